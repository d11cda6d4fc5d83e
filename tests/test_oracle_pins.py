"""Pins of the FP64 oracle against facts outside it (CPU only).

Every quantity the GPU path is later compared with is fixed here by something
other than the oracle itself: published known-answer vectors, hand-derived
poses, closed forms, an independent formulation (product of exponentials via
scipy's matrix exponential), library routines (scipy rotations, LAPACK
solves, pairwise distances), finite differences and brute-force sweeps.
"""
import math
import os

import numpy as np
import pytest
from scipy import stats
from scipy.linalg import expm
from scipy.spatial.distance import cdist
from scipy.spatial.transform import Rotation as Rot

import oracle as orc
from paper_2510_07514_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLD, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


@pytest.fixture(scope="module")
def panda():
    return orc.Robot(inputs.panda())


@pytest.fixture(scope="module")
def chains():
    rng = np.random.default_rng(11)
    return [orc.Robot(inputs.random_chain(rng, n)) for n in (3, 7, 12, 20)]


def _poses(rob, th):
    return orc.pose(rob, th)


# ----------------------------------------------------------------------------
# random numbers

def test_philox_known_answers():
    rows = _rows("philox4x32_10_kat.txt")
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = orc.philox(v[0:4], v[4:6])
        assert [int(x) for x in out] == v[6:10]


def test_u01_exact_and_open_interval():
    assert orc.u01(0) == 2.0 ** -24
    assert orc.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    rng = np.random.default_rng(0)
    for x in rng.integers(0, 2 ** 32, 200, dtype=np.uint64):
        u = orc.u01(int(x))
        assert float(np.float32(u)) == u          # exact in binary32 too
        assert u == ((int(x) >> 9) + 0.5) / 2 ** 23


def test_normal_is_standard_normal():
    key = (0x1234, 0xABCD)
    z = []
    for c in range(6000):
        w = orc.philox([c, 7, 2 << 24, 0], key)
        z.append(orc.normal(w[0], w[1]))
        z.append(orc.normal(w[2], w[3]))
    z = np.asarray(z)
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 0.03 and abs(z.var() - 1) < 0.05


def test_seed_sampling_stream_layout(panda):
    P = orc.make_params(seed=0x0123456789ABCDEF)
    tgt = np.repeat(np.arange(5), 40)
    cand = np.tile(np.arange(40), 5)
    th = orc.sample_seeds(panda, P, tgt, cand)
    key = (P.key[0], P.key[1])
    for c in (0, 17, 199):
        for j in range(7):
            w = orc.philox([cand[c], tgt[c], 1 << 24, j // 4], key)
            u = ((int(w[j % 4]) >> 9) + 0.5) / 2 ** 23
            assert th[c, j] == pytest.approx(panda.lo[j] + u * (panda.hi[j] - panda.lo[j]), abs=1e-15)
    assert np.all(th >= panda.lo) and np.all(th <= panda.hi)
    for j in range(7):
        uj = (th[:, j] - panda.lo[j]) / (panda.hi[j] - panda.lo[j])
        assert stats.kstest(uj, "uniform").pvalue > 1e-3


# ----------------------------------------------------------------------------
# kinematics (Eq. fk)

def test_panda_rest_pose(panda):
    gold = np.array([float(x) for x in _rows("panda_rest_pose.txt")[0]])
    pq = _poses(panda, np.zeros(7))[0]
    assert np.allclose(pq[:3], gold[:3], atol=1e-12)
    assert abs(abs(np.dot(pq[3:], gold[3:])) - 1) < 1e-12
    F = orc.fk_frames(panda, np.zeros(7))
    assert np.allclose(F[-1][:3, :3], np.diag([1.0, -1.0, -1.0]), atol=1e-12)


def test_planar_chain_closed_form():
    L = [0.5, 0.3, 0.2]
    rob = orc.Robot(inputs.planar(L))
    rng = np.random.default_rng(3)
    for th in rng.uniform(-math.pi, math.pi, (20, 3)):
        cum = np.cumsum(th)
        x = sum(L[i] * math.cos(cum[i]) for i in range(3))
        y = sum(L[i] * math.sin(cum[i]) for i in range(3))
        pq = _poses(rob, th)[0]
        assert np.allclose(pq[:3], [x, y, 0.0], atol=1e-12)
        yaw = cum[-1]
        q = np.array([math.cos(yaw / 2), 0, 0, math.sin(yaw / 2)])
        assert abs(abs(np.dot(q, pq[3:])) - 1) < 1e-12


def _se3_hat(w, v):
    X = np.zeros((4, 4))
    X[:3, :3] = [[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]]
    X[:3, 3] = v
    return X


@pytest.mark.parametrize("which", ["panda", 0, 1, 2, 3])
def test_fk_equals_product_of_exponentials(which, panda, chains):
    """T(theta) = prod_i exp([S_i] theta_i) T(0) with the screw axes of the rest
    configuration -- an independent formula for the same chain."""
    rob = panda if which == "panda" else chains[which]
    n = rob.n
    F0 = orc.fk_frames(rob, np.zeros(n))
    S = []
    for i in range(n):
        z = F0[i + 1][:3, 2]
        p = F0[i + 1][:3, 3]
        S.append(_se3_hat(z, -np.cross(z, p)))
    rng = np.random.default_rng(5 + n)
    for th in rng.uniform(rob.lo, rob.hi, (5, n)):
        F = orc.fk_frames(rob, th)
        G = np.eye(4)
        for i in range(n):
            G = G @ expm(S[i] * th[i])
            assert np.allclose(F[i + 1], G @ F0[i + 1], atol=1e-10)
        assert np.allclose(F[n + 1], G @ F0[n + 1], atol=1e-10)


# ----------------------------------------------------------------------------
# orientation error (Eq. quat_diff)

def test_quat_from_rot_matches_scipy():
    rs = list(Rot.random(200, random_state=1))
    rs += [Rot.from_rotvec(a * (math.pi - 1e-9)) for a in Rot.random(20, random_state=2).as_rotvec()
           / np.linalg.norm(Rot.random(20, random_state=2).as_rotvec(), axis=1)[:, None]]
    rs += [Rot.identity()]
    for r in rs:
        q = orc.quat_from_rot(r.as_matrix())
        xyzw = r.as_quat()
        ref = np.array([xyzw[3], *xyzw[:3]])
        assert q[0] >= 0
        assert abs(abs(np.dot(q, ref)) - 1) < 1e-12


def test_omega_is_the_rotation_log():
    rt = Rot.random(300, random_state=4)
    re = Rot.random(300, random_state=5)
    for a, b in zip(rt, re):
        qa, qb = a.as_quat(), b.as_quat()
        w = orc.omega([qa[3], *qa[:3]], [qb[3], *qb[:3]])
        ref = Rot.from_matrix(a.as_matrix() @ b.as_matrix().T).as_rotvec()
        assert np.linalg.norm(w) <= math.pi + 1e-12
        if np.linalg.norm(ref) < math.pi - 1e-6:
            assert np.allclose(w, ref, atol=1e-10)
    assert np.allclose(orc.omega([1, 0, 0, 0], [1, 0, 0, 0]), 0.0)
    # the same rotation given with a negated quaternion
    assert np.allclose(orc.omega([0.6, 0.8, 0, 0], [-1, 0, 0, 0]), Rot.from_quat([0.8, 0, 0, 0.6]).as_rotvec())


def test_residual_sign_convention(panda):
    rng = np.random.default_rng(6)
    th = rng.uniform(panda.lo, panda.hi)
    pq = _poses(panda, th)[0]
    dp = np.array([0.01, -0.02, 0.03])
    dr = Rot.from_rotvec([0.05, -0.02, 0.01])
    qe = Rot.from_quat([*pq[4:], pq[3]])
    qt = (dr * qe).as_quat()
    tgt = np.array([*(pq[:3] + dp), qt[3], *qt[:3]])
    e = orc.residual(panda, th, tgt)
    assert np.allclose(e[:3], dp, atol=1e-12)
    assert np.allclose(e[3:], dr.as_rotvec(), atol=1e-12)


# ----------------------------------------------------------------------------
# Jacobian (Eq. jacobian)

@pytest.mark.parametrize("which", ["panda", 0, 2, 3])
def test_jacobian_finite_differences(which, panda, chains):
    rob = panda if which == "panda" else chains[which]
    n = rob.n
    rng = np.random.default_rng(8)
    h = 1e-6
    for th in rng.uniform(rob.lo, rob.hi, (3, n)):
        J = orc.jacobian(rob, th)
        for i in range(n):
            tp, tm = th.copy(), th.copy()
            tp[i] += h
            tm[i] -= h
            Fp, Fm = orc.fk_frames(rob, tp)[-1], orc.fk_frames(rob, tm)[-1]
            assert np.allclose((Fp[:3, 3] - Fm[:3, 3]) / (2 * h), J[:3, i], atol=1e-7)
            w = Rot.from_matrix(Fp[:3, :3] @ Fm[:3, :3].T).as_rotvec() / (2 * h)
            assert np.allclose(w, J[3:, i], atol=1e-7)


# ----------------------------------------------------------------------------
# PO-CCD (Alg. 3)

def _targets(rob, rng, count):
    th = rng.uniform(rob.lo, rob.hi, (count, rob.n))
    return _poses(rob, th)


def test_ccd_position_step_is_the_optimal_joint_rotation():
    """Eq. vec_proj/theta_proj move the EE to the point of its circle about
    joint j that is closest to the target: with limits too wide to bind, a
    brute-force sweep of the joint over a full turn cannot find a smaller
    position error.  With the real limits the step is that optimum clamped
    to the limits (no angle wrapping)."""
    wide = inputs.panda()
    wide.lo, wide.hi = np.full(7, -10.0), np.full(7, 10.0)
    rw, rl = orc.Robot(wide), orc.Robot(inputs.panda())
    rng = np.random.default_rng(9)
    C = 12
    tg = _targets(rl, rng, C)
    th = rng.uniform(rl.lo, rl.hi, (C, 7))
    P = orc.make_params(seed=1)
    tw = orc.ccd_iteration(rw, P, tg, np.arange(C), np.zeros(C), 0, th)
    tl = orc.ccd_iteration(rl, P, tg, np.arange(C), np.zeros(C), 0, th)
    grid = np.linspace(-math.pi, math.pi, 4001)
    for c in range(C):
        for j in range(7):
            sweep = np.repeat(th[c][None], len(grid), 0)
            sweep[:, j] = th[c, j] + grid
            err = np.linalg.norm(_poses(rw, sweep)[:, :3] - tg[c, :3], axis=1)
            assert tw["rp"][c, j] <= err.min() + 1e-12
            assert abs(tw["dp"][c, j]) <= math.pi
            t1 = th[c].copy()
            t1[j] += tw["dp"][c, j]
            assert tw["rp"][c, j] == pytest.approx(np.linalg.norm(_poses(rw, t1)[0, :3] - tg[c, :3]), abs=1e-12)
            clamped = np.clip(th[c, j] + tw["dp"][c, j], rl.lo[j], rl.hi[j]) - th[c, j]
            assert tl["dp"][c, j] == pytest.approx(clamped, abs=1e-15)


def test_ccd_orientation_step_closed_form():
    """One revolute joint about z, target rotated about the same axis by phi0:
    Eq. angle_axis gives axis +-z and angle |phi0|, Eq. ori_update the step
    delta(k) * phi0."""
    rob = orc.Robot(inputs.planar([0.4]))
    P = orc.make_params(seed=2)
    for phi0 in (0.7, -1.3, 2.0, -0.2):
        q = (math.cos(phi0 / 2), 0.0, 0.0, math.sin(phi0 / 2))
        tgt = np.array([[0.4 * math.cos(phi0), 0.4 * math.sin(phi0), 0.0, *q]])
        for k in (0, 1, 5):
            tr = orc.ccd_iteration(rob, P, tgt, [0], [0], k, np.zeros((1, 1)))
            dk = P.cd_delta0 * P.cd_rho ** k
            assert tr["dq"][0, 0] == pytest.approx(dk * phi0, abs=1e-12)
            assert tr["rq"][0, 0] == pytest.approx(abs(phi0) * (1 - dk), abs=1e-12)
            assert tr["dp"][0, 0] == pytest.approx(phi0, abs=1e-12)   # position step hits the target point


def test_ccd_greedy_ties_go_to_the_lower_joint():
    """Planar chain with a zero-length link between joints 1 and 2: the two
    joints share axis and origin, so their position updates and their
    orientation updates are the same rotation and leave the same residual.
    That exact tie must go to joint 1, never to joint 2.  Parallel axes also
    make every orientation update leave the same orientation error.  Limits
    too wide to bind keep the clamp from telling the two joints apart."""
    chain = inputs.planar([0.5, 0.0, 0.4, 0.3])
    chain.lo, chain.hi = np.full(4, -10.0), np.full(4, 10.0)
    rob = orc.Robot(chain)
    P = orc.make_params(seed=8)
    rng = np.random.default_rng(7)
    C = 64
    tg = _targets(rob, rng, C)
    th = rng.uniform(-1.0, 1.0, (C, 4))
    tr = orc.ccd_iteration(rob, P, tg, np.arange(C), np.zeros(C), 0, th)
    picked_1 = 0
    for c in range(C):
        assert np.ptp(tr["rq"][c]) < 1e-12
        for key in ("rp", "op", "pq", "rq"):
            assert tr[key][c, 1] == pytest.approx(tr[key][c, 2], abs=1e-12)
        assert tr["jp"][c] != 2 and tr["jo"][c] != 2
        picked_1 += int(tr["jp"][c] == 1) + int(tr["jo"][c] == 1)
        sp = _score(P, tr["rp"][c], tr["op"][c])
        if tr["margin_p"][c] > 1e-9:
            assert sp[tr["jp"][c]] <= sp.min() * (1 + 1e-9)
    assert picked_1 > 0


def _score(P, ep, eo):
    return (np.asarray(ep) / P.eps_pos) ** 2 + (np.asarray(eo) / P.eps_ori) ** 2


def _normal_stream(P, cand, tgt, phase, it, n):
    key = (P.key[0], P.key[1])
    out = []
    for j in range(n):
        w = orc.philox([cand, tgt, (phase << 24) | it, j // 2], key)
        h = 2 * (j % 2)
        out.append(orc.normal(w[h], w[h + 1]))
    return np.asarray(out)


def test_ccd_selection_acceptance_and_perturbation(panda):
    rng = np.random.default_rng(10)
    C, k = 64, 3
    tg = _targets(panda, rng, C)
    th = rng.uniform(panda.lo, panda.hi, (C, 7))
    P = orc.make_params(seed=3)
    tgt_idx, cand = np.arange(C), np.arange(C) * 3
    tr = orc.ccd_iteration(panda, P, tg, tgt_idx, cand, k, th)
    n_acc = 0
    for c in range(C):
        # Alg. 3: greedy argmin of the residual score each trial leaves
        sp = _score(P, tr["rp"][c], tr["op"][c])
        so = _score(P, tr["pq"][c], tr["rq"][c])
        if tr["margin_p"][c] > P.cd_tie:
            assert tr["jp"][c] == int(np.argmin(sp))
        if tr["margin_o"][c] > P.cd_tie:
            assert tr["jo"][c] == int(np.argmin(so))
        jp, jo = tr["jp"][c], tr["jo"][c]
        for j in range(7):      # the trial errors are those of the stepped configuration
            t1 = th[c].copy()
            t1[j] += tr["dp"][c, j]
            e = orc.residual(panda, t1, tg[c])
            assert tr["rp"][c, j] == pytest.approx(np.linalg.norm(e[:3]), abs=1e-12)
            assert tr["op"][c, j] == pytest.approx(np.linalg.norm(e[3:]), abs=1e-12)
            t1 = th[c].copy()
            t1[j] += tr["dq"][c, j]
            e = orc.residual(panda, t1, tg[c])
            assert tr["pq"][c, j] == pytest.approx(np.linalg.norm(e[:3]), abs=1e-12)
            assert tr["rq"][c, j] == pytest.approx(np.linalg.norm(e[3:]), abs=1e-12)
        hat = th[c].copy()
        if jp != jo:
            hat[jp] += tr["dp"][c, jp]
            hat[jo] += tr["dq"][c, jo]
        elif abs(tr["dp"][c, jp]) >= abs(tr["dq"][c, jo]):
            hat[jp] += tr["dp"][c, jp]
        else:
            hat[jo] += tr["dq"][c, jo]
        assert np.allclose(tr["theta_hat"][c], hat, atol=0)
        e0 = orc.residual(panda, th[c], tg[c])
        e1 = orc.residual(panda, hat, tg[c])
        acc = ((np.linalg.norm(e0[:3]) - np.linalg.norm(e1[:3]) > P.cd_gamma_pos)
               or (np.linalg.norm(e0[3:]) - np.linalg.norm(e1[3:]) > P.cd_gamma_ori))
        assert bool(tr["accepted"][c]) == acc
        if acc:
            assert np.array_equal(tr["theta"][c], hat)
            n_acc += 1
        else:
            z = _normal_stream(P, cand[c], tgt_idx[c], 2, k, 7)
            assert np.allclose(tr["theta"][c], np.clip(th[c] + P.cd_sigma * z, panda.lo, panda.hi), atol=1e-14)
        e2 = orc.residual(panda, tr["theta"][c], tg[c])
        conv = (np.sum(e2[:3] ** 2) < P.cd_eps_pos2) and (np.sum(e2[3:] ** 2) < P.cd_eps_ori2)
        assert bool(tr["converged"][c]) == conv
    assert 0 < n_acc < C


# ----------------------------------------------------------------------------
# top-K and duplication (Alg. 2)

def test_dup_layout():
    assert orc.dup_layout(1000, 4) == (250, 4, 1000)
    assert orc.dup_layout(33, 4) == (8, 4, 32)
    assert orc.dup_layout(3, 4) == (1, 3, 3)
    assert orc.dup_layout(0, 4) == (0, 0, 0)


def test_topk_dup_matches_stable_sort(panda):
    rng = np.random.default_rng(12)
    T, M = 3, 64
    P = orc.make_params(seed=4)
    m_off = np.arange(T + 1) * M
    score = np.round(rng.uniform(0, 5, T * M), 1)   # many ties
    thM = rng.uniform(panda.lo, panda.hi, (T * M, 7))
    out = orc.topk_dup(panda, P, m_off, score, thM)
    K, cp, B = orc.dup_layout(M, P.dup_ratio)
    for t in range(T):
        best = np.argsort(score[t * M:(t + 1) * M], kind="stable")[:K]
        for r in range(cp):
            for i in range(K):
                b = r * K + i
                g = out["b_off"][t] + b
                assert out["src"][g] == best[i]
                z = _normal_stream(P, b, t, 3, 0, 7)
                ref = np.clip(thM[t * M + best[i]] + P.dup_sigma * z, panda.lo, panda.hi)
                assert np.allclose(out["theta"][g], ref, atol=1e-14)


# ----------------------------------------------------------------------------
# PJ-IK (Alg. 4)

def test_lm_step_matches_lapack():
    rng = np.random.default_rng(13)
    for n in (3, 6, 7, 12, 20):
        Jw = rng.normal(size=(6, n))
        b = rng.normal(size=6)
        lam = 1e-3
        A = Jw.T @ Jw
        ref = np.linalg.solve(A + lam * np.diag(np.diag(A) + 1e-9), Jw.T @ b)
        got = orc.lm_step(Jw, b, lam, 1e9)
        assert np.allclose(got, ref, rtol=1e-9, atol=1e-12)
        got_r = orc.lm_step(Jw, b, lam, 0.05)
        assert np.allclose(got_r, np.clip(ref, -0.05, 0.05), rtol=1e-9, atol=1e-12)


def test_push_through_form_equals_normal_equations():
    """The identity the GPU solves with: with S = D^(-1/2) and A_hat = Jw S,
    (Jw^T Jw + lam D)^-1 Jw^T b = S A_hat^T (A_hat A_hat^T + lam I_6)^-1 b."""
    rng = np.random.default_rng(14)
    for n in (7, 12, 20):
        Jw = rng.normal(size=(6, n))
        b = rng.normal(size=6)
        lam = 1e-3
        Dg = np.sum(Jw * Jw, axis=0) + 1e-9
        S = 1 / np.sqrt(Dg)
        Ah = Jw * S
        pt = S * (Ah.T @ np.linalg.solve(Ah @ Ah.T + lam * np.eye(6), b))
        assert np.allclose(pt, orc.lm_step(Jw, b, lam, 1e9), rtol=1e-8, atol=1e-12)


def test_dogleg_cases():
    rng = np.random.default_rng(15)
    for n in (7, 12):
        Jw = rng.normal(size=(6, n))
        b = rng.normal(size=6)
        mu = 1e-12
        gn = np.linalg.pinv(Jw) @ b
        g = Jw.T @ b
        gd = (g @ g) / np.sum((Jw @ g) ** 2) * g
        # tau = 0: the minimum-norm Gauss-Newton step
        assert np.allclose(orc.dogleg_step(Jw, b, 1e6, mu), gn, rtol=1e-8, atol=1e-10)
        # boundary: |GD| < R < |GN| -> step of length R on the segment GN -> GD
        R = 0.5 * (np.linalg.norm(gd) + np.linalg.norm(gn))
        if np.linalg.norm(gd) < R < np.linalg.norm(gn):
            st = orc.dogleg_step(Jw, b, R, mu)
            assert np.linalg.norm(st) == pytest.approx(R, rel=1e-10)
            tau = np.dot(st - gn, gd - gn) / np.dot(gd - gn, gd - gn)
            assert 0 <= tau <= 1
            assert np.allclose(gn + tau * (gd - gn), st, atol=1e-10)
        # R below |GD|: the gradient step scaled to the boundary
        R = 0.3 * np.linalg.norm(gd)
        assert np.allclose(orc.dogleg_step(Jw, b, R, mu), R * gd / np.linalg.norm(gd), rtol=1e-10)


def _cost(rob, th, tgt, W):
    e = orc.residual(rob, th, tgt)
    return 0.5 * np.sum((W * e) ** 2)


def test_lm_iteration_weights_step_and_line_search(panda):
    rng = np.random.default_rng(16)
    C = 24
    tth = rng.uniform(panda.lo, panda.hi, (C, 7))
    tg = _poses(panda, tth)
    th = np.clip(tth + rng.normal(0, 0.1, (C, 7)), panda.lo, panda.hi)
    P = orc.make_params(seed=5)
    tr = orc.lm_iteration(panda, P, tg, np.arange(C), np.arange(C), 0, th)
    for c in range(C):
        J = tr["J"][c]
        assert np.allclose(J, orc.jacobian(panda, th[c]), atol=0)
        wc = np.array([1, 1, 1, P.eps_pos / P.eps_ori, P.eps_pos / P.eps_ori, P.eps_pos / P.eps_ori])
        W = wc / np.maximum(np.linalg.norm(J, axis=1), 1e-6)
        assert np.allclose(tr["W"][c], W, rtol=1e-14)
        e = orc.residual(panda, th[c], tg[c])
        Jw = W[:, None] * J
        A = Jw.T @ Jw
        ref = np.clip(np.linalg.solve(A + P.lm_lambda * np.diag(np.diag(A) + 1e-9), Jw.T @ (W * e)),
                      -P.lm_trust_R, P.lm_trust_R)
        assert np.allclose(tr["d_lm"][c], ref, rtol=1e-8, atol=1e-12)
        c0 = _cost(panda, th[c], tg[c], W)
        first = None
        for i in range(P.lm_A + 1):
            a = 1.0 / P.lm_beta ** i
            if _cost(panda, np.clip(th[c] + a * ref, panda.lo, panda.hi), tg[c], W) < c0:
                first = a
                break
        if first is not None:
            assert tr["branch"][c] == 0 and tr["alpha"][c] == first
            assert np.allclose(tr["theta"][c], np.clip(th[c] + first * tr["d_lm"][c], panda.lo, panda.hi), atol=0)
        else:
            assert tr["branch"][c] != 0
    assert np.mean(tr["branch"] == 0) > 0.5


def test_single_coordinate_step_is_the_1d_gauss_newton_minimiser():
    """Eq. single-coord (reading c16): the joint whose cost derivative at 0 is
    steepest -- measured by central differences of 1/2 |b - x (WJ)_j|^2, not
    from the gradient formula -- and on it the minimiser of that 1-D cost,
    found by a dense scan, clamped to the trust region."""
    rng = np.random.default_rng(21)
    for n in (3, 7, 12, 24):
        for trial in range(4):
            Jw = rng.normal(size=(6, n))
            b = rng.normal(size=6)
            q = lambda j, x: 0.5 * np.sum((b[:, None] - np.outer(Jw[:, j], np.atleast_1d(x))) ** 2, axis=0)
            h = 1e-6
            slope = np.array([abs(q(j, h)[0] - q(j, -h)[0]) / (2 * h) for j in range(n)])
            i, st = orc.single_coord_step(Jw, b, 1e9)
            assert slope[i] >= slope.max() * (1 - 1e-6)
            xs = np.linspace(-10, 10, 2_000_001)
            x_best = xs[np.argmin(q(i, xs))]
            assert st[i] == pytest.approx(x_best, abs=2e-5)
            assert np.count_nonzero(st) <= 1
            # clamped: the scan restricted to [-R, R]
            R = 0.25 * abs(x_best)
            _, st_r = orc.single_coord_step(Jw, b, R)
            xr = np.linspace(-R, R, 200_001)
            assert st_r[i] == pytest.approx(xr[np.argmin(q(i, xr))], abs=1e-9)
    # ties between equally steep joints go to the lower one
    Jw = 0.1 * rng.normal(size=(6, 7))
    Jw[:, 2] = Jw[:, 5] = 2.0 * np.array([1.0, -0.5, 0.25, 0.0, 0.3, -0.2])
    b = np.array([1.0, -0.5, 0.25, 0.0, 0.3, -0.2])
    assert orc.single_coord_step(Jw, b, 1e9)[0] == 2
    Jw[:, 5] *= -1  # same magnitude, opposite sign: still a tie on |g|
    assert orc.single_coord_step(Jw, b, 1e9)[0] == 2


def test_single_coordinate_step_recovers_a_small_joint_motion():
    """A one-joint arm whose target is its own pose after turning the joint by
    delta: the residual is then zero at the answer, so the Gauss-Newton step of
    Eq. single-coord equals delta up to O(delta^2) (a dropped term or a wrong
    sign leaves an O(delta) error)."""
    rob = orc.Robot(inputs.planar([0.7]))
    P = orc.make_params(seed=1)
    errs = []
    for delta in (1e-1, 1e-2, 1e-3):
        th0 = np.array([0.3])
        tgt = orc.pose(rob, th0 + delta)
        tr = orc.lm_iteration(rob, P, tgt, [0], [0], 0, th0)
        assert tr["sc_joint"][0] == 0
        errs.append(abs(tr["sc_step"][0] - delta) / delta ** 2)
    assert max(errs) < 1.0


def _lm_cost(rob, th, tgt, W):
    e = orc.residual(rob, th, tgt)
    return 0.5 * np.sum((W * e) ** 2)


def _lm_expected(rob, P, tgt, th, tr, c):
    """The outcome Alg. 4 prescribes for candidate c, recomputed from pinned
    parts (the residual, the LM step checked against LAPACK, the dogleg step
    checked against pinv, the single-coordinate step checked by a scan): the
    first of LM line search, dogleg, single-coordinate line search that strictly
    lowers the weighted cost; else the perturbation.  Returns (branch, alpha, theta)."""
    W = tr["W"][c]
    clip = lambda x: np.clip(x, rob.lo, rob.hi)
    c0 = _lm_cost(rob, th, tgt, W)
    alphas = [1.0 / P.lm_beta ** i for i in range(P.lm_A + 1)]
    for a in alphas:
        if _lm_cost(rob, clip(th + a * tr["d_lm"][c]), tgt, W) < c0:
            return 0, a, clip(th + a * tr["d_lm"][c])
    if _lm_cost(rob, clip(th + tr["d_dog"][c]), tgt, W) < c0:
        return 1, 0.0, clip(th + tr["d_dog"][c])
    sc = np.zeros(rob.n)
    sc[tr["sc_joint"][c]] = tr["sc_step"][c]
    for a in alphas:
        if _lm_cost(rob, clip(th + a * sc), tgt, W) < c0:
            return 2, a, clip(th + a * sc)
    return 3, 0.0, None


def test_lm_iteration_follows_the_branch_order_of_alg4(panda):
    """Alg. 4's fallback chain on candidates part-way through PJ-IK from
    uniform seeds (where a third or more of the iterations fail the full step):
    each candidate's dogleg and single-coordinate steps equal the pinned step
    functions on its weighted Jacobian, and the branch, alpha and new theta are
    the first successful step in the order LM, dogleg, single coordinate, else
    the perturbation drawn from the PJ-IK normal stream."""
    rng = np.random.default_rng(22)
    T, C, k = 6, 400, 10
    tth = rng.uniform(panda.lo, panda.hi, (T, 7))
    tg = _poses(panda, tth)
    tgt = rng.integers(0, T, C)
    cand = np.arange(C)
    seen = set()
    for A in (4, 0):
        P = orc.make_params(seed=9, lm_A=A, lm_max_iters=k)
        th = orc.pjik(panda, P, tg, tgt, cand, rng.uniform(panda.lo, panda.hi, (C, 7)))["theta"]
        tr = orc.lm_iteration(panda, P, tg, tgt, cand, k, th)
        for c in range(C):
            J = orc.jacobian(panda, th[c])
            assert np.array_equal(tr["J"][c], J)
            Jw = tr["W"][c][:, None] * J
            bw = tr["W"][c] * orc.residual(panda, th[c], tg[tgt[c]])
            assert np.array_equal(tr["d_dog"][c], orc.dogleg_step(Jw, bw, P.lm_trust_R, P.lm_gn_reg))
            i, st = orc.single_coord_step(Jw, bw, P.lm_trust_R)
            assert tr["sc_joint"][c] == i and tr["sc_step"][c] == st[i]
            br, al, th_new = _lm_expected(panda, P, tg[tgt[c]], th[c], tr, c)
            assert tr["branch"][c] == br, c
            assert tr["alpha"][c] == al
            if br < 3:
                assert np.array_equal(tr["theta"][c], th_new)
            else:
                z = _normal_stream(P, c, tgt[c], inputs.PHASE_LM, k, 7)
                assert np.allclose(tr["theta"][c], np.clip(th[c] + P.lm_sigma * z, panda.lo, panda.hi), atol=1e-15)
            seen.add(br)
    assert seen >= {0, 1, 2}


def test_lm_perturbation_when_no_step_lowers_the_cost():
    """A stretched planar arm with its target straight ahead beyond reach and
    the same orientation: the gradient (WJ)^T W r is exactly zero (the
    position Jacobian is orthogonal to the error), so the LM, dogleg and
    single-coordinate steps are zero and none lowers the cost; Alg. 4 then
    perturbs with N(0, sigma^2 I) from the PJ-IK stream (phase 4) of the
    candidate's counter, and iteration k keys the draw."""
    rob = orc.Robot(inputs.planar([0.5, 0.4, 0.3]))
    th = np.zeros((2, 3))
    tgt = orc.pose(rob, th[:1]).copy()
    assert np.allclose(tgt[0, 3:], [1, 0, 0, 0])
    tgt[0, 0] += 0.6
    for k in (0, 7):
        P = orc.make_params(seed=3)
        tr = orc.lm_iteration(rob, P, tgt, [0, 0], [0, 5], k, th)
        assert np.all(tr["branch"] == 3)
        assert np.all(tr["d_lm"] == 0) and np.all(tr["d_dog"] == 0) and np.all(tr["sc_step"] == 0)
        for c, cand in enumerate((0, 5)):
            z = _normal_stream(P, cand, 0, inputs.PHASE_LM, k, 3)
            assert np.allclose(tr["theta"][c], np.clip(P.lm_sigma * z, rob.lo, rob.hi), atol=1e-15)
        assert not np.allclose(tr["theta"][0], tr["theta"][1])


def test_pjik_converges_from_nearby_seeds(panda):
    rng = np.random.default_rng(17)
    C = 32
    tth = rng.uniform(panda.lo + 0.3, panda.hi - 0.3, (C, 7))
    tg = _poses(panda, tth)
    th = tth + rng.normal(0, 0.05, (C, 7))
    P = orc.make_params(seed=6)
    o = orc.pjik(panda, P, tg, np.arange(C), np.arange(C), th)
    ok = (o["perr"] < P.eps_pos) & (o["oerr"] < P.eps_ori)
    assert ok.mean() > 0.9
    for c in np.nonzero(ok)[0]:
        e = orc.residual(panda, o["theta"][c], tg[c])
        assert np.linalg.norm(e[:3]) == pytest.approx(o["perr"][c], abs=1e-15)


# ----------------------------------------------------------------------------
# collision filter (Sec. V-C)

def _one_sphere_robot(r=0.1):
    rob = inputs.planar([1.0])
    rob.sph_body = np.array([2], np.int32)         # flange body
    rob.sph_xyzr = np.array([[0.0, 0.0, 0.0, r]])
    rob.ignore = inputs.default_ignore(rob)
    return orc.Robot(rob)


def test_collision_closed_form_cases():
    rob = _one_sphere_robot(0.1)   # sphere centre at (1, 0, 0) for theta = 0
    th = np.zeros((1, 1))

    def verdict(sph=(), box=()):
        sc = orc.Scene(inputs.Scene(np.asarray(sph, float).reshape(-1, 4), np.asarray(box, float).reshape(-1, 6)))
        return bool(orc.collide(rob, sc, th)[0][0])

    d = 1e-9
    assert verdict(sph=[[1.25 + d, 0, 0, 0.15]]) is False
    assert verdict(sph=[[1.25 - d, 0, 0, 0.15]]) is True
    assert verdict(box=[[1.1 + d, -0.1, -0.1, 1.3, 0.1, 0.1]]) is False    # face distance 0.1 + d
    assert verdict(box=[[1.1 - d, -0.1, -0.1, 1.3, 0.1, 0.1]]) is True
    a = 0.1 / math.sqrt(3)
    assert verdict(box=[[1 + a + d, a + d, a + d, 2, 1, 1]]) is False        # corner at distance > r
    assert verdict(box=[[1 + a - d, a - d, a - d, 2, 1, 1]]) is True
    assert verdict(box=[[0.5, -0.5, -0.5, 1.5, 0.5, 0.5]]) is True            # centre inside the box
    assert verdict() is False


def test_self_collision_and_ignore_mask():
    # two joints about z, links of 1.0; body 1 sphere at its origin (0,0,0),
    # flange-body sphere at the tip; folding joint 2 back brings the tip home.
    base = inputs.planar([1.0, 1.0])
    base.sph_body = np.array([1, 3], np.int32)
    base.sph_xyzr = np.array([[0, 0, 0, 0.2], [0, 0, 0, 0.2]])
    base.ignore = np.zeros((4, 4), np.uint8)
    rob = orc.Robot(base)
    folded = np.array([[0.0, math.pi * 0.999]])
    straight = np.array([[0.0, 0.0]])
    assert orc.collide(rob, None, folded)[0][0]
    assert not orc.collide(rob, None, straight)[0][0]
    base.ignore[1, 3] = base.ignore[3, 1] = 1
    assert not orc.collide(orc.Robot(base), None, folded)[0][0]


def test_collision_matches_pairwise_distances():
    rng = np.random.default_rng(inputs.CFG_SEED[2])
    robd = inputs.panda_with_spheres(rng)
    scene = inputs.random_scene(rng, 200, 20)
    rob, sc = orc.Robot(robd), orc.Scene(scene)
    th = rng.uniform(robd.lo, robd.hi, (120, 7))
    hit, margin = orc.collide(rob, sc, th)
    bodies = robd.sph_body
    ign = robd.ignore
    for c in range(len(th)):
        F = orc.fk_frames(rob, th[c])
        W = np.array([F[b][:3, :3] @ s[:3] + F[b][:3, 3] for b, s in zip(bodies, robd.sph_xyzr)])
        r = robd.sph_xyzr[:, 3]
        D = cdist(W, W)
        pair_ok = (bodies[:, None] != bodies[None, :]) & (ign[bodies][:, bodies] == 0)
        h_self = np.any((D < r[:, None] + r[None, :]) & pair_ok)
        De = cdist(W, scene.sph_xyzr[:, :3])
        h_sph = np.any(De < r[:, None] + scene.sph_xyzr[None, :, 3])
        lo, hi = scene.box_lohi[:, :3], scene.box_lohi[:, 3:]
        cl = np.clip(W[:, None, :], lo[None], hi[None])
        h_box = np.any(np.linalg.norm(W[:, None, :] - cl, axis=2) < r[:, None])
        assert bool(hit[c]) == bool(h_self or h_sph or h_box)
    assert 0 < hit.mean() < 1


# ----------------------------------------------------------------------------
# ranking (Alg. 2) and the whole method

def _rank_reference(th, score, perr, oerr, hit, b_off, k, eps_pos, eps_ori, q_ref=None):
    """Alg. 2's final ranking by a stable library sort: per target the
    collision-free candidates, those within the tolerances first (reading c20),
    each group by score -- or by joint distance to q_ref[t] (reading c24)."""
    out = []
    for t in range(len(b_off) - 1):
        g = np.arange(b_off[t], b_off[t + 1])
        g = g[~hit[g]]
        conv = (perr[g] <= eps_pos) & (oerr[g] <= eps_ori)
        key = score[g].copy()
        if q_ref is not None:
            key = np.where(conv, np.sum((th[g] - q_ref[t]) ** 2, axis=1), key)
        order = np.lexsort((g, key, ~conv))
        out.append(g[order][:k])
    return out


def test_rank_matches_sorted_collision_free(panda):
    rng = np.random.default_rng(18)
    T, B, k = 4, 50, 5
    b_off = np.arange(T + 1) * B
    th = rng.uniform(panda.lo, panda.hi, (T * B, 7))
    score = np.round(rng.uniform(0, 3, T * B), 1)
    perr, oerr = rng.uniform(0, 2e-3, T * B), rng.uniform(0, 2e-2, T * B)
    hit = rng.uniform(size=T * B) < 0.7
    hit[B:2 * B] = True       # a target with no collision-free candidate
    o = orc.rank(panda, b_off, th, score, perr, oerr, hit, k, 1e-3, 1e-2)
    ref = _rank_reference(th, score, perr, oerr, hit, b_off, k, 1e-3, 1e-2)
    for t in range(T):
        assert o["count"][t] == len(ref[t])
        for r, g in enumerate(ref[t]):
            assert np.array_equal(o["q"][t, r], th[g])
            assert np.array_equal(o["err"][t, r], [perr[g], oerr[g]])


def test_rank_puts_converged_candidates_first(panda):
    """Reading c20: a candidate just outside the position tolerance can have a
    lower score than one inside both tolerances (|e_p| = 1.05 eps_pos, omega = 0
    gives s = 1.1025; 0.9 eps_pos and 0.9 eps_ori give s = 1.62); the converged
    one is returned first, so the target counts as solved."""
    th = np.array([[0.1] * 7, [0.2] * 7, [0.3] * 7])
    perr = np.array([1.05e-3, 0.9e-3, 3e-3])
    oerr = np.array([0.0, 0.9e-2, 0.0])
    score = (perr / 1e-3) ** 2 + (oerr / 1e-2) ** 2
    assert score[0] < score[1] < score[2]
    o = orc.rank(panda, [0, 3], th, score, perr, oerr, None, 3, 1e-3, 1e-2)
    assert o["count"][0] == 3
    assert np.array_equal(o["q"][0, :, 0], [0.2, 0.1, 0.3])
    # exactly on the tolerance counts as inside it (the success test is <=)
    o = orc.rank(panda, [0, 2], th[:2], score[:2], np.array([1.05e-3, 1e-3]), np.array([0.0, 1e-2]), None, 1,
                 1e-3, 1e-2)
    assert o["q"][0, 0, 0] == 0.2


def test_rank_nearest_orders_converged_by_joint_distance(panda):
    """Reading c24 (tracking): inside the tolerances by squared joint distance
    to the reference configuration, then the rest by score; collisions never."""
    rng = np.random.default_rng(19)
    T, B, k = 3, 40, 12
    b_off = np.arange(T + 1) * B
    th = rng.uniform(panda.lo, panda.hi, (T * B, 7))
    q_ref = rng.uniform(panda.lo, panda.hi, (T, 7))
    score = rng.uniform(0, 3, T * B)
    perr, oerr = rng.uniform(0, 2e-3, T * B), rng.uniform(0, 2e-2, T * B)
    hit = rng.uniform(size=T * B) < 0.3
    o = orc.rank(panda, b_off, th, score, perr, oerr, hit, k, 1e-3, 1e-2, q_ref=q_ref)
    ref = _rank_reference(th, score, perr, oerr, hit, b_off, k, 1e-3, 1e-2, q_ref=q_ref)
    for t in range(T):
        assert o["count"][t] == len(ref[t])
        assert np.array_equal(o["q"][t, :len(ref[t])], th[ref[t]])
        # the converged prefix is nearest-first, measured independently of the oracle
        conv = (o["err"][t, :o["count"][t], 0] <= 1e-3) & (o["err"][t, :o["count"][t], 1] <= 1e-2)
        nconv = int(conv.sum())
        assert np.all(conv[:nconv]) and not np.any(conv[nconv:])
        d = np.linalg.norm(o["q"][t, :nconv] - q_ref[t], axis=1)
        assert np.all(np.diff(d) >= 0)


def test_solve_round_trip_open_world(panda):
    wl = inputs.cfg1()
    T = 4
    tg = _poses(panda, wl.theta_gen[:T])
    P = orc.make_params(wl.eps_pos, wl.eps_ori, seed=wl.seed)
    o = orc.solve(panda, None, P, tg, wl.n_samples, top_k=4)
    succ = 0
    for t in range(T):
        assert o["count"][t] == 4
        for r in range(4):
            q = o["q"][t, r]
            assert np.all(q >= panda.lo) and np.all(q <= panda.hi)
            e = orc.residual(panda, q, tg[t])
            assert np.allclose([np.linalg.norm(e[:3]), np.linalg.norm(e[3:])], o["err"][t, r], atol=1e-15)
        # converged rows first (reading c20), each group by score
        conv = (o["err"][t, :, 0] <= wl.eps_pos) & (o["err"][t, :, 1] <= wl.eps_ori)
        assert np.all(np.diff(conv.astype(int)) <= 0)
        s_ = o["err"][t, :, 0] ** 2 / wl.eps_pos ** 2 + o["err"][t, :, 1] ** 2 / wl.eps_ori ** 2
        for grp in (conv, ~conv):
            assert np.all(np.diff(s_[grp]) >= -1e-12)
        succ += (o["err"][t, 0, 0] <= wl.eps_pos) and (o["err"][t, 0, 1] <= wl.eps_ori)
    assert succ >= 3


# ----------------------------------------------------------------------------
# the position-only CCD baseline (Alg. 1)

def test_classic_ccd_sweep_order_by_hand():
    """Planar 2R chain of unit links at theta = 0, target (0, 1.5): Alg. 1
    turns the last joint first (about (1, 0): from direction (1, 0) to the
    target's direction (-1, 1.5)), then the first joint (about the origin:
    from the moved end effector's direction to the target's)."""
    rob = orc.Robot(inputs.planar([1.0, 1.0]))
    P = orc.make_params(seed=1, cd_variant=1)
    tg = np.array([[0.0, 1.5, 0.0, 1.0, 0.0, 0.0, 0.0]])
    tr = orc.ccd_iteration(rob, P, tg, [0], [0], 0, np.zeros((1, 2)))
    d2 = math.atan2(1.5, -1.0)
    ee = (1.0 + math.cos(d2), math.sin(d2))
    d1 = math.atan2(1.5, 0.0) - math.atan2(ee[1], ee[0])
    assert tr["dp"][0, 1] == pytest.approx(d2, abs=1e-12)
    assert tr["dp"][0, 0] == pytest.approx(d1, abs=1e-12)
    assert np.allclose(tr["theta"][0], [d1, d2], atol=1e-12)


def test_classic_ccd_reaches_planar_targets_and_respects_limits():
    """On a planar 3R chain the sweeps drive reachable targets to zero position
    error (the break test ends the run); with tight limits every joint stays
    inside them."""
    chain = inputs.planar([0.5, 0.4, 0.3])
    chain.lo, chain.hi = np.full(3, -20.0), np.full(3, 20.0)  # too wide to bind (no angle wrapping)
    rob = orc.Robot(chain)
    P = orc.make_params(seed=2, cd_variant=1, cd_max_iters=200, cd_eps_pos2=1e-16)
    rng = np.random.default_rng(3)
    th = rng.uniform(-math.pi, math.pi, (40, 3))
    tg = _poses(rob, th)
    out = orc.po_ccd(rob, P, tg, np.arange(40), np.zeros(40, np.int32))
    # CCD can wind joints up or crawl near a singular pose; a wrong order or sign fails almost everywhere
    assert np.mean(out["perr"] < 1e-8) > 0.9
    assert np.mean(out["iters"] < 200) > 0.9
    tight = inputs.planar([0.5, 0.4, 0.3])
    tight.lo, tight.hi = np.full(3, -0.3), np.full(3, 0.3)
    rt = orc.Robot(tight)
    o2 = orc.po_ccd(rt, P, tg, np.arange(40), np.zeros(40, np.int32))
    assert np.all(o2["theta"] >= -0.3 - 1e-15) and np.all(o2["theta"] <= 0.3 + 1e-15)
    assert np.mean(o2["perr"] > 1e-3) > 0.5  # most of those targets lie outside the reachable set


def test_target_wide_break_equals_per_seed_runs_capped_at_the_first_convergence(panda):
    """cd_variant 2 stops every seed of a target after the first iteration that
    leaves any of them inside the coarse tolerance.  Seeds do not interact
    before that, so each seed's result is its own PO-CCD run capped at
    K* = min over the target's converged seeds of their iteration count
    (the whole cap when none converges) -- exactly, in double precision."""
    rng = np.random.default_rng(17)
    T, S = 6, 40
    tg = _targets(panda, rng, T)
    tgt = np.repeat(np.arange(T), S).astype(np.int32)
    cand = np.tile(np.arange(S), T).astype(np.int32)
    P0 = orc.make_params(seed=4)
    full = orc.po_ccd(panda, P0, tg, tgt, cand)
    conv = (full["perr"] ** 2 < P0.cd_eps_pos2) & (full["oerr"] ** 2 < P0.cd_eps_ori2)
    brk = orc.po_ccd(panda, orc.make_params(seed=4, cd_variant=2), tg, tgt, cand)
    n_break = 0
    for t in range(T):
        sel = tgt == t
        ks = full["iters"][sel][conv[sel]]
        kstar = int(ks.min()) if len(ks) else P0.cd_max_iters
        n_break += kstar < P0.cd_max_iters
        capped = orc.po_ccd(panda, orc.make_params(seed=4, cd_max_iters=kstar), tg, tgt[sel], cand[sel])
        assert np.array_equal(brk["theta"][sel], capped["theta"])
        assert np.all(brk["iters"][sel] == kstar)
    assert n_break > 0
