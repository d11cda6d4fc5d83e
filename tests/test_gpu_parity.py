"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Both sides receive the same inputs: every array is rounded to binary32 first
and the oracle gets those values in double.  Floating-point outputs must agree
within 1e-5 m / 1e-5 rad (per stage, from identical inputs).  Where a float
decides a branch, outputs are compared only where the decision is clear: the
greedy joint choice where every score gap exceeds the tie band plus the score
error the trial tolerances allow, acceptance where the oracle's margin
exceeds 1e-5, line search where it exceeds 1e-4 relative; integer and index
outputs are compared bit-exactly.
Collision verdicts are compared bit-exactly where the oracle's verdict margin
is at least 1e-6 m.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2510_07514_gb300 import api, build, hjcd, inputs

pytestmark = pytest.mark.gpu


def ranked_order_ok(err, eps_pos, eps_ori):
    """Rows of one target in the order of Alg. 2's final step (reading c20):
    those within the tolerances first, each group by non-decreasing score."""
    conv = (err[:, 0] <= eps_pos) & (err[:, 1] <= eps_ori)
    if np.any(np.diff(conv.astype(int)) > 0):
        return False
    s = err[:, 0] ** 2 / eps_pos ** 2 + err[:, 1] ** 2 / eps_ori ** 2
    for grp in (conv, ~conv):
        g = s[grp]
        if np.any(np.diff(g) < -1e-3 * np.maximum(g[1:], 1e-6)):
            return False
    return True

TOL = 1e-5
MARGIN = 1e-5


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    c = api.Context(0)
    yield c
    c.close()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def dev(a, dtype=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def soa(theta):
    """[C, n] host -> [n, C] device"""
    return dev(np.ascontiguousarray(np.asarray(theta).T))


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def reach(r):
    return max(1.0, float(np.sum(np.abs(r.a)) + np.sum(np.abs(r.d)) + 0.2))


def robots():
    rng = np.random.default_rng(21)
    out = [("panda", inputs.panda())]
    for n in (3, 12, 20, 24):
        out.append((f"chain{n}", inputs.random_chain(rng, n)))
    return out


def _targets(orob, rng, T, lo, hi):
    th = rng.uniform(lo, hi, (T, len(lo)))
    return f32(orc.pose(orob, f32(th)))


# ----------------------------------------------------------------------------
# a2: forward kinematics

@pytest.mark.parametrize("name,rob", robots())
def test_fk_parity(ctx, name, rob):
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(1)
    C = 4096 + 37  # several blocks and a ragged tail
    th = f32(rng.uniform(rob.lo, rob.hi, (C, rob.n)))
    got = host(ctx.fk(rid, soa(th)))
    ref = orc.pose(orob, th)
    tol = TOL * reach(rob) / 1.5 if rob.n > 7 else TOL
    assert np.max(np.abs(got[:, :3] - ref[:, :3])) < tol
    # quaternions component-wise, up to the sign of the whole quaternion
    sgn = np.sign(np.sum(got[:, 3:] * ref[:, 3:], axis=1))[:, None]
    assert np.max(np.abs(got[:, 3:] - sgn * ref[:, 3:])) < tol
    assert np.all(got[:, 3] >= 0)


def test_fk_empty(ctx):
    rid = ctx.add_robot(inputs.panda())
    th = torch.zeros((7, 0), device="cuda")
    out = ctx.fk(rid, th)
    assert out.shape == (0, 7)


# ----------------------------------------------------------------------------
# a1: seeds

def test_seed_sampling_parity(ctx):
    rob = inputs.panda()
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    T, S = 7, 301
    tgt = np.repeat(np.arange(T), S).astype(np.int32)
    cand = np.tile(np.arange(S), T).astype(np.int32)
    seed = 0xDEADBEEF12345678
    th = torch.empty((7, T * S), device="cuda")
    hjcd.hjcd_sample_seeds(ctx.h, rid, T * S, dev(tgt, torch.int32), dev(cand, torch.int32), seed, th, T * S)
    ref = orc.sample_seeds(orob, orc.make_params(seed=seed), tgt, cand)
    assert np.max(np.abs(host(th).T - ref)) < 1e-6


# ----------------------------------------------------------------------------
# a3 + a4: one PO-CCD iteration, traced

def _proj_lengths(orob, th, tgt_pose):
    """|u_p|, |v_p|, |u|, |v| (m) of Eq. vec_proj for every joint (degenerate-projection guard)."""
    n = orob.n
    F = orc.fk_frames(orob, th)
    pee = F[-1][:3, 3]
    out = np.zeros((4, n))
    for j in range(n):
        z, p = F[j + 1][:3, 2], F[j + 1][:3, 3]
        u, v = pee - p, tgt_pose[:3] - p
        out[0, j] = np.linalg.norm(u - np.dot(u, z) * z)
        out[1, j] = np.linalg.norm(v - np.dot(v, z) * z)
        out[2, j], out[3, j] = np.linalg.norm(u), np.linalg.norm(v)
    return out


def _ccd_sensitivity(orob, rob, th, tg, tgt, proj_eps):
    """Bound on the binary32 error of each position step of Eq. theta_proj.

    The angle between the projected vectors u_p, v_p moves by about
    u (|u|/|u_p| + |v|/|v_p|) when its inputs are rounded (u = 2^-24).  A
    projection far below the degeneracy threshold gives a zero step on both
    sides (bound 0); one near the threshold may go either way (bound inf)."""
    C = len(tgt)
    sens = np.zeros((C, rob.n))
    for c in range(C):
        pl = _proj_lengths(orob, th[c], tg[tgt[c]])
        rel = np.minimum(pl[0] / np.maximum(pl[2], 1e-30), pl[1] / np.maximum(pl[3], 1e-30))
        sens[c] = 4 * 2.0 ** -24 * reach(rob) * (1 / np.maximum(pl[0], 1e-9) + 1 / np.maximum(pl[1], 1e-9))
        sens[c][rel < 0.25 * proj_eps] = 0.0
        sens[c][(rel >= 0.25 * proj_eps) & (rel <= 4 * proj_eps)] = np.inf
    return sens


def _ccd_gpu(ctx, rid, n, tg, tgt, cand, th, k, params, seed):
    C = len(tgt)
    th_in = soa(th)
    th_out = torch.empty_like(th_in)
    buf = {k_: torch.zeros((n, C), device="cuda") for k_ in ("dp", "rp", "op", "dq", "pq", "rq", "th_hat")}
    ints = {k_: torch.zeros((C,), dtype=torch.int32, device="cuda") for k_ in ("jp", "jo")}
    acc = torch.zeros((C,), dtype=torch.uint8, device="cuda")
    tr = hjcd.hjcd_ccd_trace(*[hjcd.ptr(x) for x in (buf["dp"], buf["rp"], buf["dq"], buf["rq"], ints["jp"],
                                                     ints["jo"], acc, buf["th_hat"], buf["op"], buf["pq"])])
    hjcd.hjcd_po_ccd(ctx.h, rid, len(tg), dev(tg), 1e-3, 1e-2, seed, params, C, dev(tgt, torch.int32),
                     dev(cand, torch.int32), th_in, th_out, C, k, 1, trace=tr)
    out = {k_: host(v).T for k_, v in buf.items()}
    out.update({k_: host(v).astype(np.int64) for k_, v in ints.items()})
    out["accepted"] = host(acc).astype(bool)
    out["theta"] = host(th_out).T
    return out


@pytest.mark.parametrize("which", ["panda", "chain3", "chain12", "chain20", "chain24"])
def test_ccd_iteration_trace_parity(ctx, which):
    rob = dict(robots())[which]
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(2)
    T, C, k, seed = 13, 2053, 3, 77
    tg = _targets(orob, rng, T, rob.lo, rob.hi)
    tgt = rng.integers(0, T, C).astype(np.int32)
    cand = rng.integers(0, 4096, C).astype(np.int32)
    th = f32(rng.uniform(rob.lo, rob.hi, (C, rob.n)))
    P64 = orc.make_params(seed=seed)
    g = _ccd_gpu(ctx, rid, rob.n, tg, tgt, cand, th, k, api.make_params(), seed)
    o = orc.ccd_iteration(orob, P64, tg, tgt, cand, k, th)
    tol = TOL * max(1.0, reach(rob) / 1.5)
    # Trial residuals everywhere: at the optimal rotation the residual is
    # stationary in the angle.  Position steps within the bound of their
    # binary32 sensitivity (strict 1e-5 where that bound is below it).
    sens = _ccd_sensitivity(orob, rob, th, tg, tgt, P64.proj_eps)
    good_j = sens < tol
    assert good_j.mean() > 0.4
    assert np.max(np.abs(g["rp"] - o["rp"])) < tol
    tol_j = np.maximum(tol, sens)
    assert np.all(np.abs(g["dp"] - o["dp"]) < tol_j)
    # the orientation a position step leaves moves with the step (slope <= 1)
    assert np.all(np.abs(g["op"] - o["op"]) < tol_j)
    for key in ("dq", "pq", "rq"):
        assert np.max(np.abs(g[key] - o[key])) < tol, key
    # Greedy choices where no comparison of the greedy choice of Alg. 3 is within reach of
    # rounding: every other trial's score differs from the chosen one's by more
    # than the tie band plus twice the score error the trial errors allow
    # (d s = 2 |e_p| d|e_p| / eps_p^2 + 2 |w| d|w| / eps_o^2 + squares).
    def score(ep, eo):
        return (ep / P64.eps_pos) ** 2 + (eo / P64.eps_ori) ** 2

    def dscore(ep, eo, dep, deo):
        return (2 * ep * dep + dep ** 2) / P64.eps_pos ** 2 + (2 * eo * deo + deo ** 2) / P64.eps_ori ** 2

    def clear(s_, ds_, pick):
        sb, db = s_[np.arange(C), pick][:, None], ds_[np.arange(C), pick][:, None]
        gap = np.abs(s_ - sb) - P64.cd_tie * np.maximum(s_, sb) * 2 - 2 * (ds_ + db)
        gap[np.arange(C), pick] = np.inf
        return gap.min(axis=1) > 0

    sp, so = score(o["rp"], o["op"]), score(o["pq"], o["rq"])
    robust = clear(sp, dscore(o["rp"], o["op"], tol, tol_j), o["jp"]) & \
        clear(so, dscore(o["pq"], o["rq"], tol, tol), o["jo"])
    same = o["jp"] == o["jo"]
    step_gap = np.abs(np.abs(o["dp"][np.arange(C), o["jp"]]) - np.abs(o["dq"][np.arange(C), o["jo"]]))
    robust &= ~same | (step_gap > 2 * tol_j[np.arange(C), o["jp"]])
    assert robust.mean() > 0.6, robust.mean()
    assert np.array_equal(g["jp"][robust], o["jp"][robust])
    assert np.array_equal(g["jo"][robust], o["jo"][robust])
    tol_c = np.maximum(tol, sens[np.arange(C), o["jp"]])[:, None]
    assert np.all((np.abs(g["th_hat"] - o["theta_hat"]) < tol_c)[robust])
    robust_a = robust & (o["margin_acc"] > MARGIN)
    assert np.array_equal(g["accepted"][robust_a], o["accepted"][robust_a].astype(bool))
    assert 0.05 < o["accepted"][robust_a].mean() <= 1.0
    assert np.all((np.abs(g["theta"] - o["theta"]) < tol_c)[robust_a])


def test_po_ccd_trajectories_match(ctx):
    """Alg. 3 from sampled seeds for max_iters iterations: most candidates
    follow the oracle's trajectory exactly (divergence needs a near-tie)."""
    wl = inputs.cfg1()
    rob = wl.robot
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    T, S = 16, 64
    tg = f32(orc.pose(orob, f32(wl.theta_gen[:T])))
    tgt = np.repeat(np.arange(T), S).astype(np.int32)
    cand = np.tile(np.arange(S), T).astype(np.int32)
    C = T * S
    th = torch.empty((7, C), device="cuda")
    score = torch.empty((C,), device="cuda")
    perr = torch.empty((C,), device="cuda")
    oerr = torch.empty((C,), device="cuda")
    iters = torch.empty((C,), dtype=torch.int32, device="cuda")
    P = api.make_params()
    hjcd.hjcd_po_ccd(ctx.h, rid, T, dev(tg), wl.eps_pos, wl.eps_ori, wl.seed, P, C, dev(tgt, torch.int32),
                     dev(cand, torch.int32), None, th, C, 0, P.cd_max_iters, score, perr, oerr, iters)
    o = orc.po_ccd(orob, orc.make_params(wl.eps_pos, wl.eps_ori, seed=wl.seed), tg, tgt, cand)
    same = np.max(np.abs(host(th).T - o["theta"]), axis=1) < 1e-4
    assert same.mean() > 0.85
    it = host(iters).astype(int)
    assert np.mean(it[same] == o["iters"][same]) > 0.98
    conv_g = (host(perr) ** 2 < P.cd_eps_pos2) & (host(oerr) ** 2 < P.cd_eps_ori2)
    conv_o = (o["perr"] ** 2 < P.cd_eps_pos2) & (o["oerr"] ** 2 < P.cd_eps_ori2)
    assert abs(conv_g.mean() - conv_o.mean()) < 0.03
    sc = host(score)
    assert np.allclose(sc[same], o["score"][same], rtol=1e-3, atol=1e-3)


# ----------------------------------------------------------------------------
# a5: top-K and perturbed duplication

def test_topk_dup_parity(ctx):
    rob = inputs.panda()
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(3)
    Ms = np.array([64, 1, 3, 1000, 333, 4096], np.int64)
    m_off = np.concatenate([[0], np.cumsum(Ms)])
    score = np.round(rng.uniform(0, 4, m_off[-1]), 1).astype(np.float32)   # ties
    score[::17] = np.float32(0.5)
    thM = f32(rng.uniform(rob.lo, rob.hi, (m_off[-1], 7)))
    seed = 99
    P64 = orc.make_params(seed=seed)
    o = orc.topk_dup(orob, P64, m_off, score.astype(np.float64), thM)
    b_off = o["b_off"]
    CB = int(b_off[-1])
    thB = torch.empty((7, CB), device="cuda")
    src = torch.empty((CB,), dtype=torch.int32, device="cuda")
    hjcd.hjcd_topk_dup(ctx.h, rid, len(Ms), dev(m_off, torch.int64), dev(score), soa(thM), int(m_off[-1]),
                       dev(b_off, torch.int64), thB, CB, src, seed, api.make_params())
    assert np.array_equal(host(src).astype(np.int32), o["src"])
    assert np.max(np.abs(host(thB).T - o["theta"])) < 1e-6


# ----------------------------------------------------------------------------
# a6: one PJ-IK iteration, traced

def _lm_gpu(ctx, rid, n, tg, tgt, cand, th, k, params, seed):
    C = len(tgt)
    theta = soa(th)
    J = torch.zeros((6 * n, C), device="cuda")
    W = torch.zeros((6, C), device="cuda")
    d = torch.zeros((n, C), device="cuda")
    br = torch.zeros((C,), dtype=torch.int32, device="cuda")
    al = torch.zeros((C,), device="cuda")
    # the fallback steps are written only where the full step failed: NaN / -1 elsewhere
    dd = torch.full((n, C), float("nan"), device="cuda")
    sj = torch.full((C,), -1, dtype=torch.int32, device="cuda")
    ss = torch.full((C,), float("nan"), device="cuda")
    tr = hjcd.hjcd_lm_trace(*[hjcd.ptr(x) for x in (J, W, d, br, al, dd, sj, ss)])
    hjcd.hjcd_pjik(ctx.h, rid, len(tg), dev(tg), 1e-3, 1e-2, seed, params, C, dev(tgt, torch.int32),
                   dev(cand, torch.int32), theta, C, k, 1, trace=tr)
    return dict(J=host(J).T.reshape(C, 6, n), W=host(W).T, d_lm=host(d).T, branch=host(br).astype(int),
                alpha=host(al), theta=host(theta).T, d_dog=host(dd).T, sc_joint=host(sj).astype(int),
                sc_step=host(ss))


def _cond(J, W, lam):
    """Condition number of the 6x6 system after diagonal equilibration (the
    one that bounds a Cholesky solve's rounding error, van der Sluis)."""
    Jw = W[:, None] * J
    Dg = np.sum(Jw * Jw, axis=0) + 1e-9
    Ah = Jw / np.sqrt(Dg)
    M = Ah @ Ah.T + lam * np.eye(6)
    s = 1 / np.sqrt(np.diag(M))
    ev = np.linalg.eigvalsh(M * s[:, None] * s[None, :])
    return ev[-1] / ev[0]


@pytest.mark.parametrize("which", ["panda", "chain12", "chain20", "chain24"])
def test_lm_iteration_trace_parity(ctx, which):
    rob = dict(robots())[which]
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(4)
    T, C, k, seed = 11, 1031, 0, 5
    tth = rng.uniform(rob.lo, rob.hi, (T, rob.n))
    tg = f32(orc.pose(orob, f32(tth)))
    tgt = rng.integers(0, T, C).astype(np.int32)
    cand = np.arange(C).astype(np.int32)
    sig = np.where(np.arange(C) % 3 == 0, 0.3, 0.05)[:, None]
    th = f32(np.clip(tth[tgt] + rng.normal(0, 1, (C, rob.n)) * sig, rob.lo, rob.hi))
    P64 = orc.make_params(seed=seed)
    g = _lm_gpu(ctx, rid, rob.n, tg, tgt, cand, th, k, api.make_params(), seed)
    o = orc.lm_iteration(orob, P64, tg, tgt, cand, k, th)
    tol = TOL * max(1.0, reach(rob) / 1.5)
    assert np.max(np.abs(g["J"] - o["J"])) < tol
    assert np.max(np.abs(g["W"] / o["W"] - 1)) < 1e-5
    # The LM step solves a 6x6 SPD system of condition number cond; rounding the
    # inputs to binary32 (u = 2^-24) already moves its exact solution by about
    # cond * u * |step|.  Strict 1e-5 agreement where that is below the
    # tolerance (cond < 300), and the derived bound 1e-5 + 8 cond u |step| everywhere.
    cond = np.array([_cond(o["J"][c], o["W"][c], P64.lm_lambda) for c in range(C)])
    u = 2.0 ** -24
    bound = tol + 8 * cond * u * np.max(np.abs(o["d_lm"]), axis=1)
    assert np.all(np.max(np.abs(g["d_lm"] - o["d_lm"]), axis=1) < bound)
    well = cond < 100
    assert well.mean() > 0.15
    assert np.max(np.abs(g["d_lm"] - o["d_lm"])[well]) < tol
    robust = well & (o["ls_margin"] > 1e-4)
    assert np.array_equal(g["branch"][robust], o["branch"][robust])
    assert np.array_equal(g["alpha"][robust], o["alpha"][robust].astype(np.float32).astype(np.float64))
    assert np.max(np.abs(g["theta"] - o["theta"])[robust]) < tol
    assert set(np.unique(o["branch"][robust])) >= {0}


def _dogleg_sensitivity(J, e, wo, R, mu, reach_m, rng, ulps):
    """How far the dogleg step of Eq. dogleg moves when its inputs carry the
    errors of binary32 kinematics: absolute errors of `ulps` u reach on the
    Jacobian's position rows and the position residual, `ulps` u on its axis
    rows and the orientation residual (u = 2^-24), with W recomputed from the
    perturbed Jacobian; the largest change of the oracle's step over eight
    random perturbations.  The step is continuous but not Lipschitz where the
    dogleg segment touches the trust-region sphere (the boundary point moves
    like the square root of the input error) and it amplifies errors by the
    condition of the Gauss-Newton system, so no fixed tolerance fits every
    candidate."""
    u = 2.0 ** -24
    scale = np.array([reach_m] * 3 + [1.0] * 3) * ulps * u
    wc = np.array([1.0, 1.0, 1.0, wo, wo, wo])

    def step(J_, e_):
        W = wc / np.maximum(np.linalg.norm(J_, axis=1), 1e-6)
        return orc.dogleg_step(W[:, None] * J_, W * e_, R, mu)

    d0 = step(J, e)
    worst = 0.0
    for _ in range(8):
        d1 = step(J + scale[:, None] * rng.standard_normal(J.shape), e + scale * rng.standard_normal(6))
        worst = max(worst, float(np.max(np.abs(d1 - d0))))
    return worst


@pytest.mark.parametrize("which,A", [("panda", 4), ("chain12", 4), ("chain20", 1), ("chain24", 0)])
def test_lm_fallback_branch_trace_parity(ctx, which, A):
    """Alg. 4's failure path, branch by branch.  Inputs: candidates after 10
    oracle PJ-IK iterations from uniform seeds, where a third or more of the
    iterations fail the full step.  Where the full step failed on the GPU the
    trace holds its dogleg step (Eq. dogleg), its single-coordinate joint and
    step (Eq. single-coord); they are compared with the oracle's, and where
    the oracle's decisions are clear so are the branch, the accepted alpha
    and the new theta.  The dogleg (branch 1) and the single coordinate
    (branch 2) must both occur among the compared candidates (the
    perturbation, branch 3, has its own forced case below); the longer chains
    fail the full step less often, so they run with a shallower line search
    (depth A) to reach the fallbacks."""
    rob = dict(robots())[which]
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(61)
    T, C, k, seed = 11, 4099, 10, 5
    tg = f32(orc.pose(orob, f32(rng.uniform(rob.lo, rob.hi, (T, rob.n)))))
    tgt = rng.integers(0, T, C).astype(np.int32)
    cand = np.arange(C).astype(np.int32)
    P64 = orc.make_params(seed=seed, lm_max_iters=k, lm_A=A)
    th = f32(orc.pjik(orob, P64, tg, tgt, cand, rng.uniform(rob.lo, rob.hi, (C, rob.n)))["theta"])
    g = _lm_gpu(ctx, rid, rob.n, tg, tgt, cand, th, k, api.make_params(lm_A=A), seed)
    o = orc.lm_iteration(orob, P64, tg, tgt, cand, k, th)
    tol = TOL * max(1.0, reach(rob) / 1.5)
    u = 2.0 ** -24
    fell = g["sc_joint"] >= 0                     # the GPU took the failure path
    assert np.array_equal(fell, (g["branch"] != 0) | (g["alpha"] < 1))
    assert fell.sum() > 100
    cond_lm = np.array([_cond(o["J"][c], o["W"][c], P64.lm_lambda) for c in range(C)])
    res = np.array([orc.residual(orob, th[c], tg[tgt[c]]) for c in range(C)])
    Jw = o["W"][:, :, None] * o["J"]
    bw = o["W"] * res
    # dogleg step: 1e-5 where it moves less than a third of that under 16-ulp input errors,
    # everywhere the tolerance plus twenty times that movement (the device's own binary32
    # solve and sums add errors of their own beyond those of its inputs)
    sens = np.zeros(C)
    srng = np.random.default_rng(62)
    for c in np.nonzero(fell)[0]:
        sens[c] = _dogleg_sensitivity(o["J"][c], res[c], P64.eps_pos / P64.eps_ori, P64.lm_trust_R,
                                      P64.lm_gn_reg, max(1.0, reach(rob)), srng, 16)
    ddog_err = np.max(np.abs(g["d_dog"] - o["d_dog"]), axis=1)
    assert np.all(ddog_err[fell] < (tol + 20 * sens)[fell])
    steady = fell & (sens < 0.3 * tol)
    assert steady.sum() > 25
    assert np.max(ddog_err[steady]) < tol
    # the device's steps stay in the trust region, up to the rounding of the boundary point (a
    # binary32 |d_gn|^2 taken as the 6x6 form y2.M0 y2 once let Gauss-Newton steps of norm 2.7
    # through with R = 0.3)
    assert np.all(np.linalg.norm(g["d_dog"][fell], axis=1) <= P64.lm_trust_R * 1.01)
    # single coordinate: the joint wherever the largest |g_i| is clear, the step on that joint
    gr = np.einsum("cri,cr->ci", Jw, bw)
    ag = np.sort(np.abs(gr), axis=1)
    clear = fell & ((ag[:, -1] - ag[:, -2]) > 1e-4 * ag[:, -1])
    assert clear.sum() > 50
    assert np.array_equal(g["sc_joint"][clear], o["sc_joint"][clear])
    # the 1-D step g_i / |(WJ)_i|^2: its rounding grows with the cancellation in g_i
    i_s = o["sc_joint"]
    canc = np.array([np.sum(np.abs(Jw[c, :, i_s[c]] * bw[c])) / max(abs(gr[c, i_s[c]]), 1e-300) for c in range(C)])
    sc_bound = tol + 16 * canc * u * np.abs(o["sc_step"])
    assert np.all(np.abs(g["sc_step"] - o["sc_step"])[clear] < sc_bound[clear])
    # decisions where the oracle's cost comparisons are clear (relative margin 1e-4) and the
    # steps they compare are known well: the LM step well conditioned, the dogleg step within
    # 1e-3; the new theta within the tolerance of the step taken
    ddog_bound = tol + 20 * sens
    robust = fell & clear & (cond_lm < 100) & (ddog_bound < 1e-3) & (o["ls_margin"] > 1e-4)
    assert np.array_equal(g["branch"][robust], o["branch"][robust])
    assert np.array_equal(g["alpha"][robust], o["alpha"][robust].astype(np.float32).astype(np.float64))
    dth = np.max(np.abs(g["theta"] - o["theta"]), axis=1)
    assert np.all(dth[robust & ((o["branch"] == 0) | (o["branch"] == 2))] < tol)
    assert np.all(dth[robust & (o["branch"] == 1)] < ddog_bound[robust & (o["branch"] == 1)])
    br = set(np.unique(o["branch"][robust]))
    assert {1, 2} <= br, br


def test_lm_perturbation_branch_parity(ctx):
    """Branch 3 of Alg. 4, forced: a stretched planar arm whose target lies
    straight ahead beyond reach with the same orientation has a zero gradient,
    so the LM, dogleg and single-coordinate steps are zero on both sides and no
    trial lowers the cost; both perturb with the candidate's PJ-IK normal
    stream, whose draws must agree."""
    rob = inputs.planar([0.5, 0.4, 0.3])
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    C, seed = 64, 21
    th = np.zeros((C, 3))
    tg = f32(orc.pose(orob, th[:1]))
    tg[0, 0] += 0.6
    tgt = np.zeros(C, np.int32)
    cand = np.arange(C).astype(np.int32)
    for k in (0, 13):
        g = _lm_gpu(ctx, rid, 3, tg, tgt, cand, th, k, api.make_params(), seed)
        o = orc.lm_iteration(orob, orc.make_params(seed=seed), tg, tgt, cand, k, th)
        assert np.all(o["branch"] == 3) and np.all(g["branch"] == 3)
        assert np.all(g["d_lm"] == 0) and np.all(g["d_dog"] == 0) and np.all(g["sc_step"] == 0)
        assert np.max(np.abs(g["theta"] - o["theta"])) < TOL
        assert np.std(g["theta"]) > 0.005  # the draws differ per candidate


def test_pjik_converges_like_the_oracle(ctx):
    rob = inputs.panda()
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(5)
    T, C = 32, 2048
    tth = rng.uniform(rob.lo, rob.hi, (T, 7))
    tg = f32(orc.pose(orob, f32(tth)))
    tgt = np.repeat(np.arange(T), C // T).astype(np.int32)
    cand = np.tile(np.arange(C // T), T).astype(np.int32)
    th = f32(np.clip(tth[tgt] + rng.normal(0, 0.08, (C, 7)), rob.lo, rob.hi))
    theta = soa(th)
    perr = torch.empty((C,), device="cuda")
    oerr = torch.empty((C,), device="cuda")
    P = api.make_params()
    hjcd.hjcd_pjik(ctx.h, rid, T, dev(tg), 1e-3, 1e-2, 7, P, C, dev(tgt, torch.int32), dev(cand, torch.int32),
                   theta, C, 0, P.lm_max_iters, None, perr, oerr)
    o = orc.pjik(orob, orc.make_params(seed=7), tg, tgt, cand, th)
    ok_g = (host(perr) < 1e-3) & (host(oerr) < 1e-2)
    ok_o = (o["perr"] < 1e-3) & (o["oerr"] < 1e-2)
    assert abs(ok_g.mean() - ok_o.mean()) < 0.01
    # every GPU result claimed converged is converged under the oracle's kinematics
    gth = host(theta).T
    for c in np.nonzero(ok_g)[0][:400]:
        e = orc.residual(orob, gth[c], tg[tgt[c]])
        assert np.linalg.norm(e[:3]) < 1e-3 + 1e-5 and np.linalg.norm(e[3:]) < 1e-2 + 1e-5
    assert np.all(gth >= rob.lo - 1e-7) and np.all(gth <= rob.hi + 1e-7)


@pytest.mark.parametrize("A,beta", [(0, 2.0), (2, 3.0), (7, 2.0)])
def test_pjik_line_search_depths(ctx, A, beta):
    """Other line-search depths A and ratios beta (the trial rows, the alpha
    table and the single-coordinate search all follow A): convergence as the
    oracle's with the same parameters, every claimed solution verified."""
    rob = inputs.panda()
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(40 + A)
    T, C = 16, 1024
    tth = rng.uniform(rob.lo, rob.hi, (T, 7))
    tg = f32(orc.pose(orob, f32(tth)))
    tgt = np.repeat(np.arange(T), C // T).astype(np.int32)
    cand = np.tile(np.arange(C // T), T).astype(np.int32)
    th = f32(np.clip(tth[tgt] + rng.normal(0, 0.1, (C, 7)), rob.lo, rob.hi))
    theta = soa(th)
    perr = torch.empty((C,), device="cuda")
    oerr = torch.empty((C,), device="cuda")
    P = api.make_params(lm_A=A, lm_beta=beta)
    hjcd.hjcd_pjik(ctx.h, rid, T, dev(tg), 1e-3, 1e-2, 7, P, C, dev(tgt, torch.int32), dev(cand, torch.int32),
                   theta, C, 0, P.lm_max_iters, None, perr, oerr)
    o = orc.pjik(orob, orc.make_params(seed=7, lm_A=A, lm_beta=beta), tg, tgt, cand, th)
    ok_g = (host(perr) < 1e-3) & (host(oerr) < 1e-2)
    ok_o = (o["perr"] < 1e-3) & (o["oerr"] < 1e-2)
    assert abs(ok_g.mean() - ok_o.mean()) < 0.02
    gth = host(theta).T
    for c in np.nonzero(ok_g)[0][:200]:
        e = orc.residual(orob, gth[c], tg[tgt[c]])
        assert np.linalg.norm(e[:3]) < 1e-3 + 1e-5 and np.linalg.norm(e[3:]) < 1e-2 + 1e-5
    assert np.all(gth >= rob.lo - 1e-7) and np.all(gth <= rob.hi + 1e-7)


# ----------------------------------------------------------------------------
# a7: collision filter

def _collision_case(rob, scene, C, seed):
    rng = np.random.default_rng(seed)
    return f32(rng.uniform(rob.lo, rob.hi, (C, rob.n)))


@pytest.mark.parametrize("case", ["panda_scene", "panda_self", "chain20_scene"])
def test_collision_verdict_parity(ctx, case):
    if case.startswith("panda"):
        rng = np.random.default_rng(inputs.CFG_SEED[2])
        rob = inputs.panda_with_spheres(rng)
        scene = inputs.random_scene(rng, 200, 20)
    else:
        rob = inputs.cfg3_chains()[5]
        rng = np.random.default_rng(8)
        scene = inputs.random_scene(rng, 100, 0, lo=(-2, -2, -1), hi=(2, 2, 2))
    use_scene = not case.endswith("self")
    rid = ctx.add_robot(rob)
    sid = ctx.set_scene(scene) if use_scene else -1
    orob = orc.Robot(rob)
    osc = orc.Scene(scene) if use_scene else None
    C = 6000 + 11
    th = _collision_case(rob, scene, C, 9)
    hit = host(ctx.collide(rid, sid, soa(th))).astype(bool)
    ref, margin = orc.collide(orob, osc, th)
    certain = margin >= 1e-6
    assert certain.mean() > 0.99
    assert np.array_equal(hit[certain], ref[certain])
    assert 0.0 < ref.mean() < 1.0


# ----------------------------------------------------------------------------
# a8: ranking

def _rank_gpu(ctx, rid, b_off, th, score, perr, oerr, hit, k, eps, q_ref=None):
    T, CB = len(b_off) - 1, int(b_off[-1])
    n = th.shape[1]
    oq = torch.zeros((T, k, n), device="cuda")
    oe = torch.zeros((T, k, 2), device="cuda")
    oc = torch.zeros((T,), dtype=torch.int32, device="cuda")
    hjcd.hjcd_rank(ctx.h, rid, T, dev(b_off, torch.int64), soa(th), CB, dev(score), dev(perr), dev(oerr),
                   None if hit is None else dev(hit, torch.uint8), eps[0], eps[1],
                   None if q_ref is None else dev(q_ref), k, oq, oe, oc)
    return host(oq), host(oe), host(oc).astype(int)


def test_rank_parity(ctx):
    """Alg. 2's final ranking, bit-exact: collision-free candidates, those
    within the tolerances first (reading c20), each group by score, ties to the
    lower index; rows past the count NaN."""
    rob = inputs.panda()
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(10)
    Bs = np.array([50, 1, 1000, 7, 4096], np.int64)
    b_off = np.concatenate([[0], np.cumsum(Bs)])
    CB = int(b_off[-1])
    th = f32(rng.uniform(rob.lo, rob.hi, (CB, 7)))
    score = np.round(rng.uniform(0, 3, CB), 1).astype(np.float32)
    perr = rng.uniform(0, 2e-3, CB).astype(np.float32)
    oerr = rng.uniform(0, 2e-2, CB).astype(np.float32)
    # a converged candidate whose score is above a non-converged one's, at the head of target 0
    perr[0:2], oerr[0:2], score[0:2] = [1.05e-3, 0.9e-3], [0.0, 0.9e-2], [0.0, 0.05]
    hit = (rng.uniform(size=CB) < 0.6).astype(np.uint8)
    hit[0:2] = 0
    hit[b_off[1]:b_off[2]] = 1
    k = 16
    T = len(Bs)
    eps = (np.float32(1e-3), np.float32(1e-2))  # both sides compare in binary32 values
    q, e, cnt = _rank_gpu(ctx, rid, b_off, th, score, perr, oerr, hit, k, eps)
    o = orc.rank(orob, b_off, th, score.astype(np.float64), f32(perr), f32(oerr), hit, k,
                 float(eps[0]), float(eps[1]))
    assert np.array_equal(cnt, o["count"])
    assert np.array_equal(q[0, 0], th[1])  # converged first although its score is higher
    for t in range(T):
        assert np.array_equal(q[t, :cnt[t]], o["q"][t, :cnt[t]])
        assert np.array_equal(e[t, :cnt[t]], o["err"][t, :cnt[t]])
        assert np.all(np.isnan(q[t, cnt[t]:])) and np.all(np.isnan(e[t, cnt[t]:]))
    # without a collision mask every target fills its rows
    q2, e2, c2 = _rank_gpu(ctx, rid, b_off, th, score, perr, oerr, None, k, eps)
    o2 = orc.rank(orob, b_off, th, score.astype(np.float64), f32(perr), f32(oerr), None, k,
                  float(eps[0]), float(eps[1]))
    assert np.array_equal(c2, o2["count"]) and np.array_equal(q2[:, :1], o2["q"][:, :1])


def test_rank_nearest_parity(ctx):
    """The tracking ranking (reading c24) against the oracle's: within the
    tolerances by squared joint distance to the reference, then by score.  The
    distances are sums in binary32 on the GPU and in double in the oracle, so
    the order is compared where consecutive distances differ clearly."""
    rob = inputs.panda()
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(12)
    Bs = np.array([64, 300, 1, 2000], np.int64)
    b_off = np.concatenate([[0], np.cumsum(Bs)])
    CB, T, k = int(b_off[-1]), len(Bs), 24
    th = f32(rng.uniform(rob.lo, rob.hi, (CB, 7)))
    q_ref = f32(rng.uniform(rob.lo, rob.hi, (T, 7)))
    score = rng.uniform(0, 3, CB).astype(np.float32)
    perr = rng.uniform(0, 2e-3, CB).astype(np.float32)
    oerr = rng.uniform(0, 2e-2, CB).astype(np.float32)
    hit = (rng.uniform(size=CB) < 0.3).astype(np.uint8)
    eps = (np.float32(1e-3), np.float32(1e-2))
    q, e, cnt = _rank_gpu(ctx, rid, b_off, th, score, perr, oerr, hit, k, eps, q_ref=q_ref)
    o = orc.rank(orob, b_off, th, score.astype(np.float64), f32(perr), f32(oerr), hit, k,
                 float(eps[0]), float(eps[1]), q_ref=q_ref)
    assert np.array_equal(cnt, o["count"])
    compared = 0
    for t in range(T):
        c = cnt[t]
        conv = (o["err"][t, :c, 0] <= eps[0]) & (o["err"][t, :c, 1] <= eps[1])
        d = np.sum((o["q"][t, :c] - q_ref[t]) ** 2, axis=1)
        # rows whose distance is clear of both neighbours' (relative 1e-5) must match exactly
        gap = np.full(c, np.inf)
        dd = np.abs(np.diff(d)) / np.maximum(d[1:], 1e-12)
        gap[1:] = np.minimum(gap[1:], dd)
        gap[:-1] = np.minimum(gap[:-1], dd)
        sure = ~conv | (gap > 1e-5)
        assert np.array_equal(q[t, :c][sure], o["q"][t, :c][sure])
        compared += int((sure & conv).sum())
    assert compared > 20


def test_philox_blocks_are_bit_exact(ctx):
    """The kernels' Philox4x32-10 generator, word for word: the published
    known-answer vectors and the oracle's generator on the counters of every
    phase of the method's streams."""
    gold = []
    with open(os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")) as f:
        for ln in f:
            if ln.strip() and not ln.startswith("#"):
                gold.append([int(x, 16) for x in ln.split()])
    assert len(gold) == 3
    for r in gold:
        ctr = torch.tensor(np.array(r[0:4], np.uint32).view(np.int32), dtype=torch.int32, device="cuda")
        out = torch.zeros(4, dtype=torch.int32, device="cuda")
        hjcd.hjcd_philox(ctx.h, 1, ctr, r[4] | (r[5] << 32), out)
        got = out.cpu().numpy().view(np.uint32)
        assert [int(x) for x in got] == r[6:10]
    rng = np.random.default_rng(13)
    N = 4096
    ctr = rng.integers(0, 2 ** 32, (N, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:512, 2] = (rng.integers(1, 5, 512) << 24) | rng.integers(0, 64, 512)  # phase << 24 | iteration
    key = int(rng.integers(0, 2 ** 63)) * 2 + 1
    d_ctr = torch.tensor(ctr.view(np.int32), device="cuda")
    d_out = torch.zeros((N, 4), dtype=torch.int32, device="cuda")
    hjcd.hjcd_philox(ctx.h, N, d_ctr, key, d_out)
    got = d_out.cpu().numpy().view(np.uint32)
    kw = np.array([key & 0xFFFFFFFF, key >> 32], np.uint32)
    for i in range(N):
        assert np.array_equal(got[i], orc.philox(ctr[i], kw)), i


# ----------------------------------------------------------------------------
# the whole method (Alg. 2)

def _verify(orob, osc, rob, tg, q, err, cnt, eps_pos, eps_ori):
    """Every returned solution: oracle errors equal the reported ones, inside
    the limits, collision-free under brute force; returns the success mask."""
    T = len(tg)
    succ = np.zeros(T, bool)
    for t in range(T):
        for r in range(cnt[t]):
            e = orc.residual(orob, q[t, r], tg[t])
            assert abs(np.linalg.norm(e[:3]) - err[t, r, 0]) < 1e-5
            assert abs(np.linalg.norm(e[3:]) - err[t, r, 1]) < 1e-5
            assert np.all(q[t, r] >= rob.lo - 1e-7) and np.all(q[t, r] <= rob.hi + 1e-7)
        if cnt[t] and len(rob.sph_body):
            hit, margin = orc.collide(orob, osc, q[t, :cnt[t]])
            assert not np.any(hit & (margin >= 1e-6))
        succ[t] = cnt[t] > 0 and err[t, 0, 0] <= eps_pos and err[t, 0, 1] <= eps_ori
    return succ


def test_solve_open_world_matches_oracle(ctx):
    """cfg1 workload shape (Panda, 64 seeds, no obstacles) on 200 targets."""
    wl = inputs.cfg1()
    rob = wl.robot
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(11)
    T = 200
    tg = f32(orc.pose(orob, f32(np.concatenate([wl.theta_gen, rng.uniform(rob.lo, rob.hi, (T - 16, 7))]))))
    q, err, cnt = ctx.solve(rid, -1, dev(tg), wl.n_samples, 4, wl.seed, 7)
    q, err, cnt = host(q), host(err), host(cnt).astype(int)
    succ_g = _verify(orob, None, rob, tg, q, err, cnt, wl.eps_pos, wl.eps_ori)
    o = orc.solve(orob, None, orc.make_params(wl.eps_pos, wl.eps_ori, seed=wl.seed), tg, wl.n_samples, 4)
    succ_o = (o["count"] > 0) & (o["err"][:, 0, 0] <= wl.eps_pos) & (o["err"][:, 0, 1] <= wl.eps_ori)
    assert abs(succ_g.mean() - succ_o.mean()) <= 0.01 + 1e-12
    assert succ_g.mean() > 0.9


def _cfg2_targets(ctx, rid, sid, orob, osc, wl, T):
    """Targets from joint samples the oracle finds collision-free."""
    pool = f32(wl.theta_gen)
    hit, _ = orc.collide(orob, osc, pool[: 12 * T])
    keep = pool[: 12 * T][~hit][:T]
    assert len(keep) == T
    return f32(orc.pose(orob, keep))


def test_solve_with_obstacles_matches_oracle(ctx):
    """cfg2 workload shape (Panda + 60 spheres, 200 spheres + 20 boxes) with
    256 seeds on 200 targets: success within 1 point of the oracle."""
    wl = inputs.cfg2(200, 256)
    rob, sc = wl.robot, wl.scene
    rid, sid = ctx.add_robot(rob), ctx.set_scene(sc)
    orob, osc = orc.Robot(rob), orc.Scene(sc)
    T, S, k = 200, 256, 4
    tg = _cfg2_targets(ctx, rid, sid, orob, osc, wl, T)
    q, err, cnt = ctx.solve(rid, sid, dev(tg), S, k, wl.seed, 7)
    q, err, cnt = host(q), host(err), host(cnt).astype(int)
    succ_g = _verify(orob, osc, rob, tg, q, err, cnt, wl.eps_pos, wl.eps_ori)
    o = orc.solve(orob, osc, orc.make_params(wl.eps_pos, wl.eps_ori, seed=wl.seed), tg, S, k)
    succ_o = (o["count"] > 0) & (o["err"][:, 0, 0] <= wl.eps_pos) & (o["err"][:, 0, 1] <= wl.eps_ori)
    assert abs(succ_g.mean() - succ_o.mean()) <= 0.01 + 1e-12
    assert succ_g.mean() > 0.8


def test_solve_full_size_sampled_verification(ctx):
    """cfg2 at full size (1000 targets x 1000 seeds, one batched launch per
    phase, as the benchmark runs it): every solution of a sample of targets
    is re-verified by the oracle."""
    wl = inputs.cfg2()
    rob, sc = wl.robot, wl.scene
    rid, sid = ctx.add_robot(rob), ctx.set_scene(sc)
    orob, osc = orc.Robot(rob), orc.Scene(sc)
    tg = _cfg2_targets(ctx, rid, sid, orob, osc, wl, wl.n_targets)
    q, err, cnt = ctx.solve(rid, sid, dev(tg), wl.n_samples, 16, wl.seed, 7)
    q, err, cnt = host(q), host(err), host(cnt).astype(int)
    idx = np.random.default_rng(12).choice(wl.n_targets, 24, replace=False)
    succ = _verify(orob, osc, rob, tg[idx], q[idx], err[idx], cnt[idx], wl.eps_pos, wl.eps_ori)
    assert succ.mean() > 0.8
    # ranking invariants over all targets
    for t in range(wl.n_targets):
        assert ranked_order_ok(err[t, :cnt[t]], wl.eps_pos, wl.eps_ori), t


# ----------------------------------------------------------------------------
# boundary behaviour

def test_host_and_device_buffers_give_identical_results(ctx):
    wl = inputs.cfg1()
    rid = ctx.add_robot(wl.robot)
    orob = orc.Robot(wl.robot)
    tg = f32(orc.pose(orob, f32(wl.theta_gen)))
    a = ctx.solve(rid, -1, dev(tg), 64, 4, wl.seed, 7)
    hq = torch.zeros((16, 4, 7)).pin_memory()
    he = torch.zeros((16, 4, 2)).pin_memory()
    hc = torch.zeros((16,), dtype=torch.int32)
    ctx.solve(rid, -1, torch.as_tensor(tg, dtype=torch.float32), 64, 4, wl.seed, 7, out=(hq, he, hc))
    assert torch.equal(a[0].cpu(), hq) and torch.equal(a[1].cpu(), he) and torch.equal(a[2].cpu(), hc)
    b = ctx.solve(rid, -1, dev(tg), 64, 4, wl.seed, 7)
    assert all(torch.equal(x, y) for x, y in zip(a, b))


def test_edge_cases(ctx):
    rob = inputs.panda()
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    tg = f32(orc.pose(orob, f32(inputs.cfg1().theta_gen[:3])))
    # no targets
    o = ctx.opts(8, 1, 0)
    hjcd.hjcd_solve(ctx.h, rid, -1, 0, None, o, None, None, None)
    # one seed per target: K = 1, B = 1
    q, err, cnt = ctx.solve(rid, -1, dev(tg), 1, 3, 1, 7)
    assert np.all(host(cnt) == 1)
    # top_k above B returns B solutions
    q, err, cnt = ctx.solve(rid, -1, dev(tg), 6, 64, 1, 7)
    assert np.all(host(cnt) == 6)
    # the largest seed count
    q, err, cnt = ctx.solve(rid, -1, dev(tg[:2]), hjcd.HJCD_MAX_SAMPLES, 2, 1, 7)
    assert np.all(host(cnt) == 2)
    # argument errors
    with pytest.raises(hjcd.HjcdError) as ei:
        ctx.solve(rid, -1, dev(tg), hjcd.HJCD_MAX_SAMPLES + 1, 1, 1, 7)
    assert ei.value.status == hjcd.HJCD_EINVAL
    with pytest.raises(hjcd.HjcdError) as ei:
        ctx.solve(rid + 100, -1, dev(tg), 8, 1, 1, 7)
    assert ei.value.status == hjcd.HJCD_ENOTFOUND
    with pytest.raises(hjcd.HjcdError) as ei:
        ctx.solve(rid, 12345, dev(tg), 8, 1, 1, 7)
    assert ei.value.status == hjcd.HJCD_ENOTFOUND
    bad = tg.copy()
    bad[1, 3:] = 0
    with pytest.raises(hjcd.HjcdError) as ei:
        ctx.solve(rid, -1, torch.as_tensor(bad, dtype=torch.float32), 8, 1, 1, 7,
                  out=(torch.zeros((3, 1, 7)), torch.zeros((3, 1, 2)), torch.zeros((3,), dtype=torch.int32)))
    assert ei.value.status == hjcd.HJCD_EINVAL
    # a zero quaternion on the device marks that target unsolved
    q, err, cnt = ctx.solve(rid, -1, dev(bad), 8, 1, 1, 7)
    assert list(host(cnt).astype(int)) == [1, 0, 1]
    with pytest.raises(hjcd.HjcdError):
        ctx.solve(rid, -1, dev(tg), 8, 1, 1, 7, params=api.make_params(dup_ratio=0))
    # robot table validation
    bad_rob = inputs.panda()
    bad_rob.lo = bad_rob.hi.copy()
    with pytest.raises(hjcd.HjcdError):
        ctx.add_robot(bad_rob)


def test_long_chain_solves(ctx):
    rob = inputs.random_chain(np.random.default_rng(13), 24)
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    tg = f32(orc.pose(orob, f32(np.random.default_rng(14).uniform(rob.lo, rob.hi, (8, 24)))))
    q, err, cnt = ctx.solve(rid, -1, dev(tg), 256, 2, 3, 24)
    q, err, cnt = host(q), host(err), host(cnt).astype(int)
    succ = _verify(orob, None, rob, tg, q, err, cnt, 1e-3, 1e-2)
    assert succ.mean() >= 0.75


# ----------------------------------------------------------------------------
# the position-only CCD baseline (Alg. 1)

@pytest.mark.parametrize("which", ["panda", "chain12"])
def test_classic_ccd_matches_the_oracle(ctx, which):
    """cd_variant = 1: one sweep from identical inputs (per-joint steps and the
    resulting joint vector), then whole PO-CCD runs (break on the position
    error only) -- steps agree to the binary32 sensitivity of the sweep, most
    candidates to 1e-5."""
    rob = dict(robots())[which]
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(91)
    T, C = 11, 1500
    tg = _targets(orob, rng, T, rob.lo, rob.hi)
    tgt = rng.integers(0, T, C).astype(np.int32)
    cand = rng.integers(0, 4096, C).astype(np.int32)
    th = f32(rng.uniform(rob.lo, rob.hi, (C, rob.n)))
    gp = api.make_params(cd_variant=1)
    g = _ccd_gpu(ctx, rid, rob.n, tg, tgt, cand, th, 0, gp, 5)
    o = orc.ccd_iteration(orob, orc.make_params(seed=5, cd_variant=1), tg, tgt, cand, 0, th)
    tol = TOL * max(1.0, reach(rob) / 1.5)
    err = np.max(np.abs(g["theta"] - o["theta"]), axis=1)
    assert np.mean(err < tol) > 0.9, np.mean(err < tol)
    assert np.all(np.abs(g["dp"] - o["dp"])[err < tol] < tol)
    assert np.all(g["theta"] >= rob.lo - 1e-6) and np.all(g["theta"] <= rob.hi + 1e-6)
    # whole runs: the same seeds, break on |e_p|^2 < cd_eps_pos2 only
    S = 64
    t2 = np.repeat(np.arange(T), S).astype(np.int32)
    c2 = np.tile(np.arange(S), T).astype(np.int32)
    C2 = T * S
    th_o = torch.empty((rob.n, C2), device="cuda")
    perr = torch.empty((C2,), device="cuda")
    iters = torch.empty((C2,), dtype=torch.int32, device="cuda")
    hjcd.hjcd_po_ccd(ctx.h, rid, T, dev(tg), 1e-3, 1e-2, 5, gp, C2, dev(t2, torch.int32), dev(c2, torch.int32),
                     None, th_o, C2, 0, 32, None, perr, None, iters)
    o2 = orc.po_ccd(orob, orc.make_params(seed=5, cd_variant=1), tg, t2, c2)
    same = np.max(np.abs(host(th_o).T - o2["theta"]), axis=1) < 1e-3
    assert same.mean() > 0.8, same.mean()
    conv_g, conv_o = host(perr) ** 2 < 1e-4, o2["perr"] ** 2 < 1e-4
    assert abs(conv_g.mean() - conv_o.mean()) < 0.03


def test_classic_ccd_as_the_initialiser_of_the_whole_method(ctx):
    """Alg. 2 with the position-only CCD in place of PO-CCD: success within 3
    points of the oracle on 100 Panda targets x 128 seeds."""
    wl = inputs.cfg1()
    rob = wl.robot
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(92)
    tg = f32(orc.pose(orob, f32(rng.uniform(rob.lo, rob.hi, (100, 7)))))
    q, err, cnt = ctx.solve(rid, -1, dev(tg), 128, 1, 9, 7, params=api.make_params(cd_variant=1))
    q, err, cnt = host(q), host(err), host(cnt).astype(int)
    succ_g = _verify(orob, None, rob, tg, q, err, cnt, 1e-3, 1e-2)
    o = orc.solve(orob, None, orc.make_params(1e-3, 1e-2, seed=9, cd_variant=1), tg, 128, 1)
    succ_o = (o["count"] > 0) & (o["err"][:, 0, 0] <= 1e-3) & (o["err"][:, 0, 1] <= 1e-2)
    assert abs(succ_g.mean() - succ_o.mean()) <= 0.03 + 1e-12


def test_target_wide_break_solves_like_the_oracle(ctx):
    """cd_variant 2 (lock-step PO-CCD per target, all seeds stop at the first
    convergence) through the whole method: success within 3 points of the
    oracle on cfg2's robot and scene (80 targets x 256 seeds), every solution
    re-verified, and a target-wide iteration count no larger than the cap."""
    wl = inputs.cfg2(80, 256)
    rob, sc = wl.robot, wl.scene
    rid, sid = ctx.add_robot(rob), ctx.set_scene(sc)
    orob, osc = orc.Robot(rob), orc.Scene(sc)
    tg = _cfg2_targets(ctx, rid, sid, orob, osc, wl, 80)
    p2 = api.make_params(cd_variant=2)
    q, err, cnt = ctx.solve(rid, sid, dev(tg), 256, 2, wl.seed, 7, params=p2)
    q, err, cnt = host(q), host(err), host(cnt).astype(int)
    succ_g = _verify(orob, osc, rob, tg, q, err, cnt, wl.eps_pos, wl.eps_ori)
    o = orc.solve(orob, osc, orc.make_params(wl.eps_pos, wl.eps_ori, seed=wl.seed, cd_variant=2), tg, 256, 2)
    succ_o = (o["count"] > 0) & (o["err"][:, 0, 0] <= wl.eps_pos) & (o["err"][:, 0, 1] <= wl.eps_ori)
    assert abs(succ_g.mean() - succ_o.mean()) <= 0.03 + 1e-12
    assert succ_g.mean() > 0.8
    with pytest.raises(hjcd.HjcdError):  # per-candidate stage entry: not for whole targets
        C = 8
        th = torch.zeros((7, C), device="cuda")
        hjcd.hjcd_po_ccd(ctx.h, rid, 1, dev(tg[:1]), 1e-3, 1e-2, 1, p2, C, dev(np.zeros(C), torch.int32),
                         dev(np.arange(C), torch.int32), None, th, C, 0, 4)
