"""FP64 CPU oracle of batched HJCD-IK (arXiv 2510.07514).

TEST INFRASTRUCTURE ONLY.  The test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it; the product library never imports it.
The arithmetic lives in ``hjcd_oracle.c`` (plain C, double precision); this
module compiles it with gcc and marshals numpy arrays into it.

Joint vectors here are row-major ``(C, n)`` float64 arrays, poses ``(C, 7)``
as ``px py pz qw qx qy qz``.
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hjcd_oracle.c")
_HDR = os.path.join(_HERE, "hjcd_oracle.h")
_LIB_DIR = os.path.join(_HERE, "lib")
_LIB_PATH = os.path.join(_LIB_DIR, "libhjcd_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/lib/libhjcd_oracle.so`` (gcc, OpenMP).

    ``-ffp-contract=off`` keeps every multiply and add separately rounded, so
    the x86 and Arm builds give the same bits."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(ct.Structure):
    _fields_ = [
        ("eps_pos", ct.c_double), ("eps_ori", ct.c_double),
        ("cd_max_iters", ct.c_int32),
        ("cd_eps_pos2", ct.c_double), ("cd_eps_ori2", ct.c_double),
        ("cd_gamma_pos", ct.c_double), ("cd_gamma_ori", ct.c_double),
        ("cd_sigma", ct.c_double),
        ("cd_delta0", ct.c_double), ("cd_rho", ct.c_double),
        ("proj_eps", ct.c_double),
        ("dup_ratio", ct.c_int32),
        ("dup_sigma", ct.c_double),
        ("lm_max_iters", ct.c_int32),
        ("lm_lambda", ct.c_double), ("lm_trust_R", ct.c_double), ("lm_beta", ct.c_double),
        ("lm_A", ct.c_int32),
        ("lm_sigma", ct.c_double), ("lm_gn_reg", ct.c_double),
        ("cd_tie", ct.c_double),
        ("cd_variant", ct.c_int32),
        ("key", ct.c_uint32 * 2),
    ]


_P = ct.c_void_p
_D = ct.POINTER(ct.c_double)
_I32 = ct.POINTER(ct.c_int32)
_I64 = ct.POINTER(ct.c_int64)
_U8 = ct.POINTER(ct.c_uint8)
_U32 = ct.POINTER(ct.c_uint32)

_SIGS = {
    "orc_robot_new": (_P, [ct.c_int, _D, _D, _D, _D, _D, _D, _D, ct.c_int, _I32, _D, _U8]),
    "orc_robot_free": (None, [_P]),
    "orc_scene_new": (_P, [ct.c_int, _D, ct.c_int, _D]),
    "orc_scene_free": (None, [_P]),
    "orc_set_threads": (None, [ct.c_int]),
    "orc_get_threads": (ct.c_int, []),
    "orc_philox4x32_10": (None, [_U32, _U32, _U32]),
    "orc_u01": (ct.c_double, [ct.c_uint32]),
    "orc_normal": (ct.c_double, [ct.c_uint32, ct.c_uint32]),
    "orc_fk_frames": (None, [_P, _D, _D]),
    "orc_pose": (None, [_P, _D, _D]),
    "orc_quat_from_rot": (None, [_D, _D]),
    "orc_omega": (None, [_D, _D, _D]),
    "orc_residual": (None, [_P, _D, _D, _D]),
    "orc_jacobian": (None, [_P, _D, _D]),
    "orc_fk_batch": (None, [_P, ct.c_int64, _D, _D]),
    "orc_sample_seeds": (None, [_P, ct.POINTER(Params), ct.c_int64, _I32, _I32, _D]),
    "orc_ccd_iteration_batch": (None, [_P, ct.POINTER(Params), _D, ct.c_int64, _I32, _I32, ct.c_int,
                                       _D, _D, _D, _D, _D, _D, _D, _D, _I32, _I32, _U8, _D, _D, _D, _D, _U8]),
    "orc_po_ccd_batch": (None, [_P, ct.POINTER(Params), _D, ct.c_int64, _I32, _I32, _D, _D, _D, _D, _I32]),
    "orc_dup_layout": (ct.c_int64, [ct.c_int64, ct.c_int32, _I64, _I64]),
    "orc_topk_dup": (None, [_P, ct.POINTER(Params), ct.c_int64, _I64, _D, _D, _I64, _D, _I32]),
    "orc_lm_iteration_batch": (None, [_P, ct.POINTER(Params), _D, ct.c_int64, _I32, _I32, ct.c_int,
                                      _D, _D, _D, _D, _D, _I32, _D, _D, _U8, _D, _I32, _D]),
    "orc_lm_step": (None, [ct.c_int, _D, _D, ct.c_double, ct.c_double, _D]),
    "orc_dogleg_step": (None, [ct.c_int, _D, _D, ct.c_double, ct.c_double, _D]),
    "orc_single_coord_step": (None, [ct.c_int, _D, _D, ct.c_double, _I32, _D]),
    "orc_pjik_batch": (None, [_P, ct.POINTER(Params), _D, ct.c_int64, _I32, _I32, _D, _D, _D, _D, _I32]),
    "orc_collide_batch": (None, [_P, _P, ct.c_int64, _D, _U8, _D]),
    "orc_rank": (None, [_P, ct.c_int64, _I64, _D, _D, _D, _D, _U8, ct.c_double, ct.c_double, _D, ct.c_int,
                        _D, _D, _I32]),
    "orc_solve": (None, [_P, _P, ct.POINTER(Params), ct.c_int64, _D, _I64, _D, ct.c_int, _D, _D, _I32]),
}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ct.CDLL(_LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _d(a):
    return None if a is None else a.ctypes.data_as(_D)


def _i32(a):
    return None if a is None else a.ctypes.data_as(_I32)


def _i64(a):
    return None if a is None else a.ctypes.data_as(_I64)


def _u8(a):
    return None if a is None else a.ctypes.data_as(_U8)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def make_params(eps_pos=1e-3, eps_ori=1e-2, seed=0, **over) -> Params:
    """Parameter table from keyword values (missing keys raise)."""
    from paper_2510_07514_gb300.inputs import DEFAULT_PARAMS, seed_key
    vals = dict(DEFAULT_PARAMS)
    vals.update(over)
    p = Params()
    p.eps_pos, p.eps_ori = eps_pos, eps_ori
    for k, v in vals.items():
        setattr(p, k, v)
    lo, hi = seed_key(seed)
    p.key[0], p.key[1] = lo, hi
    return p


class Robot:
    """Oracle copy of a robot description (see ``inputs.Robot``)."""

    def __init__(self, r):
        L = lib()
        self.n = int(r.n)
        self._keep = [_f64(r.a), _f64(r.alpha), _f64(r.d), _f64(r.theta_off), _f64(r.flange, (16,)),
                      _f64(r.lo), _f64(r.hi)]
        nsph = int(len(r.sph_body))
        self.sph_body = np.ascontiguousarray(r.sph_body, np.int32)
        self.sph = _f64(r.sph_xyzr, (-1, 4)) if nsph else np.zeros((1, 4))
        ign = None if r.ignore is None else np.ascontiguousarray(r.ignore, np.uint8)
        self._ign = ign
        self.n_sph = nsph
        self.ptr = L.orc_robot_new(self.n, *[_d(x) for x in self._keep], nsph, _i32(self.sph_body),
                                   _d(self.sph), _u8(ign))
        if not self.ptr:
            raise ValueError("oracle rejected the robot description")
        self.lo = np.asarray(r.lo, float)
        self.hi = np.asarray(r.hi, float)

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.orc_robot_free(self.ptr)
            self.ptr = None


class Scene:
    def __init__(self, s):
        L = lib()
        self._s = _f64(s.sph_xyzr, (-1, 4)) if len(s.sph_xyzr) else np.zeros((1, 4))
        self._b = _f64(s.box_lohi, (-1, 6)) if len(s.box_lohi) else np.zeros((1, 6))
        self.ptr = L.orc_scene_new(len(s.sph_xyzr), _d(self._s), len(s.box_lohi), _d(self._b))

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.orc_scene_free(self.ptr)
            self.ptr = None


# ----------------------------------------------------------------------------
# thin wrappers

def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def threads() -> int:
    return lib().orc_get_threads()


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(c.ctypes.data_as(_U32), k.ctypes.data_as(_U32), out.ctypes.data_as(_U32))
    return out


def u01(x: int) -> float:
    return lib().orc_u01(int(x) & 0xFFFFFFFF)


def normal(x0: int, x1: int) -> float:
    return lib().orc_normal(int(x0) & 0xFFFFFFFF, int(x1) & 0xFFFFFFFF)


def fk_frames(rob: Robot, theta) -> np.ndarray:
    th = _f64(theta)
    out = np.zeros((rob.n + 2, 4, 4))
    lib().orc_fk_frames(rob.ptr, _d(th), _d(out))
    return out


def pose(rob: Robot, theta) -> np.ndarray:
    th = _f64(theta, (-1, rob.n))
    out = np.zeros((th.shape[0], 7))
    lib().orc_fk_batch(rob.ptr, th.shape[0], _d(th), _d(out))
    return out


def quat_from_rot(Rm) -> np.ndarray:
    m = _f64(Rm, (9,))
    q = np.zeros(4)
    lib().orc_quat_from_rot(_d(m), _d(q))
    return q


def omega(qt, qe) -> np.ndarray:
    a, b = _f64(qt, (4,)), _f64(qe, (4,))
    w = np.zeros(3)
    lib().orc_omega(_d(a), _d(b), _d(w))
    return w


def residual(rob: Robot, theta, target) -> np.ndarray:
    th, tg = _f64(theta, (rob.n,)), _f64(target, (7,))
    e = np.zeros(6)
    lib().orc_residual(rob.ptr, _d(th), _d(tg), _d(e))
    return e


def jacobian(rob: Robot, theta) -> np.ndarray:
    th = _f64(theta, (rob.n,))
    J = np.zeros((6, rob.n))
    lib().orc_jacobian(rob.ptr, _d(th), _d(J))
    return J


def _idx(tgt, cand):
    return np.ascontiguousarray(tgt, np.int32), np.ascontiguousarray(cand, np.int32)


def sample_seeds(rob: Robot, P: Params, tgt, cand) -> np.ndarray:
    t, c = _idx(tgt, cand)
    out = np.zeros((len(t), rob.n))
    lib().orc_sample_seeds(rob.ptr, ct.byref(P), len(t), _i32(t), _i32(c), _d(out))
    return out


def ccd_iteration(rob: Robot, P: Params, targets, tgt, cand, k: int, theta) -> dict:
    """One PO-CCD iteration per candidate, with its trace: per joint the position
    step dp and the position / orientation error it leaves (rp, op), the
    orientation step dq and the errors it leaves (pq, rq)."""
    t, c = _idx(tgt, cand)
    C, n = len(t), rob.n
    tg = _f64(targets, (-1, 7))
    th = _f64(theta, (C, n))
    o = dict(theta=np.zeros((C, n)), dp=np.zeros((C, n)), rp=np.zeros((C, n)), op=np.zeros((C, n)),
             dq=np.zeros((C, n)), pq=np.zeros((C, n)), rq=np.zeros((C, n)),
             jp=np.zeros(C, np.int32), jo=np.zeros(C, np.int32),
             accepted=np.zeros(C, np.uint8), theta_hat=np.zeros((C, n)), margin_p=np.zeros(C),
             margin_o=np.zeros(C), margin_acc=np.zeros(C), converged=np.zeros(C, np.uint8))
    lib().orc_ccd_iteration_batch(rob.ptr, ct.byref(P), _d(tg), C, _i32(t), _i32(c), int(k), _d(th),
                                  _d(o["theta"]), _d(o["dp"]), _d(o["rp"]), _d(o["op"]), _d(o["dq"]), _d(o["pq"]),
                                  _d(o["rq"]),
                                  _i32(o["jp"]), _i32(o["jo"]), _u8(o["accepted"]), _d(o["theta_hat"]),
                                  _d(o["margin_p"]), _d(o["margin_o"]), _d(o["margin_acc"]),
                                  _u8(o["converged"]))
    return o


def po_ccd(rob: Robot, P: Params, targets, tgt, cand) -> dict:
    t, c = _idx(tgt, cand)
    C, n = len(t), rob.n
    tg = _f64(targets, (-1, 7))
    o = dict(theta=np.zeros((C, n)), score=np.zeros(C), perr=np.zeros(C), oerr=np.zeros(C),
             iters=np.zeros(C, np.int32))
    lib().orc_po_ccd_batch(rob.ptr, ct.byref(P), _d(tg), C, _i32(t), _i32(c), _d(o["theta"]),
                           _d(o["score"]), _d(o["perr"]), _d(o["oerr"]), _i32(o["iters"]))
    return o


def dup_layout(M: int, ratio: int) -> tuple[int, int, int]:
    K = ct.c_int64()
    cp = ct.c_int64()
    B = lib().orc_dup_layout(int(M), int(ratio), ct.byref(K), ct.byref(cp))
    return int(K.value), int(cp.value), int(B)


def topk_dup(rob: Robot, P: Params, m_off, score_M, theta_M) -> dict:
    m_off = np.ascontiguousarray(m_off, np.int64)
    T = len(m_off) - 1
    b_off = np.zeros(T + 1, np.int64)
    for t in range(T):
        b_off[t + 1] = b_off[t] + dup_layout(m_off[t + 1] - m_off[t], P.dup_ratio)[2]
    s = _f64(score_M)
    th = _f64(theta_M, (-1, rob.n))
    out = np.zeros((int(b_off[-1]), rob.n))
    src = np.zeros(int(b_off[-1]), np.int32)
    lib().orc_topk_dup(rob.ptr, ct.byref(P), T, _i64(m_off), _d(s), _d(th), _i64(b_off), _d(out), _i32(src))
    return dict(theta=out, src=src, b_off=b_off)


def lm_iteration(rob: Robot, P: Params, targets, tgt, cand, k: int, theta) -> dict:
    """One PJ-IK iteration per candidate, with its trace: J, W, the clamped LM
    step d_lm, the dogleg step d_dog, the single-coordinate joint sc_joint and
    step sc_step (all three computed whether or not the LM step succeeds), the
    branch taken (0 LM, 1 dogleg, 2 single coordinate, 3 perturbation), the
    accepted line-search alpha and the smallest relative cost gap of the trials
    evaluated (ls_margin)."""
    t, c = _idx(tgt, cand)
    C, n = len(t), rob.n
    tg = _f64(targets, (-1, 7))
    th = _f64(theta, (C, n))
    o = dict(theta=np.zeros((C, n)), J=np.zeros((C, 6, n)), W=np.zeros((C, 6)), d_lm=np.zeros((C, n)),
             branch=np.zeros(C, np.int32), alpha=np.zeros(C), ls_margin=np.zeros(C),
             converged=np.zeros(C, np.uint8), d_dog=np.zeros((C, n)), sc_joint=np.zeros(C, np.int32),
             sc_step=np.zeros(C))
    lib().orc_lm_iteration_batch(rob.ptr, ct.byref(P), _d(tg), C, _i32(t), _i32(c), int(k), _d(th),
                                 _d(o["theta"]), _d(o["J"]), _d(o["W"]), _d(o["d_lm"]), _i32(o["branch"]),
                                 _d(o["alpha"]), _d(o["ls_margin"]), _u8(o["converged"]), _d(o["d_dog"]),
                                 _i32(o["sc_joint"]), _d(o["sc_step"]))
    return o


def lm_step(Jw, b, lam: float, R: float) -> np.ndarray:
    """Damped normal-equation step of Eq. normal-eqs, clamped to +-R."""
    Jw = _f64(Jw)
    n = Jw.shape[1]
    out = np.zeros(n)
    lib().orc_lm_step(n, _d(Jw), _d(_f64(b, (6,))), float(lam), float(R), _d(out))
    return out


def dogleg_step(Jw, b, R: float, gn_reg: float) -> np.ndarray:
    """Dogleg step of Eq. dogleg."""
    Jw = _f64(Jw)
    n = Jw.shape[1]
    out = np.zeros(n)
    lib().orc_dogleg_step(n, _d(Jw), _d(_f64(b, (6,))), float(R), float(gn_reg), _d(out))
    return out


def single_coord_step(Jw, b, R: float) -> tuple[int, np.ndarray]:
    """Joint i* and step of Eq. single-coord, clamped to +-R."""
    Jw = _f64(Jw)
    n = Jw.shape[1]
    out = np.zeros(n)
    i = ct.c_int32()
    lib().orc_single_coord_step(n, _d(Jw), _d(_f64(b, (6,))), float(R), ct.byref(i), _d(out))
    return int(i.value), out


def pjik(rob: Robot, P: Params, targets, tgt, cand, theta) -> dict:
    t, c = _idx(tgt, cand)
    C, n = len(t), rob.n
    tg = _f64(targets, (-1, 7))
    th = np.array(_f64(theta, (C, n)), copy=True)
    o = dict(score=np.zeros(C), perr=np.zeros(C), oerr=np.zeros(C), iters=np.zeros(C, np.int32))
    lib().orc_pjik_batch(rob.ptr, ct.byref(P), _d(tg), C, _i32(t), _i32(c), _d(th), _d(o["score"]),
                         _d(o["perr"]), _d(o["oerr"]), _i32(o["iters"]))
    o["theta"] = th
    return o


def collide(rob: Robot, scene: Scene | None, theta) -> tuple[np.ndarray, np.ndarray]:
    th = _f64(theta, (-1, rob.n))
    C = th.shape[0]
    hit = np.zeros(C, np.uint8)
    margin = np.zeros(C)
    lib().orc_collide_batch(rob.ptr, scene.ptr if scene is not None else None, C, _d(th), _u8(hit), _d(margin))
    return hit.astype(bool), margin


def rank(rob: Robot, b_off, theta_B, score, perr, oerr, hit, top_k: int, eps_pos: float, eps_ori: float,
         q_ref=None) -> dict:
    """Final ranking of Alg. 2: per target the collision-free candidates, those
    within (eps_pos, eps_ori) first, each group by score -- or, with q_ref
    ([T][n]), the group within the tolerances by joint distance to q_ref[t]."""
    b_off = np.ascontiguousarray(b_off, np.int64)
    T = len(b_off) - 1
    n = rob.n
    th = _f64(theta_B, (-1, n))
    h = None if hit is None else np.ascontiguousarray(hit, np.uint8)
    qr = None if q_ref is None else _f64(q_ref, (T, n))
    o = dict(q=np.zeros((T, top_k, n)), err=np.zeros((T, top_k, 2)), count=np.zeros(T, np.int32))
    lib().orc_rank(rob.ptr, T, _i64(b_off), _d(th), _d(_f64(score)), _d(_f64(perr)), _d(_f64(oerr)),
                   _u8(h), float(eps_pos), float(eps_ori), _d(qr), int(top_k), _d(o["q"]), _d(o["err"]),
                   _i32(o["count"]))
    return o


def solve(rob: Robot, scene: Scene | None, P: Params, targets, samples, top_k: int, q_ref=None) -> dict:
    """The whole method (Alg. 2); q_ref ([T][n]) ranks as the tracking loop does."""
    tg = _f64(targets, (-1, 7))
    T = tg.shape[0]
    s = np.ascontiguousarray(np.broadcast_to(np.asarray(samples, np.int64), (T,)), np.int64)
    n = rob.n
    qr = None if q_ref is None else _f64(q_ref, (T, n))
    o = dict(q=np.zeros((T, top_k, n)), err=np.zeros((T, top_k, 2)), count=np.zeros(T, np.int32))
    lib().orc_solve(rob.ptr, scene.ptr if scene is not None else None, ct.byref(P), T, _d(tg), _i64(s),
                    _d(qr), int(top_k), _d(o["q"]), _d(o["err"]), _i32(o["count"]))
    return o
