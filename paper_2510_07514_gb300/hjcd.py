"""Python binding of the HJCD-IK C ABI (``include/hjcd.h``).

Argument marshalling only: every function here has the name of the C entry
point it calls, converts Python arguments (torch tensors, numpy arrays, ints)
into pointers and sizes, and raises :class:`HjcdError` when the call returns a
non-zero status.  All computation happens in ``lib/libhjcd.so``; there is no
fallback when it is missing -- loading raises instead.
"""
from __future__ import annotations

import ctypes as ct
import os
import threading

from . import build as _build

HJCD_OK = 0
HJCD_EINVAL = -1
HJCD_ENOMEM = -2
HJCD_ECUDA = -3
HJCD_ETIMEOUT = -4
HJCD_ENOTFOUND = -5
HJCD_MAX_DOF = 24
HJCD_MAX_SPHERES = 256
HJCD_MAX_SAMPLES = 8192
HJCD_MAX_TOPK = 64
HJCD_MAX_BATCH_ROBOTS = 16

# Every function the header declares (checked by the test-suite against include/hjcd.h).
EXPORTS = (
    "hjcd_init", "hjcd_destroy", "hjcd_last_error", "hjcd_status_string", "hjcd_default_params",
    "hjcd_create_robot", "hjcd_set_scene", "hjcd_solve", "hjcd_fk", "hjcd_sample_seeds",
    "hjcd_po_ccd", "hjcd_topk_dup", "hjcd_pjik", "hjcd_collide", "hjcd_rank",
    "hjcd_set_profiling", "hjcd_phase_times", "hjcd_counters", "hjcd_launch_count", "hjcd_ffma_probe",
    "hjcd_solve_noalloc", "hjcd_solve_batch", "hjcd_solve_nearest",
    "hjcd_server_start", "hjcd_server_stop", "hjcd_submit", "hjcd_poll", "hjcd_wait",
    "hjcd_graph_create", "hjcd_graph_launch", "hjcd_graph_check", "hjcd_graph_destroy",
    "hjcd_set_launch_config", "hjcd_autotune", "hjcd_set_memory_budget", "hjcd_scene_contacts",
    "hjcd_shard_topk", "hjcd_topk_merge", "hjcd_solve_from_topk", "hjcd_set_collision_mode",
    "hjcd_philox", "hjcd_set_wait_limit",
)


class HjcdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"hjcd status {status}: {message}")
        self.status = status


class hjcd_params(ct.Structure):
    _fields_ = [
        ("cd_max_iters", ct.c_int32), ("cd_eps_pos2", ct.c_float), ("cd_eps_ori2", ct.c_float),
        ("cd_gamma_pos", ct.c_float), ("cd_gamma_ori", ct.c_float), ("cd_sigma", ct.c_float),
        ("cd_delta0", ct.c_float), ("cd_rho", ct.c_float), ("proj_eps", ct.c_float),
        ("dup_ratio", ct.c_int32), ("dup_sigma", ct.c_float),
        ("lm_max_iters", ct.c_int32), ("lm_lambda", ct.c_float), ("lm_trust_R", ct.c_float),
        ("lm_beta", ct.c_float), ("lm_A", ct.c_int32), ("lm_sigma", ct.c_float), ("lm_gn_reg", ct.c_float),
        ("cd_tie", ct.c_float), ("cd_variant", ct.c_int32),
    ]


class hjcd_solve_opts(ct.Structure):
    _fields_ = [
        ("eps_pos", ct.c_float), ("eps_ori", ct.c_float), ("n_samples", ct.c_int32), ("top_k", ct.c_int32),
        ("seed", ct.c_uint64), ("params", ct.POINTER(hjcd_params)), ("samples_per_target", ct.c_void_p),
    ]


class hjcd_batch_item(ct.Structure):
    _fields_ = [
        ("robot_id", ct.c_int32), ("scene_id", ct.c_int32), ("n_inline_spheres", ct.c_int32),
        ("n_inline_boxes", ct.c_int32), ("inline_spheres", ct.c_void_p), ("inline_boxes", ct.c_void_p),
        ("n_targets", ct.c_int32), ("pad_", ct.c_int32), ("targets_pq", ct.c_void_p), ("opts", hjcd_solve_opts),
        ("out_q", ct.c_void_p), ("out_err", ct.c_void_p), ("out_count", ct.c_void_p), ("q_current", ct.c_void_p),
    ]


class hjcd_server_opts(ct.Structure):
    _fields_ = [
        ("max_inflight", ct.c_int32), ("max_batch_requests", ct.c_int32), ("max_batch_seeds", ct.c_int64),
        ("memory_budget", ct.c_uint64), ("params", ct.POINTER(hjcd_params)),
    ]


class hjcd_request_info(ct.Structure):
    _fields_ = [("status", ct.c_int32), ("batch_requests", ct.c_int32), ("queued_ms", ct.c_double),
                ("total_ms", ct.c_double)]


class hjcd_tune_report(ct.Structure):
    _fields_ = [("ccd_block", ct.c_int32), ("lm_warps", ct.c_int32), ("cd_max_iters", ct.c_int32),
                ("lm_max_iters", ct.c_int32), ("success_rate", ct.c_float), ("best_success_rate", ct.c_float),
                ("ms", ct.c_double), ("trials", ct.c_int32)]


class hjcd_ccd_trace(ct.Structure):
    _fields_ = [(k, ct.c_void_p) for k in ("dp", "rp", "dq", "rq", "jp", "jo", "accepted", "th_hat",
                                                   "op", "pq")]


class hjcd_lm_trace(ct.Structure):
    _fields_ = [(k, ct.c_void_p) for k in ("J", "W", "d_lm", "branch", "alpha", "d_dog", "sc_joint", "sc_step")]


_V = ct.c_void_p
_I = ct.c_int
_I32 = ct.c_int32
_I64 = ct.c_int64
_U64 = ct.c_uint64
_F = ct.c_float
_ST = ct.c_int32

_SIGS = {
    "hjcd_init": (_ST, [_I, ct.POINTER(_V)]),
    "hjcd_destroy": (None, [_V]),
    "hjcd_last_error": (ct.c_char_p, [_V]),
    "hjcd_status_string": (ct.c_char_p, [_ST]),
    "hjcd_default_params": (None, [ct.POINTER(hjcd_params)]),
    "hjcd_create_robot": (_ST, [_V, _I, _V, _V, _V, _V, _V, _V, _V, _I, _V, _V, _V, ct.POINTER(_I32)]),
    "hjcd_set_scene": (_ST, [_V, _I32, _I, _V, _I, _V, ct.POINTER(_I32)]),
    "hjcd_solve": (_ST, [_V, _I32, _I32, _I, _V, ct.POINTER(hjcd_solve_opts), _V, _V, _V, _V]),
    "hjcd_solve_noalloc": (_ST, [_V, _I32, _I32, _I, _V, ct.POINTER(hjcd_solve_opts), _V, _V, _V, _V]),
    "hjcd_solve_batch": (_ST, [_V, _I, ct.POINTER(hjcd_batch_item), ct.POINTER(hjcd_params), _V]),
    "hjcd_solve_nearest": (_ST, [_V, _I32, _I32, _I, _V, _V, ct.POINTER(hjcd_solve_opts), _V, _V, _V, _V]),
    "hjcd_server_start": (_ST, [_V, ct.POINTER(hjcd_server_opts)]),
    "hjcd_set_launch_config": (_ST, [_V, _I32, _I32]),
    "hjcd_set_memory_budget": (_ST, [_V, _U64]),
    "hjcd_set_collision_mode": (_ST, [_V, _I32]),
    "hjcd_scene_contacts": (_ST, [_V, _I32, _I32, _I64, _V, _I64, _V, _V]),
    "hjcd_shard_topk": (_ST, [_V, _I32, _I, _V, ct.POINTER(hjcd_solve_opts), _I32, _I32, _V, _V, _V, _V]),
    "hjcd_topk_merge": (_ST, [_V, _I, _I, _I, _I, _V, _V, _V, _V, _V, _V, _V]),
    "hjcd_solve_from_topk": (_ST, [_V, _I32, _I32, _I, _V, _I32, ct.POINTER(hjcd_solve_opts), _V, _V, _V, _V, _V]),
    "hjcd_autotune": (_ST, [_V, _I, ct.POINTER(hjcd_batch_item), ct.POINTER(hjcd_params), _F, _I32,
                            ct.POINTER(hjcd_params), ct.POINTER(hjcd_tune_report)]),
    "hjcd_graph_create": (_ST, [_V, _I, ct.POINTER(hjcd_batch_item), ct.POINTER(hjcd_params), ct.POINTER(_V)]),
    "hjcd_graph_launch": (_ST, [_V, _V]),
    "hjcd_graph_check": (_ST, [_V]),
    "hjcd_graph_destroy": (None, [_V]),
    "hjcd_server_stop": (_ST, [_V]),
    "hjcd_submit": (_ST, [_V, ct.POINTER(hjcd_batch_item), ct.POINTER(_I64)]),
    "hjcd_poll": (_ST, [_V, _I64, ct.POINTER(_I32), ct.POINTER(hjcd_request_info)]),
    "hjcd_wait": (_ST, [_V, _I64, ct.c_double, ct.POINTER(hjcd_request_info)]),
    "hjcd_fk": (_ST, [_V, _I32, _I64, _V, _I64, _V, _V]),
    "hjcd_sample_seeds": (_ST, [_V, _I32, _I64, _V, _V, _U64, _V, _I64, _V]),
    "hjcd_po_ccd": (_ST, [_V, _I32, _I, _V, _F, _F, _U64, ct.POINTER(hjcd_params), _I64, _V, _V, _V, _V, _I64,
                          _I, _I, _V, _V, _V, _V, ct.POINTER(hjcd_ccd_trace), _V]),
    "hjcd_topk_dup": (_ST, [_V, _I32, _I, _V, _V, _V, _I64, _V, _V, _I64, _V, _U64, ct.POINTER(hjcd_params), _V]),
    "hjcd_pjik": (_ST, [_V, _I32, _I, _V, _F, _F, _U64, ct.POINTER(hjcd_params), _I64, _V, _V, _V, _I64, _I, _I,
                        _V, _V, _V, _V, ct.POINTER(hjcd_lm_trace), _V]),
    "hjcd_collide": (_ST, [_V, _I32, _I32, _I64, _V, _I64, _V, _V]),
    "hjcd_rank": (_ST, [_V, _I32, _I, _V, _V, _I64, _V, _V, _V, _V, _F, _F, _V, _I, _V, _V, _V, _V]),
    "hjcd_philox": (_ST, [_V, _I64, _V, _U64, _V, _V]),
    "hjcd_set_wait_limit": (_ST, [_V, _I64]),
    "hjcd_set_profiling": (_ST, [_V, _I]),
    "hjcd_phase_times": (_ST, [_V, ct.POINTER(_F)]),
    "hjcd_counters": (_ST, [_V, ct.POINTER(_U64), _I]),
    "hjcd_launch_count": (_I64, [_V]),
    "hjcd_ffma_probe": (_ST, [_V, _I, ct.POINTER(ct.c_double), _V]),
}

_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _build.LIB_PATH


def load() -> ct.CDLL:
    """Load libhjcd.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB_PATH):
                raise ImportError(f"{_build.LIB_PATH} is missing: build it with "
                                  "`python -m paper_2510_07514_gb300.build` (needs nvcc)")
            L = ct.CDLL(_build.LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def ptr(x):
    """Pointer of a torch tensor, numpy array, int address or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr() if x.numel() else None
    if hasattr(x, "ctypes"):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)!r}")


def stream_handle(stream) -> int | None:
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(ctx, status: int) -> None:
    if status != HJCD_OK:
        L = load()
        msg = L.hjcd_last_error(ctx).decode() if ctx else L.hjcd_status_string(status).decode()
        raise HjcdError(status, msg)


# ----------------------------------------------------------------------------

def hjcd_init(device: int = 0) -> int:
    h = _V()
    _check(None, load().hjcd_init(int(device), ct.byref(h)))
    return h.value


def hjcd_destroy(ctx) -> None:
    load().hjcd_destroy(ctx)


def hjcd_last_error(ctx) -> str:
    return load().hjcd_last_error(ctx).decode()


def hjcd_status_string(status: int) -> str:
    return load().hjcd_status_string(int(status)).decode()


def hjcd_default_params() -> hjcd_params:
    p = hjcd_params()
    load().hjcd_default_params(ct.byref(p))
    return p


def hjcd_create_robot(ctx, n_dof, dh_a, dh_alpha, dh_d, dh_theta_off, flange, q_lo, q_hi,
                      n_spheres, sph_link, sph_xyzr, ignore_pairs) -> int:
    rid = _I32()
    _check(ctx, load().hjcd_create_robot(ctx, int(n_dof), ptr(dh_a), ptr(dh_alpha), ptr(dh_d), ptr(dh_theta_off),
                                         ptr(flange), ptr(q_lo), ptr(q_hi), int(n_spheres), ptr(sph_link),
                                         ptr(sph_xyzr), ptr(ignore_pairs), ct.byref(rid)))
    return rid.value


def hjcd_set_scene(ctx, scene_id_or_new, n_sph, sph_xyzr, n_box, box_lohi) -> int:
    sid = _I32()
    _check(ctx, load().hjcd_set_scene(ctx, int(scene_id_or_new), int(n_sph), ptr(sph_xyzr), int(n_box),
                                      ptr(box_lohi), ct.byref(sid)))
    return sid.value


def hjcd_solve(ctx, robot_id, scene_id, n_targets, targets_pq, opts: hjcd_solve_opts, out_q, out_err, out_count,
               stream=None) -> None:
    _check(ctx, load().hjcd_solve(ctx, int(robot_id), int(scene_id), int(n_targets), ptr(targets_pq),
                                  ct.byref(opts), ptr(out_q), ptr(out_err), ptr(out_count), stream_handle(stream)))


def hjcd_solve_noalloc(ctx, robot_id, scene_id, n_targets, targets_pq, opts: hjcd_solve_opts, out_q, out_err,
                       out_count, stream=None) -> None:
    """hjcd_solve without allocation (device buffers; scratch in a static device array)."""
    _check(ctx, load().hjcd_solve_noalloc(ctx, int(robot_id), int(scene_id), int(n_targets), ptr(targets_pq),
                                          ct.byref(opts), ptr(out_q), ptr(out_err), ptr(out_count),
                                          stream_handle(stream)))


def hjcd_solve_nearest(ctx, robot_id, scene_id, n_targets, targets_pq, q_current, opts: hjcd_solve_opts, out_q,
                       out_err, out_count, stream=None) -> None:
    _check(ctx, load().hjcd_solve_nearest(ctx, int(robot_id), int(scene_id), int(n_targets), ptr(targets_pq),
                                          ptr(q_current), ct.byref(opts), ptr(out_q), ptr(out_err), ptr(out_count),
                                          stream_handle(stream)))


def hjcd_solve_batch(ctx, items, params=None, stream=None) -> None:
    """Solve several requests (a sequence of hjcd_batch_item) in one launch per phase."""
    arr = (hjcd_batch_item * len(items))(*items)
    _check(ctx, load().hjcd_solve_batch(ctx, len(items), arr, ct.byref(params) if params is not None else None,
                                        stream_handle(stream)))


def hjcd_scene_contacts(ctx, robot_id, scene_id, n_cand, theta, ld, touched, stream=None) -> None:
    _check(ctx, load().hjcd_scene_contacts(ctx, int(robot_id), int(scene_id), int(n_cand), ptr(theta), int(ld),
                                           ptr(touched), stream_handle(stream)))


def hjcd_shard_topk(ctx, robot_id, n_targets, targets_pq, opts, seed_begin, seed_end, out_score, out_index,
                    out_theta, stream=None) -> None:
    _check(ctx, load().hjcd_shard_topk(ctx, int(robot_id), int(n_targets), ptr(targets_pq), ct.byref(opts),
                                       int(seed_begin), int(seed_end), ptr(out_score), ptr(out_index), ptr(out_theta),
                                       stream_handle(stream)))


def hjcd_topk_merge(ctx, n_targets, n_lists, K, n, in_score, in_index, in_theta, out_score, out_index, out_theta,
                    stream=None) -> None:
    _check(ctx, load().hjcd_topk_merge(ctx, int(n_targets), int(n_lists), int(K), int(n), ptr(in_score),
                                       ptr(in_index), ptr(in_theta), ptr(out_score), ptr(out_index), ptr(out_theta),
                                       stream_handle(stream)))


def hjcd_solve_from_topk(ctx, robot_id, scene_id, n_targets, targets_pq, first_target, opts, kept_theta, out_q,
                         out_err, out_count, stream=None) -> None:
    _check(ctx, load().hjcd_solve_from_topk(ctx, int(robot_id), int(scene_id), int(n_targets), ptr(targets_pq),
                                            int(first_target), ct.byref(opts), ptr(kept_theta), ptr(out_q),
                                            ptr(out_err), ptr(out_count), stream_handle(stream)))


def hjcd_set_collision_mode(ctx, mode: int) -> None:
    """1: collision-check candidates in rank order until top_k are found (default); 0: check all."""
    _check(ctx, load().hjcd_set_collision_mode(ctx, int(mode)))


def hjcd_set_memory_budget(ctx, nbytes: int) -> None:
    _check(ctx, load().hjcd_set_memory_budget(ctx, int(nbytes)))


def hjcd_set_launch_config(ctx, ccd_block: int, lm_warps: int) -> None:
    _check(ctx, load().hjcd_set_launch_config(ctx, int(ccd_block), int(lm_warps)))


def hjcd_autotune(ctx, items, base=None, success_tol: float = 0.01, repeats: int = 3):
    """(tuned hjcd_params, hjcd_tune_report) for a calibration batch."""
    arr = (hjcd_batch_item * len(items))(*items)
    tuned, rep = hjcd_params(), hjcd_tune_report()
    _check(ctx, load().hjcd_autotune(ctx, len(items), arr, ct.byref(base) if base is not None else None,
                                     float(success_tol), int(repeats), ct.byref(tuned), ct.byref(rep)))
    return tuned, rep


def hjcd_graph_create(ctx, items, params=None) -> int:
    """Capture a batch (device targets and outputs) as a replayable graph; returns its handle."""
    arr = (hjcd_batch_item * len(items))(*items)
    g = _V()
    _check(ctx, load().hjcd_graph_create(ctx, len(items), arr, ct.byref(params) if params is not None else None,
                                         ct.byref(g)))
    return g.value


def hjcd_graph_launch(ctx, graph, stream=None) -> None:
    _check(ctx, load().hjcd_graph_launch(graph, stream_handle(stream)))


def hjcd_graph_check(ctx, graph) -> None:
    _check(ctx, load().hjcd_graph_check(graph))


def hjcd_graph_destroy(graph) -> None:
    load().hjcd_graph_destroy(graph)


def hjcd_server_start(ctx, max_inflight=0, max_batch_requests=0, max_batch_seeds=0, memory_budget=0,
                      params=None) -> None:
    o = hjcd_server_opts(int(max_inflight), int(max_batch_requests), int(max_batch_seeds), int(memory_budget),
                         ct.pointer(params) if params is not None else None)
    _check(ctx, load().hjcd_server_start(ctx, ct.byref(o)))


def hjcd_server_stop(ctx) -> None:
    _check(ctx, load().hjcd_server_stop(ctx))


def hjcd_submit(ctx, item: hjcd_batch_item) -> int:
    rid = _I64()
    _check(ctx, load().hjcd_submit(ctx, ct.byref(item), ct.byref(rid)))
    return rid.value


def hjcd_poll(ctx, request_id) -> hjcd_request_info | None:
    """The request's info once it is done, else None."""
    done = _I32()
    info = hjcd_request_info()
    _check(ctx, load().hjcd_poll(ctx, int(request_id), ct.byref(done), ct.byref(info)))
    return info if done.value else None


def hjcd_wait(ctx, request_id, timeout_s: float = 60.0) -> hjcd_request_info:
    info = hjcd_request_info()
    _check(ctx, load().hjcd_wait(ctx, int(request_id), float(timeout_s), ct.byref(info)))
    return info


def hjcd_fk(ctx, robot_id, n_cand, theta, ld, out_pq, stream=None) -> None:
    _check(ctx, load().hjcd_fk(ctx, int(robot_id), int(n_cand), ptr(theta), int(ld), ptr(out_pq),
                               stream_handle(stream)))


def hjcd_sample_seeds(ctx, robot_id, n_cand, tgt, cand, seed, theta, ld, stream=None) -> None:
    _check(ctx, load().hjcd_sample_seeds(ctx, int(robot_id), int(n_cand), ptr(tgt), ptr(cand),
                                         int(seed) & (2 ** 64 - 1), ptr(theta), int(ld), stream_handle(stream)))


def hjcd_po_ccd(ctx, robot_id, n_targets, targets_pq, eps_pos, eps_ori, seed, params, n_cand, tgt, cand,
                theta_in, theta_out, ld, k0, n_iters, score=None, perr=None, oerr=None, iters=None,
                trace: hjcd_ccd_trace | None = None, stream=None) -> None:
    _check(ctx, load().hjcd_po_ccd(ctx, int(robot_id), int(n_targets), ptr(targets_pq), float(eps_pos),
                                   float(eps_ori), int(seed) & (2 ** 64 - 1),
                                   ct.byref(params) if params is not None else None, int(n_cand), ptr(tgt),
                                   ptr(cand), ptr(theta_in), ptr(theta_out), int(ld), int(k0), int(n_iters),
                                   ptr(score), ptr(perr), ptr(oerr), ptr(iters),
                                   ct.byref(trace) if trace is not None else None, stream_handle(stream)))


def hjcd_topk_dup(ctx, robot_id, n_targets, m_off, score_M, theta_M, ld_M, b_off, theta_B, ld_B, src_B, seed,
                  params, stream=None) -> None:
    _check(ctx, load().hjcd_topk_dup(ctx, int(robot_id), int(n_targets), ptr(m_off), ptr(score_M), ptr(theta_M),
                                     int(ld_M), ptr(b_off), ptr(theta_B), int(ld_B), ptr(src_B),
                                     int(seed) & (2 ** 64 - 1), ct.byref(params) if params is not None else None,
                                     stream_handle(stream)))


def hjcd_pjik(ctx, robot_id, n_targets, targets_pq, eps_pos, eps_ori, seed, params, n_cand, tgt, cand, theta, ld,
              k0, n_iters, score=None, perr=None, oerr=None, iters=None, trace: hjcd_lm_trace | None = None,
              stream=None) -> None:
    _check(ctx, load().hjcd_pjik(ctx, int(robot_id), int(n_targets), ptr(targets_pq), float(eps_pos),
                                 float(eps_ori), int(seed) & (2 ** 64 - 1),
                                 ct.byref(params) if params is not None else None, int(n_cand), ptr(tgt),
                                 ptr(cand), ptr(theta), int(ld), int(k0), int(n_iters), ptr(score), ptr(perr),
                                 ptr(oerr), ptr(iters), ct.byref(trace) if trace is not None else None,
                                 stream_handle(stream)))


def hjcd_collide(ctx, robot_id, scene_id, n_cand, theta, ld, hit, stream=None) -> None:
    _check(ctx, load().hjcd_collide(ctx, int(robot_id), int(scene_id), int(n_cand), ptr(theta), int(ld), ptr(hit),
                                    stream_handle(stream)))


def hjcd_rank(ctx, robot_id, n_targets, b_off, theta_B, ld, score, perr, oerr, hit, eps_pos, eps_ori, q_ref,
              top_k, out_q, out_err, out_count, stream=None) -> None:
    _check(ctx, load().hjcd_rank(ctx, int(robot_id), int(n_targets), ptr(b_off), ptr(theta_B), int(ld), ptr(score),
                                 ptr(perr), ptr(oerr), ptr(hit), float(eps_pos), float(eps_ori), ptr(q_ref),
                                 int(top_k), ptr(out_q), ptr(out_err), ptr(out_count), stream_handle(stream)))


def hjcd_philox(ctx, n_blocks, ctr, key, out, stream=None) -> None:
    _check(ctx, load().hjcd_philox(ctx, int(n_blocks), ptr(ctr), int(key) & (2 ** 64 - 1), ptr(out),
                                   stream_handle(stream)))


def hjcd_set_wait_limit(ctx, polls: int) -> None:
    _check(ctx, load().hjcd_set_wait_limit(ctx, int(polls)))


def hjcd_set_profiling(ctx, on: bool) -> None:
    _check(ctx, load().hjcd_set_profiling(ctx, 1 if on else 0))


def hjcd_phase_times(ctx) -> list[float]:
    ms = (_F * 6)()
    _check(ctx, load().hjcd_phase_times(ctx, ms))
    return list(ms)


def hjcd_counters(ctx, reset: bool = False) -> list[int]:
    out = (_U64 * 8)()
    _check(ctx, load().hjcd_counters(ctx, out, 1 if reset else 0))
    return list(out)


def hjcd_launch_count(ctx) -> int:
    return int(load().hjcd_launch_count(ctx))


def hjcd_ffma_probe(ctx, iters: int = 4096, stream=None) -> float:
    tf = ct.c_double()
    _check(ctx, load().hjcd_ffma_probe(ctx, int(iters), ct.byref(tf), stream_handle(stream)))
    return tf.value
