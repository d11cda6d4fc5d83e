"""Convenience layer over the C ABI for Python callers.

Allocation (torch tensors) and argument marshalling only; every step of the
method runs in the CUDA library through :mod:`hjcd`.
"""
from __future__ import annotations

import numpy as np
import torch

from . import hjcd
from .inputs import DEFAULT_PARAMS, Robot, Scene


def make_params(**over) -> hjcd.hjcd_params:
    """hjcd_params from the workload parameter table, with overrides."""
    vals = dict(DEFAULT_PARAMS)
    vals.update(over)
    p = hjcd.hjcd_params()
    for k, v in vals.items():
        setattr(p, k, v)
    return p


def _f32(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    return a if shape is None else a.reshape(shape)


class Context:
    """An hjcd context on one CUDA device."""

    def __init__(self, device: int = 0):
        self.device = int(device)
        self.h = hjcd.hjcd_init(self.device)
        self._keep = []

    def close(self) -> None:
        if self.h:
            hjcd.hjcd_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def add_robot(self, r: Robot) -> int:
        n = int(r.n)
        ns = int(len(r.sph_body))
        ign = None if r.ignore is None else np.ascontiguousarray(r.ignore, np.uint8)
        return hjcd.hjcd_create_robot(
            self.h, n, _f32(r.a), _f32(r.alpha), _f32(r.d), _f32(r.theta_off), _f32(r.flange, (16,)),
            _f32(r.lo), _f32(r.hi), ns, np.ascontiguousarray(r.sph_body, np.int32) if ns else None,
            _f32(r.sph_xyzr, (-1,)) if ns else None, ign)

    def set_scene(self, s: Scene, scene_id: int = -1) -> int:
        return hjcd.hjcd_set_scene(self.h, scene_id, len(s.sph_xyzr), _f32(s.sph_xyzr, (-1,)) if len(s.sph_xyzr) else None,
                                   len(s.box_lohi), _f32(s.box_lohi, (-1,)) if len(s.box_lohi) else None)

    def opts(self, n_samples: int, top_k: int, seed: int, eps_pos=1e-3, eps_ori=1e-2, params=None,
             samples_per_target=None) -> hjcd.hjcd_solve_opts:
        o = hjcd.hjcd_solve_opts()
        o.eps_pos, o.eps_ori = eps_pos, eps_ori
        o.n_samples, o.top_k = int(n_samples), int(top_k)
        o.seed = int(seed) & (2 ** 64 - 1)
        if params is not None:
            self._keep.append(params)
            o.params = hjcd.ct.pointer(params)
        if samples_per_target is not None:
            spt = np.ascontiguousarray(samples_per_target, np.int32)
            self._keep.append(spt)
            o.samples_per_target = spt.ctypes.data
        return o

    def solve(self, robot_id: int, scene_id: int, targets: torch.Tensor, n_samples: int, top_k: int, seed: int,
              n_dof: int, eps_pos=1e-3, eps_ori=1e-2, params=None, stream=None, out=None,
              samples_per_target=None, q_current=None):
        """Solve `targets` ([T, 7] float32, host or device); results are
        allocated on the targets' device unless `out` = (q, err, count) is given."""
        T = int(targets.shape[0])
        if out is None:
            dev = targets.device
            out = (torch.empty((T, top_k, n_dof), dtype=torch.float32, device=dev),
                   torch.empty((T, top_k, 2), dtype=torch.float32, device=dev),
                   torch.zeros((T,), dtype=torch.int32, device=dev))
        o = self.opts(n_samples, top_k, seed, eps_pos, eps_ori, params, samples_per_target)
        if q_current is None:
            hjcd.hjcd_solve(self.h, robot_id, scene_id, T, targets, o, out[0], out[1], out[2], stream)
        else:
            hjcd.hjcd_solve_nearest(self.h, robot_id, scene_id, T, targets, q_current, o, out[0], out[1], out[2],
                                    stream)
        return out

    def batch_item(self, robot_id: int, scene_id: int, targets, n_samples: int, top_k: int, seed: int, n_dof: int,
                   eps_pos=1e-3, eps_ori=1e-2, params=None, samples_per_target=None, spheres=None, boxes=None,
                   device=None, q_current=None):
        """An hjcd_batch_item with freshly allocated outputs (returned beside it).
        `spheres` [k, 4] / `boxes` [k, 6] give the request's own obstacles
        (scene_id < 0).  Outputs live on `device` (default: the targets')."""
        T = int(targets.shape[0])
        dev = targets.device if device is None else device
        out = (torch.empty((T, top_k, n_dof), dtype=torch.float32, device=dev),
               torch.empty((T, top_k, 2), dtype=torch.float32, device=dev),
               torch.zeros((T,), dtype=torch.int32, device=dev))
        it = hjcd.hjcd_batch_item()
        it.robot_id, it.scene_id, it.n_targets = int(robot_id), int(scene_id), T
        it.targets_pq = hjcd.ptr(targets)
        it.opts = self.opts(n_samples, top_k, seed, eps_pos, eps_ori, params, samples_per_target)
        if spheres is not None and len(spheres):
            sp = _f32(spheres, (-1,))
            self._keep.append(sp)
            it.n_inline_spheres, it.inline_spheres = len(spheres), sp.ctypes.data
        if boxes is not None and len(boxes):
            bx = _f32(boxes, (-1,))
            self._keep.append(bx)
            it.n_inline_boxes, it.inline_boxes = len(boxes), bx.ctypes.data
        it.out_q, it.out_err, it.out_count = (hjcd.ptr(x) for x in out)
        if q_current is not None:
            self._keep.append(q_current)
            it.q_current = hjcd.ptr(q_current)
        self._keep.append(targets)
        return it, out

    def solve_batch(self, items, params=None, stream=None) -> None:
        hjcd.hjcd_solve_batch(self.h, items, params, stream)

    def fk(self, robot_id: int, theta_soa: torch.Tensor, stream=None) -> torch.Tensor:
        """Flange poses [C, 7] of joint vectors given as a device tensor [n, C]."""
        C = int(theta_soa.shape[1])
        out = torch.empty((C, 7), dtype=torch.float32, device=theta_soa.device)
        hjcd.hjcd_fk(self.h, robot_id, C, theta_soa, theta_soa.stride(0), out, stream)
        return out

    def collide(self, robot_id: int, scene_id: int, theta_soa: torch.Tensor, stream=None) -> torch.Tensor:
        C = int(theta_soa.shape[1])
        hit = torch.zeros((C,), dtype=torch.uint8, device=theta_soa.device)
        hjcd.hjcd_collide(self.h, robot_id, scene_id, C, theta_soa, theta_soa.stride(0), hit, stream)
        return hit
