"""The seeds of a target sharded across devices (one process per GPU).

Each rank runs PO-CCD on its share of every target's seeds and keeps its
top-K (hjcd_shard_topk); the ranks exchange those lists -- the one collective,
K x (n + 2) values per target and rank -- and merge them (hjcd_topk_merge);
each rank then runs the rest of Alg. 2 for its share of the targets
(hjcd_solve_from_topk).  Results equal a single-device hjcd_solve.  Argument
marshalling and the exchange only: every step of the method runs in the CUDA
library.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import hjcd


def seed_range(M: int, rank: int, world: int) -> tuple[int, int]:
    """Seeds [begin, end) of rank `rank`: consecutive, as even as possible."""
    return rank * M // world, (rank + 1) * M // world


def target_range(T: int, rank: int, world: int) -> tuple[int, int]:
    return rank * T // world, (rank + 1) * T // world


def allgather_lists(score: torch.Tensor, index: torch.Tensor, theta: torch.Tensor, group=None):
    """Every rank's (score [T,K], seed index [T,K], joint vectors [T,K,n]),
    stacked in rank order: ([L,T,K], [L,T,K], [L,T,K,n]), on the inputs'
    device.  Over a gloo group device tensors travel through host memory (gloo
    gathers host tensors); over NCCL they stay on the device."""
    world = dist.get_world_size(group)
    via_host = score.is_cuda and dist.get_backend(group) == "gloo"
    out = []
    for x in (score, index, theta):
        y = x.contiguous().cpu() if via_host else x.contiguous()
        parts = [torch.empty_like(y) for _ in range(world)]
        dist.all_gather(parts, y, group=group)
        st = torch.stack(parts)
        out.append(st.to(x.device) if via_host else st)
    return tuple(out)


def solve_sharded(ctx, robot_id: int, scene_id: int, targets: torch.Tensor, opts: hjcd.hjcd_solve_opts, n_dof: int,
                  rank: int, world: int, group=None, stream=None):
    """This rank's part of a sharded solve: (first target, q, err, count) for
    its share of the targets.  `targets` ([T, 7], device) and `opts` must be
    the same on every rank."""
    T, M = int(targets.shape[0]), int(opts.n_samples)
    P = opts.params.contents if opts.params else hjcd.hjcd_default_params()
    K = max(1, M // int(P.dup_ratio))
    dev = targets.device
    s0, s1 = seed_range(M, rank, world)
    sc = torch.empty((T, K), dtype=torch.float32, device=dev)
    ix = torch.empty((T, K), dtype=torch.int32, device=dev)
    th = torch.empty((T, K, n_dof), dtype=torch.float32, device=dev)
    hjcd.hjcd_shard_topk(ctx.h, robot_id, T, targets, opts, s0, s1, sc, ix, th, stream)
    if world > 1:
        torch.cuda.synchronize(dev)
        gs, gi, gt = allgather_lists(sc, ix, th, group)
    else:
        gs, gi, gt = sc[None], ix[None], th[None]
    ms = torch.empty((T, K), dtype=torch.float32, device=dev)
    mi = torch.empty((T, K), dtype=torch.int32, device=dev)
    mt = torch.empty((T, K, n_dof), dtype=torch.float32, device=dev)
    hjcd.hjcd_topk_merge(ctx.h, T, gs.shape[0], K, n_dof, gs, gi, gt, ms, mi, mt, stream)
    t0, t1 = target_range(T, rank, world)
    k = int(opts.top_k)
    q = torch.empty((t1 - t0, k, n_dof), dtype=torch.float32, device=dev)
    e = torch.empty((t1 - t0, k, 2), dtype=torch.float32, device=dev)
    c = torch.empty((t1 - t0,), dtype=torch.int32, device=dev)
    if t1 > t0:
        hjcd.hjcd_solve_from_topk(ctx.h, robot_id, scene_id, t1 - t0, targets[t0:t1].contiguous(), t0, opts,
                                  mt[t0:t1].contiguous(), q, e, c, stream)
    return t0, q, e, c
