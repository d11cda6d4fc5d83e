"""Seeds of a target sharded across devices: the exchange step on CPU ranks
(gloo, world size 2) and, on the GPU, shards simulated in one process whose
merged result must equal the single-device solve bit for bit."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2510_07514_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_lists(rank, T=3, K=4, n=5):
    g = torch.Generator().manual_seed(100 + rank)
    return (torch.rand((T, K), generator=g), torch.randint(0, 1000, (T, K), generator=g, dtype=torch.int32),
            torch.rand((T, K, n), generator=g))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        gs, gi, gt = shard.allgather_lists(*_rank_lists(rank))
        q.put((rank, gs.numpy(), gi.numpy(), gt.numpy()))
    finally:
        dist.destroy_process_group()


def test_allgather_of_shard_lists_on_two_cpu_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict((r, (a, b, c)) for r, a, b, c in (q.get(timeout=120) for _ in ps))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        gs, gi, gt = got[r]
        assert gs.shape == (2, 3, 4) and gt.shape == (2, 3, 4, 5)
        for src in range(2):  # rank order, identical on every rank
            a, b, c = _rank_lists(src)
            assert np.array_equal(gs[src], a.numpy())
            assert np.array_equal(gi[src], b.numpy())
            assert np.array_equal(gt[src], c.numpy())


def test_seed_and_target_ranges_partition():
    for M in (1, 7, 1000, 4096):
        for world in (1, 2, 3, 8):
            r = [shard.seed_range(M, k, world) for k in range(world)]
            assert r[0][0] == 0 and r[-1][1] == M
            assert all(r[k][1] == r[k + 1][0] for k in range(world - 1))


@pytest.mark.gpu
def test_sharded_seeds_equal_the_single_device_solve():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as orc
    from paper_2510_07514_gb300 import api, build, hjcd, inputs
    build.build()
    c = api.Context(0)
    try:
        wl = inputs.cfg2(40, 1024)
        rid, sid = c.add_robot(wl.robot), c.set_scene(wl.scene)
        orob = orc.Robot(wl.robot)
        rng = np.random.default_rng(5)
        tg = torch.as_tensor(np.asarray(orc.pose(orob, rng.uniform(wl.robot.lo, wl.robot.hi, (40, 7))), np.float32),
                             device="cuda")
        M, k = 1024, 4
        ref = c.solve(rid, sid, tg, M, k, 13, 7)
        o = c.opts(M, k, 13)
        K = M // 4
        # three uneven shards in one process, lists gathered in a shuffled order
        bounds = [(0, 100), (100, 400), (400, 1024)]
        lists = []
        for s0, s1 in bounds:
            sc = torch.empty((40, K), device="cuda")
            ix = torch.empty((40, K), dtype=torch.int32, device="cuda")
            th = torch.empty((40, K, 7), device="cuda")
            hjcd.hjcd_shard_topk(c.h, rid, 40, tg, o, s0, s1, sc, ix, th)
            lists.append((sc, ix, th))
        order = [2, 0, 1]
        gs = torch.stack([lists[i][0] for i in order])
        gi = torch.stack([lists[i][1] for i in order])
        gt = torch.stack([lists[i][2] for i in order])
        ms, mi = torch.empty((40, K), device="cuda"), torch.empty((40, K), dtype=torch.int32, device="cuda")
        mt = torch.empty((40, K, 7), device="cuda")
        hjcd.hjcd_topk_merge(c.h, 40, 3, K, 7, gs, gi, gt, ms, mi, mt)
        q = torch.empty((40, k, 7), device="cuda")
        e = torch.empty((40, k, 2), device="cuda")
        cn = torch.empty((40,), dtype=torch.int32, device="cuda")
        hjcd.hjcd_solve_from_topk(c.h, rid, sid, 40, tg, 0, o, mt, q, e, cn)
        torch.cuda.synchronize()
        a = [x.cpu().numpy() for x in ref]
        b = [x.cpu().numpy() for x in (q, e, cn)]
        assert np.array_equal(a[2], b[2])
        for t in range(40):
            assert np.array_equal(a[0][t, :a[2][t]], b[0][t, :b[2][t]])
            assert np.array_equal(a[1][t, :a[2][t]], b[1][t, :b[2][t]])
        # the merged indices are each target's K best seeds of all 1024, best first
        assert np.all(np.diff(ms.cpu().numpy(), axis=1) >= 0)
        assert np.all((mi.cpu().numpy() >= 0) & (mi.cpu().numpy() < M))
        # and through the per-rank helper with one rank
        t0, q1, e1, c1 = shard.solve_sharded(c, rid, sid, tg, o, 7, 0, 1)
        assert t0 == 0 and np.array_equal(c1.cpu().numpy(), a[2])
        # a later range of the targets polished on its own keeps its targets' streams
        q2 = torch.empty((15, k, 7), device="cuda")
        e2 = torch.empty((15, k, 2), device="cuda")
        c2 = torch.empty((15,), dtype=torch.int32, device="cuda")
        hjcd.hjcd_solve_from_topk(c.h, rid, sid, 15, tg[25:].contiguous(), 25, o, mt[25:].contiguous(), q2, e2, c2)
        torch.cuda.synchronize()
        assert np.array_equal(c2.cpu().numpy(), a[2][25:])
        for t in range(15):
            assert np.array_equal(q2.cpu().numpy()[t, :a[2][25 + t]], a[0][25 + t, :a[2][25 + t]])
    finally:
        c.close()


def _cfg2_free_targets(T):
    """Poses of the first T joint samples of the 1000 x 1000 workload's
    generator that the oracle finds collision-free (a witness exists)."""
    import oracle as orc
    from paper_2510_07514_gb300 import inputs
    wl = inputs.cfg2(T, 512)
    orob, osc = orc.Robot(wl.robot), orc.Scene(wl.scene)
    pool = np.asarray(wl.theta_gen, np.float32).astype(np.float64)
    hit, _ = orc.collide(orob, osc, pool)
    keep = pool[~hit][:T]
    assert len(keep) == T
    return wl, np.asarray(orc.pose(orob, keep), np.float32)


def _gpu_worker(rank, world, port, q, T, M, k, seed):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2510_07514_gb300 import api
        wl, tg = _cfg2_free_targets(T)
        c = api.Context(0)
        try:
            rid, sid = c.add_robot(wl.robot), c.set_scene(wl.scene)
            t0, qq, ee, cc = shard.solve_sharded(c, rid, sid, torch.as_tensor(tg, device="cuda"), c.opts(M, k, seed),
                                                 7, rank, world)
            torch.cuda.synchronize()
            q.put((rank, t0, qq.cpu().numpy(), ee.cpu().numpy(), cc.cpu().numpy()))
        finally:
            c.close()
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_sharded_solve_on_two_ranks_matches_the_oracle():
    """Two processes (gloo ranks; both on the one GPU, their kernels
    independent) each run PO-CCD on half of every target's seeds, exchange
    their top-K lists, merge them and polish half of the targets.  Together
    their results equal the single-device solve bit for bit and solve like
    the oracle's whole method: success within one point, every solution
    re-verified by oracle kinematics and brute-force collision."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import oracle as orc
    from paper_2510_07514_gb300 import api, build
    build.build()
    orc.build()
    T, M, k, seed = 200, 512, 2, 29
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_gpu_worker, args=(r, 2, port, q, T, M, k, seed)) for r in range(2)]
    for p in ps:
        p.start()
    parts = sorted((q.get(timeout=600) for _ in ps), key=lambda x: x[1])
    for p in ps:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert [x[1] for x in parts] == [0, T // 2]
    qs = np.concatenate([x[2] for x in parts])
    es = np.concatenate([x[3] for x in parts])
    cs = np.concatenate([x[4] for x in parts]).astype(int)
    wl, tg = _cfg2_free_targets(T)
    c = api.Context(0)
    try:
        rid, sid = c.add_robot(wl.robot), c.set_scene(wl.scene)
        ref = [x.cpu().numpy() for x in c.solve(rid, sid, torch.as_tensor(tg, device="cuda"), M, k, seed, 7)]
    finally:
        c.close()
    assert np.array_equal(cs, ref[2])
    for t in range(T):
        assert np.array_equal(qs[t, :cs[t]], ref[0][t, :cs[t]])
        assert np.array_equal(es[t, :cs[t]], ref[1][t, :cs[t]])
    orob, osc = orc.Robot(wl.robot), orc.Scene(wl.scene)
    tg64 = tg.astype(np.float64)
    for t in range(T):
        for r in range(cs[t]):
            e = orc.residual(orob, qs[t, r].astype(np.float64), tg64[t])
            assert abs(np.linalg.norm(e[:3]) - es[t, r, 0]) < 1e-5 and abs(np.linalg.norm(e[3:]) - es[t, r, 1]) < 1e-5
            assert np.all(qs[t, r] >= wl.robot.lo - 1e-7) and np.all(qs[t, r] <= wl.robot.hi + 1e-7)
        if cs[t]:
            hit, margin = orc.collide(orob, osc, qs[t, :cs[t]].astype(np.float64))
            assert not np.any(hit & (margin >= 1e-6))
    sg = (cs > 0) & (es[:, 0, 0] <= 1e-3) & (es[:, 0, 1] <= 1e-2)
    o = orc.solve(orob, osc, orc.make_params(1e-3, 1e-2, seed=seed), tg64, M, k)
    so = (o["count"] > 0) & (o["err"][:, 0, 0] <= 1e-3) & (o["err"][:, 0, 1] <= 1e-2)
    assert abs(sg.mean() - so.mean()) <= 0.01 + 1e-12, (sg.mean(), so.mean())
