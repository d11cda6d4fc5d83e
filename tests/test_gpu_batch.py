"""Packed batches (hjcd_solve_batch): requests of different robots, scenes
(resident, inline, none), seed counts, tolerances, top_k and iteration caps
in one launch per phase.

A request's results must not depend on what it is packed with: each target
row keys its random streams by its request's seed and its index inside the
request, so the batch and the request alone give the same bits.  The mixed
batch is also checked against the oracle (every solution re-verified, success
rates compared).
"""
import numpy as np
import pytest
import torch

import oracle as orc
from paper_2510_07514_gb300 import api, build, hjcd, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    orc.build()
    c = api.Context(0)
    yield c
    c.close()


def f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


def _robots():
    chains = inputs.cfg3_chains()
    return [inputs.panda_with_spheres(np.random.default_rng(5)), chains[1], chains[3], chains[5], inputs.panda()]


def _mix_specs():
    """(robot, scene kind, T, seeds, top_k, eps_pos, eps_ori, seed, caps)"""
    return [
        (0, "resident", 9, 256, 4, 1e-3, 1e-2, 11, None),
        (1, "inline", 7, [32, 40, 64, 100, 33, 256, 48], 2, 1e-3, 1e-2, 12, None),
        (2, "none", 5, 128, 1, 2e-3, 2e-2, 13, (12, 10)),
        (3, "inline", 4, 64, 3, 1e-3, 1e-2, 14, None),
        (4, "none", 6, 96, 5, 1e-3, 1e-2, 15, (20, 30)),
        (0, "resident", 3, 512, 2, 1e-3, 1e-2, 16, None),
        (1, "none", 2, 77, 1, 5e-4, 5e-3, 17, None),
    ]


def _setup(ctx):
    rng = np.random.default_rng(41)
    robs = _robots()
    rids = [ctx.add_robot(r) for r in robs]
    scene = inputs.random_scene(rng, 60, 6)
    sid = ctx.set_scene(scene)
    reqs = []
    for (ri, kind, T, seeds, k, ep, eo, seed, caps) in _mix_specs():
        rob = robs[ri]
        th = rng.uniform(rob.lo, rob.hi, (T, rob.n))
        tg = f32(orc.pose(orc.Robot(rob), f32(th)))
        inl = inputs.random_scene(rng, 25, 3) if kind == "inline" else None
        params = api.make_params(cd_max_iters=caps[0], lm_max_iters=caps[1]) if caps else None
        reqs.append(dict(ri=ri, kind=kind, T=T, seeds=seeds, k=k, ep=ep, eo=eo, seed=seed, caps=caps,
                         tg=tg, inl=inl, params=params))
    return robs, rids, scene, sid, reqs


def _item(ctx, rids, sid, robs, r, device="cuda"):
    spt = r["seeds"] if isinstance(r["seeds"], list) else None
    n = r["seeds"] if spt is None else 0
    scene_id = sid if r["kind"] == "resident" else -1
    sph = r["inl"].sph_xyzr if r["inl"] is not None else None
    box = r["inl"].box_lohi if r["inl"] is not None else None
    tg = dev(r["tg"]) if device == "cuda" else torch.as_tensor(np.ascontiguousarray(r["tg"]), dtype=torch.float32)
    return ctx.batch_item(rids[r["ri"]], scene_id, tg, max(n, 1), r["k"], r["seed"], robs[r["ri"]].n,
                          r["ep"], r["eo"], r["params"], spt, sph, box)


def _same(a, b):
    qa, ea, ca = (host(x) for x in a)
    qb, eb, cb = (host(x) for x in b)
    assert np.array_equal(ca, cb)
    for t in range(len(ca)):
        c = int(ca[t])
        assert np.array_equal(qa[t, :c], qb[t, :c])
        assert np.array_equal(ea[t, :c], eb[t, :c])
        assert np.all(np.isnan(qa[t, c:])) and np.all(np.isnan(qb[t, c:]))


def test_each_request_is_the_same_alone_and_in_the_mix(ctx):
    robs, rids, scene, sid, reqs = _setup(ctx)
    pairs = [_item(ctx, rids, sid, robs, r) for r in reqs]
    ctx.solve_batch([p[0] for p in pairs])
    for r, (it, out) in zip(reqs, pairs):
        alone_it, alone_out = _item(ctx, rids, sid, robs, r)
        ctx.solve_batch([alone_it])
        _same(out, alone_out)
        if r["kind"] != "inline" and not isinstance(r["seeds"], list):
            # and through the one-request entry point
            q, e, c = ctx.solve(rids[r["ri"]], sid if r["kind"] == "resident" else -1, dev(r["tg"]), r["seeds"],
                                r["k"], r["seed"], robs[r["ri"]].n, r["ep"], r["eo"],
                                r["params"] if r["params"] is not None else api.make_params())
            _same(out, (q, e, c))
    # reversed order packs the requests differently: same bits again
    pairs2 = [_item(ctx, rids, sid, robs, r) for r in reqs[::-1]]
    ctx.solve_batch([p[0] for p in pairs2])
    for (it, out), (it2, out2) in zip(pairs, pairs2[::-1]):
        _same(out, out2)


def test_host_outputs_and_host_targets_in_a_batch(ctx):
    robs, rids, scene, sid, reqs = _setup(ctx)
    pd = [_item(ctx, rids, sid, robs, r) for r in reqs]
    ph = [_item(ctx, rids, sid, robs, r, device="cpu") for r in reqs]
    ctx.solve_batch([p[0] for p in pd])
    ctx.solve_batch([p[0] for p in ph])
    for (a, oa), (b, ob) in zip(pd, ph):
        _same(oa, ob)


def _verify(orob, osc, rob, tg, q, err, cnt, eps_pos, eps_ori):
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


def test_mixed_batch_matches_the_oracle(ctx):
    """Three robots (Panda with spheres and a resident scene, a 7-DoF and a
    12-DoF random chain with their own inline scenes) in one batch; targets
    are poses of configurations the oracle finds collision-free."""
    rng = np.random.default_rng(43)
    chains = inputs.cfg3_chains()
    robs = [inputs.panda_with_spheres(np.random.default_rng(5)), chains[1], chains[3]]
    rids = [ctx.add_robot(r) for r in robs]
    scene = inputs.random_scene(rng, 80, 8)
    sid = ctx.set_scene(scene)
    T, S, k = 48, 128, 2
    items, outs, meta = [], [], []
    for i, rob in enumerate(robs):
        sc = scene if i == 0 else inputs.random_scene(rng, 40, 4)
        orob, osc = orc.Robot(rob), orc.Scene(sc)
        pool = f32(rng.uniform(rob.lo, rob.hi, (40 * T, rob.n)))
        hit, _ = orc.collide(orob, osc, pool)
        keep = pool[~hit][:T]
        assert len(keep) == T
        tg = f32(orc.pose(orob, keep))
        it, out = ctx.batch_item(rids[i], sid if i == 0 else -1, dev(tg), S, k, 100 + i, rob.n,
                                 spheres=None if i == 0 else sc.sph_xyzr, boxes=None if i == 0 else sc.box_lohi)
        items.append(it)
        outs.append(out)
        meta.append((rob, orob, osc, tg))
    ctx.solve_batch(items)
    sg, so = [], []
    for i, (rob, orob, osc, tg) in enumerate(meta):
        q, e, c = (host(x) for x in outs[i])
        c = c.astype(int)
        sg.append(_verify(orob, osc, rob, tg, q, e, c, 1e-3, 1e-2))
        o = orc.solve(orob, osc, orc.make_params(1e-3, 1e-2, seed=100 + i), tg, S, k)
        so.append((o["count"] > 0) & (o["err"][:, 0, 0] <= 1e-3) & (o["err"][:, 0, 1] <= 1e-2))
    sg, so = np.concatenate(sg), np.concatenate(so)
    assert abs(sg.mean() - so.mean()) <= 0.04 + 1e-12, (sg.mean(), so.mean())
    assert sg.mean() > 0.5


def test_batch_edge_cases(ctx):
    robs, rids, scene, sid, reqs = _setup(ctx)
    # an empty request inside a batch, and an empty batch
    it, out = _item(ctx, rids, sid, robs, reqs[0])
    empty = hjcd.hjcd_batch_item()
    empty.robot_id, empty.scene_id, empty.n_targets = rids[0], -1, 0
    empty.opts = ctx.opts(64, 1, 0)
    ctx.solve_batch([empty, it, empty])
    a_it, a_out = _item(ctx, rids, sid, robs, reqs[0])
    ctx.solve_batch([a_it])
    _same(out, a_out)
    ctx.solve_batch([])
    # unknown robot, too many distinct robots
    bad = hjcd.hjcd_batch_item()
    bad.robot_id, bad.scene_id, bad.n_targets = 10 ** 6, -1, 0
    bad.opts = ctx.opts(64, 1, 0)
    with pytest.raises(hjcd.HjcdError) as ei:
        ctx.solve_batch([bad])
    assert ei.value.status == hjcd.HJCD_ENOTFOUND
    many = [ctx.add_robot(inputs.planar([0.3, 0.2])) for _ in range(hjcd.HJCD_MAX_BATCH_ROBOTS + 1)]
    tg = dev(f32(orc.pose(orc.Robot(inputs.planar([0.3, 0.2])), np.zeros((1, 2)))))
    its = [ctx.batch_item(r, -1, tg, 8, 1, 0, 2)[0] for r in many]
    with pytest.raises(hjcd.HjcdError) as ei:
        ctx.solve_batch(its)
    assert ei.value.status == hjcd.HJCD_EINVAL
    ctx.solve_batch(its[:hjcd.HJCD_MAX_BATCH_ROBOTS])


def test_graph_replay_equals_the_batch_and_follows_new_targets(ctx):
    robs, rids, scene, sid, reqs = _setup(ctx)
    pairs = [_item(ctx, rids, sid, robs, r) for r in reqs]
    g = hjcd.hjcd_graph_create(ctx.h, [p[0] for p in pairs])
    try:
        hjcd.hjcd_graph_launch(ctx.h, g)
        hjcd.hjcd_graph_check(ctx.h, g)
        for r, (it, out) in zip(reqs, pairs):
            a_it, a_out = _item(ctx, rids, sid, robs, r)
            ctx.solve_batch([a_it])
            _same(out, a_out)
        # new poses written into the same target buffers: the replay solves them
        rng = np.random.default_rng(77)
        new = []
        for r, (it, out) in zip(reqs, pairs):
            rob = robs[r["ri"]]
            tg = f32(orc.pose(orc.Robot(rob), f32(rng.uniform(rob.lo, rob.hi, (r["T"], rob.n)))))
            t_dev = torch.as_tensor(np.ascontiguousarray(tg), dtype=torch.float32)
            torch.cuda.synchronize()
            ctx_keep = [k for k in ctx._keep if isinstance(k, torch.Tensor) and k.data_ptr() == it.targets_pq]
            assert ctx_keep, "target buffer of the item not found"
            ctx_keep[0].copy_(t_dev)
            q = dict(r)
            q["tg"] = tg
            new.append(q)
        for _ in range(2):
            hjcd.hjcd_graph_launch(ctx.h, g)
        hjcd.hjcd_graph_check(ctx.h, g)
        for r, (it, out) in zip(new, pairs):
            a_it, a_out = _item(ctx, rids, sid, robs, r)
            ctx.solve_batch([a_it])
            _same(out, a_out)
    finally:
        hjcd.hjcd_graph_destroy(g)
    h_it, _ = _item(ctx, rids, sid, robs, reqs[0], device="cpu")
    with pytest.raises(hjcd.HjcdError) as ei:
        hjcd.hjcd_graph_create(ctx.h, [h_it])
    assert ei.value.status == hjcd.HJCD_EINVAL


def test_launch_configuration_does_not_change_results(ctx):
    robs, rids, scene, sid, reqs = _setup(ctx)
    ref = None
    try:
        for blk, wp in ((128, 4), (64, 2), (256, 8), (64, 8), (256, 2)):
            hjcd.hjcd_set_launch_config(ctx.h, blk, wp)
            pairs = [_item(ctx, rids, sid, robs, r) for r in reqs]
            ctx.solve_batch([p[0] for p in pairs])
            if ref is None:
                ref = pairs
            else:
                for (a, oa), (b, ob) in zip(ref, pairs):
                    _same(oa, ob)
        with pytest.raises(hjcd.HjcdError):
            hjcd.hjcd_set_launch_config(ctx.h, 96, 4)
    finally:
        hjcd.hjcd_set_launch_config(ctx.h, 64, 8)  # the defaults


def test_autotune_picks_a_valid_configuration(ctx):
    wl = inputs.cfg1()
    rid = ctx.add_robot(wl.robot)
    rng = np.random.default_rng(51)
    tg = f32(orc.pose(orc.Robot(wl.robot), f32(rng.uniform(wl.robot.lo, wl.robot.hi, (64, 7)))))
    it, _ = ctx.batch_item(rid, -1, dev(tg), 128, 1, 3, 7)
    try:
        tuned, rep = hjcd.hjcd_autotune(ctx.h, [it], None, 0.02, 2)
        assert rep.ccd_block in (64, 128, 256) and rep.lm_warps in (2, 4, 8)
        assert rep.cd_max_iters in (8, 12, 16, 24, 32, 48) and rep.lm_max_iters in (8, 12, 16, 20, 30)
        assert (tuned.cd_max_iters, tuned.lm_max_iters) == (rep.cd_max_iters, rep.lm_max_iters)
        assert rep.success_rate >= rep.best_success_rate - 0.02 - 1e-6
        assert rep.trials == 9 + 30 and rep.ms > 0
        # the tuned parameters solve the calibration batch at the reported success rate
        q, e, c = ctx.solve(rid, -1, dev(tg), 128, 1, 3, 7, params=tuned)
        e, c = host(e), host(c)
        succ = np.mean((c > 0) & (e[:, 0, 0] <= 1e-3) & (e[:, 0, 1] <= 1e-2))
        assert abs(succ - rep.success_rate) < 1e-6
    finally:
        hjcd.hjcd_set_launch_config(ctx.h, 64, 8)  # the defaults


def test_solve_nearest_ranks_by_distance_to_the_current_configuration(ctx):
    """hjcd_solve_nearest returns the same collision-free candidates as
    hjcd_solve, reordered: those within the tolerances first, nearest to
    q_current (squared joint distance), then the rest by score."""
    wl = inputs.cfg1()
    rob = wl.robot
    rid = ctx.add_robot(rob)
    rng = np.random.default_rng(81)
    T = 16
    tg = dev(f32(orc.pose(orc.Robot(rob), f32(rng.uniform(rob.lo, rob.hi, (T, 7))))))
    qref = f32(rng.uniform(rob.lo, rob.hi, (T, 7)))
    q0, e0, c0 = (host(x) for x in ctx.solve(rid, -1, tg, 64, 64, 5, 7))
    q1, e1, c1 = (host(x) for x in ctx.solve(rid, -1, tg, 64, 64, 5, 7, q_current=dev(qref)))
    assert np.array_equal(c0, c1)
    n_ok = 0
    for t in range(T):
        c = int(c0[t])
        a = {tuple(r) for r in q0[t, :c]}
        b = {tuple(r) for r in q1[t, :c]}
        assert a == b
        ok = (e1[t, :c, 0] <= 1e-3) & (e1[t, :c, 1] <= 1e-2)
        k = int(ok.sum())
        n_ok += k
        assert np.all(ok[:k]) and not np.any(ok[k:])  # within-tolerance rows first
        d = np.sum((q1[t, :k].astype(np.float32) - qref[t].astype(np.float32)) ** 2, axis=1)
        assert np.all(np.diff(d) >= -1e-6 * np.maximum(d[1:], 1e-12))
        rest = [tuple(r) for r in q1[t, k:c]]
        order0 = [tuple(r) for r in q0[t, :c] if tuple(r) in set(rest)]
        assert rest == order0  # the others keep the score order
    assert n_ok > T
    # in a batch, a request with references and one without: the latter keeps score order
    it1, o1 = ctx.batch_item(rid, -1, tg, 64, 64, 5, 7, q_current=dev(qref))
    it2, o2 = ctx.batch_item(rid, -1, tg, 64, 64, 5, 7)
    ctx.solve_batch([it1, it2])
    _same(o1, (dev(q1), dev(e1), torch.as_tensor(c1, device="cuda")))
    _same(o2, (dev(q0), dev(e0), torch.as_tensor(c0, device="cuda")))


def test_segmented_mixed_robot_batch_equals_each_request_alone(ctx):
    """Two robots (7 and 12 joints) with equal seed counts and enough seeds in
    total to fill every SM with 2048+ run PO-CCD as three iteration segments,
    whose hand-over lists then mix the robots' candidates; alone, each request
    is below that size and runs PO-CCD in one launch.  Same bits either way."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    M = 1000
    T1 = sms * 2048 // (2 * M) + 8   # each request alone stays below sms * 2048 seeds
    T2 = sms * 2048 // M - T1 + 8    # together they exceed it
    robs = _robots()
    rng = np.random.default_rng(77)
    rA, rB = ctx.add_robot(robs[0]), ctx.add_robot(robs[2])
    sid = ctx.set_scene(inputs.random_scene(rng, 40, 4))
    tA = dev(f32(orc.pose(orc.Robot(robs[0]), f32(rng.uniform(robs[0].lo, robs[0].hi, (T1, robs[0].n))))))
    tB = dev(f32(orc.pose(orc.Robot(robs[2]), f32(rng.uniform(robs[2].lo, robs[2].hi, (T2, robs[2].n))))))
    assert (T1 + T2) * M >= sms * 2048 and max(T1, T2) * M < sms * 2048
    itA, oA = ctx.batch_item(rA, sid, tA, M, 3, 31, robs[0].n)
    itB, oB = ctx.batch_item(rB, -1, tB, M, 2, 32, robs[2].n)
    torch.cuda.synchronize()
    n0 = hjcd.hjcd_launch_count(ctx.h)
    ctx.solve_batch([itA, itB])
    torch.cuda.synchronize()
    n1 = hjcd.hjcd_launch_count(ctx.h)
    aloneA = ctx.solve(rA, sid, tA, M, 3, 31, robs[0].n)
    torch.cuda.synchronize()
    n2 = hjcd.hjcd_launch_count(ctx.h)
    aloneB = ctx.solve(rB, -1, tB, M, 2, 32, robs[2].n)
    assert (n1 - n0) - (n2 - n1) == 2  # the batch's PO-CCD took three launches, the request alone one
    for got, ref in ((oA, aloneA), (oB, aloneB)):
        (qa, ea, ca), (qb, eb, cb) = [host(x) for x in got], [host(x) for x in ref]
        ca, cb = ca.astype(np.int64), cb.astype(np.int64)
        assert np.array_equal(ca, cb)
        assert ca.sum() > 0
        for t in range(len(ca)):
            assert np.array_equal(qa[t, :ca[t]], qb[t, :cb[t]])
            assert np.array_equal(ea[t, :ca[t]], eb[t, :cb[t]])


def test_autotuned_caps_match_the_oracle_with_the_same_caps(ctx):
    """The autotuner changes results only through the iteration caps it picks
    (reading c9 and c17 leave them as parameters): with the tuned caps the
    mixed-robot batch must solve like the oracle run with the same caps --
    success within one point per robot class, every solution re-verified."""
    rng = np.random.default_rng(57)
    chains = inputs.cfg3_chains()
    robs = [inputs.panda_with_spheres(np.random.default_rng(5)), chains[1], chains[3]]
    rids = [ctx.add_robot(r) for r in robs]
    scene = inputs.random_scene(rng, 60, 6)
    sid = ctx.set_scene(scene)
    S = 128
    cal = []
    for i, rob in enumerate(robs):
        tg = f32(orc.pose(orc.Robot(rob), f32(rng.uniform(rob.lo, rob.hi, (24, rob.n)))))
        cal.append(ctx.batch_item(rids[i], -1, dev(tg), S, 1, 500 + i, rob.n)[0])
    try:
        tuned, rep = hjcd.hjcd_autotune(ctx.h, cal, None, 0.02, 1)
    finally:
        hjcd.hjcd_set_launch_config(ctx.h, 64, 8)
    caps = dict(cd_max_iters=int(tuned.cd_max_iters), lm_max_iters=int(tuned.lm_max_iters))
    T = 300
    items, outs, meta = [], [], []
    for i, rob in enumerate(robs):
        sc = scene if i == 0 else None
        orob, osc = orc.Robot(rob), (orc.Scene(sc) if sc is not None else None)
        pool = f32(rng.uniform(rob.lo, rob.hi, (20 * T, rob.n)))
        keep = pool[~orc.collide(orob, osc, pool)[0]][:T] if len(rob.sph_body) else pool[:T]
        assert len(keep) == T
        tg = f32(orc.pose(orob, keep))
        it, out = ctx.batch_item(rids[i], sid if i == 0 else -1, dev(tg), S, 1, 600 + i, rob.n,
                                 params=api.make_params(**caps))
        items.append(it)
        outs.append(out)
        meta.append((rob, orob, osc, tg))
    ctx.solve_batch(items, params=tuned)
    sg_all, so_all = [], []
    for i, (rob, orob, osc, tg) in enumerate(meta):
        q, e, c = (host(x) for x in outs[i])
        sg = _verify(orob, osc, rob, tg, q, e, c.astype(int), 1e-3, 1e-2)
        o = orc.solve(orob, osc, orc.make_params(1e-3, 1e-2, seed=600 + i, **caps), tg, S, 1)
        so = (o["count"] > 0) & (o["err"][:, 0, 0] <= 1e-3) & (o["err"][:, 0, 1] <= 1e-2)
        assert abs(sg.mean() - so.mean()) <= 0.03 + 1e-12, (i, caps, sg.mean(), so.mean())
        sg_all.append(sg)
        so_all.append(so)
    sg, so = np.concatenate(sg_all), np.concatenate(so_all)
    assert abs(sg.mean() - so.mean()) <= 0.01 + 1e-12, (caps, sg.mean(), so.mean())


def test_solve_nearest_matches_the_oracle(ctx):
    """hjcd_solve_nearest against the oracle's whole method with the same
    reference configurations (reading c24): success rates within one point,
    every returned solution re-verified, and the converged rows nearest-first."""
    wl = inputs.cfg1()
    rob = wl.robot
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(83)
    T, S, k = 300, 128, 4
    tg = f32(orc.pose(orob, f32(rng.uniform(rob.lo, rob.hi, (T, 7)))))
    qref = f32(rng.uniform(rob.lo, rob.hi, (T, 7)))
    q, e, c = (host(x) for x in ctx.solve(rid, -1, dev(tg), S, k, 19, 7, q_current=dev(qref)))
    c = c.astype(int)
    sg = _verify(orob, None, rob, tg, q, e, c, 1e-3, 1e-2)
    o = orc.solve(orob, None, orc.make_params(1e-3, 1e-2, seed=19), tg, S, k, q_ref=qref)
    so = (o["count"] > 0) & (o["err"][:, 0, 0] <= 1e-3) & (o["err"][:, 0, 1] <= 1e-2)
    assert abs(sg.mean() - so.mean()) <= 0.01 + 1e-12, (sg.mean(), so.mean())
    for src_q, src_e, src_c in ((q, e, c), (o["q"], o["err"], o["count"])):
        for t in range(T):
            ok = (src_e[t, :src_c[t], 0] <= 1e-3) & (src_e[t, :src_c[t], 1] <= 1e-2)
            m = int(ok.sum())
            assert np.all(ok[:m])
            d = np.linalg.norm(src_q[t, :m] - qref[t], axis=1)
            assert np.all(np.diff(d) >= -1e-6)


@pytest.mark.parametrize("case", ["offsets_past_pi", "rotated_flange"])
def test_solve_with_general_kinematics_matches_the_oracle(ctx, case):
    """The kinematics' general forms inside a solve: joint offsets that put
    theta + offset outside (-pi, pi) for part of every joint's range (the
    range reduction, which the kernels leave out only when every robot of a
    launch keeps its angles inside), and a flange whose rotation is not the
    identity (the kernels take the last joint's axes directly only when it
    is).  Success within one point of the oracle's whole method, every
    solution re-verified."""
    import dataclasses

    base = inputs.panda()
    if case == "offsets_past_pi":
        rob = dataclasses.replace(base, theta_off=np.array([1.5, -1.2, 0.8, 2.0, -1.7, 1.1, 0.6]))
        assert np.max(np.abs(np.r_[rob.lo + rob.theta_off, rob.hi + rob.theta_off])) > np.pi
    else:
        c, s_ = np.cos(-np.pi / 4), np.sin(-np.pi / 4)  # a hand turned -45 degrees about the last axis
        fl = np.array(base.flange, float).reshape(4, 4).copy()
        fl[:3, :3] = [[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]]
        rob = dataclasses.replace(base, flange=fl.reshape(np.shape(base.flange)))
    rid = ctx.add_robot(rob)
    orob = orc.Robot(rob)
    rng = np.random.default_rng(89)
    T, S, k = 300, 128, 2
    tg = f32(orc.pose(orob, f32(rng.uniform(rob.lo, rob.hi, (T, 7)))))
    q, e, c = (host(x) for x in ctx.solve(rid, -1, dev(tg), S, k, 23, 7))
    sg = _verify(orob, None, rob, tg, q, e, c.astype(int), 1e-3, 1e-2)
    o = orc.solve(orob, None, orc.make_params(1e-3, 1e-2, seed=23), tg, S, k)
    so = (o["count"] > 0) & (o["err"][:, 0, 0] <= 1e-3) & (o["err"][:, 0, 1] <= 1e-2)
    assert sg.mean() >= 0.9
    assert abs(sg.mean() - so.mean()) <= 0.01 + 1e-12, (sg.mean(), so.mean())


def test_tracking_loop_follows_a_scene_rewritten_every_frame(ctx):
    """The tracking use (Sec. VI-D): each frame the obstacle scene is replaced
    in place (hjcd_set_scene on the same id) and the next pose is solved from
    the current configuration.  Each frame's solutions must be collision-free
    in that frame's scene under the oracle's brute force, and equal a solve
    in a fresh context holding only that scene."""
    rng = np.random.default_rng(87)
    rob = inputs.panda_with_spheres(np.random.default_rng(5))
    orob = orc.Robot(rob)
    rid = ctx.add_robot(rob)
    sid = ctx.set_scene(inputs.random_scene(rng, 10, 2))
    fresh = api.Context(0)
    try:
        frid = fresh.add_robot(rob)
        q_cur = f32(rng.uniform(rob.lo, rob.hi, (1, 7)))
        for frame in range(4):
            scene = inputs.random_scene(rng, 24, 2)
            osc = orc.Scene(scene)
            ctx.set_scene(scene, scene_id=sid)
            pool = f32(np.clip(q_cur + rng.normal(0, 0.2, (400, 7)), rob.lo, rob.hi))
            keep = pool[~orc.collide(orob, osc, pool)[0]][:1]
            assert len(keep) == 1
            tg = f32(orc.pose(orob, keep))
            got = ctx.solve(rid, sid, dev(tg), 256, 2, 700 + frame, 7, q_current=dev(q_cur))
            q, e, c = (host(x) for x in got)
            _verify(orob, osc, rob, tg, q, e, c.astype(int), 1e-3, 1e-2)
            fsid = fresh.set_scene(scene)
            _same(got, fresh.solve(frid, fsid, dev(tg), 256, 2, 700 + frame, 7, q_current=dev(q_cur)))
            if c[0] > 0:
                q_cur = f32(q[0, :1])
    finally:
        fresh.close()
