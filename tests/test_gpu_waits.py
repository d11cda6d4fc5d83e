"""The collision kernels' bounded wait for their bulk-copied obstacle tables
(the library's fault detection; the paper has none).

The wait is made to run out on purpose by giving its first poll loop a limit
of zero (hjcd_set_wait_limit): the kernel then sets its error flag, waits for
its own copy to land with the full limit -- so nothing stays in flight -- and
returns without verdicts.  The calls must report HJCD_ETIMEOUT, and the next
calls with the default limit must succeed and give the results of a fresh
context.
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


def test_staging_wait_that_runs_out_is_reported_and_the_context_recovers(ctx):
    rng = np.random.default_rng(91)
    rob = inputs.panda_with_spheres(np.random.default_rng(5))
    rid = ctx.add_robot(rob)
    sid = ctx.set_scene(inputs.random_scene(rng, 200, 20))
    orob = orc.Robot(rob)
    tg = np.asarray(orc.pose(orob, rng.uniform(rob.lo, rob.hi, (8, 7))), np.float32)
    th = torch.tensor(np.ascontiguousarray(rng.uniform(rob.lo, rob.hi, (512, 7)).T), dtype=torch.float32,
                      device="cuda")
    hit = torch.zeros((512,), dtype=torch.uint8, device="cuda")
    hjcd.hjcd_counters(ctx.h, reset=True)

    def solve_host():
        q = np.zeros((8, 2, 7), np.float32)
        e = np.zeros((8, 2, 2), np.float32)
        c = np.zeros((8,), np.int32)
        o = ctx.opts(128, 2, 5)
        hjcd.hjcd_solve(ctx.h, rid, sid, 8, tg, o, q, e, c)
        return q, e, c

    ref_hit = ctx.collide(rid, sid, th).cpu().numpy()
    ref = solve_host()
    try:
        hjcd.hjcd_set_wait_limit(ctx.h, 0)
        hjcd.hjcd_collide(ctx.h, rid, sid, 512, th, 512, hit)
        with pytest.raises(hjcd.HjcdError) as ei:
            hjcd.hjcd_counters(ctx.h)
        assert ei.value.status == hjcd.HJCD_ETIMEOUT
        for mode in (1, 0):  # the ranked filter's kernel and the filter over every candidate
            hjcd.hjcd_set_collision_mode(ctx.h, mode)
            with pytest.raises(hjcd.HjcdError) as ei:
                solve_host()
            assert ei.value.status == hjcd.HJCD_ETIMEOUT
    finally:
        hjcd.hjcd_set_wait_limit(ctx.h, -1)
        hjcd.hjcd_set_collision_mode(ctx.h, 1)
    # the default limit again: the same answers as before, and no error left behind
    got_hit = ctx.collide(rid, sid, th).cpu().numpy()
    assert np.array_equal(got_hit, ref_hit)
    hjcd.hjcd_counters(ctx.h)
    got = solve_host()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b, equal_nan=True)
