"""hjcd_solve_noalloc: the solve for callers that cannot allocate device memory
while they run (real-time control loops, processes whose device memory belongs
to another allocator).  Its scratch is a static device array shared by every
call; it must give the results of hjcd_solve on the same inputs, call after
call.  This file is collected last on purpose: a run that stops at the first
failure has then already run every other test."""
import numpy as np
import pytest
import torch

from paper_2510_07514_gb300 import api, build, hjcd, inputs

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    build.build()
    ctx = api.Context(0)
    wl = inputs.cfg2(64, 256)
    rid, sid = ctx.add_robot(wl.robot), ctx.set_scene(wl.scene)
    pool = torch.as_tensor(np.ascontiguousarray(wl.theta_gen.T), dtype=torch.float32, device="cuda")
    free = ctx.collide(rid, sid, pool) == 0
    tg = ctx.fk(rid, pool[:, free][:, :64].contiguous()).contiguous()
    yield ctx, wl, rid, sid, tg
    ctx.close()


def _noalloc(ctx, rid, sid, tg, S, K, seed, n):
    T = int(tg.shape[0])
    out = (torch.full((T, K, n), -7.0, device="cuda"), torch.full((T, K, 2), -7.0, device="cuda"),
           torch.full((T,), -1, dtype=torch.int32, device="cuda"))
    hjcd.hjcd_solve_noalloc(ctx.h, rid, sid, T, tg, ctx.opts(S, K, seed), out[0], out[1], out[2])
    return out


def _same(a, b):
    qa, ea, ca = (x.cpu().numpy() for x in a)
    qb, eb, cb = (x.cpu().numpy() for x in b)
    assert np.array_equal(ca, cb)
    for t in range(len(ca)):
        assert np.allclose(qa[t, :ca[t]], qb[t, :cb[t]], atol=TOL, rtol=0)
        assert np.allclose(ea[t, :ca[t]], eb[t, :cb[t]], atol=TOL, rtol=0)
        # rows past the count are NaN on both paths, whatever the buffers held before
        for x in (qa, ea, qb, eb):
            assert np.all(np.isnan(x[t, ca[t]:]))


def test_noalloc_matches_solve_on_consecutive_calls(setup):
    ctx, wl, rid, sid, tg = setup
    n = wl.robot.n
    # two calls in a row with different requests: the second finds the first's
    # data in the shared scratch and must not be affected by it
    for seed, T, S, K in ((wl.seed, 64, 256, 4), (wl.seed + 1, 48, 200, 3)):
        ref = ctx.solve(rid, sid, tg[:T], S, K, seed, n)
        got = _noalloc(ctx, rid, sid, tg[:T], S, K, seed, n)
        torch.cuda.synchronize()
        _same(ref, got)
        assert got[2].min().item() >= 1


def test_noalloc_fills_rows_past_the_count(setup):
    """Fewer collision-free solutions than top_k (8 seeds, top_k 20): the rows
    past each target's count read NaN, as hjcd_solve leaves them, on two calls
    in a row."""
    ctx, wl, rid, sid, tg = setup
    n = wl.robot.n
    for seed in (3, 4):
        ref = ctx.solve(rid, sid, tg[:16], 8, 20, seed, n)
        got = _noalloc(ctx, rid, sid, tg[:16], 8, 20, seed, n)
        torch.cuda.synchronize()
        _same(ref, got)
        assert got[2].max().item() < 20


def test_noalloc_rejects_work_beyond_its_scratch(setup):
    ctx, wl, rid, sid, tg = setup
    with pytest.raises(hjcd.HjcdError) as ei:
        _noalloc(ctx, rid, sid, tg, hjcd.HJCD_MAX_SAMPLES, 1, 1, wl.robot.n)   # 64 x 8192 candidates
    assert ei.value.status == hjcd.HJCD_EINVAL
    assert "scratch" in str(ei.value)
    with pytest.raises(hjcd.HjcdError):   # host buffers are refused
        hjcd.hjcd_solve_noalloc(ctx.h, rid, sid, 2, tg[:2].cpu(), ctx.opts(8, 1, 1),
                                torch.zeros((2, 1, 7)), torch.zeros((2, 1, 2)), torch.zeros(2, dtype=torch.int32))
