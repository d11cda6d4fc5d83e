"""The serving loop (hjcd_server_start / hjcd_submit / hjcd_wait): continuous
batching of requests of different robots, scenes and sizes.

Each served result must equal the request solved alone (hjcd_solve_batch with
that request only), bit for bit: a request's random streams are keyed by its
own seed and target indices, whatever batch it lands in.
"""
import threading
import time

import numpy as np
import pytest
import torch

import oracle as orc
from paper_2510_07514_gb300 import api, build, hjcd, inputs
from test_gpu_batch import _item, _same, _setup

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


def _alone(ctx, rids, sid, robs, r):
    it, out = _item(ctx, rids, sid, robs, r)
    ctx.solve_batch([it])
    return out


def _reqs_with_seeds(reqs, rounds):
    out = []
    for k in range(rounds):
        for r in reqs:
            q = dict(r)
            q["seed"] = r["seed"] + 1000 * k
            out.append(q)
    return out


def test_served_results_equal_the_request_alone(ctx):
    robs, rids, scene, sid, reqs = _setup(ctx)
    all_reqs = _reqs_with_seeds(reqs, 4)
    hjcd.hjcd_server_start(ctx.h, max_inflight=3)
    try:
        pairs = [_item(ctx, rids, sid, robs, r, device="cpu") for r in all_reqs]
        ids = []
        # two submitting threads, so requests arrive while others run
        def submit(part):
            for it, _ in part:
                ids.append(hjcd.hjcd_submit(ctx.h, it))
                time.sleep(0.0003)
        ths = [threading.Thread(target=submit, args=(pairs[i::2],)) for i in range(2)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        infos = [hjcd.hjcd_wait(ctx.h, i, 120.0) for i in ids]
    finally:
        hjcd.hjcd_server_stop(ctx.h)
    assert all(inf.status == 0 for inf in infos)
    assert max(inf.batch_requests for inf in infos) > 1  # the mix really was batched
    assert all(inf.total_ms >= inf.queued_ms >= 0.0 for inf in infos)
    for r, (it, out) in zip(all_reqs, pairs):
        _same(out, _alone(ctx, rids, sid, robs, r))


def test_admission_by_memory_and_plain_mode(ctx):
    robs, rids, scene, sid, reqs = _setup(ctx)
    # 6 MB of workspace per batch: the mix fits, one request of 40 x 8192 seeds needs more
    hjcd.hjcd_server_start(ctx.h, max_inflight=2, memory_budget=2 * 6 * 2 ** 20)
    try:
        pairs = [_item(ctx, rids, sid, robs, r, device="cpu") for r in reqs]
        ids = [hjcd.hjcd_submit(ctx.h, it) for it, _ in pairs]
        big = dict(reqs[0])
        big["T"], big["seeds"] = 40, 8192
        big["tg"] = np.repeat(reqs[0]["tg"][:1], 40, axis=0)
        bit, bout = _item(ctx, rids, sid, robs, big, device="cpu")
        bid = hjcd.hjcd_submit(ctx.h, bit)
        infos = [hjcd.hjcd_wait(ctx.h, i, 120.0) for i in ids]
        binfo = hjcd.hjcd_wait(ctx.h, bid, 120.0)
    finally:
        hjcd.hjcd_server_stop(ctx.h)
    assert binfo.status == hjcd.HJCD_ENOMEM
    assert all(inf.status == 0 for inf in infos)
    for r, (it, out) in zip(reqs, pairs):
        _same(out, _alone(ctx, rids, sid, robs, r))
    # plain path: one request per batch, one batch at a time
    hjcd.hjcd_server_start(ctx.h, max_inflight=1, max_batch_requests=1)
    try:
        pairs = [_item(ctx, rids, sid, robs, r, device="cpu") for r in reqs]
        ids = [hjcd.hjcd_submit(ctx.h, it) for it, _ in pairs]
        infos = [hjcd.hjcd_wait(ctx.h, i, 120.0) for i in ids]
    finally:
        hjcd.hjcd_server_stop(ctx.h)
    assert all(inf.batch_requests == 1 and inf.status == 0 for inf in infos)
    for r, (it, out) in zip(reqs, pairs):
        _same(out, _alone(ctx, rids, sid, robs, r))


def test_stop_finishes_admitted_requests_and_rejects_bad_ones(ctx):
    robs, rids, scene, sid, reqs = _setup(ctx)
    hjcd.hjcd_server_start(ctx.h)
    pairs = [_item(ctx, rids, sid, robs, r, device="cpu") for r in reqs]
    for it, _ in pairs:
        hjcd.hjcd_submit(ctx.h, it)
    with pytest.raises(hjcd.HjcdError):
        hjcd.hjcd_server_start(ctx.h)  # one server per context
    dit, _ = _item(ctx, rids, sid, robs, reqs[0])  # device buffers are not served
    with pytest.raises(hjcd.HjcdError) as ei:
        hjcd.hjcd_submit(ctx.h, dit)
    assert ei.value.status == hjcd.HJCD_EINVAL
    hjcd.hjcd_server_stop(ctx.h)  # returns after every admitted request finished
    for r, (it, out) in zip(reqs, pairs):
        _same(out, _alone(ctx, rids, sid, robs, r))
    with pytest.raises(hjcd.HjcdError):
        hjcd.hjcd_submit(ctx.h, pairs[0][0])  # no server


_FRESH_PROCESS = r"""
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
from paper_2510_07514_gb300 import api, hjcd, inputs
wl = inputs.cfg2(16, 64)
ctx = api.Context(0)
rid, sid = ctx.add_robot(wl.robot), ctx.set_scene(wl.scene)
th = torch.as_tensor(np.ascontiguousarray(wl.theta_gen[:16].T), dtype=torch.float32, device="cuda")
tg = ctx.fk(rid, th).cpu()
hjcd.hjcd_server_start(ctx.h, max_inflight=3)
ids, outs = [], []
try:
    # small requests first (the kernels' first launches need little shared memory), then large
    # ones while those still run
    for k, (T, S) in enumerate([(2, 64)] * 6 + [(4, 8192)] * 4):
        it, out = ctx.batch_item(rid, sid, tg[:T].contiguous(), S, 1, 100 + k, wl.robot.n, device=torch.device("cpu"))
        ids.append(hjcd.hjcd_submit(ctx.h, it))
        outs.append((it, out))
    infos = [hjcd.hjcd_wait(ctx.h, i, 120.0) for i in ids]
finally:
    hjcd.hjcd_server_stop(ctx.h)
bad = [inf.status for inf in infos if inf.status != 0]
print("statuses", [inf.status for inf in infos])
sys.exit(1 if bad else 0)
"""


def test_first_launches_small_then_large_on_concurrent_streams():
    """In a fresh process, small requests are served first and large ones
    (more than 48 KB of shared memory in the ranking kernel) arrive while they
    run on other streams: every request must succeed (a kernel's shared-memory
    limit raised at a later launch used to make that launch fail)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import os
    import subprocess
    import sys
    build.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _FRESH_PROCESS, root], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
