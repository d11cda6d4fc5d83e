"""The C-ABI library builds, loads without a GPU and exports what its header declares."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2510_07514_gb300 import build, hjcd, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hjcd.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return hjcd.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hjcd_[a-z0-9_]+)\s*\(", src)))


def test_header_declarations_are_exported(lib):
    names = _declared()
    assert len(names) >= 20
    raw = ctypes.CDLL(hjcd.lib_path())
    for nm in names:
        assert hasattr(raw, nm), f"{nm} declared in hjcd.h but not exported"
    assert sorted(hjcd.EXPORTS) == names


def test_default_params_match_the_parameter_table(lib):
    p = hjcd.hjcd_default_params()
    for k, v in inputs.DEFAULT_PARAMS.items():
        got = getattr(p, k)
        if isinstance(got, int):
            assert got == v, k
        else:
            assert got == pytest.approx(float(np.float32(v)), rel=1e-7), k


def test_status_strings(lib):
    assert hjcd.hjcd_status_string(0) == "ok"
    assert "invalid" in hjcd.hjcd_status_string(-1)


def test_init_without_gpu_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(hjcd.HjcdError):
        hjcd.hjcd_init(0)


def test_struct_layouts(lib):
    # field order and sizes of the structs passed by pointer
    assert ctypes.sizeof(hjcd.hjcd_params) == 20 * 4
    assert ctypes.sizeof(hjcd.hjcd_solve_opts) == 4 * 4 + 8 + 8 + 8
    assert ctypes.sizeof(hjcd.hjcd_ccd_trace) == 10 * 8
    assert ctypes.sizeof(hjcd.hjcd_lm_trace) == 5 * 8
    assert ctypes.sizeof(hjcd.hjcd_batch_item) == 4 * 4 + 2 * 8 + 2 * 4 + 8 + ctypes.sizeof(hjcd.hjcd_solve_opts) + 4 * 8
    assert ctypes.sizeof(hjcd.hjcd_server_opts) == 4 + 4 + 8 + 8 + 8
    assert ctypes.sizeof(hjcd.hjcd_request_info) == 4 + 4 + 8 + 8
    assert ctypes.sizeof(hjcd.hjcd_tune_report) == 6 * 4 + 8 + 8


def test_inputs_are_deterministic():
    a, b = inputs.cfg2(8, 16), inputs.cfg2(8, 16)
    assert np.array_equal(a.theta_gen, b.theta_gen)
    assert np.array_equal(a.robot.sph_xyzr, b.robot.sph_xyzr)
    assert np.array_equal(a.scene.sph_xyzr, b.scene.sph_xyzr)
    assert a.robot.sph_xyzr.shape == (60, 4) and a.scene.sph_xyzr.shape == (200, 4) and a.scene.box_lohi.shape == (20, 6)
    assert np.all(a.theta_gen >= a.robot.lo) and np.all(a.theta_gen <= a.robot.hi)
    r = a.robot.sph_xyzr[:, 3]
    assert r.min() >= 0.04 and r.max() <= 0.08
    chains = inputs.cfg3_chains()
    assert [c.n for c in chains] == list(inputs.CFG3_DOFS)
