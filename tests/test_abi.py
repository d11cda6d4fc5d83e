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
    assert ctypes.sizeof(hjcd.hjcd_lm_trace) == 8 * 8
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


def test_device_arctangent_polynomial_error_bound():
    """The kernels' arctangent (hjcd_internal.cuh, atan01): its coefficients,
    read from the source, evaluated in binary32 with fused multiply-adds, stay
    within 1.5e-7 rad of atan over [0, 1] (float64 reference), and the
    quadrant reductions reproduce atan2 on a grid of all four quadrants."""
    import re
    src = open(os.path.join(ROOT, "paper_2510_07514_gb300", "csrc", "hjcd_internal.cuh")).read()
    body = src[src.index("float atan01(float t)"):src.index("float atan2_q1(")]
    c = [np.float32(float(x)) for x in re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", body)]
    assert len(c) == 8
    t = np.linspace(0, 1, 400001, dtype=np.float32)
    s = (t * t).astype(np.float32)

    def fma(a, b, d):  # one rounding, as the device's fmaf
        return (a.astype(np.float64) * b.astype(np.float64) + np.float64(d)).astype(np.float32)

    p = np.full_like(t, c[0])
    for ci in c[1:]:
        p = fma(p, s, ci)
    r = (t * p).astype(np.float32)
    assert np.max(np.abs(r.astype(np.float64) - np.arctan(t.astype(np.float64)))) < 1.5e-7

    def atan2_all(y, x):
        ay, ax = np.abs(y), np.abs(x)
        mx, mn = np.maximum(ax, ay), np.minimum(ax, ay)
        tt = np.where(mx > 0, mn / np.where(mx > 0, mx, 1), 0).astype(np.float32)
        ss = (tt * tt).astype(np.float32)
        pp = np.full_like(tt, c[0])
        for ci in c[1:]:
            pp = fma(pp, ss, ci)
        a = (tt * pp).astype(np.float64)
        a = np.where(ay > ax, np.pi / 2 - a, a)
        a = np.where(x < 0, np.pi - a, a)
        return np.copysign(a, y)

    g = np.linspace(-3, 3, 301, dtype=np.float32)
    Y, X = np.meshgrid(g, g)
    ref = np.arctan2(Y.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(atan2_all(Y, X) - ref)) < 3e-7


def test_arctangent_coefficients_are_the_fitting_scripts():
    """The kernels' arctangent coefficients are what csrc/fit_atan.py computes
    (the minimax fit of t P(t^2) to atan on [0, 1]), digit for digit."""
    import importlib.util
    import re
    csrc = os.path.join(ROOT, "paper_2510_07514_gb300", "csrc")
    spec = importlib.util.spec_from_file_location("fit_atan", os.path.join(csrc, "fit_atan.py"))
    fa = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(fa)
    c, z = fa.fit()
    assert z < 3e-8
    inc = open(os.path.join(csrc, "hjcd_internal.cuh")).read()
    got = re.findall(r"([-+]?\d\.\d+e[-+]\d+)f", inc[inc.index("float atan01(float t)"):inc.index("float atan2_q1(")])
    assert got == fa.formatted(c)


def test_device_ccd_constants():
    """Constants of the PO-CCD kernel read from its source: the table that
    replaces the division of the perturbation items (k_ccd.cu, kDivMagic) gives
    w / nb exactly, without overflowing 32 bits, for every item w < 32 nb of
    1..12 normal pairs; and the packed arctangent of the trials uses the
    coefficients of the scalar one (hjcd_internal.cuh, atan01)."""
    import re
    csrc = os.path.join(ROOT, "paper_2510_07514_gb300", "csrc")
    ccd = open(os.path.join(csrc, "k_ccd.cu")).read()
    table = re.search(r"kDivMagic\[13\] = \{([^}]*)\}", ccd).group(1)
    magic = [int(x) for x in table.split(",")]
    assert len(magic) == 13
    for nb in range(1, 13):
        w = np.arange(32 * nb, dtype=np.uint64)
        prod = w * np.uint64(magic[nb])
        assert int(prod.max()) < 2 ** 32
        assert np.array_equal(prod >> np.uint64(16), w // np.uint64(nb)), nb
    coef = r"([-+]?\d\.\d+e[-+]\d+)f"
    inc = open(os.path.join(csrc, "hjcd_internal.cuh")).read()
    scalar = re.findall(coef, inc[inc.index("float atan01(float t)"):inc.index("float atan2_q1(")])
    packed = re.findall(coef, ccd[ccd.index("float2 atan_poly2(float2 t)"):ccd.index("float2 quat_angle2(")])
    assert len(scalar) == 8 and packed == scalar


def test_serving_crossing_interpolation():
    """The bench's equal-p99 crossing: log-linear between the fastest point at
    or below the target p99 and the next faster one; unbracketed and
    unreachable sweeps reported as such."""
    import bench
    pts = [(100.0, 1.5, 400.0), (125.0, 1.7, 500.0), (156.0, 1.9, 625.0), (195.0, 2.4, 780.0)]
    r = bench._crossing(pts, 1.8)
    assert r["bracketed"]
    f = (1.8 - 1.7) / (1.9 - 1.7)
    assert r["rate"] == pytest.approx(np.exp(np.log(125.0) + f * np.log(156.0 / 125.0)), rel=1e-12)
    assert r["solves_per_s"] == pytest.approx(np.exp(np.log(500.0) + f * np.log(625.0 / 500.0)), rel=1e-12)
    assert 125.0 < r["rate"] < 156.0
    # every point meets the target: the fastest one, not bracketed
    r = bench._crossing(pts, 3.0)
    assert not r["bracketed"] and r["rate"] == 195.0
    # no point meets it
    assert bench._crossing(pts, 1.0) is None
    # a non-monotone sweep: the fastest point at or below the target decides
    r = bench._crossing([(100.0, 1.5, 1.0), (125.0, 1.9, 1.2), (156.0, 1.7, 1.5), (195.0, 2.5, 2.0)], 1.8)
    assert r["bracketed"] and 156.0 < r["rate"] < 195.0
