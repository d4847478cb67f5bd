"""Forward parity of the CUDA path against the FP64 oracle, through the C-ABI.

Sizes span several tiles per warp and a ragged tail; full-size workloads are
checked at every point, the oracle spread over the host cores (full_parity).
"""

import numpy as np
import pytest
import torch

import full_parity
import oracle
from paper_2302_08381_gb300 import _capi as C
from paper_2302_08381_gb300 import api, inputs
from parity_utils import (
    BF16_TOL,
    F32_GRAD,
    F32_VAL,
    F64_TOL,
    assert_grads,
    assert_values,
    grad_errors,
    value_bound,
    value_errors,
)

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _run(xyz_np, l_max, normalized, grad, kernel="auto", dtype=torch.float32, out_dtype=None, qprec="native", launch=None):
    xyz = torch.from_numpy(np.ascontiguousarray(xyz_np)).to(DEV, dtype)
    res = api.spherical_harmonics(
        xyz, l_max, normalized, gradients=grad, out_dtype=out_dtype, qprec=qprec, kernel=kernel, launch=launch
    )
    torch.cuda.synchronize()

    def host(t):
        return (t.float() if t.dtype == torch.bfloat16 else t).double().cpu().numpy()

    if grad:
        return host(res[0]), host(res[1])
    return host(res)


# --------------------------------------------------------------- small, every l_max
@pytest.mark.parametrize("kernel", ["point", "slice"])
@pytest.mark.parametrize("normalized", [False, True])
def test_f32_values_and_gradients_every_lmax(kernel, normalized):
    n = 1000 + 13
    xyz = inputs.shell_points(n, 0.5, 2.0, seed=100).astype(np.float64)
    xyz32 = xyz.astype(np.float32).astype(np.float64)
    for l_max in range(0, 17):
        v, g = _run(xyz32, l_max, normalized, True, kernel)
        rv, rg = oracle.spherical_harmonics_grad(xyz32, l_max, normalized)
        assert_values(v, xyz32, l_max, normalized, F32_VAL, ref=rv)
        assert_grads(g, xyz32, l_max, normalized, F32_GRAD, ref=rg)


@pytest.mark.parametrize("kernel", ["point", "slice"])
@pytest.mark.parametrize("normalized", [False, True])
def test_f64_values_and_gradients(kernel, normalized):
    n = 777
    xyz = inputs.normal_points(n, seed=101)
    for l_max in (0, 1, 2, 3, 5, 8, 12, 16):
        v, g = _run(xyz, l_max, normalized, True, kernel, dtype=torch.float64)
        rv, rg = oracle.spherical_harmonics_grad(xyz, l_max, normalized)
        assert_values(v, xyz, l_max, normalized, F64_TOL, ref=rv)
        assert_grads(g, xyz, l_max, normalized, F64_TOL, ref=rg)


def test_values_only_matches_values_with_gradients():
    xyz = inputs.normal_points(3001, seed=102).astype(np.float32)
    for kernel in ("point", "slice"):
        for l_max in (3, 8, 13):
            v0 = _run(xyz, l_max, False, False, kernel)
            v1, _ = _run(xyz, l_max, False, True, kernel)
            np.testing.assert_array_equal(v0, v1)


# --------------------------------------------------------------- workloads
def test_workload_small_f64_n10000():
    """N = 10,000 i.i.d. normal FP64 points (seed 0), l_max = 8, values,
    normalized and scaled, every point checked."""
    xyz = inputs.normal_points(10_000, seed=0)
    for normalized in (False, True):
        for kernel in ("point", "slice"):
            v = _run(xyz, 8, normalized, False, kernel, dtype=torch.float64)
            assert_values(v, xyz, 8, normalized, F64_TOL)


@pytest.mark.parametrize("out_dtype", [None, torch.bfloat16])
def test_workload_f32_n1m_lmax10_full(out_dtype):
    """N = 1,000,000 FP32 points, uniform directions, r ~ U[0.5, 5], l_max = 10,
    values + gradients (FP32 and bf16 store): every point against the oracle."""
    n, l_max = 1_000_000, 10
    xyz = inputs.shell_points(n, 0.5, 5.0, seed=2)
    v, g = _run(xyz, l_max, False, True, out_dtype=out_dtype)
    tol_v, tol_g = (F32_VAL, F32_GRAD) if out_dtype is None else (BF16_TOL, BF16_TOL)
    ev, eg, finite = full_parity.forward_errors(xyz.astype(np.float64), l_max, False, v, g)
    assert finite
    assert np.all(ev <= value_bound(l_max, tol_v)), ev
    assert np.all(eg <= tol_g), eg


def test_headline_lmax8_n4m_full():
    """l_max = 8, N = 4,194,304 FP32 (the benchmark workload, in the launch
    shape the benchmark times: the autotuner's pick): every point against the oracle."""
    n, l_max = 4_194_304, 8
    xyz = inputs.shell_points(n, 0.5, 5.0, seed=8)
    x = torch.from_numpy(xyz).to(DEV)
    api.autotune(x, l_max, False, True)  # installs the shape later calls use
    try:
        sph, dsph = api.spherical_harmonics(x, l_max, gradients=True)
        torch.cuda.synchronize()
    finally:
        C.sphericart_tune_clear()  # process-wide: later tests see the defaults
    ev, eg, finite = full_parity.forward_errors(xyz.astype(np.float64), l_max, False,
                                                sph.cpu().numpy(), dsph.cpu().numpy())
    assert finite
    assert np.all(ev <= value_bound(l_max, F32_VAL)), ev
    assert np.all(eg <= F32_GRAD), eg


# --------------------------------------------------------------- edge cases
def test_edge_points():
    pts = np.array(
        [
            [0.0, 0.0, 0.0],
            [0.0, 0.0, 1.0],
            [0.0, 0.0, -2.0],
            [1e-20, 0.0, 1.0],
            [3.0, 0.0, 0.0],
            [0.0, -4.0, 0.0],
            [1e-6, 2e-6, -3e-6],
            [1e3, -2e3, 5e2],
        ]
    )
    for kernel in ("point", "slice"):
        for normalized in (False, True):
            for l_max in (0, 1, 4, 8):
                v, g = _run(pts, l_max, normalized, True, kernel, dtype=torch.float64)
                rv, rg = oracle.spherical_harmonics_grad(pts, l_max, normalized)
                assert np.all(np.isfinite(v)) and np.all(np.isfinite(g))
                assert_values(v, pts, l_max, normalized, F64_TOL, ref=rv)
                assert_grads(g, pts, l_max, normalized, F64_TOL, ref=rg)


def test_empty_and_tiny():
    for n in (0, 1, 2, 3, 5, 31, 33):
        xyz = inputs.normal_points(n, seed=103).astype(np.float32)
        for kernel in ("point", "slice"):
            v, g = _run(xyz, 6, False, True, kernel)
            assert v.shape == (n, 49) and g.shape == (n, 3, 49)
            if n:
                assert_values(v, xyz.astype(np.float64), 6, False, F32_VAL)


@pytest.mark.parametrize("l_max", [7, 8])
def test_launch_shapes_and_persistent_loop(l_max):
    """Several tiles per warp (one CTA per SM), every tile size, ragged tail;
    l_max = 7 takes the padded-row path, l_max = 8 the bulk-copy path."""
    n = 20_011
    xyz = inputs.normal_points(n, seed=104).astype(np.float32)
    ref = oracle.spherical_harmonics_grad(xyz.astype(np.float64), l_max, False)
    base = None
    for P in (4, 8, 12, 16, 20, 24, 28, 32):
        for W in (1, 2, 4):
            lau = C.make_launch(P, W, 1, 0)
            v, g = _run(xyz, l_max, False, True, "point", launch=lau)
            if base is None:
                base = (v, g)
                assert_values(v, xyz.astype(np.float64), l_max, False, F32_VAL, ref=ref[0])
                assert_grads(g, xyz.astype(np.float64), l_max, False, F32_GRAD, ref=ref[1])
            else:
                np.testing.assert_array_equal(v, base[0])
                np.testing.assert_array_equal(g, base[1])


def test_unaligned_outputs_take_plain_stores():
    n, l_max = 2049, 6
    xyz = torch.from_numpy(inputs.normal_points(n, seed=105).astype(np.float32)).to(DEV)
    K = (l_max + 1) ** 2
    buf = torch.full((n * K + 1,), float("nan"), device=DEV)
    dbuf = torch.full((n * 3 * K + 1,), float("nan"), device=DEV)
    sph = buf[1:].view(n, K)
    dsph = dbuf[1:].view(n, 3, K)
    assert sph.data_ptr() % 16 != 0
    api.spherical_harmonics(xyz, l_max, False, gradients=True, kernel="point", out=(sph, dsph))
    ref_v, ref_g = api.spherical_harmonics(xyz, l_max, False, gradients=True, kernel="point")
    torch.cuda.synchronize()
    assert torch.equal(sph, ref_v) and torch.equal(dsph, ref_g)
    assert torch.isnan(buf[0]) and torch.isnan(dbuf[0])


def test_outputs_do_not_overrun():
    """Canary elements after the outputs stay untouched."""
    n, l_max = 1001, 8
    K = (l_max + 1) ** 2
    xyz = torch.from_numpy(inputs.normal_points(n, seed=106).astype(np.float32)).to(DEV)
    for kernel in ("point", "slice"):
        buf = torch.full((n * K + 64,), -7.0, device=DEV)
        dbuf = torch.full((n * 3 * K + 64,), -7.0, device=DEV)
        api.spherical_harmonics(
            xyz, l_max, gradients=True, kernel=kernel, out=(buf[: n * K].view(n, K), dbuf[: 3 * n * K].view(n, 3, K))
        )
        torch.cuda.synchronize()
        assert torch.all(buf[n * K:] == -7.0) and torch.all(dbuf[3 * n * K:] == -7.0)


# --------------------------------------------------------------- large l_max, precision
@pytest.mark.parametrize("kernel", ["auto", "slice"])
@pytest.mark.parametrize("l_max", [17, 20, 31, 33])
def test_slice_large_lmax_f32(l_max, kernel):
    xyz = inputs.shell_points(500, 0.7, 1.3, seed=107).astype(np.float64)
    x32 = xyz.astype(np.float32).astype(np.float64)
    v, g = _run(x32, l_max, False, True, kernel)
    rv, rg = oracle.spherical_harmonics_grad(x32, l_max, False)
    ev = value_errors(v, rv, x32, l_max, False)
    eg = grad_errors(g, rg, x32, l_max, False)
    if l_max <= 20:
        assert np.all(ev <= F32_VAL * np.sqrt(2 * np.arange(l_max + 1) + 1))
        assert np.all(eg <= F32_GRAD)
    else:  # reported, bounded loosely: FP32 accumulates over l
        assert np.all(ev <= 1e-4) and np.all(eg <= 1e-3)


@pytest.mark.parametrize("l_max", [20, 30, 50])
def test_pole_mix_f64_and_mixed(l_max):
    """Half uniform on the sphere, half within 1e-4 rad of the poles."""
    xyz = inputs.pole_mix_points(400, seed=108)
    rv, rg = oracle.spherical_harmonics_grad(xyz, l_max, True)
    v, g = _run(xyz, l_max, True, True, "slice", dtype=torch.float64)
    assert_values(v, xyz, l_max, True, F64_TOL, ref=rv)
    assert_grads(g, xyz, l_max, True, F64_TOL, ref=rg)
    x32 = xyz.astype(np.float32).astype(np.float64)
    rv32, rg32 = oracle.spherical_harmonics_grad(x32, l_max, True)
    for qprec in ("native", "f64"):
        v, g = _run(x32, l_max, True, True, "slice", qprec=qprec)
        ev = value_errors(v, rv32, x32, l_max, True)
        eg = grad_errors(g, rg32, x32, l_max, True)
        assert np.all(np.isfinite(v)) and np.all(np.isfinite(g))
        assert np.max(ev) < 1e-4 and np.max(eg) < 1e-3, (qprec, ev, eg)
