"""Parity of the DEGREE kernel families (one thread per point, degree
outermost; Eq. iter-q upward in l, or Eq. iter-q-alt downward in m) against
the FP64 oracle, through the C-ABI.

Sizes span several 32-point tiles and a ragged tail; l_max covers the
whole-degree stage groups (l <= 15), the chunked degrees (l >= 16, one and
several 16-wide m chunks) and the high-degree sweep.
"""

import numpy as np
import pytest
import torch

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
    value_errors,
)

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
KERNELS = ("degree", "degree_down")


def _run(xyz_np, l_max, normalized, grad, kernel, dtype=torch.float32, out_dtype=None, qprec="native", launch=None):
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


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("normalized", [False, True])
def test_f32_every_lmax_to_20(kernel, normalized):
    n = 1000 + 13
    xyz = inputs.shell_points(n, 0.5, 2.0, seed=300).astype(np.float32).astype(np.float64)
    for l_max in range(0, 21):
        v, g = _run(xyz, l_max, normalized, True, kernel)
        rv, rg = oracle.spherical_harmonics_grad(xyz, l_max, normalized)
        assert_values(v, xyz, l_max, normalized, F32_VAL, ref=rv)
        assert_grads(g, xyz, l_max, normalized, F32_GRAD, ref=rg)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("l_max", [31, 32, 33, 47, 50, 64, 65, 80])
def test_f32_high_degree(kernel, l_max):
    """Several m chunks per degree; FP32 error grows with l (reported, bounded)."""
    xyz = inputs.shell_points(300, 0.7, 1.3, seed=301).astype(np.float32).astype(np.float64)
    for normalized in (False, True):
        v, g = _run(xyz, l_max, normalized, True, kernel)
        rv, rg = oracle.spherical_harmonics_grad(xyz, l_max, normalized)
        ev = value_errors(v, rv, xyz, l_max, normalized)
        eg = grad_errors(g, rg, xyz, l_max, normalized)
        assert np.all(np.isfinite(v)) and np.all(np.isfinite(g))
        assert np.all(ev <= 1e-4) and np.all(eg <= 1e-3), (kernel, l_max, normalized, ev.max(), eg.max())


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("normalized", [False, True])
def test_f64_values_and_gradients(kernel, normalized):
    n = 777
    xyz = inputs.normal_points(n, seed=302)
    for l_max in (0, 1, 2, 3, 5, 8, 12, 16, 17, 25, 40):
        v, g = _run(xyz, l_max, normalized, True, kernel, dtype=torch.float64)
        rv, rg = oracle.spherical_harmonics_grad(xyz, l_max, normalized)
        assert_values(v, xyz, l_max, normalized, F64_TOL, ref=rv)
        assert_grads(g, xyz, l_max, normalized, F64_TOL, ref=rg)


@pytest.mark.parametrize("kernel", KERNELS)
def test_values_only_matches_values_with_gradients(kernel):
    xyz = inputs.normal_points(3001, seed=303).astype(np.float32)
    for l_max in (3, 8, 15, 16, 40):
        for normalized in (False, True):
            v0 = _run(xyz, l_max, normalized, False, kernel)
            v1, _ = _run(xyz, l_max, normalized, True, kernel)
            np.testing.assert_array_equal(v0, v1)


@pytest.mark.parametrize("kernel", KERNELS)
def test_bf16_store_and_mixed_mode(kernel):
    xyz = inputs.pole_mix_points(600, seed=304)
    x32 = xyz.astype(np.float32).astype(np.float64)
    for l_max in (10, 30):
        rv, rg = oracle.spherical_harmonics_grad(x32, l_max, True)
        v, g = _run(x32, l_max, True, True, kernel, out_dtype=torch.bfloat16)
        assert_values(v, x32, l_max, True, BF16_TOL, ref=rv)
        assert_grads(g, x32, l_max, True, BF16_TOL, ref=rg)
        # FP64 arithmetic on FP32 storage: only the final rounding remains
        v, g = _run(x32, l_max, True, True, kernel, qprec="f64")
        ev = value_errors(v, rv, x32, l_max, True)
        eg = grad_errors(g, rg, x32, l_max, True)
        assert ev.max() < 1e-6 and eg.max() < 1e-6, (ev.max(), eg.max())
        v, g = _run(x32, l_max, True, True, kernel, qprec="f64", out_dtype=torch.bfloat16)
        assert_values(v, x32, l_max, True, BF16_TOL, ref=rv)


@pytest.mark.parametrize("kernel", KERNELS)
@pytest.mark.parametrize("l_max", [20, 30, 50])
def test_pole_mix_f64(kernel, l_max):
    """Half uniform on the sphere, half within 1e-4 rad of the poles, FP64."""
    xyz = inputs.pole_mix_points(400, seed=305)
    rv, rg = oracle.spherical_harmonics_grad(xyz, l_max, True)
    v, g = _run(xyz, l_max, True, True, kernel, dtype=torch.float64)
    assert_values(v, xyz, l_max, True, F64_TOL, ref=rv)
    assert_grads(g, xyz, l_max, True, F64_TOL, ref=rg)


@pytest.mark.parametrize("kernel", KERNELS)
def test_edge_points(kernel):
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
    for normalized in (False, True):
        for l_max in (0, 1, 4, 8, 20):
            v, g = _run(pts, l_max, normalized, True, kernel, dtype=torch.float64)
            rv, rg = oracle.spherical_harmonics_grad(pts, l_max, normalized)
            assert np.all(np.isfinite(v)) and np.all(np.isfinite(g))
            assert_values(v, pts, l_max, normalized, F64_TOL, ref=rv)
            assert_grads(g, pts, l_max, normalized, F64_TOL, ref=rg)


@pytest.mark.parametrize("kernel", KERNELS)
def test_empty_tiny_and_canaries(kernel):
    for n in (0, 1, 2, 31, 32, 33, 65):
        xyz = inputs.normal_points(n, seed=306).astype(np.float32)
        v, g = _run(xyz, 18, False, True, kernel)
        assert v.shape == (n, 361) and g.shape == (n, 3, 361)
        if n:
            assert_values(v, xyz.astype(np.float64), 18, False, F32_VAL)
    n, l_max = 1001, 21
    K = (l_max + 1) ** 2
    x = torch.from_numpy(inputs.normal_points(n, seed=307).astype(np.float32)).to(DEV)
    buf = torch.full((n * K + 64,), -7.0, device=DEV)
    dbuf = torch.full((n * 3 * K + 64,), -7.0, device=DEV)
    api.spherical_harmonics(
        x, l_max, gradients=True, kernel=kernel, out=(buf[: n * K].view(n, K), dbuf[: 3 * n * K].view(n, 3, K))
    )
    torch.cuda.synchronize()
    assert torch.all(buf[n * K:] == -7.0) and torch.all(dbuf[3 * n * K:] == -7.0)
    assert not torch.any(buf[: n * K] == -7.0) and not torch.any(dbuf[: 3 * n * K] == -7.0)


@pytest.mark.parametrize("kernel,lpp", [("degree", 1), ("degree", 2), ("degree", 4), ("degree_down", 0)])
def test_launch_shapes_give_identical_results(kernel, lpp):
    """Several tiles per warp (persistent loop) and every warps-per-block, for
    each lanes-per-point split of the upward recursion."""
    n, l_max = 20_011, 24
    xyz = inputs.normal_points(n, seed=308).astype(np.float32)
    base = None
    for W in (1, 2, 3, 4, 8):
        for B in (0, 1):
            v, g = _run(xyz, l_max, False, True, kernel, launch=C.make_launch(0, W, B, lpp))
            if base is None:
                base = (v, g)
                p = xyz[::97].astype(np.float64)
                rv, rg = oracle.spherical_harmonics_grad(p, l_max, False)
                assert_values(v[::97], p, l_max, False, F32_VAL, ref=rv)
                assert_grads(g[::97], p, l_max, False, F32_GRAD, ref=rg)
            else:
                np.testing.assert_array_equal(v, base[0])
                np.testing.assert_array_equal(g, base[1])


@pytest.mark.parametrize("lpp", [1, 2, 4])
def test_lanes_per_point_parity(lpp):
    """The upward kernel with a point split over 1, 2 or 4 lanes (channels
    m = h mod LPP per lane, c_m/s_m stepped by (x+iy)^LPP): FP32 and FP64
    values and gradients vs the oracle, whole-degree groups and m chunks,
    ragged tiles."""
    lau = C.make_launch(0, 0, 0, lpp)
    x64 = inputs.normal_points(1000 + 7, seed=309)
    x32 = x64.astype(np.float32).astype(np.float64)
    for l_max in (0, 1, 2, 3, 7, 15, 16, 20, 33):
        for normalized in (False, True):
            rv, rg = oracle.spherical_harmonics_grad(x32, l_max, normalized)
            v, g = _run(x32, l_max, normalized, True, "degree", launch=lau)
            if l_max <= 20:
                assert_values(v, x32, l_max, normalized, F32_VAL, ref=rv)
                assert_grads(g, x32, l_max, normalized, F32_GRAD, ref=rg)
            else:
                assert value_errors(v, rv, x32, l_max, normalized).max() < 1e-4
                assert grad_errors(g, rg, x32, l_max, normalized).max() < 1e-3
            v0 = _run(x32, l_max, normalized, False, "degree", launch=lau)
            np.testing.assert_array_equal(v0, v)
        rv, rg = oracle.spherical_harmonics_grad(x64, l_max, True)
        v, g = _run(x64, l_max, True, True, "degree", dtype=torch.float64, launch=lau)
        assert_values(v, x64, l_max, True, F64_TOL, ref=rv)
        assert_grads(g, x64, l_max, True, F64_TOL, ref=rg)


@pytest.mark.parametrize("kernel", KERNELS)
def test_sweep_workload_sampled(kernel):
    """The high-degree workload at full size (200,000 points, half near the
    poles, l_max = 20, normalized, FP32): 2,000 sampled points vs the oracle."""
    N, l_max = 200_000, 20
    xyz = inputs.pole_mix_points(N, seed=4).astype(np.float32)
    v, g = _run(xyz, l_max, True, True, kernel)
    rng = np.random.default_rng(45)
    idx = np.concatenate([rng.choice(N // 2, 1000, replace=False), N // 2 + rng.choice(N // 2, 1000, replace=False)])
    p = xyz[idx].astype(np.float64)
    rv, rg = oracle.spherical_harmonics_grad(p, l_max, True)
    assert_values(v[idx], p, l_max, True, F32_VAL, ref=rv)
    assert_grads(g[idx], p, l_max, True, F32_GRAD, ref=rg)
    assert np.all(np.isfinite(v)) and np.all(np.isfinite(g))
