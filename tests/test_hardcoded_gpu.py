"""POINT_HC: degrees l <= 3 from the generated straight-line expressions, the
recursion above them (the paper's GPU kernel design, Section 3.2), against the
FP64 oracle and against the all-recursion POINT kernel."""

import numpy as np
import pytest
import torch

import oracle
from paper_2302_08381_gb300 import _capi as C
from paper_2302_08381_gb300 import api, inputs
from parity_utils import F32_GRAD, F32_VAL, F64_TOL, assert_grads, assert_values

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _pts(tiny=True):
    """Shell points, both poles' neighbourhoods, the z axis, the origin and
    (FP64 only: r^l underflows FP32 there) a point of radius ~4e-7."""
    extra = [[0.0, 0.0, 0.0], [0.0, 0.0, 2.0], [0.0, 0.0, -1.0]] + ([[1e-7, -2e-7, 3e-7]] if tiny else [])
    return np.concatenate([
        inputs.shell_points(2000, 0.5, 3.0, seed=960).astype(np.float64),
        inputs.pole_mix_points(200, seed=961),
        np.array(extra),
    ])


@pytest.mark.parametrize("normalized", [False, True])
def test_point_hc_fp64_against_oracle(normalized):
    x = _pts()
    xt = torch.from_numpy(x).to(DEV)
    for l_max in range(0, 9):
        rv, rg = oracle.spherical_harmonics_grad(x, l_max, normalized)
        v, g = api.spherical_harmonics(xt, l_max, normalized, gradients=True, kernel="point_hc")
        torch.cuda.synchronize()
        assert_values(v.cpu().numpy(), x, l_max, normalized, F64_TOL, ref=rv)
        assert_grads(g.cpu().numpy(), x, l_max, normalized, F64_TOL, ref=rg)
        # values only: the same polynomials, CSE'd on their own
        v0 = api.spherical_harmonics(xt, l_max, normalized, kernel="point_hc")
        assert_values(v0.cpu().numpy(), x, l_max, normalized, F64_TOL, ref=rv)


@pytest.mark.parametrize("normalized", [False, True])
def test_point_hc_fp32_against_oracle_and_point(normalized):
    x = _pts(tiny=False).astype(np.float32).astype(np.float64)
    xt = torch.from_numpy(x).to(DEV, torch.float32)
    for l_max in range(0, 9):
        rv, rg = oracle.spherical_harmonics_grad(x, l_max, normalized)
        v, g = api.spherical_harmonics(xt, l_max, normalized, gradients=True, kernel="point_hc")
        v1, g1 = api.spherical_harmonics(xt, l_max, normalized, gradients=True, kernel="point")
        torch.cuda.synchronize()
        assert_values(v.double().cpu().numpy(), x, l_max, normalized, F32_VAL, ref=rv)
        assert_grads(g.double().cpu().numpy(), x, l_max, normalized, F32_GRAD, ref=rg)
        # same polynomials, other operation order: a few FP32 roundings apart
        assert_values(v.double().cpu().numpy(), x, l_max, normalized, F32_VAL, ref=v1.double().cpu().numpy())


def test_point_hc_full_workload_fp64_n10000():
    """N = 10,000 i.i.d. normal FP64 points (seed 0), l_max = 8, values,
    normalized and scaled: every point."""
    x = inputs.normal_points(10_000, seed=0)
    xt = torch.from_numpy(x).to(DEV)
    for normalized in (False, True):
        v = api.spherical_harmonics(xt, 8, normalized, kernel="point_hc")
        torch.cuda.synchronize()
        assert_values(v.cpu().numpy(), x, 8, normalized, F64_TOL)


def test_point_hc_limits():
    x = torch.zeros((4, 3), device=DEV)
    with pytest.raises(C.SphericartError):
        api.spherical_harmonics(x, 9, kernel="point_hc")
    with pytest.raises(C.SphericartError):
        api.spherical_harmonics(x, 4, gradients=True, hessians=True, kernel="point_hc")
    with pytest.raises(C.SphericartError):
        api.spherical_harmonics(x, 4, out_dtype=torch.bfloat16, kernel="point_hc")
    with pytest.raises(C.SphericartError):
        api.backward(x, torch.zeros((4, 25), device=DEV), 4, kernel="point_hc")
    assert C.lib().sphericart_max_l(C.SPH_F64, C.SPH_Q_NATIVE, C.SPH_KERNEL_POINT_HC) == 8
