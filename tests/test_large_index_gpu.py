"""Outputs and inputs beyond 2^31 elements (64-bit element offsets in every
kernel family's addressing): each case computes a full-size launch whose
largest array holds more than 2,147,483,648 elements, then checks sampled
points at the start, in the middle and at the end against the FP64 oracle."""

import numpy as np
import pytest
import torch

import oracle
from paper_2302_08381_gb300 import api, inputs
from parity_utils import F32_GRAD, F32_VAL, assert_grads, assert_values, hess_errors

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
F32_HESS = 5e-5
BIG = 2**31


def _sample(n, k=192):
    """Point indices at the start, around n/2 and at the end."""
    return np.concatenate([np.arange(k), n // 2 + np.arange(k), n - k + np.arange(k)])


def _points(n, seed):
    return inputs.shell_points(n, 0.5, 5.0, seed=seed)  # FP32


def test_point_forward_gradients_l8():
    """POINT (AUTO), FP32 values + gradients, l_max 8: dsph has 2.19e9
    elements."""
    n, l_max = 9_000_000, 8
    K = (l_max + 1) ** 2
    assert 3 * n * K > BIG
    x = _points(n, 600)
    sph, dsph = api.spherical_harmonics(torch.from_numpy(x).to(DEV), l_max, gradients=True)
    idx = _sample(n)
    ti = torch.from_numpy(idx).to(DEV)
    v, g = sph[ti].double().cpu().numpy(), dsph[ti].double().cpu().numpy()
    del sph, dsph
    xs = x[idx].astype(np.float64)
    rv, rg = oracle.spherical_harmonics_grad(xs, l_max, False)
    assert_values(v, xs, l_max, False, F32_VAL, ref=rv)
    assert_grads(g, xs, l_max, False, F32_GRAD, ref=rg)


def test_point4_forward_gradients_l12():
    """POINT with 4 lanes per point (AUTO for FP32 gradients from l_max 10),
    l_max 12: dsph has 2.28e9 elements."""
    n, l_max = 4_500_000, 12
    K = (l_max + 1) ** 2
    assert 3 * n * K > BIG
    x = _points(n, 605)
    sph, dsph = api.spherical_harmonics(torch.from_numpy(x).to(DEV), l_max, gradients=True)
    idx = _sample(n)
    ti = torch.from_numpy(idx).to(DEV)
    v, g = sph[ti].double().cpu().numpy(), dsph[ti].double().cpu().numpy()
    del sph, dsph
    xs = x[idx].astype(np.float64)
    rv, rg = oracle.spherical_harmonics_grad(xs, l_max, False)
    assert_values(v, xs, l_max, False, F32_VAL, ref=rv)
    assert_grads(g, xs, l_max, False, F32_GRAD, ref=rg)


def test_point10_hessians_l8():
    """POINT with 10 lanes per point (AUTO for FP32 Hessians), l_max 8: ddsph
    has 2.19e9 elements."""
    n, l_max = 3_000_000, 8
    K = (l_max + 1) ** 2
    assert 9 * n * K > BIG
    x = _points(n, 601)
    sph, dsph, ddsph = api.spherical_harmonics(torch.from_numpy(x).to(DEV), l_max, gradients=True, hessians=True)
    idx = _sample(n)
    ti = torch.from_numpy(idx).to(DEV)
    v, g, H = (t[ti].double().cpu().numpy() for t in (sph, dsph, ddsph))
    del sph, dsph, ddsph
    xs = x[idx].astype(np.float64)
    rv, rg = oracle.spherical_harmonics_grad(xs, l_max, False)
    assert_values(v, xs, l_max, False, F32_VAL, ref=rv)
    assert_grads(g, xs, l_max, False, F32_GRAD, ref=rg)
    e = hess_errors(H, oracle.spherical_harmonics_hessian(xs, l_max, False), xs, l_max, False)
    assert np.all(e <= F32_HESS), e


def test_row_forward_gradients_l20_normalized():
    """ROW (AUTO above POINT's range), FP32 values + gradients, l_max 20,
    normalized: dsph has 2.25e9 elements."""
    n, l_max = 1_700_000, 20
    K = (l_max + 1) ** 2
    assert 3 * n * K > BIG
    x = _points(n, 602)
    sph, dsph = api.spherical_harmonics(torch.from_numpy(x).to(DEV), l_max, True, gradients=True)
    idx = _sample(n)
    ti = torch.from_numpy(idx).to(DEV)
    v, g = sph[ti].double().cpu().numpy(), dsph[ti].double().cpu().numpy()
    del sph, dsph
    xs = x[idx].astype(np.float64)
    rv, rg = oracle.spherical_harmonics_grad(xs, l_max, True)
    assert_values(v, xs, l_max, True, F32_VAL, ref=rv)
    assert_grads(g, xs, l_max, True, F32_GRAD, ref=rg)


def test_row_backward_l20():
    """Fused recompute-backward (AUTO: ROW), l_max 20: the upstream gradient
    g has 2.2e9 elements (filled from one seeded block, repeated)."""
    n, l_max = 5_000_000, 20
    K = (l_max + 1) ** 2
    assert n * K > BIG
    x = _points(n, 603)
    block = inputs.upstream(65_536, K, seed=604)
    g = torch.empty((n, K), dtype=torch.float32, device=DEV)
    gb = torch.from_numpy(block).to(DEV)
    for s in range(0, n, block.shape[0]):
        e = min(n, s + block.shape[0])
        g[s:e] = gb[: e - s]
    dx = api.backward(torch.from_numpy(x).to(DEV), g, l_max)
    idx = _sample(n)
    got = dx[torch.from_numpy(idx).to(DEV)].double().cpu().numpy()
    del g, dx
    xs = x[idx].astype(np.float64)
    ref = oracle.backward(xs, block[idx % block.shape[0]].astype(np.float64), l_max, False)
    err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
    assert err < 2e-5, err
