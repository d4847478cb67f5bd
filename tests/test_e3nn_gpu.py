"""sphericart_compute_e3nn: the harmonics in e3nn's convention (Section 3.2
wrappers). e3nn is not installed here, so the convention is pinned by the
properties e3nn documents (l = 1 proportional to (x, y, z) in input order,
m = 0 proportional to P_l(y / r), the three normalizations), and the adapter's
arithmetic against the FP64 oracle evaluated at the permuted point."""

import math

import numpy as np
import pytest
import torch
from numpy.polynomial import legendre as npl

import oracle
from paper_2302_08381_gb300 import api, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _reference(x, l_max, normalize, normalization):
    """The oracle at (x', y', z') = (z, x, y), gradient planes to (d/dx, d/dy, d/dz), scaled per l."""
    xp = x[:, [2, 0, 1]]
    v, g = oracle.spherical_harmonics_grad(xp, l_max, normalize)
    g = g[:, [1, 2, 0], :]
    lv = np.concatenate([np.full(2 * l + 1, l) for l in range(l_max + 1)]).astype(np.float64)
    f = {"integral": np.ones_like(lv), "component": np.full_like(lv, math.sqrt(4 * math.pi)),
         "norm": np.sqrt(4 * math.pi / (2 * lv + 1))}[normalization]
    return v * f, g * f[None, None, :]


@pytest.mark.parametrize("normalization", ["integral", "component", "norm"])
@pytest.mark.parametrize("normalize", [False, True])
def test_e3nn_adapter_against_oracle(normalize, normalization):
    x = np.concatenate([inputs.shell_points(3000, 0.5, 2.0, seed=980).astype(np.float64),
                        inputs.pole_mix_points(200, seed=981)])
    for l_max in (0, 1, 2, 5, 8, 12, 20):
        rv, rg = _reference(x, l_max, normalize, normalization)
        scale = np.max(np.abs(rv), axis=0) + 1.0
        v, g = api.e3nn_spherical_harmonics(torch.from_numpy(x).to(DEV), l_max, normalize, normalization, True)
        torch.cuda.synchronize()
        assert np.max(np.abs(v.cpu().numpy() - rv) / scale) < 1e-12, l_max
        gs = np.max(np.abs(rg), axis=(0, 1)) + 1.0
        assert np.max(np.abs(g.cpu().numpy() - rg) / gs) < 1e-12, l_max
        v32 = api.e3nn_spherical_harmonics(torch.from_numpy(x).to(DEV, torch.float32), l_max, normalize,
                                           normalization)
        x32 = x.astype(np.float32).astype(np.float64)
        rv32, _ = _reference(x32, l_max, normalize, normalization)
        assert np.max(np.abs(v32.double().cpu().numpy() - rv32) / scale) < 2e-5 * math.sqrt(2 * l_max + 1), l_max


def test_e3nn_documented_properties():
    """component normalization: Y_1 = sqrt(3) (x, y, z) / r; Y_l^0 = sqrt(2l+1) P_l(y / r);
    sum_m Y_l^m(u)^2 = 2l + 1 (component), 1 (norm), (2l+1)/(4 pi) (integral)."""
    x = inputs.shell_points(500, 0.5, 2.0, seed=982).astype(np.float64)
    u = x / np.linalg.norm(x, axis=1, keepdims=True)
    xt = torch.from_numpy(x).to(DEV)
    l_max = 10
    comp = api.e3nn_spherical_harmonics(xt, l_max, True, "component").cpu().numpy()
    np.testing.assert_allclose(comp[:, 1:4], math.sqrt(3) * u, rtol=0, atol=1e-13)
    for l in range(l_max + 1):
        e = np.zeros(l + 1)
        e[l] = 1.0
        np.testing.assert_allclose(comp[:, l * l + l], math.sqrt(2 * l + 1) * npl.legval(u[:, 1], e), atol=1e-12)
    for name, want in (("component", lambda l: 2 * l + 1.0), ("norm", lambda l: 1.0),
                       ("integral", lambda l: (2 * l + 1) / (4 * math.pi))):
        y = api.e3nn_spherical_harmonics(xt, l_max, True, name).cpu().numpy()
        for l in range(l_max + 1):
            np.testing.assert_allclose(np.sum(y[:, l * l:(l + 1) ** 2] ** 2, axis=1), want(l), rtol=1e-12)
    # normalize=False is the polynomial form: degree-l homogeneous
    y1 = api.e3nn_spherical_harmonics(xt, l_max, False, "component").cpu().numpy()
    y2 = api.e3nn_spherical_harmonics(2.0 * xt, l_max, False, "component").cpu().numpy()
    lv = np.concatenate([np.full(2 * l + 1, l) for l in range(l_max + 1)])
    np.testing.assert_allclose(y2, y1 * 2.0 ** lv[None, :], rtol=1e-12, atol=1e-12)
