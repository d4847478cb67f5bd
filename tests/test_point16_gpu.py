"""POINT Hessians with 16 lanes per point (lanes_per_point = 16: one lane per
output plane, FP32) against the FP64 oracle's analytic Hessians, through the
C-ABI: every l_max, scaled and normalized, pole neighbourhoods, ragged tails,
launch shapes and limits."""

import numpy as np
import pytest
import torch

import oracle
from paper_2302_08381_gb300 import _capi as C
from paper_2302_08381_gb300 import api, inputs
from parity_utils import F32_GRAD, F32_VAL, assert_grads, assert_values, hess_errors

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
F32_HESS = 5e-5  # per l block of the Hessian scale, as for the one-lane kernel


def _t(x, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype)


def _sixteen(P=4, W=0, B=0):
    return C.make_launch(P, W, B, 16)


@pytest.mark.parametrize("normalized", [False, True])
def test_every_lmax_against_oracle(normalized):
    x = np.concatenate([inputs.shell_points(500 + 9, 0.7, 2.0, seed=330).astype(np.float64),
                        inputs.pole_mix_points(40, seed=331) * 1.3]).astype(np.float32).astype(np.float64)
    for l_max in range(0, 17):
        v, g, H = api.spherical_harmonics(_t(x), l_max, normalized, gradients=True, hessians=True, kernel="point",
                                          launch=_sixteen())
        rv, rg = oracle.spherical_harmonics_grad(x, l_max, normalized)
        assert_values(v.double().cpu().numpy(), x, l_max, normalized, F32_VAL, ref=rv)
        assert_grads(g.double().cpu().numpy(), x, l_max, normalized, F32_GRAD, ref=rg)
        rh = oracle.spherical_harmonics_hessian(x, l_max, normalized)
        e = hess_errors(H.double().cpu().numpy(), rh, x, l_max, normalized)
        assert np.all(e <= F32_HESS), (l_max, e)


def test_matches_one_lane_kernel():
    x = _t(inputs.shell_points(3001, 0.5, 3.0, seed=332))
    for l_max in (3, 8, 11, 16):
        for normalized in (False, True):
            a = api.spherical_harmonics(x, l_max, normalized, gradients=True, hessians=True, kernel="point",
                                        launch=C.make_launch(4, 1, 0, 1))
            b = api.spherical_harmonics(x, l_max, normalized, gradients=True, hessians=True, kernel="point",
                                        launch=_sixteen())
            for u, w in zip(a, b):
                tol = 2e-6 * max(1.0, u.abs().max().item())
                assert (u - w).abs().max().item() <= tol, (l_max, normalized)
            Hb = b[2]
            assert torch.equal(Hb, Hb.transpose(1, 2)), (l_max, normalized)  # symmetric planes written


@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 9])
def test_edge_sizes_and_bounds(n):
    for l_max in (0, 6, 8, 9):
        K = (l_max + 1) ** 2
        x = inputs.normal_points(max(n, 1), seed=333)[:n].astype(np.float32)
        big = [torch.full((n + 2, K), 7.0, device=DEV), torch.full((n + 2, 3, K), 7.0, device=DEV),
               torch.full((n + 2, 3, 3, K), 7.0, device=DEV)]
        out = [t[1:n + 1] for t in big]
        api.spherical_harmonics(_t(x), l_max, False, gradients=True, hessians=True, kernel="point",
                                launch=_sixteen(), out=out)
        torch.cuda.synchronize()
        for t in big:
            assert bool((t[0] == 7.0).all()) and bool((t[-1] == 7.0).all()), (n, l_max)
        if n:
            x64 = x.astype(np.float64)
            e = hess_errors(out[2].double().cpu().numpy(), oracle.spherical_harmonics_hessian(x64, l_max), x64,
                            l_max, False)
            assert np.all(e <= F32_HESS), (n, l_max, e)


def test_launch_shapes_and_limits():
    x = _t(inputs.normal_points(2051, seed=334))
    ref = api.spherical_harmonics(x, 9, False, gradients=True, hessians=True, kernel="point", launch=_sixteen())
    for P, W, B in ((2, 1, 0), (4, 2, 16), (6, 3, 0), (8, 4, 1), (4, 1, 32)):
        out = api.spherical_harmonics(x, 9, False, gradients=True, hessians=True, kernel="point",
                                      launch=_sixteen(P, W, B))
        assert all(torch.equal(u, w) for u, w in zip(ref, out)), (P, W, B)
    for lau in (_sixteen(3, 1, 0), _sixteen(10, 1, 0), _sixteen(4, 5, 0), _sixteen(2, 1, 0)):
        L = 8 if lau.points_per_tile == 2 else 9  # a 2-point tile of odd K is not 16-byte aligned
        with pytest.raises(C.SphericartError):
            api.spherical_harmonics(x, L, False, gradients=True, hessians=True, kernel="point", launch=lau)
    with pytest.raises(C.SphericartError):  # no Hessians
        api.spherical_harmonics(x, 9, False, gradients=True, kernel="point", launch=_sixteen())
    with pytest.raises(C.SphericartError):  # FP64 arithmetic
        api.spherical_harmonics(x.double(), 9, False, gradients=True, hessians=True, kernel="point",
                                launch=_sixteen())
