"""POINT with 4 lanes per point (lanes_per_point = 4: one lane per output
plane) against the FP64 oracle, through the C-ABI: every l_max, scaled and
normalized, bf16 storage, ragged tails, launch shapes, the AUTO default and a
full-size workload checked at every point."""

import numpy as np
import pytest
import torch

import full_parity
import oracle
from paper_2302_08381_gb300 import _capi as C
from paper_2302_08381_gb300 import api, inputs
from parity_utils import BF16_TOL, F32_GRAD, F32_VAL, assert_grads, assert_values

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(x, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype)


def _host(t):
    return (t.float() if t.dtype == torch.bfloat16 else t).double().cpu().numpy()


def _four(P=8, W=1, B=0):
    return C.make_launch(P, W, B, 4)


@pytest.mark.parametrize("normalized", [False, True])
def test_every_lmax_against_oracle(normalized):
    n = 1000 + 13  # 126 full 8-point tiles and a ragged tail of 5
    x = inputs.shell_points(n, 0.5, 2.0, seed=320).astype(np.float32).astype(np.float64)
    for l_max in range(0, 17):
        for P in (8, 4):
            v, g = api.spherical_harmonics(_t(x), l_max, normalized, gradients=True, kernel="point",
                                           launch=_four(P))
            rv, rg = oracle.spherical_harmonics_grad(x, l_max, normalized)
            assert_values(_host(v), x, l_max, normalized, F32_VAL, ref=rv)
            assert_grads(_host(g), x, l_max, normalized, F32_GRAD, ref=rg)


def test_matches_one_lane_point():
    """Same recursion, the planes assembled per lane: results agree with the
    one-lane POINT kernel to rounding."""
    x = _t(inputs.shell_points(5000 + 3, 0.5, 3.0, seed=321))
    for l_max in (5, 10, 12, 15, 16):
        for normalized in (False, True):
            a = api.spherical_harmonics(x, l_max, normalized, gradients=True, kernel="point",
                                        launch=C.make_launch(4, 1, 0, 1))
            b = api.spherical_harmonics(x, l_max, normalized, gradients=True, kernel="point", launch=_four())
            for u, w in zip(a, b):
                tol = 2e-6 * max(1.0, u.abs().max().item())
                assert (u - w).abs().max().item() <= tol, (l_max, normalized)


def test_bf16_storage_against_oracle():
    x = inputs.shell_points(2000 + 7, 0.5, 2.0, seed=322).astype(np.float32).astype(np.float64)
    for l_max in (4, 9, 11, 12, 13, 15, 16):
        v, g = api.spherical_harmonics(_t(x), l_max, True, gradients=True, kernel="point", launch=_four(),
                                       out_dtype=torch.bfloat16)
        rv, rg = oracle.spherical_harmonics_grad(x, l_max, True)
        assert_values(_host(v), x, l_max, True, BF16_TOL, ref=rv)
        assert_grads(_host(g), x, l_max, True, BF16_TOL, ref=rg)


@pytest.mark.parametrize("n", [0, 1, 7, 8, 9, 33])
def test_edge_sizes(n):
    x = inputs.normal_points(max(n, 1), seed=323)[:n].astype(np.float32)
    for l_max in (0, 7, 12, 15):
        K = (l_max + 1) ** 2
        v = torch.full((n, K), 7.0, device=DEV)
        g = torch.full((n, 3, K), 7.0, device=DEV)
        api.spherical_harmonics(_t(x), l_max, False, gradients=True, kernel="point", launch=_four(), out=(v, g))
        if n:
            x64 = x.astype(np.float64)
            rv, rg = oracle.spherical_harmonics_grad(x64, l_max, False)
            assert_values(_host(v), x64, l_max, False, F32_VAL, ref=rv)
            assert_grads(_host(g), x64, l_max, False, F32_GRAD, ref=rg)


def test_output_buffers_bounded():
    """Writes stay inside [n, K] / [n, 3, K] (odd and even K): guard rows
    around the outputs keep their sentinel."""
    n = 77
    for l_max, odt in ((11, torch.float32), (12, torch.float32), (13, torch.float32), (15, torch.float32),
                       (11, torch.bfloat16), (13, torch.bfloat16)):
        K = (l_max + 1) ** 2
        big_v = torch.full((n + 2, K), 7.0, device=DEV, dtype=odt)
        big_g = torch.full((n + 2, 3, K), 7.0, device=DEV, dtype=odt)
        v, g = big_v[1:n + 1], big_g[1:n + 1]
        api.spherical_harmonics(_t(inputs.normal_points(n, seed=324)), l_max, True, gradients=True,
                                kernel="point", launch=_four(), out=(v, g), out_dtype=odt)
        torch.cuda.synchronize()
        for t in (big_v[0], big_v[-1], big_g[0], big_g[-1]):
            assert bool((t == 7.0).all()), (l_max, odt)
        assert bool(torch.isfinite(v.float()).all()) and not bool((g == 7.0).all(dim=2).any()), (l_max, odt)


def test_launch_shapes_and_limits():
    x = _t(inputs.normal_points(4099, seed=325))
    ref = api.spherical_harmonics(x, 14, False, gradients=True, kernel="point", launch=_four())
    for P, W, B in ((8, 2, 0), (8, 4, 1), (8, 8, 0), (4, 3, 16), (8, 1, 32)):
        out = api.spherical_harmonics(x, 14, False, gradients=True, kernel="point", launch=_four(P, W, B))
        assert all(torch.equal(u, w) for u, w in zip(ref, out)), (P, W, B)
    bad = [C.make_launch(12, 1, 0, 4), C.make_launch(8, 1, 0, 3), C.make_launch(8, 9, 0, 4)]
    for lau in bad:
        with pytest.raises(C.SphericartError):
            api.spherical_harmonics(x, 14, False, gradients=True, kernel="point", launch=lau)
    with pytest.raises(C.SphericartError):  # values only
        api.spherical_harmonics(x, 14, False, kernel="point", launch=_four())
    with pytest.raises(C.SphericartError):  # Hessians
        api.spherical_harmonics(x, 8, False, gradients=True, hessians=True, kernel="point", launch=_four())
    with pytest.raises(C.SphericartError):  # FP64 arithmetic
        api.spherical_harmonics(x.double(), 8, False, gradients=True, kernel="point", launch=_four())


def test_auto_default_runs_four_lanes():
    """AUTO with FP32 gradients from l_max 10 runs 4 lanes per point (no tuned
    shape installed for these keys in this process)."""
    fam, s = C.sphericart_launch_info(12, C.SPH_F32, C.SPH_OUT_SAME, 1, 0)
    assert fam == C.SPH_KERNEL_POINT and s.lanes_per_point == 4 and s.points_per_tile == 8
    fam, s = C.sphericart_launch_info(8, C.SPH_F32, C.SPH_OUT_SAME, 1, 0)
    assert s.lanes_per_point == 0
    x = _t(inputs.shell_points(3000, 0.5, 2.0, seed=326))
    a = api.spherical_harmonics(x, 12, False, gradients=True)
    b = api.spherical_harmonics(x, 12, False, gradients=True, kernel="point", launch=_four())
    assert all(torch.equal(u, w) for u, w in zip(a, b))


def test_full_size_lmax16_every_point():
    """200,000 points (pole mix), l_max 16, normalized, FP32 values and
    gradients on 4 lanes per point: every element against the oracle."""
    n, l_max = 200_000, 16
    x = inputs.pole_mix_points(n, seed=327).astype(np.float32)
    v, g = api.spherical_harmonics(_t(x), l_max, True, gradients=True, kernel="point", launch=_four())
    ev, eg, finite = full_parity.forward_errors(x.astype(np.float64), l_max, True, _host(v), _host(g))
    assert finite
    lv = np.arange(l_max + 1)
    assert np.all(ev <= 4e-6 * (lv + 1)), ev
    assert np.all(eg <= 1e-5 * (lv + 1)), eg
