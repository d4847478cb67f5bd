"""ROW Hessians (FP32 values, gradients and Hessians for 0 <= l_max <= 63 on
the 8-lanes-per-point ROW decomposition) against the FP64 oracle's analytic
Hessians, through the C-ABI: scaled and normalized, pole neighbourhoods,
both window capacities, ragged tails and output bounds."""

import numpy as np
import pytest
import torch

import oracle
from paper_2302_08381_gb300 import _capi as C
from paper_2302_08381_gb300 import api, inputs
from parity_utils import grad_errors, hess_errors, value_errors

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(x, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV, dtype)


def _run(x, l_max, normalized, cap=0, W=0):
    return api.spherical_harmonics(_t(x), l_max, normalized, gradients=True, hessians=True, kernel="row",
                                   launch=C.make_launch(0, W, 0, cap))


@pytest.mark.parametrize("normalized", [False, True])
def test_against_oracle(normalized):
    """Per l block, max error relative to the block's scale (values,
    gradients, Hessians) within 5e-6 (l + 1) in FP32 (FP32 rounding grows
    about linearly in l: ~2.2e-6 per degree at l_max 63, as on the other FP32
    paths), at the FP32-rounded coordinates; shell points and points
    1e-9..1e-4 rad from the poles."""
    x = np.concatenate([inputs.shell_points(90 + 3, 0.7, 2.0, seed=340).astype(np.float64),
                        inputs.pole_mix_points(30, seed=341) * 1.2]).astype(np.float32).astype(np.float64)
    for l_max in (0, 1, 2, 5, 7, 8, 12, 15, 16, 17, 20, 23, 31, 32, 40, 47, 48, 55, 63):
        v, g, H = _run(x, l_max, normalized)
        lv = np.arange(l_max + 1)
        rv, rg = oracle.spherical_harmonics_grad(x, l_max, normalized)
        rh = oracle.spherical_harmonics_hessian(x, l_max, normalized)
        ev = value_errors(v.double().cpu().numpy(), rv, x, l_max, normalized)
        eg = grad_errors(g.double().cpu().numpy(), rg, x, l_max, normalized)
        eh = hess_errors(H.double().cpu().numpy(), rh, x, l_max, normalized)
        assert np.all(ev <= 5e-6 * (lv + 1)), (l_max, ev)
        assert np.all(eg <= 5e-6 * (lv + 1)), (l_max, eg)
        assert np.all(eh <= 5e-6 * (lv + 1)), (l_max, eh)
        Hn = H.cpu().numpy()
        assert np.array_equal(Hn, Hn.transpose(0, 2, 1, 3)), l_max


def test_window_capacities_and_shapes_agree():
    x = _t(inputs.shell_points(1003, 0.5, 3.0, seed=342))
    for l_max in (20, 41, 63):
        ref = api.spherical_harmonics(x, l_max, True, gradients=True, hessians=True, kernel="row")
        for cap, W in ((2, 1), (0, 2), (3, 2), (1, 1), (3, 1)):
            out = api.spherical_harmonics(x, l_max, True, gradients=True, hessians=True, kernel="row",
                                          launch=C.make_launch(0, W, 0, cap))
            assert all(torch.equal(u, w) for u, w in zip(ref, out)), (l_max, cap, W)


def test_matches_slice():
    """Same Eq. iter-deri terms as SLICE: results agree to FP32 rounding."""
    x = _t(inputs.shell_points(777, 0.5, 3.0, seed=343))
    for l_max, normalized in ((18, False), (30, True), (50, True)):
        a = api.spherical_harmonics(x, l_max, normalized, gradients=True, hessians=True, kernel="slice")
        b = api.spherical_harmonics(x, l_max, normalized, gradients=True, hessians=True, kernel="row")
        for u, w in zip(a, b):
            scale = u.abs().amax(dim=0, keepdim=True).clamp_min(1e-30)
            assert ((u - w).abs() / scale).max().item() <= 2e-5 * l_max, (l_max, normalized)


@pytest.mark.parametrize("n", [0, 1, 5, 9])
def test_edge_sizes_and_bounds(n):
    # l_max 0 and 1: rows shorter than one 32-byte sector (the unaligned head
    # must stay inside the row)
    for l_max in (0, 1, 2, 16, 33):
        if n == 0 and l_max < 16:
            continue  # empty outputs pass NULL: a gradients-only request, which ROW serves from l_max 16
        K = (l_max + 1) ** 2
        x = inputs.normal_points(max(n, 1), seed=344)[:n].astype(np.float32)
        big = [torch.full((n + 2, K), 7.0, device=DEV), torch.full((n + 2, 3, K), 7.0, device=DEV),
               torch.full((n + 2, 3, 3, K), 7.0, device=DEV)]
        out = [t[1:n + 1] for t in big]
        api.spherical_harmonics(_t(x), l_max, False, gradients=True, hessians=True, kernel="row", out=out)
        torch.cuda.synchronize()
        for t in big:
            assert bool((t[0] == 7.0).all()) and bool((t[-1] == 7.0).all()), (n, l_max)
        if n:
            x64 = x.astype(np.float64)
            eh = hess_errors(out[2].double().cpu().numpy(), oracle.spherical_harmonics_hessian(x64, l_max), x64,
                             l_max, False)
            assert np.all(eh <= 5e-6 * (np.arange(l_max + 1) + 1)), (n, l_max, eh)


def test_limits():
    x = _t(inputs.normal_points(64, seed=345))
    with pytest.raises(C.SphericartError):  # bf16 Hessians
        api.spherical_harmonics(x, 20, gradients=True, hessians=True, kernel="row", out_dtype=torch.bfloat16)
    with pytest.raises(C.SphericartError):  # FP64
        api.spherical_harmonics(x.double(), 20, gradients=True, hessians=True, kernel="row")
    with pytest.raises(C.SphericartError):  # gradients without Hessians below l_max 16
        api.spherical_harmonics(x, 12, gradients=True, kernel="row")
    with pytest.raises(C.SphericartError):  # beyond l_max 63
        api.spherical_harmonics(x, 64, gradients=True, hessians=True, kernel="row")
    with pytest.raises(C.SphericartError):  # 3 warps per block
        api.spherical_harmonics(x, 20, gradients=True, hessians=True, kernel="row", launch=C.make_launch(0, 3, 0, 0))


def test_full_size_lmax20_every_point():
    """100,000 points (half within 1e-4 rad of the poles), l_max 20,
    normalized, FP32 Hessians on the AUTO path (ROW): every element of ddsph
    against the oracle, symmetric planes bit for bit."""
    import full_parity

    n, l_max = 100_000, 20
    x = inputs.pole_mix_points(n, seed=346).astype(np.float32)
    _, _, H = api.spherical_harmonics(_t(x), l_max, True, gradients=True, hessians=True)
    eh, finite, sym = full_parity.hessian_errors(x.astype(np.float64), l_max, True, H.cpu().numpy())
    assert finite and sym
    assert np.all(eh <= 5e-6 * (np.arange(l_max + 1) + 1)), eh
