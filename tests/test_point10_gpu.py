"""POINT Hessians with 10 lanes per point (lanes_per_point = 10: one lane per
distinct plane of a point, three points per warp pass, FP32) against the FP64
oracle's analytic Hessians, through the C-ABI: every l_max, scaled and
normalized, pole neighbourhoods, tile starts at every 16-byte phase, ragged
tails, output bounds, launch shapes and limits."""

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


def _ten(P=6, W=0, B=0):
    return C.make_launch(P, W, B, 10)


@pytest.mark.parametrize("normalized", [False, True])
def test_every_lmax_against_oracle(normalized):
    x = np.concatenate([inputs.shell_points(500 + 7, 0.7, 2.0, seed=350).astype(np.float64),
                        inputs.pole_mix_points(40, seed=351) * 1.3]).astype(np.float32).astype(np.float64)
    for l_max in range(0, 17):
        v, g, H = api.spherical_harmonics(_t(x), l_max, normalized, gradients=True, hessians=True, kernel="point",
                                          launch=_ten(W=1 if l_max > 12 else 0))
        rv, rg = oracle.spherical_harmonics_grad(x, l_max, normalized)
        assert_values(v.double().cpu().numpy(), x, l_max, normalized, F32_VAL, ref=rv)
        assert_grads(g.double().cpu().numpy(), x, l_max, normalized, F32_GRAD, ref=rg)
        rh = oracle.spherical_harmonics_hessian(x, l_max, normalized)
        e = hess_errors(H.double().cpu().numpy(), rh, x, l_max, normalized)
        assert np.all(e <= F32_HESS), (l_max, e)
        Hn = H.cpu().numpy()
        assert np.array_equal(Hn, Hn.transpose(0, 2, 1, 3)), l_max  # mirrors written by the owner lane


def test_matches_sixteen_lanes():
    """The same role weights as the 16-lane map: the planes agree to FP32
    rounding (the two kernels' instruction selection may fuse the
    normalization's products differently)."""
    x = _t(inputs.shell_points(3001, 0.5, 3.0, seed=352))
    for l_max in (3, 8, 9, 11):
        for normalized in (False, True):
            a = api.spherical_harmonics(x, l_max, normalized, gradients=True, hessians=True, kernel="point",
                                        launch=C.make_launch(4, 1, 0, 16))
            b = api.spherical_harmonics(x, l_max, normalized, gradients=True, hessians=True, kernel="point",
                                        launch=_ten())
            for u, w in zip(a, b):
                tol = 2e-6 * max(1.0, u.abs().max().item())
                assert (u - w).abs().max().item() <= tol, (l_max, normalized, (u - w).abs().max().item())


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 7, 13])
def test_edge_sizes_phases_and_bounds(n):
    """Outputs that start at each of the four 4-byte offsets within 16 bytes:
    bulk copies need all three arrays 16-byte aligned, so these take the
    warp's plain copy-out (the bulk image at every 16-byte phase of a tile
    start is covered by 3-point tiles of odd K below, checked bit for bit
    against 6-point tiles); guard elements on both sides untouched."""
    for l_max in (0, 1, 2, 3, 8, 9):
        K = (l_max + 1) ** 2
        x = inputs.normal_points(max(n, 1), seed=353)[:n].astype(np.float32)
        ref = None
        if n:
            x64 = x.astype(np.float64)
            ref = oracle.spherical_harmonics_hessian(x64, l_max)
        for off in range(4):
            flat = [torch.full(((n + 2) * m * K + 8,), 7.0, device=DEV) for m in (1, 3, 9)]
            out = [flat[0][off + K:off + K + n * K].view(n, K),
                   flat[1][off + 3 * K:off + 3 * K + 3 * n * K].view(n, 3, K),
                   flat[2][off + 9 * K:off + 9 * K + 9 * n * K].view(n, 3, 3, K)]
            api.spherical_harmonics(_t(x), l_max, False, gradients=True, hessians=True, kernel="point",
                                    launch=_ten(), out=out)
            torch.cuda.synchronize()
            for f, m in zip(flat, (1, 3, 9)):
                assert bool((f[:off + m * K] == 7.0).all()), (n, l_max, off)
                assert bool((f[off + m * K + n * m * K:] == 7.0).all()), (n, l_max, off)
            if n:
                e = hess_errors(out[2].double().cpu().numpy(), ref, x64, l_max, False)
                assert np.all(e <= F32_HESS), (n, l_max, off, e)


def test_launch_shapes_and_limits():
    x = _t(inputs.normal_points(2051, seed=354))
    for L in (8, 9):
        ref = api.spherical_harmonics(x, L, False, gradients=True, hessians=True, kernel="point", launch=_ten())
        for P, W, B in ((3, 1, 0), (6, 2, 16), (9, 3, 0), (12, 3, 1), (3, 4, 32)):
            out = api.spherical_harmonics(x, L, False, gradients=True, hessians=True, kernel="point",
                                          launch=_ten(P, W, B))
            assert all(torch.equal(u, w) for u, w in zip(ref, out)), (L, P, W, B)
    for lau in (_ten(4, 1, 0), _ten(15, 1, 0), _ten(6, 5, 0)):
        with pytest.raises(C.SphericartError):
            api.spherical_harmonics(x, 9, False, gradients=True, hessians=True, kernel="point", launch=lau)
    with pytest.raises(C.SphericartError):  # no Hessians
        api.spherical_harmonics(x, 9, False, gradients=True, kernel="point", launch=_ten())
    with pytest.raises(C.SphericartError):  # FP64 arithmetic
        api.spherical_harmonics(x.double(), 9, False, gradients=True, hessians=True, kernel="point", launch=_ten())
    with pytest.raises(C.SphericartError):  # bf16 storage
        api.spherical_harmonics(x, 9, False, gradients=True, hessians=True, kernel="point", launch=_ten(),
                                out_dtype=torch.bfloat16)


def test_auto_default():
    """AUTO runs 10 lanes per point for FP32 Hessians where measured faster
    (scaled l_max 7..16, normalized 6..13), the one-lane tile below, ROW for
    the normalized form from l_max 14 and beyond POINT's range."""
    fam, s = C.sphericart_launch_info(8, C.SPH_F32, C.SPH_OUT_SAME, 1, 1)
    assert fam == C.SPH_KERNEL_POINT and s.lanes_per_point == 10 and s.points_per_tile == 6
    fam, s = C.sphericart_launch_info(6, C.SPH_F32, C.SPH_OUT_SAME, 1, 1)
    assert s.lanes_per_point == 0  # (launch_info reports the scaled form's choice)
    fam, s = C.sphericart_launch_info(8, C.SPH_F64, C.SPH_OUT_SAME, 1, 1)
    assert s.lanes_per_point == 0
    fam, s = C.sphericart_launch_info(16, C.SPH_F32, C.SPH_OUT_SAME, 1, 1)
    assert fam == C.SPH_KERNEL_POINT and s.lanes_per_point == 10
    x = _t(inputs.shell_points(1000, 0.5, 2.0, seed=355))
    for l_max, normalized, P in ((8, False, 6), (6, True, 6), (13, True, 3), (15, False, 3), (16, False, 3)):
        a = api.spherical_harmonics(x, l_max, normalized, gradients=True, hessians=True)
        b = api.spherical_harmonics(x, l_max, normalized, gradients=True, hessians=True, kernel="point",
                                    launch=_ten(P, 1))
        assert all(torch.equal(u, w) for u, w in zip(a, b)), (l_max, normalized)
    for l_max in (14, 16):  # normalized: ROW
        a = api.spherical_harmonics(x, l_max, True, gradients=True, hessians=True)
        b = api.spherical_harmonics(x, l_max, True, gradients=True, hessians=True, kernel="row")
        assert all(torch.equal(u, w) for u, w in zip(a, b)), l_max


def test_full_size_lmax8_every_point():
    """400,000 points, l_max 8, scaled, FP32 Hessians on the AUTO path (10
    lanes per point): every element of ddsph against the oracle, symmetric
    planes bit for bit."""
    import full_parity

    n, l_max = 400_000, 8
    x = inputs.shell_points(n, 0.5, 5.0, seed=336).astype(np.float32)
    _, _, H = api.spherical_harmonics(_t(x), l_max, False, gradients=True, hessians=True)
    eh, finite, sym = full_parity.hessian_errors(x.astype(np.float64), l_max, False, H.cpu().numpy())
    assert finite and sym
    assert np.all(eh <= 5e-6 * (np.arange(l_max + 1) + 1)), eh


def test_full_size_lmax13_normalized_every_point():
    """200,000 points (half within 1e-4 rad of the poles), l_max 13 (even K:
    row slots, mirrors sent from one slot), normalized, FP32 Hessians on the
    AUTO path (10 lanes per point): every element of ddsph against the
    oracle, symmetric planes bit for bit."""
    import full_parity

    n, l_max = 200_000, 13
    x = inputs.pole_mix_points(n, seed=356).astype(np.float32)
    _, _, H = api.spherical_harmonics(_t(x), l_max, True, gradients=True, hessians=True)
    eh, finite, sym = full_parity.hessian_errors(x.astype(np.float64), l_max, True, H.cpu().numpy())
    assert finite and sym
    assert np.all(eh <= 5e-6 * (np.arange(l_max + 1) + 1)), eh


def test_installed_shapes_and_clear():
    """set_launch installs 10- and 16-lane Hessian shapes for AUTO calls
    (validated like explicit launches); tune_clear restores the defaults."""
    x = _t(inputs.shell_points(2000, 0.5, 2.0, seed=357))
    L = 9
    ref = api.spherical_harmonics(x, L, False, gradients=True, hessians=True, kernel="point", launch=_ten(3, 1))
    try:
        C.sphericart_set_launch(L, C.SPH_F32, C.SPH_OUT_SAME, 2, _ten(6, 2, 0))
        fam, s = C.sphericart_launch_info(L, C.SPH_F32, C.SPH_OUT_SAME, 1, 1)
        assert fam == C.SPH_KERNEL_POINT and (s.points_per_tile, s.warps_per_block, s.lanes_per_point) == (6, 2, 10)
        out = api.spherical_harmonics(x, L, False, gradients=True, hessians=True)
        assert all(torch.equal(u, w) for u, w in zip(ref, out))
        C.sphericart_set_launch(L, C.SPH_F32, C.SPH_OUT_SAME, 2, C.make_launch(4, 1, 0, 16))
        fam, s = C.sphericart_launch_info(L, C.SPH_F32, C.SPH_OUT_SAME, 1, 1)
        assert s.lanes_per_point == 16
        out = api.spherical_harmonics(x, L, False, gradients=True, hessians=True)
        for u, w in zip(ref, out):
            assert (u - w).abs().max().item() <= 2e-6 * max(1.0, u.abs().max().item())
        for grad, lau in ((1, _ten()), (2, _ten(4, 1)), (2, _ten(6, 5)), (2, C.make_launch(3, 1, 0, 16))):
            with pytest.raises(C.SphericartError):
                C.sphericart_set_launch(L, C.SPH_F32, C.SPH_OUT_SAME, grad, lau)
        with pytest.raises(C.SphericartError):  # FP64
            C.sphericart_set_launch(L, C.SPH_F64, C.SPH_OUT_SAME, 2, _ten())
    finally:
        C.sphericart_tune_clear()
    fam, s = C.sphericart_launch_info(L, C.SPH_F32, C.SPH_OUT_SAME, 1, 1)
    assert (s.points_per_tile, s.lanes_per_point) == (3, 10)
