"""Fused recompute-backward and double backward against the oracle, central
finite differences (FP64, h = 1e-3) and torch.autograd's own checks.
"""

import numpy as np
import pytest
import torch

import full_parity
import oracle
from paper_2302_08381_gb300 import _capi as C
from paper_2302_08381_gb300 import api, inputs
from paper_2302_08381_gb300.autograd import spherical_harmonics_autograd
from parity_utils import F64_TOL, hess_errors, hess_scale

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _t(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV, dtype)


def _rel(got, ref, floor=0.0):
    """max |got - ref| / max(max |ref|, floor)."""
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(np.asarray(got, np.float64) - ref)) / max(np.max(np.abs(ref)), floor, 1e-300))


@pytest.mark.parametrize("kernel", ["point", "slice"])
@pytest.mark.parametrize("normalized", [False, True])
def test_backward_matches_oracle_every_lmax(kernel, normalized):
    n = 1500 + 7
    x = inputs.shell_points(n, 0.7, 3.0, seed=200).astype(np.float32).astype(np.float64)
    for l_max in list(range(0, 17)) + ([20, 27] if kernel == "slice" else []):
        K = (l_max + 1) ** 2
        g = inputs.upstream(n, K, seed=201 + l_max).astype(np.float32).astype(np.float64)
        dx = api.backward(_t(x), _t(g), l_max, normalized, kernel=kernel)
        ref = oracle.backward(x, g, l_max, normalized)
        assert _rel(dx.cpu().numpy(), ref) < 2e-5, l_max
        # FP64 path
        dx64 = api.backward(_t(x, torch.float64), _t(g, torch.float64), l_max, normalized, kernel=kernel)
        assert _rel(dx64.cpu().numpy(), ref) < 1e-12, l_max


def test_backward_equals_materialized_contraction():
    n, l_max = 4099, 6
    x = _t(inputs.shell_points(n, 0.7, 6.0, seed=202))
    g = _t(inputs.upstream(n, 49, seed=203))
    fused = api.backward(x, g, l_max)
    plain = api.materialized_backward(x, g, l_max)
    torch.cuda.synchronize()
    assert _rel(fused.cpu().numpy(), plain.double().cpu().numpy()) < 1e-5


@pytest.mark.parametrize("l_max", [0, 1, 2, 3, 4, 6, 8, 12, 16, 20])
@pytest.mark.parametrize("kernel", ["point", "slice"])
@pytest.mark.parametrize("normalized", [False, True])
def test_double_backward_matches_oracle(kernel, normalized, l_max):
    if kernel == "point" and l_max > 16:
        pytest.skip("POINT kernels stop at l_max = 16")
    n = 700 + 3
    x = inputs.shell_points(n, 0.7, 3.0, seed=204).astype(np.float64)
    K = (l_max + 1) ** 2
    g = inputs.upstream(n, K, seed=205 + l_max).astype(np.float64)
    v = inputs.upstream(n, 3, seed=305 + l_max).astype(np.float64)
    rgg, rgx = oracle.double_backward(x, g, v, l_max, normalized)
    gg, gx = api.double_backward(_t(x, torch.float64), _t(g, torch.float64), _t(v, torch.float64), l_max,
                                 normalized, kernel=kernel)
    # grad_xyz is exactly 0 for l_max <= 1 (linear harmonics): compare on a
    # scale of 1e-3 |g| |v| at least.
    floor = 1e-3 * np.max(np.abs(g)) * np.max(np.abs(v))
    assert _rel(gg.cpu().numpy(), rgg) < 1e-12
    assert _rel(gx.cpu().numpy(), rgx, floor) < 1e-12
    gg32, gx32 = api.double_backward(_t(x), _t(g), _t(v), l_max, normalized, kernel=kernel)
    assert _rel(gg32.cpu().numpy(), rgg) < 1e-5
    assert _rel(gx32.cpu().numpy(), rgx, floor) < 1e-4


@pytest.mark.parametrize("kernel", ["point", "slice"])
def test_hessian_output(kernel):
    """ddsph of the forward vs the oracle's analytic Hessian (FP64 at 1e-12 of
    each l block's Hessian scale, scaled and normalized), plus exact
    invariants: symmetric, trace-free (solid harmonics are harmonic), Euler
    relation. Points include both poles' neighbourhoods."""
    x = np.concatenate([inputs.shell_points(300, 0.7, 2.0, seed=206).astype(np.float64),
                        inputs.pole_mix_points(60, seed=207) * 1.3])
    for l_max in (0, 1, 2, 5, 8, 9, 16) + ((20,) if kernel == "slice" else ()):
        sph, dsph, ddsph = api.spherical_harmonics(_t(x, torch.float64), l_max, gradients=True, hessians=True,
                                                   kernel=kernel)
        H = ddsph.cpu().numpy()
        G = dsph.cpu().numpy()
        ref = oracle.spherical_harmonics_hessian(x, l_max)
        lv = np.concatenate([np.full(2 * l + 1, l) for l in range(l_max + 1)])
        hs = hess_scale(x, l_max, False)
        e = hess_errors(H, ref, x, l_max, False)
        assert np.all(e <= F64_TOL), (l_max, e)
        assert np.array_equal(H, H.transpose(0, 2, 1, 3))
        assert np.max(np.abs(np.trace(H, axis1=1, axis2=2)) / hs) < F64_TOL, l_max
        euler = np.einsum("nj,nijk->nik", x, H) - (lv[None, None, :] - 1.0) * G
        assert np.max(np.abs(euler) / hs[:, None, :]) < F64_TOL, l_max
        # normalized Hessians against the oracle
        _, _, Hn = api.spherical_harmonics(_t(x, torch.float64), l_max, True, hessians=True, kernel=kernel)
        refn = oracle.spherical_harmonics_hessian(x, l_max, True)
        en = hess_errors(Hn.cpu().numpy(), refn, x, l_max, True)
        assert np.all(en <= F64_TOL), (l_max, en)
        # FP32 Hessians against the oracle at the FP32-rounded coordinates
        _, _, H32 = api.spherical_harmonics(_t(x), l_max, gradients=True, hessians=True, kernel=kernel)
        x32 = x.astype(np.float32).astype(np.float64)
        ref32 = oracle.spherical_harmonics_hessian(x32, l_max)
        e32 = hess_errors(H32.double().cpu().numpy(), ref32, x32, l_max, False)
        assert np.all(e32 <= 5e-5), (l_max, e32)


def test_hessian_point_matches_slice_and_tiles():
    """POINT and SLICE Hessians agree (FP64); POINT over several tile shapes."""
    n = 5003
    x = _t(inputs.shell_points(n, 0.5, 3.0, seed=230), torch.float64)
    for l_max in (3, 8):
        a = api.spherical_harmonics(x, l_max, gradients=True, hessians=True, kernel="slice")
        for P, W in ((2, 1), (4, 2), (8, 1)):
            b = api.spherical_harmonics(x, l_max, gradients=True, hessians=True, kernel="point",
                                        launch=C.make_launch(P, W, 1, 0))
            for u, v in zip(a, b):
                assert (u - v).abs().max().item() <= 1e-12 * max(1.0, u.abs().max().item()), (l_max, P, W)


@pytest.mark.parametrize("l_max,normalized", [(3, False), (6, True), (8, False), (19, False)])
def test_autograd_gradcheck_fp64(l_max, normalized):
    torch.manual_seed(l_max)
    # radii in [0.85, 1] keep r^l <= 1, so the difference quotients' rounding
    # (~1e-16 |f| / eps) stays below atol at every l_max tested
    x = torch.randn(16, 3, dtype=torch.float64, device=DEV)
    x = x / x.norm(dim=1, keepdim=True) * (0.85 + 0.15 * torch.rand(16, 1, dtype=torch.float64, device=DEV))
    x = x.requires_grad_()
    f = lambda p: spherical_harmonics_autograd(p, l_max, normalized)  # noqa: E731
    assert torch.autograd.gradcheck(f, (x,), eps=1e-6, atol=1e-8, rtol=1e-6)
    assert torch.autograd.gradgradcheck(f, (x,), eps=1e-6, atol=1e-7, rtol=1e-5)


def test_double_backward_grad_g_is_exact_contraction():
    """grad_g = sum_j v_j dY/dx_j exactly (FP64), against the FP64 forward's dsph."""
    n = 333
    for l_max in (1, 3, 6, 8, 16, 19):
        x = _t(inputs.shell_points(n, 0.6, 1.4, seed=220 + l_max), torch.float64)
        g = _t(inputs.upstream(n, (l_max + 1) ** 2, seed=221), torch.float64)
        v = _t(inputs.upstream(n, 3, seed=222), torch.float64)
        for normalized in (False, True):
            _, dsph = api.spherical_harmonics(x, l_max, normalized, gradients=True)
            want = torch.einsum("njk,nj->nk", dsph, v)
            for kernel in ("point", "slice"):
                if kernel == "point" and l_max > 16:
                    continue
                gg, _ = api.double_backward(x, g, v, l_max, normalized, kernel=kernel)
                err = (gg - want).abs().max().item() / want.abs().max().item()
                assert err < 1e-12, (l_max, normalized, kernel, err)


def test_backward_central_fd_fp64_h1e3():
    """Config-3 distribution: dL/dxyz of L = sum(g * Y) vs central FD, h = 1e-3."""
    n, l_max = 256, 6
    x = inputs.shell_points(n, 0.7, 6.0, seed=207).astype(np.float64)
    g = inputs.upstream(n, 49, seed=208).astype(np.float64)
    dx = api.backward(_t(x, torch.float64), _t(g, torch.float64), l_max).cpu().numpy()
    fd = np.zeros_like(x)
    for j in range(3):
        e = np.zeros_like(x)
        e[:, j] = 1e-3
        yp = api.spherical_harmonics(_t(x + e, torch.float64), l_max).cpu().numpy()
        ym = api.spherical_harmonics(_t(x - e, torch.float64), l_max).cpu().numpy()
        fd[:, j] = np.sum((yp - ym) * g, axis=1) / 2e-3
    # FD truncation at h = 1e-3 for degree-6 polynomials with |r| <= 6
    assert _rel(dx, fd) < 1e-5


def test_workload_backward_full_size():
    """N = 4,194,304 edge vectors, l_max = 6: fused backward and double
    backward at full size, every point against the oracle; the fused backward
    equals the materialised contraction."""
    n, l_max = 4_194_304, 6
    x_np = inputs.shell_points(n, 0.7, 6.0, seed=3)
    g_np = inputs.upstream(n, 49, seed=33)
    v_np = inputs.upstream(n, 3, seed=34)
    x, g = _t(x_np), _t(g_np)
    dx = api.backward(x, g, l_max)
    plain = api.materialized_backward(x, g, l_max)
    gg, gx = api.double_backward(x, g, _t(v_np), l_max)
    torch.cuda.synchronize()
    assert api.device_status() == 0
    assert _rel(dx.cpu().numpy(), plain.double().cpu().numpy()) < 2e-5
    err = full_parity.adjoint_errors(x_np, g_np, l_max, False, dxyz=dx.cpu().numpy(), v=v_np,
                                     grad_g=gg.cpu().numpy(), grad_xyz=gx.cpu().numpy())
    assert err["dxyz"] < 2e-5 and err["grad_g"] < 2e-5 and err["grad_xyz"] < 1e-4, err


def test_backward_launch_shapes_and_unaligned():
    n, l_max = 9001, 5
    x_np = inputs.normal_points(n, seed=209).astype(np.float32)
    g_np = inputs.upstream(n, 36, seed=210)
    x = _t(x_np)
    base = api.backward(x, _t(g_np), l_max, kernel="point")
    for P in (4, 8, 16, 28, 32):
        for W in (1, 3, 8):
            d = api.backward(x, _t(g_np), l_max, kernel="point", launch=C.make_launch(P, W, 1, 0))
            assert torch.equal(d, base)
    # g at a 4-byte (not 16-byte) offset takes the plain-load path
    gb = torch.empty(n * 36 + 1, device=DEV)
    gb[1:] = _t(g_np).reshape(-1)
    d = api.backward(x, gb[1:].view(n, 36), l_max, kernel="point")
    assert torch.equal(d, base)
    ref = oracle.backward(x_np.astype(np.float64), g_np.astype(np.float64), l_max)
    assert _rel(base.cpu().numpy(), ref) < 2e-5
