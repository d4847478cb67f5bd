"""Parity of the ROW kernel family (8 lanes per point, recursion state in
registers, output rows staged in windows of whole degrees and written with
TMA bulk copies of sector-aligned runs) against the FP64 oracle, through the
C-ABI.

Covers every channel count (l_max 16..63), ragged tiles (n not a multiple of
the 4 points a warp owns), every alignment phase of the output rows (outputs
offset by 0..7 elements: row heads, carried partial sectors and row tails),
bf16 storage, and the high-degree workload at full size.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_2302_08381_gb300 import _capi as C
from paper_2302_08381_gb300 import api, inputs
from parity_utils import BF16_TOL, F32_GRAD, F32_VAL, assert_grads, assert_values, grad_errors, value_errors

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _run(xyz_np, l_max, normalized, grad, out_dtype=None, launch=None):
    xyz = torch.from_numpy(np.ascontiguousarray(xyz_np, dtype=np.float32)).to(DEV)
    res = api.spherical_harmonics(xyz, l_max, normalized, gradients=grad, out_dtype=out_dtype, kernel="row",
                                  launch=launch)
    torch.cuda.synchronize()

    def host(t):
        return (t.float() if t.dtype == torch.bfloat16 else t).double().cpu().numpy()

    if grad:
        return host(res[0]), host(res[1])
    return host(res)


@pytest.mark.parametrize("normalized", [False, True])
def test_f32_every_lmax(normalized):
    n = 203  # 50 full 4-point tiles and a ragged one
    x = inputs.shell_points(n, 0.5, 2.0, seed=400).astype(np.float64)
    for l_max in range(16, 64):
        v, g = _run(x, l_max, normalized, True)
        rv, rg = oracle.spherical_harmonics_grad(x, l_max, normalized)
        assert np.all(np.isfinite(v)) and np.all(np.isfinite(g))
        if l_max <= 20:
            assert_values(v, x, l_max, normalized, F32_VAL, ref=rv)
            assert_grads(g, x, l_max, normalized, F32_GRAD, ref=rg)
        else:  # FP32 rounding accumulated over the recursion: bounded loosely
            ev = value_errors(v, rv, x, l_max, normalized)
            eg = grad_errors(g, rg, x, l_max, normalized)
            assert ev.max() < 1e-4 and eg.max() < 1e-3, (l_max, ev.max(), eg.max())


def test_values_only_matches_values_with_gradients():
    x = inputs.normal_points(1001, seed=401)
    for l_max in (16, 23, 40, 63):
        for normalized in (False, True):
            v0 = _run(x, l_max, normalized, False)
            v1, _ = _run(x, l_max, normalized, True)
            np.testing.assert_array_equal(v0, v1)


@pytest.mark.parametrize("offset", [0, 1, 3, 5, 7])
def test_every_alignment_phase(offset):
    """Output buffers offset by `offset` elements from a 256-byte boundary:
    the bulk runs start at a different column of every row, the row heads and
    tails take plain stores, and the element before the buffers is untouched."""
    n, l_max = 97, 21
    K = (l_max + 1) ** 2
    x = torch.from_numpy(inputs.normal_points(n, seed=402).astype(np.float32)).to(DEV)
    buf = torch.full((offset + n * K + 32,), -7.0, device=DEV)
    dbuf = torch.full((offset + 3 * n * K + 32,), -7.0, device=DEV)
    sph = buf[offset: offset + n * K].view(n, K)
    dsph = dbuf[offset: offset + 3 * n * K].view(n, 3, K)
    api.spherical_harmonics(x, l_max, True, gradients=True, kernel="row", out=(sph, dsph))
    ref_v, ref_g = api.spherical_harmonics(x, l_max, True, gradients=True, kernel="row")
    torch.cuda.synchronize()
    assert torch.equal(sph, ref_v) and torch.equal(dsph, ref_g)
    assert torch.all(buf[:offset] == -7.0) and torch.all(buf[offset + n * K:] == -7.0)
    assert torch.all(dbuf[:offset] == -7.0) and torch.all(dbuf[offset + 3 * n * K:] == -7.0)
    p = x.double().cpu().numpy()
    rv, rg = oracle.spherical_harmonics_grad(p, l_max, True)
    assert_values(sph.double().cpu().numpy(), p, l_max, True, F32_VAL, ref=rv)
    assert_grads(dsph.double().cpu().numpy(), p, l_max, True, F32_GRAD, ref=rg)


def test_bf16_store():
    x = inputs.pole_mix_points(402, seed=403)
    x32 = x.astype(np.float32).astype(np.float64)
    for l_max in (16, 30, 47, 48):
        for offset_view in (False, True):
            xt = torch.from_numpy(x32.astype(np.float32)).to(DEV)
            K = (l_max + 1) ** 2
            n = xt.shape[0]
            if offset_view:  # bf16 rows starting 2 bytes past a sector boundary
                b = torch.empty(1 + n * K, dtype=torch.bfloat16, device=DEV)
                d = torch.empty(1 + 3 * n * K, dtype=torch.bfloat16, device=DEV)
                out = (b[1:].view(n, K), d[1:].view(n, 3, K))
                v, g = api.spherical_harmonics(xt, l_max, True, gradients=True, out_dtype=torch.bfloat16,
                                               kernel="row", out=out)
            else:
                v, g = api.spherical_harmonics(xt, l_max, True, gradients=True, out_dtype=torch.bfloat16,
                                               kernel="row")
            torch.cuda.synchronize()
            rv, rg = oracle.spherical_harmonics_grad(x32, l_max, True)
            assert_values(v.float().double().cpu().numpy(), x32, l_max, True, BF16_TOL, ref=rv)
            assert_grads(g.float().double().cpu().numpy(), x32, l_max, True, BF16_TOL, ref=rg)


def test_empty_tiny_and_canaries():
    for n in (0, 1, 2, 3, 4, 5, 7):
        x = inputs.normal_points(n, seed=404)
        v, g = _run(x, 18, False, True)
        assert v.shape == (n, 361) and g.shape == (n, 3, 361)
        if n:
            assert_values(v, x.astype(np.float32).astype(np.float64), 18, False, F32_VAL)
    n, l_max = 1003, 33
    K = (l_max + 1) ** 2
    x = torch.from_numpy(inputs.normal_points(n, seed=405).astype(np.float32)).to(DEV)
    buf = torch.full((n * K + 64,), -7.0, device=DEV)
    dbuf = torch.full((n * 3 * K + 64,), -7.0, device=DEV)
    api.spherical_harmonics(x, l_max, gradients=True, kernel="row",
                            out=(buf[: n * K].view(n, K), dbuf[: 3 * n * K].view(n, 3, K)))
    torch.cuda.synchronize()
    assert torch.all(buf[n * K:] == -7.0) and torch.all(dbuf[3 * n * K:] == -7.0)
    assert not torch.any(buf[: n * K] == -7.0) and not torch.any(dbuf[: 3 * n * K] == -7.0)


def test_launch_shapes_give_identical_results():
    n, l_max = 20_011, 30
    x = inputs.normal_points(n, seed=406)
    base = None
    for W in (1, 2):
        for B in (0, 1, 3):
            v, g = _run(x, l_max, False, True, launch=C.make_launch(0, W, B, 0))
            if base is None:
                base = (v, g)
            else:
                np.testing.assert_array_equal(v, base[0])
                np.testing.assert_array_equal(g, base[1])
    # the forward runs at most 2 warps per block (its launch bound)
    with pytest.raises(C.SphericartError):
        _run(x, l_max, False, True, launch=C.make_launch(0, 3, 0, 0))
    p = x[::101].astype(np.float32).astype(np.float64)
    rv, rg = oracle.spherical_harmonics_grad(p, l_max, False)
    assert value_errors(base[0][::101], rv, p, l_max, False).max() < 1e-4


def test_unsupported_requests():
    x = torch.zeros((4, 3), device=DEV)
    for l_max in (15, 64):
        with pytest.raises(C.SphericartError):
            api.spherical_harmonics(x, l_max, gradients=True, kernel="row")
    with pytest.raises(C.SphericartError):
        api.spherical_harmonics(x, 20, gradients=True, kernel="row", qprec="f64")
    with pytest.raises(C.SphericartError):
        api.spherical_harmonics(x.double(), 20, gradients=True, kernel="row")
    with pytest.raises(C.SphericartError):  # Hessians: FP32 storage only (tests/test_row_hess_gpu.py)
        api.spherical_harmonics(x, 20, hessians=True, kernel="row", out_dtype=torch.bfloat16)


@pytest.mark.parametrize("l_max", [20, 30, 50])
def test_sweep_workload_sampled(l_max):
    """The high-degree workload at full size (200,000 points, half within
    1e-4 rad of the poles, normalized, FP32): 2,000 sampled points vs the
    oracle, every output finite."""
    N = 200_000
    xyz = inputs.pole_mix_points(N, seed=4).astype(np.float32)
    v, g = _run(xyz, l_max, True, True)
    rng = np.random.default_rng(46)
    idx = np.concatenate([rng.choice(N // 2, 1000, replace=False), N // 2 + rng.choice(N // 2, 1000, replace=False)])
    p = xyz[idx].astype(np.float64)
    rv, rg = oracle.spherical_harmonics_grad(p, l_max, True)
    assert np.all(np.isfinite(v)) and np.all(np.isfinite(g))
    if l_max <= 20:
        assert_values(v[idx], p, l_max, True, F32_VAL, ref=rv)
        assert_grads(g[idx], p, l_max, True, F32_GRAD, ref=rg)
    else:
        assert value_errors(v[idx], rv, p, l_max, True).max() < 1e-4
        assert grad_errors(g[idx], rg, p, l_max, True).max() < 1e-3


# --------------------------------------------------------------- fused backward
def _rel(got, ref):
    ref = np.asarray(ref, np.float64)
    return float(np.max(np.abs(np.asarray(got, np.float64) - ref)) / max(np.max(np.abs(ref)), 1e-300))


@pytest.mark.parametrize("normalized", [False, True])
def test_backward_matches_oracle(normalized):
    """dxyz = sum_k g_k dY_k/dx (recomputed recursion, g read by bulk-loaded
    windows) vs the oracle's contraction, every channel count."""
    n = 203
    x = inputs.shell_points(n, 0.7, 3.0, seed=410).astype(np.float32).astype(np.float64)
    xt = torch.from_numpy(x.astype(np.float32)).to(DEV)
    for l_max in (16, 17, 20, 23, 24, 31, 32, 39, 40, 47, 48, 55, 56, 63):
        K = (l_max + 1) ** 2
        g = inputs.upstream(n, K, seed=411 + l_max).astype(np.float32)
        dx = api.backward(xt, torch.from_numpy(g).to(DEV), l_max, normalized, kernel="row")
        torch.cuda.synchronize()
        ref = oracle.backward(x, g.astype(np.float64), l_max, normalized)
        tol = 2e-5 if l_max <= 20 else 1e-4  # FP32 rounding accumulated over the recursion
        assert _rel(dx.cpu().numpy(), ref) < tol, (l_max, _rel(dx.cpu().numpy(), ref))
    assert api.device_status() == 0


@pytest.mark.parametrize("offset", [0, 1, 2, 3])
def test_backward_unaligned_rows_and_ragged_tiles(offset):
    """g rows starting at every 4-byte offset from a 16-byte boundary (bulk
    loads of the aligned middle, plain loads of the edges), n not a multiple
    of the 4 points a warp owns; AUTO picks ROW here and matches SLICE."""
    n, l_max = 1001, 27
    K = (l_max + 1) ** 2
    x = torch.from_numpy(inputs.normal_points(n, seed=412).astype(np.float32)).to(DEV)
    buf = torch.from_numpy(inputs.upstream(n * K + offset, 1, seed=413).astype(np.float32)[:, 0]).to(DEV)
    g = buf[offset:].view(n, K)
    for normalized in (False, True):
        a = api.backward(x, g, l_max, normalized)  # AUTO
        b = api.backward(x, g, l_max, normalized, kernel="slice")
        torch.cuda.synchronize()
        assert _rel(a.cpu().numpy(), b.double().cpu().numpy()) < 2e-5
    assert api.device_status() == 0


def test_backward_launch_shapes_identical():
    n, l_max = 20_011, 33
    K = (l_max + 1) ** 2
    x = torch.from_numpy(inputs.normal_points(n, seed=414).astype(np.float32)).to(DEV)
    g = torch.from_numpy(inputs.upstream(n, K, seed=415)).to(DEV)
    base = None
    for W in (1, 2, 4, 8):
        for B in (0, 1):
            d = api.backward(x, g, l_max, True, kernel="row", launch=C.make_launch(0, W, B, 0))
            torch.cuda.synchronize()
            if base is None:
                base = d.clone()
            else:
                assert torch.equal(d, base)
    p = x[::97].double().cpu().numpy()
    ref = oracle.backward(p, g[::97].double().cpu().numpy(), l_max, True)
    assert _rel(base[::97].cpu().numpy(), ref) < 1e-4
