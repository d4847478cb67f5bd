"""Host-side checks of the C-ABI library (no GPU needed).

The library must load, export every function the public header declares,
produce host FP64 tables that agree with the closed forms, and reject bad
arguments before touching any CUDA API.
"""

import math
import os
import re

import numpy as np
import pytest

import oracle
from paper_2302_08381_gb300 import _capi as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def _declared_functions():
    names = set()
    for f in os.listdir(HEADER_DIR):
        if f.endswith(".h"):
            text = open(os.path.join(HEADER_DIR, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(sphericart_\w+)\s*\(", text))
    return sorted(names)


def test_library_loads_and_exports_header_symbols():
    lib = C.lib()
    declared = _declared_functions()
    assert len(declared) >= 10
    missing = [n for n in declared if not hasattr(lib, n)]
    assert not missing, missing
    assert set(declared) == set(C._PROTOS), "binding and header list different entry points"


def test_version_and_limits():
    assert C.sphericart_version() >= 10000
    assert C.sphericart_max_l(C.SPH_F32, C.SPH_Q_NATIVE, C.SPH_KERNEL_POINT) == C.SPH_MAX_L_POINT
    assert C.sphericart_max_l(C.SPH_F32, C.SPH_Q_NATIVE, C.SPH_KERNEL_SLICE) == C.SPH_MAX_L
    assert C.sphericart_max_l(C.SPH_F32, C.SPH_Q_F64, C.SPH_KERNEL_POINT) == -1
    assert C.sphericart_max_l(C.SPH_F32, C.SPH_Q_F64, C.SPH_KERNEL_DEGREE) == C.SPH_MAX_L
    assert C.sphericart_max_l(C.SPH_F64, C.SPH_Q_NATIVE, C.SPH_KERNEL_DEGREE_DOWN) == C.SPH_MAX_L


def _tri(l, m):
    return l * (l + 1) // 2 + m


def test_host_prefactor_table_matches_closed_form():
    """Appendix C iteration (host, C++) vs Eq. Flm's closed form (oracle)."""
    L = 128
    F = C.sphericart_host_table(L, 0)
    for l in range(L + 1):
        for m in range(l + 1):
            ref = oracle.prefactor(l, m)
            assert F[_tri(l, m)] == pytest.approx(ref, rel=2e-13), (l, m)


def test_host_recursion_coefficients():
    L = 60
    qll, a, b, e, fz, d = (C.sphericart_host_table(L, w) for w in (1, 2, 3, 4, 5, 6))
    F = oracle.prefactor
    s2 = 1 / math.sqrt(2)
    for l in range(L + 1):
        # Qtilde_l^l = F_l^l (-1)^l (2l-1)!!
        dfact = 1
        for k in range(1, 2 * l, 2):
            dfact *= k
        want = F(l, l) * (-1) ** l * float(dfact) if l < 150 else None
        assert qll[_tri(l, l)] == pytest.approx(want, rel=1e-12)
        if l >= 1:
            assert d[_tri(l, l - 1)] == pytest.approx((2 * l - 1) * F(l, l - 1) / F(l - 1, l - 1), rel=1e-12)
        for m in range(l + 1):
            i = _tri(l, m)
            sc = s2 if m == 0 else 1.0
            if m <= l - 2:
                assert a[i] == pytest.approx((2 * l - 1) / (l - m) * F(l, m) / F(l - 1, m), rel=1e-12)
                assert b[i] == pytest.approx((l + m - 1) / (l - m) * F(l, m) / F(l - 2, m), rel=1e-12)
                assert e[i] == pytest.approx(sc * F(l, m) / F(l - 1, m + 1), rel=1e-12)
            else:
                assert a[i] == 0 and b[i] == 0 and e[i] == 0
            if m <= l - 1:
                assert fz[i] == pytest.approx(sc * (l + m) * F(l, m) / F(l - 1, m), rel=1e-12)
            else:
                assert fz[i] == 0


def test_host_downward_coefficients_closed_form():
    """Folded coefficients of Eq. iter-q-alt (sign-corrected) from the F table
    ratios vs their closed forms: al = 2(m+1)/sqrt((l+m+1)(l-m)),
    be = sqrt((l+m+2)(l-m-1)/((l+m+1)(l-m)))."""
    L = 128
    al, be = C.sphericart_host_table(L, 7), C.sphericart_host_table(L, 8)
    for l in range(L + 1):
        for m in range(l + 1):
            i = _tri(l, m)
            want_a = 2 * (m + 1) / math.sqrt((l + m + 1) * (l - m)) if m <= l - 1 else 0.0
            want_b = math.sqrt((l + m + 2) * (l - m - 1) / ((l + m + 1) * (l - m))) if m <= l - 2 else 0.0
            assert al[i] == pytest.approx(want_a, rel=1e-12, abs=0), (l, m)
            assert be[i] == pytest.approx(want_b, rel=1e-12, abs=0), (l, m)


def test_host_downward_tables_reproduce_oracle():
    """The library's downward-in-m tables, run on the host in FP64 (c_m, s_m
    by Eq. iter-sc, Qtilde_l^m from the tabulated Qtilde_l^l downwards),
    reproduce the oracle's scaled harmonics (Eq. real-sh-spherical) up to
    l_max = 40, including points near the poles and on the equator."""
    L = 40
    qll, al, be = (C.sphericart_host_table(L, w) for w in (1, 7, 8))
    rng = np.random.default_rng(3)
    xyz = rng.normal(size=(64, 3))
    xyz[:4] = [[1e-5, 2e-5, 1.0], [3e-6, -1e-6, -0.7], [0.6, -0.8, 0.0], [0.0, 0.0, 1.3]]
    ref = oracle.spherical_harmonics(xyz, L, False)
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    rxy2 = x * x + y * y
    c = [np.ones_like(x)]
    s = [np.zeros_like(x)]
    for m in range(1, L + 1):
        c.append(x * c[-1] - y * s[-1])
        s.append(x * s[-1] + y * c[-2])
    got = np.zeros_like(ref)
    for l in range(L + 1):
        q1 = np.zeros_like(x)  # Qtilde_l^{m+1}
        q2 = np.zeros_like(x)  # Qtilde_l^{m+2}
        for m in range(l, -1, -1):
            i = _tri(l, m)
            q = al[i] * z * q1 - be[i] * rxy2 * q2 + (qll[i] if m == l else 0.0)
            q2, q1 = q1, q
            if m == 0:
                got[:, l * l + l] = q / math.sqrt(2)
            else:
                got[:, l * l + l + m] = q * c[m]
                got[:, l * l + l - m] = q * s[m]
    r = np.linalg.norm(xyz, axis=1)
    lv = np.concatenate([np.full(2 * l + 1, l) for l in range(L + 1)])
    err = np.abs(got - ref) / r[:, None] ** lv[None, :]
    assert err.max() < 1e-12, err.max()


def test_auto_family_choice():
    """AUTO: DEGREE for FP64 arithmetic from l_max 14 (with gradients from
    9); ROW for FP32 arithmetic from POINT's range to l_max 63 and for FP32
    Hessians beyond it (scaled form; normalized from l_max 14); then SLICE
    (FP32 storage) or DEGREE (bf16
    storage); FP64 Hessians on SLICE (host-only query)."""
    fam, shape = C.sphericart_launch_info(16, C.SPH_F64, C.SPH_OUT_SAME, 1, 0)
    assert fam == C.SPH_KERNEL_DEGREE and shape.lanes_per_point in (1, 2, 4)
    fam, shape = C.sphericart_launch_info(10, C.SPH_F64, C.SPH_OUT_SAME, 1, 0)
    assert fam == C.SPH_KERNEL_DEGREE and shape.lanes_per_point == 2
    assert C.sphericart_launch_info(9, C.SPH_F64, C.SPH_OUT_SAME, 1, 0)[0] == C.SPH_KERNEL_DEGREE
    assert C.sphericart_launch_info(10, C.SPH_F64, C.SPH_OUT_SAME, 0, 0)[0] == C.SPH_KERNEL_POINT  # values
    assert C.sphericart_launch_info(13, C.SPH_F64, C.SPH_OUT_SAME, 0, 0)[0] == C.SPH_KERNEL_POINT
    assert C.sphericart_launch_info(14, C.SPH_F64, C.SPH_OUT_SAME, 0, 0)[0] == C.SPH_KERNEL_DEGREE
    assert C.sphericart_launch_info(20, C.SPH_F32, C.SPH_OUT_SAME, 1, 1)[0] == C.SPH_KERNEL_ROW  # FP32 Hessians
    assert C.sphericart_launch_info(17, C.SPH_F32, C.SPH_OUT_SAME, 1, 1)[0] == C.SPH_KERNEL_ROW
    fam, shape = C.sphericart_launch_info(16, C.SPH_F32, C.SPH_OUT_SAME, 1, 1)
    assert fam == C.SPH_KERNEL_POINT and shape.lanes_per_point == 10
    fam, _ = C.sphericart_launch_info(30, C.SPH_F32, C.SPH_OUT_BF16, 1, 0)
    assert fam == C.SPH_KERNEL_ROW
    fam, _ = C.sphericart_launch_info(30, C.SPH_F32, C.SPH_OUT_SAME, 1, 0)
    assert fam == C.SPH_KERNEL_ROW
    fam, _ = C.sphericart_launch_info(64, C.SPH_F32, C.SPH_OUT_SAME, 1, 0)
    assert fam == C.SPH_KERNEL_SLICE
    fam, _ = C.sphericart_launch_info(64, C.SPH_F32, C.SPH_OUT_BF16, 1, 0)
    assert fam == C.SPH_KERNEL_DEGREE
    fam, _ = C.sphericart_launch_info(30, C.SPH_F64, C.SPH_OUT_SAME, 1, 1)
    assert fam == C.SPH_KERNEL_SLICE  # Hessians


def _err(fn, *args):
    with pytest.raises(C.SphericartError) as ei:
        fn(*args)
    return ei.value.code


def test_argument_errors_before_any_cuda_call():
    none = None
    launch = None
    # n < 0
    assert _err(C.sphericart_compute_ex, 16, -1, 8, 0, 0, 0, 0, 0, launch, 16, none, none, none) == C.SPH_EINVAL
    # l_max out of range
    assert _err(C.sphericart_compute_ex, 16, 4, -1, 0, 0, 0, 0, 0, launch, 16, none, none, none) == C.SPH_EINVAL
    assert _err(C.sphericart_compute_ex, 16, 4, 129, 0, 0, 0, 0, 0, launch, 16, none, none, none) == C.SPH_EINVAL
    # bad enums
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 7, 0, 0, 0, launch, 16, none, none, none) == C.SPH_EINVAL
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 0, 9, 0, 0, launch, 16, none, none, none) == C.SPH_EINVAL
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 0, 0, 5, 0, launch, 16, none, none, none) == C.SPH_EINVAL
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 0, 0, 0, 9, launch, 16, none, none, none) == C.SPH_EINVAL
    # ddsph without dsph
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 0, 0, 0, 0, launch, 16, none, 32, none) == C.SPH_EINVAL
    # bf16 with FP64 arithmetic; POINT beyond its l_max, with bf16 Hessians, or mixed Q
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 1, 1, 0, 0, launch, 16, none, none, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_compute_ex, 16, 4, 17, 0, 0, 0, 0, 1, launch, 16, none, none, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 0, 1, 0, 1, launch, 16, 32, 48, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 0, 0, 1, 1, launch, 16, none, none, none) == C.SPH_EUNSUPPORTED
    # DEGREE families: no Hessians, no backward
    for k in (C.SPH_KERNEL_DEGREE, C.SPH_KERNEL_DEGREE_DOWN):
        assert _err(C.sphericart_compute_ex, 16, 4, 30, 0, 0, 0, 0, k, launch, 16, 32, 48, none) == C.SPH_EUNSUPPORTED
        assert _err(C.sphericart_backward, 16, 16, 4, 20, 0, 0, k, launch, 16, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 0, 0, 0, 7, launch, 16, none, none, none) == C.SPH_EINVAL
    # e3nn convention: bad normalization / dtype / l_max, NULL workspace
    lib = C.lib()
    assert lib.sphericart_compute_e3nn(16, 4, 8, 0, 3, 0, 16, 16, None, None) == C.SPH_EINVAL
    assert lib.sphericart_compute_e3nn(16, 4, 8, 0, 0, 2, 16, 16, None, None) == C.SPH_EINVAL
    assert lib.sphericart_compute_e3nn(16, 4, 129, 0, 0, 0, 16, 16, None, None) == C.SPH_EINVAL
    assert lib.sphericart_compute_e3nn(16, 4, 8, 0, 0, 0, None, 16, None, None) == C.SPH_EINVAL
    assert lib.sphericart_compute_e3nn(16, 0, 8, 0, 0, 0, None, None, None, None) == C.SPH_OK
    # POINT_HC (hard-coded l <= 3 + recursion): l_max <= 8, no Hessians, no bf16 storage
    hc = C.SPH_KERNEL_POINT_HC
    assert _err(C.sphericart_compute_ex, 16, 4, 9, 0, 0, 0, 0, hc, launch, 16, none, none, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 0, 1, 0, hc, launch, 16, none, none, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 0, 0, 0, hc, launch, 16, 32, 32, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 0, 0, 1, hc, launch, 16, none, none, none) == C.SPH_EUNSUPPORTED
    # ROW: FP32 arithmetic, 16 <= l_max <= 63; backward (FP32) but no double backward
    R = C.SPH_KERNEL_ROW
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 0, 0, 0, R, launch, 16, 32, none, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_compute_ex, 16, 4, 64, 0, 0, 0, 0, R, launch, 16, 32, none, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_compute_ex, 16, 4, 20, 0, 1, 0, 0, R, launch, 16, 32, none, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_compute_ex, 16, 4, 20, 0, 0, 0, 1, R, launch, 16, 32, none, none) == C.SPH_EUNSUPPORTED
    # (ROW Hessians: FP32 storage only)
    assert _err(C.sphericart_compute_ex, 16, 4, 20, 0, 0, 1, 0, R, launch, 16, 32, 48, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_backward, 16, 16, 4, 15, 0, 0, R, launch, 16, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_backward, 16, 16, 4, 20, 0, 1, R, launch, 16, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_double_backward, 16, 16, 16, 4, 20, 0, 0, R, launch, 16, 16, none) == C.SPH_EUNSUPPORTED
    assert C.sphericart_max_l(C.SPH_F32, C.SPH_Q_NATIVE, R) == 63
    # NULL required pointers
    assert _err(C.sphericart_compute_ex, none, 4, 8, 0, 0, 0, 0, 0, launch, 16, none, none, none) == C.SPH_EINVAL
    assert _err(C.sphericart_compute_ex, 16, 4, 8, 0, 0, 0, 0, 0, launch, none, none, none, none) == C.SPH_EINVAL
    # misaligned element pointers
    assert _err(C.sphericart_compute_ex, 18, 4, 8, 0, 0, 0, 0, 0, launch, 16, none, none, none) == C.SPH_EINVAL
    # backward / double backward
    assert _err(C.sphericart_backward, 16, 16, -2, 6, 0, 0, 0, launch, 16, none) == C.SPH_EINVAL
    assert _err(C.sphericart_backward, 16, none, 4, 6, 0, 0, 0, launch, 16, none) == C.SPH_EINVAL
    assert _err(C.sphericart_backward, 16, 16, 4, 6, 0, 0, 0, launch, none, none) == C.SPH_EINVAL
    assert _err(C.sphericart_backward, 16, 16, 4, 20, 0, 0, 1, launch, 16, none) == C.SPH_EUNSUPPORTED
    assert _err(C.sphericart_double_backward, 16, 16, none, 4, 6, 0, 0, 0, launch, 16, 16, none) == C.SPH_EINVAL
    # batch plan mode
    import ctypes

    arr = (C.sph_batch_set * 1)()
    arr[0] = C.sph_batch_set(16, 16, None, 4, 3, 0)
    h = ctypes.c_void_p()
    assert C.lib().sphericart_batch_plan_create_ex(arr, 1, None, 7, ctypes.byref(h)) == C.SPH_EINVAL
    assert "mode" in C.last_error()
    # host table
    with pytest.raises(C.SphericartError):
        C.sphericart_host_table(200, 0)
    assert "l_max" in C.last_error() or "host_table" in C.last_error()


def test_zero_points_is_a_noop():
    # n == 0 returns OK without a device and without touching pointers.
    C.sphericart_compute_ex(None, 0, 8, 0, 0, 0, 0, 0, None, None, None, None, None)
    C.sphericart_backward(None, None, 0, 8, 0, 0, 0, None, None, None)
    C.sphericart_double_backward(None, None, None, 0, 8, 0, 0, 0, None, None, None, None)


def test_compute_without_device_reports_cuda_error():
    import torch

    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(C.SphericartError) as ei:
        C.sphericart_compute_ex(16, 4, 8, 0, 0, 0, 0, 0, None, 16, None, None, None)
    assert ei.value.code == C.SPH_ECUDA


def test_product_path_has_no_cpu_fallback():
    """The tensor API rejects CPU tensors instead of computing elsewhere."""
    import torch

    from paper_2302_08381_gb300 import api

    with pytest.raises(ValueError):
        api.spherical_harmonics(torch.zeros(4, 3), 4)
    # the package never imports the oracle
    import paper_2302_08381_gb300 as pkg

    src_dir = os.path.dirname(pkg.__file__)
    for name in os.listdir(src_dir):
        if name.endswith(".py"):
            text = open(os.path.join(src_dir, name)).read()
            assert "import oracle" not in text and "from oracle" not in text, name


def test_fma_peak_argument_errors():
    assert _err(C.sphericart_fma_peak, 7, None, 3) == C.SPH_EINVAL
    assert _err(C.sphericart_fma_peak, C.SPH_F32, None, 0) == C.SPH_EINVAL


def test_point_default_shapes():
    """The POINT default (no shape given, none tuned): FP32 fills ~48 KB
    tiles with several warps per block; FP64, bound by the FP64 pipe, fills
    up to 32 points within 74 KB with one warp per block."""
    fam, s = C.sphericart_launch_info(8, C.SPH_F32, C.SPH_OUT_SAME, 1, 0)
    assert fam == C.SPH_KERNEL_POINT and (s.points_per_tile, s.warps_per_block, s.blocks_per_sm) == (32, 4, 16)
    # FP64 with gradients up to l_max 8 runs the hybrid (hard-coded l <= 3) on the same shapes
    fam, s = C.sphericart_launch_info(8, C.SPH_F64, C.SPH_OUT_SAME, 1, 0)
    assert fam == C.SPH_KERNEL_POINT_HC and (s.points_per_tile, s.warps_per_block, s.blocks_per_sm) == (28, 1, 16)
    assert C.sphericart_launch_info(3, C.SPH_F64, C.SPH_OUT_SAME, 0, 0)[0] == C.SPH_KERNEL_POINT_HC
    assert C.sphericart_launch_info(4, C.SPH_F64, C.SPH_OUT_SAME, 0, 0)[0] == C.SPH_KERNEL_POINT
    assert C.sphericart_launch_info(9, C.SPH_F64, C.SPH_OUT_SAME, 1, 0)[0] == C.SPH_KERNEL_DEGREE  # gradients from 9
    assert C.sphericart_launch_info(3, C.SPH_F32, C.SPH_OUT_SAME, 1, 0)[0] == C.SPH_KERNEL_POINT
    assert 28 * 4 * 81 * 8 <= 74 * 1024 < 30 * 4 * 81 * 8  # the largest even tile inside 74 KB
    _, s = C.sphericart_launch_info(8, C.SPH_F64, C.SPH_OUT_SAME, 0, 0)
    assert (s.points_per_tile, s.warps_per_block) == (32, 1)
    fam, s = C.sphericart_launch_info(11, C.SPH_F64, C.SPH_OUT_SAME, 1, 0)  # DEGREE from l_max 9 with gradients
    assert fam == C.SPH_KERNEL_DEGREE and s.lanes_per_point == 2
