"""Autotuner: picks a valid shape, installs it, results unchanged; the tuned
table round-trips through its text export keyed by GPU name."""

import numpy as np
import pytest
import torch

from paper_2302_08381_gb300 import _capi as C
from paper_2302_08381_gb300 import api, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(autouse=True)
def _restore_defaults():
    """Tuned shapes are process-wide: drop them after each test, so that later
    tests see the library defaults whatever the test order."""
    yield
    C.sphericart_tune_clear()


def test_autotune_installs_a_valid_shape_with_identical_results():
    n, L = 200_003, 8
    x = torch.from_numpy(inputs.shell_points(n, 0.5, 5.0, seed=400)).to(DEV)
    ref_v, ref_g = api.spherical_harmonics(x, L, gradients=True, launch=C.make_launch(32, 1, 0, 0))
    sph = torch.empty_like(ref_v)
    dsph = torch.empty_like(ref_g)
    best, ms = C.sphericart_autotune(
        x.data_ptr(), n, L, 0, C.SPH_F32, C.SPH_OUT_SAME, sph.data_ptr(), dsph.data_ptr(),
        torch.cuda.current_stream().cuda_stream, 2,
    )
    assert ms > 0 and 1 <= best.points_per_tile <= 32 and 1 <= best.warps_per_block <= 8
    fam, shape = C.sphericart_launch_info(L, C.SPH_F32, C.SPH_OUT_SAME, 1, 0)
    assert fam == C.SPH_KERNEL_POINT
    assert (shape.points_per_tile, shape.warps_per_block, shape.blocks_per_sm) == (
        best.points_per_tile, best.warps_per_block, best.blocks_per_sm)
    v, g = api.spherical_harmonics(x, L, gradients=True)  # uses the tuned shape
    torch.cuda.synchronize()
    assert torch.equal(v, ref_v) and torch.equal(g, ref_g)
    text = C.sphericart_tune_export()
    assert f" {L} 0 0 1 {best.points_per_tile} " in text
    name = text.split()[0]
    other = text.replace(name, "SOME_OTHER_GPU")
    assert C.sphericart_tune_import(other) == 0
    assert C.sphericart_tune_import(text) >= 1


def test_batch_autotune_returns_a_plan_shape():
    sizes, lmax, xyz = inputs.ragged_sets(24, [3, 6, 8, 12], 1000, 20000, seed=401)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    xt = torch.from_numpy(xyz).to(DEV)
    xs = [xt[offs[i]:offs[i + 1]] for i in range(len(sizes))]
    plan = api.BatchPlan(xs, [int(v) for v in lmax])
    import ctypes

    arr = (C.sph_batch_set * len(xs))()
    for i, x in enumerate(xs):
        arr[i] = C.sph_batch_set(x.data_ptr(), plan.sph[i].data_ptr(), plan.dsph[i].data_ptr(), x.shape[0],
                                 int(lmax[i]), 0)
    best = C.sph_launch()
    ms = ctypes.c_float()
    C.check("sphericart_batch_autotune", C.lib().sphericart_batch_autotune(
        arr, len(xs), torch.cuda.current_stream().cuda_stream, 2, ctypes.byref(best), ctypes.byref(ms)))
    # a per-warp budget, or (0, 0): every l_max class on its single-set POINT shape
    assert ms.value > 0 and (best.points_per_tile > 0 or best.warps_per_block == 0)
    tuned = api.BatchPlan(xs, [int(v) for v in lmax], launch=best)
    tuned.execute()
    plan.execute()
    torch.cuda.synchronize()
    for a, b in zip(tuned.sph, plan.sph):
        assert torch.allclose(a, b, rtol=1e-6, atol=1e-6)


def test_tuning_save_and_load_roundtrip(tmp_path):
    x = torch.from_numpy(inputs.shell_points(50_000, 0.5, 5.0, seed=402)).to(DEV)
    shape, ms = api.autotune(x, 6, reps=1)
    assert ms > 0 and shape["points_per_tile"] > 0
    path = tmp_path / "tune.txt"
    api.save_tuning(str(path))
    assert api.load_tuning(str(path)) >= 1


def test_fma_peak_is_measured_and_fp32_outruns_fp64():
    """The FMA-throughput probe gives positive rates below the nominal
    per-SM ceilings (FP32: 128 FMA per clock per SM at the maximum clock)."""
    stream = torch.cuda.current_stream().cuda_stream
    f32 = C.sphericart_fma_peak(C.SPH_F32, stream, 2)
    f64 = C.sphericart_fma_peak(C.SPH_F64, stream, 2)
    props = torch.cuda.get_device_properties(0)
    ceiling = props.multi_processor_count * 128 * 2 * 2.2e9 / 1e12  # TFLOP/s at 2.2 GHz
    assert 0 < f64 < f32 < ceiling, (f32, f64, ceiling)
