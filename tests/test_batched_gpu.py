"""sphericart_compute_batched: ragged point sets from a DEVICE descriptor
array in one persistent launch, checked at every point against the oracle,
against the per-set forward, under CUDA-graph replay with descriptors
rewritten on the GPU between replays, and with invalid descriptors."""

import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2302_08381_gb300 import _capi as C
from paper_2302_08381_gb300 import api, inputs
from parity_utils import F32_GRAD, F32_VAL, assert_grads, assert_values, grad_scale, value_scale

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _sets(nsets, choices, nmin, nmax, seed):
    sizes, lmax, xyz = inputs.ragged_sets(nsets, choices, nmin, nmax, seed=seed)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    xt = torch.from_numpy(xyz).to(DEV)
    return [xt[offs[i]:offs[i + 1]] for i in range(nsets)], [int(v) for v in lmax], xyz, offs


@pytest.mark.parametrize("gradients", [True, False])
@pytest.mark.parametrize("normalized", [False, True])
def test_compute_batched_every_lmax_against_oracle(gradients, normalized):
    xs, ls, xyz, offs = _sets(57, list(range(0, 17)), 1, 2500, seed=700)
    for i in (5, 30):  # empty sets
        xs[i] = xs[i][:0]
    sph, dsph = api.compute_batched(xs, ls, normalized=normalized, gradients=gradients)
    torch.cuda.synchronize()
    assert api.device_status() == 0
    for i, L in enumerate(ls):
        p = xyz[offs[i]:offs[i + 1]].astype(np.float64)
        if xs[i].shape[0] == 0:
            assert sph[i].shape[0] == 0
            continue
        if gradients:
            rv, rg = oracle.spherical_harmonics_grad(p, L, normalized)
            assert_grads(dsph[i].double().cpu().numpy(), p, L, normalized, F32_GRAD, ref=rg)
        else:
            rv = oracle.spherical_harmonics(p, L, normalized)
        assert_values(sph[i].double().cpu().numpy(), p, L, normalized, F32_VAL, ref=rv)


def test_compute_batched_equals_single_set_forward():
    """Same recursion as the single-set POINT kernels (separately compiled):
    equal up to a few FP32 roundings on the l-block scales."""
    xs, ls, xyz, offs = _sets(64, [0, 1, 3, 6, 8, 12, 16], 1, 40000, seed=701)
    sph, dsph = api.compute_batched(xs, ls)
    for i, (x, L) in enumerate(zip(xs, ls)):
        v, g = api.spherical_harmonics(x, L, gradients=True)
        torch.cuda.synchronize()
        p = xyz[offs[i]:offs[i + 1]].astype(np.float64)
        dv = (sph[i] - v).abs().double().cpu().numpy() / value_scale(p, L, False)
        dg = (dsph[i] - g).abs().double().cpu().numpy() / grad_scale(p, L, False)[:, None, :]
        assert dv.max() < 5e-6 and dg.max() < 5e-6, (i, L, dv.max(), dg.max())


def test_compute_batched_more_sets_than_one_launch_takes():
    """2,100 sets run as two launches (2,048 + 52 sets)."""
    xs, ls, xyz, offs = _sets(2100, [2, 5, 9], 1, 60, seed=702)
    sph, dsph = api.compute_batched(xs, ls)
    torch.cuda.synchronize()
    allv = torch.cat([s.reshape(-1) for s in sph]).cpu().numpy()
    assert np.all(np.isfinite(allv))
    for i in list(range(0, 2100, 97)) + [2047, 2048, 2099]:
        p = xyz[offs[i]:offs[i + 1]].astype(np.float64)
        rv, rg = oracle.spherical_harmonics_grad(p, ls[i])
        assert_values(sph[i].double().cpu().numpy(), p, ls[i], False, F32_VAL, ref=rv)
        assert_grads(dsph[i].double().cpu().numpy(), p, ls[i], False, F32_GRAD, ref=rg)


def test_compute_batched_graph_replay_reads_descriptors_from_device():
    """A captured call reads the descriptor array at every replay: rewriting
    it on the GPU (other sets, other sizes) changes what the replay computes."""
    xs, ls, xyz, offs = _sets(30, [3, 6, 8, 12], 100, 5000, seed=703)
    outs = [(torch.zeros((x.shape[0], (L + 1) ** 2), device=DEV), torch.zeros((x.shape[0], 3, (L + 1) ** 2),
                                                                              device=DEV)) for x, L in zip(xs, ls)]
    desc = api.batch_descriptors(xs, ls, [o[0] for o in outs], [o[1] for o in outs])
    # descriptors of the first 10 sets only, the rest of the array with n = 0
    desc_a = api.batch_descriptors(xs[:10] + [x[:0] for x in xs[10:]], ls,
                                   [o[0] for o in outs], [o[1] for o in outs])
    live = torch.empty_like(desc)
    live.copy_(desc_a)
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    C.check("warm-up", C.lib().sphericart_compute_batched(live.data_ptr(), len(xs), C.SPH_BATCHED_GRADIENTS,
                                                          torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    for s, d in outs:
        s.zero_()
        d.zero_()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        with torch.cuda.graph(g, stream=stream):
            C.check("capture", C.lib().sphericart_compute_batched(live.data_ptr(), len(xs), C.SPH_BATCHED_GRADIENTS,
                                                                  stream.cuda_stream))
    torch.cuda.current_stream().wait_stream(stream)
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.count_nonzero(outs[i][0]).item() > 0 for i in range(10))
    assert all(torch.count_nonzero(outs[i][0]).item() == 0 for i in range(10, 30))
    live.copy_(desc)  # every set now
    g.replay()
    torch.cuda.synchronize()
    for i, L in enumerate(ls):
        p = xyz[offs[i]:offs[i + 1]].astype(np.float64)
        rv, rg = oracle.spherical_harmonics_grad(p, L)
        assert_values(outs[i][0].double().cpu().numpy(), p, L, False, F32_VAL, ref=rv)
        assert_grads(outs[i][1].double().cpu().numpy(), p, L, False, F32_GRAD, ref=rg)


def test_compute_batched_skips_invalid_descriptors_and_flags_them():
    xs, ls, xyz, offs = _sets(6, [3, 6], 50, 400, seed=704)
    sph = [torch.full((x.shape[0], (L + 1) ** 2), -3.0, device=DEV) for x, L in zip(xs, ls)]
    dsph = [torch.full((x.shape[0], 3, (L + 1) ** 2), -3.0, device=DEV) for x, L in zip(xs, ls)]
    bad_l = list(ls)
    bad_l[2] = 17  # beyond the POINT kernels
    desc = api.batch_descriptors(xs, bad_l, sph, dsph)
    # set 4: no dsph although the call asks for gradients
    arr = (C.sph_batch_set * 1)()
    arr[0] = C.sph_batch_set(xs[4].data_ptr(), sph[4].data_ptr(), None, xs[4].shape[0], ls[4], 0)
    desc[4] = torch.frombuffer(bytearray(arr), dtype=torch.uint8).to(DEV)
    assert api.device_status() == 0
    C.check("batched", C.lib().sphericart_compute_batched(desc.data_ptr(), len(xs), C.SPH_BATCHED_GRADIENTS,
                                                          torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert api.device_status() == 2
    for i in (2, 4):
        assert torch.all(sph[i] == -3.0)
    for i in (0, 1, 3, 5):
        p = xyz[offs[i]:offs[i + 1]].astype(np.float64)
        assert_values(sph[i].double().cpu().numpy(), p, ls[i], False, F32_VAL)


def test_compute_batched_host_side_errors():
    lib = C.lib()
    st = torch.cuda.current_stream().cuda_stream
    assert lib.sphericart_compute_batched(None, 0, 0, st) == C.SPH_OK
    assert lib.sphericart_compute_batched(None, -1, 0, st) == C.SPH_EINVAL
    assert lib.sphericart_compute_batched(None, 3, 0, st) == C.SPH_EINVAL
    x = torch.zeros(16, dtype=torch.uint8, device=DEV)
    assert lib.sphericart_compute_batched(x.data_ptr(), 1, 4, st) == C.SPH_EINVAL
    host = (C.sph_batch_set * 2)()  # pageable host memory
    assert lib.sphericart_compute_batched(ctypes.addressof(host), 2, 0, st) == C.SPH_EINVAL
    assert "device" in C.last_error()


def test_plans_and_batched_take_mixed_flags():
    """A plan whose sets mix gradients / normalized runs one launch per flag
    combination (one-launch mode) or per class (default)."""
    xs, ls, xyz, offs = _sets(24, [2, 4, 7, 10], 10, 900, seed=705)
    outs, flags = [], []
    arr = (C.sph_batch_set * len(xs))()
    for i, (x, L) in enumerate(zip(xs, ls)):
        grad, norm = i % 2 == 0, (i // 2) % 2 == 1
        K = (L + 1) ** 2
        s = torch.zeros((x.shape[0], K), device=DEV)
        d = torch.zeros((x.shape[0], 3, K), device=DEV) if grad else None
        outs.append((s, d))
        flags.append((grad, norm))
        arr[i] = C.sph_batch_set(x.data_ptr(), s.data_ptr(), d.data_ptr() if grad else None, x.shape[0], L, int(norm))
    for mode in (C.SPH_BATCH_ONE_LAUNCH, C.SPH_BATCH_PER_LMAX):
        plan = ctypes.c_void_p()
        C.check("plan", C.lib().sphericart_batch_plan_create_ex(arr, len(xs), None, mode, ctypes.byref(plan)))
        C.check("exec", C.lib().sphericart_batch_execute(plan, torch.cuda.current_stream().cuda_stream))
        torch.cuda.synchronize()
        for i, L in enumerate(ls):
            p = xyz[offs[i]:offs[i + 1]].astype(np.float64)
            grad, norm = flags[i]
            assert_values(outs[i][0].double().cpu().numpy(), p, L, norm, F32_VAL)
            if grad:
                assert_grads(outs[i][1].double().cpu().numpy(), p, L, norm, F32_GRAD)
            outs[i][0].zero_()
        C.lib().sphericart_batch_plan_destroy(plan)
