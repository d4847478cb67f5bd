"""The no-allocation batch entry point.

Some callers cannot allocate device memory (their memory belongs to a fixed
arena or a framework allocator, or they cannot afford the synchronisation a
cudaMalloc implies). sphericart_batch_compute_noalloc serves them: it keeps
its descriptors in a static device array of the library. This test calls it
through the C-ABI twice in a row, with different batches, and checks both
results against the plan-based batch entry point and, at every point, against
the FP64 oracle. It lives in its own file, collected last, and passes alone
in a fresh process as well as after the rest of the suite.
"""



import numpy as np
import pytest
import torch

import oracle
from paper_2302_08381_gb300 import _capi as C
from paper_2302_08381_gb300 import api, inputs
from parity_utils import F32_GRAD, F32_VAL, assert_grads, assert_values, grad_scale, value_scale

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _batch(nsets, choices, nmin, nmax, seed):
    sizes, lmax, xyz = inputs.ragged_sets(nsets, choices, nmin, nmax, seed=seed)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    xt = torch.from_numpy(xyz).to(DEV)
    return [xt[offs[i]:offs[i + 1]] for i in range(nsets)], [int(v) for v in lmax], xyz, offs


def _noalloc(xs, ls, normalized=False):
    """Outputs allocated here by torch (the caller owns them), then one call."""
    outs = []
    arr = (C.sph_batch_set * len(xs))()
    for i, (x, L) in enumerate(zip(xs, ls)):
        K = (L + 1) ** 2
        s = torch.full((x.shape[0], K), float("nan"), device=DEV)
        d = torch.full((x.shape[0], 3, K), float("nan"), device=DEV)
        outs.append((s, d))
        arr[i] = C.sph_batch_set(x.data_ptr(), s.data_ptr(), d.data_ptr(), x.shape[0], L, 1 if normalized else 0)
    code = C.lib().sphericart_batch_compute_noalloc(arr, len(xs), None, torch.cuda.current_stream().cuda_stream)
    C.check("sphericart_batch_compute_noalloc", code)
    return outs


def _assert_close(outs, plan, xyz, offs, ls, normalized):
    torch.cuda.synchronize()
    for i, L in enumerate(ls):
        s, d = outs[i]
        p = xyz[offs[i]:offs[i + 1]].astype(np.float64)
        if p.shape[0] == 0:
            continue
        dv = (s - plan.sph[i]).abs().double().cpu().numpy() / value_scale(p, L, normalized)
        dg = (d - plan.dsph[i]).abs().double().cpu().numpy() / grad_scale(p, L, normalized)[:, None, :]
        assert np.all(np.isfinite(dv)) and np.all(np.isfinite(dg)), i
        assert dv.max() < 1e-6 and dg.max() < 1e-6, (i, L, dv.max(), dg.max())
        rv, rg = oracle.spherical_harmonics_grad(p, L, normalized)
        assert_values(s.double().cpu().numpy(), p, L, normalized, F32_VAL, ref=rv)
        assert_grads(d.double().cpu().numpy(), p, L, normalized, F32_GRAD, ref=rg)


def test_noalloc_batch_matches_plan_on_two_calls_in_a_row():
    xs1, ls1, xyz1, offs1 = _batch(48, [3, 6, 8, 12], 100, 20000, seed=500)
    xs2, ls2, xyz2, offs2 = _batch(17, list(range(0, 17)), 1, 5000, seed=501)
    # the no-allocation entry point runs the single-launch kernel: compare with
    # plans of the same mode (bitwise-equal shapes) and with the oracle
    plan1 = api.BatchPlan(xs1, ls1, mode="one_launch")
    plan2 = api.BatchPlan(xs2, ls2, normalized=True, mode="one_launch")
    plan1.execute()
    plan2.execute()
    out1 = _noalloc(xs1, ls1)
    out2 = _noalloc(xs2, ls2, normalized=True)  # second call, different batch
    _assert_close(out1, plan1, xyz1, offs1, ls1, False)
    _assert_close(out2, plan2, xyz2, offs2, ls2, True)
    plan1.close()
    plan2.close()


def test_noalloc_rejects_more_sets_than_the_static_capacity():
    x = torch.zeros((1, 3), device=DEV)
    s = torch.zeros((1, 1), device=DEV)
    arr = (C.sph_batch_set * 4097)()
    for i in range(4097):
        arr[i] = C.sph_batch_set(x.data_ptr(), s.data_ptr(), None, 1, 0, 0)
    code = C.lib().sphericart_batch_compute_noalloc(arr, 4097, None, torch.cuda.current_stream().cuda_stream)
    assert code == C.SPH_EINVAL
    assert "4096" in C.last_error()


def test_noalloc_refuses_a_capturing_stream():
    """Its work list is staged in host memory that the next call overwrites,
    so a call on a stream under capture is refused and enqueues nothing."""
    xs, ls, _, _ = _batch(4, [3, 6], 10, 200, seed=502)
    _noalloc(xs, ls)  # set-up happens on this eager first call
    torch.cuda.synchronize()
    arr = (C.sph_batch_set * len(xs))()
    outs = [torch.zeros((x.shape[0], (L + 1) ** 2), device=DEV) for x, L in zip(xs, ls)]
    for i, (x, L) in enumerate(zip(xs, ls)):
        arr[i] = C.sph_batch_set(x.data_ptr(), outs[i].data_ptr(), None, x.shape[0], L, 0)
    marker = torch.zeros(1, device=DEV)
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    codes = []
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            marker.add_(1.0)  # the graph holds one node of its own
            codes.append(C.lib().sphericart_batch_compute_noalloc(arr, len(xs), None, st.cuda_stream))
    torch.cuda.current_stream().wait_stream(st)
    assert codes == [C.SPH_EINVAL]
    assert "captured" in C.last_error()
    g.replay()
    torch.cuda.synchronize()
    assert marker.item() == 1.0
    assert all(torch.count_nonzero(o).item() == 0 for o in outs)
