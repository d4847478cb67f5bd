"""Ragged persistent batch: every set equals its own single-set launch
(within FP32 rounding) and, at every point, the oracle; the 512-set serving
workload is checked at every point too."""

import numpy as np
import pytest
import torch

import full_parity
import oracle
from paper_2302_08381_gb300 import api, inputs
from parity_utils import F32_GRAD, F32_VAL, assert_grads, assert_values, grad_scale, value_bound, value_scale

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _sets(nsets, choices, nmin, nmax, seed):
    sizes, lmax, xyz = inputs.ragged_sets(nsets, choices, nmin, nmax, seed=seed)
    offs = np.concatenate([[0], np.cumsum(sizes)])
    xt = torch.from_numpy(xyz).to(DEV)
    return [xt[offs[i]:offs[i + 1]] for i in range(nsets)], [int(v) for v in lmax], xyz, offs


@pytest.mark.parametrize("mode", ["per_lmax", "one_launch"])
@pytest.mark.parametrize("normalized", [False, True])
def test_batch_matches_single_launch_and_oracle(normalized, mode):
    xs, ls, xyz, offs = _sets(40, list(range(0, 17)), 1, 3000, seed=300)
    plan = api.BatchPlan(xs, ls, normalized=normalized, mode=mode)
    plan.execute()
    torch.cuda.synchronize()
    for i, (x, L) in enumerate(zip(xs, ls)):
        v, g = api.spherical_harmonics(x, L, normalized, gradients=True)
        torch.cuda.synchronize()
        p = xyz[offs[i]:offs[i + 1]].astype(np.float64)
        # Same recursion, separately compiled kernels (different FMA
        # contraction): equal up to a few FP32 roundings on the l-block scales.
        if p.shape[0]:
            dv = (plan.sph[i] - v).abs().double().cpu().numpy() / value_scale(p, L, normalized)
            dg = (plan.dsph[i] - g).abs().double().cpu().numpy() / grad_scale(p, L, normalized)[:, None, :]
            assert dv.max() < 5e-6 and dg.max() < 5e-6, (i, L, dv.max(), dg.max())
        if p.shape[0]:
            assert_values(plan.sph[i].double().cpu().numpy(), p, L, normalized, F32_VAL)
            assert_grads(plan.dsph[i].double().cpu().numpy(), p, L, normalized, F32_GRAD)
    n, t = plan.info()
    assert n == sum(x.shape[0] for x in xs) and t > 0
    plan.close()


@pytest.mark.parametrize("mode", ["per_lmax", "one_launch"])
def test_batch_values_only_and_empty_sets(mode):
    xs, ls, xyz, offs = _sets(12, [3, 6, 8, 12], 1, 500, seed=301)
    xs[3] = xs[3][:0]
    plan = api.BatchPlan(xs, ls, gradients=False, mode=mode)
    plan.execute()
    torch.cuda.synchronize()
    for i, (x, L) in enumerate(zip(xs, ls)):
        assert plan.dsph[i] is None
        if x.shape[0]:
            ref = oracle.spherical_harmonics(x.double().cpu().numpy(), L)
            assert_values(plan.sph[i].double().cpu().numpy(), x.double().cpu().numpy(), L, False, F32_VAL, ref=ref)


@pytest.mark.parametrize("mode", ["per_lmax", "one_launch"])
def test_batch_graph_capture_replay(mode):
    xs, ls, _, _ = _sets(64, [3, 6, 8, 12], 1000, 20000, seed=302)
    plan = api.BatchPlan(xs, ls, mode=mode)
    plan.execute()
    torch.cuda.synchronize()
    want = [s.clone() for s in plan.sph]
    for s in plan.sph:
        s.zero_()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            plan.execute()
    torch.cuda.current_stream().wait_stream(st)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(plan.sph, want):
        assert torch.equal(a, b)


def test_batch_modes_agree():
    """One launch per l_max class and one launch for all sets compute the same
    outputs (the same recursion in separately compiled kernels: equal up to a
    few FP32 roundings on the l-block scales)."""
    xs, ls, xyz, offs = _sets(80, [0, 2, 3, 6, 8, 12, 16], 1, 6000, seed=303)
    a = api.BatchPlan(xs, ls, mode="per_lmax")
    b = api.BatchPlan(xs, ls, mode="one_launch")
    a.execute()
    b.execute()
    torch.cuda.synchronize()
    for i, L in enumerate(ls):
        p = xyz[offs[i]:offs[i + 1]].astype(np.float64)
        if not p.shape[0]:
            continue
        dv = (a.sph[i] - b.sph[i]).abs().double().cpu().numpy() / value_scale(p, L, False)
        dg = (a.dsph[i] - b.dsph[i]).abs().double().cpu().numpy() / grad_scale(p, L, False)[:, None, :]
        assert dv.max() < 5e-6 and dg.max() < 5e-6, (i, L, dv.max(), dg.max())
    a.close()
    b.close()


@pytest.mark.parametrize("mode", ["per_lmax", "one_launch"])
def test_batch_serving_workload_full(mode):
    """512 sets, sizes log-uniform in [1,000, 200,000], l_max from {3, 6, 8, 12},
    N(0,1) FP32 points (seed 5), values + gradients in the batch launch the
    benchmark times: every point of every set against the oracle, one l_max
    class at a time."""
    xs, ls, xyz, offs = _sets(512, [3, 6, 8, 12], 1000, 200000, seed=5)
    plan = api.BatchPlan(xs, ls, mode=mode)
    plan.execute()
    torch.cuda.synchronize()
    for L in sorted(set(ls)):
        ids = [i for i, v in enumerate(ls) if v == L]
        p = np.concatenate([xyz[offs[i]:offs[i + 1]] for i in ids]).astype(np.float64)
        s = torch.cat([plan.sph[i] for i in ids]).cpu().numpy()
        d = torch.cat([plan.dsph[i] for i in ids]).cpu().numpy()
        ev, eg, finite = full_parity.forward_errors(p, L, False, s, d)
        assert finite
        assert np.all(ev <= value_bound(L, F32_VAL)), (L, ev)
        assert np.all(eg <= F32_GRAD), (L, eg)
        del s, d
    plan.close()
