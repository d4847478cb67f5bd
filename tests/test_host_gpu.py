"""Forward from host buffers through the chunked pipeline: identical to the
device path for every chunking, ragged tails and consecutive calls."""

import numpy as np
import pytest
import torch

from paper_2302_08381_gb300 import _capi as C
from paper_2302_08381_gb300 import api, inputs
from parity_utils import F32_GRAD, F32_VAL, assert_grads, assert_values

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.mark.parametrize("pinned", [True, False])
def test_host_pipeline_matches_device_path(pinned):
    n = 100_003
    for l_max in (3, 8):
        x_np = inputs.shell_points(n, 0.5, 5.0, seed=700 + l_max)
        xh = torch.from_numpy(x_np)
        if pinned:
            xh = xh.pin_memory()
        ref_v, ref_g = api.spherical_harmonics(xh.to(DEV), l_max, gradients=True)
        for chunk in (0, 32, 4096, 30_000, 1 << 20):
            v, g = api.spherical_harmonics_host(xh, l_max, gradients=True, chunk_points=chunk)
            v2 = api.spherical_harmonics_host(xh, l_max, chunk_points=chunk)  # second call, values only
            torch.cuda.synchronize()
            assert torch.equal(v, ref_v.cpu()) and torch.equal(g, ref_g.cpu()), (l_max, chunk)
            assert torch.equal(v2, ref_v.cpu())
        k = 500
        assert_values(v[:k].double().numpy(), x_np[:k].astype(np.float64), l_max, False, F32_VAL)
        assert_grads(g[:k].double().numpy(), x_np[:k].astype(np.float64), l_max, False, F32_GRAD)


def test_host_pipeline_small_workspace_and_errors():
    n, l_max = 5000, 6
    xh = torch.from_numpy(inputs.normal_points(n, seed=710).astype(np.float32)).pin_memory()
    ref = api.spherical_harmonics(xh.to(DEV), l_max).cpu()
    K = 49
    ws = torch.empty(2 * 64 * 4 * (3 + K) + 2048, dtype=torch.uint8, device=DEV)  # forces 64-point chunks
    v = api.spherical_harmonics_host(xh, l_max, workspace=ws)
    torch.cuda.synchronize()
    assert torch.equal(v, ref)
    tiny = torch.empty(64, dtype=torch.uint8, device=DEV)
    with pytest.raises(C.SphericartError) as ei:
        api.spherical_harmonics_host(xh, l_max, workspace=tiny)
    assert ei.value.code == C.SPH_EINVAL
