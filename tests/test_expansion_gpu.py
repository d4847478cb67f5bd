"""Fused radial expansion (Eq. expansion) against the oracle and against the
materialise-then-contract comparator."""

import numpy as np
import pytest
import torch

import oracle
from paper_2302_08381_gb300 import api, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _workload(ncent, mean_nb, nr, l_max, seed, maxnb=None):
    rng = np.random.default_rng(seed)
    counts = np.clip(rng.normal(mean_nb, mean_nb / 4, size=ncent).round(), 0, maxnb or 3 * mean_nb).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    E = int(offs[-1])
    xyz = inputs.shell_points(E, 0.7, 5.0, seed=seed + 1)
    R = inputs.upstream(E, nr * (l_max + 1), seed=seed + 2).reshape(E, nr, l_max + 1)
    return xyz, R, offs


def _scale(xyz, R, offs, l_max, normalized):
    """Per-output scale sum_k |R[k,n,l]| * (block size of Y at x_k)."""
    r = np.linalg.norm(xyz.astype(np.float64), axis=1)
    lv = np.concatenate([np.full(2 * l + 1, l) for l in range(l_max + 1)])
    ys = np.sqrt((2 * lv + 1) / (4 * np.pi))[None, :] * (1.0 if normalized else r[:, None] ** lv[None, :])
    S = np.abs(R.astype(np.float64))[:, :, lv] * ys[:, None, :]
    out = np.zeros((offs.shape[0] - 1,) + S.shape[1:])
    for i in range(offs.shape[0] - 1):
        out[i] = S[offs[i]:offs[i + 1]].sum(0)
    return np.maximum(out, 1e-30)


@pytest.mark.parametrize("normalized", [False, True])
@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_expansion_matches_oracle(normalized, dtype):
    for l_max, nr in ((0, 1), (1, 3), (3, 8), (6, 8), (8, 17), (11, 4), (16, 2)):
        xyz, R, offs = _workload(53, 30, nr, l_max, seed=600 + l_max, maxnb=90)
        offs[5] = offs[4]  # an empty centre
        offs[6:] = np.maximum(offs[6:], offs[5])
        c = api.expansion(torch.from_numpy(xyz).to(DEV, dtype), torch.from_numpy(R).to(DEV, dtype),
                          torch.from_numpy(offs).to(DEV), l_max, normalized)
        torch.cuda.synchronize()
        x64 = xyz.astype(dtype == torch.float32 and np.float32 or np.float64).astype(np.float64)
        R64 = R.astype(dtype == torch.float32 and np.float32 or np.float64).astype(np.float64)
        ref = oracle.expansion(x64, R64, offs, l_max, normalized)
        err = np.abs(c.double().cpu().numpy() - ref) / _scale(x64, R64, offs, l_max, normalized)
        tol = 2e-6 if dtype == torch.float32 else 1e-13
        assert err.max() < tol, (l_max, nr, err.max())
        assert np.all(c.cpu().numpy()[4] == 0)


def test_expansion_full_size_sampled_and_vs_materialized():
    """100,000 centres x ~40 points (4M points), l_max = 6, 8 radial channels."""
    l_max, nr = 6, 8
    xyz, R, offs = _workload(100_000, 40, nr, l_max, seed=610)
    x = torch.from_numpy(xyz).to(DEV)
    Rt = torch.from_numpy(R).to(DEV)
    ot = torch.from_numpy(offs).to(DEV)
    c = api.expansion(x, Rt, ot, l_max)
    plain = api.materialized_expansion(x, Rt, ot, l_max)
    torch.cuda.synchronize()
    scale = _scale(xyz[: offs[2001]], R[: offs[2001]], offs[:2001], l_max, False)
    diff = np.abs(c[:2000].double().cpu().numpy() - plain[:2000].double().cpu().numpy()) / scale
    assert diff.max() < 2e-6
    idx = np.random.default_rng(611).choice(100_000, 200, replace=False)
    for i in idx:
        a, b = offs[i], offs[i + 1]
        ref = oracle.expansion(xyz[a:b].astype(np.float64), R[a:b].astype(np.float64), np.array([0, b - a]), l_max)
        sc = _scale(xyz[a:b], R[a:b], np.array([0, b - a]), l_max, False)
        assert (np.abs(c[i].double().cpu().numpy() - ref[0]) / sc[0]).max() < 2e-6, i
    assert api.device_status() == 0


def test_expansion_malformed_offsets_flagged_without_fault():
    l_max, nr = 4, 2
    xyz, R, offs = _workload(10, 20, nr, l_max, seed=620)
    bad = offs.copy()
    bad[3] = bad[2] - 1          # decreasing
    bad[7] = int(offs[-1]) + 50  # beyond n_points
    c = api.expansion(torch.from_numpy(xyz).to(DEV), torch.from_numpy(R).to(DEV), torch.from_numpy(bad).to(DEV), l_max)
    torch.cuda.synchronize()
    assert api.device_status() & 2
    cc = c.cpu().numpy()
    assert np.all(cc[2] == 0) and np.all(cc[6] == 0) and np.all(cc[7] == 0)
    assert np.any(cc[0] != 0)
    assert api.device_status() == 0  # read-and-clear


@pytest.mark.parametrize("l_max,nr,dtype", [(3, 5, torch.float32), (2, 3, torch.float32), (6, 8, torch.float64)])
def test_expansion_many_centres_per_warp(l_max, nr, dtype):
    """150,000 centres of mixed sizes (empty, a few points, around one and two
    32-point chunks), so that every warp streams several batches of 32
    centres whose points cross chunk boundaries, with a few malformed centres
    in between. The oracle checks a prefix of 4,000 centres (whole warp
    ranges), 300 sampled centres and the centres next to the malformed ones.
    (l_max 2 with 3 channels has 36-byte radial rows: the plain-load path.)"""
    rng = np.random.default_rng(630 + l_max)
    ncent = 150_000
    counts = rng.choice([0, 0, 1, 1, 2, 3, 5, 31, 33, 64], size=ncent)
    offs = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    E = int(offs[-1])
    bad = offs.copy()
    for i in (17, 70_011, 149_999):  # centre i-1 decreasing; centre i starts one point early
        bad[i] = bad[i - 1] - 1
    xyz = inputs.shell_points(E, 0.7, 5.0, seed=631)
    R = inputs.upstream(E, nr * (l_max + 1), seed=632).reshape(E, nr, l_max + 1)
    npd = np.float32 if dtype == torch.float32 else np.float64
    xyz, R = xyz.astype(npd), R.astype(npd)
    c = api.expansion(torch.from_numpy(xyz).to(DEV), torch.from_numpy(R).to(DEV), torch.from_numpy(bad).to(DEV),
                      l_max)
    torch.cuda.synchronize()
    assert api.device_status() & 2
    cc = c.double().cpu().numpy()
    ok = (bad[:-1] >= 0) & (bad[:-1] <= bad[1:]) & (bad[1:] <= E)
    assert (~ok).sum() == 3 and np.all(cc[~ok] == 0)
    tol = 2e-6 if dtype == torch.float32 else 1e-13
    x64, R64 = xyz.astype(np.float64), R.astype(np.float64)
    n0 = 4000
    ref = oracle.expansion(x64[: bad[n0]], R64[: bad[n0]], bad[: n0 + 1], l_max)
    err = np.abs(cc[:n0] - ref) / _scale(x64[: bad[n0]], R64[: bad[n0]], bad[: n0 + 1], l_max, False)
    assert err.max() < tol, err.max()
    sample = np.concatenate([rng.choice(ncent, 300, replace=False), [70_009, 70_011, 70_012, 149_999]])
    for i in sample:
        if not ok[i]:
            continue
        a, b = bad[i], bad[i + 1]
        one = np.array([0, b - a])
        ref = oracle.expansion(x64[a:b], R64[a:b], one, l_max)[0]
        sc = _scale(x64[a:b], R64[a:b], one, l_max, False)[0]
        assert (np.abs(cc[i] - ref) / sc).max() < tol, i
