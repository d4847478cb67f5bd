"""Element-by-element parity at full workload sizes, the oracle spread over
the host cores.

The GPU outputs are staged on the host as .npy files in a temporary
directory; a process pool started with ``spawn`` (never forked from a process
that holds a CUDA context) maps them read-only and each worker runs the FP64
oracle on one chunk of points and returns the chunk's per-l maximum errors
(``parity_utils`` scales) or, for the adjoints, the chunk's maximum absolute
difference and maximum reference magnitude. Nothing here computes harmonics
itself: every expected value comes from ``oracle``.
"""

from __future__ import annotations

import multiprocessing as mp
import os
import tempfile

import numpy as np

_ARR: dict = {}


def _init(paths):
    global _ARR
    _ARR = {k: np.load(p, mmap_mode="r") for k, p in paths.items()}


def _fwd_chunk(job):
    import oracle
    from parity_utils import grad_errors, value_errors

    a, b, l_max, normalized = job
    x = np.asarray(_ARR["xyz"][a:b], dtype=np.float64)
    if "dsph" in _ARR:
        rv, rg = oracle.spherical_harmonics_grad(x, l_max, normalized)
        eg = grad_errors(np.asarray(_ARR["dsph"][a:b], np.float64), rg, x, l_max, normalized)
    else:
        rv, eg = oracle.spherical_harmonics(x, l_max, normalized), None
    ev = value_errors(np.asarray(_ARR["sph"][a:b], np.float64), rv, x, l_max, normalized)
    finite = bool(np.all(np.isfinite(_ARR["sph"][a:b]))) and (
        "dsph" not in _ARR or bool(np.all(np.isfinite(_ARR["dsph"][a:b]))))
    return ev, eg, finite


def _hess_chunk(job):
    import oracle
    from parity_utils import hess_errors

    a, b, l_max, normalized = job
    x = np.asarray(_ARR["xyz"][a:b], dtype=np.float64)
    ref = oracle.spherical_harmonics_hessian(x, l_max, normalized)
    got = np.asarray(_ARR["ddsph"][a:b], np.float64)
    eh = hess_errors(got, ref, x, l_max, normalized)
    sym = bool(np.array_equal(got, got.transpose(0, 2, 1, 3)))
    return eh, bool(np.all(np.isfinite(got))), sym


def _bwd_chunk(job):
    import oracle

    a, b, l_max, normalized = job
    x = np.asarray(_ARR["xyz"][a:b], np.float64)
    g = np.asarray(_ARR["g"][a:b], np.float64)
    out = []
    if "dxyz" in _ARR:
        ref = oracle.backward(x, g, l_max, normalized)
        out.append((float(np.max(np.abs(np.asarray(_ARR["dxyz"][a:b], np.float64) - ref))),
                    float(np.max(np.abs(ref)))))
    if "grad_g" in _ARR:
        v = np.asarray(_ARR["v"][a:b], np.float64)
        rgg, rgx = oracle.double_backward(x, g, v, l_max, normalized)
        for name, ref in (("grad_g", rgg), ("grad_xyz", rgx)):
            out.append((float(np.max(np.abs(np.asarray(_ARR[name][a:b], np.float64) - ref))),
                        float(np.max(np.abs(ref)))))
    return out


def _chunks(n, K, per_chunk=None):
    step = per_chunk or int(min(32768, max(256, (1 << 22) // max(K, 1))))
    return [(a, min(n, a + step)) for a in range(0, n, step)]


def _pool_map(arrays, fn, jobs, processes):
    with tempfile.TemporaryDirectory(prefix="sph_parity_") as d:
        paths = {}
        for k, arr in arrays.items():
            p = os.path.join(d, k + ".npy")
            np.save(p, np.ascontiguousarray(arr))
            paths[k] = p
        ctx = mp.get_context("spawn")
        procs = processes or os.cpu_count() or 1
        with ctx.Pool(procs, initializer=_init, initargs=(paths,)) as pool:
            return pool.map(fn, jobs, chunksize=1)


def forward_errors(xyz, l_max, normalized, sph, dsph=None, processes=None):
    """Per-l maximum value and gradient errors over every point.

    ``xyz`` [n, 3] (the coordinates the GPU saw), ``sph`` [n, K], ``dsph``
    [n, 3, K] or None, all numpy. Returns (ev [l_max+1], eg [l_max+1] or
    None, all_finite).
    """
    n = xyz.shape[0]
    K = (l_max + 1) ** 2
    arrays = {"xyz": xyz, "sph": sph}
    if dsph is not None:
        arrays["dsph"] = dsph
    jobs = [(a, b, l_max, bool(normalized)) for a, b in _chunks(n, K * (4 if dsph is not None else 1))]
    res = _pool_map(arrays, _fwd_chunk, jobs, processes)
    ev = np.max(np.stack([r[0] for r in res]), axis=0)
    eg = None if dsph is None else np.max(np.stack([r[1] for r in res]), axis=0)
    return ev, eg, all(r[2] for r in res)


def adjoint_errors(xyz, g, l_max, normalized, dxyz=None, v=None, grad_g=None, grad_xyz=None, processes=None):
    """max |got - ref| / max |ref| over every point for the fused backward
    (``dxyz``) and/or the double backward (``grad_g``, ``grad_xyz``)."""
    n = xyz.shape[0]
    K = (l_max + 1) ** 2
    arrays = {"xyz": xyz, "g": g}
    names = []
    if dxyz is not None:
        arrays["dxyz"] = dxyz
        names.append("dxyz")
    if grad_g is not None:
        arrays.update(v=v, grad_g=grad_g, grad_xyz=grad_xyz)
        names += ["grad_g", "grad_xyz"]
    jobs = [(a, b, l_max, bool(normalized)) for a, b in _chunks(n, K * (12 if grad_g is not None else 4))]
    res = _pool_map(arrays, _bwd_chunk, jobs, processes)
    out = {}
    for i, name in enumerate(names):
        diff = max(r[i][0] for r in res)
        ref = max(r[i][1] for r in res)
        out[name] = diff / max(ref, 1e-300)
    return out


def hessian_errors(xyz, l_max, normalized, ddsph, processes=None):
    """Per-l maximum Hessian error over every point (``parity_utils`` scale),
    whether every output is finite, and whether every point's [3, 3] planes
    are symmetric bit for bit. ``ddsph`` [n, 3, 3, K] numpy (any float
    dtype; staged as given)."""
    n = xyz.shape[0]
    K = (l_max + 1) ** 2
    jobs = [(a, b, l_max, bool(normalized)) for a, b in _chunks(n, 9 * K)]
    res = _pool_map({"xyz": xyz, "ddsph": ddsph}, _hess_chunk, jobs, processes)
    eh = np.max(np.stack([r[0] for r in res]), axis=0)
    return eh, all(r[1] for r in res), all(r[2] for r in res)
