"""Tensor-level calls of the C-ABI: allocate outputs with torch on the input's
device, pass raw pointers and torch's current stream, raise on any error.
Every computation runs in the CUDA library; CPU tensors are rejected.
"""

from __future__ import annotations

import torch

from . import _capi as C

_KERNELS = {
    "auto": C.SPH_KERNEL_AUTO,
    "point": C.SPH_KERNEL_POINT,
    "slice": C.SPH_KERNEL_SLICE,
    "degree": C.SPH_KERNEL_DEGREE,
    "degree_down": C.SPH_KERNEL_DEGREE_DOWN,
    "row": C.SPH_KERNEL_ROW,
    "point_hc": C.SPH_KERNEL_POINT_HC,
}
_QPREC = {"native": C.SPH_Q_NATIVE, "f64": C.SPH_Q_F64}


def n_columns(l_max: int) -> int:
    return (l_max + 1) ** 2


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return C.SPH_F32
    if t.dtype == torch.float64:
        return C.SPH_F64
    raise TypeError(f"xyz must be float32 or float64, got {t.dtype}")


def _check_points(xyz: torch.Tensor, name: str = "xyz") -> None:
    if not isinstance(xyz, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if not xyz.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor (the library has no CPU path)")
    if xyz.dim() != 2 or xyz.shape[1] != 3:
        raise ValueError(f"{name} must have shape [n, 3], got {tuple(xyz.shape)}")
    if not xyz.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _stream(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def _launch(launch):
    if launch is None:
        return None
    if isinstance(launch, C.sph_launch):
        return launch
    return C.make_launch(**launch)


def spherical_harmonics(
    xyz: torch.Tensor,
    l_max: int,
    normalized: bool = False,
    gradients: bool = False,
    hessians: bool = False,
    out_dtype: torch.dtype | None = None,
    qprec: str = "native",
    kernel: str = "auto",
    launch=None,
    out=None,
):
    """Real spherical harmonics of every (l, m), l <= l_max, at each point.

    Returns ``sph`` [n, K]; with ``gradients`` also ``dsph`` [n, 3, K]; with
    ``hessians`` also ``ddsph`` [n, 3, 3, K]. ``normalized=False`` gives the
    scaled r^l Y_l^m. ``out_dtype=torch.bfloat16`` stores FP32 results as
    bfloat16 (round to nearest even). ``qprec="f64"`` keeps FP32 inputs and
    outputs but computes in FP64 (unit vector, recursions, assembly).
    ``out`` may supply preallocated outputs.
    """
    _check_points(xyz)
    dt = _dtype_code(xyz)
    hessians = bool(hessians)
    gradients = bool(gradients) or hessians
    if out_dtype is None or out_dtype == xyz.dtype:
        oc, odt = C.SPH_OUT_SAME, xyz.dtype
    elif out_dtype == torch.bfloat16:
        oc, odt = C.SPH_OUT_BF16, torch.bfloat16
    else:
        raise TypeError(f"unsupported out_dtype {out_dtype}")
    n = xyz.shape[0]
    K = n_columns(l_max)
    if out is not None:
        sph, dsph, ddsph = (list(out) + [None, None, None])[:3]
    else:
        sph = torch.empty((n, K), dtype=odt, device=xyz.device)
        dsph = torch.empty((n, 3, K), dtype=odt, device=xyz.device) if gradients else None
        ddsph = torch.empty((n, 3, 3, K), dtype=odt, device=xyz.device) if hessians else None
    L = _launch(launch)
    C.sphericart_compute_ex(
        xyz.data_ptr(),
        n,
        l_max,
        1 if normalized else 0,
        dt,
        oc,
        _QPREC[qprec],
        _KERNELS[kernel],
        L,
        sph.data_ptr() if sph is not None else None,
        dsph.data_ptr() if dsph is not None else None,
        ddsph.data_ptr() if ddsph is not None else None,
        _stream(xyz.device),
    )
    if hessians:
        return sph, dsph, ddsph
    if gradients:
        return sph, dsph
    return sph


def spherical_harmonics_host(xyz, l_max, normalized=False, gradients=False, out=None, workspace=None,
                             chunk_points=0, device=None):
    """Forward from host tensors, pipelined in chunks through a device
    workspace (host->device copy, kernel and device->host copy overlap).

    ``xyz``: CPU tensor [n, 3] (pinned for asynchronous copies). Outputs are
    pinned CPU tensors (allocated here unless ``out`` gives them). Returns
    after the copies are enqueued on the current stream of ``device``; call
    torch.cuda.synchronize() (or sync that stream) before reading them.
    """
    if xyz.is_cuda or xyz.dim() != 2 or xyz.shape[1] != 3 or not xyz.is_contiguous():
        raise ValueError("xyz must be a contiguous CPU tensor [n, 3]")
    device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    n, K = xyz.shape[0], n_columns(l_max)
    if out is None:
        sph = torch.empty((n, K), dtype=xyz.dtype, pin_memory=True)
        dsph = torch.empty((n, 3, K), dtype=xyz.dtype, pin_memory=True) if gradients else None
    else:
        sph, dsph = out
    if workspace is None:
        chunk = chunk_points or (1 << 20)
        per = xyz.element_size() * (3 + K * (4 if gradients else 1))
        workspace = torch.empty(2 * (min(chunk, max(n, 32)) + 32) * per + 4096, dtype=torch.uint8, device=device)
    C.sphericart_compute_host(
        xyz.data_ptr(), n, l_max, 1 if normalized else 0, _dtype_code(xyz), C.SPH_OUT_SAME,
        sph.data_ptr(), dsph.data_ptr() if dsph is not None else None,
        workspace.data_ptr(), workspace.numel(), chunk_points, _stream(device),
    )
    return (sph, dsph) if gradients else sph


def backward(xyz, g, l_max, normalized=False, kernel="auto", launch=None, out=None):
    """Fused recompute-backward: dxyz[n, i] = sum_k g[n, k] d sph[n, k] / d x_i."""
    _check_points(xyz)
    g = g.contiguous()
    if g.shape != (xyz.shape[0], n_columns(l_max)) or g.dtype != xyz.dtype or g.device != xyz.device:
        raise ValueError("g must be [n, (l_max+1)^2] with the dtype and device of xyz")
    dxyz = torch.empty_like(xyz) if out is None else out
    C.sphericart_backward(
        xyz.data_ptr(),
        g.data_ptr(),
        xyz.shape[0],
        l_max,
        1 if normalized else 0,
        _dtype_code(xyz),
        _KERNELS[kernel],
        _launch(launch),
        dxyz.data_ptr(),
        _stream(xyz.device),
    )
    return dxyz


def double_backward(xyz, g, v, l_max, normalized=False, kernel="auto", launch=None, need_g=True, need_xyz=True):
    """grad_g[n, k] = sum_j v_j d sph_k/dx_j; grad_xyz[n, i] = sum_k g_k sum_j v_j d2 sph_k/dx_i dx_j."""
    _check_points(xyz)
    g = g.contiguous()
    v = v.contiguous()
    if g.shape != (xyz.shape[0], n_columns(l_max)) or v.shape != xyz.shape:
        raise ValueError("g must be [n, K] and v [n, 3]")
    grad_g = torch.empty_like(g) if need_g else None
    grad_xyz = torch.empty_like(xyz) if need_xyz else None
    C.sphericart_double_backward(
        xyz.data_ptr(),
        g.data_ptr(),
        v.data_ptr(),
        xyz.shape[0],
        l_max,
        1 if normalized else 0,
        _dtype_code(xyz),
        _KERNELS[kernel],
        _launch(launch),
        grad_g.data_ptr() if grad_g is not None else None,
        grad_xyz.data_ptr() if grad_xyz is not None else None,
        _stream(xyz.device),
    )
    return grad_g, grad_xyz


def materialized_backward(xyz, g, l_max, normalized=False, dsph=None):
    """The paper's PyTorch-layer backward (Section 3): the forward writes dsph,
    then dxyz = einsum('nik,nk->ni', dsph, g). Kept as the comparator of the
    fused backward; the einsum is torch's."""
    if dsph is None:
        _, dsph = spherical_harmonics(xyz, l_max, normalized, gradients=True)
    return torch.einsum("nik,nk->ni", dsph, g)


def expansion(xyz, radial, offsets, l_max, normalized=False, out=None):
    """Eq. expansion per centre, fused: c[i, n, (l,m)] = sum_k R[k, n, l] Y_l^m(x_k).

    ``xyz`` [E, 3] grouped by centre, ``radial`` [E, n_rad, l_max+1],
    ``offsets`` int64 [n_centres+1] (CSR). Returns c [n_centres, n_rad, K].
    """
    _check_points(xyz)
    radial = radial.contiguous()
    offsets = offsets.contiguous()
    if radial.dim() != 3 or radial.shape[0] != xyz.shape[0] or radial.shape[2] != l_max + 1:
        raise ValueError("radial must be [n_points, n_rad, l_max+1]")
    if radial.dtype != xyz.dtype or offsets.dtype != torch.int64 or not offsets.is_cuda:
        raise ValueError("radial must match xyz's dtype; offsets must be a CUDA int64 tensor")
    ncent = offsets.shape[0] - 1
    nr = radial.shape[1]
    c = torch.empty((ncent, nr, n_columns(l_max)), dtype=xyz.dtype, device=xyz.device) if out is None else out
    C.sphericart_expansion(
        xyz.data_ptr(), radial.data_ptr(), offsets.data_ptr(), ncent, xyz.shape[0], nr, l_max,
        1 if normalized else 0, _dtype_code(xyz), c.data_ptr(), _stream(xyz.device),
    )
    return c


def materialized_expansion(xyz, radial, offsets, l_max, normalized=False):
    """Comparator: the harmonics written by the forward kernel, then the
    contraction and the per-centre sum in torch (index_add)."""
    Y = spherical_harmonics(xyz, l_max, normalized)
    lv = torch.repeat_interleave(torch.arange(l_max + 1, device=xyz.device), 2 * torch.arange(l_max + 1, device=xyz.device) + 1)
    counts = offsets[1:] - offsets[:-1]
    centre = torch.repeat_interleave(torch.arange(offsets.shape[0] - 1, device=xyz.device), counts)
    contrib = radial[:, :, lv] * Y[:, None, :]
    out = torch.zeros((offsets.shape[0] - 1, radial.shape[1], Y.shape[1]), dtype=Y.dtype, device=xyz.device)
    return out.index_add_(0, centre, contrib)


def autotune(xyz, l_max, normalized=False, gradients=True, out_dtype=None, reps=3):
    """Runs the library's autotuner for this forward request on the current
    device (outputs are scratch) and installs the fastest launch shape for
    later calls. Returns (shape dict, best ms)."""
    _check_points(xyz)
    K = n_columns(l_max)
    odt = torch.bfloat16 if out_dtype == torch.bfloat16 else xyz.dtype
    sph = torch.empty((xyz.shape[0], K), dtype=odt, device=xyz.device)
    dsph = torch.empty((xyz.shape[0], 3, K), dtype=odt, device=xyz.device) if gradients else None
    best, ms = C.sphericart_autotune(
        xyz.data_ptr(), xyz.shape[0], l_max, 1 if normalized else 0, _dtype_code(xyz),
        C.SPH_OUT_BF16 if odt == torch.bfloat16 else C.SPH_OUT_SAME, sph.data_ptr(),
        dsph.data_ptr() if dsph is not None else None, _stream(xyz.device), reps,
    )
    return {"points_per_tile": best.points_per_tile, "warps_per_block": best.warps_per_block,
            "blocks_per_sm": best.blocks_per_sm}, ms


def save_tuning(path: str) -> None:
    """Writes the tuned launch shapes of the current device (keyed by GPU name)."""
    with open(path, "w") as f:
        f.write(C.sphericart_tune_export())


def load_tuning(path: str) -> int:
    """Installs the shapes of a saved table whose GPU name matches the current
    device; returns how many were installed."""
    with open(path) as f:
        return C.sphericart_tune_import(f.read())


def device_status() -> int:
    """Reads and clears the device status word (nonzero: a bounded wait timed out)."""
    return C.sphericart_device_status()


_E3NN_NORMS = {"integral": C.SPH_E3NN_INTEGRAL, "component": C.SPH_E3NN_COMPONENT, "norm": C.SPH_E3NN_NORM}


def e3nn_spherical_harmonics(xyz, l_max, normalize=False, normalization="integral", gradients=False):
    """The harmonics in e3nn's convention (``sphericart_compute_e3nn``): y is
    the polar axis, l = 1 is proportional to (x, y, z), and ``normalization``
    is "integral", "component" or "norm" as in e3nn. Returns sph [n, K] and,
    with ``gradients``, dsph [n, 3, K] (d/dx, d/dy, d/dz)."""
    _check_points(xyz)
    if normalization not in _E3NN_NORMS:
        raise ValueError("normalization must be 'integral', 'component' or 'norm'")
    n, K = xyz.shape[0], n_columns(l_max)
    ws = torch.empty_like(xyz)
    sph = torch.empty((n, K), dtype=xyz.dtype, device=xyz.device)
    dsph = torch.empty((n, 3, K), dtype=xyz.dtype, device=xyz.device) if gradients else None
    C.check("sphericart_compute_e3nn", C.lib().sphericart_compute_e3nn(
        xyz.data_ptr(), n, int(l_max), 1 if normalize else 0, _E3NN_NORMS[normalization], _dtype_code(xyz),
        ws.data_ptr(), sph.data_ptr(), dsph.data_ptr() if dsph is not None else None, _stream(xyz.device)))
    return (sph, dsph) if gradients else sph


def batch_descriptors(xyz_list, lmax_list, sph_list, dsph_list, normalized=False, device=None):
    """sph_batch_set descriptors of point sets as a CUDA uint8 tensor [nsets, 40]
    (the device array ``sphericart_compute_batched`` reads)."""
    n = len(xyz_list)
    arr = (C.sph_batch_set * n)()
    for i in range(n):
        x, s, d = xyz_list[i], sph_list[i], dsph_list[i] if dsph_list is not None else None
        arr[i] = C.sph_batch_set(x.data_ptr(), s.data_ptr(), d.data_ptr() if d is not None else None, x.shape[0],
                                 int(lmax_list[i]), 1 if normalized else 0)
    host = torch.frombuffer(bytearray(arr), dtype=torch.uint8).view(n, -1)
    return host.to(device or xyz_list[0].device)


def compute_batched(xyz_list, lmax_list, normalized=False, gradients=True, outputs=None, launch=None):
    """Ragged point sets (CUDA float32 [n_s, 3], l_max_s <= 16) in one persistent
    launch (``sphericart_compute_batched``) on torch's current stream.

    Returns ``(sph_list, dsph_list)`` (``dsph_list`` None without gradients);
    ``outputs`` may supply them as a list of (sph, dsph) pairs.
    """
    if len(xyz_list) != len(lmax_list) or not xyz_list:
        raise ValueError("need one l_max per point set")
    dev = xyz_list[0].device
    sph_list, dsph_list = [], [] if gradients else None
    for i, (x, L) in enumerate(zip(xyz_list, lmax_list)):
        _check_points(x)
        if x.dtype != torch.float32:
            raise TypeError("batched sets are float32")
        K = n_columns(int(L))
        if outputs is not None:
            s, d = outputs[i]
        else:
            s = torch.empty((x.shape[0], K), device=dev)
            d = torch.empty((x.shape[0], 3, K), device=dev) if gradients else None
        sph_list.append(s)
        if gradients:
            dsph_list.append(d)
    desc = batch_descriptors(xyz_list, lmax_list, sph_list, dsph_list, normalized, dev)
    flags = (C.SPH_BATCHED_GRADIENTS if gradients else 0) | (C.SPH_BATCHED_NORMALIZED if normalized else 0)
    C.check("sphericart_compute_batched_ex",
            C.lib().sphericart_compute_batched_ex(desc.data_ptr(), len(xyz_list), flags, _launch(launch),
                                                  _stream(dev)))
    return sph_list, dsph_list


class BatchPlan:
    """A ragged batch evaluated by persistent launches (FP32, l_max <= 16).

    ``xyz_list``: CUDA float32 tensors [n_s, 3]; ``lmax_list``: l_max per set.
    Outputs are allocated here (``self.sph[s]`` [n_s, K_s], ``self.dsph[s]``
    [n_s, 3, K_s] when ``gradients``) unless ``outputs`` supplies them.
    ``mode``: "per_lmax" (one launch per distinct l_max, the default) or
    "one_launch" (a single launch for every set). ``execute()`` enqueues the
    launches on torch's current stream; it can be captured in a CUDA graph.
    """

    def __init__(self, xyz_list, lmax_list, normalized=False, gradients=True, launch=None, outputs=None,
                 mode="per_lmax"):
        import ctypes

        if len(xyz_list) != len(lmax_list) or not xyz_list:
            raise ValueError("need one l_max per point set")
        self.device = xyz_list[0].device
        self.xyz = []
        self.sph, self.dsph = [], []
        arr = (C.sph_batch_set * len(xyz_list))()
        for i, (x, L) in enumerate(zip(xyz_list, lmax_list)):
            _check_points(x)
            if x.dtype != torch.float32:
                raise TypeError("batched sets are float32")
            K = n_columns(int(L))
            if outputs is not None:
                s, d = outputs[i]
            else:
                s = torch.empty((x.shape[0], K), device=x.device)
                d = torch.empty((x.shape[0], 3, K), device=x.device) if gradients else None
            self.xyz.append(x)
            self.sph.append(s)
            self.dsph.append(d)
            arr[i] = C.sph_batch_set(
                x.data_ptr(), s.data_ptr(), d.data_ptr() if d is not None else None, x.shape[0], int(L),
                1 if normalized else 0,
            )
        self._plan = ctypes.c_void_p()
        C.check(
            "sphericart_batch_plan_create_ex",
            C.lib().sphericart_batch_plan_create_ex(
                arr, len(xyz_list), _launch(launch), {"per_lmax": C.SPH_BATCH_PER_LMAX,
                                                      "one_launch": C.SPH_BATCH_ONE_LAUNCH}[mode],
                ctypes.byref(self._plan)),
        )

    def execute(self):
        C.check("sphericart_batch_execute", C.lib().sphericart_batch_execute(self._plan, _stream(self.device)))

    def info(self):
        import ctypes

        p, t = ctypes.c_int64(), ctypes.c_int64()
        C.check("sphericart_batch_plan_info", C.lib().sphericart_batch_plan_info(self._plan, ctypes.byref(p), ctypes.byref(t)))
        return int(p.value), int(t.value)

    def close(self):
        if getattr(self, "_plan", None):
            C.lib().sphericart_batch_plan_destroy(self._plan)
            self._plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
