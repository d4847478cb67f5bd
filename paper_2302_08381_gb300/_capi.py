"""ctypes binding of libsphericart_gb300.so: the C-ABI of
``include/sphericart_gb300.h`` under the same names, with argument
marshalling only. There is no fallback: if the library is missing, every call
raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsphericart_gb300.so")

SPH_OK, SPH_EINVAL, SPH_EUNSUPPORTED, SPH_ECUDA, SPH_ENOMEM, SPH_ETIMEOUT = range(6)
SPH_F32, SPH_F64 = 0, 1
SPH_OUT_SAME, SPH_OUT_BF16 = 0, 1
SPH_Q_NATIVE, SPH_Q_F64 = 0, 1
SPH_KERNEL_AUTO, SPH_KERNEL_POINT, SPH_KERNEL_SLICE, SPH_KERNEL_DEGREE, SPH_KERNEL_DEGREE_DOWN, SPH_KERNEL_ROW = (
    0, 1, 2, 3, 4, 5)
SPH_KERNEL_POINT_HC = 6
SPH_BATCH_PER_LMAX, SPH_BATCH_ONE_LAUNCH = 0, 1
SPH_BATCHED_GRADIENTS, SPH_BATCHED_NORMALIZED = 1, 2
SPH_E3NN_INTEGRAL, SPH_E3NN_COMPONENT, SPH_E3NN_NORM = 0, 1, 2
SPH_MAX_L = 128
SPH_MAX_L_POINT = 16

STATUS_NAMES = {
    SPH_OK: "SPH_OK",
    SPH_EINVAL: "SPH_EINVAL",
    SPH_EUNSUPPORTED: "SPH_EUNSUPPORTED",
    SPH_ECUDA: "SPH_ECUDA",
    SPH_ENOMEM: "SPH_ENOMEM",
    SPH_ETIMEOUT: "SPH_ETIMEOUT",
}


class sph_launch(ctypes.Structure):
    _fields_ = [
        ("points_per_tile", ctypes.c_int32),
        ("warps_per_block", ctypes.c_int32),
        ("blocks_per_sm", ctypes.c_int32),
        ("lanes_per_point", ctypes.c_int32),
    ]


class sph_batch_set(ctypes.Structure):
    _fields_ = [
        ("xyz", ctypes.c_void_p),
        ("sph", ctypes.c_void_p),
        ("dsph", ctypes.c_void_p),
        ("n", ctypes.c_int64),
        ("l_max", ctypes.c_int32),
        ("normalized", ctypes.c_int32),
    ]


class SphericartError(RuntimeError):
    def __init__(self, func: str, code: int, message: str):
        super().__init__(f"{func} failed with {STATUS_NAMES.get(code, code)}: {message}")
        self.code = code
        self.func = func


_P = ctypes.c_void_p
_I = ctypes.c_int
_I64 = ctypes.c_int64
_PROTOS = {
    "sphericart_compute": (_I, [_P, _I64, _I, _I, _P, _P, _P, _P]),
    "sphericart_compute_ex": (_I, [_P, _I64, _I, _I, _I, _I, _I, _I, ctypes.POINTER(sph_launch), _P, _P, _P, _P]),
    "sphericart_compute_host": (_I, [_P, _I64, _I, _I, _I, _I, _P, _P, _P, ctypes.c_size_t, _I64, _P]),
    "sphericart_backward": (_I, [_P, _P, _I64, _I, _I, _I, _I, ctypes.POINTER(sph_launch), _P, _P]),
    "sphericart_double_backward": (
        _I,
        [_P, _P, _P, _I64, _I, _I, _I, _I, ctypes.POINTER(sph_launch), _P, _P, _P],
    ),
    "sphericart_expansion": (_I, [_P, _P, _P, _I64, _I64, _I, _I, _I, _I, _P, _P]),
    "sphericart_batch_plan_create": (_I, [ctypes.POINTER(sph_batch_set), _I, ctypes.POINTER(sph_launch), ctypes.POINTER(_P)]),
    "sphericart_batch_plan_create_ex": (
        _I, [ctypes.POINTER(sph_batch_set), _I, ctypes.POINTER(sph_launch), _I, ctypes.POINTER(_P)]),
    "sphericart_batch_execute": (_I, [_P, _P]),
    "sphericart_batch_plan_destroy": (_I, [_P]),
    "sphericart_batch_plan_info": (_I, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "sphericart_batch_compute_noalloc": (_I, [ctypes.POINTER(sph_batch_set), _I, ctypes.POINTER(sph_launch), _P]),
    "sphericart_compute_batched": (_I, [_P, _I, _I, _P]),
    "sphericart_compute_e3nn": (_I, [_P, _I64, _I, _I, _I, _I, _P, _P, _P, _P]),
    "sphericart_compute_batched_ex": (_I, [_P, _I, _I, ctypes.POINTER(sph_launch), _P]),
    "sphericart_last_error": (ctypes.c_char_p, []),
    "sphericart_max_l": (_I, [_I, _I, _I]),
    "sphericart_host_table": (_I, [_I, _I, ctypes.POINTER(ctypes.c_double)]),
    "sphericart_device_status": (_I, [ctypes.POINTER(ctypes.c_uint32)]),
    "sphericart_launch_info": (_I, [_I, _I, _I, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(sph_launch)]),
    "sphericart_set_launch": (_I, [_I, _I, _I, _I, ctypes.POINTER(sph_launch)]),
    "sphericart_version": (_I, []),
    "sphericart_autotune": (
        _I,
        [_P, _I64, _I, _I, _I, _I, _P, _P, _P, _I, ctypes.POINTER(sph_launch), ctypes.POINTER(ctypes.c_float)],
    ),
    "sphericart_batch_autotune": (
        _I,
        [ctypes.POINTER(sph_batch_set), _I, _P, _I, ctypes.POINTER(sph_launch), ctypes.POINTER(ctypes.c_float)],
    ),
    "sphericart_tune_export": (_I, [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "sphericart_tune_import": (_I, [ctypes.c_char_p, ctypes.POINTER(_I)]),
    "sphericart_tune_clear": (_I, []),
    "sphericart_fma_peak": (_I, [_I, _P, _I, ctypes.POINTER(ctypes.c_double)]),
}

_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'`"
                )
            handle = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _PROTOS.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
    return _lib


def last_error() -> str:
    msg = lib().sphericart_last_error()
    return msg.decode() if msg else ""


def check(func: str, code: int) -> None:
    if code != SPH_OK:
        raise SphericartError(func, code, last_error())


def _call(name, *args):
    code = getattr(lib(), name)(*args)
    check(name, code)
    return code


# Raw entry points under their C names (pointers as ints or None).
def sphericart_compute(xyz, n, l_max, normalized, sph, dsph, ddsph, stream):
    return _call("sphericart_compute", xyz, n, l_max, normalized, sph, dsph, ddsph, stream)


def sphericart_compute_ex(xyz, n, l_max, normalized, dtype, out, qprec, kernel, launch, sph, dsph, ddsph, stream):
    return _call(
        "sphericart_compute_ex", xyz, n, l_max, normalized, dtype, out, qprec, kernel, launch, sph, dsph, ddsph, stream
    )


def sphericart_compute_host(xyz_host, n, l_max, normalized, dtype, out, sph_host, dsph_host, workspace,
                            workspace_bytes, chunk_points, stream):
    return _call("sphericart_compute_host", xyz_host, n, l_max, normalized, dtype, out, sph_host, dsph_host,
                 workspace, workspace_bytes, chunk_points, stream)


def sphericart_backward(xyz, g, n, l_max, normalized, dtype, kernel, launch, dxyz, stream):
    return _call("sphericart_backward", xyz, g, n, l_max, normalized, dtype, kernel, launch, dxyz, stream)


def sphericart_double_backward(xyz, g, v, n, l_max, normalized, dtype, kernel, launch, grad_g, grad_xyz, stream):
    return _call(
        "sphericart_double_backward", xyz, g, v, n, l_max, normalized, dtype, kernel, launch, grad_g, grad_xyz, stream
    )


def sphericart_expansion(xyz, radial, offsets, n_centres, n_points, n_rad, l_max, normalized, dtype, c, stream):
    return _call(
        "sphericart_expansion", xyz, radial, offsets, n_centres, n_points, n_rad, l_max, normalized, dtype, c, stream
    )


def sphericart_host_table(l_max: int, which: int):
    import numpy as np

    n = (l_max + 1) * (l_max + 2) // 2
    out = (ctypes.c_double * n)()
    _call("sphericart_host_table", l_max, which, out)
    return np.frombuffer(out, dtype=np.float64).copy()


def sphericart_max_l(dtype: int, qprec: int, kernel: int) -> int:
    return lib().sphericart_max_l(dtype, qprec, kernel)


def sphericart_device_status() -> int:
    v = ctypes.c_uint32(0)
    _call("sphericart_device_status", ctypes.byref(v))
    return int(v.value)


def sphericart_launch_info(l_max, dtype, out, grad, hess):
    k = ctypes.c_int(0)
    s = sph_launch()
    _call("sphericart_launch_info", l_max, dtype, out, grad, hess, ctypes.byref(k), ctypes.byref(s))
    return int(k.value), s


def sphericart_set_launch(l_max, dtype, out, grad, launch: sph_launch):
    return _call("sphericart_set_launch", l_max, dtype, out, grad, ctypes.byref(launch))


def sphericart_version() -> int:
    return lib().sphericart_version()


def sphericart_autotune(xyz, n, l_max, normalized, dtype, out, sph, dsph, stream, reps=3):
    best = sph_launch()
    ms = ctypes.c_float(0)
    _call("sphericart_autotune", xyz, n, l_max, normalized, dtype, out, sph, dsph, stream, reps, ctypes.byref(best),
          ctypes.byref(ms))
    return best, float(ms.value)


def sphericart_tune_export() -> str:
    need = ctypes.c_size_t(0)
    _call("sphericart_tune_export", None, 0, ctypes.byref(need))
    buf = ctypes.create_string_buffer(max(1, need.value))
    _call("sphericart_tune_export", buf, need.value, ctypes.byref(need))
    return buf.value.decode()


def sphericart_tune_import(text: str) -> int:
    k = ctypes.c_int(0)
    _call("sphericart_tune_import", text.encode(), ctypes.byref(k))
    return int(k.value)


def sphericart_tune_clear():
    return _call("sphericart_tune_clear")


def sphericart_fma_peak(dtype, stream, reps=3) -> float:
    v = ctypes.c_double(0)
    _call("sphericart_fma_peak", dtype, stream, reps, ctypes.byref(v))
    return float(v.value)


def make_launch(points_per_tile=0, warps_per_block=0, blocks_per_sm=0, lanes_per_point=0):
    return sph_launch(points_per_tile, warps_per_block, blocks_per_sm, lanes_per_point)
