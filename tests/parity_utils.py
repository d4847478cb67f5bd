"""Error metrics and helpers shared by the parity tests.

Tolerances (FP32 unless stated) follow the acceptance bar for this method:
values <= 1e-5 * sqrt(2l+1) as absolute error on the unit sphere (scaled
outputs are divided by r^l), gradients <= 1e-4 relative to the exact l-block
gradient norm, FP64 paths <= 1e-12 on the same scales; bfloat16 storage
<= 2^-8 relative to the same scales (one bf16 rounding is <= 2^-9 relative).
"""

import math

import numpy as np

import oracle

F32_VAL = 1e-5
F32_GRAD = 1e-4
F64_TOL = 1e-12
BF16_TOL = 2.0**-8


def lvec(l_max):
    return np.concatenate([np.full(2 * l + 1, l) for l in range(l_max + 1)])


def value_scale(xyz, l_max, normalized):
    """[n, K]: r^l (scaled) or 1 (normalized)."""
    r = np.linalg.norm(np.asarray(xyz, dtype=np.float64), axis=1)
    lv = lvec(l_max)
    if normalized:
        return np.ones((r.shape[0], lv.shape[0]))
    s = r[:, None] ** lv[None, :]
    return np.where(s > 0, s, 1.0)  # r = 0: the exact values are 0 for l >= 1


def grad_scale(xyz, l_max, normalized):
    """[n, K]: exact rms size of an l block's gradient.

    scaled: sum_m |grad r^l Y_l^m|^2 = r^(2l-2) l (2l+1)^2 / (4 pi);
    normalized: sum_m |grad Y_l^m|^2 = l (l+1) (2l+1) / (4 pi r^2).
    """
    r = np.linalg.norm(np.asarray(xyz, dtype=np.float64), axis=1)
    lv = lvec(l_max).astype(np.float64)
    if normalized:
        s = np.sqrt(lv * (lv + 1) * (2 * lv + 1) / (4 * math.pi))[None, :] / np.where(r > 0, r, 1.0)[:, None]
    else:
        s = r[:, None] ** np.maximum(lv - 1, 0)[None, :] * np.sqrt(lv * (2 * lv + 1) ** 2 / (4 * math.pi))[None, :]
    return np.where(s > 0, s, 1.0)


def hess_scale(xyz, l_max, normalized):
    r = np.linalg.norm(np.asarray(xyz, dtype=np.float64), axis=1)
    lv = lvec(l_max).astype(np.float64)
    base = (lv + 1) ** 2 * np.sqrt((2 * lv + 1) / (4 * math.pi))
    if normalized:
        s = base[None, :] / np.where(r > 0, r, 1.0)[:, None] ** 2
    else:
        s = r[:, None] ** np.maximum(lv - 2, 0)[None, :] * base[None, :]
    return np.where(s > 0, s, 1.0)


def per_l_max(err, l_max):
    """err [..., K] -> [l_max+1] max over everything but the l block."""
    e = np.asarray(err).reshape(-1, (l_max + 1) ** 2)
    return np.array([np.max(e[:, l * l:(l + 1) ** 2]) if e.size else 0.0 for l in range(l_max + 1)])


def value_errors(got, ref, xyz, l_max, normalized):
    s = value_scale(xyz, l_max, normalized)
    return per_l_max(np.abs(np.asarray(got, np.float64) - ref) / s, l_max)


def grad_errors(got, ref, xyz, l_max, normalized):
    s = grad_scale(xyz, l_max, normalized)[:, None, :]
    return per_l_max(np.abs(np.asarray(got, np.float64) - ref) / s, l_max)


def hess_errors(got, ref, xyz, l_max, normalized):
    s = hess_scale(xyz, l_max, normalized)[:, None, None, :]
    return per_l_max(np.abs(np.asarray(got, np.float64) - ref) / s, l_max)


def value_bound(l_max, tol):
    return tol * np.sqrt(2 * np.arange(l_max + 1) + 1.0)


def assert_values(got, xyz, l_max, normalized, tol, ref=None):
    if ref is None:
        ref = oracle.spherical_harmonics(xyz, l_max, normalized)
    e = value_errors(got, ref, xyz, l_max, normalized)
    bound = value_bound(l_max, tol)
    bad = np.nonzero(~(e <= bound))[0]
    assert bad.size == 0, f"value error per l {e} exceeds {bound} at l={bad}"
    return e


def assert_grads(got, xyz, l_max, normalized, tol, ref=None):
    if ref is None:
        _, ref = oracle.spherical_harmonics_grad(xyz, l_max, normalized)
    e = grad_errors(got, ref, xyz, l_max, normalized)
    bad = np.nonzero(~(e <= tol))[0]
    assert bad.size == 0, f"gradient error per l {e} exceeds {tol} at l={bad}"
    return e
