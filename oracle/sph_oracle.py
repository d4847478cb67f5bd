"""Plain FP64 CPU oracle: real spherical harmonics from the textbook definition.

TEST INFRASTRUCTURE ONLY. Imported by ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline / reference legs of ``bench.py``; never by the product package.

What it computes (arXiv 2302.08381, Section 2):

* ``Y_l^m(theta, phi) = F_l^|m| P_l^|m|(cos theta) * {sin(|m| phi), 1/sqrt2, cos(m phi)}``
  for m < 0, m = 0, m > 0 (Eq. real-sh-spherical), with the prefactor of Eq. Flm
  taken from its closed form (exact factorial ratio), and ``P_l^m`` from the
  textbook three-term recursion of Eq. recur-p (Condon-Shortley sign included
  there; the ``(-1)^m`` of F cancels it).
* the scaled (solid) form ``r^l Y_l^m`` of Section 2 and the "normalized" form
  ``Y_l^m`` on the unit sphere of Section 3.
* Cartesian gradients by the analytic chain rule in spherical coordinates.
* Hessians by the analytic second derivative of the same spherical-coordinate
  definition (the paper gives no Hessian formulas; it only claims derivatives
  of any order follow from Eq. iter-deri). The theta dependence is written with
  the t-derivatives of the Legendre polynomials, P_l^m = (-1)^m sin^m(theta)
  d^m P_l/dt^m, so every power of sin(theta) is explicit and no term divides by
  it; a finite-difference Hessian (Richardson-extrapolated central differences
  of the analytic gradient) is kept as a cross-check.
* the adjoints used by autograd: ``dL/dxyz = sum_k g_k dY_k/dxyz`` and the double
  backward built on the Hessian.
* the radial expansion of Eq. expansion, ``c_{nlm} = sum_k R_{nl}(r_k) Y_l^m(r_k)``
  per centre, with the radial values given.

This route deliberately does NOT use the Cartesian recursions the CUDA path is
built on (Eqs. define-q, iter-q, iter-sc, iter-deri): it goes through theta and
phi. The only shared element is the mathematical definition.

Readings of the paper taken here (the paper is silent or ambiguous):

* column order inside an l block is m = -l..l, so entry (l, m) is column
  ``l*l + l + m`` (Section 3 asks for "all (l,m) up to l_max" but prints no order);
* the ``sqrt(1 - t^2)`` of Eq. recur-p is evaluated as ``r_xy / r`` (never from
  t), and cos(theta) as ``z / r``, so that points 1e-9 rad from the poles keep
  their digits;
* at r = 0 the scaled output is the polynomial's value (only l = 0 is nonzero)
  and its gradient is the polynomial's gradient (constant for l = 1, zero for
  l >= 2); the normalized output at r = 0 is defined as Y_0^0 = 1/sqrt(4 pi),
  all other values and all derivatives 0;
* on the z axis phi = atan2(0, 0) = 0, which is the limit the formulas need.

Pins (tests/test_oracle_pins.py): textbook closed forms for l <= 3, a library
routine (scipy's complex spherical harmonics), the addition theorem, exact
quadrature orthonormality, rotation invariance, central finite differences for
gradients, the gradient block-norm identity, and for the Hessian the closed
forms, the finite-difference Hessian, the addition theorem differentiated twice
(with numpy's Legendre series), the exact Hessian block norm
sum_m |d_i d_j r^l Y_l^m|^2 = r^(2l-4) l (l-1) (2l-1) (2l+1)^2 / (4 pi), its
symmetry, the harmonic (Laplace) property and Euler's homogeneity relation.
Every function below is pinned; none is "parity unpinned".
"""

from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np

__all__ = [
    "column",
    "prefactor",
    "prefactor_table",
    "legendre_table",
    "legendre_derivative_table",
    "spherical_harmonics",
    "spherical_harmonics_grad",
    "spherical_harmonics_hessian",
    "spherical_harmonics_hessian_fd",
    "backward",
    "double_backward",
    "expansion",
]


def column(l: int, m: int) -> int:
    """Column of (l, m) in an output row: blocks by l, m = -l..l inside a block."""
    return l * l + l + m


@lru_cache(maxsize=None)
def prefactor(l: int, m: int) -> float:
    """F_l^m of Eq. Flm: (-1)^m sqrt((2l+1)/(2 pi) * (l-m)!/(l+m)!), 0 <= m <= l.

    The factorial ratio is formed exactly as a rational number and brought into
    the normal floating-point range by an exact power-of-four scaling before the
    square root, so F is accurate to a few ulp for any l used here.
    """
    if not (0 <= m <= l):
        raise ValueError("need 0 <= m <= l")
    ratio = Fraction(math.factorial(l - m), math.factorial(l + m))
    # ratio * 4**e lies in [1, 4) for e chosen from the bit lengths.
    e = (ratio.denominator.bit_length() - ratio.numerator.bit_length()) // 2 + 1
    scaled = float(ratio * (Fraction(4) ** e))
    root = math.ldexp(math.sqrt(scaled), -e)
    sign = -1.0 if (m % 2) else 1.0
    return sign * math.sqrt((2 * l + 1) / (2.0 * math.pi)) * root


def prefactor_table(l_max: int) -> np.ndarray:
    """[l_max+1, l_max+1] array with F_l^m at [l, m] (m <= l), zero elsewhere."""
    t = np.zeros((l_max + 1, l_max + 1))
    for l in range(l_max + 1):
        for m in range(l + 1):
            t[l, m] = prefactor(l, m)
    return t


def legendre_table(l_max: int, t: np.ndarray, u: np.ndarray):
    """Associated Legendre functions by the textbook recursion, Eq. recur-p.

    ``t`` is cos(theta) and ``u`` is sin(theta) >= 0, both given (``u`` stands
    for the ``sqrt(1 - t^2)`` of Eq. recur-p). Returns ``(P, Pbar)`` with
    ``P[l, m]`` = P_l^m(t) (Condon-Shortley sign as in Eq. recur-p) and, for
    m >= 1, ``Pbar[l, m]`` = P_l^m / sin(theta). ``Pbar`` obeys the same
    recursion in l (its coefficients depend on t only) and is seeded from
    ``P_m^m / u = -(2m-1) P_{m-1}^{m-1}``, so it needs no division and stays
    finite on the z axis.
    """
    t = np.asarray(t, dtype=np.float64)
    u = np.asarray(u, dtype=np.float64)
    shape = (l_max + 1, l_max + 1) + t.shape
    P = np.zeros(shape)
    Pbar = np.zeros(shape)
    P[0, 0] = 1.0
    for m in range(1, l_max + 1):
        P[m, m] = -(2 * m - 1) * u * P[m - 1, m - 1]
        Pbar[m, m] = -(2 * m - 1) * P[m - 1, m - 1]
    for m in range(0, l_max):
        P[m + 1, m] = (2 * m + 1) * t * P[m, m]
        if m >= 1:
            Pbar[m + 1, m] = (2 * m + 1) * t * Pbar[m, m]
    for m in range(0, l_max + 1):
        for l in range(m + 2, l_max + 1):
            P[l, m] = ((2 * l - 1) * t * P[l - 1, m] - (l + m - 1) * P[l - 2, m]) / (l - m)
            if m >= 1:
                Pbar[l, m] = (
                    (2 * l - 1) * t * Pbar[l - 1, m] - (l + m - 1) * Pbar[l - 2, m]
                ) / (l - m)
    return P, Pbar


def _angles(xyz: np.ndarray):
    """r, cos(theta), sin(theta), phi for each point (theta = 0, phi = 0 at r = 0)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    if xyz.ndim != 2 or xyz.shape[1] != 3:
        raise ValueError("xyz must be [n, 3]")
    x, y, z = xyz[:, 0], xyz[:, 1], xyz[:, 2]
    r = np.sqrt(x * x + y * y + z * z)
    rxy = np.hypot(x, y)
    safe = np.where(r > 0, r, 1.0)
    t = np.where(r > 0, z / safe, 1.0)
    u = np.where(r > 0, rxy / safe, 0.0)
    phi = np.arctan2(y, x)
    return r, t, u, phi


def _unit_sphere_parts(xyz: np.ndarray, l_max: int):
    """Y_l^m on the unit sphere and its two angular derivatives, all [n, K].

    Returns ``(r, t, u, phi, Y, dYdtheta, dYdphi_over_sin)`` where the last is
    (1/sin theta) dY/dphi, evaluated through Pbar so it is finite at the poles.
    """
    r, t, u, phi = _angles(xyz)
    n = r.shape[0]
    K = (l_max + 1) ** 2
    P, Pbar = legendre_table(l_max + 1, t, u)
    Y = np.zeros((n, K))
    dth = np.zeros((n, K))
    dph = np.zeros((n, K))
    inv_sqrt2 = 1.0 / math.sqrt(2.0)
    for l in range(l_max + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            F = prefactor(l, am)
            # dP_l^m/dtheta in the Condon-Shortley convention of Eq. recur-p.
            if am == 0:
                dP = P[l, 1]
            else:
                dP = 0.5 * (P[l, am + 1] - (l + am) * (l - am + 1) * P[l, am - 1])
            k = column(l, m)
            if m < 0:
                trig, dtrig = np.sin(am * phi), am * np.cos(am * phi)
            elif m == 0:
                trig, dtrig = inv_sqrt2, 0.0
            else:
                trig, dtrig = np.cos(m * phi), -m * np.sin(m * phi)
            Y[:, k] = F * P[l, am] * trig
            dth[:, k] = F * dP * trig
            if am > 0:
                dph[:, k] = F * Pbar[l, am] * dtrig
    return r, t, u, phi, Y, dth, dph


def _lvec(l_max: int) -> np.ndarray:
    return np.concatenate([np.full(2 * l + 1, l, dtype=np.float64) for l in range(l_max + 1)])


def spherical_harmonics(xyz, l_max: int, normalized: bool = False) -> np.ndarray:
    """Real spherical harmonics, [n, (l_max+1)^2] in FP64.

    normalized=False: the scaled form r^l Y_l^m (Section 2).
    normalized=True: Y_l^m on the unit sphere (Section 3).
    """
    r, t, u, phi, Y, _, _ = _unit_sphere_parts(xyz, l_max)
    if normalized:
        out = Y.copy()
        zero = r == 0
        out[zero, :] = 0.0
        out[zero, 0] = 1.0 / math.sqrt(4.0 * math.pi)
        return out
    rl = r[:, None] ** _lvec(l_max)[None, :]
    return Y * rl


def spherical_harmonics_grad(xyz, l_max: int, normalized: bool = False):
    """(values [n, K], gradients [n, 3, K]) in FP64, analytic chain rule.

    With unit vectors r_hat, theta_hat, phi_hat, the scaled form has
    grad(r^l Y) = r^(l-1) (l Y r_hat + dY/dtheta theta_hat
    + (1/sin theta) dY/dphi phi_hat); the normalized form drops the radial term
    and carries 1/r instead of r^(l-1).
    """
    r, t, u, phi, Y, dth, dph = _unit_sphere_parts(xyz, l_max)
    cp, sp_ = np.cos(phi), np.sin(phi)
    rhat = np.stack([u * cp, u * sp_, t], axis=1)  # [n, 3]
    that = np.stack([t * cp, t * sp_, -u], axis=1)
    phat = np.stack([-sp_, cp, np.zeros_like(cp)], axis=1)
    lv = _lvec(l_max)
    ang = that[:, :, None] * dth[:, None, :] + phat[:, :, None] * dph[:, None, :]
    if normalized:
        zero = r == 0
        inv_r = np.where(zero, 0.0, 1.0 / np.where(zero, 1.0, r))
        grad = ang * inv_r[:, None, None]
        vals = Y.copy()
        vals[zero, :] = 0.0
        vals[zero, 0] = 1.0 / math.sqrt(4.0 * math.pi)
        return vals, grad
    rad = lv[None, None, :] * Y[:, None, :] * rhat[:, :, None]
    rl1 = r[:, None] ** np.maximum(lv - 1.0, 0.0)[None, :]
    # r^(l-1) is 0 at r = 0 for l >= 2 and 1 for l = 1 (0**0); l = 0 has no gradient.
    rl1 = np.where(lv[None, :] == 0, 0.0, rl1)
    grad = (rad + ang) * rl1[:, None, :]
    vals = Y * (r[:, None] ** lv[None, :])
    return vals, grad


def legendre_derivative_table(l_max: int, t: np.ndarray, extra: int = 2) -> np.ndarray:
    """t-derivatives of the Legendre polynomials: ``A[l, m]`` = d^m P_l / dt^m.

    Shape [l_max+1, l_max+1+extra, ...t.shape]; entries with m > l are 0 (P_l
    has degree l). With the Condon-Shortley sign of Eq. recur-p,
    P_l^m(t) = (-1)^m (1-t^2)^(m/2) A[l, m], so A obeys the recursion of Eq.
    recur-p with the common factor (-1)^m sin^m(theta) divided out:
    A_m^m = (2m-1)!!, A_{m+1}^m = (2m+1) t A_m^m and
    (l-m) A_l^m = (2l-1) t A_{l-1}^m - (l+m-1) A_{l-2}^m.
    """
    t = np.asarray(t, dtype=np.float64)
    A = np.zeros((l_max + 1, l_max + 1 + extra) + t.shape)
    seed = 1.0  # (2m-1)!!, starting from (-1)!! = 1
    for m in range(0, l_max + 1):
        if m > 0:
            seed *= 2 * m - 1
        A[m, m] = seed
        if m + 1 <= l_max:
            A[m + 1, m] = (2 * m + 1) * t * seed
        for l in range(m + 2, l_max + 1):
            A[l, m] = ((2 * l - 1) * t * A[l - 1, m] - (l + m - 1) * A[l - 2, m]) / (l - m)
    return A


def _sin_power(u: np.ndarray, k: int) -> np.ndarray:
    """sin(theta)^k for k >= 0; 0 for k < 0, where every caller's coefficient is 0."""
    if k < 0:
        return np.zeros_like(u)
    return u ** k


def spherical_harmonics_hessian(xyz, l_max: int, normalized: bool = False) -> np.ndarray:
    """Hessians [n, 3, 3, K] in FP64, analytic; H[:, i, j, k] = d^2 Y_k / dx_i dx_j.

    With f = r^p Y(theta, phi) (p = l for the scaled form, p = 0 for the
    normalized one), the gradient is G = r^(p-1) v with
    v = p Y r_hat + Y_theta theta_hat + W phi_hat and W = Y_phi / sin(theta).
    Differentiating G once more in spherical coordinates (d r_hat/d theta =
    theta_hat, d theta_hat/d theta = -r_hat, d r_hat/d phi = sin(theta) phi_hat,
    d theta_hat/d phi = cos(theta) phi_hat, d phi_hat/d phi =
    -(sin(theta) r_hat + cos(theta) theta_hat)) gives

        H_ij = r^(p-2) [ (p-1) v_i r_hat_j + a_i theta_hat_j + b_i phi_hat_j ],
        a = (p-1) Y_theta r_hat + (p Y + Y_theta_theta) theta_hat + W_theta phi_hat,
        b = (p-1) W r_hat + W_theta theta_hat + (p Y + Z) phi_hat,

    with Z = cot(theta) Y_theta + Y_phi_phi / sin^2(theta). For one (l, m),
    Y = F_l^|m| P_l^|m|(cos theta) T(phi) (Eq. real-sh-spherical). Writing
    P = (-1)^m s^m A0 with s = sin(theta), t = cos(theta) and A0, A1, A2 the
    m-th, (m+1)-th and (m+2)-th t-derivatives of P_l (dt/dtheta = -s):

        P_theta       = (-1)^m [m s^(m-1) t A0 - s^(m+1) A1]
        P_theta_theta = (-1)^m [m(m-1) s^(m-2) t^2 A0 - m s^m A0
                                - (2m+1) s^m t A1 + s^(m+2) A2]
        d(P/s)/dtheta = (-1)^m [(m-1) s^(m-2) t A0 - s^m A1]
        cot P_theta - m^2 P/s^2 = (-1)^m [m(1-m) s^(m-2) A0 - m s^m A0 - t s^m A1]

    (the last uses t^2 = 1 - s^2). Every negative power of s carries a
    coefficient that vanishes for the m where it would be negative, so the
    expressions are finite on the z axis. At r = 0 the scaled Hessian is the
    polynomial's (constant for l = 2, zero otherwise); the normalized one is 0.
    """
    r, t, u, phi = _angles(xyz)
    n = r.shape[0]
    K = (l_max + 1) ** 2
    H = np.zeros((n, 3, 3, K))
    A = legendre_derivative_table(l_max, t)
    cp, sp_ = np.cos(phi), np.sin(phi)
    zero = np.zeros_like(cp)
    rhat = np.stack([u * cp, u * sp_, t], axis=1)  # [n, 3]
    that = np.stack([t * cp, t * sp_, -u], axis=1)
    phat = np.stack([-sp_, cp, zero], axis=1)
    at_origin = r == 0
    rsafe = np.where(at_origin, 1.0, r)
    inv_sqrt2 = 1.0 / math.sqrt(2.0)
    for l in range(l_max + 1):
        p = 0.0 if normalized else float(l)
        # r^(p-2); the origin is filled in below.
        rp2 = rsafe ** (p - 2.0)
        for m in range(-l, l + 1):
            am = abs(m)
            cF = prefactor(l, am) * (-1.0 if am % 2 else 1.0)
            A0, A1, A2 = A[l, am], A[l, am + 1], A[l, am + 2]
            s_m2, s_m1 = _sin_power(u, am - 2), _sin_power(u, am - 1)
            s_m, s_p1, s_p2 = _sin_power(u, am), _sin_power(u, am + 1), _sin_power(u, am + 2)
            P0 = cF * s_m * A0
            Pt = cF * (am * s_m1 * t * A0 - s_p1 * A1)
            Ptt = cF * (am * (am - 1) * s_m2 * t * t * A0 - am * s_m * A0
                        - (2 * am + 1) * s_m * t * A1 + s_p2 * A2)
            Pbt = cF * ((am - 1) * s_m2 * t * A0 - s_m * A1)
            Pz = cF * (am * (1 - am) * s_m2 * A0 - am * s_m * A0 - t * s_m * A1)
            Pb = cF * s_m1 * A0
            if m < 0:
                T, dT = np.sin(am * phi), am * np.cos(am * phi)
            elif m == 0:
                T, dT = np.full_like(phi, inv_sqrt2), zero
            else:
                T, dT = np.cos(m * phi), -m * np.sin(m * phi)
            Yv, Yt, Ytt, Z = P0 * T, Pt * T, Ptt * T, Pz * T
            W, Wt = Pb * dT, Pbt * dT
            v = p * Yv[:, None] * rhat + Yt[:, None] * that + W[:, None] * phat
            a = (p - 1.0) * Yt[:, None] * rhat + (p * Yv + Ytt)[:, None] * that + Wt[:, None] * phat
            b = (p - 1.0) * W[:, None] * rhat + Wt[:, None] * that + (p * Yv + Z)[:, None] * phat
            Hk = ((p - 1.0) * v[:, :, None] * rhat[:, None, :] + a[:, :, None] * that[:, None, :]
                  + b[:, :, None] * phat[:, None, :])
            Hk = Hk * rp2[:, None, None]
            if normalized or l != 2:
                Hk[at_origin] = 0.0
            H[:, :, :, column(l, m)] = Hk
    return H


def spherical_harmonics_hessian_fd(xyz, l_max: int, normalized: bool = False, h=None):
    """Hessians [n, 3, 3, K] by differences of the analytic gradient (cross-check).

    Central differences with step h and h/2 combined by one Richardson step
    (error O(h^4)); h defaults to 1e-3 * max(r, 1e-3). H[:, i, j, k] is
    d^2 Y_k / dx_i dx_j. Used at l_max <= 16, where the truncation error is
    below ~1e-8 relative to the Hessian's block scale. It shares only the
    gradient with ``spherical_harmonics_hessian`` and pins it.
    """
    xyz = np.asarray(xyz, dtype=np.float64)
    n = xyz.shape[0]
    K = (l_max + 1) ** 2
    r = np.linalg.norm(xyz, axis=1)
    if h is None:
        h = 1e-3 * np.maximum(r, 1e-3)
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), (n,))
    H = np.zeros((n, 3, 3, K))

    def central(step, j):
        e = np.zeros((n, 3))
        e[:, j] = step
        _, gp = spherical_harmonics_grad(xyz + e, l_max, normalized)
        _, gm = spherical_harmonics_grad(xyz - e, l_max, normalized)
        return (gp - gm) / (2.0 * step)[:, None, None]

    for j in range(3):
        d1 = central(h, j)
        d2 = central(0.5 * h, j)
        H[:, :, j, :] = (4.0 * d2 - d1) / 3.0
    return 0.5 * (H + H.transpose(0, 2, 1, 3))


def backward(xyz, g, l_max: int, normalized: bool = False) -> np.ndarray:
    """dL/dxyz [n, 3] = sum_k g[n, k] dY_k/dxyz for an upstream gradient g [n, K]."""
    _, grad = spherical_harmonics_grad(xyz, l_max, normalized)
    return np.einsum("nik,nk->ni", grad, np.asarray(g, dtype=np.float64))


def double_backward(xyz, g, v, l_max: int, normalized: bool = False, hessian=None):
    """Adjoint of ``backward`` for a cotangent v [n, 3] of its output.

    grad_g[n, k] = sum_j v[n, j] dY_k/dx_j and
    grad_xyz[n, i] = sum_k g[n, k] sum_j v[n, j] d^2 Y_k/dx_i dx_j.
    """
    _, grad = spherical_harmonics_grad(xyz, l_max, normalized)
    v = np.asarray(v, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    H = spherical_harmonics_hessian(xyz, l_max, normalized) if hessian is None else hessian
    grad_g = np.einsum("njk,nj->nk", grad, v)
    grad_xyz = np.einsum("nijk,nj,nk->ni", H, v, g)
    return grad_g, grad_xyz


def expansion(xyz, radial, offsets, l_max: int, normalized: bool = False) -> np.ndarray:
    """Eq. expansion per centre: c[i, n, (l,m)] = sum_k R[k, n, l] Y_l^m(x_k).

    ``xyz`` [E, 3] are the points (edge vectors) grouped by centre, centre i
    owning rows offsets[i]:offsets[i+1]; ``radial`` [E, n_rad, l_max+1] holds
    R_nl evaluated at each point; Y is the scaled r^l Y_l^m (the paper absorbs
    r^-l into R) or, with ``normalized``, Y_l^m. Returns [n_centres, n_rad, K].
    """
    Y = spherical_harmonics(xyz, l_max, normalized)
    R = np.asarray(radial, dtype=np.float64)
    offsets = np.asarray(offsets, dtype=np.int64)
    lv = np.concatenate([np.full(2 * l + 1, l) for l in range(l_max + 1)])
    n_centres = offsets.shape[0] - 1
    out = np.zeros((n_centres, R.shape[1], Y.shape[1]))
    for i in range(n_centres):
        a, b = offsets[i], offsets[i + 1]
        if b > a:
            out[i] = np.einsum("knl,kl->nl", R[a:b][:, :, lv], Y[a:b])
    return out
