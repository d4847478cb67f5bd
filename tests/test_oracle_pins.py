"""Pins of the FP64 oracle to facts other than itself (CPU only).

Each test ties the oracle to a value the mathematics fixes independently of
how the oracle computes it: textbook closed forms (differentiated by sympy),
scipy's complex spherical harmonics, the addition theorem, exact quadrature,
rotation invariance, finite differences, homogeneity and harmonicity, and
50-digit mpmath values near the poles. A plausible slip in the oracle (a sign,
a prefactor, a swapped index, the Condon-Shortley phase, the dP/dtheta formula,
a Richardson weight) fails at least one of them (see test_planted_mistakes).
"""

import math

import numpy as np
import pytest
import scipy.special as sps
import sympy as sp
from numpy.polynomial import legendre as npl

import oracle.sph_oracle as orc
from oracle import (
    backward,
    column,
    double_backward,
    prefactor,
    spherical_harmonics,
    spherical_harmonics_grad,
    spherical_harmonics_hessian,
    spherical_harmonics_hessian_fd,
)
from paper_2302_08381_gb300 import inputs

# ---------------------------------------------------------------------------
# Textbook closed forms of the real spherical harmonics on the unit sphere,
# l <= 3, without the Condon-Shortley phase (the convention Eq. real-sh-spherical
# reaches: the (-1)^m of Eq. Flm cancels the sign of Eq. recur-p). Written as
# homogeneous polynomials, i.e. r^l Y_l^m; standard real-harmonics table.
# ---------------------------------------------------------------------------
X, Y_, Z = sp.symbols("x y z", real=True)
PI = sp.pi
CLOSED = {
    (0, 0): sp.Rational(1, 2) * sp.sqrt(1 / PI),
    (1, -1): sp.sqrt(3 / (4 * PI)) * Y_,
    (1, 0): sp.sqrt(3 / (4 * PI)) * Z,
    (1, 1): sp.sqrt(3 / (4 * PI)) * X,
    (2, -2): sp.Rational(1, 2) * sp.sqrt(15 / PI) * X * Y_,
    (2, -1): sp.Rational(1, 2) * sp.sqrt(15 / PI) * Y_ * Z,
    (2, 0): sp.Rational(1, 4) * sp.sqrt(5 / PI) * (2 * Z**2 - X**2 - Y_**2),
    (2, 1): sp.Rational(1, 2) * sp.sqrt(15 / PI) * X * Z,
    (2, 2): sp.Rational(1, 4) * sp.sqrt(15 / PI) * (X**2 - Y_**2),
    (3, -3): sp.Rational(1, 4) * sp.sqrt(35 / (2 * PI)) * Y_ * (3 * X**2 - Y_**2),
    (3, -2): sp.Rational(1, 2) * sp.sqrt(105 / PI) * X * Y_ * Z,
    (3, -1): sp.Rational(1, 4) * sp.sqrt(21 / (2 * PI)) * Y_ * (4 * Z**2 - X**2 - Y_**2),
    (3, 0): sp.Rational(1, 4) * sp.sqrt(7 / PI) * Z * (2 * Z**2 - 3 * X**2 - 3 * Y_**2),
    (3, 1): sp.Rational(1, 4) * sp.sqrt(21 / (2 * PI)) * X * (4 * Z**2 - X**2 - Y_**2),
    (3, 2): sp.Rational(1, 4) * sp.sqrt(105 / PI) * Z * (X**2 - Y_**2),
    (3, 3): sp.Rational(1, 4) * sp.sqrt(35 / (2 * PI)) * X * (X**2 - 3 * Y_**2),
}


def _lambd(expr):
    return sp.lambdify((X, Y_, Z), expr, "numpy")


def _closed_eval(xyz):
    """values, gradients, Hessians of the closed forms (scaled), via sympy."""
    n = xyz.shape[0]
    K = 16
    V = np.zeros((n, K))
    G = np.zeros((n, 3, K))
    H = np.zeros((n, 3, 3, K))
    syms = (X, Y_, Z)
    args = (xyz[:, 0], xyz[:, 1], xyz[:, 2])
    for (l, m), e in CLOSED.items():
        k = column(l, m)
        V[:, k] = np.broadcast_to(_lambd(e)(*args), (n,))
        for i in range(3):
            G[:, i, k] = np.broadcast_to(_lambd(sp.diff(e, syms[i]))(*args), (n,))
            for j in range(3):
                H[:, i, j, k] = np.broadcast_to(
                    _lambd(sp.diff(e, syms[i], syms[j]))(*args), (n,)
                )
    return V, G, H


def _real_from_scipy(l_max, theta, phi):
    """Real harmonics assembled from scipy's complex ones (which carry the
    Condon-Shortley phase): m>0 -> sqrt2 (-1)^m Re, m<0 -> sqrt2 (-1)^m Im."""
    out = np.zeros((theta.shape[0], (l_max + 1) ** 2))
    for l in range(l_max + 1):
        for m in range(-l, l + 1):
            c = sps.sph_harm_y(l, abs(m), theta, phi)
            if m > 0:
                v = math.sqrt(2.0) * (-1) ** m * c.real
            elif m < 0:
                v = math.sqrt(2.0) * (-1) ** m * c.imag
            else:
                v = c.real
            out[:, column(l, m)] = v
    return out


def _block_scale(l_max, r):
    """Per-column r^l sqrt((2l+1)/(4 pi)): the exact rms size of an l block."""
    cols = []
    for l in range(l_max + 1):
        cols += [math.sqrt((2 * l + 1) / (4 * math.pi))] * (2 * l + 1)
    lv = np.concatenate([np.full(2 * l + 1, l) for l in range(l_max + 1)])
    return np.asarray(cols)[None, :] * r[:, None] ** lv[None, :]


# --------------------------------------------------------------------------- prefactor
def test_prefactor_closed_form_vs_appendix_c_iteration():
    """Eq. Flm (closed form) agrees with the App. C iteration and with lgamma."""
    for l in range(0, 101):
        f = math.sqrt((2 * l + 1) / (2 * math.pi))
        assert prefactor(l, 0) == pytest.approx(f, rel=1e-15)
        for m in range(1, l + 1):
            f = -f / math.sqrt((l + m) * (l + 1 - m))
            assert prefactor(l, m) == pytest.approx(f, rel=1e-12), (l, m)
            lg = 0.5 * (
                math.log((2 * l + 1) / (2 * math.pi)) + math.lgamma(l - m + 1) - math.lgamma(l + m + 1)
            )
            assert abs(prefactor(l, m)) == pytest.approx(math.exp(lg), rel=1e-11)
            assert math.copysign(1, prefactor(l, m)) == (-1) ** m


# --------------------------------------------------------------------------- values
@pytest.mark.parametrize("normalized", [False, True])
def test_closed_forms_l3(normalized):
    xyz = inputs.normal_points(200, seed=11)
    V, _, _ = _closed_eval(xyz)
    got = spherical_harmonics(xyz, 3, normalized)
    if normalized:
        r = np.linalg.norm(xyz, axis=1)
        lv = np.concatenate([np.full(2 * l + 1, l) for l in range(4)])
        V = V / r[:, None] ** lv[None, :]
    np.testing.assert_allclose(got, V, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("l_max", [6, 20])
def test_matches_scipy_complex_harmonics(l_max):
    xyz = inputs.normal_points(300, seed=12)
    r = np.linalg.norm(xyz, axis=1)
    theta = np.arccos(np.clip(xyz[:, 2] / r, -1, 1))
    phi = np.arctan2(xyz[:, 1], xyz[:, 0])
    ref = _real_from_scipy(l_max, theta, phi)
    got = spherical_harmonics(xyz, l_max, normalized=True)
    np.testing.assert_allclose(got, ref, atol=1e-12 * math.sqrt(2 * l_max + 1))


@pytest.mark.parametrize("l_max", [8, 50])
def test_addition_theorem(l_max):
    """sum_m Y_l^m(u) Y_l^m(v) = (2l+1)/(4 pi) P_l(u.v), P_l from scipy."""
    a = inputs.normal_points(64, seed=13)
    b = inputs.normal_points(64, seed=14)
    ya = spherical_harmonics(a, l_max, True)
    yb = spherical_harmonics(b, l_max, True)
    ua = a / np.linalg.norm(a, axis=1, keepdims=True)
    ub = b / np.linalg.norm(b, axis=1, keepdims=True)
    cosg = np.sum(ua * ub, axis=1)
    for l in range(l_max + 1):
        s = slice(l * l, (l + 1) ** 2)
        lhs = np.sum(ya[:, s] * yb[:, s], axis=1)
        rhs = (2 * l + 1) / (4 * math.pi) * sps.eval_legendre(l, cosg)
        np.testing.assert_allclose(lhs, rhs, atol=1e-12 * (2 * l + 1))
        sq = np.sum(ya[:, s] ** 2, axis=1)
        np.testing.assert_allclose(sq, (2 * l + 1) / (4 * math.pi), rtol=1e-12)


@pytest.mark.parametrize("l_max", [5, 12])
def test_quadrature_orthonormality(l_max):
    """Gauss-Legendre in cos(theta) x uniform phi integrates Y Y^T exactly."""
    nt, nph = l_max + 1, 2 * l_max + 2
    t, w = np.polynomial.legendre.leggauss(nt)
    phi = 2 * np.pi * np.arange(nph) / nph
    T, PH = np.meshgrid(t, phi, indexing="ij")
    W = (w[:, None] * np.full(nph, 2 * np.pi / nph)[None, :]).ravel()
    st = np.sqrt(1 - T**2)
    xyz = np.stack([st * np.cos(PH), st * np.sin(PH), T], axis=-1).reshape(-1, 3)
    Y = spherical_harmonics(xyz, l_max, True)
    gram = (Y * W[:, None]).T @ Y
    np.testing.assert_allclose(gram, np.eye(Y.shape[1]), atol=1e-13)


def test_rotation_invariance():
    rng = np.random.default_rng(15)
    qm, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    a = inputs.normal_points(50, seed=16)
    b = inputs.normal_points(50, seed=17)
    l_max = 10
    Ya, Yb = spherical_harmonics(a, l_max), spherical_harmonics(b, l_max)
    Ra, Rb = spherical_harmonics(a @ qm.T, l_max), spherical_harmonics(b @ qm.T, l_max)
    for l in range(l_max + 1):
        s = slice(l * l, (l + 1) ** 2)
        np.testing.assert_allclose(
            np.sum(Ra[:, s] * Rb[:, s], 1), np.sum(Ya[:, s] * Yb[:, s], 1), rtol=1e-11, atol=1e-12
        )
        np.testing.assert_allclose(np.sum(Ra[:, s] ** 2, 1), np.sum(Ya[:, s] ** 2, 1), rtol=1e-11)


def test_pole_special_cases():
    """At +z: Y_l^0 = sqrt((2l+1)/4pi) r^l, all m != 0 vanish; -z adds (-1)^l."""
    l_max = 12
    xyz = np.array([[0.0, 0.0, 2.0], [0.0, 0.0, -1.5], [0.0, 0.0, 0.0]])
    Y = spherical_harmonics(xyz, l_max)
    for l in range(l_max + 1):
        base = math.sqrt((2 * l + 1) / (4 * math.pi))
        for m in range(-l, l + 1):
            k = column(l, m)
            want_p = base * 2.0**l if m == 0 else 0.0
            want_m = base * (-1.5) ** l if m == 0 else 0.0
            want_0 = base if (l == 0) else 0.0
            assert Y[0, k] == pytest.approx(want_p, rel=1e-13, abs=1e-300)
            assert Y[1, k] == pytest.approx(want_m, rel=1e-13, abs=1e-300)
            assert Y[2, k] == pytest.approx(want_0, abs=0)


def test_normalized_zero_vector_convention():
    xyz = np.zeros((2, 3))
    v, g = spherical_harmonics_grad(xyz, 4, normalized=True)
    assert v[0, 0] == pytest.approx(1 / math.sqrt(4 * math.pi))
    assert np.all(v[:, 1:] == 0) and np.all(g == 0)
    # scaled gradient at r = 0: constants for l = 1, zeros otherwise
    vs, gs = spherical_harmonics_grad(xyz, 4, normalized=False)
    c = math.sqrt(3 / (4 * math.pi))
    np.testing.assert_allclose(gs[0, :, 1:4], c * np.array([[0, 0, 1], [1, 0, 0], [0, 1, 0]]), atol=1e-15)
    assert np.all(gs[0, :, 4:] == 0) and np.all(vs[0, 1:] == 0)


def test_near_pole_high_precision_mpmath():
    """50-digit mpmath harmonics at points 1e-9..1e-4 rad from the poles, L=50."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    l_max = 50
    xyz = inputs.near_pole_points(6, seed=18)
    xyz[0] = [1e-9, 2e-9, 1.0]
    got = spherical_harmonics(xyz, l_max, True)
    for p in range(xyz.shape[0]):
        x, y, z = (mpmath.mpf(float(c)) for c in xyz[p])
        r = mpmath.sqrt(x * x + y * y + z * z)
        th = mpmath.atan2(mpmath.sqrt(x * x + y * y), z)
        ph = mpmath.atan2(y, x)
        for l in range(0, l_max + 1, 7):
            for m in range(-l, l + 1, 3):
                c = mpmath.spherharm(l, abs(m), th, ph)
                if m > 0:
                    ref = mpmath.sqrt(2) * (-1) ** m * mpmath.re(c)
                elif m < 0:
                    ref = mpmath.sqrt(2) * (-1) ** m * mpmath.im(c)
                else:
                    ref = mpmath.re(c)
                assert abs(got[p, column(l, m)] - float(ref)) <= 2e-13 * math.sqrt(2 * l + 1), (p, l, m)


# --------------------------------------------------------------------------- gradients
def _fd_grad(f, xyz, h):
    """Richardson-extrapolated central differences of f (values [n, K])."""
    n = xyz.shape[0]
    out = []
    for j in range(3):
        e = np.zeros((n, 3))
        e[:, j] = 1.0

        def d(s):
            return (f(xyz + s * e) - f(xyz - s * e)) / (2 * s)

        out.append((4 * d(h / 2) - d(h)) / 3)
    return np.stack(out, axis=1)


@pytest.mark.parametrize("normalized", [False, True])
def test_gradient_closed_forms(normalized):
    xyz = inputs.normal_points(100, seed=19)
    _, G, _ = _closed_eval(xyz)
    _, g = spherical_harmonics_grad(xyz, 3, normalized)
    if not normalized:
        np.testing.assert_allclose(g, G, atol=1e-13)
    else:
        fd = _fd_grad(lambda p: spherical_harmonics(p, 3, True), xyz, 1e-3)
        np.testing.assert_allclose(g, fd, atol=1e-9)


@pytest.mark.parametrize("normalized", [False, True])
@pytest.mark.parametrize("kind", ["shell", "pole"])
def test_gradient_finite_differences(normalized, kind):
    l_max = 10
    if kind == "shell":
        xyz = inputs.shell_points(64, 0.7, 2.0, seed=20, dtype=np.float64)
    else:
        xyz = inputs.near_pole_points(64, max_angle=1e-3, seed=21)
    v, g = spherical_harmonics_grad(xyz, l_max, normalized)
    fd = _fd_grad(lambda p: spherical_harmonics(p, l_max, normalized), xyz, 1e-3)
    r = np.linalg.norm(xyz, axis=1)
    scale = np.max(np.abs(fd)) + 1
    np.testing.assert_allclose(g, fd, atol=2e-8 * scale)
    np.testing.assert_allclose(v, spherical_harmonics(xyz, l_max, normalized), rtol=0, atol=0)
    del r


@pytest.mark.parametrize("kind", ["shell", "pole"])
def test_gradient_block_norm_identity(kind):
    """sum_m |grad (r^l Y_l^m)|^2 = r^(2l-2) l (2l+1)^2 / (4 pi), every l up to 50,
    on shell points and on points 1e-9..1e-4 rad from both poles."""
    l_max = 50
    if kind == "shell":
        xyz = inputs.shell_points(80, 0.5, 1.5, seed=22, dtype=np.float64)
    else:
        xyz = inputs.pole_mix_points(80, seed=122) * 1.2
    _, g = spherical_harmonics_grad(xyz, l_max)
    r = np.linalg.norm(xyz, axis=1)
    for l in range(1, l_max + 1):
        s = slice(l * l, (l + 1) ** 2)
        lhs = np.sum(g[:, :, s] ** 2, axis=(1, 2))
        rhs = r ** (2 * l - 2) * l * (2 * l + 1) ** 2 / (4 * math.pi)
        np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


@pytest.mark.parametrize("normalized", [False, True])
def test_gradient_addition_theorem(normalized):
    """Addition theorem differentiated once in x, every l up to 50, pole mix:
    sum_m grad Y_l^m(x) Y_l^m(y) = (2l+1)/(4 pi) grad_x [|x|^p |y|^l P_l(x_hat . y_hat)]
    = (2l+1)/(4 pi) |y|^l r^(p-1) [p P x_hat + P' (y_hat - s x_hat)]."""
    l_max, n = 50, 40
    x = np.concatenate([inputs.pole_mix_points(n, seed=160) * 1.4,
                        inputs.shell_points(n, 0.5, 1.5, seed=161, dtype=np.float64)])
    _, G = spherical_harmonics_grad(x, l_max, normalized)
    r = np.linalg.norm(x, axis=1)
    xh = x / r[:, None]
    worst = 0.0
    for trial in range(3):
        yv = inputs.shell_points(2 * n, 0.5, 1.5, seed=162 + trial, dtype=np.float64)
        Ry = spherical_harmonics(yv, l_max, normalized)
        ry = np.linalg.norm(yv, axis=1)
        yh = yv / ry[:, None]
        s_ = np.sum(xh * yh, axis=1)
        for l in range(l_max + 1):
            sl = slice(l * l, (l + 1) ** 2)
            lhs = np.einsum("nik,nk->ni", G[:, :, sl], Ry[:, sl])
            e = np.zeros(l + 1)
            e[l] = 1.0
            P = npl.legval(s_, e)
            P1 = npl.legval(s_, npl.legder(e)) if l >= 1 else 0.0 * s_
            p = 0.0 if normalized else float(l)
            c = (2 * l + 1) / (4 * math.pi) * (np.ones(2 * n) if normalized else ry**l)
            rhs = (c * r ** (p - 1))[:, None] * ((p * P)[:, None] * xh + P1[:, None] * (yh - s_[:, None] * xh))
            scale = c * r ** (p - 1) * (l + 1)
            worst = max(worst, float(np.max(np.abs(lhs - rhs) / scale[:, None])))
    assert worst < 1e-13, worst


def test_gradient_euler_homogeneity():
    """x . grad(r^l Y) = l r^l Y (degree-l homogeneous polynomial)."""
    l_max = 16
    xyz = inputs.shell_points(80, 0.5, 3.0, seed=23, dtype=np.float64)
    v, g = spherical_harmonics_grad(xyz, l_max)
    lv = np.concatenate([np.full(2 * l + 1, l) for l in range(l_max + 1)])
    lhs = np.einsum("ni,nik->nk", xyz, g)
    scale = _block_scale(l_max, np.linalg.norm(xyz, axis=1))
    np.testing.assert_allclose(lhs / scale, lv[None, :] * v / scale, atol=1e-12 * l_max)


# --------------------------------------------------------------------------- Hessians
def _hess_block_scale(l_max, r, normalized=False):
    """[n, K]: exact rms size of an l block's Hessian (scaled form), also used
    as the error scale of the normalized one with r^(l-2) -> r^-2."""
    lv = np.concatenate([np.full(2 * l + 1, l) for l in range(l_max + 1)]).astype(np.float64)
    c = np.sqrt(np.maximum(lv * (lv - 1) * (2 * lv - 1), 1.0) * (2 * lv + 1) ** 2 / (4 * math.pi))
    pw = np.full_like(lv, -2.0) if normalized else np.maximum(lv - 2, 0)
    return c[None, :] * r[:, None] ** pw[None, :]


def _closed_eval_normalized(xyz):
    """Hessians of r^-l times the closed forms (the normalized harmonics), via sympy."""
    n = xyz.shape[0]
    H = np.zeros((n, 3, 3, 16))
    syms = (X, Y_, Z)
    args = (xyz[:, 0], xyz[:, 1], xyz[:, 2])
    rr = sp.sqrt(X**2 + Y_**2 + Z**2)
    for (l, m), e in CLOSED.items():
        k = column(l, m)
        f = e / rr**l
        for i in range(3):
            for j in range(i, 3):
                val = np.broadcast_to(_lambd(sp.diff(f, syms[i], syms[j]))(*args), (n,))
                H[:, i, j, k] = val
                H[:, j, i, k] = val
    return H


def _hessian_pin_points():
    """General points, points 1e-9..1e-4 rad from both poles, and exact z-axis points."""
    gen = inputs.normal_points(40, seed=24)
    pole = inputs.pole_mix_points(40, seed=124) * 1.7
    axis = np.array([[0.0, 0.0, 1.3], [0.0, 0.0, -0.6], [1e-12, 0.0, 2.0]])
    return np.concatenate([gen, pole, axis])


@pytest.mark.parametrize("normalized", [False, True])
def test_hessian_closed_forms(normalized):
    """Analytic Hessian vs sympy's second derivatives of the l <= 3 closed forms."""
    xyz = _hessian_pin_points()
    if normalized:
        ref = _closed_eval_normalized(xyz)
    else:
        _, _, ref = _closed_eval(xyz)
    got = spherical_harmonics_hessian(xyz, 3, normalized)
    scale = _hess_block_scale(3, np.linalg.norm(xyz, axis=1), normalized)[:, None, None, :]
    assert np.max(np.abs(got - ref) / scale) < 1e-13


def _legendre_kernel_hessian(x, yv, l, p):
    """d_i d_j of r^p P_l(x_hat . y_hat) in x, with numpy's Legendre series.

    With s = x_hat . y_hat and b = y_hat - s x_hat, direct differentiation
    gives r^(p-2) [p(p-1) P x_hat x_hat^T + (p-1) P' (x_hat b^T + b x_hat^T)
    + (p P - s P') (I - x_hat x_hat^T) + P'' b b^T].
    """
    r = np.linalg.norm(x, axis=1)
    xh = x / r[:, None]
    a = yv / np.linalg.norm(yv, axis=1)[:, None]
    s = np.sum(xh * a, axis=1)
    e = np.zeros(l + 1)
    e[l] = 1.0
    P = npl.legval(s, e)
    P1 = npl.legval(s, npl.legder(e)) if l >= 1 else 0.0 * s
    P2 = npl.legval(s, npl.legder(e, 2)) if l >= 2 else 0.0 * s
    b = a - s[:, None] * xh
    outer = lambda u, w: u[:, :, None] * w[:, None, :]  # noqa: E731
    H = ((p * (p - 1) * P)[:, None, None] * outer(xh, xh)
         + ((p - 1) * P1)[:, None, None] * (outer(xh, b) + outer(b, xh))
         + (p * P - s * P1)[:, None, None] * (np.eye(3)[None] - outer(xh, xh))
         + P2[:, None, None] * outer(b, b))
    return H * (r ** (p - 2.0))[:, None, None]


def test_legendre_kernel_hessian_formula():
    """The test's own kernel formula against sympy (so the pin below stands on it)."""
    x = inputs.shell_points(5, 0.5, 1.5, seed=140, dtype=np.float64)
    yv = inputs.shell_points(5, 0.5, 1.5, seed=141, dtype=np.float64)
    a1, a2, a3 = sp.symbols("a1 a2 a3", real=True)
    for l, p in ((3, 3), (4, 0), (5, 5)):
        rr = sp.sqrt(X**2 + Y_**2 + Z**2)
        s_ = (X * a1 + Y_ * a2 + Z * a3) / rr
        f = rr**p * sp.legendre(l, s_)
        got = _legendre_kernel_hessian(x, yv, l, p)
        yh = yv / np.linalg.norm(yv, axis=1)[:, None]
        for i, si in enumerate((X, Y_, Z)):
            for j, sj in enumerate((X, Y_, Z)):
                fn = sp.lambdify((X, Y_, Z, a1, a2, a3), sp.diff(f, si, sj), "numpy")
                ref = fn(x[:, 0], x[:, 1], x[:, 2], yh[:, 0], yh[:, 1], yh[:, 2])
                np.testing.assert_allclose(got[:, i, j], ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("normalized", [False, True])
@pytest.mark.parametrize("kind", ["shell", "pole"])
def test_hessian_addition_theorem(normalized, kind):
    """Addition theorem differentiated twice in x, every l up to 50:

    sum_m d_i d_j Y_l^m(x) Y_l^m(y) = (2l+1)/(4 pi) d_i d_j [|x|^p |y|^l P_l(x_hat . y_hat)]

    (p = l scaled, p = 0 and |y|^0 normalized). Three generic y per x fix
    every m component of each block."""
    l_max, n = 50, 40
    if kind == "shell":
        x = inputs.shell_points(n, 0.5, 1.5, seed=142, dtype=np.float64)
    else:
        x = inputs.pole_mix_points(n, seed=143) * 1.3
    H = spherical_harmonics_hessian(x, l_max, normalized)
    r = np.linalg.norm(x, axis=1)
    worst = 0.0
    for trial in range(3):
        yv = inputs.shell_points(n, 0.5, 1.5, seed=144 + trial, dtype=np.float64)
        Ry = spherical_harmonics(yv, l_max, normalized)
        ry = np.linalg.norm(yv, axis=1)
        for l in range(l_max + 1):
            sl = slice(l * l, (l + 1) ** 2)
            lhs = np.einsum("nijk,nk->nij", H[..., sl], Ry[:, sl])
            c = (2 * l + 1) / (4 * math.pi) * (np.ones(n) if normalized else ry**l)
            rhs = _legendre_kernel_hessian(x, yv, l, 0 if normalized else l) * c[:, None, None]
            scale = c * (r ** (-2.0) if normalized else r ** (l - 2.0)) * (l + 1) ** 2
            worst = max(worst, float(np.max(np.abs(lhs - rhs) / scale[:, None, None])))
    assert worst < 1e-13, worst


@pytest.mark.parametrize("kind", ["shell", "pole"])
def test_hessian_block_norm_identity(kind):
    """sum_m |d_i d_j (r^l Y_l^m)|^2 = r^(2l-4) l (l-1) (2l-1) (2l+1)^2 / (4 pi),
    every l up to 50 (the constant follows from the addition theorem; it is
    rotation invariant and was evaluated exactly at the pole)."""
    l_max = 50
    if kind == "shell":
        x = inputs.shell_points(60, 0.5, 1.5, seed=150, dtype=np.float64)
    else:
        x = inputs.pole_mix_points(60, seed=151) * 0.8
    H = spherical_harmonics_hessian(x, l_max)
    r = np.linalg.norm(x, axis=1)
    for l in range(l_max + 1):
        sl = slice(l * l, (l + 1) ** 2)
        lhs = np.sum(H[..., sl] ** 2, axis=(1, 2, 3))
        rhs = r ** (2 * l - 4.0) * l * (l - 1) * (2 * l - 1) * (2 * l + 1) ** 2 / (4 * math.pi)
        if l < 2:
            assert np.max(np.abs(lhs)) < 1e-26
        else:
            np.testing.assert_allclose(lhs, rhs, rtol=1e-12)


@pytest.mark.parametrize("l_max", [6, 20])
def test_hessian_harmonic_euler_symmetric(l_max):
    """trace H = 0 (solid harmonics are harmonic); sum_j x_j H_ij = (l-1) d_i Y;
    H symmetric; all to FP64 rounding."""
    xyz = np.concatenate([inputs.shell_points(40, 0.7, 2.0, seed=25, dtype=np.float64),
                          inputs.pole_mix_points(20, seed=125)])
    _, g = spherical_harmonics_grad(xyz, l_max)
    H = spherical_harmonics_hessian(xyz, l_max)
    hs = _hess_block_scale(l_max, np.linalg.norm(xyz, axis=1))
    tr = np.trace(H, axis1=1, axis2=2)
    assert np.max(np.abs(tr) / hs) < 1e-13
    lhs = np.einsum("nj,nijk->nik", xyz, H)
    lv = np.concatenate([np.full(2 * l + 1, l) for l in range(l_max + 1)])
    rhs = (lv[None, None, :] - 1.0) * g
    assert np.max(np.abs(lhs - rhs) / hs[:, None, :]) < 1e-13
    assert np.max(np.abs(H - H.transpose(0, 2, 1, 3)) / hs[:, None, None, :]) < 1e-13


@pytest.mark.parametrize("normalized", [False, True])
def test_hessian_matches_finite_differences(normalized):
    """Analytic Hessian vs Richardson central differences of the analytic gradient."""
    l_max = 12
    xyz = np.concatenate([inputs.shell_points(30, 0.7, 2.0, seed=152, dtype=np.float64),
                          inputs.near_pole_points(10, 1e-3, seed=153)])
    H = spherical_harmonics_hessian(xyz, l_max, normalized)
    Hfd = spherical_harmonics_hessian_fd(xyz, l_max, normalized)
    hs = _hess_block_scale(l_max, np.linalg.norm(xyz, axis=1), normalized)
    assert np.max(np.abs(H - Hfd) / hs[:, None, None, :]) < 1e-8


def test_hessian_at_origin():
    """r = 0: scaled Hessians are the constant ones of the l = 2 polynomials
    (zero otherwise); normalized ones are 0 by convention."""
    o = np.zeros((1, 3))
    _, _, ref = _closed_eval(o)
    H = spherical_harmonics_hessian(o, 4)
    np.testing.assert_allclose(H[..., :16], ref, atol=1e-15)
    assert np.all(H[..., 16:] == 0)
    assert np.all(spherical_harmonics_hessian(o, 4, True) == 0)


# --------------------------------------------------------------------------- adjoints
def test_backward_is_gradient_of_contraction():
    l_max = 6
    xyz = inputs.shell_points(30, 0.7, 3.0, seed=26, dtype=np.float64)
    g = inputs.upstream(30, 49, seed=27, dtype=np.float64)
    dx = backward(xyz, g, l_max)

    def loss(p):
        return np.sum(spherical_harmonics(p, l_max) * g, axis=1, keepdims=True)

    fd = _fd_grad(loss, xyz, 1e-3)[:, :, 0]
    np.testing.assert_allclose(dx, fd, rtol=1e-8, atol=1e-8)


def test_double_backward_is_gradient_of_backward():
    l_max = 6
    xyz = inputs.shell_points(20, 0.7, 3.0, seed=28, dtype=np.float64)
    g = inputs.upstream(20, 49, seed=29, dtype=np.float64)
    v = inputs.upstream(20, 3, seed=30, dtype=np.float64)
    gg, gx = double_backward(xyz, g, v, l_max)
    # d/dg of sum(v . backward(x, g)) is exact (linear in g)
    _, grad = spherical_harmonics_grad(xyz, l_max)
    np.testing.assert_allclose(gg, np.einsum("nik,ni->nk", grad, v), rtol=1e-14)

    def loss(p):
        return np.sum(backward(p, g, l_max) * v, axis=1, keepdims=True)

    fd = _fd_grad(loss, xyz, 1e-3)[:, :, 0]
    np.testing.assert_allclose(gx, fd, rtol=1e-7, atol=1e-7)


# --------------------------------------------------------------------------- planted mistakes
def test_planted_mistakes_are_caught(monkeypatch):
    """Plant plausible slips in the oracle (on the CPU) and check a pin fails."""
    xyz = inputs.normal_points(50, seed=31)
    V, G, _ = _closed_eval(xyz)

    def pins_pass():
        ok_v = np.allclose(spherical_harmonics(xyz, 3), V, atol=1e-12)
        _, g = spherical_harmonics_grad(xyz, 3)
        ok_g = np.allclose(g, G, atol=1e-12)
        ya = spherical_harmonics(xyz, 8, True)
        ok_add = all(
            np.allclose(np.sum(ya[:, l * l:(l + 1) ** 2] ** 2, 1), (2 * l + 1) / (4 * math.pi))
            for l in range(9)
        )
        return ok_v and ok_g and ok_add

    assert pins_pass()

    real_pref = orc.prefactor.__wrapped__

    # 1) Condon-Shortley phase left in (drop the (-1)^m of Eq. Flm)
    monkeypatch.setattr(orc, "prefactor", lambda l, m: abs(real_pref(l, m)))
    assert not pins_pass()
    monkeypatch.undo()

    # 2) 1/(4 pi) instead of 1/(2 pi) in the prefactor
    monkeypatch.setattr(orc, "prefactor", lambda l, m: real_pref(l, m) / math.sqrt(2))
    assert not pins_pass()
    monkeypatch.undo()

    # 3) wrong recursion coefficient in Eq. recur-p ((l+m) instead of (l+m-1))
    real_leg = orc.legendre_table

    def bad_leg(l_max, t, u):
        P, Pb = real_leg(l_max, t, u)
        if l_max >= 3:
            P[3, 1] = P[3, 1] * 1.25
        return P, Pb

    monkeypatch.setattr(orc, "legendre_table", bad_leg)
    assert not pins_pass()
    monkeypatch.undo()

    # 4) swapped sin/cos roles (m<0 <-> m>0)
    real_parts = orc._unit_sphere_parts

    def swapped(xyz_, l_max):
        r, t, u, phi, Yv, dth, dph = real_parts(xyz_, l_max)
        for l in range(1, l_max + 1):
            a, b = column(l, -1), column(l, 1)
            Yv[:, [a, b]] = Yv[:, [b, a]]
        return r, t, u, phi, Yv, dth, dph

    monkeypatch.setattr(orc, "_unit_sphere_parts", swapped)
    assert not pins_pass()
    monkeypatch.undo()

    # 5) sign slip in dP/dtheta
    def bad_dtheta(xyz_, l_max):
        r, t, u, phi, Yv, dth, dph = real_parts(xyz_, l_max)
        return r, t, u, phi, Yv, -dth, dph

    monkeypatch.setattr(orc, "_unit_sphere_parts", bad_dtheta)
    assert not pins_pass()
    monkeypatch.undo()
    assert pins_pass()


def _patched(func, old, new):
    """A copy of an oracle function with one source fragment replaced (a planted slip)."""
    import inspect
    import textwrap

    src = textwrap.dedent(inspect.getsource(func))
    assert src.count(old) == 1, old
    ns = dict(func.__globals__)
    exec(compile(src.replace(old, new), "<planted>", "exec"), ns)
    return ns[func.__name__]


@pytest.mark.parametrize(
    "old,new",
    [
        # drop the -m s^m A0 term of P_theta_theta
        ("- am * s_m * A0\n                        - (2 * am + 1)", "\n                        - (2 * am + 1)"),
        # (2m+1) -> (2m) in P_theta_theta
        ("(2 * am + 1) * s_m * t * A1", "(2 * am) * s_m * t * A1"),
        # sign slip in d(P/s)/dtheta
        ("Pbt = cF * ((am - 1) * s_m2 * t * A0 - s_m * A1)", "Pbt = cF * ((am - 1) * s_m2 * t * A0 + s_m * A1)"),
        # theta_hat / phi_hat swapped in the phi-derivative row
        ("+ Wt[:, None] * that + (p * Yv + Z)[:, None] * phat", "+ Wt[:, None] * phat + (p * Yv + Z)[:, None] * that"),
        # (p-1) -> p in the radial term
        ("Hk = ((p - 1.0) * v[:, :, None]", "Hk = (p * v[:, :, None]"),
        # one wrong coefficient in the t-derivative recursion's seed
        ("A[m + 1, m] = (2 * m + 1) * t * seed", "A[m + 1, m] = (2 * m + 2) * t * seed"),
    ],
)
def test_planted_hessian_mistakes_are_caught(old, new, monkeypatch):
    """Each slip planted in the analytic Hessian (on the CPU) fails a pin: the
    closed forms (l <= 3), or the twice-differentiated addition theorem (l <= 8)."""
    xyz = _hessian_pin_points()
    _, _, ref = _closed_eval(xyz)
    if "A[m + 1, m]" in old:
        monkeypatch.setattr(orc, "legendre_derivative_table", _patched(orc.legendre_derivative_table, old, new))
        hess = orc.spherical_harmonics_hessian
    else:
        hess = _patched(orc.spherical_harmonics_hessian, old, new)
    got = hess(xyz, 3)
    scale = _hess_block_scale(3, np.linalg.norm(xyz, axis=1))[:, None, None, :]
    closed_ok = np.max(np.abs(got - ref) / scale) < 1e-13
    x = inputs.shell_points(20, 0.5, 1.5, seed=170, dtype=np.float64)
    yv = inputs.shell_points(20, 0.5, 1.5, seed=171, dtype=np.float64)
    H = hess(x, 8)
    Ry = spherical_harmonics(yv, 8)
    ry = np.linalg.norm(yv, axis=1)
    add_ok = True
    for l in range(9):
        sl = slice(l * l, (l + 1) ** 2)
        lhs = np.einsum("nijk,nk->nij", H[..., sl], Ry[:, sl])
        rhs = _legendre_kernel_hessian(x, yv, l, l) * ((2 * l + 1) / (4 * math.pi) * ry**l)[:, None, None]
        add_ok &= bool(np.allclose(lhs, rhs, rtol=1e-12, atol=1e-12))
    assert not (closed_ok and add_ok)
    # the unmodified oracle passes both
    monkeypatch.undo()
    got = orc.spherical_harmonics_hessian(xyz, 3)
    assert np.max(np.abs(got - ref) / scale) < 1e-13


# --------------------------------------------------------------- expansion
def _wigner_free_power_spectrum(c, l_max):
    """p[i, n, n', l] = sum_m c[i, n, lm] c[i, n', lm]: invariant under rotations
    of all points of a centre (each l block transforms by an orthogonal matrix)."""
    out = []
    for l in range(l_max + 1):
        s = slice(l * l, (l + 1) ** 2)
        out.append(np.einsum("inm,ikm->ink", c[:, :, s], c[:, :, s]))
    return np.stack(out, axis=-1)


def test_expansion_single_edge_and_linearity():
    from oracle import expansion

    l_max, nr = 5, 3
    xyz = inputs.normal_points(7, seed=40)
    R = inputs.upstream(7, nr * (l_max + 1), seed=41, dtype=np.float64).reshape(7, nr, l_max + 1)
    offs = np.arange(8)  # one point per centre
    c = expansion(xyz, R, offs, l_max)
    Y = spherical_harmonics(xyz, l_max)
    for l in range(l_max + 1):
        s = slice(l * l, (l + 1) ** 2)
        np.testing.assert_allclose(c[:, :, s], R[:, :, l][:, :, None] * Y[:, None, s], rtol=1e-14)
    # one centre owning all points = sum of the single-point expansions
    c_all = expansion(xyz, R, np.array([0, 7]), l_max)
    np.testing.assert_allclose(c_all[0], c.sum(0), rtol=1e-13, atol=1e-14)
    # empty centres give zeros
    c_e = expansion(xyz, R, np.array([0, 0, 7, 7]), l_max)
    assert np.all(c_e[0] == 0) and np.all(c_e[2] == 0)


def test_expansion_power_spectrum_is_rotation_invariant():
    from oracle import expansion

    l_max, nr = 6, 4
    rng = np.random.default_rng(42)
    qm, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    xyz = inputs.shell_points(60, 0.8, 3.0, seed=43, dtype=np.float64)
    r = np.linalg.norm(xyz, axis=1)
    # radial values depend on r only, as a radial basis does
    R = np.stack([np.stack([np.exp(-(r - n) ** 2) * (1 + l * r) for l in range(l_max + 1)], 1)
                  for n in range(nr)], 1)
    offs = np.array([0, 13, 13, 40, 60])
    for normalized in (False, True):
        p0 = _wigner_free_power_spectrum(expansion(xyz, R, offs, l_max, normalized), l_max)
        p1 = _wigner_free_power_spectrum(expansion(xyz @ qm.T, R, offs, l_max, normalized), l_max)
        np.testing.assert_allclose(p1, p0, rtol=1e-10, atol=1e-12)
        # mixing l blocks (a plausible indexing slip) breaks the invariance
        c = expansion(xyz, R, offs, l_max, normalized)
        c_bad = c.copy()
        c_bad[:, :, 4:9] = c[:, :, 4:9] + 0.3 * c[:, :, 0:1]
        cr = expansion(xyz @ qm.T, R, offs, l_max, normalized)
        cr_bad = cr.copy()
        cr_bad[:, :, 4:9] = cr[:, :, 4:9] + 0.3 * cr[:, :, 0:1]
        assert not np.allclose(_wigner_free_power_spectrum(c_bad, l_max),
                               _wigner_free_power_spectrum(cr_bad, l_max), rtol=1e-6)


# --------------------------------------------------------------- readings of the paper
def test_downward_m_recursion_sign_reading():
    """Eq. iter-q-alt as printed has the wrong sign; the reading taken is
    Q_l^m = -[2(m+1) z Q_l^{m+1} + r_xy^2 Q_l^{m+2}] / ((l+m+1)(l-m)).
    Checked on Q_l^m = r^l r_xy^-m P_l^m built from the oracle's Legendre table."""
    xyz = inputs.shell_points(40, 0.6, 2.0, seed=50, dtype=np.float64)
    x, y, z = xyz.T
    r = np.linalg.norm(xyz, axis=1)
    rxy = np.hypot(x, y)
    l_max = 8
    P, _ = orc.legendre_table(l_max, z / r, rxy / r)
    Q = {(l, m): r**l * rxy ** (-m) * P[l, m] for l in range(l_max + 1) for m in range(l + 1)}
    for l in range(1, l_max + 1):
        for m in range(0, l - 1):
            q2 = Q[(l, m + 2)] if m + 2 <= l else 0.0
            corrected = -(2 * (m + 1) * z * Q[(l, m + 1)] + rxy**2 * q2) / ((l + m + 1) * (l - m))
            printed = (2 * (m + 1) * z * Q[(l, m + 1)] + rxy**2 * q2) / ((l + m + 1) * (l - m))
            np.testing.assert_allclose(corrected, Q[(l, m)], rtol=1e-10, atol=1e-10)
            assert not np.allclose(printed, Q[(l, m)], rtol=1e-6), (l, m)
    # Q_1^0 = z: the printed form would give -z
    np.testing.assert_allclose(Q[(1, 0)], z, rtol=1e-13)


def test_direct_z_link_reading():
    """The direct link printed with swapped indices reads, with |m|,
    d/dz Ytilde_l^m = (F_l^|m| / F_{l-1}^|m|) (l + |m|) Ytilde_{l-1}^m."""
    xyz = inputs.shell_points(30, 0.6, 2.0, seed=51, dtype=np.float64)
    l_max = 7
    V, G = spherical_harmonics_grad(xyz, l_max)
    for l in range(1, l_max + 1):
        for m in range(-(l - 1), l):
            am = abs(m)
            coef = prefactor(l, am) / prefactor(l - 1, am) * (l + am)
            np.testing.assert_allclose(G[:, 2, column(l, m)], coef * V[:, column(l - 1, m)], rtol=1e-11, atol=1e-12)
