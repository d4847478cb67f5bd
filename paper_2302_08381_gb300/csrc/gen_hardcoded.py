#!/usr/bin/env python
"""Writes sph_hardcoded.cuh: straight-line ("hard-coded") expressions for the
scaled harmonics of degree l <= LH and their Cartesian gradients, LH = 0..3,
with common subexpressions eliminated by sympy.

The paper evaluates low degrees from ad hoc expressions (Section 3.1, Table 1
"hard-coded"; Section 3.2: the GPU kernel hard-codes l <= 3) and the general
recursion above them. Here every expression is derived, not transcribed:

* c_m, s_m from Eq. iter-sc;
* Q_l^m from Eq. iter-q (Q_m^m = (-1)^m (2m-1)!!, then the three-term
  recursion in z and r^2), with the prefactor F_l^m of Eq. Flm folded in
  (Appendix C): Qtilde_l^m = F_l^m Q_l^m;
* Ytilde_l^{+m} = Qtilde_l^m c_m, Ytilde_l^{-m} = Qtilde_l^m s_m,
  Ytilde_l^0 = Qtilde_l^0 / sqrt2 (Eq. real-sh-cartesian);
* gradients by differentiation, r^2 kept as an input symbol (the kernels pass
  the r^2 they use, |u|^2 of the rounded unit vector in the normalized form)
  with d r^2/dx_i = 2 x_i applied by the chain rule.

Each generated function also returns Qtilde_LH^m and Qtilde_{LH-1}^m, the
state the recursion of Eq. iter-q continues from at degree LH + 1.

Run from anywhere: ``python gen_hardcoded.py`` rewrites the header next to
this file; ``python gen_hardcoded.py --check`` exits 1 if it is out of date.
"""

from __future__ import annotations

import os
import sys

import sympy as sp
from sympy.printing.c import C99CodePrinter

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(HERE, "sph_hardcoded.cuh")
LH_MAX = 3

X, Y, Z, R2 = sp.symbols("x y z r2", real=True)


def prefactor(l: int, m: int):
    """F_l^m of Eq. Flm, exact."""
    return (-1) ** m * sp.sqrt(sp.Rational(2 * l + 1, 2) / sp.pi * sp.factorial(l - m) / sp.factorial(l + m))


def q_table(L: int):
    """Q_l^m(z, r2) of Eq. iter-q for 0 <= m <= l <= L."""
    Q = {}
    for m in range(L + 1):
        Q[(m, m)] = sp.Integer((-1) ** m) * sp.factorial2(2 * m - 1)
        for l in range(m + 1, L + 1):
            prev2 = Q.get((l - 2, m), sp.Integer(0))
            Q[(l, m)] = sp.expand(((2 * l - 1) * Z * Q[(l - 1, m)] - (l + m - 1) * R2 * prev2) / (l - m))
    return Q


def cs_table(L: int):
    """(c_m, s_m) of Eq. iter-sc for 0 <= m <= L."""
    c, s = [sp.Integer(1)], [sp.Integer(0)]
    for m in range(1, L + 1):
        c.append(sp.expand(X * c[m - 1] - Y * s[m - 1]))
        s.append(sp.expand(X * s[m - 1] + Y * c[m - 1]))
    return c, s


def grad(f):
    """Cartesian gradient with r2 = x^2 + y^2 + z^2 held as a symbol."""
    fr = sp.diff(f, R2)
    return [sp.diff(f, X) + 2 * X * fr, sp.diff(f, Y) + 2 * Y * fr, sp.diff(f, Z) + 2 * Z * fr]


def numeric(e):
    """Rationals and irrational constants as 30-digit floats (integers stay exact)."""
    e = sp.nsimplify(e) if False else e
    e = e.evalf(30)
    return e


class TPrinter(C99CodePrinter):
    """C++ for a template arithmetic type T: constants as T(...) literals,
    integer powers as products."""

    def _print_Float(self, e):
        return f"T({float(e)!r})"

    def _print_Integer(self, e):
        return f"T({int(e)})"

    def _print_Rational(self, e):
        return f"T({float(e)!r})"

    def _print_Pow(self, e):
        b, ex = e.as_base_exp()
        if ex.is_Integer and int(ex) > 0:
            return "(" + "*".join([self.parenthesize(b, 100)] * int(ex)) + ")"
        raise ValueError(f"unexpected power {e}")


def build(LH: int, with_grad: bool):
    Q = q_table(LH)
    c, s = cs_table(LH)
    outs = []  # (kind, l, k or m, expr)
    for l in range(LH + 1):
        for m in range(-l, l + 1):
            am = abs(m)
            qt = prefactor(l, am) * Q[(l, am)]
            if m < 0:
                f = qt * s[am]
            elif m == 0:
                f = qt / sp.sqrt(2)
            else:
                f = qt * c[m]
            f = sp.expand(f)
            k = l * l + l + m
            outs.append(("v", l, k, f))
            if with_grad:
                for i, g in enumerate(grad(f)):
                    outs.append(("gxyz"[1 + i], l, k, sp.expand(g)))
    for l in (LH - 1, LH):
        if l < 0:
            continue
        for m in range(l + 1):
            outs.append(("qa" if l == LH else "qb", l, m, sp.expand(prefactor(l, m) * Q[(l, m)])))
    exprs = [numeric(o[3]) for o in outs]
    reps, reduced = sp.cse(exprs, symbols=sp.numbered_symbols("t"), optimizations="basic")
    return outs, reps, reduced


def emit_function(LH: int, with_grad: bool, pr: TPrinter):
    outs, reps, reduced = build(LH, with_grad)
    name = f"hardcoded_l{LH}_{'grad' if with_grad else 'val'}"
    lines = [
        f"// l <= {LH}, {'values and gradients' if with_grad else 'values'}: "
        f"{sum(sp.count_ops(r[1]) for r in reps) + sum(sp.count_ops(e) for e in reduced)} operations after CSE.",
        "template <typename T, typename Vis>",
        f"__device__ __forceinline__ void {name}(T x, T y, T z, T r2, Vis& vis, T* qa, T* qb) {{",
    ]
    for sym, e in reps:
        lines.append(f"    const T {sym} = {pr.doprint(e)};")
    by_col = {}
    for o, e in zip(outs, reduced):
        kind, l, k, _ = o
        if kind in ("qa", "qb"):
            lines.append(f"    {kind}[{k}] = {pr.doprint(e)};")
        else:
            by_col.setdefault((l, k), {})[kind] = pr.doprint(e)
    for (l, k), d in sorted(by_col.items(), key=lambda t: t[0][1]):
        lines.append("    {")
        lines.append("        Deriv<T> d;")
        lines.append(f"        d.v = {d['v']};")
        if with_grad:
            lines.append(f"        d.gx = {d['x']};")
            lines.append(f"        d.gy = {d['y']};")
            lines.append(f"        d.gz = {d['z']};")
        lines.append(f"        vis.emit({l}, {k}, d);")
        lines.append("    }")
    lines.append("}")
    return "\n".join(lines)


def generate() -> str:
    pr = TPrinter()
    parts = [
        "// GENERATED by gen_hardcoded.py from the paper's Eqs. iter-sc, iter-q, Flm",
        "// and real-sh-cartesian (Appendix C folding); do not edit by hand.",
        "//",
        "// hardcoded_l<LH>_<val|grad>(x, y, z, r2, vis, qa, qb) emits every column",
        "// of degree l <= LH through vis.emit(l, k, Deriv) (k = l*l + l + m) and",
        "// writes qa[m] = Qtilde_LH^m (m <= LH) and qb[m] = Qtilde_{LH-1}^m",
        "// (m <= LH - 1), the state Eq. iter-q continues from at degree LH + 1.",
        "#pragma once",
        "",
        '#include "sph_core.cuh"',
        "",
        "namespace sph {",
        "",
    ]
    for LH in range(LH_MAX + 1):
        for g in (False, True):
            parts.append(emit_function(LH, g, pr))
            parts.append("")
    parts.append("}  // namespace sph")
    parts.append("")
    return "\n".join(parts)


def main(argv):
    text = generate()
    if "--check" in argv:
        with open(OUT) as f:
            ok = f.read() == text
        print("up to date" if ok else "OUT OF DATE")
        return 0 if ok else 1
    with open(OUT, "w") as f:
        f.write(text)
    print(f"wrote {OUT}")
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
