"""The generated hard-coded low-degree expressions (csrc/sph_hardcoded.cuh):
the committed header is what the generator writes, and the generator's
expressions equal the FP64 oracle (values, gradients, and the Qtilde seeds
the recursion continues from) at random points, on the CPU."""

import importlib.util
import math
import os

import numpy as np
import sympy as sp

import oracle
from paper_2302_08381_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GEN = os.path.join(ROOT, "paper_2302_08381_gb300", "csrc", "gen_hardcoded.py")


def _gen():
    spec = importlib.util.spec_from_file_location("gen_hardcoded", GEN)
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_committed_header_is_up_to_date():
    g = _gen()
    with open(g.OUT) as f:
        assert f.read() == g.generate(), "run paper_2302_08381_gb300/csrc/gen_hardcoded.py"


def test_generated_expressions_equal_the_oracle():
    g = _gen()
    xyz = np.concatenate([inputs.shell_points(30, 0.5, 2.0, seed=950, dtype=np.float64),
                          inputs.pole_mix_points(10, seed=951)])
    r2 = np.sum(xyz ** 2, axis=1)
    for LH in range(4):
        outs, _, _ = g.build(LH, True)
        rv, rg = oracle.spherical_harmonics_grad(xyz, LH)
        for (kind, l, k, expr) in outs:
            f = sp.lambdify((g.X, g.Y, g.Z, g.R2), expr, "numpy")
            val = np.broadcast_to(f(xyz[:, 0], xyz[:, 1], xyz[:, 2], r2), (xyz.shape[0],))
            if kind == "v":
                ref = rv[:, k]
            elif kind in ("x", "y", "z"):
                ref = rg[:, "xyz".index(kind), k]
            else:
                # the seeds Qtilde_l^m, through the +m column of the oracle:
                # Ytilde_l^m = Qtilde_l^m c_m (m > 0), Ytilde_l^0 = Qtilde_l^0 / sqrt2
                m = k
                col = l * l + l + m
                c = np.real((xyz[:, 0] + 1j * xyz[:, 1]) ** m)
                yv = oracle.spherical_harmonics(xyz, l)[:, col]
                ok = np.abs(c) > 1e-3
                want = yv * (math.sqrt(2.0) if m == 0 else 1.0)
                np.testing.assert_allclose(val[ok] * (1.0 if m == 0 else c[ok]), want[ok], rtol=1e-12, atol=1e-12)
                continue
            np.testing.assert_allclose(val, ref, rtol=1e-12, atol=1e-12)
