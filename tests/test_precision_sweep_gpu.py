"""High-degree precision sweep: N = 200,000 points (half uniform on the unit
sphere, half within 1e-4 rad of the +/-z poles), l_max in {20, 30, 50},
values + gradients, normalized. The GPU runs the full workload for each
precision variant (FP32; FP32 storage with FP64 arithmetic for the unit
vector, the c/s and Q recursions and the assembly; FP64); every point is
compared with the FP64 oracle (spread over the host cores) and the per-l
maximum errors are printed (run with -s to see the table).
"""

import json
import os

import numpy as np
import pytest
import torch

import full_parity
from paper_2302_08381_gb300 import api, inputs
from parity_utils import F64_TOL

pytestmark = pytest.mark.gpu
DEV = "cuda:0"
N = 200_000


@pytest.mark.parametrize("l_max", [20, 30, 50])
def test_precision_sweep(l_max):
    xyz64 = inputs.pole_mix_points(N, seed=4)
    xyz32 = xyz64.astype(np.float32)
    h = N // 2  # first half uniform, second half near the poles
    rows = {}
    for name, arr, dtype, qprec in (
        ("f32", xyz32, torch.float32, "native"),
        ("f32+f64Q", xyz32, torch.float32, "f64"),
        ("f64", xyz64, torch.float64, "native"),
    ):
        x = torch.from_numpy(arr).to(DEV)
        sph, dsph = api.spherical_harmonics(x, l_max, True, gradients=True, qprec=qprec)
        torch.cuda.synchronize()
        s, d = sph.cpu().numpy(), dsph.cpu().numpy()
        del sph, dsph
        p = arr.astype(np.float64)  # compare at the coordinates the GPU saw
        ev_u, eg_u, fin_u = full_parity.forward_errors(p[:h], l_max, True, s[:h], d[:h])
        ev_p, eg_p, fin_p = full_parity.forward_errors(p[h:], l_max, True, s[h:], d[h:])
        assert fin_u and fin_p
        ev, eg = np.maximum(ev_u, ev_p), np.maximum(eg_u, eg_p)
        rows[name] = {
            "value_err_per_l": ev.tolist(),
            "grad_err_per_l": eg.tolist(),
            "value_err_uniform": float(ev_u.max()),
            "value_err_pole": float(ev_p.max()),
            "grad_err_uniform": float(eg_u.max()),
            "grad_err_pole": float(eg_p.max()),
        }
        bound = np.sqrt(2 * np.arange(l_max + 1) + 1.0)
        if name == "f64":
            assert np.all(ev <= F64_TOL * bound), ev
            assert np.all(eg <= F64_TOL), eg
        elif name == "f32+f64Q":
            # FP64 arithmetic, FP32 storage: only the final rounding remains.
            assert np.max(ev) < 1e-6 and np.max(eg) < 1e-6, (ev.max(), eg.max())
        else:
            # FP32: the error grows about linearly in l (rounding of the unit
            # vector and of the c_m/s_m powers, ~2e-6 l measured over all
            # 200,000 points); bounded per l at twice that here, the
            # acceptance bar applying at l_max <= 20.
            lv = np.arange(l_max + 1)
            assert np.all(ev <= 4e-6 * (lv + 1)) and np.all(eg <= 2e-6 * (lv + 1)), (name, ev, eg)
            if l_max <= 20:
                assert np.all(ev <= 1e-5 * bound) and np.all(eg <= 1e-4), (name, ev, eg)
    print(f"\nprecision sweep l_max={l_max} (max over all {N} points, per-l scaled errors)")
    print("   l   " + "  ".join(f"{n:>12s}v {n:>12s}g" for n in rows))
    for l in range(0, l_max + 1, 5 if l_max > 20 else 2):
        print(f"{l:4d}   " + "  ".join(f"{rows[n]['value_err_per_l'][l]:13.2e} {rows[n]['grad_err_per_l'][l]:13.2e}"
                                       for n in rows))
    out = os.environ.get("SPH_PRECISION_REPORT")
    if out:
        with open(out, "a") as f:
            f.write(json.dumps({"l_max": l_max, "n": N, "checked": N, "variants": rows}) + "\n")
