"""The full-size parity helper on the CPU: its spawn pool reports the per-l
maximum over every chunk, so one wrong element anywhere is found."""

import numpy as np

import full_parity
import oracle
from paper_2302_08381_gb300 import inputs


def test_forward_errors_find_one_planted_element():
    n, l_max = 3000, 5
    x = inputs.shell_points(n, 0.5, 2.0, seed=900).astype(np.float64)
    v, g = oracle.spherical_harmonics_grad(x, l_max)
    v32, g32 = v.astype(np.float32), g.astype(np.float32)
    ev, eg, finite = full_parity.forward_errors(x, l_max, False, v32, g32, processes=2)
    assert finite and ev.shape == (l_max + 1,) and np.max(ev) < 1e-6 and np.max(eg) < 1e-6
    g32[2999, 1, 20] += 1e-2  # last point, l = 4
    v32[1234, 9] = np.nan  # l = 3
    ev2, eg2, finite2 = full_parity.forward_errors(x, l_max, False, v32, g32, processes=2)
    assert not finite2
    assert eg2[4] > 1e-4 and np.all(np.delete(eg2, 4) < 1e-6)
    assert not (ev2[3] <= 1.0)  # NaN propagates into the l = 3 maximum


def test_adjoint_errors_match_direct_evaluation():
    n, l_max = 1200, 4
    x = inputs.shell_points(n, 0.7, 3.0, seed=901).astype(np.float64)
    g = inputs.upstream(n, 25, seed=902).astype(np.float64)
    v = inputs.upstream(n, 3, seed=903).astype(np.float64)
    dx = oracle.backward(x, g, l_max)
    gg, gx = oracle.double_backward(x, g, v, l_max)
    gx_bad = gx.copy()
    gx_bad[n - 1, 2] += 1e-3 * np.max(np.abs(gx))
    err = full_parity.adjoint_errors(x, g, l_max, False, dxyz=dx, v=v, grad_g=gg, grad_xyz=gx_bad, processes=2)
    assert err["dxyz"] < 1e-15 and err["grad_g"] < 1e-15
    assert abs(err["grad_xyz"] - 1e-3) < 1e-9


def test_hessian_pool_finds_a_planted_error():
    """The Hessian pool reproduces the oracle on exact inputs (error 0), and
    one wrong element or one broken symmetric pair is found."""
    import oracle

    x = inputs.shell_points(700, 0.5, 2.0, seed=52).astype(np.float64)
    L = 5
    H = oracle.spherical_harmonics_hessian(x, L, True)
    H = 0.5 * (H + H.transpose(0, 2, 1, 3))  # the oracle's entries (i, k), (k, i) differ in rounding
    eh, finite, sym = full_parity.hessian_errors(x, L, True, H, processes=2)
    assert finite and sym and np.all(eh < 1e-14)
    H2 = H.copy()
    H2[613, 1, 2, 20] += 1e-3 * abs(H2[613, 1, 2, 20]) + 1e-6  # l = 4 block
    eh2, _, sym2 = full_parity.hessian_errors(x, L, True, H2, processes=2)
    assert eh2[4] > 1e-9 and np.all(np.delete(eh2, 4) < 1e-14) and not sym2
