"""The oracle's 1-D shock tube (Sec. VI B) against the exact Riemann solution.

D2Q33 (Table D2Q33), open ends in x (reading R16), periodic in y; (rho, T, u) = (4, 1, 0)
on the left half and (1, 1, 0) on the right; gamma = 1.4 (N_f = 3), tau = 2/3; the paper's
time t = steps / (X r) (X cells across the tube, r the lattice scale).  At t = 0.15
(174 steps on 1000 cells) the rarefaction, contact and shock are inside the tube.  The
scheme's viscosity and conductivity smear the discontinuities over a few cells, so the
error is measured in L1 relative to the jump, and must fall as the grid is refined at the
same t (87 steps on 500 cells).  The exact solution is the textbook one (tests/riemann.py).
"""
import os
import sys

import numpy as np

from oracle import oracle as O

sys.path.insert(0, os.path.dirname(__file__))
import riemann as R  # noqa: E402

LEFT, RIGHT, GAMMA = (4.0, 0.0, 4.0), (1.0, 0.0, 1.0), 1.4  # (rho, u, p = rho T)


def shock_tube(X, steps, ny=4):
    o = O.Sim(O.D2Q33, nx=X, ny=ny, Pr=0.71, gamma=GAMMA, kappa=0.2, tau=2.0 / 3.0, open_x=True)
    rho = np.where(np.arange(X) < X // 2, 4.0, 1.0)[None, :].repeat(ny, 0)
    o.init(rho, np.zeros((2, ny, X)), np.ones((ny, X)))
    o.step(steps)
    m = o.moments()
    o.close()
    return m


def l1_errors(m, X, steps):
    """L1 errors of rho, u, p against the exact solution, relative to the jump (rho, p)
    and to the star-state velocity (u)."""
    r = O.lattice(O.D2Q33)[1]
    t = steps / (X * r)
    s = (np.arange(X) + 0.5 - X / 2) / X / t
    ex = R.sample(s, LEFT, RIGHT, GAMMA)
    rho, u, p = m["rho"].mean(0), m["u"][0].mean(0), (m["rho"] * m["T"]).mean(0)
    return (np.abs(rho - ex[0]).mean() / 3.0, np.abs(u - ex[1]).mean() / ex[1].max(),
            np.abs(p - ex[2]).mean() / 3.0), t


def test_shock_tube_matches_exact_riemann_solution():
    e1000, t = l1_errors(shock_tube(1000, 174), 1000, 174)
    assert abs(t - 0.15) < 2e-3                        # the paper's t ~ 0.15
    assert e1000[0] < 0.01 and e1000[2] < 0.01 and e1000[1] < 0.02, e1000
    e500, _ = l1_errors(shock_tube(500, 87), 500, 87)
    assert all(b < 0.8 * a for a, b in zip(e500, e1000)), (e500, e1000)


def test_open_ends_keep_an_undisturbed_state():
    # the waves do not reach the ends by t = 0.15 (only the kinetic tail of the fastest
    # populations, 4 cells per step, at ~1e-10): the open (zero-gradient) ends must keep
    # the initial states there
    m = shock_tube(200, 35)
    assert np.abs(m["rho"][:, :5] - 4.0).max() < 1e-8 and np.abs(m["rho"][:, -5:] - 1.0).max() < 1e-8
    assert np.abs(m["u"][:, :, :5]).max() < 1e-8 and np.abs(m["u"][:, :, -5:]).max() < 1e-8
