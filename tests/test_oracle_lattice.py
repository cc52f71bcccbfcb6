"""Pins of the oracle's lattices (Sec. VI, Tables D2Q37 and D2Q33; 3-D lattice reading R4).

The oracle re-solves the D2Q37 shell weights and scale r in FP64.  They must round to the
paper's printed 9-digit table, and both lattices must reproduce every moment of the unit
Gaussian up to degree 9 (what a "fourth-order" lattice needs for the G^(4) equilibrium).
"""
import itertools
import os
from math import prod

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "d2q37_table.txt")


def _table():
    rows, r = [], None
    for line in open(GOLDEN):
        if line.startswith("# r "):
            r = float(line.split()[2])
        elif line.strip() and not line.startswith("#"):
            cx, cy, k, w = line.split()
            rows.append((int(cx), int(cy), int(k), float(w)))
    return r, rows


def test_d2q37_matches_printed_table():
    r_printed, rows = _table()
    D, r, c, w = O.lattice(O.D2Q37)
    assert D == 2 and len(c) == 37 == sum(k for _, _, k, _ in rows)
    assert abs(r - r_printed) < 5e-9  # printed to 9 significant digits
    for cx, cy, k, wp in rows:
        sel = [i for i in range(37) if sorted(map(abs, c[i, :2])) == sorted((cx, cy))]
        assert len(sel) == k
        # the printed weights carry the rounding of r and their own 9 digits
        assert np.allclose(w[sel], wp, rtol=3e-7, atol=0), (cx, cy, w[sel][0], wp)


def _gauss_moment(alpha):
    return prod(0 if a % 2 else prod(range(a - 1, 0, -2)) for a in alpha)


def test_d2q33_matches_printed_table():
    # Table D2Q33: the 8 shells' 9 moment conditions fix r (a root of the augmented
    # system's determinant) and the weights; they must round to the printed 6 digits
    golden = os.path.join(os.path.dirname(__file__), "golden", "d2q33_table.txt")
    rows, r_over = [], None
    for line in open(golden):
        if line.startswith("# r_over_sqrt2 "):
            r_over = float(line.split()[2])
        elif line.strip() and not line.startswith("#"):
            cx, cy, k, wp = line.split()
            rows.append((int(cx), int(cy), int(k), float(wp)))
    D, r, c, w = O.lattice(O.D2Q33)
    assert D == 2 and len(c) == 33 == sum(k for _, _, k, _ in rows)
    assert abs(r / np.sqrt(2) - r_over) < 5e-7          # printed to 6 digits
    assert np.abs(c).max() == 4
    for cx, cy, k, wp in rows:
        sel = [i for i in range(33) if sorted(map(abs, c[i, :2])) == sorted((cx, cy))]
        assert len(sel) == k
        assert np.allclose(w[sel], wp, rtol=6e-6, atol=0), (cx, cy, w[sel][0], wp)


@pytest.mark.parametrize("which,Q", [(O.D2Q37, 37), (O.D3Q103, 103), (O.D2Q33, 33)])
def test_lattice_moments_degree9(which, Q):
    D, r, c, w = O.lattice(which)
    assert len(c) == Q and np.all(w > 0)
    xi = r * c[:, :D].astype(float)
    for deg in range(10):
        for alpha in itertools.product(range(deg + 1), repeat=D):
            if sum(alpha) != deg:
                continue
            m = np.sum(w * np.prod(xi ** np.array(alpha), axis=1))
            assert abs(m - _gauss_moment(alpha)) < 1e-11 * max(1, _gauss_moment(alpha)), (alpha, m)


def test_d2q37_is_not_exact_at_degree_10():
    # a degree-9 lattice must fail somewhere at degree 10 (else the check above is vacuous)
    D, r, c, w = O.lattice(O.D2Q37)
    xi = r * c[:, :2].astype(float)
    m = np.sum(w * xi[:, 0] ** 10)
    assert abs(m - _gauss_moment((10, 0))) > 1e-3


def test_lattice_velocity_set_symmetric():
    for which, reach in ((O.D2Q37, 3), (O.D3Q103, 3), (O.D2Q33, 4), (O.D2Q77, 5)):
        D, r, c, w = O.lattice(which)
        vs = {tuple(v) for v in c}
        assert len(vs) == len(c)
        for i, v in enumerate(c):
            j = [k for k in range(len(c)) if tuple(c[k]) == tuple(-v)][0]
            assert w[i] == pytest.approx(w[j], rel=1e-14)
        assert np.abs(c).max() == reach


def test_d2q77_moments_degree13():
    D, r, c, w = O.lattice(O.D2Q77)
    assert len(c) == 77 and np.all(w > 0) and w.sum() == pytest.approx(1.0, abs=1e-14)
    assert r == pytest.approx(0.9700084987393947, abs=1e-12)  # the only root in [0.8, 1.4]
    xi = r * c[:, :2].astype(float)
    for deg in range(14):
        for a in range(deg + 1):
            alpha = (a, deg - a)
            m = np.sum(w * xi[:, 0] ** alpha[0] * xi[:, 1] ** alpha[1])
            ref = _gauss_moment(alpha)
            assert abs(m - ref) < 1e-10 * max(1, ref), (alpha, m, ref)
    # degree 14 is not exact (so the check above is not vacuous)
    assert abs(np.sum(w * xi[:, 0] ** 8 * xi[:, 1] ** 6) / _gauss_moment((8, 6)) - 1) > 1e-2
