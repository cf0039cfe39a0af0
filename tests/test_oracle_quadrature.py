"""Pins of the oracle's quadrature (Eq. 2.4 entries) against facts that do not come
from the oracle: polynomial exactness, closed forms, and brute-force integrals."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import bruteforce
from tests._golden import capacity_reference, pair_integrals


def test_gauss_legendre_exactness():
    for n in (1, 2, 3, 4, 8, 16):
        x, w = O.gauss_legendre01(n)
        assert np.all(np.diff(x) > 0) and x[0] > 0 and x[-1] < 1
        for k in range(2 * n):
            assert abs(np.dot(w, x ** k) - 1.0 / (k + 1)) < 1e-14
        if n <= 8:  # not exact one degree above
            assert abs(np.dot(w, x ** (2 * n)) - 1.0 / (2 * n + 1)) > 1e-12


def _ref_triangle_monomial(a, b):
    # int over {x,y >= 0, x + y <= 1} of x^a y^b = a! b! / (a+b+2)!
    return math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)


def test_radon7_degree5_exact():
    bary, w = O.radon7()
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.allclose(bary.sum(axis=1), 1.0, atol=1e-15)
    pts = bary[:, 1:]  # (x, y) = barycentric weights of vertices (1,0) and (0,1)
    for a in range(6):
        for b in range(6 - a):
            q = 0.5 * np.dot(w, pts[:, 0] ** a * pts[:, 1] ** b)
            assert abs(q - _ref_triangle_monomial(a, b)) < 1e-15, (a, b)
    # degree 6 is not integrated exactly
    errs = [abs(0.5 * np.dot(w, pts[:, 0] ** a * pts[:, 1] ** (6 - a)) - _ref_triangle_monomial(a, 6 - a))
            for a in range(7)]
    assert max(errs) > 1e-6


def test_geometry_known_triangles():
    v = np.array([[0, 0, 0], [3, 0, 0], [0, 4, 0], [1, 1, 1], [1, 1, 3], [1, 3, 1.0]])
    t = np.array([[0, 1, 2], [3, 4, 5]], dtype=np.int32)
    area, diam = O.geometry(v, t)
    assert area[0] == 6.0 and diam[0] == 5.0
    assert area[1] == 2.0 and abs(diam[1] - math.sqrt(8.0)) < 1e-15


SHAPES = [
    np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0.0]]),
    np.array([[0, 0, 0], [1, 0, 0], [0.5, math.sqrt(3) / 2, 0]]),
    np.array([[0.1, -0.2, 0.3], [1.3, 0.4, -0.2], [0.2, 0.9, 0.8]]),
]


@pytest.mark.parametrize("P", SHAPES)
def test_identical_panel_closed_form(P):
    exact = bruteforce.identical_closed_form(P)
    assert abs(O.pair_identical(P, 20) / exact - 1) < 1e-11
    assert abs(O.pair_identical(P, 4) / exact - 1) < 2e-3
    # vertex order does not matter
    assert abs(O.pair_identical(P[[2, 0, 1]], 20) / exact - 1) < 1e-11
    assert abs(O.pair_identical(P[[1, 0, 2]], 20) / exact - 1) < 1e-11
    assert O.pair_identical(P * 2.0, 20) == 8 * O.pair_identical(P, 20)  # |x-y|^-1 on 4-d: s^3


def test_identical_needle_converges():
    """A needle (aspect ~20) converges slowly at low order but to the closed form."""
    P = np.array([[0, 0, 0], [4, 0, 0], [0.3, 0.2, 0.0]])
    exact = bruteforce.identical_closed_form(P)
    errs = [abs(O.pair_identical(P, n) / exact - 1) for n in (4, 16, 48)]
    assert errs[0] < 0.1 and errs[2] < 1e-9 and errs[2] < errs[1] < errs[0]


def test_unit_square_closed_form():
    """Two triangles of the unit square: 2 identical + 2 edge-adjacent pairs sum to
    the mean inverse distance in the unit square (textbook closed form)."""
    ref = capacity_reference()["unit_square_mean_inverse_distance"]
    assert abs(ref - ((4 / 3) * (1 - math.sqrt(2)) + 4 * math.log(1 + math.sqrt(2)))) < 1e-12
    A, B, C, D = (np.array(p, dtype=float) for p in ([0, 0, 0], [1, 0, 0], [1, 1, 0], [0, 1, 0]))
    for n, tol in ((16, 1e-12), (4, 2e-4)):
        tot = (O.pair_identical(np.array([A, B, C]), n) + O.pair_identical(np.array([A, C, D]), n)
               + 2 * O.pair_edge(np.array([A, C, B]), np.array([A, C, D]), n)) * 4 * math.pi
        assert abs(tot / ref - 1) < tol, (n, tot)


def test_pairs_against_brute_force_golden():
    rows = pair_integrals()
    assert len(rows) >= 4
    seen = set()
    for name, typ, P, Q, ref in rows:
        seen.add(typ)
        if typ == "vertex":
            f = O.pair_vertex
        elif typ == "edge":
            f = O.pair_edge
        else:
            assert abs(O.pair_far(P, Q) / ref - 1) < 1e-4, name
            continue
        assert abs(f(P, Q, 16) / ref - 1) < 1e-9, name
        assert abs(f(P, Q, 4) / ref - 1) < 1e-3, name
        # sign, and panel roles swapped give the same value
        assert f(P, Q, 16) > 0
        assert abs(f(Q, P, 16) / ref - 1) < 1e-9, name
    assert {"vertex", "edge"} <= seen


def test_far_pair_brute_force_live():
    P = np.array([[0, 0, 0], [1, 0, 0], [0.3, 0.9, 0.0]])
    for shift, tol in (([0.5, 2.0, 0.3], 1e-5), ([3.0, 4.0, -2.0], 1e-8)):
        Q = np.array([[0.1, 0.0, 0.0], [0.9, 0.3, 0.2], [0.2, 0.8, -0.3]]) + np.array(shift)
        ref = bruteforce.pair_integral(P, Q)
        assert abs(O.pair_far(P, Q) / ref - 1) < tol


def test_far_pair_point_limit():
    """Very distant pairs: |P||Q| / (4 pi d)."""
    P = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0.0]])
    Q = P + np.array([1e4, 0, 0])
    c = np.array([1 / 3, 1 / 3, 0])
    approx = 0.25 / (4 * math.pi * np.linalg.norm((Q.mean(0)) - c))
    assert abs(O.pair_far(P, Q) / approx - 1) < 1e-8


@pytest.mark.parametrize("n_lo,n_hi", [(4, 12)])
def test_sauter_schwab_converges_on_mesh(n_lo, n_hi):
    from paper_1901_08393_gb300 import inputs

    m = inputs.icosphere_mesh(2)
    t = O.canonical(m.verts, m.tris)
    near = [(i, j) for i in range(m.N) for j in range(m.N) if O.pair_type(t, i, j) > 0][:200]
    I = np.array([p[0] for p in near])
    J = np.array([p[1] for p in near])
    lo = O.entries(m.verts, t, I, J, n_lo, raw=True)
    hi = O.entries(m.verts, t, I, J, n_hi, raw=True)
    assert np.all(np.abs(lo / hi - 1) < 2e-3)
    # V_ij and V_ji computed separately (panel roles swapped) agree to quadrature accuracy
    hi_t = O.entries(m.verts, t, J, I, n_hi, raw=True)
    assert np.all(np.abs(hi_t / hi - 1) < 1e-9)
    # the matrix entry is the mirrored one
    assert np.array_equal(O.entries(m.verts, t, J, I, 4), O.entries(m.verts, t, I, J, 4))
