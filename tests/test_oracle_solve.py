"""Pins of the oracle's Galerkin matrix, solve and capacity (Eq. 2.4-2.8, Prop. 1,
Corollary of App. A) against invariants and values the paper prints."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1901_08393_gb300 import inputs
from tests._golden import capacity_reference

REF = capacity_reference()


def _cap(m, **kw):
    t = O.canonical(m.verts, m.tris)
    return O.solve_capacity(m.verts, t, **kw)


def test_V_symmetric_positive_definite():
    m = inputs.cube_mesh(2)
    cap, x, its, V = _cap(m)
    assert np.array_equal(V, V.T)
    assert np.all(V > 0)
    np.linalg.cholesky(V)  # raises if not SPD
    assert np.all(np.diag(V) >= V.max(axis=1) * (1 - 1e-15))


def test_pcg_matches_cholesky():
    m = inputs.workload_polycube_adaptive()
    t = O.canonical(m.verts, m.tris)
    V = O.assemble(m.verts, t)
    area, _ = O.geometry(m.verts, t)
    x, its, rr, rc = O.pcg(V, area, tol=1e-13)
    assert rc == 0 and rr <= 1e-13
    xc = O.solve_cholesky(V, area)
    assert np.max(np.abs(x - xc)) / np.max(np.abs(xc)) < 1e-10
    x0, its0, _, rc0 = O.pcg(V, area, tol=1e-13, precond=0)
    assert rc0 == 0 and np.max(np.abs(x0 - xc)) / np.max(np.abs(xc)) < 1e-10


def test_cube_sequence_increases_below_reference():
    """Nested uniform cube meshes: Cap_l increases (Corollary, App. A) and stays
    below the reference value of Sec. 3.1 (Prop. 1) and inside Polya's bounds."""
    caps = [_cap(inputs.cube_mesh(n))[0] for n in (1, 2, 4, 8)]
    assert all(b > a for a, b in zip(caps, caps[1:]))
    assert caps[-1] < REF["unit_cube_capacity"]
    assert REF["polya_lower"] < caps[2] < REF["polya_upper"]
    # O(N^{-2/3}) uniform rate (Sec. 3.1): error shrinks by about 4^{2/3} per level
    err = [REF["unit_cube_capacity"] - c for c in caps]
    ratios = [err[i] / err[i + 1] for i in range(1, 3)]
    assert all(2.0 < r < 3.5 for r in ratios), ratios


def test_sphere_limit():
    """Inscribed polyhedra of the unit sphere: 0 < Cap_h < 1 and Cap_h -> 1 (Sec. 1.2)."""
    caps = [_cap(inputs.icosphere_mesh(k, 1.0))[0] for k in (2, 4, 8)]
    assert all(0 < c < REF["sphere_capacity_over_radius"] for c in caps)
    assert all(b > a for a, b in zip(caps, caps[1:]))
    assert 1 - caps[-1] < 0.01
    c2 = _cap(inputs.icosphere_mesh(4, 2.5))[0]
    assert abs(c2 / (2.5 * caps[1]) - 1) < 1e-12


def test_scaling_and_rigid_motion():
    m = inputs.workload_polycube_adaptive()
    c1 = _cap(m)[0]
    c2 = _cap(inputs.Mesh(m.verts * 2.0, m.tris))[0]
    assert abs(c2 / (2 * c1) - 1) < 1e-14
    R = inputs.random_rotation(inputs.SplitMix64(7))
    c3 = _cap(inputs.transformed(m, R, 1.0, (0.3, -1.0, 2.0)))[0]
    assert abs(c3 / c1 - 1) < 1e-10


def test_prolongation_pythagoras():
    """Corollary (App. A): with nested P0 spaces and the coarse Galerkin matrix
    P^T V_f P, 4 pi (Cap_f - Cap_c) = |||Phi_f - Phi_c|||^2."""
    m = inputs.cube_mesh(2)
    t = O.canonical(m.verts, m.tris)
    rng = np.random.default_rng(0)
    marked = (rng.random(m.N) < 0.3).astype(np.uint8)
    vf, tf, parent, kept = O.refine(m.verts, t, marked)
    Vf = O.assemble(vf, tf)
    af, _ = O.geometry(vf, tf)
    P = np.zeros((tf.shape[0], m.N))
    P[np.arange(tf.shape[0]), parent] = 1.0
    Vc = P.T @ Vf @ P
    ac = P.T @ af
    xf = O.solve_cholesky(Vf, af)
    xc = O.solve_cholesky(Vc, ac)
    capf = O.capacity(af, xf)
    capc = float(ac @ xc) / (4 * math.pi)
    e = xf - P @ xc
    assert capf > capc > 0
    assert abs(4 * math.pi * (capf - capc) - e @ Vf @ e) < 1e-10 * (capf - capc)


def test_capacity_positive_and_rhs():
    m = inputs.tetra_mesh(3)
    cap, x, its, V = _cap(m)
    assert cap > 0 and np.all(x > 0)  # equilibrium charge density is positive
    area, _ = O.geometry(m.verts, O.canonical(m.verts, m.tris))
    assert abs(O.capacity(area, x) - cap) == 0.0


def test_cluster_order_morton_and_ties():
    """Morton order of the centroids over their bounding box, ties by index."""
    cents = [(1.0, 1.0, 1.0), (0.0, 0.5, 0.0), (0.5, 0.0, 0.0), (0.0, 0.0, 0.0), (0.5, 0.0, 0.0)]
    d = 0.25
    verts, tris = [], []
    for c in cents:  # triangle (c + d e1, c + d e2, c - d e1 - d e2): centroid exactly c
        c = np.array(c)
        k = len(verts)
        verts += [c + [d, 0, 0], c + [0, d, 0], c - [d, d, 0]]
        tris.append([k, k + 1, k + 2])
    order = O.cluster_order(np.array(verts), np.array(tris, dtype=np.int32))
    # codes: (0,0,0) -> 0; (0.5,0,0) -> x = 511 (bits 0..8 at 3b); (0,0.5,0) -> y = 511
    # (bits at 3b + 1, larger); (1,1,1) -> all 30 bits
    assert list(order) == [3, 2, 4, 1, 0]


def test_block_jacobi_pcg_special_cases():
    """One block = V^-1 exactly: one iteration to the Cholesky solution; blocks of one
    = Jacobi: the same iterates as the oracle's Jacobi PCG."""
    m = inputs.cube_mesh(2)
    t = O.canonical(m.verts, m.tris)
    V = O.assemble(m.verts, t)
    b = O.geometry(m.verts, t)[0]
    order = O.cluster_order(m.verts, t)
    x1, its1 = O.block_jacobi_pcg(V, b, order, B=len(b), tol=1e-13)
    assert its1 == 1
    xc = O.solve_cholesky(V, b)
    assert np.max(np.abs(x1 - xc)) < 1e-12 * np.max(np.abs(xc))
    xj, itsj = O.block_jacobi_pcg(V, b, np.arange(len(b)), B=1, tol=1e-12)
    xo, itso, _, _ = O.pcg(V, b, tol=1e-12, precond=1)
    assert abs(itsj - itso) <= 1 and np.max(np.abs(xj - xo)) < 1e-10 * np.max(np.abs(xo))


def test_block_jacobi_fewer_iterations_on_adaptive_mesh():
    """Spatial clusters of 64 beat the diagonal on an adaptively refined polycube."""
    hist = O.adaptive_run(*[getattr(inputs.workload_polycube_adaptive(), k) for k in ("verts", "tris")],
                          theta=0.5, max_N=1000, tol=1e-10)
    v, t = hist[-1]["verts"], hist[-1]["tris"]
    V = O.assemble(v, t)
    b = O.geometry(v, t)[0]
    _, its_b = O.block_jacobi_pcg(V, b, O.cluster_order(v, t), tol=1e-10)
    _, its_j, _, _ = O.pcg(V, b, tol=1e-10, precond=1)
    assert its_b < its_j


def test_block_jacobi_indefinite_block_falls_back_to_diagonal():
    V = np.array([[1.0, 2.0, 0.1], [2.0, 1.0, 0.1], [0.1, 0.1, 1.0]])
    blocks, inv = O.block_jacobi_inverses(V, np.arange(3), B=2)
    assert np.array_equal(inv[0], np.eye(2))  # [[1, 2], [2, 1]] is indefinite
    assert np.allclose(inv[1], [[1.0]])
    blocks, inv = O.block_jacobi_inverses(np.eye(3) * 2 + 0.5, np.arange(3), B=2)
    assert np.allclose(inv[0], np.linalg.inv(np.eye(2) * 2 + 0.5))


def test_cg_lanczos_extremes():
    """Diagonal system: the Lanczos matrix of a full CG run has exactly the eigenvalues
    of the system; BEM matrix: the estimates approach the exact extremes of the
    preconditioned operator, for no and for diagonal preconditioning."""
    A = np.diag(np.arange(1.0, 11.0))
    lo, hi, k = O.cg_lanczos_extremes(A, np.ones(10), precond=0, tol=1e-14)
    assert k == 10 and abs(lo - 1.0) < 1e-8 and abs(hi - 10.0) < 1e-8
    m = inputs.cube_mesh(3)
    t = O.canonical(m.verts, m.tris)
    V = O.assemble(m.verts, t)
    b = O.geometry(m.verts, t)[0]
    rnd = np.random.default_rng(0).standard_normal(len(b))
    for pc in (0, 1):
        elo, ehi = O.preconditioned_extremes(V, pc)
        lo, hi, k = O.cg_lanczos_extremes(V, b, precond=pc, tol=1e-14)
        assert abs(hi / ehi - 1) < 1e-6, (pc, hi, ehi)
        assert lo >= elo * (1 - 1e-9) and hi <= ehi * (1 + 1e-9)  # Ritz values lie inside the spectrum
        lo, hi, k = O.cg_lanczos_extremes(V, rnd, precond=pc, tol=1e-14)  # a right-hand side with every mode
        assert abs(lo / elo - 1) < 1e-3 and abs(hi / ehi - 1) < 1e-6, (pc, lo, elo, hi, ehi)
    # diagonal scaling lowers the condition number of V on a graded mesh (Sec. 3)
    g = inputs.graded_cube_mesh(8)
    tg = O.canonical(g.verts, g.tris)
    Vg = O.assemble(g.verts, tg)
    k0 = np.divide(*reversed(O.preconditioned_extremes(Vg, 0)))
    k1 = np.divide(*reversed(O.preconditioned_extremes(Vg, 1)))
    assert k1 < k0


def test_pcg_inexact_stopping_rule():
    """The rule of the Remark after Alg. 1 (i): it holds at the returned iterate and at
    no earlier one; lambda -> 0 gives the tolerance-stopped Jacobi PCG."""
    m = inputs.workload_polycube_adaptive()
    t = O.canonical(m.verts, m.tris)
    V = O.assemble(m.verts, t)
    b = O.geometry(m.verts, t)[0]
    x, its, rule, hist = O.pcg_inexact(V, b, m.verts, t, 1e-2, tol=1e-12)
    assert rule and len(hist) == its
    assert hist[-1][0] <= 1e-4 * hist[-1][1]
    assert all(u > 1e-4 * e for u, e in hist[:-1])
    x0, its0, rule0, _ = O.pcg_inexact(V, b, m.verts, t, 0.0, tol=1e-12)
    xo, itso, _, _ = O.pcg(V, b, tol=1e-12, precond=1)
    assert not rule0 and abs(its0 - itso) <= 1 and its < its0
    assert np.max(np.abs(x0 - xo)) < 1e-10 * np.max(np.abs(xo))
    # the capacity of the early-stopped iterate is within lambda * eta of the solution
    area = b
    assert abs(O.capacity(area, x) / O.capacity(area, xo) - 1) < 1e-3
