"""Pins of the dual-basis oracle (oracle/dual.py; Sec. 2.1, 2.6, Eq. 1.6, 2.8)."""
import numpy as np

import oracle as O
from oracle import dual as D
from paper_1901_08393_gb300 import inputs


def _mesh(m):
    return np.asarray(m.verts, dtype=np.float64), O.canonical(m.verts, m.tris)


def test_barycentric_refinement():
    v, t = _mesh(inputs.cube_mesh(2))
    vb, tb = D.barycentric(v, t)
    N, M = t.shape[0], v.shape[0]
    assert tb.shape[0] == 6 * N and vb.shape[0] == M + 3 * N // 2 + N
    area = O.geometry(v, t)[0]
    ab = O.geometry(vb, tb)[0]
    assert np.allclose(ab.reshape(N, 6), area[:, None] / 6.0, rtol=1e-14, atol=0)
    # orientation kept: child normals point like the parent's
    def normals(vv, tt):
        return np.cross(vv[tt[:, 1]] - vv[tt[:, 0]], vv[tt[:, 2]] - vv[tt[:, 0]])
    nb, n = normals(vb, tb).reshape(N, 6, 3), normals(v, t)
    assert np.all(np.einsum("nkc,nc->nk", nb, n) > 0)
    # closed and conforming: every edge is shared by exactly two children, once each way
    e = {}
    for tri in tb:
        for k in range(3):
            a, b = int(tri[k]), int(tri[(k + 1) % 3])
            assert (a, b) not in e
            e[(a, b)] = 1
    assert all((b, a) in e for (a, b) in e)


def test_dual_cells_partition_the_surface():
    v, t = _mesh(inputs.workload_polycube_adaptive())
    da = D.dual_areas(v, t)
    area = O.geometry(v, t)[0]
    assert abs(da.sum() / area.sum() - 1) < 1e-13 and np.all(da > 0)
    cell = D.child_cell(t)
    vb, tb = D.barycentric(v, t)
    ab = O.geometry(vb, tb)[0]
    per = np.zeros(v.shape[0])
    np.add.at(per, cell, ab)
    assert np.allclose(per, da, rtol=1e-13)


def test_zz_dual_closed_form_against_quadrature():
    """The closed form integrates (Phi - I Phi)^2 exactly: compare with a degree-2
    exact rule on every child (independent evaluation of Phi and I Phi)."""
    v, t = _mesh(inputs.cube_mesh(2))
    rng = np.random.default_rng(1)
    x = rng.standard_normal(v.shape[0])
    area, diam = O.geometry(v, t)
    ref = np.zeros(t.shape[0])
    vb, tb = D.barycentric(v, t)
    cell = D.child_cell(t)
    for ti in range(t.shape[0]):
        P = v[t[ti]]
        xv = x[t[ti]]
        s = 0.0
        for k in range(6):
            B = vb[tb[6 * ti + k]]
            for w, lam in ((1 / 3, (2 / 3, 1 / 6, 1 / 6)), (1 / 3, (1 / 6, 2 / 3, 1 / 6)), (1 / 3, (1 / 6, 1 / 6, 2 / 3))):
                y = lam[0] * B[0] + lam[1] * B[1] + lam[2] * B[2]
                # barycentric coordinates of y in T: I Phi(y)
                A = np.array([P[1] - P[0], P[2] - P[0]]).T
                mu = np.linalg.lstsq(A, y - P[0], rcond=None)[0]
                ipy = xv[0] * (1 - mu[0] - mu[1]) + xv[1] * mu[0] + xv[2] * mu[1]
                s += w * (area[ti] / 6.0) * (x[cell[6 * ti + k]] - ipy) ** 2
        ref[ti] = diam[ti] * s
    got = D.zz_dual(v, t, x)
    assert np.allclose(got, ref, rtol=1e-11, atol=1e-15)
    assert np.all(D.zz_dual(v, t, np.full(v.shape[0], 2.5)) == 0.0)


def test_dual_solution_against_primal_and_the_paper():
    """The dual-basis Galerkin capacity on the 12-triangle cube is the paper's level-0
    value (Sec. 3.1 table, 0.6492810516, computed by Bempp with its own quadrature;
    loose pin), and on finer cubes dual and primal capacities approach the reference
    0.66067815409957 from below."""
    v, t = _mesh(inputs.cube_mesh(1))
    cap0, x0, its, Vd = D.solve_dual(v, t)
    assert np.allclose(Vd, Vd.T, rtol=1e-13, atol=0)
    np.linalg.cholesky(Vd)
    assert abs(cap0 - 0.6492810516) < 2e-3, cap0
    ref = 0.66067815409957
    errs = []
    for n in (2, 3):
        vv, tt = _mesh(inputs.cube_mesh(n))
        cd = D.solve_dual(vv, tt)[0]
        cp = O.solve_capacity(vv, tt)[0]
        assert cd < ref and cp < ref
        errs.append(ref - cd)
    assert errs[1] < errs[0]


# ---------------------------------------------------------------- operator preconditioning (Sec. 2.6)

def test_surface_curls_of_linear_functions():
    """For a linear function c.x restricted to a flat triangle, sum_k (c.p_k) phi_k is the
    function itself, so sum_k (c.p_k) curl phi_k = n x grad_G(c.x) = n x c; the curls of
    the three hats sum to zero (constants have no curl)."""
    v, t = _mesh(inputs.workload_polycube_adaptive())
    g = D.surface_curls(v, t)
    rng = np.random.default_rng(3)
    for _ in range(3):
        c = rng.standard_normal(3)
        for ti in range(0, t.shape[0], 7):
            P = v[t[ti]]
            n = np.cross(P[1] - P[0], P[2] - P[0])
            n /= np.linalg.norm(n)
            got = sum((c @ P[k]) * g[ti, k] for k in range(3))
            assert np.allclose(got, np.cross(n, c), rtol=0, atol=1e-12 * np.linalg.norm(c))
    assert np.max(np.abs(g.sum(axis=1))) < 1e-12 * np.max(np.abs(g))


def test_mass_matrix_reproduces_cell_moments():
    """M[i, j] = int phi_j chi_i^dual: sum_j M[i, j] (c.p_j) = int_{cell i} c.x, the cell's
    first moment taken from the barycentric children's centroids; rows sum to the cell
    areas, columns to the hat integrals; symmetric on a barycentric refinement."""
    v, t = _mesh(inputs.fichera_mesh(1))
    Mm = D.mass_dual(v, t)
    vb, tb = D.barycentric(v, t)
    ab = O.geometry(vb, tb)[0]
    cell = D.child_cell(t)
    mom = np.zeros((v.shape[0], 3))
    for B in range(tb.shape[0]):
        mom[cell[B]] += ab[B] * vb[tb[B]].mean(axis=0)
    c = np.array([0.3, -1.2, 0.7])
    assert np.allclose(Mm @ (v @ c), mom @ c, rtol=1e-12, atol=1e-14)
    assert np.allclose(Mm.sum(axis=1), D.dual_areas(v, t), rtol=1e-13)
    assert np.allclose(Mm.sum(axis=0), D.hat_integrals(v, t), rtol=1e-13)
    assert np.array_equal(Mm, Mm.T)


def test_hypersingular_kernel_and_regularisation():
    """D annihilates constants (a one-dimensional kernel on a connected surface), is
    symmetric positive semi-definite; D^reg = D + a a^T is SPD and maps 1 to |Gamma| a."""
    v, t = _mesh(inputs.cube_mesh(2))
    vb, tb = D.barycentric(v, t)
    Vb = O.assemble(vb, O.canonical(vb, tb))
    Dm, Dreg = D.hypersingular(v, t, Vb)
    one = np.ones(v.shape[0])
    scale = np.max(np.abs(Dm))
    assert np.max(np.abs(Dm @ one)) < 1e-12 * scale
    assert np.allclose(Dm, Dm.T, rtol=0, atol=1e-14 * scale)
    ev = np.linalg.eigvalsh(Dm)
    assert ev[0] > -1e-12 * scale and ev[1] > 1e-3 * scale
    gamma = O.geometry(v, t)[0].sum()
    assert np.allclose(Dreg @ one, gamma * D.hat_integrals(v, t), rtol=1e-12)
    np.linalg.cholesky(Dreg)


def test_hypersingular_on_the_sphere():
    """On the unit sphere the spherical harmonics of degree n are eigenfunctions of D with
    eigenvalue n(n+1)/(2n+1); for the degree-1 function z: <D z, z> = (2/3)(4 pi / 3).  The
    discrete form of the interpolant of z on inscribed icospheres (20 k^2 triangles)
    approaches it at O(h^2)."""
    errs = []
    for k in (1, 2, 3):
        m = inputs.icosphere_mesh(k)
        v, t = _mesh(m)
        vb, tb = D.barycentric(v, t)
        Dm, _ = D.hypersingular(v, t, O.assemble(vb, O.canonical(vb, tb)))
        z = v[:, 2]
        errs.append(abs((z @ Dm @ z) / (8.0 * np.pi / 9.0) - 1.0))
    assert errs[1] < 0.4 * errs[0] and errs[2] < 0.6 * errs[1] and errs[2] < 0.08, errs


def test_gmres():
    """Restarted GMRES: exact (up to rounding) in as many steps as the matrix has distinct
    eigenvalues; with restarts on a nonsymmetric system it reaches the LAPACK solution."""
    A = np.diag([1.0] * 5 + [2.0] * 4 + [5.0] * 3)
    b = np.arange(1.0, 13.0)
    x, its = D.gmres(lambda y: A @ y, b, tol=1e-12)
    assert its == 3 and np.allclose(x, b / np.diag(A), rtol=1e-12)
    rng = np.random.default_rng(5)
    A = np.eye(40) * 4 + rng.standard_normal((40, 40)) * 0.3
    b = rng.standard_normal(40)
    x, its = D.gmres(lambda y: A @ y, b, tol=1e-11, restart=8)
    assert its > 8 and np.linalg.norm(A @ x - b) <= 1e-10 * np.linalg.norm(b)
    assert np.allclose(x, np.linalg.solve(A, b), rtol=1e-9, atol=1e-12)


def test_operator_preconditioned_solve():
    """The system of Sec. 2.6 gives the Galerkin solution of V^dual x = f (the same x as
    Jacobi PCG); on the 12-triangle cube GMRES needs 4 iterations, the count Table 1
    reports for level 0; the preconditioned condition number stays nearly constant under
    uniform refinement while diagonal scaling's grows like h^-1."""
    v, t = _mesh(inputs.cube_mesh(1))
    cap, x, its = D.solve_dual_calderon(v, t)
    cap_p, x_p, _, _ = D.solve_dual(v, t)
    assert its == 4
    assert abs(cap / cap_p - 1) < 1e-10 and np.max(np.abs(x - x_p)) < 1e-8 * np.max(np.abs(x_p))
    kc, kd = [], []
    for n in (1, 4):
        vv, tt = _mesh(inputs.cube_mesh(n))
        Vd, Dreg, Mm, _ = D.calderon_system(vv, tt)
        lo, hi = D.calderon_extremes(Vd, Dreg, Mm)
        kc.append(hi / lo)
        d = np.sqrt(np.diag(Vd))
        ev = np.linalg.eigvalsh(Vd / np.outer(d, d))
        kd.append(ev[-1] / ev[0])
    assert kc[1] < 1.5 * kc[0] and kd[1] > 3 * kd[0], (kc, kd)


def test_operator_preconditioned_adaptive_iterations():
    """Table 1 reports 12 GMRES iterations on every listed level past the first; along the
    adaptive cube sequence to N ~ 1000 the count stays bounded at that size."""
    m = inputs.cube_mesh(1)
    hist = D.adaptive_run_dual(m.verts, m.tris, max_N=600, tol=1e-10, solver="calderon")
    its = [h["its"] for h in hist]
    assert its[0] == 4 and max(its) <= 13, its
    caps = [h["cap"] for h in hist]
    assert all(b > a for a, b in zip(caps, caps[1:]))


def test_chebyshev_inverse_of_the_mass_matrix():
    """S_K is the degree-K Chebyshev polynomial in D^-1 M times D^-1: symmetric, and the
    eigenvalues of S_K M lie within 2 q^K of 1, q = (sqrt(k) - 1)/(sqrt(k) + 1) for the
    interval's k = 36/15 -- the bound that fixes K = 6 at 2e-4."""
    v, t = _mesh(inputs.workload_polycube_adaptive())
    Mm = D.mass_dual(v, t)
    d = np.diag(Mm)
    ev = np.linalg.eigvalsh(Mm / np.sqrt(np.outer(d, d)))
    assert ev[0] >= 15 / 22 - 1e-12 and ev[-1] <= 36 / 22 + 1e-12
    q = (np.sqrt(2.4) - 1) / (np.sqrt(2.4) + 1)
    for K in (2, 4, 6):
        S = D.chebyshev_inverse(Mm, K)
        assert np.allclose(S, S.T, rtol=0, atol=1e-14 * np.max(np.abs(S)))
        e = np.linalg.eigvals(S @ Mm).real
        assert np.max(np.abs(e - 1)) <= 2 * q ** K * (1 + 1e-9), (K, np.max(np.abs(e - 1)))
    assert 2 * q ** 6 < 2.2e-4
