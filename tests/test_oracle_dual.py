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
