"""Dual-basis Galerkin formulation of Sec. 2 (the paper's own discretisation).

TEST INFRASTRUCTURE ONLY: plain numpy on top of the FP64 oracle (`oracle.assemble`,
`oracle.pcg`, ...); shares no code with the CUDA path.

* Barycentric refinement (Sec. 2.1): every triangle T = (v0, v1, v2) of the mesh is
  split into six triangles by its centroid c and its edge midpoints m01, m12, m20:
  (v0, m01, c), (m01, v1, c), (v1, m12, c), (m12, v2, c), (v2, m20, c), (m20, v0, c)
  (orientation kept).  New vertices: the edge midpoints 0.5 (a + b), numbered after
  the M old vertices by the first appearance of their edge in (triangle, local edge)
  order, then the centroids ((v0 + v1) + v2) / 3 in triangle order.
* Dual cells (Sec. 2.1): the cell of vertex z is the union of the barycentric
  children that contain z: of T, children 0 and 5 belong to v0, 1 and 2 to v1, 3 and
  4 to v2.  |T_z^dual| = (sum over the triangles T at z, ascending, of |T|) / 3.
* V^dual = P^T V^bary P (Sec. 2.6), P the 0/1 map from dual cells to their children;
  the Galerkin solution solves V^dual x = f^dual, f^dual_z = |T_z^dual| (f = 1), and
  Cap_l = (1/4 pi) sum_z |T_z^dual| x_z (Eq. 2.8).  The paper solves the same Galerkin
  system with operator preconditioning and GMRES; any convergent solver gives the same
  x, and this oracle uses Jacobi PCG.
* Operator preconditioning (Sec. 2.6): the regularised hypersingular operator
  D^reg = D + a a^T on S^1 (hat functions phi_j of the primal vertices), a_j = int phi_j,
  with D = sum_m Q_m^T V^bary Q_m, Q_m (6N x M) the m-th component of the surface curl
  n x grad_G phi_j, constant on each primal triangle and so on its six children; the
  mass matrix M[i, j] = int phi_j chi_i^dual (exact: phi_j is linear on every child);
  the paper's system M^-T V^dual M^-1 D^reg x~ = M^-T f^dual, solved by restarted
  GMRES (restart 20, relative residual 1e-10, the solver the paper uses), and
  x = M^-1 D^reg x~.
* ZZ (Eq. 1.6) on the dual solution: eta(T)^2 = diam(T) ||Phi - I Phi||^2_{L2(T)}, Phi
  piecewise constant on the dual cells, I Phi the S^1 interpolant of the cell values.
  On each child the difference is affine; with its vertex values (a, b, c) the integral
  is (|T|/6)/12 (a^2 + b^2 + c^2 + (a + b + c)^2).  Vertex values on the children: 0 at
  the child's own vertex, (x_own - x_other)/2 at the midpoint, x_own - s/3 at the
  centroid, s = (x0 + x1) + x2.  Operation order: per child q = ((a a + b b) + c c) +
  (a + b + c)^2 with (a + b) + c; children summed in order 0..5; eta^2 = (h (|T| / 72)) q.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as O

CHILD_VERTEX = (0, 1, 1, 2, 2, 0)  # local primal vertex of barycentric child k


def barycentric(verts, tris):
    """(verts_b, tris_b) of the barycentric refinement, children of T at 6T .. 6T+5."""
    v = np.asarray(verts, dtype=np.float64)
    t = np.asarray(tris, dtype=np.int32)
    M, N = v.shape[0], t.shape[0]
    edge_id = {}
    mids = []
    for ti in range(N):
        for k in range(3):
            a, b = int(t[ti, k]), int(t[ti, (k + 1) % 3])
            key = (min(a, b), max(a, b))
            if key not in edge_id:
                edge_id[key] = M + len(mids)
                mids.append(0.5 * (v[a] + v[b]))
    E = len(mids)
    cent = (v[t[:, 0]] + v[t[:, 1]] + v[t[:, 2]]) / 3.0
    vb = np.concatenate([v, np.array(mids).reshape(E, 3), cent])
    tb = np.zeros((6 * N, 3), dtype=np.int32)
    for ti in range(N):
        v0, v1, v2 = (int(x) for x in t[ti])
        m01 = edge_id[(min(v0, v1), max(v0, v1))]
        m12 = edge_id[(min(v1, v2), max(v1, v2))]
        m20 = edge_id[(min(v2, v0), max(v2, v0))]
        c = M + E + ti
        tb[6 * ti:6 * ti + 6] = [(v0, m01, c), (m01, v1, c), (v1, m12, c), (m12, v2, c), (v2, m20, c),
                                 (m20, v0, c)]
    return vb, tb


def child_cell(tris):
    """Dual cell (primal vertex) of every barycentric child, length 6N."""
    t = np.asarray(tris, dtype=np.int32)
    return np.stack([t[:, k] for k in CHILD_VERTEX], axis=1).reshape(-1)


def dual_areas(verts, tris):
    """|T_z^dual| = (sum of |T| over the triangles at z, ascending) / 3."""
    area = O.geometry(verts, tris)[0]
    M = np.asarray(verts).shape[0]
    t = np.asarray(tris, dtype=np.int32)
    out = np.zeros(M)
    for z in range(M):
        s = 0.0
        for ti in np.flatnonzero(np.any(t == z, axis=1)):
            s = s + area[ti]
        out[z] = s / 3.0
    return out


def dual_operator(Vb, cell, M):
    """V^dual = P^T V^bary P (P[B, z] = 1 if child B belongs to cell z)."""
    P = np.zeros((len(cell), M))
    P[np.arange(len(cell)), cell] = 1.0
    return P.T @ Vb @ P


def zz_dual(verts, tris, x, h_mode=0):
    """eta(T)^2 of Eq. 1.6 for the dual solution x (one value per vertex)."""
    area, diam = O.geometry(verts, tris)
    t = np.asarray(tris, dtype=np.int32)
    xd = np.asarray(x, dtype=np.float64)
    out = np.zeros(t.shape[0])
    for ti in range(t.shape[0]):
        x0, x1, x2 = (float(xd[k]) for k in t[ti])
        s = (x0 + x1) + x2
        c3 = s / 3.0
        own = (x0, x1, x1, x2, x2, x0)
        mid = (0.5 * (x0 - x1), 0.5 * (x1 - x0), 0.5 * (x1 - x2), 0.5 * (x2 - x1), 0.5 * (x2 - x0),
               0.5 * (x0 - x2))
        q = 0.0
        for k in range(6):
            # child vertex order: own vertex first for even k, midpoint first for odd k
            a, b, c = (0.0, mid[k], own[k] - c3) if k % 2 == 0 else (mid[k], 0.0, own[k] - c3)
            ab = a + b
            q = q + (((a * a + b * b) + c * c) + (ab + c) * (ab + c))
        h = math.sqrt(area[ti]) if h_mode == 1 else diam[ti]
        out[ti] = (h * (area[ti] / 72.0)) * q
    return out


def solve_dual(verts, tris, tol=1e-12, precond=1, maxit=20000, n_ss=4):
    """Cap_l, x (per vertex), iterations, V^dual of the dual-basis Galerkin system."""
    vb, tb = barycentric(verts, tris)
    tbc = O.canonical(vb, tb)
    Vb = O.assemble(vb, tbc, n_ss)
    M = np.asarray(verts).shape[0]
    Vd = dual_operator(Vb, child_cell(tris), M)
    f = dual_areas(verts, tris)
    x, its, _, _ = O.pcg(Vd, f, tol=tol, maxit=maxit, precond=precond)
    return O.capacity(f, x), x, its, Vd


def adaptive_run_dual(verts, tris, theta=0.5, max_N=1000, tol=1e-12, h_mode=0, max_levels=100, solver="pcg"):
    """Alg. 1 with the dual-basis solution: solve -> ZZ (Eq. 1.6) -> Doerfler -> NVB on
    the primal mesh, each solve from zero, until N >= max_N.  The vanishing-estimator
    rule of the primal loop applies with x_T = (x0 + x1 + x2) / 3.  solver: "pcg"
    (Jacobi PCG on V^dual) or "calderon" (GMRES on the operator-preconditioned system
    of Sec. 2.6, tol as its relative residual)."""
    t = O.canonical(verts, tris)
    v = np.asarray(verts, dtype=np.float64)
    hist = []
    for lvl in range(max_levels):
        if solver == "calderon":
            cap, x, its = solve_dual_calderon(v, t, tol=tol)
        else:
            cap, x, its, _ = solve_dual(v, t, tol=tol)
        eta2 = zz_dual(v, t, x, h_mode)
        rec = {"level": lvl, "N": t.shape[0], "M": v.shape[0], "cap": cap, "its": its,
               "eta2_total": float(np.sum(eta2)), "x": x, "verts": v, "tris": t}
        hist.append(rec)
        if t.shape[0] >= max_N:
            break
        area, diam = O.geometry(v, t)
        xm = (x[t[:, 0]] + x[t[:, 1]] + x[t[:, 2]]) / 3.0
        h = np.sqrt(area) if h_mode == 1 else diam
        scale = float(np.sum(h * area * xm * xm / 12.0))
        m = O.mark(eta2, scale, theta)
        rec["marked"] = m
        v, t, _, _ = O.refine(v, t, m)
    return hist


# ---------------------------------------------------------------- operator preconditioning (Sec. 2.6)

def surface_curls(verts, tris):
    """curl_G phi_k = n x grad_G phi_k on every triangle, shape (N, 3 local vertices, 3).

    grad_G of the linear hat: J (J^T J)^-1 times the reference gradients of
    (1 - s - t, s, t), J = [p1 - p0, p2 - p0]; n the unit normal (p1 - p0) x (p2 - p0)."""
    v = np.asarray(verts, dtype=np.float64)
    t = np.asarray(tris, dtype=np.int64)
    out = np.zeros((t.shape[0], 3, 3))
    gref = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])
    for ti in range(t.shape[0]):
        p0, p1, p2 = v[t[ti, 0]], v[t[ti, 1]], v[t[ti, 2]]
        J = np.stack([p1 - p0, p2 - p0], axis=1)
        grads = J @ np.linalg.solve(J.T @ J, gref.T)  # columns: grad_G phi_k
        n = np.cross(p1 - p0, p2 - p0)
        n = n / np.linalg.norm(n)
        for k in range(3):
            out[ti, k] = np.cross(n, grads[:, k])
    return out


def curl_maps(verts, tris):
    """Q_m (6N x M), m = 0, 1, 2: coefficients of S^1 -> the m-th curl component on the
    barycentric children (the same value on all six children of a triangle)."""
    t = np.asarray(tris, dtype=np.int64)
    N, M = t.shape[0], np.asarray(verts).shape[0]
    g = surface_curls(verts, tris)
    Q = np.zeros((3, 6 * N, M))
    for ti in range(N):
        for k in range(3):
            for m in range(3):
                Q[m, 6 * ti:6 * ti + 6, t[ti, k]] += g[ti, k, m]
    return Q


def hat_integrals(verts, tris):
    """a_j = int_Gamma phi_j (the hat is linear on each triangle: |T| / 3 per triangle)."""
    area = O.geometry(verts, tris)[0]
    t = np.asarray(tris, dtype=np.int64)
    a = np.zeros(np.asarray(verts).shape[0])
    for ti in range(t.shape[0]):
        for k in range(3):
            a[t[ti, k]] += area[ti] / 3.0
    return a


def hypersingular(verts, tris, Vb):
    """D = sum_m Q_m^T V^bary Q_m and D^reg = D + a a^T (Sec. 2.6)."""
    Q = curl_maps(verts, tris)
    D = sum(Q[m].T @ Vb @ Q[m] for m in range(3))
    a = hat_integrals(verts, tris)
    return D, D + np.outer(a, a)


def mass_dual(verts, tris):
    """M[i, j] = int phi_j chi_i^dual: on each barycentric child of the cell of i the
    integral of the linear phi_j is |child| times the mean of its three vertex values;
    the values come from the barycentric coordinates of the child's vertices in T."""
    v = np.asarray(verts, dtype=np.float64)
    t = np.asarray(tris, dtype=np.int64)
    M = np.zeros((v.shape[0], v.shape[0]))
    area = O.geometry(v, t)[0]
    corner = np.eye(3)
    mid = {(0, 1): np.array([0.5, 0.5, 0.0]), (1, 2): np.array([0.0, 0.5, 0.5]),
           (2, 0): np.array([0.5, 0.0, 0.5])}
    cen = np.full(3, 1.0 / 3.0)
    # children in barycentric coordinates of T, same order as barycentric()
    kids = [(corner[0], mid[(0, 1)], cen), (mid[(0, 1)], corner[1], cen), (corner[1], mid[(1, 2)], cen),
            (mid[(1, 2)], corner[2], cen), (corner[2], mid[(2, 0)], cen), (mid[(2, 0)], corner[0], cen)]
    for ti in range(t.shape[0]):
        for k, kid in enumerate(kids):
            i = t[ti, CHILD_VERTEX[k]]
            mean = (kid[0] + kid[1] + kid[2]) / 3.0  # mean of phi_(local j) over the child
            for jl in range(3):
                M[i, t[ti, jl]] += (area[ti] / 6.0) * mean[jl]
    return M


def gmres(apply_A, b, tol=1e-10, restart=20, maxit=2000):
    """Restarted GMRES (Arnoldi with modified Gram-Schmidt, Givens rotations); stops
    when the residual norm is <= tol ||b||.  Returns x and the number of inner
    iterations (Arnoldi steps)."""
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    x = np.zeros(n)
    bn = np.linalg.norm(b)
    if bn == 0.0:
        return x, 0
    its = 0
    while its < maxit:
        r = b - apply_A(x)
        beta = np.linalg.norm(r)
        if beta <= tol * bn:
            break
        m = min(restart, n)
        Vk = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs, sn = np.zeros(m), np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        Vk[0] = r / beta
        k_used = 0
        for k in range(m):
            w = apply_A(Vk[k])
            for j in range(k + 1):
                H[j, k] = Vk[j] @ w
                w = w - H[j, k] * Vk[j]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0.0:
                Vk[k + 1] = w / H[k + 1, k]
            for j in range(k):  # previous rotations
                h0, h1 = H[j, k], H[j + 1, k]
                H[j, k], H[j + 1, k] = cs[j] * h0 + sn[j] * h1, -sn[j] * h0 + cs[j] * h1
            den = math.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k], H[k + 1, k] = den, 0.0
            g[k], g[k + 1] = cs[k] * g[k], -sn[k] * g[k]
            its += 1
            k_used = k + 1
            if abs(g[k + 1]) <= tol * bn or its >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:k_used, :k_used]), g[:k_used])
        x = x + Vk[:k_used].T @ y
        if abs(g[k_used]) <= tol * bn:
            break
    return x, its


def calderon_system(verts, tris, n_ss=4):
    """The matrices of the preconditioned dual system of one mesh: V^dual, D^reg, M,
    f^dual (Sec. 2.6)."""
    vb, tb = barycentric(verts, tris)
    Vb = O.assemble(vb, O.canonical(vb, tb), n_ss)
    M_ = np.asarray(verts).shape[0]
    Vd = dual_operator(Vb, child_cell(tris), M_)
    _, Dreg = hypersingular(verts, tris, Vb)
    return Vd, Dreg, mass_dual(verts, tris), dual_areas(verts, tris)


def solve_dual_calderon(verts, tris, tol=1e-10, n_ss=4):
    """Cap, x (per vertex), GMRES iterations of M^-T V^dual M^-1 D^reg x~ = M^-T f,
    x = M^-1 D^reg x~ (Sec. 2.6)."""
    Vd, Dreg, Mm, f = calderon_system(verts, tris, n_ss)
    MT = Mm.T

    def apply_A(y):
        return np.linalg.solve(MT, Vd @ np.linalg.solve(Mm, Dreg @ y))

    xt, its = gmres(apply_A, np.linalg.solve(MT, f), tol=tol)
    x = np.linalg.solve(Mm, Dreg @ xt)
    return O.capacity(f, x), x, its


def calderon_extremes(Vd, Dreg, Mm):
    """Extreme eigenvalues of the preconditioned operator: C V^dual with
    C = M^-1 D^reg M^-T (the spectrum of M^-T V^dual M^-1 D^reg)."""
    C = np.linalg.solve(Mm, np.linalg.solve(Mm, Dreg).T).T  # M^-1 D^reg M^-T (M^-T = (M^-1)^T)
    L = np.linalg.cholesky(Vd)
    ev = np.linalg.eigvalsh(L.T @ C @ L)
    return float(ev[0]), float(ev[-1])


def chebyshev_inverse(Mm, K=6, lo=15.0 / 22.0, hi=36.0 / 22.0):
    """S_K ~ M^-1: K steps of Chebyshev iteration for M s = r from s = 0, Jacobi-scaled,
    with the spectral interval [lo, hi] of D^-1 M (per triangle the mass matrix is
    (|T|/108)(15 I + 7 J) against the diagonal 22 |T|/108, so [15/22, 36/22] holds on
    every mesh), applied to the columns of the identity.  Not the paper's (it factors
    M): the GPU's operator preconditioner uses this polynomial, C = S_K D^reg S_K."""
    A = np.asarray(Mm, dtype=np.float64)
    dinv = 1.0 / np.diag(A)
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    sigma = theta / delta
    res = np.eye(A.shape[0])
    d = (dinv[:, None] * res) / theta
    S = d.copy()
    rho = 1.0 / sigma
    for _ in range(1, K):
        res = res - A @ d
        rn = 1.0 / (2.0 * sigma - rho)
        d = rn * rho * d + (2.0 * rn / delta) * (dinv[:, None] * res)
        S = S + d
        rho = rn
    return S
