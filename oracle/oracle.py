"""ctypes front end of the FP64 oracle (``bem_oracle.c``) plus the adaptive loop.

TEST INFRASTRUCTURE ONLY.  Each function names the passage of Betcke, Haberl and
Praetorius (arXiv 1901.08393) it follows; the arithmetic lives in bem_oracle.c
(plain FP64 C, no FMA contraction) and, for the cross-check solve, in LAPACK via
numpy (a library primitive).
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bem_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lib = None
_lock = threading.Lock()

__all__ = [
    "build", "lib", "gauss_legendre01", "radon7", "geometry", "pair_far", "pair_identical",
    "pair_edge", "pair_vertex", "pair_type", "entry", "entries", "assemble", "pcg",
    "solve_cholesky", "capacity", "zz", "dorfler", "canonical", "refine", "num_threads",
    "solve_capacity", "adaptive_run", "mark", "VANISHING_ETA", "set_num_threads", "cluster_order", "block_jacobi_inverses", "block_jacobi_pcg", "cg_lanczos_extremes", "pcg_inexact",
    "preconditioned_extremes",
]


def build(force: bool = False) -> str:
    """Compile bem_oracle.c into liborc.so (gcc, OpenMP, no FP contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            d, i64, i32, vp = C.c_double, C.c_int64, C.c_int, C.c_void_p
            L.orc_gauss_legendre01.argtypes = [i32, vp, vp]
            L.orc_radon7.argtypes = [vp, vp]
            L.orc_geometry.argtypes = [vp, i64, vp, i64, vp, vp]
            L.orc_pair_far.argtypes = [vp, vp]
            L.orc_pair_far.restype = d
            L.orc_pair_identical.argtypes = [vp, i32]
            L.orc_pair_identical.restype = d
            L.orc_pair_edge.argtypes = [vp, vp, i32]
            L.orc_pair_edge.restype = d
            L.orc_pair_vertex.argtypes = [vp, vp, i32]
            L.orc_pair_vertex.restype = d
            L.orc_pair_type.argtypes = [vp, i64, i64]
            L.orc_entry.argtypes = [vp, vp, i64, i64, i32]
            L.orc_entry.restype = d
            L.orc_entries.argtypes = [vp, vp, vp, vp, i64, i32, vp]
            L.orc_entries_raw.argtypes = [vp, vp, vp, vp, i64, i32, vp]
            L.orc_assemble.argtypes = [vp, i64, vp, i64, i32, vp]
            L.orc_pcg.argtypes = [vp, i64, vp, vp, vp, d, i32, i32, vp, vp]
            L.orc_matvec.argtypes = [vp, i64, vp, vp]
            L.orc_capacity.argtypes = [vp, vp, i64]
            L.orc_capacity.restype = d
            L.orc_zz.argtypes = [vp, i64, vp, i64, vp, i32, vp, vp]
            L.orc_dorfler.argtypes = [vp, i64, d, vp, vp]
            L.orc_canonical.argtypes = [vp, vp, i64, vp, vp]
            L.orc_refine.argtypes = [vp, i64, vp, i64, vp, i32, vp, vp, vp, vp, vp, vp]
            L.orc_num_threads.restype = i32
            L.orc_set_num_threads.argtypes = [i32]
            L.orc_set_num_threads.restype = None
            _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (n <= 0: all processors); timing only."""
    lib().orc_set_num_threads(int(n))


def gauss_legendre01(n: int):
    x, w = np.zeros(n), np.zeros(n)
    lib().orc_gauss_legendre01(n, _p(x), _p(w))
    return x, w


def radon7():
    """Radon's 7-point degree-5 triangle rule: barycentric points (7,3), weights (7,)."""
    b, w = np.zeros((7, 3)), np.zeros(7)
    lib().orc_radon7(_p(b), _p(w))
    return b, w


def geometry(verts, tris):
    """(area, diam) per triangle, in the exact operation order the GPU also uses."""
    v, t = _f64(verts), _i32(tris)
    N = t.shape[0]
    a, d = np.zeros(N), np.zeros(N)
    lib().orc_geometry(_p(v), v.shape[0], _p(t), N, _p(a), _p(d))
    return a, d


def pair_far(P, Q):
    """int_P int_Q 1/(4 pi |x-y|) by the 7x7 Radon product rule."""
    return float(lib().orc_pair_far(_p(_f64(P)), _p(_f64(Q))))


def pair_identical(P, n=4):
    return float(lib().orc_pair_identical(_p(_f64(P)), n))


def pair_edge(P, Q, n=4):
    """P = (A,B,C), Q = (A,B,D) share the edge AB (same vertex order)."""
    return float(lib().orc_pair_edge(_p(_f64(P)), _p(_f64(Q)), n))


def pair_vertex(P, Q, n=4):
    """P = (A,B,C), Q = (A,D,E) share the vertex A."""
    return float(lib().orc_pair_vertex(_p(_f64(P)), _p(_f64(Q)), n))


def pair_type(tris, i, j) -> int:
    t = _i32(tris)
    return int(lib().orc_pair_type(_p(t), i, j))


def entry(verts, tris, i, j, n=4) -> float:
    v, t = _f64(verts), _i32(tris)
    return float(lib().orc_entry(_p(v), _p(t), i, j, n))


def entries(verts, tris, I, J, n=4, raw=False):
    """V[I[k]][J[k]] (the matrix: i <= j computed, mirrored); raw=True evaluates with
    triangle I[k] as the first panel (not symmetric at finite order)."""
    v, t = _f64(verts), _i32(tris)
    I = np.ascontiguousarray(I, dtype=np.int64)
    J = np.ascontiguousarray(J, dtype=np.int64)
    out = np.zeros(I.shape[0])
    f = lib().orc_entries_raw if raw else lib().orc_entries
    f(_p(v), _p(t), _p(I), _p(J), I.shape[0], n, _p(out))
    return out


def assemble(verts, tris, n=4):
    """Dense Galerkin matrix V (Eq. 2.4 on primal P0, App. A Eq. A.1), FP64."""
    v, t = _f64(verts), _i32(tris)
    N = t.shape[0]
    out = np.zeros((N, N))
    lib().orc_assemble(_p(v), v.shape[0], _p(t), N, n, _p(out))
    return out


def pcg(A, b, x0=None, tol=1e-12, maxit=10000, precond=1):
    """Jacobi (precond=1) or plain (0) CG on the SPD system A x = b."""
    A = _f64(A)
    b = _f64(b)
    N = b.shape[0]
    x = np.zeros(N)
    its = C.c_int(0)
    rr = C.c_double(0.0)
    x0a = _f64(x0) if x0 is not None else None
    rc = lib().orc_pcg(_p(A), N, _p(b), _p(x0a), _p(x), tol, maxit, precond,
                       C.byref(its), C.byref(rr))
    return x, int(its.value), float(rr.value), int(rc)


def solve_cholesky(A, b):
    """Cross-check solve through LAPACK's Cholesky (fails if A is not SPD)."""
    L = np.linalg.cholesky(A)
    y = np.linalg.solve(L, b)
    return np.linalg.solve(L.T, y)


def capacity(area, x) -> float:
    """Cap_l = (1/4pi) <Phi_l, 1> = (1/4pi) sum |T_i| x_i   (Eq. 2.8)."""
    a, xx = _f64(area), _f64(x)
    return float(lib().orc_capacity(_p(a), _p(xx), a.shape[0]))


def zz(verts, tris, x, h_mode=0, with_scale=False):
    """ZZ-type indicators eta(T)^2 (Eq. 1.6, primal-P0 reading); with_scale also
    returns sum_T h_T |T| x_T^2 / 12."""
    v, t, xx = _f64(verts), _i32(tris), _f64(x)
    N = t.shape[0]
    out = np.zeros(N)
    sc = C.c_double(0.0)
    lib().orc_zz(_p(v), v.shape[0], _p(t), N, _p(xx), h_mode, _p(out), C.byref(sc))
    return (out, float(sc.value)) if with_scale else out


# An estimator whose total is below this fraction of sum h|T|x^2/12 is rounding
# noise of a solution that is constant up to rounding (a fully symmetric mesh).
VANISHING_ETA = 1e-20


def mark(eta2, scale, theta=0.5):
    """Alg. 1 (iii): Doerfler marking; when the estimator vanishes up to rounding
    the empty set satisfies Eq. 2.6 and the step refines uniformly instead."""
    if not np.sum(eta2) > VANISHING_ETA * scale:
        return np.ones(eta2.shape[0], dtype=np.uint8)
    return dorfler(eta2, theta)


def dorfler(eta2, theta=0.5):
    """Doerfler marking (Eq. 2.6); returns a uint8 flag per element."""
    e = _f64(eta2)
    N = e.shape[0]
    m = np.zeros(N, dtype=np.uint8)
    nm = C.c_int64(0)
    lib().orc_dorfler(_p(e), N, theta, _p(m), C.byref(nm))
    return m


def canonical(verts, tris, ref_edge=None):
    """Rotate triangles so that the reference edge is local edge 0 (Fig. 3)."""
    v, t = _f64(verts), _i32(tris)
    out = np.zeros_like(t)
    re = np.ascontiguousarray(ref_edge, dtype=np.uint8) if ref_edge is not None else None
    lib().orc_canonical(_p(v), _p(t), t.shape[0], _p(re), _p(out))
    return out


def refine(verts, tris, marked, bisec3=False):
    """NVB refinement with closure (Fig. 3).  Returns (verts, tris, parent, kept)."""
    v, t = _f64(verts), _i32(tris)
    M, N = v.shape[0], t.shape[0]
    mk = np.ascontiguousarray(marked, dtype=np.uint8)
    vo = np.zeros((M + 3 * N, 3))
    to = np.zeros((4 * N, 3), dtype=np.int32)
    par = np.zeros(4 * N, dtype=np.int32)
    kept = np.zeros(4 * N, dtype=np.uint8)
    Mo, No = C.c_int64(0), C.c_int64(0)
    lib().orc_refine(_p(v), M, _p(t), N, _p(mk), int(bisec3), _p(vo), _p(to), _p(par),
                     _p(kept), C.byref(Mo), C.byref(No))
    Mo, No = Mo.value, No.value
    return vo[:Mo].copy(), to[:No].copy(), par[:No].copy(), kept[:No].copy()


def solve_capacity(verts, tris, n_ss=4, tol=1e-12, maxit=20000, precond=1, x0=None):
    """Assemble V, solve V x = |T| by PCG, return (cap, x, its, V)."""
    V = assemble(verts, tris, n_ss)
    area, _ = geometry(verts, tris)
    x, its, rr, rc = pcg(V, area, x0=x0, tol=tol, maxit=maxit, precond=precond)
    return capacity(area, x), x, its, V


def cluster_order(verts, tris, B=64):
    """Triangle order of the block-Jacobi preconditioner (not part of the paper's
    method, which preconditions differently; any SPD preconditioner leaves the
    solution of Eq. 2.8 unchanged): Morton code of the centroid ((v0 + v1) + v2) / 3,
    10 bits per axis over the centroids' bounding box (q = trunc((c - lo) * (1023 /
    (hi - lo))), clamped to 0..1023; bit b of axis k at bit 3b + k), ascending, ties
    by index.  Consecutive groups of B triangles form the clusters."""
    v, t = _f64(verts), _i32(tris)
    c = (v[t[:, 0]] + v[t[:, 1]] + v[t[:, 2]]) / 3.0
    lo = c.min(axis=0)
    ext = c.max(axis=0) - lo
    code = np.zeros(t.shape[0], dtype=np.int64)
    for k in range(3):
        sc = 1023.0 / ext[k] if ext[k] > 0.0 else 0.0
        q = np.clip((c[:, k] - lo[k]) * sc, 0.0, 1023.0).astype(np.int64)
        for b in range(10):
            code |= ((q >> b) & 1) << (3 * b + k)
    return np.lexsort((np.arange(t.shape[0]), code))


def block_jacobi_inverses(V, order, B=64):
    """Clusters order[kB:(k+1)B] and the inverse of V on each (numpy Cholesky and
    inverse, library primitives); a block that is not positive definite is replaced
    by its diagonal, so that the preconditioner stays symmetric positive definite."""
    blocks = [order[k:k + B] for k in range(0, len(order), B)]
    inv = []
    for ix in blocks:
        A = V[np.ix_(ix, ix)]
        try:
            np.linalg.cholesky(A)
            inv.append(np.linalg.inv(A))
        except np.linalg.LinAlgError:
            inv.append(np.diag(1.0 / np.diag(A)))
    return blocks, inv


def block_jacobi_pcg(V, b, order, B=64, tol=1e-12, maxit=20000, x0=None):
    """CG on V x = b preconditioned by block_jacobi_inverses (the discrete V is not
    positive definite everywhere on strongly graded meshes: such blocks fall back to
    their diagonal).  Stops at ||r|| <= tol ||b||.  Returns (x, iterations)."""
    V, b = np.asarray(V, dtype=np.float64), np.asarray(b, dtype=np.float64)
    blocks, inv = block_jacobi_inverses(V, order, B)

    def apply(r):
        z = np.empty_like(r)
        for ix, Mi in zip(blocks, inv):
            z[ix] = Mi @ r[ix]
        return z

    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - V @ x
    z = apply(r)
    p = z.copy()
    rz = float(r @ z)
    bn = float(np.linalg.norm(b))
    for it in range(maxit + 1):
        if np.linalg.norm(r) <= tol * bn or it == maxit:
            return x, it
        q = V @ p
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        z = apply(r)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit


def cg_lanczos_extremes(V, b, precond=1, tol=1e-12, maxit=20000):
    """Estimates of the extreme eigenvalues of the preconditioned operator (Sec. 3,
    Figs. 6 and 12 report its condition number) from CG: plain numpy PCG (precond 0:
    none, 1: diag(V)) records alpha_j and beta_j; the Lanczos tridiagonal matrix has
    diagonal 1/alpha_j + beta_(j-1)/alpha_(j-1) and off-diagonal sqrt(beta_j)/alpha_j;
    its extreme eigenvalues (numpy eigvalsh, a library primitive).  Returns
    (lambda_min, lambda_max, iterations)."""
    V, b = np.asarray(V, dtype=np.float64), np.asarray(b, dtype=np.float64)
    dinv = 1.0 / np.diag(V) if precond == 1 else np.ones_like(b)
    x = np.zeros_like(b)
    r = b.copy()
    z = dinv * r
    p = z.copy()
    rz = float(r @ z)
    bn = float(np.linalg.norm(b))
    alphas, betas = [], []
    for _ in range(maxit):
        if np.linalg.norm(r) <= tol * bn:
            break
        q = V @ p
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        z = dinv * r
        rz_new = float(r @ z)
        beta = rz_new / rz
        alphas.append(alpha)
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    k = len(alphas)
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k:
            T[j, j + 1] = T[j + 1, j] = math.sqrt(betas[j]) / alphas[j]
    w = np.linalg.eigvalsh(T)
    return float(w[0]), float(w[-1]), k


def preconditioned_extremes(V, precond=1):
    """Exact extreme eigenvalues of D^-1/2 V D^-1/2 (precond 1, D = diag(V)) or of V
    (precond 0), by numpy eigvalsh."""
    V = np.asarray(V, dtype=np.float64)
    if precond == 1:
        s = 1.0 / np.sqrt(np.diag(V))
        V = V * s[:, None] * s[None, :]
    w = np.linalg.eigvalsh(V)
    return float(w[0]), float(w[-1])


def pcg_inexact(V, b, verts, tris, lam, x0=None, precond=1, tol=1e-12, maxit=20000, h_mode=0):
    """Jacobi (precond 1) or plain PCG with the stopping rule of the Remark after
    Alg. 1 (i), on the primal P0 space: after iteration k stop if
    |||x_k - x_(k-1)|||^2 = alpha_k (r.z) <= lam^2 sum_T eta_T^2(x_k), eta the ZZ
    indicators of the iterate (Eq. 1.6, `zz`); also at ||r|| <= tol ||b||.  Plain
    numpy.  Returns (x, iterations, stopped_by_rule, history of (upd2, eta2))."""
    V, b = np.asarray(V, dtype=np.float64), np.asarray(b, dtype=np.float64)
    dinv = 1.0 / np.diag(V) if precond == 1 else np.ones_like(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b - V @ x
    z = dinv * r
    p = z.copy()
    rz = float(r @ z)
    bn = float(np.linalg.norm(b))
    hist = []
    for it in range(maxit):
        if np.linalg.norm(r) <= tol * bn:
            return x, it, False, hist
        q = V @ p
        alpha = rz / float(p @ q)
        x = x + alpha * p
        r = r - alpha * q
        upd2 = alpha * rz
        eta2 = float(np.sum(zz(verts, tris, x, h_mode)))
        hist.append((upd2, eta2))
        if upd2 <= lam * lam * eta2:
            return x, it + 1, True, hist
        z = dinv * r
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit, False, hist


def adaptive_run(verts, tris, theta=0.5, max_N=2000, n_ss=4, tol=1e-12, h_mode=0,
                 max_levels=100, callback=None, inexact_lambda=0.0):
    """Algorithm 1 on the primal P0 space: solve -> estimate -> mark -> refine
    until the mesh has at least max_N triangles; the previous level's solution,
    copied to the children, starts the next solve (inexact_lambda > 0: stopped by
    the rule of the Remark after Alg. 1 (i), `pcg_inexact`).  Returns one record per
    level."""
    t = canonical(verts, tris)
    v = _f64(verts)
    hist = []
    x_prev = None
    for lvl in range(max_levels):
        if inexact_lambda > 0.0:
            V = assemble(v, t, n_ss)
            area = geometry(v, t)[0]
            x, its, _, _ = pcg_inexact(V, area, v, t, inexact_lambda, x0=x_prev, tol=tol, h_mode=h_mode)
            cap = capacity(area, x)
        else:
            cap, x, its, _ = solve_capacity(v, t, n_ss=n_ss, tol=tol, x0=x_prev)
        eta2, scale = zz(v, t, x, h_mode, with_scale=True)
        rec = {"level": lvl, "N": t.shape[0], "M": v.shape[0], "cap": cap, "its": its,
               "eta2_total": float(np.sum(eta2)), "x": x, "eta2": eta2,
               "verts": v, "tris": t}
        if t.shape[0] >= max_N:
            hist.append(rec)
            if callback:
                callback(rec)
            break
        m = mark(eta2, scale, theta)
        rec["marked"] = m
        hist.append(rec)
        if callback:
            callback(rec)
        v, t, parent, kept = refine(v, t, m)
        x_prev = x[parent]
    return hist


FOUR_PI = 4.0 * math.pi
