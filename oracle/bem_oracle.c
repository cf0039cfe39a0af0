/*
 * bem_oracle.c -- plain, slow FP64 CPU oracle for the dense P0 single-layer BEM
 * capacity computation (Betcke, Haberl, Praetorius, arXiv 1901.08393).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  It shares no code, header,
 * table or constant generator with the CUDA library; every quantity here is
 * written out from its definition, in FP64, in the order the definition states.
 *
 * What it computes (paper sections / equations):
 *   - Galerkin matrix of the single-layer operator V on piecewise constants,
 *     V[i][j] = (1/4pi) int_Ti int_Tj 1/|x-y|                  (Eq. 2.1, 2.4-2.5; App. A, Eq. A.1)
 *       * pairs with no common vertex: 7 x 7 product of Radon's degree-5 rule
 *       * pairs with a common vertex / edge / identical pairs: Sauter-Schwab type
 *         regularising transformations, n Gauss-Legendre points in each of the
 *         four integration variables (the paper cites the Sauter-Schwab textbook
 *         for these integrals; the regions used here are derived in the comments)
 *       * i <= j computed, the lower triangle mirrored
 *   - Jacobi-preconditioned CG for V x = b, b_i = |T_i|      (Remark after Alg. 1; Sec. 3 "diag")
 *   - Cap = (1/4pi) sum_i |T_i| x_i                          (Eq. 2.8)
 *   - ZZ-type indicators eta(T)^2 = h_T ||x_T - I x||^2_{L2(T)}  (Eq. 1.6, Sec. 2.4)
 *   - Doerfler marking                                       (Eq. 2.6, Alg. 1 (iii))
 *   - newest-vertex bisection with closure                   (Fig. 3, Alg. 1 (iv))
 *
 * Floating point: compile with -ffp-contract=off so that every product and sum
 * is rounded separately, in the order written (the geometry, ZZ and marking
 * results must match the GPU bit for bit when both are fed the same bytes).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------ helpers */

/* Gauss-Legendre nodes/weights on [0,1]: Newton iteration on the Legendre
 * polynomial P_n from the three-term recurrence (Abramowitz & Stegun 25.4.29). */
static void gauss_legendre01(int n, double *x, double *w)
{
    for (int k = 0; k < n; ++k) {
        double z = cos(ORC_PI * (k + 0.75) / (n + 0.5));
        double pn = 0.0, dp = 0.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            pn = (n == 1) ? z : p1;
            double pm = (n == 1) ? 1.0 : p0;
            dp = n * (z * pn - pm) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        /* recompute derivative at the converged root */
        {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            double pnn = (n == 1) ? z : p1, pm = (n == 1) ? 1.0 : p0;
            dp = n * (z * pnn - pm) / (z * z - 1.0);
        }
        x[k] = 0.5 * (1.0 - z);
        w[k] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

void orc_gauss_legendre01(int n, double *x, double *w) { gauss_legendre01(n, x, w); }

/* Radon's 7-point degree-5 rule on a triangle, barycentric coordinates and
 * weights normalised to sum 1: the centroid, and the two orbits (a,a,1-2a) with
 * a = (6 -+ sqrt 15)/21 and weights (155 -+ sqrt 15)/1200. */
static void radon7(double bary[7][3], double w[7])
{
    const double s15 = sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
    const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    double B[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                      {a1, a1, 1 - 2 * a1}, {a1, 1 - 2 * a1, a1}, {1 - 2 * a1, a1, a1},
                      {a2, a2, 1 - 2 * a2}, {a2, 1 - 2 * a2, a2}, {1 - 2 * a2, a2, a2}};
    double W[7] = {9.0 / 40, w1, w1, w1, w2, w2, w2};
    memcpy(bary, B, sizeof(B));
    memcpy(w, W, sizeof(W));
}

void orc_radon7(double *bary21, double *w7)
{
    double b[7][3];
    radon7(b, w7);
    memcpy(bary21, b, sizeof(b));
}

static void tri_points(const double *V, const int32_t *t, double P[3][3])
{
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c) P[k][c] = V[3 * (int64_t)t[k] + c];
}

/* |T| = |(P1-P0) x (P2-P0)| / 2, rounded step by step in this order. */
static double tri_area(const double P[3][3])
{
    double e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = P[1][c] - P[0][c];
        e2[c] = P[2][c] - P[0][c];
    }
    double cx = e1[1] * e2[2] - e1[2] * e2[1];
    double cy = e1[2] * e2[0] - e1[0] * e2[2];
    double cz = e1[0] * e2[1] - e1[1] * e2[0];
    return 0.5 * sqrt((cx * cx + cy * cy) + cz * cz);
}

static double edge_len2(const double *a, const double *b)
{
    double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
    return (dx * dx + dy * dy) + dz * dz;
}

/* diam(T) = longest edge (edges P0P1, P1P2, P2P0). */
static double tri_diam(const double P[3][3])
{
    double l0 = sqrt(edge_len2(P[0], P[1]));
    double l1 = sqrt(edge_len2(P[1], P[2]));
    double l2 = sqrt(edge_len2(P[2], P[0]));
    double m = l0 > l1 ? l0 : l1;
    return m > l2 ? m : l2;
}

int orc_geometry(const double *V, int64_t M, const int32_t *T, int64_t N,
                 double *area, double *diam)
{
    (void)M;
    for (int64_t i = 0; i < N; ++i) {
        double P[3][3];
        tri_points(V, T + 3 * i, P);
        if (area) area[i] = tri_area(P);
        if (diam) diam[i] = tri_diam(P);
    }
    return 0;
}

static inline double dist3(const double *x, const double *y)
{
    double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
    return sqrt(dx * dx + dy * dy + dz * dz);
}

/* chi(s,t) = P0 + s (P1 - P0) + t (P2 - P1), (s,t) in the reference triangle
 * {0 <= t <= s <= 1}; |d chi| = 2|T|. */
static inline void chi(const double P[3][3], double s, double t, double *x)
{
    for (int c = 0; c < 3; ++c) x[c] = P[0][c] + s * (P[1][c] - P[0][c]) + t * (P[2][c] - P[1][c]);
}

/* ------------------------------------------------------------ far field */
/* int_P int_Q 1/(4 pi |x-y|) by the 7x7 product rule. */
double orc_pair_far(const double *P9, const double *Q9)
{
    double P[3][3], Q[3][3], B[7][3], w[7];
    memcpy(P, P9, sizeof(P));
    memcpy(Q, Q9, sizeof(Q));
    radon7(B, w);
    double xa[7][3], yb[7][3];
    for (int a = 0; a < 7; ++a)
        for (int c = 0; c < 3; ++c) {
            xa[a][c] = B[a][0] * P[0][c] + B[a][1] * P[1][c] + B[a][2] * P[2][c];
            yb[a][c] = B[a][0] * Q[0][c] + B[a][1] * Q[1][c] + B[a][2] * Q[2][c];
        }
    double s = 0.0;
    for (int a = 0; a < 7; ++a)
        for (int b = 0; b < 7; ++b) s += w[a] * w[b] / dist3(xa[a], yb[b]);
    return tri_area(P) * tri_area(Q) * s / (4.0 * ORC_PI);
}

/* ------------------------------------------------------------ Sauter-Schwab */
/*
 * Identical panels.  With z = y^ - x^, the set {x^ in tau, x^ + z in tau} is, for
 * z in the difference hexagon with corners (1,0),(1,1),(0,1),(-1,0),(-1,-1),
 * (0,-1), a copy of tau shrunk by the factor (1 - L(z)), L the hexagon gauge.
 * Sector k of the hexagon (corners p, q): z = xi (p + eta (q - p)), dz = xi dxi deta;
 * x^ = x_c(z) + (1 - L)(sigma, sigma tau), dx^ = (1 - L)^2 sigma dsigma dtau.
 * The 1/|x-y| singularity at z = 0 is cancelled by the factor xi.
 */
static const double HEX[6][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 0}, {-1, -1}, {0, -1}};

double orc_pair_identical(const double *P9, int n)
{
    double P[3][3];
    memcpy(P, P9, sizeof(P));
    double g[64], gw[64];
    gauss_legendre01(n, g, gw);
    double I = 0.0;
    for (int k = 0; k < 6; ++k) {
        const double *p = HEX[k], *q = HEX[(k + 1) % 6];
        double cross = fabs(p[0] * q[1] - p[1] * q[0]);
        for (int a = 0; a < n; ++a)
            for (int b = 0; b < n; ++b)
                for (int c = 0; c < n; ++c)
                    for (int d = 0; d < n; ++d) {
                        double xi = g[a], eta = g[b], sg = g[c], ta = g[d];
                        double z1 = xi * (p[0] + eta * (q[0] - p[0]));
                        double z2 = xi * (p[1] + eta * (q[1] - p[1]));
                        /* barycentric linear parts of z: -z1, z1 - z2, z2 */
                        double c0 = fmax(0.0, z1), c1 = fmax(0.0, -(z1 - z2)), c2 = fmax(0.0, -z2);
                        double L = c0 + c1 + c2;
                        double xs = c1 + c2 + (1.0 - L) * sg;
                        double xt = c2 + (1.0 - L) * sg * ta;
                        double x[3], y[3];
                        chi(P, xs, xt, x);
                        chi(P, xs + z1, xt + z2, y);
                        double jac = xi * cross * (1.0 - L) * (1.0 - L) * sg;
                        I += gw[a] * gw[b] * gw[c] * gw[d] * jac / dist3(x, y);
                    }
    }
    double A = tri_area(P);
    return 4.0 * A * A * I / (4.0 * ORC_PI);
}

/*
 * Common edge.  Panels P = (A, B, C), Q = (A, B, D): chi_P(s,0) = chi_Q(s,0) on AB.
 * The 4-d domain tau x tau is a cone from the origin over its far faces
 * {s1 = 1} (region 1) and {s2 = 1} (region 2): (s1,t1,s2,t2) = xi * w, Jacobian
 * xi^3.  On face s1 = 1 put a = 1 - s2: the kernel is singular only at
 * (t1, a, t2) = 0 and that face is [0,1]_{t1} x {a, t2 >= 0, a + t2 <= 1}, again a
 * cone from 0 over {t1 = 1} (sub-region a) and {a + t2 = 1} (sub-region b):
 *   a: (t1, a, t2) = rho (1, m1 (1 - m2), m1 m2),  Jacobian rho^2 m1
 *   b: (t1, a, t2) = rho (nu, 1 - lam, lam),       Jacobian rho^2
 * Region 2 is the same with the roles of the panels swapped.
 */
double orc_pair_edge(const double *P9, const double *Q9, int n)
{
    double P[3][3], Q[3][3];
    memcpy(P, P9, sizeof(P));
    memcpy(Q, Q9, sizeof(Q));
    double g[64], gw[64];
    gauss_legendre01(n, g, gw);
    double I = 0.0;
    for (int reg = 0; reg < 2; ++reg)
        for (int sub = 0; sub < 2; ++sub)
            for (int ia = 0; ia < n; ++ia)
                for (int ib = 0; ib < n; ++ib)
                    for (int ic = 0; ic < n; ++ic)
                        for (int id = 0; id < n; ++id) {
                            double xi = g[ia], rho = g[ib], u = g[ic], v = g[id];
                            double wq = gw[ia] * gw[ib] * gw[ic] * gw[id];
                            double f, aa, h, jac; /* far-face coords: own t, a, other t */
                            if (sub == 0) {
                                f = rho;
                                aa = rho * u * (1.0 - v);
                                h = rho * u * v;
                                jac = xi * xi * xi * rho * rho * u;
                            } else {
                                f = rho * u;
                                aa = rho * (1.0 - v);
                                h = rho * v;
                                jac = xi * xi * xi * rho * rho;
                            }
                            double s1, t1, s2, t2;
                            if (reg == 0) { /* s1 = xi, face s1 = 1 */
                                s1 = xi; t1 = xi * f; s2 = xi * (1.0 - aa); t2 = xi * h;
                            } else {        /* s2 = xi, face s2 = 1 */
                                s2 = xi; t2 = xi * f; s1 = xi * (1.0 - aa); t1 = xi * h;
                            }
                            double x[3], y[3];
                            chi(P, s1, t1, x);
                            chi(Q, s2, t2, y);
                            I += wq * jac / dist3(x, y);
                        }
    return 4.0 * tri_area(P) * tri_area(Q) * I / (4.0 * ORC_PI);
}

/*
 * Common vertex.  Panels P = (A, B, C), Q = (A, D, E).  Duffy maps x^ = s1 (1, t),
 * y^ = s2 (1, t') and the split s2 <= s1 / s1 <= s2 give
 *   region 1: x^ = xi (1, e1),     y^ = xi e2 (1, e3)
 *   region 2: x^ = xi e2 (1, e1),  y^ = xi (1, e3)
 * each with Jacobian xi^3 e2.
 */
double orc_pair_vertex(const double *P9, const double *Q9, int n)
{
    double P[3][3], Q[3][3];
    memcpy(P, P9, sizeof(P));
    memcpy(Q, Q9, sizeof(Q));
    double g[64], gw[64];
    gauss_legendre01(n, g, gw);
    double I = 0.0;
    for (int reg = 0; reg < 2; ++reg)
        for (int ia = 0; ia < n; ++ia)
            for (int ib = 0; ib < n; ++ib)
                for (int ic = 0; ic < n; ++ic)
                    for (int id = 0; id < n; ++id) {
                        double xi = g[ia], e1 = g[ib], e2 = g[ic], e3 = g[id];
                        double wq = gw[ia] * gw[ib] * gw[ic] * gw[id];
                        double sx, tx, sy, ty;
                        if (reg == 0) {
                            sx = xi; tx = xi * e1; sy = xi * e2; ty = xi * e2 * e3;
                        } else {
                            sx = xi * e2; tx = xi * e2 * e1; sy = xi; ty = xi * e3;
                        }
                        double x[3], y[3];
                        chi(P, sx, tx, x);
                        chi(Q, sy, ty, y);
                        I += wq * xi * xi * xi * e2 / dist3(x, y);
                    }
    return 4.0 * tri_area(P) * tri_area(Q) * I / (4.0 * ORC_PI);
}

/* ------------------------------------------------------------ one entry */
/* Number of vertex indices two triangles share. */
static int shared_count(const int32_t *a, const int32_t *b)
{
    int s = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s += (a[i] == b[j]);
    return s;
}

int orc_pair_type(const int32_t *T, int64_t i, int64_t j)
{
    if (i == j) return 3;
    return shared_count(T + 3 * i, T + 3 * j);
}

/* The integral with triangle i as the first panel (Sauter-Schwab order n for
 * touching pairs).  For touching pairs this is not symmetric in (i, j) at finite
 * n; the matrix entry is orc_entry. */
double orc_entry_raw(const double *V, const int32_t *T, int64_t i, int64_t j, int n)
{
    const int32_t *ti = T + 3 * i, *tj = T + 3 * j;
    double P[3][3], Q[3][3];
    if (i == j) {
        tri_points(V, ti, P);
        return orc_pair_identical(&P[0][0], n);
    }
    int s = shared_count(ti, tj);
    if (s == 0) {
        tri_points(V, ti, P);
        tri_points(V, tj, Q);
        return orc_pair_far(&P[0][0], &Q[0][0]);
    }
    int32_t pi[3], pj[3];
    if (s == 2) {
        /* order both as (u, v, other) with the shared edge (u, v) in the same order */
        int32_t u = -1, v = -1, ci = -1, cj = -1;
        for (int k = 0; k < 3; ++k) {
            int in = (ti[k] == tj[0] || ti[k] == tj[1] || ti[k] == tj[2]);
            if (in) {
                if (u < 0) u = ti[k]; else v = ti[k];
            } else {
                ci = ti[k];
            }
        }
        for (int k = 0; k < 3; ++k)
            if (tj[k] != u && tj[k] != v) cj = tj[k];
        pi[0] = u; pi[1] = v; pi[2] = ci;
        pj[0] = u; pj[1] = v; pj[2] = cj;
        tri_points(V, pi, P);
        tri_points(V, pj, Q);
        return orc_pair_edge(&P[0][0], &Q[0][0], n);
    }
    if (s == 1) {
        int ki = 0, kj = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                if (ti[a] == tj[b]) { ki = a; kj = b; }
        for (int k = 0; k < 3; ++k) {
            pi[k] = ti[(ki + k) % 3];
            pj[k] = tj[(kj + k) % 3];
        }
        tri_points(V, pi, P);
        tri_points(V, pj, Q);
        return orc_pair_vertex(&P[0][0], &Q[0][0], n);
    }
    return NAN; /* duplicate triangle: not a valid mesh */
}

/* V[i][j]: the entry with i <= j is computed and mirrored. */
double orc_entry(const double *V, const int32_t *T, int64_t i, int64_t j, int n)
{
    return i <= j ? orc_entry_raw(V, T, i, j, n) : orc_entry_raw(V, T, j, i, n);
}

int orc_entries(const double *V, const int32_t *T, const int64_t *I, const int64_t *J,
                int64_t K, int n, double *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < K; ++k) out[k] = orc_entry(V, T, I[k], J[k], n);
    return 0;
}

int orc_entries_raw(const double *V, const int32_t *T, const int64_t *I, const int64_t *J,
                    int64_t K, int n, double *out)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t k = 0; k < K; ++k) out[k] = orc_entry_raw(V, T, I[k], J[k], n);
    return 0;
}

/* Full dense V (row-major N x N): i <= j computed, j < i mirrored. */
int orc_assemble(const double *V, int64_t M, const int32_t *T, int64_t N, int n, double *out)
{
    (void)M;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = i; j < N; ++j) out[i * N + j] = orc_entry_raw(V, T, i, j, n);
    for (int64_t i = 0; i < N; ++i)
        for (int64_t j = 0; j < i; ++j) out[i * N + j] = out[j * N + i];
    return 0;
}

/* ------------------------------------------------------------ solve */
static void matvec(const double *A, int64_t N, const double *x, double *y)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        double s = 0.0;
        const double *row = A + i * N;
        for (int64_t j = 0; j < N; ++j) s += row[j] * x[j];
        y[i] = s;
    }
}

static double dot(const double *a, const double *b, int64_t N)
{
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) s += a[i] * b[i];
    return s;
}

/* Preconditioned CG (precond 1: Jacobi diag(A); 0: none) until
 * ||b - A x||_2 <= tol ||b||_2.  Returns 0 on convergence, 1 otherwise. */
int orc_pcg(const double *A, int64_t N, const double *b, const double *x0, double *x,
            double tol, int maxit, int precond, int *its, double *relres)
{
    double *r = malloc(N * sizeof(double)), *z = malloc(N * sizeof(double));
    double *p = malloc(N * sizeof(double)), *q = malloc(N * sizeof(double));
    for (int64_t i = 0; i < N; ++i) x[i] = x0 ? x0[i] : 0.0;
    matvec(A, N, x, q);
    for (int64_t i = 0; i < N; ++i) r[i] = b[i] - q[i];
    double bn = sqrt(dot(b, b, N));
    if (bn == 0.0) bn = 1.0;
    for (int64_t i = 0; i < N; ++i) z[i] = precond ? r[i] / A[i * N + i] : r[i];
    memcpy(p, z, N * sizeof(double));
    double rz = dot(r, z, N);
    double rr = sqrt(dot(r, r, N)) / bn;
    int k = 0, rc = 1;
    if (rr <= tol) rc = 0;
    while (rc && k < maxit) {
        matvec(A, N, p, q);
        double alpha = rz / dot(p, q, N);
        for (int64_t i = 0; i < N; ++i) {
            x[i] += alpha * p[i];
            r[i] -= alpha * q[i];
        }
        ++k;
        rr = sqrt(dot(r, r, N)) / bn;
        if (rr <= tol) { rc = 0; break; }
        for (int64_t i = 0; i < N; ++i) z[i] = precond ? r[i] / A[i * N + i] : r[i];
        double rz2 = dot(r, z, N);
        double beta = rz2 / rz;
        rz = rz2;
        for (int64_t i = 0; i < N; ++i) p[i] = z[i] + beta * p[i];
    }
    if (its) *its = k;
    if (relres) *relres = rr;
    free(r); free(z); free(p); free(q);
    return rc;
}

int orc_matvec(const double *A, int64_t N, const double *x, double *y)
{
    matvec(A, N, x, y);
    return 0;
}

/* Cap = (1/4pi) <Phi, 1> = (1/4pi) sum_i |T_i| x_i   (Eq. 2.8) */
double orc_capacity(const double *area, const double *x, int64_t N)
{
    double s = 0.0;
    for (int64_t i = 0; i < N; ++i) s += area[i] * x[i];
    return s / (4.0 * ORC_PI);
}

/* ------------------------------------------------------------ ZZ estimator */
/*
 * Primal-P0 reading of Eq. 1.6: the nodal value at vertex z is the area-weighted
 * mean of x over the triangles at z (Zienkiewicz-Zhu recovery), summed in
 * ascending triangle order; I x is the S1 function with those nodal values and
 * eta(T)^2 = h_T ||x_T - I x||^2_{L2(T)} = h_T |T|/12 (sum d_k^2 + (sum d_k)^2),
 * d_k = u_{z_k} - x_T.  h_mode 0: h_T = diam(T) (Eq. 1.6); 1: h_T = |T|^{1/2}.
 * scale_total = sum_T h_T |T| x_T^2 / 12, the size of the indicators of a
 * solution with O(1) relative variation (used to recognise an estimator that
 * vanishes up to rounding).
 */
int orc_zz(const double *V, int64_t M, const int32_t *T, int64_t N, const double *x,
           int h_mode, double *eta2, double *scale_total)
{
    double scale = 0.0;
    double *num = calloc(M, sizeof(double)), *den = calloc(M, sizeof(double));
    double *area = malloc(N * sizeof(double)), *diam = malloc(N * sizeof(double));
    orc_geometry(V, M, T, N, area, diam);
    for (int64_t t = 0; t < N; ++t)
        for (int k = 0; k < 3; ++k) {
            int32_t z = T[3 * t + k];
            double ax = area[t] * x[t];
            num[z] = num[z] + ax;
            den[z] = den[z] + area[t];
        }
    for (int64_t t = 0; t < N; ++t) {
        double d[3];
        for (int k = 0; k < 3; ++k) {
            int32_t z = T[3 * t + k];
            double u = num[z] / den[z];
            d[k] = u - x[t];
        }
        double s2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        double s1 = (d[0] + d[1]) + d[2];
        double q = s2 + s1 * s1;
        double h = h_mode == 1 ? sqrt(area[t]) : diam[t];
        eta2[t] = ((h * area[t]) / 12.0) * q;
        scale += ((h * area[t]) / 12.0) * (x[t] * x[t]);
    }
    if (scale_total) *scale_total = scale;
    free(num); free(den); free(area); free(diam);
    return 0;
}

/* ------------------------------------------------------------ Doerfler */
typedef struct { float key; int64_t idx; } orc_kv;

static int kv_cmp(const void *a, const void *b)
{
    const orc_kv *x = a, *y = b;
    if (x->key > y->key) return -1;
    if (x->key < y->key) return 1;
    return (x->idx > y->idx) - (x->idx < y->idx);
}

/*
 * Eq. 2.6 / Alg. 1 (iii): order the elements by decreasing indicator (compared
 * in single precision, ties by index), form the running sums of eta^2 in that
 * order in FP64, mark the shortest prefix whose running sum reaches
 * theta * total (total = the last running sum), then extend it over elements
 * whose single-precision indicator equals the last marked one.
 *
 * Summation order of the running sums (the paper fixes none; Eq. 2.6 is an
 * inequality between exact sums): the sorted sequence is cut into blocks of
 * ORC_DORFLER_BLOCK consecutive elements; l = the running sum inside a block
 * (from 0, left to right), o_b = the offset of block b (o_0 = 0,
 * o_(b+1) = o_b + the block's full sum l), and the running sum at an element of
 * block b is o_b + l.  For N <= ORC_DORFLER_BLOCK this is the plain left-to-right
 * sum.  Every addition is one IEEE-754 double addition in this order.
 */
#define ORC_DORFLER_BLOCK 128
int orc_dorfler(const double *eta2, int64_t N, double theta, uint8_t *marked, int64_t *n_marked)
{
    orc_kv *kv = malloc((N ? N : 1) * sizeof(orc_kv));
    for (int64_t i = 0; i < N; ++i) {
        kv[i].key = (float)eta2[i];
        kv[i].idx = i;
    }
    qsort(kv, N, sizeof(orc_kv), kv_cmp);
    /* running sums in the two-level order */
    double *run = malloc((N ? N : 1) * sizeof(double));
    double off = 0.0;
    for (int64_t b0 = 0; b0 < N; b0 += ORC_DORFLER_BLOCK) {
        double l = 0.0;
        for (int64_t k = b0; k < N && k < b0 + ORC_DORFLER_BLOCK; ++k) {
            l = l + eta2[kv[k].idx];
            run[k] = off + l;
        }
        off = off + l;
    }
    const double total = N > 0 ? run[N - 1] : 0.0;
    const double thr = theta * total;
    int64_t k = 0;
    while (k < N && (k == 0 ? 0.0 : run[k - 1]) < thr) ++k;
    free(run);
    while (k > 0 && k < N && kv[k].key == kv[k - 1].key) ++k;
    if (N > 0) memset(marked, 0, (size_t)N);
    for (int64_t i = 0; i < k; ++i) marked[kv[i].idx] = 1;
    *n_marked = k;
    free(kv);
    return 0;
}

/* ------------------------------------------------------------ NVB */
/*
 * Reference edge convention: triangle (a, b, c) has reference edge (a, b).
 * orc_canonical rotates each triangle so that its reference edge comes first:
 * the given local edge e (edge (v_e, v_{e+1})) or, by default, the longest edge,
 * ties to the lowest local index.  Rotation keeps the orientation.
 */
int orc_canonical(const double *V, const int32_t *T, int64_t N, const uint8_t *ref_edge,
                  int32_t *T_out)
{
    for (int64_t t = 0; t < N; ++t) {
        const int32_t *v = T + 3 * t;
        int e = 0;
        if (ref_edge) {
            e = ref_edge[t] % 3;
        } else {
            double l[3];
            for (int k = 0; k < 3; ++k) l[k] = edge_len2(V + 3 * (int64_t)v[k], V + 3 * (int64_t)v[(k + 1) % 3]);
            e = 0;
            if (l[1] > l[e]) e = 1;
            if (l[2] > l[e]) e = 2;
        }
        for (int k = 0; k < 3; ++k) T_out[3 * t + k] = v[(e + k) % 3];
    }
    return 0;
}

typedef struct { int32_t u, v; int64_t he; } orc_edge;

static int edge_cmp(const void *a, const void *b)
{
    const orc_edge *x = a, *y = b;
    if (x->u != y->u) return x->u < y->u ? -1 : 1;
    if (x->v != y->v) return x->v < y->v ? -1 : 1;
    return (x->he > y->he) - (x->he < y->he);
}

/*
 * Newest-vertex bisection of the marked triangles plus closure (Fig. 3):
 *   - a marked triangle marks its reference edge (bisec3: all three edges);
 *   - repeat until stable: a triangle with any marked edge marks its reference edge;
 *   - each marked edge gets one new vertex 0.5 (a + b), numbered M, M+1, ... by
 *     first appearance in (triangle index, local edge) order;
 *   - triangle (a,b,c), midpoints m0 of ab, m1 of bc, m2 of ca:
 *       ab        -> (c,a,m0) (b,c,m0)
 *       ab,bc     -> (c,a,m0) (m0,b,m1) (c,m0,m1)
 *       ab,ca     -> (m0,c,m2) (a,m0,m2) (b,c,m0)
 *       ab,bc,ca  -> (m0,c,m2) (a,m0,m2) (m0,b,m1) (c,m0,m1)
 *   - numbering: the unrefined triangles first, in their order, then the children
 *     of the refined ones, parent by parent, each in the order listed above.
 *     parent_out[i] is the source triangle of triangle i and kept_out[i] is 1
 *     when triangle i is that source triangle unchanged.
 * Output capacity: M + 3N vertices, 4N triangles.  Returns the number of
 * closure sweeps.
 */
int orc_refine(const double *V, int64_t M, const int32_t *T, int64_t N, const uint8_t *marked,
               int bisec3, double *V_out, int32_t *T_out, int32_t *parent_out, uint8_t *kept_out,
               int64_t *M_out, int64_t *N_out)
{
    int64_t H = 3 * N;
    orc_edge *E = malloc((H ? H : 1) * sizeof(orc_edge));
    for (int64_t t = 0; t < N; ++t)
        for (int k = 0; k < 3; ++k) {
            int32_t a = T[3 * t + k], b = T[3 * t + (k + 1) % 3];
            E[3 * t + k].u = a < b ? a : b;
            E[3 * t + k].v = a < b ? b : a;
            E[3 * t + k].he = 3 * t + k;
        }
    qsort(E, H, sizeof(orc_edge), edge_cmp);
    int64_t *owner = malloc((H ? H : 1) * sizeof(int64_t)); /* half-edge -> first half-edge of its edge */
    for (int64_t s = 0; s < H;) {
        int64_t e = s;
        while (e < H && E[e].u == E[s].u && E[e].v == E[s].v) ++e;
        for (int64_t r = s; r < e; ++r) owner[E[r].he] = E[s].he;
        s = e;
    }
    uint8_t *flag = calloc(H ? H : 1, 1);
    for (int64_t t = 0; t < N; ++t)
        if (marked[t]) {
            flag[owner[3 * t]] = 1;
            if (bisec3) { flag[owner[3 * t + 1]] = 1; flag[owner[3 * t + 2]] = 1; }
        }
    int sweeps = 0;
    for (int changed = 1; changed;) {
        changed = 0;
        ++sweeps;
        for (int64_t t = 0; t < N; ++t) {
            int any = flag[owner[3 * t]] | flag[owner[3 * t + 1]] | flag[owner[3 * t + 2]];
            if (any && !flag[owner[3 * t]]) { flag[owner[3 * t]] = 1; changed = 1; }
        }
    }
    memcpy(V_out, V, 3 * M * sizeof(double));
    int64_t *mid = malloc((H ? H : 1) * sizeof(int64_t));
    int64_t Mn = M;
    for (int64_t h = 0; h < H; ++h) {
        mid[h] = -1;
        if (owner[h] == h && flag[h]) {
            int32_t a = T[h], b = T[(h / 3) * 3 + (h % 3 + 1) % 3];
            for (int c = 0; c < 3; ++c) V_out[3 * Mn + c] = 0.5 * (V[3 * (int64_t)a + c] + V[3 * (int64_t)b + c]);
            mid[h] = Mn++;
        }
    }
    /* children patterns; unrefined triangles first (in order), then the
     * children of refined triangles, parent by parent, in the pattern order */
    int64_t Nn = 0;
    for (int64_t t = 0; t < N; ++t)
        if (!flag[owner[3 * t]]) {
            for (int k = 0; k < 3; ++k) T_out[3 * Nn + k] = T[3 * t + k];
            parent_out[Nn] = (int32_t)t;
            kept_out[Nn] = 1;
            ++Nn;
        }
    for (int64_t t = 0; t < N; ++t) {
        int32_t a = T[3 * t], b = T[3 * t + 1], c = T[3 * t + 2];
        int f0 = flag[owner[3 * t]], f1 = flag[owner[3 * t + 1]], f2 = flag[owner[3 * t + 2]];
        if (!f0) continue;
        int32_t ch[4][3];
        int nc = 0;
        int32_t m0 = (int32_t)mid[owner[3 * t]];
        int32_t m1 = f1 ? (int32_t)mid[owner[3 * t + 1]] : -1;
        int32_t m2 = f2 ? (int32_t)mid[owner[3 * t + 2]] : -1;
        if (!f1 && !f2) {
            int32_t L[2][3] = {{c, a, m0}, {b, c, m0}};
            memcpy(ch, L, sizeof(L)); nc = 2;
        } else if (f1 && !f2) {
            int32_t L[3][3] = {{c, a, m0}, {m0, b, m1}, {c, m0, m1}};
            memcpy(ch, L, sizeof(L)); nc = 3;
        } else if (!f1 && f2) {
            int32_t L[3][3] = {{m0, c, m2}, {a, m0, m2}, {b, c, m0}};
            memcpy(ch, L, sizeof(L)); nc = 3;
        } else {
            int32_t L[4][3] = {{m0, c, m2}, {a, m0, m2}, {m0, b, m1}, {c, m0, m1}};
            memcpy(ch, L, sizeof(L)); nc = 4;
        }
        for (int r = 0; r < nc; ++r) {
            for (int k = 0; k < 3; ++k) T_out[3 * Nn + k] = ch[r][k];
            parent_out[Nn] = (int32_t)t;
            kept_out[Nn] = 0;
            ++Nn;
        }
    }
    *M_out = Mn;
    *N_out = Nn;
    free(E); free(owner); free(flag); free(mid);
    return sweeps;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel regions (n <= 0: all processors).  Timing only:
 * every reduction of the oracle is sequential, so results do not depend on it. */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    omp_set_num_threads(n > 0 ? n : omp_get_num_procs());
#else
    (void)n;
#endif
}
