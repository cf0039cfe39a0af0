// Assembly of the Galerkin matrix V[i][j] = (1/4pi) int_Ti int_Tj 1/|x-y| on
// piecewise constants (Eq. 2.4-2.5; primal P0 form of App. A, Eq. A.1).
//
//  * Far field (no common vertex): 7 x 7 product of Radon's degree-5 rule,
//      V_ij = |Ti||Tj|/(4pi) sum_a w_a sum_b w_b / |x_a - y_b|.
//    One thread per column j holds its 7 points (FP64, FP32: in registers; DF64: on
//    the current pair's grid in shared memory); the CTA stages R row triangles in
//    shared memory and walks them (broadcast reads; R x C tile variants, chosen per
//    size class by timing them).  Only
//    entries with i <= j are computed; the strict lower triangle is mirrored, so
//    V is exactly symmetric and an incremental re-assembly reproduces the full
//    one bit for bit.  Three arithmetic variants:
//      DF64 -- FP64-accurate double-float on the FP32 pipe: x_a - y_b is formed as
//              (c_i - c_j) + (o_a - o_b) with the centroid difference taken exactly
//              from three-float centroids and the offsets o from the centroid as
//              hi/lo pairs.  Pairs whose centroids are at least 1.12 (R_i + R_j)
//              apart (R: the largest distance of a triangle's points from its
//              centroid; almost all far pairs) split every term on one power-of-two
//              grid chosen for the pair, so that the hi part of x_a - y_b is a single
//              exact subtraction; closer pairs take it by two-sums.  |r|^2 by
//              two-product/two-sum; 1/|r| by the MUFU reciprocal square root and one
//              Newton step in double-float (error ~1.5 e^2 ~ 1e-14); sums by
//              two-sum.  Entries within ~1e-12 of FP64.  V stored as hi/lo pairs.
//      F64  -- native FP64 (GB300 issues FP64 at 1/64 of the FP32 rate).
//      F32  -- centroid difference from hi + lo float centroids, offsets in FP32, MUFU rsqrt;
//              no FP64 operation per pair (GB300 issues FP64 at 1/64 of the FP32 rate).
//  * Near field (common vertex, common edge, identical): Sauter-Schwab
//    regularising transformations.  The 4-d integrand of each region is a power
//    of the radial variables times a function of the others (the kernel is
//    homogeneous of degree -1 on flat panels), so the radial integrals are taken
//    exactly (1/3 for xi^2, 1/2 for rho) -- the same value that a Gauss-Legendre
//    rule with >= 2 points gives in those variables -- and the remaining
//    variables use n Gauss-Legendre points each: identical 6 hexagon sectors x n,
//    common edge 4 sub-regions x n^2, common vertex 2 regions x n^3.  FP64.
#include <cmath>
#include <type_traits>

#include "bem_internal.cuh"
#include "dfloat.cuh"

namespace bem {

__constant__ double c_w7[kQ];
__constant__ float2 c_w7df[kQ];
__constant__ float2 c_inv4pi_df;
__constant__ double c_inv4pi_f32;  // 1 / (4 pi (sum of the FP32 Radon weights)^2)
__constant__ double c_glx[kMaxSS + 1][kMaxSS];
__constant__ double c_glw[kMaxSS + 1][kMaxSS];

static bool g_asm_ready[64] = {false};

// Gauss-Legendre rule with n points on [0, 1]: roots of P_n by Newton's method on
// the three-term recurrence, weights 2 / ((1 - x^2) P_n'(x)^2) halved.
static void gauss_legendre(int n, double *x, double *w)
{
    const double pi = 3.14159265358979323846;
    for (int i = 0; i < n; ++i) {
        double r = std::cos(pi * (i + 0.75) / (n + 0.5));
        double d = 0.0;
        for (int it = 0; it < 60; ++it) {
            double pm1 = 1.0, p = r;  // P_0, P_1
            for (int k = 1; k < n; ++k) {
                const double pn = ((2.0 * k + 1.0) * r * p - k * pm1) / (k + 1.0);
                pm1 = p;
                p = pn;
            }
            if (n == 1) { p = r; pm1 = 1.0; }
            d = n * (pm1 - r * p) / (1.0 - r * r);  // P_n'(r)
            const double step = p / d;
            r -= step;
            if (std::fabs(step) <= 1e-17) break;
        }
        double pm1 = 1.0, p = r;
        for (int k = 1; k < n; ++k) {
            const double pn = ((2.0 * k + 1.0) * r * p - k * pm1) / (k + 1.0);
            pm1 = p;
            p = pn;
        }
        if (n == 1) { p = r; pm1 = 1.0; }
        d = n * (pm1 - r * p) / (1.0 - r * r);
        x[n - 1 - i] = 0.5 * (1.0 + r);
        w[n - 1 - i] = 1.0 / ((1.0 - r * r) * d * d);
    }
}

static bem_status far_df_attributes(bem_ctx *ctx);

static bem_status assembly_constants(bem_ctx *ctx)
{
    if (ctx->device < 64 && g_asm_ready[ctx->device]) return BEM_OK;
    if (bem_status st = far_df_attributes(ctx)) return st;
    const double r15 = std::sqrt(15.0);
    const double wa = (155.0 - r15) / 1200.0, wb = (155.0 + r15) / 1200.0;
    const double w7[kQ] = {9.0 / 40.0, wa, wa, wa, wb, wb, wb};
    double X[kMaxSS + 1][kMaxSS] = {}, W[kMaxSS + 1][kMaxSS] = {};
    for (int n = 1; n <= kMaxSS; ++n) gauss_legendre(n, X[n], W[n]);
    float2 w7df[kQ];
    for (int a = 0; a < kQ; ++a) {
        const float h = (float)w7[a];
        w7df[a] = make_float2(h, (float)(w7[a] - (double)h));
    }
    BEM_CK(ctx, cudaMemcpyToSymbol(c_w7, w7, sizeof(w7)));
    BEM_CK(ctx, cudaMemcpyToSymbol(c_w7df, w7df, sizeof(w7df)));
    const float ih = (float)kInv4Pi;
    const float2 inv4pi = make_float2(ih, (float)(kInv4Pi - (double)ih));
    BEM_CK(ctx, cudaMemcpyToSymbol(c_inv4pi_df, &inv4pi, sizeof(inv4pi)));
    double wsum = 0.0;  // exact: seven floats of similar size
    for (int a = 0; a < kQ; ++a) wsum += (double)w7df[a].x;
    const double inv4pi_f32 = kInv4Pi / (wsum * wsum);
    BEM_CK(ctx, cudaMemcpyToSymbol(c_inv4pi_f32, &inv4pi_f32, sizeof(inv4pi_f32)));
    BEM_CK(ctx, cudaMemcpyToSymbol(c_glx, X, sizeof(X)));
    BEM_CK(ctx, cudaMemcpyToSymbol(c_glw, W, sizeof(W)));
    if (ctx->device < 64) g_asm_ready[ctx->device] = true;
    return BEM_OK;
}

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// Element storage: FP64, double-float hi/lo pair, or FP32.
template <typename T> struct Elem;
template <> struct Elem<double> {
    __device__ static double from_double(double v) { return v; }
    __host__ __device__ static double to_double(double v) { return v; }
};
template <> struct Elem<float> {
    __device__ static float from_double(double v) { return (float)v; }
    __host__ __device__ static double to_double(float v) { return (double)v; }
};
template <> struct Elem<float2> {
    __device__ static float2 from_double(double v) { return df_from_double(v); }
    __host__ __device__ static double to_double(float2 v) { return df_to_double(v); }
};

// ------------------------------------------------------------------ far field
// Pair tiles: a CTA of C threads (one column each) walks R row triangles staged in
// shared memory.  Every variant computes each entry with the same operations, so V
// is bit-identical whichever is used; the fastest depends on N (small meshes want
// more, smaller CTAs) and on the arithmetic, and is chosen by timing (autotune).
struct FarTileS {
    int rows, cols;
    int min_ctas;  // DF64: > 0 -- point loops rolled, this many CTAs per SM requested
                   // (the other arithmetics use their unrolled register form)
};
constexpr FarTileS kFarTiles[kFarTileVariants] = {
    {32, 256, 0}, {16, 256, 0}, {64, 256, 0}, {8, 128, 0}, {16, 128, 0}, {32, 128, 0}, {8, 128, 8},
    {16, 128, 8}, {32, 128, 8}, {8, 128, 9},  {8, 64, 16},  {8, 64, 18},  {8, 128, 6}, {32, 128, 6}};

// The far-field bodies take the tile origin (first row i0, first column cbase) as
// arguments: the per-operator kernels derive it from the block index, the batched
// kernel (several operators in one launch) from its work list.
template <int R, int C>
__device__ __forceinline__ void far_f64_body(const double *__restrict__ q64, double *__restrict__ V, int64_t ld,
                                             int64_t r1, int64_t c1, int64_t i0, int64_t cbase)
{
    __shared__ double sx[R][22];
    if (i0 > cbase + C - 1 || i0 >= r1) return;  // tile strictly below the diagonal
    for (int k = threadIdx.x; k < R * 22; k += C) {
        const int r = k / 22, c = k % 22;
        const int64_t i = i0 + r;
        sx[r][c] = (i < r1) ? q64[i * kQ64Stride + c] : 0.0;
    }
    __syncthreads();
    const int64_t j = cbase + threadIdx.x;
    if (j >= c1) return;
    double y[3 * kQ];
#pragma unroll
    for (int c = 0; c < 3 * kQ; ++c) y[c] = q64[j * kQ64Stride + c];
    const double Aj = q64[j * kQ64Stride + 21] * kInv4Pi;
    const int rows = (int)((r1 - i0) < R ? (r1 - i0) : R);
    for (int r = 0; r < rows; ++r) {
        const int64_t i = i0 + r;
        if (i > j) break;
        double acc = 0.0;
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
            const double xa = sx[r][3 * a], ya = sx[r][3 * a + 1], za = sx[r][3 * a + 2];
            double s = 0.0;
#pragma unroll
            for (int b = 0; b < kQ; ++b) {
                const double dx = xa - y[3 * b], dy = ya - y[3 * b + 1], dz = za - y[3 * b + 2];
                s += c_w7[b] * rsqrt(dx * dx + dy * dy + dz * dz);
            }
            acc += c_w7[a] * s;
        }
        V[i * ld + j] = sx[r][21] * Aj * acc;
    }
}

template <int R, int C>
__global__ void __launch_bounds__(C) k_far_f64(const double *__restrict__ q64, double *__restrict__ V,
                                                      int64_t ld, int64_t r0, int64_t r1, int64_t c0,
                                                      int64_t c1)
{
    far_f64_body<R, C>(q64, V, ld, r1, c1, r0 + (int64_t)blockIdx.y * R, c0 + (int64_t)blockIdx.x * C);
}

template <int R, int C>
__device__ __forceinline__ void far_f32_body(const float *__restrict__ q32, const double *__restrict__ cent,
                                             float *__restrict__ V, int64_t ld, int64_t r1, int64_t c1,
                                             int64_t i0, int64_t cbase)
{
    // FP32 only in the pair loop: centroids as hi + lo floats, so that the centroid
    // difference (hi_i - hi_j) + (lo_i - lo_j) keeps FP32 relative accuracy for
    // distant pairs; weights and areas rounded to FP32 once
    __shared__ float so[R][3 * kQ];
    __shared__ float sc[R][7];  // centroid hi (3), lo (3), area
    if (i0 > cbase + C - 1 || i0 >= r1) return;
    for (int k = threadIdx.x; k < R * 3 * kQ; k += C) {
        const int r = k / (3 * kQ), c = k % (3 * kQ);
        const int64_t i = i0 + r;
        so[r][c] = (i < r1) ? q32[i * kQ32Stride + c] : 0.0f;
    }
    for (int k = threadIdx.x; k < R * 4; k += C) {
        const int r = k / 4, c = k % 4;
        const int64_t i = i0 + r;
        const double v = (i < r1) ? cent[i * 4 + c] : 0.0;
        const float h = (float)v;
        if (c < 3) {
            sc[r][c] = h;
            sc[r][3 + c] = (float)(v - (double)h);
        } else {
            sc[r][6] = h;
        }
    }
    __syncthreads();
    const int64_t j = cbase + threadIdx.x;
    if (j >= c1) return;
    float y[3 * kQ];
#pragma unroll
    for (int c = 0; c < 3 * kQ; ++c) y[c] = q32[j * kQ32Stride + c];
    float ch[3], cl[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double v = cent[4 * j + c];
        ch[c] = (float)v;
        cl[c] = (float)(v - (double)ch[c]);
    }
    // 1/(4pi) with the weights' rounding undone: the FP32 Radon weights all round down
    // (their sum is 1 - 2.98e-8), which would scale every far entry by (sum w)^2; the
    // factor 1 / (sum of the FP32 weights)^2 is folded into the column's area term
    const float Aj = (float)(cent[4 * j + 3] * c_inv4pi_f32);
    float wf[kQ];  // the weights rounded to FP32 once (c_w7df[.].x = nearest float)
#pragma unroll
    for (int a = 0; a < kQ; ++a) wf[a] = c_w7df[a].x;
    const int rows = (int)((r1 - i0) < R ? (r1 - i0) : R);
    for (int r = 0; r < rows; ++r) {
        const int64_t i = i0 + r;
        if (i > j) break;
        const float Dx = (sc[r][0] - ch[0]) + (sc[r][3] - cl[0]);
        const float Dy = (sc[r][1] - ch[1]) + (sc[r][4] - cl[1]);
        const float Dz = (sc[r][2] - ch[2]) + (sc[r][5] - cl[2]);
        float acc = 0.0f;
#pragma unroll
        for (int a = 0; a < kQ; ++a) {
            const float xa = Dx + so[r][3 * a], ya = Dy + so[r][3 * a + 1], za = Dz + so[r][3 * a + 2];
            float s = 0.0f;
#pragma unroll
            for (int b = 0; b < kQ; ++b) {
                const float dx = xa - y[3 * b], dy = ya - y[3 * b + 1], dz = za - y[3 * b + 2];
                s += wf[b] * rsqrtf(dx * dx + dy * dy + dz * dz);
            }
            acc += wf[a] * s;
        }
        V[i * ld + j] = sc[r][6] * Aj * acc;
    }
}

template <int R, int C>
__global__ void __launch_bounds__(C) k_far_f32(const float *__restrict__ q32,
                                                      const double *__restrict__ cent, float *__restrict__ V,
                                                      int64_t ld, int64_t r0, int64_t r1, int64_t c0,
                                                      int64_t c1)
{
    far_f32_body<R, C>(q32, cent, V, ld, r1, c1, r0 + (int64_t)blockIdx.y * R, c0 + (int64_t)blockIdx.x * C);
}

// Double-float far field: see the file comment.
//
// v rounded to the nearest multiple of q = 2^(e-23), for |v| < 2^(e-1) and big =
// 1.5 * 2^e: v + big lies in [2^e, 2^(e+1)], whose spacing is q, and the subtraction
// of big is exact (Sterbenz).
__device__ __forceinline__ float grid_snap(float v, float big) { return __fsub_rn(__fadd_rn(v, big), big); }

// s + e = a + b exactly for a, b >= 0 (Dekker's fast two-sum with the larger first).
__device__ __forceinline__ void pos_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(fminf(a, b), __fsub_rn(s, fmaxf(a, b)));
}

// 1/|d| = y + yl for |d|^2 = Sh + Sl: the MUFU estimate y and one Newton step in
// double-float, yl = y t / 2 with t = 1 - S y^2 and y^2 = y2 + y2e by a two-product.
// The estimate's relative error is below 2^-22, so 1 - Sh y2 is below 2^-20 in size
// and its single rounding in the FMA is below 2^-44; the other terms are of order
// 2^-24 and enter by FMAs.
template <bool FTZ = false>
__device__ __forceinline__ void df_rsqrt_newton(float Sh, float Sl, float &y, float &yl)
{
    if (FTZ)  // Sh known to be a normal number: the bare MUFU estimate
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(Sh));
    else
        y = rsqrtf(Sh);
    float y2, y2e;
    two_prod(y, y, y2, y2e);
    float t = __fmaf_rn(-Sh, y2, 1.0f);
    t = __fmaf_rn(-Sh, y2e, t);
    t = __fmaf_rn(-Sl, y2, t);
    yl = __fmul_rn(__fmul_rn(0.5f, y), t);
}

// sh + sl += w (y + yl) with the two-sum of the running sum (pos: sh and w y are not
// negative, the larger added first)
template <bool POS = false>
__device__ __forceinline__ void df_acc_w(float2 w, float y, float yl, float &sh, float &sl)
{
    float ph, pe, u, ue;
    two_prod(w.x, y, ph, pe);
    pe = __fmaf_rn(w.x, yl, pe);
    pe = __fmaf_rn(w.y, y, pe);
    if (POS)
        pos_two_sum(sh, ph, u, ue);
    else
        two_sum(sh, ph, u, ue);
    sh = u;
    sl = __fadd_rn(sl, __fadd_rn(pe, ue));
}

// Entry sum sum_a w_a sum_b w_b / |x_a - y_b| of a pair whose bounding balls are close
// (|c_i - c_j| < 1.12 (R_i + R_j)): x_a - y_b = (D + o_a) - o_b in double-float by
// two-sums, D = c_i - c_j, o the offsets from the centroids (o_b from the table).
__device__ __forceinline__ void far_df_exact(const float *qi, const float *Dh, const float *Dl,
                                             const float2 *__restrict__ oj, float &h_out, float &l_out)
{
    float acc_h = 0.0f, acc_l = 0.0f;
#pragma unroll 1
    for (int a = 0; a < kQ; ++a) {
        float eh[3], el[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float s, e;
            two_sum(Dh[c], qi[2 * (3 * a + c)], s, e);
            e = __fadd_rn(e, __fadd_rn(Dl[c], qi[2 * (3 * a + c) + 1]));
            fast_two_sum(s, e, eh[c], el[c]);
        }
        float sh = 0.0f, sl = 0.0f;
#pragma unroll 1
        for (int b = 0; b < kQ; ++b) {
            // d = e_a - o_b; |d|^2 = sum h^2 + 2 h l (two-product, two-sum)
            float Sh = 0.0f, Sl = 0.0f;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float h, e;
                const float2 o = oj[3 * b + c];
                two_sum(eh[c], -o.x, h, e);
                const float l = __fadd_rn(e, __fsub_rn(el[c], o.y));
                float p, pe;
                two_prod(h, h, p, pe);
                pe = __fmaf_rn(__fmul_rn(2.0f, h), l, pe);
                if (c == 0) {
                    Sh = p;
                    Sl = pe;
                } else {
                    float t, te;
                    two_sum(Sh, p, t, te);
                    Sh = t;
                    Sl = __fadd_rn(Sl, __fadd_rn(pe, te));
                }
            }
            float y, yl;
            df_rsqrt_newton(Sh, Sl, y, yl);
            df_acc_w(c_w7df[b], y, yl, sh, sl);
        }
        df_acc_w(c_w7df[a], sh, sl, acc_h, acc_l);
    }
    fast_two_sum(acc_h, acc_l, h_out, l_out);
}

// The same sum for a pair with |D| >= 1.12 (R_i + R_j) (R: the largest distance of a
// triangle's points from its centroid): D, o_a and o_b are split on the pair's grid
// q = 2^(e-23), 2^(e-1) > max(|D|_inf, r_i, r_j) (r: the largest |hi| of the offset
// coordinates) with e odd -- hi parts multiples of q (exact), lo parts the rest -- so
// that the hi part h of x_a - y_b is one exact subtraction and its lo part l one
// rounded one; |d|^2 = h^2 + 2 h l + l^2 with h^2 by a two-product.  Every |x_a - y_b|
// is at least 0.107 |D| and 2^e <= 8 |D|, so the lo parts' roundings (a few units of
// 2^-24 q each) stay below 1e-11 of the entry.  sg: o_b on the grid, (hi, 2 lo),
// stride C.
template <int C, bool UNROLL>
__device__ __forceinline__ void far_df_grid(const float *qi, const float *Dh, const float *Dl, float big,
                                            const float2 *sg, float &h_out, float &l_out)
{
    float Dg[3], Dl2[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Dg[c] = grid_snap(Dh[c], big);
        Dl2[c] = __fmul_rn(2.0f, __fadd_rn(__fsub_rn(Dh[c], Dg[c]), Dl[c]));
    }
    float acc_h = 0.0f, acc_l = 0.0f;
#pragma unroll(UNROLL ? kQ : 1)
    for (int a = 0; a < kQ; ++a) {
        float eh[3], el2[3];  // x_a - c_j: hi on the grid, twice the lo part
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const float oh = qi[2 * (3 * a + c)], og = grid_snap(oh, big);
            eh[c] = __fadd_rn(Dg[c], og);
            el2[c] = __fmaf_rn(2.0f, __fadd_rn(__fsub_rn(oh, og), qi[2 * (3 * a + c) + 1]), Dl2[c]);
        }
        float sh = 0.0f, sl = 0.0f;
        auto point_pair = [&](int b) {
            float p[3], pe[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 o = sg[(3 * b + c) * C];
                const float dh = __fsub_rn(eh[c], o.x);  // exact
                const float dl2 = __fsub_rn(el2[c], o.y);
                p[c] = __fmul_rn(dh, dh);
                pe[c] = __fmaf_rn(dh, dh, -p[c]);
                pe[c] = __fmaf_rn(dl2, __fmaf_rn(0.25f, dl2, dh), pe[c]);  // 2 h l + l^2
            }
            float s1, e1, s2, e2, y, yl;
            pos_two_sum(p[0], p[1], s1, e1);
            pos_two_sum(s1, p[2], s2, e2);
            df_rsqrt_newton<true>(s2, __fadd_rn(__fadd_rn(pe[0], pe[1]), __fadd_rn(pe[2], __fadd_rn(e1, e2))), y,
                                  yl);
            df_acc_w<true>(c_w7df[b], y, yl, sh, sl);
        };
        if (UNROLL) {
#pragma unroll
            for (int b = 0; b < kQ; ++b) point_pair(b);
        } else {  // two point pairs per trip: half the loop control
            point_pair(0);
#pragma unroll 2
            for (int b = 1; b < kQ; ++b) point_pair(b);
        }
        df_acc_w<true>(c_w7df[a], sh, sl, acc_h, acc_l);
    }
    fast_two_sum(acc_h, acc_l, h_out, l_out);
}

// MB > 0: MB CTAs per SM requested (registers capped to fit), the point loops rolled
// unless UB.  The column triangle's offsets on the current pair's grid are kept in
// dynamic shared memory (3 kQ x C pairs, thread-major: conflict-free), re-split only
// when the grid changes from one row to the next.
template <int C>
constexpr size_t far_df_smem() { return sizeof(float2) * 3 * kQ * C; }

template <int R, int C, int MB, bool UB = false>
__device__ __forceinline__ void far_df_body(const float *__restrict__ qdf, float2 *__restrict__ V, int64_t ld,
                                            int64_t r1, int64_t c1, int64_t i0, int64_t cbase)
{
    constexpr bool UNROLL = MB == 0 || UB;
    __shared__ float sq[R][55];
    extern __shared__ float2 far_dsm[];
    if (i0 > cbase + C - 1 || i0 >= r1) return;
    for (int k = threadIdx.x; k < R * 55; k += C) {
        const int r = k / 55, c = k % 55;
        const int64_t i = i0 + r;
        sq[r][c] = (i < r1) ? qdf[i * kQdfStride + c] : 0.0f;
    }
    __syncthreads();
    const int64_t j = cbase + threadIdx.x;
    if (j >= c1) return;
    const float *qj = qdf + j * kQdfStride;
    const float2 *oj = reinterpret_cast<const float2 *>(qj);
    float2 *sg = far_dsm + threadIdx.x;
    float cj[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) cj[k] = qj[42 + k];
    const float rj = qj[53], Rj = qj[54];
    const float2 Aj = df_mul(make_float2(qj[51], qj[52]), c_inv4pi_df);
    unsigned eg = 0u;  // exponent field of the grid bound sg holds (0: none)
    const int rows = (int)((r1 - i0) < R ? (r1 - i0) : R);
    for (int r = 0; r < rows; ++r) {
        const int64_t i = i0 + r;
        if (i > j) break;
        const float *qi = sq[r];
        // centroid difference c_i - c_j from the three-float centroids
        float Dh[3], Dl[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float s1, e1, s2, e2, h, l;
            two_sum(qi[42 + 3 * c], -cj[3 * c], s1, e1);
            two_sum(qi[43 + 3 * c], -cj[3 * c + 1], s2, e2);
            const float s3 = __fsub_rn(qi[44 + 3 * c], cj[3 * c + 2]);
            two_sum(s1, s2, h, l);
            l = __fadd_rn(l, __fadd_rn(__fadd_rn(e1, e2), s3));
            fast_two_sum(h, l, Dh[c], Dl[c]);
        }
        const float ri = qi[53], Rs = qi[54] + Rj;
        const float bound = fmaxf(fmaxf(fabsf(Dh[0]), fabsf(Dh[1])), fmaxf(fmaxf(fabsf(Dh[2]), ri), rj));
        // bound in [2^(eb-127), 2^(eb-126)); odd eb, so that the grid changes less often
        // from one row to the next
        const unsigned eb = (__float_as_uint(bound) >> 23) | 1u;
        const float D2 = Dh[0] * Dh[0] + Dh[1] * Dh[1] + Dh[2] * Dh[2];
        float h, l;
        // the grid path where its bounds hold (and no product of it can leave the
        // normal FP32 range); the two-sum path otherwise
        if (D2 >= 1.26f * (Rs * Rs) && eb >= 93u && eb <= 185u) {
            const float big = __uint_as_float(((eb + 2u) << 23) | 0x400000u);  // 1.5 * 2^(eb-125)
            if (eb != eg) {
#pragma unroll 1
                for (int k = 0; k < 3 * kQ; ++k) {
                    const float2 o = oj[k];
                    const float g = grid_snap(o.x, big);
                    sg[k * C] = make_float2(g, __fmul_rn(2.0f, __fadd_rn(__fsub_rn(o.x, g), o.y)));
                }
                eg = eb;
            }
            far_df_grid<C, UNROLL>(qi, Dh, Dl, big, sg, h, l);
        } else {
            far_df_exact(qi, Dh, Dl, oj, h, l);
        }
        V[i * ld + j] = df_mul(df_mul(make_float2(qi[51], qi[52]), Aj), make_float2(h, l));
    }
}

template <int R, int C>
__global__ void __launch_bounds__(C) k_far_df(const float *__restrict__ qdf, float2 *__restrict__ V, int64_t ld,
                                              int64_t r0, int64_t r1, int64_t c0, int64_t c1)
{
    far_df_body<R, C, 0>(qdf, V, ld, r1, c1, r0 + (int64_t)blockIdx.y * R, c0 + (int64_t)blockIdx.x * C);
}

// UB: the inner point loop unrolled (more registers: fewer CTAs per SM requested)
template <int R, int C, int MB, bool UB = false>
__global__ void __launch_bounds__(C, MB) k_far_df_s(const float *__restrict__ qdf, float2 *__restrict__ V, int64_t ld,
                                                    int64_t r0, int64_t r1, int64_t c0, int64_t c1)
{
    far_df_body<R, C, MB, UB>(qdf, V, ld, r1, c1, r0 + (int64_t)blockIdx.y * R, c0 + (int64_t)blockIdx.x * C);
}

// Mirror the strict lower triangle of rows [r0, r1): V[i][j] = V[j][i], j < i,
// through 32 x 32 shared-memory tiles (coalesced on both sides).
template <typename T>
__device__ __forceinline__ void mirror_tile(T *V, int64_t ld, int64_t r0, int64_t r1, int64_t bi, int64_t bj)
{
    __shared__ T tile[32][33];
    if (bj > bi) return;
    const int tx = threadIdx.x, ty = threadIdx.y;
    // load source block rows bj.., cols bi.. (upper part)
    for (int k = ty; k < 32; k += 8) {
        const int64_t sr = bj + k, sc = bi + tx;
        tile[k][tx] = (sr < r1 && sc < r1) ? V[sr * ld + sc] : T();
    }
    __syncthreads();
    for (int k = ty; k < 32; k += 8) {
        const int64_t i = bi + k, j = bj + tx;
        if (i >= r0 && i < r1 && j < i) V[i * ld + j] = tile[tx][k];
    }
}

template <typename T>
__global__ void k_mirror(T *V, int64_t ld, int64_t r0, int64_t r1)
{
    // destination row tile, destination column tile
    mirror_tile<T>(V, ld, r0, r1, (int64_t)blockIdx.y * 32 + (r0 / 32) * 32, (int64_t)blockIdx.x * 32);
}

// ------------------------------------------------------------------ near field
struct Tri {
    double p[3][3];
};

__device__ __forceinline__ double inv_norm3(double x, double y, double z)
{
    return rsqrt(x * x + y * y + z * z);
}

// The near-field quadratures below return one thread's share of the sum: thread sub of
// a group of kNearGroup takes every kNearGroup-th index of the outermost loop, and the
// group's shares are added in a fixed order before the constant factor is applied.
constexpr int kNearGroup = 4;

// Identical panels: (1/6) sum over the 6 hexagon sectors of int_0^1 1/|J w(eta)|.
__device__ double ss_identical(const Tri &P, int n, int sub)
{
    const double *gx = c_glx[n], *gw = c_glw[n];
    const double J1[3] = {P.p[1][0] - P.p[0][0], P.p[1][1] - P.p[0][1], P.p[1][2] - P.p[0][2]};
    const double J2[3] = {P.p[2][0] - P.p[1][0], P.p[2][1] - P.p[1][1], P.p[2][2] - P.p[1][2]};
    const double H[7][2] = {{1, 0}, {1, 1}, {0, 1}, {-1, 0}, {-1, -1}, {0, -1}, {1, 0}};
    double s = 0.0;
    for (int k = sub; k < 6; k += kNearGroup) {
        const double px = H[k][0], py = H[k][1], qx = H[k + 1][0], qy = H[k + 1][1];
        for (int g = 0; g < n; ++g) {
            const double z1 = px + gx[g] * (qx - px), z2 = py + gx[g] * (qy - py);
            s += gw[g] * inv_norm3(z1 * J1[0] + z2 * J2[0], z1 * J1[1] + z2 * J2[1], z1 * J1[2] + z2 * J2[2]);
        }
    }
    return s;  // times 1/6
}

// Common edge: P = (A,B,C), Q = (A,B,D).  x - y = xi rho (+-a e + t1 fP - t2 fQ).
__device__ double ss_edge(const Tri &P, const Tri &Q, int n, int sub)
{
    const double *gx = c_glx[n], *gw = c_glw[n];
    double e[3], fP[3], fQ[3];
    for (int c = 0; c < 3; ++c) {
        e[c] = P.p[1][c] - P.p[0][c];
        fP[c] = P.p[2][c] - P.p[1][c];
        fQ[c] = Q.p[2][c] - Q.p[1][c];
    }
    double s = 0.0;
    for (int iu = sub; iu < n; iu += kNearGroup)
        for (int iv = 0; iv < n; ++iv) {
            const double u = gx[iu], v = gx[iv], w = gw[iu] * gw[iv];
            // sub-region a: (own, a, other) = (1, u(1-v), uv), weight u
            // sub-region b: (own, a, other) = (u, 1-v, v),    weight 1
            const double oa = 1.0, aa = u * (1.0 - v), ha = u * v;
            const double ob = u, ab = 1.0 - v, hb = v;
            double t = 0.0;
            // region 1 (s1 = xi): vec = a e + own fP - other fQ
            t += u * inv_norm3(aa * e[0] + oa * fP[0] - ha * fQ[0], aa * e[1] + oa * fP[1] - ha * fQ[1],
                               aa * e[2] + oa * fP[2] - ha * fQ[2]);
            t += inv_norm3(ab * e[0] + ob * fP[0] - hb * fQ[0], ab * e[1] + ob * fP[1] - hb * fQ[1],
                           ab * e[2] + ob * fP[2] - hb * fQ[2]);
            // region 2 (s2 = xi): vec = -a e + other fP - own fQ
            t += u * inv_norm3(-aa * e[0] + ha * fP[0] - oa * fQ[0], -aa * e[1] + ha * fP[1] - oa * fQ[1],
                               -aa * e[2] + ha * fP[2] - oa * fQ[2]);
            t += inv_norm3(-ab * e[0] + hb * fP[0] - ob * fQ[0], -ab * e[1] + hb * fP[1] - ob * fQ[1],
                           -ab * e[2] + hb * fP[2] - ob * fQ[2]);
            s += w * t;
        }
    return s;  // times 1/6
}

// Common vertex: P = (A,B,C), Q = (A,D,E).  Regions x = (1,e1), y = e2 (1,e3) and
// x = e2 (1,e1), y = (1,e3), weight e2.
__device__ double ss_vertex(const Tri &P, const Tri &Q, int n, int sub)
{
    const double *gx = c_glx[n], *gw = c_glw[n];
    double a1[3], a2[3], b1[3], b2[3];
    for (int c = 0; c < 3; ++c) {
        a1[c] = P.p[1][c] - P.p[0][c];
        a2[c] = P.p[2][c] - P.p[1][c];
        b1[c] = Q.p[1][c] - Q.p[0][c];
        b2[c] = Q.p[2][c] - Q.p[1][c];
    }
    double s = 0.0;
    for (int i1 = sub; i1 < n; i1 += kNearGroup) {
        double xa[3];
        for (int c = 0; c < 3; ++c) xa[c] = a1[c] + gx[i1] * a2[c];
        for (int i3 = 0; i3 < n; ++i3) {
            double yb[3];
            for (int c = 0; c < 3; ++c) yb[c] = b1[c] + gx[i3] * b2[c];
            double t = 0.0;
            for (int i2 = 0; i2 < n; ++i2) {
                const double e2 = gx[i2];
                const double r1 = inv_norm3(xa[0] - e2 * yb[0], xa[1] - e2 * yb[1], xa[2] - e2 * yb[2]);
                const double r2 = inv_norm3(e2 * xa[0] - yb[0], e2 * xa[1] - yb[1], e2 * xa[2] - yb[2]);
                t += gw[i2] * e2 * (r1 + r2);
            }
            s += gw[i1] * gw[i3] * t;
        }
    }
    return s;  // times 1/3
}

__device__ __forceinline__ void load_tri(const double *verts, const int32_t *v, Tri &T)
{
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c) T.p[k][c] = verts[3 * (int64_t)v[k] + c];
}

// kind 0: identical pairs i = j = K + idx; 1: common-vertex list; 2: common-edge list.
// Pairs (i < j) with j < K are skipped (their entries are reused).  Called by every
// thread of a warp (valid false for the padding): the kNearGroup threads of a pair each
// integrate their share, the shares are summed in a fixed order ((s0 + s1) + (s2 + s3))
// by shuffles, and the group's first thread writes the entry.
template <typename T>
__device__ __forceinline__ void near_entry(const double *__restrict__ verts, const int32_t *__restrict__ tris,
                                           const double *__restrict__ area, const int32_t *__restrict__ pairs,
                                           int64_t idx, int kind, int64_t K, int n, T *V, int64_t ld, bool valid)
{
    static_assert(kNearGroup == 4, "the group sum below adds four shares");
    const int sub = (int)(threadIdx.x % kNearGroup);
    int64_t i = 0, j = 0;
    bool write = false;
    double I = 0.0;
    if (valid) {
        if (kind == 0) {
            i = j = K + idx;
        } else {
            i = pairs[2 * idx];
            j = pairs[2 * idx + 1];
        }
        write = kind == 0 || j >= K;
    }
    if (write) {
        const int32_t *ti = tris + 3 * i, *tj = tris + 3 * j;
        if (kind == 0) {
            Tri P;
            load_tri(verts, ti, P);
            I = ss_identical(P, n, sub);
        } else if (kind == 2) {
            // (u, v) = the shared vertices in the order they appear in triangle i
            int32_t u = -1, v = -1, ci = -1, cj = -1;
            for (int k = 0; k < 3; ++k) {
                const bool in = (ti[k] == tj[0] || ti[k] == tj[1] || ti[k] == tj[2]);
                if (in) {
                    if (u < 0) u = ti[k];
                    else v = ti[k];
                } else {
                    ci = ti[k];
                }
            }
            for (int k = 0; k < 3; ++k)
                if (tj[k] != u && tj[k] != v) cj = tj[k];
            const int32_t pi[3] = {u, v, ci}, pj[3] = {u, v, cj};
            Tri P, Q;
            load_tri(verts, pi, P);
            load_tri(verts, pj, Q);
            I = ss_edge(P, Q, n, sub);
        } else {
            int ki = 0, kj = 0;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    if (ti[a] == tj[b]) {
                        ki = a;
                        kj = b;
                    }
            const int32_t pi[3] = {ti[ki], ti[(ki + 1) % 3], ti[(ki + 2) % 3]};
            const int32_t pj[3] = {tj[kj], tj[(kj + 1) % 3], tj[(kj + 2) % 3]};
            Tri P, Q;
            load_tri(verts, pi, P);
            load_tri(verts, pj, Q);
            I = ss_vertex(P, Q, n, sub);
        }
    }
    I += __shfl_xor_sync(0xffffffffu, I, 1);
    I += __shfl_xor_sync(0xffffffffu, I, 2);
    if (write && sub == 0) {
        I = kind == 1 ? I / 3.0 : I / 6.0;
        const double v = 4.0 * area[i] * area[j] * I * kInv4Pi;
        const T e = Elem<T>::from_double(v);
        V[i * ld + j] = e;
        if (i != j) V[j * ld + i] = e;
    }
}

// All touching pairs of an assembly in one launch, kNearGroup threads per pair: the
// common-vertex pairs (the longest quadrature) first, then the common-edge pairs, then
// the identical pairs of the new triangles, so that the three lists overlap instead of
// running one after another.  Each list starts on a warp boundary (its pair count
// rounded up to kNearPairsPerWarp), so that no warp runs two of the quadratures.
constexpr int kNearPairsPerWarp = 32 / kNearGroup;
inline int64_t near_pad(int64_t n) { return (n + kNearPairsPerWarp - 1) / kNearPairsPerWarp * kNearPairsPerWarp; }

template <typename T>
__global__ void k_near(const double *__restrict__ verts, const int32_t *__restrict__ tris,
                       const double *__restrict__ area, const int32_t *__restrict__ vert_pairs, int64_t n_vert,
                       const int32_t *__restrict__ edge_pairs, int64_t n_edge, int64_t n_ident, int64_t K, int n,
                       T *V, int64_t ld)
{
    const int64_t nvp = (n_vert + kNearPairsPerWarp - 1) / kNearPairsPerWarp * kNearPairsPerWarp;
    const int64_t nep = (n_edge + kNearPairsPerWarp - 1) / kNearPairsPerWarp * kNearPairsPerWarp;
    int64_t idx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kNearGroup;
    if (idx < nvp) {
        near_entry<T>(verts, tris, area, vert_pairs, idx, 1, K, n, V, ld, idx < n_vert);
    } else if ((idx -= nvp) < nep) {
        near_entry<T>(verts, tris, area, edge_pairs, idx, 2, K, n, V, ld, idx < n_edge);
    } else {
        idx -= nep;
        near_entry<T>(verts, tris, area, nullptr, idx, 0, K, n, V, ld, idx < n_ident);
    }
}

// ------------------------------------------------------------------ reuse and diagonal
// V'[i][j] = Vc[parent[i]][parent[j]] for i, j < K (unrefined triangles), by 64 x 64
// tiles: CTA (bx, by) copies rows 64 by.. and columns 64 bx.., thread t column t % 64 and
// the 16 rows 16 (t / 64).. of the tile (16 independent loads in flight; a warp reads
// 32 nearly consecutive entries of a coarse row, the kept triangles keeping their
// order).  upper: entries i <= j only (tiles below the diagonal return at once; the
// kept triangles keep their order, so these come from the coarse operator's upper
// triangle).
template <typename T>
__global__ void __launch_bounds__(256) k_gather_kept(const T *__restrict__ Vc, int64_t ldc,
                                                     const int32_t *__restrict__ parent, int64_t K,
                                                     T *__restrict__ V, int64_t ld, int upper)
{
    if (upper && blockIdx.y > blockIdx.x) return;
    const int64_t j = (int64_t)blockIdx.x * 64 + (threadIdx.x & 63);
    const int64_t i0 = (int64_t)blockIdx.y * 64 + 16 * (threadIdx.x >> 6);
    if (j >= K) return;
    const int64_t pj = parent[j];
    const int64_t iend = upper ? (j + 1 < K ? j + 1 : K) : K;
    T v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r)
        if (i0 + r < iend) v[r] = Vc[(int64_t)parent[i0 + r] * ldc + pj];
#pragma unroll
    for (int r = 0; r < 16; ++r)
        if (i0 + r < iend) V[(i0 + r) * ld + j] = v[r];
}

// Mirror of the diagonal 64 x 64 blocks only: 32 x 32 tiles (2D, 2D), (2D+1, 2D),
// (2D+1, 2D+1) of block D, item t = 3 D + (0, 1, 2).
template <typename T>
__global__ void k_mirror_diag(T *V, int64_t ld, int64_t N)
{
    const int64_t t = blockIdx.x, D = t / 3, r = t % 3;
    const int64_t bi = 2 * D + (r > 0 ? 1 : 0), bj = 2 * D + (r == 2 ? 1 : 0);
    mirror_tile<T>(V, ld, 0, N, 32 * bi, 32 * bj);
}

template <typename T>
__global__ void k_diag(const T *V, int64_t ld, int64_t N, double *d)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) d[i] = Elem<T>::to_double(V[i * ld + i]);
}

// ------------------------------------------------------------------ drivers
template <typename T, int R, int C, int MB = 0, bool UB = false>
static void far_kernel(bem_operator *op, dim3 grid, int64_t r0, int64_t r1, int64_t c0, int64_t c1)
{
    bem_mesh *m = op->mesh;
    cudaStream_t s = m->ctx->stream;
    if (op->precision == BEM_PREC_F64)
        k_far_f64<R, C><<<grid, C, 0, s>>>(m->q64, (double *)op->V, op->ld, r0, r1, c0, c1);
    else if (op->precision == BEM_PREC_DF64)
    {
        if constexpr (MB > 0)
            k_far_df_s<R, C, MB, UB><<<grid, C, far_df_smem<C>(), s>>>(m->qdf, (float2 *)op->V, op->ld, r0, r1,
                                                                       c0, c1);
        else
            k_far_df<R, C><<<grid, C, far_df_smem<C>(), s>>>(m->qdf, (float2 *)op->V, op->ld, r0, r1, c0, c1);
    }
    else
        k_far_f32<R, C><<<grid, C, 0, s>>>(m->q32, m->cent, (float *)op->V, op->ld, r0, r1, c0, c1);
}

// Far-field entries i <= j of the block [r0, r1) x [c0, c1) with tile variant v.
template <typename T>
static bem_status launch_far(bem_operator *op, int v, int64_t r0, int64_t r1, int64_t c0, int64_t c1,
                             bool profile = true)
{
    if (r1 <= r0 || c1 <= c0) return BEM_OK;
    bem_mesh *m = op->mesh;
    bem_ctx *ctx = m->ctx;
    const int R = kFarTiles[v].rows, C = kFarTiles[v].cols;
    const int64_t gx = (c1 - c0 + C - 1) / C;
    const int64_t gy = (r1 - r0 + R - 1) / R;
    if (gy > 65535) {
        // split rows into chunks that fit the grid's y limit
        for (int64_t rs = r0; rs < r1; rs += 65535LL * R) {
            const int64_t re = rs + 65535LL * R < r1 ? rs + 65535LL * R : r1;
            bem_status st = launch_far<T>(op, v, rs, re, c0, c1, profile);
            if (st) return st;
        }
        return BEM_OK;
    }
    dim3 grid((unsigned)gx, (unsigned)gy);
    double units = 0.0;  // entries with i <= j in the block
    for (int64_t i = r0; i < r1; ++i) {
        const int64_t lo = i > c0 ? i : c0;
        if (c1 > lo) units += (double)(c1 - lo);
    }
    const int prof = profile ? prof_start(ctx, BEM_KERNEL_FAR, units) : -1;
    switch (v) {
    case 0: far_kernel<T, 32, 256>(op, grid, r0, r1, c0, c1); break;
    case 1: far_kernel<T, 16, 256>(op, grid, r0, r1, c0, c1); break;
    case 2: far_kernel<T, 64, 256>(op, grid, r0, r1, c0, c1); break;
    case 3: far_kernel<T, 8, 128>(op, grid, r0, r1, c0, c1); break;
    case 4: far_kernel<T, 16, 128>(op, grid, r0, r1, c0, c1); break;
    case 5: far_kernel<T, 32, 128>(op, grid, r0, r1, c0, c1); break;
    case 6: far_kernel<T, 8, 128, 8>(op, grid, r0, r1, c0, c1); break;
    case 7: far_kernel<T, 16, 128, 8>(op, grid, r0, r1, c0, c1); break;
    case 8: far_kernel<T, 32, 128, 8>(op, grid, r0, r1, c0, c1); break;
    case 9: far_kernel<T, 8, 128, 9>(op, grid, r0, r1, c0, c1); break;
    case 10: far_kernel<T, 8, 64, 16>(op, grid, r0, r1, c0, c1); break;
    case 11: far_kernel<T, 8, 64, 18>(op, grid, r0, r1, c0, c1); break;
    case 12: far_kernel<T, 8, 128, 6, true>(op, grid, r0, r1, c0, c1); break;
    default: far_kernel<T, 32, 128, 6, true>(op, grid, r0, r1, c0, c1); break;
    }
    BEM_COUNT(ctx);
    if (profile) prof_stop(ctx, prof);
    BEM_CK_LAUNCH(ctx);
    return BEM_OK;
}

// Size classes of the tile cache: N < 1,024, < 4,096, < 16,384, larger.
static int far_bucket(int64_t N) { return N < 1024 ? 0 : N < 4096 ? 1 : N < 16384 ? 2 : 3; }

// The tile variant of this assembly: the requested one, else the context's choice
// for (precision, size class), timed now on this assembly's own far-field block if
// the class has none yet -- every variant once to load its module, then once timed,
// the fastest kept.  No timing while the stream is being captured into a graph (the
// variant is then the cached one, or variant 0).
template <typename T>
static bem_status far_variant(bem_operator *op, int64_t K, int64_t N, int *v_out)
{
    bem_ctx *ctx = op->mesh->ctx;
    if (op->tile > 0) {
        *v_out = op->tile - 1;
        return BEM_OK;
    }
    int8_t &slot = ctx->far_tile[op->precision][far_bucket(N)];
    *v_out = slot >= 0 ? slot : 0;
    if (slot >= 0 || N - K <= 0) return BEM_OK;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    BEM_CK(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
    if (cs != cudaStreamCaptureStatusNone) return BEM_OK;
    float best = 0.0f;
    int bv = 0;
    for (int pass = 0; pass < 2; ++pass)
        for (int v = 0; v < kFarTileVariants; ++v) {
            BEM_CK(ctx, cudaEventRecord(ctx->ev[4], ctx->stream));
            bem_status st = launch_far<T>(op, v, K, N, K, N, false);
            if (st) return st;
            BEM_CK(ctx, cudaEventRecord(ctx->ev[5], ctx->stream));
            BEM_CK(ctx, cudaEventSynchronize(ctx->ev[5]));
            float ms = 0.0f;
            BEM_CK(ctx, cudaEventElapsedTime(&ms, ctx->ev[4], ctx->ev[5]));
            if (pass == 1 && (v == 0 || ms < best)) {
                best = ms;
                bv = v;
            }
        }
    slot = (int8_t)bv;
    *v_out = bv;
    return BEM_OK;
}

int far_cached_variant(const bem_ctx *ctx, int precision, int64_t N) { return ctx->far_tile[precision][far_bucket(N)]; }

bem_status far_tune(bem_operator *op)
{
    int v = 0;
    const int64_t N = op->mesh->N;
    if (op->precision == BEM_PREC_F64) return far_variant<double>(op, 0, N, &v);
    if (op->precision == BEM_PREC_DF64) return far_variant<float2>(op, 0, N, &v);
    return far_variant<float>(op, 0, N, &v);
}

template <typename T>
static bem_status launch_mirror(bem_operator *op, int64_t r0, int64_t r1)
{
    if (r1 <= r0) return BEM_OK;
    bem_ctx *ctx = op->mesh->ctx;
    const int64_t t0 = r0 / 32, t1 = (r1 + 31) / 32;
    for (int64_t ts = t0; ts < t1; ts += 65535) {
        const int64_t te = ts + 65535 < t1 ? ts + 65535 : t1;
        dim3 grid((unsigned)te, (unsigned)(te - ts));
        k_mirror<T><<<grid, dim3(32, 8), 0, ctx->stream>>>((T *)op->V, op->ld, ts * 32 > r0 ? ts * 32 : r0,
                                                           te * 32 < r1 ? te * 32 : r1); BEM_COUNT(ctx);
        BEM_CK_LAUNCH(ctx);
    }
    return BEM_OK;
}

template <typename T>
static bem_status launch_near(bem_operator *op, int64_t K)
{
    bem_mesh *m = op->mesh;
    bem_ctx *ctx = m->ctx;
    const int n = op->ss_order;
    const int prof = prof_start(ctx, BEM_KERNEL_NEAR, (double)(m->N - K + m->n_vert_pairs + m->n_edge_pairs));
    const int64_t n_ident = m->N > K ? m->N - K : 0;
    const int64_t total = near_pad(m->n_vert_pairs) + near_pad(m->n_edge_pairs) + n_ident;
    if (total > 0) {
        k_near<T><<<nblk(total * kNearGroup, 128), 128, 0, ctx->stream>>>(m->verts, m->tris, m->area, m->vert_pairs,
                                                             m->n_vert_pairs, m->edge_pairs, m->n_edge_pairs, n_ident,
                                                             K, n, (T *)op->V, op->ld);
        BEM_COUNT(ctx);
    }
    prof_stop(ctx, prof);
    BEM_CK_LAUNCH(ctx);
    return BEM_OK;
}

// Zero the padding columns [N, ld) of every row (the far field, the mirror, the near
// field and the reused block write every entry of [0, N) x [0, N)).
template <typename T>
__global__ void k_zero_padding(T *V, int64_t ld, int64_t N)
{
    const int64_t i = blockIdx.x, j = N + threadIdx.x;
    if (i < N && j < ld) V[i * ld + j] = T();
}

template <typename T>
static bem_status launch_mirror_diag(bem_operator *op)
{
    bem_ctx *ctx = op->mesh->ctx;
    const int64_t T32 = (op->N + 31) / 32, items = 3 * (T32 / 2) + (T32 % 2);
    if (items > 0) {
        k_mirror_diag<T><<<(unsigned)items, dim3(32, 8), 0, ctx->stream>>>((T *)op->V, op->ld, op->N); BEM_COUNT(ctx);
        BEM_CK_LAUNCH(ctx);
    }
    return BEM_OK;
}

// upper: fill only the upper triangle and the diagonal blocks (op->upper_only)
template <typename T>
static bem_status assemble_t(bem_operator *op, const bem_operator *coarse, bool upper)
{
    bem_mesh *m = op->mesh;
    bem_ctx *ctx = m->ctx;
    const int64_t N = m->N;
    if (op->ld > N) {
        k_zero_padding<T><<<(unsigned)N, 64, 0, ctx->stream>>>((T *)op->V, op->ld, N); BEM_COUNT(ctx);
    }
    bem_status st;
    int64_t K = 0;
    if (coarse) {
        K = m->n_kept;
        if (K > 0) {
            dim3 grid(nblk(K, 64), nblk(K, 64));
            k_gather_kept<T><<<grid, 256, 0, ctx->stream>>>((const T *)coarse->V, coarse->ld, m->parent, K,
                                                            (T *)op->V, op->ld,
                                                            (upper || coarse->upper_only) ? 1 : 0); BEM_COUNT(ctx);
            BEM_CK_LAUNCH(ctx);
        }
    }
    int v = 0;
    if ((st = far_variant<T>(op, K, N, &v))) return st;
    if (K > 0 && (st = launch_far<T>(op, v, 0, K, K, N))) return st;
    if ((st = launch_far<T>(op, v, K, N, K, N))) return st;
    if (upper) {
        if ((st = launch_mirror_diag<T>(op))) return st;
    } else {
        // a coarse operator with its upper triangle alone gave the kept block's upper half
        const int64_t m0 = (coarse && coarse->upper_only) ? 0 : (K > 0 ? K : 0);
        if ((st = launch_mirror<T>(op, m0, N))) return st;
    }
    op->upper_only = upper ? 1 : 0;
    if ((st = launch_near<T>(op, K))) return st;
    k_diag<T><<<nblk(N, 256), 256, 0, ctx->stream>>>((const T *)op->V, op->ld, N, op->diag); BEM_COUNT(ctx);
    BEM_CK_LAUNCH(ctx);
    return BEM_OK;
}

// ------------------------------------------------------------------ batched assembly
// The assembly of every operator of a batch wave in one launch per phase: the far
// field over a work list of (problem, row tile, column tile) items, the mirror over
// the 32 x 32 tile pairs of all problems, the near field over the concatenated
// identical / common-vertex / common-edge lists.  Every entry is computed by the same
// device code as the per-operator kernels, so the operators are bit-identical to
// bem_assemble_V's.

// Problem p with prefix[p] <= k < prefix[p + 1] (prefix: P + 1 ascending entries).
__device__ __forceinline__ int batch_find(const int64_t *__restrict__ prefix, int P, int64_t k)
{
    int lo = 0, hi = P - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= k)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

template <typename T, int R, int C, int MB, bool UB>
__global__ void __launch_bounds__(C, (MB > 0 ? MB : 1))
    k_far_batch(const BatchAsmProb *__restrict__ prob, const int4 *__restrict__ items)
{
    const int4 it = items[blockIdx.x];
    const BatchAsmProb *pb = prob + it.x;
    const int64_t N = pb->N, ld = pb->ld;
    if constexpr (std::is_same<T, double>::value)
        far_f64_body<R, C>(pb->q64, (double *)pb->V, ld, N, N, it.y, it.z);
    else if constexpr (std::is_same<T, float2>::value)
        far_df_body<R, C, MB, UB>(pb->qdf, (float2 *)pb->V, ld, N, N, it.y, it.z);
    else
        far_f32_body<R, C>(pb->q32, pb->cent, (float *)pb->V, ld, N, N, it.y, it.z);
}

// Tile pair t of a problem: row tile bi >= column tile bj, t = bi (bi + 1) / 2 + bj.
// A batch's operators are read only through their upper triangle (the packed tiles, the
// DF64 tile products, the symmetric reads of the block preconditioner), so only the
// 64 x 64 diagonal blocks, whose lower halves those tiles include, are mirrored: 32 x 32
// tiles (2D, 2D), (2D+1, 2D), (2D+1, 2D+1) of block D, item t = 3 D + (0, 1, 2).
template <typename T>
__global__ void k_mirror_batch(const BatchAsmProb *__restrict__ prob, const int64_t *__restrict__ pref, int P)
{
    const int64_t k = blockIdx.x;
    const int p = batch_find(pref, P, k);
    const int64_t t = k - pref[p];
    const int64_t D = t / 3, r = t % 3;
    const int64_t bi = 2 * D + (r > 0 ? 1 : 0), bj = 2 * D + (r == 2 ? 1 : 0);
    const BatchAsmProb *pb = prob + p;
    mirror_tile<T>((T *)pb->V, pb->ld, 0, pb->N, 32 * bi, 32 * bj);
}

// Item k of a problem: identical pairs [0, N), common-vertex pairs, common-edge pairs.
// kNearGroup threads per item (every thread of a warp reaches near_entry's group sum).
template <typename T>
__global__ void k_near_batch(const BatchAsmProb *__restrict__ prob, const int64_t *__restrict__ pref, int P,
                             int64_t total, int n)
{
    const int64_t k = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / kNearGroup;
    const bool valid = k < total;
    const int p = batch_find(pref, P, valid ? k : total - 1);
    const BatchAsmProb *pb = prob + p;
    int64_t idx = (valid ? k : total - 1) - pref[p];
    const int64_t N = pb->N;
    if (idx < N) {
        near_entry<T>(pb->verts, pb->tris, pb->area, nullptr, idx, 0, 0, n, (T *)pb->V, pb->ld, valid);
    } else if ((idx -= N) < pb->n_vert) {
        near_entry<T>(pb->verts, pb->tris, pb->area, pb->vert_pairs, idx, 1, 0, n, (T *)pb->V, pb->ld, valid);
    } else {
        idx -= pb->n_vert;
        near_entry<T>(pb->verts, pb->tris, pb->area, pb->edge_pairs, idx, 2, 0, n, (T *)pb->V, pb->ld, valid);
    }
}

int far_variant_rows(int v) { return kFarTiles[v].rows; }
int far_variant_cols(int v) { return kFarTiles[v].cols; }

void batch_far_items(int v, int p, int64_t N, std::vector<int4> &items)
{
    const int64_t R = kFarTiles[v].rows, C = kFarTiles[v].cols;
    for (int64_t i0 = 0; i0 < N; i0 += R)
        for (int64_t c = (i0 / C) * C; c < N; c += C)  // tiles reaching the diagonal or above
            if (i0 <= c + C - 1) items.push_back(make_int4(p, (int)i0, (int)c, 0));
}

template <typename T, int R, int C, int MB = 0, bool UB = false>
static void far_batch_launch(const BatchAsm &b, cudaStream_t s)
{
    const size_t smem = std::is_same<T, float2>::value ? far_df_smem<C>() : 0;
    k_far_batch<T, R, C, MB, UB><<<(unsigned)b.n_far, C, smem, s>>>(b.prob, b.far_items);
}

// The DF64 tiles of 256 columns whose shared memory (row staging + the column
// offsets on the pair grid) exceeds the default 48 KB per CTA.
static bem_status far_df_attributes(bem_ctx *ctx)
{
    const int dyn = (int)far_df_smem<256>();
    BEM_CK(ctx, cudaFuncSetAttribute(k_far_df<32, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    BEM_CK(ctx, cudaFuncSetAttribute(k_far_df<64, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    BEM_CK(ctx, cudaFuncSetAttribute(k_far_batch<float2, 32, 256, 0, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    BEM_CK(ctx, cudaFuncSetAttribute(k_far_batch<float2, 64, 256, 0, false>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, dyn));
    return BEM_OK;
}

// Event record that also fires when a captured graph replays (an external event node
// while the stream is being captured; a plain record otherwise).
bem_status record_timing_event(bem_ctx *ctx, cudaEvent_t e)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    BEM_CK(ctx, cudaStreamIsCapturing(ctx->stream, &cs));
    BEM_CK(ctx, cudaEventRecordWithFlags(e, ctx->stream,
                                         cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                             : cudaEventRecordDefault));
    return BEM_OK;
}

template <typename T>
static bem_status batch_assemble_t(bem_ctx *ctx, const BatchAsm &b, cudaEvent_t *ev)
{
    cudaStream_t s = ctx->stream;
    bem_status st;
    if (ev && (st = record_timing_event(ctx, ev[0]))) return st;
    if (b.n_far > 0) {
        switch (b.variant) {
        case 0: far_batch_launch<T, 32, 256>(b, s); break;
        case 1: far_batch_launch<T, 16, 256>(b, s); break;
        case 2: far_batch_launch<T, 64, 256>(b, s); break;
        case 3: far_batch_launch<T, 8, 128>(b, s); break;
        case 4: far_batch_launch<T, 16, 128>(b, s); break;
        case 5: far_batch_launch<T, 32, 128>(b, s); break;
        case 6: far_batch_launch<T, 8, 128, 8>(b, s); break;
        case 7: far_batch_launch<T, 16, 128, 8>(b, s); break;
        case 8: far_batch_launch<T, 32, 128, 8>(b, s); break;
        case 9: far_batch_launch<T, 8, 128, 9>(b, s); break;
        case 10: far_batch_launch<T, 8, 64, 16>(b, s); break;
        case 11: far_batch_launch<T, 8, 64, 18>(b, s); break;
        case 12: far_batch_launch<T, 8, 128, 6, true>(b, s); break;
        default: far_batch_launch<T, 32, 128, 6, true>(b, s); break;
        }
        BEM_COUNT(ctx);
        BEM_CK_LAUNCH(ctx);
    }
    if (ev && (st = record_timing_event(ctx, ev[1]))) return st;
    if (b.n_mirror > 0) {
        k_mirror_batch<T><<<(unsigned)b.n_mirror, dim3(32, 8), 0, s>>>(b.prob, b.mirror_pref, b.P); BEM_COUNT(ctx);
        BEM_CK_LAUNCH(ctx);
    }
    if (ev && (st = record_timing_event(ctx, ev[2]))) return st;
    if (b.n_near > 0) {
        k_near_batch<T><<<nblk(b.n_near * kNearGroup, 128), 128, 0, s>>>(b.prob, b.near_pref, b.P, b.n_near,
                                                                          b.ss_order);
        BEM_COUNT(ctx);
        BEM_CK_LAUNCH(ctx);
    }
    if (ev && (st = record_timing_event(ctx, ev[3]))) return st;
    return BEM_OK;
}

bem_status batch_assemble(bem_ctx *ctx, const BatchAsm &b, cudaEvent_t *ev)
{
    if (b.precision == BEM_PREC_F64) return batch_assemble_t<double>(ctx, b, ev);
    if (b.precision == BEM_PREC_DF64) return batch_assemble_t<float2>(ctx, b, ev);
    return batch_assemble_t<float>(ctx, b, ev);
}

bem_status assembly_prepare(bem_ctx *ctx) { return assembly_constants(ctx); }

bem_status gauss_legendre_upload(int n)
{
    (void)n;
    return BEM_OK;
}

bem_status assemble_full(bem_operator *op, bool upper_only)
{
    bem_status st = assembly_constants(op->mesh->ctx);
    if (st) return st;
    if (op->precision == BEM_PREC_F64) return assemble_t<double>(op, nullptr, upper_only);
    if (op->precision == BEM_PREC_DF64) return assemble_t<float2>(op, nullptr, upper_only);
    return assemble_t<float>(op, nullptr, upper_only);
}

bem_status assemble_update(bem_operator *op, const bem_operator *coarse, bool upper_only)
{
    bem_status st = assembly_constants(op->mesh->ctx);
    if (st) return st;
    if (op->precision == BEM_PREC_F64) return assemble_t<double>(op, coarse, upper_only);
    if (op->precision == BEM_PREC_DF64) return assemble_t<float2>(op, coarse, upper_only);
    return assemble_t<float>(op, coarse, upper_only);
}

// The lower triangle of an upper-only operator, mirrored from the upper one (bit-
// identical copies) before a reader of whole rows.
bem_status ensure_full(bem_operator *op)
{
    if (!op || !op->upper_only) return BEM_OK;
    bem_status st;
    if (op->precision == BEM_PREC_F64) st = launch_mirror<double>(op, 0, op->N);
    else if (op->precision == BEM_PREC_DF64) st = launch_mirror<float2>(op, 0, op->N);
    else st = launch_mirror<float>(op, 0, op->N);
    if (!st) op->upper_only = 0;
    return st;
}

bem_status operator_diag(bem_operator *op)
{
    bem_ctx *ctx = op->mesh->ctx;
    if (op->precision == BEM_PREC_F64)
        { k_diag<double><<<nblk(op->N, 256), 256, 0, ctx->stream>>>((const double *)op->V, op->ld, op->N, op->diag); BEM_COUNT(ctx); }
    else if (op->precision == BEM_PREC_DF64)
        { k_diag<float2><<<nblk(op->N, 256), 256, 0, ctx->stream>>>((const float2 *)op->V, op->ld, op->N, op->diag); BEM_COUNT(ctx); }
    else
        { k_diag<float><<<nblk(op->N, 256), 256, 0, ctx->stream>>>((const float *)op->V, op->ld, op->N, op->diag); BEM_COUNT(ctx); }
    BEM_CK_LAUNCH(ctx);
    return BEM_OK;
}

}  // namespace bem
