// Solve V x = b, b_i = |T_i| (Eq. 2.5 with f = 1) and Cap = (1/4pi) b.x (Eq. 2.8).
//
// Dense V x (the paper needs "only matrix-vector products", Sec. 1.4) streams V
// once per product: one warp per row, 16-byte vector loads with the streaming
// cache hint, x served from L1/L2, a fixed warp-shuffle reduction (deterministic).
// The PCG recurrences (Jacobi preconditioner diag(V), the paper's "diag",
// Sec. 3) run in FP64 in three launches per iteration; every global sum is taken
// over per-block partials in a fixed order, so a solve is bit-reproducible.
// FP32 operators: FP64 iterative refinement -- r = b - V x with FP64-accurate
// accumulation, an inner PCG on that residual, x += d.  The inner products also
// accumulate in double-float: with FP32 sums the error (~sqrt(N) 2^-24, 1.5e-5 at
// N = 60k) would sit at the inner tolerance, and the product is HBM-bound either way.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include <cuda_fp16.h>

#include "bem_internal.cuh"
#include "dfloat.cuh"
#include "grid_sync.cuh"

namespace bem {

constexpr int kMvThreads = 256;               // 8 rows per CTA
constexpr int kMvRows = kMvThreads / 32;
constexpr int kVecThreads = 256;

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Block sum of one value per thread into out[blockIdx.x] (fixed tree).
__device__ __forceinline__ void block_partial(double v, double *out)
{
    __shared__ double sw[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sw[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? sw[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) out[blockIdx.x] = t;
    }
    __syncthreads();
}

// Fixed-order sum of n partials, computed by every thread block that needs it.
__device__ double sum_partials(const double *p, int n)
{
    __shared__ double sw[32];
    __shared__ double res;
    double v = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) v += p[k];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sw[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? sw[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) res = t;
    }
    __syncthreads();
    return res;
}

// y = V x for V stored as T (double or float); x, y FP64 of length ld (x zero-padded).
// kAcc64: accumulate in FP64 (else FP32 products and sums per lane).
// If dot_partial: also block partials of sum_i w_i y_i.
template <typename T, bool kAcc64>
__global__ void __launch_bounds__(kMvThreads) k_matvec(const T *__restrict__ V, int64_t ld, int64_t N,
                                                       const double *__restrict__ x, double *__restrict__ y,
                                                       const double *__restrict__ w, double *dot_partial)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t row = (int64_t)blockIdx.x * kMvRows + warp;
    double acc = 0.0;
    if (row < N) {
        if (sizeof(T) == 8) {
            const double2 *r = reinterpret_cast<const double2 *>(V + row * ld);
            const double2 *xv = reinterpret_cast<const double2 *>(x);
            const int64_t n2 = ld / 2;
#pragma unroll 4
            for (int64_t k = lane; k < n2; k += 32) {
                const double2 a = __ldcs(r + k);
                const double2 b = __ldg(xv + k);
                acc = fma(a.x, b.x, acc);
                acc = fma(a.y, b.y, acc);
            }
        } else {
            const float4 *r = reinterpret_cast<const float4 *>(V + row * ld);
            const double2 *xv = reinterpret_cast<const double2 *>(x);
            const int64_t n4 = ld / 4;
            float accf = 0.0f;
#pragma unroll 4
            for (int64_t k = lane; k < n4; k += 32) {
                const float4 a = __ldcs(r + k);
                const double2 b0 = __ldg(xv + 2 * k), b1 = __ldg(xv + 2 * k + 1);
                if (kAcc64) {
                    acc = fma((double)a.x, b0.x, acc);
                    acc = fma((double)a.y, b0.y, acc);
                    acc = fma((double)a.z, b1.x, acc);
                    acc = fma((double)a.w, b1.y, acc);
                } else {
                    accf = fmaf(a.x, (float)b0.x, accf);
                    accf = fmaf(a.y, (float)b0.y, accf);
                    accf = fmaf(a.z, (float)b1.x, accf);
                    accf = fmaf(a.w, (float)b1.y, accf);
                }
            }
            if (!kAcc64) acc = (double)accf;
        }
        acc = warp_sum(acc);
        if (lane == 0) y[row] = acc;
    }
    if (dot_partial) {
        __shared__ double sd[kMvRows];
        if (lane == 0) sd[warp] = (row < N) ? w[row] * acc : 0.0;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kMvRows; ++k) t += sd[k];
            dot_partial[blockIdx.x] = t;
        }
    }
}

// Double-float y = V x for V entries stored as hi/lo pairs (float2) or as FP32
// (float), x given as hi/lo pairs: every product is exact up to the neglected
// lo*lo term and every sum is a two-sum, so y carries ~2^-46 relative error while
// only the FP32 pipe is used (HBM-bound on GB300, where FP64 FMA would not be).
__device__ __forceinline__ void acc_df(float &sh, float &sl, float vh, float vl, float xh, float xl)
{
    float p, e, s, t;
    two_prod(vh, xh, p, e);
    e = __fmaf_rn(vh, xl, e);
    e = __fmaf_rn(vl, xh, e);
    two_sum(sh, p, s, t);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(e, t));
}

template <typename T>
__global__ void __launch_bounds__(kMvThreads) k_matvec_df(const T *__restrict__ V, int64_t ld, int64_t N,
                                                          const float2 *__restrict__ xdf, double *__restrict__ y,
                                                          const double *__restrict__ w, double *dot_partial)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t row = (int64_t)blockIdx.x * kMvRows + warp;
    double acc = 0.0;
    if (row < N) {
        float sh = 0.0f, sl = 0.0f;
        const float4 *r = reinterpret_cast<const float4 *>(V + row * ld);
        const float4 *xv = reinterpret_cast<const float4 *>(xdf);
        if (sizeof(T) == 8) {
            const int64_t n2 = ld / 2;
#pragma unroll 4
            for (int64_t k = lane; k < n2; k += 32) {
                const float4 a = __ldcs(r + k);
                const float4 b = __ldg(xv + k);
                acc_df(sh, sl, a.x, a.y, b.x, b.y);
                acc_df(sh, sl, a.z, a.w, b.z, b.w);
            }
        } else {
            const int64_t n4 = ld / 4;
#pragma unroll 4
            for (int64_t k = lane; k < n4; k += 32) {
                const float4 a = __ldcs(r + k);
                const float4 b0 = __ldg(xv + 2 * k), b1 = __ldg(xv + 2 * k + 1);
                acc_df(sh, sl, a.x, 0.0f, b0.x, b0.y);
                acc_df(sh, sl, a.y, 0.0f, b0.z, b0.w);
                acc_df(sh, sl, a.z, 0.0f, b1.x, b1.y);
                acc_df(sh, sl, a.w, 0.0f, b1.z, b1.w);
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, sh, o), ol = __shfl_xor_sync(0xffffffffu, sl, o);
            const float2 t = df_add(make_float2(sh, sl), make_float2(oh, ol));
            sh = t.x;
            sl = t.y;
        }
        acc = (double)sh + (double)sl;
        if (lane == 0) y[row] = acc;
    }
    if (dot_partial) {
        __shared__ double sd[kMvRows];
        if (lane == 0) sd[warp] = (row < N) ? w[row] * acc : 0.0;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < kMvRows; ++k) t += sd[k];
            dot_partial[blockIdx.x] = t;
        }
    }
}

// Symmetric V x from the upper triangle only (half the HBM traffic).  A
// persistent CTA walks a list of tiles (I, J), I <= J, of 64 x 64 entries; each
// tile is streamed once into shared memory by 16-byte cp.async copies, double
// buffered so that the next tile is in flight while this one is used, into rows
// padded to 68 pairs (bank-conflict-free for both passes).  Row pass: four threads
// per row form V_IJ x_J (row partials of block I); column pass, off the diagonal:
// four threads per column form V_IJ^T x_I (column partials of block J).  All sums
// in double-float.  k_symv_reduce adds the partials of each row in a fixed order.
constexpr int kSB = 64;
constexpr int kSP = 68;  // padded row stride (pairs)
constexpr int kSymThreads = 256;
constexpr size_t kSymSmem = 2 * (kSB * kSP + 2 * kSB) * sizeof(float2) + 4 * kSB * sizeof(float2);

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;  // src-size 0: zero fill
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Stage tile (I, J) and the x segments of blocks I and J into one buffer.
__device__ __forceinline__ void symv_stage(const float2 *V, int64_t ld, int64_t N, const float2 *xdf, int2 tj,
                                           float2 *tile, float2 *xs)
{
    const int t = threadIdx.x;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        const int id = t + kSymThreads * k;  // 2048 chunks of 16 bytes
        const int r = id >> 5, c16 = id & 31;
        const int64_t row = (int64_t)tj.x * kSB + r;
        const bool ok = row < N;
        const float2 *src = V + (ok ? row : 0) * ld + (int64_t)tj.y * kSB + 2 * c16;
        cp_async16(tile + r * kSP + 2 * c16, src, ok);
    }
    if (t < 64) {  // x_I (pairs 0..63) then x_J (64..127), 2 pairs per copy
        const int blk = t < 32 ? tj.x : tj.y;
        const int off = 2 * (t & 31);
        cp_async16(xs + (t < 32 ? 0 : kSB) + off, xdf + (int64_t)blk * kSB + off, true);
    }
}

// Tile loop of the symmetric product for CTA cta of G (shared by the standalone
// kernel and the persistent solver); sm: kSymSmem bytes of dynamic shared memory.
// Tiles are taken either statically (k = cta, cta + G, ...) or, when ctr is given,
// dynamically: each grab is an atomicAdd on *ctr, which never decreases; a grab
// returns tile (value - base) and each CTA makes exactly one grab past the last
// tile, so one pass consumes ntiles + G grabs.  A tile's partials do not depend on
// which CTA computes it.
__device__ __forceinline__ int symv_grab(unsigned long long *ctr, unsigned long long base)
{
    __shared__ int s_k;
    __syncthreads();
    if (threadIdx.x == 0) s_k = (int)(atomicAdd(ctr, 1ull) - base);
    __syncthreads();
    return s_k;
}

// pack (nullable): also write the FP32 hi parts of each staged tile, row-major
// 64 x 64 at pack + 4096 k for tile k of the list (the packed upper triangle).
constexpr int kTileF = kSB * kSB;
// BEM_PRODUCTS_FP16: replaced residual after every 10^2-fold drop of ||r|| (r.r by
// 10^4); fallback to the exact products when a replacement finds r.r above
// kH16Progress times the previous replacement's (||r|| fallen by less than 10x)
constexpr double kH16Delta2 = 1e-4;
constexpr double kH16Progress = 1e-2;
// a segment this long without reaching its drop also ends in a replaced residual (and
// so in the progress test): the FP16 products can hold the recursion itself back
constexpr int kH16SegMax = 400;

__device__ void symv_tiles(const float2 *__restrict__ V, int64_t ld, int64_t N, const int2 *__restrict__ tiles,
                           int ntiles, const float2 *__restrict__ xdf, float2 *__restrict__ prow,
                           float2 *__restrict__ pcol, float2 *sm, int cta, int G,
                           unsigned long long *ctr = nullptr, unsigned long long base = 0, float *pack = nullptr)
{
    // [tile buffer 0][tile buffer 1][x segments 0][x segments 1][column partials 4 x 64]
    float2 *const xs0 = sm + 2 * kSB * kSP;
    float2 *cpart = sm + 2 * kSB * kSP + 4 * kSB;
    const int t = threadIdx.x;
    int it = 0;
    int k = ctr ? symv_grab(ctr, base) : cta;
    if (k < ntiles) symv_stage(V, ld, N, xdf, tiles[k], sm, xs0);
    cp_async_commit();
    for (; k < ntiles; ++it) {
        const int cur = it & 1;
        const int nk = ctr ? symv_grab(ctr, base) : k + G;
        if (nk < ntiles) symv_stage(V, ld, N, xdf, tiles[nk], sm + (cur ^ 1) * kSB * kSP, xs0 + (cur ^ 1) * 2 * kSB);
        cp_async_commit();
        cp_async_wait1();
        __syncthreads();
        const int2 tj = tiles[k];
        const float2 *T = sm + cur * kSB * kSP;
        const float2 *xi = xs0 + cur * 2 * kSB, *xj = xi + kSB;
        const int64_t base = (int64_t)k * kSB;
        if (pack) {
            float4 *dst = reinterpret_cast<float4 *>(pack + (int64_t)k * kTileF);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int f = t + kSymThreads * u;  // float4 f: row f / 16, columns 4 (f % 16) ..
                const float2 *src = T + (f >> 4) * kSP + 4 * (f & 15);
                dst[f] = make_float4(src[0].x, src[1].x, src[2].x, src[3].x);
            }
        }
        {  // row pass: row r, columns q, q+4, ..., q+60
            const int r = t >> 2, q = t & 3;
            float h = 0.f, l = 0.f;
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                const int c = q + 4 * m;
                const float2 v = T[r * kSP + c], x = xj[c];
                acc_df(h, l, v.x, v.y, x.x, x.y);
            }
#pragma unroll
            for (int o = 1; o < 4; o <<= 1) {
                const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
                const float2 s = df_add(make_float2(h, l), make_float2(oh, ol));
                h = s.x;
                l = s.y;
            }
            if (q == 0) prow[base + r] = make_float2(h, l);
        }
        if (tj.x != tj.y) {  // column pass: column c, rows 16 q .. 16 q + 15
            const int c = t & 63, q = t >> 6;
            float h = 0.f, l = 0.f;
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                const int r = 16 * q + m;
                const float2 v = T[r * kSP + c], x = xi[r];
                acc_df(h, l, v.x, v.y, x.x, x.y);
            }
            cpart[q * kSB + c] = make_float2(h, l);
            __syncthreads();
            if (t < kSB) {
                float2 s = cpart[t];
                s = df_add(s, cpart[kSB + t]);
                s = df_add(s, cpart[2 * kSB + t]);
                s = df_add(s, cpart[3 * kSB + t]);
                pcol[base + t] = s;
            }
        }
        __syncthreads();  // buffer cur is refilled in the next iteration
        k = nk;
    }
    cp_async_wait_all();
}

__global__ void __launch_bounds__(kSymThreads) k_symv_df(const float2 *__restrict__ V, int64_t ld, int64_t N, int nb,
                                                         const int2 *__restrict__ tiles, int ntiles,
                                                         const float2 *__restrict__ xdf, float2 *__restrict__ prow,
                                                         float2 *__restrict__ pcol)
{
    extern __shared__ float2 sm[];
    (void)nb;
    symv_tiles(V, ld, N, tiles, ntiles, xdf, prow, pcol, sm, blockIdx.x, gridDim.x);
}

// y_i = sum of the column partials of tiles (J', I), J' < I, then of the row
// partials of tiles (I, J), J >= I (tile (a, b) sits at position
// a nb - a (a - 1) / 2 + (b - a) of the list).  Loads bypass L1 (the partials are
// written by other CTAs of the persistent solver).
__device__ __forceinline__ int64_t tile_pos(int a, int b, int nb)
{
    return (int64_t)a * nb - (int64_t)a * (a - 1) / 2 + (b - a);
}

__device__ __forceinline__ double symv_row(const float2 *__restrict__ prow, const float2 *__restrict__ pcol, int nb,
                                           int64_t i)
{
    // the partials are added in the order J = 0, 1, ..., nb-1; loads are issued 8 at
    // a time so that their L2 latency overlaps
    const int I = (int)(i / kSB), r = (int)(i % kSB);
    float2 s = make_float2(0.f, 0.f);
    int J = 0;
    for (; J + 8 <= I; J += 8) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(pcol + tile_pos(J + u, I, nb) * kSB + r);
#pragma unroll
        for (int u = 0; u < 8; ++u) s = df_add(s, v[u]);
    }
    for (; J < I; ++J) s = df_add(s, __ldcg(pcol + tile_pos(J, I, nb) * kSB + r));
    const int64_t rbase = tile_pos(I, I, nb) * kSB + r;  // tiles (I, J), J >= I, are consecutive
    for (; J + 8 <= nb; J += 8) {
        float2 v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(prow + rbase + (int64_t)(J + u - I) * kSB);
#pragma unroll
        for (int u = 0; u < 8; ++u) s = df_add(s, v[u]);
    }
    for (; J < nb; ++J) s = df_add(s, __ldcg(prow + rbase + (int64_t)(J - I) * kSB));
    return df_to_double(s);
}

// Row i by four consecutive threads (q = 0..3): thread q adds the partials
// J in [q nb/4, (q+1) nb/4) in order, then (q0 + q1) + (q2 + q3); every thread of the
// group returns the row's value.
__device__ __forceinline__ double symv_row4(const float2 *__restrict__ prow, const float2 *__restrict__ pcol, int nb,
                                            int64_t i, int q)
{
    const int I = (int)(i / kSB), r = (int)(i % kSB);
    const int J0 = (q * nb) >> 2, J1 = ((q + 1) * nb) >> 2;
    const int64_t rbase = tile_pos(I, I, nb) * kSB + r;
    float2 s = make_float2(0.f, 0.f);
    int J = J0;
    // 16 partials in flight per thread (L2 round trips, not the adds, bound this pass)
    for (; J + 16 <= J1; J += 16) {
        float2 v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int j = J + u;
            v[u] = j < I ? __ldcg(pcol + tile_pos(j, I, nb) * kSB + r) : __ldcg(prow + rbase + (int64_t)(j - I) * kSB);
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) s = df_add(s, v[u]);
    }
    for (; J + 4 <= J1; J += 4) {
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int j = J + u;
            v[u] = j < I ? __ldcg(pcol + tile_pos(j, I, nb) * kSB + r) : __ldcg(prow + rbase + (int64_t)(j - I) * kSB);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) s = df_add(s, v[u]);
    }
    for (; J < J1; ++J)
        s = df_add(s, J < I ? __ldcg(pcol + tile_pos(J, I, nb) * kSB + r) : __ldcg(prow + rbase + (int64_t)(J - I) * kSB));
    float2 o;
    o.x = __shfl_xor_sync(0xffffffffu, s.x, 1);
    o.y = __shfl_xor_sync(0xffffffffu, s.y, 1);
    s = (q & 1) ? df_add(o, s) : df_add(s, o);
    o.x = __shfl_xor_sync(0xffffffffu, s.x, 2);
    o.y = __shfl_xor_sync(0xffffffffu, s.y, 2);
    s = (q & 2) ? df_add(o, s) : df_add(s, o);
    return df_to_double(s);
}

// Product of the packed FP32 hi parts V_hi with a double-float vector (the
// iteration products of the mixed-precision solver): exact FP32 x FP32 products
// and double-float sums, as the DF64 product but reading 4 instead of 8 bytes per
// entry.  Each warp takes whole tiles from the counter (one 16 KB contiguous
// block per tile); lane l covers columns 4 (l % 16) .. +3 and rows 32 (l / 16) ..
// +31, eight rows per step.  Row partials (V_IJ x_J) are summed over the 16 lanes
// of a row half by a halving butterfly, column partials (V_IJ^T x_I, off the
// diagonal) over the two row halves; both in the DF64 partial layout.
// xsw: 128 pairs of shared memory per warp.
__device__ __forceinline__ int warp_grab(unsigned long long *ctr, unsigned long long base)
{
    int k = 0;
    if ((threadIdx.x & 31) == 0) k = (int)(atomicAdd(ctr, 1ull) - base);
    return __shfl_sync(0xffffffffu, k, 0);
}

// sh + sl += v (xh + xl): acc_df with a single-float matrix entry
__device__ __forceinline__ void acc_hi(float &sh, float &sl, float v, float xh, float xl)
{
    float p, e, s, t;
    two_prod(v, xh, p, e);
    e = __fmaf_rn(v, xl, e);
    two_sum(sh, p, s, t);
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(e, t));
}

__device__ __forceinline__ float2 shfl_df(float2 v, int o)
{
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// static_k >= 0: at most one tile per warp, this one (no counter: when there are no
// more tiles than warps, dynamic grabs only add two L2 atomic round trips)
__device__ void symv_hi_tiles(const float *__restrict__ vp, const int2 *__restrict__ tiles, int ntiles,
                              const float2 *__restrict__ xdf, float2 *__restrict__ prow, float2 *__restrict__ pcol,
                              float2 *xsw, unsigned long long *ctr, unsigned long long base, int static_k = -1)
{
    const int lane = threadIdx.x & 31, cg = lane & 15, par = lane >> 4;
    const bool b1 = lane & 2, b2 = lane & 4, b3 = lane & 8;
    for (int k = static_k >= 0 ? static_k : warp_grab(ctr, base); k < ntiles;
         k = static_k >= 0 ? ntiles : warp_grab(ctr, base)) {
        const int2 tj = tiles[k];
        __syncwarp();
        // x_I in xsw[0..63] (lanes 0..15), x_J in xsw[64..127] (lanes 16..31)
        {
            const float4 *src = reinterpret_cast<const float4 *>(xdf + (int64_t)(par ? tj.y : tj.x) * kSB) + 2 * cg;
            float4 *dst = reinterpret_cast<float4 *>(xsw) + 2 * lane;
            dst[0] = __ldcg(src);
            dst[1] = __ldcg(src + 1);
        }
        __syncwarp();
        float2 xc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xc[u] = xsw[kSB + 4 * cg + u];
        const float4 *T = reinterpret_cast<const float4 *>(vp + (int64_t)k * kTileF);
        float2 cs[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) cs[u] = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int ch = 0; ch < 4; ++ch) {
            const int r0 = 32 * par + 8 * ch;
            float4 v[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) v[m] = __ldcs(T + (r0 + m) * 16 + cg);
            float2 sr[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const float2 xr = xsw[r0 + m];
                const float e[4] = {v[m].x, v[m].y, v[m].z, v[m].w};
                // the row sum starts from the first exact product itself (a two-sum
                // with zero adds nothing)
                float h, l;
                two_prod(e[0], xc[0].x, h, l);
                l = __fmaf_rn(e[0], xc[0].y, l);
#pragma unroll
                for (int u = 1; u < 4; ++u) acc_hi(h, l, e[u], xc[u].x, xc[u].y);
#pragma unroll
                for (int u = 0; u < 4; ++u) acc_hi(cs[u].x, cs[u].y, e[u], xr.x, xr.y);
                sr[m] = make_float2(h, l);
            }
            // rows m of this lane: 8 -> 4 (xor 8) -> 2 (xor 4) -> 1 (xor 2), then xor 1
            // (renormalised there); lane keeps row (l / 2) % 8
            float2 t4[4], t2[2];
#pragma unroll
            for (int j = 0; j < 4; ++j) t4[j] = df_add_u(b3 ? sr[j + 4] : sr[j], shfl_df(b3 ? sr[j] : sr[j + 4], 8));
#pragma unroll
            for (int j = 0; j < 2; ++j) t2[j] = df_add_u(b2 ? t4[j + 2] : t4[j], shfl_df(b2 ? t4[j] : t4[j + 2], 4));
            float2 w = df_add_u(b1 ? t2[1] : t2[0], shfl_df(b1 ? t2[0] : t2[1], 2));
            const float2 o = shfl_df(w, 1);
            w = (lane & 1) ? df_add(o, w) : df_add(w, o);
            if (!(lane & 1)) prow[(int64_t)k * kSB + r0 + ((lane >> 1) & 7)] = w;
        }
        if (tj.x != tj.y) {  // lane keeps columns 4 (l % 16) + 2 (l / 16) + {0, 1}, rows 0..31 first
            const float2 a0 = shfl_df(par ? cs[0] : cs[2], 16), a1 = shfl_df(par ? cs[1] : cs[3], 16);
            float4 out;
            const float2 s0 = par ? df_add(a0, cs[2]) : df_add(cs[0], a0);
            const float2 s1 = par ? df_add(a1, cs[3]) : df_add(cs[1], a1);
            out = make_float4(s0.x, s0.y, s1.x, s1.y);
            reinterpret_cast<float4 *>(pcol + (int64_t)k * kSB)[2 * cg + par] = out;
        }
    }
}

// FP16 working copy of the packed tiles (BEM_PRODUCTS_FP16).  Each 64 x 64 tile is
// stored as halves of its entries divided by a power of two s_k >= max |entry| of the
// tile (exact in FP32, so only the FP16 rounding remains: 2^-11 of the tile's largest
// entry).  One warp per tile: the maximum by a butterfly, then the halves.
__device__ __forceinline__ void pack_h16_tiles(const float *__restrict__ vp, int ntiles, __half *__restrict__ vh,
                                               float *__restrict__ vsc, int64_t w0, int64_t nw)
{
    const int lane = threadIdx.x & 31;
    for (int64_t k = w0; k < ntiles; k += nw) {
        const float4 *T = reinterpret_cast<const float4 *>(vp + k * kTileF);
        float mx = 0.f;
        for (int f = lane; f < kTileF / 4; f += 32) {
            const float4 v = __ldcg(T + f);
            mx = fmaxf(mx, fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fmaxf(fabsf(v.z), fabsf(v.w))));
        }
        for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        int ex = 0;
        if (mx > 0.f) frexpf(mx, &ex);  // mx = m 2^ex, m in [0.5, 1): s = 2^ex > mx
        const float inv = ldexpf(1.f, -ex);
        if (lane == 0) vsc[k] = ldexpf(1.f, ex);
        __half2 *H = reinterpret_cast<__half2 *>(vh + k * kTileF);
        for (int f = lane; f < kTileF / 4; f += 32) {
            const float4 v = __ldcg(T + f);
            H[2 * f] = __floats2half2_rn(v.x * inv, v.y * inv);
            H[2 * f + 1] = __floats2half2_rn(v.z * inv, v.w * inv);
        }
    }
}

__global__ void k_pack_h16(const float *__restrict__ vp, int ntiles, __half *__restrict__ vh, float *__restrict__ vsc)
{
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    pack_h16_tiles(vp, ntiles, vh, vsc, w0, ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// Product with the FP16 working copy: the layout and partials of symv_hi_tiles (lane
// l: columns 4 (l % 16) .. +3, rows 32 (l / 16) + 8 c .. +7 in step c), 8 bytes per
// lane and row, FP32 products of the half entries with the hi part of x and FP32
// sums; the tile's scale multiplies its partials.  The iteration products of
// BEM_PRODUCTS_FP16 only: the residuals that decide convergence use the exact form.
__device__ void symv_h16_tiles(const __half *__restrict__ vh, const float *__restrict__ vsc,
                               const int2 *__restrict__ tiles, int ntiles, const float2 *__restrict__ xdf,
                               float2 *__restrict__ prow, float2 *__restrict__ pcol, float2 *xsw,
                               unsigned long long *ctr, unsigned long long base, int static_k = -1)
{
    const int lane = threadIdx.x & 31, cg = lane & 15, par = lane >> 4;
    const bool b1 = lane & 2, b2 = lane & 4, b3 = lane & 8;
    for (int k = static_k >= 0 ? static_k : warp_grab(ctr, base); k < ntiles;
         k = static_k >= 0 ? ntiles : warp_grab(ctr, base)) {
        const int2 tj = tiles[k];
        const float sk = vsc[k];
        __syncwarp();
        {
            const float4 *src = reinterpret_cast<const float4 *>(xdf + (int64_t)(par ? tj.y : tj.x) * kSB) + 2 * cg;
            float4 *dst = reinterpret_cast<float4 *>(xsw) + 2 * lane;
            dst[0] = __ldcg(src);
            dst[1] = __ldcg(src + 1);
        }
        __syncwarp();
        float xc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) xc[u] = xsw[kSB + 4 * cg + u].x;
        const uint2 *T = reinterpret_cast<const uint2 *>(vh + (int64_t)k * kTileF);
        float cs[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
        for (int ch = 0; ch < 4; ++ch) {
            const int r0 = 32 * par + 8 * ch;
            uint2 raw[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) raw[m] = __ldcs(T + (r0 + m) * 16 + cg);
            float sr[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const float xr = xsw[r0 + m].x;
                __half2 h01, h23;
                memcpy(&h01, &raw[m].x, 4);
                memcpy(&h23, &raw[m].y, 4);
                const float2 a01 = __half22float2(h01), a23 = __half22float2(h23);
                const float e[4] = {a01.x, a01.y, a23.x, a23.y};
                float h = e[0] * xc[0];
#pragma unroll
                for (int u = 1; u < 4; ++u) h = __fmaf_rn(e[u], xc[u], h);
                sr[m] = h;
#pragma unroll
                for (int u = 0; u < 4; ++u) cs[u] = __fmaf_rn(e[u], xr, cs[u]);
            }
            // rows m: 8 -> 4 (xor 8) -> 2 (xor 4) -> 1 (xor 2), then xor 1
            float t4[4], t2[2];
#pragma unroll
            for (int j = 0; j < 4; ++j)
                t4[j] = (b3 ? sr[j + 4] : sr[j]) + __shfl_xor_sync(0xffffffffu, b3 ? sr[j] : sr[j + 4], 8);
#pragma unroll
            for (int j = 0; j < 2; ++j)
                t2[j] = (b2 ? t4[j + 2] : t4[j]) + __shfl_xor_sync(0xffffffffu, b2 ? t4[j] : t4[j + 2], 4);
            float w = (b1 ? t2[1] : t2[0]) + __shfl_xor_sync(0xffffffffu, b1 ? t2[0] : t2[1], 2);
            w += __shfl_xor_sync(0xffffffffu, w, 1);
            if (!(lane & 1)) prow[(int64_t)k * kSB + r0 + ((lane >> 1) & 7)] = make_float2(w * sk, 0.f);
        }
        if (tj.x != tj.y) {  // lane keeps columns 4 (l % 16) + 2 (l / 16) + {0, 1}
            const float a0 = __shfl_xor_sync(0xffffffffu, par ? cs[0] : cs[2], 16);
            const float a1 = __shfl_xor_sync(0xffffffffu, par ? cs[1] : cs[3], 16);
            const float s0 = (par ? cs[2] : cs[0]) + a0, s1 = (par ? cs[3] : cs[1]) + a1;
            reinterpret_cast<float4 *>(pcol + (int64_t)k * kSB)[2 * cg + par] = make_float4(s0 * sk, 0.f, s1 * sk, 0.f);
        }
    }
}

// y = reduction of the tile partials; optional block partials of sum w_i y_i.
__global__ void k_symv_reduce(const float2 *__restrict__ prow, const float2 *__restrict__ pcol, int nb, int64_t N,
                              double *__restrict__ y, const double *__restrict__ w, double *dot_partial)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < N) {
        v = symv_row(prow, pcol, nb, i);
        y[i] = v;
    }
    if (dot_partial) block_partial(i < N ? w[i] * v : 0.0, dot_partial);
}

__global__ void k_tile_list(int nb, int2 *tiles)
{
    const int I = blockIdx.x;
    for (int J = I + threadIdx.x; J < nb; J += blockDim.x) tiles[tile_pos(I, J, nb)] = make_int2(I, J);
}

// x (FP64, N) -> hi/lo pairs, zero-padded to ld
__global__ void k_to_df(const double *x, int64_t N, int64_t ld, float2 *xdf)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ld) xdf[i] = i < N ? df_from_double(x[i]) : make_float2(0.0f, 0.0f);
}

// r = b - q; z = M^-1 r; p = z; partials of r.z, r.r, b.b
__global__ void k_pcg_init(int64_t N, const double *b, const double *q, const double *d, int precond,
                           double *r, double *z, double *p, double *prz, double *prr, double *pbb)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rz = 0.0, rr = 0.0, bb = 0.0;
    if (i < N) {
        const double ri = b[i] - q[i];
        const double zi = precond ? ri / d[i] : ri;
        r[i] = ri;
        z[i] = zi;
        p[i] = zi;
        rz = ri * zi;
        rr = ri * ri;
        bb = b[i] * b[i];
    }
    block_partial(rz, prz);
    block_partial(rr, prr);
    block_partial(bb, pbb);
}

// alpha = rz / p.q; x += alpha p; r -= alpha q; z = M^-1 r; partials of r.z, r.r
__global__ void k_pcg_update1(int64_t N, const double *ppq, int npq, const double *rz_old, double *x,
                              double *r, double *z, const double *p, const double *q, const double *d,
                              int precond, double *prz, double *prr)
{
    const double pq = sum_partials(ppq, npq);
    const double alpha = *rz_old / pq;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double rz = 0.0, rr = 0.0;
    if (i < N) {
        x[i] += alpha * p[i];
        const double ri = r[i] - alpha * q[i];
        const double zi = precond ? ri / d[i] : ri;
        r[i] = ri;
        z[i] = zi;
        rz = ri * zi;
        rr = ri * ri;
    }
    block_partial(rz, prz);
    block_partial(rr, prr);
}

// beta = rz_new / rz_old; p = z + beta p; block 0 stores rz_new and r.r
__global__ void k_pcg_update2(int64_t N, const double *prz, const double *prr, int nparts,
                              const double *rz_old, double *rz_new, double *rr_out, const double *z, double *p)
{
    const double rz = sum_partials(prz, nparts);
    const double rr = sum_partials(prr, nparts);
    const double beta = rz / *rz_old;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) p[i] = z[i] + beta * p[i];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *rz_new = rz;
        *rr_out = rr;
    }
}

// out[0] = sum of partials a, out[1] = sum b, out[2] = sum c (one block).
__global__ void k_reduce3(const double *a, const double *b, const double *c, int n, double *out)
{
    const double sa = sum_partials(a, n);
    const double sb = b ? sum_partials(b, n) : 0.0;
    const double sc = c ? sum_partials(c, n) : 0.0;
    if (threadIdx.x == 0) {
        out[0] = sa;
        out[1] = sb;
        out[2] = sc;
    }
}

// partials of sum_i u_i v_i
__global__ void k_dot_partial(int64_t N, const double *u, const double *v, double *part)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    block_partial(i < N ? u[i] * v[i] : 0.0, part);
}

__global__ void k_axpy(int64_t N, double a, const double *x, double *y)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) y[i] += a * x[i];
}

// r = b - q, partials of r.r
__global__ void k_residual(int64_t N, const double *b, const double *q, double *r, double *prr)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < N) {
        v = b[i] - q[i];
        r[i] = v;
    }
    block_partial(v * v, prr);
}

// ------------------------------------------------------------------ block-Jacobi clusters
// Spatial clusters of kBJ triangles: Morton order of the centroids (10 bits per axis
// over the bounding box of the centroids, ties by index), cut into consecutive
// groups; the preconditioner is the block diagonal of V over the clusters, each block
// inverted in FP64 (Cholesky, inverse of the factor, Gram product: symmetric positive
// definite by construction).
constexpr int kBJ = 64;

// Bounding box of the centroids: per-CTA min/max (part: gridDim.x x 6), then one
// CTA folds the partials (min and max are exact, so the order does not matter).
__global__ void __launch_bounds__(256) k_cent_box(const double *cent, int64_t N, double *part)
{
    __shared__ double s[6][256];
    double v[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        for (int c = 0; c < 3; ++c) {
            const double x = cent[4 * i + c];
            v[c] = fmin(v[c], x);
            v[3 + c] = fmax(v[3 + c], x);
        }
    for (int c = 0; c < 6; ++c) s[c][threadIdx.x] = v[c];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int c = 0; c < 6; ++c)
                s[c][threadIdx.x] = c < 3 ? fmin(s[c][threadIdx.x], s[c][threadIdx.x + w])
                                          : fmax(s[c][threadIdx.x], s[c][threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void k_box_fold(const double *part, int nparts, double *box)
{
    const int c = threadIdx.x;
    if (c >= 6) return;
    double r = part[c];
    for (int k = 1; k < nparts; ++k) r = c < 3 ? fmin(r, part[6 * k + c]) : fmax(r, part[6 * k + c]);
    box[c] = r;
}

__device__ __forceinline__ unsigned spread3(unsigned q)  // bit b of q -> bit 3b
{
    unsigned r = 0;
    for (int b = 0; b < 10; ++b) r |= ((q >> b) & 1u) << (3 * b);
    return r;
}

__global__ void k_morton_keys(const double *cent, int64_t N, int64_t n2, const double *box,
                              unsigned long long *keys)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    if (i >= N) {
        keys[i] = ~0ull;
        return;
    }
    unsigned code = 0;
    for (int c = 0; c < 3; ++c) {
        const double lo = box[c], ext = __dsub_rn(box[3 + c], lo);
        const double sc = ext > 0.0 ? __ddiv_rn(1023.0, ext) : 0.0;
        double t = __dmul_rn(__dsub_rn(cent[4 * i + c], lo), sc);
        t = t < 0.0 ? 0.0 : (t > 1023.0 ? 1023.0 : t);
        code |= spread3((unsigned)t) << c;
    }
    keys[i] = ((unsigned long long)code << 32) | (unsigned long long)(uint32_t)i;
}

__global__ void k_cluster_perm(const unsigned long long *keys, int64_t N, int64_t nperm, int32_t *perm)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < nperm) perm[k] = k < N ? (int32_t)(keys[k] & 0xFFFFFFFFull) : -1;
}

__device__ __forceinline__ double elem_f64(const double *V, int64_t o) { return V[o]; }
__device__ __forceinline__ double elem_f64(const float2 *V, int64_t o) { return (double)V[o].x + (double)V[o].y; }
__device__ __forceinline__ double elem_f64(const float *V, int64_t o) { return (double)V[o]; }

// One CTA per cluster block.  A = V[perm, perm] (identity on padding) is scaled to
// unit diagonal, S A S with S = diag(A)^-1/2 (FP64), factored A = L L^T in FP32,
// L^-1 formed column by column in FP32, and M^-1 = S L^-T L^-1 S with the Gram sums
// taken in double-float (exact FP32 products): symmetric (upper triangle formed,
// mirrored) and positive definite for any nonsingular L, whatever the FP32 rounding
// of L.  The discrete V is not positive definite everywhere (on strongly graded
// meshes the fixed 7 x 7 rule for close disjoint pairs leaves some diagonal blocks
// with a non-positive eigenvalue); a block whose factorisation meets a pivot <= 0
// is replaced by its diagonal, so that M stays symmetric positive definite.
template <typename T>
__device__ __forceinline__ void block_inverse_body(const T *__restrict__ V, int64_t ld,
                                                   const int32_t *__restrict__ perm, double *__restrict__ binv,
                                                   int64_t blk)
{
    __shared__ float A[kBJ][kBJ + 1];
    __shared__ float B[kBJ][kBJ + 1];
    __shared__ double sc[kBJ], d0[kBJ];
    __shared__ int32_t pk[kBJ];  // the cluster's rows, read once
    __shared__ int s_fail;
    const int t = threadIdx.x;
    if (t == 0) s_fail = 0;
    if (t < kBJ) pk[t] = perm[blk * kBJ + t];
    __syncthreads();
    if (t < kBJ) {
        const int32_t g = pk[t];
        const double d = g >= 0 ? elem_f64(V, (int64_t)g * ld + g) : 1.0;
        d0[t] = d;
        if (!(d > 0.0)) s_fail = 1;
        sc[t] = d > 0.0 ? 1.0 / sqrt(d) : 1.0;
    }
    __syncthreads();
    // 16 entries per thread (blockDim.x = 256), their scattered reads issued together
    constexpr int kPer = kBJ * kBJ / 256;
    double av[kPer];
#pragma unroll
    for (int m = 0; m < kPer; ++m) {
        const int idx = t + 256 * m, i = idx / kBJ, j = idx % kBJ;
        const int32_t gi = pk[i], gj = pk[j];
        // upper-triangle read: V (i, j) for i <= j (batch operators mirror only their
        // diagonal blocks; mirrored entries are bit-identical copies)
        const int64_t lo = gi < gj ? gi : gj, hi = gi < gj ? gj : gi;
        av[m] = (gi >= 0 && gj >= 0) ? elem_f64(V, lo * ld + hi) : (i == j ? 1.0 : 0.0);
    }
#pragma unroll
    for (int m = 0; m < kPer; ++m) {
        const int idx = t + 256 * m, i = idx / kBJ, j = idx % kBJ;
        A[i][j] = (float)(av[m] * sc[i] * sc[j]);
    }
    __syncthreads();
    const int ri = t >> 2, rc = t & 3;  // trailing update: row ri, columns rc + 4 m
    __shared__ float dg[kBJ];
    for (int k = 0; k < kBJ; ++k) {
        // every thread that scales column k takes the pivot itself (nothing writes A[k][k]
        // during step k; the factor's diagonal is stored after the loop), so the step
        // needs two barriers, not three
        // the pivot's reciprocal square root scales the column (a multiplication instead
        // of a division per entry); the factor's diagonal is d times it
        const float d = A[k][k];
        const float rk = d > 0.f ? rsqrtf(d) : 1.f;
        if (t == 0) {
            if (!(d > 0.f)) s_fail = 1;
            dg[k] = d > 0.f ? d * rk : 1.f;
        }
        if (t > k && t < kBJ) A[t][k] *= rk;
        __syncthreads();
        if (ri > k) {
            // the row's entries and the column's, read before any is written (no shared
            // load waits on a store of this thread)
            const float lik = A[ri][k];
            float aj[kBJ / 4], cj[kBJ / 4];
#pragma unroll
            for (int m = 0; m < kBJ / 4; ++m) {
                const int j = k + 1 + rc + 4 * m;
                if (j <= ri) {
                    aj[m] = A[j][k];
                    cj[m] = A[ri][j];
                }
            }
#pragma unroll
            for (int m = 0; m < kBJ / 4; ++m) {
                const int j = k + 1 + rc + 4 * m;
                if (j <= ri) A[ri][j] = cj[m] - lik * aj[m];
            }
        }
        __syncthreads();
    }
    if (t < kBJ) A[t][t] = dg[t];
    __syncthreads();
    double *out = binv + blk * kBJ * kBJ;
    if (s_fail) {  // diagonal block (Jacobi)
        for (int idx = t; idx < kBJ * kBJ; idx += blockDim.x) {
            const int i = idx / kBJ, j = idx % kBJ;
            out[idx] = i == j ? 1.0 / d0[i] : 0.0;
        }
        return;
    }
    if (t < kBJ) {  // column t of L^-1 (lower), forward substitution
        // four partial sums over k (c + 4 q + r), so that four shared loads and FMAs are
        // in flight instead of one dependent chain; (s0 + s1) + (s2 + s3) at the end
        const int c = t;
        for (int i = 0; i < kBJ; ++i) {
            float v = 0.f;
            if (i >= c) {
                float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
                int k = c;
                for (; k + 4 <= i; k += 4) {
                    s0 = __fmaf_rn(A[i][k], B[k][c], s0);
                    s1 = __fmaf_rn(A[i][k + 1], B[k + 1][c], s1);
                    s2 = __fmaf_rn(A[i][k + 2], B[k + 2][c], s2);
                    s3 = __fmaf_rn(A[i][k + 3], B[k + 3][c], s3);
                }
                if (k < i) s0 = __fmaf_rn(A[i][k], B[k][c], s0);
                if (k + 1 < i) s1 = __fmaf_rn(A[i][k + 1], B[k + 1][c], s1);
                if (k + 2 < i) s2 = __fmaf_rn(A[i][k + 2], B[k + 2][c], s2);
                v = ((i == c ? 1.f : 0.f) - ((s0 + s1) + (s2 + s3))) / A[i][i];
            }
            B[i][c] = v;
        }
    }
    __syncthreads();
    for (int idx = t; idx < kBJ * kBJ; idx += blockDim.x) {
        const int i = idx / kBJ, j = idx % kBJ;
        if (i > j) continue;
        float h = 0.f, l = 0.f;
        for (int k = j; k < kBJ; ++k) acc_hi(h, l, B[k][i], B[k][j], 0.f);
        const double v = ((double)h + (double)l) * sc[i] * sc[j];
        out[i * kBJ + j] = v;
        out[j * kBJ + i] = v;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_block_inverse(const T *__restrict__ V, int64_t ld,
                                                       const int32_t *__restrict__ perm, double *__restrict__ binv)
{
    block_inverse_body<T>(V, ld, perm, binv, blockIdx.x);
}

// z = M^-1 r on the rows of cluster blk, by one CTA.  Thread t < 64 handles row t of
// the cluster: with update, x += alpha p and r -= alpha q first; r is staged in rs
// (64 doubles of shared memory).  Then 4 threads per row (t = 4 i + c) add 16
// products each and combine them by shuffles ((c0 + c1) + (c2 + c3)).  init: also
// p = z and pdf = z in double-float.  Adds the cluster's r.z and r.r to the thread's
// partials.
__device__ __forceinline__ void block_apply(const int32_t *__restrict__ perm, const double *__restrict__ binv, int blk,
                                            double *x, double *r, double *z, double *p, const double *q,
                                            float2 *pdf, double alpha, bool update, bool init, double *rs,
                                            double &rz_l, double &rr_l)
{
    const int t = threadIdx.x;
    const int32_t *pk = perm + (int64_t)blk * kBJ;
    // this thread's row slice of the inverse block, loaded first: it does not depend
    // on r, so its latency overlaps the gather below
    const int i = t >> 2, c = t & 3;
    const double2 *Mi = reinterpret_cast<const double2 *>(binv + (int64_t)blk * kBJ * kBJ + i * kBJ + 16 * c);
    double2 m[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) m[u] = Mi[u];
    if (t < kBJ) {
        const int32_t g = pk[t];
        double v = 0.0;
        if (g >= 0) {
            if (update) {
                x[g] += alpha * p[g];
                v = r[g] - alpha * q[g];
                r[g] = v;
            } else {
                v = r[g];
            }
        }
        rs[t] = v;
    }
    __syncthreads();
    double sacc = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        sacc += m[u].x * rs[16 * c + 2 * u];
        sacc += m[u].y * rs[16 * c + 2 * u + 1];
    }
    sacc += __shfl_xor_sync(0xffffffffu, sacc, 1);
    sacc += __shfl_xor_sync(0xffffffffu, sacc, 2);
    if (c == 0) {
        const int32_t g = pk[i];
        if (g >= 0) {
            const double rv = rs[i];
            z[g] = sacc;
            if (init) {
                p[g] = sacc;
                pdf[g] = df_from_double(sacc);
            }
            rz_l += rv * sacc;
            rr_l += rv * rv;
        }
    }
    __syncthreads();  // rs is refilled for the next cluster
}

// Packed upper triangle of an FP32 operator: tile k of the list, row-major 64 x 64 at
// vp + 4096 k (rows past N zero; columns past N are the operator's zero padding).
__global__ void k_pack_f32(const float *__restrict__ V, int64_t ld, int64_t N, const int2 *__restrict__ tiles,
                           int64_t ntiles, float *__restrict__ vp)
{
    const int64_t n4 = ntiles * (kTileF / 4);
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < n4; f += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = f / (kTileF / 4);
        const int e = (int)(f % (kTileF / 4)), r = e >> 4, c4 = e & 15;
        const int2 tj = tiles[k];
        const int64_t row = (int64_t)tj.x * kSB + r;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < N) v = __ldcs(reinterpret_cast<const float4 *>(V + row * ld + (int64_t)tj.y * kSB) + c4);
        reinterpret_cast<float4 *>(vp)[f] = v;
    }
}

// ------------------------------------------------------------------ persistent DF64 solver
// The whole Jacobi-PCG of a DF64 operator in one cooperative launch: every CTA
// takes part in the tile loop of the symmetric product, then owns rows
// cta*256 + t + k*G*256 for the vector updates; global sums are fixed-order sums
// of per-CTA partials that every CTA evaluates identically, so all CTAs take the
// same convergence decision.  CTAs meet at a grid barrier whose wait is bounded
// (about 1.7 s): on time-out it raises err and the kernel returns.
struct PcgArgs {
    const float2 *V;
    int64_t ld, N;
    int nb, ntiles;
    const int2 *tiles;
    float2 *prow, *pcol, *pdf;
    double *x, *r, *z, *p, *q;
    const double *d, *b;
    double *part;             // 3 x G per-CTA partials
    unsigned *bar;            // [0] grid-barrier arrival counter (zero at launch)
    unsigned long long *ctr;  // tile counter (never decreases)
    int *err;
    double *out;              // [0] r.r, [1] b.b, [2] iterations, [3] DF64 residuals
    float *vp;                // packed FP32 hi parts of the tiles (mixed mode), else null
    const int32_t *bperm;     // block preconditioner: cluster order (nbj x kBJ, -1 padding)
    const double *binv;       // block preconditioner: inverse blocks (nbj x kBJ x kBJ)
    double tol, delta2;
    int max_it, precond, has_x0, nbj;
    int f32op;                // FP32 operator: every product (residuals too) from vp
    double *lanczos;          // nullable: (alpha_j, beta_j) of iteration j < lanczos_cap
    int lanczos_cap;
    // inexact stopping (Remark (i) after Alg. 1): stop once the energy norm of the
    // update satisfies |||x_k - x_(k-1)|||^2 <= lam2 * eta^2(x_k), eta the ZZ estimator
    // of the iterate (Eq. 1.6, primal P0 reading); lam2 = 0: off
    double lam2;
    const int32_t *tris, *v2t_off, *v2t;
    const double *area, *hdiam;  // hdiam: diam(T), or null for h_T = |T|^1/2
    double *u;                   // M nodal values
    int64_t M;
    // operator preconditioning (Sec. 2.6): packed FP32 upper triangle of the
    // preconditioner C = S D^reg S (the tiles of vp)
    const float *dvp;
    long long bar_limit_ns;   // grid-barrier wait limit (ns)
    int absent_cta;           // failure-detection tests: this CTA leaves at its first barrier (-1: none)
    // BEM_PRODUCTS_FP16: the FP16 working copy of the packed tiles and their scales
    // (null: off).  FP32 operators: packed by the host before the launch; DF64: by
    // the kernel from its packed hi parts after the first product.
    __half *vh;
    float *vsc;
    double *n16_out;          // nullable: iterations that used the FP16 copy
};

// Per-CTA partial of one value per thread (fixed tree) into slot[cta].
__device__ __forceinline__ void cta_partial(double v, double *slot, int cta)
{
    __shared__ double sw[kSymThreads / 32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sw[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kSymThreads / 32; ++k) t += sw[k];
        slot[cta] = t;
    }
    __syncthreads();
}

// Two values at once, each summed exactly as cta_partial sums it.
__device__ __forceinline__ void cta_partial2(double v1, double v2, double *slot1, double *slot2, int cta)
{
    __shared__ double sw1[kSymThreads / 32], sw2[kSymThreads / 32];
    v1 = warp_sum(v1);
    v2 = warp_sum(v2);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sw1[w] = v1;
        sw2[w] = v2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < kSymThreads / 32; ++k) {
            t1 += sw1[k];
            t2 += sw2[k];
        }
        slot1[cta] = t1;
        slot2[cta] = t2;
    }
    __syncthreads();
}

// Fixed-order sum of the G per-CTA partials (L2 loads: written by other CTAs).
__device__ __forceinline__ double grid_total(const double *slot, int G)
{
    __shared__ double sw[kSymThreads / 32];
    __shared__ double res;
    double v = 0.0;
    for (int k = threadIdx.x; k < G; k += blockDim.x) v += __ldcg(slot + k);
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sw[w] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < kSymThreads / 32; ++k) t += sw[k];
        res = t;
    }
    __syncthreads();
    return res;
}

// Two totals at once, each summed exactly as grid_total sums it.
__device__ __forceinline__ void grid_total2(const double *slot1, const double *slot2, int G, double &r1, double &r2)
{
    __shared__ double sw1[kSymThreads / 32], sw2[kSymThreads / 32];
    __shared__ double res1, res2;
    double v1 = 0.0, v2 = 0.0;
    for (int k = threadIdx.x; k < G; k += blockDim.x) {
        v1 += __ldcg(slot1 + k);
        v2 += __ldcg(slot2 + k);
    }
    v1 = warp_sum(v1);
    v2 = warp_sum(v2);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) {
        sw1[w] = v1;
        sw2[w] = v2;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t1 = 0.0, t2 = 0.0;
        for (int k = 0; k < kSymThreads / 32; ++k) {
            t1 += sw1[k];
            t2 += sw2[k];
        }
        res1 = t1;
        res2 = t2;
    }
    __syncthreads();
    r1 = res1;
    r2 = res2;
}

// kCal: the build with the operator preconditioner (BEM_PRECOND_CALDERON), kept out of
// the other solvers' kernels (its Chebyshev and D^reg phases cost registers).
template <bool kCal>
__device__ __forceinline__ void pcg_body(const PcgArgs &a, const int G, const int cta)
{
    extern __shared__ float2 sm[];
    const int64_t stride = (int64_t)G * kSymThreads;
    const int64_t i0 = (int64_t)cta * kSymThreads + threadIdx.x;
    double *pA = a.part, *pB = a.part + G, *pC = a.part + 2 * G;
    const bool mixed = a.vp != nullptr;
    const bool blockpc = a.precond == BEM_PRECOND_BLOCK, jacobi = a.precond == BEM_PRECOND_JACOBI;
    const bool calpc = kCal && a.precond == BEM_PRECOND_CALDERON;
    const bool zlocal = !blockpc && !calpc;  // z_i from r_i alone
    float2 *const xsw = sm + (threadIdx.x >> 5) * 2 * kSB;
    __shared__ double rs[kBJ];
    const int lane = threadIdx.x & 31, q4 = lane & 3;
    const int64_t warp_g = ((int64_t)cta * kSymThreads + threadIdx.x) >> 5, nwarps = stride >> 5;
    unsigned long long tbase = 0ull;
    GridBar gb{a.bar, a.err, 0u, a.bar_limit_ns > 0 ? a.bar_limit_ns : kBarrierLimitNs, a.absent_cta == cta};
    // packed products: tiles taken statically when every warp gets one at most
    const int hi_static = a.ntiles <= nwarps ? (int)warp_g : -1;
    auto hi_product = [&](const float *packed) {
        symv_hi_tiles(packed, a.tiles, a.ntiles, a.pdf, a.prow, a.pcol, xsw, a.ctr, tbase, hi_static);
        if (hi_static < 0) tbase += (unsigned long long)(a.ntiles + G * (kSymThreads / 32));
    };
    // DF64 product V x into the tile partials (x = the FP64 iterate); the first one
    // of the mixed mode also packs the hi parts
    auto df64_product = [&](bool pack) -> bool {
        for (int64_t i = i0; i < a.ld; i += stride) a.pdf[i] = i < a.N ? df_from_double(a.x[i]) : make_float2(0.f, 0.f);
        if (!grid_barrier(gb, G)) return false;
        if (a.f32op) {  // the stored operator is the packed copy itself
            hi_product(a.vp);
        } else {
            symv_tiles(a.V, a.ld, a.N, a.tiles, a.ntiles, a.pdf, a.prow, a.pcol, sm, cta, G, a.ctr, tbase,
                       pack ? a.vp : nullptr);
            tbase += (unsigned long long)(a.ntiles + G);
        }
        return grid_barrier(gb, G);
    };
    // z = C r (operator preconditioning, Sec. 2.6): the product with the packed FP32 C
    // (exact products, double-float sums); its row pass also forms the partial of r.z,
    // and with init p = z
    auto calderon = [&](bool init, double &rz_part) -> bool {
        for (int64_t i = i0; i < a.ld; i += stride) a.pdf[i] = i < a.N ? df_from_double(a.r[i]) : make_float2(0.f, 0.f);
        if (!grid_barrier(gb, G)) return false;
        hi_product(a.dvp);
        if (!grid_barrier(gb, G)) return false;
        for (int64_t ib = warp_g * 8; ib < a.N; ib += nwarps * 8) {
            const int64_t i = ib + (lane >> 2);
            const bool valid = i < a.N;
            const double zi = symv_row4(a.prow, a.pcol, a.nb, valid ? i : a.N - 1, q4);
            if (valid && q4 == 0) {
                a.z[i] = zi;
                rz_part += __ldcg(a.r + i) * zi;  // r of other threads' rows: L2
                if (init) {
                    a.p[i] = zi;
                    a.pdf[i] = df_from_double(zi);
                }
            }
        }
        return true;
    };
    // r = b - V x0 (or b), z = M^-1 r, p = z
    const bool prod0 = a.has_x0 || mixed;
    if (prod0 && !df64_product(mixed)) return;
    // FP16 iteration products (mixed mode): residuals replaced after every 10^2-fold
    // drop of ||r||; back to the exact products for good if a replacement finds that
    // the true residual fell by less than 10x since the previous one
    bool use16 = mixed && a.vh != nullptr && !calpc;
    if (use16 && !a.f32op) {  // the halves of the hi parts packed by the first product
        pack_h16_tiles(a.vp, a.ntiles, a.vh, a.vsc, warp_g, nwarps);
        if (!grid_barrier(gb, G)) return;
    }
    int n16 = 0, seg = 0;
    double rz_l = 0.0, rr_l = 0.0, bb_l = 0.0;
    for (int64_t i = i0; i < a.ld; i += stride) {
        if (i < a.N) {
            const double ri = a.b[i] - (a.has_x0 ? symv_row(a.prow, a.pcol, a.nb, i) : 0.0);
            a.r[i] = ri;
            bb_l += a.b[i] * a.b[i];
            if (zlocal) {
                const double zi = jacobi ? ri / a.d[i] : ri;
                a.z[i] = zi;
                a.p[i] = zi;
                a.pdf[i] = df_from_double(zi);
                rz_l += ri * zi;
                rr_l += ri * ri;
            }
        } else {
            a.pdf[i] = make_float2(0.f, 0.f);
        }
    }
    if (blockpc) {  // z = M^-1 r over whole clusters: every r written first
        if (!grid_barrier(gb, G)) return;
        for (int blk = cta; blk < a.nbj; blk += G)
            block_apply(a.bperm, a.binv, blk, a.x, a.r, a.z, a.p, a.q, a.pdf, 0.0, false, true, rs, rz_l, rr_l);
    }
    if (calpc) {  // r.r of this thread's rows, then z = C r (r written by its own rows)
        for (int64_t i = i0; i < a.N; i += stride) rr_l += a.r[i] * a.r[i];
        if (!calderon(true, rz_l)) return;
    }
    cta_partial(rz_l, pA, cta);
    cta_partial(rr_l, pB, cta);
    cta_partial(bb_l, pC, cta);
    if (!grid_barrier(gb, G)) return;
    double rz = grid_total(pA, G), rr = grid_total(pB, G);
    const double bb = grid_total(pC, G);
    const double thr = a.tol * a.tol * (bb > 0.0 ? bb : 1.0);
    double rr_true = rr;  // r.r at the last residual formed with the DF64 product
    double rr_true_prev = rr;
    int it = 0, ndf = prod0 ? 1 : 0, inexact_stop = 0;
    if (!grid_barrier(gb, G)) return;  // partial slots are reused below
    while (!(rr <= thr) && it < a.max_it) {
        double alpha, rz_new, rz_n = 0.0;
        if (use16) {
            symv_h16_tiles(a.vh, a.vsc, a.tiles, a.ntiles, a.pdf, a.prow, a.pcol, xsw, a.ctr, tbase, hi_static);
            if (hi_static < 0) tbase += (unsigned long long)(a.ntiles + G * (kSymThreads / 32));
            ++n16;
        } else if (mixed) {
            hi_product(a.vp);
        } else {
            symv_tiles(a.V, a.ld, a.N, a.tiles, a.ntiles, a.pdf, a.prow, a.pcol, sm, cta, G, a.ctr, tbase);
            tbase += (unsigned long long)(a.ntiles + G);
        }
        if (!grid_barrier(gb, G)) return;
        double pq_l = 0.0;
        // 8 rows per warp and pass, 4 threads per row; the loop is uniform across the
        // warp (rows past N recompute row N-1 and are discarded) because the row sum
        // combines the 4 threads with shuffles
        for (int64_t ib = warp_g * 8; ib < a.N; ib += nwarps * 8) {
            const int64_t i = ib + (lane >> 2);
            const bool valid = i < a.N;
            const int64_t ic = valid ? i : a.N - 1;
            const double qi = symv_row4(a.prow, a.pcol, a.nb, ic, q4);
            if (valid && q4 == 0) {
                a.q[i] = qi;
                pq_l += a.p[i] * qi;
            }
        }
        cta_partial(pq_l, pA, cta);
        if (!grid_barrier(gb, G)) return;
        alpha = rz / grid_total(pA, G);
        rr_l = 0.0;
        if (blockpc) {
            for (int blk = cta; blk < a.nbj; blk += G)
                block_apply(a.bperm, a.binv, blk, a.x, a.r, a.z, a.p, a.q, a.pdf, alpha, true, false, rs, rz_n, rr_l);
        } else if (calpc) {
            for (int64_t i = i0; i < a.N; i += stride) {
                a.x[i] += alpha * a.p[i];
                const double ri = a.r[i] - alpha * a.q[i];
                a.r[i] = ri;
                rr_l += ri * ri;
            }
            if (!calderon(false, rz_n)) return;
        } else {
            for (int64_t i = i0; i < a.N; i += stride) {
                a.x[i] += alpha * a.p[i];
                const double ri = a.r[i] - alpha * a.q[i];
                const double zi = jacobi ? ri / a.d[i] : ri;
                a.r[i] = ri;
                a.z[i] = zi;
                rz_n += ri * zi;
                rr_l += ri * ri;
            }
        }
        cta_partial2(rz_n, rr_l, pB, pC, cta);
        if (!grid_barrier(gb, G)) return;
        grid_total2(pB, pC, G, rz_new, rr);
        ++it;
        if (a.lam2 > 0.0) {
            // |||alpha p|||^2 = alpha^2 p.Vp = alpha (r.z); ZZ estimator of the iterate
            const double upd2 = alpha * rz;
            for (int64_t z = i0; z < a.M; z += stride) {
                double num = 0.0, den = 0.0;
                for (int32_t q = a.v2t_off[z]; q < a.v2t_off[z + 1]; ++q) {
                    const int32_t t = a.v2t[q];
                    num += a.area[t] * __ldcg(a.x + t);  // x of other CTAs' rows: L2
                    den += a.area[t];
                }
                a.u[z] = den > 0.0 ? num / den : 0.0;
            }
            if (!grid_barrier(gb, G)) return;
            double el = 0.0;
            for (int64_t t = i0; t < a.N; t += stride) {
                double d[3];
                for (int k = 0; k < 3; ++k) d[k] = __ldcg(a.u + a.tris[3 * t + k]) - a.x[t];
                const double s2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
                const double s1 = (d[0] + d[1]) + d[2];
                const double h = a.hdiam ? a.hdiam[t] : sqrt(a.area[t]);
                el += (h * a.area[t]) / 12.0 * (s2 + s1 * s1);
            }
            cta_partial(el, pA, cta);
            if (!grid_barrier(gb, G)) return;
            if (upd2 <= a.lam2 * grid_total(pA, G)) {
                inexact_stop = 1;
                break;
            }
        }
        ++seg;
        if (mixed && (rr <= (use16 ? kH16Delta2 : a.delta2) * rr_true || rr <= thr || (use16 && seg >= kH16SegMax))) {
            seg = 0;
            // reliable update: replace the recursive residual by b - V x with the
            // DF64 product (the direction p is kept)
            if (!df64_product(false)) return;
            rz_n = 0.0;
            rr_l = 0.0;
            for (int64_t ib = warp_g * 8; ib < a.N; ib += nwarps * 8) {
                const int64_t i = ib + (lane >> 2);
                const bool valid = i < a.N;
                const double vi = symv_row4(a.prow, a.pcol, a.nb, valid ? i : a.N - 1, q4);
                if (valid && q4 == 0) {
                    const double ri = a.b[i] - vi;
                    a.r[i] = ri;
                    if (zlocal) {
                        const double zi = jacobi ? ri / a.d[i] : ri;
                        a.z[i] = zi;
                        rz_n += ri * zi;
                        rr_l += ri * ri;
                    }
                }
            }
            if (blockpc) {
                if (!grid_barrier(gb, G)) return;
                for (int blk = cta; blk < a.nbj; blk += G)
                    block_apply(a.bperm, a.binv, blk, a.x, a.r, a.z, a.p, a.q, a.pdf, 0.0, false, false, rs, rz_n,
                                rr_l);
            } else if (calpc) {  // r was written in the row-pass layout: barrier first
                if (!grid_barrier(gb, G)) return;
                for (int64_t i = i0; i < a.N; i += stride) rr_l += a.r[i] * a.r[i];
                if (!calderon(false, rz_n)) return;
            }
            cta_partial2(rz_n, rr_l, pB, pC, cta);
            if (!grid_barrier(gb, G)) return;
            grid_total2(pB, pC, G, rz_new, rr);
            rr_true_prev = rr_true;
            rr_true = rr;
            ++ndf;
            if (use16 && rr_true > kH16Progress * rr_true_prev) use16 = false;  // the same in every CTA
        }
        const double beta = rz_new / rz;
        if (a.lanczos && cta == 0 && threadIdx.x == 0 && it - 1 < a.lanczos_cap) {
            a.lanczos[2 * (it - 1)] = alpha;
            a.lanczos[2 * (it - 1) + 1] = beta;
        }
        rz = rz_new;
        for (int64_t i = i0; i < a.N; i += stride) {
            const double pi = a.z[i] + beta * a.p[i];
            a.p[i] = pi;
            a.pdf[i] = df_from_double(pi);
        }
        if (!grid_barrier(gb, G)) return;
    }
    if (cta == 0 && threadIdx.x == 0) {
        a.out[0] = rr;
        a.out[1] = bb;
        a.out[2] = (double)it;
        a.out[3] = (double)ndf;
        a.out[4] = (double)inexact_stop;
        if (a.n16_out) a.n16_out[0] = (double)n16;
    }
}

__global__ void __launch_bounds__(kSymThreads, 3) k_pcg_df(PcgArgs a) { pcg_body<false>(a, gridDim.x, blockIdx.x); }
__global__ void __launch_bounds__(kSymThreads, 3) k_pcg_cal(PcgArgs a) { pcg_body<true>(a, gridDim.x, blockIdx.x); }

// Independent solves in one cooperative launch: problem p owns the CTAs
// [begin[p], begin[p + 1]) and runs the same solver on them, with its own grid
// barrier, tile counter and partials; a problem that converges releases its CTAs.
__global__ void __launch_bounds__(kSymThreads, 3) k_pcg_batch(const PcgArgs *__restrict__ args,
                                                              const int *__restrict__ begin, int P)
{
    __shared__ PcgArgs sa;
    __shared__ int s_p;
    if (threadIdx.x == 0) {
        int lo = 0, hi = P - 1;  // last p with begin[p] <= blockIdx.x
        while (lo < hi) {
            const int mid = (lo + hi + 1) / 2;
            if (begin[mid] <= (int)blockIdx.x)
                lo = mid;
            else
                hi = mid - 1;
        }
        s_p = lo;
        sa = args[lo];
    }
    __syncthreads();
    const int p = s_p;
    const int b0 = begin[p], b1 = begin[p + 1];
    if ((int)blockIdx.x >= b1) return;  // CTAs past the last group
    pcg_body<false>(sa, b1 - b0, (int)blockIdx.x - b0);
}

// ------------------------------------------------------------------ host side
struct Work {
    double *r, *z, *p, *q, *b, *x, *d;  // vectors of length ld
    float2 *xdf;                        // hi/lo copy of the matvec input (double-float paths)
    float2 *prow, *pcol;                // symmetric matvec tile partials (DF64), one 64-vector per tile
    int2 *tiles;                        // upper-triangle tile list
    double *part1, *part2, *part3;      // per-block partials
    double *scal;                       // device scalars: [0..1] rz slots, [2] rr, [3..5] reduce3
    int nb_vec, nb_mv;
};

// y = V x.  acc64: FP64-accurate products and sums (double-float arithmetic for
// DF64 and F32 storage, native FP64 for F64); otherwise FP32 (F32 storage only).
// xdf: scratch of ld hi/lo pairs for the double-float paths.
static bem_status launch_mv(bem_operator *op, bool acc64, const double *x, double *y, const double *w,
                            double *part, float2 *xdf, float2 *prow, float2 *pcol, const int2 *tiles, int *nparts)
{
    bem_ctx *ctx = op->mesh->ctx;
    const unsigned g = nblk(op->N, kMvRows);
    const double es = op->precision == BEM_PREC_F32 ? 4.0 : 8.0;
    const bool df = op->precision == BEM_PREC_DF64 || (op->precision == BEM_PREC_F32 && acc64);
    const bool sym = op->precision == BEM_PREC_DF64 && prow && pcol && tiles;
    if (!sym && op->upper_only) {  // the row kernels read whole rows
        const bem_status st = ensure_full(op);
        if (st) return st;
    }
    if (df) {
        k_to_df<<<nblk(op->ld, 256), 256, 0, ctx->stream>>>(x, op->N, op->ld, xdf); BEM_COUNT(ctx);
    }
    // algorithmic bytes: the half of V that a symmetric product must read, else all of V
    const double bytes = es * (double)op->N * (double)op->N * (sym ? 0.5 : 1.0);
    const int prof = prof_start(ctx, BEM_KERNEL_MATVEC, bytes);
    if (nparts) *nparts = (int)g;
    if (sym) {
        const int nb = (int)(op->ld / kSB);
        const int ntiles = nb * (nb + 1) / 2;
        BEM_CK(ctx, cudaFuncSetAttribute(k_symv_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSymSmem));
        const int grid = ntiles < 3 * ctx->sm_count ? ntiles : 3 * ctx->sm_count;
        k_symv_df<<<grid, kSymThreads, kSymSmem, ctx->stream>>>((const float2 *)op->V, op->ld, op->N, nb, tiles, ntiles,
                                                                xdf, prow, pcol); BEM_COUNT(ctx);
        k_symv_reduce<<<nblk(op->N, kVecThreads), kVecThreads, 0, ctx->stream>>>(prow, pcol, nb, op->N, y, w, part); BEM_COUNT(ctx);
        if (nparts) *nparts = (int)nblk(op->N, kVecThreads);
    } else if (op->precision == BEM_PREC_F64)
        { k_matvec<double, true><<<g, kMvThreads, 0, ctx->stream>>>((const double *)op->V, op->ld, op->N, x, y, w,
                                                                  part); BEM_COUNT(ctx); }
    else if (op->precision == BEM_PREC_DF64)
        { k_matvec_df<float2><<<g, kMvThreads, 0, ctx->stream>>>((const float2 *)op->V, op->ld, op->N, xdf, y, w,
                                                                part); BEM_COUNT(ctx); }
    else if (acc64)
        { k_matvec_df<float><<<g, kMvThreads, 0, ctx->stream>>>((const float *)op->V, op->ld, op->N, xdf, y, w,
                                                               part); BEM_COUNT(ctx); }
    else
        { k_matvec<float, false><<<g, kMvThreads, 0, ctx->stream>>>((const float *)op->V, op->ld, op->N, x, y, w,
                                                                  part); BEM_COUNT(ctx); }
    prof_stop(ctx, prof);
    BEM_CK_LAUNCH(ctx);
    return BEM_OK;
}

// Scratch of the symmetric product: per tile 64 hi/lo pairs for rows and for
// columns, then the tile list.
static size_t symv_scratch_bytes(const bem_operator *op)
{
    if (op->precision == BEM_PREC_F64) return 0;
    const size_t nb = (size_t)(op->ld / kSB), nt = nb * (nb + 1) / 2;
    return 2 * nt * kSB * sizeof(float2) + nt * sizeof(int2);
}

// Carve the scratch and write the tile list.
static bem_status symv_setup(bem_operator *op, void *scratch, float2 **prow, float2 **pcol, int2 **tiles)
{
    const int nb = (int)(op->ld / kSB);
    const size_t nt = (size_t)nb * (nb + 1) / 2;
    *prow = static_cast<float2 *>(scratch);
    *pcol = *prow + nt * kSB;
    *tiles = reinterpret_cast<int2 *>(*pcol + nt * kSB);
    bem_ctx *ctx = op->mesh->ctx;
    k_tile_list<<<nb, 128, 0, ctx->stream>>>(nb, *tiles); BEM_COUNT(ctx);
    BEM_CK_LAUNCH(ctx);
    return BEM_OK;
}

bem_status matvec_f64(bem_operator *op, const double *x, double *y)
{
    bem_ctx *ctx = op->mesh->ctx;
    Allocs tmp;
    float2 *xdf = nullptr, *pr = nullptr, *pc = nullptr;
    int2 *tl = nullptr;
    void *scr = nullptr;
    const size_t ps = symv_scratch_bytes(op);
    bem_status st = dalloc(ctx, tmp, (void **)&xdf, sizeof(float2) * op->ld, false);
    if (!st && ps) st = dalloc(ctx, tmp, &scr, ps, false);
    if (!st && ps) st = symv_setup(op, scr, &pr, &pc, &tl);
    if (!st) st = launch_mv(op, true, x, y, nullptr, nullptr, xdf, pr, pc, tl, nullptr);
    dfree_all(ctx, tmp);
    return st;
}

static bem_status read_scalars(bem_ctx *ctx, const double *d, int n, double *h)
{
    BEM_CK(ctx, cudaMemcpyAsync(ctx->h_pinned, d, sizeof(double) * n, cudaMemcpyDeviceToHost, ctx->stream));
    BEM_CK(ctx, cudaStreamSynchronize(ctx->stream));
    memcpy(h, ctx->h_pinned, sizeof(double) * n);
    return BEM_OK;
}

// PCG on V x = rhs from the initial x already in W.x.  acc64: FP64 products for
// FP32 operators.  Stops at ||r|| <= tol ||rhs|| (recursive residual) or max_it.
static bem_status pcg(bem_operator *op, Work &W, const double *rhs, double tol, int max_it, int precond,
                      bool acc64, int *its_out, double *rel_out)
{
    bem_ctx *ctx = op->mesh->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t N = op->N;
    bem_status st;
    if ((st = launch_mv(op, acc64, W.x, W.q, nullptr, nullptr, W.xdf, W.prow, W.pcol, W.tiles, nullptr))) return st;
    k_pcg_init<<<W.nb_vec, kVecThreads, 0, s>>>(N, rhs, W.q, W.d, precond, W.r, W.z, W.p, W.part1, W.part2,
                                                W.part3); BEM_COUNT(ctx);
    k_reduce3<<<1, 1024, 0, s>>>(W.part1, W.part2, W.part3, W.nb_vec, W.scal + 3); BEM_COUNT(ctx);
    BEM_CK_LAUNCH(ctx);
    BEM_CK(ctx, cudaMemcpyAsync(W.scal + 0, W.scal + 3, sizeof(double), cudaMemcpyDeviceToDevice, s));
    double h[3];
    if ((st = read_scalars(ctx, W.scal + 3, 3, h))) return st;
    const double bnorm = std::sqrt(h[2]) > 0 ? std::sqrt(h[2]) : 1.0;
    double rel = std::sqrt(h[1]) / bnorm;
    int it = 0;
    while (rel > tol && it < max_it) {
        int npq = 0;
        if ((st = launch_mv(op, acc64, W.p, W.q, W.p, W.part3, W.xdf, W.prow, W.pcol, W.tiles, &npq))) return st;
        const int cur = it & 1, nxt = cur ^ 1;
        k_pcg_update1<<<W.nb_vec, kVecThreads, 0, s>>>(N, W.part3, npq, W.scal + cur, W.x, W.r, W.z, W.p,
                                                       W.q, W.d, precond, W.part1, W.part2); BEM_COUNT(ctx);
        k_pcg_update2<<<W.nb_vec, kVecThreads, 0, s>>>(N, W.part1, W.part2, W.nb_vec, W.scal + cur,
                                                       W.scal + nxt, W.scal + 2, W.z, W.p); BEM_COUNT(ctx);
        BEM_CK_LAUNCH(ctx);
        ++it;
        double rr;
        if ((st = read_scalars(ctx, W.scal + 2, 1, &rr))) return st;
        rel = std::sqrt(rr) / bnorm;
    }
    *its_out = it;
    *rel_out = rel;
    return BEM_OK;
}

// The persistent DF64 solver (k_pcg_df).  Returns BEM_OK with *ran = false when a
// cooperative launch of the needed size is not possible (the caller then runs the
// host-driven loop).
// Cluster order and inverse blocks of the block-Jacobi preconditioner (scratch in tmp).
// Cluster order of the block preconditioner (depends on the mesh only): scratch and
// perm (nbj x kBJ, -1 padding) in a.
static bem_status cluster_setup(bem_operator *op, Allocs &a, int32_t **perm_out, int *nbj_out)
{
    bem_ctx *ctx = op->mesh->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t N = op->N;
    const int nbj = (int)((N + kBJ - 1) / kBJ);
    int64_t n2 = 2;
    while (n2 < N) n2 <<= 1;
    unsigned long long *keys = nullptr;
    const size_t kb = sizeof(unsigned long long) * n2, pb = sizeof(int32_t) * nbj * kBJ;
    const int nbox = (int)std::min<int64_t>((N + 255) / 256, 64);
    bem_status st = dalloc(ctx, a, (void **)&keys, kb + pb + (6 + 6 * nbox) * sizeof(double) + 64, false);
    if (st) return st;
    int32_t *perm = reinterpret_cast<int32_t *>(keys + n2);
    double *box = reinterpret_cast<double *>(reinterpret_cast<char *>(perm) + (pb + 7) / 8 * 8);
    k_cent_box<<<nbox, 256, 0, s>>>(op->mesh->cent, N, box + 6); BEM_COUNT(ctx);
    k_box_fold<<<1, 32, 0, s>>>(box + 6, nbox, box); BEM_COUNT(ctx);
    k_morton_keys<<<nblk(n2, 256), 256, 0, s>>>(op->mesh->cent, N, n2, box, keys); BEM_COUNT(ctx);
    sort_u64(ctx, keys, n2);
    k_cluster_perm<<<nblk((int64_t)nbj * kBJ, 256), 256, 0, s>>>(keys, N, (int64_t)nbj * kBJ, perm); BEM_COUNT(ctx);
    BEM_CK_LAUNCH(ctx);
    *perm_out = perm;
    *nbj_out = nbj;
    return BEM_OK;
}

// Inverse blocks of the block preconditioner from the assembled operator.
static bem_status block_inverse_launch(bem_operator *op, const int32_t *perm, int nbj, double *binv)
{
    bem_ctx *ctx = op->mesh->ctx;
    cudaStream_t s = ctx->stream;
    if (op->precision == BEM_PREC_DF64) {
        k_block_inverse<float2><<<nbj, 256, 0, s>>>((const float2 *)op->V, op->ld, perm, binv); BEM_COUNT(ctx);
    } else if (op->precision == BEM_PREC_F64) {
        k_block_inverse<double><<<nbj, 256, 0, s>>>((const double *)op->V, op->ld, perm, binv); BEM_COUNT(ctx);
    } else {
        k_block_inverse<float><<<nbj, 256, 0, s>>>((const float *)op->V, op->ld, perm, binv); BEM_COUNT(ctx);
    }
    BEM_CK_LAUNCH(ctx);
    return BEM_OK;
}

// Cluster order and inverse blocks of the block-Jacobi preconditioner (scratch in tmp).
static bem_status block_setup(bem_operator *op, Allocs &tmp, int32_t **perm_out, double **binv_out, int *nbj_out)
{
    int32_t *perm = nullptr;
    double *binv = nullptr;
    int nbj = 0;
    bem_status st = cluster_setup(op, tmp, &perm, &nbj);
    if (!st) st = dalloc(op->mesh->ctx, tmp, (void **)&binv, sizeof(double) * kBJ * kBJ * nbj, false);
    if (!st) st = block_inverse_launch(op, perm, nbj, binv);
    if (st) return st;
    *perm_out = perm;
    *binv_out = binv;
    *nbj_out = nbj;
    return BEM_OK;
}

// Extreme eigenvalues of the symmetric tridiagonal matrix with diagonal d and
// off-diagonal e, by bisection on Sturm counts inside the Gershgorin interval.
static void tridiag_extremes(const std::vector<double> &d, const std::vector<double> &e, double *lmin, double *lmax)
{
    const int k = (int)d.size();
    double gl = INFINITY, gh = -INFINITY;
    for (int i = 0; i < k; ++i) {
        const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i + 1 < k ? std::fabs(e[i]) : 0.0);
        gl = std::min(gl, d[i] - r);
        gh = std::max(gh, d[i] + r);
    }
    auto below = [&](double x) {  // eigenvalues < x
        int c = 0;
        double q = 1.0;
        for (int i = 0; i < k; ++i) {
            q = (d[i] - x) - (i > 0 ? e[i - 1] * e[i - 1] / q : 0.0);
            if (q == 0.0) q = -1e-300;
            if (q < 0.0) ++c;
        }
        return c;
    };
    auto bisect = [&](int target) {  // smallest x with below(x) >= target
        double a = gl, b = gh;
        for (int it = 0; it < 200 && b - a > 1e-15 * std::max(std::fabs(a), std::fabs(b)); ++it) {
            const double m = 0.5 * (a + b);
            if (below(m) >= target)
                b = m;
            else
                a = m;
        }
        return b;
    };
    *lmin = bisect(1);
    *lmax = bisect(k);
}

// delta > 0 selects the mixed mode: the products of the iteration use the packed
// FP32 hi parts of the upper triangle, and the residual is recomputed with the DF64
// product whenever ||r|| has dropped by delta since the last such residual (and at
// convergence).  Without room for the packed copy in the context's budget the
// solve runs with DF64 products only.
// Results of a finished persistent solve from their pinned copy h ([0..4] the
// solver's out, [5] the barrier error flag).
static bem_status persistent_results(bem_ctx *ctx, const double *h, const PersistentRun &r, int *its, int *ndf,
                                     double *rel, bool *inexact)
{
    if (*reinterpret_cast<const int *>(h + 5)) return set_error(ctx, BEM_ERR_CUDA, "persistent solve: grid barrier timed out");
    *inexact = h[4] != 0.0;
    *its = (int)h[2];
    *ndf = r.mixed ? (int)h[3] : 1;
    *rel = std::sqrt(h[0] / (h[1] > 0.0 ? h[1] : 1.0));
    // algorithmic bytes: a DF64 product reads the upper triangle of V (8 bytes x N^2 /
    // 2); a mixed-mode iteration reads the packed FP32 upper triangle (4 x N^2 / 2),
    // written once by the first product (+ the packed FP32 C once per preconditioner
    // application)
    // (FP16 working copy: N^2 bytes per iteration that used it, h[7] of them, and
    // for DF64 its packing, 2 N^2 read and N^2 written once)
    const double n2 = r.n2;
    const double i16 = r.h16 ? h[7] : 0.0, i32 = h[2] - i16;
    const double bytes = (r.f32op  ? 2.0 * n2 * (i32 + h[3]) + n2 * i16
                          : r.mixed ? 4.0 * n2 * h[3] + 2.0 * n2 * (i32 + 1.0) + n2 * i16 + (r.h16 ? 3.0 * n2 : 0.0)
                                    : 4.0 * n2 * (h[2] + h[3])) +
                         (r.calpc ? 2.0 * n2 * (h[2] + h[3]) : 0.0);
    prof_set_units(ctx, r.prof, bytes);
    return BEM_OK;
}

static bem_status pcg_persistent(bem_operator *op, Work &W, const double *rhs, bool has_x0, double tol, int max_it,
                                 int precond, double delta, const int32_t *bperm, const double *binv, int nbj,
                                 double inexact_lambda, int h_mode, int *its_out, int *ndf_out, double *rel_out,
                                 bool *ran, double *lmin, double *lmax, bool *inexact_out, SolveDeferred *def,
                                 int products)
{
    // FP32 operators: the products of the iteration and of the residuals read the
    // packed copy of the stored operator (the residual, formed from x with
    // FP64-accurate sums, confirms convergence)
    const bool f32op = op->precision == BEM_PREC_F32;
    bem_ctx *ctx = op->mesh->ctx;
    *ran = false;
    int coop = 0, per_sm = 0;
    BEM_CK(ctx, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
    if (!coop || !W.tiles) return BEM_OK;
    if (f32op) delta = 1.0;  // a packed copy is needed; residuals are replaced only at convergence
    const int nb_ = (int)(op->ld / kSB), nt_ = nb_ * (nb_ + 1) / 2;
    const void *kern = precond == BEM_PRECOND_CALDERON ? (const void *)k_pcg_cal : (const void *)k_pcg_df;
    BEM_CK(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSymSmem));
    BEM_CK(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSymThreads, kSymSmem));
    if (per_sm < 1) return BEM_OK;
    Allocs tmp;
    bem_status st = BEM_OK;
    float *vp = nullptr;
    if (delta > 0.0) {
        const size_t vbytes = (size_t)nt_ * kTileF * sizeof(float);
        if (ctx->budget <= 0 || ctx->in_use + (int64_t)vbytes + (64 << 10) <= ctx->budget)
            if ((st = dalloc(ctx, tmp, (void **)&vp, vbytes, false))) return st;
    }
    if (f32op && !vp) return BEM_OK;  // no room for the packed copy: host-driven refinement
    const bool calpc = precond == BEM_PRECOND_CALDERON;
    float *dvp = nullptr;
    if (calpc) {  // packed C (the tiles of the operator's packed copy)
        if ((st = dalloc(ctx, tmp, (void **)&dvp, (size_t)nt_ * kTileF * sizeof(float), false))) {
            dfree_all(ctx, tmp);
            return st;
        }
        k_pack_f32<<<(unsigned)std::min<int64_t>(((int64_t)nt_ * (kTileF / 4) + 255) / 256, 8 * ctx->sm_count), 256, 0,
                     ctx->stream>>>(op->cal_C, op->ld, op->N, W.tiles, nt_, dvp); BEM_COUNT(ctx);
    }
    if (f32op) {
        k_pack_f32<<<(unsigned)std::min<int64_t>(((int64_t)nt_ * (kTileF / 4) + 255) / 256, 8 * ctx->sm_count), 256, 0,
                     ctx->stream>>>((const float *)op->V, op->ld, op->N, W.tiles, nt_, vp); BEM_COUNT(ctx);
    }
    // FP16 working copy for the iteration products (N^2 bytes and a scale per tile)
    __half *vh = nullptr;
    float *vsc = nullptr;
    // default: FP16 for FP32 operators (whose stored entries are FP32 roundings already)
    // under the block preconditioner (a condition number the FP16 copy's perturbation
    // leaves room for; diag(V) on strongly graded meshes does not), else the packed
    // FP32 hi parts
    if (products == BEM_PRODUCTS_DEFAULT)
        products = (f32op && precond == BEM_PRECOND_BLOCK) ? BEM_PRODUCTS_FP16 : BEM_PRODUCTS_FP32;
    if (products == BEM_PRODUCTS_FP16 && vp && !calpc) {
        const size_t hb = (size_t)nt_ * kTileF * sizeof(__half), sb = ((size_t)nt_ * sizeof(float) + 255) / 256 * 256;
        if (ctx->budget <= 0 || ctx->in_use + (int64_t)(hb + sb) + (64 << 10) <= ctx->budget) {
            if ((st = dalloc(ctx, tmp, (void **)&vh, hb + sb, false))) {
                dfree_all(ctx, tmp);
                return st;
            }
            vsc = reinterpret_cast<float *>(reinterpret_cast<char *>(vh) + hb);
            if (f32op) {
                k_pack_h16<<<(unsigned)std::min<int64_t>(((int64_t)nt_ * 32 + 255) / 256, 8 * ctx->sm_count), 256, 0,
                             ctx->stream>>>(vp, nt_, vh, vsc); BEM_COUNT(ctx);
            }
        }
    }
    // Up to 3 CTAs per SM.  On small levels, CTAs that would only wait at the grid
    // barriers are left out: DF64 products take one tile per CTA, the mixed mode's
    // products one tile per warp (8 per CTA), its row passes 8 rows per warp.
    const int Gmax = (per_sm < 3 ? per_sm : 3) * ctx->sm_count;
    int G = vp ? (int)std::max<int64_t>((nt_ + 7) / 8, (op->N + 63) / 64) : nt_;
    G = std::min(std::max(G, 8), Gmax);
    double *part = nullptr;
    if ((st = dalloc(ctx, tmp, (void **)&part, sizeof(double) * (3 * G + 8) + 64, true))) {
        dfree_all(ctx, tmp);
        return st;
    }
    double *out = part + 3 * G;  // [0..4]: r.r, b.b, iterations, DF64 residuals, inexact stop
    unsigned long long *ctr = reinterpret_cast<unsigned long long *>(out + 6);
    unsigned *bar = reinterpret_cast<unsigned *>(ctr + 1);
    int *err = reinterpret_cast<int *>(bar + 2);
    const int lcap = std::min(max_it, 20000);
    double *unod = nullptr;
    if (inexact_lambda > 0.0 && (st = dalloc(ctx, tmp, (void **)&unod, sizeof(double) * op->mesh->M, false))) {
        dfree_all(ctx, tmp);
        return st;
    }
    double *lanczos = nullptr;
    if ((st = dalloc(ctx, tmp, (void **)&lanczos, sizeof(double) * 2 * lcap, false))) {
        dfree_all(ctx, tmp);
        return st;
    }
    PcgArgs a{};
    a.V = (const float2 *)op->V;
    a.ld = op->ld;
    a.N = op->N;
    a.nb = (int)(op->ld / kSB);
    a.ntiles = a.nb * (a.nb + 1) / 2;
    a.tiles = W.tiles;
    a.prow = W.prow;
    a.pcol = W.pcol;
    a.pdf = W.xdf;
    a.x = W.x;
    a.r = W.r;
    a.z = W.z;
    a.p = W.p;
    a.q = W.q;
    a.d = W.d;
    a.b = rhs;
    a.part = part;
    a.bar = bar;
    a.ctr = ctr;
    a.err = err;
    a.out = out;
    a.vp = vp;
    a.lanczos = lanczos;
    a.lanczos_cap = lcap;
    a.lam2 = inexact_lambda > 0.0 ? inexact_lambda * inexact_lambda : 0.0;
    a.tris = op->mesh->tris;
    a.v2t_off = op->mesh->v2t_off;
    a.v2t = op->mesh->v2t;
    a.area = op->mesh->area;
    a.hdiam = h_mode == 1 ? nullptr : op->mesh->diam;
    a.u = unod;
    a.M = op->mesh->M;
    a.bperm = bperm;
    a.binv = binv;
    a.nbj = nbj;
    a.tol = tol;
    a.f32op = f32op ? 1 : 0;
    a.delta2 = f32op ? 0.0 : delta * delta;
    a.max_it = max_it;
    a.precond = precond;
    a.has_x0 = has_x0 ? 1 : 0;
    a.dvp = dvp;
    a.vh = vh;
    a.vsc = vsc;
    a.n16_out = out + 5;
    a.bar_limit_ns = ctx->bar_limit_ns;
    a.absent_cta = ctx->bar_absent_cta < G ? ctx->bar_absent_cta : -1;
    void *args[] = {&a};
    const int prof = prof_start(ctx, BEM_KERNEL_MATVEC, 0.0);
    cudaError_t e = cudaLaunchCooperativeKernel(kern, dim3(G), dim3(kSymThreads), args, kSymSmem,
                                                ctx->stream);
    BEM_COUNT(ctx);
    prof_stop(ctx, prof);
    if (e != cudaSuccess) {
        cudaGetLastError();
        dfree_all(ctx, tmp);
        return BEM_OK;  // not launchable here: fall back
    }
    // the solver's out[0..4] and its barrier error flag to pinned host memory: read
    // now (synchronous solve), or after a later synchronisation of the stream
    // (deferred: the caller finishes the solve with solve_capacity_end)
    double *hres = def ? def->h : ctx->h_pinned;
    PersistentRun run;
    run.prof = prof;
    run.f32op = f32op;
    run.mixed = vp != nullptr;
    run.calpc = calpc;
    run.n2 = (double)op->N * (double)op->N;
    run.h16 = vh != nullptr;
    e = cudaMemcpyAsync(hres, out, 5 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hres + 5, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hres + 7, out + 5, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess && !def) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) st = cuda_error(ctx, e, "persistent solve");
    if (!st && def) {
        def->run = run;
        *ran = true;
        *lmin = *lmax = 0.0;  // no condition estimates for deferred solves
    } else if (!st) {
        double h[8];
        memcpy(h, hres, sizeof(h));
        st = persistent_results(ctx, h, run, its_out, ndf_out, rel_out, inexact_out);
        if (!st) {
            *ran = true;
            // Lanczos tridiagonal matrix of the CG coefficients
            const int k = std::min((int)h[2] - (h[4] != 0.0 ? 1 : 0), lcap);  // an inexact stop records no beta
            *lmin = *lmax = 0.0;
            if (k > 0) {
                std::vector<double> ab(2 * (size_t)k);
                e = cudaMemcpy(ab.data(), lanczos, sizeof(double) * 2 * k, cudaMemcpyDeviceToHost);
                if (e != cudaSuccess) {
                    st = cuda_error(ctx, e, "CG coefficients");
                } else {
                    std::vector<double> dg(k), od(k > 1 ? k - 1 : 0);
                    for (int j = 0; j < k; ++j) {
                        dg[j] = 1.0 / ab[2 * j] + (j > 0 ? ab[2 * j - 1] / ab[2 * (j - 1)] : 0.0);
                        if (j + 1 < k) od[j] = std::sqrt(ab[2 * j + 1]) / ab[2 * j];
                    }
                    tridiag_extremes(dg, od, lmin, lmax);
                }
            }
        }
    }
    dfree_all(ctx, tmp);
    return st;
}

__global__ void k_capacity(int64_t N, const double *area, const double *x, double *out)
{
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) v += area[i] * x[i];
    __shared__ double part[1];
    block_partial(v, part);
    if (threadIdx.x == 0) out[0] = part[0] * kInv4Pi;
}

bem_status solve_capacity_end(bem_ctx *ctx, SolveDeferred &def, double *cap, bem_solve_info *info)
{
    if (!def.pending) return BEM_OK;
    def.pending = false;
    int its = 0, ndf = 0;
    double rel = 0.0;
    bool inexact = false;
    bem_status st = persistent_results(ctx, def.h, def.run, &its, &ndf, &rel, &inexact);
    if (st) return st;
    *cap = def.h[6];
    if (info) {
        info->iterations = its;
        info->outer = ndf;
        info->relres = rel;
        info->converged = rel <= def.tol || inexact;
        info->lambda_min = info->lambda_max = 0.0;
    }
    if (rel > def.tol && !inexact)
        return set_error(ctx, BEM_ERR_NOT_CONVERGED, "solve stopped at relative residual %.3e > %.3e", rel, def.tol);
    return BEM_OK;
}

bem_status solve_capacity(bem_operator *op, const bem_solve_opts *o, const double *d_x0, double *d_x,
                          double *cap, bem_solve_info *info, SolveDeferred *def)
{
    if (def) def->pending = false;
    bem_mesh *m = op->mesh;
    bem_ctx *ctx = m->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t N = op->N, L = op->ld;
    if (o->precond < BEM_PRECOND_NONE || o->precond > BEM_PRECOND_CALDERON)
        return set_error(ctx, BEM_ERR_INVALID, "unknown preconditioner %d", o->precond);
    if (o->precond == BEM_PRECOND_CALDERON &&
        (!op->cal_C || op->precision == BEM_PREC_F64 || !ctx->persistent_solver))
        return set_error(ctx, BEM_ERR_INVALID,
                         "BEM_PRECOND_CALDERON needs a DF64 dual operator (bem_operator_dual) and the persistent solver");
    if (o->inexact_lambda > 0.0 && m->cells_only)
        return set_error(ctx, BEM_ERR_INVALID, "the inexact stopping rule needs a triangle mesh (not a dual operator)");
    if (o->precond == BEM_PRECOND_BLOCK && (op->precision == BEM_PREC_F64 || !ctx->persistent_solver))
        return set_error(ctx, BEM_ERR_INVALID,
                         "BEM_PRECOND_BLOCK is implemented by the persistent solver (DF64 and FP32 operators)");
    Allocs tmp;
    Work W{};
    W.nb_vec = (int)nblk(N, kVecThreads);
    W.nb_mv = (int)nblk(N, kMvRows);
    const int np = W.nb_mv > W.nb_vec ? W.nb_mv : W.nb_vec;
    bem_status st = BEM_OK;
    double *base = nullptr;
    const size_t vecs = 7;
    if ((st = dalloc(ctx, tmp, (void **)&base, sizeof(double) * (vecs * L + 3 * np + 8), true))) return st;
    if ((st = dalloc(ctx, tmp, (void **)&W.xdf, sizeof(float2) * L, true))) {
        dfree_all(ctx, tmp);
        return st;
    }
    W.prow = W.pcol = nullptr;
    W.tiles = nullptr;
    if (const size_t ps = symv_scratch_bytes(op)) {
        void *scr = nullptr;
        if ((st = dalloc(ctx, tmp, &scr, ps, false)) || (st = symv_setup(op, scr, &W.prow, &W.pcol, &W.tiles))) {
            dfree_all(ctx, tmp);
            return st;
        }
    }
    W.r = base;
    W.z = base + L;
    W.p = base + 2 * L;
    W.q = base + 3 * L;
    W.b = base + 4 * L;
    W.x = base + 5 * L;
    W.d = base + 6 * L;
    W.part1 = base + vecs * L;
    W.part2 = W.part1 + np;
    W.part3 = W.part2 + np;
    W.scal = W.part3 + np;
    const double tol = o->tol > 0 ? o->tol : 1e-10;
    const int max_it = o->max_it > 0 ? o->max_it : 10000;
    const int precond = o->precond;
    int its = 0, outer = 0;
    double rel = 0.0;
    bool ran = false;
    double lam_min = 0.0, lam_max = 0.0;
    bool inexact = false;
    cudaError_t e = cudaMemcpyAsync(W.b, m->area, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(W.d, op->diag, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && d_x0) e = cudaMemcpyAsync(W.x, d_x0, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        st = cuda_error(ctx, e, "solve setup");
        goto out;
    }
    outer = 1;
    {
        // persistent solver (DF64 and FP32 operators).  DF64: FP32 products of the
        // packed hi parts between DF64 residuals whenever ||r|| drops by
        // reliable_delta (default 1e-4; < 0: DF64 products only).  FP32: products of
        // the packed operator, residual confirmed at convergence.
        const double delta = o->reliable_delta == 0.0 ? 1e-4 : (o->reliable_delta > 0.0 ? o->reliable_delta : 0.0);
        int32_t *bperm = nullptr;
        double *binv = nullptr;
        int nbj = 0;
        if (precond == BEM_PRECOND_BLOCK && (st = block_setup(op, tmp, &bperm, &binv, &nbj))) goto out;
        if (op->precision != BEM_PREC_F64 && ctx->persistent_solver)
            st = pcg_persistent(op, W, W.b, d_x0 != nullptr, tol, max_it, precond, delta < 1.0 ? delta : 0.0, bperm,
                                binv, nbj, o->inexact_lambda, o->h_mode, &its, &outer, &rel, &ran, &lam_min, &lam_max,
                                &inexact, def, o->products);
        if (!st && !ran && (precond == BEM_PRECOND_BLOCK || precond == BEM_PRECOND_CALDERON))
            st = set_error(ctx, BEM_ERR_CUDA, "this preconditioner needs the persistent solver, which could not be launched");
        if (st) goto out;
    }
    if (ran) {
    } else if (op->precision != BEM_PREC_F32) {
        st = pcg(op, W, W.b, tol, max_it, precond, true, &its, &rel);
        outer = 1;
    } else {
        // FP64 iterative refinement around FP32-product inner CG
        const int max_outer = o->max_outer > 0 ? o->max_outer : 20;
        const double inner_tol = o->inner_tol > 0 ? o->inner_tol : 1e-5;
        double *xs = nullptr, *rhs = nullptr;
        if ((st = dalloc(ctx, tmp, (void **)&xs, sizeof(double) * 2 * L, true))) goto out;
        rhs = xs + L;
        e = cudaMemcpyAsync(xs, W.x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) { st = cuda_error(ctx, e, "refinement setup"); goto out; }
        double bb = 0.0;
        for (outer = 0; outer < max_outer; ++outer) {
            // rhs = b - V xs in FP64 accumulation
            if ((st = launch_mv(op, true, xs, W.q, nullptr, nullptr, W.xdf, W.prow, W.pcol, W.tiles, nullptr))) goto out;
            k_residual<<<W.nb_vec, kVecThreads, 0, s>>>(N, W.b, W.q, rhs, W.part1); BEM_COUNT(ctx);
            k_dot_partial<<<W.nb_vec, kVecThreads, 0, s>>>(N, W.b, W.b, W.part2); BEM_COUNT(ctx);
            k_reduce3<<<1, 1024, 0, s>>>(W.part1, W.part2, nullptr, W.nb_vec, W.scal + 3); BEM_COUNT(ctx);
            double h[3];
            if ((st = read_scalars(ctx, W.scal + 3, 3, h))) goto out;
            bb = h[1] > 0 ? h[1] : 1.0;
            rel = std::sqrt(h[0] / bb);
            if (rel <= tol) break;
            cudaMemsetAsync(W.x, 0, sizeof(double) * L, s);
            int it_in = 0;
            double rel_in = 0.0;
            if ((st = pcg(op, W, rhs, inner_tol, max_it, precond, true, &it_in, &rel_in))) goto out;
            its += it_in;
            k_axpy<<<W.nb_vec, kVecThreads, 0, s>>>(N, 1.0, W.x, xs); BEM_COUNT(ctx);
            BEM_CK_LAUNCH(ctx);
        }
        if (outer == max_outer) {
            // residual of the last update
            if ((st = launch_mv(op, true, xs, W.q, nullptr, nullptr, W.xdf, W.prow, W.pcol, W.tiles, nullptr))) goto out;
            k_residual<<<W.nb_vec, kVecThreads, 0, s>>>(N, W.b, W.q, rhs, W.part1); BEM_COUNT(ctx);
            k_reduce3<<<1, 1024, 0, s>>>(W.part1, nullptr, nullptr, W.nb_vec, W.scal + 3); BEM_COUNT(ctx);
            double h[3];
            if ((st = read_scalars(ctx, W.scal + 3, 3, h))) goto out;
            rel = std::sqrt(h[0] / bb);
        }
        outer = outer < max_outer ? outer + 1 : outer;
        e = cudaMemcpyAsync(W.x, xs, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) { st = cuda_error(ctx, e, "refinement result"); goto out; }
    }
    {
        k_capacity<<<1, 1024, 0, s>>>(N, m->area, W.x, W.scal + 6); BEM_COUNT(ctx);
        BEM_CK_LAUNCH(ctx);
        if (d_x) {
            e = cudaMemcpyAsync(d_x, W.x, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) { st = cuda_error(ctx, e, "solution copy"); goto out; }
        }
        if (def && ran) {  // deferred: Cap joins the solver's results in pinned memory
            e = cudaMemcpyAsync(def->h + 6, W.scal + 6, sizeof(double), cudaMemcpyDeviceToHost, s);
            if (e != cudaSuccess) { st = cuda_error(ctx, e, "Cap copy"); goto out; }
            def->pending = true;
            def->tol = tol;
            goto out;
        }
        double c;
        if ((st = read_scalars(ctx, W.scal + 6, 1, &c))) goto out;
        *cap = c;
    }
    if (info) {
        info->iterations = its;
        info->outer = outer;
        info->relres = rel;
        info->converged = rel <= tol || inexact;
        info->lambda_min = lam_min;
        info->lambda_max = lam_max;
    }
    if (rel > tol && !inexact)
        st = set_error(ctx, BEM_ERR_NOT_CONVERGED, "solve stopped at relative residual %.3e > %.3e", rel, tol);
out:
    dfree_all(ctx, tmp);
    return st;
}

// ------------------------------------------------------------------ batch
// Independent problems assembled and solved together (bem_batch_*).  The problems are
// cut, in their given order, into waves whose device memory fits the budget (the
// context's HBM budget and the device's free memory, read at creation); one arena
// sized for the largest wave holds the operators and solver state of whichever wave
// runs, and a wave is one launch per phase for all its problems: the batched far
// field (a work list of (problem, tile) items), mirror and near field, the set-up of
// diagonals, right-hand sides and preconditioners, ONE cooperative launch of the
// persistent solver in which every problem owns a share of the CTAs, the capacities,
// and a copy of the results to pinned host memory.  With use_graph each wave's
// sequence is recorded once as a CUDA graph (its arena layout is fixed) and replayed
// by later runs; the waves of a run follow each other on the batch's stream.
struct BatchSolveProb {
    const void *V;
    int64_t ld, N;
    double *d, *b, *x;
    const double *area;
    double *part;
    int64_t part_n;  // doubles of part zeroed per run
    float *vp;       // packed FP32 upper triangle (FP32 operators: formed per run)
    __half *vh;      // its FP16 working copy (BEM_PRODUCTS_FP16, FP32 operators), else null
    float *vsc;      // and the tiles' scales
    const int2 *tiles;
    int64_t nt;
    const int32_t *perm;
    double *binv;
    int nbj;
    double *res;     // kBatchRes doubles: out[0..4] of the solver, [5] Cap, [6] error flag
};

constexpr int kBatchRes = 8;

// Per run, after the assembly: x = 0, the diagonal, b = |T|, zero padding columns
// of V, zero partials, barrier counter and results.  Grid (rows / 256, problems).
template <typename T>
__global__ void k_batch_init(const BatchSolveProb *__restrict__ prob)
{
    const BatchSolveProb *pb = prob + blockIdx.y;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t N = pb->N, ld = pb->ld;
    if (i < ld) {
        pb->x[i] = 0.0;
        if (i < N) {
            T *V = (T *)pb->V;
            pb->d[i] = elem_f64(V, i * ld + i);
            pb->b[i] = pb->area[i];
            for (int64_t j = N; j < ld; ++j) V[i * ld + j] = T();
        }
    }
    if (i < pb->part_n) pb->part[i] = 0.0;
    if (i < kBatchRes) pb->res[i] = 0.0;
}

// Packed upper triangles of FP32 operators; grid (blocks, problems).
__global__ void k_batch_pack(const BatchSolveProb *__restrict__ prob)
{
    const BatchSolveProb *pb = prob + blockIdx.y;
    const int64_t n4 = pb->nt * (kTileF / 4);
    const float *V = (const float *)pb->V;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < n4; f += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = f / (kTileF / 4);
        const int e = (int)(f % (kTileF / 4)), r = e >> 4, c4 = e & 15;
        const int2 tj = pb->tiles[k];
        const int64_t row = (int64_t)tj.x * kSB + r;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (row < pb->N) v = __ldcs(reinterpret_cast<const float4 *>(V + row * pb->ld + (int64_t)tj.y * kSB) + c4);
        reinterpret_cast<float4 *>(pb->vp)[f] = v;
    }
}

// FP16 working copies of the packed FP32 operators; grid (blocks, problems).
__global__ void k_batch_pack_h16(const BatchSolveProb *__restrict__ prob)
{
    const BatchSolveProb *pb = prob + blockIdx.y;
    if (!pb->vh) return;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    pack_h16_tiles(pb->vp, (int)pb->nt, pb->vh, pb->vsc, w0, ((int64_t)gridDim.x * blockDim.x) >> 5);
}

// Inverse cluster blocks of every problem; grid (largest cluster count, problems).
template <typename T>
__global__ void __launch_bounds__(256) k_batch_block_inverse(const BatchSolveProb *__restrict__ prob)
{
    const BatchSolveProb *pb = prob + blockIdx.y;
    if ((int)blockIdx.x >= pb->nbj) return;
    block_inverse_body<T>((const T *)pb->V, pb->ld, pb->perm, pb->binv, blockIdx.x);
}

// Cap = (1/4pi) sum |T_i| x_i of every problem (Eq. 2.8); one CTA per problem.
__global__ void k_batch_capacity(const BatchSolveProb *__restrict__ prob)
{
    const BatchSolveProb *pb = prob + blockIdx.x;
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < pb->N; i += blockDim.x) v += pb->area[i] * pb->x[i];
    // the fixed tree of block_partial (warps, then the warp sums), kept in this CTA
    __shared__ double sw[32];
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sw[w] = v;
    __syncthreads();
    if (w == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? sw[lane] : 0.0;
        t = warp_sum(t);
        if (lane == 0) pb->res[5] = t * kInv4Pi;
    }
}

struct BatchProblem {
    bem_operator *op = nullptr;  // V and diag in the arena (the handle owns no memory)
    int wave = 0;
    size_t off = 0;              // offset of this problem's block in the arena
    size_t bytes = 0;
    int64_t nt = 0;
    int2 *tiles = nullptr;       // persistent tile list
    int32_t *perm = nullptr;     // persistent cluster order (block preconditioner)
    int nbj = 0;
};

// Problems of a wave solved by one cooperative launch: similar sizes, CTAs shared in
// proportion to N^2, so that they finish at about the same time.
struct BatchGroup {
    int count = 0, G = 0;
    std::vector<int> idx;    // problems (batch indices), in launch order
    std::vector<int> begin;  // CTA ranges
    PcgArgs *d_args = nullptr;
    int *d_begin = nullptr;
};

struct BatchWave {
    int first = 0, count = 0, variant = 0, max_nbj = 0;
    int64_t max_rows = 0;
    std::vector<BatchGroup> groups;
    BatchSolveProb *d_sprob = nullptr;
    BatchAsm asmb;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0;        // kernels of one replay
    // recorded around the far field (0, 1), the near field (2, 3) and the solver
    // launch (4, 5) of every run, captured into the graph too, so that profiling sees
    // the replayed runs themselves
    cudaEvent_t ev[6] = {};
};

}  // namespace bem

struct bem_batch {
    bem_ctx *ctx = nullptr;
    int P = 0, use_graph = 1, graph_used = 0, precond = BEM_PRECOND_JACOBI, precision = BEM_PREC_F32;
    bool h16 = false;  // BEM_PRODUCTS_FP16: FP16 working copies for the iteration products
    double tol = 1e-10;
    void *arena = nullptr;
    size_t arena_bytes = 0;
    std::vector<bem::BatchProblem> prob;
    std::vector<bem::PcgArgs> args;  // per problem (pointers into the arena)
    std::vector<bem::BatchWave> waves;
    double *d_res = nullptr;  // P x kBatchRes
    double *h_res = nullptr;  // pinned copy
    cudaStream_t stream = nullptr;
    bem::Allocs allocs;
};

namespace bem {

static bem_status batch_enqueue(bem_batch *bt, BatchWave &w)
{
    bem_ctx *ctx = bt->ctx;
    cudaStream_t s = ctx->stream;
    bem_status st;
    if ((st = batch_assemble(ctx, w.asmb, w.ev))) return st;
    const dim3 gi((unsigned)((w.max_rows + 255) / 256), (unsigned)w.count);
    if (bt->precision == BEM_PREC_F32)
        k_batch_init<float><<<gi, 256, 0, s>>>(w.d_sprob);
    else
        k_batch_init<float2><<<gi, 256, 0, s>>>(w.d_sprob);
    BEM_COUNT(ctx);
    if (bt->precision == BEM_PREC_F32) {
        k_batch_pack<<<dim3(64, (unsigned)w.count), 256, 0, s>>>(w.d_sprob); BEM_COUNT(ctx);
        if (bt->h16) {
            k_batch_pack_h16<<<dim3(64, (unsigned)w.count), 256, 0, s>>>(w.d_sprob); BEM_COUNT(ctx);
        }
    }
    if (bt->precond == BEM_PRECOND_BLOCK) {
        const dim3 gb((unsigned)w.max_nbj, (unsigned)w.count);
        if (bt->precision == BEM_PREC_F32)
            k_batch_block_inverse<float><<<gb, 256, 0, s>>>(w.d_sprob);
        else
            k_batch_block_inverse<float2><<<gb, 256, 0, s>>>(w.d_sprob);
        BEM_COUNT(ctx);
    }
    BEM_CK_LAUNCH(ctx);
    if ((st = record_timing_event(ctx, w.ev[4]))) return st;
    for (const auto &gr : w.groups) {  // one cooperative launch per group of similar sizes
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)gr.G);
        cfg.blockDim = dim3(kSymThreads);
        cfg.dynamicSmemBytes = kSymSmem;
        cfg.stream = s;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        BEM_CK(ctx, cudaLaunchKernelEx(&cfg, k_pcg_batch, (const PcgArgs *)gr.d_args, (const int *)gr.d_begin, gr.count));
        BEM_COUNT(ctx);
    }
    if ((st = record_timing_event(ctx, w.ev[5]))) return st;
    k_batch_capacity<<<w.count, 1024, 0, s>>>(w.d_sprob); BEM_COUNT(ctx);
    BEM_CK_LAUNCH(ctx);
    BEM_CK(ctx, cudaMemcpyAsync(bt->h_res + (size_t)kBatchRes * w.first, bt->d_res + (size_t)kBatchRes * w.first,
                                sizeof(double) * kBatchRes * w.count, cudaMemcpyDeviceToHost, s));
    return BEM_OK;
}

// Device bytes of one problem's block in the arena: V, diagonal, 7 solver vectors, the
// double-float copy of the product's input, the tile partials of the product, the
// packed FP32 upper triangle, the CTA partials and the inverse cluster blocks.
static size_t batch_problem_bytes(int64_t N, int prec, bool packed, bool block, int G, bool h16)
{
    auto al = [](size_t b) { return (b + 255) / 256 * 256; };
    const int64_t L = padded_ld(N), nb = L / kSB, nt = nb * (nb + 1) / 2;
    const size_t es = prec == BEM_PREC_F32 ? 4 : 8;
    size_t b = al(es * (size_t)N * (size_t)L) + al(8 * (size_t)N) + al(8 * 7 * (size_t)L) + al(8 * (size_t)L) +
               al(2 * (size_t)nt * kSB * 8) + al(sizeof(double) * (3 * (size_t)G + 8) + 64);
    if (packed) b += al((size_t)nt * kTileF * 4);
    if (packed && h16) b += al((size_t)nt * kTileF * 2) + al((size_t)nt * 4);
    if (block) b += al(8 * (size_t)kBJ * kBJ * (size_t)((N + kBJ - 1) / kBJ));
    return b;
}

}  // namespace bem

extern "C" {

bem_status bem_batch_create(bem_ctx *ctx, int32_t count, bem_mesh *const *meshes, const bem_assembly_opts *aopts,
                            const bem_solve_opts *sopts, int32_t use_graph, bem_batch **out)
{
    using namespace bem;
    if (!ctx || !meshes || !out || count < 1) return ctx ? set_error(ctx, BEM_ERR_INVALID, "bad batch arguments") : BEM_ERR_INVALID;
    *out = nullptr;
    const int prec = aopts ? aopts->precision : BEM_PREC_DF64;
    if (prec != BEM_PREC_DF64 && prec != BEM_PREC_F32)
        return set_error(ctx, BEM_ERR_INVALID, "a batch needs BEM_PREC_DF64 or BEM_PREC_F32 operators");
    const int precond = sopts ? sopts->precond : BEM_PRECOND_JACOBI;
    if (precond < BEM_PRECOND_NONE || precond > BEM_PRECOND_BLOCK)
        return set_error(ctx, BEM_ERR_INVALID, "preconditioner %d: a batch takes NONE, JACOBI or BLOCK", precond);
    for (int p = 0; p < count; ++p)
        if (!meshes[p] || meshes[p]->ctx != ctx || meshes[p]->cells_only)
            return set_error(ctx, BEM_ERR_INVALID, "mesh %d is not a triangle mesh of this context", p);
    const int ss = (aopts && aopts->ss_order > 0) ? aopts->ss_order : 4;
    if (ss < 2 || ss > kMaxSS) return set_error(ctx, BEM_ERR_INVALID, "ss_order outside 2..16");
    int coop = 0, per_sm = 0;
    BEM_CK(ctx, cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->device));
    if (!coop) return set_error(ctx, BEM_ERR_CUDA, "the device has no cooperative launch");
    BEM_CK(ctx, cudaFuncSetAttribute(k_pcg_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSymSmem));
    BEM_CK(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_batch, kSymThreads, kSymSmem));
    const int Gmax = (per_sm < 3 ? per_sm : 3) * ctx->sm_count;
    if (Gmax < 1) return set_error(ctx, BEM_ERR_CUDA, "the batch solver cannot be resident on this device");
    bem_status st = assembly_prepare(ctx);
    if (st) return st;
    BEM_CK(ctx, cudaStreamSynchronize(ctx->stream));  // meshes built on the context's stream
    bem_batch *bt = new (std::nothrow) bem_batch();
    if (!bt) return set_error(ctx, BEM_ERR_OOM, "host allocation");
    bt->ctx = ctx;
    bt->P = count;
    bt->use_graph = use_graph ? 1 : 0;
    bt->precond = precond;
    bt->precision = prec;
    bt->tol = (sopts && sopts->tol > 0) ? sopts->tol : 1e-10;
    const int max_it = (sopts && sopts->max_it > 0) ? sopts->max_it : 10000;
    const double rd = sopts ? sopts->reliable_delta : 0.0;
    const double delta = rd == 0.0 ? 1e-4 : (rd > 0.0 && rd < 1.0 ? rd : 0.0);
    const bool packed = prec == BEM_PREC_F32 || delta > 0.0;
    const bool block = precond == BEM_PRECOND_BLOCK;
    {
        const int pr = sopts ? sopts->products : BEM_PRODUCTS_DEFAULT;
        bt->h16 = packed && (pr == BEM_PRODUCTS_FP16 ||
                             (pr == BEM_PRODUCTS_DEFAULT && prec == BEM_PREC_F32 && precond == BEM_PRECOND_BLOCK));
    }
    bt->prob.resize(count);
    bt->args.resize(count);
    auto fail = [&](bem_status code) {
        bem_batch_destroy(bt);
        return code;
    };
    // persistent per-problem data: tile lists, cluster orders, results
    for (int p = 0; p < count && !st; ++p) {
        BatchProblem &pr = bt->prob[p];
        const int64_t N = meshes[p]->N, nb = padded_ld(N) / kSB;
        pr.nt = nb * (nb + 1) / 2;
        if ((st = dalloc(ctx, bt->allocs, (void **)&pr.tiles, sizeof(int2) * (size_t)pr.nt, false))) break;
        k_tile_list<<<(unsigned)nb, 128, 0, ctx->stream>>>((int)nb, pr.tiles); BEM_COUNT(ctx);
    }
    if (!st) st = dalloc(ctx, bt->allocs, (void **)&bt->d_res, sizeof(double) * kBatchRes * count, true);
    if (st) return fail(st);
    // waves: problems in their order, a new wave when the next one does not fit the
    // memory left for the arena or the CTAs of one cooperative launch
    int64_t avail = 0;
    {
        cache_release(ctx);  // the kept blocks go back to the pool, then to the device
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e == cudaSuccess) e = cudaMemPoolTrimTo(ctx->pool, 0);
        size_t fr = 0, tot = 0;
        if (e == cudaSuccess) e = cudaMemGetInfo(&fr, &tot);
        if (e != cudaSuccess) return fail(cuda_error(ctx, e, "batch memory query"));
        // room for what is allocated after the arena: the far-field work lists (bounded
        // by the smallest tile, 8 x 64), the cluster orders and the wave tables
        double later = 4.0 * 1048576.0;
        for (int p = 0; p < count; ++p) {
            const double N = (double)meshes[p]->N;
            int64_t n2 = 2;
            while (n2 < meshes[p]->N) n2 <<= 1;
            later += 16.0 * (N * N / 1024.0 + N / 8.0 + 2.0) + 1024.0 + sizeof(PcgArgs) + 512.0;
            if (block) later += 8.0 * (double)n2 + 4.0 * kBJ * std::ceil(N / kBJ) + 6.0 * 8.0 * 80.0 + 1024.0;
        }
        avail = (int64_t)((double)fr * 0.9) - (int64_t)later;
        if (ctx->budget > 0) avail = std::min<int64_t>(avail, ctx->budget - ctx->in_use - (int64_t)later);
    }
    // CTA share of each problem (within its wave, below) needs the wave; size the
    // partials for the largest share a problem can get
    {
        int w = 0, n_in = 0;
        size_t wbytes = 0, maxw = 0;
        for (int p = 0; p < count; ++p) {
            const size_t b = batch_problem_bytes(meshes[p]->N, prec, packed, block, Gmax, bt->h16);
            if ((int64_t)b > avail) {
                return fail(set_error(ctx, BEM_ERR_OOM,
                                      "problem %d (N = %lld) needs %zu bytes, more than the %lld available to a wave",
                                      p, (long long)meshes[p]->N, b, (long long)avail));
            }
            if (n_in > 0 && ((int64_t)(wbytes + b) > avail || n_in == Gmax)) {
                ++w;
                n_in = 0;
                wbytes = 0;
            }
            bt->prob[p].wave = w;
            bt->prob[p].off = wbytes;
            bt->prob[p].bytes = b;
            wbytes += b;
            ++n_in;
            maxw = std::max(maxw, wbytes);
        }
        bt->waves.resize(w + 1);
        for (int p = 0; p < count; ++p) {
            BatchWave &wv = bt->waves[bt->prob[p].wave];
            if (wv.count == 0) wv.first = p;
            ++wv.count;
        }
        bt->arena_bytes = maxw;
        if ((st = dalloc(ctx, bt->allocs, &bt->arena, maxw, false))) return fail(st);
    }
    // operator handles over the arena; far-field tiles timed per size class now (a
    // run may be captured as a graph); cluster orders
    for (int p = 0; p < count && !st; ++p) {
        BatchProblem &pr = bt->prob[p];
        bem_operator *op = new (std::nothrow) bem_operator();
        if (!op) {
            st = set_error(ctx, BEM_ERR_OOM, "host allocation");
            break;
        }
        pr.op = op;
        op->mesh = meshes[p];
        op->ctx = ctx;
        op->precision = prec;
        op->ss_order = ss;
        op->tile = aopts ? aopts->tile : 0;
        op->N = meshes[p]->N;
        op->ld = padded_ld(op->N);
        char *base = static_cast<char *>(bt->arena) + pr.off;
        op->V = base;
        const size_t es = prec == BEM_PREC_F32 ? 4 : 8;
        op->diag = reinterpret_cast<double *>(base + (es * (size_t)op->N * op->ld + 255) / 256 * 256);
        if (op->tile < 0 || op->tile > BEM_FAR_TILE_VARIANTS) {
            st = set_error(ctx, BEM_ERR_INVALID, "tile outside 0..BEM_FAR_TILE_VARIANTS");
            break;
        }
        if ((st = far_tune(op))) break;
        if (block && (st = cluster_setup(op, bt->allocs, &pr.perm, &pr.nbj))) break;
    }
    if (st) return fail(st);
    // per wave: CTA shares, solver arguments, device tables and work lists
    std::vector<int4> items;
    for (size_t wi = 0; wi < bt->waves.size() && !st; ++wi) {
        BatchWave &w = bt->waves[wi];
        const int P = w.count;
        // Groups: the wave's problems by decreasing N, a new group when N^2 falls below
        // half the group's first or the group has as many problems as CTAs can serve
        // (8 per problem that can use them, else what it can use).  Within a group, CTAs
        // per problem in proportion to its bytes per product (N^2; iteration counts are
        // alike), at least one, at most what the single-problem rule can use (a tile per
        // warp, 8 rows per warp), so that the group's problems finish at about the same
        // time; small, latency-bound problems share one launch instead of holding CTAs
        // that the large ones need.
        std::vector<int64_t> want(P);
        for (int k = 0; k < P; ++k) {
            const int64_t N = meshes[w.first + k]->N, nt = bt->prob[w.first + k].nt;
            want[k] = std::min<int64_t>(std::max<int64_t>(std::max<int64_t>((nt + 7) / 8, (N + 63) / 64), 1), Gmax);
        }
        std::vector<int> order(P);
        for (int k = 0; k < P; ++k) order[k] = k;
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return meshes[w.first + a]->N > meshes[w.first + b]->N; });
        std::vector<int> g(P, 1);
        w.groups.clear();
        for (size_t pos = 0; pos < order.size();) {
            BatchGroup gr;
            const int k0 = order[pos];
            const double n0 = (double)meshes[w.first + k0]->N;
            const int per = (int)std::min<int64_t>(want[k0], 8);
            const int cap = std::max(1, Gmax / std::max(per, 1));
            while (pos < order.size() && (int)gr.idx.size() < cap) {
                const int k = order[pos];
                const double n = (double)meshes[w.first + k]->N;
                if (!gr.idx.empty() && 2.0 * n * n < n0 * n0) break;
                gr.idx.push_back(k);
                ++pos;
            }
            const int Pg = (int)gr.idx.size();
            double wsum = 0.0;
            for (int k : gr.idx) wsum += (double)meshes[w.first + k]->N * (double)meshes[w.first + k]->N;
            int gsum = 0;
            for (int k : gr.idx) {
                const double N = (double)meshes[w.first + k]->N;
                const int64_t share = (int64_t)((double)(Gmax - Pg) * N * N / wsum) + 1;
                g[k] = (int)std::min<int64_t>(share, want[k]);
                gsum += g[k];
            }
            while (gsum > Gmax) {  // rounding: take from the largest
                int km = gr.idx[0];
                for (int k : gr.idx)
                    if (g[k] > g[km]) km = k;
                --g[km];
                --gsum;
            }
            gr.count = Pg;
            gr.begin.assign(Pg + 1, 0);
            for (int q = 0; q < Pg; ++q) gr.begin[q + 1] = gr.begin[q] + g[gr.idx[q]];
            gr.G = gr.begin[Pg];
            for (int &k : gr.idx) k += w.first;  // batch indices from here on
            w.groups.push_back(std::move(gr));
        }
        std::vector<BatchSolveProb> sp(P);
        std::vector<BatchAsmProb> ap(P);
        std::vector<int64_t> mpref(P + 1, 0), npref(P + 1, 0);
        int64_t nmax = 0;
        double far_entries = 0.0;
        for (int k = 0; k < P; ++k) {
            const int p = w.first + k;
            BatchProblem &pr = bt->prob[p];
            bem_operator *op = pr.op;
            bem_mesh *m = op->mesh;
            const int64_t N = op->N, L = op->ld;
            nmax = std::max(nmax, N);
            auto al = [](size_t b) { return (b + 255) / 256 * 256; };
            char *cur = static_cast<char *>(bt->arena) + pr.off;
            const size_t es = prec == BEM_PREC_F32 ? 4 : 8;
            cur += al(es * (size_t)N * L) + al(8 * (size_t)N);  // V, diag
            double *vec = reinterpret_cast<double *>(cur);
            cur += al(8 * 7 * (size_t)L);
            float2 *xdf = reinterpret_cast<float2 *>(cur);
            cur += al(8 * (size_t)L);
            float2 *prow = reinterpret_cast<float2 *>(cur);
            float2 *pcol = prow + (size_t)pr.nt * kSB;
            cur += al(2 * (size_t)pr.nt * kSB * 8);
            double *part = reinterpret_cast<double *>(cur);
            const size_t part_bytes = sizeof(double) * (3 * (size_t)g[k] + 8) + 64;
            cur += al(sizeof(double) * (3 * (size_t)Gmax + 8) + 64);
            float *vp = nullptr;
            __half *vh = nullptr;
            float *vsc = nullptr;
            if (packed) {
                vp = reinterpret_cast<float *>(cur);
                cur += al((size_t)pr.nt * kTileF * 4);
                if (bt->h16) {
                    vh = reinterpret_cast<__half *>(cur);
                    cur += al((size_t)pr.nt * kTileF * 2);
                    vsc = reinterpret_cast<float *>(cur);
                    cur += al((size_t)pr.nt * 4);
                }
            }
            double *binv = nullptr;
            if (block) {
                binv = reinterpret_cast<double *>(cur);
                cur += al(8 * (size_t)kBJ * kBJ * (size_t)((N + kBJ - 1) / kBJ));
            }
            PcgArgs &a = bt->args[p];
            a = PcgArgs{};
            a.V = prec == BEM_PREC_DF64 ? (const float2 *)op->V : nullptr;
            a.ld = L;
            a.N = N;
            a.nb = (int)(L / kSB);
            a.ntiles = (int)pr.nt;
            a.tiles = pr.tiles;
            a.prow = prow;
            a.pcol = pcol;
            a.pdf = xdf;
            a.r = vec;
            a.z = vec + L;
            a.p = vec + 2 * L;
            a.q = vec + 3 * L;
            a.b = vec + 4 * L;
            a.x = vec + 5 * L;
            a.d = vec + 6 * L;
            a.part = part;
            double *outp = part + 3 * g[k];
            a.ctr = reinterpret_cast<unsigned long long *>(outp + 4);
            a.bar = reinterpret_cast<unsigned *>(a.ctr + 1);
            a.out = bt->d_res + (size_t)kBatchRes * p;
            a.err = reinterpret_cast<int *>(bt->d_res + (size_t)kBatchRes * p + 6);
            a.vp = vp;
            a.vh = vh;
            a.vsc = vsc;
            a.n16_out = bt->d_res + (size_t)kBatchRes * p + 7;
            a.bperm = pr.perm;
            a.binv = binv;
            a.nbj = pr.nbj;
            a.tol = bt->tol;
            a.f32op = prec == BEM_PREC_F32 ? 1 : 0;
            a.delta2 = a.f32op ? 0.0 : (delta > 0.0 ? delta * delta : 0.0);
            a.max_it = max_it;
            a.precond = precond;
            a.has_x0 = 0;
            a.bar_limit_ns = ctx->bar_limit_ns;
            a.absent_cta = -1;
            BatchSolveProb &q = sp[k];
            q.V = op->V;
            q.ld = L;
            q.N = N;
            q.d = vec + 6 * L;
            q.b = vec + 4 * L;
            q.x = a.x;
            q.area = m->area;
            q.part = part;
            q.part_n = (int64_t)(part_bytes / 8);
            q.vp = prec == BEM_PREC_F32 ? vp : nullptr;
            q.vh = prec == BEM_PREC_F32 ? vh : nullptr;
            q.vsc = vsc;
            q.tiles = pr.tiles;
            q.nt = pr.nt;
            q.perm = pr.perm;
            q.binv = binv;
            q.nbj = pr.nbj;
            q.res = bt->d_res + (size_t)kBatchRes * p;
            w.max_rows = std::max<int64_t>(w.max_rows, std::max<int64_t>(L, q.part_n));
            w.max_nbj = std::max(w.max_nbj, pr.nbj);
            BatchAsmProb &c = ap[k];
            c.q64 = m->q64;
            c.q32 = m->q32;
            c.cent = m->cent;
            c.qdf = m->qdf;
            c.verts = m->verts;
            c.tris = m->tris;
            c.area = m->area;
            c.edge_pairs = m->edge_pairs;
            c.vert_pairs = m->vert_pairs;
            c.n_edge = m->n_edge_pairs;
            c.n_vert = m->n_vert_pairs;
            c.V = op->V;
            c.ld = L;
            c.N = N;
            const int64_t T = (N + 31) / 32;  // 32 x 32 tiles inside the diagonal 64 x 64 blocks
            mpref[k + 1] = mpref[k] + 3 * (T / 2) + (T % 2);
            npref[k + 1] = npref[k] + N + m->n_vert_pairs + m->n_edge_pairs;
            far_entries += 0.5 * (double)N * (double)(N + 1);
        }
        // one far-field tile for the wave: the autotuned one of its largest size class
        // (or the requested one)
        const int tile_req = aopts ? aopts->tile : 0;
        w.variant = tile_req > 0 ? tile_req - 1 : std::max(0, far_cached_variant(ctx, prec, nmax));
        items.clear();
        for (int k = 0; k < P; ++k) batch_far_items(w.variant, k, bt->prob[w.first + k].op->N, items);
        int4 *d_items = nullptr;
        BatchAsmProb *d_ap = nullptr;
        int64_t *d_pref = nullptr;
        for (auto &gr : w.groups) {
            if ((st = dalloc(ctx, bt->allocs, (void **)&gr.d_args, sizeof(PcgArgs) * gr.count, false))) break;
            if ((st = dalloc(ctx, bt->allocs, (void **)&gr.d_begin, sizeof(int) * (gr.count + 1), false))) break;
        }
        if (st) break;
        if ((st = dalloc(ctx, bt->allocs, (void **)&w.d_sprob, sizeof(BatchSolveProb) * P, false))) break;
        if ((st = dalloc(ctx, bt->allocs, (void **)&d_ap, sizeof(BatchAsmProb) * P, false))) break;
        if ((st = dalloc(ctx, bt->allocs, (void **)&d_pref, sizeof(int64_t) * 2 * (P + 1), false))) break;
        if ((st = dalloc(ctx, bt->allocs, (void **)&d_items, sizeof(int4) * std::max<size_t>(items.size(), 1), false)))
            break;
        std::vector<int64_t> prefs(mpref);
        prefs.insert(prefs.end(), npref.begin(), npref.end());
        // on the context's stream, which orders them after the stream-ordered
        // allocations; copies from pageable memory return once the data is staged
        cudaStream_t s = ctx->stream;
        const cudaMemcpyKind h2d = cudaMemcpyHostToDevice;
        cudaError_t e = cudaSuccess;
        std::vector<std::vector<PcgArgs>> gargs(w.groups.size());
        for (size_t gi = 0; gi < w.groups.size() && e == cudaSuccess; ++gi) {
            const BatchGroup &gr = w.groups[gi];
            for (int p : gr.idx) gargs[gi].push_back(bt->args[p]);
            e = cudaMemcpyAsync(gr.d_args, gargs[gi].data(), sizeof(PcgArgs) * gr.count, h2d, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(gr.d_begin, gr.begin.data(), sizeof(int) * (gr.count + 1), h2d, s);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(w.d_sprob, sp.data(), sizeof(BatchSolveProb) * P, h2d, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_ap, ap.data(), sizeof(BatchAsmProb) * P, h2d, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_pref, prefs.data(), sizeof(int64_t) * prefs.size(), h2d, s);
        if (e == cudaSuccess && !items.empty())
            e = cudaMemcpyAsync(d_items, items.data(), sizeof(int4) * items.size(), h2d, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);  // the host tables go out of scope
        if (e != cudaSuccess) {
            st = cuda_error(ctx, e, "batch set-up");
            break;
        }
        for (auto &ev : w.ev)
            if (e == cudaSuccess) e = cudaEventCreate(&ev);
        if (e != cudaSuccess) {
            st = cuda_error(ctx, e, "batch events");
            break;
        }
        w.asmb.P = P;
        w.asmb.precision = prec;
        w.asmb.variant = w.variant;
        w.asmb.ss_order = ss;
        w.asmb.prob = d_ap;
        w.asmb.far_items = d_items;
        w.asmb.n_far = (int64_t)items.size();
        w.asmb.mirror_pref = d_pref;
        w.asmb.n_mirror = mpref[P];
        w.asmb.near_pref = d_pref + (P + 1);
        w.asmb.n_near = npref[P];
        w.asmb.far_entries = far_entries;
    }
    if (!st) {
        cudaError_t e = cudaMallocHost((void **)&bt->h_res, sizeof(double) * kBatchRes * count);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_error(ctx, e, "batch set-up");
    }
    if (st) return fail(st);
    *out = bt;
    return BEM_OK;
}

bem_status bem_batch_run(bem_batch *bt, bem_batch_result *results)
{
    using namespace bem;
    if (!bt) return BEM_ERR_INVALID;
    bem_ctx *ctx = bt->ctx;
    cudaStream_t saved = ctx->stream;
    const int saved_profile = ctx->profile;
    ctx->stream = bt->stream;  // the batch's work runs on its own (capturable) stream
    bem_status st = BEM_OK;
    cudaError_t e = cudaSuccess;
    int replayed = 0;
    for (auto &w : bt->waves) {
        if (bt->use_graph && !w.exec) {
            ctx->profile = 0;  // no profiler events inside a captured graph
            const int64_t l0 = ctx->n_launch;
            e = cudaStreamBeginCapture(bt->stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                st = batch_enqueue(bt, w);
                cudaGraph_t graph = nullptr;
                const cudaError_t e2 = cudaStreamEndCapture(bt->stream, &graph);
                if (!st && e2 == cudaSuccess) {
                    w.graph = graph;
                    e = cudaGraphInstantiate(&w.exec, graph, 0);
                } else {
                    if (graph) cudaGraphDestroy(graph);
                    if (!st) e = e2;
                }
            }
            w.launches = ctx->n_launch - l0;
            ctx->n_launch = l0;
            ctx->profile = saved_profile;
            if (st || e != cudaSuccess) {
                // not capturable here: run the sequence directly from now on
                cudaGetLastError();
                for (auto &x : bt->waves) {
                    if (x.exec) cudaGraphExecDestroy(x.exec);
                    if (x.graph) cudaGraphDestroy(x.graph);
                    x.exec = nullptr;
                    x.graph = nullptr;
                }
                bt->use_graph = 0;
                st = BEM_OK;
                e = cudaSuccess;
            }
        }
        if (bt->use_graph && w.exec) {
            e = cudaGraphLaunch(w.exec, bt->stream);
            ctx->n_launch += w.launches;
            ++replayed;
        } else {
            st = batch_enqueue(bt, w);
        }
        if (st || e != cudaSuccess) break;
    }
    bt->graph_used = replayed == (int)bt->waves.size() ? 1 : 0;
    if (!st && e == cudaSuccess) e = cudaStreamSynchronize(bt->stream);
    ctx->stream = saved;
    ctx->profile = saved_profile;
    if (!st && e != cudaSuccess) st = cuda_error(ctx, e, "batch run");
    if (st) return st;
    bool timeout = false, unconverged = false;
    for (auto &w : bt->waves) {
        double bytes = 0.0;  // algorithmic bytes of the wave's solver launch, as for a single solve
        for (int p = w.first; p < w.first + w.count; ++p) {
            const double *r = bt->h_res + (size_t)kBatchRes * p;
            const double n2 = (double)bt->prob[p].op->N * (double)bt->prob[p].op->N;
            // iterations with the FP16 copy read N^2 bytes (r[7]); DF64 problems also
            // pack it once from the hi parts (2 N^2 read, N^2 written)
            const double i16 = bt->h16 ? r[7] : 0.0;
            bytes += bt->precision == BEM_PREC_F32
                         ? 2.0 * n2 * (r[2] - i16 + r[3]) + n2 * i16
                         : 4.0 * n2 * r[3] + 2.0 * n2 * (r[2] - i16 + 1.0) + n2 * i16 + (bt->h16 ? 3.0 * n2 : 0.0);
            const int err = *reinterpret_cast<const int *>(r + 6);
            const double rel = std::sqrt(r[0] / (r[1] > 0.0 ? r[1] : 1.0));
            timeout |= err != 0;
            unconverged |= !(rel <= bt->tol);
            if (results) {
                bem_batch_result &o = results[p];
                o.cap = r[5];
                o.iterations = (int32_t)r[2];
                o.outer = (int32_t)r[3];
                o.relres = rel;
                o.converged = (err == 0 && rel <= bt->tol) ? 1 : 0;
                o.status = err ? BEM_ERR_CUDA : (rel <= bt->tol ? BEM_OK : BEM_ERR_NOT_CONVERGED);
            }
        }
        if (ctx->profile) {
            // the wave's own events (recorded by direct runs and by graph replays alike)
            float ms[3] = {0.f, 0.f, 0.f};
            for (int k = 0; k < 3; ++k)
                if (cudaEventElapsedTime(&ms[k], w.ev[2 * k], w.ev[2 * k + 1]) != cudaSuccess) {
                    cudaGetLastError();
                    ms[k] = 0.f;
                }
            const double units[3] = {w.asmb.far_entries, (double)w.asmb.n_near, bytes};
            const int kinds[3] = {BEM_KERNEL_FAR, BEM_KERNEL_NEAR, BEM_KERNEL_MATVEC};
            for (int k = 0; k < 3; ++k) {
                ctx->prof_launches[kinds[k]] += 1;
                ctx->prof_ms[kinds[k]] += ms[k];
                ctx->prof_units[kinds[k]] += units[k];
            }
        }
    }
    if (timeout) return set_error(ctx, BEM_ERR_CUDA, "batch solve: a grid barrier timed out");
    if (unconverged) return set_error(ctx, BEM_ERR_NOT_CONVERGED, "batch solve: a problem did not reach the tolerance");
    return BEM_OK;
}

bem_status bem_batch_info(const bem_batch *bt, int32_t *count, int32_t *ctas, int32_t *graph_used)
{
    if (!bt) return BEM_ERR_INVALID;
    if (count) *count = bt->P;
    if (ctas) {
        int g = 0;
        for (const auto &w : bt->waves)
            for (const auto &gr : w.groups) g = std::max(g, gr.G);
        *ctas = g;
    }
    if (graph_used) *graph_used = bt->graph_used;
    return BEM_OK;
}

bem_status bem_batch_waves(const bem_batch *bt, int32_t *waves, int64_t *arena_bytes, int32_t *wave_of)
{
    if (!bt) return BEM_ERR_INVALID;
    if (waves) *waves = (int32_t)bt->waves.size();
    if (arena_bytes) *arena_bytes = (int64_t)bt->arena_bytes;
    if (wave_of)
        for (int p = 0; p < bt->P; ++p) wave_of[p] = bt->prob[p].wave;
    return BEM_OK;
}

bem_status bem_batch_destroy(bem_batch *bt)
{
    using namespace bem;
    if (!bt) return BEM_ERR_INVALID;
    bem_ctx *ctx = bt->ctx;
    if (bt->stream) cudaStreamSynchronize(bt->stream);
    for (auto &w : bt->waves) {
        if (w.exec) cudaGraphExecDestroy(w.exec);
        if (w.graph) cudaGraphDestroy(w.graph);
        for (auto &ev : w.ev)
            if (ev) cudaEventDestroy(ev);
    }
    for (auto &pr : bt->prob)
        if (pr.op) bem_operator_destroy(pr.op);  // the handles own no memory: V lives in the arena
    dfree_all(ctx, bt->allocs);
    cudaStreamSynchronize(ctx->stream);
    if (bt->h_res) cudaFreeHost(bt->h_res);
    if (bt->stream) cudaStreamDestroy(bt->stream);
    delete bt;
    return BEM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ no-allocation product
// Some callers cannot let a library allocate device memory in the middle of a
// call: code that is being captured into a CUDA graph (cudaMalloc and cudaFree
// are not permitted during stream capture), serving loops that run inside a fixed,
// pre-reserved memory footprint, and hosts whose device memory is owned by another
// framework's allocator.  For them bem_operator_matvec_noalloc computes the same
// symmetric double-float product as bem_operator_matvec, with its scratch in the
// static device array below instead of in allocated buffers.
namespace bem {

constexpr int64_t kNoAllocMaxN = 4096;  // largest operator accepted
// padded_ld(N) <= kNoAllocMaxN for every N <= kNoAllocMaxN only if the limit is a
// whole number of tiles (rows are padded to 64 entries, one tile side)
static_assert(kNoAllocMaxN % kSB == 0, "the no-allocation limit must be a multiple of the tile side");
static_assert(kSB == 64, "rows are padded to 64 entries (padded_ld): one tile side");
constexpr int kNoAllocNb = (int)(kNoAllocMaxN / kSB);
constexpr int64_t kNoAllocTiles = (int64_t)kNoAllocNb * (kNoAllocNb + 1) / 2;
constexpr size_t kNoAllocXBytes = (size_t)kNoAllocMaxN * sizeof(float2);           // x as hi/lo pairs
constexpr size_t kNoAllocPartBytes = (size_t)kNoAllocTiles * kSB * sizeof(float2);  // row (or column) partials
constexpr size_t kNoAllocBytes = kNoAllocXBytes + 2 * kNoAllocPartBytes + kNoAllocTiles * sizeof(int2);

// Every GPU that loads the library holds this array (about 2.1 MiB) until exit.
// Each call writes every word it reads, so nothing has to start at zero; calls
// that overlap on the GPU (other streams, other threads) share it and race.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Device address of the array, per device: looked up once per device under
// std::call_once (slot threads of a server may make their first calls at once).
// A device reset (cudaDeviceReset) invalidates the cached address: the library
// does not support calls after one.
constexpr int kNoAllocDevices = 64;
static std::once_flag g_noalloc_once[kNoAllocDevices];
static void *g_noalloc_addr[kNoAllocDevices] = {nullptr};
static cudaError_t g_noalloc_err[kNoAllocDevices] = {cudaSuccess};

}  // namespace bem

extern "C" bem_status bem_operator_matvec_noalloc(const bem_operator *op, const double *x, double *y)
{
    using namespace bem;
    if (!op) return BEM_ERR_INVALID;
    bem_ctx *ctx = op->mesh->ctx;
    if (op->precision != BEM_PREC_DF64)
        return set_error(ctx, BEM_ERR_INVALID, "bem_operator_matvec_noalloc needs a BEM_PREC_DF64 operator");
    if (op->N > kNoAllocMaxN)
        return set_error(ctx, BEM_ERR_INVALID,
                         "operator size N = %lld exceeds the no-allocation limit N <= %lld; use bem_operator_matvec",
                         (long long)op->N, (long long)kNoAllocMaxN);
    if (op->ld > kNoAllocMaxN)
        return set_error(ctx, BEM_ERR_INVALID, "padded row length %lld exceeds the no-allocation limit %lld",
                         (long long)op->ld, (long long)kNoAllocMaxN);
    int xdev = -1, ydev = -1;
    if (!x || !y || !is_device_ptr(x, &xdev) || !is_device_ptr(y, &ydev))
        return set_error(ctx, BEM_ERR_INVALID,
                         "x and y must be device pointers (host arrays would need staging buffers)");
    // plain device memory must sit on the context's device (a peer pointer would be
    // read by the kernels directly, without a copy); managed memory is reachable
    if ((xdev >= 0 && xdev != ctx->device) || (ydev >= 0 && ydev != ctx->device))
        return set_error(ctx, BEM_ERR_INVALID, "x and y must be memory of the context's device (%d)", ctx->device);
    int dev = -1;
    BEM_CK(ctx, cudaGetDevice(&dev));
    if (dev != ctx->device || dev < 0 || dev >= kNoAllocDevices)
        return set_error(ctx, BEM_ERR_INVALID, "call with the context's device (%d) current", ctx->device);
    // set-up on the first call on this device: the host-side name of the array is
    // not a device address, so ask the runtime for it (with this device current)
    std::call_once(g_noalloc_once[dev], [dev] {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        g_noalloc_err[dev] = (e == cudaSuccess && !p) ? cudaErrorInvalidSymbol : e;
        if (e != cudaSuccess) cudaGetLastError();
        g_noalloc_addr[dev] = e == cudaSuccess ? p : nullptr;
    });
    if (g_noalloc_err[dev] != cudaSuccess || !g_noalloc_addr[dev])
        return cuda_error(ctx, g_noalloc_err[dev], "cudaGetSymbolAddress of the no-allocation scratch");
    unsigned char *base = static_cast<unsigned char *>(g_noalloc_addr[dev]);
    float2 *xdf = reinterpret_cast<float2 *>(base);
    float2 *prow = reinterpret_cast<float2 *>(base + kNoAllocXBytes);
    float2 *pcol = reinterpret_cast<float2 *>(base + kNoAllocXBytes + kNoAllocPartBytes);
    int2 *tiles = reinterpret_cast<int2 *>(base + kNoAllocXBytes + 2 * kNoAllocPartBytes);
    const int nb = (int)(op->ld / kSB);
    const int ntiles = nb * (nb + 1) / 2;
    cudaStream_t s = ctx->stream;
    k_tile_list<<<nb, 128, 0, s>>>(nb, tiles); BEM_COUNT(ctx);
    k_to_df<<<nblk(op->ld, 256), 256, 0, s>>>(x, op->N, op->ld, xdf); BEM_COUNT(ctx);
    BEM_CK(ctx, cudaFuncSetAttribute(k_symv_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSymSmem));
    const int grid = ntiles < 3 * ctx->sm_count ? ntiles : 3 * ctx->sm_count;
    k_symv_df<<<grid, kSymThreads, kSymSmem, s>>>((const float2 *)op->V, op->ld, op->N, nb, tiles, ntiles, xdf, prow,
                                                  pcol); BEM_COUNT(ctx);
    k_symv_reduce<<<nblk(op->N, kVecThreads), kVecThreads, 0, s>>>(prow, pcol, nb, op->N, y, nullptr, nullptr); BEM_COUNT(ctx);
    BEM_CK_LAUNCH(ctx);
    return BEM_OK;
}
