// Adaptive steps of Alg. 1 on the device: ZZ-type estimate (Eq. 1.6), Doerfler
// marking (Eq. 2.6) and newest-vertex bisection with closure (Fig. 3).
//
// Compiled with -fmad=false: every product and sum of the estimator is rounded
// separately in the order written, so the indicators, and the decisions taken
// from them, are bit-identical to a plain IEEE-754 evaluation of the same
// formulas.
#include <algorithm>
#include <cmath>
#include <new>
#include <type_traits>

#include "bem_internal.cuh"

namespace bem {

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

// ------------------------------------------------------------------ ZZ estimate
// u_z = sum_{T at z} |T| x_T / sum_{T at z} |T|, triangles in ascending order.
__global__ void k_zz_nodal(const int32_t *off, const int32_t *v2t, const double *area, const double *x,
                           double *u, int64_t M)
{
    const int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= M) return;
    double num = 0.0, den = 0.0;
    for (int32_t p = off[z]; p < off[z + 1]; ++p) {
        const int32_t t = v2t[p];
        const double ax = area[t] * x[t];
        num = num + ax;
        den = den + area[t];
    }
    u[z] = den > 0.0 ? num / den : 0.0;
}

// eta(T)^2 = (h |T| / 12) (sum d_k^2 + (sum d_k)^2), d_k = u_{z_k} - x_T; block
// partials of the total and of sum h|T| x_T^2 / 12.
__global__ void k_zz_eta(const int32_t *tris, const double *area, const double *diam, const double *x,
                         const double *u, int64_t N, int h_mode, double *eta2, double *part_eta, double *part_scale)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0, sc = 0.0;
    if (t < N) {
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = u[tris[3 * t + k]] - x[t];
        const double s2 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2];
        const double s1 = (d[0] + d[1]) + d[2];
        const double q = s2 + s1 * s1;
        const double h = h_mode == 1 ? sqrt(area[t]) : diam[t];
        const double f = (h * area[t]) / 12.0;
        e = f * q;
        sc = f * (x[t] * x[t]);
        eta2[t] = e;
    }
    __shared__ double se[256], ss[256];
    se[threadIdx.x] = e;
    ss[threadIdx.x] = sc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            se[threadIdx.x] += se[threadIdx.x + o];
            ss[threadIdx.x] += ss[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part_eta[blockIdx.x] = se[0];
        part_scale[blockIdx.x] = ss[0];
    }
}

__global__ void k_sum2(const double *a, const double *b, int n, double *out)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0, t = 0.0;
        for (int k = 0; k < n; ++k) {
            s += a[k];
            t += b[k];
        }
        out[0] = s;
        out[1] = t;
    }
}

bem_status zz_estimate(bem_mesh *m, const double *d_phi, int h_mode, double *d_eta2, double *h_totals,
                       double *d_totals)
{
    bem_ctx *ctx = m->ctx;
    cudaStream_t s = ctx->stream;
    Allocs tmp;
    double *u = nullptr;
    const int nb = (int)nblk(m->N, 256);
    bem_status st = dalloc(ctx, tmp, (void **)&u, sizeof(double) * (m->M + 2 * nb + 2), false);
    if (st) return st;
    double *pe = u + m->M, *ps = pe + nb, *tot = d_totals ? d_totals : ps + nb;
    k_zz_nodal<<<nblk(m->M, 128), 128, 0, s>>>(m->v2t_off, m->v2t, m->area, d_phi, u, m->M); BEM_COUNT(ctx);
    k_zz_eta<<<nb, 256, 0, s>>>(m->tris, m->area, m->diam, d_phi, u, m->N, h_mode, d_eta2, pe, ps); BEM_COUNT(ctx);
    k_sum2<<<1, 32, 0, s>>>(pe, ps, nb, tot); BEM_COUNT(ctx);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_error(ctx, e, "zz kernels");
    if (!st && h_totals) {
        e = cudaMemcpyAsync(ctx->h_pinned, tot, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(ctx, e, "zz totals");
        else {
            h_totals[0] = ctx->h_pinned[0];
            h_totals[1] = ctx->h_pinned[1];
        }
    }
    dfree_all(ctx, tmp);
    return st;
}

// ------------------------------------------------------------------ Doerfler
// key = (~float_bits(eta2) << 32) | index: ascending key order = descending
// single-precision indicator, ties by index.
__global__ void k_keys(const double *eta2, int64_t N, int64_t n2, unsigned long long *keys)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n2) return;
    if (i < N) {
        const float f = __double2float_rn(eta2[i]);
        const unsigned int bits = __float_as_uint(f);
        keys[i] = ((unsigned long long)(0xFFFFFFFFu - bits) << 32) | (unsigned long long)(uint32_t)i;
    } else {
        keys[i] = ~0ull;
    }
}

__device__ __forceinline__ void cmp_swap(unsigned long long *keys, int64_t i, int64_t l, bool asc)
{
    const unsigned long long a = keys[i], b = keys[l];
    if ((a > b) == asc) {
        keys[i] = b;
        keys[l] = a;
    }
}

// One bitonic stage (k, j) over all n2/2 pairs.
__global__ void k_bitonic_global(unsigned long long *keys, int64_t n2, int64_t k, int64_t j)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n2 / 2) return;
    const int64_t i = ((t & ~(j - 1)) << 1) | (t & (j - 1));  // 2 j (t / j) + t % j, j a power of two
    cmp_swap(keys, i, i + j, (i & k) == 0);
}

// Stages j = j0, j0/2, ..., 1 of step k inside chunks of 2 * blockDim.x keys.
__global__ void k_bitonic_shared(unsigned long long *keys, int64_t n2, int64_t k, int64_t j0)
{
    extern __shared__ unsigned long long sk[];
    const int chunk = 2 * blockDim.x;
    const int64_t base = (int64_t)blockIdx.x * chunk;
    for (int q = threadIdx.x; q < chunk; q += blockDim.x) sk[q] = keys[base + q];
    __syncthreads();
    for (int64_t j = j0; j >= 1; j >>= 1) {
        const int t = threadIdx.x;
        const int i = (int)(((t & ~(j - 1)) << 1) | (t & (j - 1)));  // j a power of two
        const bool asc = ((base + i) & k) == 0;
        const unsigned long long a = sk[i], b = sk[i + j];
        if ((a > b) == asc) {
            sk[i] = b;
            sk[i + j] = a;
        }
        __syncthreads();
    }
    for (int q = threadIdx.x; q < chunk; q += blockDim.x) keys[base + q] = sk[q];
}

// The whole bitonic network of n2 <= kSortBlockMax keys in one CTA's shared memory
// (one launch instead of one per stage for the arrays of the first adaptive levels);
// the keys are unique, so the result is the array the per-stage kernels produce.
constexpr int64_t kSortBlockMax = 16384;  // 128 KB of shared memory
constexpr int kSortBlockThreads = 1024;

__global__ void __launch_bounds__(kSortBlockThreads) k_bitonic_block(unsigned long long *keys, int64_t n2)
{
    extern __shared__ unsigned long long sk[];
    const int n = (int)n2, half = n / 2;
    for (int q = threadIdx.x; q < n; q += blockDim.x) sk[q] = keys[q];
    __syncthreads();
    for (int k = 2; k <= n; k <<= 1)
        for (int j = k >> 1; j >= 1; j >>= 1) {
            for (int t = threadIdx.x; t < half; t += blockDim.x) {
                const int i = ((t & ~(j - 1)) << 1) | (t & (j - 1));  // 2 j (t / j) + t % j
                const bool asc = (i & k) == 0;
                const unsigned long long a = sk[i], b = sk[i + j];
                if ((a > b) == asc) {
                    sk[i] = b;
                    sk[i + j] = a;
                }
            }
            __syncthreads();
        }
    for (int q = threadIdx.x; q < n; q += blockDim.x) keys[q] = sk[q];
}

// Running FP64 sums of eta2 in key order, in a fixed two-level order: the sorted
// sequence is cut into blocks of kDorflerBlock; l = the running sum inside a block
// (from 0, left to right), o_b = the offset of block b (o_0 = 0, o_(b+1) = o_b +
// the block's full sum), and prefix[k] = o_b + l for k in block b.  The marking
// rule (Eq. 2.6) fixes no order; this one is the oracle's, addition for addition, and
// its chains are 128 (blocks, in parallel) plus N / 128 (offsets) additions long
// instead of N.
constexpr int kDorflerBlock = 128;

// One thread per block: the running sums inside the block and the block's sum.
__global__ void k_dorfler_blocks(const unsigned long long *__restrict__ keys, const double *__restrict__ eta2,
                                 int64_t N, double *__restrict__ prefix, double *__restrict__ bsum)
{
    const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b0 = b * kDorflerBlock;
    if (b0 >= N) return;
    const int n = (int)((N - b0) < kDorflerBlock ? (N - b0) : kDorflerBlock);
    double l = 0.0;
    int q = 0;
    for (; q + 16 <= n; q += 16) {  // loads of a group issued before its additions
        double r[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) r[u] = eta2[keys[b0 + q + u] & 0xFFFFFFFFull];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            l = l + r[u];
            prefix[b0 + q + u] = l;
        }
    }
    for (; q < n; ++q) {
        l = l + eta2[keys[b0 + q] & 0xFFFFFFFFull];
        prefix[b0 + q] = l;
    }
    bsum[b] = l;
}

// The block offsets, by one thread: off[0] = 0, off[b + 1] = off[b] + bsum[b].
__global__ void k_dorfler_offsets(const double *__restrict__ bsum, int64_t nb, double *__restrict__ off)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double o = 0.0;
    off[0] = 0.0;
    for (int64_t b = 0; b < nb; ++b) {
        o = o + bsum[b];
        off[b + 1] = o;
    }
}

// prefix[k] = off[block of k] + (running sum inside the block).
__global__ void k_dorfler_finish(const double *__restrict__ off, int64_t N, double *__restrict__ prefix)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) prefix[k] = off[k / kDorflerBlock] + prefix[k];
}

// The shortest prefix whose running sum reaches theta * total (total = prefix[N-1];
// none if theta * total <= 0), by bisection over the non-decreasing prefix sums,
// then extended over equal keys.
__global__ void k_dorfler_select(const unsigned long long *keys, const double *prefix, int64_t N, double theta,
                                 const double *vanish, long long *K_out)
{
    // vanish (nullable): [sum eta^2, sum h|T|x^2/12]; when every indicator vanishes up
    // to rounding (sum eta^2 <= 1e-20 of the scale) Eq. 2.6 holds for the empty set and
    // every element is marked (uniform refinement)
    if (vanish && !(vanish[0] > 1e-20 * vanish[1])) {
        *K_out = N;
        return;
    }
    const double thr = theta * prefix[N - 1];
    int64_t kk = 0;
    if (0.0 < thr) {
        int64_t lo = 0, hi = N - 1;  // prefix[hi] >= thr
        if (!(prefix[hi] >= thr)) lo = hi = N;
        while (lo < hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            if (prefix[mid] >= thr)
                hi = mid;
            else
                lo = mid + 1;
        }
        kk = lo < N ? lo + 1 : N;
    }
    while (kk > 0 && kk < N && (keys[kk] >> 32) == (keys[kk - 1] >> 32)) ++kk;
    *K_out = kk;
}

__global__ void k_mark(const unsigned long long *keys, int64_t N, const long long *K, uint8_t *marked)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    marked[keys[k] & 0xFFFFFFFFull] = (k < *K) ? 1 : 0;
}

void sort_u64(bem_ctx *ctx, unsigned long long *keys, int64_t n2)
{
    cudaStream_t s = ctx->stream;
    if (n2 <= kSortBlockMax) {
        const size_t smem = sizeof(unsigned long long) * (size_t)n2;
        bool ok = true;  // shared memory beyond 48 KB needs the opt-in
        if (smem > 48 * 1024 && cudaFuncSetAttribute(k_bitonic_block, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                     (int)(sizeof(unsigned long long) * kSortBlockMax)) != cudaSuccess) {
            cudaGetLastError();
            ok = false;
        }
        if (ok) {
            const int threads = (int)std::min<int64_t>(kSortBlockThreads, std::max<int64_t>(n2 / 2, 32));
            k_bitonic_block<<<1, threads, smem, s>>>(keys, n2); BEM_COUNT(ctx);
            return;
        }
    }
    const int64_t chunk = n2 < 2048 ? n2 : 2048;
    const int sthreads = (int)(chunk / 2);
    for (int64_t k = 2; k <= n2; k <<= 1) {
        int64_t j = k >> 1;
        for (; j >= chunk; j >>= 1)
            { k_bitonic_global<<<nblk(n2 / 2, 256), 256, 0, s>>>(keys, n2, k, j); BEM_COUNT(ctx); }
        k_bitonic_shared<<<(unsigned)(n2 / chunk), sthreads, chunk * sizeof(unsigned long long), s>>>(keys, n2, k, j); BEM_COUNT(ctx);
    }
}

bem_status dorfler(bem_ctx *ctx, const double *d_eta2, int64_t N, double theta, uint8_t *d_marked,
                   int64_t *n_marked, const double *d_vanish, long long *d_count)
{
    if (N <= 0) {
        if (n_marked) *n_marked = 0;
        if (d_count) BEM_CK(ctx, cudaMemsetAsync(d_count, 0, sizeof(long long), ctx->stream));
        return BEM_OK;
    }
    if (N > 0x7FFFFFFFLL) return set_error(ctx, BEM_ERR_INVALID, "too many elements for marking");
    cudaStream_t s = ctx->stream;
    int64_t n2 = 1;
    while (n2 < N) n2 <<= 1;
    if (n2 < 2) n2 = 2;
    Allocs tmp;
    unsigned long long *keys = nullptr;
    const int64_t nb = (N + kDorflerBlock - 1) / kDorflerBlock;
    bem_status st = dalloc(ctx, tmp, (void **)&keys,
                           sizeof(unsigned long long) * n2 + sizeof(double) * (N + 2 * nb + 1) + 64, false);
    if (st) return st;
    double *prefix = reinterpret_cast<double *>(keys + n2);
    double *bsum = prefix + N, *off = bsum + nb;
    long long *dK = reinterpret_cast<long long *>(off + nb + 1);
    k_keys<<<nblk(n2, 256), 256, 0, s>>>(d_eta2, N, n2, keys); BEM_COUNT(ctx);
    sort_u64(ctx, keys, n2);
    k_dorfler_blocks<<<nblk(nb, 64), 64, 0, s>>>(keys, d_eta2, N, prefix, bsum); BEM_COUNT(ctx);
    k_dorfler_offsets<<<1, 32, 0, s>>>(bsum, nb, off); BEM_COUNT(ctx);
    k_dorfler_finish<<<nblk(N, 256), 256, 0, s>>>(off, N, prefix); BEM_COUNT(ctx);
    k_dorfler_select<<<1, 1, 0, s>>>(keys, prefix, N, theta, d_vanish, dK); BEM_COUNT(ctx);
    k_mark<<<nblk(N, 256), 256, 0, s>>>(keys, N, dK, d_marked); BEM_COUNT(ctx);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && d_count) e = cudaMemcpyAsync(d_count, dK, sizeof(long long), cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) st = cuda_error(ctx, e, "doerfler kernels");
    if (!st && n_marked) {
        e = cudaMemcpyAsync(ctx->h_pinned, dK, sizeof(long long), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(ctx, e, "doerfler count");
        else *n_marked = *reinterpret_cast<long long *>(ctx->h_pinned);
    }
    dfree_all(ctx, tmp);
    return st;
}

// ------------------------------------------------------------------ NVB
__global__ void k_nvb_seed(const int32_t *owner, const uint8_t *marked, int64_t N, int bisec3, uint8_t *flag)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N || !marked[t]) return;
    flag[owner[3 * t]] = 1;
    if (bisec3) {
        flag[owner[3 * t + 1]] = 1;
        flag[owner[3 * t + 2]] = 1;
    }
}

// One closure sweep: a triangle with a marked edge marks its reference edge.
// The closure to its fixed point in one CTA (meshes up to kCloseBlockMax triangles):
// sweeps until one changes nothing.  Flags only go from 0 to 1, so the fixed point
// (the least closed set containing the seeds) does not depend on the order of the
// updates; each sweep that changes something sets at least one of the 3N flags, so
// 3N + 1 sweeps always reach it.
constexpr int64_t kCloseBlockMax = 65536;

__global__ void __launch_bounds__(1024) k_nvb_close_block(const int32_t *owner, int64_t N, uint8_t *flag)
{
    __shared__ int changed;
    for (int64_t sweep = 0; sweep <= 3 * N; ++sweep) {
        if (threadIdx.x == 0) changed = 0;
        __syncthreads();
        int c = 0;
        for (int64_t t = threadIdx.x; t < N; t += blockDim.x) {
            const int32_t o0 = owner[3 * t];
            if (!flag[o0] && (flag[owner[3 * t + 1]] | flag[owner[3 * t + 2]])) {
                flag[o0] = 1;
                c = 1;
            }
        }
        if (c) changed = 1;
        __syncthreads();
        const int done = !changed;
        __syncthreads();  // every thread has read changed before thread 0 clears it
        if (done) return;
    }
}

__global__ void k_nvb_close(const int32_t *owner, int64_t N, uint8_t *flag, int32_t *changed)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const int32_t o0 = owner[3 * t];
    if (!flag[o0] && (flag[owner[3 * t + 1]] | flag[owner[3 * t + 2]])) {
        flag[o0] = 1;
        *changed = 1;
    }
}

// Per half-edge: 1 if it owns a marked edge (a new vertex).  Per triangle: kept
// flag and number of children.
__global__ void k_nvb_counts(const int32_t *owner, const uint8_t *flag, int64_t N, int32_t *is_new,
                             int32_t *is_kept, int32_t *n_child)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    for (int k = 0; k < 3; ++k) {
        const int64_t h = 3 * t + k;
        is_new[h] = (owner[h] == h && flag[h]) ? 1 : 0;
    }
    const int f0 = flag[owner[3 * t]], f1 = flag[owner[3 * t + 1]], f2 = flag[owner[3 * t + 2]];
    is_kept[t] = f0 ? 0 : 1;
    n_child[t] = f0 ? 2 + f1 + f2 : 0;
}

__global__ void k_nvb_verts(const double *V, const int32_t *tris, const int32_t *owner, const uint8_t *flag,
                            const int32_t *new_pos, int64_t N, int64_t M, double *Vn)
{
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= 3 * N || owner[h] != h || !flag[h]) return;
    const int64_t t = h / 3;
    const int k = (int)(h % 3);
    const int32_t a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
    const int64_t m = M + new_pos[h];
    for (int c = 0; c < 3; ++c) Vn[3 * m + c] = 0.5 * (V[3 * (int64_t)a + c] + V[3 * (int64_t)b + c]);
}

__global__ void k_nvb_tris(const int32_t *tris, const int32_t *owner, const uint8_t *flag, const int32_t *new_pos,
                           const int32_t *kept_pos, const int32_t *child_pos, int64_t n_kept, int64_t N, int64_t M,
                           int32_t *Tn, int32_t *parent, uint8_t *kept)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const int32_t a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
    const int32_t o0 = owner[3 * t], o1 = owner[3 * t + 1], o2 = owner[3 * t + 2];
    const int f0 = flag[o0], f1 = flag[o1], f2 = flag[o2];
    if (!f0) {
        const int64_t p = kept_pos[t];
        Tn[3 * p] = a;
        Tn[3 * p + 1] = b;
        Tn[3 * p + 2] = c;
        parent[p] = (int32_t)t;
        kept[p] = 1;
        return;
    }
    const int32_t m0 = (int32_t)(M + new_pos[o0]);
    const int32_t m1 = f1 ? (int32_t)(M + new_pos[o1]) : -1;
    const int32_t m2 = f2 ? (int32_t)(M + new_pos[o2]) : -1;
    int32_t ch[4][3];
    int nc;
    if (!f1 && !f2) {
        const int32_t L[2][3] = {{c, a, m0}, {b, c, m0}};
        memcpy(ch, L, sizeof(L));
        nc = 2;
    } else if (f1 && !f2) {
        const int32_t L[3][3] = {{c, a, m0}, {m0, b, m1}, {c, m0, m1}};
        memcpy(ch, L, sizeof(L));
        nc = 3;
    } else if (!f1 && f2) {
        const int32_t L[3][3] = {{m0, c, m2}, {a, m0, m2}, {b, c, m0}};
        memcpy(ch, L, sizeof(L));
        nc = 3;
    } else {
        const int32_t L[4][3] = {{m0, c, m2}, {a, m0, m2}, {m0, b, m1}, {c, m0, m1}};
        memcpy(ch, L, sizeof(L));
        nc = 4;
    }
    const int64_t base = n_kept + child_pos[t];
    for (int r = 0; r < nc; ++r) {
        for (int q = 0; q < 3; ++q) Tn[3 * (base + r) + q] = ch[r][q];
        parent[base + r] = (int32_t)t;
        kept[base + r] = 0;
    }
}

bem_status refine(bem_mesh *m, const uint8_t *d_marked, int flags, bem_mesh **out, bool defer_check)
{
    bem_ctx *ctx = m->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t N = m->N, M = m->M, H = 3 * N;
    Allocs tmp;
    bem_mesh *r = nullptr;
    bem_status st = BEM_OK;
    uint8_t *flag = nullptr;
    int32_t *is_new = nullptr, *new_pos = nullptr, *is_kept = nullptr, *kept_pos = nullptr, *n_child = nullptr,
            *child_pos = nullptr, *changed = nullptr;
    int64_t n_new = 0, n_kept = 0, n_children = 0;
#define TRY(x)             \
    do {                   \
        st = (x);          \
        if (st) goto fail; \
    } while (0)
    TRY(dalloc(ctx, tmp, (void **)&flag, H + 16, true));
    TRY(dalloc(ctx, tmp, (void **)&changed, sizeof(int32_t) * 4, true));
    TRY(dalloc(ctx, tmp, (void **)&is_new, sizeof(int32_t) * (H + 1), false));
    TRY(dalloc(ctx, tmp, (void **)&new_pos, sizeof(int32_t) * (H + 1), false));
    TRY(dalloc(ctx, tmp, (void **)&is_kept, sizeof(int32_t) * (N + 1), false));
    TRY(dalloc(ctx, tmp, (void **)&kept_pos, sizeof(int32_t) * (N + 1), false));
    TRY(dalloc(ctx, tmp, (void **)&n_child, sizeof(int32_t) * (N + 1), false));
    TRY(dalloc(ctx, tmp, (void **)&child_pos, sizeof(int32_t) * (N + 1), false));
    k_nvb_seed<<<nblk(N, 256), 256, 0, s>>>(m->owner, d_marked, N, flags & BEM_REFINE_BISEC3, flag); BEM_COUNT(ctx);
    // closure: in one CTA for meshes up to kCloseBlockMax triangles; larger ones by
    // sweeps over the grid, eight per check of the changed flag (a sweep after the
    // fixed point changes nothing; a level's closure rarely needs more than eight)
    if (N <= kCloseBlockMax) {
        k_nvb_close_block<<<1, 1024, 0, s>>>(m->owner, N, flag); BEM_COUNT(ctx);
    }
    for (int sweep = 0; N > kCloseBlockMax; sweep += 8) {
        if (sweep > 100000) {
            st = set_error(ctx, BEM_ERR_MESH, "NVB closure did not terminate");
            goto fail;
        }
        if (cudaMemsetAsync(changed, 0, sizeof(int32_t), s) != cudaSuccess) {
            st = set_error(ctx, BEM_ERR_CUDA, "closure flag reset");
            goto fail;
        }
        for (int k = 0; k < 8; ++k)
            { k_nvb_close<<<nblk(N, 256), 256, 0, s>>>(m->owner, N, flag, changed); BEM_COUNT(ctx); }
        cudaError_t e = cudaMemcpyAsync(ctx->h_pinned, changed, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            st = cuda_error(ctx, e, "closure sweep");
            goto fail;
        }
        if (*reinterpret_cast<int32_t *>(ctx->h_pinned) == 0) break;
    }
    k_nvb_counts<<<nblk(N, 256), 256, 0, s>>>(m->owner, flag, N, is_new, is_kept, n_child); BEM_COUNT(ctx);
    TRY(exclusive_scan_i32(ctx, is_new, new_pos, H, nullptr));
    TRY(exclusive_scan_i32(ctx, is_kept, kept_pos, N, nullptr));
    TRY(exclusive_scan_i32(ctx, n_child, child_pos, N, nullptr));
    {  // the three totals in one read, with the source mesh's deferred checks
        const bool chk = m->bad_pending != 0;
        const int32_t *src[6] = {new_pos + H, kept_pos + N, child_pos + N, nullptr, nullptr, nullptr};
        if (chk) {
            src[3] = m->d_bad + 1;
            src[4] = m->d_bad + 2;
            src[5] = m->d_bad + 3;
        }
        int64_t tot[6] = {0, 0, 0, 0, 0, 0};
        TRY(read_i32s(ctx, src, chk ? 6 : 3, tot));
        if (chk) {
            m->bad_pending = 0;
            TRY(mesh_bad_status(ctx, tot + 3));
        }
        n_new = tot[0];
        n_kept = tot[1];
        n_children = tot[2];
    }
    r = new bem_mesh();
    r->ctx = ctx;
    r->M = M + n_new;
    r->N = n_kept + n_children;
    r->n_kept = n_kept;
    r->src_N = N;
    if (r->M > 0x7FFFFFFFLL || r->N > 0x7FFFFFFFLL) {
        st = set_error(ctx, BEM_ERR_INVALID, "refined mesh exceeds 2^31 entries");
        goto fail;
    }
    TRY(dalloc(ctx, r->allocs, (void **)&r->verts, sizeof(double) * 3 * r->M, false));
    TRY(dalloc(ctx, r->allocs, (void **)&r->tris, sizeof(int32_t) * 3 * r->N, false));
    TRY(dalloc(ctx, r->allocs, (void **)&r->parent, sizeof(int32_t) * r->N, false));
    TRY(dalloc(ctx, r->allocs, (void **)&r->kept, r->N + 16, false));
    if (cudaMemcpyAsync(r->verts, m->verts, sizeof(double) * 3 * M, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        st = set_error(ctx, BEM_ERR_CUDA, "copy vertices");
        goto fail;
    }
    k_nvb_verts<<<nblk(H, 256), 256, 0, s>>>(m->verts, m->tris, m->owner, flag, new_pos, N, M, r->verts); BEM_COUNT(ctx);
    k_nvb_tris<<<nblk(N, 256), 256, 0, s>>>(m->tris, m->owner, flag, new_pos, kept_pos, child_pos, n_kept, N, M,
                                            r->tris, r->parent, r->kept); BEM_COUNT(ctx);
    if (cudaGetLastError() != cudaSuccess) {
        st = set_error(ctx, BEM_ERR_CUDA, "refinement kernels");
        goto fail;
    }
    TRY(mesh_build(r, false, nullptr, defer_check));
    dfree_all(ctx, tmp);
    *out = r;
    return BEM_OK;
fail:
#undef TRY
    if (r) {
        dfree_all(ctx, r->allocs);
        delete r;
    }
    dfree_all(ctx, tmp);
    return st;
}

}  // namespace bem

// ------------------------------------------------------------------ dual basis (Sec. 2.1, 2.6)
namespace bem {

// Barycentric refinement: vertices = the old ones, the edge midpoints 0.5 (a + b)
// numbered by the first appearance of their edge in (triangle, local edge) order (the
// owner half-edge), then the centroids ((v0 + v1) + v2) / 3; children of T at 6T .. 6T+5:
// (v0, m01, c), (m01, v1, c), (v1, m12, c), (m12, v2, c), (v2, m20, c), (m20, v0, c).
__global__ void k_bary_verts(const double *V, const int32_t *tris, const int32_t *owner, const int32_t *edge_pos,
                             int64_t N, int64_t M, int64_t E, double *Vb)
{
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= 3 * N) return;
    const int64_t t = h / 3;
    const int k = (int)(h % 3);
    if (owner[h] == h) {
        const int32_t a = tris[3 * t + k], b = tris[3 * t + (k + 1) % 3];
        const int64_t m = M + edge_pos[h];
        for (int c = 0; c < 3; ++c) Vb[3 * m + c] = 0.5 * (V[3 * (int64_t)a + c] + V[3 * (int64_t)b + c]);
    }
    if (k == 0) {
        const int32_t a = tris[3 * t], b = tris[3 * t + 1], c0 = tris[3 * t + 2];
        for (int c = 0; c < 3; ++c)
            Vb[3 * (M + E + t) + c] = (V[3 * (int64_t)a + c] + V[3 * (int64_t)b + c] + V[3 * (int64_t)c0 + c]) / 3.0;
    }
}

__global__ void k_bary_tris(const int32_t *tris, const int32_t *owner, const int32_t *edge_pos, int64_t N, int64_t M,
                            int64_t E, int32_t *Tb)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const int32_t v0 = tris[3 * t], v1 = tris[3 * t + 1], v2 = tris[3 * t + 2];
    const int32_t m01 = (int32_t)(M + edge_pos[owner[3 * t]]), m12 = (int32_t)(M + edge_pos[owner[3 * t + 1]]),
                  m20 = (int32_t)(M + edge_pos[owner[3 * t + 2]]);
    const int32_t c = (int32_t)(M + E + t);
    const int32_t ch[6][3] = {{v0, m01, c}, {m01, v1, c}, {v1, m12, c}, {m12, v2, c}, {v2, m20, c}, {m20, v0, c}};
    for (int k = 0; k < 6; ++k)
        for (int j = 0; j < 3; ++j) Tb[3 * (6 * t + k) + j] = ch[k][j];
}

__global__ void k_owner_flag(const int32_t *owner, int64_t H, int32_t *flag)
{
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h < H) flag[h] = owner[h] == h ? 1 : 0;
}

bem_status barycentric(bem_mesh *m, bem_mesh **out)
{
    bem_ctx *ctx = m->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t N = m->N, M = m->M, H = 3 * N;
    Allocs tmp;
    int32_t *flag = nullptr, *pos = nullptr;
    int64_t E = 0;
    bem_status st = dalloc(ctx, tmp, (void **)&flag, sizeof(int32_t) * (2 * H + 2), false);
    if (st) return st;
    pos = flag + H + 1;
    k_owner_flag<<<nblk(H, 256), 256, 0, s>>>(m->owner, H, flag); BEM_COUNT(ctx);
    if ((st = exclusive_scan_i32(ctx, flag, pos, H, &E))) {
        dfree_all(ctx, tmp);
        return st;
    }
    bem_mesh *r = new (std::nothrow) bem_mesh();
    if (!r) {
        dfree_all(ctx, tmp);
        return set_error(ctx, BEM_ERR_OOM, "host allocation");
    }
    r->ctx = ctx;
    r->M = M + E + N;
    r->N = 6 * N;
    if (r->M > 0x7FFFFFFFLL || r->N > 0x7FFFFFFFLL) st = set_error(ctx, BEM_ERR_INVALID, "barycentric mesh too large");
    if (!st) st = dalloc(ctx, r->allocs, (void **)&r->verts, sizeof(double) * 3 * r->M, false);
    if (!st) st = dalloc(ctx, r->allocs, (void **)&r->tris, sizeof(int32_t) * 3 * r->N, false);
    if (!st) {
        cudaError_t e = cudaMemcpyAsync(r->verts, m->verts, sizeof(double) * 3 * M, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) st = cuda_error(ctx, e, "barycentric vertices");
    }
    if (!st) {
        k_bary_verts<<<nblk(H, 256), 256, 0, s>>>(m->verts, m->tris, m->owner, pos, N, M, E, r->verts); BEM_COUNT(ctx);
        k_bary_tris<<<nblk(N, 256), 256, 0, s>>>(m->tris, m->owner, pos, N, M, E, r->tris); BEM_COUNT(ctx);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = cuda_error(ctx, e, "barycentric kernels");
    }
    if (!st) st = mesh_build(r, true, nullptr);
    dfree_all(ctx, tmp);
    if (st) {
        dfree_all(ctx, r->allocs);
        delete r;
        return st;
    }
    *out = r;
    return BEM_OK;
}

// Dual-cell table of the primal mesh: cell areas |T_z^dual| = (sum of |T| at z,
// ascending) / 3 and cell "centroids" (the vertex) for the cells mesh.
__global__ void k_dual_cells(const double *V, const int32_t *v2t_off, const int32_t *v2t, const double *area,
                             int64_t M, double *darea, double *dcent)
{
    const int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= M) return;
    double sum = 0.0;
    for (int32_t p = v2t_off[z]; p < v2t_off[z + 1]; ++p) sum = sum + area[v2t[p]];
    const double a = sum / 3.0;
    darea[z] = a;
    for (int c = 0; c < 3; ++c) dcent[4 * z + c] = V[3 * z + c];
    dcent[4 * z + 3] = a;
}

template <typename T> __device__ __forceinline__ double vb_elem(const T *V, int64_t o);
template <> __device__ __forceinline__ double vb_elem<double>(const double *V, int64_t o) { return V[o]; }
template <> __device__ __forceinline__ double vb_elem<float2>(const float2 *V, int64_t o)
{
    return (double)V[o].x + (double)V[o].y;
}
template <> __device__ __forceinline__ double vb_elem<float>(const float *V, int64_t o) { return (double)V[o]; }

// Children of primal vertex z that belong to its dual cell, in ascending order:
// local vertex k of triangle t owns children 6t + {0,5} (k = 0), {1,2} (k = 1),
// {3,4} (k = 2).
__device__ __forceinline__ int cell_children(const int32_t *tris, const int32_t *v2t_off, const int32_t *v2t,
                                             int64_t z, int32_t *out, int cap)
{
    int n = 0;
    for (int32_t p = v2t_off[z]; p < v2t_off[z + 1]; ++p) {
        const int32_t t = v2t[p];
        const int k = tris[3 * t] == z ? 0 : (tris[3 * t + 1] == z ? 1 : 2);
        const int c0 = k == 0 ? 0 : 2 * k - 1, c1 = k == 0 ? 5 : 2 * k;
        if (n + 2 <= cap) {
            out[n++] = 6 * t + c0;
            out[n++] = 6 * t + c1;
        }
    }
    return n;
}

// V^dual[z][w] = sum over children B of z and B' of w of V^bary[B][B'] (FP64 sums in
// the order of the children lists), z <= w, mirrored; output double (F64) or hi/lo
// pairs (DF64).  One thread per (z, w) of a row z; the children lists come from the
// primal vertex-to-triangle table.
constexpr int kMaxCellChildren = 64;  // valence <= 32

template <typename T, typename O>
__global__ void k_dual_operator(const T *__restrict__ Vb, int64_t ldb, const int32_t *tris, const int32_t *v2t_off,
                                const int32_t *v2t, int64_t M, O *Vd, int64_t ldd, int *bad)
{
    const int64_t z = blockIdx.y;
    const int64_t w = z + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    __shared__ int32_t cz[kMaxCellChildren];
    __shared__ int s_nz;
    if (threadIdx.x == 0) s_nz = cell_children(tris, v2t_off, v2t, z, cz, kMaxCellChildren);
    __syncthreads();
    if (w >= M) return;
    int32_t cw[kMaxCellChildren];
    const int nw = cell_children(tris, v2t_off, v2t, w, cw, kMaxCellChildren);
    if ((v2t_off[w + 1] - v2t_off[w]) * 2 > kMaxCellChildren || (v2t_off[z + 1] - v2t_off[z]) * 2 > kMaxCellChildren)
        atomicExch(bad, 1);
    double sum = 0.0;
    for (int a = 0; a < s_nz; ++a) {
        const int64_t row = (int64_t)cz[a] * ldb;
        for (int b = 0; b < nw; ++b) sum = sum + vb_elem(Vb, row + cw[b]);
    }
    if constexpr (std::is_same<O, double>::value) {
        Vd[z * ldd + w] = sum;
        Vd[w * ldd + z] = sum;
    } else {
        const float h = __double2float_rn(sum);
        const float2 v = make_float2(h, __double2float_rn(sum - (double)h));
        Vd[z * ldd + w] = v;
        Vd[w * ldd + z] = v;
    }
}

// eta(T)^2 of Eq. 1.6 for a dual solution x (one value per vertex): Phi piecewise
// constant on the dual cells, I Phi its S^1 interpolant; closed form per barycentric
// child (see the oracle of the same name for the operation order); block partials of
// the total and of sum h |T| xbar^2 / 12, xbar = (x0 + x1 + x2) / 3.
__global__ void k_zz_dual(const int32_t *tris, const double *area, const double *diam, const double *x, int64_t N,
                          int h_mode, double *eta2, double *part_eta, double *part_scale)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double e = 0.0, sc = 0.0;
    if (t < N) {
        const double x0 = x[tris[3 * t]], x1 = x[tris[3 * t + 1]], x2 = x[tris[3 * t + 2]];
        const double s = (x0 + x1) + x2;
        const double c3 = s / 3.0;
        const double own[6] = {x0, x1, x1, x2, x2, x0};
        const double mid[6] = {0.5 * (x0 - x1), 0.5 * (x1 - x0), 0.5 * (x1 - x2),
                               0.5 * (x2 - x1), 0.5 * (x2 - x0), 0.5 * (x0 - x2)};
        double q = 0.0;
        for (int k = 0; k < 6; ++k) {
            const double a = (k % 2 == 0) ? 0.0 : mid[k], b = (k % 2 == 0) ? mid[k] : 0.0, c = own[k] - c3;
            const double ab = a + b;
            q = q + (((a * a + b * b) + c * c) + (ab + c) * (ab + c));
        }
        const double h = h_mode == 1 ? sqrt(area[t]) : diam[t];
        e = (h * (area[t] / 72.0)) * q;
        const double xm = s / 3.0;
        sc = h * area[t] * xm * xm / 12.0;
        eta2[t] = e;
    }
    __shared__ double se[256], ss[256];
    se[threadIdx.x] = e;
    ss[threadIdx.x] = sc;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            se[threadIdx.x] += se[threadIdx.x + o];
            ss[threadIdx.x] += ss[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part_eta[blockIdx.x] = se[0];
        part_scale[blockIdx.x] = ss[0];
    }
}

bem_status zz_estimate_dual(bem_mesh *m, const double *d_x, int h_mode, double *d_eta2, double *h_totals)
{
    bem_ctx *ctx = m->ctx;
    cudaStream_t s = ctx->stream;
    Allocs tmp;
    const int nb = (int)nblk(m->N, 256);
    double *pe = nullptr;
    bem_status st = dalloc(ctx, tmp, (void **)&pe, sizeof(double) * (2 * nb + 2), false);
    if (st) return st;
    double *ps = pe + nb, *tot = ps + nb;
    k_zz_dual<<<nb, 256, 0, s>>>(m->tris, m->area, m->diam, d_x, m->N, h_mode, d_eta2, pe, ps); BEM_COUNT(ctx);
    k_sum2<<<1, 32, 0, s>>>(pe, ps, nb, tot); BEM_COUNT(ctx);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) st = cuda_error(ctx, e, "dual zz kernels");
    if (!st && h_totals) {
        e = cudaMemcpyAsync(ctx->h_pinned, tot, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(ctx, e, "dual zz totals");
        else {
            h_totals[0] = ctx->h_pinned[0];
            h_totals[1] = ctx->h_pinned[1];
        }
    }
    dfree_all(ctx, tmp);
    return st;
}

// ---- operator preconditioner (Sec. 2.6)
// V^T[T][T'] = sum of V^bary over the 6 x 6 children of T and T' (R^T V^bary R, R the
// map of a primal triangle to its six children): the P0 Galerkin matrix of the primal
// triangles evaluated with the barycentric quadrature.  Rows strided over grid y.
template <typename T>
__global__ void k_contract_children(const T *__restrict__ Vb, int64_t ldb, int64_t N, double *__restrict__ VT)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= N) return;
    for (int64_t i = blockIdx.y; i < N; i += gridDim.y) {
        double s = 0.0;
        for (int a = 0; a < 6; ++a) {
            const int64_t row = (6 * i + a) * ldb + 6 * j;
            for (int b = 0; b < 6; ++b) s += vb_elem(Vb, row + b);
        }
        VT[i * N + j] = s;
    }
}

// Surface curl of the hat of vertex z on triangle t: n x grad phi_z = (p_(k+1) - p_(k+2))
// / (2 |T|) for z the local vertex k of t (n the unit normal of the vertex order).
__device__ __forceinline__ void hat_curl(const double *V, const int32_t *tris, const double *area, int32_t t, int64_t z,
                                         double g[3])
{
    const int32_t *tv = tris + 3 * (int64_t)t;
    const int k = tv[0] == z ? 0 : (tv[1] == z ? 1 : 2);
    const double *p1 = V + 3 * (int64_t)tv[(k + 1) % 3], *p2 = V + 3 * (int64_t)tv[(k + 2) % 3];
    const double s = 1.0 / (2.0 * area[t]);
    for (int c = 0; c < 3; ++c) g[c] = (p1[c] - p2[c]) * s;
}

// D^reg[i][j] = sum_{T at i} sum_{T' at j} (curl phi_i|T . curl phi_j|T') V^T[T][T'] +
// a_i a_j, j >= i, mirrored, stored FP32.  One CTA row i: its star and curls in
// shared memory; one thread per column j.
constexpr int kMaxStar = 32;

__global__ void k_hypersingular(const double *V, const int32_t *tris, const int32_t *v2t_off, const int32_t *v2t,
                                const double *area, const double *__restrict__ VT, int64_t N, const double *a_int,
                                int64_t M, float *Dm, int64_t ldd, int *bad)
{
    __shared__ int32_t st[kMaxStar];
    __shared__ double sg[kMaxStar][3];
    __shared__ int s_n;
    for (int64_t i = blockIdx.y; i < M; i += gridDim.y) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const int n = v2t_off[i + 1] - v2t_off[i];
            if (n > kMaxStar) atomicExch(bad, 1);
            s_n = n < kMaxStar ? n : kMaxStar;
        }
        __syncthreads();
        if ((int)threadIdx.x < s_n) {
            const int32_t t = v2t[v2t_off[i] + threadIdx.x];
            st[threadIdx.x] = t;
            hat_curl(V, tris, area, t, i, sg[threadIdx.x]);
        }
        __syncthreads();
        const int64_t j = i + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
        if (j >= M) continue;
        double acc = 0.0;
        const int nj = min(v2t_off[j + 1] - v2t_off[j], kMaxStar);
        for (int q = 0; q < nj; ++q) {
            const int32_t tj = v2t[v2t_off[j] + q];
            double g[3];
            hat_curl(V, tris, area, tj, j, g);
            for (int p = 0; p < s_n; ++p) {
                const double dot = (sg[p][0] * g[0] + sg[p][1] * g[1]) + sg[p][2] * g[2];
                acc += dot * __ldg(VT + (int64_t)st[p] * N + tj);
            }
        }
        const float v = __double2float_rn(acc + a_int[i] * a_int[j]);
        Dm[i * ldd + j] = v;
        Dm[j * ldd + i] = v;
    }
}

// 1 / diag of the mass matrix M[i][j] = int phi_j chi_i^dual: M_ii = sum_{T at i} 22 |T| / 108.
__global__ void k_mass_dinv(const int32_t *v2t_off, const int32_t *v2t, const double *area, int64_t M, float *dinv)
{
    const int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= M) return;
    double s = 0.0;
    for (int32_t p = v2t_off[z]; p < v2t_off[z + 1]; ++p) s += area[v2t[p]];
    dinv[z] = (float)(108.0 / (22.0 * s));
}

// S ~ M^-1 applied to every column of B (M x ld, FP32): kChebSteps steps of Chebyshev
// iteration on the Jacobi-scaled mass matrix, whose spectrum lies in [15/22, 36/22] on
// every mesh (per triangle M_T = (|T| / 108)(15 I + 7 J) against diag 22 |T| / 108);
// theta and delta are the interval's centre and half-width.  One thread per (row i,
// column j), columns fastest: (M X)_ij = sum_{T at i} |T| / 108 (22 X_ij + 7 (X_kj + X_lj)).
constexpr double kChebTheta = 51.0 / 44.0, kChebDelta = 21.0 / 44.0;
constexpr int kChebSteps = 6;  // error factor 2 ((sqrt(2.4) - 1) / (sqrt(2.4) + 1))^6 = 2e-4

__global__ void k_cheb_cols(const int32_t *tris, const int32_t *v2t_off, const int32_t *v2t, const double *area,
                            const float *dinv, int64_t M, int64_t ld, const float *B, const float *dc, float *dn,
                            float *res, float *out, float c_old, float c_res, int first)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    for (int64_t i = blockIdx.y; i < M; i += gridDim.y) {
        const int64_t o = i * ld + j;
        if (first) {  // res = B, d = D^-1 B / theta, out = d
            const float b = B[o];
            const float d = b * dinv[i] * (float)(1.0 / kChebTheta);
            res[o] = b;
            dn[o] = d;
            out[o] = d;
            continue;
        }
        const float di = dc[o];
        float md = 0.0f;
        for (int32_t q = v2t_off[i]; q < v2t_off[i + 1]; ++q) {
            const int32_t t = v2t[q];
            float nb = 0.0f;
            for (int c = 0; c < 3; ++c) {
                const int32_t v = tris[3 * (int64_t)t + c];
                if (v != i) nb += dc[(int64_t)v * ld + j];
            }
            md += (float)area[t] * (22.0f * di + 7.0f * nb);
        }
        const float r = res[o] - md * (1.0f / 108.0f);
        res[o] = r;
        const float d = c_old * di + c_res * r * dinv[i];
        dn[o] = d;
        out[o] += d;
    }
}

// out[j][i] = in[i][j] over 32 x 32 tiles (M x ld, FP32).
__global__ void k_transpose_f32(const float *in, int64_t M, int64_t ld, float *out)
{
    __shared__ float t[32][33];
    const int64_t bx = (int64_t)blockIdx.x * 32, by = (int64_t)blockIdx.y * 32;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = by + r, j = bx + threadIdx.x;
        t[r][threadIdx.x] = (i < M && j < M) ? in[i * ld + j] : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {
        const int64_t i = bx + r, j = by + threadIdx.x;
        if (i < M && j < M) out[i * ld + j] = t[threadIdx.x][r];
    }
}

// C[i][j] = C[j][i] for i > j through 32 x 32 tiles: the rounded S W^T made exactly
// symmetric (the packed product reads both halves of the diagonal tiles).
__global__ void k_mirror_upper_f32(float *C, int64_t M, int64_t ld)
{
    __shared__ float t[32][33];
    const int64_t bi = blockIdx.y, bj = blockIdx.x;
    if (bj > bi) return;
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {  // upper block (bj, bi)
        const int64_t i = bj * 32 + r, j = bi * 32 + threadIdx.x;
        t[r][threadIdx.x] = (i < M && j < M) ? C[i * ld + j] : 0.0f;
    }
    __syncthreads();
    for (int r = threadIdx.y; r < 32; r += blockDim.y) {  // lower block (bi, bj)
        const int64_t i = bi * 32 + r, j = bj * 32 + threadIdx.x;
        if (i < M && j < M && i > j) C[i * ld + j] = t[threadIdx.x][r];
    }
}

static bem_status cheb_cols(bem_ctx *ctx, bem_mesh *pm, const float *dinv, int64_t ld, const float *B, float *out,
                            float *w)
{
    const int64_t M = pm->M;
    float *res = w, *dA = w + M * ld, *dB = w + 2 * M * ld;
    const dim3 grid((unsigned)nblk(M, 128), (unsigned)std::min<int64_t>(M, 65535));
    k_cheb_cols<<<grid, 128, 0, ctx->stream>>>(pm->tris, pm->v2t_off, pm->v2t, pm->area, dinv, M, ld, B, nullptr, dA,
                                               res, out, 0.f, 0.f, 1); BEM_COUNT(ctx);
    double rho = kChebDelta / kChebTheta;
    for (int k = 1; k < kChebSteps; ++k) {
        const double rn = 1.0 / (2.0 * (kChebTheta / kChebDelta) - rho);
        k_cheb_cols<<<grid, 128, 0, ctx->stream>>>(pm->tris, pm->v2t_off, pm->v2t, pm->area, dinv, M, ld, B, dA, dB,
                                                   res, out, (float)(rn * rho), (float)(2.0 * rn / kChebDelta), 0);
        BEM_COUNT(ctx);
        rho = rn;
        float *t = dA;
        dA = dB;
        dB = t;
    }
    BEM_CK_LAUNCH(ctx);
    return BEM_OK;
}

// The operator preconditioner of Sec. 2.6 for CG on V^dual: D^reg (FP32, from V^bary),
// then C = S D^reg S with S the Chebyshev approximation of M^-1 (W = S D^reg by
// columns, C = S W^T, which equals S D^reg S since it is symmetric), stored FP32.
static bem_status calderon_setup(bem_operator *ob, bem_mesh *pm, bem_operator *op, int *bad)
{
    bem_ctx *ctx = pm->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t N = pm->N, M = pm->M, ld = op->ld;
    Allocs tmp;
    double *VT = nullptr;
    float *W = nullptr, *work = nullptr, *dinv = nullptr;
    bem_status st = dalloc(ctx, op->allocs, (void **)&op->cal_D, sizeof(float) * (size_t)M * (size_t)ld, true);
    if (!st) st = dalloc(ctx, op->allocs, (void **)&op->cal_C, sizeof(float) * (size_t)M * (size_t)ld, true);
    if (!st) st = dalloc(ctx, tmp, (void **)&VT, sizeof(double) * (size_t)N * (size_t)N, false);
    if (st) {
        dfree_all(ctx, tmp);
        return st;
    }
    const dim3 gc((unsigned)nblk(N, 128), (unsigned)std::min<int64_t>(N, 65535));
    if (ob->precision == BEM_PREC_F64)
        { k_contract_children<double><<<gc, 128, 0, s>>>((const double *)ob->V, ob->ld, N, VT); BEM_COUNT(ctx); }
    else if (ob->precision == BEM_PREC_DF64)
        { k_contract_children<float2><<<gc, 128, 0, s>>>((const float2 *)ob->V, ob->ld, N, VT); BEM_COUNT(ctx); }
    else
        { k_contract_children<float><<<gc, 128, 0, s>>>((const float *)ob->V, ob->ld, N, VT); BEM_COUNT(ctx); }
    const dim3 gh((unsigned)nblk(M, 128), (unsigned)std::min<int64_t>(M, 65535));
    k_hypersingular<<<gh, 128, 0, s>>>(pm->verts, pm->tris, pm->v2t_off, pm->v2t, pm->area, VT, N,
                                       op->mesh->area, M, op->cal_D, ld, bad); BEM_COUNT(ctx);
    dfree_all(ctx, tmp);  // stream-ordered: V^T is freed after the kernel that reads it
    // C = S D^reg S: W = S D^reg, then S W^T (all buffers zeroed: padding columns stay 0)
    st = dalloc(ctx, tmp, (void **)&W, sizeof(float) * ((size_t)M * (size_t)ld * 5 + (size_t)M), true);
    if (st) return st;
    float *Wt = W + M * ld;
    work = W + 2 * M * ld;  // residuals and two directions
    dinv = W + 5 * M * ld;
    k_mass_dinv<<<nblk(M, 256), 256, 0, s>>>(pm->v2t_off, pm->v2t, pm->area, M, dinv); BEM_COUNT(ctx);
    if (!(st = cheb_cols(ctx, pm, dinv, ld, op->cal_D, W, work))) {
        k_transpose_f32<<<dim3(nblk(M, 32), nblk(M, 32)), dim3(32, 8), 0, s>>>(W, M, ld, Wt); BEM_COUNT(ctx);
        st = cheb_cols(ctx, pm, dinv, ld, Wt, op->cal_C, work);
    }
    if (!st) {
        k_mirror_upper_f32<<<dim3(nblk(M, 32), nblk(M, 32)), dim3(32, 8), 0, s>>>(op->cal_C, M, ld); BEM_COUNT(ctx);
    }
    cudaError_t e = cudaGetLastError();
    dfree_all(ctx, tmp);
    if (st) return st;
    return e == cudaSuccess ? BEM_OK : cuda_error(ctx, e, "preconditioner kernels");
}

// The dual operator of primal mesh pm from the operator of its barycentric refinement:
// an M x M operator (DF64, or F64 for an F64 barycentric operator) over a cells mesh
// (N = M cells: dual areas as |T|, the vertices as centroids) owned by the operator.
bem_status dual_operator(bem_operator *ob, bem_mesh *pm, bem_operator **out)
{
    bem_ctx *ctx = pm->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t M = pm->M;
    bem_mesh *cm = new (std::nothrow) bem_mesh();
    bem_operator *op = new (std::nothrow) bem_operator();
    if (!cm || !op) {
        delete cm;
        delete op;
        return set_error(ctx, BEM_ERR_OOM, "host allocation");
    }
    cm->ctx = ctx;
    cm->N = M;
    cm->M = 0;
    cm->cells_only = 1;
    op->mesh = cm;
    op->ctx = ctx;
    op->owns_mesh = 1;
    op->precision = ob->precision == BEM_PREC_F64 ? BEM_PREC_F64 : BEM_PREC_DF64;
    op->ss_order = ob->ss_order;
    op->N = M;
    op->ld = padded_ld(M);
    Allocs tmp;
    int *bad = nullptr;
    bem_status st = dalloc(ctx, cm->allocs, (void **)&cm->area, sizeof(double) * M, false);
    if (!st) st = dalloc(ctx, cm->allocs, (void **)&cm->cent, sizeof(double) * 4 * M, false);
    if (!st) st = dalloc(ctx, op->allocs, &op->V, 8 * (size_t)M * (size_t)op->ld, true);
    if (!st) st = dalloc(ctx, op->allocs, (void **)&op->diag, sizeof(double) * M, false);
    if (!st) st = dalloc(ctx, tmp, (void **)&bad, sizeof(int), true);
    if (!st) {
        k_dual_cells<<<nblk(M, 256), 256, 0, s>>>(pm->verts, pm->v2t_off, pm->v2t, pm->area, M, cm->area, cm->cent); BEM_COUNT(ctx);
        const dim3 grid((unsigned)nblk(M, 128), (unsigned)M);
        if (M > 65535) st = set_error(ctx, BEM_ERR_INVALID, "dual operator: more than 65535 vertices");
        else if (ob->precision == BEM_PREC_F64)
            { k_dual_operator<double, double><<<grid, 128, 0, s>>>((const double *)ob->V, ob->ld, pm->tris, pm->v2t_off, pm->v2t, M, (double *)op->V, op->ld, bad); BEM_COUNT(ctx); }
        else if (ob->precision == BEM_PREC_DF64)
            { k_dual_operator<float2, float2><<<grid, 128, 0, s>>>((const float2 *)ob->V, ob->ld, pm->tris, pm->v2t_off, pm->v2t, M, (float2 *)op->V, op->ld, bad); BEM_COUNT(ctx); }
        else
            { k_dual_operator<float, float2><<<grid, 128, 0, s>>>((const float *)ob->V, ob->ld, pm->tris, pm->v2t_off, pm->v2t, M, (float2 *)op->V, op->ld, bad); BEM_COUNT(ctx); }
    }
    if (!st) st = operator_diag(op);
    if (!st) st = calderon_setup(ob, pm, op, bad);
    if (!st) {
        cudaError_t e = cudaMemcpyAsync(ctx->h_pinned, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = cuda_error(ctx, e, "dual operator");
        else if (*reinterpret_cast<int *>(ctx->h_pinned))
            st = set_error(ctx, BEM_ERR_MESH, "dual operator: a vertex has more than %d triangles", kMaxCellChildren / 2);
    }
    dfree_all(ctx, tmp);
    if (st) {
        bem_operator_destroy(op);
        return st;
    }
    *out = op;
    return BEM_OK;
}

}  // namespace bem
