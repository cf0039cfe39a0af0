// Mesh on the device (Sec. 2.1): validation, reference-edge rotation, per-triangle
// geometry and quadrature points, vertex->triangle incidence, edge owners and the
// lists of touching pairs that route entries to the singular quadrature.
//
// Compiled with -fmad=false: area and diameter are formed with every product and
// sum rounded separately, in the order written, so that the estimator that uses
// them is bit-identical to a plain IEEE-754 evaluation.
#include <climits>

#include "bem_internal.cuh"

namespace bem {

__constant__ double c_radon_bary[kQ][3];

static bool g_radon_ready[64] = {false};

// Radon's 7-point degree-5 rule: the centroid and the orbits (a,a,1-2a),
// a = (6 -+ sqrt 15)/21.
static bem_status radon_upload(bem_ctx *ctx)
{
    if (ctx->device < 64 && g_radon_ready[ctx->device]) return BEM_OK;
    const double r = std::sqrt(15.0);
    const double a = (6.0 - r) / 21.0, b = (6.0 + r) / 21.0;
    double B[kQ][3] = {{1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0},
                       {a, a, 1.0 - 2.0 * a}, {a, 1.0 - 2.0 * a, a}, {1.0 - 2.0 * a, a, a},
                       {b, b, 1.0 - 2.0 * b}, {b, 1.0 - 2.0 * b, b}, {1.0 - 2.0 * b, b, b}};
    BEM_CK(ctx, cudaMemcpyToSymbol(c_radon_bary, B, sizeof(B)));
    if (ctx->device < 64) g_radon_ready[ctx->device] = true;
    return BEM_OK;
}

// ------------------------------------------------------------------ scan
__global__ void k_scan_blocks(const int32_t *in, int32_t *out, int64_t n, int32_t *block_sums)
{
    __shared__ int32_t wsum[32];
    const int64_t base = (int64_t)blockIdx.x * 4096 + threadIdx.x * 4;
    int32_t v[4], s = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = (base + k < n) ? in[base + k] : 0;
        s += v[k];
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t x = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int32_t t = wsum[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        wsum[lane] = t;
    }
    __syncthreads();
    int32_t excl = x - s + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        if (base + k < n) out[base + k] = excl;
        excl += v[k];
    }
    if (threadIdx.x == blockDim.x - 1) block_sums[blockIdx.x] = wsum[31];
}

__global__ void k_scan_add(int32_t *out, int64_t n, const int32_t *block_offsets)
{
    const int64_t i = (int64_t)blockIdx.x * 4096 + threadIdx.x * 4;
    const int32_t off = block_offsets[blockIdx.x];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (i + k < n) out[i + k] += off;
}

// Whole scan in one CTA for short inputs (up to kScanSingleMax): chunks of 4096 scanned
// in turn with a running carry, out[n] = total written by the kernel.  Saves the
// second-level launches, allocations and the total's copy of the multi-block scan for
// the per-level tables of the adaptive loop.
constexpr int64_t kScanSingleMax = 16384;
__global__ void __launch_bounds__(1024) k_scan_single(const int32_t *in, int32_t *out, int64_t n)
{
    __shared__ int32_t wsum[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t carry = 0;
    for (int64_t c0 = 0; c0 < n; c0 += 4096) {
        const int64_t base = c0 + threadIdx.x * 4;
        int32_t v[4], s = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = (base + k < n) ? in[base + k] : 0;
            s += v[k];
        }
        int32_t x = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) wsum[w] = x;
        __syncthreads();
        if (w == 0) {
            int32_t t = wsum[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int32_t y = __shfl_up_sync(0xffffffffu, t, o);
                if (lane >= o) t += y;
            }
            wsum[lane] = t;
        }
        __syncthreads();
        int32_t excl = carry + x - s + (w > 0 ? wsum[w - 1] : 0);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (base + k < n) out[base + k] = excl;
            excl += v[k];
        }
        carry += wsum[31];
        __syncthreads();  // wsum is rewritten by the next chunk
    }
    if (threadIdx.x == 0) out[n] = carry;
}

static bem_status scan_rec(bem_ctx *ctx, const int32_t *in, int32_t *out, int64_t n, Allocs &tmp)
{
    // out[0..n) exclusive, out[n] = total
    if (n <= kScanSingleMax) {
        k_scan_single<<<1, 1024, 0, ctx->stream>>>(in, out, n); BEM_COUNT(ctx);
        BEM_CK_LAUNCH(ctx);
        return BEM_OK;
    }
    const int64_t nb = (n + 4095) / 4096;
    int32_t *bs = nullptr;
    bem_status st = dalloc(ctx, tmp, (void **)&bs, sizeof(int32_t) * (nb + 1), false);
    if (st) return st;
    k_scan_blocks<<<(unsigned)nb, 1024, 0, ctx->stream>>>(in, out, n, bs); BEM_COUNT(ctx);
    BEM_CK_LAUNCH(ctx);
    if (nb == 1) {
        BEM_CK(ctx, cudaMemcpyAsync(out + n, bs, sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->stream));
        return BEM_OK;
    }
    int32_t *bo = nullptr;
    st = dalloc(ctx, tmp, (void **)&bo, sizeof(int32_t) * (nb + 1), false);
    if (st) return st;
    st = scan_rec(ctx, bs, bo, nb, tmp);
    if (st) return st;
    k_scan_add<<<(unsigned)nb, 1024, 0, ctx->stream>>>(out, n, bo); BEM_COUNT(ctx);
    BEM_CK_LAUNCH(ctx);
    BEM_CK(ctx, cudaMemcpyAsync(out + n, bo + nb, sizeof(int32_t), cudaMemcpyDeviceToDevice, ctx->stream));
    return BEM_OK;
}

bem_status read_i32s(bem_ctx *ctx, const int32_t *const *src, int n, int64_t *out)
{
    int32_t *h = reinterpret_cast<int32_t *>(ctx->h_pinned);
    if (n > 64) return set_error(ctx, BEM_ERR_INVALID, "too many scalars in one read");
    for (int k = 0; k < n; ++k)
        BEM_CK(ctx, cudaMemcpyAsync(h + k, src[k], sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    BEM_CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (int k = 0; k < n; ++k) out[k] = h[k];
    return BEM_OK;
}

bem_status exclusive_scan_i32(bem_ctx *ctx, const int32_t *in, int32_t *out, int64_t n,
                              int64_t *total)
{
    if (n <= 0) {
        BEM_CK(ctx, cudaMemsetAsync(out, 0, sizeof(int32_t), ctx->stream));
        if (total) *total = 0;
        return BEM_OK;
    }
    Allocs tmp;
    bem_status st = scan_rec(ctx, in, out, n, tmp);
    if (!st && total) {
        int32_t *h = reinterpret_cast<int32_t *>(ctx->h_pinned);
        cudaError_t e = cudaMemcpyAsync(h, out + n, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_error(ctx, e, "scan total");
        else *total = *h;
    }
    dfree_all(ctx, tmp);
    return st;
}

// ------------------------------------------------------------------ validation
// bad[0]: index out of range / repeated vertex; bad[1]: zero area; bad[2]: open
// edge (odd or single use); bad[3]: duplicate triangle.
__global__ void k_check_indices(const int32_t *tris, int64_t N, int64_t M, int32_t *bad)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    const int32_t a = tris[3 * t], b = tris[3 * t + 1], c = tris[3 * t + 2];
    if (a < 0 || b < 0 || c < 0 || a >= M || b >= M || c >= M || a == b || b == c || a == c)
        atomicOr(&bad[0], 1);
}

__device__ __forceinline__ double len2(const double *p, const double *q)
{
    const double dx = q[0] - p[0], dy = q[1] - p[1], dz = q[2] - p[2];
    return (dx * dx + dy * dy) + dz * dz;
}

// Rotate every triangle so that its reference edge (given, or the longest with
// ties to the lowest local index) is local edge 0 = (v0, v1).
__global__ void k_canonical(const double *verts, const int32_t *tin, const uint8_t *ref_edge,
                            int32_t *tout, int64_t N)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    int32_t v[3] = {tin[3 * t], tin[3 * t + 1], tin[3 * t + 2]};
    int e = 0;
    if (ref_edge) {
        e = ref_edge[t] % 3;
    } else {
        double l[3];
        for (int k = 0; k < 3; ++k) l[k] = len2(verts + 3 * (int64_t)v[k], verts + 3 * (int64_t)v[(k + 1) % 3]);
        if (l[1] > l[e]) e = 1;
        if (l[2] > l[e]) e = 2;
    }
    for (int k = 0; k < 3; ++k) tout[3 * t + k] = v[(e + k) % 3];
}

// Per triangle: |T| = |(P1-P0) x (P2-P0)|/2 and diam = longest edge in the fixed
// operation order; the 7 Radon points (FP64), their offsets from the centroid
// (FP32) and the centroid (FP64).
__device__ __forceinline__ void split2(double v, float *out)
{
    const float h = __double2float_rn(v);
    out[0] = h;
    out[1] = __double2float_rn(v - (double)h);
}

__device__ __forceinline__ void split3(double v, float *out)
{
    const float a = __double2float_rn(v);
    const double r = v - (double)a;  // exact
    const float b = __double2float_rn(r);
    out[0] = a;
    out[1] = b;
    out[2] = __double2float_rn(r - (double)b);
}

__global__ void k_geometry(const double *verts, const int32_t *tris, int64_t N, double *area,
                           double *diam, double *q64, float *q32, double *cent, float *qdf, int32_t *bad)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    double P[3][3];
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c) P[k][c] = verts[3 * (int64_t)tris[3 * t + k] + c];
    double e1[3], e2[3];
    for (int c = 0; c < 3; ++c) {
        e1[c] = P[1][c] - P[0][c];
        e2[c] = P[2][c] - P[0][c];
    }
    const double cx = e1[1] * e2[2] - e1[2] * e2[1];
    const double cy = e1[2] * e2[0] - e1[0] * e2[2];
    const double cz = e1[0] * e2[1] - e1[1] * e2[0];
    const double A = 0.5 * sqrt((cx * cx + cy * cy) + cz * cz);
    const double l0 = sqrt(len2(P[0], P[1])), l1 = sqrt(len2(P[1], P[2])), l2 = sqrt(len2(P[2], P[0]));
    double d = l0 > l1 ? l0 : l1;
    d = d > l2 ? d : l2;
    area[t] = A;
    diam[t] = d;
    if (!(A > 0.0)) atomicOr(&bad[1], 1);
    double c3[3];
    for (int c = 0; c < 3; ++c) c3[c] = (P[0][c] + P[1][c] + P[2][c]) / 3.0;
    double *q = q64 + (int64_t)kQ64Stride * t;
    float *o = q32 + (int64_t)kQ32Stride * t;
    for (int a = 0; a < kQ; ++a)
        for (int c = 0; c < 3; ++c) {
            const double x = c_radon_bary[a][0] * P[0][c] + c_radon_bary[a][1] * P[1][c] +
                             c_radon_bary[a][2] * P[2][c];
            q[3 * a + c] = x;
            o[3 * a + c] = (float)(x - c3[c]);
        }
    q[21] = A;
    q[22] = d;
    q[23] = 0.0;
    o[21] = o[22] = o[23] = 0.0f;
    // double-float table: offsets lambda . (P - c) from the centroid, the centroid
    // itself as an exact sum of three floats, and the area
    float *f = qdf + (int64_t)kQdfStride * t;
    double R[3][3];
    for (int k = 0; k < 3; ++k)
        for (int c = 0; c < 3; ++c) R[k][c] = P[k][c] - c3[c];
    for (int a = 0; a < kQ; ++a)
        for (int c = 0; c < 3; ++c) {
            const double off = c_radon_bary[a][0] * R[0][c] + c_radon_bary[a][1] * R[1][c] +
                               c_radon_bary[a][2] * R[2][c];
            split2(off, f + 2 * (3 * a + c));
        }
    for (int c = 0; c < 3; ++c) split3(c3[c], f + 42 + 3 * c);
    split2(A, f + 51);
    // the largest |hi part| of the 21 offset coordinates (the far field's grid bound)
    // and the largest distance of a point from the centroid, rounded up
    float rm = 0.0f;
    for (int k = 0; k < 3 * kQ; ++k) rm = fmaxf(rm, fabsf(f[2 * k]));
    double rd2 = 0.0;
    for (int a = 0; a < kQ; ++a) {
        double s2 = 0.0;
        for (int c = 0; c < 3; ++c) {
            const double off = c_radon_bary[a][0] * R[0][c] + c_radon_bary[a][1] * R[1][c] +
                               c_radon_bary[a][2] * R[2][c];
            s2 += off * off;
        }
        rd2 = rd2 > s2 ? rd2 : s2;
    }
    f[53] = rm;
    f[54] = __double2float_ru(sqrt(rd2) * (1.0 + 1e-12));
    f[55] = 0.0f;
    cent[4 * t + 0] = c3[0];
    cent[4 * t + 1] = c3[1];
    cent[4 * t + 2] = c3[2];
    cent[4 * t + 3] = A;
}

// ------------------------------------------------------------------ incidence
__global__ void k_v2t_count(const int32_t *tris, int64_t N, int32_t *cnt)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    for (int k = 0; k < 3; ++k) atomicAdd(&cnt[tris[3 * t + k]], 1);
}

__global__ void k_v2t_fill(const int32_t *tris, int64_t N, const int32_t *off, int32_t *cursor,
                           int32_t *v2t)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= N) return;
    for (int k = 0; k < 3; ++k) {
        const int32_t z = tris[3 * t + k];
        const int32_t pos = off[z] + atomicAdd(&cursor[z], 1);
        v2t[pos] = (int32_t)t;
    }
}

// Sort each vertex's list ascending (insertion sort; lists are short).
__global__ void k_v2t_sort(const int32_t *off, int32_t *v2t, int64_t M)
{
    const int64_t z = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= M) return;
    const int32_t b = off[z], e = off[z + 1];
    for (int32_t i = b + 1; i < e; ++i) {
        const int32_t key = v2t[i];
        int32_t j = i - 1;
        while (j >= b && v2t[j] > key) {
            v2t[j + 1] = v2t[j];
            --j;
        }
        v2t[j + 1] = key;
    }
}

// Owner of half-edge h = (t, k): the smallest half-edge index among the
// triangles' edges with the same two vertices, found in vertex u's ascending list.
__global__ void k_owner(const int32_t *tris, int64_t N, const int32_t *off, const int32_t *v2t,
                        int32_t *owner)
{
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= 3 * N) return;
    const int64_t t = h / 3;
    const int k = (int)(h % 3);
    const int32_t u = tris[3 * t + k], v = tris[3 * t + (k + 1) % 3];
    int32_t own = (int32_t)h;
    for (int32_t p = off[u]; p < off[u + 1]; ++p) {
        const int32_t s = v2t[p];
        bool found = false;
        for (int k2 = 0; k2 < 3; ++k2) {
            const int32_t a = tris[3 * (int64_t)s + k2], b = tris[3 * (int64_t)s + (k2 + 1) % 3];
            if ((a == u && b == v) || (a == v && b == u)) {
                own = 3 * s + k2;
                found = true;
                break;
            }
        }
        if (found) break;
    }
    owner[h] = own;
}

__global__ void k_edge_use(const int32_t *owner, int64_t H, int32_t *cnt)
{
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= H) return;
    atomicAdd(&cnt[owner[h]], 1);
}

__global__ void k_edge_closed(const int32_t *owner, const int32_t *cnt, int64_t H, int32_t *bad)
{
    const int64_t h = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (h >= H) return;
    if (owner[h] == h && ((cnt[h] & 1) || cnt[h] < 2)) atomicOr(&bad[2], 1);
}

// ------------------------------------------------------------------ touching pairs
// Walk the three ascending incidence lists of triangle i together; every j > i met
// c times shares c vertices with i (c = 1: vertex pair, 2: edge pair, 3: duplicate).
template <bool kFill>
__global__ void k_touch(const int32_t *tris, int64_t N, const int32_t *off, const int32_t *v2t,
                        int32_t *n_edge, int32_t *n_vert, const int32_t *off_edge,
                        const int32_t *off_vert, int32_t *edge_pairs, int32_t *vert_pairs,
                        int64_t ne_total, int64_t nv_total, int32_t *bad)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    int32_t p[3], e[3];
    for (int k = 0; k < 3; ++k) {
        const int32_t z = tris[3 * i + k];
        p[k] = off[z];
        e[k] = off[z + 1];
        while (p[k] < e[k] && v2t[p[k]] <= i) ++p[k];
    }
    int32_t ce = 0, cv = 0;
    int64_t we = kFill ? off_edge[i] : 0, wv = kFill ? off_vert[i] : 0;
    for (;;) {
        int32_t j = INT_MAX;
        for (int k = 0; k < 3; ++k)
            if (p[k] < e[k] && v2t[p[k]] < j) j = v2t[p[k]];
        if (j == INT_MAX) break;
        int c = 0;
        for (int k = 0; k < 3; ++k)
            if (p[k] < e[k] && v2t[p[k]] == j) {
                ++c;
                ++p[k];
            }
        if (c == 2) {
            if (kFill && we < ne_total) {
                edge_pairs[2 * we] = (int32_t)i;
                edge_pairs[2 * we + 1] = j;
            }
            ++we;
            ++ce;
        } else if (c == 1) {
            if (kFill && wv < nv_total) {
                vert_pairs[2 * wv] = (int32_t)i;
                vert_pairs[2 * wv + 1] = j;
            }
            ++wv;
            ++cv;
        } else if (!kFill) {
            atomicOr(&bad[3], 1);
        }
    }
    if (!kFill) {
        n_edge[i] = ce;
        n_vert[i] = cv;
    }
}

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

static bem_status read_bad(bem_ctx *ctx, const int32_t *d_bad, int32_t *h_bad)
{
    int32_t *h = reinterpret_cast<int32_t *>(ctx->h_pinned);
    BEM_CK(ctx, cudaMemcpyAsync(h, d_bad, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    BEM_CK(ctx, cudaStreamSynchronize(ctx->stream));
    memcpy(h_bad, h, 4 * sizeof(int32_t));
    return BEM_OK;
}

bem_status mesh_bad_status(bem_ctx *ctx, const int64_t *bad3)
{
    if (bad3[0]) return set_error(ctx, BEM_ERR_MESH, "degenerate triangle (zero area)");
    if (bad3[1]) return set_error(ctx, BEM_ERR_MESH, "mesh is not closed (an edge is used an odd number of times)");
    if (bad3[2]) return set_error(ctx, BEM_ERR_MESH, "duplicate triangle");
    return BEM_OK;
}

bem_status mesh_check_pending(bem_mesh *m)
{
    if (!m->bad_pending) return BEM_OK;
    const int32_t *src[3] = {m->d_bad + 1, m->d_bad + 2, m->d_bad + 3};
    int64_t b[3] = {0, 0, 0};
    bem_status st = read_i32s(m->ctx, src, 3, b);
    if (st) return st;
    m->bad_pending = 0;
    return mesh_bad_status(m->ctx, b);
}

bem_status mesh_build(bem_mesh *m, bool canonicalize, const uint8_t *d_ref_edge, bool defer_check)
{
    bem_ctx *ctx = m->ctx;
    const int64_t N = m->N, M = m->M;
    cudaStream_t s = ctx->stream;
    bem_status st = radon_upload(ctx);
    if (st) return st;
    Allocs tmp;
    int32_t *bad = nullptr, hb[4] = {0, 0, 0, 0};
#define TRY(x)                    \
    do {                          \
        st = (x);                 \
        if (st) goto done;        \
    } while (0)
    TRY(dalloc(ctx, defer_check ? m->allocs : tmp, (void **)&bad, 4 * sizeof(int32_t), true));
    if (canonicalize) {
        // a caller's mesh: indices checked before any kernel follows them (meshes made
        // by the library's refinements have valid indices by construction)
        k_check_indices<<<nblk(N, 256), 256, 0, s>>>(m->tris, N, M, bad); BEM_COUNT(ctx);
        TRY(read_bad(ctx, bad, hb));
        if (hb[0]) {
            st = set_error(ctx, BEM_ERR_MESH, "triangle with a vertex index outside [0, M) or repeated");
            goto done;
        }
    }
    if (canonicalize) {
        int32_t *t2 = nullptr;
        TRY(dalloc(ctx, tmp, (void **)&t2, sizeof(int32_t) * 3 * N, false));
        k_canonical<<<nblk(N, 256), 256, 0, s>>>(m->verts, m->tris, d_ref_edge, t2, N); BEM_COUNT(ctx);
        if (cudaGetLastError() != cudaSuccess) { st = set_error(ctx, BEM_ERR_CUDA, "k_canonical launch"); goto done; }
        if (cudaMemcpyAsync(m->tris, t2, sizeof(int32_t) * 3 * N, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            st = set_error(ctx, BEM_ERR_CUDA, "copy canonical triangles");
            goto done;
        }
    }
    TRY(dalloc(ctx, m->allocs, (void **)&m->area, sizeof(double) * N, false));
    TRY(dalloc(ctx, m->allocs, (void **)&m->diam, sizeof(double) * N, false));
    TRY(dalloc(ctx, m->allocs, (void **)&m->q64, sizeof(double) * kQ64Stride * N, false));
    TRY(dalloc(ctx, m->allocs, (void **)&m->q32, sizeof(float) * kQ32Stride * N, false));
    TRY(dalloc(ctx, m->allocs, (void **)&m->cent, sizeof(double) * 4 * N, false));
    TRY(dalloc(ctx, m->allocs, (void **)&m->qdf, sizeof(float) * kQdfStride * N, false));
    k_geometry<<<nblk(N, 128), 128, 0, s>>>(m->verts, m->tris, N, m->area, m->diam, m->q64, m->q32,
                                            m->cent, m->qdf, bad); BEM_COUNT(ctx);
    {
        int32_t *cnt = nullptr, *cursor = nullptr;
        TRY(dalloc(ctx, m->allocs, (void **)&m->v2t_off, sizeof(int32_t) * (M + 1), false));
        TRY(dalloc(ctx, m->allocs, (void **)&m->v2t, sizeof(int32_t) * 3 * N, false));
        TRY(dalloc(ctx, tmp, (void **)&cnt, sizeof(int32_t) * (M + 1), true));
        TRY(dalloc(ctx, tmp, (void **)&cursor, sizeof(int32_t) * (M + 1), true));
        k_v2t_count<<<nblk(N, 256), 256, 0, s>>>(m->tris, N, cnt); BEM_COUNT(ctx);
        TRY(exclusive_scan_i32(ctx, cnt, m->v2t_off, M, nullptr));
        k_v2t_fill<<<nblk(N, 256), 256, 0, s>>>(m->tris, N, m->v2t_off, cursor, m->v2t); BEM_COUNT(ctx);
        k_v2t_sort<<<nblk(M, 128), 128, 0, s>>>(m->v2t_off, m->v2t, M); BEM_COUNT(ctx);
    }
    {
        const int64_t H = 3 * N;
        int32_t *ecnt = nullptr;
        TRY(dalloc(ctx, m->allocs, (void **)&m->owner, sizeof(int32_t) * H, false));
        TRY(dalloc(ctx, tmp, (void **)&ecnt, sizeof(int32_t) * H, true));
        k_owner<<<nblk(H, 256), 256, 0, s>>>(m->tris, N, m->v2t_off, m->v2t, m->owner); BEM_COUNT(ctx);
        k_edge_use<<<nblk(H, 256), 256, 0, s>>>(m->owner, H, ecnt); BEM_COUNT(ctx);
        k_edge_closed<<<nblk(H, 256), 256, 0, s>>>(m->owner, ecnt, H, bad); BEM_COUNT(ctx);
    }
    {
        int32_t *ne = nullptr, *nv = nullptr, *oe = nullptr, *ov = nullptr;
        TRY(dalloc(ctx, tmp, (void **)&ne, sizeof(int32_t) * (N + 1), true));
        TRY(dalloc(ctx, tmp, (void **)&nv, sizeof(int32_t) * (N + 1), true));
        TRY(dalloc(ctx, tmp, (void **)&oe, sizeof(int32_t) * (N + 1), false));
        TRY(dalloc(ctx, tmp, (void **)&ov, sizeof(int32_t) * (N + 1), false));
        k_touch<false><<<nblk(N, 128), 128, 0, s>>>(m->tris, N, m->v2t_off, m->v2t, ne, nv, nullptr,
                                                    nullptr, nullptr, nullptr, 0, 0, bad); BEM_COUNT(ctx);
        BEM_CK_LAUNCH(ctx);
        int64_t tt[2] = {0, 0};
        TRY(exclusive_scan_i32(ctx, ne, oe, N, nullptr));
        TRY(exclusive_scan_i32(ctx, nv, ov, N, nullptr));
        const int32_t *src[2] = {oe + N, ov + N};
        TRY(read_i32s(ctx, src, 2, tt));  // both totals in one read
        const int64_t te = tt[0], tv = tt[1];
        m->n_edge_pairs = te;
        m->n_vert_pairs = tv;
        TRY(dalloc(ctx, m->allocs, (void **)&m->edge_pairs, sizeof(int32_t) * 2 * (te > 0 ? te : 1), false));
        TRY(dalloc(ctx, m->allocs, (void **)&m->vert_pairs, sizeof(int32_t) * 2 * (tv > 0 ? tv : 1), false));
        k_touch<true><<<nblk(N, 128), 128, 0, s>>>(m->tris, N, m->v2t_off, m->v2t, nullptr, nullptr, oe,
                                                   ov, m->edge_pairs, m->vert_pairs, te, tv, bad); BEM_COUNT(ctx);
        BEM_CK_LAUNCH(ctx);
    }
    if (defer_check) {
        m->d_bad = bad;
        m->bad_pending = 1;
    } else {
        TRY(read_bad(ctx, bad, hb));
        const int64_t b3[3] = {hb[1], hb[2], hb[3]};
        st = mesh_bad_status(ctx, b3);
    }
done:
#undef TRY
    dfree_all(ctx, tmp);
    return st;
}

}  // namespace bem
