// Solve V x = b, b_i = |T_i| (Eq. 2.5 with f = 1) and Cap = (1/4pi) b.x (Eq. 2.8).
//
// Dense V x (the paper needs "only matrix-vector products", Sec. 1.4) streams V
// once per product: one warp per row, 16-byte vector loads with the streaming
// cache hint, x served from L1/L2, a fixed warp-shuffle reduction (deterministic).
// The PCG recurrences (Jacobi preconditioner diag(V), the paper's "diag",
// Sec. 3) run in FP64 in three launches per iteration; every global sum is taken
// over per-block partials in a fixed order, so a solve is bit-reproducible.
// FP32 operators: FP64 iterative refinement -- r = b - V x with FP64
// accumulation, an inner PCG with FP32 products on that residual, x += d.
#include <cmath>

#include "bem_internal.cuh"

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

// ------------------------------------------------------------------ host side
struct Work {
    double *r, *z, *p, *q, *b, *x, *d;  // vectors of length ld
    double *part1, *part2, *part3;      // per-block partials
    double *scal;                       // device scalars: [0..1] rz slots, [2] rr, [3..5] reduce3
    int nb_vec, nb_mv;
};

bem_status matvec_f64(bem_operator *op, const double *x, double *y)
{
    bem_ctx *ctx = op->mesh->ctx;
    const unsigned g = nblk(op->N, kMvRows);
    if (op->precision == BEM_PREC_F64)
        { k_matvec<double, true><<<g, kMvThreads, 0, ctx->stream>>>((const double *)op->V, op->ld, op->N, x, y,
                                                                  nullptr, nullptr); BEM_COUNT(ctx); }
    else
        { k_matvec<float, true><<<g, kMvThreads, 0, ctx->stream>>>((const float *)op->V, op->ld, op->N, x, y,
                                                                 nullptr, nullptr); BEM_COUNT(ctx); }
    BEM_CK_LAUNCH(ctx);
    return BEM_OK;
}

static bem_status launch_mv(bem_operator *op, bool acc64, const double *x, double *y, const double *w,
                            double *part)
{
    bem_ctx *ctx = op->mesh->ctx;
    const unsigned g = nblk(op->N, kMvRows);
    const double es = op->precision == BEM_PREC_F64 ? 8.0 : 4.0;
    const int prof = prof_start(ctx, BEM_KERNEL_MATVEC, es * (double)op->N * (double)op->N);
    if (op->precision == BEM_PREC_F64)
        { k_matvec<double, true><<<g, kMvThreads, 0, ctx->stream>>>((const double *)op->V, op->ld, op->N, x, y, w,
                                                                  part); BEM_COUNT(ctx); }
    else if (acc64)
        { k_matvec<float, true><<<g, kMvThreads, 0, ctx->stream>>>((const float *)op->V, op->ld, op->N, x, y, w,
                                                                 part); BEM_COUNT(ctx); }
    else
        { k_matvec<float, false><<<g, kMvThreads, 0, ctx->stream>>>((const float *)op->V, op->ld, op->N, x, y, w,
                                                                  part); BEM_COUNT(ctx); }
    prof_stop(ctx, prof);
    BEM_CK_LAUNCH(ctx);
    return BEM_OK;
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
    if ((st = launch_mv(op, acc64, W.x, W.q, nullptr, nullptr))) return st;
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
        if ((st = launch_mv(op, acc64, W.p, W.q, W.p, W.part3))) return st;
        const int cur = it & 1, nxt = cur ^ 1;
        k_pcg_update1<<<W.nb_vec, kVecThreads, 0, s>>>(N, W.part3, W.nb_mv, W.scal + cur, W.x, W.r, W.z, W.p,
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

__global__ void k_capacity(int64_t N, const double *area, const double *x, double *out)
{
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) v += area[i] * x[i];
    __shared__ double part[1];
    block_partial(v, part);
    if (threadIdx.x == 0) out[0] = part[0] * kInv4Pi;
}

bem_status solve_capacity(bem_operator *op, const bem_solve_opts *o, const double *d_x0, double *d_x,
                          double *cap, bem_solve_info *info)
{
    bem_mesh *m = op->mesh;
    bem_ctx *ctx = m->ctx;
    cudaStream_t s = ctx->stream;
    const int64_t N = op->N, L = op->ld;
    Allocs tmp;
    Work W{};
    W.nb_vec = (int)nblk(N, kVecThreads);
    W.nb_mv = (int)nblk(N, kMvRows);
    const int np = W.nb_mv > W.nb_vec ? W.nb_mv : W.nb_vec;
    bem_status st = BEM_OK;
    double *base = nullptr;
    const size_t vecs = 7;
    if ((st = dalloc(ctx, tmp, (void **)&base, sizeof(double) * (vecs * L + 3 * np + 8), true))) return st;
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
    cudaError_t e = cudaMemcpyAsync(W.b, m->area, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(W.d, op->diag, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess && d_x0) e = cudaMemcpyAsync(W.x, d_x0, sizeof(double) * N, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
        st = cuda_error(ctx, e, "solve setup");
        goto out;
    }
    if (op->precision == BEM_PREC_F64) {
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
            if ((st = launch_mv(op, true, xs, W.q, nullptr, nullptr))) goto out;
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
            if ((st = pcg(op, W, rhs, inner_tol, max_it, precond, false, &it_in, &rel_in))) goto out;
            its += it_in;
            k_axpy<<<W.nb_vec, kVecThreads, 0, s>>>(N, 1.0, W.x, xs); BEM_COUNT(ctx);
            BEM_CK_LAUNCH(ctx);
        }
        if (outer == max_outer) {
            // residual of the last update
            if ((st = launch_mv(op, true, xs, W.q, nullptr, nullptr))) goto out;
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
        double c;
        if ((st = read_scalars(ctx, W.scal + 6, 1, &c))) goto out;
        *cap = c;
    }
    if (info) {
        info->iterations = its;
        info->outer = outer;
        info->relres = rel;
        info->converged = rel <= tol;
    }
    if (rel > tol) st = set_error(ctx, BEM_ERR_NOT_CONVERGED, "solve stopped at relative residual %.3e > %.3e", rel, tol);
out:
    dfree_all(ctx, tmp);
    return st;
}

}  // namespace bem
