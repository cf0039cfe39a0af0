// C ABI of the library (include/bem.h): handles, argument checks, host/device
// marshalling of caller arrays, and the adaptive loop of Alg. 1.
#include <cmath>
#include <cstdarg>
#include <new>

#include <mutex>
#include <unordered_map>

#include "bem_internal.cuh"
#include "dfloat.cuh"

namespace bem {

bem_status set_error(bem_ctx *ctx, bem_status code, const char *fmt, ...)
{
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

bem_status cuda_error(bem_ctx *ctx, cudaError_t e, const char *what)
{
    cudaGetLastError();
    return set_error(ctx, e == cudaErrorMemoryAllocation ? BEM_ERR_OOM : BEM_ERR_CUDA, "%s: %s", what,
                     cudaGetErrorString(e));
}

// Freed large blocks kept by contexts without an HBM budget: the stream-ordered pool
// keeps freed memory mapped but seldom hands an operator's block to the next
// operator of another size, and mapping new memory cost about 1 ms of host time per
// GB for every adaptive level while the GPU waited; a block is reused by a request on
// the same stream that it fits with at most 2x to spare.
constexpr size_t kCacheMaxBlock = size_t(8) << 30, kCacheMaxTotal = size_t(16) << 30;
constexpr int kCacheMaxBlocks = 6;

static void cache_put(bem_ctx *ctx, void *p, size_t bytes)
{
    ctx->block_cache.push_back(CachedBlock{p, bytes, ctx->stream});
    ctx->cache_bytes += bytes;
    while ((int)ctx->block_cache.size() > kCacheMaxBlocks || ctx->cache_bytes > kCacheMaxTotal) {
        size_t k = 0;  // drop the smallest
        for (size_t j = 1; j < ctx->block_cache.size(); ++j)
            if (ctx->block_cache[j].bytes < ctx->block_cache[k].bytes) k = j;
        cudaFreeAsync(ctx->block_cache[k].p, ctx->block_cache[k].stream);
        ctx->cache_bytes -= ctx->block_cache[k].bytes;
        ctx->block_cache.erase(ctx->block_cache.begin() + (std::ptrdiff_t)k);
    }
}

void cache_release(bem_ctx *ctx)
{
    for (auto &b : ctx->block_cache) cudaFreeAsync(b.p, b.stream);
    ctx->block_cache.clear();
    ctx->cache_bytes = 0;
}

bem_status dalloc(bem_ctx *ctx, Allocs &a, void **p, size_t bytes, bool zero)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) / 256 * 256;
    if (ctx->budget > 0 && ctx->in_use + (int64_t)bytes > ctx->budget)
        return set_error(ctx, BEM_ERR_OOM, "HBM budget exceeded: %lld in use + %zu requested > %lld",
                         (long long)ctx->in_use, bytes, (long long)ctx->budget);
    if (ctx->budget <= 0 && bytes >= kLargeAlloc) {  // a kept block that fits
        int best = -1;
        for (int k = 0; k < (int)ctx->block_cache.size(); ++k) {
            const CachedBlock &b = ctx->block_cache[k];
            if (b.stream == ctx->stream && b.bytes >= bytes && b.bytes <= 2 * bytes &&
                (best < 0 || b.bytes < ctx->block_cache[best].bytes))
                best = k;
        }
        if (best >= 0) {
            const CachedBlock b = ctx->block_cache[best];
            ctx->block_cache.erase(ctx->block_cache.begin() + best);
            ctx->cache_bytes -= b.bytes;
            *p = b.p;
            if (zero) {
                const cudaError_t e = cudaMemsetAsync(*p, 0, bytes, ctx->stream);
                if (e != cudaSuccess) {
                    cudaFreeAsync(*p, ctx->stream);
                    return cuda_error(ctx, e, "memset");
                }
            }
            a.list.emplace_back(*p, b.bytes);
            a.bytes += b.bytes;
            ctx->in_use += (int64_t)b.bytes;
            return BEM_OK;
        }
    }
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, ctx->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return set_error(ctx, BEM_ERR_OOM, "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    }
    if (zero) {
        e = cudaMemsetAsync(*p, 0, bytes, ctx->stream);
        if (e != cudaSuccess) {
            cudaFreeAsync(*p, ctx->stream);
            return cuda_error(ctx, e, "memset");
        }
    }
    a.list.emplace_back(*p, bytes);
    a.bytes += bytes;
    ctx->in_use += (int64_t)bytes;
    return BEM_OK;
}

void dfree_all(bem_ctx *ctx, Allocs &a)
{
    for (auto &pb : a.list) {
        if (ctx->budget <= 0 && pb.second >= kLargeAlloc && pb.second <= kCacheMaxBlock)
            cache_put(ctx, pb.first, pb.second);
        else
            cudaFreeAsync(pb.first, ctx->stream);
    }
    ctx->in_use -= (int64_t)a.bytes;
    a.list.clear();
    a.bytes = 0;
}

bool is_device_ptr(const void *p, int *device)
{
    if (device) *device = -1;
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (device && at.type == cudaMemoryTypeDevice) *device = at.device;
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

DevBuf::~DevBuf()
{
    if (owned && ctx) cudaFreeAsync(owned, ctx->stream);
}

bem_status dev_in(bem_ctx *ctx, const void *src, size_t bytes, DevBuf &buf)
{
    buf.ctx = ctx;
    buf.bytes = bytes;
    if (is_device_ptr(src)) {
        buf.dptr = const_cast<void *>(src);
        return BEM_OK;
    }
    BEM_CK(ctx, cudaMallocFromPoolAsync(&buf.owned, bytes ? bytes : 16, ctx->pool, ctx->stream));
    buf.dptr = buf.owned;
    if (bytes) BEM_CK(ctx, cudaMemcpyAsync(buf.owned, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    return BEM_OK;
}

bem_status dev_out_begin(bem_ctx *ctx, void *dst, size_t bytes, DevBuf &buf)
{
    buf.ctx = ctx;
    buf.bytes = bytes;
    if (is_device_ptr(dst)) {
        buf.dptr = dst;
        return BEM_OK;
    }
    BEM_CK(ctx, cudaMallocFromPoolAsync(&buf.owned, bytes ? bytes : 16, ctx->pool, ctx->stream));
    buf.dptr = buf.owned;
    return BEM_OK;
}

bem_status dev_out_end(bem_ctx *ctx, void *dst, DevBuf &buf)
{
    if (buf.owned && buf.bytes)
        BEM_CK(ctx, cudaMemcpyAsync(dst, buf.owned, buf.bytes, cudaMemcpyDeviceToHost, ctx->stream));
    BEM_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return BEM_OK;
}

template <typename T>
__global__ void k_entries(const T *V, int64_t ld, int64_t N, const int64_t *I, const int64_t *J, int64_t K,
                          double *out, int32_t *bad)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int64_t i = I[k], j = J[k];
    if (i < 0 || j < 0 || i >= N || j >= N) {
        out[k] = NAN;
        atomicOr(bad, 1);
        return;
    }
    out[k] = (double)V[i * ld + j];
}

__global__ void k_entries_df(const float2 *V, int64_t ld, int64_t N, const int64_t *I, const int64_t *J, int64_t K,
                             double *out, int32_t *bad)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= K) return;
    const int64_t i = I[k], j = J[k];
    if (i < 0 || j < 0 || i >= N || j >= N) {
        out[k] = NAN;
        atomicOr(bad, 1);
        return;
    }
    out[k] = df_to_double(V[i * ld + j]);
}

// dst[r * nj + c] = V[(i0 + r) * ld + j0 + c] as FP64
__global__ void k_block_df(const float2 *V, int64_t ld, int64_t i0, int64_t ni, int64_t j0, int64_t nj, double *dst)
{
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t r = blockIdx.y; r < ni; r += gridDim.y)
        if (c < nj) dst[r * nj + c] = df_to_double(V[(i0 + r) * ld + j0 + c]);
}

__global__ void k_prolong(const double *xc, const int32_t *parent, int64_t N, double *x)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) x[i] = xc[parent[i]];
}

static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

int prof_start(bem_ctx *ctx, int id, double units)
{
    if (!ctx->profile) return -1;
    ProfRec r{id, nullptr, nullptr, units};
    for (cudaEvent_t *e : {&r.a, &r.b}) {
        if (!ctx->ev_pool.empty()) {
            *e = ctx->ev_pool.back();
            ctx->ev_pool.pop_back();
        } else if (cudaEventCreate(e) != cudaSuccess) {
            cudaGetLastError();
            return -1;
        }
    }
    cudaEventRecord(r.a, ctx->stream);
    ctx->prof.push_back(r);
    return (int)ctx->prof.size() - 1;
}

void prof_stop(bem_ctx *ctx, int rec)
{
    if (rec >= 0 && rec < (int)ctx->prof.size()) cudaEventRecord(ctx->prof[rec].b, ctx->stream);
}

void prof_set_units(bem_ctx *ctx, int rec, double units)
{
    if (rec >= 0 && rec < (int)ctx->prof.size()) ctx->prof[rec].units = units;
}

static void prof_collect(bem_ctx *ctx)
{
    if (ctx->prof.empty()) return;
    cudaStreamSynchronize(ctx->stream);
    for (auto &r : ctx->prof) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess && r.id >= 0 && r.id < kProfKinds) {
            ctx->prof_launches[r.id] += 1;
            ctx->prof_ms[r.id] += ms;
            ctx->prof_units[r.id] += r.units;
        }
        cudaGetLastError();
        ctx->ev_pool.push_back(r.a);
        ctx->ev_pool.push_back(r.b);
    }
    ctx->prof.clear();
}

}  // namespace bem

using namespace bem;

#define CHECK_ARG(ctx, cond, msg) \
    do {                          \
        if (!(cond)) return set_error(ctx, BEM_ERR_INVALID, "%s", msg); \
    } while (0)

extern "C" {

// One stream-ordered memory pool per device for all contexts of the library.  Its
// release threshold keeps freed blocks reserved instead of returning them to the CUDA
// driver at every synchronisation; the pool is trimmed when the last context of the
// device is destroyed.  (Operator-sized blocks were seldom handed back by the pool to
// the next level's operator; contexts without a budget keep those blocks themselves,
// see dalloc.)
namespace {
std::mutex g_pool_mu;
std::unordered_map<int, std::pair<cudaMemPool_t, int>> g_pools;  // device -> (pool, contexts)

cudaError_t pool_acquire(int device, cudaMemPool_t *out)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(device);
    if (it == g_pools.end()) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t pool;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        unsigned long long keep = ~0ull;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        it = g_pools.emplace(device, std::make_pair(pool, 0)).first;
    }
    it->second.second += 1;
    *out = it->second.first;
    return cudaSuccess;
}

void pool_release(int device)
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    auto it = g_pools.find(device);
    if (it != g_pools.end() && --it->second.second == 0) cudaMemPoolTrimTo(it->second.first, 0);
}
}  // namespace

bem_status bem_context_create(void *cuda_stream, int64_t hbm_budget_bytes, bem_ctx **out)
{
    if (!out) return BEM_ERR_INVALID;
    *out = nullptr;
    bem_ctx *ctx = new (std::nothrow) bem_ctx();
    if (!ctx) return BEM_ERR_OOM;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&ctx->h_pinned, 64 * sizeof(double));
    for (int k = 0; k < 8 && e == cudaSuccess; ++k) e = cudaEventCreate(&ctx->ev[k]);
    if (e == cudaSuccess) e = pool_acquire(ctx->device, &ctx->pool);
    if (e != cudaSuccess) {
        cudaGetLastError();
        for (int k = 0; k < 8; ++k)
            if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
        if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
        delete ctx;
        return BEM_ERR_CUDA;
    }
    ctx->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    ctx->budget = hbm_budget_bytes;
    *out = ctx;
    return BEM_OK;
}

bem_status bem_profile_enable(bem_ctx *ctx, int32_t on)
{
    if (!ctx) return BEM_ERR_INVALID;
    prof_collect(ctx);
    if (on) {
        for (int k = 0; k < kProfKinds; ++k) {
            ctx->prof_launches[k] = 0;
            ctx->prof_ms[k] = 0.0;
            ctx->prof_units[k] = 0.0;
        }
    }
    ctx->profile = on ? 1 : 0;
    return BEM_OK;
}

bem_status bem_profile_read(bem_ctx *ctx, int32_t kernel, int64_t *launches, double *ms, double *units)
{
    if (!ctx) return BEM_ERR_INVALID;
    CHECK_ARG(ctx, kernel >= 0 && kernel < kProfKinds, "unknown kernel id");
    prof_collect(ctx);
    if (launches) *launches = ctx->prof_launches[kernel];
    if (ms) *ms = ctx->prof_ms[kernel];
    if (units) *units = ctx->prof_units[kernel];
    return BEM_OK;
}

bem_status bem_context_set_persistent(bem_ctx *ctx, int32_t on)
{
    if (!ctx) return BEM_ERR_INVALID;
    ctx->persistent_solver = on ? 1 : 0;
    return BEM_OK;
}

bem_status bem_debug_barrier_fault(bem_ctx *ctx, int64_t wait_limit_ns, int32_t absent_cta)
{
    if (!ctx) return BEM_ERR_INVALID;
    CHECK_ARG(ctx, absent_cta >= -1, "absent_cta must be -1 or a CTA index");
    ctx->bar_limit_ns = wait_limit_ns > 0 ? wait_limit_ns : 0;
    ctx->bar_absent_cta = absent_cta;
    return BEM_OK;
}

bem_status bem_launch_count(const bem_ctx *ctx, int64_t *n)
{
    if (!ctx || !n) return BEM_ERR_INVALID;
    *n = ctx->n_launch;
    return BEM_OK;
}

bem_status bem_context_destroy(bem_ctx *ctx)
{
    if (!ctx) return BEM_ERR_INVALID;
    cudaStreamSynchronize(ctx->stream);
    prof_collect(ctx);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
    for (int k = 0; k < 8; ++k)
        if (ctx->ev[k]) cudaEventDestroy(ctx->ev[k]);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    cache_release(ctx);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->h_levels) cudaFreeHost(ctx->h_levels);
    for (cudaEvent_t e : ctx->lvl_ev) cudaEventDestroy(e);
    if (ctx->pool) pool_release(ctx->device);
    delete ctx;
    return BEM_OK;
}

const char *bem_last_error(const bem_ctx *ctx) { return ctx ? ctx->err : "null context"; }

bem_status bem_far_tiles(const bem_ctx *ctx, int32_t out[12])
{
    if (!ctx || !out) return BEM_ERR_INVALID;
    for (int p = 0; p < 3; ++p)
        for (int c = 0; c < 4; ++c) out[4 * p + c] = ctx->far_tile[p][c] + 1;
    return BEM_OK;
}

bem_status bem_context_memory(const bem_ctx *ctx, int64_t *bytes_in_use)
{
    if (!ctx || !bytes_in_use) return BEM_ERR_INVALID;
    *bytes_in_use = ctx->in_use;
    return BEM_OK;
}

// ------------------------------------------------------------------ mesh
bem_status bem_mesh_upload(bem_ctx *ctx, const double *verts, int64_t M, const int32_t *tris, int64_t N,
                           const uint8_t *ref_edge, bem_mesh **out)
{
    if (!ctx) return BEM_ERR_INVALID;
    CHECK_ARG(ctx, out && verts && tris, "null argument");
    *out = nullptr;
    CHECK_ARG(ctx, N >= 1, "empty mesh (N = 0)");
    CHECK_ARG(ctx, M >= 3, "fewer than 3 vertices");
    CHECK_ARG(ctx, M < 0x7FFFFFFFLL && 3 * N < 0x7FFFFFFFLL, "mesh too large for 32-bit indices");
    bem_mesh *m = new (std::nothrow) bem_mesh();
    if (!m) return set_error(ctx, BEM_ERR_OOM, "host allocation");
    m->ctx = ctx;
    m->M = M;
    m->N = N;
    bem_status st = dalloc(ctx, m->allocs, (void **)&m->verts, sizeof(double) * 3 * M, false);
    if (!st) st = dalloc(ctx, m->allocs, (void **)&m->tris, sizeof(int32_t) * 3 * N, false);
    if (!st) {
        cudaError_t e = cudaMemcpyAsync(m->verts, verts, sizeof(double) * 3 * M, cudaMemcpyDefault, ctx->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(m->tris, tris, sizeof(int32_t) * 3 * N, cudaMemcpyDefault, ctx->stream);
        if (e != cudaSuccess) st = cuda_error(ctx, e, "mesh copy");
    }
    if (!st) {
        DevBuf re;
        if (ref_edge) st = dev_in(ctx, ref_edge, (size_t)N, re);
        if (!st) st = mesh_build(m, true, ref_edge ? (const uint8_t *)re.dptr : nullptr);
    }
    if (st) {
        dfree_all(ctx, m->allocs);
        delete m;
        return st;
    }
    *out = m;
    return BEM_OK;
}

bem_status bem_mesh_destroy(bem_mesh *mesh)
{
    if (!mesh) return BEM_ERR_INVALID;
    dfree_all(mesh->ctx, mesh->allocs);
    delete mesh;
    return BEM_OK;
}

bem_status bem_mesh_info(const bem_mesh *mesh, int64_t *M, int64_t *N, int64_t *n_near)
{
    if (!mesh) return BEM_ERR_INVALID;
    if (M) *M = mesh->M;
    if (N) *N = mesh->N;
    if (n_near) *n_near = 2 * (mesh->n_edge_pairs + mesh->n_vert_pairs);
    return BEM_OK;
}

bem_status bem_mesh_download(const bem_mesh *mesh, double *verts, int32_t *tris, int32_t *parent, uint8_t *kept)
{
    if (!mesh) return BEM_ERR_INVALID;
    bem_ctx *ctx = mesh->ctx;
    cudaStream_t s = ctx->stream;
    if (verts) BEM_CK(ctx, cudaMemcpyAsync(verts, mesh->verts, sizeof(double) * 3 * mesh->M, cudaMemcpyDefault, s));
    if (tris) BEM_CK(ctx, cudaMemcpyAsync(tris, mesh->tris, sizeof(int32_t) * 3 * mesh->N, cudaMemcpyDefault, s));
    BEM_CK(ctx, cudaStreamSynchronize(s));
    if (parent) {
        if (mesh->parent) {
            BEM_CK(ctx, cudaMemcpyAsync(parent, mesh->parent, sizeof(int32_t) * mesh->N, cudaMemcpyDefault, s));
        } else if (is_device_ptr(parent)) {
            BEM_CK(ctx, cudaMemsetAsync(parent, 0xFF, sizeof(int32_t) * mesh->N, s));
        } else {
            for (int64_t i = 0; i < mesh->N; ++i) parent[i] = -1;
        }
    }
    if (kept) {
        if (mesh->kept) {
            BEM_CK(ctx, cudaMemcpyAsync(kept, mesh->kept, mesh->N, cudaMemcpyDefault, s));
        } else if (is_device_ptr(kept)) {
            BEM_CK(ctx, cudaMemsetAsync(kept, 0, mesh->N, s));
        } else {
            memset(kept, 0, mesh->N);
        }
    }
    BEM_CK(ctx, cudaStreamSynchronize(s));
    return BEM_OK;
}

bem_status bem_mesh_geometry(const bem_mesh *mesh, double *area, double *diam)
{
    if (!mesh) return BEM_ERR_INVALID;
    bem_ctx *ctx = mesh->ctx;
    if (area) BEM_CK(ctx, cudaMemcpyAsync(area, mesh->area, sizeof(double) * mesh->N, cudaMemcpyDefault, ctx->stream));
    if (diam) BEM_CK(ctx, cudaMemcpyAsync(diam, mesh->diam, sizeof(double) * mesh->N, cudaMemcpyDefault, ctx->stream));
    BEM_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return BEM_OK;
}

// ------------------------------------------------------------------ operator
static bem_status operator_alloc(bem_mesh *mesh, const bem_assembly_opts *opts, bem_operator **out)
{
    bem_ctx *ctx = mesh->ctx;
    const int prec = opts ? opts->precision : BEM_PREC_F64;
    const int ss = (opts && opts->ss_order > 0) ? opts->ss_order : 4;
    CHECK_ARG(ctx, prec == BEM_PREC_F64 || prec == BEM_PREC_F32 || prec == BEM_PREC_DF64, "unknown precision");
    CHECK_ARG(ctx, ss >= 2 && ss <= kMaxSS, "ss_order outside 2..16");
    const int tile = opts ? opts->tile : 0;
    CHECK_ARG(ctx, tile >= 0 && tile <= BEM_FAR_TILE_VARIANTS, "tile outside 0..BEM_FAR_TILE_VARIANTS");
    bem_operator *op = new (std::nothrow) bem_operator();
    if (!op) return set_error(ctx, BEM_ERR_OOM, "host allocation");
    op->mesh = mesh;
    op->ctx = mesh->ctx;
    op->precision = prec;
    op->ss_order = ss;
    op->tile = tile;
    op->N = mesh->N;
    op->ld = padded_ld(mesh->N);
    const size_t es = prec == BEM_PREC_F32 ? 4 : 8;
    bem_status st = dalloc(ctx, op->allocs, &op->V, es * (size_t)op->N * (size_t)op->ld, false);
    if (!st) st = dalloc(ctx, op->allocs, (void **)&op->diag, sizeof(double) * op->N, false);
    if (st) {
        dfree_all(ctx, op->allocs);
        delete op;
        return st;
    }
    *out = op;
    return BEM_OK;
}

// Assembly of a new operator for mesh: from scratch (coarse null) or reusing the
// entries of unrefined pairs from coarse.  sync: wait for the kernels (the public
// entry points; the adaptive loop lets them run on).
static bem_status assemble_impl(bem_mesh *mesh, const bem_assembly_opts *opts, const bem_operator *coarse, bool sync,
                                bem_operator **out, bool upper_only = false)
{
    bem_ctx *ctx = mesh->ctx;
    *out = nullptr;
    bem_assembly_opts o{};
    const bem_assembly_opts *use = opts;
    if (coarse) {
        CHECK_ARG(ctx, coarse->mesh->ctx == ctx, "operator and mesh belong to different contexts");
        CHECK_ARG(ctx, !coarse->mesh->cells_only, "a dual operator has no incremental update");
        CHECK_ARG(ctx, mesh->parent != nullptr && mesh->src_N == coarse->N,
                  "mesh was not refined from the operator's mesh");
        o = bem_assembly_opts{coarse->precision, coarse->ss_order, opts ? opts->tile : coarse->tile};
        if (opts) {
            CHECK_ARG(ctx, opts->precision == coarse->precision, "precision differs from the coarse operator");
            CHECK_ARG(ctx, (opts->ss_order > 0 ? opts->ss_order : 4) == coarse->ss_order,
                      "ss_order differs from the coarse operator");
        }
        use = &o;
    }
    bem_operator *op = nullptr;
    bem_status st = operator_alloc(mesh, use, &op);
    if (st) return st;
    st = coarse ? assemble_update(op, coarse, upper_only) : assemble_full(op, upper_only);
    if (!st && sync) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_error(ctx, e, coarse ? "incremental assembly" : "assembly");
    }
    if (st) {
        bem_operator_destroy(op);
        return st;
    }
    *out = op;
    return BEM_OK;
}

bem_status bem_assemble_V(bem_mesh *mesh, const bem_assembly_opts *opts, bem_operator **out)
{
    if (!mesh || !out) return BEM_ERR_INVALID;
    return assemble_impl(mesh, opts, nullptr, true, out);
}

bem_status bem_assemble_V_update(bem_mesh *fine, const bem_operator *coarse, const bem_assembly_opts *opts,
                                 bem_operator **out)
{
    if (!fine || !coarse || !out) return BEM_ERR_INVALID;
    return assemble_impl(fine, opts, coarse, true, out);
}

bem_status bem_operator_destroy(bem_operator *op)
{
    if (!op) return BEM_ERR_INVALID;
    dfree_all(op->ctx, op->allocs);
    if (op->owns_mesh && op->mesh) {
        dfree_all(op->ctx, op->mesh->allocs);
        delete op->mesh;
    }
    delete op;
    return BEM_OK;
}

bem_status bem_mesh_barycentric(bem_mesh *mesh, bem_mesh **out)
{
    if (!mesh || !out) return BEM_ERR_INVALID;
    *out = nullptr;
    CHECK_ARG(mesh->ctx, !mesh->cells_only, "not a triangle mesh");
    bem_status st = barycentric(mesh, out);
    if (!st) {
        cudaError_t e = cudaStreamSynchronize(mesh->ctx->stream);
        if (e != cudaSuccess) st = cuda_error(mesh->ctx, e, "barycentric refinement");
    }
    return st;
}

bem_status bem_operator_dual(bem_operator *bary_op, bem_mesh *mesh, bem_operator **out)
{
    if (!bary_op || !mesh || !out) return BEM_ERR_INVALID;
    bem_ctx *ctx = mesh->ctx;
    *out = nullptr;
    CHECK_ARG(ctx, bary_op->ctx == ctx, "operator and mesh belong to different contexts");
    CHECK_ARG(ctx, !mesh->cells_only && bary_op->N == 6 * mesh->N,
              "the operator must be that of the barycentric refinement of the mesh (6 N triangles)");
    return dual_operator(bary_op, mesh, out);
}

bem_status bem_zz_estimate_dual(bem_mesh *mesh, const double *x, int32_t h_mode, double *eta2_out, double *totals)
{
    if (!mesh) return BEM_ERR_INVALID;
    bem_ctx *ctx = mesh->ctx;
    CHECK_ARG(ctx, x && eta2_out && !mesh->cells_only, "null argument");
    CHECK_ARG(ctx, h_mode == 0 || h_mode == 1, "h_mode must be 0 or 1");
    DevBuf dx, de;
    bem_status st;
    if ((st = dev_in(ctx, x, sizeof(double) * (size_t)mesh->M, dx))) return st;
    if ((st = dev_out_begin(ctx, eta2_out, sizeof(double) * (size_t)mesh->N, de))) return st;
    if ((st = zz_estimate_dual(mesh, (const double *)dx.dptr, h_mode, (double *)de.dptr, totals))) return st;
    return dev_out_end(ctx, eta2_out, de);
}

bem_status bem_operator_preconditioner(const bem_operator *op, int32_t which, float *dst)
{
    if (!op) return BEM_ERR_INVALID;
    bem_ctx *ctx = op->ctx;
    CHECK_ARG(ctx, dst != nullptr, "null destination");
    CHECK_ARG(ctx, which == 0 || which == 1, "which must be 0 (D^reg) or 1 (C)");
    CHECK_ARG(ctx, op->cal_D != nullptr, "the operator carries no preconditioner (not a dual operator)");
    cudaError_t e = cudaMemcpy2DAsync(dst, sizeof(float) * op->N, which ? op->cal_C : op->cal_D, sizeof(float) * op->ld,
                                      sizeof(float) * op->N, op->N, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    return e == cudaSuccess ? BEM_OK : cuda_error(ctx, e, "preconditioner read");
}

bem_status bem_operator_info(const bem_operator *op, int64_t *N, int32_t *precision)
{
    if (!op) return BEM_ERR_INVALID;
    if (N) *N = op->N;
    if (precision) *precision = op->precision;
    return BEM_OK;
}

bem_status bem_operator_read(const bem_operator *op, int64_t i0, int64_t ni, int64_t j0, int64_t nj, void *dst)
{
    if (!op) return BEM_ERR_INVALID;
    bem_ctx *ctx = op->mesh->ctx;
    CHECK_ARG(ctx, dst != nullptr, "null destination");
    CHECK_ARG(ctx, i0 >= 0 && j0 >= 0 && ni >= 0 && nj >= 0 && i0 + ni <= op->N && j0 + nj <= op->N,
              "block outside the operator");
    if (ni == 0 || nj == 0) return BEM_OK;
    if (op->upper_only) {  // never the case for operators handed to callers; kept safe
        bem_status sf = ensure_full(const_cast<bem_operator *>(op));
        if (sf) return sf;
    }
    if (op->precision == BEM_PREC_DF64) {
        Allocs tmp;
        double *blk = nullptr;
        bem_status st = dalloc(ctx, tmp, (void **)&blk, sizeof(double) * ni * nj, false);
        if (st) return st;
        dim3 grid(nblk(nj, 256), (unsigned)(ni < 65535 ? ni : 65535));
        k_block_df<<<grid, 256, 0, ctx->stream>>>((const float2 *)op->V, op->ld, i0, ni, j0, nj, blk); BEM_COUNT(ctx);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaMemcpyAsync(dst, blk, sizeof(double) * ni * nj, cudaMemcpyDefault, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_error(ctx, e, "operator read");
        dfree_all(ctx, tmp);
        return st;
    }
    const size_t es = op->precision == BEM_PREC_F64 ? 8 : 4;
    const char *src = static_cast<const char *>(op->V) + es * (size_t)(i0 * op->ld + j0);
    BEM_CK(ctx, cudaMemcpy2DAsync(dst, es * nj, src, es * op->ld, es * nj, ni, cudaMemcpyDefault, ctx->stream));
    BEM_CK(ctx, cudaStreamSynchronize(ctx->stream));
    return BEM_OK;
}

bem_status bem_operator_entries(const bem_operator *op, const int64_t *I, const int64_t *J, int64_t K, double *out)
{
    if (!op) return BEM_ERR_INVALID;
    bem_ctx *ctx = op->mesh->ctx;
    CHECK_ARG(ctx, K >= 0, "negative count");
    if (K == 0) return BEM_OK;
    CHECK_ARG(ctx, I && J && out, "null argument");
    DevBuf dI, dJ, dO;
    bem_status st;
    if ((st = dev_in(ctx, I, sizeof(int64_t) * K, dI))) return st;
    if ((st = dev_in(ctx, J, sizeof(int64_t) * K, dJ))) return st;
    if ((st = dev_out_begin(ctx, out, sizeof(double) * K, dO))) return st;
    Allocs tmp;
    int32_t *bad = nullptr;
    if (op->upper_only && (st = ensure_full(const_cast<bem_operator *>(op)))) return st;
    if ((st = dalloc(ctx, tmp, (void **)&bad, sizeof(int32_t), true))) return st;
    if (op->precision == BEM_PREC_DF64)
        { k_entries_df<<<nblk(K, 256), 256, 0, ctx->stream>>>((const float2 *)op->V, op->ld, op->N,
                                                               (const int64_t *)dI.dptr, (const int64_t *)dJ.dptr, K,
                                                               (double *)dO.dptr, bad); BEM_COUNT(ctx); }
    else if (op->precision == BEM_PREC_F64)
        { k_entries<double><<<nblk(K, 256), 256, 0, ctx->stream>>>((const double *)op->V, op->ld, op->N,
                                                                 (const int64_t *)dI.dptr, (const int64_t *)dJ.dptr, K,
                                                                 (double *)dO.dptr, bad); BEM_COUNT(ctx); }
    else
        { k_entries<float><<<nblk(K, 256), 256, 0, ctx->stream>>>((const float *)op->V, op->ld, op->N,
                                                                (const int64_t *)dI.dptr, (const int64_t *)dJ.dptr, K,
                                                                (double *)dO.dptr, bad); BEM_COUNT(ctx); }
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->h_pinned, bad, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream);
    if (e != cudaSuccess) st = cuda_error(ctx, e, "entries");
    if (!st) st = dev_out_end(ctx, out, dO);
    if (!st && *reinterpret_cast<int32_t *>(ctx->h_pinned)) st = set_error(ctx, BEM_ERR_INVALID, "entry index out of range");
    dfree_all(ctx, tmp);
    return st;
}

bem_status bem_operator_matvec(const bem_operator *op, const double *x, double *y)
{
    if (!op) return BEM_ERR_INVALID;
    bem_ctx *ctx = op->mesh->ctx;
    CHECK_ARG(ctx, x && y, "null argument");
    Allocs tmp;
    double *xb = nullptr;
    bem_status st = dalloc(ctx, tmp, (void **)&xb, sizeof(double) * 2 * op->ld, true);
    if (st) return st;
    double *yb = xb + op->ld;
    cudaError_t e = cudaMemcpyAsync(xb, x, sizeof(double) * op->N, cudaMemcpyDefault, ctx->stream);
    if (e != cudaSuccess) st = cuda_error(ctx, e, "matvec input");
    if (!st) st = matvec_f64(const_cast<bem_operator *>(op), xb, yb);
    if (!st) {
        e = cudaMemcpyAsync(y, yb, sizeof(double) * op->N, cudaMemcpyDefault, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_error(ctx, e, "matvec output");
    }
    dfree_all(ctx, tmp);
    return st;
}

// ------------------------------------------------------------------ solve
static bem_solve_opts default_solve_opts()
{
    bem_solve_opts o;
    o.tol = 1e-10;
    o.max_it = 10000;
    o.precond = BEM_PRECOND_JACOBI;
    o.max_outer = 20;
    o.inner_tol = 1e-5;
    o.reliable_delta = 0.0;
    o.inexact_lambda = 0.0;
    o.h_mode = 0;
    return o;
}

bem_status bem_solve_capacity(bem_operator *op, const bem_solve_opts *opts, const double *x0, double *cap_out,
                              double *phi_out, bem_solve_info *info)
{
    if (!op) return BEM_ERR_INVALID;
    bem_ctx *ctx = op->mesh->ctx;
    CHECK_ARG(ctx, cap_out != nullptr, "null cap_out");
    const bem_solve_opts o = opts ? *opts : default_solve_opts();
    CHECK_ARG(ctx, o.precond >= BEM_PRECOND_NONE && o.precond <= BEM_PRECOND_CALDERON, "unknown preconditioner");
    CHECK_ARG(ctx, !(o.tol < 0), "negative tolerance");
    const size_t vb = sizeof(double) * op->N;
    DevBuf dx0, dphi;
    bem_status st;
    if (x0 && (st = dev_in(ctx, x0, vb, dx0))) return st;
    if (phi_out && (st = dev_out_begin(ctx, phi_out, vb, dphi))) return st;
    st = solve_capacity(op, &o, x0 ? (const double *)dx0.dptr : nullptr,
                        phi_out ? (double *)dphi.dptr : nullptr, cap_out, info);
    if ((st == BEM_OK || st == BEM_ERR_NOT_CONVERGED) && phi_out) {
        bem_status s2 = dev_out_end(ctx, phi_out, dphi);
        if (s2) return s2;
    }
    return st;
}

// ------------------------------------------------------------------ adaptivity
bem_status bem_zz_estimate(bem_mesh *mesh, const double *phi, int32_t h_mode, double *eta2_out, double *totals)
{
    if (!mesh) return BEM_ERR_INVALID;
    bem_ctx *ctx = mesh->ctx;
    CHECK_ARG(ctx, phi && eta2_out, "null argument");
    CHECK_ARG(ctx, h_mode == 0 || h_mode == 1, "h_mode must be 0 or 1");
    const size_t vb = sizeof(double) * mesh->N;
    DevBuf dphi, deta;
    bem_status st;
    if ((st = dev_in(ctx, phi, vb, dphi))) return st;
    if ((st = dev_out_begin(ctx, eta2_out, vb, deta))) return st;
    if ((st = zz_estimate(mesh, (const double *)dphi.dptr, h_mode, (double *)deta.dptr, totals))) return st;
    return dev_out_end(ctx, eta2_out, deta);
}

bem_status bem_dorfler(bem_ctx *ctx, const double *eta2, int64_t N, double theta, uint8_t *marked, int64_t *n_marked)
{
    if (!ctx) return BEM_ERR_INVALID;
    CHECK_ARG(ctx, N >= 0, "negative size");
    CHECK_ARG(ctx, theta > 0.0 && theta <= 1.0, "theta must lie in (0, 1]");
    if (N == 0) {
        if (n_marked) *n_marked = 0;
        return BEM_OK;
    }
    CHECK_ARG(ctx, eta2 && marked, "null argument");
    DevBuf de, dm;
    bem_status st;
    if ((st = dev_in(ctx, eta2, sizeof(double) * N, de))) return st;
    if ((st = dev_out_begin(ctx, marked, (size_t)N, dm))) return st;
    if ((st = dorfler(ctx, (const double *)de.dptr, N, theta, (uint8_t *)dm.dptr, n_marked))) return st;
    return dev_out_end(ctx, marked, dm);
}

bem_status bem_refine(bem_mesh *mesh, const uint8_t *marked, int32_t flags, bem_mesh **refined_out)
{
    if (!mesh) return BEM_ERR_INVALID;
    bem_ctx *ctx = mesh->ctx;
    CHECK_ARG(ctx, marked && refined_out, "null argument");
    *refined_out = nullptr;
    DevBuf dm;
    bem_status st;
    if ((st = dev_in(ctx, marked, (size_t)mesh->N, dm))) return st;
    return refine(mesh, (const uint8_t *)dm.dptr, flags, refined_out);
}

bem_status bem_mark_refine(bem_mesh *mesh, const double *eta2, double theta, int32_t flags, uint8_t *marked_out,
                           int64_t *n_marked, bem_mesh **refined_out)
{
    if (!mesh) return BEM_ERR_INVALID;
    bem_ctx *ctx = mesh->ctx;
    CHECK_ARG(ctx, eta2 && refined_out, "null argument");
    CHECK_ARG(ctx, theta > 0.0 && theta <= 1.0, "theta must lie in (0, 1]");
    *refined_out = nullptr;
    Allocs tmp;
    uint8_t *dm = nullptr;
    bem_status st = dalloc(ctx, tmp, (void **)&dm, (size_t)mesh->N, false);
    if (st) return st;
    DevBuf de;
    int64_t nm = 0;
    if (!st) st = dev_in(ctx, eta2, sizeof(double) * mesh->N, de);
    if (!st) st = dorfler(ctx, (const double *)de.dptr, mesh->N, theta, dm, &nm);
    if (!st && marked_out) {
        cudaError_t e = cudaMemcpyAsync(marked_out, dm, (size_t)mesh->N, cudaMemcpyDefault, ctx->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) st = cuda_error(ctx, e, "marked copy");
    }
    if (!st && n_marked) *n_marked = nm;
    if (!st) st = refine(mesh, dm, flags, refined_out);
    dfree_all(ctx, tmp);
    return st;
}

// ------------------------------------------------------------------ adaptive loop
static float elapsed(cudaEvent_t a, cudaEvent_t b)
{
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        ms = 0.0f;
    }
    return ms;
}

// Children 6t .. 6t+5 of the kept primal triangles t < K keep their parent's children
// 6 parent[t] .. 6 parent[t] + 5: the parent map of the barycentric refinement.
__global__ void k_bary_parent(const int32_t *parent, int64_t K, int32_t *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 6 * K) out[i] = 6 * parent[i / 6] + (int32_t)(i % 6);
}

// The barycentric refinement and its operator of the previous level, kept for the
// incremental assembly of the next one.
struct BaryLevel {
    bem_mesh *mesh = nullptr;
    bem_operator *op = nullptr;
    void release()
    {
        if (op) bem_operator_destroy(op);
        if (mesh) bem_mesh_destroy(mesh);
        op = nullptr;
        mesh = nullptr;
    }
};

// Operator of one level of the dual-basis loop: barycentric refinement, its operator,
// V^dual.  With incremental, the children of the kept primal triangles (the first 6K
// barycentric triangles, geometry and adjacency unchanged under conforming NVB) take
// their entries from the previous level's barycentric operator (bem_assemble_V_update);
// the refinement and its operator are then kept for the next level.
static bem_status dual_level_operator(bem_mesh *cur, const bem_assembly_opts *aopts, bool incremental,
                                      BaryLevel &prev, bem_operator **out)
{
    bem_ctx *ctx = cur->ctx;
    bem_mesh *b = nullptr;
    bem_operator *ob = nullptr;
    bem_status st = barycentric(cur, &b);
    const bool inc = incremental && prev.op && cur->parent && cur->n_kept > 0 && prev.op->N == 6 * cur->src_N;
    if (!st && inc) {
        st = dalloc(ctx, b->allocs, (void **)&b->parent, sizeof(int32_t) * (size_t)b->N, false);
        if (!st) {
            k_bary_parent<<<nblk(6 * cur->n_kept, 256), 256, 0, ctx->stream>>>(cur->parent, cur->n_kept, b->parent);
            BEM_COUNT(ctx);
            b->n_kept = 6 * cur->n_kept;
            b->src_N = prev.op->N;
            st = bem_assemble_V_update(b, prev.op, aopts, &ob);
        }
    } else if (!st) {
        st = bem_assemble_V(b, aopts, &ob);
    }
    prev.release();
    if (!st) st = dual_operator(ob, cur, out);
    if (!st && incremental) {
        prev.mesh = b;
        prev.op = ob;
    } else {
        if (ob) bem_operator_destroy(ob);
        if (b) bem_mesh_destroy(b);
    }
    return st;
}

// Pinned result slots and timing events for `levels` levels of the adaptive loop.
static bem_status level_slots(bem_ctx *ctx, int levels)
{
    if (ctx->h_levels_cap < levels) {
        cache_release(ctx);
    cudaStreamSynchronize(ctx->stream);
    if (ctx->h_levels) cudaFreeHost(ctx->h_levels);
        ctx->h_levels = nullptr;
        ctx->h_levels_cap = 0;
        BEM_CK(ctx, cudaMallocHost((void **)&ctx->h_levels, sizeof(double) * 16 * (size_t)levels));
        ctx->h_levels_cap = levels;
    }
    while ((int)ctx->lvl_ev.size() < 4 * levels) {
        cudaEvent_t e = nullptr;
        BEM_CK(ctx, cudaEventCreate(&e));
        ctx->lvl_ev.push_back(e);
    }
    return BEM_OK;
}

bem_status bem_adaptive_run(bem_mesh *mesh, const bem_adaptive_opts *opts, bem_level_record *records, int32_t *n_levels,
                            bem_mesh **final_mesh)
{
    if (!mesh) return BEM_ERR_INVALID;
    bem_ctx *ctx = mesh->ctx;
    CHECK_ARG(ctx, opts && records && n_levels, "null argument");
    CHECK_ARG(ctx, opts->max_levels >= 1, "max_levels < 1");
    CHECK_ARG(ctx, opts->theta > 0.0 && opts->theta <= 1.0, "theta must lie in (0, 1]");
    CHECK_ARG(ctx, opts->basis == BEM_BASIS_P0 || opts->basis == BEM_BASIS_DUAL, "unknown basis");
    const bool dual = opts->basis == BEM_BASIS_DUAL;
    CHECK_ARG(ctx, !(dual && opts->solve.inexact_lambda > 0.0), "the inexact stopping rule needs the P0 basis");
    CHECK_ARG(ctx, dual || opts->solve.precond != BEM_PRECOND_CALDERON, "BEM_PRECOND_CALDERON needs the dual basis");
    if (final_mesh) *final_mesh = nullptr;
    *n_levels = 0;
    bem_status st = level_slots(ctx, opts->max_levels);
    if (st) return st;
    // The loop synchronises with the host only where it needs a count: the sizes of the
    // refined mesh (refine) and its touching-pair lists.  The solve's results, the ZZ
    // totals and the Doerfler count travel to pinned slots meanwhile and are read after
    // that synchronisation; the per-phase times come from events read once at the end.
    cudaStream_t s = ctx->stream;
    bem_mesh *cur = mesh;
    bem_mesh *prev_mesh = nullptr;  // mesh of op_prev, destroyed after op_prev
    bem_operator *op_prev = nullptr;
    BaryLevel bary_prev;  // dual basis: the previous level's barycentric operator
    Allocs xprev_alloc;
    double *x_prev = nullptr;
    for (int lvl = 0; lvl < opts->max_levels; ++lvl) {
        bem_level_record &rec = records[lvl];
        memset(&rec, 0, sizeof(rec));
        rec.N = cur->N;
        rec.M = cur->M;
        double *slot = ctx->h_levels + 16 * (size_t)lvl;
        cudaEvent_t *ev = &ctx->lvl_ev[4 * (size_t)lvl];
        cudaEventRecord(ev[0], s);
        bem_operator *op = nullptr;
        if (dual)
            st = dual_level_operator(cur, &opts->assembly, opts->incremental != 0, bary_prev, &op);
        else if (op_prev && opts->incremental && cur->parent)
            st = assemble_impl(cur, &opts->assembly, op_prev, false, &op, true);
        else
            st = assemble_impl(cur, &opts->assembly, nullptr, false, &op, true);
        if (op_prev) {
            bem_operator_destroy(op_prev);
            op_prev = nullptr;
        }
        if (prev_mesh && prev_mesh != mesh) bem_mesh_destroy(prev_mesh);
        prev_mesh = nullptr;
        if (st) break;
        cudaEventRecord(ev[1], s);
        Allocs lv;
        double *x0 = nullptr, *x = nullptr, *eta2 = nullptr, *dsc = nullptr;
        const int64_t nx = dual ? cur->M : cur->N;  // unknowns: vertices or triangles
        st = dalloc(ctx, lv, (void **)&x, sizeof(double) * (2 * nx + cur->N + 4), false);
        if (st) { bem_operator_destroy(op); break; }
        x0 = x + nx;
        eta2 = x + 2 * nx;
        dsc = eta2 + cur->N;  // [0..1] ZZ totals, [2] Doerfler count (long long)
        if (!dual && x_prev && cur->parent) {
            k_prolong<<<nblk(cur->N, 256), 256, 0, s>>>(x_prev, cur->parent, cur->N, x0); BEM_COUNT(ctx);
        } else {
            x0 = nullptr;
        }
        bem_solve_info info{};
        double cap = 0.0;
        bem_solve_opts so = opts->solve;
        so.h_mode = opts->h_mode;  // the estimator of the inexact stopping rule
        SolveDeferred def;
        def.h = slot;
        st = solve_capacity(op, &so, x0, x, &cap, &info, &def);
        if (st) { dfree_all(ctx, lv); bem_operator_destroy(op); break; }
        cudaEventRecord(ev[2], s);
        double tot[2] = {0.0, 0.0};
        if (dual) {
            st = zz_estimate_dual(cur, x, opts->h_mode, eta2, tot);
            slot[8] = tot[0];
            slot[9] = tot[1];
        } else {
            st = zz_estimate(cur, x, opts->h_mode, eta2, nullptr, dsc);
            if (!st) {
                cudaError_t e = cudaMemcpyAsync(slot + 8, dsc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
                if (e != cudaSuccess) st = cuda_error(ctx, e, "ZZ totals");
            }
        }
        bem_mesh *next = nullptr;
        const bool last = cur->N >= opts->max_N || lvl == opts->max_levels - 1;
        long long *hcount = reinterpret_cast<long long *>(slot + 10);
        *hcount = 0;
        if (!st && !last) {
            Allocs mk;
            uint8_t *dm = nullptr;
            st = dalloc(ctx, mk, (void **)&dm, (size_t)cur->N, false);
            if (!st && dual) {
                int64_t nm = 0;
                if (!(tot[0] > 1e-20 * tot[1])) {
                    // every indicator vanishes up to rounding: refine uniformly
                    cudaMemsetAsync(dm, 1, (size_t)cur->N, s);
                    nm = cur->N;
                } else {
                    st = dorfler(ctx, eta2, cur->N, opts->theta, dm, &nm);
                }
                *hcount = nm;
            } else if (!st) {
                // the vanishing-estimator rule is taken on the device from the totals
                long long *dcount = reinterpret_cast<long long *>(dsc + 2);
                st = dorfler(ctx, eta2, cur->N, opts->theta, dm, nullptr, dsc, dcount);
                if (!st) {
                    cudaError_t e = cudaMemcpyAsync(hcount, dcount, sizeof(long long), cudaMemcpyDeviceToHost, s);
                    if (e != cudaSuccess) st = cuda_error(ctx, e, "Doerfler count");
                }
            }
            // synchronises: the new mesh's sizes; the new mesh's checks are read with
            // the next level's sizes (or at the end)
            if (!st) st = refine(cur, dm, 0, &next, true);
            dfree_all(ctx, mk);
        }
        cudaEventRecord(ev[3], s);
        if (last || st) cudaEventSynchronize(ev[3]);
        // the level's results are in their pinned slot now
        bem_status st_solve = BEM_OK;
        if (def.pending) st_solve = solve_capacity_end(ctx, def, &cap, &info);
        rec.cap = cap;
        rec.iterations = info.iterations;
        rec.outer = info.outer;
        rec.relres = info.relres;
        rec.eta2_total = slot[8];
        rec.n_marked = last ? 0 : (int32_t)*hcount;
        if (st_solve) {  // a failed solve ends the loop; its level is not counted
            st = st_solve;
        } else {
            *n_levels = lvl + 1;
        }
        // keep this level's solution for the warm start of the next one
        dfree_all(ctx, xprev_alloc);
        x_prev = nullptr;
        if (!st && next && !dual) {
            if ((st = dalloc(ctx, xprev_alloc, (void **)&x_prev, sizeof(double) * cur->N, false)) == BEM_OK) {
                cudaError_t e = cudaMemcpyAsync(x_prev, x, sizeof(double) * cur->N, cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) st = cuda_error(ctx, e, "warm start copy");
            }
        }
        dfree_all(ctx, lv);
        if (st || !next) {
            if (next) bem_mesh_destroy(next);
            bem_operator_destroy(op);
            break;
        }
        op_prev = op;
        prev_mesh = cur;
        cur = next;
    }
    // the last mesh's deferred checks, then the per-phase device times of every level
    if (!st && cur != mesh) st = mesh_check_pending(cur);
    cudaStreamSynchronize(s);
    for (int l = 0; l < *n_levels; ++l) {
        cudaEvent_t *ev = &ctx->lvl_ev[4 * (size_t)l];
        records[l].ms_assemble = elapsed(ev[0], ev[1]);
        records[l].ms_solve = elapsed(ev[1], ev[2]);
        records[l].ms_adapt = elapsed(ev[2], ev[3]);
    }
    if (op_prev) bem_operator_destroy(op_prev);
    if (prev_mesh && prev_mesh != mesh) bem_mesh_destroy(prev_mesh);
    bary_prev.release();
    dfree_all(ctx, xprev_alloc);
    if (final_mesh && cur != mesh && !st) {
        *final_mesh = cur;
    } else if (cur != mesh) {
        bem_mesh_destroy(cur);
    }
    return st;
}

}  // extern "C"

namespace bem {
bem_status new_operator(bem_mesh *mesh, const bem_assembly_opts *opts, bem_operator **out)
{
    return operator_alloc(mesh, opts, out);
}
}  // namespace bem
