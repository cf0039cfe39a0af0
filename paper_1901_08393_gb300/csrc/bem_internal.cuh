// Internal declarations of the GB300 BEM capacity library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/bem.h"

namespace bem {

constexpr int kQ = 7;              // far-field points per triangle (Radon degree 5)
constexpr int kQ64Stride = 24;     // doubles per triangle in the FP64 point table
constexpr int kQ32Stride = 24;     // floats per triangle in the FP32 offset table
constexpr int kQdfStride = 56;     // floats per triangle in the double-float table:
                                   // [0,42) offsets hi/lo, [42,51) centroid as 3 floats
                                   // per coordinate, [51,53) area hi/lo, [53] the
                                   // largest |hi| of the offsets, [54] the largest
                                   // distance of a point from the centroid
constexpr int kMaxSS = 16;         // largest Sauter-Schwab order accepted
constexpr int kMaxValence = 96;    // triangles per vertex accepted by the pair builder
constexpr double kInv4Pi = 0.079577471545947668;  // 1 / (4 pi)
constexpr int kFarTileVariants = BEM_FAR_TILE_VARIANTS;  // far-field pair tile shapes

// Row stride of the dense operator: N rounded up to 64 elements so that every row
// starts on a 256-byte boundary (vector loads) and whole 64 x 64 tiles fit (the
// symmetric matvec); the padding columns are zero.
inline int64_t padded_ld(int64_t n) { return (n + 63) / 64 * 64; }

constexpr size_t kLargeAlloc = size_t(64) << 20;  // blocks from this size up are kept for reuse (dalloc)

struct Allocs {
    std::vector<std::pair<void *, size_t>> list;
    size_t bytes = 0;
};

}  // namespace bem

namespace bem {
struct CachedBlock {
    void *p;
    size_t bytes;
    cudaStream_t stream;  // the stream it was freed on (reused only there)
};
struct ProfRec {
    int id;
    cudaEvent_t a, b;
    double units;
};
constexpr int kProfKinds = 4;
}  // namespace bem

struct bem_ctx {
    int64_t n_launch = 0;  // kernels launched by this context
    int profile = 0;       // record CUDA events around the hot kernels
    int persistent_solver = 1;  // DF64 solves in one cooperative launch
    std::vector<bem::ProfRec> prof;
    std::vector<cudaEvent_t> ev_pool;
    int64_t prof_launches[bem::kProfKinds] = {0, 0, 0, 0};
    double prof_ms[bem::kProfKinds] = {0, 0, 0, 0};
    double prof_units[bem::kProfKinds] = {0, 0, 0, 0};
    cudaStream_t stream = nullptr;
    cudaMemPool_t pool = nullptr;  // the library's stream-ordered pool of this device
    int device = 0;
    int sm_count = 0;
    int64_t budget = 0;  // <= 0: unlimited
    int64_t in_use = 0;
    char err[1024] = {0};
    double *h_pinned = nullptr;  // 64 doubles of pinned host memory for scalar readbacks
    cudaEvent_t ev[8] = {};
    int8_t far_tile[3][4] = {{-1, -1, -1, -1}, {-1, -1, -1, -1}, {-1, -1, -1, -1}};  // autotuned variant
    // freed large blocks kept for reuse (contexts without a budget; see dalloc)
    std::vector<bem::CachedBlock> block_cache;
    size_t cache_bytes = 0;
    // adaptive loop: pinned per-level result slots (16 doubles each) and timing events
    double *h_levels = nullptr;
    int h_levels_cap = 0;
    std::vector<cudaEvent_t> lvl_ev;
    int64_t bar_limit_ns = 0;   // persistent solver: grid-barrier wait limit (0: default)
    int32_t bar_absent_cta = -1;  // failure-detection tests: CTA that leaves at its first barrier
};

struct bem_mesh {
    bem_ctx *ctx = nullptr;
    int64_t M = 0, N = 0;
    double *verts = nullptr;    // M x 3
    int32_t *tris = nullptr;    // N x 3, reference edge first
    double *area = nullptr;     // N
    double *diam = nullptr;     // N
    double *q64 = nullptr;      // N x 24: 7 points (x,y,z), [21] = area
    float *q32 = nullptr;       // N x 24: 7 offsets from the centroid (x,y,z)
    double *cent = nullptr;     // N x 4: centroid (x,y,z), area
    float *qdf = nullptr;       // N x 56: double-float table (see kQdfStride)
    int32_t *v2t_off = nullptr; // M + 1
    int32_t *v2t = nullptr;     // 3N, ascending triangle index per vertex
    int32_t *owner = nullptr;   // 3N: half-edge -> first half-edge of its edge
    int64_t n_edge_pairs = 0;   // touching pairs i < j sharing an edge
    int64_t n_vert_pairs = 0;   // touching pairs i < j sharing one vertex
    int32_t *edge_pairs = nullptr;  // 2 x n_edge_pairs (i, j), ascending (i, j)
    int32_t *vert_pairs = nullptr;  // 2 x n_vert_pairs
    int32_t *parent = nullptr;  // N or null (refined meshes)
    uint8_t *kept = nullptr;    // N or null
    int64_t n_kept = 0;         // refined meshes: triangles [0, n_kept) are unrefined
    int64_t src_N = 0;          // refined meshes: N of the source mesh
    int cells_only = 0;         // dual cells of an operator from bem_operator_dual: N, area, cent only
    // checks of a mesh built by the adaptive loop's refinement (degenerate, not closed,
    // duplicate: flags 1..3 of d_bad), read with the next count the loop needs anyway
    int32_t *d_bad = nullptr;
    int bad_pending = 0;
    bem::Allocs allocs;
};

struct bem_operator {
    bem_mesh *mesh = nullptr;
    bem_ctx *ctx = nullptr;  // kept apart from mesh: an operator may be destroyed after its mesh
    int32_t precision = BEM_PREC_F64;
    int32_t ss_order = 4;
    int32_t tile = 0;       // requested far-field tile variant (1-based), 0: autotuned
    int64_t N = 0, ld = 0;
    void *V = nullptr;      // N x ld, row-major: double (F64), float2 hi/lo (DF64), float (F32)
    double *diag = nullptr; // N, FP64 diagonal
    int owns_mesh = 0;      // 1: mesh is a cells mesh freed with the operator
    // 1: only the upper triangle (i <= j) and the diagonal 64 x 64 blocks hold entries
    // (operators of the adaptive loop, read by the symmetric products alone);
    // ensure_full mirrors the rest before any reader of whole rows
    int upper_only = 0;
    // dual operators: the regularised hypersingular operator D^reg and the operator
    // preconditioner C = S D^reg S (both FP32, N x ld)
    float *cal_D = nullptr, *cal_C = nullptr;
    bem::Allocs allocs;
};

namespace bem {

// ----------------------------------------------------------------- host helpers
bem_status set_error(bem_ctx *ctx, bem_status code, const char *fmt, ...);
bem_status cuda_error(bem_ctx *ctx, cudaError_t e, const char *what);
bem_status dalloc(bem_ctx *ctx, Allocs &a, void **p, size_t bytes, bool zero);
void dfree_all(bem_ctx *ctx, Allocs &a);
void cache_release(bem_ctx *ctx);  // free the kept blocks (stream-ordered)
// True for device or managed memory; device (nullable) receives the device that holds
// plain device memory (-1 for managed or host memory).
bool is_device_ptr(const void *p, int *device = nullptr);

#define BEM_CK(ctx, call)                                              \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return ::bem::cuda_error(ctx, e_, #call); \
    } while (0)

#define BEM_CK_LAUNCH(ctx) BEM_CK(ctx, cudaGetLastError())
#define BEM_COUNT(ctx) (++(ctx)->n_launch)

// Event pair around one hot-kernel launch (no-op unless profiling is on).
int prof_start(bem_ctx *ctx, int id, double units);
void prof_stop(bem_ctx *ctx, int rec);
void prof_set_units(bem_ctx *ctx, int rec, double units);

// Temporary device copy of a caller array (host or device).
struct DevBuf {
    bem_ctx *ctx = nullptr;
    void *dptr = nullptr;
    void *owned = nullptr;
    size_t bytes = 0;
    ~DevBuf();
};
bem_status dev_in(bem_ctx *ctx, const void *src, size_t bytes, DevBuf &buf);
bem_status dev_out_begin(bem_ctx *ctx, void *dst, size_t bytes, DevBuf &buf);
bem_status dev_out_end(bem_ctx *ctx, void *dst, DevBuf &buf);

// Exclusive prefix sum of n int32 counts into out (n + 1 entries), on the stream;
// returns the total through a synchronous read when total != nullptr.
bem_status exclusive_scan_i32(bem_ctx *ctx, const int32_t *in, int32_t *out, int64_t n,
                              int64_t *total);
// Read n (<= 64) int32 device scalars with one synchronisation of the stream.
bem_status read_i32s(bem_ctx *ctx, const int32_t *const *src, int n, int64_t *out);

// ----------------------------------------------------------------- mesh (mesh.cu)
// Build every derived array of a mesh whose verts / tris are already on the device.
bem_status mesh_build(bem_mesh *m, bool canonicalize, const uint8_t *d_ref_edge, bool defer_check = false);
// the error of the mesh check flags bad[1..3] (BEM_OK if none is raised)
bem_status mesh_bad_status(bem_ctx *ctx, const int64_t *bad3);

// ----------------------------------------------------------------- assembly (assemble.cu)
bem_status gauss_legendre_upload(int n);
bem_status assemble_full(bem_operator *op, bool upper_only = false);
// Operator handle with V (uninitialised) and diag allocated for mesh (api.cu).
bem_status new_operator(bem_mesh *mesh, const bem_assembly_opts *opts, bem_operator **out);
bem_status assembly_prepare(bem_ctx *ctx);  // constant tables on the device (once)
bem_status far_tune(bem_operator *op);       // time the far-field tile variants for op's size class
bem_status assemble_update(bem_operator *op, const bem_operator *coarse, bool upper_only = false);
bem_status ensure_full(bem_operator *op);
bem_status operator_diag(bem_operator *op);

// ----------------------------------------------------------------- batched assembly (assemble.cu)
// One problem of a batch wave as the batched assembly kernels see it.
struct BatchAsmProb {
    const double *q64;
    const float *q32;
    const double *cent;
    const float *qdf;
    const double *verts;
    const int32_t *tris;
    const double *area;
    const int32_t *edge_pairs, *vert_pairs;
    int64_t n_edge, n_vert;
    void *V;
    int64_t ld, N;
};
// The batched assembly of one wave: device arrays owned by the batch.
struct BatchAsm {
    int P = 0, precision = 0, variant = 0, ss_order = 4;
    const BatchAsmProb *prob = nullptr;    // P entries
    const int4 *far_items = nullptr;       // (problem, first row, first column, 0) per far-field tile
    int64_t n_far = 0;
    const int64_t *mirror_pref = nullptr;  // P + 1: prefix of the 32 x 32 tiles in the diagonal 64 x 64 blocks
    int64_t n_mirror = 0;
    const int64_t *near_pref = nullptr;    // P + 1: prefix of N + touching pairs
    int64_t n_near = 0;
    double far_entries = 0.0;              // entries i <= j (profiler units)
};
int far_variant_rows(int v);
int far_variant_cols(int v);
// Host: append the far-field tiles (i <= j part) of problem p of size N for tile variant v.
void batch_far_items(int v, int p, int64_t N, std::vector<int4> &items);
// Enqueue the far field, the mirror and the near field of every problem of b; ev
// (nullable, 4 events) is recorded before the far field, after it, before and after
// the near field.
bem_status batch_assemble(bem_ctx *ctx, const BatchAsm &b, cudaEvent_t *ev);
// Record e on the context's stream so that it also fires in replays of a graph being
// captured from that stream.
bem_status record_timing_event(bem_ctx *ctx, cudaEvent_t e);
// The autotuned far-field variant of (precision, N) in ctx, or -1 while not timed.
int far_cached_variant(const bem_ctx *ctx, int precision, int64_t N);

// ----------------------------------------------------------------- solve (solve.cu)
bem_status matvec_f64(bem_operator *op, const double *x, double *y);
// How the algorithmic bytes of a persistent solve are counted once its counts are read.
struct PersistentRun {
    int prof = -1;  // profiler record of the launch
    bool f32op = false, mixed = false, calpc = false, h16 = false;
    double n2 = 0.0;  // N^2
};
// A solve whose results are still travelling to pinned host memory: solve_capacity
// with a SolveDeferred enqueues the persistent solve, the Cap reduction and the
// copies of their results to h without synchronising (when the persistent solver
// runs; other paths finish at once and leave pending false); after any later
// synchronisation of the context's stream, solve_capacity_end reads them.
struct SolveDeferred {
    double *h = nullptr;  // pinned, 8 doubles: [0..4] solver out, [5] barrier error flag, [6] Cap,
                          // [7] iterations with FP16 products
    bool pending = false;
    PersistentRun run;
    double tol = 0.0;
};
bem_status solve_capacity(bem_operator *op, const bem_solve_opts *o, const double *d_x0,
                          double *d_x, double *cap, bem_solve_info *info, SolveDeferred *def = nullptr);
bem_status solve_capacity_end(bem_ctx *ctx, SolveDeferred &def, double *cap, bem_solve_info *info);

// ----------------------------------------------------------------- adaptivity (adapt.cu)
bem_status barycentric(bem_mesh *m, bem_mesh **out);
bem_status dual_operator(bem_operator *ob, bem_mesh *pm, bem_operator **out);
bem_status zz_estimate_dual(bem_mesh *m, const double *d_x, int h_mode, double *d_eta2, double *h_totals);
// d_totals (nullable, device, 2 doubles): where the totals are formed (the host copy
// h_totals, nullable, synchronises the stream).
bem_status zz_estimate(bem_mesh *m, const double *d_phi, int h_mode, double *d_eta2,
                       double *h_totals, double *d_totals = nullptr);
// Ascending sort of n2 (a power of two) 64-bit keys on the context's stream.
void sort_u64(bem_ctx *ctx, unsigned long long *keys, int64_t n2);
// n_marked (nullable) synchronises the stream; d_vanish (nullable, device: the ZZ
// totals) marks everything when the estimator vanishes up to rounding; d_count
// (nullable, device) receives the count without synchronising.
bem_status dorfler(bem_ctx *ctx, const double *d_eta2, int64_t N, double theta, uint8_t *d_marked,
                   int64_t *n_marked, const double *d_vanish = nullptr, long long *d_count = nullptr);
// defer_check: the refined mesh's checks are read by the next refine of it (or by
// mesh_check_pending) instead of a synchronisation of their own
bem_status refine(bem_mesh *m, const uint8_t *d_marked, int flags, bem_mesh **out, bool defer_check = false);
bem_status mesh_check_pending(bem_mesh *m);

}  // namespace bem
