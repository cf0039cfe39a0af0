// Continuous-batching request server for adaptive capacity computations.
//
// Requests (a surface mesh plus a level budget) arrive at any time.  A request is
// admitted as soon as a slot is free and its device-memory estimate fits in the
// server's HBM budget next to the requests already running (first fitting request
// in arrival order, so small requests backfill around a large one).  Each slot is a
// host thread with its own CUDA stream and library context, so the kernels of the
// admitted requests overlap on the device; each request keeps its mesh, operator
// and Krylov state on the device across its adaptive levels (bem_adaptive_run).
// Results and timestamps (steady clock, seconds since the server started) are
// kept until the caller collects them.
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bem_internal.cuh"

namespace {

struct Request {
    int64_t id = 0;
    std::vector<double> verts;
    std::vector<int32_t> tris;
    int32_t max_levels = 0;
    int64_t max_N = 0;
    int64_t estimate = 0;
    bem_request_result res{};
};

}  // namespace

struct bem_server {
    int device = 0;
    int64_t budget = 0;
    bem_adaptive_opts opts{};
    std::vector<std::thread> workers;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request *> queue;
    std::unordered_map<int64_t, Request *> all;
    int64_t next_id = 1;
    int64_t in_flight_bytes = 0, peak_bytes = 0;
    int in_flight = 0, peak_in_flight = 0;
    bool stop = false;
    int profile = 0;                 // slots profile their hot kernels (bem_profile_enable)
    std::vector<bem_ctx *> ctxs;     // the slots' contexts, for the profile read
    std::chrono::steady_clock::time_point t0;

    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// Device bytes a request may need: for one level, its operator plus the packed FP32
// upper triangle the solver reads (2 N^2 bytes: a quarter of a DF64 operator, half
// of an FP32 one);
// otherwise the operators of two consecutive levels (the coarse one is read by the
// incremental assembly of the fine one and freed before the solve) at the largest
// level the request can reach -- the first with N >= max_N, which Doerfler marking
// can overshoot by about 1.5x, or N0 grown by at most 2.2x per level (bisection of
// every element plus closure) -- plus per-triangle tables and solver vectors.  The
// dual basis holds, at its largest level, the operators of the barycentric refinements
// of two consecutive levels (6 n triangles: 36 times the bytes of a level operator,
// the coarse one read by the incremental assembly of the fine one) and V^dual with its
// preconditioner (about n / 2 vertices: DF64, packed copies, FP32 D^reg, 4 n^2 bytes).
int64_t estimate_bytes(int64_t N0, int64_t max_N, int32_t levels, int precision, int basis)
{
    const double es = precision == BEM_PREC_F32 ? 4.0 : 8.0;
    double reach = 1.5 * (double)(max_N > N0 ? max_N : N0);
    const double grown = (double)N0 * std::pow(2.2, (double)(levels - 1));
    if (grown < reach) reach = grown;
    const double n = (levels <= 1 ? (double)N0 : reach) + 64.0;
    if (basis == BEM_BASIS_DUAL) return (int64_t)((72.0 * es + 4.0) * n * n + 6.0 * 4096.0 * n) + (64ll << 20);
    const double ops = levels <= 1 ? (precision == BEM_PREC_DF64 ? 1.25 : precision == BEM_PREC_F32 ? 1.5 : 1.0) : 2.0;
    return (int64_t)(ops * es * n * n + 4096.0 * n) + (64ll << 20);
}

// A request on its slot's context (one per slot, kept across requests: its stream,
// pinned buffers, events and autotuned far-field tiles are reused), held to the
// request's admission estimate by the context's HBM budget.
void run_request(bem_server *srv, Request *r, bem_ctx *ctx)
{
    bem_mesh *mesh = nullptr;
    bem_request_result &res = r->res;
    bem_status st = ctx ? BEM_OK : BEM_ERR_CUDA;
    if (ctx) {
        ctx->budget = ctx->in_use + r->estimate;
        ctx->err[0] = 0;
    } else {
        snprintf(res.message, sizeof(res.message), "the slot has no library context");
    }
    if (!st)
        st = bem_mesh_upload(ctx, r->verts.data(), (int64_t)(r->verts.size() / 3), r->tris.data(),
                             (int64_t)(r->tris.size() / 3), nullptr, &mesh);
    if (!st) {
        bem_adaptive_opts o = srv->opts;
        o.max_levels = r->max_levels;
        o.max_N = r->max_N;
        std::vector<bem_level_record> rec((size_t)r->max_levels);
        int32_t n = 0;
        st = bem_adaptive_run(mesh, &o, rec.data(), &n, nullptr);
        res.levels = n;
        for (int k = 0; k < n && k < BEM_SERVER_HISTORY; ++k) {
            res.cap_history[k] = rec[k].cap;
            res.N_history[k] = rec[k].N;
        }
        if (n > 0) {
            res.cap = rec[n - 1].cap;
            res.N_final = rec[n - 1].N;
        }
    }
    if (st && ctx) snprintf(res.message, sizeof(res.message), "%s", bem_last_error(ctx));
    res.status = st;
    if (mesh) bem_mesh_destroy(mesh);
    if (ctx) cudaStreamSynchronize(ctx->stream);  // the request's frees are done before the next one
}

void worker_main(bem_server *srv)
{
    cudaSetDevice(srv->device);
    cudaStream_t stream = nullptr;
    if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        stream = nullptr;
    }
    bem_ctx *ctx = nullptr;
    if (bem_context_create(stream, 0, &ctx) != BEM_OK) ctx = nullptr;
    if (ctx) {
        std::lock_guard<std::mutex> lk(srv->mu);
        srv->ctxs.push_back(ctx);
    }
    int prof_on = 0;
    for (;;) {
        Request *r = nullptr;
        int want_prof = 0;
        {
            std::unique_lock<std::mutex> lk(srv->mu);
            for (;;) {
                if (srv->stop && srv->queue.empty()) break;
                // first queued request that fits next to the running ones (always one
                // when nothing runs, so an oversized request still makes progress)
                for (auto it = srv->queue.begin(); it != srv->queue.end(); ++it)
                    if (srv->in_flight == 0 || srv->in_flight_bytes + (*it)->estimate <= srv->budget) {
                        r = *it;
                        srv->queue.erase(it);
                        break;
                    }
                if (r) break;
                srv->cv_work.wait(lk);
            }
            if (!r) break;
            srv->in_flight_bytes += r->estimate;
            srv->in_flight += 1;
            if (srv->in_flight_bytes > srv->peak_bytes) srv->peak_bytes = srv->in_flight_bytes;
            if (srv->in_flight > srv->peak_in_flight) srv->peak_in_flight = srv->in_flight;
            r->res.t_start = srv->now();
            want_prof = srv->profile;
        }
        if (ctx && want_prof != prof_on) {  // this slot's context, on its own thread
            bem_profile_enable(ctx, want_prof);
            prof_on = want_prof;
        }
        run_request(srv, r, ctx);
        {
            std::lock_guard<std::mutex> lk(srv->mu);
            r->res.t_done = srv->now();
            r->res.done = 1;
            srv->in_flight_bytes -= r->estimate;
            srv->in_flight -= 1;
            r->verts.clear();
            r->verts.shrink_to_fit();
            r->tris.clear();
            r->tris.shrink_to_fit();
        }
        srv->cv_work.notify_all();
        srv->cv_done.notify_all();
    }
    if (ctx) bem_context_destroy(ctx);
    if (stream) cudaStreamDestroy(stream);
}

}  // namespace

extern "C" {

bem_status bem_server_create(int32_t slots, int64_t hbm_budget_bytes, const bem_adaptive_opts *opts, bem_server **out)
{
    if (!out || !opts || slots < 1 || slots > 256 || hbm_budget_bytes <= 0) return BEM_ERR_INVALID;
    if (!(opts->theta > 0.0 && opts->theta <= 1.0)) return BEM_ERR_INVALID;
    if (opts->basis != BEM_BASIS_P0 && opts->basis != BEM_BASIS_DUAL) return BEM_ERR_INVALID;
    bem_server *s = new (std::nothrow) bem_server();
    if (!s) return BEM_ERR_OOM;
    if (cudaGetDevice(&s->device) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return BEM_ERR_CUDA;
    }
    s->budget = hbm_budget_bytes;
    s->opts = *opts;
    s->t0 = std::chrono::steady_clock::now();
    for (int k = 0; k < slots; ++k) s->workers.emplace_back(worker_main, s);
    *out = s;
    return BEM_OK;
}

bem_status bem_server_submit(bem_server *s, const double *verts, int64_t M, const int32_t *tris, int64_t N,
                             int32_t max_levels, int64_t max_N, int64_t *id_out)
{
    if (!s || !verts || !tris || M < 3 || N < 1 || max_levels < 1 || !id_out) return BEM_ERR_INVALID;
    Request *r = new (std::nothrow) Request();
    if (!r) return BEM_ERR_OOM;
    r->verts.assign(verts, verts + 3 * M);
    r->tris.assign(tris, tris + 3 * N);
    r->max_levels = max_levels;
    r->max_N = max_N > 0 ? max_N : N;
    r->estimate = estimate_bytes(N, r->max_N, max_levels, s->opts.assembly.precision, s->opts.basis);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) {
            delete r;
            return BEM_ERR_INVALID;
        }
        r->id = s->next_id++;
        r->res.id = r->id;
        r->res.t_submit = s->now();
        r->res.estimate_bytes = r->estimate;
        s->all[r->id] = r;
        s->queue.push_back(r);
        *id_out = r->id;
    }
    s->cv_work.notify_all();
    return BEM_OK;
}

bem_status bem_server_wait(bem_server *s, int64_t id, bem_request_result *out)
{
    if (!s || !out) return BEM_ERR_INVALID;
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->all.find(id);
    if (it == s->all.end()) return BEM_ERR_INVALID;
    Request *r = it->second;
    s->cv_done.wait(lk, [&] { return r->res.done != 0; });
    *out = r->res;
    s->all.erase(it);
    delete r;
    return BEM_OK;
}

bem_status bem_server_stats(bem_server *s, bem_server_stats_t *out)
{
    if (!s || !out) return BEM_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    out->queued = (int64_t)s->queue.size();
    out->in_flight = s->in_flight;
    out->peak_in_flight = s->peak_in_flight;
    out->in_flight_bytes = s->in_flight_bytes;
    out->peak_bytes = s->peak_bytes;
    out->budget = s->budget;
    out->clock = s->now();
    return BEM_OK;
}

bem_status bem_server_profile_enable(bem_server *s, int32_t on)
{
    if (!s) return BEM_ERR_INVALID;
    std::lock_guard<std::mutex> lk(s->mu);
    s->profile = on ? 1 : 0;
    return BEM_OK;
}

bem_status bem_server_profile_read(bem_server *s, int32_t kernel, int64_t *launches, double *ms, double *units)
{
    if (!s || kernel < 0 || kernel >= bem::kProfKinds) return BEM_ERR_INVALID;
    // the lock is held throughout, so that no slot starts a request on its context
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->in_flight != 0 || !s->queue.empty()) return BEM_ERR_INVALID;
    int64_t n = 0;
    double t = 0.0, u = 0.0;
    for (bem_ctx *c : s->ctxs) {
        int64_t cn = 0;
        double cms = 0.0, cu = 0.0;
        const bem_status st = bem_profile_read(c, kernel, &cn, &cms, &cu);
        if (st) return st;
        n += cn;
        t += cms;
        u += cu;
    }
    if (launches) *launches = n;
    if (ms) *ms = t;
    if (units) *units = u;
    return BEM_OK;
}

bem_status bem_server_destroy(bem_server *s)
{
    if (!s) return BEM_ERR_INVALID;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    for (auto &t : s->workers) t.join();
    for (auto &kv : s->all) delete kv.second;
    delete s;
    return BEM_OK;
}

}  // extern "C"
