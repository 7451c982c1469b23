// Serving: continuous batching of BSGD reconstructions on one GPU.
//
// Two host threads drive the GPU:
//   admission  (two threads, one stream each) takes queued requests in arrival
//              order while slots and the byte budget allow, builds each one's
//              geometry and solver state (power-iteration step, unless a
//              request with the same geometry and step rule ran before: its
//              step is reused), draws its first iteration's blocks and hands
//              the ready request to the round thread;
//   rounds     keeps a device table of the resident requests and replays one
//              captured CUDA graph per round: persistent kernels (FP,
//              residual and BP of each ray; one per class of request present:
//              one or several column blocks per iteration x storage type) that
//              share all requests' detector tiles through atomic work
//              counters, then every request's block update with the draw of
//              its next iteration beside it, then the promotion of those
//              draws. After the last iteration of a request the round thread
//              copies its image out, and once that copy has finished it frees
//              the request and releases its budget.
// A graph is kept per set of classes present: the kernels read the table and
// the number of entries from memory, which the round thread rewrites between
// rounds when requests join or leave.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>

#include "bsgd_internal.h"

using namespace bsgd;

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum ReqStatus { kQueued, kAdmitting, kReady, kResident, kFinishing, kDone, kFailed };

constexpr int kAdmitThreads = 2;   // requests set up concurrently

struct Request {
    int64_t id = 0;
    bsgd_geometry_desc desc{};
    std::vector<double> angles;
    std::vector<int32_t> view_block;
    int M = 1, N = 1;
    bsgd_solve_params p{};
    std::vector<char> y;          // host copy of the data
    bsgd_dtype yt = BSGD_F32;
    float *x_out = nullptr;       // caller's result buffer
    size_t bytes = 0;             // budget charged while admitted
    int64_t target = 0, done = 0; // iterations
    int period = 1;               // rounds per iteration while resident (age priority)
    ReqStatus status = kQueued;
    std::string error;
    std::string geo_key;          // geometry cache entry this request holds
    bsgd_geometry *g = nullptr;
    bsgd_state *st = nullptr;
    void *x = nullptr;            // device image (storage type), from the pool
    float *xf = nullptr;          // device float copy for the result, from the pool
    float *stage = nullptr;       // pinned host staging of the result (+ update count)
    size_t stage_bytes = 0;
    unsigned long long *upd_host = nullptr;  // inside stage
    // inside stage too: the step, the residual-norm table and the sampling
    // trace, copied out with the image
    size_t off_mu = 0, off_S = 0, off_trace = 0;
    int64_t n_S = 0, trace_rows = 0, stride = 0;
    std::vector<int32_t> trace;   // the draws, kept after the request retires
    cudaEvent_t ev = nullptr;
    double t_submit = 0, t_done = 0;
    bsgd_report rep{};
};

}  // namespace

struct bsgd_server {
    bsgd_server_params prm{};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> queue;
    std::vector<Request *> ready, resident, finishing;
    std::map<int64_t, Request *> all;
    int64_t next_id = 1;
    int admitting = 0;
    size_t bytes = 0, peak_bytes = 0;
    bool stopping = false;
    std::vector<std::thread> admit_thr;
    std::thread round_thr;
    std::map<std::string, double> mu_cache;  // step size per geometry and step rule
    // geometries shared by requests of the same set-up (their update counts are
    // computed once): entry -> (geometry, requests holding it, last use)
    struct GeoEntry {
        bsgd_geometry *g = nullptr;
        int refs = 0;
        int64_t last = 0;
    };
    std::map<std::string, GeoEntry> geo_cache;
    int64_t geo_clock = 0;
    std::multimap<size_t, float *> pinned_free;   // reusable pinned staging buffers
    cudaStream_t round_stream = nullptr;
    std::vector<cudaStream_t> admit_streams;
    ReqDesc *d_table = nullptr;
    RoundCtl *d_ctl = nullptr;
    ReqDesc *h_table = nullptr;   // pinned
    RoundCtl *h_ctl = nullptr;    // pinned
    std::map<int, cudaGraphExec_t> graphs;   // round graph per set of classes present
    int class_mask = 0;                      // classes of the current table
    unsigned long long host_round = 0;       // rounds launched (the device's round index)
    int grid[kRoundClasses] = {};   // persistent grid of each class's kernel
    bool const_table = false;       // this server holds the device's constant request table
    // stats
    int64_t submitted = 0, admitted = 0, completed = 0, failed = 0, rounds = 0;
    int peak_resident = 0;
    std::vector<double> latencies_ms;
    int64_t updates = 0;
    double busy_s = 0, busy_since = -1;
    std::string thread_error;
};

namespace {

constexpr size_t kGeoKeep = 16;   // unreferenced geometries kept for reuse

// The constant-memory request table holds one server's table per device: the
// first server created on a device takes it, later ones (while it lives) read
// their table from global memory.
std::mutex g_const_mu;
std::map<int, bool> g_const_taken;

bool claim_const_table(int device) {
    std::lock_guard<std::mutex> lk(g_const_mu);
    if (g_const_taken[device]) return false;
    g_const_taken[device] = true;
    return true;
}

void release_const_table(int device) {
    std::lock_guard<std::mutex> lk(g_const_mu);
    g_const_taken[device] = false;
}

// Key of a geometry: everything its tables depend on.
std::string geometry_key(const Request *r) {
    const bsgd_geometry_desc &d = r->desc;
    std::string k;
    auto put = [&](const void *p, size_t n) { k.append((const char *)p, n); };
    put(&d.kind, sizeof d.kind);
    put(&d.nx, 3 * sizeof(int));
    put(&d.dx, 3 * sizeof(double));
    put(&d.n_views, sizeof(int));
    put(&d.nu, 2 * sizeof(int));
    put(&d.du, 4 * sizeof(double));
    if (d.angles) put(d.angles, sizeof(double) * d.n_views);
    if (d.view_block) put(d.view_block, sizeof(int32_t) * d.n_views);
    put(&r->M, sizeof(int));
    put(&r->N, sizeof(int));
    return k;
}

// The geometry of r's set-up, shared through the server's cache.
bsgd_status acquire_geometry(bsgd_server *S, Request *r) {
    r->geo_key = geometry_key(r);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->geo_cache.find(r->geo_key);
        if (it != S->geo_cache.end()) {
            it->second.refs++;
            it->second.last = ++S->geo_clock;
            r->g = it->second.g;
            return BSGD_OK;
        }
    }
    bsgd_geometry *g = nullptr;
    BSGD_TRY(bsgd_geometry_create(&r->desc, r->M, r->N, &g));
    std::lock_guard<std::mutex> lk(S->mu);
    auto &e = S->geo_cache[r->geo_key];
    if (e.g) {                       // another admission thread built it meanwhile
        bsgd_geometry_destroy(g);
    } else {
        e.g = g;
    }
    e.refs++;
    e.last = ++S->geo_clock;
    r->g = e.g;
    return BSGD_OK;
}

// Drop r's hold on its geometry; beyond kGeoKeep unreferenced entries the
// least recently used one is destroyed. Called without S->mu held.
void release_geometry(bsgd_server *S, Request *r) {
    if (!r->g) return;
    bsgd_geometry *drop = nullptr;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->geo_cache.find(r->geo_key);
        if (it != S->geo_cache.end()) it->second.refs--;
        size_t idle = 0;
        auto oldest = S->geo_cache.end();
        for (auto jt = S->geo_cache.begin(); jt != S->geo_cache.end(); ++jt) {
            if (jt->second.refs > 0) continue;
            ++idle;
            if (oldest == S->geo_cache.end() || jt->second.last < oldest->second.last) oldest = jt;
        }
        if (idle > kGeoKeep) {
            drop = oldest->second.g;
            S->geo_cache.erase(oldest);
        }
    }
    if (drop) bsgd_geometry_destroy(drop);
    r->g = nullptr;
}

float *take_pinned(bsgd_server *S, size_t bytes) {
    {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->pinned_free.lower_bound(bytes);
        if (it != S->pinned_free.end() && it->first <= 2 * bytes) {
            float *p = it->second;
            S->pinned_free.erase(it);
            return p;
        }
    }
    float *p = nullptr;
    if (cudaHostAlloc((void **)&p, bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

// Release what a request holds. Its device work is ordered on `st` (the round
// stream once it has been resident), so the pool memory is freed in stream
// order there; nothing here synchronises the device.
void free_request_gpu(bsgd_server *S, Request *r, cudaStream_t st) {
    if (r->st) state_release(r->st, st);
    pool_free(r->x, st);
    pool_free(r->xf, st);
    release_geometry(S, r);
    if (r->stage) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->pinned_free.emplace(r->stage_bytes, r->stage);
    }
    if (r->ev) cudaEventDestroy(r->ev);
    r->st = nullptr;
    r->x = r->xf = nullptr;
    r->stage = nullptr;
    r->upd_host = nullptr;
    r->ev = nullptr;
}

// Key of the step size: everything the power iteration's result depends on.
std::string mu_key(const Request *r) {
    const bsgd_geometry_desc &d = r->desc;
    std::string k;
    auto put = [&](const void *p, size_t n) { k.append((const char *)p, n); };
    put(&d.kind, sizeof d.kind);
    put(&d.nx, 3 * sizeof(int));
    put(&d.dx, 3 * sizeof(double));
    put(&d.n_views, sizeof(int));
    put(&d.nu, 2 * sizeof(int));
    put(&d.du, 4 * sizeof(double));
    if (d.angles) put(d.angles, sizeof(double) * d.n_views);
    if (d.view_block) put(d.view_block, sizeof(int32_t) * d.n_views);
    put(&r->M, sizeof(int));
    put(&r->N, sizeof(int));
    put(&r->p.step_rule, sizeof(int));
    put(&r->p.rho, sizeof(double));
    put(&r->p.power_iters, sizeof(int));
    return k;
}

// Build geometry, state and buffers of one request on an admission stream. A
// request whose geometry and step rule were seen before reuses that step size
// instead of running the power iteration again.
bsgd_status admit_one(bsgd_server *S, Request *r, cudaStream_t stream) {
    const std::string key = r->p.step_rule == BSGD_STEP_FIXED ? std::string() : mu_key(r);
    bsgd_solve_params prm = r->p;
    if (!key.empty()) {
        std::lock_guard<std::mutex> lk(S->mu);
        auto it = S->mu_cache.find(key);
        if (it != S->mu_cache.end()) {
            prm.step_rule = BSGD_STEP_FIXED;
            prm.mu = it->second;
        }
    }
    BSGD_TRY(acquire_geometry(S, r));
    const int64_t R = r->g->n_rows(), C = r->g->n_cols();
    const size_t ys = dtype_size(r->yt), es = dtype_size((bsgd_dtype)r->p.storage);
    void *dy = nullptr;
    BSGD_TRY(pool_alloc(&dy, R * ys, stream));
    cudaError_t e = cudaMemcpyAsync(dy, r->y.data(), R * ys, cudaMemcpyHostToDevice, stream);
    bsgd_status st = e == cudaSuccess ? BSGD_OK : cuda_fail(e, "copy of y");
    if (!st) st = bsgd_state_create(r->g, &prm, dy, r->yt, stream, &r->st);
    cudaStreamSynchronize(stream);
    pool_free(dy, stream);
    BSGD_TRY(st);
    if (!key.empty()) {
        bsgd_report rep{};
        if (bsgd_state_query(r->st, &rep, stream) == BSGD_OK) {
            std::lock_guard<std::mutex> lk(S->mu);
            S->mu_cache.emplace(key, rep.mu);
        }
    }
    r->y.clear();
    r->y.shrink_to_fit();
    BSGD_TRY(pool_alloc(&r->x, C * es, stream));
    BSGD_TRY(pool_alloc((void **)&r->xf, C * 4, stream));
    BSGD_CUDA(cudaMemsetAsync(r->x, 0, C * es, stream));
    {
        ReqDesc d;
        BSGD_TRY(state_descriptor(r->st, r->x, &d));
        r->n_S = (int64_t)r->g->M * r->g->desc.nv;
        r->stride = d.A.stride;
        r->trace_rows = std::min<int64_t>(r->target, d.A.trace_cap);
    }
    r->off_mu = (size_t)C * 4 + 64;
    r->off_S = r->off_mu + 8;
    r->off_trace = r->off_S + 8 * (size_t)r->n_S;
    r->stage_bytes = r->off_trace + 4 * (size_t)r->trace_rows * r->stride;
    r->stage = take_pinned(S, r->stage_bytes);
    if (!r->stage) return fail(BSGD_ERR_OOM, "pinned staging buffer");
    r->upd_host = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(r->stage) + (size_t)C * 4 + 32);
    BSGD_CUDA(cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming));
    ReqDesc tmp;
    BSGD_TRY(state_descriptor(r->st, r->x, &tmp));   // rejects what rounds cannot run
    BSGD_TRY(state_first_draw(r->st, stream));        // iteration 0's blocks, before the first round
    BSGD_CUDA(cudaStreamSynchronize(stream));
    return BSGD_OK;
}

void admission_loop(bsgd_server *S, cudaStream_t stream) {
    cudaSetDevice(S->prm.device);
    for (;;) {
        Request *r = nullptr;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait(lk, [&] {
                if (S->stopping) return true;
                if (S->queue.empty()) return false;
                const int live = (int)(S->resident.size() + S->ready.size()) + S->admitting;
                return live < S->prm.max_slots && S->bytes + S->queue.front()->bytes <= S->prm.budget_bytes;
            });
            if (S->stopping) return;
            r = S->queue.front();
            S->queue.pop_front();
            r->status = kAdmitting;
            S->admitting++;
            S->bytes += r->bytes;
            S->peak_bytes = std::max(S->peak_bytes, S->bytes);
        }
        bsgd_status st = admit_one(S, r, stream);
        std::string err = st ? bsgd_last_error() : "";
        {
            std::lock_guard<std::mutex> lk(S->mu);
            S->admitting--;
            if (st) {
                r->status = kFailed;
                r->error = err;
                r->t_done = now_s();
                S->failed++;
                S->bytes -= r->bytes;
            } else {
                r->status = kReady;
                S->ready.push_back(r);
                S->admitted++;
            }
        }
        if (st) free_request_gpu(S, r, stream);
        S->cv.notify_all();
    }
}

// The round graph for a set of request classes (bit c = class c present):
// the persistent kernel of each present class, then the block updates with
// the next iteration's draws, and the promotion of those draws.
bsgd_status round_graph(bsgd_server *S, int mask, cudaGraphExec_t *out) {
    auto it = S->graphs.find(mask);
    if (it != S->graphs.end()) {
        *out = it->second;
        return BSGD_OK;
    }
    cudaGraph_t graph = nullptr;
    BSGD_CUDA(cudaStreamBeginCapture(S->round_stream, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(&S->d_ctl->next[0], 0, kRoundClasses * sizeof(unsigned long long), S->round_stream);
    bsgd_status st = BSGD_OK;
    for (int c = 0; c < kRoundClasses && !st; ++c)
        if (mask & (1 << c))
            st = launch_round_solve(S->d_table, S->d_ctl, c, S->const_table, S->grid[c], S->round_stream);
    if (!st) st = launch_round_update(S->d_table, S->d_ctl, S->prm.max_slots, S->round_stream);
    cudaError_t e = cudaStreamEndCapture(S->round_stream, &graph);
    BSGD_TRY(st);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    S->graphs[mask] = exec;
    *out = exec;
    return BSGD_OK;
}

// Rewrite the device table from the resident list (called with no round in
// flight: the round stream is synchronised first).
bsgd_status upload_table(bsgd_server *S) {
    BSGD_CUDA(cudaStreamSynchronize(S->round_stream));
    // age priority: the request submitted first advances every round, the
    // others in every other round (shared: everyone every round)
    Request *oldest = nullptr;
    for (Request *r : S->resident)
        if (!oldest || r->t_submit < oldest->t_submit) oldest = r;
    for (Request *r : S->resident)
        r->period = S->prm.priority == BSGD_SERVE_AGE && S->resident.size() > 1 && r != oldest ? 2 : 1;
    // sorted by class (round_class: one or several column blocks per
    // iteration x storage type); work items are numbered within each class
    int n = 0, mask = 0;
    for (int cls = 0; cls < kRoundClasses; ++cls) {
        int64_t begin = 0;
        S->h_ctl->lo[cls] = n;
        for (Request *r : S->resident) {
            ReqDesc d;
            BSGD_TRY(state_descriptor(r->st, r->x, &d));
            if (round_class(d.kN, d.dtype) != cls) continue;
            d.target = r->target;
            d.period = r->period;
            d.work_begin = begin;
            begin += d.work_count;
            S->h_table[n++] = d;
        }
        S->h_ctl->hi[cls] = n;
        S->h_ctl->total_items[cls] = begin;
        S->h_ctl->next[cls] = 0;
        if (S->h_ctl->hi[cls] > S->h_ctl->lo[cls]) mask |= 1 << cls;
    }
    S->h_ctl->n = n;
    S->h_ctl->round = S->host_round;
    S->class_mask = mask;
    if (n) BSGD_CUDA(cudaMemcpyAsync(S->d_table, S->h_table, sizeof(ReqDesc) * n,
                                     cudaMemcpyHostToDevice, S->round_stream));
    if (S->const_table) BSGD_TRY(upload_round_const_table(S->h_table, n, S->round_stream));
    BSGD_CUDA(cudaMemcpyAsync(S->d_ctl, S->h_ctl, sizeof(RoundCtl), cudaMemcpyHostToDevice,
                              S->round_stream));
    BSGD_CUDA(cudaStreamSynchronize(S->round_stream));
    return BSGD_OK;
}

// After a request's last iteration: its image to the host, asynchronously.
bsgd_status start_finish(bsgd_server *S, Request *r) {
    const int64_t C = r->g->n_cols();
    BSGD_TRY(convert(r->x, (bsgd_dtype)r->p.storage, r->xf, BSGD_F32, C, S->round_stream));
    BSGD_CUDA(cudaMemcpyAsync(r->stage, r->xf, C * 4, cudaMemcpyDeviceToHost, S->round_stream));
    ReqDesc d;
    BSGD_TRY(state_descriptor(r->st, r->x, &d));
    BSGD_CUDA(cudaMemcpyAsync(r->upd_host, d.A.updates, 8, cudaMemcpyDeviceToHost, S->round_stream));
    char *base = reinterpret_cast<char *>(r->stage);
    BSGD_CUDA(cudaMemcpyAsync(base + r->off_mu, d.S.mu, 8, cudaMemcpyDeviceToHost, S->round_stream));
    BSGD_CUDA(cudaMemcpyAsync(base + r->off_S, d.S.S, 8 * (size_t)r->n_S, cudaMemcpyDeviceToHost,
                              S->round_stream));
    if (r->trace_rows > 0)
        BSGD_CUDA(cudaMemcpyAsync(base + r->off_trace, d.A.trace, 4 * (size_t)r->trace_rows * r->stride,
                                  cudaMemcpyDeviceToHost, S->round_stream));
    BSGD_CUDA(cudaEventRecord(r->ev, S->round_stream));
    return BSGD_OK;
}

void round_loop(bsgd_server *S) {
    cudaSetDevice(S->prm.device);
    bool dirty = true;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->cv.wait_for(lk, std::chrono::milliseconds(S->resident.empty() && S->finishing.empty() ? 20 : 0), [&] {
                return S->stopping || !S->ready.empty() || !S->resident.empty() || !S->finishing.empty();
            });
            if (S->stopping && S->ready.empty() && S->resident.empty() && S->finishing.empty()) break;
            while (!S->ready.empty() && (int)S->resident.size() < S->prm.max_slots) {
                Request *r = S->ready.front();
                S->ready.erase(S->ready.begin());
                r->status = kResident;
                S->resident.push_back(r);
                dirty = true;
            }
            S->peak_resident = std::max(S->peak_resident, (int)S->resident.size());
            if (!S->resident.empty() && S->busy_since < 0) S->busy_since = now_s();
        }
        if (dirty) {
            bsgd_status st = upload_table(S);
            if (st) {
                std::lock_guard<std::mutex> lk(S->mu);
                S->thread_error = bsgd_last_error();
                for (Request *r : S->resident) {
                    r->status = kFailed;
                    r->error = S->thread_error;
                    r->t_done = now_s();
                    S->failed++;
                }
                S->resident.clear();
                S->cv.notify_all();
                continue;
            }
            dirty = false;
        }
        if (!S->resident.empty()) {
            cudaGraphExec_t graph = nullptr;
            if (round_graph(S, S->class_mask, &graph) == BSGD_OK) cudaGraphLaunch(graph, S->round_stream);
            S->rounds++;
            const unsigned long long t = S->host_round++;
            std::vector<Request *> leaving;
            for (Request *r : S->resident)
                if (!round_skips(r->period, t) && ++r->done >= r->target) leaving.push_back(r);
            for (Request *r : leaving) {
                bsgd_status st = start_finish(S, r);
                std::lock_guard<std::mutex> lk(S->mu);
                S->resident.erase(std::find(S->resident.begin(), S->resident.end(), r));
                if (st) {
                    r->status = kFailed;
                    r->error = bsgd_last_error();
                    r->t_done = now_s();
                    S->failed++;
                } else {
                    r->status = kFinishing;
                    S->finishing.push_back(r);
                }
                dirty = true;
            }
            // keep at most a few rounds in flight so completions are seen early
            if (S->rounds % 4 == 0) cudaStreamSynchronize(S->round_stream);
        } else {
            cudaStreamSynchronize(S->round_stream);
        }
        // retire finished requests whose result copy has completed
        std::vector<Request *> done;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            for (Request *r : S->finishing)
                if (cudaEventQuery(r->ev) == cudaSuccess) done.push_back(r);
            for (Request *r : done) S->finishing.erase(std::find(S->finishing.begin(), S->finishing.end(), r));
        }
        for (Request *r : done) {
            const int64_t C = r->g->n_cols();
            std::memcpy(r->x_out, r->stage, C * 4);
            const unsigned long long upd = *r->upd_host;
            const char *base = reinterpret_cast<const char *>(r->stage);
            double mu = 0.0, rr = 0.0;
            std::memcpy(&mu, base + r->off_mu, 8);
            for (int64_t k = 0; k < r->n_S; ++k) {
                double v;
                std::memcpy(&v, base + r->off_S + 8 * k, 8);
                rr += v;
            }
            r->trace.resize((size_t)r->trace_rows * r->stride);
            if (!r->trace.empty()) std::memcpy(r->trace.data(), base + r->off_trace, 4 * r->trace.size());
            free_request_gpu(S, r, S->round_stream);
            std::lock_guard<std::mutex> lk(S->mu);
            r->t_done = now_s();
            r->rep.iteration = r->target;
            r->rep.updates = (int64_t)upd;
            r->rep.mu = mu;
            r->rep.residual_norm = std::sqrt(std::max(rr, 0.0));
            r->rep.epoch = (double)r->p.epochs;
            r->status = kDone;
            S->completed++;
            S->updates += (int64_t)upd;
            S->latencies_ms.push_back(1e3 * (r->t_done - r->t_submit));
            S->bytes -= r->bytes;
        }
        {
            std::lock_guard<std::mutex> lk(S->mu);
            if (S->resident.empty() && S->ready.empty() && S->finishing.empty() && S->busy_since >= 0) {
                S->busy_s += now_s() - S->busy_since;
                S->busy_since = -1;
            }
        }
        if (!done.empty()) S->cv.notify_all();
    }
}

}  // namespace

extern "C" bsgd_status bsgd_request_bytes(const bsgd_geometry_desc *desc, int M, int N,
                                          const bsgd_solve_params *p, size_t *out) {
    if (!desc || !p || !out) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    BSGD_TRY(validate_desc(desc, M, N));
    if (!dtype_ok(p->storage)) return fail(BSGD_ERR_INVALID_ARG, "bad storage dtype");
    size_t transient = 0;
    size_t b = state_bytes(*desc, M, N, *p, &transient);
    const size_t C = (size_t)desc->nx * desc->ny * desc->nz;
    const size_t R = (size_t)desc->n_views * desc->nu * desc->nv;
    b += C * dtype_size((bsgd_dtype)p->storage) + C * 4;   // image and its float copy
    transient = std::max(transient, R * 4);                 // the device copy of y
    *out = b + transient + ((size_t)16 << 20);               // allocation granularity
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_server_create(const bsgd_server_params *p, bsgd_server **out) {
    if (!p || !out) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (p->max_slots < 1 || p->max_slots > 64) return fail(BSGD_ERR_INVALID_ARG, "max_slots in [1, 64]");
    if (p->budget_bytes == 0) return fail(BSGD_ERR_INVALID_ARG, "budget_bytes must be > 0");
    if (p->priority != BSGD_SERVE_SHARED && p->priority != BSGD_SERVE_AGE)
        return fail(BSGD_ERR_INVALID_ARG, "priority must be BSGD_SERVE_SHARED or BSGD_SERVE_AGE");
    BSGD_CUDA(cudaSetDevice(p->device));
    bsgd_server *S = new (std::nothrow) bsgd_server();
    if (!S) return fail(BSGD_ERR_OOM, "host allocation failed");
    S->prm = *p;
    auto init = [&]() -> bsgd_status {
        BSGD_CUDA(cudaStreamCreateWithFlags(&S->round_stream, cudaStreamNonBlocking));
        for (int k = 0; k < kAdmitThreads; ++k) {
            cudaStream_t a = nullptr;
            BSGD_CUDA(cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
            S->admit_streams.push_back(a);
        }
        BSGD_CUDA(cudaMalloc((void **)&S->d_table, sizeof(ReqDesc) * p->max_slots));
        BSGD_CUDA(cudaMalloc((void **)&S->d_ctl, sizeof(RoundCtl)));
        BSGD_CUDA(cudaHostAlloc((void **)&S->h_table, sizeof(ReqDesc) * p->max_slots, cudaHostAllocDefault));
        BSGD_CUDA(cudaHostAlloc((void **)&S->h_ctl, sizeof(RoundCtl), cudaHostAllocDefault));
        std::memset(S->h_ctl, 0, sizeof(RoundCtl));
        BSGD_CUDA(cudaMemset(S->d_ctl, 0, sizeof(RoundCtl)));
        S->const_table = claim_const_table(p->device);   // max_slots <= 64 = kRoundConstSlots
        for (int c = 0; c < kRoundClasses; ++c) S->grid[c] = round_persistent_grid(c, S->const_table);
        return BSGD_OK;
    };
    bsgd_status st = init();
    if (st) {
        if (S->const_table) release_const_table(p->device);
        for (auto &kv : S->graphs) cudaGraphExecDestroy(kv.second);
        cudaFree(S->d_table);
        cudaFree(S->d_ctl);
        if (S->h_table) cudaFreeHost(S->h_table);
        if (S->h_ctl) cudaFreeHost(S->h_ctl);
        if (S->round_stream) cudaStreamDestroy(S->round_stream);
        for (cudaStream_t a : S->admit_streams) cudaStreamDestroy(a);
        delete S;
        return st;
    }
    for (cudaStream_t a : S->admit_streams) S->admit_thr.emplace_back(admission_loop, S, a);
    S->round_thr = std::thread(round_loop, S);
    *out = S;
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_server_destroy(bsgd_server *S) {
    if (!S) return fail(BSGD_ERR_INVALID_ARG, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stopping = true;
        for (Request *r : S->queue) {
            r->status = kFailed;
            r->error = "server stopped";
        }
        S->queue.clear();
    }
    S->cv.notify_all();
    for (auto &t : S->admit_thr)
        if (t.joinable()) t.join();
    if (S->round_thr.joinable()) S->round_thr.join();
    cudaSetDevice(S->prm.device);
    cudaStreamSynchronize(S->round_stream);
    for (auto &kv : S->all) {
        free_request_gpu(S, kv.second, S->round_stream);
        delete kv.second;
    }
    cudaStreamSynchronize(S->round_stream);
    for (auto &kv : S->geo_cache) bsgd_geometry_destroy(kv.second.g);
    for (auto &kv : S->pinned_free) cudaFreeHost(kv.second);
    for (auto &kv : S->graphs) cudaGraphExecDestroy(kv.second);
    cudaFree(S->d_table);
    cudaFree(S->d_ctl);
    cudaFreeHost(S->h_table);
    cudaFreeHost(S->h_ctl);
    cudaStreamDestroy(S->round_stream);
    for (cudaStream_t a : S->admit_streams) cudaStreamDestroy(a);
    if (S->const_table) release_const_table(S->prm.device);
    delete S;
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_server_submit(bsgd_server *S, const bsgd_geometry_desc *desc, int M,
                                          int N, const bsgd_solve_params *p, const void *y,
                                          bsgd_dtype yt, float *x_out, int64_t *id) {
    if (!S || !desc || !p || !y || !x_out || !id) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    if (!dtype_ok(yt)) return fail(BSGD_ERR_INVALID_ARG, "bad y dtype");
    size_t bytes = 0;
    BSGD_TRY(bsgd_request_bytes(desc, M, N, p, &bytes));
    const int kN = std::max(1, (int)std::lround(p->gamma * N));
    if (kN > kMaxFusedCols) return fail(BSGD_ERR_INVALID_ARG, "serving needs gamma * N <= 4");
    if (kN > 1 && p->pair_sampling != BSGD_PAIRS_UNIFORM)
        return fail(BSGD_ERR_INVALID_ARG, "serving with several column blocks needs uniform pairs");
    if (p->tv_lambda > 0) return fail(BSGD_ERR_INVALID_ARG, "serving runs no TV prox");
    if (p->auto_mu) return fail(BSGD_ERR_INVALID_ARG, "serving runs no automatic step length");
    if (p->epochs < 1) return fail(BSGD_ERR_INVALID_ARG, "epochs must be >= 1");
    if (!(p->alpha > 0 && p->alpha <= 1)) return fail(BSGD_ERR_INVALID_ARG, "alpha in (0, 1]");
    if (bytes > S->prm.budget_bytes)
        return fail(BSGD_ERR_BUDGET, "request needs " + std::to_string(bytes) +
                                         " bytes, more than the server's budget");
    Request *r = new (std::nothrow) Request();
    if (!r) return fail(BSGD_ERR_OOM, "host allocation failed");
    r->desc = *desc;
    r->angles.assign(desc->angles ? desc->angles : nullptr, desc->angles ? desc->angles + desc->n_views : nullptr);
    if (desc->view_block) r->view_block.assign(desc->view_block, desc->view_block + desc->n_views);
    r->desc.angles = desc->angles ? r->angles.data() : nullptr;
    r->desc.view_block = desc->view_block ? r->view_block.data() : nullptr;
    r->M = M;
    r->N = N;
    r->p = *p;
    const size_t R = (size_t)desc->n_views * desc->nu * desc->nv;
    r->y.assign((const char *)y, (const char *)y + R * dtype_size(yt));
    r->yt = yt;
    r->x_out = x_out;
    r->bytes = bytes;
    const int kM = std::max(1, (int)std::lround(p->alpha * M));
    const int epoch_len = std::max(1, (int)std::lround(1.0 / (p->alpha * p->gamma)));
    (void)kM;
    r->target = (int64_t)p->epochs * epoch_len;
    r->t_submit = now_s();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stopping) {
            delete r;
            return fail(BSGD_ERR_STATE, "server is stopping");
        }
        r->id = S->next_id++;
        S->all[r->id] = r;
        S->queue.push_back(r);
        S->submitted++;
        *id = r->id;
    }
    S->cv.notify_all();
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_server_poll(bsgd_server *S, int64_t id, int *done) {
    if (!S || !done) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail(BSGD_ERR_INVALID_ARG, "unknown request id");
    *done = it->second->status == kDone || it->second->status == kFailed;
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_server_wait(bsgd_server *S, int64_t id, int timeout_ms, bsgd_report *out) {
    if (!S) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail(BSGD_ERR_INVALID_ARG, "unknown request id");
    Request *r = it->second;
    const bool fin = S->cv.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)), [&] {
        return r->status == kDone || r->status == kFailed;
    });
    if (!fin) return fail(BSGD_ERR_TIMEOUT, "request " + std::to_string(id) + " still running");
    if (r->status == kFailed) return fail(BSGD_ERR_CUDA, "request failed: " + r->error);
    if (out) *out = r->rep;
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_server_read_trace(bsgd_server *S, int64_t id, int32_t *host, int64_t cap,
                                              int64_t *stride, int64_t *n_iters) {
    if (!S || !stride || !n_iters) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->all.find(id);
    if (it == S->all.end()) return fail(BSGD_ERR_INVALID_ARG, "unknown request id");
    const Request *r = it->second;
    if (r->status != kDone) return fail(BSGD_ERR_STATE, "request has not finished");
    *stride = r->stride;
    *n_iters = r->stride > 0 ? (int64_t)r->trace.size() / r->stride : 0;
    if (!host) return BSGD_OK;
    if (cap < 0) return fail(BSGD_ERR_INVALID_ARG, "cap < 0");
    const int64_t n = std::min(*n_iters, r->stride > 0 ? cap / r->stride : 0);
    std::memcpy(host, r->trace.data(), 4 * (size_t)n * r->stride);
    *n_iters = n;
    return BSGD_OK;
}

extern "C" bsgd_status bsgd_server_get_stats(bsgd_server *S, bsgd_server_stats *out) {
    if (!S || !out) return fail(BSGD_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    bsgd_server_stats z{};
    z.submitted = S->submitted;
    z.admitted = S->admitted;
    z.completed = S->completed;
    z.failed = S->failed;
    z.queued = (int64_t)S->queue.size();
    z.resident = (int64_t)S->resident.size();
    z.peak_resident = S->peak_resident;
    z.bytes_resident = S->bytes;
    z.peak_bytes = S->peak_bytes;
    std::vector<double> l = S->latencies_ms;
    std::sort(l.begin(), l.end());
    if (!l.empty()) {
        auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)std::floor(f * (l.size() - 1) + 0.5))]; };
        z.p50_ms = q(0.50);
        z.p99_ms = q(0.99);
        double s = 0;
        for (double v : l) s += v;
        z.mean_ms = s / l.size();
        z.max_ms = l.back();
    }
    z.updates = S->updates;
    z.busy_s = S->busy_s + (S->busy_since >= 0 ? now_s() - S->busy_since : 0.0);
    z.rounds = S->rounds;
    *out = z;
    return BSGD_OK;
}
