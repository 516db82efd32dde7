// server.cpp -- serving loop: admission by device-memory budget, one stream
// per in-flight request, resident per-slot indices, completion by stream
// callback (Sec. 3.1: Run-3 timeframes arrive continuously and are tracked
// synchronously with data taking).
//
// A scheduler thread admits queued requests in arrival order whenever a slot
// is free and the request's device bytes fit the budget.  An admitted request
// is enqueued on its slot's stream: host-to-device copies, index rebuild,
// follower, device-to-host copy of the results, and a host callback that
// time-stamps completion.  Requests on different slots overlap on the device
// (copies of one with kernels of another), and a request that arrives while
// others run is admitted as soon as a slot and memory free up.  There are no
// device-side waits; every host wait is bounded.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "trd_internal.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_s() { return std::chrono::duration<double>(Clock::now().time_since_epoch()).count(); }

struct Request {
    uint64_t ticket = 0;
    trd_seeds_t seeds{};       // host pointers
    trd_tracklets_t trk{};     // host pointers
    trd_results_t out{};       // host pointers
    size_t bytes = 0;          // device bytes charged against the budget
    double t_submit = 0, t_admit = 0;
    std::atomic<double> t_done{0.0};
    std::atomic<int> state{0};  // 0 queued, 1 in flight, 2 done, 3 failed
    int slot = -1;
    int error = TRD_OK;
    // device buffers (stream-ordered allocations on the slot's stream)
    void *dbuf = nullptr;
    // stream-ordered marks: before the input copies, after them, after the
    // index build and follower, after the result copies
    cudaEvent_t ev0 = nullptr, ev_in = nullptr, ev_k = nullptr, ev1 = nullptr;
    float gpu_ms = 0;
    float stage_ms[4] = {0, 0, 0, 0};  // the four marks on the server's device clock
};

bool create_events(Request *r)
{
    if (cudaEventCreate(&r->ev0) == cudaSuccess && cudaEventCreate(&r->ev_in) == cudaSuccess &&
        cudaEventCreate(&r->ev_k) == cudaSuccess && cudaEventCreate(&r->ev1) == cudaSuccess)
        return true;
    (void)cudaGetLastError();
    return false;
}

void destroy_events(Request *r)
{
    cudaEvent_t *ev[4] = {&r->ev0, &r->ev_in, &r->ev_k, &r->ev1};
    for (cudaEvent_t *e : ev)
        if (*e) {
            cudaEventDestroy(*e);
            *e = nullptr;
        }
}

struct Slot {
    cudaStream_t stream = nullptr;
    trd_index *index = nullptr;  // resident, grows when a larger request arrives
    Request *busy = nullptr;
};

size_t align_up(size_t v) { return (v + 255) & ~static_cast<size_t>(255); }

// bytes of one request's device buffer: inputs (seeds 22 rows of n,
// tracklets 7 rows of m, interaction ids of seeds and tracklets, tracklet
// radii) and outputs (23 float rows and 9 int rows of n), each packed without
// gaps (4-byte elements) so that a caller's packed host block moves in one
// copy, then the follower's scratch
size_t io_bytes(int n_seeds, int n_trk)
{
    const size_t n = static_cast<size_t>(n_seeds), m = static_cast<size_t>(n_trk);
    return align_up(sizeof(float) * (22 * n + 7 * m + n + m + m)) + align_up(sizeof(float) * 32 * n) +
           align_up(trd_host::parked_bytes(n_seeds));
}

// bytes of an index for n_trk tracklets (records + build scratch + buckets)
size_t index_bytes(int n_trk, float w)
{
    const size_t nb = static_cast<size_t>(ceilf(2.0f * 66.0f / w));
    const size_t buckets = static_cast<size_t>(TRD_N_CHAMBERS) * 18 * nb;
    return 40 * static_cast<size_t>(n_trk) + 8 * buckets + 4096;  // records, radii, bucket
}

void CUDART_CB on_done(void *p)
{
    Request *r = static_cast<Request *>(p);
    r->t_done.store(now_s());
    r->state.store(2);
}

}  // namespace

struct trd_server {
    trd_ctx *ctx;
    trd_server_cfg_t cfg;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request *> queue;
    std::unordered_map<uint64_t, Request *> all;
    std::vector<Request *> inflight;
    uint64_t next_ticket = 1;
    size_t used = 0;       // bytes of admitted requests' I/O buffers
    size_t index_used = 0; // bytes of the slots' resident indices
    bool stop = false;
    cudaEvent_t ev_ref = nullptr;  // origin of the requests' device-clock marks
    std::thread worker;
    int fatal = TRD_OK;
};

namespace {

// One request's copies in one direction, merged where both the host and the
// device ranges continue the previous copy: a caller that keeps its arrays in
// one block in the library's order gets one copy per block instead of one per
// array (every copy costs the copy engine a fixed set-up time).
struct CopyList {
    struct Copy {
        char *dst;
        const char *src;
        size_t bytes;
    };
    Copy c[32];
    int k = 0;
    void add(void *dst, const void *src, size_t bytes)
    {
        if (!bytes) return;
        char *d = static_cast<char *>(dst);
        const char *s = static_cast<const char *>(src);
        if (k && c[k - 1].dst + c[k - 1].bytes == d && c[k - 1].src + c[k - 1].bytes == s) {
            c[k - 1].bytes += bytes;
            return;
        }
        c[k++] = {d, s, bytes};
    }
    int issue(cudaMemcpyKind kind, cudaStream_t st) const
    {
        for (int j = 0; j < k; ++j) TRD_CUDA_TRY(cudaMemcpyAsync(c[j].dst, c[j].src, c[j].bytes, kind, st));
        return TRD_OK;
    }
};

// enqueue one admitted request on its slot (scheduler thread, lock held)
int start_request(trd_server *S, Slot &slot, Request *r)
{
    cudaStream_t st = slot.stream;
    const int n = r->seeds.n, m = r->trk.n;
    const size_t need = io_bytes(n, m);
    TRD_CUDA_TRY(cudaMallocAsync(&r->dbuf, std::max<size_t>(need, 256), st));
    char *p = static_cast<char *>(r->dbuf);
    float *ds = reinterpret_cast<float *>(p);                  // seeds [22][n]
    char *dt = reinterpret_cast<char *>(ds + 22 * static_cast<size_t>(n));  // tracklets [7][m]
    int32_t *dtrig_s = reinterpret_cast<int32_t *>(dt) + 7 * static_cast<size_t>(m);
    int32_t *dtrig_t = dtrig_s + n;
    float *dx_t = reinterpret_cast<float *>(dtrig_t + m);
    p += align_up(sizeof(float) * (22 * static_cast<size_t>(n) + 9 * static_cast<size_t>(m) + n));
    float *dr = reinterpret_cast<float *>(p);                  // float results [23][n]
    int32_t *di = reinterpret_cast<int32_t *>(dr + 23 * static_cast<size_t>(n));  // int results [9][n]
    p += align_up(sizeof(float) * 32 * static_cast<size_t>(n));
    void *parked = n ? p : nullptr;                            // 256-byte aligned
    // inputs in device order: seeds alpha x y z snp tgl q2pt cov[15] (22 rows
    // of n), tracklets chamber y z dy vyy vzz vyz (7 rows of m), interaction
    // ids of seeds and tracklets, tracklet radii
    const float *hs[7] = {r->seeds.alpha, r->seeds.x, r->seeds.y, r->seeds.z, r->seeds.snp, r->seeds.tgl,
                          r->seeds.q2pt};
    int32_t *dch = reinterpret_cast<int32_t *>(dt);
    float *dtf = reinterpret_cast<float *>(dt) + m;
    const float *ht[6] = {r->trk.y, r->trk.z, r->trk.dy, r->trk.vyy, r->trk.vzz, r->trk.vyz};
    CopyList in;
    if (n) {
        for (int k = 0; k < 7; ++k) in.add(ds + static_cast<size_t>(k) * n, hs[k], sizeof(float) * n);
        in.add(ds + 7 * static_cast<size_t>(n), r->seeds.cov, sizeof(float) * 15 * n);
    }
    if (m) {
        in.add(dch, r->trk.chamber, sizeof(int32_t) * m);
        for (int k = 0; k < 6; ++k) in.add(dtf + static_cast<size_t>(k) * m, ht[k], sizeof(float) * m);
    }
    if (n && r->seeds.trigger) in.add(dtrig_s, r->seeds.trigger, sizeof(int32_t) * n);
    if (m && r->trk.trigger) in.add(dtrig_t, r->trk.trigger, sizeof(int32_t) * m);
    if (m && r->trk.x) in.add(dx_t, r->trk.x, sizeof(float) * m);
    TRD_CUDA_TRY(cudaEventRecord(r->ev0, st));
    int rc = in.issue(cudaMemcpyHostToDevice, st);
    if (rc) return rc;
    TRD_CUDA_TRY(cudaEventRecord(r->ev_in, st));
    trd_seeds_t dseeds{ds, ds + n, ds + 2 * static_cast<size_t>(n), ds + 3 * static_cast<size_t>(n),
                       ds + 4 * static_cast<size_t>(n), ds + 5 * static_cast<size_t>(n),
                       ds + 6 * static_cast<size_t>(n), ds + 7 * static_cast<size_t>(n), n,
                       r->seeds.trigger ? dtrig_s : nullptr};
    trd_tracklets_t dtrk{dch, dtf, dtf + m, dtf + 2 * static_cast<size_t>(m), dtf + 3 * static_cast<size_t>(m),
                         dtf + 4 * static_cast<size_t>(m), dtf + 5 * static_cast<size_t>(m), m,
                         r->trk.trigger ? dtrig_t : nullptr, r->trk.x ? dx_t : nullptr};
    trd_results_t dres{dr, dr + n, dr + 2 * static_cast<size_t>(n), dr + 7 * static_cast<size_t>(n),
                       dr + 22 * static_cast<size_t>(n), di, di + n, di + 2 * static_cast<size_t>(n),
                       di + 3 * static_cast<size_t>(n)};
    rc = trd_index_rebuild(slot.index, &dtrk, st);
    if (rc) return rc;
    rc = trd_host::follow_checked(S->ctx, &dseeds, slot.index, &S->cfg.params, nullptr, &dres, st, &S->cfg.launch,
                                  parked);
    if (rc) return rc;
    TRD_CUDA_TRY(cudaEventRecord(r->ev_k, st));
    // results back: alpha x par[5] cov[15] chi2 (23 float rows), then 9 int rows
    float *hf[5] = {r->out.alpha, r->out.x, r->out.par, r->out.cov, r->out.chi2};
    const int rows_f[5] = {1, 1, 5, 15, 1};
    int32_t *hi[4] = {r->out.n_trk, r->out.n_miss, r->out.status, r->out.tracklet_id};
    const int rows_i[4] = {1, 1, 1, 6};
    CopyList out;
    if (n) {
        size_t off = 0;
        for (int k = 0; k < 5; ++k) {
            out.add(hf[k], dr + off, sizeof(float) * rows_f[k] * n);
            off += static_cast<size_t>(rows_f[k]) * n;
        }
        off = 0;
        for (int k = 0; k < 4; ++k) {
            out.add(hi[k], di + off, sizeof(int32_t) * rows_i[k] * n);
            off += static_cast<size_t>(rows_i[k]) * n;
        }
    }
    rc = out.issue(cudaMemcpyDeviceToHost, st);
    if (rc) return rc;
    TRD_CUDA_TRY(cudaEventRecord(r->ev1, st));
    TRD_CUDA_TRY(cudaFreeAsync(r->dbuf, st));
    r->dbuf = nullptr;
    TRD_CUDA_TRY(cudaLaunchHostFunc(st, on_done, r));
    return TRD_OK;
}

// make the slot's resident index large enough (scheduler thread, lock NOT
// held, slot reserved and idle); *added = index bytes added (may be negative)
int ensure_index(trd_server *S, Slot &slot, int n_trk, long long *added)
{
    *added = 0;
    if (slot.index && slot.index->capacity >= n_trk) return TRD_OK;
    const int cap = std::max(n_trk, slot.index ? 2 * slot.index->capacity : n_trk);
    if (slot.index) {
        *added -= static_cast<long long>(index_bytes(slot.index->capacity, S->cfg.y_bin_width));
        cudaStreamSynchronize(slot.stream);
        trd_host::index_release(slot.index);
        slot.index = nullptr;
    }
    int rc = trd_host::index_alloc(S->ctx, cap, S->cfg.y_bin_width, 1, &slot.index);
    if (rc) return rc;
    *added += static_cast<long long>(index_bytes(cap, S->cfg.y_bin_width));
    return TRD_OK;
}

void worker_loop(trd_server *S)
{
    cudaSetDevice(S->ctx->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // retire finished requests
        for (size_t k = 0; k < S->inflight.size();) {
            Request *r = S->inflight[k];
            if (r->state.load() == 2) {
                cudaEventElapsedTime(&r->gpu_ms, r->ev0, r->ev1);
                const cudaEvent_t marks[4] = {r->ev0, r->ev_in, r->ev_k, r->ev1};
                for (int k2 = 0; k2 < 4; ++k2) cudaEventElapsedTime(&r->stage_ms[k2], S->ev_ref, marks[k2]);
                S->used -= r->bytes;
                S->slots[r->slot].busy = nullptr;
                S->inflight[k] = S->inflight.back();
                S->inflight.pop_back();
                S->cv.notify_all();
            } else {
                ++k;
            }
        }
        // admit in arrival order while a slot and the budget allow
        while (!S->queue.empty()) {
            Request *r = S->queue.front();
            int free_slot = -1;
            for (size_t k = 0; k < S->slots.size(); ++k)
                if (!S->slots[k].busy) {
                    free_slot = static_cast<int>(k);
                    break;
                }
            if (free_slot < 0) break;
            Slot &slot = S->slots[free_slot];
            const size_t grow = (!slot.index || slot.index->capacity < r->trk.n)
                                    ? index_bytes(std::max(r->trk.n, slot.index ? 2 * slot.index->capacity : 0),
                                                  S->cfg.y_bin_width)
                                    : 0;
            if (S->used + S->index_used + r->bytes + grow > S->cfg.mem_budget_bytes && !S->inflight.empty()) break;
            // reserve the slot and the budget, then enqueue without the lock so
            // that submit and poll never wait for copies or allocations
            S->queue.pop_front();
            r->slot = free_slot;
            r->t_admit = now_s();
            r->state.store(1);
            slot.busy = r;
            S->used += r->bytes;
            S->index_used += grow;
            S->inflight.push_back(r);
            lk.unlock();
            long long added = 0;
            int rc = ensure_index(S, slot, r->trk.n, &added);
            if (!rc) rc = start_request(S, slot, r);
            if (rc) {
                cudaStreamSynchronize(slot.stream);
                if (r->dbuf) cudaFree(r->dbuf);
                r->dbuf = nullptr;
                (void)cudaGetLastError();
            }
            lk.lock();
            S->index_used += static_cast<size_t>(static_cast<long long>(added) - static_cast<long long>(grow));
            if (rc) {  // the request fails on its own; the server keeps going
                r->error = rc;
                r->t_done.store(now_s());
                S->used -= r->bytes;
                slot.busy = nullptr;
                for (size_t k = 0; k < S->inflight.size(); ++k)
                    if (S->inflight[k] == r) {
                        S->inflight[k] = S->inflight.back();
                        S->inflight.pop_back();
                        break;
                    }
                r->state.store(3);
                S->cv.notify_all();
            }
        }
        if (S->stop && S->queue.empty() && S->inflight.empty()) break;
        S->cv.wait_for(lk, std::chrono::microseconds(S->inflight.empty() ? 2000 : 20));
    }
}

}  // namespace

extern "C" {

int trd_server_create(trd_ctx_t *ctx, const trd_server_cfg_t *cfg, trd_server_t **out)
{
    if (!ctx || !cfg || !out) return TRD_EINVAL;
    *out = nullptr;
    if (cfg->max_slots < 0 || cfg->max_slots > 64 || cfg->max_queue < 0) return TRD_EINVAL;
    trd_server *S = new (std::nothrow) trd_server;
    if (!S) return TRD_ENOMEM;
    S->ctx = ctx;
    S->cfg = *cfg;
    if (S->cfg.mem_budget_bytes == 0) S->cfg.mem_budget_bytes = 60ull << 30;
    if (S->cfg.max_slots == 0) S->cfg.max_slots = 4;
    if (S->cfg.max_queue == 0) S->cfg.max_queue = 1024;
    if (S->cfg.y_bin_width == 0.0f) S->cfg.y_bin_width = 2.0f;
    // validate parameters and launch shape once (no work: zero seeds)
    trd_index *probe = nullptr;
    int rc = trd_host::index_alloc(ctx, 0, S->cfg.y_bin_width, 1, &probe);
    if (!rc) {
        trd_seeds_t none{};
        trd_results_t nores{};
        rc = trd_follow_tuned(ctx, &none, probe, &S->cfg.params, &nores, nullptr, &S->cfg.launch);
        trd_host::index_release(probe);
    }
    if (rc) {
        delete S;
        return rc;
    }
    cudaSetDevice(ctx->device);
    S->slots.resize(S->cfg.max_slots);
    for (auto &sl : S->slots)
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) {
            for (auto &z : S->slots)
                if (z.stream) cudaStreamDestroy(z.stream);
            delete S;
            return TRD_ECUDA;
        }
    // the origin of the requests' device-clock marks
    if (cudaEventCreate(&S->ev_ref) != cudaSuccess || cudaEventRecord(S->ev_ref, S->slots[0].stream) != cudaSuccess ||
        cudaEventSynchronize(S->ev_ref) != cudaSuccess) {
        if (S->ev_ref) cudaEventDestroy(S->ev_ref);
        for (auto &z : S->slots) cudaStreamDestroy(z.stream);
        (void)cudaGetLastError();
        delete S;
        return TRD_ECUDA;
    }
    // keep freed stream-ordered memory in the pool between requests
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
        uint64_t keep = S->cfg.mem_budget_bytes;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    (void)cudaGetLastError();
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return TRD_OK;
}

int trd_server_submit(trd_server_t *S, const trd_seeds_t *seeds, const trd_tracklets_t *trk,
                      trd_results_t *results, uint64_t *ticket)
{
    if (!S || !seeds || !trk || !results || !ticket || seeds->n < 0 || trk->n < 0) return TRD_EINVAL;
    if (seeds->n > 0 && (!seeds->alpha || !seeds->x || !seeds->y || !seeds->z || !seeds->snp || !seeds->tgl ||
                         !seeds->q2pt || !seeds->cov || !results->alpha || !results->x || !results->par ||
                         !results->cov || !results->chi2 || !results->n_trk || !results->n_miss ||
                         !results->status || !results->tracklet_id))
        return TRD_EINVAL;
    if (trk->n > 0 && (!trk->chamber || !trk->y || !trk->z || !trk->dy || !trk->vyy || !trk->vzz || !trk->vyz))
        return TRD_EINVAL;
    const size_t bytes = io_bytes(seeds->n, trk->n);
    if (bytes + index_bytes(trk->n, S->cfg.y_bin_width) > S->cfg.mem_budget_bytes) return TRD_ENOMEM;
    Request *r = new (std::nothrow) Request;
    if (!r) return TRD_ENOMEM;
    r->seeds = *seeds;
    r->trk = *trk;
    r->out = *results;
    r->bytes = bytes;
    if (!create_events(r)) {
        destroy_events(r);
        delete r;
        return TRD_ECUDA;
    }
    std::lock_guard<std::mutex> g(S->mu);
    if (S->stop) {
        destroy_events(r);
        delete r;
        return TRD_EINVAL;
    }
    if (static_cast<int>(S->queue.size()) >= S->cfg.max_queue) {
        destroy_events(r);
        delete r;
        return TRD_EAGAIN;
    }
    r->ticket = S->next_ticket++;
    r->t_submit = now_s();
    S->queue.push_back(r);
    S->all[r->ticket] = r;
    *ticket = r->ticket;
    S->cv.notify_all();
    return TRD_OK;
}

static int finish(trd_server *S, Request *r, trd_timing_t *t)
{
    // called with S->mu held, request done or failed
    if (t) {
        t->submit_s = r->t_submit;
        t->admit_s = r->t_admit;
        t->done_s = r->t_done.load();
        t->gpu_ms = r->gpu_ms;
        t->slot = r->slot;
        t->start_ms = r->stage_ms[0];
        t->inputs_ms = r->stage_ms[1];
        t->kernels_ms = r->stage_ms[2];
        t->results_ms = r->stage_ms[3];
    }
    const int rc = r->state.load() == 3 ? r->error : TRD_OK;
    destroy_events(r);
    S->all.erase(r->ticket);
    delete r;
    return rc;
}

int trd_server_poll(trd_server_t *S, uint64_t ticket, trd_timing_t *timing)
{
    if (!S) return TRD_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return TRD_EINVAL;
    Request *r = it->second;
    const int st = r->state.load();
    if (st == 3) return finish(S, r, timing);
    if (st != 2) return TRD_EAGAIN;
    // done on the device; the scheduler retires it (timing, budget) first
    for (Request *q : S->inflight)
        if (q == r) return TRD_EAGAIN;
    return finish(S, r, timing);
}

int trd_server_wait(trd_server_t *S, uint64_t ticket, int32_t timeout_ms, trd_timing_t *timing)
{
    if (!S || timeout_ms < 0) return TRD_EINVAL;
    const auto until = Clock::now() + std::chrono::milliseconds(timeout_ms);
    while (true) {
        const int rc = trd_server_poll(S, ticket, timing);
        if (rc != TRD_EAGAIN) return rc;
        if (Clock::now() >= until) return TRD_ETIMEOUT;
        std::unique_lock<std::mutex> lk(S->mu);
        S->cv.wait_for(lk, std::chrono::microseconds(200));
    }
}

int trd_server_stats(trd_server_t *S, int32_t *queued, int32_t *in_flight, uint64_t *device_bytes)
{
    if (!S) return TRD_EINVAL;
    std::lock_guard<std::mutex> g(S->mu);
    if (queued) *queued = static_cast<int32_t>(S->queue.size());
    if (in_flight) *in_flight = static_cast<int32_t>(S->inflight.size());
    if (device_bytes) *device_bytes = S->used + S->index_used;
    return TRD_OK;
}

int trd_server_destroy(trd_server_t *S)
{
    if (!S) return TRD_EINVAL;
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    S->worker.join();  // drains the queue and the work in flight
    cudaSetDevice(S->ctx->device);
    for (auto &sl : S->slots) {
        cudaStreamSynchronize(sl.stream);
        if (sl.index) trd_host::index_release(sl.index);
        cudaStreamDestroy(sl.stream);
    }
    for (auto &kv : S->all) {
        destroy_events(kv.second);
        delete kv.second;
    }
    if (S->ev_ref) cudaEventDestroy(S->ev_ref);
    (void)cudaGetLastError();
    delete S;
    return TRD_OK;
}

}  // extern "C"
