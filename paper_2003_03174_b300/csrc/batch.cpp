// batch.cpp -- many timeframes in one CUDA-graph replay.
//
// The timeframes of a batch are concatenated (seeds, tracklets, results) and
// described by offset tables.  One index covers all of them (its key carries
// the timeframe), and one persistent follower launch pulls seeds of every
// timeframe from a single work counter, so small timeframes share the GPU
// with large ones instead of each running a half-empty launch.  The whole
// sequence (index build, counter reset, follower) is captured once into a
// CUDA graph at creation and replayed by trd_batch_run.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "trd_internal.h"

struct trd_batch {
    trd_ctx *ctx;
    int n_tf;
    trd_index *index;
    int32_t *soff;      // [n_tf + 1] device seed offsets
    int32_t *counter;   // the follower's work counter (private to this batch)
    void *parked;       // the seeds' pre-pass output (sorted, rotated states)
    cudaGraph_t graph;
    cudaGraphExec_t exec;
};

namespace {

bool valid_offsets(const int32_t *off, int n_tf, int32_t total)
{
    if (!off || off[0] != 0 || off[n_tf] != total) return false;
    for (int t = 0; t < n_tf; ++t)
        if (off[t + 1] < off[t]) return false;
    return true;
}

void release(trd_batch *b)
{
    cudaSetDevice(b->ctx->device);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->index) trd_host::index_release(b->index);
    cudaFree(b->soff);
    cudaFree(b->counter);
    cudaFree(b->parked);
    (void)cudaGetLastError();
    delete b;
}

}  // namespace

extern "C" {

int trd_batch_create(trd_ctx_t *ctx, int32_t n_tf, const int32_t *seed_offsets, const int32_t *tracklet_offsets,
                     const trd_seeds_t *seeds, const trd_tracklets_t *tracklets, const trd_params_t *params,
                     trd_results_t *results, float y_bin_width, const trd_launch_t *launch, trd_batch_t **out)
{
    if (!ctx || !seeds || !tracklets || !params || !results || !out || n_tf < 1) return TRD_EINVAL;
    *out = nullptr;
    if (seeds->n < 0 || tracklets->n < 0) return TRD_EINVAL;
    if (!valid_offsets(seed_offsets, n_tf, seeds->n) || !valid_offsets(tracklet_offsets, n_tf, tracklets->n))
        return TRD_EINVAL;
    TRD_CUDA_TRY(cudaSetDevice(ctx->device));
    trd_batch *b = new (std::nothrow) trd_batch;
    if (!b) return TRD_ENOMEM;
    memset(b, 0, sizeof *b);
    b->ctx = ctx;
    b->n_tf = n_tf;
    int rc = trd_host::index_alloc(ctx, tracklets->n, y_bin_width, n_tf, &b->index);
    if (rc) {
        delete b;
        return rc;
    }
    if (cudaMalloc(&b->soff, sizeof(int32_t) * (n_tf + 1)) != cudaSuccess ||
        cudaMalloc(&b->counter, sizeof(int32_t)) != cudaSuccess ||
        (seeds->n > 0 && cudaMalloc(&b->parked, trd_host::parked_bytes(seeds->n, n_tf)) != cudaSuccess)) {
        release(b);
        return TRD_ENOMEM;
    }
    if (cudaMemcpy(b->soff, seed_offsets, sizeof(int32_t) * (n_tf + 1), cudaMemcpyHostToDevice) != cudaSuccess ||
        (n_tf > 1 && cudaMemcpy(b->index->toff, tracklet_offsets, sizeof(int32_t) * (n_tf + 1),
                                cudaMemcpyHostToDevice) != cudaSuccess)) {
        release(b);
        return TRD_ECUDA;
    }
    // the index's bucket counters zeroed before the capture, so that the
    // captured build does not repeat that memset on every replay
    if (cudaMemset(b->index->counts, 0, sizeof(int32_t) * b->index->n_buckets) != cudaSuccess ||
        cudaDeviceSynchronize() != cudaSuccess) {
        release(b);
        return TRD_ECUDA;
    }
    b->index->counts_zero = true;
    // validate the follower's arguments once, with the plain entry point's rules
    trd_seeds_t none = *seeds;
    none.n = 0;
    rc = trd_follow_tuned(ctx, &none, b->index, params, results, nullptr, launch);
    if (rc) {
        release(b);
        return rc;
    }
    if (seeds->n > 0 && (!results->alpha || !results->x || !results->par || !results->cov || !results->chi2 ||
                         !results->n_trk || !results->n_miss || !results->status || !results->tracklet_id)) {
        release(b);
        return TRD_EINVAL;
    }

    // the graph: the seeds' pre-pass on a branch beside the index build (it
    // does not read the index), joined before the follower
    cudaStream_t cs = nullptr, cs2 = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&cs2, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
        if (cs) cudaStreamDestroy(cs);
        if (cs2) cudaStreamDestroy(cs2);
        if (fork) cudaEventDestroy(fork);
        (void)cudaGetLastError();
        release(b);
        return TRD_ECUDA;
    }
    bool ok = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
        ok = cudaEventRecord(fork, cs) == cudaSuccess && cudaStreamWaitEvent(cs2, fork, 0) == cudaSuccess;
        if (ok)
            rc = trd_host::prepare_launch(seeds, params, results, cs2, b->parked, b->counter,
                                          n_tf > 1 ? b->soff : nullptr, n_tf);
        if (ok && !rc) ok = cudaEventRecord(join, cs2) == cudaSuccess;
        if (ok && !rc) rc = trd_host::index_rebuild_launch(b->index, tracklets, cs);
        if (ok && !rc) ok = cudaStreamWaitEvent(cs, join, 0) == cudaSuccess;
        if (ok && !rc) {
            int32_t most = 0;
            for (int t = 0; t < n_tf; ++t) most = std::max(most, tracklet_offsets[t + 1] - tracklet_offsets[t]);
            IndexView iv{b->index->offsets, b->index->rec, b->index->stats, b->index->nb, b->index->inv_w,
                         tracklets->x ? b->index->recx : nullptr, most};
            rc = trd_host::follow_launch(ctx, seeds, iv, params, results, cs, launch ? launch->lanes_per_track : 0,
                                         launch ? launch->block_threads : 0, launch ? launch->min_blocks_per_sm : 0,
                                         b->counter, n_tf > 1 ? b->soff : nullptr, n_tf, nullptr, false,
                                         b->parked);
        }
        const bool ended = cudaStreamEndCapture(cs, &b->graph) == cudaSuccess;
        ok = ok && !rc && ended && cudaGraphInstantiate(&b->exec, b->graph, 0) == cudaSuccess;
    }
    cudaStreamDestroy(cs);
    cudaStreamDestroy(cs2);
    cudaEventDestroy(fork);
    cudaEventDestroy(join);
    if (!ok) {
        (void)cudaGetLastError();
        release(b);
        return rc ? rc : TRD_ECUDA;
    }
    b->index->n_input = tracklets->n;
    *out = b;
    return TRD_OK;
}

int trd_batch_run(trd_batch_t *b, void *stream)
{
    if (!b) return TRD_EINVAL;
    TRD_CUDA_TRY(cudaSetDevice(b->ctx->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TRD_CUDA_TRY(cudaGraphLaunch(b->exec, s));
    TRD_CUDA_TRY(cudaEventRecord(b->index->built, s));
    return TRD_OK;
}

int trd_batch_free(trd_batch_t *b)
{
    if (!b) return TRD_EINVAL;
    release(b);
    return TRD_OK;
}

}  // extern "C"
