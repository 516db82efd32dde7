// trd_internal.h -- host-side definitions shared by the library's sources.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/trd_abi.h"

struct trd_ctx {
    int device;
    int sm_count;
    int max_threads_per_sm;
    size_t l2_bytes;
};

// Device-resident tracklet index (built by trd_index_build / rebuild).
struct trd_index {
    trd_ctx *ctx;
    int device;
    int32_t capacity;   // tracklets the buffers can hold
    int32_t n_input;    // tracklets given to the last build
    float y_bin_width;  // cm
    float inv_w;
    int32_t nb;         // y bins per (chamber, pad row)
    int32_t n_tf;       // timeframes indexed together (1 for a plain index)
    int32_t *toff;      // [n_tf + 1] tracklet offsets per timeframe (device), null when n_tf = 1
    int32_t n_buckets;  // n_tf * 540 * 18 * nb
    // index proper
    int32_t *offsets;   // [n_buckets + 1] exclusive prefix of bucket sizes
    float4 *rec;        // [2 * capacity]: per tracklet, in bucket order, a 32-byte
                        // record {y, z, dy, id (bits)}, {vyy, vzz, vyz, 0}
    uint32_t *stats;    // [4]: max vyy bits, max vzz bits, rejected count, max |x - x_layer| bits
    float *recx;        // [capacity]: per tracklet, in bucket order, its radius (when given)
    int has_x;          // the last build's tracklets carried radii
    // build scratch
    int32_t *bucket;    // [capacity] bucket of each input tracklet (-1: rejected)
    int32_t *counts;    // [n_buckets], zero between builds (each build's scan re-zeroes them)
    bool counts_zero;   // the counters are zero for the next build (set by a build whose scan
                        // was enqueued, or by the batch before its capture)
    int32_t *partials;  // [scan blocks + 1] tile sums, then [scan blocks + 1] each tile's last counter
    int32_t n_partials;
    cudaStream_t stream;  // stream of the last build
    cudaEvent_t built;
};

// Plain-pointer views passed to kernels.
struct IndexView {
    const int32_t *offsets;
    const float4 *rec;  // 2 float4 per tracklet
    const uint32_t *stats;
    int32_t nb;
    float inv_w;
    const float *recx = nullptr;  // radius per record, or null (every tracklet at its layer's radius)
    int32_t max_tf_tracklets = 0; // most tracklets of one timeframe (their ids' bound)
};

namespace trd_host {
// Caller-owned events recorded just before and just after the follower
// kernel's launch (trd_follow_timed).
struct KernelEvents {
    cudaEvent_t start, end;
};
int index_rebuild_launch(trd_index *idx, const trd_tracklets_t *t, cudaStream_t s);
int follow_launch(const trd_ctx *ctx, const trd_seeds_t *seeds, const IndexView &iv,
                  const trd_params_t *p, trd_results_t *out, cudaStream_t s, int lanes_per_track,
                  int block_threads, int min_blocks, int *counter, const int32_t *seed_offsets = nullptr,
                  int n_tf = 1, const trd_alignment_t *align = nullptr, bool prepare = true,
                  void *parked = nullptr, const KernelEvents *kev = nullptr);
// Device scratch of the seeds' pre-pass for n seeds (sorted, rotated states).
size_t parked_bytes(int32_t n, int32_t n_tf = 1);
int prepare_launch(const trd_seeds_t *seeds, const trd_params_t *p, trd_results_t *out, cudaStream_t s,
                   void *parked, int *counter, const int32_t *seed_offsets = nullptr, int n_tf = 1,
                   const trd_alignment_t *align = nullptr);
int follow_checked(trd_ctx *ctx, const trd_seeds_t *seeds, const trd_index *index, const trd_params_t *p,
                   const trd_alignment_t *align, trd_results_t *out, void *stream, const trd_launch_t *launch,
                   void *parked, const KernelEvents *kev = nullptr);
int index_alloc(trd_ctx *ctx, int32_t capacity, float y_bin_width, int32_t n_tf, trd_index **out);
void index_release(trd_index *x);
int scan_blocks_for(int n);
}  // namespace trd_host

namespace trd_host {
// Launch `kernel` after the previous kernel in stream s with programmatic
// serialization: its blocks may be scheduled before that kernel has finished
// (hiding the launch latency), and they wait in trd::wait_prior_grid(), which
// every kernel launched this way calls first.
template <typename... K, typename... A>
inline cudaError_t launch_after(void (*kernel)(K...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                                A &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<A &&>(args)...);
}
}  // namespace trd_host

#define TRD_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) {                             \
            (void)cudaGetLastError();                        \
            return TRD_ECUDA;                                \
        }                                                    \
    } while (0)
