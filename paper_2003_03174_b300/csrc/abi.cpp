// abi.cpp -- the C entry points of libtrd.so (declared in include/trd_abi.h).
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>

#include "trd_internal.h"

namespace {

constexpr int kRowsPerStack = 18;
constexpr float kYHalf = 66.0f;
constexpr float kDefaultBinWidth = 2.0f;

bool finite_pos(float v) { return isfinite(v) && v > 0.0f; }

int check_device(int device)
{
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || n <= 0) {
        (void)cudaGetLastError();
        return TRD_ECUDA;
    }
    if (device < 0 || device >= n) return TRD_ECUDA;
    return TRD_OK;
}

void free_index_buffers(trd_index *x)
{
    cudaFree(x->offsets);
    cudaFree(x->rec);
    cudaFree(x->recx);
    cudaFree(x->stats);
    cudaFree(x->bucket);
    cudaFree(x->counts);
    cudaFree(x->partials);
    cudaFree(x->toff);
    if (x->built) cudaEventDestroy(x->built);
    (void)cudaGetLastError();
}

}  // namespace

namespace trd_host {
// Allocate an index for up to `capacity` tracklets of `n_tf` timeframes.
int index_alloc(trd_ctx *ctx, int32_t capacity, float y_bin_width, int32_t n_tf, trd_index **out)
{
    if (!ctx || !out || capacity < 0 || n_tf < 1) return TRD_EINVAL;
    *out = nullptr;
    if (y_bin_width == 0.0f) y_bin_width = kDefaultBinWidth;
    if (!finite_pos(y_bin_width) || y_bin_width < 0.05f) return TRD_EINVAL;
    const int32_t nb = static_cast<int32_t>(ceilf(2.0f * kYHalf / y_bin_width));
    const long long n_buckets = static_cast<long long>(n_tf) * TRD_N_CHAMBERS * kRowsPerStack * nb;
    if (n_buckets >= (1LL << 31) - 1) return TRD_EINVAL;
    TRD_CUDA_TRY(cudaSetDevice(ctx->device));
    trd_index *x = new (std::nothrow) trd_index;
    if (!x) return TRD_ENOMEM;
    memset(x, 0, sizeof *x);
    x->ctx = ctx;
    x->device = ctx->device;
    x->capacity = capacity;
    x->y_bin_width = y_bin_width;
    x->nb = nb;
    x->inv_w = 1.0f / y_bin_width;
    x->n_tf = n_tf;
    x->n_buckets = static_cast<int32_t>(n_buckets);
    x->n_partials = scan_blocks_for(x->n_buckets);
    const size_t cap = static_cast<size_t>(std::max(capacity, 1));
    bool ok = cudaMalloc(&x->offsets, sizeof(int32_t) * (x->n_buckets + 1)) == cudaSuccess &&
              cudaMalloc(&x->rec, 2 * sizeof(float4) * cap) == cudaSuccess &&
              cudaMalloc(&x->recx, sizeof(float) * cap) == cudaSuccess &&
              cudaMalloc(&x->stats, sizeof(uint32_t) * 4) == cudaSuccess &&
              cudaMalloc(&x->bucket, sizeof(int32_t) * cap) == cudaSuccess &&
              cudaMalloc(&x->counts, sizeof(int32_t) * x->n_buckets) == cudaSuccess &&
              cudaMalloc(&x->partials, sizeof(int32_t) * 2 * (x->n_partials + 1)) == cudaSuccess &&
              (n_tf == 1 || cudaMalloc(&x->toff, sizeof(int32_t) * (n_tf + 1)) == cudaSuccess) &&
              cudaEventCreateWithFlags(&x->built, cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        free_index_buffers(x);
        delete x;
        return TRD_ENOMEM;
    }
    *out = x;
    return TRD_OK;
}

void index_release(trd_index *x)
{
    cudaSetDevice(x->device);
    free_index_buffers(x);
    delete x;
}
}  // namespace trd_host

extern "C" {

const char *trd_version(void) { return "trd-b300 0.1 (sm_103a, FP32)"; }

int trd_geometry(double *out, int n)
{
    if (!out || n < 0) return TRD_EINVAL;
    const double v[] = {18, 5, 6, 540, 300.0, 12.6, 144.0, -360.0, 2.0, 3.0, 8.0, 2.99792458e-3, 0.95};
    for (int i = 0; i < n && i < static_cast<int>(sizeof v / sizeof v[0]); ++i) out[i] = v[i];
    return TRD_OK;
}

int trd_ctx_create(int device, trd_ctx_t **ctx)
{
    if (!ctx) return TRD_EINVAL;
    *ctx = nullptr;
    int rc = check_device(device);
    if (rc) return rc;
    TRD_CUDA_TRY(cudaSetDevice(device));
    cudaDeviceProp prop;
    TRD_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (prop.major * 10 + prop.minor != 103) return TRD_ECUDA;  // kernels are built for sm_103a only
    trd_ctx *c = new (std::nothrow) trd_ctx;
    if (!c) return TRD_ENOMEM;
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    c->max_threads_per_sm = prop.maxThreadsPerMultiProcessor;
    c->l2_bytes = static_cast<size_t>(prop.l2CacheSize);
    // the follower and the server take stream-ordered scratch from the
    // device's default pool on every call: keep freed blocks in the pool
    // (the default threshold of 0 returns them to the system at every
    // synchronisation, and the next call maps fresh memory)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
        uint64_t keep = ~0ull;
        (void)cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    (void)cudaGetLastError();
    *ctx = c;
    return TRD_OK;
}

int trd_ctx_destroy(trd_ctx_t *ctx)
{
    if (!ctx) return TRD_EINVAL;
    delete ctx;
    return TRD_OK;
}

int trd_ctx_sm_count(const trd_ctx_t *ctx) { return ctx ? ctx->sm_count : TRD_EINVAL; }

int trd_index_create(trd_ctx_t *ctx, int32_t capacity, float y_bin_width, trd_index_t **out)
{
    return trd_host::index_alloc(ctx, capacity, y_bin_width, 1, out);
}

int trd_index_rebuild(trd_index_t *index, const trd_tracklets_t *t, void *stream)
{
    if (!index || !t || t->n < 0 || t->n > index->capacity) return TRD_EINVAL;
    if (t->n > 0 && (!t->chamber || !t->y || !t->z || !t->dy || !t->vyy || !t->vzz || !t->vyz)) return TRD_EINVAL;
    TRD_CUDA_TRY(cudaSetDevice(index->device));
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int rc = trd_host::index_rebuild_launch(index, t, s);
    if (rc) return rc;
    index->n_input = t->n;
    index->stream = s;
    TRD_CUDA_TRY(cudaEventRecord(index->built, s));
    return TRD_OK;
}

int trd_index_build(trd_ctx_t *ctx, const trd_tracklets_t *t, float y_bin_width, void *stream,
                    trd_index_t **out)
{
    if (!ctx || !t || !out || t->n < 0) return TRD_EINVAL;
    trd_index_t *x = nullptr;
    int rc = trd_index_create(ctx, t->n, y_bin_width, &x);
    if (rc) return rc;
    rc = trd_index_rebuild(x, t, stream);
    if (rc) {
        trd_index_free(x);
        return rc;
    }
    *out = x;
    return TRD_OK;
}

int trd_index_free(trd_index_t *index)
{
    if (!index) return TRD_EINVAL;
    cudaSetDevice(index->device);
    free_index_buffers(index);  // cudaFree waits for work that uses the buffers
    delete index;
    return TRD_OK;
}

int trd_index_info(const trd_index_t *index, int32_t *n_indexed, int32_t *n_rejected, int32_t *n_buckets)
{
    if (!index) return TRD_EINVAL;
    TRD_CUDA_TRY(cudaSetDevice(index->device));
    TRD_CUDA_TRY(cudaEventSynchronize(index->built));
    uint32_t st[4] = {0, 0, 0, 0};
    TRD_CUDA_TRY(cudaMemcpy(st, index->stats, sizeof st, cudaMemcpyDeviceToHost));
    if (n_rejected) *n_rejected = static_cast<int32_t>(st[2]);
    if (n_indexed) *n_indexed = index->n_input - static_cast<int32_t>(st[2]);
    if (n_buckets) *n_buckets = index->n_buckets;
    return TRD_OK;
}

int trd_index_copy_out(const trd_index_t *index, int32_t *offsets, int32_t *ids)
{
    if (!index) return TRD_EINVAL;
    TRD_CUDA_TRY(cudaSetDevice(index->device));
    TRD_CUDA_TRY(cudaEventSynchronize(index->built));
    if (offsets)
        TRD_CUDA_TRY(cudaMemcpy(offsets, index->offsets, sizeof(int32_t) * (index->n_buckets + 1),
                                cudaMemcpyDeviceToHost));
    if (ids) {
        int32_t total = 0;
        TRD_CUDA_TRY(cudaMemcpy(&total, index->offsets + index->n_buckets, sizeof total, cudaMemcpyDeviceToHost));
        // word 3 of each 32-byte record holds the input index bits
        if (total > 0)
            TRD_CUDA_TRY(cudaMemcpy2D(ids, sizeof(int32_t), reinterpret_cast<const char *>(index->rec) + 12,
                                      2 * sizeof(float4), sizeof(int32_t), total, cudaMemcpyDeviceToHost));
    }
    return TRD_OK;
}

int trd_follow_tuned(trd_ctx_t *ctx, const trd_seeds_t *seeds, const trd_index_t *index,
                     const trd_params_t *p, trd_results_t *out, void *stream, const trd_launch_t *launch)
{
    return trd_follow_aligned(ctx, seeds, index, p, nullptr, out, stream, launch);
}

int trd_follow_aligned(trd_ctx_t *ctx, const trd_seeds_t *seeds, const trd_index_t *index,
                       const trd_params_t *p, const trd_alignment_t *align, trd_results_t *out, void *stream,
                       const trd_launch_t *launch)
{
    return trd_host::follow_checked(ctx, seeds, index, p, align, out, stream, launch, nullptr);
}

}  // extern "C"

// The follower's public entry points after validation; parked: the
// pre-pass's scratch (trd_host::parked_bytes), or null to take it from the
// device's pool on the stream.
int trd_host::follow_checked(trd_ctx *ctx, const trd_seeds_t *seeds, const trd_index *index, const trd_params_t *p,
                             const trd_alignment_t *align, trd_results_t *out, void *stream,
                             const trd_launch_t *launch, void *parked, const KernelEvents *kev)
{
    if (align && align->bz_map &&
        (align->nr < 2 || align->nz < 2 || !(align->r_max > align->r_min) || !(align->z_max > align->z_min) ||
         !isfinite(align->r_min) || !isfinite(align->r_max) || !isfinite(align->z_min) || !isfinite(align->z_max)))
        return TRD_EINVAL;
    const int lanes_per_track = launch ? launch->lanes_per_track : 0;
    const int block_threads = launch ? launch->block_threads : 0;
    const int min_blocks = launch ? launch->min_blocks_per_sm : 0;
    if (!ctx || !seeds || !index || !p || !out || seeds->n < 0) return TRD_EINVAL;
    if (p->n_hyp < 1 || p->n_hyp > TRD_MAX_HYP || p->max_missing < 0 || p->max_missing > TRD_N_LAYERS) return TRD_EINVAL;
    if (!finite_pos(p->n_sigma_road) || !finite_pos(p->chi2_cut) || !finite_pos(p->dy_gate_sigma) ||
        !isfinite(p->p_miss) || !isfinite(p->bz))
        return TRD_EINVAL;
    if (block_threads != 0 && block_threads != 64 && block_threads != 128) return TRD_EINVAL;
    if (seeds->n > 0) {
        if (!seeds->alpha || !seeds->x || !seeds->y || !seeds->z || !seeds->snp || !seeds->tgl || !seeds->q2pt ||
            !seeds->cov)
            return TRD_EINVAL;
        if (!out->alpha || !out->x || !out->par || !out->cov || !out->chi2 || !out->n_trk || !out->n_miss ||
            !out->status || !out->tracklet_id)
            return TRD_EINVAL;
    }
    TRD_CUDA_TRY(cudaSetDevice(ctx->device));
    IndexView iv{index->offsets, index->rec, index->stats, index->nb, index->inv_w,
                 index->has_x ? index->recx : nullptr, index->n_input};
    return trd_host::follow_launch(ctx, seeds, iv, p, out, static_cast<cudaStream_t>(stream), lanes_per_track,
                                   block_threads, min_blocks, nullptr, nullptr, 1, align, true,
                                   parked, kev);
}

extern "C" {

int trd_follow(trd_ctx_t *ctx, const trd_seeds_t *seeds, const trd_index_t *index, const trd_params_t *p,
               trd_results_t *out, void *stream)
{
    return trd_follow_tuned(ctx, seeds, index, p, out, stream, nullptr);
}

int trd_follow_timed(trd_ctx_t *ctx, const trd_seeds_t *seeds, const trd_index_t *index, const trd_params_t *p,
                     trd_results_t *out, void *stream, const trd_launch_t *launch, void *ev_start, void *ev_end)
{
    if (!ev_start || !ev_end) return TRD_EINVAL;
    const trd_host::KernelEvents kev{static_cast<cudaEvent_t>(ev_start), static_cast<cudaEvent_t>(ev_end)};
    return trd_host::follow_checked(ctx, seeds, index, p, nullptr, out, stream, launch, nullptr, &kev);
}

}  // extern "C"
