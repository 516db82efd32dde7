// index.cu -- the tracklet index (Sec. 3: "all tracklets inside a search road
// based on the covariance matrices of the tracks are considered").
//
// Tracklets are bucketed by (chamber, pad row, y bin) with a counting sort:
//   1. count: bucket of each tracklet; a fire-and-forget atomic add on the
//      bucket's counter (nothing waits for its return); block-reduced maxima
//      of vyy and vzz bound the road width.
//   2. exclusive scan of the bucket counters (tile sums, then apply),
//      written one slot late: offsets[b + 1] = first position of bucket b,
//      offsets[0] = 0.
//   3. scatter: atomicAdd on offsets[bucket + 1] returns the tracklet's
//      position, where its 32-byte record goes; when every tracklet is placed,
//      offsets[b + 1] holds the end of bucket b, i.e. the start of bucket
//      b + 1, so offsets[b] is the first position of bucket b for every b.
// The y bins of one (chamber, pad row) are adjacent, so the follower reads
// one contiguous range per pad row.  Order inside a bucket is not defined;
// the follower's selection does not depend on it (ties break on tracklet id).
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>
#include <mutex>

#include "noalloc_cache.h"
#include "trd_device.cuh"
#include "trd_internal.h"

namespace {

constexpr int kCountThreads = 256;
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;
constexpr int kDirectTiles = 1024;  // up to this many scan tiles, each apply block adds up the sums before it

constexpr int kIlp = 4;  // tracklets per thread per loop iteration (loads issued together)

__global__ void __launch_bounds__(kCountThreads)
k_index_count(const int32_t *__restrict__ ch, const float *__restrict__ y, const float *__restrict__ z,
              const float *__restrict__ dy, const float *__restrict__ vyy, const float *__restrict__ vzz,
              const float *__restrict__ vyz, int n, float inv_w, int nb, int32_t *__restrict__ bucket,
              int32_t *__restrict__ counts, uint32_t *__restrict__ stats,
              const int32_t *__restrict__ toff, int n_tf, const float *__restrict__ xs)
{
    float myy = 0.0f, mzz = 0.0f, mdx = 0.0f;
    int rejected = 0;
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * kIlp) {
        int c[kIlp];
        float yy[kIlp], zz[kIlp], dd[kIlp], a[kIlp], b[kIlp], cc[kIlp];
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            const int i = i0 + u * stride;
            const bool in = i < n;
            c[u] = in ? __ldg(&ch[i]) : -1;
            yy[u] = in ? __ldg(&y[i]) : 0.0f;
            zz[u] = in ? __ldg(&z[i]) : 0.0f;
            dd[u] = in ? __ldg(&dy[i]) : 0.0f;
            a[u] = in ? __ldg(&vyy[i]) : 0.0f;
            b[u] = in ? __ldg(&vzz[i]) : 0.0f;
            cc[u] = in ? __ldg(&vyz[i]) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            const int i = i0 + u * stride;
            if (i >= n) continue;
            // a tracklet's radius (misalignment) and its offset from the layer's
            const float xt = xs ? __ldg(&xs[i]) : 0.0f;
            const bool ok = c[u] >= 0 && c[u] < trd::kChambers && isfinite(yy[u]) && isfinite(zz[u]) &&
                            isfinite(dd[u]) && isfinite(a[u]) && isfinite(b[u]) && isfinite(cc[u]) &&
                            a[u] >= 0.0f && b[u] >= 0.0f && isfinite(xt);
            if (!ok) {
                bucket[i] = -1;
                ++rejected;
                continue;
            }
            const int row = trd::row_of_z(zz[u], trd::stack_z_lo(trd::stack_of_chamber(c[u])));
            const int yb = trd::ybin_of(yy[u], inv_w, nb);
            const int bk = trd::bucket_of(trd::tf_of(i, toff, n_tf) * trd::kChambers + c[u], yb, row, nb);
            bucket[i] = bk;
            atomicAdd(&counts[bk], 1);  // return value unused: a reduction, no round trip
            myy = fmaxf(myy, a[u]);
            mzz = fmaxf(mzz, b[u]);
            if (xs) {
                const trd::df xl = trd::layer_x_df(c[u] % trd::kLayers);
                mdx = fmaxf(mdx, fabsf((xt - xl.hi) - xl.lo));
            }
        }
    }
    // block reduction of the maxima and the rejected count
    for (int o = 16; o > 0; o >>= 1) {
        myy = fmaxf(myy, __shfl_xor_sync(0xffffffffu, myy, o));
        mzz = fmaxf(mzz, __shfl_xor_sync(0xffffffffu, mzz, o));
        mdx = fmaxf(mdx, __shfl_xor_sync(0xffffffffu, mdx, o));
        rejected += __shfl_xor_sync(0xffffffffu, rejected, o);
    }
    __shared__ float s_yy[kCountThreads / 32], s_zz[kCountThreads / 32], s_dx[kCountThreads / 32];
    __shared__ int s_rej[kCountThreads / 32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        s_yy[w] = myy;
        s_zz[w] = mzz;
        s_dx[w] = mdx;
        s_rej[w] = rejected;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float am = 0.0f, bm = 0.0f, dm = 0.0f;
        int r = 0;
        for (int k = 0; k < kCountThreads / 32; ++k) {
            am = fmaxf(am, s_yy[k]);
            bm = fmaxf(bm, s_zz[k]);
            dm = fmaxf(dm, s_dx[k]);
            r += s_rej[k];
        }
        // non-negative floats order like their bit patterns
        atomicMax(&stats[0], __float_as_uint(am));
        atomicMax(&stats[1], __float_as_uint(bm));
        if (r) atomicAdd(&stats[2], static_cast<uint32_t>(r));
        if (xs) atomicMax(&stats[3], __float_as_uint(dm));
    }
}

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ __forceinline__ int block_exclusive_scan(int v, int *s_warp, int *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += t;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int s = lane < nw ? s_warp[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        if (lane < nw) s_warp[lane] = s;
    }
    __syncthreads();
    const int before = w ? s_warp[w - 1] : 0;
    *total = s_warp[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before + x - v;
}

// partials[t] = sum of tile t's counters; lastc[t] = its last counter (the
// apply kernel's first thread of tile t + 1 needs it, and by then tile t may
// have zeroed it).
__global__ void __launch_bounds__(kScanThreads)
k_scan_reduce(const int32_t *__restrict__ in, int n, int32_t *__restrict__ partials, int32_t *__restrict__ lastc)
{
    trd::wait_prior_grid();
    const int base = blockIdx.x * kScanTile;
    int s = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; ++k) {
        const int i = base + k * kScanThreads + threadIdx.x;
        if (i < n) {
            const int c = in[i];
            s += c;
            if (k == kScanItems - 1 && threadIdx.x == kScanThreads - 1) lastc[blockIdx.x] = c;
        }
    }
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ int s_w[kScanThreads / 32];
    if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        int t = threadIdx.x < kScanThreads / 32 ? s_w[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) partials[blockIdx.x] = t;
    }
}

// Exclusive scan of the m tile sums in place, one block: for an index of
// more than kDirectTiles tiles (a batch of timeframes), where every apply
// block adding up the sums before it would cost O(m^2) loads.
__global__ void __launch_bounds__(kScanThreads) k_scan_partials(int32_t *__restrict__ p, int m)
{
    trd::wait_prior_grid();
    __shared__ int s_w[kScanThreads / 32];
    int carry = 0;
    for (int base = 0; base < m; base += kScanTile) {
        const int j = base + threadIdx.x * kScanItems;
        int v[kScanItems];
        int sum = 0;
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            v[k] = j + k < m ? p[j + k] : 0;
            sum += v[k];
        }
        int total;
        int run = carry + block_exclusive_scan(sum, s_w, &total);  // its last barrier ends the reads
#pragma unroll
        for (int k = 0; k < kScanItems; ++k) {
            if (j + k < m) p[j + k] = run;
            run += v[k];
        }
        carry += total;
    }
}

// out[b + 1] = exclusive prefix of the counters at b (the scatter's cursor for
// bucket b), out[0] = 0.  A block's base is the sum of the partial sums of the
// tiles before it: added up here by one warp for up to kDirectTiles tiles (no
// separate scan of the partials is launched), else already scanned by
// k_scan_partials (scanned != 0).  The counters are zeroed after they are
// read, so every build leaves them ready for the next one (they start zeroed).
// Each thread takes four consecutive counters with one 16-byte load, zeroes
// them with one 16-byte store and writes out[4t .. 4t + 3] (the prefixes at
// buckets 4t - 1 .. 4t + 2) with one 16-byte store where out is 16-byte
// aligned: a quarter of the L2 transactions of four 4-byte accesses.  The
// counter before its first comes from the previous lane, the previous warp
// or the previous tile (lastc); the thread of the last bucket also writes
// out[n].  n is a multiple of 4.
static_assert(kScanItems == 4, "one 16-byte vector of counters per thread");
static_assert((trd::kChambers * trd::kRowsPerStack) % 4 == 0, "bucket counts come in whole vectors");
__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(int32_t *__restrict__ in, int n, const int32_t *__restrict__ partials,
             const int32_t *__restrict__ lastc, int32_t *__restrict__ out, int scanned)
{
    trd::wait_prior_grid();
    __shared__ int s_w[kScanThreads / 32];
    __shared__ int s_last[kScanThreads / 32];
    __shared__ int s_base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (scanned) {
        if (threadIdx.x == 0) s_base = partials[blockIdx.x];
    } else if (threadIdx.x < 32) {
        int b = 0;
        for (int j = threadIdx.x; j < static_cast<int>(blockIdx.x); j += 32) b += partials[j];
        for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
        if (threadIdx.x == 0) s_base = b;
    }
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanItems;
    const bool in_range = base < n;
    int4 c = make_int4(0, 0, 0, 0);
    if (in_range) {
        c = *reinterpret_cast<const int4 *>(in + base);
        *reinterpret_cast<int4 *>(in + base) = make_int4(0, 0, 0, 0);
    }
    if (lane == 31) s_last[w] = c.w;
    int total;
    // its barriers also publish s_base and s_last
    const int ex = block_exclusive_scan(c.x + c.y + c.z + c.w, s_w, &total);
    int prev = __shfl_up_sync(0xffffffffu, c.w, 1);
    if (lane == 0) prev = w ? s_last[w - 1] : (blockIdx.x ? lastc[blockIdx.x - 1] : 0);
    if (!in_range) return;
    const int run = s_base + ex;  // first position of bucket base
    const int4 o = make_int4(run - prev, run, run + c.x, run + c.x + c.y);
    if ((reinterpret_cast<uintptr_t>(out) & 15u) == 0) {
        *reinterpret_cast<int4 *>(out + base) = o;
    } else {  // a caller's buffer aligned to 4 bytes only
        out[base] = o.x;
        out[base + 1] = o.y;
        out[base + 2] = o.z;
        out[base + 3] = o.w;
    }
    if (base + 4 == n) out[n] = o.w + c.z;
}

__global__ void __launch_bounds__(kCountThreads)
k_index_scatter(const float *__restrict__ y, const float *__restrict__ z, const float *__restrict__ dy,
                const float *__restrict__ vyy, const float *__restrict__ vzz, const float *__restrict__ vyz,
                int n, const int32_t *__restrict__ bucket, int32_t *__restrict__ offsets,
                float4 *__restrict__ rec, const int32_t *__restrict__ toff,
                int n_tf, const int32_t *__restrict__ trig, const float *__restrict__ xs, float *__restrict__ recx)
{
    trd::wait_prior_grid();
    const bool wide = (reinterpret_cast<uintptr_t>(rec) & 31u) == 0;  // 32-byte stores need 32-byte alignment
    const int stride = gridDim.x * blockDim.x;
    for (int i0 = blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += stride * kIlp) {
        // the records' contents are loaded before the position atomics, so
        // the two latencies overlap
        int bk[kIlp], at[kIlp];
        float4 ra[kIlp], rb[kIlp];
        float rx[kIlp];
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            const int i = i0 + u * stride;
            bk[u] = i < n ? __ldg(&bucket[i]) : -1;
            const bool in = i < n;
            // ids are local to the tracklet's timeframe
            const int local = in && toff ? i - __ldg(&toff[trd::tf_of(i, toff, n_tf)]) : i;
            ra[u] = in ? make_float4(__ldg(&y[i]), __ldg(&z[i]), __ldg(&dy[i]), __int_as_float(local))
                       : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            rb[u] = in ? make_float4(__ldg(&vyy[i]), __ldg(&vzz[i]), __ldg(&vyz[i]),
                                     __int_as_float(trig ? __ldg(&trig[i]) : -1))
                       : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            rx[u] = in && xs ? __ldg(&xs[i]) : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < kIlp; ++u) at[u] = bk[u] >= 0 ? atomicAdd(&offsets[bk[u] + 1], 1) : 0;
#pragma unroll
        for (int u = 0; u < kIlp; ++u) {
            if (bk[u] < 0) continue;
            const int pos = at[u];
            if (wide) {
                // the 32-byte record in one store (one L2 transaction where
                // two 16-byte stores take two: the scattered stores and the
                // atomics bound this kernel)
                asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(rec + 2 * pos),
                             "f"(ra[u].x), "f"(ra[u].y), "f"(ra[u].z), "f"(ra[u].w), "f"(rb[u].x), "f"(rb[u].y),
                             "f"(rb[u].z), "f"(rb[u].w)
                             : "memory");
            } else {  // records only 16-byte aligned (a caller's buffer)
                rec[2 * pos] = ra[u];
                rec[2 * pos + 1] = rb[u];
            }
            if (xs) recx[pos] = rx[u];
        }
    }
}

}  // namespace

namespace trd_host {

int scan_blocks_for(int n) { return (n + kScanTile - 1) / kScanTile; }

int index_rebuild_launch(trd_index *idx, const trd_tracklets_t *t, cudaStream_t s)
{
    const int n = t->n;
    // the bucket counters are zero between builds: cleared here when no
    // complete build has run since they were (first build, or a build that
    // stopped on an error), otherwise by the previous build's scan after it
    // read them; the flag is set again once this build's scan is enqueued
    const bool clear = !idx->counts_zero;
    idx->counts_zero = false;
    if (clear) TRD_CUDA_TRY(cudaMemsetAsync(idx->counts, 0, sizeof(int32_t) * idx->n_buckets, s));
    TRD_CUDA_TRY(cudaMemsetAsync(idx->stats, 0, sizeof(uint32_t) * 4, s));
    const int grid_n =
        n > 0 ? std::min((n + kCountThreads * kIlp - 1) / (kCountThreads * kIlp), idx->ctx->sm_count * 8) : 0;
    if (n > 0) {
        k_index_count<<<grid_n, kCountThreads, 0, s>>>(t->chamber, t->y, t->z, t->dy, t->vyy, t->vzz, t->vyz, n,
                                                       idx->inv_w, idx->nb, idx->bucket, idx->counts,
                                                       idx->stats, idx->toff, idx->n_tf, t->x);
        TRD_CUDA_TRY(cudaGetLastError());
    }
    const int m = scan_blocks_for(idx->n_buckets);
    // the scan and the scatter start while their predecessor drains
    int32_t *lastc = idx->partials + idx->n_partials + 1;
    TRD_CUDA_TRY(launch_after(k_scan_reduce, dim3(m), dim3(kScanThreads), 0, s, idx->counts, idx->n_buckets,
                              idx->partials, lastc));
    const int scanned = m > kDirectTiles;
    if (scanned) TRD_CUDA_TRY(launch_after(k_scan_partials, dim3(1), dim3(kScanThreads), 0, s, idx->partials, m));
    TRD_CUDA_TRY(launch_after(k_scan_apply, dim3(m), dim3(kScanThreads), 0, s, idx->counts, idx->n_buckets,
                              idx->partials, static_cast<const int32_t *>(lastc), idx->offsets, scanned));
    idx->counts_zero = true;  // the scan just enqueued leaves them zero
    if (n > 0) {
        TRD_CUDA_TRY(launch_after(k_index_scatter, dim3(grid_n), dim3(kCountThreads), 0, s, t->y, t->z, t->dy,
                                  t->vyy, t->vzz, t->vyz, n, idx->bucket, idx->offsets, idx->rec, idx->toff,
                                  idx->n_tf, t->trigger, t->x, idx->recx));
    }
    idx->has_x = t->x != nullptr;
    return TRD_OK;
}

}  // namespace trd_host

// ---- index build into caller buffers, with no allocation --------------------
// Some callers cannot allocate device memory at the point where they build an
// index: code running inside a framework that owns every device allocation
// through its own pool, or a real-time loop that must not call cudaMalloc
// because it may synchronise the device.  For them the build's scratch (the
// bucket of every tracklet, one counter per bucket, scan partials) lives in
// the file-scope array below, sized for kNoAllocMaxTracklets tracklets and
// y bins of at least kNoAllocMinBinWidth cm.  Every GPU that loads the library
// holds it (about 9.3 MB) until the process exits, and all calls on a device
// share it.
namespace {

constexpr int kNoAllocMaxTracklets = 1 << 20;
constexpr float kNoAllocMinBinWidth = 1.0f;
constexpr int kNoAllocMaxBins = 132;  // ceil(2 * 66 cm / 1 cm)
constexpr int kNoAllocMaxBuckets = trd::kChambers * trd::kRowsPerStack * kNoAllocMaxBins;
constexpr int kNoAllocMaxPartials = (kNoAllocMaxBuckets + kScanTile - 1) / kScanTile + 1;
constexpr size_t kNoAllocWords =
    static_cast<size_t>(kNoAllocMaxTracklets) + kNoAllocMaxBuckets + 2 * kNoAllocMaxPartials;

static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocWords];

constexpr int kNoAllocMaxDevices = 64;
trd_host::NoAllocEntry g_noalloc_dev[kNoAllocMaxDevices];
std::mutex g_noalloc_mu;

// The current context's id through the driver API (resolved once through the
// runtime, so the library needs no link against the driver library).
bool current_ctx_id(unsigned long long *id)
{
    using GetCurrent = CUresult (*)(CUcontext *);
    using GetId = CUresult (*)(CUcontext, unsigned long long *);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *a = nullptr, *b = nullptr;
        cudaDriverEntryPointQueryResult qa{}, qb{};
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) == cudaSuccess &&
            qa == cudaDriverEntryPointSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) == cudaSuccess &&
            qb == cudaDriverEntryPointSuccess) {
            get_current = reinterpret_cast<GetCurrent>(a);
            get_id = reinterpret_cast<GetId>(b);
        }
        (void)cudaGetLastError();
    });
    if (!get_current || !get_id) return false;
    CUcontext c = nullptr;
    if (get_current(&c) != CUDA_SUCCESS || !c) return false;
    return get_id(c, id) == CUDA_SUCCESS;
}

// With the device current: fetch the address the kernels must be given (the
// host-side name of the array is not a device address) and the SM count.
int noalloc_lookup(int dev, trd_host::NoAllocEntry *e)
{
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        (void)cudaGetLastError();
        return TRD_ECUDA;
    }
    e->scratch = static_cast<int32_t *>(p);
    if (cudaDeviceGetAttribute(&e->sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return TRD_ECUDA;
    }
    return TRD_OK;
}

// Once per device and context (again after the context was re-created).
int noalloc_setup(int dev, trd_host::NoAllocEntry *out)
{
    const int rc = trd_host::noalloc_resolve(g_noalloc_dev, kNoAllocMaxDevices, g_noalloc_mu, dev, current_ctx_id,
                                             noalloc_lookup, out);
    return rc ? TRD_ECUDA : TRD_OK;
}

}  // namespace

extern "C" int trd_index_build_noalloc(const trd_tracklets_t *t, float y_bin_width, int32_t *offsets,
                                       float *records, uint32_t *stats, void *stream)
{
    if (!t || !offsets || !records || !stats || t->n < 0) return TRD_EINVAL;
    if (t->n > kNoAllocMaxTracklets) return TRD_EINVAL;  // larger than the static scratch
    if (y_bin_width == 0.0f) y_bin_width = 2.0f;
    if (!(y_bin_width >= kNoAllocMinBinWidth) || !isfinite(y_bin_width)) return TRD_EINVAL;
    if (reinterpret_cast<uintptr_t>(records) % 16 != 0) return TRD_EINVAL;
    if (t->n > 0 && (!t->chamber || !t->y || !t->z || !t->dy || !t->vyy || !t->vzz || !t->vyz)) return TRD_EINVAL;
    if (t->x) return TRD_EINVAL;  // no room for per-tracklet radii in the caller's buffers
    int dev = 0;
    TRD_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kNoAllocMaxDevices) return TRD_ECUDA;
    trd_host::NoAllocEntry d;
    const int rc = noalloc_setup(dev, &d);
    if (rc) return rc;

    const int n = t->n;
    const int nb = static_cast<int>(ceilf(2.0f * trd::kYHalf / y_bin_width));
    const float inv_w = 1.0f / y_bin_width;
    const int n_buckets = trd::kChambers * trd::kRowsPerStack * nb;
    const int m = (n_buckets + kScanTile - 1) / kScanTile;
    int32_t *bucket = d.scratch;
    int32_t *counts = bucket + kNoAllocMaxTracklets;
    int32_t *partials = counts + kNoAllocMaxBuckets;
    int32_t *lastc = partials + kNoAllocMaxPartials;
    float4 *rec = reinterpret_cast<float4 *>(records);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    // the counters and the caller's stats must start at zero: the shared array
    // keeps whatever the last call left (its scan re-zeroes the counters, but
    // a call that did not complete would not), so they are cleared here; the
    // rest of the scratch is fully written before it is read
    TRD_CUDA_TRY(cudaMemsetAsync(counts, 0, sizeof(int32_t) * n_buckets, s));
    TRD_CUDA_TRY(cudaMemsetAsync(stats, 0, sizeof(uint32_t) * 4, s));
    const int grid_n = n > 0 ? std::min((n + kCountThreads * kIlp - 1) / (kCountThreads * kIlp), d.sm_count * 8) : 0;
    if (n > 0) {
        k_index_count<<<grid_n, kCountThreads, 0, s>>>(t->chamber, t->y, t->z, t->dy, t->vyy, t->vzz, t->vyz, n,
                                                       inv_w, nb, bucket, counts, stats, nullptr, 1, nullptr);
        TRD_CUDA_TRY(cudaGetLastError());
    }
    k_scan_reduce<<<m, kScanThreads, 0, s>>>(counts, n_buckets, partials, lastc);
    TRD_CUDA_TRY(cudaGetLastError());
    static_assert(kNoAllocMaxPartials - 1 <= kDirectTiles, "the allocation-free build adds up tile sums directly");
    k_scan_apply<<<m, kScanThreads, 0, s>>>(counts, n_buckets, partials, lastc, offsets, 0);
    TRD_CUDA_TRY(cudaGetLastError());
    if (n > 0) {
        k_index_scatter<<<grid_n, kCountThreads, 0, s>>>(t->y, t->z, t->dy, t->vyy, t->vzz, t->vyz, n, bucket,
                                                         offsets, rec, nullptr, 1, t->trigger, nullptr, nullptr);
        TRD_CUDA_TRY(cudaGetLastError());
    }
    return TRD_OK;
}
