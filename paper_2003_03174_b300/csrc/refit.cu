// refit.cu -- the TRD-only refit of matched tracks (arXiv:2003.03174, Sec. 2,
// step 3: two independent refits, from the ITS and from TRD+TOF, ignore the
// TPC clusters; this is the TRD one).
//
// One thread per track.  The thread gathers the track's tracklets (six
// random 4-byte loads per tracklet, issued together before any arithmetic),
// starts from the follower's final state with a diagonal, widened
// covariance, and runs the Kalman filter inward from the outermost matched
// layer to layer 0 with the follower's own transport, rotation, update and
// (inward) material step.  No device-side waits, no shared memory.
#include <cuda_runtime.h>
#include <math.h>

#include "trd_device.cuh"
#include "trd_internal.h"
#include "track_model.cuh"

namespace trd {

struct RefitIn {
    const float *alpha, *x, *par, *cov;
    const int32_t *status, *ids;
    int n;
};

struct TrackletSoA {
    const int32_t *ch;
    const float *y, *z, *vyy, *vzz, *vyz;
    int n;
    const float *x;  // own radius per tracklet (misalignment), or null
};

struct RefitOut {
    float *alpha, *x, *par, *cov, *chi2;
    int32_t *nupd, *status;
};

struct RefitParams {
    float bz, cov_scale;
    int resmode, material;
};

__device__ __forceinline__ int sector_of_alpha(float a)
{
    const float u = a - kTwoPiHi * floorf(a * (1.0f / kTwoPiHi));
    return min(max(static_cast<int>(u * (1.0f / kSectorWidthHi)), 0), kSectors - 1);
}

// Rotate the state from the frame `frame` into the frame of sector `target`.
__device__ __forceinline__ bool enter_sector(TrackState &s, df &frame, int target, float bz)
{
    const df to = sector_alpha_df(target);
    df d = df_add(to, df_neg(frame));
    if (d.hi > 3.14159265f) d = df_add(d, df{-kTwoPiHi, -kTwoPiLo});
    if (d.hi < -3.14159265f) d = df_add(d, df{kTwoPiHi, kTwoPiLo});
    if (!rotate(s, d, target, bz)) return false;
    frame = to;
    return true;
}

__global__ void __launch_bounds__(128) k_refit(RefitIn in, TrackletSoA T, RefitParams P, RefitOut o)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = in.n;
    if (i >= n) return;

    // ids and the tracklets they name, all loads issued up front
    int ids[kLayers], ch[kLayers];
    float ty[kLayers], tz[kLayers], tvy[kLayers], tvz[kLayers], tvyz[kLayers], tx[kLayers];
    int ntrk = 0, ltop = -1;
    bool bad = false;
#pragma unroll
    for (int l = 0; l < kLayers; ++l) {
        ids[l] = in.ids[l * n + i];
        const int j = ids[l];
        const bool have = j >= 0 && j < T.n;
        bad = bad || j >= T.n;
        ch[l] = have ? T.ch[j] : -1;
        ty[l] = have ? T.y[j] : 0.0f;
        tz[l] = have ? T.z[j] : 0.0f;
        tvy[l] = have ? T.vyy[j] : 0.0f;
        tvz[l] = have ? T.vzz[j] : 0.0f;
        tvyz[l] = have ? T.vyz[j] : 0.0f;
        tx[l] = have && T.x ? T.x[j] : 0.0f;
        if (j >= 0) {
            ++ntrk;
            ltop = l;
        }
    }
    const float alpha_in = in.alpha[i];
    TrackState s;
    s.x = {in.x[i], 0.0f};
    s.y = {in.par[0 * n + i], 0.0f};
    s.z = in.par[1 * n + i];
    s.f = in.par[2 * n + i];
    s.t = in.par[3 * n + i];
    s.k = in.par[4 * n + i];
#pragma unroll
    for (int k = 0; k < 15; ++k) s.c[k] = 0.0f;
#pragma unroll
    for (int l = 0; l < kLayers; ++l) bad = bad || (ids[l] >= 0 && (ch[l] < 0 || ch[l] >= kChambers));
    const bool skip = ntrk < 2 || (in.status[i] & TRD_ST_SEED_INVALID) || bad;

    float chi2 = 0.0f;
    int nupd = 0, status = TRD_RF_SKIPPED;
    df frame = {alpha_in, 0.0f};
    if (!skip) {
        // diagonal prior, widened
#pragma unroll
        for (int d = 0; d < 5; ++d) s.c[cidx(d, d)] = P.cov_scale * in.cov[cidx(d, d) * n + i];
        s.sector = sector_of_alpha(alpha_in);
        status = TRD_RF_OK;
#pragma unroll 1
        for (int l = ltop; l >= 0; --l) {
            // this layer's tracklet, selected without indexing the register
            // arrays by a runtime layer number
            int jl = -1, cl = 0;
            float yl = 0.0f, zl = 0.0f, vyl = 0.0f, vzl = 0.0f, vyzl = 0.0f, xtl = 0.0f;
#pragma unroll
            for (int q = 0; q < kLayers; ++q)
                if (q == l) {
                    jl = ids[q];
                    cl = ch[q];
                    yl = ty[q];
                    zl = tz[q];
                    vyl = tvy[q];
                    vzl = tvz[q];
                    vyzl = tvyz[q];
                    xtl = tx[q];
                }
            // a layer's plane: its tracklet's own radius when given (misalignment)
            const df xl = (jl >= 0 && T.x) ? df{xtl, 0.0f} : layer_x_df(l);
            if (!propagate(s, xl, P.bz)) { status = TRD_RF_PROP_FAIL; break; }
            int target = s.sector;
            if (jl >= 0)
                target = cl / (kStacks * kLayers);
            else if (fabsf(s.y.hi) > xl.hi * half_sector_tan())
                target = (s.sector + (s.y.hi > 0.0f ? 1 : -1) + kSectors) % kSectors;
            if (target != s.sector) {
                if (!enter_sector(s, frame, target, P.bz)) { status = TRD_RF_PROP_FAIL; break; }
                if (!propagate(s, xl, P.bz)) { status = TRD_RF_PROP_FAIL; break; }
            }
            if (jl >= 0) {
                float vyy = vyl;
                if (P.resmode) {
                    const float r = sqrtf((1.0f - s.f) * (1.0f + s.f));
                    const float u = s.f / r - lorentz_tan(P.bz);
                    vyy = kSigY0 * kSigY0 + kSigY1 * kSigY1 * u * u;
                }
                chi2 += kalman_update(s, layer_tilt_tan(l), yl, zl, vyy, vzl, vyzl);
                ++nupd;
            }
            if (P.material && !material<true>(s)) { status = TRD_RF_PROP_FAIL; break; }
        }
    }

    o.alpha[i] = df_to_f(frame);
    o.x[i] = df_to_f(s.x);
    o.par[0 * n + i] = df_to_f(s.y);
    o.par[1 * n + i] = s.z;
    o.par[2 * n + i] = s.f;
    o.par[3 * n + i] = s.t;
    o.par[4 * n + i] = s.k;
#pragma unroll
    for (int k = 0; k < 15; ++k) o.cov[k * n + i] = s.c[k];
    o.chi2[i] = chi2;
    o.nupd[i] = nupd;
    o.status[i] = status;
}

}  // namespace trd

namespace {
bool finite_positive(float v) { return isfinite(v) && v > 0.0f; }
}  // namespace

extern "C" int trd_refit(trd_ctx_t *ctx, const trd_results_t *tracks, int32_t n, const trd_tracklets_t *tracklets,
                         const trd_params_t *params, float cov_scale, trd_refit_t *out, void *stream)
{
    if (!ctx || !tracks || !tracklets || !params || !out || n < 0 || tracklets->n < 0) return TRD_EINVAL;
    if (!finite_positive(cov_scale) || !isfinite(params->bz)) return TRD_EINVAL;
    if (n == 0) return TRD_OK;
    if (!tracks->alpha || !tracks->x || !tracks->par || !tracks->cov || !tracks->status || !tracks->tracklet_id)
        return TRD_EINVAL;
    if (tracklets->n > 0 && (!tracklets->chamber || !tracklets->y || !tracklets->z || !tracklets->vyy ||
                             !tracklets->vzz || !tracklets->vyz))
        return TRD_EINVAL;
    if (!out->alpha || !out->x || !out->par || !out->cov || !out->chi2 || !out->n_upd || !out->status)
        return TRD_EINVAL;
    TRD_CUDA_TRY(cudaSetDevice(ctx->device));
    trd::RefitIn in{tracks->alpha, tracks->x, tracks->par, tracks->cov, tracks->status, tracks->tracklet_id, n};
    trd::TrackletSoA T{tracklets->chamber, tracklets->y, tracklets->z, tracklets->vyy, tracklets->vzz,
                       tracklets->vyz, tracklets->n, tracklets->x};
    trd::RefitParams P{params->bz, cov_scale, params->res_mode, params->material_on};
    trd::RefitOut o{out->alpha, out->x, out->par, out->cov, out->chi2, out->n_upd, out->status};
    const int threads = 128;
    const int blocks = (n + threads - 1) / threads;
    trd::k_refit<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(in, T, P, o);
    TRD_CUDA_TRY(cudaGetLastError());
    return TRD_OK;
}
