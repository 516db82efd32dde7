// residuals.cu -- residuals of distorted TPC clusters to the combined external
// refits, collected per TPC sub-volume, and the distortion vector of each
// sub-volume (arXiv:2003.03174, Sec. 2, steps 4 and 5).
//
// k_residuals: two lanes per track (one per refit).  The ITS refit (inside the TPC) and the
// TRD-only refit (outside) are carried along the track to every pad row that
// holds a cluster of that track.  Each refit is transported to the row plane
// (in one step from its state after the last rotation);
// where the cluster lies in another sector than the refit's frame, the refit
// is first transported to the plane in its old frame, rotated there into the
// cluster's sector and transported again, so every rotation happens next to
// the cluster.  The ITS refit goes outward, the TRD refit inward; to combine
// them at the same row without storing one side, the thread first carries the
// ITS refit outward to the track's last row (stopping only where the cluster
// sector changes, which are the only points where the path matters), then
// carries both inward together, row by row.  At each cluster the two (y, z)
// estimates are combined with their inverse 2x2 covariances, in residual
// space (cluster - estimate, small numbers) so FP32 keeps ~2e-5 cm; sin(phi)
// and tan(lambda) are combined with their inverse variances.  Eleven sums per
// sub-volume (n, t, u, t^2, u^2, dy, dz, t dy, u dz, dy^2, dz^2) are added as
// 64-bit fixed-point integers (2^-24 units): exact, order-independent sums.
//
// k_voxel_solve: one thread per sub-volume, the least-squares solution of
// dy_i = Dy - Dx t_i, dz_i = Dz - Dx u_i from the sums; the numerator and
// denominator of Dx are formed exactly in 128-bit integers.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "trd_device.cuh"
#include "trd_internal.h"
#include "track_model.cuh"

namespace trd {

constexpr int kRows = TRD_TPC_ROWS;
constexpr int kVoxY = TRD_VOX_Y_BINS;
constexpr int kVoxZ = TRD_VOX_Z_BINS;
constexpr int kVoxSums = TRD_VOX_SUMS;

struct RowTable {
    float x[kRows];
};

// pad-row centres, x_r = 85 + 160 (r + 1/2) / 152 cm, rounded to float at
// compile time (the device sees only the float values)
constexpr RowTable make_rows()
{
    RowTable t{};
    for (int r = 0; r < kRows; ++r) t.x[r] = static_cast<float>(85.0 + (r + 0.5) * 160.0 / kRows);
    return t;
}
__constant__ RowTable c_rows = make_rows();

struct StatesView {
    const float *alpha, *x, *par, *cov;
    const int32_t *status;
};

struct ClustersView {
    const float *y, *z;
    const int8_t *sector;
};

__device__ __forceinline__ void load_state(const StatesView &v, int n, int i, TrackState &s)
{
    s.x = {v.x[i], 0.0f};
    s.y = {v.par[0 * n + i], 0.0f};
    s.z = v.par[1 * n + i];
    s.f = v.par[2 * n + i];
    s.t = v.par[3 * n + i];
    s.k = v.par[4 * n + i];
#pragma unroll
    for (int k = 0; k < 15; ++k) s.c[k] = v.cov[k * n + i];
    s.sector = -1;
}

// A refit being carried along its track: the anchor is the state right after
// its last rotation (or as given), and every row is reached by one transport
// from the anchor, so FP32 rounding does not accumulate over the ~150 rows
// (a row-to-row chain would add ~1e-4 cm to z at 250 cm).  frame: the
// azimuth of the anchor's frame; anchor.sector = -1 until the first rotation.
struct Carrier {
    TrackState anchor;
    df frame;
};

// The refit at the row plane xr in the frame of sector sec, in w.  When sec
// is not the anchor's sector: transport to the plane in the old frame (if
// that fails, from where the anchor is), rotate into sec there (the rotated
// state becomes the new anchor), transport to the plane.  Returns false
// when the rotation or the final transport fails (the |sin(phi)| limit).
__device__ __forceinline__ bool carry(Carrier &c, int sec, df xr, float bz, TrackState &w)
{
    w = c.anchor;
    if (c.anchor.sector != sec) {
        (void)propagate(w, xr, bz);
        const df to = sector_alpha_df(sec);
        df d = df_add(to, df_neg(c.frame));
        if (d.hi > 3.14159265f) d = df_add(d, df{-kTwoPiHi, -kTwoPiLo});
        if (d.hi < -3.14159265f) d = df_add(d, df{kTwoPiHi, kTwoPiLo});
        if (!rotate(w, d, sec, bz)) return false;
        c.anchor = w;
        c.frame = to;
    }
    // the row's copy needs only the (y, z) block and the angle variances
    return propagate_t<false>(w, xr, bz);
}

// Sub-volume of a cluster, decided in FP32 with correctly rounded operations
// in the order written (no contraction), so that the decision is the same
// wherever it is evaluated.
__device__ __forceinline__ int voxel_of(float y, float z, int sec, int row, float xr)
{
    constexpr float T = hi_of(0.17632698070846498);  // tan 10 deg
    constexpr float ys = static_cast<float>(kVoxY) / (2.0f * T);
    const float u = __fdiv_rn(y, xr);
    const float v = __fadd_rn(u, T);
    const float fy = fminf(fmaxf(__fmul_rn(v, ys), -1.0f), static_cast<float>(kVoxY));  // bounded before the cast
    const int iy = min(max(static_cast<int>(floorf(fy)), 0), kVoxY - 1);
    const float w = __fdiv_rn(fabsf(z), xr);
    const float fz = fminf(__fmul_rn(w, static_cast<float>(kVoxZ)), static_cast<float>(kVoxZ));
    const int iz = min(max(static_cast<int>(floorf(fz)), 0), kVoxZ - 1);
    const int side = z < 0.0f ? 1 : 0;
    return (((side * kSectors + sec) * kRows + row) * kVoxY + iy) * kVoxZ + iz;
}

__device__ __forceinline__ long long fixed24(float v) { return __float2ll_rn(v * 16777216.0f); }

// Resident 128-thread blocks per SM the register budget is sized for: 7 (72
// registers, no spill) ran the 450k-track map 2.8 % faster than 6 (76
// registers); 8 (64 registers) spills and is slower.
#ifndef TRD_RESIDUALS_MIN_BLOCKS
#define TRD_RESIDUALS_MIN_BLOCKS 7
#endif

// Two lanes per track: the even lane carries the ITS refit, the odd lane the
// TRD refit.  Both lanes of a pair walk the same rows (their control flow is
// identical), exchange what the combination needs by shuffles, compute it
// the same way, and split the eleven atomics.
__global__ void __launch_bounds__(128, TRD_RESIDUALS_MIN_BLOCKS)
k_residuals(StatesView I, StatesView Tr, ClustersView cl, int n, float bz, unsigned long long *sums, float *res_out)
{
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = g >> 1;
    if (i >= n) return;  // pair-uniform
    const int role = g & 1;  // 0: ITS refit, 1: TRD refit
    const unsigned pmask = 3u << ((threadIdx.x & 31) & ~1);
    const size_t plane = static_cast<size_t>(kRows) * n;
    const float nan = __int_as_float(0x7fc00000);
    if (I.status[i] != 0 || Tr.status[i] != 0) {
        if (res_out)
            for (int r = 0; r < kRows; ++r)
#pragma unroll
                for (int k = 0; k < 2; ++k) res_out[(2 * role + k) * plane + static_cast<size_t>(r) * n + i] = nan;
        return;
    }
    const StatesView &V = role ? Tr : I;
    Carrier C;
    load_state(V, n, i, C.anchor);
    C.frame = {V.alpha[i], 0.0f};
    TrackState w;

    // the ITS refit outward (even lane): only where the cluster sector
    // changes does the path matter; both lanes find the last row
    int last = -1;
#pragma unroll 4
    for (int r = 0; r < kRows; ++r) {
        const size_t q = static_cast<size_t>(r) * n + i;
        const int s = cl.sector[q];
        if (s < 0 || s >= kSectors) continue;
        last = r;
        if (role == 0 && s != C.anchor.sector && isfinite(cl.y[q]) && isfinite(cl.z[q]))
            (void)carry(C, s, df{c_rows.x[r], 0.0f}, bz, w);
    }

    // both inward, row by row; the next row's cluster is loaded while this
    // row is computed
    int s_next = last >= 0 ? cl.sector[static_cast<size_t>(last) * n + i] : -1;
    float y_next = last >= 0 ? cl.y[static_cast<size_t>(last) * n + i] : 0.0f;
    float z_next = last >= 0 ? cl.z[static_cast<size_t>(last) * n + i] : 0.0f;
    if (res_out)
        for (int r = kRows - 1; r > last; --r)
#pragma unroll
            for (int k = 0; k < 2; ++k) res_out[(2 * role + k) * plane + static_cast<size_t>(r) * n + i] = nan;
#pragma unroll 1
    for (int r = last; r >= 0; --r) {
        const size_t q = static_cast<size_t>(r) * n + i;
        const int s = s_next;
        const float ycl = y_next, zcl = z_next;
        if (r > 0) {
            const size_t qn = q - n;
            s_next = cl.sector[qn];
            y_next = cl.y[qn];
            z_next = cl.z[qn];
        }
        float o0 = nan, o1 = nan;  // this lane's outputs: (dy, dz) or (t, u)
        if (s >= 0 && s < kSectors && isfinite(ycl) && isfinite(zcl)) {
            const df xr = {c_rows.x[r], 0.0f};
            const bool ok = carry(C, s, xr, bz, w);
            // this refit's share of the combination: V^-1, V^-1 (cluster - estimate),
            // and the inverse-variance weighted angles (y carried as a double-float)
            const float ry = __fsub_rn(ycl, w.y.hi) - w.y.lo, rz = zcl - w.z;
            const float d = 1.0f / (w.c[0] * w.c[2] - w.c[1] * w.c[1]);
            const float A00 = w.c[2] * d, A01 = -w.c[1] * d, A11 = w.c[0] * d;
            const float wf = 1.0f / w.c[5], wt = 1.0f / w.c[9];
            float v[9] = {A00, A01, A11, A00 * ry + A01 * rz, A01 * ry + A11 * rz, wf, w.f * wf, wt, w.t * wt};
            const int both = __shfl_xor_sync(pmask, static_cast<int>(ok), 1) & static_cast<int>(ok);
#pragma unroll
            for (int k = 0; k < 9; ++k) v[k] += __shfl_xor_sync(pmask, v[k], 1);
            if (both) {
                const float dw = 1.0f / (v[0] * v[2] - v[1] * v[1]);
                const float dy = (v[2] * v[3] - v[1] * v[4]) * dw;
                const float dz = (v[0] * v[4] - v[1] * v[3]) * dw;
                const float f = v[6] / v[5], tl = v[8] / v[7];
                const float ir = rsqrtf((1.0f - f) * (1.0f + f));
                const float t = f * ir, u = tl * ir;
                o0 = role ? t : dy;
                o1 = role ? u : dz;
                unsigned long long *S = sums + static_cast<size_t>(voxel_of(ycl, zcl, s, r, xr.hi)) * kVoxSums;
                if (role == 0) {
                    atomicAdd(S + 0, 1ull);
                    atomicAdd(S + 1, static_cast<unsigned long long>(fixed24(t)));
                    atomicAdd(S + 2, static_cast<unsigned long long>(fixed24(u)));
                    atomicAdd(S + 3, static_cast<unsigned long long>(fixed24(t * t)));
                    atomicAdd(S + 4, static_cast<unsigned long long>(fixed24(u * u)));
                    atomicAdd(S + 5, static_cast<unsigned long long>(fixed24(dy)));
                } else {
                    atomicAdd(S + 6, static_cast<unsigned long long>(fixed24(dz)));
                    atomicAdd(S + 7, static_cast<unsigned long long>(fixed24(t * dy)));
                    atomicAdd(S + 8, static_cast<unsigned long long>(fixed24(u * dz)));
                    atomicAdd(S + 9, static_cast<unsigned long long>(fixed24(dy * dy)));
                    atomicAdd(S + 10, static_cast<unsigned long long>(fixed24(dz * dz)));
                }
            }
        }
        if (res_out) {
            res_out[(2 * role + 0) * plane + q] = o0;
            res_out[(2 * role + 1) * plane + q] = o1;
        }
    }
}

// ---- the distortion vector of each sub-volume --------------------------------
__device__ __forceinline__ float i128_to_float(__int128 v)
{
    const bool neg = v < 0;
    const unsigned __int128 m = neg ? static_cast<unsigned __int128>(-v) : static_cast<unsigned __int128>(v);
    const float f = __ull2float_rn(static_cast<unsigned long long>(m >> 64)) * 18446744073709551616.0f +
                    __ull2float_rn(static_cast<unsigned long long>(m));
    return neg ? -f : f;
}

__global__ void __launch_bounds__(256) k_voxel_solve(const long long *sums, int nvox, int min_count, float *map)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nvox) return;
    const long long *S = sums + static_cast<size_t>(v) * kVoxSums;
    const long long n = S[0];
    float *o = map + static_cast<size_t>(v) * 6;
    const float nan = __int_as_float(0x7fc00000);
    float Dx = nan, Dy = nan, Dz = nan, ry = nan, rz = nan;
    if (n >= max(min_count, 1)) {
        const __int128 N = n;
        const __int128 two24 = static_cast<__int128>(1) << 24;
        // exact, in units of 2^-48: n (Stt + Suu) - St^2 - Su^2, and the
        // numerator of Dx; n Sdydy - Sdy^2, n Sdzdz - Sdz^2 for the spreads
        const __int128 den = N * (static_cast<__int128>(S[3]) + S[4]) * two24 -
                             static_cast<__int128>(S[1]) * S[1] - static_cast<__int128>(S[2]) * S[2];
        const __int128 num = N * (static_cast<__int128>(S[7]) + S[8]) * two24 -
                             static_cast<__int128>(S[1]) * S[5] - static_cast<__int128>(S[2]) * S[6];
        const __int128 vy = N * static_cast<__int128>(S[9]) * two24 - static_cast<__int128>(S[5]) * S[5];
        const __int128 vz = N * static_cast<__int128>(S[10]) * two24 - static_cast<__int128>(S[6]) * S[6];
        const float nf = static_cast<float>(n);
        const float inv48 = 1.0f / (16777216.0f * 16777216.0f);
        const float inv24 = 1.0f / 16777216.0f;
        ry = sqrtf(fmaxf(i128_to_float(vy) * inv48, 0.0f)) / nf;
        rz = sqrtf(fmaxf(i128_to_float(vz) * inv48, 0.0f)) / nf;
        const float denf = i128_to_float(den) * inv48;
        if (denf > 1e-12f * nf * nf) {
            Dx = -(i128_to_float(num) * inv48) / denf;
            Dy = (static_cast<float>(S[5]) * inv24 + static_cast<float>(S[1]) * inv24 * Dx) / nf;
            Dz = (static_cast<float>(S[6]) * inv24 + static_cast<float>(S[2]) * inv24 * Dx) / nf;
        }
    }
    o[0] = Dx;
    o[1] = Dy;
    o[2] = Dz;
    o[3] = static_cast<float>(n);
    o[4] = ry;
    o[5] = rz;
}

}  // namespace trd

extern "C" int trd_residuals(trd_ctx_t *ctx, int32_t n, const trd_states_t *its, const trd_states_t *trd_refit,
                             const trd_tpc_clusters_t *clusters, float bz, int64_t *voxel_sums, float *cluster_res,
                             void *stream)
{
    if (!ctx || !its || !trd_refit || !clusters || !voxel_sums || n < 0 || !isfinite(bz)) return TRD_EINVAL;
    if (n == 0) return TRD_OK;
    if (!its->alpha || !its->x || !its->par || !its->cov || !its->status || !trd_refit->alpha || !trd_refit->x ||
        !trd_refit->par || !trd_refit->cov || !trd_refit->status || !clusters->y || !clusters->z ||
        !clusters->sector)
        return TRD_EINVAL;
    if (static_cast<long long>(n) * TRD_TPC_ROWS > 0x7fffffffLL) return TRD_EINVAL;
    TRD_CUDA_TRY(cudaSetDevice(ctx->device));
    trd::StatesView I{its->alpha, its->x, its->par, its->cov, its->status};
    trd::StatesView T{trd_refit->alpha, trd_refit->x, trd_refit->par, trd_refit->cov, trd_refit->status};
    trd::ClustersView C{clusters->y, clusters->z, clusters->sector};
    const int threads = 128;  // 64 tracks, two lanes each
    const long long lanes = 2LL * n;
    trd::k_residuals<<<static_cast<int>((lanes + threads - 1) / threads), threads, 0,
                        static_cast<cudaStream_t>(stream)>>>(
        I, T, C, n, bz, reinterpret_cast<unsigned long long *>(voxel_sums), cluster_res);
    TRD_CUDA_TRY(cudaGetLastError());
    return TRD_OK;
}

extern "C" int trd_voxel_solve(trd_ctx_t *ctx, const int64_t *voxel_sums, int32_t min_count, float *map,
                               void *stream)
{
    if (!ctx || !voxel_sums || !map) return TRD_EINVAL;
    TRD_CUDA_TRY(cudaSetDevice(ctx->device));
    const int threads = 256;
    trd::k_voxel_solve<<<(TRD_N_VOXELS + threads - 1) / threads, threads, 0, static_cast<cudaStream_t>(stream)>>>(
        reinterpret_cast<const long long *>(voxel_sums), TRD_N_VOXELS, min_count, map);
    TRD_CUDA_TRY(cudaGetLastError());
    return TRD_OK;
}
