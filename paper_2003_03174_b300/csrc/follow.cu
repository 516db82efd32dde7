// follow.cu -- the FP32 TRD tracklet follower (arXiv:2003.03174, Sec. 3).
//
// One group of G lanes follows one seed; lane q holds hypothesis q (N <= G).
// Per layer every live lane transports its hypothesis to the layer plane,
// scans the index over the road and keeps its own best N extensions; the
// group then merges the lanes' lists with shuffles into the best N overall,
// and every lane adopts one winner (parent state by shuffle) and applies the
// Kalman update.  With N = 1 the group is a single thread per seed, which
// keeps 32x more seeds in flight than a warp per seed: the per-layer chain of
// dependent loads (road offsets, then records) is latency-bound, so memory
// parallelism comes from many independent seeds per SM.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "trd_device.cuh"
#include "trd_internal.h"
#include "track_model.cuh"

namespace trd {

struct Params {
    float bz, road, cut, pmiss, gate;
    int nhyp, maxmiss, resmode, material;
    // misalignment and field map (the EXT kernels only; Sec. 3): average
    // radius per chamber, Bz on a regular (r, z) grid, or null
    const float *chamber_x = nullptr;
    const float *bzmap = nullptr;
    int nr = 0, nz = 0;
    float r0 = 0.0f, ir = 0.0f, z0 = 0.0f, iz = 0.0f;  // grid origin and nodes per cm
};

// ---- field map --------------------------------------------------------------
// Bilinear between the nodes, the grid box clamps.  A transport step uses the
// field at its midpoint, estimated along the straight line from the start; a
// rotation the field at the state's point.  Without a map: the homogeneous bz.
__device__ __forceinline__ float field_at(const Params &P, float r, float z)
{
    const float fr = fminf(fmaxf((r - P.r0) * P.ir, 0.0f), static_cast<float>(P.nr - 1));
    const float fz = fminf(fmaxf((z - P.z0) * P.iz, 0.0f), static_cast<float>(P.nz - 1));
    const int i = min(static_cast<int>(fr), P.nr - 2), j = min(static_cast<int>(fz), P.nz - 2);
    const float wr = fr - static_cast<float>(i), wz = fz - static_cast<float>(j);
    const float *F = P.bzmap + j * P.nr + i;
    const float b00 = __ldg(F), b01 = __ldg(F + 1), b10 = __ldg(F + P.nr), b11 = __ldg(F + P.nr + 1);
    return (1.0f - wz) * ((1.0f - wr) * b00 + wr * b01) + wz * ((1.0f - wr) * b10 + wr * b11);
}

template <bool EXT>
__device__ __forceinline__ float point_bz(const Params &P, const TrackState &s)
{
    if (!EXT || !P.bzmap) return P.bz;
    return field_at(P, hypotf(s.x.hi, s.y.hi), s.z);
}

template <bool EXT>
__device__ __forceinline__ float step_bz(const Params &P, const TrackState &s, df x1)
{
    if (!EXT || !P.bzmap) return P.bz;
    const float f = s.f;
    if (!(fabsf(f) < 1.0f)) return point_bz<EXT>(P, s);
    const float ir = rsqrtf((1.0f - f) * (1.0f + f));
    const float h = 0.5f * df_to_f(df_add(x1, df_neg(s.x)));
    return field_at(P, hypotf(s.x.hi + h, s.y.hi + h * f * ir), s.z + h * s.t * ir);
}

struct SeedsView {
    const float *alpha, *x, *y, *z, *snp, *tgl, *q2pt, *cov;
    int n;
    const int32_t *soff;  // [n_tf + 1] seed offsets of a batch of timeframes, or null
    int n_tf;
    const int32_t *trig;  // interaction id per seed, or null
};

struct ResultsView {
    float *alpha, *x, *par, *cov, *chi2;
    int32_t *ntrk, *nmiss, *status, *ids;
};

// Carry a hypothesis to the plane of layer l; returns false if it is lost.
// chamber = -1 when z is outside the 5 stacks.
// With EXT, the steps use the field map and a hypothesis in a chamber moves on
// to the chamber's average radius (misalignment, Sec. 3).
template <bool EXT>
__device__ bool to_layer(TrackState &s, int l, const Params &P, int &chamber)
{
    const df xl = layer_x_df(l);
    if (!propagate(s, xl, step_bz<EXT>(P, s, xl))) return false;
    const float lim = xl.hi * half_sector_tan();
    if (fabsf(s.y.hi) > lim) {
        const int dir = s.y.hi > 0.0f ? 1 : -1;
        const int ns = (s.sector + dir + kSectors) % kSectors;
        const df d = dir > 0 ? df{kSectorWidthHi, kSectorWidthLo} : df{-kSectorWidthHi, -kSectorWidthLo};
        if (!rotate(s, d, ns, point_bz<EXT>(P, s))) return false;
        if (!propagate(s, xl, step_bz<EXT>(P, s, xl))) return false;
    }
    if (P.material && !material<false>(s)) return false;
    const float u = (s.z - kZMin) * (1.0f / kStackLength);
    if (u >= 0.0f && u < static_cast<float>(kStacks)) {
        const int stack = static_cast<int>(u);
        chamber = s.sector * (kStacks * kLayers) + stack * kLayers + l;
        if (EXT && P.chamber_x) {
            const float xc = __ldg(&P.chamber_x[chamber]);
            if (!(xc == xl.hi && xl.lo == 0.0f)) {
                const df xcd = {xc, 0.0f};
                if (!propagate(s, xcd, step_bz<EXT>(P, s, xcd))) return false;
            }
        }
    } else {
        chamber = -1;
    }
    return true;
}

// ---- small sorted extension list (per lane) ---------------------------------
template <int NH>
struct ExtList {
    // extensions kept in the selection order (score, parent rank, tracklet
    // id; a missing layer has id kMissing and sorts after tracklets)
    float score[NH];
    float chi2[NH];
    int par[NH];
    int id[NH];
    int pos[NH];
    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int k = 0; k < NH; ++k) {
            score[k] = INFINITY;
            chi2[k] = 0.0f;
            par[k] = 0x7fffffff;
            id[k] = kMissing;
            pos[k] = -1;
        }
    }
    __device__ __forceinline__ static bool less(float sa, int pa, int ia, float sb, int pb, int ib)
    {
        return sa < sb || (sa == sb && (pa < pb || (pa == pb && ia < ib)));
    }
    __device__ __forceinline__ void insert(float sc, int parent, int tid, int p, float c2)
    {
        if (!less(sc, parent, tid, score[NH - 1], par[NH - 1], id[NH - 1])) return;
        // shift larger entries up, then place (unrolled, stays in registers)
        bool placed = false;
#pragma unroll
        for (int k = NH - 1; k >= 0; --k) {
            if (placed) continue;
            const bool move = k > 0 && less(sc, parent, tid, score[k - 1], par[k - 1], id[k - 1]);
            if (move) {
                score[k] = score[k - 1];
                chi2[k] = chi2[k - 1];
                par[k] = par[k - 1];
                id[k] = id[k - 1];
                pos[k] = pos[k - 1];
            } else {
                score[k] = sc;
                chi2[k] = c2;
                par[k] = parent;
                id[k] = tid;
                pos[k] = p;
                placed = true;
            }
        }
    }
    __device__ __forceinline__ void pop()
    {
#pragma unroll
        for (int k = 0; k + 1 < NH; ++k) {
            score[k] = score[k + 1];
            chi2[k] = chi2[k + 1];
            par[k] = par[k + 1];
            id[k] = id[k + 1];
            pos[k] = pos[k + 1];
        }
        score[NH - 1] = INFINITY;
        par[NH - 1] = 0x7fffffff;
        id[NH - 1] = kMissing;
        pos[NH - 1] = -1;
    }
};

// Road query + candidate tests for one hypothesis at layer l (Sec. 3).
// The road bounds z_tl to z +- Rz (pad rows r_lo..r_hi) and the measured y to
// y +- (W + |tan tau| Rz) (y bins b_lo..b_hi); each y bin is one contiguous
// range of the index over those rows.  The candidates of the first two bins
// form one list: their {y, z} are read eight at a time (one dependent L2
// round trip, which also brings each 32-byte record into L1), a bit mask
// keeps those inside the road's y/z bounds, and only those get the full test
// (record read again from L1).  More than two bins (very wide roads) are
// handled the same way, two at a time.
// Road geometry of a hypothesis for the EXT kernels: its radius and the
// straight-line slopes dy/dx = tan(phi), dz/dx = tan(lambda)/cos(phi).
struct LinExt {
    float xh, xl, fr, tr;
};

template <int NH, bool EXT>
__device__ __forceinline__ void full_test(int pos, const IndexView &ix, float tt, float z, float yh, float yl,
                                          float n2, float syy_trk, float syz_trk, float c11, float vyy_res,
                                          int resmode, float dy_pred, float gate, float cut, float score,
                                          int parent, int trig, const LinExt &e, ExtList<NH> &L)
{
    const float4 a = __ldg(&ix.rec[2 * pos]);
    const float4 v = __ldg(&ix.rec[2 * pos + 1]);
    // per-interaction association (Sec. 4): other interactions' tracklets are not candidates
    const int ttrig = __float_as_int(v.w);
    if (trig >= 0 && ttrig >= 0 && ttrig != trig) return;
    if (EXT && ix.recx) {
        // a tracklet at its own radius (misalignment, Sec. 3): the fast linear
        // extrapolation of the hypothesis to it, covariance as at the chamber
        const float dx = __fsub_rn(__ldg(&ix.recx[pos]), e.xh) - e.xl;
        const df yy = df_add_f(df{yh, yl}, dx * e.fr);
        yh = yy.hi;
        yl = yy.lo;
        z = fmaf(dx, e.tr, z);
    }
    const float ry = (__fsub_rn(a.x, yh) - yl) + tt * (z - a.y);
    const float rz = a.y - z;
    const float vyy = resmode ? vyy_res : v.x;
    const float S00 = syy_trk + vyy;
    const float S01 = syz_trk + v.z;
    const float S11 = c11 + v.y;
    if (ry * ry > n2 * S00 || rz * rz > n2 * S11) return;
    if (fabsf(a.z - dy_pred) > gate) return;
    const float chi2 = (S11 * ry * ry - 2.0f * S01 * ry * rz + S00 * rz * rz) / (S00 * S11 - S01 * S01);
    if (!(chi2 < cut)) return;
    L.insert(score + chi2, parent, __float_as_int(a.w), pos, chi2);
}

template <int NH, bool EXT>
__device__ void scan_candidates(const TrackState &s, int l, int chamber, int cbase, float score, const Params &P,
                                const IndexView &ix, float vyy_max_in, float vzz_max, float dx_max, int trig,
                                ExtList<NH> &L)
{
    const float tt = layer_tilt_tan(l);
    const float f = s.f;
    const float r = sqrtf((1.0f - f) * (1.0f + f));
    const float uu = f / r - lorentz_tan(P.bz);
    const float vyy_res = kSigY0 * kSigY0 + kSigY1 * kSigY1 * uu * uu;
    const float vyy_max = P.resmode ? vyy_res : vyy_max_in;
    const float c10 = s.c[1], c11 = s.c[2];
    const float syy_trk = s.c[0] - 2.0f * tt * c10 + tt * tt * c11;
    const float syz_trk = c10 - tt * c11;
    const float n2 = P.road * P.road;
    float W = P.road * sqrtf(fmaxf(syy_trk + vyy_max, 0.0f)) * 1.0001f + 1e-4f;
    float Rz = P.road * sqrtf(fmaxf(c11 + vzz_max, 0.0f)) * 1.0001f + 1e-4f;
    LinExt e{s.x.hi, s.x.lo, 0.0f, 0.0f};
    if (EXT && ix.recx) {
        // tracklets up to dxb from this radius: the window holds their roads
        e.fr = f / r;
        e.tr = s.t / r;
        const float dxb = dx_max + fabsf(df_to_f(df_add(s.x, df_neg(layer_x_df(l))))) + 1e-4f;
        W += dxb * fabsf(e.fr) * 1.0001f;
        Rz += dxb * fabsf(e.tr) * 1.0001f;
    }
    const float dy_pred = kDriftLength * uu;
    const float gate = P.gate * sqrtf(kSigDy0 * kSigDy0 + kSigDy1 * kSigDy1 * uu * uu);
    const float z = s.z;
    const float yh = s.y.hi, yl = s.y.lo;
    const float zlo = stack_z_lo(stack_of_chamber(chamber));
    const int r_lo = row_of_z(z - Rz, zlo), r_hi = row_of_z(z + Rz, zlo);
    const float half = W + fabsf(tt) * Rz + 1e-3f + 1e-6f * fabsf(yh);
    const int b_lo = ybin_of(yh - half, ix.inv_w, ix.nb), b_hi = ybin_of(yh + half, ix.inv_w, ix.nb);
    const float2 *yz = reinterpret_cast<const float2 *>(ix.rec);  // {y, z} of record p at yz[4 p]
    for (int b = b_lo; b <= b_hi; b += 2) {
        const int base = bucket_of(cbase + chamber, b, 0, ix.nb);
        const bool two = b + 1 <= b_hi;
        const int beg0 = __ldg(&ix.offsets[base + r_lo]);
        const int end0 = __ldg(&ix.offsets[base + r_hi + 1]);
        int beg1 = 0, end1 = 0;
        if (two) {
            beg1 = __ldg(&ix.offsets[base + kRowsPerStack + r_lo]);
            end1 = __ldg(&ix.offsets[base + kRowsPerStack + r_hi + 1]);
        }
        const int n0 = end0 - beg0;
        const int n = n0 + (end1 - beg1);
#pragma unroll 1
        for (int j0 = 0; j0 < n; j0 += 8) {
            float2 c[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u;
                const int pos = j < n0 ? beg0 + j : beg1 + (j - n0);
                c[u] = j < n ? __ldg(&yz[4 * pos]) : make_float2(INFINITY, INFINITY);
            }
            unsigned mask = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const float ry = (__fsub_rn(c[u].x, yh) - yl) + tt * (z - c[u].y);
                const float rz = c[u].y - z;
                if (fabsf(ry) <= W && fabsf(rz) <= Rz) mask |= 1u << u;
            }
            while (mask) {
                const int u = __ffs(mask) - 1;
                mask &= mask - 1u;
                const int j = j0 + u;
                const int pos = j < n0 ? beg0 + j : beg1 + (j - n0);
                full_test<NH, EXT>(pos, ix, tt, z, yh, yl, n2, syy_trk, syz_trk, c11, vyy_res, P.resmode, dy_pred,
                                   gate, P.cut, score, 0, trig, e, L);
            }
        }
    }
}

// Group scan (N > 1): the lanes of a seed's group take its hypotheses one at
// a time and share each one's road: the road is broadcast from the lane that
// holds the hypothesis, lane q tests candidates q, q + G, ... (eight at a
// time), and every extension records its parent.  The candidate set, the
// arithmetic and the selection order are those of one lane scanning its own
// hypothesis; the work is spread evenly over the group.
template <int G, int NH, bool EXT>
__device__ void scan_group(bool mine, const TrackState &s, int l, int chamber, int cbase, float score,
                           const Params &P, const IndexView &ix, float vyy_max_in, float vzz_max, float dx_max,
                           unsigned gmask, int q, int trig, ExtList<NH> &L)
{
    const float tt = layer_tilt_tan(l);
    // this lane's own road (used when it is broadcast)
    float z = 0, yh = 0, yl = 0, W = 0, Rz = 0, syy = 0, syz = 0, c11 = 0, vres = 0, dyp = 0, gate = 0;
    int r_lo = 0, r_hi = 0, b_lo = 0, b_hi = -1, base_ch = 0;
    LinExt e{s.x.hi, s.x.lo, 0.0f, 0.0f};
    if (mine) {
        const float f = s.f;
        const float r = sqrtf((1.0f - f) * (1.0f + f));
        const float uu = f / r - lorentz_tan(P.bz);
        vres = kSigY0 * kSigY0 + kSigY1 * kSigY1 * uu * uu;
        const float vyy_max = P.resmode ? vres : vyy_max_in;
        const float c10 = s.c[1];
        c11 = s.c[2];
        syy = s.c[0] - 2.0f * tt * c10 + tt * tt * c11;
        syz = c10 - tt * c11;
        W = P.road * sqrtf(fmaxf(syy + vyy_max, 0.0f)) * 1.0001f + 1e-4f;
        Rz = P.road * sqrtf(fmaxf(c11 + vzz_max, 0.0f)) * 1.0001f + 1e-4f;
        if (EXT && ix.recx) {
            e.fr = f / r;
            e.tr = s.t / r;
            const float dxb = dx_max + fabsf(df_to_f(df_add(s.x, df_neg(layer_x_df(l))))) + 1e-4f;
            W += dxb * fabsf(e.fr) * 1.0001f;
            Rz += dxb * fabsf(e.tr) * 1.0001f;
        }
        dyp = kDriftLength * uu;
        gate = P.gate * sqrtf(kSigDy0 * kSigDy0 + kSigDy1 * kSigDy1 * uu * uu);
        z = s.z;
        yh = s.y.hi;
        yl = s.y.lo;
        const float zlo = stack_z_lo(stack_of_chamber(chamber));
        r_lo = row_of_z(z - Rz, zlo);
        r_hi = row_of_z(z + Rz, zlo);
        const float half = W + fabsf(tt) * Rz + 1e-3f + 1e-6f * fabsf(yh);
        b_lo = ybin_of(yh - half, ix.inv_w, ix.nb);
        b_hi = ybin_of(yh + half, ix.inv_w, ix.nb);
        base_ch = bucket_of(cbase + chamber, 0, 0, ix.nb);
    }
    const float n2 = P.road * P.road;
    const float2 *yzs = reinterpret_cast<const float2 *>(ix.rec);
    for (int h = 0; h < NH; ++h) {  // hypotheses live in lanes 0..NH-1
        if (!__shfl_sync(gmask, static_cast<int>(mine), h, G)) continue;
        const float hz = __shfl_sync(gmask, z, h, G), hyh = __shfl_sync(gmask, yh, h, G);
        const float hyl = __shfl_sync(gmask, yl, h, G), hW = __shfl_sync(gmask, W, h, G);
        const float hRz = __shfl_sync(gmask, Rz, h, G), hsyy = __shfl_sync(gmask, syy, h, G);
        const float hsyz = __shfl_sync(gmask, syz, h, G), hc11 = __shfl_sync(gmask, c11, h, G);
        const float hvres = __shfl_sync(gmask, vres, h, G), hdyp = __shfl_sync(gmask, dyp, h, G);
        const float hgate = __shfl_sync(gmask, gate, h, G), hscore = __shfl_sync(gmask, score, h, G);
        const int hr_lo = __shfl_sync(gmask, r_lo, h, G), hr_hi = __shfl_sync(gmask, r_hi, h, G);
        const int hb_lo = __shfl_sync(gmask, b_lo, h, G), hb_hi = __shfl_sync(gmask, b_hi, h, G);
        const int hbase = __shfl_sync(gmask, base_ch, h, G);
        LinExt he{};
        if (EXT) {
            he.xh = __shfl_sync(gmask, e.xh, h, G);
            he.xl = __shfl_sync(gmask, e.xl, h, G);
            he.fr = __shfl_sync(gmask, e.fr, h, G);
            he.tr = __shfl_sync(gmask, e.tr, h, G);
        }
        for (int b = hb_lo; b <= hb_hi; b += 2) {
            const int base = hbase + b * kRowsPerStack;
            const int beg0 = __ldg(&ix.offsets[base + hr_lo]);
            const int end0 = __ldg(&ix.offsets[base + hr_hi + 1]);
            int beg1 = 0, end1 = 0;
            if (b + 1 <= hb_hi) {
                beg1 = __ldg(&ix.offsets[base + kRowsPerStack + hr_lo]);
                end1 = __ldg(&ix.offsets[base + kRowsPerStack + hr_hi + 1]);
            }
            const int n0 = end0 - beg0;
            const int n = n0 + (end1 - beg1);
            // lane q takes candidates q, q + G, ...: ceil(n / G) of them, four at a time
            const int per_lane = (n + G - 1) / G;
            for (int u0 = 0; u0 < per_lane; u0 += 4) {
                float2 c[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = q + G * (u0 + u);
                    const int pos = j < n0 ? beg0 + j : beg1 + (j - n0);
                    c[u] = j < n ? __ldg(&yzs[4 * pos]) : make_float2(INFINITY, INFINITY);
                }
                unsigned mask = 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float ry = (__fsub_rn(c[u].x, hyh) - hyl) + tt * (hz - c[u].y);
                    const float rz = c[u].y - hz;
                    if (fabsf(ry) <= hW && fabsf(rz) <= hRz) mask |= 1u << u;
                }
                while (mask) {
                    const int u = __ffs(mask) - 1;
                    mask &= mask - 1u;
                    const int j = q + G * (u0 + u);
                    const int pos = j < n0 ? beg0 + j : beg1 + (j - n0);
                    full_test<NH, EXT>(pos, ix, tt, hz, hyh, hyl, n2, hsyy, hsyz, hc11, hvres, P.resmode, hdyp,
                                       hgate, P.cut, hscore, h, trig, he, L);
                }
            }
        }
    }
}

struct Snapshot {  // pre-transport copy of lane 0's state, in shared memory
    float v[24];
};

__device__ __forceinline__ void save_state(float *sm, int stride, const TrackState &s)
{
    sm[0 * stride] = s.x.hi;
    sm[1 * stride] = s.x.lo;
    sm[2 * stride] = s.y.hi;
    sm[3 * stride] = s.y.lo;
    sm[4 * stride] = s.z;
    sm[5 * stride] = s.f;
    sm[6 * stride] = s.t;
    sm[7 * stride] = s.k;
#pragma unroll
    for (int k = 0; k < 15; ++k) sm[(8 + k) * stride] = s.c[k];
    sm[23 * stride] = __int_as_float(s.sector);
}

__device__ __forceinline__ void load_state(const float *sm, int stride, TrackState &s)
{
    s.x = {sm[0 * stride], sm[1 * stride]};
    s.y = {sm[2 * stride], sm[3 * stride]};
    s.z = sm[4 * stride];
    s.f = sm[5 * stride];
    s.t = sm[6 * stride];
    s.k = sm[7 * stride];
#pragma unroll
    for (int k = 0; k < 15; ++k) s.c[k] = sm[(8 + k) * stride];
    s.sector = __float_as_int(sm[23 * stride]);
}

__device__ __forceinline__ bool cov_pd(const float *c)
{
    // Cholesky of the 5x5 (seed validity), without early exits: every pivot
    // is computed and the matrix is positive definite when all are > 0.
    float L[15];
    bool pd = true;
#pragma unroll
    for (int j = 0; j < 5; ++j) {
        float d = c[cidx(j, j)];
#pragma unroll
        for (int k = 0; k < j; ++k) d -= L[cidx(j, k)] * L[cidx(j, k)];
        pd = pd && d > 0.0f;
        const float inv = rsqrtf(fmaxf(d, 1e-30f));
        L[cidx(j, j)] = d * inv;
#pragma unroll
        for (int i = j + 1; i < 5; ++i) {
            float x = c[cidx(i, j)];
#pragma unroll
            for (int k = 0; k < j; ++k) x -= L[cidx(i, k)] * L[cidx(j, k)];
            L[cidx(i, j)] = x * inv;
        }
    }
    return pd;
}

__device__ __forceinline__ void write_result(const ResultsView &o, int n, int i, const TrackState &s, float chi2,
                                             int ntrk, int nmiss, int status, const int (&ids)[kLayers])
{
    o.alpha[i] = sector_alpha_df(s.sector).hi;
    o.x[i] = df_to_f(s.x);
    o.par[0 * n + i] = df_to_f(s.y);
    o.par[1 * n + i] = s.z;
    o.par[2 * n + i] = s.f;
    o.par[3 * n + i] = s.t;
    o.par[4 * n + i] = s.k;
#pragma unroll
    for (int k = 0; k < 15; ++k) o.cov[k * n + i] = s.c[k];
    o.chi2[i] = chi2;
    o.ntrk[i] = ntrk;
    o.nmiss[i] = nmiss;
    o.status[i] = status;
#pragma unroll
    for (int l = 0; l < kLayers; ++l) o.ids[l * n + i] = ids[l];
}

__device__ __forceinline__ void write_seed_result(const ResultsView &o, const SeedsView &sv, int n, int i,
                                                  int status)
{
    o.alpha[i] = sv.alpha[i];
    o.x[i] = sv.x[i];
    o.par[0 * n + i] = sv.y[i];
    o.par[1 * n + i] = sv.z[i];
    o.par[2 * n + i] = sv.snp[i];
    o.par[3 * n + i] = sv.tgl[i];
    o.par[4 * n + i] = sv.q2pt[i];
#pragma unroll
    for (int k = 0; k < 15; ++k) o.cov[k * n + i] = sv.cov[k * n + i];
    o.chi2[i] = 0.0f;
    o.ntrk[i] = 0;
    o.nmiss[i] = 0;
    o.status[i] = status;
#pragma unroll
    for (int l = 0; l < kLayers; ++l) o.ids[l * n + i] = -1;
}

template <int G>
__device__ __forceinline__ float gshfl(unsigned mask, float v, int src)
{
    return G == 1 ? v : __shfl_sync(mask, v, src, G);
}
template <int G>
__device__ __forceinline__ int gshfl(unsigned mask, int v, int src)
{
    return G == 1 ? v : __shfl_sync(mask, v, src, G);
}

// Next seed for this group from the launch's work counter.  G == 1: the lanes
// that ask together share one atomicAdd (warp-aggregated).
template <int G>
__device__ __forceinline__ int fetch_seed(int *counter, unsigned gmask, int q)
{
    if (G == 1) {
        const unsigned mask = __activemask();
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(mask) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(counter, __popc(mask));
        base = __shfl_sync(mask, base, leader);
        return base + __popc(mask & ((1u << lane) - 1u));
    } else {
        int t = 0;
        if (q == 0) t = atomicAdd(counter, 1);
        return __shfl_sync(gmask, t, 0, G);
    }
}

// Per-seed registers of one lane (hypothesis q of its group).
struct Lane {
    TrackState s;
    float score, chisum;
    int ntrk, nmiss;
    int cbase;  // first chamber of the seed's timeframe in the index (timeframe * 540)
    int trig;   // the seed's interaction id (-1: no association)
    int ids[kLayers];
    bool alive;
};

// Seed preparation, one thread per seed (all seeds take the same path, so
// this runs without divergence): load the seed, validate it, rotate it into
// the sector of its position.  A seed that ends here gets its final result;
// a live seed's rotated state is parked in its own result slots (which the
// follower overwrites at the end) with status -1:
//   alpha <- sector, x <- x.hi, chi2 <- x.lo, par <- (y.hi, z, snp, tgl, q2pt),
//   cov <- cov, n_miss <- bits of y.lo.
__global__ void __launch_bounds__(256) k_seed_prepare(SeedsView sv, Params P, ResultsView o)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sv.n;
    if (i >= n) return;
    TrackState s;
    const float alpha = sv.alpha[i];
    const float sx = sv.x[i], sy = sv.y[i];
    s.x = {sx, 0.0f};
    s.y = {sy, 0.0f};
    s.z = sv.z[i];
    s.f = sv.snp[i];
    s.t = sv.tgl[i];
    s.k = sv.q2pt[i];
#pragma unroll
    for (int k = 0; k < 15; ++k) s.c[k] = sv.cov[k * n + i];
    if (!(fabsf(s.f) < kMaxSnp) || !cov_pd(s.c)) {
        write_seed_result(o, sv, n, i, TRD_ST_SEED_INVALID);
        return;
    }
    const float phi = alpha + atan2f(sy, sx);
    float u = phi - kTwoPiHi * floorf(phi * (1.0f / kTwoPiHi));
    int sec = static_cast<int>(u * (1.0f / kSectorWidthHi));
    sec = min(max(sec, 0), kSectors - 1);
    df d = df_add_f(sector_alpha_df(sec), -alpha);
    if (d.hi > 3.14159265f) d = df_add(d, df{-kTwoPiHi, -kTwoPiLo});
    if (d.hi < -3.14159265f) d = df_add(d, df{kTwoPiHi, kTwoPiLo});
    s.sector = sec;
    if (!rotate(s, d, sec, P.bzmap ? field_at(P, hypotf(sx, sy), s.z) : P.bz)) {
        write_seed_result(o, sv, n, i, TRD_ST_PROP_FAIL);
        return;
    }
    o.alpha[i] = static_cast<float>(sec);
    o.x[i] = s.x.hi;
    o.chi2[i] = s.x.lo;
    o.par[0 * n + i] = s.y.hi;
    o.par[1 * n + i] = s.z;
    o.par[2 * n + i] = s.f;
    o.par[3 * n + i] = s.t;
    o.par[4 * n + i] = s.k;
#pragma unroll
    for (int k = 0; k < 15; ++k) o.cov[k * n + i] = s.c[k];
    o.nmiss[i] = __float_as_int(s.y.lo);
    o.status[i] = -1;
}

// Pick up seed i as prepared by k_seed_prepare.  Returns false when the seed
// already has its final result.
template <int G>
__device__ __forceinline__ bool start_seed(int i, int q, const SeedsView &sv, const ResultsView &o, Lane &L)
{
    const int n = sv.n;
    if (o.status[i] != -1) return false;
    TrackState &s = L.s;
    s.sector = static_cast<int>(o.alpha[i]);
    s.x = {o.x[i], o.chi2[i]};
    s.y = {o.par[0 * n + i], __int_as_float(o.nmiss[i])};
    s.z = o.par[1 * n + i];
    s.f = o.par[2 * n + i];
    s.t = o.par[3 * n + i];
    s.k = o.par[4 * n + i];
#pragma unroll
    for (int k = 0; k < 15; ++k) s.c[k] = o.cov[k * n + i];
    L.cbase = tf_of(i, sv.soff, sv.n_tf) * kChambers;
    L.trig = sv.trig ? sv.trig[i] : -1;
    L.alive = q == 0;
    L.score = 0.0f;
    L.chisum = 0.0f;
    L.ntrk = 0;
    L.nmiss = 0;
#pragma unroll
    for (int k = 0; k < kLayers; ++k) L.ids[k] = -1;
    return true;
}

// One layer of seed i for the group.  Returns true when the seed is finished
// (result written).
template <int G, int NH, bool EXT>
__device__ __forceinline__ bool layer_step(int i, int l, int q, unsigned gmask, const IndexView &ix, const Params &P,
                                           const ResultsView &o, int n, float *sm, int stride, float vyy_max,
                                           float vzz_max, float dx_max, Lane &H)
{
    TrackState &s = H.s;
    if (q == 0) save_state(sm, stride, s);
    int chamber = -1;
    const bool live = H.alive && to_layer<EXT>(s, l, P, chamber);
    ExtList<NH> L;
    L.clear();
    if (G == 1) {
        if (live && chamber >= 0)
            scan_candidates<NH, EXT>(s, l, chamber, H.cbase, H.score, P, ix, vyy_max, vzz_max, dx_max, H.trig, L);
    } else {
        scan_group<G, NH, EXT>(live && chamber >= 0, s, l, chamber, H.cbase, H.score, P, ix, vyy_max, vzz_max,
                               dx_max, gmask, q, H.trig, L);
    }
    if (live && H.nmiss < P.maxmiss) L.insert(H.score + P.pmiss, q, kMissing, -1, 0.0f);

    // merge the lanes' lists: the k-th best extension goes to lane k
    int my_parent = q, my_id = kMissing, my_pos = -1;
    float my_score = INFINITY, my_chi2 = 0.0f;
    int kept = 0;
    if (G == 1) {
        if (L.score[0] < INFINITY) {
            my_score = L.score[0];
            my_id = L.id[0];
            my_pos = L.pos[0];
            my_chi2 = L.chi2[0];
            kept = 1;
        }
    } else {
        for (int rr = 0; rr < P.nhyp; ++rr) {
            // group minimum of the lanes' heads in (score, parent, id) order;
            // bh is the lane holding it
            float bs = L.score[0];
            int bp = L.par[0], bid = L.id[0], bh = q;
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                const float os = __shfl_xor_sync(gmask, bs, off, G);
                const int op = __shfl_xor_sync(gmask, bp, off, G);
                const int oid = __shfl_xor_sync(gmask, bid, off, G);
                const int oh = __shfl_xor_sync(gmask, bh, off, G);
                if (ExtList<NH>::less(os, op, oid, bs, bp, bid)) {
                    bs = os;
                    bp = op;
                    bid = oid;
                    bh = oh;
                }
            }
            if (!(bs < INFINITY)) break;
            const float wchi2 = __shfl_sync(gmask, L.chi2[0], bh, G);
            const int wpos = __shfl_sync(gmask, L.pos[0], bh, G);
            if (q == rr) {
                my_parent = bp;
                my_id = bid;
                my_pos = wpos;
                my_score = bs;
                my_chi2 = wchi2;
            }
            if (q == bh) L.pop();
            kept = rr + 1;
        }
    }
    if (kept == 0) {
        // no extension for any hypothesis: the seed ends with the best
        // hypothesis as it was after the previous layer
        const bool any_live = G == 1 ? live : (__any_sync(gmask, live) != 0);
        if (q == 0) {
            TrackState b;
            load_state(sm, stride, b);
            write_result(o, n, i, b, H.chisum, H.ntrk, H.nmiss, any_live ? TRD_ST_STOPPED : TRD_ST_PROP_FAIL, H.ids);
        }
        return true;
    }
    if (G > 1) {  // adopt the parent's transported state
        const int src = my_parent;
        s.x.hi = gshfl<G>(gmask, s.x.hi, src);
        s.x.lo = gshfl<G>(gmask, s.x.lo, src);
        s.y.hi = gshfl<G>(gmask, s.y.hi, src);
        s.y.lo = gshfl<G>(gmask, s.y.lo, src);
        s.z = gshfl<G>(gmask, s.z, src);
        s.f = gshfl<G>(gmask, s.f, src);
        s.t = gshfl<G>(gmask, s.t, src);
        s.k = gshfl<G>(gmask, s.k, src);
#pragma unroll
        for (int k = 0; k < 15; ++k) s.c[k] = gshfl<G>(gmask, s.c[k], src);
        s.sector = gshfl<G>(gmask, s.sector, src);
        H.chisum = gshfl<G>(gmask, H.chisum, src);
        H.ntrk = gshfl<G>(gmask, H.ntrk, src);
        H.nmiss = gshfl<G>(gmask, H.nmiss, src);
#pragma unroll
        for (int k = 0; k < kLayers; ++k) H.ids[k] = gshfl<G>(gmask, H.ids[k], src);
    }
    H.alive = q < kept;
    if (H.alive) {
        H.score = my_score;
        int idl = -1;
        if (my_id != kMissing) {
            const float4 a = __ldg(&ix.rec[2 * my_pos]);
            const float4 v = __ldg(&ix.rec[2 * my_pos + 1]);
            if (EXT && ix.recx) {
                // the precise transport to the matched tracklet's own radius
                // before the update (a failed transport leaves the state)
                const df xt = {__ldg(&ix.recx[my_pos]), 0.0f};
                (void)propagate(s, xt, step_bz<EXT>(P, s, xt));
            }
            float vyy = v.x;
            if (P.resmode) {
                const float r = sqrtf((1.0f - s.f) * (1.0f + s.f));
                const float uu = s.f / r - lorentz_tan(P.bz);
                vyy = kSigY0 * kSigY0 + kSigY1 * kSigY1 * uu * uu;
            }
            kalman_update(s, layer_tilt_tan(l), a.x, a.y, vyy, v.y, v.z);
            idl = my_id;
            H.ntrk += 1;
            H.chisum += my_chi2;
        } else {
            H.nmiss += 1;
        }
#pragma unroll
        for (int k = 0; k < kLayers; ++k) H.ids[k] = k == l ? idl : H.ids[k];
    }
    if (l == kLayers - 1) {
        if (q == 0) write_result(o, n, i, s, H.chisum, H.ntrk, H.nmiss, TRD_ST_OK, H.ids);
        return true;
    }
    return false;
}

// Persistent follower: every group loops over seeds taken from the launch's
// counter and over their layers in one flattened loop, so a lane whose seed
// ends takes the next seed instead of idling while its warp finishes.
template <int G, int NH, int MINB, bool EXT>
__global__ void __launch_bounds__(128, MINB) k_follow(SeedsView sv, IndexView ix, Params P, ResultsView o, int *counter)
{
    extern __shared__ float smem[];
    const int groups = blockDim.x / G;
    const int g = threadIdx.x / G;
    const int q = G == 1 ? 0 : (threadIdx.x & (G - 1));
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << ((threadIdx.x & 31) & ~(G - 1)));
    float *sm = smem + g;
    const float vyy_max = __uint_as_float(__ldg(&ix.stats[0]));
    const float vzz_max = __uint_as_float(__ldg(&ix.stats[1]));
    const float dx_max = EXT && ix.recx ? __uint_as_float(__ldg(&ix.stats[3])) : 0.0f;
    Lane H;
    int i = 0, l = 0;
    bool have = false;
    for (;;) {
        if (!have) {
            i = fetch_seed<G>(counter, gmask, q);
            if (i >= sv.n) break;
            have = start_seed<G>(i, q, sv, o, H);
            l = 0;
            if (!have) continue;
        }
        if (layer_step<G, NH, EXT>(i, l, q, gmask, ix, P, o, sv.n, sm, groups, vyy_max, vzz_max, dx_max, H))
            have = false;
        ++l;
    }
}

}  // namespace trd

namespace trd_host {

using namespace trd;

template <int G, int NH, int MINB, bool EXT>
static int launch(const trd_ctx *ctx, const SeedsView &sv, const IndexView &ix, const Params &P,
                  const ResultsView &o, cudaStream_t s, int block, int *counter, bool prepare)
{
    if (sv.n == 0) return TRD_OK;
    const int groups = block / G;
    const size_t smem = sizeof(float) * 24 * groups;
    int per_sm = 0;
    TRD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_follow<G, NH, MINB, EXT>, block, smem));
    per_sm = per_sm > 0 ? per_sm : 1;
    const long long need = (static_cast<long long>(sv.n) + groups - 1) / groups;
    const int grid = static_cast<int>(std::min<long long>(need, static_cast<long long>(ctx->sm_count) * per_sm));
    TRD_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(int), s));
    if (prepare) {
        k_seed_prepare<<<(sv.n + 255) / 256, 256, 0, s>>>(sv, P, o);
        TRD_CUDA_TRY(cudaGetLastError());
    }
    k_follow<G, NH, MINB, EXT><<<grid, block, smem, s>>>(sv, ix, P, o, counter);
    TRD_CUDA_TRY(cudaGetLastError());
    return TRD_OK;
}

template <bool EXT>
static int dispatch(const trd_ctx *ctx, const SeedsView &sv, const IndexView &iv, const Params &P,
                    const ResultsView &o, cudaStream_t s, int G, int mb, int block, int nhyp, int *counter,
                    bool prepare)
{
    switch (G * 16 + mb) {
    case 1 * 16 + 4: return nhyp == 1 ? launch<1, 1, 4, EXT>(ctx, sv, iv, P, o, s, block, counter, prepare) : TRD_EINVAL;
    case 1 * 16 + 5: return nhyp == 1 ? launch<1, 1, 5, EXT>(ctx, sv, iv, P, o, s, block, counter, prepare) : TRD_EINVAL;
    case 1 * 16 + 6: return nhyp == 1 ? launch<1, 1, 6, EXT>(ctx, sv, iv, P, o, s, block, counter, prepare) : TRD_EINVAL;
    case 1 * 16 + 8: return nhyp == 1 ? launch<1, 1, 8, EXT>(ctx, sv, iv, P, o, s, block, counter, prepare) : TRD_EINVAL;
    case 2 * 16 + 3: return launch<2, 2, 3, EXT>(ctx, sv, iv, P, o, s, block, counter, prepare);
    case 2 * 16 + 4: return launch<2, 2, 4, EXT>(ctx, sv, iv, P, o, s, block, counter, prepare);
    case 4 * 16 + 3: return launch<4, 4, 3, EXT>(ctx, sv, iv, P, o, s, block, counter, prepare);
    case 4 * 16 + 4: return launch<4, 4, 4, EXT>(ctx, sv, iv, P, o, s, block, counter, prepare);
    case 8 * 16 + 3: return launch<8, 8, 3, EXT>(ctx, sv, iv, P, o, s, block, counter, prepare);
    case 8 * 16 + 4: return launch<8, 8, 4, EXT>(ctx, sv, iv, P, o, s, block, counter, prepare);
    case 32 * 16 + 3: return launch<32, 8, 3, EXT>(ctx, sv, iv, P, o, s, block, counter, prepare);
    case 32 * 16 + 4: return launch<32, 8, 4, EXT>(ctx, sv, iv, P, o, s, block, counter, prepare);
    default: return TRD_EINVAL;
    }
}

static Params make_params(const trd_params_t *p, const trd_alignment_t *align)
{
    Params P{p->bz, p->n_sigma_road, p->chi2_cut, p->p_miss, p->dy_gate_sigma, p->n_hyp, p->max_missing,
             p->res_mode, p->material_on};
    if (align) {
        P.chamber_x = align->chamber_x;
        if (align->bz_map) {
            P.bzmap = align->bz_map;
            P.nr = align->nr;
            P.nz = align->nz;
            P.r0 = align->r_min;
            P.ir = static_cast<float>(align->nr - 1) / (align->r_max - align->r_min);
            P.z0 = align->z_min;
            P.iz = static_cast<float>(align->nz - 1) / (align->z_max - align->z_min);
        }
    }
    return P;
}

// The seeds' pre-pass alone (it does not read the index, so a captured step
// can run it beside the index build).
int prepare_launch(const trd_seeds_t *seeds, const trd_params_t *p, trd_results_t *out, cudaStream_t s,
                   const trd_alignment_t *align)
{
    if (seeds->n == 0) return TRD_OK;
    SeedsView sv{seeds->alpha, seeds->x, seeds->y, seeds->z, seeds->snp, seeds->tgl, seeds->q2pt, seeds->cov,
                 seeds->n, nullptr, 1, seeds->trigger};
    const Params P = make_params(p, align);
    ResultsView o{out->alpha, out->x, out->par, out->cov, out->chi2, out->n_trk, out->n_miss, out->status,
                  out->tracklet_id};
    k_seed_prepare<<<(sv.n + 255) / 256, 256, 0, s>>>(sv, P, o);
    TRD_CUDA_TRY(cudaGetLastError());
    return TRD_OK;
}

int follow_launch(const trd_ctx *ctx, const trd_seeds_t *seeds, const IndexView &iv, const trd_params_t *p,
                  trd_results_t *out, cudaStream_t s, int lanes_per_track, int block_threads, int min_blocks,
                  int *counter, const int32_t *seed_offsets, int n_tf, const trd_alignment_t *align,
                  bool prepare)
{
    SeedsView sv{seeds->alpha, seeds->x, seeds->y, seeds->z, seeds->snp, seeds->tgl, seeds->q2pt, seeds->cov,
                 seeds->n, seed_offsets, n_tf, seeds->trigger};
    const Params P = make_params(p, align);
    const bool ext = iv.recx || P.chamber_x || P.bzmap;
    ResultsView o{out->alpha, out->x, out->par, out->cov, out->chi2, out->n_trk, out->n_miss, out->status,
                  out->tracklet_id};
    const int block = block_threads > 0 ? block_threads : 128;
    int G = lanes_per_track;
    if (G <= 0) G = p->n_hyp <= 1 ? 1 : (p->n_hyp <= 2 ? 2 : (p->n_hyp <= 4 ? 4 : 8));
    if (G < p->n_hyp) return TRD_EINVAL;
    const int mb = min_blocks > 0 ? min_blocks : 4;
    return ext ? dispatch<true>(ctx, sv, iv, P, o, s, G, mb, block, p->n_hyp, counter, prepare)
               : dispatch<false>(ctx, sv, iv, P, o, s, G, mb, block, p->n_hyp, counter, prepare);
}

}  // namespace trd_host
