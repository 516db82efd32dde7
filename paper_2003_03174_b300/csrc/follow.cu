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
    if (EXT) {
        // the same steps through one inlined copy of the transport (the EXT
        // kernels' code is large enough that instruction fetch shows: 4 %
        // faster on the misaligned timeframe): to the layer's plane, to it
        // again in the neighbour sector's frame after a sector change, then
        // on to the chamber's radius
        df target = xl;
        chamber = -1;
        bool at_plane = false;
        for (int step = 0; step < 3; ++step) {
            if (!propagate(s, target, step_bz<EXT>(P, s, target))) return false;
            if (at_plane) break;
            if (step == 0 && fabsf(s.y.hi) > xl.hi * half_sector_tan()) {
                const int dir = s.y.hi > 0.0f ? 1 : -1;
                const int ns = (s.sector + dir + kSectors) % kSectors;
                const df d = dir > 0 ? df{kSectorWidthHi, kSectorWidthLo} : df{-kSectorWidthHi, -kSectorWidthLo};
                if (!rotate(s, d, ns, point_bz<EXT>(P, s))) return false;
                continue;
            }
            at_plane = true;
            if (P.material && !material<false>(s)) return false;
            const float u = (s.z - kZMin) * (1.0f / kStackLength);
            if (!(u >= 0.0f && u < static_cast<float>(kStacks))) break;
            chamber = s.sector * (kStacks * kLayers) + static_cast<int>(u) * kLayers + l;
            if (!P.chamber_x) break;
            const float xc = __ldg(&P.chamber_x[chamber]);
            if (xc == xl.hi && xl.lo == 0.0f) break;
            target = {xc, 0.0f};
        }
        return true;
    }
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
// The selection order (score, parent rank, tracklet id) as one unsigned
// 64-bit key: the score's bits made orderable, then the parent (3 bits) and
// the id (28 bits, kMissing as the largest, so a missing layer sorts after
// tracklets of the same score).  Needs tracklet ids below kKeyIdMask (the
// library checks the index's size); kNoKey (all ones) marks an empty slot.
constexpr unsigned kKeyIdMask = 0x0fffffffu;
constexpr unsigned long long kNoKey = ~0ull;

__device__ __forceinline__ unsigned long long sel_key(float s, int par, int id)
{
    unsigned u = __float_as_uint(s);
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    const unsigned lo = (static_cast<unsigned>(par) << 28) | (id == kMissing ? kKeyIdMask : static_cast<unsigned>(id));
    return (static_cast<unsigned long long>(u) << 32) | lo;
}

__device__ __forceinline__ float key_score(unsigned long long k)
{
    const unsigned t = static_cast<unsigned>(k >> 32);
    return __uint_as_float((t & 0x80000000u) ? (t & 0x7fffffffu) : ~t);
}

__device__ __forceinline__ int key_parent(unsigned long long k) { return static_cast<int>(static_cast<unsigned>(k) >> 28); }

__device__ __forceinline__ int key_id(unsigned long long k)
{
    const unsigned id = static_cast<unsigned>(k) & kKeyIdMask;
    return id == kKeyIdMask ? kMissing : static_cast<int>(id);
}

template <int NH>
struct ExtList {
    // extensions kept in the selection order, with their chi2 and record
    // position (-1 for a missing layer)
    unsigned long long key[NH];
    float chi2[NH];
    int pos[NH];
    __device__ __forceinline__ void clear()
    {
#pragma unroll
        for (int k = 0; k < NH; ++k) {
            key[k] = kNoKey;
            chi2[k] = 0.0f;
            pos[k] = -1;
        }
    }
    __device__ __forceinline__ void insert(float sc, int parent, int tid, int p, float c2)
    {
        const unsigned long long kk = sel_key(sc, parent, tid);
        if (!(kk < key[NH - 1])) return;
        // shift larger entries up, then place (unrolled, stays in registers)
        bool placed = false;
#pragma unroll
        for (int k = NH - 1; k >= 0; --k) {
            if (placed) continue;
            const bool move = k > 0 && kk < key[k - 1];
            if (move) {
                key[k] = key[k - 1];
                chi2[k] = chi2[k - 1];
                pos[k] = pos[k - 1];
            } else {
                key[k] = kk;
                chi2[k] = c2;
                pos[k] = p;
                placed = true;
            }
        }
    }
    __device__ __forceinline__ void pop()
    {
#pragma unroll
        for (int k = 0; k + 1 < NH; ++k) {
            key[k] = key[k + 1];
            chi2[k] = chi2[k + 1];
            pos[k] = pos[k + 1];
        }
        key[NH - 1] = kNoKey;
        pos[NH - 1] = -1;
    }
    __device__ __forceinline__ bool empty() const { return key[0] == kNoKey; }
    __device__ __forceinline__ unsigned long long head_key() const { return key[0]; }
    __device__ __forceinline__ float head_score() const { return key_score(key[0]); }
    __device__ __forceinline__ int head_id() const { return key_id(key[0]); }
    __device__ __forceinline__ float head_chi2() const { return chi2[0]; }
    __device__ __forceinline__ int head_pos() const { return pos[0]; }
};

// One entry (N = 1): plain fields, so no key is built for every candidate.
template <>
struct ExtList<1> {
    float score, c2;
    int par, id, pos;
    __device__ __forceinline__ void clear()
    {
        score = INFINITY;
        c2 = 0.0f;
        par = 0x7fffffff;
        id = kMissing;
        pos = -1;
    }
    __device__ __forceinline__ void insert(float sc, int parent, int tid, int p, float chi2)
    {
        if (sc < score || (sc == score && (parent < par || (parent == par && tid < id)))) {
            score = sc;
            c2 = chi2;
            par = parent;
            id = tid;
            pos = p;
        }
    }
    __device__ __forceinline__ void pop() { clear(); }
    __device__ __forceinline__ bool empty() const { return !(score < INFINITY); }
    __device__ __forceinline__ unsigned long long head_key() const { return empty() ? kNoKey : sel_key(score, par, id); }
    __device__ __forceinline__ float head_score() const { return score; }
    __device__ __forceinline__ int head_id() const { return id; }
    __device__ __forceinline__ float head_chi2() const { return c2; }
    __device__ __forceinline__ int head_pos() const { return pos; }
};

// Road query + candidate tests for one hypothesis at layer l (Sec. 3).
// The road bounds z_tl to z +- Rz (pad rows r_lo..r_hi) and the measured y to
// y +- (W + |tan tau| Rz) (y bins b_lo..b_hi); each pad row is one contiguous
// range of the index over those bins.  The candidates of up to three rows
// form one list: the first halves of their records, {y, z, dy, id}, are read
// eight at a time (one dependent L2 round trip, which also brings each 32-byte
// record into L1), a bit mask keeps those inside the road's y/z bounds and
// the deflection gate, and only those get the full test (record read again
// from L1).  Longer z roads are handled the same way, three rows at a time.
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
    // (the first half is an L1 hit: the pre-filter read it; taking it from
    // the pre-filter's registers would index them by a run-time slot)
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

constexpr int kScanChunk = 8;  // candidates whose loads are in flight together

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
    const int nb = ix.nb;
    for (int r = r_lo; r <= r_hi; r += 3) {
        // up to three pad rows: their six bounds are loaded together
        const int base = bucket_of(cbase + chamber, 0, r, nb);
        const int beg0 = __ldg(&ix.offsets[base + b_lo]);
        const int end0 = __ldg(&ix.offsets[base + b_hi + 1]);
        int beg1 = 0, end1 = 0, beg2 = 0, end2 = 0;
        if (r + 1 <= r_hi) {
            beg1 = __ldg(&ix.offsets[base + nb + b_lo]);
            end1 = __ldg(&ix.offsets[base + nb + b_hi + 1]);
        }
        if (r + 2 <= r_hi) {
            beg2 = __ldg(&ix.offsets[base + 2 * nb + b_lo]);
            end2 = __ldg(&ix.offsets[base + 2 * nb + b_hi + 1]);
        }
        const int n0 = end0 - beg0;
        const int n01 = n0 + (end1 - beg1);
        const int n = n01 + (end2 - beg2);
#pragma unroll 1
        for (int j0 = 0; j0 < n; j0 += kScanChunk) {
            float4 c[kScanChunk];  // the records' first halves {y, z, dy, id}
#pragma unroll
            for (int u = 0; u < kScanChunk; ++u) {
                const int j = j0 + u;
                const int pos = j < n0 ? beg0 + j : (j < n01 ? beg1 + (j - n0) : beg2 + (j - n01));
                c[u] = j < n ? __ldg(&ix.rec[2 * pos]) : make_float4(INFINITY, INFINITY, INFINITY, 0.0f);
            }
            // pre-filter: the road's y/z box and the deflection gate (the
            // gate is the full test's own condition, taken here because dy
            // arrives with y and z)
            unsigned mask = 0;
#pragma unroll
            for (int u = 0; u < kScanChunk; ++u) {
                const float ry = (__fsub_rn(c[u].x, yh) - yl) + tt * (z - c[u].y);
                const float rz = c[u].y - z;
                if (fabsf(ry) <= W && fabsf(rz) <= Rz && !(fabsf(c[u].z - dy_pred) > gate)) mask |= 1u << u;
            }
            while (mask) {
                const int u = __ffs(mask) - 1;
                mask &= mask - 1u;
                const int j = j0 + u;
                const int pos = j < n0 ? beg0 + j : (j < n01 ? beg1 + (j - n0) : beg2 + (j - n01));
                full_test<NH, EXT>(pos, ix, tt, z, yh, yl, n2, syy_trk, syz_trk, c11, vyy_res, P.resmode, dy_pred,
                                   gate, P.cut, score, 0, trig, e, L);
            }
        }
    }
}

constexpr int kRoadWords = 21;  // a hypothesis's road in the group scan's table (17 without EXT)

// Group scan (N > 1): the lanes of a seed's group take its hypotheses one at
// a time and share each one's road: the road is broadcast from the lane that
// holds the hypothesis, lane q tests candidates q, q + G, ... (four at a
// time), and every extension records its parent.  The candidate set, the
// arithmetic and the selection order are those of one lane scanning its own
// hypothesis; the work is spread evenly over the group.  This version
// broadcasts by shuffles (groups of 2 and 4); groups of 8 or more use
// group_road / group_scan below, through a road table in shared memory.
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
        for (int r = hr_lo; r <= hr_hi; r += 3) {
            // up to three pad rows: their six bounds are loaded together
            const int base = hbase + r * ix.nb;
            const int beg0 = __ldg(&ix.offsets[base + hb_lo]);
            const int end0 = __ldg(&ix.offsets[base + hb_hi + 1]);
            int beg1 = 0, end1 = 0, beg2 = 0, end2 = 0;
            if (r + 1 <= hr_hi) {
                beg1 = __ldg(&ix.offsets[base + ix.nb + hb_lo]);
                end1 = __ldg(&ix.offsets[base + ix.nb + hb_hi + 1]);
            }
            if (r + 2 <= hr_hi) {
                beg2 = __ldg(&ix.offsets[base + 2 * ix.nb + hb_lo]);
                end2 = __ldg(&ix.offsets[base + 2 * ix.nb + hb_hi + 1]);
            }
            const int n0 = end0 - beg0;
            const int n01 = n0 + (end1 - beg1);
            const int n = n01 + (end2 - beg2);
            // lane q takes candidates q, q + G, ...: ceil(n / G) of them, four at a time
            const int per_lane = (n + G - 1) / G;
            for (int u0 = 0; u0 < per_lane; u0 += 4) {
                float4 c[4];  // the records' first halves {y, z, dy, id}
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = q + G * (u0 + u);
                    const int pos = j < n0 ? beg0 + j : (j < n01 ? beg1 + (j - n0) : beg2 + (j - n01));
                    c[u] = j < n ? __ldg(&ix.rec[2 * pos]) : make_float4(INFINITY, INFINITY, INFINITY, 0.0f);
                }
                unsigned mask = 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float ry = (__fsub_rn(c[u].x, hyh) - hyl) + tt * (hz - c[u].y);
                    const float rz = c[u].y - hz;
                    if (fabsf(ry) <= hW && fabsf(rz) <= hRz && !(fabsf(c[u].z - hdyp) > hgate)) mask |= 1u << u;
                }
                while (mask) {
                    const int u = __ffs(mask) - 1;
                    mask &= mask - 1u;
                    const int j = q + G * (u0 + u);
                    const int pos = j < n0 ? beg0 + j : (j < n01 ? beg1 + (j - n0) : beg2 + (j - n01));
                    full_test<NH, EXT>(pos, ix, tt, hz, hyh, hyl, n2, hsyy, hsyz, hc11, hvres, P.resmode, hdyp,
                                       hgate, P.cut, hscore, h, trig, he, L);
                }
            }
        }
    }
}

// Groups of 8 or more, in two steps around a parking of each lane's state in
// shared memory: each lane writes its own road to its column of the block's
// road table (row stride = block size), then the group scans its hypotheses
// reading each one's road from the table.  Neither step needs the lanes'
// states, so they wait in shared memory meanwhile and the registers hold one
// road and the lists: 96 registers with 8 B of spill, 5 blocks per SM.
template <int G, bool EXT>
__device__ __forceinline__ void group_road(bool mine, const TrackState &s, int l, int chamber, int cbase, float score,
                                           const Params &P, const IndexView &ix, float vyy_max_in, float vzz_max,
                                           float dx_max, float *road)
{
    if (!mine) return;
    const int S = blockDim.x;
    const float tt = layer_tilt_tan(l);
    const float f = s.f;
    const float r = sqrtf((1.0f - f) * (1.0f + f));
    const float uu = f / r - lorentz_tan(P.bz);
    const float vres = kSigY0 * kSigY0 + kSigY1 * kSigY1 * uu * uu;
    const float vyy_max = P.resmode ? vres : vyy_max_in;
    const float c10 = s.c[1], c11 = s.c[2];
    const float syy = s.c[0] - 2.0f * tt * c10 + tt * tt * c11;
    const float syz = c10 - tt * c11;
    float W = P.road * sqrtf(fmaxf(syy + vyy_max, 0.0f)) * 1.0001f + 1e-4f;
    float Rz = P.road * sqrtf(fmaxf(c11 + vzz_max, 0.0f)) * 1.0001f + 1e-4f;
    LinExt e{s.x.hi, s.x.lo, 0.0f, 0.0f};
    if (EXT && ix.recx) {
        e.fr = f / r;
        e.tr = s.t / r;
        const float dxb = dx_max + fabsf(df_to_f(df_add(s.x, df_neg(layer_x_df(l))))) + 1e-4f;
        W += dxb * fabsf(e.fr) * 1.0001f;
        Rz += dxb * fabsf(e.tr) * 1.0001f;
    }
    const float dyp = kDriftLength * uu;
    const float gate = P.gate * sqrtf(kSigDy0 * kSigDy0 + kSigDy1 * kSigDy1 * uu * uu);
    const float z = s.z, yh = s.y.hi, yl = s.y.lo;
    const float zlo = stack_z_lo(stack_of_chamber(chamber));
    const int r_lo = row_of_z(z - Rz, zlo), r_hi = row_of_z(z + Rz, zlo);
    const float half = W + fabsf(tt) * Rz + 1e-3f + 1e-6f * fabsf(yh);
    const int b_lo = ybin_of(yh - half, ix.inv_w, ix.nb), b_hi = ybin_of(yh + half, ix.inv_w, ix.nb);
    const int base_ch = bucket_of(cbase + chamber, 0, 0, ix.nb);
    const float v[kRoadWords] = {z, yh, yl, W, Rz, syy, syz, c11, vres, dyp, gate, score,
                                 __int_as_float(r_lo), __int_as_float(r_hi), __int_as_float(b_lo),
                                 __int_as_float(b_hi), __int_as_float(base_ch), e.xh, e.xl, e.fr, e.tr};
    float *own = road + threadIdx.x;
#pragma unroll
    for (int k = 0; k < (EXT ? kRoadWords : kRoadWords - 4); ++k) own[k * S] = v[k];
}

template <int G, int NH, bool EXT>
__device__ __forceinline__ void group_scan(bool mine, int l, const Params &P, const IndexView &ix, unsigned gmask,
                                           int trig, const float *road, ExtList<NH> &L)
{
    const int S = blockDim.x;
    const float tt = layer_tilt_tan(l);
    const float n2 = P.road * P.road;
    __syncwarp(gmask);
    for (int h = 0; h < NH; ++h) {  // hypotheses live in lanes 0..NH-1
        if (!__shfl_sync(gmask, static_cast<int>(mine), h, G)) continue;
        const float *hr = road + (threadIdx.x & ~(G - 1)) + h;  // lane h of this group
        const float hz = hr[0], hyh = hr[S], hyl = hr[2 * S], hW = hr[3 * S], hRz = hr[4 * S];
        const float hsyy = hr[5 * S], hsyz = hr[6 * S], hc11 = hr[7 * S], hvres = hr[8 * S];
        const float hdyp = hr[9 * S], hgate = hr[10 * S], hscore = hr[11 * S];
        const int hr_lo = __float_as_int(hr[12 * S]), hr_hi = __float_as_int(hr[13 * S]);
        const int hb_lo = __float_as_int(hr[14 * S]), hb_hi = __float_as_int(hr[15 * S]);
        const int hbase = __float_as_int(hr[16 * S]);
        LinExt he{};
        if (EXT) {
            he.xh = hr[17 * S];
            he.xl = hr[18 * S];
            he.fr = hr[19 * S];
            he.tr = hr[20 * S];
        }
        const int q = threadIdx.x & (G - 1);
        for (int r = hr_lo; r <= hr_hi; r += 3) {
            const int base = hbase + r * ix.nb;
            const int beg0 = __ldg(&ix.offsets[base + hb_lo]);
            const int end0 = __ldg(&ix.offsets[base + hb_hi + 1]);
            int beg1 = 0, end1 = 0, beg2 = 0, end2 = 0;
            if (r + 1 <= hr_hi) {
                beg1 = __ldg(&ix.offsets[base + ix.nb + hb_lo]);
                end1 = __ldg(&ix.offsets[base + ix.nb + hb_hi + 1]);
            }
            if (r + 2 <= hr_hi) {
                beg2 = __ldg(&ix.offsets[base + 2 * ix.nb + hb_lo]);
                end2 = __ldg(&ix.offsets[base + 2 * ix.nb + hb_hi + 1]);
            }
            const int n0 = end0 - beg0;
            const int n01 = n0 + (end1 - beg1);
            const int n = n01 + (end2 - beg2);
            const int per_lane = (n + G - 1) / G;
            for (int u0 = 0; u0 < per_lane; u0 += 4) {
                float4 c[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int j = q + G * (u0 + u);
                    const int pos = j < n0 ? beg0 + j : (j < n01 ? beg1 + (j - n0) : beg2 + (j - n01));
                    c[u] = j < n ? __ldg(&ix.rec[2 * pos]) : make_float4(INFINITY, INFINITY, INFINITY, 0.0f);
                }
                unsigned mask = 0;
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const float ry = (__fsub_rn(c[u].x, hyh) - hyl) + tt * (hz - c[u].y);
                    const float rz = c[u].y - hz;
                    if (fabsf(ry) <= hW && fabsf(rz) <= hRz && !(fabsf(c[u].z - hdyp) > hgate)) mask |= 1u << u;
                }
                while (mask) {
                    const int u = __ffs(mask) - 1;
                    mask &= mask - 1u;
                    const int j = q + G * (u0 + u);
                    const int pos = j < n0 ? beg0 + j : (j < n01 ? beg1 + (j - n0) : beg2 + (j - n01));
                    full_test<NH, EXT>(pos, ix, tt, hz, hyh, hyl, n2, hsyy, hsyz, hc11, hvres, P.resmode, hdyp,
                                       hgate, P.cut, hscore, h, trig, he, L);
                }
            }
        }
    }
    __syncwarp(gmask);  // the table is rewritten at the next layer
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

// A finished seed's result as one 128-byte record at its sorted position
// (8 vector stores); k_results_gather moves it to the seed's input position.
// Words: alpha, x, par[5], cov[15], chi2, then n_trk, n_miss, status, ids[6].
// The one-lane kernel keeps the ids in the record (written per layer), not
// in registers: stage all but them.
__device__ __forceinline__ void stage_result_noids(float4 *res, int pos, const TrackState &s, float chi2, int ntrk,
                                                   int nmiss, int status)
{
    float4 *r = res + 8 * static_cast<size_t>(pos);
    r[0] = make_float4(sector_alpha_df(s.sector).hi, df_to_f(s.x), df_to_f(s.y), s.z);
    r[1] = make_float4(s.f, s.t, s.k, s.c[0]);
    r[2] = make_float4(s.c[1], s.c[2], s.c[3], s.c[4]);
    r[3] = make_float4(s.c[5], s.c[6], s.c[7], s.c[8]);
    r[4] = make_float4(s.c[9], s.c[10], s.c[11], s.c[12]);
    r[5] = make_float4(s.c[13], s.c[14], chi2, __int_as_float(ntrk));
    reinterpret_cast<float2 *>(r + 6)[0] = make_float2(__int_as_float(nmiss), __int_as_float(status));
}

__device__ __forceinline__ void stage_result(float4 *res, int pos, const TrackState &s, float chi2, int ntrk,
                                             int nmiss, int status, const int (&ids)[kLayers])
{
    float4 *r = res + 8 * static_cast<size_t>(pos);
    r[0] = make_float4(sector_alpha_df(s.sector).hi, df_to_f(s.x), df_to_f(s.y), s.z);
    r[1] = make_float4(s.f, s.t, s.k, s.c[0]);
    r[2] = make_float4(s.c[1], s.c[2], s.c[3], s.c[4]);
    r[3] = make_float4(s.c[5], s.c[6], s.c[7], s.c[8]);
    r[4] = make_float4(s.c[9], s.c[10], s.c[11], s.c[12]);
    r[5] = make_float4(s.c[13], s.c[14], chi2, __int_as_float(ntrk));
    r[6] = make_float4(__int_as_float(nmiss), __int_as_float(status), __int_as_float(ids[0]), __int_as_float(ids[1]));
    r[7] = make_float4(__int_as_float(ids[2]), __int_as_float(ids[3]), __int_as_float(ids[4]),
                       __int_as_float(ids[5]));
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

constexpr int kParkWords = 33;  // a lane's state (24) and bookkeeping (9) while its group scans

// Which instances scan through the road table with the lanes' states parked:
// groups of 8 or more always; smaller groups with 5 or more blocks per SM,
// whose register budget only that fits (with 3 or 4 blocks per SM their
// shuffle broadcast is faster).
__host__ __device__ constexpr bool parks(int G, int MINB) { return G >= 8 || (G > 1 && MINB >= 5); }

__device__ __forceinline__ void park(float *pk, int S, const TrackState &s, const Lane &H)
{
    pk[0] = s.x.hi;
    pk[S] = s.x.lo;
    pk[2 * S] = s.y.hi;
    pk[3 * S] = s.y.lo;
    pk[4 * S] = s.z;
    pk[5 * S] = s.f;
    pk[6 * S] = s.t;
    pk[7 * S] = s.k;
#pragma unroll
    for (int k = 0; k < 15; ++k) pk[(8 + k) * S] = s.c[k];
    pk[23 * S] = __int_as_float(s.sector);
    pk[24 * S] = H.chisum;
    pk[25 * S] = __int_as_float(H.ntrk);
    pk[26 * S] = __int_as_float(H.nmiss);
#pragma unroll
    for (int k = 0; k < kLayers; ++k) pk[(27 + k) * S] = __int_as_float(H.ids[k]);
}

__device__ __forceinline__ void unpark(const float *pk, int S, TrackState &s, Lane &H)
{
    s.x.hi = pk[0];
    s.x.lo = pk[S];
    s.y.hi = pk[2 * S];
    s.y.lo = pk[3 * S];
    s.z = pk[4 * S];
    s.f = pk[5 * S];
    s.t = pk[6 * S];
    s.k = pk[7 * S];
#pragma unroll
    for (int k = 0; k < 15; ++k) s.c[k] = pk[(8 + k) * S];
    s.sector = __float_as_int(pk[23 * S]);
    H.chisum = pk[24 * S];
    H.ntrk = __float_as_int(pk[25 * S]);
    H.nmiss = __float_as_int(pk[26 * S]);
#pragma unroll
    for (int k = 0; k < kLayers; ++k) H.ids[k] = __float_as_int(pk[(27 + k) * S]);
}

// ---- processing order ---------------------------------------------------------
// The follower takes seeds in order of decreasing |q/pT| (bins of 1/28 c/GeV;
// everything above 4.5 c/GeV shares the first bin): a low-momentum seed has a
// wide road (scattering), a high-momentum one a narrow road, so lanes that
// take seeds together scan roads of similar size and diverge less, and the
// slow seeds start first instead of forming the launch's tail.  Results do
// not depend on the order (every seed is followed on its own).  The rotated
// seed state is parked at the seed's sorted position and the result is staged
// there too, so the follower reads and writes consecutive addresses; a gather
// kernel then writes the results at the input positions with full lines.
constexpr int kSortBins = 128;        // momentum bins of one timeframe
constexpr int kMaxSortBins = 1024;    // bins of a batch of timeframes (128 per timeframe up to 8)
constexpr float kSortBinsPerUnit = 28.0f;
constexpr int kKeyThreads = 256;
constexpr int kKeyItems = 2;  // seeds per thread: 391 blocks for 200k seeds (8 per thread left 98, fewer than the SMs)
constexpr int kParkedWords = 25;  // words of a parked record

// A batch of timeframes is taken timeframe by timeframe (each one's tracklet
// records then stay in L2 while its seeds are followed), each in momentum
// order at the resolution its share of the bins leaves: a batch has
// sort_bins(n_tf) = 128 * min(n_tf, 8) bins and bin = (timeframe * 128 +
// momentum bin) * bins / (128 * n_tf) (all 128 momentum bins of each
// timeframe up to 8 timeframes, 16 of them at 64).
__host__ __device__ __forceinline__ int sort_bins(int n_tf) { return kSortBins * (n_tf < 8 ? n_tf : 8); }

__device__ __forceinline__ int sort_bin(float q2pt, int tf, int n_tf)
{
    const float a = fabsf(q2pt) * kSortBinsPerUnit;  // NaN fails the test: first bin
    const int local = a < static_cast<float>(kSortBins - 1) ? kSortBins - 1 - static_cast<int>(a) : 0;
    if (n_tf == 1) return local;
    return static_cast<int>((static_cast<long long>(tf) * kSortBins + local) * sort_bins(n_tf) /
                            (static_cast<long long>(kSortBins) * n_tf));
}

// Scratch of one follower call (device, n seeds of n_tf timeframes; the base
// 16-byte aligned):
//   bin_count [sort_bins]     seeds per sort bin (zeroed before k_seed_key)
//   counter   [4]             the follower's work counter (zeroed by
//                             k_seed_key), then padding: each call in flight
//                             has its own
//   rec       [n][8] float4   one 128-byte record per sorted position: first
//                             the parked seed (k_seed_prepare), then the
//                             staged result (stage_result)
//   rank      [n]             a seed's rank inside its bin (input order)
//   inv       [n]             the seed's sorted position, -1 when it ended in
//                             k_seed_prepare (input order)
// Parked record (words): sector (int bits; -1 = finished), x.hi, x.lo, y.hi,
// y.lo, z, snp, tgl, q2pt, c0..c14, input index (int bits); words 25..31
// unused until the result is staged (the one-lane follower sets words 26..31,
// the tracklet ids, to -1 when it takes the seed and writes each matched
// layer's id there, so they need no registers).
struct ParkedView {
    int32_t *bin_count;
    int32_t *counter;
    float4 *rec;
    int32_t *rank, *inv;
    int nbins;
};

// bin counts, work counter, padding (528 bytes for one timeframe: a multiple of 16)
__host__ __device__ inline int parked_head(int n_tf) { return sort_bins(n_tf) + 4; }

__host__ __device__ inline size_t parked_words(int n, int n_tf)
{
    return static_cast<size_t>(parked_head(n_tf)) + static_cast<size_t>(32 + 2) * static_cast<size_t>(n);
}

__host__ __device__ inline ParkedView parked_view(void *base, int n, int n_tf)
{
    int32_t *w = static_cast<int32_t *>(base);
    ParkedView v;
    v.nbins = sort_bins(n_tf);
    v.bin_count = w;
    v.counter = w + v.nbins;
    v.rec = reinterpret_cast<float4 *>(w + parked_head(n_tf));  // still 16-byte aligned
    v.rank = w + parked_head(n_tf) + 32 * static_cast<size_t>(n);
    v.inv = v.rank + n;
    return v;
}

// Bin of every seed and its rank inside the bin: lanes of a warp with the
// same bin share one shared-memory atomic, and each block takes its base in
// every occupied bin with one global atomic.  Also zeroes the follower's work
// counter (the follower starts after this kernel).
__global__ void __launch_bounds__(kKeyThreads)
k_seed_key(const float *__restrict__ q2pt, int n, const int32_t *__restrict__ soff, int n_tf, ParkedView pk,
           int *__restrict__ counter)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0;
    __shared__ int h[kMaxSortBins], base[kMaxSortBins];
    for (int t = threadIdx.x; t < pk.nbins; t += kKeyThreads) h[t] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int i0 = blockIdx.x * (kKeyThreads * kKeyItems) + threadIdx.x;
    int b[kKeyItems], r[kKeyItems];
#pragma unroll
    for (int u = 0; u < kKeyItems; ++u) {
        const int i = i0 + u * kKeyThreads;
        b[u] = i < n ? sort_bin(__ldg(&q2pt[i]), tf_of(i, soff, n_tf), n_tf) : -1;
        const unsigned peers = __match_any_sync(0xffffffffu, b[u]);
        const int leader = __ffs(peers) - 1;
        int first = 0;
        if (b[u] >= 0 && lane == leader) first = atomicAdd(&h[b[u]], __popc(peers));
        first = __shfl_sync(0xffffffffu, first, leader);
        r[u] = first + __popc(peers & ((1u << lane) - 1u));
    }
    __syncthreads();
    for (int t = threadIdx.x; t < pk.nbins; t += kKeyThreads) base[t] = h[t] ? atomicAdd(&pk.bin_count[t], h[t]) : 0;
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kKeyItems; ++u) {
        const int i = i0 + u * kKeyThreads;
        if (b[u] >= 0) pk.rank[i] = base[b[u]] + r[u];
    }
}

// Seed preparation, one thread per seed (all seeds take the same path, so
// this runs without divergence): load the seed, validate it, rotate it into
// the sector of its position.  A seed that ends here gets its final result
// (and sector -1 at its sorted position); a live seed's rotated state is
// parked at its sorted position.
__global__ void __launch_bounds__(256) k_seed_prepare(SeedsView sv, Params P, ResultsView o, ParkedView pk)
{
    wait_prior_grid();
    // first sorted position of every bin: exclusive scan of the bin counts
    // (one warp, nbins / 32 consecutive bins per lane)
    static_assert(kSortBins % 32 == 0 && kMaxSortBins % kSortBins == 0, "bins per lane");
    __shared__ int s_off[kMaxSortBins];
    static_assert(kParkedWords % 2 == 1, "an odd row length keeps the lanes' rows in distinct banks");
    __shared__ float s_rec[256 / 32][32][kParkedWords];  // each warp's records
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = sv.n;
    // the seed's inputs and rank, loaded before the bin scan so that their
    // latency overlaps it
    TrackState s;
    float alpha = 0.0f;
    int rank = 0;
    if (i < n) {
        alpha = sv.alpha[i];
        s.x = {sv.x[i], 0.0f};
        s.y = {sv.y[i], 0.0f};
        s.z = sv.z[i];
        s.f = sv.snp[i];
        s.t = sv.tgl[i];
        s.k = sv.q2pt[i];
#pragma unroll
        for (int k = 0; k < 15; ++k) s.c[k] = sv.cov[k * n + i];
        rank = pk.rank[i];
    }
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const int per = pk.nbins / 32;
        int sum = 0;
        for (int j = 0; j < per; ++j) {
            const int c = pk.bin_count[per * lane + j];
            s_off[per * lane + j] = c;
            sum += c;
        }
        int x = sum;
#pragma unroll
        for (int o2 = 1; o2 < 32; o2 <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, x, o2);
            if (lane >= o2) x += t;
        }
        int run = x - sum;
        for (int j = 0; j < per; ++j) {
            const int c = s_off[per * lane + j];
            s_off[per * lane + j] = run;
            run += c;
        }
    }
    __syncthreads();
    // 0: parked, 1: ended here, 2: beyond n (no early exits: the warp writes
    // its seeds' records together below)
    int state = 2, pos = -1;
    float *t = s_rec[threadIdx.x >> 5][threadIdx.x & 31];
    if (i < n) {
        pos = s_off[sort_bin(s.k, tf_of(i, sv.soff, sv.n_tf), sv.n_tf)] + rank;
        const float sx = s.x.hi, sy = s.y.hi;
        state = 1;
        if (!(fabsf(s.f) < kMaxSnp) || !cov_pd(s.c)) {
            write_seed_result(o, sv, n, i, TRD_ST_SEED_INVALID);
        } else {
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
            } else {
                state = 0;
                t[0] = __int_as_float(sec);
                t[1] = s.x.hi;
                t[2] = s.x.lo;
                t[3] = s.y.hi;
                t[4] = s.y.lo;
                t[5] = s.z;
                t[6] = s.f;
                t[7] = s.t;
                t[8] = s.k;
#pragma unroll
                for (int k = 0; k < 15; ++k) t[9 + k] = s.c[k];
                t[24] = __int_as_float(i);
            }
        }
        pk.inv[i] = state == 0 ? pos : -1;
    }
    __syncwarp();
    // the warp's records, one 100-byte record per store instruction
    const int lane = threadIdx.x & 31;
    float *recw = reinterpret_cast<float *>(pk.rec);
    for (int j = 0; j < 32; ++j) {
        const int pj = __shfl_sync(0xffffffffu, pos, j);
        const int sj = __shfl_sync(0xffffffffu, state, j);
        if (sj == 0 && lane < kParkedWords) recw[32 * static_cast<size_t>(pj) + lane] = s_rec[threadIdx.x >> 5][j][lane];
        if (sj == 1 && lane == 0) reinterpret_cast<int *>(recw)[32 * static_cast<size_t>(pj)] = -1;
    }
}

// Pick up the seed at sorted position pos as parked by k_seed_prepare; i is
// its input index.  Returns false when the seed already has its final result.
template <int G>
__device__ __forceinline__ bool start_seed(int pos, int q, const SeedsView &sv, const ParkedView &pk, Lane &L,
                                           int &i)
{
    // plain loads: the follower later stages the result in the same record
    const float4 *rec = pk.rec + 8 * static_cast<size_t>(pos);
    const float4 r0 = rec[0];
    const int sec = __float_as_int(r0.x);
    if (sec < 0) return false;
    const float4 r1 = rec[1], r2 = rec[2], r3 = rec[3], r4 = rec[4], r5 = rec[5];
    i = sv.soff || sv.trig ? __float_as_int(rec[6].x) : 0;  // the input index, for timeframe and interaction
    TrackState &s = L.s;
    s.sector = sec;
    s.x = {r0.y, r0.z};
    s.y = {r0.w, r1.x};
    s.z = r1.y;
    s.f = r1.z;
    s.t = r1.w;
    s.k = r2.x;
    const float c[15] = {r2.y, r2.z, r2.w, r3.x, r3.y, r3.z, r3.w, r4.x, r4.y, r4.z, r4.w, r5.x, r5.y, r5.z, r5.w};
#pragma unroll
    for (int k = 0; k < 15; ++k) s.c[k] = c[k];
    L.cbase = tf_of(i, sv.soff, sv.n_tf) * kChambers;
    L.trig = sv.trig ? sv.trig[i] : -1;
    L.alive = q == 0;
    L.score = 0.0f;
    L.chisum = 0.0f;
    L.ntrk = 0;
    L.nmiss = 0;
#pragma unroll
    for (int k = 0; k < kLayers; ++k) L.ids[k] = -1;
    if (G == 1) {  // the ids live in the record (words 26..31)
        const float m1 = __int_as_float(-1);
        float4 *r = pk.rec + 8 * static_cast<size_t>(pos);
        reinterpret_cast<float2 *>(r + 6)[1] = make_float2(m1, m1);
        r[7] = make_float4(m1, m1, m1, m1);
    }
    return true;
}

// One layer of seed i for the group.  Returns true when the seed is finished
// (result written).
template <int G, int NH, bool EXT, bool PARK>
__device__ __forceinline__ bool layer_step(int pos, int l, int q, unsigned gmask, const IndexView &ix, const Params &P,
                                           float4 *res, float *sm, int stride, float *road, float vyy_max,
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
    } else if (PARK) {
        const bool mine = live && chamber >= 0;
        group_road<G, EXT>(mine, s, l, chamber, H.cbase, H.score, P, ix, vyy_max, vzz_max, dx_max, road);
        const int S = blockDim.x;
        float *pk = road + (EXT ? kRoadWords : kRoadWords - 4) * S + threadIdx.x;
        park(pk, S, s, H);
        group_scan<G, NH, EXT>(mine, l, P, ix, gmask, H.trig, road, L);
        unpark(pk, S, s, H);
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
        if (!L.empty()) {
            my_score = L.head_score();
            my_id = L.head_id();
            my_pos = L.head_pos();
            my_chi2 = L.head_chi2();
            kept = 1;
        }
    } else {
        for (int rr = 0; rr < P.nhyp; ++rr) {
            // group minimum of the lanes' heads in (score, parent, id) order
            // (two shuffles a step); the keys of the lanes' heads are
            // distinct, so the holder is the lane whose head equals the minimum
            const unsigned long long mine = L.head_key();
            unsigned long long best = mine;
#pragma unroll
            for (int off = G / 2; off > 0; off >>= 1) {
                const unsigned long long o = __shfl_xor_sync(gmask, best, off, G);
                best = o < best ? o : best;
            }
            if (best == kNoKey) break;
            const float bs = key_score(best);
            const int bp = key_parent(best), bid = key_id(best);
            const int bh = (__ffs(__ballot_sync(gmask, mine == best) & gmask) - 1) & (G - 1);
            const float wchi2 = __shfl_sync(gmask, L.head_chi2(), bh, G);
            const int wpos = __shfl_sync(gmask, L.head_pos(), bh, G);
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
            if (G == 1)
                stage_result_noids(res, pos, b, H.chisum, H.ntrk, H.nmiss, any_live ? TRD_ST_STOPPED : TRD_ST_PROP_FAIL);
            else
                stage_result(res, pos, b, H.chisum, H.ntrk, H.nmiss, any_live ? TRD_ST_STOPPED : TRD_ST_PROP_FAIL, H.ids);
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
        if (G == 1) {
            if (idl >= 0) reinterpret_cast<int *>(res + 8 * static_cast<size_t>(pos))[26 + l] = idl;
        } else {
#pragma unroll
            for (int k = 0; k < kLayers; ++k) H.ids[k] = k == l ? idl : H.ids[k];
        }
    }
    if (l == kLayers - 1) {
        if (q == 0) {
            if (G == 1)
                stage_result_noids(res, pos, s, H.chisum, H.ntrk, H.nmiss, TRD_ST_OK);
            else
                stage_result(res, pos, s, H.chisum, H.ntrk, H.nmiss, TRD_ST_OK, H.ids);
        }
        return true;
    }
    return false;
}

// Persistent, layer-synchronous follower: a warp takes 32 / G consecutive
// sorted positions (seeds of similar momentum; G lanes per seed) with one
// atomic and carries its seeds through the six layers together, so every
// group of the warp runs the same layer's code at the same time: the seed
// loads, the layer's transport, road set-up and update, the merge of the
// groups' lists and the result stores are issued once per warp instead of
// once per group whose seed happens to be at that step.  A group whose seed
// ended waits for the warp's last layer.  The snapshot of each group's state
// before the layer's transport sits in shared memory (24 floats per group).
template <int G, int NH, int MINB, bool EXT>
__global__ void __launch_bounds__(128, MINB)
k_follow(SeedsView sv, IndexView ix, Params P, ParkedView pk, int *counter)
{
    wait_prior_grid();
    extern __shared__ float smem[];
    const int groups = blockDim.x / G;
    const int g = threadIdx.x / G;
    const int q = G == 1 ? 0 : (threadIdx.x & (G - 1));
    const int lane = threadIdx.x & 31;
    const unsigned gmask = G == 32 ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    float *sm = smem + g;
    float *road = smem + 24 * groups;  // the group scan's road table and parked states
    const float vyy_max = __uint_as_float(__ldg(&ix.stats[0]));
    const float vzz_max = __uint_as_float(__ldg(&ix.stats[1]));
    const float dx_max = EXT && ix.recx ? __uint_as_float(__ldg(&ix.stats[3])) : 0.0f;
    for (;;) {
        int base = 0;
        if (lane == 0) base = atomicAdd(counter, 32 / G);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (base >= sv.n) break;
        const int pos = base + lane / G;
        Lane H;
        int i;
        bool have = pos < sv.n && start_seed<G>(pos, q, sv, pk, H, i);
        for (int l = 0; l < kLayers && __any_sync(0xffffffffu, have); ++l) {
            if (have && layer_step<G, NH, EXT, parks(G, MINB)>(pos, l, q, gmask, ix, P, pk.rec, sm, groups, road, vyy_max,
                                               vzz_max, dx_max, H))
                have = false;
        }
    }
}

// The staged results to the seeds' input positions: thread i reads its
// seed's 128-byte record and writes the result arrays with full lines.  Seeds
// that ended in k_seed_prepare (inv -1) already have their results.
__global__ void __launch_bounds__(256) k_results_gather(int n, ParkedView pk, ResultsView o)
{
    wait_prior_grid();
    __shared__ float s_res[256 / 32][32][33];  // each warp's 32 records (odd row: no bank conflicts)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int pos = i < n ? pk.inv[i] : -1;
    // record j of the warp read by all lanes, one 128-byte line per load,
    // sixteen lines in flight at a time (a seed that ended in the pre-pass
    // reads record 0 in its place, and its row is not used)
    const float *recw = reinterpret_cast<const float *>(pk.rec);
#pragma unroll
    for (int j0 = 0; j0 < 32; j0 += 16) {
        float v[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const int pj = max(__shfl_sync(0xffffffffu, pos, j0 + u), 0);
            v[u] = recw[32 * static_cast<size_t>(pj) + lane];
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) s_res[w][j0 + u][lane] = v[u];
    }
    __syncwarp();
    if (pos < 0) return;
    const float *r = s_res[w][lane];
    o.alpha[i] = r[0];
    o.x[i] = r[1];
#pragma unroll
    for (int k = 0; k < 5; ++k) o.par[k * n + i] = r[2 + k];
#pragma unroll
    for (int k = 0; k < 15; ++k) o.cov[k * n + i] = r[7 + k];
    o.chi2[i] = r[22];
    o.ntrk[i] = __float_as_int(r[23]);
    o.nmiss[i] = __float_as_int(r[24]);
    o.status[i] = __float_as_int(r[25]);
#pragma unroll
    for (int l = 0; l < kLayers; ++l) o.ids[l * n + i] = __float_as_int(r[26 + l]);
}

}  // namespace trd

namespace trd_host {

using namespace trd;

// The seeds' pre-pass: bins and ranks, then the rotated states parked in
// sorted order.
static int prepare_kernels(const SeedsView &sv, const Params &P, const ResultsView &o, const ParkedView &pk,
                           int *counter, cudaStream_t s)
{
    TRD_CUDA_TRY(cudaMemsetAsync(pk.bin_count, 0, sizeof(int32_t) * pk.nbins, s));
    const int per_block = kKeyThreads * kKeyItems;
    k_seed_key<<<(sv.n + per_block - 1) / per_block, kKeyThreads, 0, s>>>(sv.q2pt, sv.n, sv.soff, sv.n_tf, pk,
                                                                           counter);
    TRD_CUDA_TRY(cudaGetLastError());
    TRD_CUDA_TRY(launch_after(k_seed_prepare, dim3((sv.n + 255) / 256), dim3(256), 0, s, sv, P, o, pk));
    return TRD_OK;
}

template <int G, int NH, int MINB, bool EXT>
static int launch(const trd_ctx *ctx, const SeedsView &sv, const IndexView &ix, const Params &P,
                  const ResultsView &o, const ParkedView &pk, cudaStream_t s, int block, int *counter, bool prepare,
                  const KernelEvents *kev)
{
    if (sv.n == 0) {
        if (kev) {  // no kernel: an empty interval
            TRD_CUDA_TRY(cudaEventRecord(kev->start, s));
            TRD_CUDA_TRY(cudaEventRecord(kev->end, s));
        }
        return TRD_OK;
    }
    const int groups = block / G;
    // snapshots (24 floats per group), then the group scan's road table
    const size_t smem =
        sizeof(float) * (24 * groups + (parks(G, MINB) ? ((EXT ? kRoadWords : kRoadWords - 4) + kParkWords) * block : 0));
    void (*kernel)(SeedsView, IndexView, Params, ParkedView, int *) = k_follow<G, NH, MINB, EXT>;
    int per_sm = 0;
    TRD_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, block, smem));
    per_sm = per_sm > 0 ? per_sm : 1;
    const long long need = (static_cast<long long>(sv.n) + groups - 1) / groups;
    const int grid = static_cast<int>(std::min<long long>(need, static_cast<long long>(ctx->sm_count) * per_sm));
    // the work counter is zeroed by the pre-pass (here, or on the caller's
    // branch when prepare is false)
    if (prepare) {
        const int rc = prepare_kernels(sv, P, o, pk, counter, s);
        if (rc) return rc;
    }
    // the follower and the gather start while their predecessor drains
    // (except around the events of a timed call)
    if (kev) TRD_CUDA_TRY(cudaEventRecord(kev->start, s));
    TRD_CUDA_TRY(launch_after(kernel, dim3(grid), dim3(block), smem, s, sv, ix, P, pk, counter));
    if (kev) TRD_CUDA_TRY(cudaEventRecord(kev->end, s));
    TRD_CUDA_TRY(launch_after(k_results_gather, dim3((sv.n + 255) / 256), dim3(256), 0, s, sv.n, pk, o));
    return TRD_OK;
}

template <bool EXT>
static int dispatch(const trd_ctx *ctx, const SeedsView &sv, const IndexView &iv, const Params &P,
                    const ResultsView &o, const ParkedView &pk, cudaStream_t s, int G, int mb, int block, int nhyp,
                    int *counter, bool prepare, const KernelEvents *kev)
{
#define TRD_LAUNCH(g, nh, m) launch<g, nh, m, EXT>(ctx, sv, iv, P, o, pk, s, block, counter, prepare, kev)
    switch (G * 16 + mb) {
    case 1 * 16 + 4: return nhyp == 1 ? TRD_LAUNCH(1, 1, 4) : TRD_EINVAL;
    case 1 * 16 + 5: return nhyp == 1 ? TRD_LAUNCH(1, 1, 5) : TRD_EINVAL;
    case 1 * 16 + 6: return nhyp == 1 ? TRD_LAUNCH(1, 1, 6) : TRD_EINVAL;
    case 1 * 16 + 8: return nhyp == 1 ? TRD_LAUNCH(1, 1, 8) : TRD_EINVAL;
    case 2 * 16 + 3: return TRD_LAUNCH(2, 2, 3);
    case 2 * 16 + 4: return TRD_LAUNCH(2, 2, 4);
    case 2 * 16 + 5: return TRD_LAUNCH(2, 2, 5);
    case 2 * 16 + 6: return TRD_LAUNCH(2, 2, 6);
    // up to three hypotheses in a group of 4: lists of 3
    case 4 * 16 + 3: return nhyp <= 3 ? TRD_LAUNCH(4, 3, 3) : TRD_LAUNCH(4, 4, 3);
    case 4 * 16 + 4: return nhyp <= 3 ? TRD_LAUNCH(4, 3, 4) : TRD_LAUNCH(4, 4, 4);
    case 4 * 16 + 5: return nhyp <= 3 ? TRD_LAUNCH(4, 3, 5) : TRD_LAUNCH(4, 4, 5);
    case 4 * 16 + 6: return nhyp <= 3 ? TRD_LAUNCH(4, 3, 6) : TRD_LAUNCH(4, 4, 6);
    // up to six hypotheses in a group of 8: lists of 6 (fewer registers)
    case 8 * 16 + 3: return nhyp <= 6 ? TRD_LAUNCH(8, 6, 3) : TRD_LAUNCH(8, 8, 3);
    case 8 * 16 + 4: return nhyp <= 6 ? TRD_LAUNCH(8, 6, 4) : TRD_LAUNCH(8, 8, 4);
    case 8 * 16 + 5: return nhyp <= 6 ? TRD_LAUNCH(8, 6, 5) : TRD_LAUNCH(8, 8, 5);
    case 8 * 16 + 6: return nhyp <= 6 ? TRD_LAUNCH(8, 6, 6) : TRD_LAUNCH(8, 8, 6);
    case 32 * 16 + 3: return TRD_LAUNCH(32, 8, 3);
    case 32 * 16 + 4: return TRD_LAUNCH(32, 8, 4);
    default: return TRD_EINVAL;
    }
#undef TRD_LAUNCH
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

size_t parked_bytes(int32_t n, int32_t n_tf) { return n > 0 ? sizeof(int32_t) * parked_words(n, n_tf) : 0; }

// The seeds' pre-pass alone (it does not read the index, so a captured step
// can run it beside the index build).  parked: parked_bytes(n) of device
// memory; counter: the work counter of the follower launch that follows.
int prepare_launch(const trd_seeds_t *seeds, const trd_params_t *p, trd_results_t *out, cudaStream_t s,
                   void *parked, int *counter, const int32_t *seed_offsets, int n_tf, const trd_alignment_t *align)
{
    if (seeds->n == 0) return TRD_OK;
    if (!parked) return TRD_EINVAL;
    const int ntf = seed_offsets ? n_tf : 1;
    if (!counter) counter = parked_view(parked, seeds->n, ntf).counter;
    SeedsView sv{seeds->alpha, seeds->x, seeds->y, seeds->z, seeds->snp, seeds->tgl, seeds->q2pt, seeds->cov,
                 seeds->n, seed_offsets, seed_offsets ? n_tf : 1, seeds->trigger};
    const Params P = make_params(p, align);
    ResultsView o{out->alpha, out->x, out->par, out->cov, out->chi2, out->n_trk, out->n_miss, out->status,
                  out->tracklet_id};
    return prepare_kernels(sv, P, o, parked_view(parked, seeds->n, ntf), counter, s);
}

int follow_launch(const trd_ctx *ctx, const trd_seeds_t *seeds, const IndexView &iv, const trd_params_t *p,
                  trd_results_t *out, cudaStream_t s, int lanes_per_track, int block_threads, int min_blocks,
                  int *counter, const int32_t *seed_offsets, int n_tf, const trd_alignment_t *align,
                  bool prepare, void *parked, const KernelEvents *kev)
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
    // the selection keys hold 28-bit tracklet ids
    if (iv.max_tf_tracklets >= static_cast<int32_t>(trd::kKeyIdMask)) return TRD_EINVAL;
    // default register budget: the fastest on the benchmark's workloads
    // (one lane: 4 blocks per SM; groups of 2 and 4 with parked states: 6;
    // groups of 8: 5; whole warps: 4)
    const int mb = min_blocks > 0 ? min_blocks : (G == 1 || G == 32 ? 4 : (G == 8 ? 5 : 6));
    // without a caller scratch: one from the device's pool, ordered on s
    void *own = nullptr;
    if (sv.n > 0 && !parked) {
        if (!prepare) return TRD_EINVAL;  // the pre-pass's output is needed
        if (cudaMallocAsync(&own, parked_bytes(sv.n, sv.n_tf), s) != cudaSuccess) {
            (void)cudaGetLastError();
            return TRD_ENOMEM;
        }
        parked = own;
    }
    const ParkedView pk = sv.n > 0 ? parked_view(parked, sv.n, sv.n_tf) : ParkedView{};
    if (!counter) counter = pk.counter;  // the call's own, inside its scratch
    const int rc = ext ? dispatch<true>(ctx, sv, iv, P, o, pk, s, G, mb, block, p->n_hyp, counter, prepare, kev)
                       : dispatch<false>(ctx, sv, iv, P, o, pk, s, G, mb, block, p->n_hyp, counter, prepare, kev);
    if (own && cudaFreeAsync(own, s) != cudaSuccess) {
        (void)cudaGetLastError();
        return rc ? rc : TRD_ECUDA;
    }
    return rc;
}

}  // namespace trd_host
