// trd_device.cuh -- device-side building blocks of the FP32 TRD follower
// (arXiv:2003.03174, Sec. 3).  Everything here runs in FP32; constants that
// need more than 24 bits (layer radii, sector azimuths, 2*pi) are stored as
// unevaluated sums of two floats computed at compile time, and the track
// position (x, y) is carried the same way, because a chi2 of y against a
// 0.04 cm tracklet resolution is sensitive to 1e-5 cm while an FP32 value
// near 300 cm has a spacing of 3e-5 cm.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace trd {

// Programmatic dependent launch: a kernel launched after another in the same
// stream with the programmatic-serialization attribute (trd_host::launch_after)
// may have its blocks start while its predecessor is still running; it calls
// wait_prior_grid() before touching any memory the predecessor reads or
// writes, and that returns once the predecessor has completed and its writes
// are visible.  In a kernel launched the ordinary way it returns at once.
__device__ __forceinline__ void wait_prior_grid() { asm volatile("griddepcontrol.wait;" ::: "memory"); }


// ---- geometry (Sec. 3: 18 sectors x 5 stacks x 6 layers; radii, pad rows
// and material are readings) ------------------------------------------------
constexpr int kLayers = 6;
constexpr int kSectors = 18;
constexpr int kStacks = 5;
constexpr int kChambers = kSectors * kStacks * kLayers;  // 540
constexpr int kRowsPerStack = 18;
constexpr float kRowLength = 8.0f;
constexpr float kStackLength = 144.0f;
constexpr float kZMin = -360.0f;
constexpr float kYHalf = 66.0f;  // index y range: |y| <= 66 cm covers x*tan(10 deg) at 363 cm
constexpr float kMaxSnp = 0.95f;
constexpr float kCLight = 2.99792458e-3f;
constexpr float kDriftLength = 3.0f;
constexpr int kMissing = 0x7fffffff;

constexpr double kPiD = 3.14159265358979323846;
constexpr double kXLayerD(int l) { return 300.0 + 12.6 * l; }
constexpr double kSectorAlphaD(int s) { return (s + 0.5) * (2.0 * kPiD / 18.0); }
constexpr float hi_of(double v) { return static_cast<float>(v); }
constexpr float lo_of(double v) { return static_cast<float>(v - static_cast<double>(static_cast<float>(v))); }

// material reading: x/X0 = 0.04 and 1 g/cm^2 per layer at normal incidence
constexpr float kX0Fraction = 0.04f;
constexpr float kXRho = 1.0f;
constexpr float kMassPion = 0.13957039f;
constexpr float kTwoMeOverI = static_cast<float>(2.0 * 0.51099895e-3 / 100e-9);  // 2 m_e c^2 / I
constexpr float kBetheKZA = static_cast<float>(0.307075 * 0.5 * 1e-3);            // GeV cm^2/g
// resolution reading (best near the Lorentz angle, Sec. 3 / Fig. 3)
constexpr float kSigDy0 = 0.04f, kSigDy1 = 0.1f;
constexpr float kSigY0 = 0.03f, kSigY1 = 0.05f;

__device__ __forceinline__ float layer_tilt_tan(int l)
{
    // +2 degrees on even layers, -2 on odd (reading of "tilted by +-2 degrees")
    constexpr float t = hi_of(0.034920769491747931);  // tan(2 deg)
    return (l & 1) ? -t : t;
}

__device__ __forceinline__ float lorentz_tan(float bz)
{
    constexpr float t = hi_of(0.14054083470239145);  // tan(8 deg)
    return bz >= 0.0f ? t : -t;
}

__device__ __forceinline__ float half_sector_tan()
{
    constexpr float t = hi_of(0.17632698070846498);  // tan(10 deg)
    return t;
}

// ---- double-float arithmetic (Knuth's two-sum; Dekker's product via FMA) ---
struct df {
    float hi, lo;
};

__device__ __forceinline__ df two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df quick_two_sum(float a, float b)
{
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df df_add_f(df a, float b)
{
    df s = two_sum(a.hi, b);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df df_add(df a, df b)
{
    df s = two_sum(a.hi, b.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ df df_neg(df a) { return {-a.hi, -a.lo}; }

// a * b with a double-float, b double-float (low-order cross terms only)
__device__ __forceinline__ df df_mul(df a, df b)
{
    float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return quick_two_sum(p, e);
}

__device__ __forceinline__ df df_mul_f(df a, float b)
{
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return quick_two_sum(p, e);
}

__device__ __forceinline__ float df_to_f(df a) { return __fadd_rn(a.hi, a.lo); }

template <int L>
struct LayerX {
    static constexpr float hi = hi_of(kXLayerD(L));
    static constexpr float lo = lo_of(kXLayerD(L));
};

__device__ __forceinline__ df layer_x_df(int l)
{
    // x_l = 300 + 12.6 l, split into two floats at compile time
    switch (l) {
    case 0: return {LayerX<0>::hi, LayerX<0>::lo};
    case 1: return {LayerX<1>::hi, LayerX<1>::lo};
    case 2: return {LayerX<2>::hi, LayerX<2>::lo};
    case 3: return {LayerX<3>::hi, LayerX<3>::lo};
    case 4: return {LayerX<4>::hi, LayerX<4>::lo};
    default: return {LayerX<5>::hi, LayerX<5>::lo};
    }
}

constexpr float kSectorWidthHi = hi_of(2.0 * kPiD / 18.0);
constexpr float kSectorWidthLo = lo_of(2.0 * kPiD / 18.0);
constexpr float kTwoPiHi = hi_of(2.0 * kPiD);
constexpr float kTwoPiLo = lo_of(2.0 * kPiD);

__device__ __forceinline__ df sector_alpha_df(int s)
{
    // (s + 0.5) * w with s + 0.5 exact in FP32
    return df_mul({kSectorWidthHi, kSectorWidthLo}, {static_cast<float>(s) + 0.5f, 0.0f});
}

// sin(d) as a double-float and 1 - cos(d) as a float, for |d| <= ~0.6 rad,
// from their Taylor series (d given as a double-float): the leading term of
// sin is kept exact and the tails are summed in FP32.
__device__ __forceinline__ void sincos_small(df d, df *s, float *omc)
{
    const float x = d.hi;
    const float x2 = x * x;
    const float tail = x * x2 * (-1.0f / 6.0f + x2 * (1.0f / 120.0f + x2 * (-1.0f / 5040.0f + x2 * (1.0f / 362880.0f))));
    *s = df_add_f(d, tail);
    *omc = x2 * (0.5f + x2 * (-1.0f / 24.0f + x2 * (1.0f / 720.0f + x2 * (-1.0f / 40320.0f + x2 * (1.0f / 3628800.0f))))) +
           x * d.lo;
}

// ---- track state ------------------------------------------------------------
struct TrackState {
    df x, y;         // reference radius and local y (double-float)
    float z, f, t, k;  // z, sin(phi), tan(lambda), q/pT
    float c[15];     // covariance, lower triangle row by row
    int sector;      // sector of the local frame (alpha = sector centre)
};

__device__ __forceinline__ int cidx(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

// ---- index bucketing (shared by the index build and the road query; the
// same monotone FP32 expressions on both sides keep the query a superset) ---
__device__ __forceinline__ int stack_of_chamber(int ch) { return (ch / kLayers) % kStacks; }

__device__ __forceinline__ float stack_z_lo(int stack) { return kZMin + kStackLength * static_cast<float>(stack); }

__device__ __forceinline__ int row_of_z(float z, float z_lo)
{
    float u = floorf((z - z_lo) * (1.0f / kRowLength));
    u = fminf(fmaxf(u, 0.0f), static_cast<float>(kRowsPerStack - 1));
    return static_cast<int>(u);
}

// Bucket order: chamber, then pad row, then y bin, so that the y bins of one
// pad row are adjacent and a road query reads one contiguous range per pad
// row, however narrow the bins.
__device__ __forceinline__ int bucket_of(int chamber, int ybin, int row, int nb)
{
    return (chamber * kRowsPerStack + row) * nb + ybin;
}

// Timeframe of element i in a batch laid out by offsets off[0..n_tf]
// (off[0] = 0, non-decreasing): the last t with off[t] <= i.  A single
// timeframe passes off = nullptr.
__device__ __forceinline__ int tf_of(int i, const int32_t *__restrict__ off, int n_tf)
{
    if (!off) return 0;
    int lo = 0, hi = n_tf - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&off[mid]) <= i)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int ybin_of(float y, float inv_w, int nb)
{
    float u = floorf((y + kYHalf) * inv_w);
    u = fminf(fmaxf(u, 0.0f), static_cast<float>(nb - 1));
    return static_cast<int>(u);
}

}  // namespace trd
