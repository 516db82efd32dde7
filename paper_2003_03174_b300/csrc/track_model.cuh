// track_model.cuh -- the FP32 track model shared by the follower and the
// refit (arXiv:2003.03174, Sec. 3): exact helix transport in a homogeneous
// Bz with its Jacobian sandwich, rotation into another sector frame, the
// material step, and the Kalman update of a tilted-pad tracklet.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "trd_device.cuh"

namespace trd {

// ---- transport (exact helix in homogeneous Bz) -----------------------------
// sin(phi) grows linearly with x at rate rho = -c Bz q/pT; the chord has
// slope (f0+f1)/(r0+r1); the arc is chord * asin(w)/w with w = rho chord / 2.
static __device__ __forceinline__ void asin_over_series(float w, float *g, float *dg)
{
    const float w2 = w * w;
    if (fabsf(w) < 0.3f) {
        *g = 1.0f + w2 * (1.0f / 6.0f + w2 * (3.0f / 40.0f + w2 * (5.0f / 112.0f + w2 * (35.0f / 1152.0f))));
        *dg = w * (1.0f / 3.0f + w2 * (0.3f + w2 * (15.0f / 56.0f + w2 * (35.0f / 144.0f))));
    } else {
        const float a = asinf(w);
        *g = a / w;
        *dg = (w * rsqrtf(1.0f - w2) - a) / w2;
    }
}

// FULL = false transports only the covariance terms a residual needs (the
// (y, z) block and the sin(phi), tan(lambda) variances); the other terms are
// then left stale.
template <bool FULL>
static __device__ bool propagate_t(TrackState &s, df xk, float bz)
{
    const float dx = df_to_f(df_add(xk, df_neg(s.x)));
    const float f0 = s.f;
    const float drho_dk = -kCLight * bz;
    const float rho = drho_dk * s.k;
    const float f1 = fmaf(rho, dx, f0);
    if (!(fabsf(f0) < kMaxSnp) || !(fabsf(f1) < kMaxSnp)) return false;
    const float r0 = sqrtf((1.0f - f0) * (1.0f + f0));
    const float r1 = sqrtf((1.0f - f1) * (1.0f + f1));
    const float rs = r0 + r1;
    const float irs = 1.0f / rs;
    const float fs = f0 + f1;
    const float h = fs * irs;
    const float q = sqrtf(fmaf(h, h, 1.0f));
    const float chord = dx * q;
    const float w = 0.5f * rho * chord;
    float g, dg;
    asin_over_series(w, &g, &dg);
    const float arc = chord * g;

    const float irs2 = irs * irs;
    const float dh_df0 = (rs + fs * f0 / r0) * irs2;
    const float dh_df1 = (rs + fs * f1 / r1) * irs2;
    const float ds_df0 = dx * fs / (r0 * r1 * rs);
    const float dchord_drho = dx * (h / q) * dh_df1 * dx;
    const float ds_drho = dchord_drho * fmaf(w, dg, g) + 0.5f * chord * chord * dg;
    const float a = dx * (dh_df0 + dh_df1);  // dy/dsnp
    const float b = dx * dh_df1 * drho_dk * dx;  // dy/dk
    const float c = s.t * ds_df0;            // dz/dsnp
    const float d = arc;                     // dz/dtgl
    const float e = s.t * ds_drho * drho_dk; // dz/dk
    const float gg = drho_dk * dx;           // dsnp/dk

    s.x = xk;
    s.y = df_add_f(s.y, dx * h);
    s.z = fmaf(s.t, arc, s.z);
    s.f = f1;

    // C <- J C J^T with J = I except rows y (a, b), z (c, d, e), snp (gg)
    float *C = s.c;
    const float C00 = C[0], C10 = C[1], C11 = C[2], C20 = C[3], C21 = C[4], C22 = C[5], C30 = C[6], C31 = C[7],
                C32 = C[8], C33 = C[9], C40 = C[10], C41 = C[11], C42 = C[12], C43 = C[13], C44 = C[14];
    if (!FULL) {
        const float T00 = C00 + a * C20 + b * C40, T02 = C20 + a * C22 + b * C42, T04 = C40 + a * C42 + b * C44;
        const float T10 = C10 + c * C20 + d * C30 + e * C40;
        const float T11 = C11 + c * C21 + d * C31 + e * C41;
        const float T12 = C21 + c * C22 + d * C32 + e * C42;
        const float T13 = C31 + c * C32 + d * C33 + e * C43;
        const float T14 = C41 + c * C42 + d * C43 + e * C44;
        C[0] = T00 + a * T02 + b * T04;
        C[1] = T10 + a * T12 + b * T14;
        C[2] = T11 + c * T12 + d * T13 + e * T14;
        C[5] = (C22 + gg * C42) + gg * (C42 + gg * C44);
        return true;
    }
    // T = J C (rows 0..2)
    const float T00 = C00 + a * C20 + b * C40, T02 = C20 + a * C22 + b * C42, T04 = C40 + a * C42 + b * C44;
    const float T10 = C10 + c * C20 + d * C30 + e * C40;
    const float T11 = C11 + c * C21 + d * C31 + e * C41;
    const float T12 = C21 + c * C22 + d * C32 + e * C42;
    const float T13 = C31 + c * C32 + d * C33 + e * C43;
    const float T14 = C41 + c * C42 + d * C43 + e * C44;
    const float T20 = C20 + gg * C40, T21 = C21 + gg * C41, T22 = C22 + gg * C42, T23 = C32 + gg * C43,
                T24 = C42 + gg * C44;
    C[0] = T00 + a * T02 + b * T04;
    C[1] = T10 + a * T12 + b * T14;
    C[2] = T11 + c * T12 + d * T13 + e * T14;
    C[3] = T20 + a * T22 + b * T24;
    C[4] = T21 + c * T22 + d * T23 + e * T24;
    C[5] = T22 + gg * T24;
    C[6] = C30 + a * C32 + b * C43;
    C[7] = C31 + c * C32 + d * C33 + e * C43;
    C[8] = C32 + gg * C43;
    // C[9] = C33 unchanged
    C[10] = C40 + a * C42 + b * C44;
    C[11] = C41 + c * C42 + d * C43 + e * C44;
    C[12] = C42 + gg * C44;
    // C[13] = C43, C[14] = C44 unchanged
    return true;
}

static __device__ __forceinline__ bool propagate(TrackState &s, df xk, float bz) { return propagate_t<true>(s, xk, bz); }

// ---- rotation into another sector frame ------------------------------------
// Exact rotation of the point (double-float), first-order transform of the
// covariance onto the new plane x' = const (slide along the track):
// dy'/dy = r/r', dz'/dy = -tgl sin(d)/r', dsnp'/dy = -rho sin(d), dsnp'/dsnp = r'/r.
static __device__ bool rotate(TrackState &s, df delta, int new_sector, float bz)
{
    df sn;
    float omc;
    if (fabsf(delta.hi) < 0.6f) {
        sincos_small(delta, &sn, &omc);
    } else {
        // rare (seed frame far from its sector): halve the angle into the
        // series' range, then apply sin 2a = 2 sin a cos a, 1 - cos 2a = 2 sin^2 a
        int halvings = 0;
        df h = delta;
        while (fabsf(h.hi) >= 0.3f && halvings < 6) {
            h = {0.5f * h.hi, 0.5f * h.lo};
            ++halvings;
        }
        sincos_small(h, &sn, &omc);
        for (int k = 0; k < halvings; ++k) {
            const float sf = df_to_f(sn);
            const float nomc = 2.0f * sf * sf;
            sn = df_mul_f(sn, 2.0f * (1.0f - omc));
            omc = nomc;
        }
    }
    const float snf = df_to_f(sn);
    const float f = s.f;
    const float r = sqrtf((1.0f - f) * (1.0f + f));
    const float fn = f - f * omc - r * snf;
    const float rn = r - r * omc + f * snf;
    if (!(fabsf(fn) < kMaxSnp) || !(rn > 0.0f)) return false;
    const float rho = -kCLight * bz * s.k;
    const float p = r / rn, qq = -s.t * snf / rn, u = -rho * snf, v = rn / r;

    const df x = s.x, y = s.y;
    // x' = x cos d + y sin d ; y' = -x sin d + y cos d   (cos d = 1 - omc)
    s.x = df_add(df_add(x, df_neg(df_mul_f(x, omc))), df_mul(y, sn));
    s.y = df_add(df_add(y, df_neg(df_mul_f(y, omc))), df_neg(df_mul(x, sn)));
    s.f = fn;
    s.sector = new_sector;

    float *C = s.c;
    const float C00 = C[0], C10 = C[1], C11 = C[2], C20 = C[3], C21 = C[4], C22 = C[5], C30 = C[6], C31 = C[7],
                C32 = C[8], C40 = C[10], C41 = C[11], C42 = C[12];
    const float T10 = qq * C00 + C10;
    const float T20 = u * C00 + v * C20;
    const float T21 = u * C10 + v * C21;
    const float T22 = u * C20 + v * C22;
    C[0] = p * p * C00;
    C[1] = p * T10;
    C[2] = qq * T10 + qq * C10 + C11;
    C[3] = p * T20;
    C[4] = qq * T20 + T21;
    C[5] = u * T20 + v * T22;
    C[6] = p * C30;
    C[7] = qq * C30 + C31;
    C[8] = u * C30 + v * C32;
    C[10] = p * C40;
    C[11] = qq * C40 + C41;
    C[12] = u * C40 + v * C42;
    return true;
}

// ---- material step (reading: Highland scattering + Bethe loss of a pion) ----
// INWARD = false: a track moving outward, the mean loss is subtracted;
// INWARD = true: a track moving inward (the refit), the loss is added back.
// Scattering at the entry momentum widens the sin(phi), tan(lambda), q/pT
// block; the loss changes |p| to p', so q/pT becomes sign(q) sqrt(1+tgl^2)/p'
// and the covariance is carried through that change by its Jacobian (the
// loss depends on q/pT through p and the slope of the Bethe curve, on sin(phi)
// and tan(lambda) through the path length, and tan(lambda) also enters p).
template <bool INWARD>
static __device__ bool material(TrackState &s)
{
    const float f = s.f, t = s.t, k = s.k;
    if (k == 0.0f) return true;
    const float r2 = (1.0f - f) * (1.0f + f);
    const float r = sqrtf(r2);
    const float t2 = fmaf(t, t, 1.0f);
    const float st2 = sqrtf(t2);
    const float path = st2 / r;
    const float xx0 = kX0Fraction * path;
    const float p = st2 / fabsf(k);
    const float m2 = kMassPion * kMassPion;
    const float e = sqrtf(fmaf(p, p, m2));
    const float beta = p / e;
    const float t0 = 0.0136f / (beta * p);
    const float lg = fmaf(0.038f, __logf(xx0), 1.0f);
    const float th2 = t0 * t0 * xx0 * lg * lg;
    float *C = s.c;
    C[5] += th2 * r2 * t2;
    C[9] += th2 * t2 * t2;
    C[13] += th2 * t * t2 * k;
    C[14] += th2 * t * t * k * k;
    const float bg = p / kMassPion;
    const float bg2 = bg * bg;
    const float b2 = bg2 / (1.0f + bg2);
    const float ib2 = 1.0f + 1.0f / bg2;  // 1 / beta^2
    const float brk = __logf(kTwoMeOverI * bg2) - b2;
    const float dedx = kBetheKZA * ib2 * brk;  // GeV cm^2/g
    // d(dedx)/d(bg) = K Z/A (d(1/beta^2)/dbg * brk + 1/beta^2 * d(brk)/dbg)
    const float ddedx = kBetheKZA * (-2.0f / (bg2 * bg) * brk + ib2 * (2.0f / bg - 2.0f * b2 * (1.0f - b2) / bg));
    const float de = dedx * kXRho * path;
    const float e1 = INWARD ? e + de : e - de;
    if (!(e1 > kMassPion)) return false;
    const float p1 = sqrtf((e1 - kMassPion) * (e1 + kMassPion));
    const float k1 = k * (p / p1);
    // d q2pt' / d(snp, tgl, q2pt) = q2pt' (d ln sqrt(1+tgl^2) - e1/p1^2 d e1), with
    // d e1 = (p/e) dp -+ d de, dp = (0, p tgl/t2, -p/q2pt), dpath = (path snp/r^2, path tgl/t2, 0)
    const float tt2 = t / t2;
    const float sgn = INWARD ? -1.0f : 1.0f;                    // e1 = e - sgn de
    const float slope = ddedx * kXRho * path * (1.0f / kMassPion);  // d de / dp
    const float w = k1 * e1 / (p1 * p1);
    const float de1_df = -sgn * dedx * kXRho * path * f / r2;
    const float dp_dt = p * tt2;
    const float de1_dt = (p / e) * dp_dt - sgn * (slope * dp_dt + de * tt2);
    const float dp_dk = -p / k;
    const float de1_dk = (p / e - sgn * slope) * dp_dk;
    const float ja = -w * de1_df;             // d q2pt' / d snp
    const float jb = k1 * tt2 - w * de1_dt;   // d q2pt' / d tgl
    const float jc = -w * de1_dk;             // d q2pt' / d q2pt
    s.k = k1;
    // C <- J C J^T with J = I except row 4 = (0, 0, ja, jb, jc)
    const float C20 = C[3], C21 = C[4], C22 = C[5], C30 = C[6], C31 = C[7], C32 = C[8], C33 = C[9];
    const float C40 = C[10], C41 = C[11], C42 = C[12], C43 = C[13], C44 = C[14];
    C[10] = ja * C20 + jb * C30 + jc * C40;
    C[11] = ja * C21 + jb * C31 + jc * C41;
    C[12] = ja * C22 + jb * C32 + jc * C42;
    C[13] = ja * C32 + jb * C33 + jc * C43;
    C[14] = ja * (ja * C22 + 2.0f * (jb * C32 + jc * C42)) + jb * (jb * C33 + 2.0f * jc * C43) + jc * jc * C44;
    return true;
}

// ---- Kalman update, Joseph form, symmetrised --------------------------------
// Measurement (y_tl, z_tl) with pad tilt: h(p) = (y - tt (z - z_tl), z).
// Returns the chi2 of the predicted residual, r^T S^-1 r.
static __device__ float kalman_update(TrackState &s, float tt, float ytl, float ztl, float vyy, float vzz, float vyz)
{
    float *C = s.c;
    const float r0 = (__fsub_rn(ytl, s.y.hi) - s.y.lo) + tt * (s.z - ztl);
    const float r1 = ztl - s.z;
    // C H^T (5x2): column 0 = C[:,0] - tt C[:,1], column 1 = C[:,1]
    float Ci0[5], Ci1[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        Ci0[i] = C[cidx(i, 0)];
        Ci1[i] = C[cidx(i, 1)];
    }
    float H0[5], H1[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        H0[i] = Ci0[i] - tt * Ci1[i];
        H1[i] = Ci1[i];
    }
    const float S00 = H0[0] - tt * H0[1] + vyy;
    const float S01 = H1[0] - tt * H1[1] + vyz;
    const float S11 = H1[1] + vzz;
    const float idet = 1.0f / (S00 * S11 - S01 * S01);
    const float Si00 = S11 * idet, Si01 = -S01 * idet, Si11 = S00 * idet;
    float K0[5], K1[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        K0[i] = H0[i] * Si00 + H1[i] * Si01;
        K1[i] = H0[i] * Si01 + H1[i] * Si11;
    }
    s.y = df_add_f(s.y, K0[0] * r0 + K1[0] * r1);
    s.z += K0[1] * r0 + K1[1] * r1;
    s.f += K0[2] * r0 + K1[2] * r1;
    s.t += K0[3] * r0 + K1[3] * r1;
    s.k += K0[4] * r0 + K1[4] * r1;
    // Joseph: (I - K H) C (I - K H)^T + K V K^T.  I - K H differs from I in
    // columns 0 and 1 only: A x = x - u x_0 - v x_1 with u = K0, v = K1 - tt K0.
    // B = A C is needed in columns 0, 1 and on and below the diagonal; the
    // product B A^T + K V K^T is evaluated for the lower triangle, which is
    // stored for both triangles (exactly symmetric).
    float u[5], v[5], kv0[5], kv1[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        u[i] = K0[i];
        v[i] = K1[i] - tt * K0[i];
        kv0[i] = vyy * K0[i] + vyz * K1[i];
        kv1[i] = vyz * K0[i] + vzz * K1[i];
    }
    float B0[5], B1[5];  // columns 0 and 1 of B
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        B0[i] = Ci0[i] - u[i] * Ci0[0] - v[i] * Ci1[0];
        B1[i] = Ci1[i] - u[i] * Ci0[1] - v[i] * Ci1[1];
    }
    float Nw[15];
#pragma unroll
    for (int i = 0; i < 5; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            const float bij = j == 0 ? B0[i] : (j == 1 ? B1[i] : C[cidx(i, j)] - u[i] * Ci0[j] - v[i] * Ci1[j]);
            Nw[cidx(i, j)] = bij - B0[i] * u[j] - B1[i] * v[j] + K0[i] * kv0[j] + K1[i] * kv1[j];
        }
#pragma unroll
    for (int k = 0; k < 15; ++k) C[k] = Nw[k];
    return r0 * (Si00 * r0 + Si01 * r1) + r1 * (Si01 * r0 + Si11 * r1);
}

}  // namespace trd
