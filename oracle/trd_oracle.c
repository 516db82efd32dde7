/*
 * trd_oracle.c -- FP64 CPU oracle of the TRD tracklet follower
 * (arXiv:2003.03174, Sec. 3 "TRD tracking algorithm").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, double-precision
 * statement of what the follower computes.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark call it; the product path
 * (the CUDA library) never links, loads or calls it, and the two share no
 * code, header or constant table.
 *
 * The paper describes the matching in prose only.  Every formula below that
 * the paper does not print is a reading, derived here from first principles
 * (helix geometry, the Kalman filter, the Highland and Bethe formulas):
 *
 *   track state (local frame of azimuth alpha, at radius x):
 *       p = (y, z, snp = sin(phi), tgl = tan(lambda), q2pt = q/pT)
 *   covariance: 15 terms, lower triangle row by row
 *       c00 c10 c11 c20 c21 c22 c30 c31 c32 c33 c40 c41 c42 c43 c44
 *   signed curvature rho = d(phi)/ds = -C_LIGHT * Bz * q2pt
 *       (Lorentz force: +q in +Bz bends towards -y)
 *
 * The material step (Highland + Bethe with the constants of the reading) has
 * no counterpart in the paper beyond "energy loss" (Sec. 3).  Its constants
 * are a reading; its action on the state and covariance is pinned: the
 * scattering increments against a Monte-Carlo of two projected angles
 * carried through the exact direction geometry, the energy taken out against
 * the Bethe curve over the geometric path, and the covariance transport
 * against finite differences of the state map.
 *
 * Build: gcc -O2 -fopenmp -shared -fPIC trd_oracle.c -o libtrd_oracle.so -lm
 */
#include <limits.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---- geometry and detector constants --------------------------------- */
/* Sec. 3: 18 sectors in azimuth, 5 stacks along z, 6 layers in radius.     */
#define ORA_NLAYER 6
#define ORA_NSECTOR 18
#define ORA_NSTACK 5
#define ORA_NCHAMBER (ORA_NSECTOR * ORA_NSTACK * ORA_NLAYER)
#define ORA_MAXHYP 65536
#define ORA_MISSING INT_MAX

static const double kPi = 3.14159265358979323846;
static const double kXLayer0 = 300.0;     /* reading: x_l = 300 + 12.6 l cm */
static const double kDXLayer = 12.6;
static const double kStackLength = 144.0; /* reading: 18 pad rows of 8 cm */
static const double kZMin = -360.0;
static const double kTiltDeg = 2.0;       /* Sec. 3: pads tilted by +-2 degrees */
static const double kDriftLength = 3.0;   /* Sec. 3: 3 cm drift region */
static const double kLorentzDeg = 8.0;    /* Fig. 3 caption: ~ +-8 deg at +-0.5 T */
static const double kCLight = 2.99792458e-3;
static const double kMaxSnp = 0.95;
/* material reading (one step per layer at normal incidence) */
static const double kX0Fraction = 0.04;   /* x / X0 */
static const double kXRho = 1.0;          /* g / cm^2 */
static const double kMassPion = 0.13957039; /* GeV */
static const double kMassElectron = 0.51099895e-3; /* GeV */
static const double kBetheK = 0.307075;   /* MeV cm^2 / g */
static const double kZOverA = 0.5;
static const double kIExcitation = 100e-9; /* GeV */
/* resolution reading (Sec. 3, Fig. 3: best near the Lorentz angle) */
static const double kSigDy0 = 0.04, kSigDy1 = 0.1;
static const double kSigY0 = 0.03, kSigY1 = 0.05;

static double sector_width(void) { return 2.0 * kPi / ORA_NSECTOR; }
static double layer_x(int l) { return kXLayer0 + kDXLayer * l; }
static double half_sector_tan(void) { return tan(0.5 * sector_width()); }
/* Reading: +2 degrees on even layers, -2 degrees on odd layers. */
static double tilt_tan(int l) { return tan((l % 2 == 0 ? 1.0 : -1.0) * kTiltDeg * kPi / 180.0); }
static double lorentz_tan(double bz) { return tan((bz >= 0 ? 1.0 : -1.0) * kLorentzDeg * kPi / 180.0); }

void ora_constants(double *out, int n)
{
    const double v[] = {ORA_NSECTOR, ORA_NSTACK, ORA_NLAYER, ORA_NCHAMBER, kXLayer0,
                        kDXLayer, kStackLength, kZMin, kTiltDeg, kDriftLength,
                        kLorentzDeg, kCLight, kMaxSnp};
    for (int i = 0; i < n && i < (int)(sizeof v / sizeof v[0]); ++i) out[i] = v[i];
}

/* ---- small dense algebra (plain loops) --------------------------------- */
static int ci(int i, int j) { return i >= j ? i * (i + 1) / 2 + j : j * (j + 1) / 2 + i; }

static void cov_full(const double c[15], double m[5][5])
{
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) m[i][j] = c[ci(i, j)];
}

static void cov_pack(double m[5][5], double c[15])
{
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j <= i; ++j) c[ci(i, j)] = 0.5 * (m[i][j] + m[j][i]);
}

/* c <- J c J^T */
static void cov_transport(const double J[5][5], double c[15])
{
    double m[5][5], t[5][5], r[5][5];
    cov_full(c, m);
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            double s = 0;
            for (int k = 0; k < 5; ++k) s += J[i][k] * m[k][j];
            t[i][j] = s;
        }
    for (int i = 0; i < 5; ++i)
        for (int j = 0; j < 5; ++j) {
            double s = 0;
            for (int k = 0; k < 5; ++k) s += t[i][k] * J[j][k];
            r[i][j] = s;
        }
    cov_pack(r, c);
}

static void eye5(double J[5][5])
{
    memset(J, 0, 25 * sizeof(double));
    for (int i = 0; i < 5; ++i) J[i][i] = 1.0;
}

static void put_jac(double *out, double J[5][5])
{
    if (out) memcpy(out, J, 25 * sizeof(double));
}

/* Cholesky test of positive definiteness (seed validity). */
int ora_cov_is_pd(const double c[15])
{
    double m[5][5], L[5][5] = {{0}};
    cov_full(c, m);
    for (int j = 0; j < 5; ++j) {
        double d = m[j][j];
        for (int k = 0; k < j; ++k) d -= L[j][k] * L[j][k];
        if (!(d > 0)) return 0;
        L[j][j] = sqrt(d);
        for (int i = j + 1; i < 5; ++i) {
            double s = m[i][j];
            for (int k = 0; k < j; ++k) s -= L[i][k] * L[j][k];
            L[i][j] = s / L[j][j];
        }
    }
    return 1;
}

/* asin(w)/w and its derivative, with the Taylor series for small |w|. */
static double asin_over(double w)
{
    if (fabs(w) < 1e-3) { double w2 = w * w; return 1.0 + w2 / 6.0 + 3.0 * w2 * w2 / 40.0; }
    return asin(w) / w;
}

static double asin_over_deriv(double w)
{
    if (fabs(w) < 1e-3) { double w2 = w * w; return w / 3.0 + 0.3 * w2 * w + 15.0 / 56.0 * w2 * w2 * w; }
    return (w / sqrt(1.0 - w * w) - asin(w)) / (w * w);
}

/* ---- transport: exact helix in a homogeneous Bz (Sec. 3, "precise
 * propagation"; the field map is replaced by a constant Bz) ------------------
 * st = {alpha, x, y, z, snp, tgl, q2pt}.  Moves the state to radius xk.
 * Geometry: sin(phi) changes linearly with x at the rate rho; the chord
 * between the end points has slope tan((phi0+phi1)/2) = (f0+f1)/(r0+r1); the
 * arc is the chord times asin(w)/w with w = rho * chord / 2; z advances by
 * tgl times the transverse arc.
 * Returns 0, or -1 when |snp| reaches kMaxSnp at either end or is not a
 * number (state untouched).
 * J (25 doubles, row major, optional) receives d(p1)/d(p0).                */
int ora_propagate(double st[7], double c[15], double xk, double bz, double *jac_out,
                  double *snp_slack)
{
    const double dx = xk - st[1];
    const double f0 = st[4], t = st[5], k = st[6];
    const double drho_dk = -kCLight * bz;
    const double rho = drho_dk * k;
    const double f1 = f0 + rho * dx;
    if (snp_slack) {
        double s = kMaxSnp - fmax(fabs(f0), fabs(f1));
        *snp_slack = fmin(*snp_slack, fabs(s));
    }
    /* a sin(phi) that is not a number has no place below the limit either */
    if (!(fabs(f0) < kMaxSnp) || !(fabs(f1) < kMaxSnp)) return -1;
    const double r0 = sqrt((1.0 - f0) * (1.0 + f0));
    const double r1 = sqrt((1.0 - f1) * (1.0 + f1));
    const double rs = r0 + r1;
    const double h = (f0 + f1) / rs;
    const double q = sqrt(1.0 + h * h);
    const double chord = dx * q;
    const double w = 0.5 * rho * chord;
    const double g = asin_over(w);
    const double s = chord * g;

    /* Jacobian */
    const double dh_df0 = (rs + (f0 + f1) * f0 / r0) / (rs * rs);
    const double dh_df1 = (rs + (f0 + f1) * f1 / r1) / (rs * rs);
    const double ds_df0 = dx * (f0 + f1) / (r0 * r1 * rs);
    const double dchord_drho = dx * (h / q) * dh_df1 * dx;
    const double ds_drho = dchord_drho * (g + w * asin_over_deriv(w)) +
                           0.5 * chord * chord * asin_over_deriv(w);
    double J[5][5];
    eye5(J);
    J[0][2] = dx * (dh_df0 + dh_df1);
    J[0][4] = dx * dh_df1 * drho_dk * dx;
    J[1][2] = t * ds_df0;
    J[1][3] = s;
    J[1][4] = t * ds_drho * drho_dk;
    J[2][4] = drho_dk * dx;
    put_jac(jac_out, J);

    st[1] = xk;
    st[2] += dx * h;
    st[3] += t * s;
    st[4] = f1;
    if (c) cov_transport(J, c);
    return 0;
}

/* ---- rotation into another sector frame (Sec. 3: the TRD shares the TPC's
 * 18-sector segmentation; tracks are followed in the sector's local frame) --
 * The point is rotated exactly; the covariance is carried to the new
 * reference plane x' = const to first order by sliding along the track:
 *   dy'/dy = r/r',  dz'/dy = -tgl sin(d)/r',  dsnp'/dy = -rho sin(d),
 *   dsnp'/dsnp = r'/r,  all else identity   (r = cos(phi), r' = cos(phi - d)).
 * Returns -1 when |snp'| >= kMaxSnp or the track would point inwards.      */
int ora_rotate(double st[7], double c[15], double alpha_new, double bz, double *jac_out,
               double *snp_slack)
{
    const double d = alpha_new - st[0];
    const double cd = cos(d), sd = sin(d);
    const double f = st[4];
    const double r = sqrt((1.0 - f) * (1.0 + f));
    const double fn = f * cd - r * sd;
    const double rn = r * cd + f * sd;
    if (snp_slack) *snp_slack = fmin(*snp_slack, fabs(kMaxSnp - fabs(fn)));
    if (!(fabs(fn) < kMaxSnp) || !(rn > 0)) return -1;  /* NaN fails too */
    const double rho = -kCLight * bz * st[6];
    double J[5][5];
    eye5(J);
    J[0][0] = r / rn;
    J[1][0] = -st[5] * sd / rn;
    J[2][0] = -rho * sd;
    J[2][2] = rn / r;
    put_jac(jac_out, J);
    const double x = st[1], y = st[2];
    st[0] = alpha_new;
    st[1] = x * cd + y * sd;
    st[2] = -x * sd + y * cd;
    st[4] = fn;
    if (c) cov_transport(J, c);
    return 0;
}

/* ---- material (Sec. 3: "energy loss"; constants are a reading) ---------- */
/* Bethe mean energy loss without the density term, MeV cm^2/g.            */
double ora_bethe(double bg)
{
    const double b2 = bg * bg / (1.0 + bg * bg);
    return kBetheK * kZOverA / b2 *
           (log(2.0 * kMassElectron * bg * bg / kIExcitation) - b2);
}

/* d(ora_bethe)/d(beta gamma): with 1/beta^2 = 1 + 1/bg^2 the curve is
 * K Z/A (1 + 1/bg^2) (ln(2 m_e bg^2 / I) - beta^2), differentiated term by
 * term (d beta^2 / d bg = 2 bg / (1 + bg^2)^2).                             */
double ora_bethe_dbg(double bg)
{
    const double bg2 = bg * bg;
    const double inv_b2 = 1.0 + 1.0 / bg2;
    const double b2 = bg2 / (1.0 + bg2);
    const double bracket = log(2.0 * kMassElectron * bg2 / kIExcitation) - b2;
    const double d_inv_b2 = -2.0 / (bg2 * bg);
    const double d_bracket = 2.0 / bg - 2.0 * bg / ((1.0 + bg2) * (1.0 + bg2));
    return kBetheK * kZOverA * (d_inv_b2 * bracket + inv_b2 * d_bracket);
}

/* Highland: variance of the projected scattering angle (rad^2). */
double ora_highland(double p, double beta, double xx0)
{
    const double t0 = 0.0136 / (beta * p);
    const double f = 1.0 + 0.038 * log(xx0);
    return t0 * t0 * xx0 * f * f;
}

/* One material step at the current position.  dir = +1 for a track moving
 * outward (the mean loss is subtracted), -1 for a track moving inward (the
 * refit of Sec. 2, step 3: the loss is added back).
 *   1. multiple scattering at the entry momentum widens snp, tgl and q2pt
 *      (two projected angles of variance theta0^2 carried onto the state);
 *   2. the mean energy loss of a pion over the path through the layer
 *      changes |p| to p', so q2pt becomes q2pt p / p' = sign(q) sqrt(1 + tgl^2) / p';
 *   3. the covariance is carried through step 2 by its Jacobian, as through
 *      a transport: q2pt' depends on snp (path length), on tgl (path length
 *      and p) and on q2pt (p, and through p the Bethe curve).
 * Returns -1 when the particle stops.                                      */
static int material_dir(double st[7], double c[15], double dir)
{
    const double f = st[4], t = st[5], k = st[6];
    if (k == 0.0) return 0;
    const double r = sqrt((1.0 - f) * (1.0 + f));
    const double t2 = 1.0 + t * t;
    const double path = sqrt(t2) / r;
    const double xx0 = kX0Fraction * path;
    const double xrho = kXRho * path;
    const double p = sqrt(t2) / fabs(k);
    const double e = sqrt(p * p + kMassPion * kMassPion);
    const double beta = p / e;
    const double th2 = ora_highland(p, beta, xx0);
    c[ci(2, 2)] += th2 * r * r * t2;
    c[ci(3, 3)] += th2 * t2 * t2;
    c[ci(4, 3)] += th2 * t * t2 * k;
    c[ci(4, 4)] += th2 * t * t * k * k;
    const double bg = p / kMassPion;
    const double de = ora_bethe(bg) * xrho * 1e-3;
    const double e1 = e - dir * de;
    if (e1 <= kMassPion) return -1;
    const double p1 = sqrt(e1 * e1 - kMassPion * kMassPion);
    const double k1 = k * p / p1;
    /* derivatives with respect to (snp, tgl, q2pt) */
    const double dp[3] = {0.0, p * t / t2, -p / k};
    const double dpath[3] = {path * f / (r * r), path * t / t2, 0.0};
    const double dlns[3] = {0.0, t / t2, 0.0}; /* d ln sqrt(1 + tgl^2) */
    double J[5][5];
    eye5(J);
    for (int a = 0; a < 3; ++a) {
        const double dde = 1e-3 * kXRho *
                           (ora_bethe_dbg(bg) * dp[a] / kMassPion * path + ora_bethe(bg) * dpath[a]);
        const double de1 = (p / e) * dp[a] - dir * dde;
        const double dp1 = (e1 / p1) * de1;
        J[4][2 + a] = k1 * (dlns[a] - dp1 / p1);
    }
    st[6] = k1;
    cov_transport(J, c);
    return 0;
}

int ora_material(double st[7], double c[15]) { return material_dir(st, c, 1.0); }
int ora_material_inward(double st[7], double c[15]) { return material_dir(st, c, -1.0); }

/* ---- measurement model with pad tilt (Sec. 3) -----------------------------
 * Only y and z enter the chi2.  The tilted pads make the measured y depend on
 * where along the pad the track crossed:  y_meas = y - tan(tau) (z - z_tl).
 * H = [[1, -tan(tau), 0, 0, 0], [0, 1, 0, 0, 0]],  S = H C H^T + V.        */
typedef struct {
    double r[2];
    double S[3]; /* S00, S01, S11 */
    double chi2;
} ora_resid_t;

static void ora_residual(const double st[7], const double c[15], double tt, double ytl,
                         double ztl, double vyy, double vzz, double vyz, ora_resid_t *o)
{
    o->r[0] = ytl - (st[2] - tt * (st[3] - ztl));
    o->r[1] = ztl - st[3];
    o->S[0] = c[0] - 2.0 * tt * c[1] + tt * tt * c[2] + vyy;
    o->S[1] = c[1] - tt * c[2] + vyz;
    o->S[2] = c[2] + vzz;
    const double det = o->S[0] * o->S[2] - o->S[1] * o->S[1];
    o->chi2 = (o->S[2] * o->r[0] * o->r[0] - 2.0 * o->S[1] * o->r[0] * o->r[1] +
               o->S[0] * o->r[1] * o->r[1]) / det;
}

/* Kalman update (Abstract; Sec. 3, "Kalman filter").  Standard gain form
 * K = C H^T S^-1, p += K r, C -= K S K^T; with joseph != 0 the covariance is
 * (I - K H) C (I - K H)^T + K V K^T instead.  meas = {y_tl, z_tl, vyy, vzz,
 * vyz}.  Returns the chi2 of the measurement.                              */
double ora_update(double st[7], double c[15], int layer, const double *meas, int joseph)
{
    const double tt = tilt_tan(layer);
    ora_resid_t o;
    ora_residual(st, c, tt, meas[0], meas[1], meas[2], meas[3], meas[4], &o);
    double C[5][5], H[2][5] = {{1, -tt, 0, 0, 0}, {0, 1, 0, 0, 0}};
    cov_full(c, C);
    const double det = o.S[0] * o.S[2] - o.S[1] * o.S[1];
    const double Si[2][2] = {{o.S[2] / det, -o.S[1] / det}, {-o.S[1] / det, o.S[0] / det}};
    double CHt[5][2], K[5][2];
    for (int i = 0; i < 5; ++i)
        for (int a = 0; a < 2; ++a) {
            double s = 0;
            for (int k = 0; k < 5; ++k) s += C[i][k] * H[a][k];
            CHt[i][a] = s;
        }
    for (int i = 0; i < 5; ++i)
        for (int a = 0; a < 2; ++a) K[i][a] = CHt[i][0] * Si[0][a] + CHt[i][1] * Si[1][a];
    for (int i = 0; i < 5; ++i) st[2 + i] += K[i][0] * o.r[0] + K[i][1] * o.r[1];
    double N[5][5];
    if (!joseph) {
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) N[i][j] = C[i][j] - (K[i][0] * CHt[j][0] + K[i][1] * CHt[j][1]);
    } else {
        double A[5][5], T[5][5];
        const double V[2][2] = {{meas[2], meas[4]}, {meas[4], meas[3]}};
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) A[i][j] = (i == j) - (K[i][0] * H[0][j] + K[i][1] * H[1][j]);
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                double s = 0;
                for (int k = 0; k < 5; ++k) s += A[i][k] * C[k][j];
                T[i][j] = s;
            }
        for (int i = 0; i < 5; ++i)
            for (int j = 0; j < 5; ++j) {
                double s = 0;
                for (int k = 0; k < 5; ++k) s += T[i][k] * A[j][k];
                for (int a = 0; a < 2; ++a)
                    for (int b = 0; b < 2; ++b) s += K[i][a] * V[a][b] * K[j][b];
                N[i][j] = s;
            }
    }
    cov_pack(N, c);
    return o.chi2;
}

/* residual + chi2 only (for tests) */
double ora_chi2(const double st[7], const double c[15], int layer, const double *meas)
{
    ora_resid_t o;
    ora_residual(st, c, tilt_tan(layer), meas[0], meas[1], meas[2], meas[3], meas[4], &o);
    return o.chi2;
}

/* ---- the follower (Sec. 3) ------------------------------------------------ */
typedef struct {
    double bz, n_sigma_road, chi2_cut, p_miss, dy_gate_sigma;
    int n_hyp, max_missing, res_mode, material_on;
    /* misalignment and field (Sec. 3, the paragraph on misalignment): an
     * optional average radius per chamber, an optional Bz(r, z) map */
    const float *chamber_x;        /* [540] or NULL: nominal layer radii */
    const float *field;            /* [nz][nr] or NULL: homogeneous bz */
    int f_nr, f_nz;
    double f_r0, f_r1, f_z0, f_z1;
} ora_params_t;

typedef struct {
    double st[7];
    double c[15];
    double score, chi2;
    int sector, ntrk, nmiss;
    int ids[ORA_NLAYER];
} ora_hyp_t;

typedef struct {
    double score, chi2;
    int parent, id; /* id = input tracklet index, ORA_MISSING for a missing layer */
} ora_ext_t;

typedef struct {
    int n;
    const int *ch;
    const float *y, *z, *dy, *vyy, *vzz, *vyz;
    const int *start; /* chamber buckets: start[ORA_NCHAMBER + 1] */
    const int *list;
    int brute;        /* 1: scan every tracklet of the input and test its chamber id */
    const int *trig;  /* interaction id per tracklet, or NULL */
    const float *x;   /* radius of each tracklet (misalignment), or NULL: the layer's */
} ora_tracklets_t;

static int cmp_ext(const void *pa, const void *pb)
{
    const ora_ext_t *a = pa, *b = pb;
    if (a->score < b->score) return -1;
    if (a->score > b->score) return 1;
    if (a->parent != b->parent) return a->parent < b->parent ? -1 : 1;
    if (a->id != b->id) return a->id < b->id ? -1 : 1; /* ORA_MISSING sorts last */
    return 0;
}

static int sector_of_alpha(double a)
{
    const double w = sector_width();
    double u = fmod(a, 2.0 * kPi);
    if (u < 0) u += 2.0 * kPi;
    int s = (int)floor(u / w);
    return ((s % ORA_NSECTOR) + ORA_NSECTOR) % ORA_NSECTOR;
}

static double sector_alpha(int s) { return (s + 0.5) * sector_width(); }

/* ---- field map (reading for the field inhomogeneities of Sec. 3) ----------
 * Bz on a regular grid in (r, z): nodes r_i = r0 + i (r1 - r0) / (nr - 1),
 * z_j likewise, value field[j * nr + i]; bilinear between the nodes, the grid
 * box clamps.  A transport step uses the field at its midpoint, estimated
 * along the straight line from the start: x_m = (x0 + x1) / 2, y_m and z_m
 * advanced by half the step along the start direction, r_m = |(x_m, y_m)|;
 * the helix of that constant field is then exact for the step (the field's
 * gradient is not carried into the Jacobian).  A rotation uses the field at
 * the state's own point.  Without a map every step uses bz.                */
static ora_params_t make_params(const double *pd, const int *pi)
{
    ora_params_t P;
    memset(&P, 0, sizeof P);
    P.bz = pd[0];
    P.n_sigma_road = pd[1];
    P.chi2_cut = pd[2];
    P.p_miss = pd[3];
    P.dy_gate_sigma = pd[4];
    P.n_hyp = pi[0];
    P.max_missing = pi[1];
    P.res_mode = pi[2];
    P.material_on = pi[3];
    return P;
}

static double field_at(const ora_params_t *P, double r, double z)
{
    if (!P->field) return P->bz;
    double fr = (P->f_nr - 1) * (r - P->f_r0) / (P->f_r1 - P->f_r0);
    double fz = (P->f_nz - 1) * (z - P->f_z0) / (P->f_z1 - P->f_z0);
    fr = fmin(fmax(fr, 0.0), (double)(P->f_nr - 1));
    fz = fmin(fmax(fz, 0.0), (double)(P->f_nz - 1));
    int i = (int)floor(fr), j = (int)floor(fz);
    if (i > P->f_nr - 2) i = P->f_nr - 2;
    if (j > P->f_nz - 2) j = P->f_nz - 2;
    const double wr = fr - i, wz = fz - j;
    const float *F = P->field;
    const int nr = P->f_nr;
    return (1 - wz) * ((1 - wr) * F[j * nr + i] + wr * F[j * nr + i + 1]) +
           wz * ((1 - wr) * F[(j + 1) * nr + i] + wr * F[(j + 1) * nr + i + 1]);
}

static double step_field(const ora_params_t *P, const double st[7], double x1)
{
    if (!P->field) return P->bz;
    const double f = st[4];
    if (!(fabs(f) < 1.0)) return field_at(P, hypot(st[1], st[2]), st[3]);
    const double r = sqrt((1.0 - f) * (1.0 + f)), h = 0.5 * (x1 - st[1]);
    return field_at(P, hypot(st[1] + h, st[2] + h * f / r), st[3] + h * st[5] / r);
}

static int fprop(double st[7], double c[15], double x1, const ora_params_t *P, double *slack)
{
    return ora_propagate(st, c, x1, step_field(P, st, x1), NULL, slack);
}

static int frot(double st[7], double c[15], double alpha, const ora_params_t *P, double *slack)
{
    return ora_rotate(st, c, alpha, field_at(P, hypot(st[1], st[2]), st[3]), NULL, slack);
}

/* Test helper: one field-map transport step (fprop above) of a state to x1.
 * field [nz][nr] with box = {r0, r1, z0, z1}; NULL field: homogeneous bz.   */
int ora_propagate_map(double st[7], double c[15], double x1, double bz, const float *field, int nr, int nz,
                      const double *box)
{
    ora_params_t P;
    memset(&P, 0, sizeof P);
    P.bz = bz;
    if (field) {
        P.field = field;
        P.f_nr = nr;
        P.f_nz = nz;
        P.f_r0 = box[0];
        P.f_r1 = box[1];
        P.f_z0 = box[2];
        P.f_z1 = box[3];
    }
    return fprop(st, c, x1, &P, NULL);
}

/* Carry a hypothesis to the plane of layer l: helix transport; if the track
 * left the sector's azimuthal extent, rotate into the neighbour sector and
 * transport again; then one material step.  Sets *chamber (-1 when z is
 * outside the 5 stacks).  Accumulates decision slacks into *margin.        */
static int to_layer(ora_hyp_t *h, int l, const ora_params_t *P, int *chamber, double *margin)
{
    const double xl = layer_x(l);
    double sl = INFINITY;
    if (fprop(h->st, h->c, xl, P, &sl)) { *margin = fmin(*margin, sl); return -1; }
    const double lim = xl * half_sector_tan();
    *margin = fmin(*margin, fabs(fabs(h->st[2]) - lim));
    if (fabs(h->st[2]) > lim) {
        const int ns = (h->sector + (h->st[2] > 0 ? 1 : -1) + ORA_NSECTOR) % ORA_NSECTOR;
        if (frot(h->st, h->c, sector_alpha(ns), P, &sl)) { *margin = fmin(*margin, sl); return -1; }
        h->sector = ns;
        if (fprop(h->st, h->c, xl, P, &sl)) { *margin = fmin(*margin, sl); return -1; }
    }
    *margin = fmin(*margin, sl);
    if (P->material_on && ora_material(h->st, h->c)) return -1;
    const double z = h->st[3];
    double zb = INFINITY;
    for (int b = 0; b <= ORA_NSTACK; ++b) zb = fmin(zb, fabs(z - (kZMin + kStackLength * b)));
    *margin = fmin(*margin, zb);
    const double u = (z - kZMin) / kStackLength;
    if (u >= 0 && u < ORA_NSTACK) {
        const int stack = (int)floor(u);
        *chamber = h->sector * (ORA_NSTACK * ORA_NLAYER) + stack * ORA_NLAYER + l;
        /* misalignment: on to the chamber's average radius (the chamber is the
         * one found at the nominal radius) */
        if (P->chamber_x && (double)P->chamber_x[*chamber] != xl) {
            sl = INFINITY;
            if (fprop(h->st, h->c, P->chamber_x[*chamber], P, &sl)) { *margin = fmin(*margin, sl); return -1; }
            *margin = fmin(*margin, sl);
        }
    } else {
        *chamber = -1;
    }
    return 0;
}

/* Tracklet tests (Sec. 3): search road from the covariance, dy deviation
 * below dy_gate_sigma (4 sigma in the paper), chi2 from y and z only below
 * the cut.  Returns 1 if accepted; *slack is the distance of the decision
 * from flipping (smallest passing slack, or largest failing one).          */
static int test_tracklet(const ora_hyp_t *h, int l, const ora_tracklets_t *T, int j,
                         const ora_params_t *P, double *chi2, double *slack, int *in_road)
{
    const double f = h->st[4];
    const double r = sqrt((1.0 - f) * (1.0 + f));
    const double u = f / r - lorentz_tan(P->bz);
    double vyy = T->vyy[j];
    if (P->res_mode) vyy = kSigY0 * kSigY0 + kSigY1 * kSigY1 * u * u;
    /* a tracklet at another radius (misalignment): the fast linear
     * extrapolation of the track to it (straight line along its direction;
     * covariance as at the chamber radius) for the tests */
    double sx[7];
    memcpy(sx, h->st, sizeof sx);
    if (T->x) {
        const double dx = (double)T->x[j] - h->st[1];
        sx[2] += dx * f / r;
        sx[3] += dx * h->st[5] / r;
    }
    ora_resid_t o;
    ora_residual(sx, h->c, tilt_tan(l), T->y[j], T->z[j], vyy, T->vzz[j], T->vyz[j], &o);
    const double ny = fabs(o.r[0]) / sqrt(o.S[0]);
    const double nz = fabs(o.r[1]) / sqrt(o.S[2]);
    const double dy_pred = kDriftLength * u;
    const double sdy = sqrt(kSigDy0 * kSigDy0 + kSigDy1 * kSigDy1 * u * u);
    const double ndy = fabs(T->dy[j] - dy_pred) / sdy;
    const double s[4] = {P->n_sigma_road - ny, P->n_sigma_road - nz, P->dy_gate_sigma - ndy,
                         P->chi2_cut - o.chi2};
    const int acc = s[0] >= 0 && s[1] >= 0 && s[2] >= 0 && s[3] > 0;
    *in_road = s[0] >= 0 && s[1] >= 0;
    double m;
    if (acc) {
        m = INFINITY;
        for (int i = 0; i < 4; ++i) m = fmin(m, s[i]);
    } else {
        m = 0;
        for (int i = 0; i < 4; ++i)
            if (s[i] < 0 || (i == 3 && s[i] <= 0)) m = fmax(m, -s[i]);
    }
    *slack = m;
    *chi2 = o.chi2;
    return acc;
}

typedef struct {
    ora_ext_t *ext;
    int cap;
    ora_hyp_t *set, *work; /* n_hyp entries each */
} ora_scratch_t;

static void push_ext(ora_scratch_t *S, int *n, ora_ext_t e)
{
    if (*n == S->cap) {
        S->cap = S->cap ? 2 * S->cap : 256;
        S->ext = realloc(S->ext, (size_t)S->cap * sizeof(ora_ext_t));
    }
    S->ext[(*n)++] = e;
}

typedef struct {
    double st[7], c[15], chi2;
    int ntrk, nmiss, status;
    int ids[ORA_NLAYER];
    double margin[ORA_NLAYER];
    int nroad[ORA_NLAYER];
} ora_result_t;

enum { ORA_ST_PROP_FAIL = 1, ORA_ST_STOPPED = 2, ORA_ST_SEED_INVALID = 4 };

/* Sec. 4: in time frames, only tracklets of the track's own interaction are
 * considered.  An id < 0 on either side means no association.             */
static int same_interaction(int seed_trig, const ora_tracklets_t *T, int j)
{
    return seed_trig < 0 || !T->trig || T->trig[j] < 0 || T->trig[j] == seed_trig;
}

static void follow_one(const double seed_st[7], const double seed_c[15], int seed_trig,
                       const ora_tracklets_t *T, const ora_params_t *P, ora_scratch_t *S, ora_result_t *R)
{
    memset(R, 0, sizeof *R);
    for (int l = 0; l < ORA_NLAYER; ++l) { R->ids[l] = -1; R->margin[l] = INFINITY; }
    memcpy(R->st, seed_st, sizeof R->st);
    memcpy(R->c, seed_c, sizeof R->c);
    if (!(fabs(seed_st[4]) < kMaxSnp) || !ora_cov_is_pd(seed_c)) { R->status = ORA_ST_SEED_INVALID; return; }

    const int nh = P->n_hyp < 1 ? 1 : (P->n_hyp > ORA_MAXHYP ? ORA_MAXHYP : P->n_hyp);
    ora_hyp_t *set = S->set, *work = S->work;
    int nset = 1;
    memset(&set[0], 0, sizeof set[0]);
    memcpy(set[0].st, seed_st, sizeof set[0].st);
    memcpy(set[0].c, seed_c, sizeof set[0].c);
    for (int l = 0; l < ORA_NLAYER; ++l) set[0].ids[l] = -1;

    /* rotate the seed into the sector that contains its position */
    {
        const double phi = seed_st[0] + atan2(seed_st[2], seed_st[1]);
        const int s = sector_of_alpha(phi);
        const double w = sector_width();
        double u = fmod(phi, w);
        if (u < 0) u += w;
        const double rad = hypot(seed_st[1], seed_st[2]);
        R->margin[0] = fmin(R->margin[0], rad * fmin(u, w - u));
        double sl = INFINITY;
        if (frot(set[0].st, set[0].c, sector_alpha(s), P, &sl)) {
            R->margin[0] = fmin(R->margin[0], sl);
            R->status = ORA_ST_PROP_FAIL;
            return;
        }
        R->margin[0] = fmin(R->margin[0], sl);
        set[0].sector = s;
    }

    int status = 0;
    for (int l = 0; l < ORA_NLAYER; ++l) {
        int next = 0, n_alive = 0;
        for (int hi = 0; hi < nset; ++hi) {
            work[hi] = set[hi];
            int chamber = -1;
            if (to_layer(&work[hi], l, P, &chamber, &R->margin[l])) { work[hi].sector = -1; continue; }
            ++n_alive;
            if (chamber >= 0) {
                const int lo = T->brute ? 0 : T->start[chamber];
                const int up = T->brute ? T->n : T->start[chamber + 1];
                for (int q = lo; q < up; ++q) {
                    const int j = T->brute ? q : T->list[q];
                    if (T->brute && T->ch[j] != chamber) continue;
                    if (!same_interaction(seed_trig, T, j)) continue;
                    double chi2, slack;
                    int in_road;
                    const int acc = test_tracklet(&work[hi], l, T, j, P, &chi2, &slack, &in_road);
                    R->margin[l] = fmin(R->margin[l], slack);
                    R->nroad[l] += in_road;
                    if (acc) push_ext(S, &next, (ora_ext_t){work[hi].score + chi2, chi2, hi, j});
                }
            }
            if (work[hi].nmiss < P->max_missing)
                push_ext(S, &next, (ora_ext_t){work[hi].score + P->p_miss, 0.0, hi, ORA_MISSING});
        }
        if (next == 0) { status = n_alive ? ORA_ST_STOPPED : ORA_ST_PROP_FAIL; break; }
        qsort(S->ext, (size_t)next, sizeof(ora_ext_t), cmp_ext);
        const int keep = next < nh ? next : nh;
        const int ngap = next > nh ? nh : next - 1;
        for (int g = 0; g < ngap; ++g)
            R->margin[l] = fmin(R->margin[l], S->ext[g + 1].score - S->ext[g].score);
        for (int e = 0; e < keep; ++e) {
            const ora_ext_t *x = &S->ext[e];
            ora_hyp_t h = work[x->parent];
            h.score = x->score;
            if (x->id == ORA_MISSING) {
                h.ids[l] = -1;
                h.nmiss += 1;
            } else {
                double m5[5] = {T->y[x->id], T->z[x->id], T->vyy[x->id], T->vzz[x->id],
                                T->vyz[x->id]};
                /* before the update: the precise transport to the tracklet's
                 * own radius (a failed transport leaves the state where it is) */
                if (T->x) (void)fprop(h.st, h.c, (double)T->x[x->id], P, NULL);
                if (P->res_mode) {
                    const double f = h.st[4], r = sqrt((1.0 - f) * (1.0 + f));
                    const double u = f / r - lorentz_tan(P->bz);
                    m5[2] = kSigY0 * kSigY0 + kSigY1 * kSigY1 * u * u;
                }
                ora_update(h.st, h.c, l, m5, 0);
                h.ids[l] = x->id;
                h.ntrk += 1;
                h.chi2 += x->chi2;
            }
            set[e] = h;
        }
        nset = keep;
    }
    const ora_hyp_t *b = &set[0];
    memcpy(R->st, b->st, sizeof R->st);
    memcpy(R->c, b->c, sizeof R->c);
    R->chi2 = b->chi2;
    R->ntrk = b->ntrk;
    R->nmiss = b->nmiss;
    R->status = status;
    memcpy(R->ids, b->ids, sizeof R->ids);
}

/* Step helpers for tests: carry a state to layer l (to_layer above) and list
 * the accepted tracklets of a chamber with their chi2 (test_tracklet above).
 * sector_io: in = current sector, out = sector after a possible rotation.   */
int ora_to_layer(double st[7], double c[15], int *sector_io, int l, const double *pd,
                 const int *pi, int *chamber)
{
    ora_params_t P = make_params(pd, pi);
    ora_hyp_t h;
    memset(&h, 0, sizeof h);
    memcpy(h.st, st, sizeof h.st);
    memcpy(h.c, c, sizeof h.c);
    h.sector = *sector_io;
    double m = INFINITY;
    if (to_layer(&h, l, &P, chamber, &m)) return -1;
    memcpy(st, h.st, sizeof h.st);
    memcpy(c, h.c, sizeof h.c);
    *sector_io = h.sector;
    return 0;
}

int ora_candidates(const double st[7], const double c[15], int l, int chamber, int n_trk,
                   const int *t_ch, const float *t_y, const float *t_z, const float *t_dy,
                   const float *t_vyy, const float *t_vzz, const float *t_vyz, const double *pd,
                   const int *pi, int max_out, int *ids_out, double *chi2_out)
{
    ora_params_t P = make_params(pd, pi);
    ora_tracklets_t T = {n_trk, t_ch, t_y, t_z, t_dy, t_vyy, t_vzz, t_vyz, NULL, NULL, 1, NULL, NULL};
    ora_hyp_t h;
    memset(&h, 0, sizeof h);
    memcpy(h.st, st, sizeof h.st);
    memcpy(h.c, c, sizeof h.c);
    int n = 0;
    for (int j = 0; j < n_trk; ++j) {
        if (t_ch[j] != chamber) continue;
        double chi2, slack;
        int in_road;
        if (test_tracklet(&h, l, &T, j, &P, &chi2, &slack, &in_road)) {
            if (n < max_out) { ids_out[n] = j; chi2_out[n] = chi2; }
            ++n;
        }
    }
    return n;
}

/* Entry point.  Inputs are the FP32 arrays the library also reads; every
 * value is widened to double.  seed_index (optional, n_out entries) selects
 * which seeds to follow.  Outputs: [n_out] or [k][n_out] arrays.
 *   st_out[7][n]   alpha, x, y, z, snp, tgl, q2pt
 *   cov_out[15][n], chi2_out[n], ntrk/nmiss/status[n], ids_out[6][n]
 *   margin_out[6][n] (smallest decision slack per layer), nroad_out[6][n]
 * pd = {bz, n_sigma_road, chi2_cut, p_miss, dy_gate_sigma}
 * pi = {n_hyp, max_missing, res_mode, material_on}
 * seed_trig, t_trig (optional): interaction ids (Sec. 4 association).
 * t_x (optional): the radius of each tracklet; chamber_x (optional, [540]):
 * the average radius of each chamber (misalignment, Sec. 3).  field
 * (optional, [f_nz][f_nr]) with f_box = {r0, r1, z0, z1}: a Bz map.
 * Returns 0, or -1 on invalid arguments.                                    */
int ora_follow(int n_seeds, const float *alpha, const float *x, const float *y, const float *z,
               const float *snp, const float *tgl, const float *q2pt, const float *cov,
               int n_trk, const int *t_ch, const float *t_y, const float *t_z, const float *t_dy,
               const float *t_vyy, const float *t_vzz, const float *t_vyz,
               const double *pd, const int *pi, int n_out, const int *seed_index, int brute,
               int n_threads, double *st_out, double *cov_out, double *chi2_out, int *ntrk_out,
               int *nmiss_out, int *status_out, int *ids_out, double *margin_out, int *nroad_out,
               const int *seed_trig, const int *t_trig, const float *t_x, const float *chamber_x,
               const float *field, int f_nr, int f_nz, const double *f_box)
{
    if (n_seeds < 0 || n_trk < 0 || n_out < 0) return -1;
    ora_params_t P = make_params(pd, pi);
    if (P.n_hyp < 1 || P.n_hyp > ORA_MAXHYP) return -1;
    P.chamber_x = chamber_x;
    if (field) {
        if (f_nr < 2 || f_nz < 2 || !f_box || !(f_box[1] > f_box[0]) || !(f_box[3] > f_box[2])) return -1;
        P.field = field;
        P.f_nr = f_nr;
        P.f_nz = f_nz;
        P.f_r0 = f_box[0];
        P.f_r1 = f_box[1];
        P.f_z0 = f_box[2];
        P.f_z1 = f_box[3];
    }

    /* chamber buckets: a counting pass, then a fill in input order */
    int *start = calloc(ORA_NCHAMBER + 1, sizeof(int));
    int *list = malloc((size_t)(n_trk > 0 ? n_trk : 1) * sizeof(int));
    for (int j = 0; j < n_trk; ++j)
        if (t_ch[j] >= 0 && t_ch[j] < ORA_NCHAMBER) start[t_ch[j] + 1]++;
    for (int c = 0; c < ORA_NCHAMBER; ++c) start[c + 1] += start[c];
    {
        int *fill = malloc(ORA_NCHAMBER * sizeof(int));
        memcpy(fill, start, ORA_NCHAMBER * sizeof(int));
        for (int j = 0; j < n_trk; ++j)
            if (t_ch[j] >= 0 && t_ch[j] < ORA_NCHAMBER) list[fill[t_ch[j]]++] = j;
        free(fill);
    }
    ora_tracklets_t T = {n_trk, t_ch, t_y, t_z, t_dy, t_vyy, t_vzz, t_vyz, start, list, brute, t_trig, t_x};

#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        ora_scratch_t S = {NULL, 0, malloc((size_t)P.n_hyp * sizeof(ora_hyp_t)),
                           malloc((size_t)P.n_hyp * sizeof(ora_hyp_t))};
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int o = 0; o < n_out; ++o) {
            const int i = seed_index ? seed_index[o] : o;
            ora_result_t R;
            if (i < 0 || i >= n_seeds) {
                memset(&R, 0, sizeof R);
                R.status = ORA_ST_SEED_INVALID;
                for (int l = 0; l < ORA_NLAYER; ++l) { R.ids[l] = -1; R.margin[l] = INFINITY; }
            } else {
                double s7[7] = {alpha[i], x[i], y[i], z[i], snp[i], tgl[i], q2pt[i]};
                double c15[15];
                for (int k = 0; k < 15; ++k) c15[k] = cov[(size_t)k * n_seeds + i];
                follow_one(s7, c15, seed_trig ? seed_trig[i] : -1, &T, &P, &S, &R);
            }
            for (int k = 0; k < 7; ++k) st_out[(size_t)k * n_out + o] = R.st[k];
            for (int k = 0; k < 15; ++k) cov_out[(size_t)k * n_out + o] = R.c[k];
            chi2_out[o] = R.chi2;
            ntrk_out[o] = R.ntrk;
            nmiss_out[o] = R.nmiss;
            status_out[o] = R.status;
            for (int l = 0; l < ORA_NLAYER; ++l) {
                ids_out[(size_t)l * n_out + o] = R.ids[l];
                if (margin_out) margin_out[(size_t)l * n_out + o] = R.margin[l];
                if (nroad_out) nroad_out[(size_t)l * n_out + o] = R.nroad[l];
            }
        }
        free(S.ext);
        free(S.set);
        free(S.work);
    }
    free(start);
    free(list);
    return 0;
}

/* ---- the TRD-only refit (Sec. 2, step 3) ------------------------------------
 * The calibration chain refits each matched track twice, once from the ITS
 * and once from TRD and TOF alone, without the TPC clusters.  This is the
 * TRD half (no TOF points are modelled).  Reading, in order:
 *   1. only tracks with at least two tracklets (matched, Sec. 3.1) whose
 *      follower status is not SEED_INVALID are refitted;
 *   2. the prior is the follower's final state with its covariance reduced
 *      to the diagonal and scaled by cov_scale (the TPC-derived correlations
 *      are dropped and the variances widened, so the prior carries little of
 *      the TPC's information);
 *   3. the prior is carried (helix, no material) into the sector frame of the
 *      outermost tracklet and to that layer's plane;
 *   4. for l from that layer down to 0: transport to x_l (from the second
 *      layer on), entering the tracklet's sector when it lies in another one
 *      (or the neighbour sector at the azimuthal edge when the layer has no
 *      tracklet), Kalman update with the layer's tracklet, then the layer's
 *      material with the energy loss added back (the material of layer l
 *      sits just inside x_l, where the outward follower meets it before its
 *      update);
 *   5. the result is the state at x_0 after the material of layer 0, with the
 *      sum of the update chi2 values and the number of updates.
 * A transport or rotation that fails (|snp| limit) stops the refit (status
 * PROP_FAIL); the result is then the state as far as it was carried (a
 * failing transport or rotation leaves the state untouched).               */
enum { ORA_RF_PROP_FAIL = 1, ORA_RF_SKIPPED = 8 };

typedef struct {
    double st[7], c[15], chi2;
    int nupd, status;
    double margin; /* smallest slack of a decision (|snp| limit, sector edge) */
} ora_refit_result_t;

static void refit_one(const double in_st[7], const double in_cdiag[5], int in_status, const int ids[ORA_NLAYER],
                      const ora_tracklets_t *T, const ora_params_t *P, double cov_scale, ora_refit_result_t *R)
{
    memset(R, 0, sizeof *R);
    memcpy(R->st, in_st, sizeof R->st);
    R->margin = INFINITY;
    int ntrk = 0, ltop = -1;
    for (int l = 0; l < ORA_NLAYER; ++l)
        if (ids[l] >= 0) { ++ntrk; ltop = l; }
    if (ntrk < 2 || (in_status & ORA_ST_SEED_INVALID)) { R->status = ORA_RF_SKIPPED; return; }
    for (int l = 0; l < ORA_NLAYER; ++l)
        if (ids[l] >= T->n || (ids[l] >= 0 && (T->ch[ids[l]] < 0 || T->ch[ids[l]] >= ORA_NCHAMBER))) {
            R->status = ORA_RF_SKIPPED;
            return;
        }

    ora_hyp_t h;
    memset(&h, 0, sizeof h);
    memcpy(h.st, in_st, sizeof h.st);
    /* step 2: diagonal prior */
    for (int i = 0; i < 5; ++i) h.c[ci(i, i)] = cov_scale * in_cdiag[i];
    h.sector = sector_of_alpha(in_st[0]);

    int fail = 0;
    for (int l = ltop; l >= 0 && !fail; --l) {
        const int j = ids[l];
        /* a layer's plane: its tracklet's own radius when given (misalignment) */
        const double xl = (j >= 0 && T->x) ? (double)T->x[j] : layer_x(l);
        /* step 3 (l == ltop) and step 4: into the tracklet's sector, to x_l */
        double sl = INFINITY;
        if (ora_propagate(h.st, h.c, xl, P->bz, NULL, &sl)) { fail = 1; }
        int target = h.sector;
        if (!fail && j >= 0) {
            target = T->ch[j] / (ORA_NSTACK * ORA_NLAYER);
        } else if (!fail) {
            const double lim = xl * half_sector_tan();
            sl = fmin(sl, fabs(fabs(h.st[2]) - lim));
            if (fabs(h.st[2]) > lim) target = (h.sector + (h.st[2] > 0 ? 1 : -1) + ORA_NSECTOR) % ORA_NSECTOR;
        }
        if (!fail && target != h.sector) {
            if (ora_rotate(h.st, h.c, sector_alpha(target), P->bz, NULL, &sl)) {
                fail = 1;
            } else {
                h.sector = target;
                if (ora_propagate(h.st, h.c, xl, P->bz, NULL, &sl)) fail = 1;
            }
        }
        R->margin = fmin(R->margin, sl);
        if (fail) break;
        if (j >= 0) {
            double m5[5] = {T->y[j], T->z[j], T->vyy[j], T->vzz[j], T->vyz[j]};
            if (P->res_mode) {
                const double f = h.st[4], r = sqrt((1.0 - f) * (1.0 + f));
                const double u = f / r - lorentz_tan(P->bz);
                m5[2] = kSigY0 * kSigY0 + kSigY1 * kSigY1 * u * u;
            }
            h.chi2 += ora_update(h.st, h.c, l, m5, 0);
            h.ntrk += 1;
        }
        if (P->material_on && material_dir(h.st, h.c, -1.0)) { fail = 1; break; }
    }
    memcpy(R->st, h.st, sizeof R->st);
    memcpy(R->c, h.c, sizeof R->c);
    R->chi2 = h.chi2;
    R->nupd = h.ntrk;
    R->status = fail ? ORA_RF_PROP_FAIL : 0;
}

/* Entry point of the refit.  The follower's results (FP32 arrays in the
 * library's layout, n tracks) and the tracklets (input order) are widened
 * to double.  Outputs: st_out[7][n], cov_out[15][n], chi2_out[n],
 * nupd_out[n], status_out[n], margin_out[n] (optional: the smallest slack of
 * a decision, |snp| limit or sector edge, in the units of its test).  pd/pi
 * as for ora_follow; t_x (optional): the tracklets' own radii.  Returns 0, or -1
 * on invalid arguments.                                                     */
int ora_refit(int n, const float *alpha, const float *x, const float *par, const float *cov,
              const int *status, const int *ids, int n_trk, const int *t_ch, const float *t_y,
              const float *t_z, const float *t_vyy, const float *t_vzz, const float *t_vyz,
              const double *pd, const int *pi, double cov_scale, int n_threads, double *st_out,
              double *cov_out, double *chi2_out, int *nupd_out, int *status_out, double *margin_out,
              const float *t_x)
{
    if (n < 0 || n_trk < 0 || !(cov_scale > 0)) return -1;
    ora_params_t P = make_params(pd, pi);
    ora_tracklets_t T = {n_trk, t_ch, t_y, NULL, NULL, t_vyy, t_vzz, t_vyz, NULL, NULL, 1, NULL, t_x};
    T.z = t_z;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
    for (int i = 0; i < n; ++i) {
        double s7[7] = {alpha[i], x[i]};
        for (int k = 0; k < 5; ++k) s7[2 + k] = par[(size_t)k * n + i];
        double cd[5];
        for (int k = 0; k < 5; ++k) cd[k] = cov[(size_t)ci(k, k) * n + i];
        int id6[ORA_NLAYER];
        for (int l = 0; l < ORA_NLAYER; ++l) id6[l] = ids[(size_t)l * n + i];
        ora_refit_result_t R;
        refit_one(s7, cd, status[i], id6, &T, &P, cov_scale, &R);
        for (int k = 0; k < 7; ++k) st_out[(size_t)k * n + i] = R.st[k];
        for (int k = 0; k < 15; ++k) cov_out[(size_t)k * n + i] = R.c[k];
        chi2_out[i] = R.chi2;
        nupd_out[i] = R.nupd;
        status_out[i] = R.status;
        if (margin_out) margin_out[i] = R.margin;
    }
    return 0;
}

/* ---- residuals in TPC sub-volumes and the distortion vector (Sec. 2,
 * steps 4 and 5) -------------------------------------------------------------
 * The space-point calibration compares each distorted TPC cluster with the
 * weighted combination of the two external refits (ITS, and TRD without the
 * TPC) and collects the residuals per TPC sub-volume; each sub-volume then
 * yields one distortion vector in x, y and z.  Readings (the paper gives no
 * numbers for them):
 *   - 152 pad rows, centres at x_r = 85 + 160 (r + 1/2) / 152 cm (as float);
 *   - a cluster of sector s (0..17) at row r is compared in the frame of s:
 *     each refit is rotated into that frame and transported (helix, no
 *     material in the gas) to x_r;
 *   - combination: the (y, z) estimates are averaged with their inverse 2x2
 *     covariances, sin(phi) and tan(lambda) with their inverse variances;
 *   - residual (dy, dz) = cluster - combination; slopes t = dy/dx =
 *     tan(phi) and u = dz/dx = tan(lambda) / cos(phi) of the combination;
 *   - sub-volume (voxel): side (z < 0) x 18 sectors x 152 rows x 15 bins of
 *     y/x in [-tan 10 deg, tan 10 deg) x 5 bins of |z|/x in [0, 1) (the last
 *     bins take what lies beyond), decided in FP32 from the cluster's own
 *     y, z and x_r;
 *   - distortion of a voxel: a cluster at row x_r was freed at the track
 *     point x_r - dx and moved by (dy, dz), so to first order its residuals
 *     are dy_i = Dy - Dx t_i and dz_i = Dz - Dx u_i; (Dx, Dy, Dz) is the
 *     least-squares solution over the voxel's clusters.
 * Per voxel the oracle keeps 11 FP64 sums: n, St, Su, Stt, Suu, Sdy, Sdz,
 * Stdy, Sudz, Sdydy, Sdzdz.                                                 */
#define ORA_TPC_ROWS 152
#define ORA_VOX_Y 15
#define ORA_VOX_Z 5
#define ORA_VOX_SECT 36
#define ORA_NVOX (ORA_VOX_SECT * ORA_TPC_ROWS * ORA_VOX_Y * ORA_VOX_Z)
#define ORA_VOX_SUMS 11

static float tpc_row_x(int r) { return (float)(85.0 + (r + 0.5) * 160.0 / ORA_TPC_ROWS); }

/* Voxel of a cluster (FP32 decisions, in the order written). */
int ora_voxel_of(float y, float z, int sector, int row)
{
    if (sector < 0 || sector >= ORA_NSECTOR || row < 0 || row >= ORA_TPC_ROWS) return -1;
    const float xr = tpc_row_x(row);
    const float T = (float)0.17632698070846498; /* tan 10 deg */
    const float ys = (float)ORA_VOX_Y / (2.0f * T);
    const float u = y / xr;
    const float v = u + T;
    const float fy = fminf(fmaxf(v * ys, -1.0f), (float)ORA_VOX_Y); /* bounded before the cast */
    int iy = (int)floorf(fy);
    iy = iy < 0 ? 0 : (iy >= ORA_VOX_Y ? ORA_VOX_Y - 1 : iy);
    const float w = fabsf(z) / xr;
    const float fz = fminf(w * (float)ORA_VOX_Z, (float)ORA_VOX_Z);
    int iz = (int)floorf(fz);
    iz = iz < 0 ? 0 : (iz >= ORA_VOX_Z ? ORA_VOX_Z - 1 : iz);
    const int side = z < 0.0f ? 1 : 0;
    return (((side * ORA_NSECTOR + sector) * ORA_TPC_ROWS + row) * ORA_VOX_Y + iy) * ORA_VOX_Z + iz;
}

/* Carry a refit state along its track to the pad-row plane x_r of sector s
 * (the cluster's frame): when s is not the state's frame, transport first in
 * the old frame to x_r (if that fails, the state stays where it is), rotate
 * there into s, then transport to x_r in s.  Every rotation thus happens
 * next to the cluster.  *frame = -1: the frame is not a sector's yet (the
 * first call always rotates).  Returns -1 when a rotation or the final
 * transport fails (|snp| limit).                                            */
static int tpc_carry(double st[7], double c[15], int *frame, int s, double xr, double bz, double *slack)
{
    if (*frame != s) {
        (void)ora_propagate(st, c, xr, bz, NULL, slack);
        if (ora_rotate(st, c, sector_alpha(s), bz, NULL, slack)) return -1;
        *frame = s;
    }
    return ora_propagate(st, c, xr, bz, NULL, slack);
}

/* The combination of the two refits at one cluster.  out = {dy, dz, t, u,
 * var y, var z} (residual = cluster - combination; slopes of the combined
 * direction; variances of the combined y and z).                           */
static void tpc_combine(const double a[2][7], const double c[2][15], float ycl, float zcl, double out[6])
{
    /* W = V1^-1 + V2^-1 on (y, z); m = W^-1 (V1^-1 m1 + V2^-1 m2) */
    double Vi[2][3], g[2][2];
    for (int k = 0; k < 2; ++k) {
        const double vyy = c[k][0], vyz = c[k][1], vzz = c[k][2];
        const double det = vyy * vzz - vyz * vyz;
        Vi[k][0] = vzz / det;
        Vi[k][1] = -vyz / det;
        Vi[k][2] = vyy / det;
        g[k][0] = Vi[k][0] * a[k][2] + Vi[k][1] * a[k][3];
        g[k][1] = Vi[k][1] * a[k][2] + Vi[k][2] * a[k][3];
    }
    const double W00 = Vi[0][0] + Vi[1][0], W01 = Vi[0][1] + Vi[1][1], W11 = Vi[0][2] + Vi[1][2];
    const double dW = W00 * W11 - W01 * W01;
    const double b0 = g[0][0] + g[1][0], b1 = g[0][1] + g[1][1];
    const double my = (W11 * b0 - W01 * b1) / dW;
    const double mz = (-W01 * b0 + W00 * b1) / dW;
    const double f = (a[0][4] / c[0][5] + a[1][4] / c[1][5]) / (1.0 / c[0][5] + 1.0 / c[1][5]);
    const double tl = (a[0][5] / c[0][9] + a[1][5] / c[1][9]) / (1.0 / c[0][9] + 1.0 / c[1][9]);
    const double r = sqrt((1.0 - f) * (1.0 + f));
    out[0] = (double)ycl - my;
    out[1] = (double)zcl - mz;
    out[2] = f / r;
    out[3] = tl / r;
    out[4] = W11 / dW;
    out[5] = W00 / dW;
}

/* Accumulate the residuals of n tracks into sums[ORA_NVOX][ORA_VOX_SUMS]
 * (added to what is there) and, optionally, abs_sums (the same sums of
 * absolute values, for tolerances).  Inputs are the FP32 arrays the library
 * reads: refit states (alpha, x [n], par [5][n], cov [15][n], status [n]; only
 * tracks with both statuses 0 contribute) and clusters (y, z [152][n], sector
 * int8 [152][n], -1 = none; a non-finite y or z is no cluster either).  Per
 * track, the TRD refit is carried inward
 * through the rows with a cluster (151 down to 0) and the ITS refit outward
 * (0 up to 151), each with tpc_carry; a cluster where both arrive gives a
 * residual.  Optional per-cluster outputs: res_out [4][152][n] (dy, dz, t, u;
 * NaN where none), vox_out [152][n] (-1 where none), var_out [2][152][n]
 * (variance of the combined y and z), and slack_out [n] (smallest slack of
 * the track's |snp| decisions).                                             */
int ora_residuals(int n, const float *ia, const float *ix, const float *ipar, const float *icov, const int *ist,
                  const float *ta, const float *tx, const float *tpar, const float *tcov, const int *tst,
                  const float *cy, const float *cz, const signed char *csec, double bz, int n_threads,
                  double *sums, double *abs_sums, float *res_out, int *vox_out, float *var_out,
                  double *slack_out)
{
    if (n < 0 || !sums) return -1;
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel
#endif
    {
        double (*trd_st)[7] = malloc(sizeof(double[7]) * ORA_TPC_ROWS);
        double (*trd_c)[15] = malloc(sizeof(double[15]) * ORA_TPC_ROWS);
        int *trd_ok = malloc(sizeof(int) * ORA_TPC_ROWS);
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int i = 0; i < n; ++i) {
            double sI[7] = {ia[i], ix[i]}, sT[7] = {ta[i], tx[i]}, cI[15], cT[15];
            for (int k = 0; k < 5; ++k) {
                sI[2 + k] = ipar[(size_t)k * n + i];
                sT[2 + k] = tpar[(size_t)k * n + i];
            }
            for (int k = 0; k < 15; ++k) {
                cI[k] = icov[(size_t)k * n + i];
                cT[k] = tcov[(size_t)k * n + i];
            }
            const int use = ist[i] == 0 && tst[i] == 0;
            double slack = INFINITY;
            /* the TRD refit, inward */
            int frame = -1;
            for (int r = ORA_TPC_ROWS - 1; r >= 0; --r) {
                const size_t q = (size_t)r * n + i;
                const int s = csec[q];
                trd_ok[r] = 0;
                if (!use || s < 0 || s >= ORA_NSECTOR || !isfinite(cy[q]) || !isfinite(cz[q])) continue;
                if (tpc_carry(sT, cT, &frame, s, tpc_row_x(r), bz, &slack)) continue;
                memcpy(trd_st[r], sT, sizeof sT);
                memcpy(trd_c[r], cT, sizeof cT);
                trd_ok[r] = 1;
            }
            /* the ITS refit, outward; combine where both arrived */
            frame = -1;
            for (int r = 0; r < ORA_TPC_ROWS; ++r) {
                const size_t q = (size_t)r * n + i;
                const int s = csec[q];
                double o[6];
                int vox = -1;
                if (use && s >= 0 && s < ORA_NSECTOR && isfinite(cy[q]) && isfinite(cz[q]) &&
                    tpc_carry(sI, cI, &frame, s, tpc_row_x(r), bz, &slack) == 0 && trd_ok[r]) {
                    double a2[2][7], c2[2][15];
                    memcpy(a2[0], sI, sizeof sI);
                    memcpy(c2[0], cI, sizeof cI);
                    memcpy(a2[1], trd_st[r], sizeof sI);
                    memcpy(c2[1], trd_c[r], sizeof cI);
                    tpc_combine(a2, c2, cy[q], cz[q], o);
                    vox = ora_voxel_of(cy[q], cz[q], s, r);
                }
                if (res_out)
                    for (int k = 0; k < 4; ++k) res_out[(size_t)k * ORA_TPC_ROWS * n + q] = vox >= 0 ? (float)o[k] : NAN;
                if (var_out)
                    for (int k = 0; k < 2; ++k)
                        var_out[(size_t)k * ORA_TPC_ROWS * n + q] = vox >= 0 ? (float)o[4 + k] : NAN;
                if (vox_out) vox_out[q] = vox;
                if (vox < 0) continue;
                const double dy = o[0], dz = o[1], t = o[2], u = o[3];
                const double term[ORA_VOX_SUMS] = {1.0, t, u, t * t, u * u, dy, dz, t * dy, u * dz, dy * dy, dz * dz};
                double *S = sums + (size_t)vox * ORA_VOX_SUMS;
                for (int k = 0; k < ORA_VOX_SUMS; ++k) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                    S[k] += term[k];
                }
                if (abs_sums) {
                    double *A = abs_sums + (size_t)vox * ORA_VOX_SUMS;
                    for (int k = 0; k < ORA_VOX_SUMS; ++k) {
#ifdef _OPENMP
#pragma omp atomic
#endif
                        A[k] += fabs(term[k]);
                    }
                }
            }
            if (slack_out) slack_out[i] = slack;
        }
        free(trd_st);
        free(trd_c);
        free(trd_ok);
    }
    return 0;
}

/* The distortion vector of each voxel: least squares of dy_i = Dy - Dx t_i,
 * dz_i = Dz - Dx u_i.  Eliminating Dy and Dz:
 *   Dx = -[n (Stdy + Sudz) - St Sdy - Su Sdz] / [n (Stt + Suu) - St^2 - Su^2],
 *   Dy = (Sdy + St Dx) / n,  Dz = (Sdz + Su Dx) / n.
 * out[nvox][6] = {Dx, Dy, Dz, n, rms dy, rms dz} (rms of the raw residuals
 * about their mean); a voxel with fewer than min_count clusters or no spread
 * in angle gets NaN for Dx, Dy, Dz.                                         */
int ora_voxel_solve(const double *sums, int nvox, int min_count, double *out)
{
    if (!sums || !out || nvox < 0) return -1;
    for (int v = 0; v < nvox; ++v) {
        const double *S = sums + (size_t)v * ORA_VOX_SUMS;
        double *o = out + (size_t)v * 6;
        const double n = S[0];
        o[3] = n;
        o[0] = o[1] = o[2] = o[4] = o[5] = NAN;
        if (n < (double)(min_count > 1 ? min_count : 1)) continue;
        o[4] = sqrt(fmax(S[9] / n - (S[5] / n) * (S[5] / n), 0.0));
        o[5] = sqrt(fmax(S[10] / n - (S[6] / n) * (S[6] / n), 0.0));
        const double den = n * (S[3] + S[4]) - S[1] * S[1] - S[2] * S[2];
        if (!(den > 1e-12 * n * n)) continue;
        const double dx = -(n * (S[7] + S[8]) - S[1] * S[5] - S[2] * S[6]) / den;
        o[0] = dx;
        o[1] = (S[5] + S[1] * dx) / n;
        o[2] = (S[6] + S[2] * dx) / n;
    }
    return 0;
}
