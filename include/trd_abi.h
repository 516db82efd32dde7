/*
 * trd_abi.h -- C ABI of the B300 TRD tracklet follower (libtrd.so).
 *
 * The library matches extrapolated ITS-TPC seed tracks to TRD tracklets with
 * a Kalman filter that keeps the best N hypotheses per layer (arXiv:2003.03174,
 * Sec. 3 and Fig. 2).  All compute runs in hand-written FP32 CUDA kernels for
 * sm_103a; there is no CPU fallback: every entry point that needs the GPU
 * returns TRD_ECUDA when no usable device is present.
 *
 * Conventions used by every call:
 *   - Return value: TRD_OK (0) or a negative TRD_E* code.  No call aborts the
 *     process or leaves a CUDA error pending on success.
 *   - Units: cm, GeV/c, Tesla.  Angles in radians.
 *   - Track state in the local frame of a sector: alpha (azimuth of the frame),
 *     x (radius of the reference plane), and five parameters
 *     p = (y, z, snp = sin(phi), tgl = tan(lambda), q2pt = q/pT).
 *   - Covariance: 15 terms, lower triangle row by row:
 *     c00 c10 c11 c20 c21 c22 c30 c31 c32 c33 c40 c41 c42 c43 c44.
 *   - Arrays are structure-of-arrays, FP32 unless stated.  A "[k][n]" array is
 *     k rows of n contiguous values (row r of track i at r*n + i).
 *   - Geometry: 18 sectors x 5 stacks x 6 layers (Sec. 3); chamber id =
 *     sector*30 + stack*6 + layer in 0..539; layer planes at x = 300 + 12.6 l;
 *     sector s centred at alpha = (s + 0.5) * 20 degrees; stacks of 18 pad rows
 *     of 8 cm covering z in [-360, 360); pads tilted by +2 degrees on even and
 *     -2 degrees on odd layers.
 *   - Streams: `stream` arguments are cudaStream_t values passed as void*;
 *     NULL means the legacy default stream.  Calls that take a stream are
 *     asynchronous with respect to the host unless stated.
 */
#ifndef TRD_ABI_H
#define TRD_ABI_H

#include <stdint.h>

#if defined(__GNUC__)
#define TRD_API __attribute__((visibility("default")))
#else
#define TRD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes -------------------------------------------------------- */
#define TRD_OK 0
#define TRD_EINVAL (-1)   /* invalid argument (null pointer, bad size, bad parameter) */
#define TRD_ENOMEM (-2)   /* device or pinned host allocation failed */
#define TRD_EAGAIN (-3)   /* resource temporarily full, or result not ready yet */
#define TRD_ETIMEOUT (-4) /* a bounded device wait ran out */
#define TRD_ECUDA (-5)    /* a CUDA runtime call failed (no device, launch error, ...) */

/* ---- per-track status bits (trd_results_t.status) ----------------------- */
#define TRD_ST_OK 0           /* followed through all 6 layers */
#define TRD_ST_PROP_FAIL 1    /* every hypothesis failed transport (|snp| >= 0.95) at some layer */
#define TRD_ST_STOPPED 2      /* no extension left: missing-layer budget spent, no candidate */
#define TRD_ST_SEED_INVALID 4 /* seed |snp| >= 0.95 or covariance not positive definite */

#define TRD_N_LAYERS 6
#define TRD_N_CHAMBERS 540
#define TRD_MAX_HYP 8 /* largest N (hypotheses kept per layer) the kernels support */

typedef struct trd_ctx trd_ctx_t;
typedef struct trd_index trd_index_t;
typedef struct trd_batch trd_batch_t;
typedef struct trd_server trd_server_t;

/* Seeds: ITS-TPC tracks extrapolated towards the TRD (Sec. 3), in any frame
 * alpha.  Device pointers, each n floats; cov is [15][n].  Read only.
 * trigger (optional, may be NULL): int32 interaction id of each seed (its
 * bunch crossing); when both a seed and a tracklet carry an id >= 0, the
 * tracklet is a candidate only if the ids are equal (Sec. 4: only tracklets
 * of the track's own interaction are considered).                           */
typedef struct {
    const float *alpha, *x, *y, *z, *snp, *tgl, *q2pt;
    const float *cov;
    int32_t n;
    const int32_t *trigger;
} trd_seeds_t;

/* Tracklets: the FEE straight-line fits of Sec. 3 (local y at the chamber's
 * reference radius, z of the pad row, deflection dy over the 3 cm drift), with
 * their 2x2 covariance (vyy, vzz, vyz).  chamber in 0..539; tracklets with a
 * chamber id outside that range, a non-finite y/z/dy, or a negative variance
 * are left out of the index and counted (trd_index_info).  Device pointers,
 * each n entries.  Read only.                                               */
typedef struct {
    const int32_t *chamber;
    const float *y, *z, *dy, *vyy, *vzz, *vyz;
    int32_t n;
    const int32_t *trigger; /* optional interaction id per tracklet (see trd_seeds_t) */
    const float *x;         /* optional radius of each tracklet in its sector frame (cm): with
                               misalignment not every tracklet sits at its layer's radius (Sec. 3);
                               NULL = the layer's nominal radius.  A non-finite x rejects the
                               tracklet.  Not accepted by trd_index_build_noalloc. */
} trd_tracklets_t;

/* Follower parameters.
 *   bz            solenoid field (T); the Lorentz angle sign follows it (Fig. 3)
 *   n_sigma_road  half-width of the search road in sigma of the residual (Sec. 3)
 *   chi2_cut      a candidate needs chi2 (y and z only, 2 dof) below this (Sec. 3)
 *   p_miss        score penalty of a layer without a tracklet
 *   dy_gate_sigma deflection deviation allowed, in sigma (4 in Sec. 3)
 *   n_hyp         hypotheses kept per layer, N_candidates of Sec. 3 (1..TRD_MAX_HYP)
 *   max_missing   layers a hypothesis may skip
 *   res_mode      0: tracklet y variance from the input; 1: from the resolution
 *                 parametrisation in sin(phi) of the track (Sec. 3, Fig. 3)
 *   material_on   1: one material step (scattering + energy loss) per layer  */
typedef struct {
    float bz, n_sigma_road, chi2_cut, p_miss, dy_gate_sigma;
    int32_t n_hyp, max_missing, res_mode, material_on;
} trd_params_t;

/* Results: device pointers written by trd_follow, caller-owned.
 *   alpha, x [n]; par [5][n]; cov [15][n]; chi2 [n] (sum of the attached
 *   tracklets' chi2); n_trk, n_miss, status [n] (int32); tracklet_id [6][n]
 *   (int32, index into the caller's tracklet arrays, -1 = no tracklet).
 * The state is the best hypothesis after its last completed layer.         */
typedef struct {
    float *alpha, *x, *par, *cov, *chi2;
    int32_t *n_trk, *n_miss, *status, *tracklet_id;
} trd_results_t;

/* ---- context ---------------------------------------------------------------
 * trd_ctx_create: bind to CUDA device `device` (makes it current on the calling
 * thread) and read its properties.  *ctx is owned by the caller and released
 * with trd_ctx_destroy.  Errors: TRD_EINVAL (ctx NULL), TRD_ECUDA (no such
 * device, or the device is not sm_103), TRD_ENOMEM.                         */
TRD_API int trd_ctx_create(int device, trd_ctx_t **ctx);
TRD_API int trd_ctx_destroy(trd_ctx_t *ctx);

/* Number of SMs of the context's device (for sizing), or a negative code. */
TRD_API int trd_ctx_sm_count(const trd_ctx_t *ctx);

/* ---- tracklet index (Sec. 3: "all tracklets inside a search road") --------
 * trd_index_build: bucket the tracklets by (chamber, pad row, y bin) with a
 * counting sort on `stream`, and record the largest vyy and vzz.  The y bins
 * of one (chamber, pad row) are adjacent, so a road query is one contiguous
 * range per pad row.  y_bin_width (cm, >= 0.05; 0 selects 2 cm)
 * sets the bin size.  The library allocates and owns the index (*out, freed
 * by trd_index_free); the input arrays may be reused once `stream` has passed
 * the build.  Errors: TRD_EINVAL, TRD_ENOMEM, TRD_ECUDA.                     */
TRD_API int trd_index_build(trd_ctx_t *ctx, const trd_tracklets_t *tracklets, float y_bin_width,
                    void *stream, trd_index_t **out);
TRD_API int trd_index_free(trd_index_t *index);

/* Resident-index pattern for repeated timeframes: trd_index_create allocates
 * an index for up to `capacity` tracklets (library-owned, freed by
 * trd_index_free); trd_index_rebuild refills it from new tracklets on
 * `stream` without allocating (TRD_EINVAL if n > capacity).  Work that still
 * reads the previous contents must be ordered before the rebuild on the
 * caller's streams.                                                         */
TRD_API int trd_index_create(trd_ctx_t *ctx, int32_t capacity, float y_bin_width, trd_index_t **out);
TRD_API int trd_index_rebuild(trd_index_t *index, const trd_tracklets_t *tracklets, void *stream);

/* Synchronises with the index's build stream, then reports the number of
 * tracklets indexed and the number rejected as invalid.                     */
TRD_API int trd_index_info(const trd_index_t *index, int32_t *n_indexed, int32_t *n_rejected,
                   int32_t *n_buckets);

/* Copies the index to host memory (synchronises with its build stream), for
 * inspection and tests.  offsets: n_buckets + 1 int32 (bucket b holds
 * entries offsets[b] .. offsets[b+1]-1; bucket = (chamber * 18 + pad row) *
 * n_ybins + y bin); ids: n_indexed int32 input indices in bucket order.
 * Either pointer may be NULL.  Host pointers, caller-owned.                 */
TRD_API int trd_index_copy_out(const trd_index_t *index, int32_t *offsets, int32_t *ids);

/* Index build that allocates nothing (the paper has no counterpart: this is
 * for callers that cannot allocate device memory where they build an index,
 * such as code inside a framework whose pool owns every device allocation, or
 * a real-time loop that must not call cudaMalloc because it can synchronise
 * the device).  It runs the same kernels as trd_index_build on the current
 * device and writes the index into the caller's device buffers:
 *   offsets  n_buckets + 1 int32, n_buckets = 540 * 18 * ceil(132 / w)
 *            (bucket = (chamber * 18 + pad row) * n_ybins + y bin)
 *   records  8 floats per tracklet (16-byte aligned): {y, z, dy, input index
 *            as int32 bits}, {vyy, vzz, vyz, trigger as int32 bits (-1 when
 *            the tracklets carry none)}, in bucket order; the first
 *            offsets[n_buckets] records are written
 *   stats    4 uint32: largest vyy and vzz (float bits), rejected count, 0
 * Its scratch is a fixed device array inside the library (about 9.3 MB on
 * every GPU that loads it, kept until exit), so it accepts at most 1,048,576
 * tracklets and y bins of at least 1 cm (w = 0 selects 2 cm); anything larger
 * returns TRD_EINVAL.  All calls on a device share that scratch: calls that
 * overlap on the GPU (other streams, other threads) race and must be ordered
 * by the caller.  The first call on each device looks up the array's device
 * address (no allocation), and so does the first call after the device's
 * context was re-created (cudaDeviceReset); make such a call before any
 * stream capture.
 * Asynchronous on `stream`; the inputs must stay valid until it completes.
 * Errors: TRD_EINVAL (NULL pointer, size or bin width beyond the limits,
 * misaligned records), TRD_ECUDA.                                           */
TRD_API int trd_index_build_noalloc(const trd_tracklets_t *tracklets, float y_bin_width,
                                    int32_t *offsets, float *records, uint32_t *stats,
                                    void *stream);

/* ---- the follower (Sec. 3) -------------------------------------------------
 * trd_follow: for every seed, rotate it into the sector of its position,
 * then for layers 0..5: transport the helix and covariance to the layer plane
 * (changing sector at the edge), apply the material step, query the index
 * inside the n-sigma road, test each candidate (pad-tilt-corrected chi2 of y
 * and z, dy gate), keep the best n_hyp extensions (a layer may be skipped
 * while max_missing allows), and update with the chosen tracklet.  Selection
 * order: lowest score (sum of chi2 plus p_miss per missing layer), then
 * parent rank, then tracklet id, a missing layer last.
 * All pointers are device pointers owned by the caller; results are written
 * asynchronously on `stream`.  The index must have been built on `stream` or
 * on a stream `stream` has synchronised with.
 * Seeds are processed in order of decreasing |q/pT| (lanes that work together
 * then have roads of similar width); results do not depend on the order and
 * are written at the seeds' input positions.  The call's scratch (136 bytes
 * per seed + 528: sorted seed states, staged results and the call's own work
 * counter, so calls in flight on any number of streams never share one) is
 * taken from the device's default memory pool, ordered on `stream`
 * (cudaMallocAsync / cudaFreeAsync).
 * Errors: TRD_EINVAL (NULL pointers, n < 0, n_hyp outside 1..TRD_MAX_HYP,
 * non-positive road/cut), TRD_ENOMEM (no scratch), TRD_ECUDA (launch
 * failure).                                                                 */
TRD_API int trd_follow(trd_ctx_t *ctx, const trd_seeds_t *seeds, const trd_index_t *index,
               const trd_params_t *params, trd_results_t *out, void *stream);

/* Launch shape of the follower (the autotuner's search space).
 *   lanes_per_track   lanes that follow one seed, one hypothesis per lane,
 *                     all of them sharing each hypothesis's road scan:
 *                     1, 2, 4, 8 or 32 (a whole warp per seed, for wide roads)
 *                     (0 = smallest power of two >= n_hyp; 1 needs n_hyp = 1)
 *   block_threads     64 or 128 (0 = 128)
 *   min_blocks_per_sm register budget: 128-thread blocks kept resident per SM
 *                     (1 lane: 4, 5, 6 or 8; 2, 4 or 8 lanes: 3, 4, 5 or 6;
 *                     32 lanes: 3 or 4; 0 = 4 for 1 or 32 lanes, 5 for 8,
 *                     6 for 2 or 4)
 * The follower orders extensions by keys that hold a tracklet id in 28 bits,
 * so an index of one timeframe may hold at most 268,435,454 tracklets
 * (TRD_EINVAL beyond).                                                      */
typedef struct {
    int32_t lanes_per_track, block_threads, min_blocks_per_sm;
} trd_launch_t;

/* trd_follow with an explicit launch shape; launch may be NULL (defaults).
 * TRD_EINVAL for a shape outside the list above.                            */
TRD_API int trd_follow_tuned(trd_ctx_t *ctx, const trd_seeds_t *seeds, const trd_index_t *index,
                             const trd_params_t *params, trd_results_t *out, void *stream,
                             const trd_launch_t *launch);

/* trd_follow_timed: trd_follow_tuned that also records two caller-owned CUDA
 * events (cudaEvent_t handles, created with timing enabled) on `stream`:
 * ev_start just before the follower kernel is launched and ev_end just after
 * it, so that cudaEventElapsedTime(ev_start, ev_end) is that kernel's device
 * time alone (the seeds' key and pre-pass before it and the gather of the
 * results after it lie outside the pair).  The events keep the kernel from
 * starting while the pre-pass drains (programmatic dependent launch), so a
 * timed call takes a little longer than an untimed one.  With no seeds both
 * events are recorded at once.  Results are those of trd_follow_tuned.
 * Errors as trd_follow_tuned, plus TRD_EINVAL for a NULL event.             */
TRD_API int trd_follow_timed(trd_ctx_t *ctx, const trd_seeds_t *seeds, const trd_index_t *index,
                             const trd_params_t *params, trd_results_t *out, void *stream,
                             const trd_launch_t *launch, void *ev_start, void *ev_end);

/* ---- misalignment and field map (Sec. 3) ---------------------------------------
 * Misaligned chambers put tracklets at different radii; the paper carries a
 * track to the average radius of the chamber (through the field's
 * inhomogeneities), compares it with each tracklet by a fast linear
 * extrapolation to that tracklet's radius, and transports it precisely to
 * the matched tracklet's radius before the update.
 *   chamber_x (device, [540] float, or NULL): average radius of each chamber
 *     (cm); a hypothesis in chamber c is carried from its layer's nominal
 *     radius (where the chamber is found from z) on to chamber_x[c].
 *   bz_map (device, [nz][nr] float, or NULL): Bz (T) at r_i = r_min + i (r_max -
 *     r_min) / (nr - 1), z_j likewise, bilinear between nodes, clamped to the
 *     box; every transport step uses the map at its midpoint (estimated along
 *     the straight line from the step's start), every rotation the map at the
 *     state's point.  The Lorentz-angle sign still follows params.bz.
 * Per-tracklet radii come with the tracklets (trd_tracklets_t.x, stored in
 * the index by trd_index_build/rebuild): a candidate is then tested at its
 * own radius by extrapolating the hypothesis along its direction
 * (covariance as at the chamber radius), and a matched tracklet's hypothesis
 * is transported to its radius before the update.
 * trd_follow_aligned: trd_follow_tuned with an alignment (NULL = none).
 * Errors as trd_follow_tuned, plus TRD_EINVAL for nr or nz < 2 or an empty
 * box.                                                                      */
typedef struct {
    const float *chamber_x;
    const float *bz_map;
    int32_t nr, nz;
    float r_min, r_max, z_min, z_max;
} trd_alignment_t;

TRD_API int trd_follow_aligned(trd_ctx_t *ctx, const trd_seeds_t *seeds, const trd_index_t *index,
                               const trd_params_t *params, const trd_alignment_t *align, trd_results_t *out,
                               void *stream, const trd_launch_t *launch);

/* ---- TRD-only refit (Sec. 2, step 3) ----------------------------------------
 * The space-point calibration refits each matched track twice without the TPC
 * clusters: from the ITS, and from TRD and TOF.  trd_refit is the TRD half
 * (no TOF point is modelled).  For every track with at least two tracklets
 * whose follower status lacks TRD_ST_SEED_INVALID:
 *   1. prior: the follower's final state, its covariance reduced to the
 *      diagonal and multiplied by cov_scale (> 0; e.g. 100 widens every
 *      error tenfold), so little of the TPC-derived information is kept
 *      (FP32: up to cov_scale ~1e3 the results stay within 1e-4 of the FP64
 *      refit; a wider prior costs accuracy in the first update);
 *   2. from the outermost layer with a tracklet down to layer 0: transport
 *      to the layer plane (entering the tracklet's sector, or the neighbour
 *      sector at the azimuthal edge of a layer without tracklet), Kalman
 *      update with the tracklet (same pad-tilt model, res_mode and Joseph
 *      form as trd_follow), then, with material_on, the layer's material
 *      with the mean energy loss added back;
 *   3. output: the state at the plane of layer 0 (x = 300 cm) in its sector
 *      frame, the covariance, the sum of the update chi2, the number of
 *      updates and a status.
 * tracks (read only, device): results of trd_follow for n tracks (alpha, x,
 *   par, cov diagonal, status, tracklet_id are read; the other fields are
 *   ignored).  tracklets (read only, device): the arrays the ids refer to
 *   (chamber, y, z, vyy, vzz, vyz, and x when given: a layer with a
 *   tracklet is then refitted at that tracklet's own radius; dy and trigger
 *   are not read).  The field is homogeneous (params.bz).
 *   params: bz, res_mode and material_on are used.
 * out (device, caller-owned): alpha, x [n]; par [5][n]; cov [15][n];
 *   chi2 [n]; n_upd, status [n] (int32).  status: TRD_RF_OK, TRD_RF_PROP_FAIL
 *   (|snp| limit reached; the state is as far as it was carried), or
 *   TRD_RF_SKIPPED (fewer than two tracklets, an invalid seed, or a tracklet
 *   id or chamber outside the tracklet arrays; the output is the input
 *   state with a zero covariance).
 * Asynchronous on `stream`.  Errors: TRD_EINVAL (NULL pointers, n < 0,
 * cov_scale not finite and positive), TRD_ECUDA.                             */
#define TRD_RF_OK 0
#define TRD_RF_PROP_FAIL 1
#define TRD_RF_SKIPPED 8

typedef struct {
    float *alpha, *x, *par, *cov, *chi2;
    int32_t *n_upd, *status;
} trd_refit_t;

TRD_API int trd_refit(trd_ctx_t *ctx, const trd_results_t *tracks, int32_t n,
                      const trd_tracklets_t *tracklets, const trd_params_t *params, float cov_scale,
                      trd_refit_t *out, void *stream);

/* ---- residuals in TPC sub-volumes and the distortion map (Sec. 2, steps 4
 * and 5) ----------------------------------------------------------------------
 * The calibration compares each distorted TPC cluster with the weighted
 * combination of the ITS refit and the TRD-only refit (trd_refit) of its
 * track, collects the residuals per TPC sub-volume, and derives one
 * distortion vector per sub-volume.
 *
 * Geometry (readings; the paper gives none): TRD_TPC_ROWS pad rows with
 * centres x_r = 85 + 160 (r + 1/2) / 152 cm, rounded to float; the 18
 * sectors of the TRD's segmentation; sub-volume (voxel) index
 *   (((side * 18 + sector) * 152 + row) * 15 + iy) * 5 + iz,
 * side = 1 for z < 0; iy = floor((y/x_r + tan 10 deg) * 15 / (2 tan 10 deg)),
 * iz = floor(|z|/x_r * 5), both clamped into range, evaluated in FP32 with
 * correctly rounded operations in that order.
 *
 * trd_residuals: for each of n tracks with both refit statuses 0, each
 * refit is carried along the track to every pad row with a cluster: to the
 * row plane in its current frame, and where the cluster lies in another
 * sector, rotated there into the cluster's sector and carried to the plane
 * again (helix transport, no material in the gas).  At each cluster the two
 * (y, z) estimates are combined with their inverse 2x2 covariances, sin(phi)
 * and tan(lambda) with their inverse variances; the residual (dy, dz) =
 * cluster - combination, with the combination's slopes t = tan(phi) and
 * u = tan(lambda) / cos(phi), is added to the cluster's voxel.
 *   its, trd (read only, device): states at any radius and frame (alpha, x
 *     [n]; par [5][n]; cov [15][n]; status [n]) -- e.g. the output of
 *     trd_refit for the TRD side.
 *   clusters (read only, device): y, z float [152][n] (local frame of the
 *     cluster's sector, z global); sector int8 [152][n], 0..17, any other
 *     value = no cluster on that row.  Non-finite y or z: no cluster.
 *   voxel_sums (device, caller-owned, accumulated into, zero it first):
 *     int64 [TRD_N_VOXELS][TRD_VOX_SUMS] = n, St, Su, Stt, Suu, Sdy, Sdz,
 *     Stdy, Sudz, Sdydy, Sdzdz; every sum except n holds round(v * 2^24) of
 *     each FP32 term (exact, order-independent integer sums).
 *   cluster_res (optional device output, NULL to skip): float [4][152][n] =
 *     dy, dz, t, u per cluster, NaN where there is none.
 * trd_voxel_solve: per voxel with at least min_count clusters, the least
 * squares solution of dy_i = Dy - Dx t_i, dz_i = Dz - Dx u_i (a cluster at
 * row x_r was freed at the track point x_r - Dx and moved by (Dy, Dz));
 * map (device, caller-owned) float [TRD_N_VOXELS][6] = Dx, Dy, Dz, n,
 * rms dy, rms dz (NaN where undetermined).
 * Both asynchronous on `stream`.  Errors: TRD_EINVAL (NULL pointers, n < 0,
 * n * 152 beyond int32), TRD_ECUDA.                                          */
#define TRD_TPC_ROWS 152
#define TRD_VOX_Y_BINS 15
#define TRD_VOX_Z_BINS 5
#define TRD_N_VOXELS (2 * 18 * TRD_TPC_ROWS * TRD_VOX_Y_BINS * TRD_VOX_Z_BINS)
#define TRD_VOX_SUMS 11

typedef struct {
    const float *alpha, *x, *par, *cov;
    const int32_t *status;
} trd_states_t;

typedef struct {
    const float *y, *z;
    const int8_t *sector;
} trd_tpc_clusters_t;

TRD_API int trd_residuals(trd_ctx_t *ctx, int32_t n, const trd_states_t *its, const trd_states_t *trd,
                          const trd_tpc_clusters_t *clusters, float bz, int64_t *voxel_sums, float *cluster_res,
                          void *stream);
TRD_API int trd_voxel_solve(trd_ctx_t *ctx, const int64_t *voxel_sums, int32_t min_count, float *map,
                            void *stream);

/* ---- batches of timeframes (Sec. 3.1: Run 3 processes time frames of many
 * collisions; here many time frames at once) ----------------------------------
 * A batched follow, "follow n_tf timeframes in one persistent, graph-captured
 * launch", is split here into create / run / free: a CUDA graph is bound to
 * its buffers when it is captured, so the capture (trd_batch_create, which
 * also sizes the batch's index and scratch) happens once and each
 * trd_batch_run replays it on fresh contents of the same buffers.  One
 * create + run + free is the single-call form; a caller that refills the
 * buffers keeps the batch and calls run again.
 * trd_batch_create: prepare one CUDA graph that, for n_tf timeframes stored
 * back to back, builds a single index over all their tracklets and follows
 * all their seeds in one persistent launch that pulls seeds of every
 * timeframe from one work queue.
 *   seed_offsets, tracklet_offsets  host arrays of n_tf + 1 int32: timeframe t
 *       owns seeds [seed_offsets[t], seed_offsets[t+1]) of `seeds` and
 *       tracklets [tracklet_offsets[t], ...) of `tracklets`; offsets[0] = 0,
 *       non-decreasing, offsets[n_tf] = n (empty timeframes are allowed).
 *   seeds, tracklets, results: device arrays of the concatenated timeframes,
 *       caller-owned, bound to the graph (refill them in place between runs).
 *       Result tracklet ids are local to each seed's timeframe.
 *   params, y_bin_width, launch: as for trd_index_build / trd_follow_tuned.
 * The library owns the batch (index, offsets, the follower's scratch of 136
 * bytes per seed + 16 + 512 * min(n_tf, 8), graph); free with trd_batch_free.
 * Seeds are taken timeframe by timeframe, each timeframe's in
 * decreasing-|q/pT| order (128 momentum bins per timeframe up to 8
 * timeframes, 1,024 bins shared out beyond); each
 * seed's arithmetic is the same as in trd_follow on its timeframe alone, so
 * results are identical.
 * trd_batch_run replays the graph on `stream` (asynchronous).  A batch must
 * not be run concurrently with itself.
 * Errors: TRD_EINVAL (bad offsets, parameters or shape), TRD_ENOMEM,
 * TRD_ECUDA.                                                                */
TRD_API int trd_batch_create(trd_ctx_t *ctx, int32_t n_tf, const int32_t *seed_offsets,
                             const int32_t *tracklet_offsets, const trd_seeds_t *seeds,
                             const trd_tracklets_t *tracklets, const trd_params_t *params,
                             trd_results_t *results, float y_bin_width, const trd_launch_t *launch,
                             trd_batch_t **out);
TRD_API int trd_batch_run(trd_batch_t *batch, void *stream);
TRD_API int trd_batch_free(trd_batch_t *batch);

/* ---- serving (Sec. 3.1: timeframes arrive continuously and are tracked
 * synchronously with data taking) -------------------------------------------
 * A server owns a scheduler thread, max_slots CUDA streams and one resident
 * index per stream.  Requests are admitted in arrival order as soon as a
 * stream is free and the request's device bytes fit mem_budget_bytes
 * (inputs + results + the stream's index); admitted requests run
 * concurrently on their streams, so the copies of one overlap the kernels of
 * another, and a request that arrives while others are on the GPU starts as
 * soon as a stream and memory free up.  Each request's arithmetic is that of
 * trd_follow on its timeframe alone.                                        */
typedef struct {
    uint64_t mem_budget_bytes; /* device bytes for requests and indices (0 = 60 GiB) */
    int32_t max_slots;         /* requests on the GPU at once, 1..64 (0 = 4) */
    int32_t max_queue;         /* requests waiting for admission (0 = 1024) */
    float y_bin_width;         /* index bin width in cm (0 = 2) */
    trd_params_t params;       /* follower parameters of every request */
    trd_launch_t launch;       /* follower launch shape (zeros = defaults) */
} trd_server_cfg_t;

/* Host-clock seconds (steady clock) of one request, its GPU time, and its
 * stages on the device clock: milliseconds since the server was created, read
 * from CUDA events recorded on the request's stream before its first input
 * copy (start_ms), after its last input copy (inputs_ms), after its index
 * build and follower (kernels_ms) and after its last result copy
 * (results_ms).  The marks of requests on different slots share that origin,
 * so they show which requests' copies ran under which requests' kernels.
 * A failed request's marks are zero.                                        */
typedef struct {
    double submit_s, admit_s, done_s; /* done_s: stream callback after the results landed */
    float gpu_ms;                     /* first input copy to last result copy, CUDA events */
    int32_t slot;
    float start_ms, inputs_ms, kernels_ms, results_ms;
} trd_timing_t;

/* trd_server_create: errors TRD_EINVAL (bad config or parameters),
 * TRD_ENOMEM, TRD_ECUDA.  The server is owned by the caller; destroy it with
 * trd_server_destroy, which finishes queued and running requests first.    */
TRD_API int trd_server_create(trd_ctx_t *ctx, const trd_server_cfg_t *cfg, trd_server_t **out);

/* trd_server_submit: queue one timeframe.  seeds, tracklets and results are
 * HOST pointers (layouts as for trd_follow) that must stay valid until the
 * request completes; page-locked host memory lets the copies overlap other
 * requests' kernels.  *ticket identifies the request.  The host result
 * buffers are named here rather than at poll time because the result copies
 * are enqueued on the request's stream right behind its kernels (they then
 * overlap the next request's work); poll only reports that they landed.  Errors: TRD_EINVAL,
 * TRD_ENOMEM (the request alone exceeds the budget), TRD_EAGAIN (queue
 * full: retry later).                                                       */
TRD_API int trd_server_submit(trd_server_t *server, const trd_seeds_t *seeds,
                              const trd_tracklets_t *tracklets, trd_results_t *results,
                              uint64_t *ticket);

/* trd_server_poll: non-blocking.  TRD_OK: the results are in the caller's
 * host buffers and the ticket is released (timing filled if not NULL);
 * TRD_EAGAIN: not finished; TRD_EINVAL: unknown or already released ticket;
 * another negative code: the request failed (ticket released).
 * trd_server_wait: the same, waiting at most timeout_ms on the host
 * (TRD_ETIMEOUT when it runs out).                                          */
TRD_API int trd_server_poll(trd_server_t *server, uint64_t ticket, trd_timing_t *timing);
TRD_API int trd_server_wait(trd_server_t *server, uint64_t ticket, int32_t timeout_ms,
                            trd_timing_t *timing);

/* Requests waiting, requests on the GPU, device bytes held (I/O + indices). */
TRD_API int trd_server_stats(trd_server_t *server, int32_t *queued, int32_t *in_flight,
                             uint64_t *device_bytes);
TRD_API int trd_server_destroy(trd_server_t *server);

/* FP32 FMA throughput of the context's device in TFLOP/s (independent FMA
 * chains on every SM, best of 5 timed launches): the denominator of the
 * follower's arithmetic roofline.  Measurement only (not a step of the
 * method); synchronises the device.                                         */
TRD_API int trd_measure_fp32_peak(trd_ctx_t *ctx, double *tflops);

/* Geometry constants the library was built with, for cross-checks:
 * out[0..12] = n_sectors, n_stacks, n_layers, n_chambers, x_layer0,
 * dx_layer, stack_length, z_min, tilt_deg, drift_length, lorentz_deg,
 * c_light, max_snp.  Host only; needs no GPU.                               */
TRD_API int trd_geometry(double *out, int n);

/* Library version string (static storage).  Host only. */
TRD_API const char *trd_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TRD_ABI_H */
