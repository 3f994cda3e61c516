/*
 * tpc.h - C ABI of the B300 TPC track-finding and refit library.
 *
 * The library implements the data-parallel hot path of the ALICE Run 3 TPC
 * tracking described in arXiv:1811.11481 ("Track Reconstruction in the ALICE
 * TPC using GPUs for LHC Run 3"):
 *   - Sec. 2: sector-local cellular-automaton seeding (neighbour finder, link
 *     cleaning "evolution", start hits), tracklet construction with a
 *     simplified Kalman filter and cluster pick-up, tracklet selection;
 *   - Sec. 4: cluster time scaled linearly to z for seeding, closest approach
 *     to the beam line as the collision-time estimate, calibration applied
 *     between seeding and fitting;
 *   - Sec. 3: final Kalman refit iterated three times (inward, outward,
 *     inward) with outlier rejection on the predicted chi2;
 *   - an adjoint of the fixed-assignment refit (not in the paper).
 *
 * Conventions shared by every entry point:
 *   - Pointers documented as "device" must point to memory of the device that
 *     was current when the context was created; "host" pointers to host memory.
 *   - Every call returns tpc_status; nothing throws across the ABI. Errors
 *     detected on the device (capacity overflow, invalid cluster fields,
 *     non-finite fits) are latched in a device error word and reported by the
 *     next call that synchronises (tpc_find_tracks, tpc_sync, tpc_get_counts).
 *     tpc_last_error() gives a text for the last non-OK status.
 *   - All work is issued on the stream given to tpc_create, in call order.
 *     A context is not thread-safe; separate contexts are independent.
 *   - Units: cm, microseconds, Tesla, GeV. Local sector frame: x along the
 *     sector's centre line (pad-row planes x = row_x[r]), y along the pad row,
 *     z along the drift direction (global z).
 *   - A track state is (y, z, sin(phi), tan(lambda), q/pT) at a local x.
 *     Covariances are packed lower triangles in the order (0,0) (1,0) (1,1)
 *     (2,0) (2,1) (2,2) ... (4,4), 15 floats.
 */
#ifndef TPC_H_
#define TPC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TPC_OK = 0,
  TPC_ERR_ARG = 1,       /* invalid argument or invalid cluster field     */
  TPC_ERR_CAPACITY = 2,  /* an internal buffer was too small (see text)   */
  TPC_ERR_CUDA = 3,      /* a CUDA runtime call failed                    */
  TPC_ERR_TIMEOUT = 4,   /* a bounded device wait gave up                 */
  TPC_ERR_STATE = 5,     /* call sequence violated (e.g. backward first)  */
  TPC_ERR_NUMERIC = 6    /* non-finite value in a fit                     */
} tpc_status;

/* Cluster flag bits (Sec. 3 lists these special cluster types). In the
 * final refit each set bit scales the cluster's position error by its
 * factor (split_scale, single_row_scale, single_time_scale, edge_scale,
 * shared_scale of tpc_params), in this bit order; track finding uses the
 * plain error. */
#define TPC_FLAG_SPLIT 0x01u
#define TPC_FLAG_SINGLE_ROW 0x02u
#define TPC_FLAG_SINGLE_TIME 0x04u
#define TPC_FLAG_EDGE 0x08u
#define TPC_FLAG_SHARED 0x10u

#define TPC_N_SECTORS 36      /* 18 in azimuth x 2 sides (Sec. 2)            */
#define TPC_MAX_ROWS 160      /* row tables are sized for up to 160 rows     */
#define TPC_SPLINE_N 8        /* control points per spline axis              */
#define TPC_SPLINE_SIZE (TPC_N_SECTORS * 2 * 8 * 8 * 8) /* floats           */
#define TPC_GRAD_CALIB_SIZE (2 + TPC_SPLINE_SIZE)        /* doubles          */

typedef struct tpc_ctx tpc_ctx;

/* Detector geometry (Sec. 2: 36 trapezoidal sectors, 152 pad rows). Sector k
 * is rotated by ((k mod 18) + 1/2) * 20 degrees; k < 18 is the A side (z > 0),
 * k >= 18 the C side. Copied at tpc_create. */
typedef struct {
  int32_t n_rows;       /* number of pad rows, 3 .. TPC_MAX_ROWS            */
  const float* row_x;   /* host [n_rows], plane positions (cm), increasing  */
  float tan_half;       /* tan of the sector half-opening angle             */
  float drift_length;   /* L (cm): |z| of the readout plane                  */
  float bz;             /* uniform field (T)                                 */
  /* Native pad coordinates (tpc_clusters.pads = 1), or NULL: a cluster at
   * pad position p (in pads, continuous) of row r lies at
   * y = (p - pad_center[r]) * pad_width[r], computed in single precision on
   * the fly by the kernels that read y. */
  const float* pad_width;   /* host [n_rows] pad pitch (cm)                 */
  const float* pad_center;  /* host [n_rows] pad position of y = 0 (pads)   */
  /* The full field for the final refit (Sec. 3: Bx and By taken into
   * account, three-dimensional polynomial field), or NULL for the uniform
   * bz: host [3][10], the coefficients of Bx, By, Bz (T) as quadratic
   * polynomials in the global coordinates (X, Y, Z) in metres, monomials
   * 1, X, Y, Z, X^2, XY, XZ, Y^2, YZ, Z^2 (X, Y: sector k's local frame
   * rotated by its angle; Z along the beam). tpc_refit then transports the
   * state by fourth-order Runge-Kutta in the field (steps <= 0.5 cm) and
   * the covariance with the helix Jacobian of the local Bz (tpc_refit_backward
   * differentiates that transport); track finding, merging and compression
   * keep the uniform bz. */
  const float* field;
} tpc_geometry;

/* Cut values of the method (the paper gives none; defaults by
 * tpc_default_params). Copied at tpc_create. */
typedef struct {
  float sigma;            /* cluster position error (cm), y and z          */
  float shared_scale;     /* error scale for TPC_FLAG_SHARED clusters      */
  float nb_wy, nb_wz;     /* neighbour window offsets (cm)                 */
  float nb_teta;          /* neighbour z-slope window, sinh(eta_max)       */
  float nb_ty;            /* neighbour y-slope window, tan(phi_max)        */
  float nb_dmax;          /* max squared deviation from straight line      */
  float chi2_pick;        /* pick-up cut on the normalised distance        */
  int32_t max_miss;       /* consecutive empty rows that end following     */
  int32_t max_gap;        /* largest row gap inside an emitted track       */
  int32_t min_track_hits; /* minimum clusters of a track                   */
  float s_max;            /* |sin(phi)| limit of the propagation           */
  float inward_cov_scale; /* covariance scale before the inward pass       */
  float c0t[5];           /* tracklet seed covariance diagonal             */
  float c0r[5];           /* refit pass-1 covariance diagonal              */
  float chi2_out;         /* refit outlier cut on the predicted chi2       */
  int32_t min_acc_reject; /* accepted clusters before rejection starts     */
  float refit_inflate;    /* covariance inflation between refit passes     */
  int32_t seed_max_hits;  /* chain hits used by the tracklet seed fit      */
  float chi2_merge;       /* segment-merging cut on the 5-parameter chi2   */
  float split_scale;      /* error scale for TPC_FLAG_SPLIT clusters       */
  float single_row_scale; /* error scale for TPC_FLAG_SINGLE_ROW clusters  */
  float single_time_scale;/* error scale for TPC_FLAG_SINGLE_TIME clusters */
  float edge_scale;       /* error scale for TPC_FLAG_EDGE clusters        */
} tpc_params;

/* Calibration (Sec. 4 and Sec. 5.2): drift velocity, time offset and a
 * per-sector distortion given as a tensor-product uniform cubic B-spline with
 * 8 control points per axis over u = (x - spl_x0)/spl_dx,
 * v = (y/x + tan_half)/(2 tan_half), w = |z|/drift_length (each clamped to
 * [0,1]). corrected = measured + spline. */
typedef struct {
  double vdrift;        /* cm/us                                            */
  double t0;            /* us                                               */
  const float* spline;  /* device [36][2][8][8][8]: [sector][dy,dz][w][v][u],
                           or NULL for no distortion. Copied by the call.   */
  float spl_x0, spl_dx; /* spline x domain (cm)                             */
} tpc_calib;

/* One batch of clusters (structure of arrays, device pointers, caller-owned;
 * they must stay valid and unchanged until the last call that reads them:
 * tpc_find_tracks / tpc_refit / tpc_refit_backward of this batch). */
typedef struct {
  int64_t n;              /* number of clusters (< 2^31)                    */
  int32_t mode;           /* 0: z given (triggered events), 1: t given
                             (continuous readout, Sec. 4)                   */
  int32_t n_events;       /* independent events in the batch (>= 1)         */
  double tf_start;        /* time-frame start (us), mode 1                  */
  const float* y;         /* device [n] local y (cm)                         */
  const float* z;         /* device [n] z (cm), mode 0; else NULL           */
  const double* t;        /* device [n] absolute drift time (us), mode 1    */
  const uint8_t* row;     /* device [n] pad row, < n_rows                   */
  const uint8_t* sector;  /* device [n] sector, < 36                        */
  const uint8_t* flags;   /* device [n] TPC_FLAG_* bits, or NULL            */
  const uint32_t* event;  /* device [n] event index < n_events, or NULL     */
  int32_t pads;           /* 1: y holds native pad positions (pads), turned
                             into cm with the geometry's pad tables on the
                             fly (the next step the paper names after
                             Sec. 4: tracking in native pad, row and time
                             coordinates); the gradient grad_y of
                             tpc_refit_backward is then per pad. 0: y in cm */
} tpc_clusters;

/* A set of tracks as CSR over cluster indices of the loaded batch.
 * Returned by tpc_find_tracks (library-owned device memory, valid until the
 * next tpc_load_clusters / tpc_find_tracks / tpc_set_tracks / tpc_destroy), or
 * given by the caller to tpc_set_tracks (caller-owned device memory). */
typedef struct {
  int64_t n_tracks;
  int64_t n_assigned;            /* = track_start[n_tracks]                  */
  const uint32_t* track_start;   /* device [n_tracks + 1]                    */
  const uint32_t* cluster_idx;   /* device [n_assigned], input cluster index,
                                    strictly increasing pad row per track.
                                    Found tracks lie in one sector; a track
                                    merged across sectors (Sec. 2, second
                                    phase) is refitted with the state
                                    rotated into the frame of each
                                    cluster's sector (sectors k and k + 18
                                    share a frame); params, cov and x are
                                    then given in the frame of the track's
                                    last fitted cluster                    */
  const double* t_coll;          /* device [n_tracks] collision time (us) used
                                    for the absolute z (mode 1)             */
  const uint32_t* start_hit;     /* device [n_tracks] input index of the
                                    chain head (found tracks), may be NULL  */
} tpc_tracks;

/* Fill *p with the default cut values. */
void tpc_default_params(tpc_params* p);

/* Create a context on the current device. stream: a cudaStream_t (NULL =
 * legacy default stream). Copies geometry and params. Allocates scratch
 * lazily as batches are loaded. Returns TPC_ERR_ARG for invalid geometry. */
tpc_status tpc_create(const tpc_geometry* geo, const tpc_params* params, void* stream,
                      tpc_ctx** out);

/* Destroy the context and free all library-owned device memory. NULL is a
 * no-op. Synchronises the context's stream. */
void tpc_destroy(tpc_ctx* ctx);

/* Set the calibration (Sec. 4: applied between seeding and fitting). The
 * spline is copied (device to device, asynchronous on the stream); its
 * bounds are reduced on the device. Must precede tpc_load_clusters for the
 * seeding transform (vdrift, t0). */
tpc_status tpc_set_calib(tpc_ctx* ctx, const tpc_calib* calib);

/* Load a batch: validates fields, converts t to the seeding z (Sec. 4: linear
 * time scaling with tf_start as reference), buckets clusters by (event,
 * sector, row) and builds the per-row search grid. Asynchronous. May
 * allocate device memory when the batch is larger than any before (not
 * while a stream capture is active). */
tpc_status tpc_load_clusters(tpc_ctx* ctx, const tpc_clusters* cl);

/* Run the track finder on the loaded batch (neighbours, link cleaning, start
 * hits, tracklets, selection) and the calibration transform of the assigned
 * clusters. Synchronises once to read the track count, then fills *out.
 * Tracks come ordered by (event, sector, pad row, input index) of their start
 * hit, whatever the tuning (tpc_set_tuning); tracklets (tpc_get_tracklets)
 * come in search-grid order, which depends on grid_tau and grid_ny_max.
 * Returns TPC_ERR_CAPACITY if the tracklet buffer overflowed (the next call
 * retries with twice the capacity). */
tpc_status tpc_find_tracks(tpc_ctx* ctx, tpc_tracks* out);

/* Batching (many events of uneven size in one launch sequence): load the
 * n_parts cluster sets ev[0 .. n_parts-1] (each as for tpc_load_clusters:
 * device SoA, caller-owned, mode and pads equal across parts, in mode 1
 * the same tf_start) as one batch and run tpc_find_tracks on it. The parts
 * are copied (device to device, on the context's stream) into
 * library-owned buffers, concatenated in order: cluster j of part i gets
 * the input index (n_0 + ... + n_{i-1}) + j, and its event index is the
 * part's own (0 when the part has no event array) plus the events of the
 * parts before it. So the returned tracks, tpc_refit and
 * tpc_refit_backward then refer to the concatenated numbering; the parts'
 * arrays may be released once the call returns. At most 4096 events and
 * 2^31 - 1 clusters in all. Synchronises once (as tpc_find_tracks); may
 * allocate. Returns TPC_ERR_ARG for inconsistent parts. */
tpc_status tpc_find_tracks_batched(tpc_ctx* ctx, const tpc_clusters* ev, int32_t n_parts,
                                   tpc_tracks* out);

/* Same as tpc_find_tracks without the synchronisation: counts stay on the
 * device (readable with tpc_get_counts) and *out is not filled. Makes the
 * whole load-find-refit sequence capturable in a CUDA graph once buffers
 * are allocated. */
tpc_status tpc_find_tracks_async(tpc_ctx* ctx);

/* Fill *out with the context's current track set (library-owned device
 * memory, as returned by tpc_find_tracks / tpc_merge_tracks). Synchronises
 * (reads the counts). */
tpc_status tpc_get_tracks(tpc_ctx* ctx, tpc_tracks* out);

/* Replace the context's track set by caller-given tracks (truth assignment,
 * merged tracks ...). Copies the CSR asynchronously and applies the
 * calibration transform to the assigned clusters. */
tpc_status tpc_set_tracks(tpc_ctx* ctx, const tpc_tracks* tracks);

/* Refit the context's track set (Sec. 3) with the current calibration: the
 * calibration transform of the assigned clusters (Sec. 4) is re-applied
 * first when tpc_set_calib changed the calibration since the track set's
 * calibrated coordinates were computed (by the find, tpc_set_tracks, a
 * merge or a time refinement), so tpc_set_calib between refits takes
 * effect. Outputs are caller-owned device
 * buffers with room for the number of tracks (params [n][5], cov [n][15],
 * x [n], chi2 [n], ndf [n]; rej [n_assigned] receives for each cluster the
 * refit pass that rejected it, 0 = kept; any output may be NULL). status[n]
 * per track: 0 ok, 1 propagation or frame rotation failed, 2 no seed (fewer than 3 clusters or
 * no circle), 3 invalid track range (also raises TPC_ERR_ARG). With save_for_backward != 0 the per-step filter states are
 * kept for tpc_refit_backward. */
tpc_status tpc_refit(tpc_ctx* ctx, int save_for_backward, float* params, float* cov, float* x,
                     float* chi2, int32_t* ndf, int32_t* status, uint8_t* rej);

/* Vertex pseudo-measurements for the refit of the current track set (not
 * in the paper; a reading of how drift velocity and time offset become
 * determinable: like a triggered event whose vertex is known). z_vertex:
 * device [n_tracks], caller-owned and valid until the refits and adjoints
 * that use it have run; entry k is the vertex z (cm) of track k, NaN for a
 * track without one. After pass 3 of tpc_refit such a track's state is
 * transported to the beam line (x = 0 of its frame) and updated with
 * (y, z) = (0, z_vertex[k]) of variance sigma^2 each: chi2 and ndf include
 * that term and params, cov and x are those at the vertex. A track whose
 * transport to x = 0 fails (|sin(phi)| would reach s_max) keeps its state
 * at the innermost cluster without the term. tpc_refit_backward
 * differentiates the term too. NULL switches the vertices off; a new track
 * set (find, tpc_set_tracks, merge) switches them off as well. Returns
 * TPC_ERR_ARG for sigma <= 0 or a geometry with a full field, TPC_ERR_STATE
 * without a track set or while capturing; tpc_refit_backward returns
 * TPC_ERR_STATE when the vertices were set or cleared after the saved
 * refit. */
tpc_status tpc_set_vertex(tpc_ctx* ctx, const float* z_vertex, float sigma);

/* Merge the context's track set, taken as sector segments (from
 * tpc_find_tracks, or given by tpc_set_tracks), into tracks across sectors
 * (Sec. 2, second phase: the segments found in the individual sectors are
 * merged before the final fit). params [n][5], cov [n][15], x [n], status
 * [n]: the segments' states from tpc_refit of this track set (device,
 * caller-owned). Segment j continues segment i when both refits converged,
 * they lie in the same event and on the same side, j's sector is i's or a
 * neighbour in azimuth, j starts on a pad row beyond i's last one, and the
 * chi2 of their states (i's rotated into j's frame and transported to j's
 * x; in mode 1 j's z expressed with i's collision time; covariances added)
 * is at most params.chi2_merge with each the other's best match (smallest
 * chi2, then smallest index). Pairs whose tan(lambda) or q/pT differ by
 * more than sqrt(2 chi2_merge) standard deviations are not compared.
 * Replaces the track set by the chains of linked segments, ordered by their
 * first segment, whose collision time and start hit they take; clusters in
 * chain order. next [n] (device, may be NULL) receives each segment's
 * continuation or -1, link_chi2 [n] (may be NULL) its chi2 (0 when
 * unlinked). *out (may be NULL): the merged set (library-owned, as for
 * tpc_find_tracks). Synchronises. */
tpc_status tpc_merge_tracks(tpc_ctx* ctx, const float* params, const float* cov, const float* x,
                            const int32_t* status, int32_t* next, float* link_chi2,
                            tpc_tracks* out);

/* The same merge without synchronising (capturable in a CUDA graph): the
 * counts stay on the device (read them with tpc_get_counts), grids are
 * sized by the track buffer's capacity, and the candidate-pair list keeps
 * the capacity it has (32 pairs per segment of capacity unless a
 * synchronous merge enlarged it). If the pairs that pass the prefilter
 * exceed it, the next synchronising call reports TPC_ERR_CAPACITY (the
 * merged set is then incomplete; tpc_merge_tracks on the same segments
 * enlarges the list). The first call allocates (not during a capture). */
tpc_status tpc_merge_tracks_async(tpc_ctx* ctx, const float* params, const float* cov,
                                  const float* x, const int32_t* status, int32_t* next,
                                  float* link_chi2);

/* Time-frame mode (mode 1; Sec. 4, after merging: the vertex estimate is
 * refined with the merged track's fit and the track is shifted in z to it;
 * a track with clusters outside the drift volume is shifted back inside):
 * each track's collision time moves so that the fitted helix (params [n][5]
 * at x [n], from tpc_refit of the current track set, device, caller-owned)
 * reaches its closest approach to the beam line at z = 0, i.e. by
 * -sg * z0 / vdrift (sg = +1 on the A side); it is then clipped so that
 * every cluster's drift time t - t0 - t_coll lies in [0, drift_length /
 * vdrift] (the lower bound wins when both apply). Tracks with status[k] !=
 * 0, and every track in mode 0, keep their time. The calibration transform
 * of the assigned clusters is re-applied; t_coll_out [n] (device, may be
 * NULL) receives the times. Asynchronous; a refit must follow before
 * tpc_refit_backward. */
tpc_status tpc_refine_time(tpc_ctx* ctx, const float* params, const float* x,
                           const int32_t* status, double* t_coll_out);

/* Track-model compression of the context's track set (Sec. 5: only the
 * residuals of the clusters attached to tracks are stored, the track being
 * fitted in the distorted coordinate system). Along each track (clusters in
 * order; the model restarts where the sector frame changes, sectors k and
 * k + 18 sharing a frame) the first cluster of a run is stored as the
 * quantised absolute (y, z), the second as the quantised difference to the
 * first, and from then on a Kalman filter (straight-line seed through the
 * first two decoded clusters, helix transport in the uniform field, update
 * with each decoded cluster, errors params.sigma, seed covariance
 * params.c0t) predicts (y, z) at the next row: residual =
 * round-half-even((measured - predicted) / q). Decoded cluster = prediction
 * + residual * q, the filter's input, so that a decoder running the same
 * single-precision operations on the residuals reproduces the decoded
 * clusters exactly. Measured coordinates: y (cm; from the pad position
 * with native pads) and z as given (mode 0) or from the drift time with the
 * track's collision time and v_drift, without distortion correction (mode
 * 1). Where the transport fails the prediction is the previous decoded
 * cluster and the filter restarts. Outputs per assigned cluster in track
 * order (device, caller-owned, [n_assigned]): ry, rz (residuals in steps of
 * qy, qz cm), dy, dz (decoded clusters, may be NULL). Asynchronous. */
tpc_status tpc_compress_tracks(tpc_ctx* ctx, float qy, float qz, int32_t* ry, int32_t* rz,
                               float* dy, float* dz);

/* Adjoint of the last saved refit (not in the paper; TPC_ERR_STATE if the
 * calibration was set again after that refit): for
 * L = sum_k dL_dchi2[k] * chi2_k with chi2_k the pass-3 chi2, writes
 * grad_y[j], grad_zt[j] = dL/d(y, t or z) of the input cluster cluster_idx[j]
 * (device [n_assigned] each, overwritten) and grad_calib = dL/d(vdrift, t0,
 * spline[36*2*512]) (device double [TPC_GRAD_CALIB_SIZE], overwritten).
 * Rejections and seed states are held fixed. dL_dchi2: device [n_tracks].
 * Returns TPC_ERR_STATE without a preceding tpc_refit(save_for_backward=1). */
tpc_status tpc_refit_backward(tpc_ctx* ctx, const float* dL_dchi2, float* grad_y,
                              float* grad_zt, double* grad_calib);

/* CUDA-graph capture of a sequence of calls on the context's stream.
 * tpc_graph_begin starts a capture; the following asynchronous calls
 * (tpc_load_clusters, tpc_find_tracks_async, tpc_set_calib, tpc_refit,
 * tpc_refit_backward) are recorded instead of run; tpc_graph_end
 * instantiates them; tpc_graph_launch replays the recorded sequence on the
 * stream (same device pointers and sizes as when captured). Buffers are
 * allocated on first use, so run the sequence once outside the capture
 * before capturing it: an allocation during capture fails with TPC_ERR_STATE.
 * Synchronising calls (tpc_find_tracks, tpc_sync, tpc_get_*) are refused with
 * TPC_ERR_STATE while capturing. */
tpc_status tpc_graph_begin(tpc_ctx* ctx);
tpc_status tpc_graph_end(tpc_ctx* ctx);
tpc_status tpc_graph_launch(tpc_ctx* ctx);

/* Synchronise the stream and report the latched device error word. */
tpc_status tpc_sync(tpc_ctx* ctx);

/* Synchronise and read the counts of the current track set. */
tpc_status tpc_get_counts(tpc_ctx* ctx, int64_t* n_tracks, int64_t* n_assigned,
                          int64_t* n_tracklets);

/* Introspection of intermediate results, for tests (device outputs, cluster
 * indices in input numbering, -1 = none; asynchronous):
 *   links: up/dn neighbour links before cleaning and upc/dnc after, [n];
 *   tracklets (capacity n_cap): start hit, hit count, collision-time
 *     estimate and the per-row hit table [n_cap][n_rows];
 *   calibrated: corrected (y, z) of each assigned cluster [n_assigned];
 *   grid: cluster index in bucket order [n] and the start of each
 *     (event, sector, row) bucket [n_events*36*n_rows + 1]. */
tpc_status tpc_get_links(tpc_ctx* ctx, int32_t* up, int32_t* dn, int32_t* upc, int32_t* dnc);
tpc_status tpc_get_tracklets(tpc_ctx* ctx, int64_t n_cap, uint32_t* start_hit, int32_t* n_hits,
                             double* t_coll, int32_t* hits);
tpc_status tpc_get_calibrated(tpc_ctx* ctx, float* yc, float* zc);
tpc_status tpc_get_grid(tpc_ctx* ctx, uint32_t* order, uint32_t* row_start);

/* Refit without any device allocation. The paper has no counterpart: this
 * is for callers that cannot allocate device memory when they need a refit --
 * code running while a stream is captured into a CUDA graph (an allocation is
 * not a stream operation), real-time loops that must not take the device-wide
 * synchronisation an allocation can cause, or plug-ins whose host framework's
 * caching allocator owns the device memory.
 * The three-pass refit of tpc_refit in the uniform field geo->bz, for tracks
 * given as CSR over assigned clusters with their calibrated coordinates
 * already computed (device). The inputs carry no sector, so every track is
 * fitted in one sector frame: each track's clusters must lie in one sector
 * frame (sectors k and k + 18 share one); refit tracks merged across
 * sectors with tpc_refit. A geometry with a full field (geo->field not
 * NULL) returns TPC_ERR_ARG: the full-field transport is tpc_refit's.
 * Arguments:
 *   track_start [n_tracks + 1], yc, zc [n_assigned] (cm), row, flags
 *   [n_assigned] (flags may be NULL); outputs (device, any may be NULL):
 *   params [n_tracks][5], cov [n_tracks][15], chi2, ndf, status [n_tracks]
 *   (status 3 marks an invalid track range or row).
 * Working memory is a fixed device array of TPC_NOALLOC_SCRATCH_BYTES that
 * every GPU loading the library holds until the process exits; n_assigned
 * above TPC_NOALLOC_MAX_ASSIGNED returns TPC_ERR_CAPACITY. The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress); make
 * that first call before any stream capture on that device. The address is
 * kept per device ordinal for the life of the process, so the entry point
 * supports neither a cudaDeviceReset between calls nor contexts other than
 * the device's primary context. All calls share
 * the array, so calls that can overlap on the GPU (other streams, other
 * threads) race; the array is rewritten by every call before it is read.
 * geo, params: host, as for tpc_create (params NULL = defaults); stream: a
 * cudaStream_t. Asynchronous: kernel errors surface at the next stream sync. */
#define TPC_NOALLOC_MAX_ASSIGNED (1 << 20)
#define TPC_NOALLOC_SCRATCH_BYTES (5 * TPC_NOALLOC_MAX_ASSIGNED + 1024)
tpc_status tpc_refit_noalloc(const tpc_geometry* geo, const tpc_params* params, void* stream,
                             int64_t n_tracks, int64_t n_assigned, const uint32_t* track_start,
                             const float* yc, const float* zc, const uint8_t* row,
                             const uint8_t* flags, float* params_out, float* cov_out,
                             float* chi2_out, int32_t* ndf_out, int32_t* status_out);

/* Kernel accounting (tracing). Every kernel launch of a context is counted.
 * tpc_profile(ctx, 1) also brackets each launch with CUDA events on the
 * context's stream (adds a few microseconds per launch); tpc_profile(ctx, 0)
 * stops timing. Both synchronise and reset the statistics.
 * tpc_profile_read synchronises and returns per-kernel launch counts and
 * summed device time (out: host [cap], n_out: number of distinct kernels,
 * launches: all launches since the last reset). */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
} tpc_kernel_stat;
tpc_status tpc_profile(tpc_ctx* ctx, int enable);
/* Restrict the event timing of tpc_profile to the launches of one kernel
 * (name as reported by tpc_profile_read; NULL or "" = every kernel), so that
 * a long run can time its dominant kernel with two events per launch. Takes
 * effect from the next launch; does not synchronise. */
tpc_status tpc_profile_only(tpc_ctx* ctx, const char* kernel);
tpc_status tpc_profile_read(tpc_ctx* ctx, tpc_kernel_stat* out, int32_t cap, int32_t* n_out,
                            int64_t* launches);

/* Launch shapes and tile sizes of the track finder (autotuning). The paper
 * does not fix them; none of them changes any output bit, only the speed (the
 * search grid breaks ties by input index, not by bin; tracks are emitted in
 * an order that does not depend on the grid; the tracklet kernel is built
 * without contracted multiply-adds, so its block size cannot change rounding).
 *   grid_tau            target clusters per search-grid bin (0.125 .. 16)
 *   grid_ny_max         grid bins across a row at most (1 .. 64)
 *   tracklet_block      threads per block of the tracklet kernel (64, 128, 256)
 *   tracklet_per_sm     resident tracklet blocks per SM (0 .. 64); 0 = as many
 *                       as fit
 *   tracklet_regs       register cap of the tracklet kernel: 0 = the compiler's
 *                       choice (128 per thread), 96 = at most 96 (a quarter
 *                       more resident threads per SM, blocks of 64 or 128)
 * tpc_set_tuning validates (TPC_ERR_ARG) and applies from the next
 * tpc_load_clusters (grid) or tpc_find_tracks (tracklet kernel);
 * TPC_ERR_STATE while capturing. tpc_autotune searches one parameter at a
 * time, in that order, over grid_tau {0.25, 0.5, 1, 2, 4}, grid_ny_max {8, 16, 32},
 * (tracklet_block, tracklet_regs) together over {(64, 0), (128, 0),
 * (256, 0), (64, 96), (128, 96)}, and tracklet_per_sm {0, 1, 2, 4}, on the loaded
 * batch: each candidate runs load + find (grid parameters) or find (tracklet
 * parameters) `repeats` times (1 .. 50; < 1 means 3) after one untimed run,
 * timed with CUDA events on the context's stream, and the fastest median is
 * kept. It synchronises, needs a loaded batch, and leaves the batch loaded
 * and found with the chosen tuning; out may be NULL. */
typedef struct {
  float grid_tau;
  int32_t grid_ny_max;
  int32_t tracklet_block;
  int32_t tracklet_per_sm;
  int32_t tracklet_regs;
} tpc_tuning;
tpc_status tpc_get_tuning(const tpc_ctx* ctx, tpc_tuning* out);
tpc_status tpc_set_tuning(tpc_ctx* ctx, const tpc_tuning* in);
tpc_status tpc_autotune(tpc_ctx* ctx, int32_t repeats, tpc_tuning* out);

/* Text of the last error of this context ("" if none). Valid until the next
 * call on the context. */
const char* tpc_last_error(const tpc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* TPC_H_ */
