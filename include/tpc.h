/*
 * tpc.h — C ABI of the B300 TPC timeframe reconstruction library.
 *
 * The library reconstructs one TPC timeframe on one GPU: zero-suppressed (ZS)
 * digit decoding, the 3x3 peak / cluster finder per pad row, cellular-automaton
 * (CA) seeding across pad rows, the in-sector segment merge and the Kalman helix
 * fit.  The paper (Rohr, "The ALICE Run 3 Online / Offline Processing",
 * section "Hardware and data flow") states that the EPN GPUs perform the full
 * online TPC track reconstruction, that this is the most computing-intense part
 * of the synchronous processing, and that zero suppression of the raw data runs
 * upstream in the readout FPGA.  The paper does not define any of the
 * algorithms; every operation below is therefore defined in this header (and
 * restated, independently, by the CPU oracle shipped for testing).
 *
 * Conventions
 *   - Every function returns tpc_status: 0 on success, a negative TPC_E_* code
 *     otherwise.  tpc_last_error() returns a thread-local message for the most
 *     recent failure on the calling thread.
 *   - Pointers are host pointers unless stated otherwise.  "Borrowed" means the
 *     caller keeps ownership and must keep the memory valid for the stated time.
 *   - Units: x, y, z in cm.  A time bin is 200 ns = 0.5 cm of drift.  The common
 *     integer unit u = 7.8125 um is used by CA and merge (see TPC coordinates).
 *
 * Geometry (sector-local frame)
 *   n_sectors sectors (36: 0..17 on side A, z > 0; 18..35 on side C), each with
 *   n_rows pad rows.  Row r has npads[r] pads of pitch 0.4 cm centred on the
 *   sector axis: y(r, p) = (p - (npads[r]-1)/2) * 0.4 cm.  Row r sits at
 *   x = row_x[r] * 0.05 cm.  Sector s has axis angle alpha_s = ((s mod 18) + 0.5)
 *   * 20 degrees.
 *
 * ZS page format (one page per window = (sector, row, fragment); a fragment is
 * 256 time bins, fragment f covers time bins [256 f, 256 f + 256)).  All
 * integers little endian.  Pages start on 16-byte boundaries and their length is
 * a multiple of 16.
 *     off  0  u32 page_bytes      total length including this header
 *     off  4  u16 n_tb            number of time-bin entries
 *     off  6  u16 n_runs          number of pad runs
 *     off  8  u16 n_digits        number of digits (= sum of run lengths)
 *     off 10  u8  sector, u8 row
 *     off 12  u16 fragment
 *     off 14  u16 magic           TPC_ZS_MAGIC
 *     off 16  u16 lo_tb, lo_runs, lo_digits   entries/runs/digits with t < 3
 *     off 22  u16 hi_tb, hi_runs, hi_digits   first entry/run/digit with t >= 253
 *     off 28  u32 reserved (0)
 *     off 32  n_tb  x {u8 t_in_fragment, u8 n_runs}   strictly increasing t, n_runs >= 1
 *             n_runs x {u8 pad_start, u8 len}          per entry: ascending, disjoint, len >= 1
 *             (4-byte aligned) ceil(n_digits/3) x u32  ADCs, digit k in bits 10*(k%3)..+9 of word k/3
 *             zero padding to a multiple of 16 bytes
 *   Digit order is time-major, pad-ascending.  The lo_/hi_ fields let the two
 *   neighbouring windows read only the 3-time-bin halo they need.
 *
 * Results
 *   Clusters are returned in canonical order: ascending (sector, row, t_peak,
 *   pad_peak); a cluster's index is its position in that order.  Tracks are
 *   returned ordered by (sector, index of their lowest cluster).
 */
#ifndef TPC_H
#define TPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tpc_status;

#define TPC_OK            0
#define TPC_E_INVAL      -1   /* bad argument (null pointer, size out of range, bad descriptor) */
#define TPC_E_NOMEM      -2   /* request larger than the context's memory budget, or allocation failed */
#define TPC_E_BUSY       -3   /* no free slot and TPC_TF_NOWAIT given */
#define TPC_E_CUDA       -4   /* a CUDA runtime call failed; message in tpc_last_error() */
#define TPC_E_CORRUPT    -5   /* a ZS page failed validation (header, ranges, counts) */
#define TPC_E_NOTREADY   -6   /* results requested before the timeframe finished */
#define TPC_E_TIMEOUT    -7   /* tpc_poll timed out, or a bounded device wait gave up */
#define TPC_E_OVERFLOW   -8   /* a capacity (clusters, chains, tracks) was exceeded */
#define TPC_E_DEVICE     -9   /* device error word set for another reason */
#define TPC_E_NOTFOUND  -10   /* unknown or released ticket */

#define TPC_ZS_MAGIC      0x5A53u
#define TPC_FRAGMENT_BINS 256
#define TPC_ZS_HALO       3
#define TPC_MAX_PADS      255
#define TPC_MAX_ROWS      255
#define TPC_MAX_SECTORS   255
#define TPC_MAX_BATCH     4096   /* events in one tpc_submit_batch */

/* Ticket states reported by tpc_poll (monotone). */
#define TPC_STATE_QUEUED          0   /* admitted, waiting for a slot */
#define TPC_STATE_RUNNING         1   /* work enqueued on the device */
#define TPC_STATE_INPUT_RELEASED  2   /* input pages copied; caller may reuse them (host input
                                          only: device input is read in place until DONE / FAILED) */
#define TPC_STATE_DONE            3   /* results resident on the device */
#define TPC_STATE_FAILED          4   /* finished with an error; tpc_poll returns it */

/* Timeframe flags. */
#define TPC_TF_DEVICE_INPUT  1u   /* pages / page_offsets are device pointers, read in place: borrowed
                                     until tpc_poll reports TPC_STATE_DONE or TPC_STATE_FAILED (a
                                     capacity overflow re-runs the pipeline from them), so such a
                                     timeframe never reports TPC_STATE_INPUT_RELEASED */
#define TPC_TF_NOWAIT        2u   /* fail with TPC_E_BUSY instead of waiting for a slot */

/* Context flags. */
#define TPC_CTX_STAGE_TIMING 1u   /* record CUDA events around each stage (tpc_get_stage_times) */
#define TPC_CTX_NO_GRAPHS    2u   /* enqueue every kernel instead of replaying the slot's captured CUDA graph */
#define TPC_CTX_DENSE_FINDER 4u   /* steps 1-4 as the dense-plane variant: pages decoded into a dense
                                     (sector row, time bin, pad) ADC plane in device memory (2 bytes per
                                     pixel, 1.6 GB for the full TPC at 1000 bins), then windows read back
                                     from it */
#define TPC_CTX_FUSED_FINDER 8u   /* steps 1-4 as the fused variant: each window's pages decoded straight
                                     into a shared-memory plane of the whole window and clustered there.
                                     Without either flag the two-pass finder runs: every page decoded
                                     into 8-byte pad-run records (pad, length, time bin, first digit) in
                                     device memory (about 1.2x the ZS bytes), then each 64-bin time chunk
                                     of a window expanded from its runs and the page's ADC words into a
                                     small shared plane and clustered there.  All three give the same clusters
                                     (split_charge = 1 needs the two-pass finder). */

/* Pipeline stages, in launch order (indices into tpc_get_stage_times). */
#define TPC_STAGE_FIND       0    /* ZS decode + peak finder + cluster moments + compaction */
#define TPC_STAGE_CA         1    /* CA neighbours, links, chains */
#define TPC_STAGE_MERGE      2    /* segment merge + track assembly */
#define TPC_STAGE_FIT        3    /* Kalman fit + emit */
#define TPC_N_STAGES         4

typedef struct tpc_geometry tpc_geometry;
typedef struct tpc_context  tpc_context;

/* Geometry descriptor.  npads and row_x are borrowed for the call only. */
typedef struct {
  int32_t n_sectors;         /* 1..TPC_MAX_SECTORS */
  int32_t n_rows;            /* 3..TPC_MAX_ROWS */
  const int32_t* npads;      /* [n_rows], each 3..TPC_MAX_PADS */
  const int32_t* row_x;      /* [n_rows], x of the row in units of 0.05 cm, strictly increasing */
} tpc_geometry_desc;

/* Reconstruction parameters.  tpc_params_default() fills the defaults listed. */
typedef struct {
  uint32_t version;          /* TPC_PARAMS_VERSION */
  int32_t  q_peak_min;       /* 10   minimum peak ADC */
  int32_t  ca_slope_y_num;   /* 1    |dY| <= (num/den) dX window, y */
  int32_t  ca_slope_y_den;   /* 1 */
  int32_t  ca_slope_z_num;   /* 11   |dZ| <= (num/den) dX window, z (1.1) */
  int32_t  ca_slope_z_den;   /* 10 */
  int32_t  ca_cut;           /* 256  straight-line deviation cut, u (0.2 cm) */
  int32_t  min_chain;        /* 5    clusters per kept CA chain */
  int32_t  merge_cut;        /* 384  merge extrapolation cut, u (0.3 cm) */
  int32_t  merge_gap_min;    /* 1    row(b1) - row(a2) lower bound */
  int32_t  merge_gap_max;    /* 6    row(b1) - row(a2) upper bound */
  int32_t  merge_max_passes; /* 8 */
  int32_t  min_track;        /* 10   clusters per output track */
  int32_t  fit_passes;       /* 3    inward, outward, inward */
  int32_t  ns_min_dip;       /* 0    5x5 noise suppression (step 2b): 0 off, else 1..1023 ADC */
  double   bz;               /* 0.5  T */
  double   sigma_y;          /* 0.02 cm */
  double   sigma_z;          /* 0.03 cm */
  double   c0[5];            /* 4, 4, 0.25, 1, 100 initial covariance diagonal */
  double   fp32_pd_margin;   /* 0    step 8's FP32 positive-definiteness check asks every factor
                                     D_i of C = U D U^T to be > 0; with a margin m in [0, 1) it asks
                                     D_i > m * c0_i (c0 in the fit's unit), so that updates whose
                                     factors shrank below that are redone in FP64 (the FP64 check
                                     stays D_i > 0) */
  int32_t  split_charge;     /* 0    charge splitting (step 3s): 1 on; two-pass finder only */
} tpc_params;

#define TPC_PARAMS_VERSION 3u

/* Timeframe descriptor.  pages / page_offsets are borrowed until tpc_poll
 * reports a state >= TPC_STATE_INPUT_RELEASED (host input) or >=
 * TPC_STATE_DONE (TPC_TF_DEVICE_INPUT). */
typedef struct {
  const void*     pages;         /* concatenated ZS pages (16-byte aligned) */
  uint64_t        pages_bytes;   /* total bytes of pages */
  const uint64_t* page_offsets;  /* [n_sectors*n_rows*n_fragments] byte offset of the page of
                                    window (s, r, f) at index (s*n_rows + r)*n_fragments + f */
  uint32_t        n_time_bins;   /* 1..65535; n_fragments = ceil(n_time_bins / 256) */
  uint32_t        flags;         /* TPC_TF_* */
} tpc_timeframe_desc;

/* Cluster record (16 bytes).  See tpc_submit_timeframe for the definition of
 * every field. */
typedef struct {
  uint16_t pad_fp;       /* 256 * pad of the charge centroid (8.8 fixed point) */
  uint16_t time_fp;      /* 128 * (centroid time - 256*fragment + 4) (9.7 fixed point) */
  uint16_t qmax;         /* ADC of the peak digit */
  uint16_t qtot;         /* min(total charge of the cluster, 65535) */
  uint8_t  sigma2_pad;   /* 16 * pad variance (4.4), saturating at 255 */
  uint8_t  sigma2_time;  /* 16 * time variance (4.4), saturating at 255 */
  uint8_t  flags;        /* TPC_CL_* */
  uint8_t  row;
  uint16_t t_peak;       /* time bin of the peak digit */
  uint8_t  pad_peak;     /* pad of the peak digit */
  uint8_t  sector;
} tpc_cluster;

#define TPC_CL_EDGE      1u   /* peak on the first/last pad of the row or first/last time bin */
#define TPC_CL_EXCLUDED  2u   /* an outer-ring digit with charge was left out */
#define TPC_CL_NEIGHBOUR 4u   /* another peak lies in the 5x5 window */
#define TPC_CL_SPLIT     8u   /* step 3s gave an included pixel less than its whole charge */

/* Track record (112 bytes). */
typedef struct {
  float    par[5];       /* y, zeta, snp = sin(phi_local), tgl_zeta = dzeta/ds_T, q/pT (1/GeV) */
  float    x;            /* cm, x of the innermost cluster: the point the parameters refer to */
  float    alpha;        /* sector axis angle, rad */
  float    chi2;         /* of the final pass */
  float    cov[15];      /* lower triangle, row major: c00, c10, c11, c20, c21, c22, ... */
  int32_t  ndf;          /* 2 * n_used - 5 */
  int32_t  n_clusters;
  int32_t  first_cluster;/* canonical index of the lowest-row cluster */
  int16_t  sector;
  uint16_t flags;        /* TPC_TRK_* */
  int32_t  n_fp64;       /* covariance updates redone in FP64 after a failed PD check */
} tpc_track;

#define TPC_TRK_STOPPED  1u   /* a pass stopped early (|snp| would reach 0.999) */
#define TPC_TRK_NOT_PD   2u   /* covariance not positive definite even after the FP64 redo */
#define TPC_TRK_XSECTOR  4u   /* refitted over pieces in several sectors (tpc_merge_sectors) */

/* Fill *p with the defaults listed in tpc_params.  Never fails for p != NULL. */
tpc_status tpc_params_default(tpc_params* p);

/* Create a geometry object from desc (validated: sizes in range, row_x strictly
 * increasing).  The caller owns *out and frees it with tpc_destroy_geometry.
 * Defines the sector-local frame of the paper's TPC ("Hardware and data flow":
 * the TPC data the EPNs reconstruct); the layout itself is this library's. */
tpc_status tpc_create_geometry(const tpc_geometry_desc* desc, tpc_geometry** out);
void       tpc_destroy_geometry(tpc_geometry* g);

/* Create a reconstruction context on CUDA device `device`.
 *   geom        borrowed for the lifetime of the context
 *   params      copied (NULL: defaults)
 *   mem_budget  device bytes the context may hold for timeframes in flight
 *               (0: 8 GiB).  Work space is allocated once, here and on growth.
 *   n_slots     timeframes that may be in flight at once (1..64)
 *   stream      cudaStream_t (as void*) to run slot 0 on, or NULL for a
 *               library-created stream.  Slots > 0 always get their own stream.
 *   flags       TPC_CTX_*
 * Errors: TPC_E_INVAL, TPC_E_CUDA, TPC_E_NOMEM. */
tpc_status tpc_create_context(const tpc_geometry* geom, const tpc_params* params, int device,
                              uint64_t mem_budget, int n_slots, void* stream, uint32_t flags,
                              tpc_context** out);
void       tpc_destroy_context(tpc_context* ctx);

/* Submit one timeframe for reconstruction (non-blocking).
 *
 * Operation (the EPN GPU step of the paper's section "Hardware and data flow";
 * the algorithm is this library's own definition, stated here):
 *   1 decode   every page is validated and decoded to digits q(p, t).  Pixels
 *              without a digit have q = 0, as do pads outside the row and times
 *              outside [0, n_time_bins).
 *   2 peaks    pixel c is a peak iff q(c) >= q_peak_min and its key
 *              (q, -(t*npads + p)) is lexicographically greater than the key of
 *              each of its 8 neighbours in the same row.
 *   2b noise suppression (only with ns_min_dip > 0): a peak c is dropped iff a
 *              peak n of step 2 with a greater key lies on the ring of c's 5x5
 *              window (max(|dp|, |dt|) = 2) and q(c) - q(m) < ns_min_dip, m the
 *              pixel between them (the inner pixel of step 3 toward n).  Decided
 *              on step 2's peak set, so the order of the peaks does not matter;
 *              flag bit 2 of a cluster keeps referring to that set too.
 *   3 cluster  5x5 window around each peak: the inner 3x3 is always included; an
 *              outer pixel (dp, dt) is included iff q(outer) <= q(inner) and
 *              q(inner) > 0, inner = (sgn dp*min(|dp|,1), sgn dt*min(|dt|,1)).
 *              With Q = sum q, Sp = sum q dp, St = sum q dt, Spp = sum q dp^2,
 *              Stt = sum q dt^2 and R(a, b) = floor((2a + b) / (2b)):
 *              pad_fp = 256 p + R(256 Sp, Q); time_fp = 128 (t - 256 f + 4) +
 *              R(128 St, Q); sigma2_pad = min(255, R(16 (Spp Q - Sp^2), Q^2)),
 *              likewise sigma2_time; qmax = q(peak); qtot = min(Q, 65535).
 *   3s split   (only with split_charge = 1) charge of pixels near several
 *              peaks is shared.  The owners O(x) of a pixel x are the step-2
 *              peaks j with max(|p_x - p_j|, |t_x - t_j|) <= 1 if there is any,
 *              else those with that distance <= 2.  Step 3's sums count an
 *              included pixel x of the cluster of c with the weight
 *              floor(q(x) q(c) / sum_{j in O(x)} q(j)) if c is in O(x), else 0
 *              (the inclusion rule and flags still read q); flag TPC_CL_SPLIT
 *              marks a cluster where some weight differed from q(x).  The owners
 *              are step 2's peaks whether or not step 2b drops them.
 *   4 coords   Y = 2 (pad_fp - 128 (npads-1)), Z = 5 (32768 f + time_fp - 512),
 *              X = 64 row_x, all in u = 7.8125 um.
 *   5 CA       for a cluster c on rows 1..n_rows-2, over d on row-1 and u on row+1
 *              with |Y_u-Y_c| <= sy (X_u-X_c), |Y_c-Y_d| <= sy (X_c-X_d) and the
 *              same for Z with sz: dev_Y = (Y_u-Y_c)(X_c-X_d) - (Y_c-Y_d)(X_u-X_c),
 *              dev_Z alike; accepted iff |dev_Y|, |dev_Z| <= ca_cut (X_u - X_d);
 *              (up[c], down[c]) = argmin of dev_Y^2 + dev_Z^2, ties to the
 *              smallest (d, u); none: -1.  Row 0: up[d] = argmin of c's score
 *              over {c on row 1: down[c] = d}, ties to the smallest c; the last
 *              row mirrors it.
 *   6 chains   link (c, u) kept iff up[c] = u and down[u] = c.  Chains are the
 *              maximal paths; chain id = index of the lowest cluster; chains with
 *              fewer than min_chain clusters are dropped.
 *   7 merge    for a chain top (a1 below a2) and a chain bottom (b1 below b2) in
 *              the same sector with merge_gap_min <= row(b1)-row(a2) <=
 *              merge_gap_max, the forward residuals trunc(((Y_b1-Y_a2)(X_a2-X_a1) -
 *              (Y_a2-Y_a1)(X_b1-X_a2)) / (X_a2-X_a1)) (and Z), and the backward
 *              ones from (b2, b1) to a2, must all be <= merge_cut in size; score =
 *              sum of squares; mutual-best pairs merge (ties to the lower chain
 *              id of the end's chain); repeated up to merge_max_passes times.
 *              Merged chains with >= min_track clusters become tracks.
 *   8 fit      Kalman helix fit of each track in FP32 (see tpc_track): exact
 *              helix transport, (y, zeta) measurements with sigma_y, sigma_z,
 *              initial state from the circle through the outermost, middle and
 *              innermost clusters, C0 = diag(c0); passes inward, outward, inward
 *              with the covariance reset at each pass start; update C' = C - K H C
 *              then symmetrised; an update whose result fails the PD check is
 *              redone in FP64.
 * Admission: a timeframe starts at once on a free slot when the memory budget
 * allows (the device buffers of idle slots are given back first if it is
 * short).  Otherwise, and whenever earlier requests are still queued, it is
 * queued (state TPC_STATE_QUEUED) and started in arrival order by the
 * tpc_release that frees a slot and enough memory, so requests that arrive
 * while others run are admitted as slots and memory free up and overlap with
 * them on the device (each slot has its own stream).  A queued request that
 * cannot fit even with every other slot idle fails with TPC_E_NOMEM (reported
 * by tpc_poll).
 * Ownership: tf->pages and tf->page_offsets are borrowed (see the descriptor),
 * for a queued request until it has started and reached
 * TPC_STATE_INPUT_RELEASED.  Results stay on the device until tpc_release.
 * *ticket identifies them.
 * Errors: TPC_E_INVAL (descriptor), TPC_E_NOMEM (over budget with nothing else
 * running), TPC_E_BUSY (TPC_TF_NOWAIT and no slot or memory), TPC_E_CUDA.
 * Page corruption and capacity overflow are reported by tpc_poll
 * (TPC_E_CORRUPT, TPC_E_OVERFLOW). */
tpc_status tpc_submit_timeframe(tpc_context* ctx, const tpc_timeframe_desc* tf, uint64_t* ticket);

/* Submit a batch of n_events independent events (timeframes of the same
 * geometry and the same n_time_bins, e.g. triggered collisions of uneven
 * multiplicity) as ONE pipeline run: every stage is one set of launches over
 * all events' windows, chains and tracks, so small events share the GPU
 * instead of each leaving it mostly idle.  The paper processes each timeframe
 * on its own; batching is this library's way to fill the GPU with small ones
 * ("Real-time reconstruction": the EPNs reconstruct complete collisions).
 * Internally the sector axis becomes (event, sector); every step of the
 * method stays inside a sector, so each event's results equal those of a
 * tpc_submit_timeframe of that event alone, bit for bit.
 *   tfs       n_events descriptors (host or device pointers, told apart by
 *             address; TPC_TF_DEVICE_INPUT is not needed); borrowed until
 *             tpc_poll reports TPC_STATE_INPUT_RELEASED
 *   n_events  1..TPC_MAX_BATCH
 * The events' pages are gathered into the slot's own buffer (one copy per
 * event) and their page tables rebased onto it; a page offset outside its
 * event's own pages is treated as corrupt.  Results: tpc_get_batch_info and
 * the tpc_get_event_* calls; the plain getters return the concatenation
 * (events in order, indices global to the batch).
 * Errors: as tpc_submit_timeframe; TPC_E_INVAL if the events' n_time_bins
 * differ. */
tpc_status tpc_submit_batch(tpc_context* ctx, const tpc_timeframe_desc* tfs, uint32_t n_events,
                            uint64_t* ticket);

/* Wait up to timeout_us (0: do not wait; UINT32_MAX: forever) for the ticket
 * and report its state in *state.  Returns TPC_OK while running or done,
 * TPC_E_TIMEOUT if the wait expired, or the timeframe's own error
 * (TPC_E_CORRUPT, TPC_E_OVERFLOW, TPC_E_TIMEOUT, TPC_E_DEVICE, TPC_E_CUDA) once it
 * has failed (state TPC_STATE_FAILED). */
tpc_status tpc_poll(tpc_context* ctx, uint64_t ticket, uint32_t timeout_us, int32_t* state);

/* Copy the clusters of a finished ticket into out (host memory, cap records).
 * out == NULL: only *n is set (size query).  TPC_E_OVERFLOW if cap < n.
 * TPC_E_NOTREADY before TPC_STATE_DONE. */
tpc_status tpc_get_clusters(tpc_context* ctx, uint64_t ticket, tpc_cluster* out, uint64_t cap,
                            uint64_t* n);

/* Copy the tracks (cap records) and, if cluster_to_track != NULL, the track
 * index of every cluster (-1: none; n_clusters entries) into host memory.
 * out == NULL: only *n is set.  Errors as tpc_get_clusters. */
tpc_status tpc_get_tracks(tpc_context* ctx, uint64_t ticket, tpc_track* out, uint64_t cap,
                          uint64_t* n, int32_t* cluster_to_track);

/* Cross-sector merge parameters (step 9). */
typedef struct {
  double chi2_cut;   /* 100  matching chi2 (5 parameters) for a link */
  double edge_cm;    /* 6    a piece's end counts as at a sector edge within this distance
                              of the pad plane's edge (rounded to u = 7.8125 um) */
  double dz_cm;      /* 250  |zeta(B innermost) - zeta(A outermost)| bound of a candidate pair
                              (the drift length: the pieces of one track lie within it),
                              rounded to u; 0 < dz_cm <= 1e4 */
} tpc_xs_params;

/* Step 9, optional: join the pieces of tracks that cross a sector border, on
 * a finished ticket's device-resident results, and refit each joined track
 * over all its clusters.  The paper names the full TPC tracking on the EPN
 * GPUs ("Hardware and data flow"); this is the library's definition of its
 * last step:
 *   - a track's end is at the +y (-y) edge of its sector when its outermost
 *     (for the exit) or innermost (for the entry) cluster has
 *     Y >= 256 (npads - 1) - E (Y <= -(256 (npads - 1) - E)), Y in u, E = edge_cm / u;
 *   - candidates: A exiting through +y (-y) of sector s, B entering through -y
 *     (+y) of the neighbouring sector s+1 (s-1) of the same side (sectors
 *     0..17 and 18..35, cyclic), A's outermost row below B's innermost row,
 *     |Z(B's innermost cluster) - Z(A's outermost cluster)| <= dz (u), neither
 *     fit flagged;
 *   - B's state is rotated into A's frame and transported to A's reference x:
 *     chi2 = d^T (C_A + J C_B J^T)^-1 d over the 5 parameters; with the
 *     rotation by delta = alpha_B - alpha_A of a state at x: (x, y) ->
 *     (x cos d - y sin d, x sin d + y cos d), snp -> sin(phi + d), and the
 *     first-order Jacobian dy' = (cos d + tan(phi') sin d) dy, dzeta' = dzeta +
 *     (tgl / cos(phi')) sin d dy, dsnp' = (cos d - sin d tan(phi)) dsnp +
 *     k sin d dy;
 *   - mutual best pairs with chi2 <= chi2_cut link (ties: lower track index);
 *   - each chain of linked pieces is one track, ordered by its innermost
 *     piece; refitted as in step 8 over all its clusters (initial circle in
 *     the outermost piece's frame; state and covariance rotated into a piece's
 *     frame before its first cluster); flagged TPC_TRK_XSECTOR; its parameters
 *     refer to the innermost cluster in the innermost piece's frame.
 *   Unlinked tracks keep their step-8 records.
 * xp: NULL for the defaults.  *n_tracks (may be NULL): tracks after the merge.
 * Runs on the ticket's stream and waits for it; results until tpc_release.
 * The candidate search bins the entering pieces of every sector by zeta (bins
 * at least dz wide), so an exiting piece is compared with the entering pieces
 * of at most three bins of the neighbouring sector: linear in the timeframe's
 * length for continuous timeframes.
 * Errors: TPC_E_NOTREADY (ticket not done), TPC_E_NOTFOUND, TPC_E_CUDA, TPC_E_NOMEM. */
tpc_status tpc_merge_sectors(tpc_context* ctx, uint64_t ticket, const tpc_xs_params* xp, uint64_t* n_tracks);

/* The tracks after tpc_merge_sectors (cap records), the cluster-to-track map
 * (n_clusters entries, may be NULL) and, per step-8 track (may be NULL), the
 * index of its outer linked piece or -1.  out == NULL: only *n is set.
 * TPC_E_NOTREADY if tpc_merge_sectors has not run on the ticket. */
tpc_status tpc_get_merged_tracks(tpc_context* ctx, uint64_t ticket, tpc_track* out, uint64_t cap, uint64_t* n,
                                 int32_t* cluster_to_track, int32_t* link);

/* Looper-leg join parameters (step 9b). */
typedef struct {
  double  chi2_cut;        /* 30   matching chi2 (5 parameters) of two legs for a link, 0..1e6 */
  double  loop_radius_cm;  /* 275  a track can loop when its circle (|q/pT| raised by 3 sigma)
                                   stays within this distance of the beam axis: the 250 cm
                                   outer field cage + 10 %; 0 < r <= 1e4 */
  int32_t max_turns;       /* 4    largest number of turns between two linked legs, 1..15 */
  int32_t pad;
} tpc_loop_params;

/* Step 9b, optional: link the legs of looping tracks within each sector, on a
 * finished ticket's device-resident step-8 tracks.  The paper names the full
 * TPC tracking on the EPN GPUs ("Hardware and data flow"); a track whose
 * circle stays inside the TPC crosses a sector once per turn on the same
 * transverse path, and steps 5-8 find each crossing as a track of its own.
 * The library's definition:
 *   - a track can loop when the circle through its fitted point and direction
 *     with |q/pT| raised by 3 sigma has |centre| + 1/|k| <= loop_radius (centre
 *     (x - snp/k, y + cos(phi)/k) in the sector frame, k = -bz c 1e-2 q/pT);
 *   - each fit's covariance is scaled by max(1, chi2/ndf);
 *   - candidates: tracks A < B of one sector (of one event) that can loop,
 *     fits unflagged, q/pT of one sign; both carried along their helices to
 *     the larger reference x; m = the integer nearest (ties away from zero)
 *     to (zeta_B - zeta_A) / S with S = tgl_A 2 pi / |k_A| (the zeta advance
 *     of one turn), 1 <= |m| <= max_turns;
 *   - chi2 = d^T (J C_A J^T + C_B)^-1 d with d = s_B - (s_A + m S e_zeta) and
 *     J the identity plus m 2 pi / |k_A| at (zeta, tgl) and -m S / (q/pT)_A at
 *     (zeta, q/pT); accepted when chi2 <= chi2_cut and directed A -> B for
 *     m > 0, B -> A for m < 0;
 *   - a track's next (previous) leg is its outgoing (incoming) accepted pair of
 *     least |m|, then least chi2, then lowest index; f -> g links when g is
 *     f's next and f is g's previous.  Chains of links are one looper's turns.
 * The chi2 is computed in FP32 on the FP32 fits.  lp: NULL for the defaults.
 * *n_links (may be NULL): links made.  Runs on the ticket's stream and waits
 * for it; results until tpc_release.
 * Errors: TPC_E_INVAL (bad parameters, 2^28 or more tracks), TPC_E_NOTREADY
 * (ticket not done), TPC_E_NOTFOUND, TPC_E_CUDA, TPC_E_NOMEM. */
tpc_status tpc_join_loopers(tpc_context* ctx, uint64_t ticket, const tpc_loop_params* lp, uint64_t* n_links);

/* The links of tpc_join_loopers: next[t] / prev[t] (host memory, one entry
 * per step-8 track, either may be NULL) = the linked following / preceding
 * leg of track t or -1; in a batch, indices over the whole batch's tracks.
 * *n_tracks (may be NULL): the number of entries.  TPC_E_NOTREADY if
 * tpc_join_loopers has not run on the ticket. */
tpc_status tpc_get_looper_links(tpc_context* ctx, uint64_t ticket, int32_t* next, int32_t* prev, uint64_t* n_tracks);

/* Track-model compression parameters (step 10). */
typedef struct {
  double step_y_cm;  /* 0.0125    quantisation step of the y residual (1/32 pad) */
  double step_z_cm;  /* 0.015625  quantisation step of the zeta residual (1/32 time bin) */
} tpc_cmp_params;

/* Step 10, optional: track-model compression of the clusters on the step-8
 * tracks of a finished ticket (the paper gives the online reconstruction as
 * the means to reduce the TPC data, "Hardware and data flow"; this is the
 * library's definition):
 *   - per track, its fitted parameters at the innermost cluster are carried
 *     along the exact helix from row to row (the predicted state only, clusters
 *     innermost first, no measurement updates);
 *   - a cluster's codes are rint(residual / step) (ties away from zero) of its
 *     measured y and zeta minus the prediction at its row;
 *   - coded if both |codes| <= 127, else escaped (kept raw); clusters after a
 *     failed transport are escaped;
 *   - decoding: prediction + code * step, within half a step of the measured
 *     position.
 * cp: NULL for the defaults.  *n_coded / *n_escaped may be NULL.  Runs on the
 * ticket's stream and waits; results until tpc_release.
 * Errors: TPC_E_NOTREADY, TPC_E_NOTFOUND, TPC_E_INVAL, TPC_E_CUDA, TPC_E_NOMEM. */
tpc_status tpc_compress_clusters(tpc_context* ctx, uint64_t ticket, const tpc_cmp_params* cp, uint64_t* n_coded,
                                 uint64_t* n_escaped);

/* Codes and status of every cluster (n_clusters entries each; any pointer may
 * be NULL): status 0 not on a track, 1 coded (code_y, code_z valid), 2 escaped.
 * TPC_E_NOTREADY if tpc_compress_clusters has not run on the ticket. */
tpc_status tpc_get_compressed(tpc_context* ctx, uint64_t ticket, int8_t* code_y, int8_t* code_z, uint8_t* status);

/* Step 10c, optional: entropy coding of the step-10 codes into a bit stream
 * (the size the compression reaches; the paper gives data reduction as the
 * reason for online tracking, "Hardware and data flow"; the code is this
 * library's definition):
 *   - symbols: code + 128 of the y and of the z codes of the coded clusters
 *     (status 1), one 256-symbol alphabet per component;
 *   - per alphabet, Huffman codeword lengths from the symbol counts: the
 *     symbols with a count, ordered by (count, symbol), form queue A; merged
 *     nodes join queue B in creation order; each merge takes the lighter of
 *     the two queue heads twice, a symbol before a node of equal weight; a
 *     symbol's length is its depth (1 for a lone symbol).  If a length exceeds
 *     24, every count c becomes (c + 1) / 2 and the lengths are built again;
 *   - canonical codewords: symbols ordered by (length, symbol), the first
 *     gets 0, each next (previous + 1) << (its length - previous length);
 *   - the stream: for each coded cluster in index order its y codeword, then
 *     its z codeword, most significant bit first; stream bit b is bit
 *     31 - b % 32 of 32-bit word b / 32; the last word is zero-padded.
 * code_y, code_z, status: NULL to encode the ticket's step-10 codes (then
 * tpc_compress_clusters must have run: TPC_E_NOTREADY otherwise), or host
 * arrays of n_clusters entries each (all three) that replace the ticket's
 * step-10 codes before encoding (tpc_get_compressed returns them afterwards).
 * lengths (may be NULL): the 512 codeword lengths, y alphabet then z (0: symbol
 * unused).  *n_bits (may be NULL): the stream's length.  words (may be NULL:
 * size query) receives the (n_bits + 31) / 32 stream words; TPC_E_INVAL if
 * cap_words is smaller.  Runs on the ticket's stream and waits.
 * Errors: TPC_E_INVAL, TPC_E_NOTREADY, TPC_E_NOTFOUND, TPC_E_NOMEM, TPC_E_CUDA. */
tpc_status tpc_entropy_encode(tpc_context* ctx, uint64_t ticket, const int8_t* code_y, const int8_t* code_z,
                              const uint8_t* status, uint8_t* lengths, uint64_t* n_bits, uint32_t* words,
                              uint64_t cap_words);

/* Step 11, optional: drift-velocity / T0 calibration from the step-8 tracks of
 * a finished ticket holding one collision whose vertex lies on the beam axis
 * at z = 0 (the paper lists calibration among the EPNs' tasks, "Hardware and
 * data flow"; this is the library's definition):
 *   - per track with >= 20 clusters and no flag, its state is carried along
 *     the exact helix to x = 0 and used if |y| < 3 cm there; its vertex time
 *     bin is t_v = zeta / 0.5 cm (zeta is 0.5 cm per time bin);
 *   - the fullest whole bin b* of floor(t_v) (over 2^20 bins, the lowest on
 *     ties) seeds a mean over |t_v - (b* + 0.5)| <= 3, then a mean over
 *     |t_v - mean| <= 1.5: *t_vertex_bins;
 *   - the vertex's charge drifts the whole length L, so with the collision
 *     time t0_bins known the drift velocity is off by
 *     *eps_vd = (L / 0.5 cm) / (t_vertex - t0) - 1, and with the drift
 *     velocity known the collision time is *t0_from_vertex = t_vertex - L / 0.5 cm.
 * Any output pointer may be NULL; *n_used: tracks in the final mean (0: no
 * estimate, outputs 0).  Runs on the ticket's stream and waits.
 * Errors: TPC_E_NOTREADY, TPC_E_NOTFOUND, TPC_E_INVAL, TPC_E_CUDA, TPC_E_NOMEM. */
tpc_status tpc_calibrate_drift(tpc_context* ctx, uint64_t ticket, double t0_bins, double drift_length_cm,
                               double* t_vertex_bins, double* eps_vd, double* t0_from_vertex, uint64_t* n_used);

/* Layout of a finished ticket's results by event: *n_events (1 for a plain
 * timeframe) and, if not NULL, cluster_start[n_events + 1] and
 * track_start[n_events + 1], each event's first cluster / track in the
 * concatenated results (last entry: the totals). */
tpc_status tpc_get_batch_info(tpc_context* ctx, uint64_t ticket, uint32_t* n_events, uint64_t* cluster_start,
                              uint64_t* track_start);

/* One event's clusters of a finished ticket, as tpc_get_clusters gives them for
 * that event submitted alone.  TPC_E_INVAL if event >= n_events. */
tpc_status tpc_get_event_clusters(tpc_context* ctx, uint64_t ticket, uint32_t event, tpc_cluster* out,
                                  uint64_t cap, uint64_t* n);

/* One event's tracks and cluster-to-track map, indices relative to the event
 * (first_cluster, map values), as tpc_get_tracks gives them for that event
 * submitted alone. */
tpc_status tpc_get_event_tracks(tpc_context* ctx, uint64_t ticket, uint32_t event, tpc_track* out,
                                uint64_t cap, uint64_t* n, int32_t* cluster_to_track);

/* Copy the CA results of a finished ticket (n_clusters entries each; any
 * pointer may be NULL): up[], down[] (step 5, cluster indices or -1) and
 * chain_of[] (step 6: id of the kept chain holding the cluster, or -1). */
tpc_status tpc_get_links(tpc_context* ctx, uint64_t ticket, int32_t* up, int32_t* down,
                         int32_t* chain_of);

/* Device pointers to a finished ticket's results (valid until tpc_release);
 * any output pointer may be NULL.  Lets device-resident callers skip the copy. */
tpc_status tpc_get_device_results(tpc_context* ctx, uint64_t ticket, const tpc_cluster** clusters,
                                  uint64_t* n_clusters, const tpc_track** tracks,
                                  uint64_t* n_tracks, const int32_t** cluster_to_track);

/* Per-stage device times (ms) of a finished ticket, from CUDA events recorded on
 * the slot's stream around each stage; requires TPC_CTX_STAGE_TIMING.
 * ms[TPC_N_STAGES]. */
tpc_status tpc_get_stage_times(tpc_context* ctx, uint64_t ticket, float* ms);

/* Counters of a finished ticket: out[0] clusters, [1] kept chains, [2] tracks,
 * [3] clusters on tracks, [4] FP64 covariance redos, [5] merge passes that
 * merged, [6] device error word, [7] ZS bytes of the timeframe, [8] kernel
 * launches of the last run, [9] runs (1; 2 or 3 after capacity regrowths).
 * n: entries requested (<= 10). */
tpc_status tpc_get_counters(tpc_context* ctx, uint64_t ticket, uint64_t* out, int n);

/* Free the ticket's slot and results, then start the oldest queued requests
 * that now fit.  A queued ticket is cancelled.  Unknown ticket: TPC_E_NOTFOUND. */
tpc_status tpc_release(tpc_context* ctx, uint64_t ticket);

/* Launch configuration of the pipeline's kernels (per context).  Every choice
 * gives the same results, bit for bit; only the speed differs.  Defaults:
 * 128, 8, 8, 8, 64, 32 (two-pass finder) or 384, 2, 8, 8, 64, 32 (fused or
 * dense-plane finder). */
typedef struct {
  int32_t find_threads;        /* two-pass finder: 128 | 256 threads per unit CTA; fused and dense-plane
                                  finders: 256 | 384 | 512 threads per persistent window CTA */
  int32_t find_ctas_per_sm;    /* two-pass: 4 | 8 unit CTAs per SM; fused and dense-plane: 1 | 2 */
  int32_t ca_blocks_per_sm;    /* 4 | 8 | 16 CA-neighbour blocks per SM */
  int32_t elem_blocks_per_sm;  /* 4 | 8 | 16 blocks per SM of the grid-stride CA / merge kernels */
  int32_t fit_threads;         /* 32 | 64 | 128 tracks per fit block */
  int32_t fit_blocks_per_sm;   /* 16 | 32 | 64 fit blocks per SM (grid cap) */
} tpc_tuning;

/* The context's current launch configuration. */
tpc_status tpc_get_tuning(tpc_context* ctx, tpc_tuning* out);

/* Set the launch configuration (e.g. one saved from an earlier tpc_autotune)
 * for the following submits.  TPC_E_INVAL if a value is outside its set. */
tpc_status tpc_set_tuning(tpc_context* ctx, const tpc_tuning* t);

/* Autotuner: run the sample timeframe (host or device input, as for
 * tpc_submit_timeframe) reps times under each of 9 joint candidate
 * configurations, time every stage with CUDA events, and keep per stage the
 * fastest choice (finder: threads x CTAs per SM; CA and merge: grid sizes; fit:
 * block and grid size); the result is set on the context and copied to *out
 * (may be NULL).  The paper describes no tuner; this picks launch parameters
 * per context and workload on the GPU at hand.  Needs an idle context (no ticket
 * in flight or queued, else TPC_E_BUSY); blocks until done; errors of a
 * sample run are returned (the configuration is then left unchanged). */
tpc_status tpc_autotune(tpc_context* ctx, const tpc_timeframe_desc* sample, int reps, tpc_tuning* out);

/* Allocation-free cluster finder (steps 1-4 only).  The paper has no
 * counterpart to this entry point; it exists for callers that cannot allocate
 * device memory: code that runs inside a device-memory budget owned by another
 * framework, or in a loop that must never reach cudaMalloc / cudaFree, whose
 * implicit device-wide synchronisation and unbounded latency such a loop
 * cannot afford.  It computes exactly the clusters tpc_submit_timeframe
 * computes, with no context and no allocation of any kind.
 *   geom          host geometry object
 *   params        NULL for defaults; only q_peak_min and ns_min_dip are used
 *                 (split_charge must be 0: TPC_E_INVAL otherwise)
 *   device        CUDA device the pointers live on
 *   pages, page_offsets, pages_bytes, n_time_bins   as in tpc_timeframe_desc,
 *                 device memory, borrowed for the call; pages 16-byte aligned
 *   clusters      device memory for cap records (16-byte aligned), written in
 *                 canonical order
 *   n_clusters    host out: clusters found (may exceed cap: TPC_E_OVERFLOW)
 *   stream        cudaStream_t (as void*) to run on, NULL for the default stream
 * Scratch: a file-scope device array of 65,536 windows' look-back states plus
 * 256 bytes of control words (about 513 KB, held on every GPU that loads the
 * library until the process exits).  A timeframe with more windows (sectors x
 * rows x 256-bin fragments) is rejected with TPC_E_INVAL.  The first call on a
 * device looks up the array's device address and sets the kernel's shared-
 * memory limit; make that first call before any stream capture.  Every call
 * shares the one array, and clears it on its stream before use: calls that
 * overlap on the GPU (other streams, other host threads) race and corrupt
 * each other's results.  The call waits for its stream before returning.
 * Errors: TPC_E_INVAL, TPC_E_CUDA, TPC_E_CORRUPT, TPC_E_OVERFLOW, TPC_E_TIMEOUT. */
tpc_status tpc_find_clusters_noalloc(const tpc_geometry* geom, const tpc_params* params, int device,
                                     const void* pages, uint64_t pages_bytes, const uint64_t* page_offsets,
                                     uint32_t n_time_bins, tpc_cluster* clusters, uint64_t cap,
                                     uint64_t* n_clusters, void* stream);

/* Diagnostics: the FP32 FMA throughput of device `device` in FLOP/s (an FMA
 * counts two), the best of `reps` (1..1000) timed launches of a kernel in
 * which every thread runs eight independent FMA chains, 8 blocks of 256
 * threads per SM.  It is the measured ALU peak the step-8 fit's achieved
 * FLOP/s is compared with; the paper has no counterpart.  Allocates and frees
 * a small scratch buffer and its own stream; changes no device setting.
 * Errors: TPC_E_INVAL, TPC_E_CUDA. */
tpc_status tpc_measure_fma_peak(int device, int reps, double* flops_per_s);

/* Thread-local message describing the last error on this thread ("" if none). */
const char* tpc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TPC_H */
