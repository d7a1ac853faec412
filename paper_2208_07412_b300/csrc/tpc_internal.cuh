// tpc_internal.cuh — shared device-side definitions of the B300 TPC library.
//
// Everything here belongs to the CUDA path.  The CPU oracle used by the tests
// is separate code and shares nothing with these files.
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/tpc.h"

// Host-side geometry object behind the opaque tpc_geometry handle.
struct tpc_geometry {
  int n_sectors, n_rows, npmax;
  std::vector<int> npads, row_x;
};

namespace tpc {

// Sets the thread-local message returned by tpc_last_error().
void set_last_error(const char* msg);

constexpr int kFrag = TPC_FRAGMENT_BINS;     // 256 time bins per window
constexpr int kHalo = TPC_ZS_HALO;           // 3 time bins of halo each side
constexpr int kWinT = kFrag + 2 * kHalo;     // 262 plane rows per window
constexpr int kMaxRowsDev = 256;

// device error word bits
constexpr uint32_t kErrCorrupt = 1u;         // a ZS page failed validation
constexpr uint32_t kErrOverflowCl = 2u;      // cluster capacity exceeded
constexpr uint32_t kErrOverflowCh = 4u;      // chain / track capacity exceeded
constexpr uint32_t kErrTimeout = 8u;         // a bounded wait gave up
constexpr uint32_t kErrRowCount = 16u;       // a row holds >= 2^23 clusters (edge keys)

// bounded spin for look-back waits: 4e6 polls with back-off is about a second
constexpr long long kSpinLimit = 4000000LL;

// Geometry + parameters, passed by value to every kernel (fits in the 32 KB
// kernel parameter space).
struct DevGeom {
  // A batch of events runs as one timeframe whose sector axis is
  // (event, sector): n_sectors = n_events * n_phys "virtual" sectors, window and
  // row tables indexed by virtual sector, records carrying the physical one.
  int n_sectors, n_rows, n_time_bins, n_frag;
  int n_phys, n_events;          // sectors of the detector, events in the batch
  int npmax, nw;                 // widest row, 32-pad words per plane row
  int npads[kMaxRowsDev];
  int xrow[kMaxRowsDev];         // X of each row in u (= 64 * row_x)
};

// Launch configuration of the pipeline's kernels.  Every choice computes the
// same results (all kernels are deterministic in their outputs); the
// autotuner picks the fastest per stage on a sample timeframe.
struct LaunchCfg {
  int find_threads = 384;        // 256 | 384 | 512 threads per finder CTA
  int find_ctas_per_sm = 2;      // 1 | 2 persistent finder CTAs per SM
  int ca_blocks_per_sm = 8;      // 4 | 8 | 16: CA neighbour blocks (one (sector, row) each at a time)
  int elem_blocks_per_sm = 8;    // 4 | 8 | 16: grid-stride kernels of the CA and merge stages
  int fit_threads = 64;          // 32 | 64 | 128 threads (tracks) per fit block
  int fit_blocks_per_sm = 32;    // 16 | 32 | 64: fit grid cap
};

struct DevParams {
  int q_peak_min;
  int ns_min_dip;                // 5x5 noise suppression: 0 off, else the minimum dip (ADC)
  int split_charge;              // step 3s charge splitting: 0 off, 1 on (two-pass finder only)
  int sy_num, sy_den, sz_num, sz_den;
  int ca_cut, min_chain;
  int merge_cut, gap_min, gap_max, merge_passes;
  int min_track, fit_passes;
  float kfac;                    // curvature per unit q/pT: -bz * c * 1e-2 (1/cm per 1/GeV)
  float sy2, sz2;                // sigma_y^2, sigma_z^2 (cm^2)
  float c0[5];
  double kfac_d, sy2_d, sz2_d;   // FP64 copies for the covariance redo
  // the same in the integer coordinate unit u = 7.8125e-4 cm (the step-8 fit's unit)
  float kfac_u;                  // 1/u per 1/GeV
  float sy2_u, sz2_u;            // u^2
  float c0_u[5];                 // y, zeta entries in u^2
  float pd_min_u[5];             // floor of each FP32 D factor: fp32_pd_margin * c0_u
  double sy2_ud, sz2_ud;         // FP64 copies for the covariance redo
};

// Per-slot device work space.  All pointers are device memory owned by the
// runtime; capacities are in elements.
struct DevWork {
  // input
  const uint8_t* pages;
  const uint64_t* page_offsets;
  uint64_t pages_bytes;
  // finder
  tpc_cluster* clusters;
  int32_t* cl_x; int32_t* cl_y; int32_t* cl_z; int32_t* cl_t;
  uint32_t* row_start;           // [n_sectors * n_rows + 1]
  uint16_t* dense;               // dense-plane finder variant: [sector row][time bin][dense_stride] ADC
  uint32_t dense_stride;         // pads per dense time row (npmax rounded up to 8)
  unsigned long long* win_state;  // look-back states of the finder windows (allocation-free mode)
  tpc_cluster* scratch_cl;       // finder output, window spans in completion order
  unsigned long long* win_cnt;   // clusters per window, scanned in place to canonical bases
  uint32_t* win_soff;            // start of each window's span in scratch_cl
  uint32_t* light_list;          // [n_windows] windows of the light path (first CTR_NLIGHT), or null
  uint32_t* heavy_list;          // [n_windows] the other windows (first CTR_NHEAVY)
  uint2* runs;                   // two-pass finder: every pad run as (pad | len << 8 | t_in << 16, index of its
                                 // first digit in the page), one span per page
  uint4* dtab;                   // [3 * n_windows] per window: (run span start lo, hi, runs, 0), the run
                                 // indices at the units' time boundaries (8 x u16), (ADC byte offset lo, hi, 0, 0)
  uint64_t cap_runs;             // runs the array holds
  uint4* udesc;                  // [7 * units] two-pass finder: unit descriptors (k_unit_descs)
  // CA
  int32_t* up; int32_t* down;
  int64_t* score;
  unsigned long long* edge_key;
  unsigned long long* jump;      // (dist << 32) | ptr
  int32_t* chain_len;            // indexed by root cluster
  uint64_t* scan_val;            // scan inputs / outputs (clusters or chains)
  unsigned long long* scan_state;
  int32_t* chain_of;
  int32_t* cl_chain;
  // chain table
  int32_t* ch_root; int32_t* ch_len; int32_t* ch_b2; int32_t* ch_top; int32_t* ch_top2;
  int32_t* ch_t;                 // t_peak of the chain's root (bottom) cluster
  uint32_t* ch_row_start;        // [n_sectors * n_rows + 1] first chain whose root lies in each row
  uint32_t* ch_bucket;           // [n_sectors * n_rows * (4 n_frag + 1) + 1] first chain whose root lies in
                                 // each (row, 64-bin bucket of its time bin) or later
  int32_t* ch_next; int32_t* ch_prev;
  unsigned long long* best_b;
  unsigned long long* best_a;    // [2 * cap_chains]
  unsigned long long* cand_ab;   // merge candidate pairs (top chain << 32 | bottom chain)
  uint32_t* cand_sc;             // their scores
  uint64_t cap_cand;
  int32_t* ch_track; int32_t* ch_off;
  int32_t* grp_total;
  // tracks
  int32_t* trk_first; int32_t* trk_ncl; int32_t* trk_off;
  uint32_t* len_hist;            // [512]: tracks per length bin (longest first), then ranks
  int32_t* fit_order;            // tracks, longest first (reuses ch_off once assignment is done)
  int32_t* track_cl;
  int4* trk_xyz;                 // (X, Y, Z, cluster) in track order, aligned with track_cl (reuses scratch_cl)
  int32_t* cl2trk;
  tpc_track* tracks;
  // counters (device scalars, one 64-byte block)
  unsigned long long* ctr;       // see CTR_* below
  uint32_t* err;
  unsigned int* tickets;         // [kNumTickets] atomic ticket counters
  // capacities
  uint64_t cap_cl, cap_ch;
};

enum {
  CTR_NCL = 0,        // clusters found (may exceed cap_cl on overflow)
  CTR_NCH = 1,        // kept chains
  CTR_NTRK = 2,       // tracks
  CTR_NFP64 = 3,      // FP64 covariance redos
  CTR_MERGED0 = 4,    // merges in pass p at CTR_MERGED0 + p (up to 16 passes)
  CTR_NCLCL = 20,     // clusters assigned to tracks
  CTR_SCURSOR = 21,   // next free scratch record of the finder
  CTR_NWIN = 22,      // windows of the timeframe
  CTR_NCAND = 23,     // merge candidate pairs found
  CTR_NLIGHT = 24,    // windows the light finder path takes
  CTR_NHEAVY = 25,    // windows the block-per-window finder takes
  CTR_NRUN = 26,      // pad runs decoded by the two-pass finder (span cursor)
  CTR_COUNT = 27
};
enum { TK_FIND = 0, TK_SCAN_A = 1, TK_SCAN_B = 2, TK_SCAN_W = 3, TK_FIND2 = 4, TK_LIGHT = 5, TK_UNIT = 6, TK_DEC = 7,
       kNumTickets = 8 };
// The control block is 256 bytes: CTR_COUNT counters, the error word and the tickets.
static_assert(8 * (CTR_COUNT + 1) + 4 * kNumTickets <= 256, "control block layout");

// ------------------------------------------------------------------ helpers
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Inclusive warp scan of a 64-bit value.
__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// Exclusive block scan of one 64-bit value per thread (blockDim.x <= 1024,
// multiple of 32).  Returns the exclusive prefix; *total gets the block sum.
// sm: >= 33 entries of shared scratch.
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long* sm,
                                                              unsigned long long* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long inc = warp_incl_scan(v);
  if (lane == 31) sm[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    unsigned long long w = lane < nw ? sm[lane] : 0ull;
    unsigned long long wi = warp_incl_scan(w);
    if (lane < nw) sm[lane] = wi - w;
    if (lane == nw - 1) sm[32] = wi;
  }
  __syncthreads();
  unsigned long long r = sm[wid] + inc - v;
  *total = sm[32];
  __syncthreads();
  return r;
}

// Decoupled look-back (single pass chained scan).  Called by warp 0 of the
// block owning tile `tile` after it knows its aggregate.  States: bits 63:62 =
// 0 empty, 1 aggregate, 2 inclusive prefix; bits 61:0 the value.  Tiles are
// handed out by an atomic ticket, so every predecessor is running or done and
// publishes its aggregate without waiting: the spin ends.  It is bounded all
// the same; on expiry the error word gets kErrTimeout and 0 is returned.
constexpr unsigned long long kStFlagAgg = 1ull << 62, kStFlagPre = 2ull << 62,
                             kStMask = (1ull << 62) - 1;
// Publish a tile's aggregate (tile 0 publishes its inclusive prefix at once).
__device__ __forceinline__ void lookback_publish(unsigned long long* state, long long tile,
                                                 unsigned long long aggregate) {
  st_release_u64(&state[tile], (tile == 0 ? kStFlagPre : kStFlagAgg) | aggregate);
}
// Wait for the exclusive prefix of `tile` (warp 0 of the block; the aggregate
// must already be published) and publish the tile's inclusive prefix.
__device__ __forceinline__ unsigned long long lookback_wait(unsigned long long* state, long long tile,
                                                            unsigned long long aggregate, uint32_t* err);
__device__ __forceinline__ unsigned long long lookback_warp0(unsigned long long* state, long long tile,
                                                             unsigned long long aggregate, uint32_t* err) {
  if ((threadIdx.x & 31) == 0) lookback_publish(state, tile, aggregate);
  return lookback_wait(state, tile, aggregate, err);
}
__device__ __forceinline__ unsigned long long lookback_wait(unsigned long long* state, long long tile,
                                                            unsigned long long aggregate, uint32_t* err) {
  const int lane = threadIdx.x & 31;
  if (tile == 0) return 0;
  unsigned long long excl = 0;
  long long base = tile - 1;
  long long spins = 0;
  while (true) {
    long long j = base - lane;
    // the state word carries the whole value, so a relaxed poll suffices
    unsigned long long s = j >= 0 ? ld_relaxed_u64(&state[j]) : kStFlagPre;
    unsigned flag = (unsigned)(s >> 62);
    unsigned empty = __ballot_sync(0xffffffffu, flag == 0);
    if (empty) {
      if (++spins > kSpinLimit) {
        if (lane == 0) atomicOr(err, kErrTimeout);
        excl = 0;
        break;
      }
      __nanosleep(spins < 8 ? 32 : 256);
      continue;
    }
    unsigned pre = __ballot_sync(0xffffffffu, flag == 2);
    // lanes up to and including the first lane holding a prefix contribute
    int stop = pre ? __ffs(pre) - 1 : 31;
    unsigned long long v = lane <= stop ? (s & kStMask) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    excl += v;
    if (pre) break;
    base -= 32;
  }
  if (lane == 0) st_release_u64(&state[tile], kStFlagPre | (excl + aggregate));
  return excl;
}

// Work space of the optional looper-leg join (step 9b), in one slot buffer.
struct LoopWork {
  uint8_t* loops;                // [cap_ch] 1: the track can loop (candidate leg)
  uint64_t* bin_off;             // [n_vs + 1] looping tracks per virtual sector -> offsets
  uint32_t* bin_cur;             // [n_vs] fill cursors
  unsigned long long* bin_state; // scan state of bin_off
  uint32_t* ent;                 // [cap_ch] looping tracks grouped by virtual sector
  uint4* ent_fit;                // [cap_ch][6] their records' first 96 bytes, in the same order
  unsigned long long* next_key;  // [cap_ch] best outgoing pair: |m| << 60 | chi2 bits << 28 | index
  unsigned long long* prev_key;  // [cap_ch] best incoming pair, same packing
  int32_t* next;                 // [cap_ch] linked following leg or -1
  int32_t* prev;                 // [cap_ch] linked preceding leg or -1
  unsigned long long* ctl;       // [0] links, [1] n_vs + 1, [2] (u32) bin scan ticket, [3] looping tracks
  float chi2_cut;
  float loop_radius;             // cm
  int max_turns;
  int n_vs;                      // virtual sectors (sectors x events)
};

// Work space of the optional cross-sector merge (step 9), in one slot buffer.
struct XsWork {
  uint8_t* side;                 // [cap_ch] exit side (bits 0-1: 1 = +y, 2 = -y), entry side (bits 2-3)
  int32_t* row_in;               // [cap_ch] row of the innermost cluster
  int32_t* row_out;              // [cap_ch] row of the outermost cluster
  unsigned long long* best_b;    // [cap_ch] best outer partner of A: chi2 bits << 32 | B
  unsigned long long* best_a;    // [cap_ch] best inner partner of B
  int32_t* link;                 // [cap_ch] outer piece or -1
  int32_t* prev;                 // [cap_ch] inner piece or -1
  int32_t* group;                // [cap_ch] merged track of every piece
  uint64_t* scan;                // [cap_ch] root flags, scanned to merged track indices
  unsigned long long* scan_state;
  unsigned long long* ctl;       // [0] merged tracks, [1] links, [2] (u32) scan ticket, [3] bins + 1,
                                 // [4] (u32) bin scan ticket, [5] entering pieces binned
  tpc_track* tracks_out;         // [cap_ch]
  int32_t* cl2trk_out;           // [cap_cl]
  int32_t* z_in;                 // [cap_ch] Z (u) of the innermost cluster
  int32_t* z_out;                // [cap_ch] Z (u) of the outermost cluster
  uint64_t* bin_off;             // [n_bins + 1] entering pieces per (virtual sector, zeta bin) -> offsets
  uint32_t* bin_cur;             // [n_bins] fill cursors
  uint4* ent;                    // [cap_ch] entering unflagged pieces grouped by bin: (piece, Z of the
                                 // innermost cluster, innermost row | entry edge << 8, 0)
  uint4* ent_fit;                // [cap_ch][6] the same pieces' first 96 bytes of tpc_track (state,
                                 // x, alpha, chi2, covariance), in the same order
  unsigned long long* bin_state; // scan state of bin_off
  float chi2_cut;
  int edge_u;
  int dz_u;                      // |Z(B innermost) - Z(A outermost)| bound of a candidate (u)
  int bin_w;                     // zeta bin width (u), >= dz_u
  int n_zb;                      // zeta bins per virtual sector
};

// Work space of the optional track-model compression (step 10).
struct CmpWork {
  int8_t* code_y;                // [cap_cl] residual codes (coded clusters)
  int8_t* code_z;
  uint8_t* status;               // [cap_cl] 0 not on a track, 1 coded, 2 escaped
  unsigned long long* ctl;       // [0] coded, [1] escaped
  float step_y, step_z;          // cm
};

// Work space of the optional entropy coding of the step-10 codes (step 10c).
struct EntWork {
  unsigned long long* hist;      // [512] symbol counts, y then z alphabet
  uint8_t* len;                  // [512] codeword lengths
  uint32_t* code;                // [512] canonical codewords
  uint64_t* bits;                // [cap_cl] bits per cluster, scanned in place to stream offsets
  unsigned long long* scan_state;
  unsigned int* ticket;          // scan ticket
  unsigned long long* total;     // stream length in bits
  uint32_t* words;               // [cap_words] the stream
  unsigned long long cap_words;
};

// Work space of the optional drift calibration (step 11).
struct CalWork {
  float* tv;                     // [cap_ch] vertex time bin per track, -1 if unused
  unsigned* hist;                // [2^20] tracks per whole vertex time bin
  unsigned long long* mode;      // count << 32 | (2^20 - 1 - bin) of the fullest bin
  double* sum;                   // [2] window sums of t_v
  unsigned long long* cnt;       // [2] window counts
  float zeta_per_bin;            // cm of the drift coordinate per time bin
};

// Warp-aggregated atomicAdd of 1 on one counter: the lanes that call it
// together take consecutive values with a single atomic (correct under
// independent thread scheduling: the group is whoever is converged here).
__device__ __forceinline__ unsigned long long aggregated_inc(unsigned long long* ctr) {
  const unsigned mask = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  unsigned long long base = 0;
  if (lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + __popc(mask & ((1u << lane) - 1u));
}

// Warp-aggregated atomicAdd of 1 on counters indexed by key: lanes with equal
// keys share one atomic and take consecutive values.
__device__ __forceinline__ unsigned aggregated_inc_keyed(unsigned* base_ptr, int key) {
  const unsigned mask = __activemask();
  const unsigned peers = __match_any_sync(mask, key);
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(peers) - 1;
  unsigned base = 0;
  if (lane == leader) base = atomicAdd(base_ptr + key, (unsigned)__popc(peers));
  base = __shfl_sync(peers, base, leader);
  return base + __popc(peers & ((1u << lane) - 1u));
}

// Event of cluster c in a batch: the last e with row_start[e * n_phys * R] <= c.
__device__ __forceinline__ int event_of(const DevGeom& G, const DevWork& W, unsigned long long c) {
  int lo = 0, hi = G.n_events - 1;
  const unsigned stride = (unsigned)(G.n_phys * G.n_rows);
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((unsigned long long)W.row_start[(unsigned)mid * stride] <= c) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Virtual sector of cluster c whose record holds physical sector s.
__device__ __forceinline__ int vsector_of(const DevGeom& G, const DevWork& W, unsigned long long c, int s) {
  return G.n_events > 1 ? s + G.n_phys * event_of(G, W, c) : s;
}

}  // namespace tpc
