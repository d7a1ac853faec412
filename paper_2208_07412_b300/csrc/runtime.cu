// runtime.cu — host side of the C ABI declared in include/tpc.h.
//
// A context owns n_slots slots.  Each slot has its own stream, its own device
// work space (allocated once, regrown only when a timeframe needs more) and a
// pinned block of counters that the pipeline copies back at its end, so
// tpc_poll never needs an extra synchronising copy.  A timeframe's whole
// pipeline (find -> CA -> merge -> fit) is enqueued on its slot's stream by
// tpc_submit_timeframe; nothing on the host waits for the device until the
// caller polls or fetches results.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "tpc_internal.cuh"

namespace tpc {
size_t find_smem_bytes(int npmax, int nw);
cudaError_t launch_find(const DevGeom&, const DevParams&, const DevWork&, unsigned int, int, const LaunchCfg&,
                        cudaStream_t, cudaStream_t, cudaEvent_t, cudaEvent_t, unsigned long long*, int*);
cudaError_t launch_ca(const DevGeom&, const DevParams&, const DevWork&, int, const LaunchCfg&, cudaStream_t, int*);
cudaError_t launch_merge(const DevGeom&, const DevParams&, const DevWork&, int, const LaunchCfg&, cudaStream_t,
                         unsigned long long*, int*);
cudaError_t launch_fit(const DevGeom&, const DevParams&, const DevWork&, int, const LaunchCfg&, cudaStream_t, int*);
size_t scan_tiles(unsigned long long cap);
cudaError_t prepare_find();
cudaError_t prepare_find2();
cudaError_t launch_find2(const DevGeom&, const DevParams&, const DevWork&, unsigned int, int, const LaunchCfg&,
                         cudaStream_t, unsigned long long*, int*);
cudaError_t launch_xsec(const DevGeom&, const DevParams&, const DevWork&, const XsWork&, int, cudaStream_t);
cudaError_t launch_loopers(const DevGeom&, const DevParams&, const DevWork&, const LoopWork&, int, cudaStream_t);
cudaError_t launch_compress(const DevParams&, const DevWork&, const CmpWork&, int, cudaStream_t);
cudaError_t launch_entropy(const DevWork&, const CmpWork&, const EntWork&, int, cudaStream_t);
cudaError_t launch_calibrate(const DevParams&, const DevWork&, const CalWork&, int, cudaStream_t);
}  // namespace tpc

using namespace tpc;

static thread_local std::string g_err;
static tpc_status fail(tpc_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
namespace tpc {
void set_last_error(const char* msg) { g_err = msg; }
}  // namespace tpc
#define CUDA_TRY(expr)                                                                          \
  do {                                                                                          \
    cudaError_t e_ = (expr);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(TPC_E_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));              \
  } while (0)

namespace {

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Slot {
  int index = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaEvent_t ev_stage[TPC_N_STAGES + 1] = {};
  cudaEvent_t ev_done = nullptr, ev_input = nullptr;
  cudaStream_t aux = nullptr;                         // second stream of the finder (light windows)
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // device buffers
  Buf pages, offsets, winstate, cl, clx, cly, clz, clt, rowstart, chrow, up, down, score, edge, jump, chlen, scanv,
      scanst, chainof, clchain, ch_i32, besta, bestb, trk_i32, trackcl, cl2trk, tracks, ctrl, scratch, wincnt, winsoff,
      candab, candsc, lenhist, evinfo, xs, lp, cmp, cal, dense, runrec, dtab;
  unsigned long long* h_ctrl = nullptr;   // pinned copy of [ctr | err]
  // batch tables, device (evinfo) and pinned host copy, same layout:
  // u64 base[kMaxBatch], u64 bytes[kMaxBatch], u32 cl_start[kMaxBatch + 1],
  // u32 trk_start[kMaxBatch + 1]
  uint64_t* h_ev = nullptr;
  uint32_t n_events = 1;
  // cross-sector merge results of the current ticket (tpc_merge_sectors)
  bool xs_done = false;
  uint64_t xs_n = 0, xs_links = 0;
  size_t xs_bytes = 0;
  // looper-leg join results of the current ticket (tpc_join_loopers)
  bool lp_done = false;
  uint64_t lp_links = 0, lp_tracks = 0;
  size_t lp_bytes = 0;
  // track-model compression of the current ticket (tpc_compress_clusters)
  bool cmp_done = false;
  size_t cmp_bytes = 0, cal_bytes = 0;
  // capacities
  uint64_t cap_pages = 0, cap_windows = 0, cap_cl = 0, cap_ch = 0, cap_runs = 0;
  // ticket
  bool in_use = false;
  uint64_t ticket = 0;
  int state = TPC_STATE_QUEUED;
  tpc_status status = TPC_OK;
  int runs = 0, launches = 0;
  // the captured pipeline of this slot, valid for one input shape
  cudaGraphExec_t gexec = nullptr;
  bool graph_broken = false;
  DevWork gk_W{};        // the work-space wiring and input shape the graph was captured with
  uint32_t gk_T = 0, gk_nwin = 0, gk_tune = 0;
  // timeframe
  const void* user_pages = nullptr;
  const uint64_t* user_offsets = nullptr;
  uint64_t pages_bytes = 0;
  unsigned n_windows = 0;
  uint32_t n_time_bins = 0, tf_flags = 0;
  DevWork W{};
};

// A submitted request that waits for a slot and memory.
struct Pending {
  uint64_t ticket = 0;
  bool batch = false;
  std::vector<tpc_timeframe_desc> descs;
};

}  // namespace

struct tpc_context {
  tpc_geometry geom;
  tpc_params params;
  DevGeom G{};
  DevParams P{};
  LaunchCfg L{};
  uint32_t tune_gen = 0;    // bumped when L changes (captured graphs are re-made)
  int device = 0, n_sm = 148;
  uint64_t budget = 0, used = 0;
  uint32_t flags = 0;
  std::vector<Slot> slots;
  std::deque<Pending> pending;                               // arrival order
  std::vector<std::pair<uint64_t, tpc_status>> failed;       // queued requests that could not start
  uint64_t next_ticket = 1;
  std::mutex mu;
};

// ------------------------------------------------------------------ params / geometry
extern "C" tpc_status tpc_params_default(tpc_params* p) {
  if (!p) return fail(TPC_E_INVAL, "tpc_params_default: null");
  std::memset(p, 0, sizeof(*p));
  p->version = TPC_PARAMS_VERSION;
  p->q_peak_min = 10;
  p->ca_slope_y_num = 1; p->ca_slope_y_den = 1;
  p->ca_slope_z_num = 11; p->ca_slope_z_den = 10;
  p->ca_cut = 256;
  p->min_chain = 5;
  p->merge_cut = 384;
  p->merge_gap_min = 1; p->merge_gap_max = 6;
  p->merge_max_passes = 8;
  p->min_track = 10;
  p->fit_passes = 3;
  p->bz = 0.5;
  p->sigma_y = 0.02; p->sigma_z = 0.03;
  p->c0[0] = 4.0; p->c0[1] = 4.0; p->c0[2] = 0.25; p->c0[3] = 1.0; p->c0[4] = 100.0;
  p->fp32_pd_margin = 0.0;
  p->split_charge = 0;
  return TPC_OK;
}

extern "C" tpc_status tpc_create_geometry(const tpc_geometry_desc* d, tpc_geometry** out) {
  if (!d || !out || !d->npads || !d->row_x) return fail(TPC_E_INVAL, "tpc_create_geometry: null argument");
  if (d->n_sectors < 1 || d->n_sectors > TPC_MAX_SECTORS) return fail(TPC_E_INVAL, "n_sectors out of range");
  if (d->n_rows < 3 || d->n_rows > TPC_MAX_ROWS) return fail(TPC_E_INVAL, "n_rows out of range");
  auto* g = new tpc_geometry;
  g->n_sectors = d->n_sectors;
  g->n_rows = d->n_rows;
  g->npmax = 0;
  for (int r = 0; r < d->n_rows; r++) {
    if (d->npads[r] < 3 || d->npads[r] > TPC_MAX_PADS) { delete g; return fail(TPC_E_INVAL, "npads out of range"); }
    if (d->row_x[r] <= 0 || d->row_x[r] > 1000000 || (r > 0 && d->row_x[r] <= d->row_x[r - 1])) {
      delete g;
      return fail(TPC_E_INVAL, "row_x must be positive and strictly increasing");
    }
    g->npads.push_back(d->npads[r]);
    g->row_x.push_back(d->row_x[r]);
    g->npmax = std::max(g->npmax, d->npads[r]);
  }
  *out = g;
  return TPC_OK;
}

extern "C" void tpc_destroy_geometry(tpc_geometry* g) { delete g; }

static tpc_status check_params(const tpc_params& p, const tpc_geometry& g) {
  if (p.version != TPC_PARAMS_VERSION) return fail(TPC_E_INVAL, "params: version mismatch");
  if (p.q_peak_min < 1 || p.q_peak_min > 1023) return fail(TPC_E_INVAL, "params: q_peak_min out of range");
  if (p.ns_min_dip < 0 || p.ns_min_dip > 1023) return fail(TPC_E_INVAL, "params: ns_min_dip out of range");
  if (p.ca_slope_y_num < 0 || p.ca_slope_y_den < 1 || p.ca_slope_z_num < 0 || p.ca_slope_z_den < 1 ||
      p.ca_slope_y_num > 1000 || p.ca_slope_z_num > 1000 || p.ca_slope_y_den > 1000 || p.ca_slope_z_den > 1000)
    return fail(TPC_E_INVAL, "params: CA slopes out of range");
  if (p.ca_cut < 0 || p.min_chain < 2 || p.min_track < 3) return fail(TPC_E_INVAL, "params: cuts out of range");
  if (p.merge_cut < 0 || p.merge_cut > 16383 || p.merge_gap_min < 1 || p.merge_gap_max < p.merge_gap_min ||
      p.merge_max_passes < 0 || p.merge_max_passes > 16)
    return fail(TPC_E_INVAL, "params: merge settings out of range");
  if (p.fit_passes < 1 || p.fit_passes > 15 || !(p.sigma_y > 0) || !(p.sigma_z > 0))
    return fail(TPC_E_INVAL, "params: fit settings out of range");
  for (int i = 0; i < 5; i++)
    if (!(p.c0[i] > 0)) return fail(TPC_E_INVAL, "params: c0 must be positive");
  if (!(p.fp32_pd_margin >= 0 && p.fp32_pd_margin < 1))
    return fail(TPC_E_INVAL, "params: fp32_pd_margin must be in [0, 1)");
  if (p.split_charge != 0 && p.split_charge != 1) return fail(TPC_E_INVAL, "params: split_charge must be 0 or 1");
  // CA scores must fit the 41-bit field of the edge-row keys
  for (int r = 1; r + 1 < g.n_rows; r++) {
    long double lim = (long double)p.ca_cut * 64.0L * (g.row_x[r + 1] - g.row_x[r - 1]);
    if (2.0L * lim * lim >= 2199023255552.0L) return fail(TPC_E_INVAL, "params: ca_cut too large for the geometry");
  }
  return TPC_OK;
}

// ------------------------------------------------------------------ buffers
static void free_buf(Buf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}
static cudaError_t ensure(Buf& b, size_t bytes) {
  if (b.bytes >= bytes && b.p) return cudaSuccess;
  free_buf(b);
  cudaError_t e = cudaMalloc(&b.p, std::max<size_t>(bytes, 256));
  if (e == cudaSuccess) b.bytes = std::max<size_t>(bytes, 256);
  return e;
}

// Steps 1-4 by the two-pass finder (the default) rather than the fused or the
// dense-plane variant.
static bool two_pass(const tpc_context* ctx) {
  return !(ctx->flags & (TPC_CTX_DENSE_FINDER | TPC_CTX_FUSED_FINDER));
}

// Units of the two-pass finder per window (its scan and span arrays are sized for them).
constexpr uint64_t kUnitsPerWindow = 4;

// Pad runs the two-pass finder's array must hold for pages_bytes of pages: a
// run takes 2 bytes of its page and at least one digit, 10 bits of an ADC word.
static uint64_t run_cap(uint64_t pages_bytes) { return pages_bytes / 3 + 3; }

static size_t slot_bytes(uint64_t pages, uint64_t windows, uint64_t cap_cl, uint64_t cap_ch, int nsr,
                         size_t dense = 0, uint64_t cap_runs = 0) {
  size_t b = dense + pages + 16 + windows * (8 + 8 + 8 * kUnitsPerWindow + 4 * (kUnitsPerWindow + 2) + 48 +
                                             112 * kUnitsPerWindow) +
             cap_runs * 8 + cap_cl * (16 + 16 + 16 + 8 + 8 + 8 + 8 + 4 + 8 + 4 + 4 + 4 + 4) +
             (scan_tiles(cap_cl) + scan_tiles(cap_ch) + scan_tiles(windows * kUnitsPerWindow)) * 8 +
             cap_ch * (14 * 4 + 8 + 16 + sizeof(tpc_track) + 4 * 12) +
             (size_t)(nsr + 1) * 8 + (size_t)(4 * windows + nsr + 2) * 4 + 1024;
  return b;
}

static tpc_status slot_reserve(tpc_context* ctx, Slot& s, uint64_t pages_bytes, uint64_t windows,
                               uint64_t cap_cl, bool need_pages) {
  const int nsr = ctx->geom.n_sectors * ctx->geom.n_rows * (int)s.n_events;
  uint64_t cap_ch = cap_cl / (uint64_t)ctx->params.min_chain + 16;
  uint64_t want_pages = need_pages ? pages_bytes : 0;
  // dense-plane finder variant: one ADC per (sector row, time bin, pad)
  const size_t dstride = (size_t)((ctx->geom.npmax + 7) & ~7);
  const size_t want_dense = (ctx->flags & TPC_CTX_DENSE_FINDER) ? (size_t)windows * kFrag * dstride * 2 : 0;
  const uint64_t want_runs = two_pass(ctx) ? run_cap(pages_bytes) : 0;
  size_t cur = slot_bytes(s.cap_pages, s.cap_windows, s.cap_cl, s.cap_ch, nsr, s.dense.bytes, s.cap_runs);
  size_t need = slot_bytes(std::max(s.cap_pages, want_pages), std::max(s.cap_windows, windows),
                           std::max(s.cap_cl, cap_cl), std::max(s.cap_ch, cap_ch), nsr,
                           std::max(s.dense.bytes, want_dense), std::max(s.cap_runs, want_runs));
  if (ctx->used - cur + need > ctx->budget)
    return fail(TPC_E_NOMEM, "timeframe needs " + std::to_string(need) + " device bytes; budget left " +
                                 std::to_string(ctx->budget - ctx->used + cur));
  if (want_pages > s.cap_pages) { CUDA_TRY(ensure(s.pages, want_pages + 16)); s.cap_pages = want_pages; }
  if (windows > s.cap_windows) {
    CUDA_TRY(ensure(s.offsets, windows * 8));
    CUDA_TRY(ensure(s.winstate, windows * 8));
    CUDA_TRY(ensure(s.wincnt, windows * kUnitsPerWindow * 8));
    // span starts (one per unit) | light list | heavy list
    CUDA_TRY(ensure(s.winsoff, windows * (kUnitsPerWindow + 2) * 4));
    // window table rows (3 x 16 bytes), then the units' descriptors (7 x 16 bytes each)
    CUDA_TRY(ensure(s.dtab, windows * (48 + 112 * kUnitsPerWindow)));
    s.cap_windows = windows;
  }
  if (want_runs > s.cap_runs) {
    CUDA_TRY(ensure(s.runrec, want_runs * 8));
    s.cap_runs = want_runs;
  }
  if (cap_cl > s.cap_cl) {
    CUDA_TRY(ensure(s.cl, cap_cl * 16));
    CUDA_TRY(ensure(s.scratch, cap_cl * 16));
    CUDA_TRY(ensure(s.clx, cap_cl * 4)); CUDA_TRY(ensure(s.cly, cap_cl * 4));
    CUDA_TRY(ensure(s.clz, cap_cl * 4)); CUDA_TRY(ensure(s.clt, cap_cl * 4));
    CUDA_TRY(ensure(s.up, cap_cl * 4)); CUDA_TRY(ensure(s.down, cap_cl * 4));
    CUDA_TRY(ensure(s.score, cap_cl * 8)); CUDA_TRY(ensure(s.edge, cap_cl * 8));
    CUDA_TRY(ensure(s.jump, cap_cl * 8)); CUDA_TRY(ensure(s.chlen, cap_cl * 4));
    CUDA_TRY(ensure(s.scanv, cap_cl * 8));
    CUDA_TRY(ensure(s.chainof, cap_cl * 4)); CUDA_TRY(ensure(s.clchain, cap_cl * 4));
    CUDA_TRY(ensure(s.trackcl, cap_cl * 4)); CUDA_TRY(ensure(s.cl2trk, cap_cl * 4));
    s.cap_cl = cap_cl;
  }
  if (cap_ch > s.cap_ch) {
    CUDA_TRY(ensure(s.ch_i32, cap_ch * 4 * 14));
    CUDA_TRY(ensure(s.bestb, cap_ch * 8));
    CUDA_TRY(ensure(s.besta, cap_ch * 16));
    CUDA_TRY(ensure(s.tracks, cap_ch * sizeof(tpc_track)));
    CUDA_TRY(ensure(s.candab, cap_ch * 4 * 8));
    CUDA_TRY(ensure(s.candsc, cap_ch * 4 * 4));
    s.cap_ch = cap_ch;
  }
  CUDA_TRY(ensure(s.scanst,
                  (scan_tiles(s.cap_cl) + scan_tiles(s.cap_ch) + scan_tiles(s.cap_windows * kUnitsPerWindow)) * 8));
  CUDA_TRY(ensure(s.rowstart, (size_t)(nsr + 1) * 4));
  // first chain per row, then per (row, 64-bin time bucket): 4 buckets per
  // fragment and one past the last, nsr * (4 n_frag + 1) + 1 entries
  CUDA_TRY(ensure(s.chrow, (size_t)(nsr + 1) * 4 + (size_t)(4 * s.cap_windows + nsr + 2) * 4));
  if (want_dense) CUDA_TRY(ensure(s.dense, want_dense));
  CUDA_TRY(ensure(s.ctrl, 256));
  CUDA_TRY(ensure(s.lenhist, 512 * 4));
  ctx->used = ctx->used - cur + slot_bytes(s.cap_pages, s.cap_windows, s.cap_cl, s.cap_ch, nsr, s.dense.bytes,
                                           s.cap_runs);
  // wire the work-space pointers
  DevWork& W = s.W;
  W.clusters = (tpc_cluster*)s.cl.p;
  W.cl_x = (int32_t*)s.clx.p; W.cl_y = (int32_t*)s.cly.p; W.cl_z = (int32_t*)s.clz.p; W.cl_t = (int32_t*)s.clt.p;
  W.row_start = (uint32_t*)s.rowstart.p;
  W.ch_row_start = (uint32_t*)s.chrow.p;
  W.ch_bucket = (uint32_t*)s.chrow.p + (nsr + 1);
  W.dense = (ctx->flags & TPC_CTX_DENSE_FINDER) ? (uint16_t*)s.dense.p : nullptr;
  W.dense_stride = (uint32_t)dstride;
  W.win_state = (unsigned long long*)s.winstate.p;
  W.scratch_cl = (tpc_cluster*)s.scratch.p;
  W.win_cnt = (unsigned long long*)s.wincnt.p;
  W.win_soff = (uint32_t*)s.winsoff.p;
  W.light_list = (uint32_t*)s.winsoff.p + kUnitsPerWindow * s.cap_windows;
  W.heavy_list = (uint32_t*)s.winsoff.p + (kUnitsPerWindow + 1) * s.cap_windows;
  W.runs = (uint2*)s.runrec.p;
  W.dtab = (uint4*)s.dtab.p;
  W.udesc = (uint4*)s.dtab.p + 3 * s.cap_windows;
  W.cap_runs = s.cap_runs;
  W.up = (int32_t*)s.up.p; W.down = (int32_t*)s.down.p;
  W.score = (int64_t*)s.score.p;
  W.edge_key = (unsigned long long*)s.edge.p;
  W.jump = (unsigned long long*)s.jump.p;
  W.chain_len = (int32_t*)s.chlen.p;
  W.scan_val = (uint64_t*)s.scanv.p;
  W.scan_state = (unsigned long long*)s.scanst.p;
  W.chain_of = (int32_t*)s.chainof.p;
  W.cl_chain = (int32_t*)s.clchain.p;
  int32_t* ci = (int32_t*)s.ch_i32.p;
  const uint64_t C = s.cap_ch;
  W.ch_root = ci; W.ch_len = ci + C; W.ch_b2 = ci + 2 * C; W.ch_top = ci + 3 * C; W.ch_top2 = ci + 4 * C;
  W.ch_next = ci + 5 * C; W.ch_prev = ci + 6 * C; W.ch_track = ci + 7 * C; W.ch_off = ci + 8 * C;
  W.grp_total = ci + 9 * C; W.trk_first = ci + 10 * C; W.trk_ncl = ci + 11 * C; W.trk_off = ci + 12 * C;
  W.ch_t = ci + 13 * C;
  W.fit_order = W.ch_off;   // free once the clusters are assigned to tracks
  W.len_hist = (uint32_t*)s.lenhist.p;
  W.best_b = (unsigned long long*)s.bestb.p;
  W.best_a = (unsigned long long*)s.besta.p;
  W.cand_ab = (unsigned long long*)s.candab.p;
  W.cand_sc = (uint32_t*)s.candsc.p;
  W.cap_cand = s.cap_ch * 4;
  W.track_cl = (int32_t*)s.trackcl.p;
  W.trk_xyz = (int4*)s.scratch.p;   // the finder's scratch is free once the clusters are compacted
  W.cl2trk = (int32_t*)s.cl2trk.p;
  W.tracks = (tpc_track*)s.tracks.p;
  W.ctr = (unsigned long long*)s.ctrl.p;
  W.err = (uint32_t*)((unsigned long long*)s.ctrl.p + CTR_COUNT);
  W.tickets = (unsigned int*)((unsigned long long*)s.ctrl.p + CTR_COUNT + 1);
  W.cap_cl = s.cap_cl;
  W.cap_ch = s.cap_ch;
  return TPC_OK;
}

static void slot_free(tpc_context* ctx, Slot& s) {
  Buf* all[] = {&s.pages, &s.offsets, &s.winstate, &s.cl, &s.clx, &s.cly, &s.clz, &s.clt, &s.rowstart, &s.chrow, &s.up,
                &s.down, &s.score, &s.edge, &s.jump, &s.chlen, &s.scanv, &s.scanst, &s.chainof, &s.clchain,
                &s.ch_i32, &s.besta, &s.bestb, &s.trk_i32, &s.trackcl, &s.cl2trk, &s.tracks, &s.ctrl,
                &s.scratch, &s.wincnt, &s.winsoff, &s.candab, &s.candsc, &s.lenhist, &s.evinfo, &s.xs, &s.lp, &s.cmp, &s.cal, &s.dense,
                &s.runrec, &s.dtab};
  for (Buf* b : all) free_buf(*b);
  for (auto& e : s.ev_stage) if (e) cudaEventDestroy(e);
  if (s.ev_done) cudaEventDestroy(s.ev_done);
  if (s.ev_input) cudaEventDestroy(s.ev_input);
  if (s.ev_fork) cudaEventDestroy(s.ev_fork);
  if (s.ev_join) cudaEventDestroy(s.ev_join);
  if (s.aux) cudaStreamDestroy(s.aux);
  if (s.gexec) cudaGraphExecDestroy(s.gexec);
  if (s.own_stream && s.stream) cudaStreamDestroy(s.stream);
  if (s.h_ctrl) cudaFreeHost(s.h_ctrl);
  if (s.h_ev) cudaFreeHost(s.h_ev);
  (void)ctx;
}

// ------------------------------------------------------------------ context
extern "C" tpc_status tpc_create_context(const tpc_geometry* geom, const tpc_params* params, int device,
                                         uint64_t mem_budget, int n_slots, void* stream, uint32_t flags,
                                         tpc_context** out) {
  if (!geom || !out) return fail(TPC_E_INVAL, "tpc_create_context: null argument");
  if (n_slots < 1 || n_slots > 64) return fail(TPC_E_INVAL, "n_slots must be 1..64");
  tpc_params p;
  if (params) p = *params; else tpc_params_default(&p);
  tpc_status st = check_params(p, *geom);
  if (st) return st;
  if (p.split_charge && (flags & (TPC_CTX_DENSE_FINDER | TPC_CTX_FUSED_FINDER)))
    return fail(TPC_E_INVAL, "params: split_charge needs the two-pass finder (no TPC_CTX_DENSE_FINDER / "
                             "TPC_CTX_FUSED_FINDER)");
  int ndev = 0;
  CUDA_TRY(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return fail(TPC_E_INVAL, "no such CUDA device");
  CUDA_TRY(cudaSetDevice(device));
  auto* ctx = new tpc_context;
  ctx->geom = *geom;
  ctx->params = p;
  ctx->device = device;
  ctx->budget = mem_budget ? mem_budget : (8ull << 30);
  ctx->flags = flags;
  cudaDeviceGetAttribute(&ctx->n_sm, cudaDevAttrMultiProcessorCount, device);
  DevGeom& G = ctx->G;
  G.n_sectors = geom->n_sectors;
  G.n_phys = geom->n_sectors;
  G.n_events = 1;
  G.n_rows = geom->n_rows;
  G.npmax = geom->npmax;
  G.nw = (geom->npmax + 31) / 32;
  for (int r = 0; r < geom->n_rows; r++) { G.npads[r] = geom->npads[r]; G.xrow[r] = 64 * geom->row_x[r]; }
  DevParams& P = ctx->P;
  P.q_peak_min = p.q_peak_min;
  P.ns_min_dip = p.ns_min_dip;
  P.split_charge = p.split_charge;
  P.sy_num = p.ca_slope_y_num; P.sy_den = p.ca_slope_y_den;
  P.sz_num = p.ca_slope_z_num; P.sz_den = p.ca_slope_z_den;
  P.ca_cut = p.ca_cut; P.min_chain = p.min_chain;
  P.merge_cut = p.merge_cut; P.gap_min = p.merge_gap_min; P.gap_max = p.merge_gap_max;
  P.merge_passes = p.merge_max_passes; P.min_track = p.min_track; P.fit_passes = p.fit_passes;
  P.kfac_d = -p.bz * 0.299792458 * 1e-2;
  P.kfac = (float)P.kfac_d;
  P.sy2_d = p.sigma_y * p.sigma_y; P.sz2_d = p.sigma_z * p.sigma_z;
  P.sy2 = (float)P.sy2_d; P.sz2 = (float)P.sz2_d;
  for (int i = 0; i < 5; i++) P.c0[i] = (float)p.c0[i];
  const double u = 7.8125e-4;   // cm per u
  P.kfac_u = (float)(P.kfac_d * u);
  P.sy2_ud = P.sy2_d / (u * u);
  P.sz2_ud = P.sz2_d / (u * u);
  P.sy2_u = (float)P.sy2_ud;
  P.sz2_u = (float)P.sz2_ud;
  for (int i = 0; i < 5; i++) {
    const double c = p.c0[i] / (i < 2 ? u * u : 1.0);
    P.c0_u[i] = (float)c;
    P.pd_min_u[i] = (float)(p.fp32_pd_margin * c);
  }
  if (find_smem_bytes(G.npmax, G.nw) > 227 * 1024) { delete ctx; return fail(TPC_E_INVAL, "rows too wide"); }
  if (prepare_find() != cudaSuccess || prepare_find2() != cudaSuccess) {
    delete ctx;
    return fail(TPC_E_CUDA, "cudaFuncSetAttribute failed");
  }
  if (two_pass(ctx)) {   // the two-pass finder's launch shape: 128-thread CTAs, 8 per SM
    ctx->L.find_threads = 128;
    ctx->L.find_ctas_per_sm = 8;
  }
  ctx->slots.resize(n_slots);
  for (int i = 0; i < n_slots; i++) {
    Slot& s = ctx->slots[i];
    s.index = i;
    cudaError_t e = cudaSuccess;
    if (i == 0 && stream) { s.stream = (cudaStream_t)stream; s.own_stream = false; }
    else { e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking); s.own_stream = true; }
    for (auto& ev : s.ev_stage) if (e == cudaSuccess) e = cudaEventCreate(&ev);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev_done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev_input, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s.aux, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&s.h_ctrl, 256);
    if (e != cudaSuccess) {
      for (auto& s2 : ctx->slots) slot_free(ctx, s2);
      delete ctx;
      return fail(TPC_E_CUDA, std::string("context setup: ") + cudaGetErrorString(e));
    }
  }
  *out = ctx;
  return TPC_OK;
}

extern "C" void tpc_destroy_context(tpc_context* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  for (auto& s : ctx->slots) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    slot_free(ctx, s);
  }
  delete ctx;
}

// ------------------------------------------------------------------ pipeline
constexpr uint32_t kMaxBatch = TPC_MAX_BATCH;
constexpr size_t kEvBytes = (size_t)kMaxBatch * 16 + 2 * ((size_t)kMaxBatch + 1) * 4;
constexpr uint64_t kBadOffset = 1ull << 62;   // fails every page-range check

// Offsets of a batch: event e's page offsets (copied in place) rebased onto its
// position in the concatenated page buffer; an offset outside the event's own
// pages becomes invalid, so a corrupt page table stays corrupt.
__global__ void k_rebase_offsets(uint64_t* offs, unsigned long long nwin_e, int n_events, const uint64_t* ev) {
  const unsigned long long n = nwin_e * (unsigned long long)n_events;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long e = i / nwin_e;
    const uint64_t o = offs[i];
    offs[i] = o < ev[kMaxBatch + e] ? o + ev[e] : kBadOffset;
  }
}

// First cluster and first track of every event of a batch (entry n_events:
// the totals).  Tracks are ordered by their lowest cluster, so an event's
// first track is the first whose lowest cluster is at or past its first cluster.
__global__ void k_event_starts(DevWork W, int n_events, unsigned stride, uint32_t* cl_start, uint32_t* trk_start) {
  const unsigned long long ntrk = min(W.ctr[CTR_NTRK], (unsigned long long)W.cap_ch);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e <= n_events; e += gridDim.x * blockDim.x) {
    const uint32_t c = W.row_start[(unsigned long long)e * stride];
    unsigned long long lo = 0, hi = ntrk;
    while (lo < hi) {
      const unsigned long long mid = (lo + hi) >> 1;
      if ((uint32_t)W.trk_first[mid] < c) lo = mid + 1; else hi = mid;
    }
    cl_start[e] = c;
    trk_start[e] = (uint32_t)lo;
  }
}

static tpc_status enqueue_body(tpc_context* ctx, Slot& s, bool capturing) {
  cudaStream_t st = s.stream;
  // inside a capture an event record must become an external event node
  const unsigned evf = capturing ? cudaEventRecordExternal : cudaEventRecordDefault;
  DevWork& W = s.W;
  DevGeom G = ctx->G;
  G.n_time_bins = (int)s.n_time_bins;
  G.n_frag = (int)((s.n_time_bins + kFrag - 1) / kFrag);
  G.n_events = (int)s.n_events;
  G.n_sectors = ctx->geom.n_sectors * (int)s.n_events;
  const bool timing = ctx->flags & TPC_CTX_STAGE_TIMING;
  s.launches = 0;
  CUDA_TRY(cudaMemsetAsync(s.ctrl.p, 0, 256, st));
  CUDA_TRY(cudaMemsetAsync(W.len_hist, 0, 512 * 4, st));
  const size_t tiles_a = scan_tiles(s.cap_cl), tiles_b = scan_tiles(s.cap_ch);
  CUDA_TRY(cudaMemsetAsync(W.scan_state, 0, (tiles_a + tiles_b + scan_tiles(s.n_windows * kUnitsPerWindow)) * 8, st));
  if (timing) CUDA_TRY(cudaEventRecordWithFlags(s.ev_stage[0], st, evf));
  const LaunchCfg& L = ctx->L;
  if (two_pass(ctx))
    CUDA_TRY(launch_find2(G, ctx->P, W, s.n_windows, ctx->n_sm, L, st, W.scan_state + tiles_a + tiles_b,
                          &s.launches));
  else
    CUDA_TRY(launch_find(G, ctx->P, W, s.n_windows, ctx->n_sm, L, st, s.aux, s.ev_fork, s.ev_join,
                         W.scan_state + tiles_a + tiles_b, &s.launches));
  if (timing) CUDA_TRY(cudaEventRecordWithFlags(s.ev_stage[1], st, evf));
  CUDA_TRY(launch_ca(G, ctx->P, W, ctx->n_sm, L, st, &s.launches));
  if (timing) CUDA_TRY(cudaEventRecordWithFlags(s.ev_stage[2], st, evf));
  CUDA_TRY(launch_merge(G, ctx->P, W, ctx->n_sm, L, st, (unsigned long long*)W.scan_state + tiles_a, &s.launches));
  if (timing) CUDA_TRY(cudaEventRecordWithFlags(s.ev_stage[3], st, evf));
  CUDA_TRY(launch_fit(G, ctx->P, W, ctx->n_sm, L, st, &s.launches));
  if (timing) CUDA_TRY(cudaEventRecordWithFlags(s.ev_stage[4], st, evf));
  if (s.n_events > 1) {
    uint32_t* d_st = (uint32_t*)((uint64_t*)s.evinfo.p + 2 * kMaxBatch);
    k_event_starts<<<(s.n_events + 256) / 256, 256, 0, st>>>(W, (int)s.n_events,
                                                             (unsigned)(ctx->geom.n_sectors * ctx->geom.n_rows),
                                                             d_st, d_st + kMaxBatch + 1);
    CUDA_TRY(cudaGetLastError());
    s.launches++;
    uint32_t* h_st = (uint32_t*)(s.h_ev + 2 * kMaxBatch);
    CUDA_TRY(cudaMemcpyAsync(h_st, d_st, (s.n_events + 1) * 4, cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(h_st + kMaxBatch + 1, d_st + kMaxBatch + 1, (s.n_events + 1) * 4,
                             cudaMemcpyDeviceToHost, st));
  }
  CUDA_TRY(cudaMemcpyAsync(s.h_ctrl, s.ctrl.p, 256, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaEventRecordWithFlags(s.ev_done, st, evf));
  return TPC_OK;
}

// The whole pipeline of a timeframe, replayed from a CUDA graph captured once
// per slot and input shape (pointers, sizes, capacities): one launch instead of
// ~40 enqueues.  A capture that fails falls back to plain launches for good.
static tpc_status enqueue(tpc_context* ctx, Slot& s) {
  const bool use_graph = !(ctx->flags & TPC_CTX_NO_GRAPHS) && !s.graph_broken;
  if (!use_graph) {
    tpc_status st = enqueue_body(ctx, s, false);
    if (st == TPC_OK) s.runs++;
    return st;
  }
  const bool same = s.gexec && s.gk_T == s.n_time_bins && s.gk_nwin == s.n_windows && s.gk_tune == ctx->tune_gen &&
                    std::memcmp(&s.gk_W, &s.W, sizeof(DevWork)) == 0;
  if (!same) {
    // capture the pipeline; a graph of the same topology (new input pointers,
    // regrown buffers) updates the instantiated one in place
    cudaGraph_t g = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(s.stream, cudaStreamCaptureModeThreadLocal));
    tpc_status st = enqueue_body(ctx, s, true);
    cudaError_t e = cudaStreamEndCapture(s.stream, &g);
    bool ok = st == TPC_OK && e == cudaSuccess && g;
    if (ok && s.gexec) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(s.gexec, g, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(s.gexec);
        s.gexec = nullptr;
      }
    }
    if (ok && !s.gexec) ok = cudaGraphInstantiate(&s.gexec, g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      if (s.gexec) cudaGraphExecDestroy(s.gexec);
      s.gexec = nullptr;
      s.graph_broken = true;
      cudaGetLastError();
      st = enqueue_body(ctx, s, false);
      if (st == TPC_OK) s.runs++;
      return st;
    }
    s.gk_W = s.W;
    s.gk_tune = ctx->tune_gen;
    s.gk_T = s.n_time_bins;
    s.gk_nwin = s.n_windows;
  }
  CUDA_TRY(cudaGraphLaunch(s.gexec, s.stream));
  s.runs++;
  return TPC_OK;
}

static Slot* find_ticket(tpc_context* ctx, uint64_t ticket) {
  for (auto& s : ctx->slots)
    if (s.in_use && s.ticket == ticket) return &s;
  return nullptr;
}

// An upper bound of the clusters any valid timeframe of pages_bytes can hold.
// A cluster needs a peak digit (4/3 B: three 10-bit ADCs per 32-bit word).
// Two peaks of one time bin are at least two pads apart (peaks are never
// adjacent), so between consecutive peaks of an entry lies either a digit
// (4/3 B) or the start of another run (2 B): at least 8/3 B per peak beyond the
// first of each entry, whose entry and run headers (4 B) cost more.  Hence
// clusters <= 3 pages_bytes / 8.
static uint64_t guaranteed_cap_cl(uint64_t pages_bytes) {
  return pages_bytes / 8 * 3 + 3 + 1024;
}

// The initial cluster capacity: one cluster per 20 page bytes (generated
// timeframes hold one per 43-65 bytes); a denser timeframe overflows it, and
// the pipeline re-runs once with the bound above.  At ~156 bytes of work space
// per cluster of capacity, a 5.7 GB timeframe's slot needs ~45 GB for it.
static uint64_t initial_cap_cl(uint64_t pages_bytes) {
  return std::min(std::max<uint64_t>(65536, pages_bytes / 20), guaranteed_cap_cl(pages_bytes));
}

// Validation of one descriptor (before any slot is touched).
static tpc_status check_desc(const tpc_timeframe_desc* tf) {
  if (tf->n_time_bins < 1 || tf->n_time_bins > 65535) return fail(TPC_E_INVAL, "n_time_bins out of range");
  if (!tf->pages || !tf->page_offsets || tf->pages_bytes < 32)
    return fail(TPC_E_INVAL, "pages / page_offsets missing");
  if ((tf->flags & TPC_TF_DEVICE_INPUT) && ((uintptr_t)tf->pages & 15))
    return fail(TPC_E_INVAL, "device pages must be 16-byte aligned");
  return TPC_OK;
}

// Start one timeframe on free slot s (lock held).
static tpc_status start_timeframe(tpc_context* ctx, Slot* s, const tpc_timeframe_desc* tf) {
  const bool dev_in = tf->flags & TPC_TF_DEVICE_INPUT;
  s->n_events = 1;
  s->xs_done = false;
  s->lp_done = false;
  s->cmp_done = false;
  const unsigned nfrag = (tf->n_time_bins + kFrag - 1) / kFrag;
  const uint64_t nwin = (uint64_t)ctx->geom.n_sectors * ctx->geom.n_rows * nfrag;
  if (nwin > 0xffffffffull) return fail(TPC_E_INVAL, "too many windows");
  const uint64_t cap_cl = std::max(initial_cap_cl(tf->pages_bytes), s->cap_cl);
  tpc_status st = slot_reserve(ctx, *s, tf->pages_bytes, nwin, cap_cl, !dev_in);
  if (st) return st;
  s->pages_bytes = tf->pages_bytes;
  s->n_windows = (unsigned)nwin;
  s->n_time_bins = tf->n_time_bins;
  s->tf_flags = tf->flags;
  s->runs = 0;
  if (dev_in) {
    s->W.pages = (const uint8_t*)tf->pages;
    s->W.page_offsets = tf->page_offsets;
  } else {
    CUDA_TRY(cudaMemcpyAsync(s->pages.p, tf->pages, tf->pages_bytes, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemcpyAsync(s->offsets.p, tf->page_offsets, nwin * 8, cudaMemcpyHostToDevice, s->stream));
    s->W.pages = (const uint8_t*)s->pages.p;
    s->W.page_offsets = (const uint64_t*)s->offsets.p;
  }
  s->W.pages_bytes = tf->pages_bytes;
  CUDA_TRY(cudaEventRecord(s->ev_input, s->stream));
  return enqueue(ctx, *s);
}

// Start a batch of events on free slot s (lock held); descriptors validated.
static tpc_status start_batch(tpc_context* ctx, Slot* s, const tpc_timeframe_desc* tfs, uint32_t n_events) {
  const uint32_t T = tfs[0].n_time_bins;
  s->xs_done = false;
  s->lp_done = false;
  s->cmp_done = false;
  std::vector<uint64_t> base(n_events), bytes(n_events);
  uint64_t total = 0;
  for (uint32_t e = 0; e < n_events; e++) {
    base[e] = total;
    bytes[e] = tfs[e].pages_bytes;
    total += (tfs[e].pages_bytes + 15) & ~15ull;
  }
  const unsigned nfrag = (T + kFrag - 1) / kFrag;
  const uint64_t nwin_e = (uint64_t)ctx->geom.n_sectors * ctx->geom.n_rows * nfrag;
  const uint64_t nwin = nwin_e * n_events;
  if (nwin > 0xffffffffull) return fail(TPC_E_INVAL, "too many windows");
  if (!s->h_ev) CUDA_TRY(cudaMallocHost((void**)&s->h_ev, kEvBytes));
  CUDA_TRY(ensure(s->evinfo, kEvBytes));
  const uint64_t cap_cl = std::max(initial_cap_cl(total), s->cap_cl);
  s->n_events = n_events;
  tpc_status st = slot_reserve(ctx, *s, total, nwin, cap_cl, true);
  if (st) { s->n_events = 1; return st; }
  s->pages_bytes = total;
  s->n_windows = (unsigned)nwin;
  s->n_time_bins = T;
  s->tf_flags = 0;   // the pages now live in the slot's own buffer
  s->runs = 0;
  // gather the events' pages and page tables, then rebase the offsets
  uint8_t* pages = (uint8_t*)s->pages.p;
  uint64_t* offs = (uint64_t*)s->offsets.p;
  for (uint32_t e = 0; e < n_events; e++) {
    CUDA_TRY(cudaMemcpyAsync(pages + base[e], tfs[e].pages, bytes[e], cudaMemcpyDefault, s->stream));
    CUDA_TRY(cudaMemcpyAsync(offs + e * nwin_e, tfs[e].page_offsets, nwin_e * 8, cudaMemcpyDefault, s->stream));
  }
  // the slot is free, so nothing in flight still reads its pinned table
  std::memcpy(s->h_ev, base.data(), n_events * 8);
  std::memcpy(s->h_ev + kMaxBatch, bytes.data(), n_events * 8);
  uint64_t* d_ev = (uint64_t*)s->evinfo.p;
  CUDA_TRY(cudaMemcpyAsync(d_ev, s->h_ev, 2 * (size_t)kMaxBatch * 8, cudaMemcpyHostToDevice, s->stream));
  const unsigned g = (unsigned)std::min<uint64_t>((nwin + 255) / 256, (uint64_t)ctx->n_sm * 8);
  k_rebase_offsets<<<g, 256, 0, s->stream>>>(offs, nwin_e, (int)n_events, d_ev);
  CUDA_TRY(cudaGetLastError());
  s->W.pages = pages;
  s->W.page_offsets = offs;
  s->W.pages_bytes = total;
  CUDA_TRY(cudaEventRecord(s->ev_input, s->stream));
  return enqueue(ctx, *s);
}

static Slot* free_slot(tpc_context* ctx) {
  for (auto& c : ctx->slots)
    if (!c.in_use) return &c;
  return nullptr;
}

static bool any_in_use(const tpc_context* ctx) {
  for (auto& c : ctx->slots)
    if (c.in_use) return true;
  return false;
}

// Give the device memory of idle slots other than keep back to the budget.
static void reclaim_idle(tpc_context* ctx, const Slot* keep) {
  const int nsr1 = ctx->geom.n_sectors * ctx->geom.n_rows;
  for (auto& c : ctx->slots) {
    if (c.in_use || &c == keep || !c.cap_pages && !c.cap_cl) continue;
    cudaStreamSynchronize(c.stream);
    ctx->used -= slot_bytes(c.cap_pages, c.cap_windows, c.cap_cl, c.cap_ch, nsr1 * (int)c.n_events, c.dense.bytes,
                            c.cap_runs);
    Buf* big[] = {&c.pages, &c.offsets, &c.winstate, &c.cl, &c.clx, &c.cly, &c.clz, &c.clt, &c.up, &c.down,
                  &c.score, &c.edge, &c.jump, &c.chlen, &c.scanv, &c.scanst, &c.chainof, &c.clchain, &c.ch_i32,
                  &c.besta, &c.bestb, &c.trk_i32, &c.trackcl, &c.cl2trk, &c.tracks, &c.scratch, &c.wincnt,
                  &c.winsoff, &c.candab, &c.candsc, &c.xs, &c.lp, &c.cmp, &c.cal, &c.dense, &c.runrec, &c.dtab};
    for (Buf* b : big) free_buf(*b);
    ctx->used -= c.xs_bytes + c.lp_bytes + c.cmp_bytes + c.cal_bytes;
    c.xs_bytes = c.lp_bytes = c.cmp_bytes = c.cal_bytes = 0;
    c.xs_done = c.lp_done = c.cmp_done = false;
    c.cap_pages = c.cap_windows = c.cap_cl = c.cap_ch = c.cap_runs = 0;
  }
}

// Start a request on a free slot, reclaiming idle slots' memory if the budget
// is short.  Returns TPC_E_NOMEM if it still does not fit.
static tpc_status start_request(tpc_context* ctx, Slot* s, const Pending& rq) {
  auto go = [&]() {
    return rq.descs.size() == 1 && !rq.batch ? start_timeframe(ctx, s, rq.descs.data())
                                             : start_batch(ctx, s, rq.descs.data(), (uint32_t)rq.descs.size());
  };
  tpc_status st = go();
  if (st == TPC_E_NOMEM) {
    reclaim_idle(ctx, s);
    st = go();
  }
  if (st) return st;
  s->in_use = true;
  s->ticket = rq.ticket;
  s->state = TPC_STATE_RUNNING;
  s->status = TPC_OK;
  return TPC_OK;
}

// Admit queued requests in arrival order while slots and memory allow (lock
// held).  A request that cannot fit even with every other slot idle fails.
static void admit(tpc_context* ctx) {
  while (!ctx->pending.empty()) {
    Slot* s = free_slot(ctx);
    if (!s) return;
    Pending& rq = ctx->pending.front();
    tpc_status st = start_request(ctx, s, rq);
    if (st == TPC_E_NOMEM && any_in_use(ctx)) return;   // wait for memory
    if (st) ctx->failed.emplace_back(rq.ticket, st);
    ctx->pending.pop_front();
  }
}

// Submit or queue one request (lock not held).
static tpc_status submit(tpc_context* ctx, Pending&& rq, bool nowait, uint64_t* ticket) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  CUDA_TRY(cudaSetDevice(ctx->device));
  rq.ticket = ctx->next_ticket;
  Slot* s = ctx->pending.empty() ? free_slot(ctx) : nullptr;
  if (s) {
    tpc_status st = start_request(ctx, s, rq);
    if (st == TPC_OK) {
      ctx->next_ticket++;
      *ticket = rq.ticket;
      return TPC_OK;
    }
    if (st != TPC_E_NOMEM || !any_in_use(ctx)) return st;
    if (nowait) return fail(TPC_E_BUSY, "not enough of the memory budget free while other timeframes run");
  } else if (nowait) {
    return fail(TPC_E_BUSY, "no free slot: release a finished ticket first");
  }
  // queued: admitted when a slot and memory free up (tpc_release)
  ctx->next_ticket++;
  *ticket = rq.ticket;
  ctx->pending.push_back(std::move(rq));
  return TPC_OK;
}

extern "C" tpc_status tpc_submit_timeframe(tpc_context* ctx, const tpc_timeframe_desc* tf, uint64_t* ticket) {
  if (!ctx || !tf || !ticket) return fail(TPC_E_INVAL, "tpc_submit_timeframe: null argument");
  tpc_status st = check_desc(tf);
  if (st) return st;
  Pending rq;
  rq.descs.assign(tf, tf + 1);
  return submit(ctx, std::move(rq), tf->flags & TPC_TF_NOWAIT, ticket);
}

extern "C" tpc_status tpc_submit_batch(tpc_context* ctx, const tpc_timeframe_desc* tfs, uint32_t n_events,
                                       uint64_t* ticket) {
  if (!ctx || !tfs || !ticket) return fail(TPC_E_INVAL, "tpc_submit_batch: null argument");
  if (n_events < 1 || n_events > kMaxBatch) return fail(TPC_E_INVAL, "n_events out of range");
  for (uint32_t e = 0; e < n_events; e++) {
    tpc_status st = check_desc(&tfs[e]);
    if (st) return st;
    if (tfs[e].n_time_bins != tfs[0].n_time_bins)
      return fail(TPC_E_INVAL, "every event of a batch needs the same n_time_bins");
  }
  const uint64_t nfrag = (tfs[0].n_time_bins + kFrag - 1) / kFrag;
  if ((uint64_t)ctx->geom.n_sectors * ctx->geom.n_rows * nfrag * n_events > 0xffffffffull)
    return fail(TPC_E_INVAL, "too many windows");
  Pending rq;
  rq.batch = true;
  rq.descs.assign(tfs, tfs + n_events);
  return submit(ctx, std::move(rq), tfs[0].flags & TPC_TF_NOWAIT, ticket);
}

static tpc_status status_from_err(uint32_t e) {
  if (e & kErrCorrupt) return TPC_E_CORRUPT;
  if (e & kErrTimeout) return TPC_E_TIMEOUT;
  if (e & (kErrOverflowCl | kErrOverflowCh | kErrRowCount)) return TPC_E_OVERFLOW;
  return e ? TPC_E_DEVICE : TPC_OK;
}

// Called with the lock held once ev_done has completed.
static tpc_status finish(tpc_context* ctx, Slot& s) {
  const uint32_t e = *(const uint32_t*)(s.h_ctrl + CTR_COUNT);
  if ((e & (kErrOverflowCl | kErrOverflowCh)) && !(e & (kErrCorrupt | kErrTimeout)) && s.runs <= 2) {
    // regrow and run again (input still resident): to 1.25x the cluster count
    // the finder reported (exact even past the capacity) or twice the old
    // capacity, and on a second overflow to the bound no timeframe can exceed
    const uint64_t ncl = s.h_ctrl[CTR_NCL];
    uint64_t cap = s.runs == 1 ? std::max<uint64_t>(2 * s.cap_cl, ncl + ncl / 4 + 1024) : ~0ull;
    cap = std::min(cap, guaranteed_cap_cl(s.pages_bytes));
    tpc_status st = slot_reserve(ctx, s, s.pages_bytes, s.n_windows, cap, !(s.tf_flags & TPC_TF_DEVICE_INPUT));
    if (st == TPC_E_NOMEM) {
      reclaim_idle(ctx, &s);
      st = slot_reserve(ctx, s, s.pages_bytes, s.n_windows, cap, !(s.tf_flags & TPC_TF_DEVICE_INPUT));
    }
    if (st) { s.state = TPC_STATE_FAILED; s.status = st; return st; }
    st = enqueue(ctx, s);
    if (st) { s.state = TPC_STATE_FAILED; s.status = st; return st; }
    return TPC_E_NOTREADY;   // still running
  }
  tpc_status st = status_from_err(e);
  if (st) {
    s.state = TPC_STATE_FAILED;
    s.status = st;
    char buf[96];
    std::snprintf(buf, sizeof buf, "timeframe failed on the device (error word 0x%x)", e);
    return fail(st, buf);
  }
  s.state = TPC_STATE_DONE;
  return TPC_OK;
}

extern "C" tpc_status tpc_poll(tpc_context* ctx, uint64_t ticket, uint32_t timeout_us, int32_t* state) {
  if (!ctx || !state) return fail(TPC_E_INVAL, "tpc_poll: null argument");
  auto t0 = std::chrono::steady_clock::now();
  while (true) {
    {
      std::lock_guard<std::mutex> lk(ctx->mu);
      Slot* s = find_ticket(ctx, ticket);
      if (!s) {
        cudaSetDevice(ctx->device);
        admit(ctx);
        s = find_ticket(ctx, ticket);
      }
      if (!s) {
        for (auto& f : ctx->failed)
          if (f.first == ticket) {
            *state = TPC_STATE_FAILED;
            return fail(f.second, "queued timeframe could not start");
          }
        bool queued = false;
        for (auto& rq : ctx->pending) queued |= rq.ticket == ticket;
        if (!queued) return fail(TPC_E_NOTFOUND, "unknown ticket");
        *state = TPC_STATE_QUEUED;
      } else if (s->state == TPC_STATE_DONE || s->state == TPC_STATE_FAILED) {
        *state = s->state;
        return s->status ? fail(s->status, "timeframe failed") : TPC_OK;
      } else {
        cudaSetDevice(ctx->device);
        cudaError_t q = cudaEventQuery(s->ev_done);
        if (q == cudaSuccess) {
          tpc_status st = finish(ctx, *s);
          if (st != TPC_E_NOTREADY) {
            *state = s->state;
            return st;
          }
        } else if (q != cudaErrorNotReady) {
          s->state = TPC_STATE_FAILED;
          s->status = TPC_E_CUDA;
          *state = s->state;
          return fail(TPC_E_CUDA, std::string("device error: ") + cudaGetErrorString(q));
        } else if (s->state == TPC_STATE_RUNNING && !(s->tf_flags & TPC_TF_DEVICE_INPUT) &&
                   cudaEventQuery(s->ev_input) == cudaSuccess) {
          // host input has been copied into the slot; device input is read in
          // place by every run (an overflow re-runs from it) until DONE
          s->state = TPC_STATE_INPUT_RELEASED;
        }
        *state = s->state;
      }
    }
    if (timeout_us == 0) return TPC_OK;
    auto el = std::chrono::duration_cast<std::chrono::microseconds>(std::chrono::steady_clock::now() - t0).count();
    if (timeout_us != UINT32_MAX && (uint64_t)el >= timeout_us) return fail(TPC_E_TIMEOUT, "tpc_poll timed out");
    std::this_thread::sleep_for(std::chrono::microseconds(el < 2000 ? 5 : 50));
  }
}

static tpc_status done_slot(tpc_context* ctx, uint64_t ticket, Slot** out) {
  Slot* s = find_ticket(ctx, ticket);
  if (!s) return fail(TPC_E_NOTFOUND, "unknown ticket");
  if (s->state == TPC_STATE_FAILED) return fail(s->status, "timeframe failed");
  if (s->state != TPC_STATE_DONE) return fail(TPC_E_NOTREADY, "timeframe not finished (poll it first)");
  *out = s;
  return TPC_OK;
}

static uint64_t ctr(const Slot& s, int i) { return s.h_ctrl[i]; }
static uint64_t n_cl_of(const Slot& s) { return std::min<uint64_t>(ctr(s, CTR_NCL), s.cap_cl); }
static uint64_t n_trk_of(const Slot& s) { return std::min<uint64_t>(ctr(s, CTR_NTRK), s.cap_ch); }

extern "C" tpc_status tpc_get_clusters(tpc_context* ctx, uint64_t ticket, tpc_cluster* out, uint64_t cap,
                                       uint64_t* n) {
  if (!ctx || !n) return fail(TPC_E_INVAL, "tpc_get_clusters: null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  *n = n_cl_of(*s);
  if (!out) return TPC_OK;
  if (cap < *n) return fail(TPC_E_OVERFLOW, "output buffer too small");
  CUDA_TRY(cudaSetDevice(ctx->device));
  if (*n) CUDA_TRY(cudaMemcpyAsync(out, s->W.clusters, *n * sizeof(tpc_cluster), cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return TPC_OK;
}

extern "C" tpc_status tpc_get_tracks(tpc_context* ctx, uint64_t ticket, tpc_track* out, uint64_t cap, uint64_t* n,
                                     int32_t* cluster_to_track) {
  if (!ctx || !n) return fail(TPC_E_INVAL, "tpc_get_tracks: null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  *n = n_trk_of(*s);
  if (!out && !cluster_to_track) return TPC_OK;
  if (out && cap < *n) return fail(TPC_E_OVERFLOW, "output buffer too small");
  CUDA_TRY(cudaSetDevice(ctx->device));
  if (out && *n) CUDA_TRY(cudaMemcpyAsync(out, s->W.tracks, *n * sizeof(tpc_track), cudaMemcpyDeviceToHost, s->stream));
  const uint64_t ncl = n_cl_of(*s);
  if (cluster_to_track && ncl)
    CUDA_TRY(cudaMemcpyAsync(cluster_to_track, s->W.cl2trk, ncl * 4, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return TPC_OK;
}

extern "C" tpc_status tpc_get_batch_info(tpc_context* ctx, uint64_t ticket, uint32_t* n_events,
                                         uint64_t* cluster_start, uint64_t* track_start) {
  if (!ctx || !n_events) return fail(TPC_E_INVAL, "tpc_get_batch_info: null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  *n_events = s->n_events;
  const uint32_t* h = (const uint32_t*)(s->h_ev + 2 * kMaxBatch);
  for (uint32_t e = 0; e <= s->n_events; e++) {
    const bool one = s->n_events == 1;
    if (cluster_start) cluster_start[e] = one ? (e ? n_cl_of(*s) : 0) : h[e];
    if (track_start) track_start[e] = one ? (e ? n_trk_of(*s) : 0) : h[kMaxBatch + 1 + e];
  }
  return TPC_OK;
}

static tpc_status event_range(const Slot& s, uint32_t event, uint64_t* c0, uint64_t* c1, uint64_t* t0,
                              uint64_t* t1) {
  if (event >= s.n_events) return fail(TPC_E_INVAL, "event index out of range");
  if (s.n_events == 1) {
    *c0 = 0; *c1 = n_cl_of(s); *t0 = 0; *t1 = n_trk_of(s);
    return TPC_OK;
  }
  const uint32_t* h = (const uint32_t*)(s.h_ev + 2 * kMaxBatch);
  *c0 = h[event]; *c1 = h[event + 1];
  *t0 = h[kMaxBatch + 1 + event]; *t1 = h[kMaxBatch + 2 + event];
  return TPC_OK;
}

extern "C" tpc_status tpc_get_event_clusters(tpc_context* ctx, uint64_t ticket, uint32_t event, tpc_cluster* out,
                                             uint64_t cap, uint64_t* n) {
  if (!ctx || !n) return fail(TPC_E_INVAL, "tpc_get_event_clusters: null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  uint64_t c0, c1, t0, t1;
  if ((st = event_range(*s, event, &c0, &c1, &t0, &t1))) return st;
  *n = c1 - c0;
  if (!out) return TPC_OK;
  if (cap < *n) return fail(TPC_E_OVERFLOW, "output buffer too small");
  CUDA_TRY(cudaSetDevice(ctx->device));
  if (*n)
    CUDA_TRY(cudaMemcpyAsync(out, s->W.clusters + c0, *n * sizeof(tpc_cluster), cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return TPC_OK;
}

extern "C" tpc_status tpc_get_event_tracks(tpc_context* ctx, uint64_t ticket, uint32_t event, tpc_track* out,
                                           uint64_t cap, uint64_t* n, int32_t* cluster_to_track) {
  if (!ctx || !n) return fail(TPC_E_INVAL, "tpc_get_event_tracks: null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  uint64_t c0, c1, t0, t1;
  if ((st = event_range(*s, event, &c0, &c1, &t0, &t1))) return st;
  *n = t1 - t0;
  if (!out && !cluster_to_track) return TPC_OK;
  if (out && cap < *n) return fail(TPC_E_OVERFLOW, "output buffer too small");
  CUDA_TRY(cudaSetDevice(ctx->device));
  if (out && *n)
    CUDA_TRY(cudaMemcpyAsync(out, s->W.tracks + t0, *n * sizeof(tpc_track), cudaMemcpyDeviceToHost, s->stream));
  if (cluster_to_track && c1 > c0)
    CUDA_TRY(cudaMemcpyAsync(cluster_to_track, s->W.cl2trk + c0, (c1 - c0) * 4, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  // indices relative to the event, as a run of the event alone gives them
  if (out)
    for (uint64_t i = 0; i < *n; i++) out[i].first_cluster -= (int32_t)c0;
  if (cluster_to_track)
    for (uint64_t i = 0; i < c1 - c0; i++)
      if (cluster_to_track[i] >= 0) cluster_to_track[i] -= (int32_t)t0;
  return TPC_OK;
}

// ------------------------------------------------------------------ step 9
extern "C" tpc_status tpc_merge_sectors(tpc_context* ctx, uint64_t ticket, const tpc_xs_params* xp,
                                        uint64_t* n_tracks) {
  if (!ctx) return fail(TPC_E_INVAL, "tpc_merge_sectors: null argument");
  const double chi2_cut = xp ? xp->chi2_cut : 100.0, edge_cm = xp ? xp->edge_cm : 6.0;
  const double dz_cm = xp ? xp->dz_cm : 250.0;
  if (!(chi2_cut >= 0.0) || !(edge_cm >= 0.0) || edge_cm > 100.0 || !(dz_cm > 0.0) || dz_cm > 1e4)
    return fail(TPC_E_INVAL, "tpc_merge_sectors: bad parameters");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  CUDA_TRY(cudaSetDevice(ctx->device));
  const uint64_t C = s->cap_ch, Ncl = s->cap_cl;
  const size_t tiles = scan_tiles(C);
  // zeta bins of the candidate search: Z = 5 (32768 f + time_fp - 512) spans
  // [-2560, zmax]; bins at least dz wide, at most ~4M bins over all virtual sectors
  const int n_vs = ctx->geom.n_sectors * (int)s->n_events;
  const long long n_frag = (long long)((s->n_time_bins + kFrag - 1) / kFrag);
  const long long zrange = 5 * (32768 * (n_frag - 1) + 65535 - 512) + 2560 + 1;
  const long long dz_u = (long long)std::floor(dz_cm / 7.8125e-4 + 0.5);
  const long long bin_w = std::max({dz_u, 1ll, (zrange * n_vs + (1ll << 22) - 1) >> 22});
  const long long n_zb = zrange / bin_w + 1;
  const uint64_t n_bins = (uint64_t)n_vs * (uint64_t)n_zb;
  const size_t btiles = scan_tiles(n_bins + 1);
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t need = al(C) + 2 * al(C * 4) + 2 * al(C * 8) + 3 * al(C * 4) + al(C * 8) + al(tiles * 8) + al(64) +
                      al(C * sizeof(tpc_track)) + al(Ncl * 4) + 2 * al(C * 4) + al(C * 16) + al(C * 96) +
                      al((n_bins + 1) * 8) +
                      al(n_bins * 4) + al(btiles * 8);
  if (need > s->xs.bytes) {
    if (ctx->used - s->xs_bytes + need > ctx->budget) return fail(TPC_E_NOMEM, "tpc_merge_sectors: over the memory budget");
    CUDA_TRY(ensure(s->xs, need));
    ctx->used = ctx->used - s->xs_bytes + need;
    s->xs_bytes = need;
  }
  uint8_t* p = (uint8_t*)s->xs.p;
  XsWork X;
  auto take = [&](size_t b) { uint8_t* q = p; p += al(b); return q; };
  X.side = take(C);
  X.row_in = (int32_t*)take(C * 4);
  X.row_out = (int32_t*)take(C * 4);
  X.best_b = (unsigned long long*)take(C * 8);
  X.best_a = (unsigned long long*)take(C * 8);
  X.link = (int32_t*)take(C * 4);
  X.prev = (int32_t*)take(C * 4);
  X.group = (int32_t*)take(C * 4);
  X.scan = (uint64_t*)take(C * 8);
  X.scan_state = (unsigned long long*)take(tiles * 8);
  X.ctl = (unsigned long long*)take(64);
  X.tracks_out = (tpc_track*)take(C * sizeof(tpc_track));
  X.cl2trk_out = (int32_t*)take(Ncl * 4);
  X.z_in = (int32_t*)take(C * 4);
  X.z_out = (int32_t*)take(C * 4);
  X.ent = (uint4*)take(C * 16);
  X.ent_fit = (uint4*)take(C * 96);
  X.bin_off = (uint64_t*)take((n_bins + 1) * 8);
  X.bin_cur = (uint32_t*)take(n_bins * 4);
  X.bin_state = (unsigned long long*)take(btiles * 8);
  X.chi2_cut = (float)chi2_cut;
  X.edge_u = (int)std::floor(edge_cm / 7.8125e-4 + 0.5);
  X.dz_u = (int)dz_u;
  X.bin_w = (int)bin_w;
  X.n_zb = (int)n_zb;
  DevGeom G = ctx->G;
  G.n_time_bins = (int)s->n_time_bins;
  G.n_frag = (int)((s->n_time_bins + kFrag - 1) / kFrag);
  G.n_events = (int)s->n_events;
  G.n_sectors = ctx->geom.n_sectors * (int)s->n_events;
  CUDA_TRY(cudaMemsetAsync(X.scan_state, 0, tiles * 8, s->stream));
  CUDA_TRY(cudaMemsetAsync(X.bin_state, 0, btiles * 8, s->stream));
  CUDA_TRY(cudaMemsetAsync(X.bin_off, 0, (n_bins + 1) * 8, s->stream));
  CUDA_TRY(cudaMemsetAsync(X.bin_cur, 0, n_bins * 4, s->stream));
  {
    // ctl: [0] merged tracks, [1] links, [2] scan ticket, [3] bins + 1, [4] bin scan ticket, [5] bin total
    unsigned long long c[8] = {0, 0, 0, n_bins + 1, 0, 0, 0, 0};
    CUDA_TRY(cudaMemcpyAsync(X.ctl, c, sizeof c, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));   // c lives on this stack frame
  }
  CUDA_TRY(launch_xsec(G, ctx->P, s->W, X, ctx->n_sm, s->stream));
  unsigned long long ctl[2];
  CUDA_TRY(cudaMemcpyAsync(ctl, X.ctl, 16, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->xs_done = true;
  s->xs_n = ctl[0];
  s->xs_links = ctl[1];
  if (n_tracks) *n_tracks = s->xs_n;
  return TPC_OK;
}

extern "C" tpc_status tpc_get_merged_tracks(tpc_context* ctx, uint64_t ticket, tpc_track* out, uint64_t cap,
                                            uint64_t* n, int32_t* cluster_to_track, int32_t* link) {
  if (!ctx || !n) return fail(TPC_E_INVAL, "tpc_get_merged_tracks: null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  if (!s->xs_done) return fail(TPC_E_NOTREADY, "tpc_merge_sectors has not run on this ticket");
  *n = s->xs_n;
  if (!out && !cluster_to_track && !link) return TPC_OK;
  if (out && cap < *n) return fail(TPC_E_OVERFLOW, "output buffer too small");
  CUDA_TRY(cudaSetDevice(ctx->device));
  const uint64_t C = s->cap_ch;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const uint8_t* base = (const uint8_t*)s->xs.p;
  const size_t o_link = al(C) + 2 * al(C * 4) + 2 * al(C * 8);
  const size_t o_tracks = o_link + 3 * al(C * 4) + al(C * 8) + al(scan_tiles(C) * 8) + al(64);
  const size_t o_map = o_tracks + al(C * sizeof(tpc_track));
  const uint64_t ncl = n_cl_of(*s), ntr = n_trk_of(*s);
  if (out && *n) CUDA_TRY(cudaMemcpyAsync(out, base + o_tracks, *n * sizeof(tpc_track), cudaMemcpyDeviceToHost, s->stream));
  if (cluster_to_track && ncl)
    CUDA_TRY(cudaMemcpyAsync(cluster_to_track, base + o_map, ncl * 4, cudaMemcpyDeviceToHost, s->stream));
  if (link && ntr) CUDA_TRY(cudaMemcpyAsync(link, base + o_link, ntr * 4, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return TPC_OK;
}

// ------------------------------------------------------------------ step 9b
extern "C" tpc_status tpc_join_loopers(tpc_context* ctx, uint64_t ticket, const tpc_loop_params* lp,
                                       uint64_t* n_links) {
  if (!ctx) return fail(TPC_E_INVAL, "tpc_join_loopers: null argument");
  const double chi2_cut = lp ? lp->chi2_cut : 30.0, radius = lp ? lp->loop_radius_cm : 275.0;
  const int max_turns = lp ? lp->max_turns : 4;
  if (!(chi2_cut >= 0.0) || chi2_cut > 1e6 || !(radius > 0.0) || radius > 1e4 || max_turns < 1 || max_turns > 15)
    return fail(TPC_E_INVAL, "tpc_join_loopers: bad parameters");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  CUDA_TRY(cudaSetDevice(ctx->device));
  const uint64_t C = s->cap_ch;
  if (C >= (1ull << 28)) return fail(TPC_E_INVAL, "tpc_join_loopers: more than 2^28 tracks");
  const int n_vs = ctx->geom.n_sectors * (int)s->n_events;
  const size_t btiles = scan_tiles((uint64_t)n_vs + 1);
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t need = al(C) + al(((size_t)n_vs + 1) * 8) + al((size_t)n_vs * 4) + al(btiles * 8) + al(C * 4) +
                      al(C * 96) + 2 * al(C * 8) + 2 * al(C * 4) + al(64);
  if (need > s->lp.bytes) {
    if (ctx->used - s->lp_bytes + need > ctx->budget) return fail(TPC_E_NOMEM, "tpc_join_loopers: over the memory budget");
    CUDA_TRY(ensure(s->lp, need));
    ctx->used = ctx->used - s->lp_bytes + need;
    s->lp_bytes = need;
  }
  uint8_t* p = (uint8_t*)s->lp.p;
  auto take = [&](size_t b) { uint8_t* q = p; p += al(b); return q; };
  LoopWork L;
  L.loops = take(C);
  L.bin_off = (uint64_t*)take(((size_t)n_vs + 1) * 8);
  L.bin_cur = (uint32_t*)take((size_t)n_vs * 4);
  L.bin_state = (unsigned long long*)take(btiles * 8);
  L.ent = (uint32_t*)take(C * 4);
  L.ent_fit = (uint4*)take(C * 96);
  L.next_key = (unsigned long long*)take(C * 8);
  L.prev_key = (unsigned long long*)take(C * 8);
  L.next = (int32_t*)take(C * 4);
  L.prev = (int32_t*)take(C * 4);
  L.ctl = (unsigned long long*)take(64);
  L.chi2_cut = (float)chi2_cut;
  L.loop_radius = (float)radius;
  L.max_turns = max_turns;
  L.n_vs = n_vs;
  DevGeom G = ctx->G;
  G.n_time_bins = (int)s->n_time_bins;
  G.n_frag = (int)((s->n_time_bins + kFrag - 1) / kFrag);
  G.n_events = (int)s->n_events;
  G.n_sectors = n_vs;
  CUDA_TRY(cudaMemsetAsync(L.bin_off, 0, ((size_t)n_vs + 1) * 8, s->stream));
  CUDA_TRY(cudaMemsetAsync(L.bin_cur, 0, (size_t)n_vs * 4, s->stream));
  CUDA_TRY(cudaMemsetAsync(L.bin_state, 0, btiles * 8, s->stream));
  {
    // ctl: [0] links, [1] n_vs + 1 (entries of the scan), [2] scan ticket, [3] looping tracks
    unsigned long long c[8] = {0, (unsigned long long)n_vs + 1, 0, 0, 0, 0, 0, 0};
    CUDA_TRY(cudaMemcpyAsync(L.ctl, c, sizeof c, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));   // c lives on this stack frame
  }
  CUDA_TRY(launch_loopers(G, ctx->P, s->W, L, ctx->n_sm, s->stream));
  unsigned long long ctl[4];
  CUDA_TRY(cudaMemcpyAsync(ctl, L.ctl, 32, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->lp_done = true;
  s->lp_links = ctl[0];
  s->lp_tracks = ctl[3];
  if (n_links) *n_links = s->lp_links;
  return TPC_OK;
}

extern "C" tpc_status tpc_get_looper_links(tpc_context* ctx, uint64_t ticket, int32_t* next, int32_t* prev,
                                           uint64_t* n_tracks) {
  if (!ctx) return fail(TPC_E_INVAL, "tpc_get_looper_links: null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  if (!s->lp_done) return fail(TPC_E_NOTREADY, "tpc_join_loopers has not run on this ticket");
  const uint64_t ntr = n_trk_of(*s);
  if (n_tracks) *n_tracks = ntr;
  if ((!next && !prev) || !ntr) return TPC_OK;
  CUDA_TRY(cudaSetDevice(ctx->device));
  const uint64_t C = s->cap_ch;
  const int n_vs = ctx->geom.n_sectors * (int)s->n_events;
  auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
  const size_t o_next = al(C) + al(((size_t)n_vs + 1) * 8) + al((size_t)n_vs * 4) +
                        al(scan_tiles((uint64_t)n_vs + 1) * 8) + al(C * 4) + al(C * 96) + 2 * al(C * 8);
  const size_t o_prev = o_next + al(C * 4);
  const uint8_t* base = (const uint8_t*)s->lp.p;
  if (next) CUDA_TRY(cudaMemcpyAsync(next, base + o_next, ntr * 4, cudaMemcpyDeviceToHost, s->stream));
  if (prev) CUDA_TRY(cudaMemcpyAsync(prev, base + o_prev, ntr * 4, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return TPC_OK;
}

// ------------------------------------------------------------------ step 10
// The step-10 buffer: codes and status (3 bytes per cluster), counters, then
// step 10c's work: tables, bits per cluster, scan state, the stream (at most
// 48 bits per cluster).
static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }
static uint64_t ent_cap_words(uint64_t cap_cl) { return cap_cl * 3 / 2 + 4; }
static size_t cmp_need(uint64_t cap_cl) {
  const size_t n = al256(cap_cl);
  return 3 * n + 256 + 8192 + al256(8 * cap_cl) + al256(8 * scan_tiles(cap_cl)) + 256 + al256(4 * ent_cap_words(cap_cl));
}
static CmpWork cmp_work(Slot& s, EntWork* E = nullptr) {
  CmpWork C;
  uint8_t* p = (uint8_t*)s.cmp.p;
  const size_t n = al256(s.cap_cl);
  C.code_y = (int8_t*)p;
  C.code_z = (int8_t*)(p + n);
  C.status = p + 2 * n;
  C.ctl = (unsigned long long*)(p + 3 * n);
  if (E) {
    uint8_t* q = p + 3 * n + 256;
    E->hist = (unsigned long long*)q;
    E->len = q + 4096;
    E->code = (uint32_t*)(q + 4096 + 1024);
    q += 8192;
    E->bits = (uint64_t*)q;
    q += al256(8 * s.cap_cl);
    E->scan_state = (unsigned long long*)q;
    q += al256(8 * scan_tiles(s.cap_cl));
    E->ticket = (unsigned int*)q;
    E->total = (unsigned long long*)(q + 16);
    q += 256;
    E->words = (uint32_t*)q;
    E->cap_words = ent_cap_words(s.cap_cl);
  }
  return C;
}

extern "C" tpc_status tpc_compress_clusters(tpc_context* ctx, uint64_t ticket, const tpc_cmp_params* cp,
                                            uint64_t* n_coded, uint64_t* n_escaped) {
  if (!ctx) return fail(TPC_E_INVAL, "tpc_compress_clusters: null argument");
  const double sy = cp ? cp->step_y_cm : 0.4 / 32, sz = cp ? cp->step_z_cm : 0.5 / 32;
  if (!(sy > 0.0) || !(sz > 0.0)) return fail(TPC_E_INVAL, "tpc_compress_clusters: steps must be positive");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  CUDA_TRY(cudaSetDevice(ctx->device));
  const size_t need = cmp_need(s->cap_cl);
  if (need > s->cmp.bytes) {
    if (ctx->used - s->cmp_bytes + need > ctx->budget) return fail(TPC_E_NOMEM, "tpc_compress_clusters: over the memory budget");
    CUDA_TRY(ensure(s->cmp, need));
    ctx->used = ctx->used - s->cmp_bytes + need;
    s->cmp_bytes = need;
  }
  CmpWork C = cmp_work(*s);
  C.step_y = (float)sy;
  C.step_z = (float)sz;
  const uint64_t ncl = n_cl_of(*s);
  CUDA_TRY(cudaMemsetAsync(C.status, 0, ncl ? ncl : 1, s->stream));
  CUDA_TRY(cudaMemsetAsync(C.ctl, 0, 16, s->stream));
  CUDA_TRY(launch_compress(ctx->P, s->W, C, ctx->n_sm, s->stream));
  unsigned long long ctl[2];
  CUDA_TRY(cudaMemcpyAsync(ctl, C.ctl, 16, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  s->cmp_done = true;
  if (n_coded) *n_coded = ctl[0];
  if (n_escaped) *n_escaped = ctl[1];
  return TPC_OK;
}

extern "C" tpc_status tpc_get_compressed(tpc_context* ctx, uint64_t ticket, int8_t* code_y, int8_t* code_z,
                                         uint8_t* status) {
  if (!ctx) return fail(TPC_E_INVAL, "tpc_get_compressed: null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  if (!s->cmp_done) return fail(TPC_E_NOTREADY, "tpc_compress_clusters has not run on this ticket");
  CUDA_TRY(cudaSetDevice(ctx->device));
  const CmpWork C = cmp_work(*s);
  const uint64_t ncl = n_cl_of(*s);
  if (ncl) {
    if (code_y) CUDA_TRY(cudaMemcpyAsync(code_y, C.code_y, ncl, cudaMemcpyDeviceToHost, s->stream));
    if (code_z) CUDA_TRY(cudaMemcpyAsync(code_z, C.code_z, ncl, cudaMemcpyDeviceToHost, s->stream));
    if (status) CUDA_TRY(cudaMemcpyAsync(status, C.status, ncl, cudaMemcpyDeviceToHost, s->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return TPC_OK;
}

extern "C" tpc_status tpc_entropy_encode(tpc_context* ctx, uint64_t ticket, const int8_t* code_y,
                                         const int8_t* code_z, const uint8_t* status, uint8_t* lengths,
                                         uint64_t* n_bits, uint32_t* words, uint64_t cap_words) {
  if (!ctx) return fail(TPC_E_INVAL, "tpc_entropy_encode: null argument");
  const bool given = code_y || code_z || status;
  if (given && !(code_y && code_z && status))
    return fail(TPC_E_INVAL, "tpc_entropy_encode: give code_y, code_z and status together, or none");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  if (!given && !s->cmp_done) return fail(TPC_E_NOTREADY, "tpc_compress_clusters has not run on this ticket");
  CUDA_TRY(cudaSetDevice(ctx->device));
  const size_t need = cmp_need(s->cap_cl);
  if (need > s->cmp.bytes) {
    if (ctx->used - s->cmp_bytes + need > ctx->budget) return fail(TPC_E_NOMEM, "tpc_entropy_encode: over the memory budget");
    CUDA_TRY(ensure(s->cmp, need));
    ctx->used = ctx->used - s->cmp_bytes + need;
    s->cmp_bytes = need;
  }
  EntWork E;
  CmpWork C = cmp_work(*s, &E);
  const uint64_t ncl = n_cl_of(*s);
  if (given && ncl) {
    CUDA_TRY(cudaMemcpyAsync(C.code_y, code_y, ncl, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemcpyAsync(C.code_z, code_z, ncl, cudaMemcpyHostToDevice, s->stream));
    CUDA_TRY(cudaMemcpyAsync(C.status, status, ncl, cudaMemcpyHostToDevice, s->stream));
  }
  CUDA_TRY(cudaMemsetAsync(E.hist, 0, 4096, s->stream));
  CUDA_TRY(cudaMemsetAsync(E.scan_state, 0, 8 * scan_tiles(s->cap_cl), s->stream));
  CUDA_TRY(cudaMemsetAsync(E.ticket, 0, 256, s->stream));
  CUDA_TRY(cudaMemsetAsync(E.words, 0, 4 * E.cap_words, s->stream));
  CUDA_TRY(launch_entropy(s->W, C, E, ctx->n_sm, s->stream));
  unsigned long long total = 0;
  CUDA_TRY(cudaMemcpyAsync(&total, E.total, 8, cudaMemcpyDeviceToHost, s->stream));
  if (lengths) CUDA_TRY(cudaMemcpyAsync(lengths, E.len, 512, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  if (given) s->cmp_done = true;
  if (n_bits) *n_bits = total;
  const uint64_t nw = (total + 31) / 32;
  if (words) {
    if (nw > cap_words) return fail(TPC_E_INVAL, "tpc_entropy_encode: words holds fewer than (n_bits + 31) / 32 words");
    if (nw) CUDA_TRY(cudaMemcpyAsync(words, E.words, 4 * nw, cudaMemcpyDeviceToHost, s->stream));
    CUDA_TRY(cudaStreamSynchronize(s->stream));
  }
  return TPC_OK;
}

// ------------------------------------------------------------------ step 11
extern "C" tpc_status tpc_calibrate_drift(tpc_context* ctx, uint64_t ticket, double t0_bins, double drift_length_cm,
                                          double* t_vertex_bins, double* eps_vd, double* t0_from_vertex,
                                          uint64_t* n_used) {
  if (!ctx) return fail(TPC_E_INVAL, "tpc_calibrate_drift: null argument");
  if (!(drift_length_cm > 0.0)) return fail(TPC_E_INVAL, "tpc_calibrate_drift: drift length must be positive");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  CUDA_TRY(cudaSetDevice(ctx->device));
  const size_t nb = (size_t)1 << 20;
  const size_t need = ((s->cap_ch * 4 + 255) & ~(size_t)255) + nb * 4 + 256;
  if (need > s->cal.bytes) {
    if (ctx->used - s->cal_bytes + need > ctx->budget) return fail(TPC_E_NOMEM, "tpc_calibrate_drift: over the memory budget");
    CUDA_TRY(ensure(s->cal, need));
    ctx->used = ctx->used - s->cal_bytes + need;
    s->cal_bytes = need;
  }
  uint8_t* p = (uint8_t*)s->cal.p;
  CalWork C;
  C.tv = (float*)p;
  p += (s->cap_ch * 4 + 255) & ~(size_t)255;
  C.hist = (unsigned*)p;
  p += nb * 4;
  C.mode = (unsigned long long*)p;
  C.sum = (double*)(p + 8);
  C.cnt = (unsigned long long*)(p + 24);
  C.zeta_per_bin = 0.5f;
  CUDA_TRY(cudaMemsetAsync(C.hist, 0, nb * 4 + 64, s->stream));
  CUDA_TRY(launch_calibrate(ctx->P, s->W, C, ctx->n_sm, s->stream));
  unsigned long long h[5];
  CUDA_TRY(cudaMemcpyAsync(h, C.mode, 40, cudaMemcpyDeviceToHost, s->stream));
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  double sums[2];
  std::memcpy(sums, &h[1], 16);
  const uint64_t n = h[4];
  const double tv = n ? sums[1] / (double)n : 0.0, full = drift_length_cm / 0.5;
  if (t_vertex_bins) *t_vertex_bins = tv;
  if (eps_vd) *eps_vd = (n && tv != t0_bins) ? full / (tv - t0_bins) - 1.0 : 0.0;
  if (t0_from_vertex) *t0_from_vertex = n ? tv - full : 0.0;
  if (n_used) *n_used = n;
  return TPC_OK;
}

extern "C" tpc_status tpc_get_links(tpc_context* ctx, uint64_t ticket, int32_t* up, int32_t* down,
                                    int32_t* chain_of) {
  if (!ctx) return fail(TPC_E_INVAL, "tpc_get_links: null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  const uint64_t ncl = n_cl_of(*s);
  CUDA_TRY(cudaSetDevice(ctx->device));
  if (ncl) {
    if (up) CUDA_TRY(cudaMemcpyAsync(up, s->W.up, ncl * 4, cudaMemcpyDeviceToHost, s->stream));
    if (down) CUDA_TRY(cudaMemcpyAsync(down, s->W.down, ncl * 4, cudaMemcpyDeviceToHost, s->stream));
    if (chain_of) CUDA_TRY(cudaMemcpyAsync(chain_of, s->W.chain_of, ncl * 4, cudaMemcpyDeviceToHost, s->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(s->stream));
  return TPC_OK;
}

extern "C" tpc_status tpc_get_device_results(tpc_context* ctx, uint64_t ticket, const tpc_cluster** clusters,
                                             uint64_t* n_clusters, const tpc_track** tracks, uint64_t* n_tracks,
                                             const int32_t** cluster_to_track) {
  if (!ctx) return fail(TPC_E_INVAL, "tpc_get_device_results: null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  if (clusters) *clusters = s->W.clusters;
  if (n_clusters) *n_clusters = n_cl_of(*s);
  if (tracks) *tracks = s->W.tracks;
  if (n_tracks) *n_tracks = n_trk_of(*s);
  if (cluster_to_track) *cluster_to_track = s->W.cl2trk;
  return TPC_OK;
}

extern "C" tpc_status tpc_get_stage_times(tpc_context* ctx, uint64_t ticket, float* ms) {
  if (!ctx || !ms) return fail(TPC_E_INVAL, "tpc_get_stage_times: null argument");
  if (!(ctx->flags & TPC_CTX_STAGE_TIMING)) return fail(TPC_E_INVAL, "context created without TPC_CTX_STAGE_TIMING");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s;
  tpc_status st = done_slot(ctx, ticket, &s);
  if (st) return st;
  CUDA_TRY(cudaSetDevice(ctx->device));
  for (int i = 0; i < TPC_N_STAGES; i++) CUDA_TRY(cudaEventElapsedTime(&ms[i], s->ev_stage[i], s->ev_stage[i + 1]));
  return TPC_OK;
}

extern "C" tpc_status tpc_get_counters(tpc_context* ctx, uint64_t ticket, uint64_t* out, int n) {
  if (!ctx || !out || n < 0 || n > 10) return fail(TPC_E_INVAL, "tpc_get_counters: bad argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  Slot* s = find_ticket(ctx, ticket);
  if (!s) return fail(TPC_E_NOTFOUND, "unknown ticket");
  if (s->state != TPC_STATE_DONE && s->state != TPC_STATE_FAILED)
    return fail(TPC_E_NOTREADY, "timeframe not finished (poll it first)");
  uint64_t passes = 0;
  for (int p = 0; p < 16; p++) passes += ctr(*s, CTR_MERGED0 + p) ? 1 : 0;
  uint64_t v[10] = {ctr(*s, CTR_NCL),
                    ctr(*s, CTR_NCH),
                    ctr(*s, CTR_NTRK),
                    ctr(*s, CTR_NCLCL) & 0xffffffffull,
                    ctr(*s, CTR_NFP64),
                    passes,
                    (uint64_t) * (const uint32_t*)(s->h_ctrl + CTR_COUNT),
                    s->pages_bytes,
                    (uint64_t)s->launches,
                    (uint64_t)s->runs};
  for (int i = 0; i < n; i++) out[i] = v[i];
  return TPC_OK;
}

extern "C" tpc_status tpc_release(tpc_context* ctx, uint64_t ticket) {
  if (!ctx) return fail(TPC_E_INVAL, "tpc_release: null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  cudaSetDevice(ctx->device);
  Slot* s = find_ticket(ctx, ticket);
  if (!s) {
    // a queued request is cancelled, a failed one forgotten
    for (auto it = ctx->pending.begin(); it != ctx->pending.end(); ++it)
      if (it->ticket == ticket) { ctx->pending.erase(it); admit(ctx); return TPC_OK; }
    for (auto it = ctx->failed.begin(); it != ctx->failed.end(); ++it)
      if (it->first == ticket) { ctx->failed.erase(it); return TPC_OK; }
    return fail(TPC_E_NOTFOUND, "unknown ticket");
  }
  cudaStreamSynchronize(s->stream);
  s->in_use = false;
  s->state = TPC_STATE_QUEUED;
  admit(ctx);   // the freed slot and memory go to the oldest queued request
  return TPC_OK;
}

// ------------------------------------------------------------------ tuning
// Finder launch shapes (threads per CTA x CTAs per SM): the two-pass finder's
// small-plane CTAs, or the fused / dense-plane finder's whole-window ones.
static const int kFind2ThreadsC[] = {128, 256};
static const int kFind2CtasC[] = {4, 8};
static const int kFindThreadsC[] = {256, 384, 512};
static const int kFindCtasC[] = {1, 2};
static const int kPerSmC[] = {4, 8, 16};
static const int kFitThreadsC[] = {32, 64, 128};
static const int kFitBlocksC[] = {16, 32, 64};

template <size_t N>
static bool one_of(int v, const int (&set)[N]) {
  for (int x : set)
    if (x == v) return true;
  return false;
}

static void to_public(const LaunchCfg& L, tpc_tuning* t) {
  t->find_threads = L.find_threads;
  t->find_ctas_per_sm = L.find_ctas_per_sm;
  t->ca_blocks_per_sm = L.ca_blocks_per_sm;
  t->elem_blocks_per_sm = L.elem_blocks_per_sm;
  t->fit_threads = L.fit_threads;
  t->fit_blocks_per_sm = L.fit_blocks_per_sm;
}

extern "C" tpc_status tpc_get_tuning(tpc_context* ctx, tpc_tuning* out) {
  if (!ctx || !out) return fail(TPC_E_INVAL, "tpc_get_tuning: null argument");
  std::lock_guard<std::mutex> lk(ctx->mu);
  to_public(ctx->L, out);
  return TPC_OK;
}

extern "C" tpc_status tpc_set_tuning(tpc_context* ctx, const tpc_tuning* t) {
  if (!ctx || !t) return fail(TPC_E_INVAL, "tpc_set_tuning: null argument");
  const bool find_ok = two_pass(ctx) ? one_of(t->find_threads, kFind2ThreadsC) && one_of(t->find_ctas_per_sm, kFind2CtasC)
                                      : one_of(t->find_threads, kFindThreadsC) && one_of(t->find_ctas_per_sm, kFindCtasC);
  if (!find_ok || !one_of(t->ca_blocks_per_sm, kPerSmC) || !one_of(t->elem_blocks_per_sm, kPerSmC) ||
      !one_of(t->fit_threads, kFitThreadsC) || !one_of(t->fit_blocks_per_sm, kFitBlocksC))
    return fail(TPC_E_INVAL, "tpc_set_tuning: a value outside its candidate set");
  std::lock_guard<std::mutex> lk(ctx->mu);
  LaunchCfg L;
  L.find_threads = t->find_threads;
  L.find_ctas_per_sm = t->find_ctas_per_sm;
  L.ca_blocks_per_sm = t->ca_blocks_per_sm;
  L.elem_blocks_per_sm = t->elem_blocks_per_sm;
  L.fit_threads = t->fit_threads;
  L.fit_blocks_per_sm = t->fit_blocks_per_sm;
  ctx->L = L;
  ctx->tune_gen++;
  return TPC_OK;
}

// Run one timeframe synchronously on slot s (lock held, slot free) with the
// current launch configuration; stage times in ms[4].
static tpc_status run_sync(tpc_context* ctx, Slot& s, const tpc_timeframe_desc* tf, float* ms) {
  tpc_status st = start_timeframe(ctx, &s, tf);
  if (st) return st;
  while (true) {
    CUDA_TRY(cudaEventSynchronize(s.ev_done));
    st = finish(ctx, s);
    if (st != TPC_E_NOTREADY) break;   // TPC_E_NOTREADY: regrown and re-enqueued
  }
  s.state = TPC_STATE_QUEUED;
  if (st) return st;
  for (int i = 0; i < TPC_N_STAGES; i++) CUDA_TRY(cudaEventElapsedTime(&ms[i], s.ev_stage[i], s.ev_stage[i + 1]));
  return TPC_OK;
}

extern "C" tpc_status tpc_autotune(tpc_context* ctx, const tpc_timeframe_desc* sample, int reps, tpc_tuning* out) {
  if (!ctx || !sample) return fail(TPC_E_INVAL, "tpc_autotune: null argument");
  if (reps < 1 || reps > 100) return fail(TPC_E_INVAL, "tpc_autotune: reps out of range");
  tpc_status st = check_desc(sample);
  if (st) return st;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (any_in_use(ctx) || !ctx->pending.empty()) return fail(TPC_E_BUSY, "tpc_autotune needs an idle context");
  CUDA_TRY(cudaSetDevice(ctx->device));
  Slot& s = ctx->slots[0];
  const uint32_t flags0 = ctx->flags;
  const LaunchCfg L0 = ctx->L;
  ctx->flags = (flags0 | TPC_CTX_STAGE_TIMING | TPC_CTX_NO_GRAPHS);
  // joint trials: trial i uses finder choice i % n_find, CA/merge choice i % 9
  // and fit choice i % 9; a stage's time depends only on its own kernels' choice
  const bool tp = two_pass(ctx);
  auto find_shape = [tp](int fi, LaunchCfg& L) {
    if (tp) {
      L.find_threads = kFind2ThreadsC[fi % 2];
      L.find_ctas_per_sm = kFind2CtasC[fi / 2];
    } else {
      L.find_threads = kFindThreadsC[fi % 3];
      L.find_ctas_per_sm = kFindCtasC[fi / 3];
    }
  };
  const int n_find = tp ? 4 : 6, n_mid = 9, n_fit = 9, n_trials = 9;
  std::vector<float> t_find(n_find, 1e30f), t_mid(n_mid, 1e30f), t_fit(n_fit, 1e30f);
  float ms[TPC_N_STAGES];
  st = run_sync(ctx, s, sample, ms);   // warm-up, grows the slot to the sample
  for (int i = 0; i < n_trials && st == TPC_OK; i++) {
    const int fi = i % n_find, mi = i % n_mid, ti = i % n_fit;
    LaunchCfg L;
    find_shape(fi, L);
    L.ca_blocks_per_sm = kPerSmC[mi % 3];
    L.elem_blocks_per_sm = kPerSmC[mi / 3];
    L.fit_threads = kFitThreadsC[ti % 3];
    L.fit_blocks_per_sm = kFitBlocksC[ti / 3];
    ctx->L = L;
    std::vector<float> a, b, c;
    for (int r = 0; r < reps && st == TPC_OK; r++) {
      st = run_sync(ctx, s, sample, ms);
      a.push_back(ms[0]);
      b.push_back(ms[1] + ms[2]);
      c.push_back(ms[3]);
    }
    if (st) break;
    auto med = [](std::vector<float>& v) {
      std::sort(v.begin(), v.end());
      return v[v.size() / 2];
    };
    t_find[fi] = std::min(t_find[fi], med(a));
    t_mid[mi] = std::min(t_mid[mi], med(b));
    t_fit[ti] = std::min(t_fit[ti], med(c));
  }
  ctx->flags = flags0;
  if (st) {
    ctx->L = L0;
    return st;
  }
  const int fi = (int)(std::min_element(t_find.begin(), t_find.end()) - t_find.begin());
  const int mi = (int)(std::min_element(t_mid.begin(), t_mid.end()) - t_mid.begin());
  const int ti = (int)(std::min_element(t_fit.begin(), t_fit.end()) - t_fit.begin());
  LaunchCfg L;
  find_shape(fi, L);
  L.ca_blocks_per_sm = kPerSmC[mi % 3];
  L.elem_blocks_per_sm = kPerSmC[mi / 3];
  L.fit_threads = kFitThreadsC[ti % 3];
  L.fit_blocks_per_sm = kFitBlocksC[ti / 3];
  ctx->L = L;
  ctx->tune_gen++;
  if (out) to_public(L, out);
  return TPC_OK;
}

extern "C" const char* tpc_last_error(void) { return g_err.c_str(); }
