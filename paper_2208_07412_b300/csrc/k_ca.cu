// k_ca.cu — cellular-automaton seeding across pad rows (steps 5-6 of the
// library's definition): best (down, up) neighbour pair per cluster by an
// integer straight-line residual, the edge-row rule, mutual links, chains by
// pointer jumping, and the kept-chain table.  Also the generic single-pass scan
// used for every stable compaction of the pipeline.
//
// The paper (section "Hardware and data flow") names full TPC track
// reconstruction on the GPU but not its algorithm; the CA here is this
// library's definition, restated independently by the CPU oracle.
#include "tpc_internal.cuh"

namespace tpc {

__device__ __forceinline__ unsigned long long n_clusters(const DevWork& W) {
  unsigned long long n = W.ctr[CTR_NCL];
  return n < W.cap_cl ? n : W.cap_cl;
}
__device__ __forceinline__ unsigned long long n_chains(const DevWork& W) {
  unsigned long long n = W.ctr[CTR_NCH];
  return n < W.cap_ch ? n : W.cap_ch;
}

// first index in [lo, hi) with t[i] >= v (t ascending within a row)
__device__ __forceinline__ unsigned lower_bound_t(const int32_t* __restrict__ t, unsigned lo, unsigned hi, int v) {
  while (lo < hi) {
    unsigned mid = (lo + hi) >> 1;
    if (__ldg(t + mid) < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ long long llabs_(long long v) { return v < 0 ? -v : v; }

// ---------------------------------------------------------------- neighbours
__global__ void k_ca_neighbours(DevGeom G, DevParams P, DevWork W) {
  const unsigned long long n = n_clusters(W);
  const int R = G.n_rows;
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < n;
       c += (unsigned long long)gridDim.x * blockDim.x) {
    const uint4 rec = __ldg(reinterpret_cast<const uint4*>(W.clusters) + c);
    const int r = (rec.z >> 24) & 0xff, s = rec.w >> 24;
    W.edge_key[c] = ~0ull;
    if (r == 0 || r >= R - 1 || s >= G.n_sectors) {
      W.up[c] = -1; W.down[c] = -1; W.score[c] = -1;
      continue;
    }
    const int sr = s * R + r;
    const long long Xc = G.xrow[r], Xd = G.xrow[r - 1], Xu = G.xrow[r + 1];
    const long long Yc = __ldg(W.cl_y + c), Zc = __ldg(W.cl_z + c);
    const int tc = __ldg(W.cl_t + c);
    const long long dxd = Xc - Xd, dxu = Xu - Xc;
    const unsigned dlo = W.row_start[sr - 1], dhi = W.row_start[sr];
    const unsigned ulo = W.row_start[sr + 1], uhi = W.row_start[sr + 2];
    const int wd = (int)((P.sz_num * dxd) / (P.sz_den * 640LL)) + 5;
    const int wu = (int)((P.sz_num * dxu) / (P.sz_den * 640LL)) + 5;
    const unsigned d0 = lower_bound_t(W.cl_t, dlo, dhi, tc - wd);
    const unsigned u0 = lower_bound_t(W.cl_t, ulo, uhi, tc - wu);
    const long long lim = (long long)P.ca_cut * (Xu - Xd);
    long long best = -1;
    int bd = -1, bu = -1;
    for (unsigned d = d0; d < dhi; d++) {
      if (__ldg(W.cl_t + d) > tc + wd) break;
      const long long Yd = __ldg(W.cl_y + d), Zd = __ldg(W.cl_z + d);
      if (llabs_(Yc - Yd) * P.sy_den > P.sy_num * dxd) continue;
      if (llabs_(Zc - Zd) * P.sz_den > P.sz_num * dxd) continue;
      for (unsigned u = u0; u < uhi; u++) {
        if (__ldg(W.cl_t + u) > tc + wu) break;
        const long long Yu = __ldg(W.cl_y + u), Zu = __ldg(W.cl_z + u);
        if (llabs_(Yu - Yc) * P.sy_den > P.sy_num * dxu) continue;
        if (llabs_(Zu - Zc) * P.sz_den > P.sz_num * dxu) continue;
        const long long devy = (Yu - Yc) * dxd - (Yc - Yd) * dxu;
        const long long devz = (Zu - Zc) * dxd - (Zc - Zd) * dxu;
        if (llabs_(devy) > lim || llabs_(devz) > lim) continue;
        const long long sc = devy * devy + devz * devz;
        // d ascending, then u ascending; strict < keeps the smallest (d, u)
        if (best < 0 || sc < best) { best = sc; bd = (int)d; bu = (int)u; }
      }
    }
    W.up[c] = bu; W.down[c] = bd; W.score[c] = best;
  }
}

// Edge rows: the first row links up to the row-1 cluster that chose it as its
// down neighbour with the smallest score (ties: smallest index); the last row
// mirrors it.  Keys pack (score << 23 | index within the row).
constexpr int kEdgeIdxBits = 23;
__global__ void k_ca_edge_min(DevGeom G, DevWork W) {
  const unsigned long long n = n_clusters(W);
  const int R = G.n_rows;
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < n;
       c += (unsigned long long)gridDim.x * blockDim.x) {
    const uint4 rec = __ldg(reinterpret_cast<const uint4*>(W.clusters) + c);
    const int r = (rec.z >> 24) & 0xff, s = rec.w >> 24;
    if ((r != 1 && r != R - 2) || s >= G.n_sectors) continue;
    const long long sc = W.score[c];
    if (sc < 0) continue;
    const unsigned local = (unsigned)(c - W.row_start[s * R + r]);
    if (local >= (1u << kEdgeIdxBits)) { atomicOr(W.err, kErrRowCount); continue; }
    const unsigned long long key = ((unsigned long long)sc << kEdgeIdxBits) | local;
    if (r == 1) atomicMin(&W.edge_key[W.down[c]], key);
    if (r == R - 2) atomicMin(&W.edge_key[W.up[c]], key);
  }
}

__global__ void k_ca_edge_apply(DevGeom G, DevWork W) {
  const unsigned long long n = n_clusters(W);
  const int R = G.n_rows;
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < n;
       c += (unsigned long long)gridDim.x * blockDim.x) {
    const uint4 rec = __ldg(reinterpret_cast<const uint4*>(W.clusters) + c);
    const int r = (rec.z >> 24) & 0xff, s = rec.w >> 24;
    if ((r != 0 && r != R - 1) || s >= G.n_sectors) continue;
    const unsigned long long key = W.edge_key[c];
    int tgt = -1;
    if (key != ~0ull) {
      const int rr = r == 0 ? 1 : R - 2;
      tgt = (int)(W.row_start[s * R + rr] + (unsigned)(key & ((1ull << kEdgeIdxBits) - 1)));
    }
    if (r == 0) { W.up[c] = tgt; W.down[c] = -1; }
    else { W.down[c] = tgt; W.up[c] = -1; }
  }
}

// ---------------------------------------------------------------- links, chains
// jump word = (distance to the chain's lowest cluster << 32) | that cluster
__global__ void k_links(DevWork W) {
  const unsigned long long n = n_clusters(W);
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < n;
       c += (unsigned long long)gridDim.x * blockDim.x) {
    const int d = W.down[c];
    const bool link = d >= 0 && W.up[d] == (int)c;
    W.jump[c] = link ? ((1ull << 32) | (unsigned)d) : (unsigned long long)c;
    W.chain_len[c] = 0;
  }
}

// Pointer jumping without a grid barrier: every value ever stored in jump[x]
// is a valid (ancestor, distance) pair of x, so reading a stale one is safe,
// and each step strictly increases the distance (bounded by the row count):
// the loop ends.
__global__ void k_jump(DevWork W) {
  const unsigned long long n = n_clusters(W);
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < n;
       c += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long w = __ldcg(W.jump + c);
    for (int it = 0; it < 4 * kMaxRowsDev; it++) {
      const unsigned p = (unsigned)w;
      const unsigned long long wp = __ldcg(W.jump + p);
      if ((unsigned)wp == p) break;
      w = (((w >> 32) + (wp >> 32)) << 32) | (unsigned)wp;
      __stcg(W.jump + c, w);
    }
    atomicMax(&W.chain_len[(unsigned)w], (int)(w >> 32) + 1);
  }
}

__global__ void k_chain_flags(DevParams P, DevWork W) {
  const unsigned long long n = n_clusters(W);
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < n;
       c += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long w = W.jump[c];
    W.scan_val[c] = ((unsigned)w == c && W.chain_len[c] >= P.min_chain) ? 1ull : 0ull;
  }
}

__global__ void k_chain_table(DevParams P, DevWork W) {
  const unsigned long long n = n_clusters(W);
  const unsigned long long nch_raw = W.ctr[CTR_NCH];
  if (blockIdx.x == 0 && threadIdx.x == 0 && nch_raw > W.cap_ch) atomicOr(W.err, kErrOverflowCh);
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < n;
       c += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long w = W.jump[c];
    const unsigned root = (unsigned)w;
    const int pos = (int)(w >> 32);
    const int L = W.chain_len[root];
    const unsigned long long k = L >= P.min_chain ? W.scan_val[root] : ~0ull;
    if (L >= P.min_chain && k < W.cap_ch) {
      W.cl_chain[c] = (int)k;
      W.chain_of[c] = (int)root;
      if (pos == 0) {
        W.ch_root[k] = (int)c; W.ch_len[k] = L; W.ch_next[k] = -1; W.ch_prev[k] = -1;
        W.best_a[k] = ~0ull;
      }
      if (pos == 1) W.ch_b2[k] = (int)c;
      if (pos == L - 1) W.ch_top[k] = (int)c;
      if (pos == L - 2) W.ch_top2[k] = (int)c;
    } else {
      W.cl_chain[c] = -1;
      W.chain_of[c] = -1;
    }
  }
}

// ---------------------------------------------------------------- scan
// Exclusive scan in place of v[0, n), n = min(*n_ptr, cap), single pass with
// decoupled look-back over 2048-element tiles taken by ticket.  *total gets the
// sum.  Blocks loop over tiles (persistent grid).
constexpr int kScanThreads = 256, kScanItems = 8, kScanTile = kScanThreads * kScanItems;

__global__ void __launch_bounds__(kScanThreads)
k_scan(uint64_t* v, const unsigned long long* n_ptr, unsigned long long cap, unsigned long long* state,
       unsigned int* ticket, unsigned long long* total, uint32_t* err) {
  __shared__ unsigned long long sm[34];
  __shared__ long long s_tile;
  unsigned long long n = *n_ptr;
  if (n > cap) n = cap;
  const long long ntiles = (long long)((n + kScanTile - 1) / kScanTile);
  while (true) {
    if (threadIdx.x == 0) s_tile = (long long)atomicAdd(ticket, 1u);
    __syncthreads();
    const long long t = s_tile;
    __syncthreads();
    if (t >= ntiles) {
      if (t == 0 && threadIdx.x == 0) *total = 0;
      break;
    }
    const unsigned long long i0 = (unsigned long long)t * kScanTile + (unsigned long long)threadIdx.x * kScanItems;
    unsigned long long x[kScanItems];
    unsigned long long sum = 0;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
      x[k] = (i0 + k < n) ? v[i0 + k] : 0ull;
      sum += x[k];
    }
    unsigned long long agg;
    unsigned long long pre = block_excl_scan(sum, sm, &agg);
    if (threadIdx.x < 32) {
      unsigned long long base = lookback_warp0(state, t, agg, err);
      if (threadIdx.x == 0) {
        sm[33] = base;
        if (t == ntiles - 1) *total = base + agg;
      }
    }
    __syncthreads();
    unsigned long long run = sm[33] + pre;
#pragma unroll
    for (int k = 0; k < kScanItems; k++) {
      if (i0 + k < n) v[i0 + k] = run;
      run += x[k];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- launchers
static inline unsigned grid_for(unsigned long long cap, int n_sm, int per_sm) {
  unsigned long long g = (cap + 255) / 256;
  unsigned long long m = (unsigned long long)n_sm * per_sm;
  if (g > m) g = m;
  return (unsigned)(g ? g : 1);
}

cudaError_t launch_ca(const DevGeom& G, const DevParams& P, const DevWork& W, int n_sm, cudaStream_t st,
                      int* launches) {
  const unsigned g = grid_for(W.cap_cl, n_sm, 8);
  k_ca_neighbours<<<g, 256, 0, st>>>(G, P, W);
  k_ca_edge_min<<<g, 256, 0, st>>>(G, W);
  k_ca_edge_apply<<<g, 256, 0, st>>>(G, W);
  k_links<<<g, 256, 0, st>>>(W);
  k_jump<<<g, 256, 0, st>>>(W);
  k_chain_flags<<<g, 256, 0, st>>>(P, W);
  const unsigned gs = grid_for((W.cap_cl + kScanItems - 1) / kScanItems, n_sm, 4);
  k_scan<<<gs, kScanThreads, 0, st>>>(W.scan_val, W.ctr + CTR_NCL, W.cap_cl, W.scan_state,
                                      W.tickets + TK_SCAN_A, W.ctr + CTR_NCH, W.err);
  k_chain_table<<<g, 256, 0, st>>>(P, W);
  *launches += 8;
  return cudaGetLastError();
}

cudaError_t launch_scan(uint64_t* v, const unsigned long long* n_ptr, unsigned long long cap,
                        unsigned long long* state, unsigned int* ticket, unsigned long long* total, uint32_t* err,
                        int n_sm, cudaStream_t st) {
  const unsigned gs = grid_for((cap + kScanItems - 1) / kScanItems, n_sm, 4);
  k_scan<<<gs, kScanThreads, 0, st>>>(v, n_ptr, cap, state, ticket, total, err);
  return cudaGetLastError();
}

size_t scan_tiles(unsigned long long cap) { return (size_t)((cap + kScanTile - 1) / kScanTile) + 1; }

}  // namespace tpc
