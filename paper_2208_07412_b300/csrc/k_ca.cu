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


__device__ __forceinline__ long long llabs_(long long v) { return v < 0 ? -v : v; }

// ---------------------------------------------------------------- neighbours
// One block per pad row (grid-stride over the sector x row list), in chunks of
// kCaChunk clusters: the slices of rows r-1 and r+1 that can hold a partner of
// the chunk (time-sorted, so two binary searches bound them) are staged in
// shared memory as (t, Y, Z); every search and candidate loop then runs there.
// A slice larger than the stage is read from global memory instead.  The
// iteration order (d ascending, then u ascending, strict <) is the definition's
// tie rule.
constexpr int kCaThreads = 128, kCaChunk = 128, kCaStage = 768;
// Per staged slice, the index of its first cluster at or past each time bin of
// [tmin - w, tmax + w + 1] (the chunk's candidate range), built while staging:
// a cluster's candidate range is then two table reads instead of two binary
// searches.  Ranges longer than the table fall back to the searches.
constexpr int kCaIdx = 1024;
static_assert(kCaThreads >= 128 && kCaThreads % 32 == 0, "four warps compute the four slice bounds");

struct Slice {
  const int32_t* t; const int32_t* y; const int32_t* z;
  unsigned base, n;   // cluster index of element 0, element count
};

// First index in [lo, hi) with t[i] >= v (hi if none), by a whole warp: each
// round the 32 lanes probe 32 evenly spaced elements and the range shrinks
// 32-fold, so a row of 10^4-10^5 clusters takes 3-4 dependent loads instead of
// 14-17.  Every lane returns the result.
__device__ __forceinline__ unsigned warp_lower_bound(const int32_t* __restrict__ t, unsigned lo, unsigned hi, int v) {
  const unsigned lane = threadIdx.x & 31;
  while (hi - lo > 32) {
    const unsigned step = (hi - lo + 31) / 32;
    const unsigned idx = lo + lane * step;
    const bool ge = idx >= hi || __ldg(t + idx) >= v;
    const unsigned m = __ballot_sync(0xffffffffu, ge);
    if (m == 0) {
      lo = lo + 31 * step + 1;
    } else {
      const unsigned f = (unsigned)(__ffs(m) - 1);
      if (f == 0) return lo;
      const unsigned nlo = lo + (f - 1) * step + 1, nhi = min(lo + f * step, hi);
      lo = nlo;
      hi = nhi;
    }
  }
  const unsigned idx = lo + lane;
  const bool ge = idx >= hi || __ldg(t + idx) >= v;
  const unsigned m = __ballot_sync(0xffffffffu, ge);
  return m ? min(lo + (unsigned)(__ffs(m) - 1), hi) : hi;
}

// The same search when the answer is most likely within 512 elements of lo
// (the chunk after a chunk whose bound was lo): one round probes [lo, lo + 512)
// at stride 16 and, if the bound lies there, one more finishes it.
__device__ __forceinline__ unsigned warp_lower_bound_near(const int32_t* __restrict__ t, unsigned lo, unsigned hi, int v) {
  const unsigned lane = threadIdx.x & 31;
  if (hi - lo > 512) {
    const unsigned idx = lo + lane * 16;
    const bool ge = __ldg(t + idx) >= v;                 // idx < lo + 512 < hi
    const unsigned m = __ballot_sync(0xffffffffu, ge);
    if (m == 0) return warp_lower_bound(t, lo + 31 * 16 + 1, hi, v);
    const unsigned f = (unsigned)(__ffs(m) - 1);
    if (f == 0) return lo;
    return warp_lower_bound(t, lo + (f - 1) * 16 + 1, lo + f * 16, v) ;
  }
  return warp_lower_bound(t, lo, hi, v);
}

__device__ __forceinline__ unsigned lb_slice(const int32_t* t, unsigned n, int v) {
  unsigned lo = 0, hi = n;
  while (lo < hi) {
    const unsigned mid = (lo + hi) >> 1;
    if (t[mid] < v) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kCaThreads)
k_ca_neighbours(DevGeom G, DevParams P, DevWork W) {
  __shared__ int32_t sm_t[2][kCaStage], sm_y[2][kCaStage], sm_z[2][kCaStage];
  __shared__ uint16_t sm_idx[2][kCaIdx];
  __shared__ unsigned sm_rng[4];
  __shared__ int sm_tmm[2];                      // the chunk's first and last time bins
  const unsigned long long n = n_clusters(W);
  const int R = G.n_rows, nsr = G.n_sectors * R;
  const int tid = threadIdx.x;
  // edge keys start empty everywhere; the first and last rows get no pair
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + tid; c < n;
       c += (unsigned long long)gridDim.x * blockDim.x)
    W.edge_key[c] = ~0ull;
  for (int sr = blockIdx.x; sr < nsr; sr += gridDim.x) {
    const int r = sr % R;
    const unsigned lo = min((unsigned long long)W.row_start[sr], n), hi = min((unsigned long long)W.row_start[sr + 1], n);
    if (r == 0 || r == R - 1) {
      for (unsigned c = lo + tid; c < hi; c += blockDim.x) { W.up[c] = -1; W.down[c] = -1; W.score[c] = -1; }
      continue;
    }
    const long long Xc = G.xrow[r], Xd = G.xrow[r - 1], Xu = G.xrow[r + 1];
    const long long dxd = Xc - Xd, dxu = Xu - Xc;
    const int wd = (int)((P.sz_num * dxd) / (P.sz_den * 640LL)) + 5;
    const int wu = (int)((P.sz_num * dxu) / (P.sz_den * 640LL)) + 5;
    const long long lim = (long long)P.ca_cut * (Xu - Xd);
    // the window cuts |dY| den > num dX as |dY| > floor(num dX / den) (den >= 1):
    // one 32-bit compare per candidate (coordinate differences fit 32 bits)
    const int yld = (int)min((P.sy_num * dxd) / P.sy_den, 2147483647LL);
    const int zld = (int)min((P.sz_num * dxd) / P.sz_den, 2147483647LL);
    const int ylu = (int)min((P.sy_num * dxu) / P.sy_den, 2147483647LL);
    const int zlu = (int)min((P.sz_num * dxu) / P.sz_den, 2147483647LL);
    const unsigned dlo = W.row_start[sr - 1], dhi = min((unsigned long long)W.row_start[sr], n);
    const unsigned ulo = min((unsigned long long)W.row_start[sr + 1], n), uhi = min((unsigned long long)W.row_start[sr + 2], n);
    for (unsigned cs = lo; cs < hi; cs += kCaChunk) {
      const unsigned ce = min(cs + kCaChunk, hi);
      // this thread's cluster, loaded before the bounds and the staging so
      // that its latency overlaps theirs
      const unsigned c = cs + tid;
      int Yc = 0, Zc = 0, tc = 0;
      if (c < ce) { Yc = W.cl_y[c]; Zc = W.cl_z[c]; tc = W.cl_t[c]; }
      if (tid < 128) {
        // slices of the neighbour rows that can pair with clusters [cs, ce):
        // warp q computes bound q (row below: 0, 1; row above: 2, 3)
        const int q = tid >> 5, side = q >> 1;
        const int tmin = W.cl_t[cs], tmax = W.cl_t[ce - 1];
        if (tid == 0) { sm_tmm[0] = tmin; sm_tmm[1] = tmax; }
        const unsigned a = side == 0 ? dlo : ulo, b = side == 0 ? dhi : uhi;
        const int w = side == 0 ? wd : wu;
        // the bounds only grow from chunk to chunk: start from the previous one
        const unsigned a1 = cs == lo ? a : max(a, min(sm_rng[q], b));
        const unsigned bound = warp_lower_bound_near(W.cl_t, a1, b, (q & 1) ? tmax + w + 1 : tmin - w);
        __syncwarp();
        if ((tid & 31) == 0) sm_rng[q] = bound;
      }
      __syncthreads();
      Slice sl[2];
      const int tmin = sm_tmm[0], tmax = sm_tmm[1];
      int tlo[2], Rk[2];
      unsigned nst[2];                                   // elements staged per slice (+1: a virtual one)
      bool use_idx[2];
#pragma unroll
      for (int k = 0; k < 2; k++) {
        const unsigned a = sm_rng[2 * k], b = sm_rng[2 * k + 1];
        const int w = k == 0 ? wd : wu;
        sl[k].base = a;
        sl[k].n = b > a ? b - a : 0;
        tlo[k] = tmin - w;
        Rk[k] = tmax + w + 1 - tlo[k];                    // table entries 0 .. Rk
        const bool staged = sl[k].n <= (unsigned)kCaStage;
        use_idx[k] = staged && Rk[k] < kCaIdx;
        nst[k] = staged ? sl[k].n + 1 : 0u;
        if (staged) {
          sl[k].t = sm_t[k]; sl[k].y = sm_y[k]; sl[k].z = sm_z[k];
        } else {
          sl[k].t = W.cl_t + a; sl[k].y = W.cl_y + a; sl[k].z = W.cl_z + a;
        }
      }
      // Both slices staged in one loop, so that their loads are in flight
      // together.  Element i (and a virtual element n past the range) fills the
      // table entries of the bins after its predecessor's time bin up to its own.
      const unsigned nloop = max(nst[0], nst[1]);
      for (unsigned i = tid; i < nloop; i += blockDim.x) {
        int ti[2], yi[2], zi[2], tp[2];
#pragma unroll
        for (int k = 0; k < 2; k++) {
          const int w = k == 0 ? wd : wu;
          const unsigned a = sl[k].base;
          const bool in = i < nst[k], real = in && i < sl[k].n;
          ti[k] = real ? W.cl_t[a + i] : tmax + w + 2;
          yi[k] = real ? W.cl_y[a + i] : 0;
          zi[k] = real ? W.cl_z[a + i] : 0;
          tp[k] = (in && use_idx[k] && i > 0) ? W.cl_t[a + i - 1] : tlo[k] - 1;
        }
#pragma unroll
        for (int k = 0; k < 2; k++) {
          if (i >= nst[k]) continue;
          if (i < sl[k].n) {
            sm_t[k][i] = ti[k];
            sm_y[k][i] = yi[k];
            sm_z[k][i] = zi[k];
          }
          if (use_idx[k]) {
            const int b1 = min(ti[k] - tlo[k], Rk[k]);
            for (int bb = max(tp[k] + 1 - tlo[k], 0); bb <= b1; bb++) sm_idx[k][bb] = (uint16_t)i;
          }
        }
      }
      __syncthreads();
      if (c < ce) {
        // candidate ranges [d0, d1), [u0, u1): the clusters within the time window
        const unsigned d0 = use_idx[0] ? sm_idx[0][tc - wd - tlo[0]] : lb_slice(sl[0].t, sl[0].n, tc - wd);
        const unsigned d1 = use_idx[0] ? sm_idx[0][tc + wd + 1 - tlo[0]] : lb_slice(sl[0].t, sl[0].n, tc + wd + 1);
        const unsigned u0 = use_idx[1] ? sm_idx[1][tc - wu - tlo[1]] : lb_slice(sl[1].t, sl[1].n, tc - wu);
        const unsigned u1 = use_idx[1] ? sm_idx[1][tc + wu + 1 - tlo[1]] : lb_slice(sl[1].t, sl[1].n, tc + wu + 1);
        // candidates passing the window cuts, in ascending index order
        constexpr int kMaxCand = 8;
        unsigned di[kMaxCand], ui[kMaxCand];
        int nd = 0, nu = 0;
        bool spill = false;
        for (unsigned i = d0; i < d1; i++) {
          if (abs(Yc - sl[0].y[i]) > yld) continue;
          if (abs(Zc - sl[0].z[i]) > zld) continue;
          if (nd < kMaxCand) di[nd] = i; else spill = true;
          nd++;
        }
        for (unsigned j = u0; nd > 0 && j < u1; j++) {
          if (abs(sl[1].y[j] - Yc) > ylu) continue;
          if (abs(sl[1].z[j] - Zc) > zlu) continue;
          if (nu < kMaxCand) ui[nu] = j; else spill = true;
          nu++;
        }
        long long best = -1;
        int bd = -1, bu = -1;
        if (!spill) {
          for (int a = 0; a < nd; a++) {
            const int Yd = sl[0].y[di[a]], Zd = sl[0].z[di[a]];
            for (int b = 0; b < nu; b++) {
              const int Yu = sl[1].y[ui[b]], Zu = sl[1].z[ui[b]];
              const long long devy = (long long)(Yu - Yc) * dxd - (long long)(Yc - Yd) * dxu;
              const long long devz = (long long)(Zu - Zc) * dxd - (long long)(Zc - Zd) * dxu;
              if (llabs_(devy) > lim || llabs_(devz) > lim) continue;
              const long long sc = devy * devy + devz * devz;
              if (best < 0 || sc < best) { best = sc; bd = (int)(sl[0].base + di[a]); bu = (int)(sl[1].base + ui[b]); }
            }
          }
        } else {
          // more candidates than the lists hold: the plain double loop
          for (unsigned i = d0; i < sl[0].n; i++) {
            if (sl[0].t[i] > tc + wd) break;
            const int Yd = sl[0].y[i], Zd = sl[0].z[i];
            if (abs(Yc - Yd) > yld) continue;
            if (abs(Zc - Zd) > zld) continue;
            for (unsigned j = u0; j < sl[1].n; j++) {
              if (sl[1].t[j] > tc + wu) break;
              const int Yu = sl[1].y[j], Zu = sl[1].z[j];
              if (abs(Yu - Yc) > ylu) continue;
              if (abs(Zu - Zc) > zlu) continue;
              const long long devy = (long long)(Yu - Yc) * dxd - (long long)(Yc - Yd) * dxu;
              const long long devz = (long long)(Zu - Zc) * dxd - (long long)(Zc - Zd) * dxu;
              if (llabs_(devy) > lim || llabs_(devz) > lim) continue;
              const long long sc = devy * devy + devz * devz;
              if (best < 0 || sc < best) { best = sc; bd = (int)(sl[0].base + i); bu = (int)(sl[1].base + j); }
            }
          }
        }
        W.up[c] = bu; W.down[c] = bd; W.score[c] = best;
      }
      __syncthreads();
    }
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
    const int r = (rec.z >> 24) & 0xff;
    if (r != 1 && r != R - 2) continue;
    const int s = vsector_of(G, W, c, (int)(rec.w >> 24));
    if (s >= G.n_sectors) continue;
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
    const int r = (rec.z >> 24) & 0xff;
    if (r != 0 && r != R - 1) continue;
    const int s = vsector_of(G, W, c, (int)(rec.w >> 24));
    if (s >= G.n_sectors) continue;
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
        W.ch_t[k] = W.cl_t[c];
        W.best_a[k] = ~0ull;
        W.best_b[k] = ~0ull;
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

// Per (sector, row): the first chain whose root (bottom cluster) lies in it.
// Chain ids follow their roots' canonical order, so the chains rooted in a row
// are a contiguous id range, ordered by the root's time bin.
__global__ void k_chain_rows(DevGeom G, DevWork W) {
  const unsigned long long nch = min(W.ctr[CTR_NCH], (unsigned long long)W.cap_ch);
  const int R = G.n_rows;
  const long long nsr = (long long)G.n_sectors * R;
  const long long NB = 4LL * G.n_frag + 1, nkeys = nsr * NB;
  if (nch == 0) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i <= nsr; i += (long long)gridDim.x * blockDim.x)
      W.ch_row_start[i] = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i <= nkeys; i += (long long)gridDim.x * blockDim.x)
      W.ch_bucket[i] = 0;
    return;
  }
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < nch;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    auto sr_of = [&](unsigned long long kk) {
      const unsigned c = (unsigned)W.ch_root[kk];
      const uint4 rec = __ldg(reinterpret_cast<const uint4*>(W.clusters) + c);
      return (long long)vsector_of(G, W, c, (int)(rec.w >> 24)) * R + ((rec.z >> 24) & 0xff);
    };
    const long long sr = sr_of(k);
    const long long prev = k > 0 ? sr_of(k - 1) : -1;
    for (long long i = prev + 1; i <= sr && i <= nsr; i++) W.ch_row_start[i] = (uint32_t)k;
    if (k == nch - 1)
      for (long long i = sr + 1; i <= nsr; i++) W.ch_row_start[i] = (uint32_t)nch;
    // the same over (row, 64-bin bucket of the root's time bin) keys, which
    // follow the chain order too
    auto key_of = [&](unsigned long long kk, long long srk) {
      return srk * NB + min((long long)(W.ch_t[kk] >> 6), NB - 1);
    };
    const long long key = key_of(k, sr);
    const long long kprev = k > 0 ? key_of(k - 1, prev) : -1;
    for (long long i = kprev + 1; i <= key && i <= nkeys; i++) W.ch_bucket[i] = (uint32_t)k;
    if (k == nch - 1)
      for (long long i = key + 1; i <= nkeys; i++) W.ch_bucket[i] = (uint32_t)nch;
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

cudaError_t launch_ca(const DevGeom& G, const DevParams& P, const DevWork& W, int n_sm, const LaunchCfg& L,
                      cudaStream_t st, int* launches) {
  const unsigned g = grid_for(W.cap_cl, n_sm, L.elem_blocks_per_sm);
  k_ca_neighbours<<<(unsigned)min(G.n_sectors * G.n_rows, n_sm * L.ca_blocks_per_sm), kCaThreads, 0, st>>>(G, P, W);
  k_ca_edge_min<<<g, 256, 0, st>>>(G, W);
  k_ca_edge_apply<<<g, 256, 0, st>>>(G, W);
  k_links<<<g, 256, 0, st>>>(W);
  k_jump<<<g, 256, 0, st>>>(W);
  k_chain_flags<<<g, 256, 0, st>>>(P, W);
  const unsigned gs = grid_for((W.cap_cl + kScanItems - 1) / kScanItems, n_sm, 4);
  k_scan<<<gs, kScanThreads, 0, st>>>(W.scan_val, W.ctr + CTR_NCL, W.cap_cl, W.scan_state,
                                      W.tickets + TK_SCAN_A, W.ctr + CTR_NCH, W.err);
  k_chain_table<<<g, 256, 0, st>>>(P, W);
  k_chain_rows<<<grid_for(W.cap_ch, n_sm, L.elem_blocks_per_sm), 256, 0, st>>>(G, W);
  *launches += 9;
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
