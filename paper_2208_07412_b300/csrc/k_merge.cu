// k_merge.cu — in-sector segment merge and track assembly (step 7 of the
// library's definition; the paper's section "Hardware and data flow" names the
// TPC tracking the EPN GPUs run, not its merge rule, which is this library's).
//
// The ends of merged groups are always ends of the original chains, so the
// candidate pairs (top end a1 below a2, bottom end b1 below b2, four integer
// straight-line residuals within the cut) do not change between passes: they
// are searched once, one thread per (top chain, gap row), and stored.  A pass
// then takes, among the stored pairs whose top is still a group top and whose
// bottom is still a group bottom, the best bottom per top and the best top per
// bottom by 64-bit atomicMin on (score << 32 | chain index), and links the
// mutual-best pairs.  Passes repeat until one links nothing; later passes exit
// at once, so a fixed number of launches gives the fixpoint (graph friendly).
#include "tpc_internal.cuh"

namespace tpc {

__device__ __forceinline__ unsigned long long n_chains_m(const DevWork& W) {
  unsigned long long n = W.ctr[CTR_NCH];
  return n < W.cap_ch ? n : W.cap_ch;
}
__device__ __forceinline__ long long floordiv_ll(long long a, long long b) {  // b > 0
  long long q = a / b;
  if ((a % b) != 0 && a < 0) q -= 1;
  return q;
}
__device__ __forceinline__ long long absll(long long v) { return v < 0 ? -v : v; }
// Residual r = trunc(n / d), n = (yb - y2)(x2 - x1) - (y2 - y1)(xb - x2),
// d = x2 - x1: true when |r| <= MC, r then set.  |trunc(n / d)| =
// floor(|n| / |d|) exceeds MC exactly when |n| >= (MC + 1) |d|, so a pair past
// the cut costs a multiply, not a 64-bit division.
__device__ __forceinline__ bool extrap_res_within(long long x1, long long y1, long long x2, long long y2,
                                                  long long xb, long long yb, long long MC, long long& r) {
  const long long n = (yb - y2) * (x2 - x1) - (y2 - y1) * (xb - x2), d = x2 - x1;
  if (absll(n) >= (MC + 1) * absll(d)) return false;
  r = n / d;
  return true;
}
__global__ void k_merge_cand(DevGeom G, DevParams P, DevWork W) {
  const unsigned long long nch = n_chains_m(W);
  const int ngap = P.gap_max - P.gap_min + 1;
  unsigned long long* bestA = W.best_a;   // pass 0 buffer
  const int R = G.n_rows;
  const long long MC = P.merge_cut;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < nch * ngap;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long k = i / ngap;
    const int a2 = W.ch_top[k], a1 = W.ch_top2[k];
    const uint4 rec = __ldg(reinterpret_cast<const uint4*>(W.clusters) + a2);
    const int r2 = (rec.z >> 24) & 0xff, s = min(vsector_of(G, W, a2, (int)(rec.w >> 24)), G.n_sectors - 1);
    const int rb = r2 + P.gap_min + (int)(i % ngap);
    if (r2 >= R || rb >= R) continue;
    const long long Xa1 = W.cl_x[a1], Ya1 = W.cl_y[a1], Za1 = W.cl_z[a1];
    const long long Xa2 = W.cl_x[a2], Ya2 = W.cl_y[a2], Za2 = W.cl_z[a2];
    const long long dxa = Xa2 - Xa1;
    const long long Xb = G.xrow[rb];
    const long long zp = Za2 + floordiv_ll((Za2 - Za1) * (Xb - Xa2), dxa);
    const long long tlo = floordiv_ll(zp - MC - 2, 640) - 3;
    const long long thi = floordiv_ll(zp + MC + 2, 640) + 3;
    // the chains whose bottom (root) cluster lies in row rb, by root time bin
    const unsigned hi = W.ch_row_start[s * R + rb + 1];
    // the first chain at or past time bin tlo: from its 64-bin bucket's first chain
    const long long NB = 4LL * G.n_frag + 1;
    unsigned kb0 = W.ch_bucket[(long long)(s * R + rb) * NB + (tlo < 0 ? 0 : min(tlo >> 6, NB - 1))];
    while (kb0 < hi && (long long)__ldg(W.ch_t + kb0) < tlo) kb0++;
    for (unsigned kb = kb0; kb < hi; kb++) {
      if ((long long)__ldg(W.ch_t + kb) > thi) break;
      const int b1 = W.ch_root[kb];
      const int b2 = W.ch_b2[kb];
      const long long Xb1 = W.cl_x[b1], Yb1 = W.cl_y[b1], Zb1 = W.cl_z[b1];
      const long long Xb2 = W.cl_x[b2], Yb2 = W.cl_y[b2], Zb2 = W.cl_z[b2];
      long long ry, rz, sy, sz;
      if (!extrap_res_within(Xa1, Ya1, Xa2, Ya2, Xb1, Yb1, MC, ry) ||
          !extrap_res_within(Xa1, Za1, Xa2, Za2, Xb1, Zb1, MC, rz) ||
          !extrap_res_within(Xb2, Yb2, Xb1, Yb1, Xa2, Ya2, MC, sy) ||
          !extrap_res_within(Xb2, Zb2, Xb1, Zb1, Xa2, Za2, MC, sz))
        continue;
      const unsigned long long sc = (unsigned long long)(ry * ry + rz * rz + sy * sy + sz * sz);
      // pass 0: every chain is both a group top and a group bottom
      atomicMin(&W.best_b[k], (sc << 32) | (unsigned)kb);
      atomicMin(&bestA[kb], (sc << 32) | (unsigned)k);
      const unsigned long long slot = aggregated_inc(&W.ctr[CTR_NCAND]);
      if (slot < W.cap_cand) {
        W.cand_ab[slot] = (k << 32) | (unsigned)kb;
        W.cand_sc[slot] = (uint32_t)sc;
      } else {
        atomicOr(W.err, kErrOverflowCh);
      }
    }
  }
}

// Passes after the first: the stored pairs whose ends are still group ends.
__global__ void k_merge_best(DevWork W, int pass) {
  if (W.ctr[CTR_MERGED0 + pass - 1] == 0) return;
  unsigned long long n = W.ctr[CTR_NCAND];
  if (n > W.cap_cand) n = W.cap_cand;
  unsigned long long* bestA = W.best_a + (size_t)(pass & 1) * W.cap_ch;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const unsigned long long ab = W.cand_ab[i];
    const unsigned k = (unsigned)(ab >> 32), kb = (unsigned)ab;
    if (W.ch_next[k] >= 0 || W.ch_prev[kb] >= 0) continue;
    const unsigned long long sc = W.cand_sc[i];
    atomicMin(&W.best_b[k], (sc << 32) | kb);
    atomicMin(&bestA[kb], (sc << 32) | k);
  }
}

__global__ void k_merge_link(DevWork W, int pass) {
  if (pass > 0 && W.ctr[CTR_MERGED0 + pass - 1] == 0) return;
  const unsigned long long nch = n_chains_m(W);
  const unsigned long long* bestA = W.best_a + (size_t)(pass & 1) * W.cap_ch;
  unsigned long long* nextA = W.best_a + (size_t)((pass + 1) & 1) * W.cap_ch;
  unsigned int linked = 0;
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < nch;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    nextA[k] = ~0ull;
    const unsigned long long key = W.best_b[k];
    W.best_b[k] = ~0ull;   // ready for the next pass
    if (key == ~0ull) continue;
    const unsigned kb = (unsigned)key;
    if ((unsigned)bestA[kb] == (unsigned)k) {
      W.ch_next[k] = (int)kb;
      W.ch_prev[kb] = (int)k;
      linked++;
    }
  }
  linked = __reduce_add_sync(0xffffffffu, linked);
  if ((threadIdx.x & 31) == 0 && linked) atomicAdd(&W.ctr[CTR_MERGED0 + pass], (unsigned long long)linked);
}

// Group roots (chains with no lower neighbour) sum their group's clusters; a
// group with >= min_track clusters becomes a track.  The scan value packs
// (is_track << 32 | clusters) so one scan gives track indices and offsets.
__global__ void k_groups(DevParams P, DevWork W) {
  const unsigned long long nch = n_chains_m(W);
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < nch;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    unsigned long long v = 0;
    int tot = 0;
    if (W.ch_prev[k] < 0) {
      int g = (int)k;
      for (int it = 0; g >= 0 && it < kMaxRowsDev; it++) { tot += W.ch_len[g]; g = W.ch_next[g]; }
      if (tot >= P.min_track) v = (1ull << 32) | (unsigned)tot;
    }
    W.grp_total[k] = tot;
    W.scan_val[k] = v;
  }
}

__global__ void k_group_assign(DevParams P, DevWork W) {
  const unsigned long long nch = n_chains_m(W);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const unsigned long long tot = W.ctr[CTR_NCLCL];
    W.ctr[CTR_NTRK] = tot >> 32;
  }
  for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < nch;
       k += (unsigned long long)gridDim.x * blockDim.x) {
    if (W.ch_prev[k] >= 0) continue;
    const bool is_trk = W.grp_total[k] >= P.min_track;
    const unsigned long long v = W.scan_val[k];
    const int t = is_trk ? (int)(v >> 32) : -1;
    if (is_trk) {
      W.trk_first[t] = W.ch_root[k];
      W.trk_ncl[t] = W.grp_total[k];
      W.trk_off[t] = (int)(unsigned)v;
      aggregated_inc_keyed(W.len_hist, 255 - min(W.grp_total[k], 255));
    }
    int g = (int)k, run = 0;
    for (int it = 0; g >= 0 && it < kMaxRowsDev; it++) {
      W.ch_track[g] = t;
      W.ch_off[g] = run;
      run += W.ch_len[g];
      g = W.ch_next[g];
    }
  }
}

__global__ void k_cluster_assign(DevWork W) {
  unsigned long long n = W.ctr[CTR_NCL];
  if (n > W.cap_cl) n = W.cap_cl;
  for (unsigned long long c = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; c < n;
       c += (unsigned long long)gridDim.x * blockDim.x) {
    const int k = W.cl_chain[c];
    int t = -1;
    if (k >= 0) {
      t = W.ch_track[k];
      if (t >= 0) {
        const int pos = (int)(W.jump[c] >> 32);
        const int idx = W.trk_off[t] + W.ch_off[k] + pos;
        W.track_cl[idx] = (int)c;
        // the fit reads the coordinates in track order, without indirection
        W.trk_xyz[idx] = make_int4(W.cl_x[c], W.cl_y[c], W.cl_z[c], (int)c);
      }
    }
    W.cl2trk[c] = t;
  }
}

// Fit order: tracks sorted by length, longest first (a counting sort over
// 256 length bins), so that a warp holds tracks of similar length and the
// longest serial chains start first.  Order within a bin is arbitrary; each
// track's fit does not depend on it.
__global__ void k_fit_order(DevWork W) {
  __shared__ unsigned long long pre[256];
  __shared__ unsigned long long sm[34];
  const unsigned long long ntrk = min(W.ctr[CTR_NTRK], (unsigned long long)W.cap_ch);
  unsigned long long tot;
  const unsigned long long v = threadIdx.x < 256 ? W.len_hist[threadIdx.x] : 0ull;
  const unsigned long long ex = block_excl_scan(v, sm, &tot);
  if (threadIdx.x < 256) pre[threadIdx.x] = ex;
  __syncthreads();
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < ntrk;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const int bin = 255 - min(W.trk_ncl[t], 255);
    const unsigned rank = aggregated_inc_keyed(W.len_hist + 256, bin);
    W.fit_order[pre[bin] + rank] = (int)t;
  }
}

static inline unsigned grid_for_m(unsigned long long cap, int n_sm, int per_sm) {
  unsigned long long g = (cap + 255) / 256;
  unsigned long long m = (unsigned long long)n_sm * per_sm;
  if (g > m) g = m;
  return (unsigned)(g ? g : 1);
}

cudaError_t launch_scan(uint64_t* v, const unsigned long long* n_ptr, unsigned long long cap,
                        unsigned long long* state, unsigned int* ticket, unsigned long long* total, uint32_t* err,
                        int n_sm, cudaStream_t st);

cudaError_t launch_merge(const DevGeom& G, const DevParams& P, const DevWork& W, int n_sm, const LaunchCfg& L,
                         cudaStream_t st, unsigned long long* scan_state_b, int* launches) {
  const int per_sm = L.elem_blocks_per_sm;
  const unsigned gc = grid_for_m(W.cap_ch, n_sm, per_sm);
  for (int p = 0; p < P.merge_passes; p++) {
    if (p == 0) {
      const int ngap = P.gap_max - P.gap_min + 1;
      k_merge_cand<<<grid_for_m(W.cap_ch * ngap, n_sm, per_sm), 256, 0, st>>>(G, P, W);
    } else {
      k_merge_best<<<grid_for_m(W.cap_cand, n_sm, per_sm), 256, 0, st>>>(W, p);
    }
    k_merge_link<<<gc, 256, 0, st>>>(W, p);
  }
  k_groups<<<gc, 256, 0, st>>>(P, W);
  cudaError_t e = launch_scan(W.scan_val, W.ctr + CTR_NCH, W.cap_ch, scan_state_b, W.tickets + TK_SCAN_B,
                              W.ctr + CTR_NCLCL, W.err, n_sm, st);
  if (e != cudaSuccess) return e;
  k_group_assign<<<gc, 256, 0, st>>>(P, W);
  const unsigned g = grid_for_m(W.cap_cl, n_sm, per_sm);
  k_cluster_assign<<<g, 256, 0, st>>>(W);
  k_fit_order<<<grid_for_m(W.cap_ch, n_sm, 4), 256, 0, st>>>(W);
  *launches += 2 * P.merge_passes + 5;
  return cudaGetLastError();
}

}  // namespace tpc
