// k_find.cu — ZS decode + 3x3 peak finder + 5x5 cluster moments + stable
// compaction, fused in one persistent kernel (steps 1-4 of the library's
// definition; the paper's section "Hardware and data flow" places this first
// step of the TPC reconstruction on the EPN GPUs, after FPGA zero suppression).
//
// One CTA iteration processes one window = (sector, row, 256-bin fragment).
// The window's page, plus the 3-time-bin halos of the neighbouring pages, are
// decoded into a shared-memory plane guarded by an occupancy bitmap: only the
// bitmap (5 KB) is cleared, never the 72 KB plane, so the work scales with the
// digits and not with the pixels.  Peaks are found by walking the bitmap in
// (t, pad) order, which is the canonical cluster order; a block scan ranks them
// and a decoupled look-back over the windows (taken in index order through an
// atomic ticket) gives the global offset, so clusters are written once, in
// their final place, with no scratch copy.
#include "tpc_internal.cuh"

namespace tpc {

constexpr int kFindThreads = 256;

struct PageHdr {
  uint32_t len;
  int n_tb, n_runs, n_dig, sector, row, frag, magic;
  int lo_tb, lo_runs, lo_dig, hi_tb, hi_runs, hi_dig;
  uint32_t body;   // byte offset of the ADC words
};

__device__ __forceinline__ bool read_header(const DevWork& W, uint64_t off, PageHdr& h) {
  if ((off & 15) || off + 32 > W.pages_bytes) return false;
  const uint4* p = reinterpret_cast<const uint4*>(W.pages + off);
  uint4 a = __ldg(p), b = __ldg(p + 1);
  h.len = a.x;
  h.n_tb = a.y & 0xffff; h.n_runs = a.y >> 16;
  h.n_dig = a.z & 0xffff; h.sector = (a.z >> 16) & 0xff; h.row = a.z >> 24;
  h.frag = a.w & 0xffff; h.magic = a.w >> 16;
  h.lo_tb = b.x & 0xffff; h.lo_runs = b.x >> 16; h.lo_dig = b.y & 0xffff;
  h.hi_tb = b.y >> 16; h.hi_runs = b.z & 0xffff; h.hi_dig = b.z >> 16;
  uint64_t body = (32ull + 2ull * h.n_tb + 2ull * h.n_runs + 3ull) & ~3ull;
  h.body = (uint32_t)body;
  if (h.magic != (int)TPC_ZS_MAGIC || (h.len & 15) || off + h.len > W.pages_bytes ||
      body + 4ull * ((h.n_dig + 2) / 3) > h.len)
    return false;
  if (h.n_tb > kFrag || h.lo_tb > h.n_tb || h.hi_tb > h.n_tb || h.lo_runs > h.n_runs ||
      h.hi_runs > h.n_runs || h.lo_dig > h.n_dig || h.hi_dig > h.n_dig)
    return false;
  return true;
}

constexpr int kStage = 256;   // clusters staged in shared memory before the look-back

struct FindSmem {
  uint16_t* plane;     // [kWinT][npmax]
  uint32_t* occ;       // [kWinT][nw]
  uint32_t* pk;        // [kWinT][nw]
  uint16_t* wpre;      // digit rank prefix over the words of plane rows 1..260, [(kWinT-2)*nw + 1]
  uint16_t* ppre;      // own-peak rank prefix over the words of rows 3..258, [kFrag*nw + 1]
  uint4* st_rec;       // [kStage] staged cluster records
  int4* st_xyz;        // [kStage] staged (X, Y, Z, t_peak)
  uint8_t* ent_t;      // [256]
  int32_t* ent_rs;     // [257]
  unsigned long long* scan;  // [34]
  int32_t* misc;       // [16]
};

__device__ __forceinline__ int floordiv64(long long n, long long d) {
  long long q = n / d;
  if ((n % d) != 0 && (n < 0)) q -= 1;
  return (int)q;
}
// R(a, b) = floor((2a + b) / (2b)), b > 0
__device__ __forceinline__ long long round_half_up(long long a, long long b) {
  long long n = 2 * a + b, d = 2 * b;
  long long q = n / d;
  if ((n % d) != 0 && (n < 0)) q -= 1;
  return q;
}

// Decode entries [e0, e1) of a page (first run r0, first digit d0) into plane
// rows tt = t_in + tt_base.  All reads are bounds-checked against the page's
// counts, all writes against the plane.  Returns true (block-uniform) if every
// check passed; `strict` adds the ordering checks of the page's own window.
__device__ bool decode_segment(const uint8_t* pg, const PageHdr& h, int e0, int e1, int r0, int d0,
                               int tt_base, int np, int stride, int nw, int t_base_abs, int T,
                               bool strict, const FindSmem& S) {
  const uint8_t* ent = pg + 32;
  const uint8_t* run = ent + 2 * h.n_tb;
  const uint8_t* adc = pg + h.body;
  const int tid = threadIdx.x;
  const int ne = e1 - e0;
  bool bad = ne < 0 || ne > kFrag;
  int t_in = 0, nr = 0;
  if (!bad && tid < ne) {
    uint32_t v = __ldg(reinterpret_cast<const uint16_t*>(ent) + e0 + tid);
    t_in = v & 0xff;
    nr = v >> 8;
    int tt = t_in + tt_base;
    if (nr < 1 || tt < 0 || tt >= kWinT || t_base_abs + t_in >= T) bad = true;
    if (strict && tid > 0) {
      uint32_t pv = __ldg(reinterpret_cast<const uint16_t*>(ent) + e0 + tid - 1);
      if ((int)(pv & 0xff) >= t_in) bad = true;
    }
  }
  unsigned long long tot;
  unsigned long long rs = block_excl_scan((unsigned long long)nr, S.scan, &tot);
  if (tid < ne) { S.ent_t[tid] = (uint8_t)t_in; S.ent_rs[tid] = (int32_t)rs; }
  const int nrun = (int)tot;
  if (r0 + nrun > h.n_runs) bad = true;
  __syncthreads();
  unsigned long long dcarry = 0;
  for (int base = 0; base < nrun; base += blockDim.x) {
    int j = base + tid;
    int ps = 0, len = 0, tt = 0;
    bool mine = j < nrun && r0 + j < h.n_runs;
    if (mine) {
      uint32_t v = __ldg(reinterpret_cast<const uint16_t*>(run) + r0 + j);
      ps = v & 0xff;
      len = v >> 8;
      int lo = 0, hi = ne - 1;
      while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (S.ent_rs[mid] <= j) lo = mid; else hi = mid - 1;
      }
      tt = (int)S.ent_t[lo] + tt_base;
      if (len < 1 || ps + len > np || tt < 0 || tt >= kWinT) { bad = true; mine = false; len = 0; }
      if (strict && j > S.ent_rs[lo]) {
        uint32_t pv = __ldg(reinterpret_cast<const uint16_t*>(run) + r0 + j - 1);
        if ((int)ps < (int)(pv & 0xff) + (int)(pv >> 8)) bad = true;
      }
    }
    unsigned long long ctot;
    unsigned long long doff = block_excl_scan((unsigned long long)len, S.scan, &ctot);
    long long di = (long long)d0 + (long long)dcarry + (long long)doff;
    if (mine && di + len > h.n_dig) { bad = true; mine = false; }
    if (mine) {
      uint16_t* prow = S.plane + tt * stride;
      for (int k = 0; k < len; k++) {
        long long d = di + k;
        uint32_t w = __ldg(reinterpret_cast<const uint32_t*>(adc) + d / 3);
        prow[ps + k] = (uint16_t)((w >> (10 * (int)(d % 3))) & 1023u);
      }
      // occupancy bits for pads [ps, ps + len)
      int p = ps, pe = ps + len;
      while (p < pe) {
        int wi = p >> 5, b0 = p & 31;
        int n = min(32 - b0, pe - p);
        uint32_t m = (n == 32) ? 0xffffffffu : (((1u << n) - 1u) << b0);
        atomicOr(&S.occ[tt * nw + wi], m);
        p += n;
      }
    }
    dcarry += ctot;
  }
  if (strict && (r0 + nrun != h.n_runs || d0 + (long long)dcarry != h.n_dig)) bad = true;
  return !__syncthreads_or(bad);
}

__device__ __forceinline__ int qat(const FindSmem& S, int stride, int nw, int np, int tt, int p) {
  if (p < 0 || p >= np) return 0;
  return ((S.occ[tt * nw + (p >> 5)] >> (p & 31)) & 1u) ? (int)S.plane[tt * stride + p] : 0;
}
__device__ __forceinline__ bool pkat(const FindSmem& S, int nw, int np, int tt, int p) {
  if (p < 0 || p >= np) return false;
  return (S.pk[tt * nw + (p >> 5)] >> (p & 31)) & 1u;
}

__device__ __forceinline__ bool peak_test(const FindSmem& S, int stride, int nw, int np, int tt, int p, int q) {
  // neighbours with a lower linear index must be strictly lower in charge,
  // those with a higher index lower or equal: key = (q, -(t * npads + p))
  return q > qat(S, stride, nw, np, tt - 1, p - 1) && q > qat(S, stride, nw, np, tt - 1, p) &&
         q > qat(S, stride, nw, np, tt - 1, p + 1) && q > qat(S, stride, nw, np, tt, p - 1) &&
         q >= qat(S, stride, nw, np, tt, p + 1) && q >= qat(S, stride, nw, np, tt + 1, p - 1) &&
         q >= qat(S, stride, nw, np, tt + 1, p) && q >= qat(S, stride, nw, np, tt + 1, p + 1);
}

// Index of the last prefix entry <= r in pre[0..n] (pre ascending, pre[0] = 0).
__device__ __forceinline__ int rank_search(const uint16_t* pre, int n, int r) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((int)pre[mid] <= r) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Cluster of the peak at (tt, p): 5x5 window with the inner/outer rule.
__device__ __forceinline__ void make_cluster(const FindSmem& S, int stride, int nw, int np, int T, int s, int r,
                                             int f, int tt, int p, int xrow, uint4& rec, int4& xyz) {
  int Q = 0, Sp = 0, St = 0, Spp = 0, Stt = 0;
  bool excl = false, other = false;
#pragma unroll
  for (int dt = -2; dt <= 2; dt++) {
#pragma unroll
    for (int dp = -2; dp <= 2; dp++) {
      const int q = qat(S, stride, nw, np, tt + dt, p + dp);
      bool inc;
      if (dp >= -1 && dp <= 1 && dt >= -1 && dt <= 1) {
        inc = true;
      } else {
        const int ip = dp > 0 ? 1 : (dp < 0 ? -1 : 0), it = dt > 0 ? 1 : (dt < 0 ? -1 : 0);
        const int qi = qat(S, stride, nw, np, tt + it, p + ip);
        inc = qi > 0 && q <= qi;
        if (!inc && q > 0) excl = true;
      }
      if (inc) {
        Q += q; Sp += q * dp; St += q * dt; Spp += q * dp * dp; Stt += q * dt * dt;
      }
      if ((dp || dt) && pkat(S, nw, np, tt + dt, p + dp)) other = true;
    }
  }
  const int t_in = tt - kHalo;
  const int t = kFrag * f + t_in;
  const long long QQ = Q;
  const int pad_fp = 256 * p + (int)round_half_up(256LL * Sp, QQ);
  const int time_fp = 128 * (t_in + 4) + (int)round_half_up(128LL * St, QQ);
  const long long vp = round_half_up(16LL * ((long long)Spp * QQ - (long long)Sp * Sp), QQ * QQ);
  const long long vt = round_half_up(16LL * ((long long)Stt * QQ - (long long)St * St), QQ * QQ);
  const int flags = ((p == 0 || p == np - 1 || t == 0 || t == T - 1) ? TPC_CL_EDGE : 0) |
                    (excl ? TPC_CL_EXCLUDED : 0) | (other ? TPC_CL_NEIGHBOUR : 0);
  rec.x = (uint32_t)(pad_fp & 0xffff) | ((uint32_t)(time_fp & 0xffff) << 16);
  rec.y = (uint32_t)S.plane[tt * stride + p] | ((uint32_t)min(Q, 65535) << 16);
  rec.z = (uint32_t)min(vp, 255LL) | ((uint32_t)min(vt, 255LL) << 8) | ((uint32_t)flags << 16) |
          ((uint32_t)r << 24);
  rec.w = (uint32_t)t | ((uint32_t)p << 16) | ((uint32_t)s << 24);
  xyz = make_int4(xrow, 2 * (pad_fp - 128 * (np - 1)), 5 * (32768 * f + time_fp - 512), t);
}

__global__ void __launch_bounds__(kFindThreads, 2)
k_find_clusters(DevGeom G, DevParams P, DevWork W, unsigned int n_windows) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int stride = G.npmax, nw = G.nw;
  const int nrow_words = (kWinT - 2) * nw;   // plane rows 1 .. 260
  const int nown_words = kFrag * nw;         // plane rows 3 .. 258
  FindSmem S;
  {
    size_t o = 0;
    S.plane = reinterpret_cast<uint16_t*>(smem_raw + o);
    o += ((size_t)kWinT * stride * 2 + 15) & ~(size_t)15;
    S.occ = reinterpret_cast<uint32_t*>(smem_raw + o);
    o += (size_t)kWinT * nw * 4;
    S.pk = reinterpret_cast<uint32_t*>(smem_raw + o);
    o += (size_t)kWinT * nw * 4;
    o = (o + 15) & ~(size_t)15;
    S.st_rec = reinterpret_cast<uint4*>(smem_raw + o);
    o += kStage * 16;
    S.st_xyz = reinterpret_cast<int4*>(smem_raw + o);
    o += kStage * 16;
    S.scan = reinterpret_cast<unsigned long long*>(smem_raw + o);
    o += 34 * 8;
    S.ent_rs = reinterpret_cast<int32_t*>(smem_raw + o);
    o += 260 * 4;
    S.misc = reinterpret_cast<int32_t*>(smem_raw + o);
    o += 16 * 4;
    S.wpre = reinterpret_cast<uint16_t*>(smem_raw + o);
    o += ((size_t)nrow_words + 1) * 2;
    S.ppre = reinterpret_cast<uint16_t*>(smem_raw + o);
    o += ((size_t)nown_words + 1) * 2;
    S.ent_t = reinterpret_cast<uint8_t*>(smem_raw + o);
  }
  const int tid = threadIdx.x;
  const int wpt = (nrow_words + blockDim.x - 1) / blockDim.x;
  const int opt = (nown_words + blockDim.x - 1) / blockDim.x;

  while (true) {
    if (tid == 0) S.misc[0] = (int)atomicAdd(&W.tickets[TK_FIND], 1u);
    // clear the occupancy bitmap
    for (int i = tid; i < kWinT * nw; i += blockDim.x) S.occ[i] = 0u;
    __syncthreads();
    const unsigned int w = (unsigned int)S.misc[0];
    if (w >= n_windows) break;
    const int f = (int)(w % G.n_frag);
    const int sr = (int)(w / G.n_frag);
    const int r = sr % G.n_rows, s = sr / G.n_rows;
    const int np = G.npads[r];
    const int T = G.n_time_bins;

    // ---- 1. decode own page and the neighbours' halos
    PageHdr h;
    uint64_t off = W.page_offsets[w];
    bool ok = read_header(W, off, h) && h.sector == s && h.row == r && h.frag == f;
    ok = __syncthreads_and(ok);
    if (ok) ok = decode_segment(W.pages + off, h, 0, h.n_tb, 0, 0, kHalo, np, stride, nw, kFrag * f, T,
                                true, S);
    if (f > 0) {
      PageHdr hp;
      uint64_t offp = W.page_offsets[w - 1];
      bool okp = __syncthreads_and(read_header(W, offp, hp));
      if (okp)
        decode_segment(W.pages + offp, hp, hp.hi_tb, hp.n_tb, hp.hi_runs, hp.hi_dig, kHalo - kFrag, np,
                       stride, nw, kFrag * (f - 1), T, false, S);
    }
    if (f + 1 < G.n_frag) {
      PageHdr hn;
      uint64_t offn = W.page_offsets[w + 1];
      bool okn = __syncthreads_and(read_header(W, offn, hn));
      if (okn)
        decode_segment(W.pages + offn, hn, 0, hn.lo_tb, 0, 0, kHalo + kFrag, np, stride, nw, kFrag * (f + 1),
                       T, false, S);
    }
    if (!ok && tid == 0) atomicOr(W.err, kErrCorrupt);

    // ---- 2. rank the digits of rows 1..260 (popcount prefix over the bitmap words)
    int ndig = 0;
    {
      const int w0 = tid * wpt, w1 = min(w0 + wpt, nrow_words);
      int c = 0;
      for (int i = w0; i < w1; i++) c += __popc(S.occ[nw + i]);
      unsigned long long tot;
      unsigned long long pre = block_excl_scan((unsigned long long)c, S.scan, &tot);
      int run = (int)pre;
      for (int i = w0; i < w1; i++) { S.wpre[i] = (uint16_t)run; run += __popc(S.occ[nw + i]); }
      if (tid == 0) S.wpre[nrow_words] = (uint16_t)tot;
      // the pk words of rows 1..260 are rebuilt by atomicOr below
      for (int i = w0; i < w1; i++) S.pk[nw + i] = 0u;
      ndig = ok ? (int)tot : 0;
    }
    __syncthreads();

    // ---- 3. peak test, one digit per thread (balanced)
    for (int rk = tid; rk < ndig; rk += blockDim.x) {
      const int wi_ = rank_search(S.wpre, nrow_words + 1, rk);
      const uint32_t word = S.occ[nw + wi_];
      const int bit = __fns(word, 0, rk - (int)S.wpre[wi_] + 1);
      const int tt = 1 + wi_ / nw, p = (wi_ % nw) * 32 + bit;
      const int q = S.plane[tt * stride + p];
      if (q >= P.q_peak_min && peak_test(S, stride, nw, np, tt, p, q)) atomicOr(&S.pk[tt * nw + (p >> 5)], 1u << bit);
    }
    __syncthreads();

    // ---- 4. rank the own peaks (rows 3..258) and publish the window's count
    int npk;
    {
      const int w0 = tid * opt, w1 = min(w0 + opt, nown_words);
      int c = 0;
      for (int i = w0; i < w1; i++) c += __popc(S.pk[kHalo * nw + i]);
      unsigned long long tot;
      unsigned long long pre = block_excl_scan((unsigned long long)c, S.scan, &tot);
      int run = (int)pre;
      for (int i = w0; i < w1; i++) { S.ppre[i] = (uint16_t)run; run += __popc(S.pk[kHalo * nw + i]); }
      if (tid == 0) {
        S.ppre[nown_words] = (uint16_t)tot;
        lookback_publish(W.win_state, (long long)w, tot);
      }
      npk = (int)tot;
    }
    __syncthreads();

    // ---- 5. clusters of the first kStage peaks, staged in shared memory
    const int nst = min(npk, kStage);
    for (int k = tid; k < nst; k += blockDim.x) {
      const int wi_ = rank_search(S.ppre, nown_words + 1, k);
      const uint32_t word = S.pk[kHalo * nw + wi_];
      const int bit = __fns(word, 0, k - (int)S.ppre[wi_] + 1);
      const int tt = kHalo + wi_ / nw, p = (wi_ % nw) * 32 + bit;
      make_cluster(S, stride, nw, np, T, s, r, f, tt, p, G.xrow[r], S.st_rec[k], S.st_xyz[k]);
    }

    // ---- 6. global offset of this window (decoupled look-back)
    if (tid < 32) {
      const unsigned long long base = lookback_wait(W.win_state, (long long)w, (unsigned long long)npk, W.err);
      if (tid == 0) {
        S.scan[33] = base;
        // row starts are clamped to the capacity so that, after an overflow,
        // every later kernel still indexes inside the cluster arrays
        if (f == 0) W.row_start[sr] = (uint32_t)min(base, (unsigned long long)W.cap_cl);
        if (w == n_windows - 1) {
          W.row_start[G.n_sectors * G.n_rows] = (uint32_t)min(base + npk, (unsigned long long)W.cap_cl);
          W.ctr[CTR_NCL] = base + npk;
        }
        if (base + npk > W.cap_cl) atomicOr(W.err, kErrOverflowCl);
      }
    }
    __syncthreads();
    const unsigned long long base = S.scan[33];

    // ---- 7. write out (coalesced), then any peaks beyond the staging buffer
    for (int k = tid; k < npk; k += blockDim.x) {
      const unsigned long long idx = base + k;
      if (idx >= W.cap_cl) break;   // overflow: keep [0, cap) free of gaps, drop the rest
      uint4 rec;
      int4 xyz;
      if (k < kStage) {
        rec = S.st_rec[k];
        xyz = S.st_xyz[k];
      } else {
        const int wi_ = rank_search(S.ppre, nown_words + 1, k);
        const uint32_t word = S.pk[kHalo * nw + wi_];
        const int bit = __fns(word, 0, k - (int)S.ppre[wi_] + 1);
        make_cluster(S, stride, nw, np, T, s, r, f, kHalo + wi_ / nw, (wi_ % nw) * 32 + bit, G.xrow[r], rec, xyz);
      }
      reinterpret_cast<uint4*>(W.clusters)[idx] = rec;
      W.cl_x[idx] = xyz.x;
      W.cl_y[idx] = xyz.y;
      W.cl_z[idx] = xyz.z;
      W.cl_t[idx] = xyz.w;
    }
    __syncthreads();
  }
}

size_t find_smem_bytes(int npmax, int nw) {
  size_t o = ((size_t)kWinT * npmax * 2 + 15) & ~(size_t)15;
  o += 2 * (size_t)kWinT * nw * 4;
  o = (o + 15) & ~(size_t)15;
  o += 2 * kStage * 16 + 34 * 8 + 260 * 4 + 16 * 4;
  o += ((size_t)(kWinT - 2) * nw + 1) * 2 + ((size_t)kFrag * nw + 1) * 2;
  o += 256;
  return o;
}

cudaError_t launch_find(const DevGeom& G, const DevParams& P, const DevWork& W, unsigned int n_windows,
                        int n_sm, cudaStream_t st) {
  size_t sm = find_smem_bytes(G.npmax, G.nw);
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(k_find_clusters, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  unsigned int grid = (unsigned int)min((long long)n_windows, (long long)n_sm * 2);
  if (grid == 0) grid = 1;
  k_find_clusters<<<grid, kFindThreads, sm, st>>>(G, P, W, n_windows);
  return cudaGetLastError();
}

}  // namespace tpc
