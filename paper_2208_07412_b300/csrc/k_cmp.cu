// k_cmp.cu — optional track-model compression of the clusters on tracks
// (step 10 of the library's definition; the paper's section "Hardware and data
// flow" gives the online reconstruction as the means to reduce the TPC data).
//
// Per step-8 track, one thread: the fitted parameters at the innermost cluster
// are carried along the exact helix from row to row (predicted state only);
// each cluster's measured (y, zeta) minus the prediction at its row, divided
// by the step and rounded (ties away from zero), is its pair of 8-bit codes
// when both are within +-127; otherwise, and after a failed transport, the
// cluster is escaped (kept raw).  Decoding adds code * step to the prediction,
// so a coded position is within half a step of the measured one.
#include "fit_common.cuh"

namespace tpc {

__global__ void k_compress(DevParams P, DevWork W, CmpWork C) {
  unsigned long long ntrk = W.ctr[CTR_NTRK];
  if (ntrk > W.cap_ch) ntrk = W.cap_ch;
  unsigned coded = 0, escaped = 0;
  const float iy = 1.f / C.step_y, iz = 1.f / C.step_z;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < ntrk;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const int n = W.trk_ncl[t];
    const int4* pts = W.trk_xyz + W.trk_off[t];   // innermost first
    const tpc_track& tr = W.tracks[t];
    float s[5] = {tr.par[0], tr.par[1], tr.par[2], tr.par[3], tr.par[4]};
    float x = tr.x;
    bool ok = true;
    for (int i = 0; i < n; i++) {
      const int4 p = pts[i];
      const float xc = (float)p.x * kU;
      if (ok && xc != x) {
        Jac<float> J;
        if (transport(P.kfac, s, xc - x, J)) x = xc; else ok = false;
      }
      uint8_t st = 2;
      if (ok) {
        const float cy = roundf(((float)p.y * kU - s[0]) * iy), cz = roundf(((float)p.z * kU - s[1]) * iz);
        if (fabsf(cy) <= 127.f && fabsf(cz) <= 127.f) {
          C.code_y[p.w] = (int8_t)cy;
          C.code_z[p.w] = (int8_t)cz;
          st = 1;
        }
      }
      C.status[p.w] = st;
      if (st == 1) coded++; else escaped++;
    }
  }
  coded = __reduce_add_sync(0xffffffffu, coded);
  escaped = __reduce_add_sync(0xffffffffu, escaped);
  if ((threadIdx.x & 31) == 0) {
    if (coded) atomicAdd(&C.ctl[0], (unsigned long long)coded);
    if (escaped) atomicAdd(&C.ctl[1], (unsigned long long)escaped);
  }
}

cudaError_t launch_compress(const DevParams& P, const DevWork& W, const CmpWork& C, int n_sm, cudaStream_t st) {
  unsigned long long g = (W.cap_ch + 63) / 64;
  const unsigned long long m = (unsigned long long)n_sm * 16;
  if (g > m) g = m;
  k_compress<<<(unsigned)(g ? g : 1), 64, 0, st>>>(P, W, C);
  return cudaGetLastError();
}

}  // namespace tpc

// ---------------------------------------------------------------------------
// Optional drift calibration (step 11 of the library's definition; the paper
// lists calibration among the EPNs' tasks, "Hardware and data flow").  Per
// step-8 track with >= 20 clusters and no flag: its state carried along the
// exact helix to x = 0 (the beam axis), used if |y| < 3 cm there; t_v = zeta /
// (zeta per time bin).  The mode of floor(t_v) over 2^20 bins (lowest bin on
// ties) seeds a mean over |t_v - (b* + 0.5)| <= 3, then one over |t_v - mean|
// <= 1.5.  Sums in FP64 atomics (order-dependent only in the last bits).
namespace tpc {

constexpr int kCalBins = 1 << 20;

__global__ void k_calib_tracks(DevParams P, DevWork W, CalWork C) {
  unsigned long long ntrk = W.ctr[CTR_NTRK];
  if (ntrk > W.cap_ch) ntrk = W.cap_ch;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < ntrk;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const tpc_track& tr = W.tracks[t];
    float tv = -1.f;
    if (tr.n_clusters >= 20 && tr.flags == 0) {
      float s[5] = {tr.par[0], tr.par[1], tr.par[2], tr.par[3], tr.par[4]};
      Jac<float> J;
      if (transport(P.kfac, s, -tr.x, J) && fabsf(s[0]) < 3.f) tv = s[1] / C.zeta_per_bin;
    }
    C.tv[t] = tv;
    if (tv >= 0.f && tv < (float)kCalBins) atomicAdd(&C.hist[(int)floorf(tv)], 1u);
  }
}

// Mode: key = count << 32 | (kCalBins - 1 - bin), maximised (lowest bin on ties).
__global__ void k_calib_mode(CalWork C) {
  unsigned long long best = 0;
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < kCalBins; b += gridDim.x * blockDim.x) {
    const unsigned n = C.hist[b];
    if (n) best = max(best, ((unsigned long long)n << 32) | (unsigned)(kCalBins - 1 - b));
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0 && best) atomicMax(C.mode, best);
}

__global__ void k_calib_mean(DevWork W, CalWork C, int pass) {
  unsigned long long ntrk = W.ctr[CTR_NTRK];
  if (ntrk > W.cap_ch) ntrk = W.cap_ch;
  double centre, win;
  if (pass == 0) {
    const unsigned long long m = *C.mode;
    if (!m) return;
    centre = (double)(kCalBins - 1 - (int)(unsigned)m) + 0.5;
    win = 3.0;
  } else {
    if (C.cnt[0] == 0) return;
    centre = C.sum[0] / (double)C.cnt[0];
    win = 1.5;
  }
  double s = 0.0;
  unsigned n = 0;
  for (unsigned long long t = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; t < ntrk;
       t += (unsigned long long)gridDim.x * blockDim.x) {
    const float tv = C.tv[t];
    if (tv >= 0.f && fabs((double)tv - centre) <= win) { s += (double)tv; n++; }
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, o);
    n += __shfl_xor_sync(0xffffffffu, n, o);
  }
  if ((threadIdx.x & 31) == 0 && n) {
    atomicAdd(&C.sum[pass], s);
    atomicAdd(&C.cnt[pass], (unsigned long long)n);
  }
}

cudaError_t launch_calibrate(const DevParams& P, const DevWork& W, const CalWork& C, int n_sm, cudaStream_t st) {
  unsigned long long g = (W.cap_ch + 255) / 256;
  const unsigned long long m = (unsigned long long)n_sm * 8;
  if (g > m) g = m;
  k_calib_tracks<<<(unsigned)(g ? g : 1), 256, 0, st>>>(P, W, C);
  k_calib_mode<<<n_sm * 4, 256, 0, st>>>(C);
  k_calib_mean<<<(unsigned)(g ? g : 1), 256, 0, st>>>(W, C, 0);
  k_calib_mean<<<(unsigned)(g ? g : 1), 256, 0, st>>>(W, C, 1);
  return cudaGetLastError();
}

}  // namespace tpc

// ---------------------------------------------------------------------------
// Optional entropy coding of the step-10 codes (step 10c of the library's
// definition): per component (y, z) a canonical Huffman code over the 256
// symbols code + 128 of the coded clusters, lengths limited to 24 bits, and
// the stream of the coded clusters' codewords in cluster order (y then z,
// most significant bit first, stream bit b in bit 31 - b % 32 of word b / 32).
// Tie rules of the code construction: the leaves ordered by (count, symbol)
// form one queue, the merged nodes a second in creation order, and each merge
// takes the lighter head twice, a leaf before a node of equal weight; over
// 24 bits every count c becomes (c + 1) / 2 and the code is built again.
namespace tpc {

constexpr int kMaxCodeLen = 24;

__global__ void k_ent_hist(DevWork W, CmpWork C, EntWork E) {
  __shared__ unsigned int h[512];
  for (int i = threadIdx.x; i < 512; i += blockDim.x) h[i] = 0;
  __syncthreads();
  unsigned long long n = W.ctr[CTR_NCL];
  if (n > W.cap_cl) n = W.cap_cl;
  // most codes fall in a few bins: lanes holding the same symbol add once
  // (their leader adds their number), so the shared counters see few atomics
  const unsigned long long n_pad = (n + 31) & ~31ull;
  const int lane = threadIdx.x & 31;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n_pad;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const bool coded = i < n && C.status[i] == 1;
    const int sy = coded ? (int)C.code_y[i] + 128 : -1, sz = coded ? 256 + (int)C.code_z[i] + 128 : -1;
    const unsigned my = __match_any_sync(0xffffffffu, sy), mz = __match_any_sync(0xffffffffu, sz);
    if (coded && (__ffs(my) - 1) == lane) atomicAdd(&h[sy], (unsigned)__popc(my));
    if (coded && (__ffs(mz) - 1) == lane) atomicAdd(&h[sz], (unsigned)__popc(mz));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 512; i += blockDim.x)
    if (h[i]) atomicAdd(&E.hist[i], (unsigned long long)h[i]);
}

// One block of 256 threads, one symbol per thread: the leaves sorted by rank,
// the merges by thread 0, the depths by every leaf walking up, then the
// canonical codewords by thread 0.
__global__ void __launch_bounds__(256) k_ent_tables(EntWork E) {
  __shared__ unsigned long long w[512];
  __shared__ int leaves[256], parent[512];
  __shared__ int maxlen;
  const int s = threadIdx.x;
  for (int comp = 0; comp < 2; comp++) {
    unsigned long long c = E.hist[256 * comp + s];
    int len = 0;
    while (true) {
      __syncthreads();
      // rank of this leaf in (count, symbol) order
      w[s] = c;
      parent[s] = parent[256 + s] = -1;
      if (s == 0) maxlen = 0;
      const int n = __syncthreads_count(c != 0);
      if (c) {
        int rank = 0;
        for (int j = 0; j < 256; j++) {
          const unsigned long long cj = w[j];
          rank += cj != 0 && (cj < c || (cj == c && j < s));
        }
        leaves[rank] = s;
      }
      __syncthreads();
      if (s == 0 && n >= 2) {
        int qa = 0, qb = 256, nb = 256;
        for (int m = 0; m < n - 1; m++) {
          int pick[2];
          for (int k = 0; k < 2; k++) {
            bool take_a;
            if (qa >= n) take_a = false;
            else if (qb >= nb) take_a = true;
            else take_a = w[leaves[qa]] <= w[qb];
            pick[k] = take_a ? leaves[qa++] : qb++;
          }
          w[nb] = w[pick[0]] + w[pick[1]];
          parent[pick[0]] = parent[pick[1]] = nb;
          nb++;
        }
      }
      __syncthreads();
      len = 0;
      if (c) {
        if (n == 1) len = 1;
        else for (int x = s; parent[x] >= 0; x = parent[x]) len++;
        atomicMax(&maxlen, len);
      }
      __syncthreads();
      if (maxlen <= kMaxCodeLen) break;   // block-uniform
      if (c) c = (c + 1) / 2;
    }
    E.len[256 * comp + s] = (uint8_t)len;
    leaves[s] = len;                      // the lengths, for thread 0
    __syncthreads();
    if (s == 0) {
      uint32_t next = 0;
      int prev = 0;
      bool first = true;
      for (int l = 1; l <= kMaxCodeLen; l++)
        for (int j = 0; j < 256; j++) {
          if (leaves[j] != l) continue;
          next = first ? 0u : (next + 1u) << (l - prev);
          first = false;
          prev = l;
          E.code[256 * comp + j] = next;
        }
    }
  }
}

// Bits of each cluster's codewords (0 unless coded), scanned afterwards.
__global__ void k_ent_bits(DevWork W, CmpWork C, EntWork E) {
  unsigned long long n = W.ctr[CTR_NCL];
  if (n > W.cap_cl) n = W.cap_cl;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x)
    E.bits[i] = C.status[i] == 1 ? (uint64_t)E.len[(int)C.code_y[i] + 128] + E.len[256 + (int)C.code_z[i] + 128] : 0ull;
}

// Each coded cluster ORs its (at most 48) bits into the zeroed stream at its
// offset; bits of different clusters never overlap.
__global__ void k_ent_pack(DevWork W, CmpWork C, EntWork E) {
  unsigned long long n = W.ctr[CTR_NCL];
  if (n > W.cap_cl) n = W.cap_cl;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    if (C.status[i] != 1) continue;
    const int sy = (int)C.code_y[i] + 128, sz = 256 + (int)C.code_z[i] + 128;
    const int lz = E.len[sz];
    int L = E.len[sy] + lz;
    const unsigned long long v = ((unsigned long long)E.code[sy] << lz) | E.code[sz];
    unsigned long long b = E.bits[i];
    while (L > 0) {
      const unsigned long long wi = b >> 5;
      const int room = 32 - (int)(b & 31);
      const int take = min(room, L);
      const uint32_t part = (uint32_t)((v >> (L - take)) & ((1ull << take) - 1ull));
      if (wi < E.cap_words) atomicOr(&E.words[wi], part << (room - take));
      L -= take;
      b += take;
    }
  }
}

cudaError_t launch_scan(uint64_t* v, const unsigned long long* n_ptr, unsigned long long cap,
                        unsigned long long* state, unsigned int* ticket, unsigned long long* total, uint32_t* err,
                        int n_sm, cudaStream_t st);

// Step 10c on the codes in C: histogram, tables, bit offsets, stream.  The
// caller has zeroed E.hist, E.scan_state, E.ticket and E.words.
cudaError_t launch_entropy(const DevWork& W, const CmpWork& C, const EntWork& E, int n_sm, cudaStream_t st) {
  unsigned long long g = (W.cap_cl + 255) / 256;
  const unsigned long long m = (unsigned long long)n_sm * 8;
  if (g > m) g = m;
  const unsigned grid = (unsigned)(g ? g : 1);
  k_ent_hist<<<grid, 256, 0, st>>>(W, C, E);
  k_ent_tables<<<1, 256, 0, st>>>(E);
  k_ent_bits<<<grid, 256, 0, st>>>(W, C, E);
  cudaError_t e = launch_scan(E.bits, W.ctr + CTR_NCL, W.cap_cl, E.scan_state, E.ticket, E.total, W.err, n_sm, st);
  if (e != cudaSuccess) return e;
  k_ent_pack<<<grid, 256, 0, st>>>(W, C, E);
  return cudaGetLastError();
}

}  // namespace tpc
