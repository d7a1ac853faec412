/*
 * oracle.c — plain, slow CPU oracle of the TPC timeframe reconstruction.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this code; the library never does.  It
 * shares no code, header, table or constant with the CUDA path.
 *
 * The paper (section "Hardware and data flow") says only that the EPN GPUs run
 * the full online TPC track reconstruction on zero-suppressed data; it defines
 * none of the algorithms.  This file therefore writes out, step by step and in
 * the plainest form, the definition the library documents: ZS decode, 3x3 peak
 * test under a total order, 5x5 cluster moments, integer CA neighbour search by
 * brute force over all candidate pairs, mutual links and chains, integer
 * segment merge, and the FP64 Kalman helix fit.  Integers are exact; the fit is
 * double precision.  No blocking, fusion or reordering beyond the definition.
 * The CA and merge searches visit candidates in the definition's order but skip
 * index ranges that a bound proves are rejected (a candidate window in time
 * bins, see ca_time_window and the merge); search_all = 1 visits every
 * candidate, and the tests check that the two give identical results.
 *
 * Pins (tests, not this file): ZS round trip, peak finder against a 3x3
 * maximum filter, centroid closed forms, CA special cases and hand-worked
 * examples, merge gap closure, fit closure on exact helices, Jacobian against
 * finite differences, Kalman update against the information form, pulls.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------ data types */
typedef struct {
  int32_t n_sectors, n_rows;
  const int32_t* npads;
  const int32_t* row_x;       /* 0.05 cm units */
  int32_t n_time_bins;
  const uint8_t* pages;
  uint64_t pages_bytes;
  const uint64_t* page_offsets;
} orc_input;

typedef struct {
  int32_t q_peak_min;
  int32_t sy_num, sy_den, sz_num, sz_den;
  int32_t ca_cut;
  int32_t min_chain;
  int32_t merge_cut, gap_min, gap_max, merge_passes;
  int32_t min_track;
  int32_t fit_passes;
  int32_t ns_min_dip;   /* 5x5 noise suppression: 0 off, else the minimum dip in ADC */
  double bz, sigma_y, sigma_z;
  double c0[5];
  int32_t search_all;   /* 1: CA and merge visit every candidate (no window) */
  int32_t split_charge; /* 1: step 3s, charge of pixels near several peaks is shared */
} orc_params;

/* 16-byte cluster record, field for field as documented by the library. */
typedef struct {
  uint16_t pad_fp, time_fp, qmax, qtot;
  uint8_t sigma2_pad, sigma2_time, flags, row;
  uint16_t t_peak;
  uint8_t pad_peak, sector;
} orc_cluster;

typedef struct {
  double par[5];   /* y, zeta, snp, tgl_zeta, q/pT (absolute y, zeta) */
  double x;
  double cov[15];
  double chi2;
  int32_t ndf, n_used, flags, pad;
} orc_fit;

#define ORC_E_CORRUPT (-5)

/* ------------------------------------------------------------ helpers */
static uint32_t rd16(const uint8_t* p) { return (uint32_t)p[0] | ((uint32_t)p[1] << 8); }
static uint32_t rd32(const uint8_t* p) {
  return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
/* R(a, b) = floor((2a + b) / (2b)) for b > 0: division rounding half up */
static int64_t round_div(int64_t a, int64_t b) {
  int64_t n = 2 * a + b, d = 2 * b;
  int64_t q = n / d;
  if ((n % d != 0) && ((n < 0) != (d < 0))) q -= 1;
  return q;
}
static int64_t iabs64(int64_t v) { return v < 0 ? -v : v; }

/* ------------------------------------------------------------ 1. decode */
/* Decode every page of (sector s, row r) into the dense plane q[t * npads + p]
 * (zero where there is no digit).  Returns 0 or ORC_E_CORRUPT. */
int orc_decode_row(const orc_input* in, int s, int r, uint16_t* plane) {
  int np = in->npads[r];
  int T = in->n_time_bins;
  int nf = (T + 255) / 256;
  memset(plane, 0, sizeof(uint16_t) * (size_t)T * np);
  for (int f = 0; f < nf; f++) {
    uint64_t off = in->page_offsets[((int64_t)s * in->n_rows + r) * nf + f];
    if (off % 16 != 0 || off + 32 > in->pages_bytes) return ORC_E_CORRUPT;
    const uint8_t* pg = in->pages + off;
    uint32_t len = rd32(pg);
    uint32_t n_tb = rd16(pg + 4), n_runs = rd16(pg + 6), n_dig = rd16(pg + 8);
    if (rd16(pg + 14) != 0x5A53u || pg[10] != s || pg[11] != r || rd16(pg + 12) != (uint32_t)f)
      return ORC_E_CORRUPT;
    uint64_t body = 32 + 2 * (uint64_t)n_tb + 2 * (uint64_t)n_runs;
    body = (body + 3) & ~(uint64_t)3;
    if (len % 16 != 0 || off + len > in->pages_bytes || body + 4 * (((uint64_t)n_dig + 2) / 3) > len)
      return ORC_E_CORRUPT;
    const uint8_t* ent = pg + 32;
    const uint8_t* run = ent + 2 * n_tb;
    const uint8_t* adcw = pg + body;
    uint32_t ri = 0, di = 0;
    int last_t = -1;
    for (uint32_t e = 0; e < n_tb; e++) {
      int t_in = ent[2 * e], nr = ent[2 * e + 1];
      int t = 256 * f + t_in;
      if (t_in <= last_t || nr < 1 || t >= T) return ORC_E_CORRUPT;
      last_t = t_in;
      int last_end = -1;
      for (int k = 0; k < nr; k++, ri++) {
        if (ri >= n_runs) return ORC_E_CORRUPT;
        int ps = run[2 * ri], ln = run[2 * ri + 1];
        if (ln < 1 || ps < last_end || ps + ln > np) return ORC_E_CORRUPT;
        last_end = ps + ln;
        for (int i = 0; i < ln; i++, di++) {
          if (di >= n_dig) return ORC_E_CORRUPT;
          uint32_t w = rd32(adcw + 4 * (di / 3));
          plane[(size_t)t * np + ps + i] = (uint16_t)((w >> (10 * (di % 3))) & 1023u);
        }
      }
    }
    if (ri != n_runs || di != n_dig) return ORC_E_CORRUPT;
  }
  return 0;
}

/* ------------------------------------------------------------ 2-3. peaks, clusters */
static int q_at(const uint16_t* plane, int np, int T, int p, int t) {
  if (p < 0 || p >= np || t < 0 || t >= T) return 0;
  return plane[(size_t)t * np + p];
}

/* key(c) > key(n) with key = (q, -(t*np + p)), lexicographic */
static int key_greater(int qc, int64_t lc, int qn, int64_t ln) {
  if (qc != qn) return qc > qn;
  return lc < ln;
}

static int is_peak(const uint16_t* plane, int np, int T, int p, int t, int qmin) {
  int q = q_at(plane, np, T, p, t);
  if (q < qmin) return 0;
  int64_t lc = (int64_t)t * np + p;
  for (int dt = -1; dt <= 1; dt++)
    for (int dp = -1; dp <= 1; dp++) {
      if (dp == 0 && dt == 0) continue;
      int pn = p + dp, tn = t + dt;
      int qn = q_at(plane, np, T, pn, tn);
      int64_t ln = (int64_t)tn * np + pn;
      if (!key_greater(q, lc, qn, ln)) return 0;
    }
  return 1;
}

static int sgn(int v) { return (v > 0) - (v < 0); }
static int imin(int a, int b) { return a < b ? a : b; }

/* Step 2b (optional noise suppression): the peak at (p, t) is dropped when some
 * other peak n of step 2, with a greater key, sits on the ring of its 5x5 window
 * (max(|dp|, |dt|) = 2) and the pixel m between them -- the inner pixel of the
 * cluster rule in n's direction -- lies less than min_dip ADC below the peak.
 * The test reads step 2's peak set, so it does not depend on any order. */
static int ns_suppressed(const uint16_t* plane, int np, int T, int p, int t, int qmin, int min_dip) {
  if (min_dip <= 0) return 0;
  int qc = q_at(plane, np, T, p, t);
  int64_t lc = (int64_t)t * np + p;
  for (int dt = -2; dt <= 2; dt++)
    for (int dp = -2; dp <= 2; dp++) {
      if (abs(dp) < 2 && abs(dt) < 2) continue;          /* ring only */
      int pn = p + dp, tn = t + dt;
      if (pn < 0 || pn >= np || tn < 0 || tn >= T) continue;
      if (!is_peak(plane, np, T, pn, tn, qmin)) continue;
      if (!key_greater(q_at(plane, np, T, pn, tn), (int64_t)tn * np + pn, qc, lc)) continue;
      int qm = q_at(plane, np, T, p + sgn(dp) * imin(abs(dp), 1), t + sgn(dt) * imin(abs(dt), 1));
      if (qc - qm < min_dip) return 1;
    }
  return 0;
}

/* Step 3s (optional charge splitting).  The owners O(x) of a pixel x are the
 * step-2 peaks j at Chebyshev distance max(|p_x - p_j|, |t_x - t_j|) <= 1 from
 * x if there is any, else those at distance <= 2 (x then lies only on the
 * outer rings of their 5x5 windows).  Cluster c counts the charge of an
 * included pixel x as its share
 *     w_c(x) = floor(q(x) q(c) / sum_{j in O(x)} q(j))   if c is in O(x),
 *     w_c(x) = 0                                          otherwise,
 * so x's charge goes to the peaks whose cores hold it, in proportion to their
 * heights, and the shares of all clusters never add up to more than q(x).  A
 * peak is alone in its own 3x3 (peaks are never adjacent), so w_c(c) = q(c).
 * Returns w_c(x) for the peak c = (pc, tc) and the pixel x = (px, pt). */
static int split_share(const uint16_t* plane, int np, int T, int px, int pt, int pc, int tc, int qmin) {
  int q = q_at(plane, np, T, px, pt);
  if (q == 0) return 0;
  for (int d = 1; d <= 2; d++) {
    int64_t sum = 0;
    int c_in = 0, any = 0;
    for (int dt = -d; dt <= d; dt++)
      for (int dp = -d; dp <= d; dp++) {
        int pj = px + dp, tj = pt + dt;
        if (pj < 0 || pj >= np || tj < 0 || tj >= T) continue;
        if (!is_peak(plane, np, T, pj, tj, qmin)) continue;
        any = 1;
        sum += q_at(plane, np, T, pj, tj);
        if (pj == pc && tj == tc) c_in = 1;
      }
    if (any) return c_in ? (int)(((int64_t)q * q_at(plane, np, T, pc, tc)) / sum) : 0;
  }
  return 0;   /* unreachable for x in the 5x5 window of the peak c */
}

static orc_cluster make_cluster(const uint16_t* plane, int np, int T, int s, int r, int p, int t,
                                int qmin, int split) {
  int64_t Q = 0, Sp = 0, St = 0, Spp = 0, Stt = 0;
  int excluded = 0, other_peak = 0, shared = 0;
  for (int dt = -2; dt <= 2; dt++)
    for (int dp = -2; dp <= 2; dp++) {
      int q = q_at(plane, np, T, p + dp, t + dt);
      int inc;
      if (abs(dp) <= 1 && abs(dt) <= 1) {
        inc = 1;
      } else {
        int ip = sgn(dp) * imin(abs(dp), 1), it = sgn(dt) * imin(abs(dt), 1);
        int qi = q_at(plane, np, T, p + ip, t + it);
        inc = (qi > 0) && (q <= qi);
        if (!inc && q > 0) excluded = 1;
      }
      if (inc && split && q > 0) {
        int w = split_share(plane, np, T, p + dp, t + dt, p, t, qmin);
        if (w != q) shared = 1;
        q = w;
      }
      if (inc) {
        Q += q; Sp += (int64_t)q * dp; St += (int64_t)q * dt;
        Spp += (int64_t)q * dp * dp; Stt += (int64_t)q * dt * dt;
      }
      if ((dp || dt) && p + dp >= 0 && p + dp < np && t + dt >= 0 && t + dt < T &&
          is_peak(plane, np, T, p + dp, t + dt, qmin))
        other_peak = 1;
    }
  int f = t / 256;
  orc_cluster c;
  c.pad_fp = (uint16_t)(256 * p + round_div(256 * Sp, Q));
  c.time_fp = (uint16_t)(128 * (t - 256 * f + 4) + round_div(128 * St, Q));
  int64_t vp = round_div(16 * (Spp * Q - Sp * Sp), Q * Q);
  int64_t vt = round_div(16 * (Stt * Q - St * St), Q * Q);
  c.sigma2_pad = (uint8_t)(vp > 255 ? 255 : vp);
  c.sigma2_time = (uint8_t)(vt > 255 ? 255 : vt);
  c.qmax = (uint16_t)q_at(plane, np, T, p, t);
  c.qtot = (uint16_t)(Q > 65535 ? 65535 : Q);
  c.flags = 0;
  if (p == 0 || p == np - 1 || t == 0 || t == T - 1) c.flags |= 1;
  if (excluded) c.flags |= 2;
  if (other_peak) c.flags |= 4;
  if (shared) c.flags |= 8;
  c.row = (uint8_t)r;
  c.t_peak = (uint16_t)t;
  c.pad_peak = (uint8_t)p;
  c.sector = (uint8_t)s;
  return c;
}

/* Clusters of the whole timeframe in canonical order (sector, row, t, p).
 * out may be NULL (count only).  Returns the count, or ORC_E_CORRUPT. */
int64_t orc_find_clusters(const orc_input* in, const orc_params* P, orc_cluster* out, int64_t cap) {
  int npmax = 0;
  for (int r = 0; r < in->n_rows; r++) if (in->npads[r] > npmax) npmax = in->npads[r];
  uint16_t* plane = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)in->n_time_bins * npmax + 2);
  int64_t n = 0;
  for (int s = 0; s < in->n_sectors; s++)
    for (int r = 0; r < in->n_rows; r++) {
      int np = in->npads[r], T = in->n_time_bins;
      if (orc_decode_row(in, s, r, plane) != 0) { free(plane); return ORC_E_CORRUPT; }
      for (int t = 0; t < T; t++)
        for (int p = 0; p < np; p++)
          if (is_peak(plane, np, T, p, t, P->q_peak_min) &&
              !ns_suppressed(plane, np, T, p, t, P->q_peak_min, P->ns_min_dip)) {
            if (out && n < cap) out[n] = make_cluster(plane, np, T, s, r, p, t, P->q_peak_min, P->split_charge);
            n++;
          }
    }
  free(plane);
  return n;
}

/* Dense decoded planes of a whole timeframe, [sector][row][t][pad] with pads
 * padded to npmax; for tests. */
int orc_decode_all(const orc_input* in, uint16_t* out, int npmax) {
  uint16_t* plane = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)in->n_time_bins * npmax + 2);
  for (int s = 0; s < in->n_sectors; s++)
    for (int r = 0; r < in->n_rows; r++) {
      int np = in->npads[r];
      if (orc_decode_row(in, s, r, plane) != 0) { free(plane); return ORC_E_CORRUPT; }
      uint16_t* o = out + ((size_t)s * in->n_rows + r) * (size_t)in->n_time_bins * npmax;
      memset(o, 0, sizeof(uint16_t) * (size_t)in->n_time_bins * npmax);
      for (int t = 0; t < in->n_time_bins; t++)
        memcpy(o + (size_t)t * npmax, plane + (size_t)t * np, sizeof(uint16_t) * np);
    }
  free(plane);
  return 0;
}

/* Peak flags of one dense plane q[t * np + p] (tests). */
void orc_peaks_plane(const uint16_t* plane, int np, int T, int qmin, uint8_t* flags) {
  for (int t = 0; t < T; t++)
    for (int p = 0; p < np; p++) flags[(size_t)t * np + p] = (uint8_t)is_peak(plane, np, T, p, t, qmin);
}

/* Surviving peaks of step 2b on one dense plane (tests). */
void orc_peaks_plane_ns(const uint16_t* plane, int np, int T, int qmin, int min_dip, uint8_t* flags) {
  for (int t = 0; t < T; t++)
    for (int p = 0; p < np; p++)
      flags[(size_t)t * np + p] =
          (uint8_t)(is_peak(plane, np, T, p, t, qmin) && !ns_suppressed(plane, np, T, p, t, qmin, min_dip));
}

/* One cluster from a dense plane (tests). */
void orc_cluster_at(const uint16_t* plane, int np, int T, int p, int t, int qmin, int split, orc_cluster* out) {
  *out = make_cluster(plane, np, T, 0, 0, p, t, qmin, split);
}

/* Step 3s share w_c(x) of the pixel x = (px, pt) in the cluster of the peak
 * c = (pc, tc) of one dense plane (tests). */
int orc_split_share(const uint16_t* plane, int np, int T, int qmin, int pc, int tc, int px, int pt) {
  return split_share(plane, np, T, px, pt, pc, tc, qmin);
}

/* ------------------------------------------------------------ 4. coordinates */
/* Integer coordinates in u = 7.8125 um. */
void orc_coords(const orc_input* in, const orc_cluster* c, int64_t* X, int64_t* Y, int64_t* Z) {
  int np = in->npads[c->row];
  int f = c->t_peak / 256;
  *Y = 2 * ((int64_t)c->pad_fp - 128 * (int64_t)(np - 1));
  *Z = 5 * ((int64_t)128 * 256 * f + c->time_fp - 512);
  *X = 64 * (int64_t)in->row_x[c->row];
}

/* ------------------------------------------------------------ 5-6. CA */
/* First index i in [lo, hi) whose cluster has t_peak >= t (clusters of one
 * (sector, row) are in (t_peak, pad) order); hi if none. */
static int64_t first_t_at_least(const orc_cluster* cl, int64_t lo, int64_t hi, int64_t t) {
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if ((int64_t)cl[mid].t_peak < t) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/* Time-bin half width of the CA candidate window between rows dX apart.  Step
 * 4 gives Z = 640 t_peak + 5 R(128 St, Q) with |St| <= 2 Q, so |5 R| <= 1280 and
 * |Z_c - Z_d| >= 640 |t_c - t_d| - 2560.  A candidate passing the window test
 * |Z_c - Z_d| sz_den <= sz_num dX thus has |t_c - t_d| <= (sz_num dX / sz_den +
 * 2560) / 640; one bin more is kept for safety. */
static int64_t ca_time_window(const orc_params* P, int64_t dx) {
  return ((int64_t)P->sz_num * dx / P->sz_den + 2560) / 640 + 1;
}

/* up / down / best score for every cluster by brute force over all (d, u) pairs,
 * then mutual links and chains.  chain_of[c] = index of the lowest cluster of
 * the chain holding c if that chain has >= min_chain clusters, else -1. */
int orc_ca(const orc_input* in, const orc_params* P, const orc_cluster* cl, int64_t n,
           int32_t* up, int32_t* down, int32_t* chain_of) {
  int64_t *X = (int64_t*)malloc(sizeof(int64_t) * (n + 1)), *Y = (int64_t*)malloc(sizeof(int64_t) * (n + 1)),
          *Z = (int64_t*)malloc(sizeof(int64_t) * (n + 1)), *score = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
  for (int64_t i = 0; i < n; i++) { orc_coords(in, &cl[i], &X[i], &Y[i], &Z[i]); up[i] = down[i] = -1; score[i] = -1; }
  /* row ranges: clusters are in canonical order, so each (sector, row) is contiguous */
  int64_t nsr = (int64_t)in->n_sectors * in->n_rows;
  int64_t* rs = (int64_t*)calloc((size_t)nsr + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) rs[(int64_t)cl[i].sector * in->n_rows + cl[i].row + 1]++;
  for (int64_t b = 0; b < nsr; b++) rs[b + 1] += rs[b];
  const int R = in->n_rows;
  for (int s = 0; s < in->n_sectors; s++)
    for (int r = 1; r <= R - 2; r++) {
      int64_t bc = (int64_t)s * R + r;
      const int64_t wd = ca_time_window(P, 64 * ((int64_t)in->row_x[r] - in->row_x[r - 1]));
      const int64_t wu = ca_time_window(P, 64 * ((int64_t)in->row_x[r + 1] - in->row_x[r]));
      for (int64_t c = rs[bc]; c < rs[bc + 1]; c++) {
        int64_t best = -1, bd = -1, bu = -1;
        int64_t d_lo = rs[bc - 1], d_hi = rs[bc], u_lo = rs[bc + 1], u_hi = rs[bc + 2];
        if (!P->search_all) {
          d_lo = first_t_at_least(cl, d_lo, d_hi, (int64_t)cl[c].t_peak - wd);
          d_hi = first_t_at_least(cl, d_lo, d_hi, (int64_t)cl[c].t_peak + wd + 1);
          u_lo = first_t_at_least(cl, u_lo, u_hi, (int64_t)cl[c].t_peak - wu);
          u_hi = first_t_at_least(cl, u_lo, u_hi, (int64_t)cl[c].t_peak + wu + 1);
        }
        for (int64_t d = d_lo; d < d_hi; d++) {
          int64_t dxd = X[c] - X[d];
          if (iabs64(Y[c] - Y[d]) * P->sy_den > (int64_t)P->sy_num * dxd) continue;
          if (iabs64(Z[c] - Z[d]) * P->sz_den > (int64_t)P->sz_num * dxd) continue;
          for (int64_t u = u_lo; u < u_hi; u++) {
            int64_t dxu = X[u] - X[c];
            if (iabs64(Y[u] - Y[c]) * P->sy_den > (int64_t)P->sy_num * dxu) continue;
            if (iabs64(Z[u] - Z[c]) * P->sz_den > (int64_t)P->sz_num * dxu) continue;
            int64_t devy = (Y[u] - Y[c]) * dxd - (Y[c] - Y[d]) * dxu;
            int64_t devz = (Z[u] - Z[c]) * dxd - (Z[c] - Z[d]) * dxu;
            int64_t lim = (int64_t)P->ca_cut * (X[u] - X[d]);
            if (iabs64(devy) > lim || iabs64(devz) > lim) continue;
            int64_t sc = devy * devy + devz * devz;
            /* d ascending, then u ascending: strict < keeps the smallest (d, u) on ties */
            if (best < 0 || sc < best) { best = sc; bd = d; bu = u; }
          }
        }
        if (best >= 0) { up[c] = (int32_t)bu; down[c] = (int32_t)bd; score[c] = best; }
      }
      (void)0;
    }
  /* edge rows: up[d] for d on row 0 is the c on row 1 with down[c] = d and
   * the smallest score (c ascending, strict <: ties to the smallest c); the
   * last row mirrors it.  One pass over the c's of row 1 (row R-2) finds it
   * for every d (u) at once. */
  int64_t* edge_best = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
  for (int s = 0; s < in->n_sectors; s++) {
    int64_t b0 = (int64_t)s * R, b1 = b0 + 1;
    for (int64_t d = rs[b0]; d < rs[b0 + 1]; d++) { up[d] = -1; edge_best[d] = -1; }
    for (int64_t c = rs[b1]; c < rs[b1 + 1]; c++) {
      int64_t d = down[c];
      if (d >= 0 && (edge_best[d] < 0 || score[c] < edge_best[d])) { edge_best[d] = score[c]; up[d] = (int32_t)c; }
    }
    for (int64_t d = rs[b0]; d < rs[b0 + 1]; d++) down[d] = -1;
    int64_t bl = (int64_t)s * R + R - 1, bm = bl - 1;
    for (int64_t u = rs[bl]; u < rs[bl + 1]; u++) { down[u] = -1; edge_best[u] = -1; }
    for (int64_t c = rs[bm]; c < rs[bm + 1]; c++) {
      int64_t u = up[c];
      if (u >= 0 && (edge_best[u] < 0 || score[c] < edge_best[u])) { edge_best[u] = score[c]; down[u] = (int32_t)c; }
    }
    for (int64_t u = rs[bl]; u < rs[bl + 1]; u++) up[u] = -1;
  }
  free(edge_best);
  /* links and chains */
  for (int64_t i = 0; i < n; i++) chain_of[i] = -1;
  for (int64_t c = 0; c < n; c++) {
    int has_down = down[c] >= 0 && up[down[c]] == c;
    if (has_down) continue;
    int64_t len = 1, cur = c;
    while (up[cur] >= 0 && down[up[cur]] == cur) { cur = up[cur]; len++; }
    if (len >= P->min_chain) {
      cur = c;
      chain_of[cur] = (int32_t)c;
      while (up[cur] >= 0 && down[up[cur]] == cur) { cur = up[cur]; chain_of[cur] = (int32_t)c; }
    }
  }
  free(X); free(Y); free(Z); free(score); free(rs);
  return 0;
}

/* ------------------------------------------------------------ 7. merge */
typedef struct {
  int64_t root;       /* chain id */
  int64_t* cl;        /* clusters bottom -> top */
  int64_t len;
  int64_t next, prev; /* merged neighbour chain (index into chain table) */
} ochain;

static int64_t trunc_div(int64_t a, int64_t b) { return a / b; /* C truncates toward zero */ }

/* Residual of point (xb, yb) from the straight line through (x1, y1) -> (x2, y2),
 * measured along y at xb: trunc(((yb-y2)(x2-x1) - (y2-y1)(xb-x2)) / (x2-x1)). */
static int64_t extrap_res(int64_t x1, int64_t y1, int64_t x2, int64_t y2, int64_t xb, int64_t yb) {
  return trunc_div((yb - y2) * (x2 - x1) - (y2 - y1) * (xb - x2), x2 - x1);
}

/* Merge kept chains into tracks.  cl2trk[c] = track index or -1; track_first[k]
 * = index of the lowest cluster of track k; track_ncl[k].  Returns the track
 * count; *passes_merged = passes that merged something. */
int64_t orc_merge(const orc_input* in, const orc_params* P, const orc_cluster* cl, int64_t n,
                  const int32_t* up, const int32_t* down, const int32_t* chain_of, int32_t* cl2trk,
                  int64_t* track_first, int64_t* track_ncl, int64_t track_cap, int32_t* passes_merged) {
  int64_t *X = (int64_t*)malloc(sizeof(int64_t) * (n + 1)), *Y = (int64_t*)malloc(sizeof(int64_t) * (n + 1)),
          *Z = (int64_t*)malloc(sizeof(int64_t) * (n + 1));
  for (int64_t i = 0; i < n; i++) orc_coords(in, &cl[i], &X[i], &Y[i], &Z[i]);
  /* chain table in chain-id order */
  int64_t nch = 0;
  for (int64_t c = 0; c < n; c++) if (chain_of[c] == c) nch++;
  ochain* ch = (ochain*)calloc((size_t)nch + 1, sizeof(ochain));
  int64_t k = 0;
  for (int64_t c = 0; c < n; c++)
    if (chain_of[c] == c) {
      int64_t len = 1, cur = c;
      while (up[cur] >= 0 && down[up[cur]] == cur) { cur = up[cur]; len++; }
      ch[k].root = c; ch[k].len = len; ch[k].next = ch[k].prev = -1;
      ch[k].cl = (int64_t*)malloc(sizeof(int64_t) * len);
      cur = c;
      for (int64_t i = 0; i < len; i++) { ch[k].cl[i] = cur; if (i + 1 < len) cur = up[cur]; }
      k++;
    }
  /* chains are in id order, hence grouped by (sector, row of the root) and,
   * within one, in (t_peak, pad) order of the root: crs[s R + r] is the first
   * chain whose root lies in (sector s, row r) or later */
  const int R = in->n_rows;
  const int64_t nsr = (int64_t)in->n_sectors * R;
  int64_t* crs = (int64_t*)calloc((size_t)nsr + 1, sizeof(int64_t));
  for (int64_t i = 0; i < nch; i++) crs[(int64_t)cl[ch[i].root].sector * R + cl[ch[i].root].row + 1]++;
  for (int64_t b = 0; b < nsr; b++) crs[b + 1] += crs[b];
  int64_t* bestB = (int64_t*)malloc(sizeof(int64_t) * (nch + 1));
  int64_t* bestBs = (int64_t*)malloc(sizeof(int64_t) * (nch + 1));
  int64_t* bestA = (int64_t*)malloc(sizeof(int64_t) * (nch + 1));
  int64_t* bestAs = (int64_t*)malloc(sizeof(int64_t) * (nch + 1));
  int merged_passes = 0;
  for (int pass = 0; pass < P->merge_passes; pass++) {
    for (int64_t i = 0; i < nch; i++) { bestB[i] = bestA[i] = -1; bestBs[i] = bestAs[i] = -1; }
    for (int64_t a = 0; a < nch; a++) {
      if (ch[a].next >= 0) continue;                 /* not a top end */
      int64_t a2 = ch[a].cl[ch[a].len - 1], a1 = ch[a].cl[ch[a].len - 2];
      /* candidate bottoms b1 lie in a2's sector, gap_min..gap_max rows above
       * a2: those chains form one id range.  The forward residual bounds b1's
       * time: |trunc(n / dX_a)| <= cut needs |Z_b1 - Zp| < cut + 1, Zp the line
       * (a1, a2) at X_b1, and Z = 640 t_peak + 5 R with |5 R| <= 1280 (see
       * ca_time_window), so only roots with t_peak within that band (one bin
       * of margin) can pass; within a row they are one id range.  Visiting the
       * rows in ascending order keeps the chains in id order. */
      const int sa = cl[a2].sector, ra = cl[a2].row;
      int r_lo = ra + P->gap_min, r_hi = ra + P->gap_max;
      if (r_hi > R - 1) r_hi = R - 1;
      if (P->search_all) { r_lo = 0; r_hi = R - 1; }
      for (int rb = r_lo; rb <= r_hi; rb++) {
        int64_t b_lo = crs[(int64_t)sa * R + rb], b_hi = crs[(int64_t)sa * R + rb + 1];
        if (!P->search_all) {
          const double xb = 64.0 * in->row_x[rb];
          const double zp = (double)Z[a2] + (double)(Z[a2] - Z[a1]) * (xb - (double)X[a2]) / (double)(X[a2] - X[a1]);
          const int64_t t_lo = (int64_t)floor((zp - P->merge_cut - 1 - 1280.0) / 640.0) - 1;
          const int64_t t_hi = (int64_t)ceil((zp + P->merge_cut + 1 + 1280.0) / 640.0) + 1;
          int64_t lo = b_lo, hi = b_hi;
          while (lo < hi) {                            /* first root with t_peak >= t_lo */
            int64_t mid = lo + (hi - lo) / 2;
            if ((int64_t)cl[ch[mid].root].t_peak < t_lo) lo = mid + 1; else hi = mid;
          }
          b_lo = lo;
          hi = b_hi;
          while (lo < hi) {                            /* first root with t_peak > t_hi */
            int64_t mid = lo + (hi - lo) / 2;
            if ((int64_t)cl[ch[mid].root].t_peak <= t_hi) lo = mid + 1; else hi = mid;
          }
          b_hi = lo;
        }
        for (int64_t b = b_lo; b < b_hi; b++) {
          if (ch[b].prev >= 0) continue;               /* not a bottom end */
          int64_t b1 = ch[b].cl[0], b2 = ch[b].cl[1];
          if (cl[b1].sector != cl[a2].sector) continue;
          int gap = (int)cl[b1].row - (int)cl[a2].row;
          if (gap < P->gap_min || gap > P->gap_max) continue;
          int64_t ry = extrap_res(X[a1], Y[a1], X[a2], Y[a2], X[b1], Y[b1]);
          int64_t rz = extrap_res(X[a1], Z[a1], X[a2], Z[a2], X[b1], Z[b1]);
          int64_t sy = extrap_res(X[b2], Y[b2], X[b1], Y[b1], X[a2], Y[a2]);
          int64_t sz = extrap_res(X[b2], Z[b2], X[b1], Z[b1], X[a2], Z[a2]);
          if (iabs64(ry) > P->merge_cut || iabs64(rz) > P->merge_cut || iabs64(sy) > P->merge_cut ||
              iabs64(sz) > P->merge_cut)
            continue;
          int64_t sc = ry * ry + rz * rz + sy * sy + sz * sz;
          /* ties to the lower chain id: chains are visited in id order, strict < */
          if (bestB[a] < 0 || sc < bestBs[a]) { bestB[a] = b; bestBs[a] = sc; }
          if (bestA[b] < 0 || sc < bestAs[b]) { bestA[b] = a; bestAs[b] = sc; }
        }
      }
    }
    int any = 0;
    for (int64_t a = 0; a < nch; a++) {
      int64_t b = bestB[a];
      if (b >= 0 && bestA[b] == a) { ch[a].next = b; ch[b].prev = a; any = 1; }
    }
    if (!any) break;
    merged_passes++;
  }
  for (int64_t i = 0; i < n; i++) cl2trk[i] = -1;
  int64_t ntr = 0;
  for (int64_t a = 0; a < nch; a++) {
    if (ch[a].prev >= 0) continue;
    int64_t tot = 0;
    for (int64_t g = a; g >= 0; g = ch[g].next) tot += ch[g].len;
    if (tot < P->min_track) continue;
    if (ntr < track_cap) { track_first[ntr] = ch[a].root; track_ncl[ntr] = tot; }
    for (int64_t g = a; g >= 0; g = ch[g].next)
      for (int64_t i = 0; i < ch[g].len; i++) cl2trk[ch[g].cl[i]] = (int32_t)ntr;
    ntr++;
  }
  if (passes_merged) *passes_merged = merged_passes;
  for (int64_t i = 0; i < nch; i++) free(ch[i].cl);
  free(crs); free(ch); free(bestB); free(bestBs); free(bestA); free(bestAs); free(X); free(Y); free(Z);
  return ntr;
}

/* ------------------------------------------------------------ 8. Kalman fit */
#define CLIGHT 0.299792458

/* Curvature per unit q/pT: k = kfac * q/pT (1/cm), kfac = -bz * c * 1e-2. */
static double kfac(const orc_params* P) { return -P->bz * CLIGHT * 1e-2; }

/* Exact helix transport of state s (y, zeta, snp, tgl, qpt) by dx along x.
 * Fills the 5x5 Jacobian F (row-major) if F != NULL.  Returns 0, or 1 if
 * |snp| would reach 0.999. */
int orc_transport(const orc_params* P, const double* s, double dx, double* out, double* F) {
  double K = kfac(P);
  double k = K * s[4];
  double s1 = s[2], s2 = s1 + k * dx;
  if (fabs(s1) >= 0.999 || fabs(s2) >= 0.999) return 1;
  double c1 = sqrt(1.0 - s1 * s1), c2 = sqrt(1.0 - s2 * s2);
  double f = (s1 + s2) / (c1 + c2);
  double dy = dx * f;
  double d = fabs(dx) * sqrt(1.0 + f * f);        /* chord length */
  double kd = k * d;
  double A;                                       /* unsigned arc length */
  if (fabs(kd) < 1e-3) A = d * (1.0 + kd * kd / 24.0);
  else {
    double h = kd / 2.0;
    if (h > 1.0) h = 1.0;
    if (h < -1.0) h = -1.0;
    A = 2.0 * asin(h) / k;
  }
  double sg = dx > 0 ? 1.0 : (dx < 0 ? -1.0 : 0.0);
  out[0] = s[0] + dy;
  out[1] = s[1] + s[3] * sg * A;
  out[2] = s2;
  out[3] = s[3];
  out[4] = s[4];
  if (F) {
    for (int i = 0; i < 25; i++) F[i] = 0.0;
    for (int i = 0; i < 5; i++) F[i * 5 + i] = 1.0;
    /* f(s1, s2) partials */
    double cc = c1 + c2;
    double fs1 = 1.0 / cc + f * (s1 / c1) / cc;
    double fs2 = 1.0 / cc + f * (s2 / c2) / cc;
    double ds2dq = K * dx;
    /* y */
    F[0 * 5 + 2] = dx * (fs1 + fs2);
    F[0 * 5 + 4] = dx * fs2 * ds2dq;
    /* snp */
    F[2 * 5 + 4] = ds2dq;
    /* zeta: A(d, k), d(f) */
    double x = kd / 2.0;
    double Ad = 1.0 / sqrt(1.0 - x * x);
    double Ak;
    if (fabs(x) < 0.1) {
      double x2 = x * x;
      Ak = (k * d * d * d / 4.0) * (1.0 / 3.0 + x2 * (0.3 + x2 * (15.0 / 56.0 + x2 * (35.0 / 144.0))));
    } else {
      Ak = (2.0 / (k * k)) * (x / sqrt(1.0 - x * x) - asin(x));
    }
    double dd_df = fabs(dx) * f / sqrt(1.0 + f * f);
    double dd_ds1 = dd_df * (fs1 + fs2);
    double dd_dq = dd_df * fs2 * ds2dq;
    F[1 * 5 + 2] = s[3] * sg * Ad * dd_ds1;
    F[1 * 5 + 3] = sg * A;
    F[1 * 5 + 4] = s[3] * sg * (Ad * dd_dq + Ak * K);
  }
  return 0;
}

/* One Kalman update with measurement (my, mz) of (y, zeta).  C is 5x5 full.
 * Returns the chi2 increment; *pd_ok reports the PD check of the result. */
double orc_update(const orc_params* P, double* s, double* C, double my, double mz, int* pd_ok) {
  double S00 = C[0] + P->sigma_y * P->sigma_y, S01 = C[1], S11 = C[6] + P->sigma_z * P->sigma_z;
  double det = S00 * S11 - S01 * S01;
  double I00 = S11 / det, I01 = -S01 / det, I11 = S00 / det;
  double r0 = my - s[0], r1 = mz - s[1];
  double Kg[5][2];
  for (int i = 0; i < 5; i++) {
    Kg[i][0] = C[i * 5 + 0] * I00 + C[i * 5 + 1] * I01;
    Kg[i][1] = C[i * 5 + 0] * I01 + C[i * 5 + 1] * I11;
  }
  for (int i = 0; i < 5; i++) s[i] += Kg[i][0] * r0 + Kg[i][1] * r1;
  double Cn[25];
  for (int i = 0; i < 5; i++)
    for (int j = 0; j < 5; j++) Cn[i * 5 + j] = C[i * 5 + j] - (Kg[i][0] * C[0 * 5 + j] + Kg[i][1] * C[1 * 5 + j]);
  for (int i = 0; i < 5; i++)
    for (int j = 0; j < 5; j++) C[i * 5 + j] = 0.5 * (Cn[i * 5 + j] + Cn[j * 5 + i]);
  int ok = 1;
  for (int i = 0; i < 5; i++) if (!(C[i * 5 + i] > 0.0)) ok = 0;
  for (int i = 0; i < 5 && ok; i++)
    for (int j = i + 1; j < 5; j++)
      if (!(C[i * 5 + j] * C[i * 5 + j] < C[i * 5 + i] * C[j * 5 + j])) ok = 0;
  if (pd_ok) *pd_ok = ok;
  return r0 * (I00 * r0 + I01 * r1) + r1 * (I01 * r0 + I11 * r1);
}

/* Initial state at the outermost point from the circle through the innermost
 * (1), middle (2) and outermost (3) points. */
static void fit_init(const orc_params* P, const double* x, const double* y, const double* z, int n,
                     double* s) {
  int i1 = 0, i2 = (n - 1) / 2, i3 = n - 1;
  double ax = x[i2] - x[i1], ay = y[i2] - y[i1];
  double bx = x[i3] - x[i2], by = y[i3] - y[i2];
  double cx = x[i3] - x[i1], cy = y[i3] - y[i1];
  double la = sqrt(ax * ax + ay * ay), lb = sqrt(bx * bx + by * by), lc = sqrt(cx * cx + cy * cy);
  double k = 2.0 * (ax * cy - ay * cx) / (la * lb * lc);
  double h = k * lc / 2.0;
  if (h > 1.0) h = 1.0;
  if (h < -1.0) h = -1.0;
  double half = asin(h);
  double phic = atan2(cy, cx);
  double arc = fabs(k * lc) < 1e-3 ? lc * (1.0 + (k * lc) * (k * lc) / 24.0) : 2.0 * half / k;
  s[0] = y[i3];
  s[1] = z[i3];
  s[2] = sin(phic + half);
  s[3] = (z[i3] - z[i1]) / arc;
  s[4] = k / kfac(P);
}

/* FP64 fit of measurement points (x, y, zeta in cm, ascending x, n >= 3).
 * Three passes inward / outward / inward; output at the innermost point. */
int orc_fit_points(const orc_params* P, int n, const double* x, const double* y, const double* z,
                   orc_fit* out) {
  double s[5], C[25];
  fit_init(P, x, y, z, n, s);
  double xcur = x[n - 1];
  int flags = 0, n_used = 0;
  double chi2 = 0.0;
  for (int pass = 0; pass < P->fit_passes; pass++) {
    for (int i = 0; i < 25; i++) C[i] = 0.0;
    for (int i = 0; i < 5; i++) C[i * 5 + i] = P->c0[i];
    chi2 = 0.0;
    n_used = 0;
    int inward = (pass % 2) == 0;
    for (int j = 0; j < n; j++) {
      int i = inward ? n - 1 - j : j;
      double dx = x[i] - xcur;
      if (dx != 0.0) {
        double ns[5], F[25], T[25], Cn[25];
        if (orc_transport(P, s, dx, ns, F)) { flags |= 1; break; }
        /* C' = F C F^T */
        for (int a = 0; a < 5; a++)
          for (int b = 0; b < 5; b++) {
            double acc = 0.0;
            for (int l = 0; l < 5; l++) acc += F[a * 5 + l] * C[l * 5 + b];
            T[a * 5 + b] = acc;
          }
        for (int a = 0; a < 5; a++)
          for (int b = 0; b < 5; b++) {
            double acc = 0.0;
            for (int l = 0; l < 5; l++) acc += T[a * 5 + l] * F[b * 5 + l];
            Cn[a * 5 + b] = acc;
          }
        memcpy(C, Cn, sizeof(Cn));
        memcpy(s, ns, sizeof(ns));
        xcur = x[i];
      }
      int ok = 1;
      chi2 += orc_update(P, s, C, y[i], z[i], &ok);
      if (!ok) flags |= 2;
      n_used++;
    }
  }
  for (int i = 0; i < 5; i++) out->par[i] = s[i];
  out->x = xcur;
  int m = 0;
  for (int i = 0; i < 5; i++)
    for (int j = 0; j <= i; j++) out->cov[m++] = C[i * 5 + j];
  out->chi2 = chi2;
  out->ndf = 2 * n_used - 5;
  out->n_used = n_used;
  out->flags = flags;
  return 0;
}

/* Fit of one track given its clusters' integer coordinates (u units, ascending
 * row).  Measurements are taken relative to the first cluster's exact integer
 * coordinates, converted to cm, and the reference is added back at the end. */
int orc_fit_track(const orc_params* P, int n, const int64_t* X, const int64_t* Y, const int64_t* Z,
                  orc_fit* out) {
  const double u = 7.8125e-4;
  double* x = (double*)malloc(sizeof(double) * 3 * n);
  double *y = x + n, *z = x + 2 * n;
  for (int i = 0; i < n; i++) {
    x[i] = (double)X[i] * u;
    y[i] = (double)(Y[i] - Y[0]) * u;
    z[i] = (double)(Z[i] - Z[0]) * u;
  }
  int rc = orc_fit_points(P, n, x, y, z, out);
  out->par[0] += (double)Y[0] * u;
  out->par[1] += (double)Z[0] * u;
  free(x);
  return rc;
}

/* Fit every track produced by orc_merge (cl2trk, n_tracks). */
int orc_fit_all(const orc_input* in, const orc_params* P, const orc_cluster* cl, int64_t n,
                const int32_t* cl2trk, int64_t n_tracks, orc_fit* out) {
  int64_t* cnt = (int64_t*)calloc((size_t)n_tracks + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) if (cl2trk[i] >= 0) cnt[cl2trk[i] + 1]++;
  for (int64_t t = 0; t < n_tracks; t++) cnt[t + 1] += cnt[t];
  int64_t* lst = (int64_t*)malloc(sizeof(int64_t) * (cnt[n_tracks] + 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (n_tracks + 1));
  memcpy(fill, cnt, sizeof(int64_t) * n_tracks);
  /* cluster indices ascend with row within a sector, so each list is in row order */
  for (int64_t i = 0; i < n; i++) if (cl2trk[i] >= 0) lst[fill[cl2trk[i]]++] = i;
  for (int64_t t = 0; t < n_tracks; t++) {
    int m = (int)(cnt[t + 1] - cnt[t]);
    int64_t* X = (int64_t*)malloc(sizeof(int64_t) * 3 * m);
    int64_t *Y = X + m, *Z = X + 2 * m;
    for (int i = 0; i < m; i++) orc_coords(in, &cl[lst[cnt[t] + i]], &X[i], &Y[i], &Z[i]);
    orc_fit_track(P, m, X, Y, Z, &out[t]);
    free(X);
  }
  free(cnt); free(lst); free(fill);
  return 0;
}

/* ------------------------------------------------------------ 9. cross-sector merge
 * Follows the library's definition of the optional cross-sector merge (the
 * paper, section "Hardware and data flow", names the full TPC tracking on the
 * EPN GPUs; matching track pieces across sector borders is this library's
 * definition of that tracking's last step):
 *   - a track piece A exits through the +y (-y) edge of its sector when its
 *     outermost cluster lies within edge_cm of that edge of the pad plane; a
 *     piece B enters through an edge when its innermost cluster does;
 *   - a candidate pair is A exiting through +y (-y) of sector s and B entering
 *     through -y (+y) of the neighbouring sector s+1 (s-1) of the same side,
 *     with A's outermost row below B's innermost row;
 *   - B's fitted state is expressed in A's frame (rotation about the beam axis)
 *     and transported to A's reference x; chi2 = d^T (C_A + J C_B J^T)^-1 d;
 *   - mutual best pairs under chi2 <= chi2_cut link (ties: lower index);
 *   - chained pieces form one track, refitted over all their clusters with the
 *     frame switched at each sector change.
 * borderline[t] (may be NULL; test output, not part of the definition) marks a
 * piece whose decision is within 1 % of flipping: a candidate chi2 within 1 %
 * of the cut, or a runner-up within 1 % of the best on either side.
 * Rotation of a state (y, zeta, snp, tgl, q/pT) at x from a frame at angle
 * alpha_old to one at alpha_new (delta = alpha_old - alpha_new): the point
 * (x, y) maps to (x cos d - y sin d, x sin d + y cos d), the direction angle
 * gains d.  Its Jacobian at the rotated reference x' (first order: the point
 * moves with y by dx' = -sin d dy, and the state is carried back along the
 * helix to the fixed x'): dy' = (cos d + tan(phi') sin d) dy;
 * dzeta' = dzeta + (tgl / cos(phi')) sin d dy; dsnp' = (cos d - sin d snp /
 * cos(phi)) dsnp + k sin d dy. */
typedef struct {
  double chi2_cut;   /* 100 */
  double edge_cm;    /* 6 */
  double dz_cm;      /* 250: |zeta(B innermost) - zeta(A outermost)| bound of a candidate pair */
} orc_xs_params;

static double sector_alpha(int s) { return ((double)(s % 18) + 0.5) * (20.0 * 3.14159265358979323846 / 180.0); }

int orc_rotate(const orc_params* P, double* s, double* x, double delta, double* R) {
  double cd = cos(delta), sd = sin(delta);
  double sn = s[2];
  if (fabs(sn) >= 0.999) return 1;
  double cs = sqrt(1.0 - sn * sn);
  double sn2 = sn * cd + cs * sd;
  if (fabs(sn2) >= 0.999) return 1;
  double cs2 = sqrt(1.0 - sn2 * sn2);
  if (R) {
    for (int i = 0; i < 25; i++) R[i] = 0.0;
    for (int i = 0; i < 5; i++) R[i * 5 + i] = 1.0;
    R[0 * 5 + 0] = cd + (sn2 / cs2) * sd;
    R[1 * 5 + 0] = (s[3] / cs2) * sd;
    R[2 * 5 + 0] = kfac(P) * s[4] * sd;
    R[2 * 5 + 2] = cd - sd * sn / cs;
  }
  double xn = *x * cd - s[0] * sd;
  double yn = *x * sd + s[0] * cd;
  s[0] = yn;
  s[2] = sn2;
  *x = xn;
  return 0;
}

static void mat_abt(const double* A, const double* B, double* C) {   /* C = A B^T (5x5) */
  for (int i = 0; i < 5; i++)
    for (int j = 0; j < 5; j++) {
      double acc = 0.0;
      for (int l = 0; l < 5; l++) acc += A[i * 5 + l] * B[j * 5 + l];
      C[i * 5 + j] = acc;
    }
}
static void mat_ab(const double* A, const double* B, double* C) {    /* C = A B (5x5) */
  for (int i = 0; i < 5; i++)
    for (int j = 0; j < 5; j++) {
      double acc = 0.0;
      for (int l = 0; l < 5; l++) acc += A[i * 5 + l] * B[l * 5 + j];
      C[i * 5 + j] = acc;
    }
}
/* C <- J C J^T */
static void sandwich(const double* J, double* C) {
  double T[25], Jt[25];
  mat_ab(J, C, T);
  for (int i = 0; i < 5; i++)
    for (int j = 0; j < 5; j++) Jt[i * 5 + j] = J[j * 5 + i];
  mat_ab(T, Jt, C);
}

static void unpack_cov(const double* tri, double* C) {
  int m = 0;
  for (int i = 0; i < 5; i++)
    for (int j = 0; j <= i; j++) { C[i * 5 + j] = tri[m]; C[j * 5 + i] = tri[m]; m++; }
}

/* chi2 of d^T M^-1 d for symmetric positive definite M (Cholesky); -1 if not PD. */
static double chi2_spd(const double* M, const double* d) {
  double L[25] = {0};
  for (int j = 0; j < 5; j++) {
    double acc = M[j * 5 + j];
    for (int k = 0; k < j; k++) acc -= L[j * 5 + k] * L[j * 5 + k];
    if (!(acc > 0.0)) return -1.0;
    L[j * 5 + j] = sqrt(acc);
    for (int i = j + 1; i < 5; i++) {
      double a = M[i * 5 + j];
      for (int k = 0; k < j; k++) a -= L[i * 5 + k] * L[j * 5 + k];
      L[i * 5 + j] = a / L[j * 5 + j];
    }
  }
  double w[5], c2 = 0.0;   /* solve L w = d */
  for (int i = 0; i < 5; i++) {
    double a = d[i];
    for (int k = 0; k < i; k++) a -= L[i * 5 + k] * w[k];
    w[i] = a / L[i * 5 + i];
    c2 += w[i] * w[i];
  }
  return c2;
}

/* Matching chi2 of pieces A (state at xa in frame aa) and B (at xb in frame ab);
 * -1 if B cannot be carried to A's reference. */
double orc_xs_chi2(const orc_params* P, const orc_fit* A, double aa, const orc_fit* B, double ab) {
  double s[5], x = B->x, R[25], F[25], J[25], CA[25], CB[25], out[5], d[5];
  for (int i = 0; i < 5; i++) s[i] = B->par[i];
  if (orc_rotate(P, s, &x, ab - aa, R)) return -1.0;
  if (orc_transport(P, s, A->x - x, out, F)) return -1.0;
  mat_ab(F, R, J);
  unpack_cov(A->cov, CA);
  unpack_cov(B->cov, CB);
  sandwich(J, CB);
  for (int i = 0; i < 25; i++) CA[i] += CB[i];
  for (int i = 0; i < 5; i++) d[i] = A->par[i] - out[i];
  return chi2_spd(CA, d);
}

/* FP64 fit over points in several sector frames: (x, y) in the frame of
 * alpha[i], zeta common; points ordered innermost first, frames changing only
 * between pieces.  Initial state from the circle through the innermost, middle
 * and outermost points expressed in the outermost point's frame; passes as in
 * orc_fit_points, the state and covariance rotated into a point's frame before
 * it is reached. */
int orc_fit_points_xs(const orc_params* P, int n, const double* x, const double* y, const double* z,
                      const double* alpha, orc_fit* out) {
  double s[5], C[25];
  {
    /* the three points in the outermost point's frame */
    int idx[3] = {0, (n - 1) / 2, n - 1};
    double px[3], py[3], pz[3];
    for (int q = 0; q < 3; q++) {
      double dd = alpha[idx[q]] - alpha[n - 1], cd = cos(dd), sd = sin(dd);
      px[q] = x[idx[q]] * cd - y[idx[q]] * sd;
      py[q] = x[idx[q]] * sd + y[idx[q]] * cd;
      pz[q] = z[idx[q]];
    }
    fit_init(P, px, py, pz, 3, s);
  }
  double xcur = x[n - 1], acur = alpha[n - 1];
  int flags = 0, n_used = 0;
  double chi2 = 0.0;
  for (int pass = 0; pass < P->fit_passes; pass++) {
    for (int i = 0; i < 25; i++) C[i] = 0.0;
    for (int i = 0; i < 5; i++) C[i * 5 + i] = P->c0[i];
    chi2 = 0.0;
    n_used = 0;
    int inward = (pass % 2) == 0;
    for (int j = 0; j < n; j++) {
      int i = inward ? n - 1 - j : j;
      if (alpha[i] != acur) {
        double R[25];
        if (orc_rotate(P, s, &xcur, acur - alpha[i], R)) { flags |= 1; break; }
        sandwich(R, C);
        acur = alpha[i];
      }
      double dx = x[i] - xcur;
      if (dx != 0.0) {
        double ns[5], F[25];
        if (orc_transport(P, s, dx, ns, F)) { flags |= 1; break; }
        sandwich(F, C);
        memcpy(s, ns, sizeof(ns));
        xcur = x[i];
      }
      int ok = 1;
      chi2 += orc_update(P, s, C, y[i], z[i], &ok);
      if (!ok) flags |= 2;
      n_used++;
    }
  }
  for (int i = 0; i < 5; i++) out->par[i] = s[i];
  out->x = xcur;
  int m = 0;
  for (int i = 0; i < 5; i++)
    for (int j = 0; j <= i; j++) out->cov[m++] = C[i * 5 + j];
  out->chi2 = chi2;
  out->ndf = 2 * n_used - 5;
  out->n_used = n_used;
  out->flags = flags;
  return 0;
}

/* Edge test in integer u (7.8125 um): the pad plane of a row spans
 * |Y| <= 256 (npads - 1); a cluster within E = edge_cm / u of an edge. */
static int side_of(int64_t Y, int np, int64_t E) {
  const int64_t hw = 256 * (int64_t)(np - 1);
  if (Y >= hw - E) return 1;
  if (Y <= -(hw - E)) return -1;
  return 0;
}
static int neighbour_sector(int s, int side) {
  int base = s < 18 ? 0 : 18, k = s - base;
  return base + (k + (side > 0 ? 1 : 17)) % 18;
}

/* Cross-sector merge of the tracks of orc_merge / orc_fit_all.  Outputs:
 * link[n_tracks] (outer piece or -1), best_chi2[n_tracks] (A's best candidate
 * chi2 or -1), group_of[n_tracks] (merged track index of every piece),
 * gfit / g_first / g_ncl / g_npieces per merged track (track order: by the
 * innermost piece's index).  Returns the number of merged tracks. */
int64_t orc_merge_sectors(const orc_input* in, const orc_params* P, const orc_xs_params* XP,
                          const orc_cluster* cl, int64_t n, const int32_t* cl2trk, int64_t nt,
                          const orc_fit* fits, int32_t* link, double* best_chi2, int32_t* group_of,
                          orc_fit* gfit, int32_t* g_first, int32_t* g_ncl, int32_t* g_npieces,
                          int8_t* borderline) {
  const double u = 7.8125e-4;
  /* per-track cluster lists in row order */
  int64_t* cnt = (int64_t*)calloc((size_t)nt + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) if (cl2trk[i] >= 0) cnt[cl2trk[i] + 1]++;
  for (int64_t t = 0; t < nt; t++) cnt[t + 1] += cnt[t];
  int64_t* lst = (int64_t*)malloc(sizeof(int64_t) * (cnt[nt] + 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (nt + 1));
  memcpy(fill, cnt, sizeof(int64_t) * nt);
  for (int64_t i = 0; i < n; i++) if (cl2trk[i] >= 0) lst[fill[cl2trk[i]]++] = i;
  /* ends */
  int* sec = (int*)malloc(sizeof(int) * (nt + 1));
  int* exit_side = (int*)malloc(sizeof(int) * (nt + 1));
  int* entry_side = (int*)malloc(sizeof(int) * (nt + 1));
  int* row_in = (int*)malloc(sizeof(int) * (nt + 1));
  int* row_out = (int*)malloc(sizeof(int) * (nt + 1));
  int64_t* z_in = (int64_t*)malloc(sizeof(int64_t) * (nt + 1));
  int64_t* z_out = (int64_t*)malloc(sizeof(int64_t) * (nt + 1));
  const int64_t Dz = (int64_t)floor(XP->dz_cm / u + 0.5);
  for (int64_t t = 0; t < nt; t++) {
    const orc_cluster* ci = &cl[lst[cnt[t]]];
    const orc_cluster* co = &cl[lst[cnt[t + 1] - 1]];
    int64_t X, Y, Z;
    sec[t] = ci->sector;
    row_in[t] = ci->row;
    row_out[t] = co->row;
    const int64_t E = (int64_t)floor(XP->edge_cm / u + 0.5);
    orc_coords(in, ci, &X, &Y, &Z);
    entry_side[t] = side_of(Y, in->npads[ci->row], E);
    z_in[t] = Z;
    orc_coords(in, co, &X, &Y, &Z);
    exit_side[t] = side_of(Y, in->npads[co->row], E);
    z_out[t] = Z;
  }
  /* best candidates (chi2, index) both ways */
  double* bb = (double*)malloc(sizeof(double) * (nt + 1));
  double* ba = (double*)malloc(sizeof(double) * (nt + 1));
  double* bb2 = (double*)malloc(sizeof(double) * (nt + 1));   /* runners-up */
  double* ba2 = (double*)malloc(sizeof(double) * (nt + 1));
  int32_t* ib = (int32_t*)malloc(sizeof(int32_t) * (nt + 1));
  int32_t* ia = (int32_t*)malloc(sizeof(int32_t) * (nt + 1));
  for (int64_t t = 0; t < nt; t++) { bb[t] = ba[t] = bb2[t] = ba2[t] = -1.0; ib[t] = ia[t] = -1; }
  if (borderline) for (int64_t t = 0; t < nt; t++) borderline[t] = 0;
  for (int64_t a = 0; a < nt; a++) {
    if (!exit_side[a] || fits[a].flags) continue;
    int sb = neighbour_sector(sec[a], exit_side[a]);
    for (int64_t b = 0; b < nt; b++) {
      if (sec[b] != sb || entry_side[b] != -exit_side[a] || row_out[a] >= row_in[b] || fits[b].flags) continue;
      if (llabs(z_in[b] - z_out[a]) > Dz) continue;
      double c2 = orc_xs_chi2(P, &fits[a], sector_alpha(sec[a]), &fits[b], sector_alpha(sec[b]));
      if (borderline && c2 >= 0.0 && fabs(c2 - XP->chi2_cut) <= 0.01 * XP->chi2_cut) borderline[a] = borderline[b] = 1;
      if (c2 < 0.0 || c2 > XP->chi2_cut) continue;
      if (ib[a] < 0 || c2 < bb[a] || (c2 == bb[a] && b < ib[a])) { bb2[a] = bb[a]; bb[a] = c2; ib[a] = (int32_t)b; }
      else if (bb2[a] < 0.0 || c2 < bb2[a]) bb2[a] = c2;
      if (ia[b] < 0 || c2 < ba[b] || (c2 == ba[b] && a < ia[b])) { ba2[b] = ba[b]; ba[b] = c2; ia[b] = (int32_t)a; }
      else if (ba2[b] < 0.0 || c2 < ba2[b]) ba2[b] = c2;
    }
  }
  /* a runner-up within 1 % of the best makes the choice borderline */
  if (borderline)
    for (int64_t t = 0; t < nt; t++) {
      if (bb2[t] >= 0.0 && bb2[t] - bb[t] <= 0.01 * (bb[t] > 1.0 ? bb[t] : 1.0)) borderline[t] = 1;
      if (ba2[t] >= 0.0 && ba2[t] - ba[t] <= 0.01 * (ba[t] > 1.0 ? ba[t] : 1.0)) borderline[t] = 1;
    }
  int32_t* prev = (int32_t*)malloc(sizeof(int32_t) * (nt + 1));
  for (int64_t t = 0; t < nt; t++) { link[t] = -1; prev[t] = -1; best_chi2[t] = bb[t]; }
  for (int64_t a = 0; a < nt; a++)
    if (ib[a] >= 0 && ia[ib[a]] == a) { link[a] = ib[a]; prev[ib[a]] = (int32_t)a; }
  /* groups in the order of their innermost piece */
  int64_t ng = 0;
  for (int64_t r = 0; r < nt; r++) {
    if (prev[r] >= 0) continue;
    int np_ = 0, ncl = 0;
    for (int64_t t = r; t >= 0; t = link[t]) { group_of[t] = (int32_t)ng; np_++; ncl += (int)(cnt[t + 1] - cnt[t]); }
    g_first[ng] = (int32_t)lst[cnt[r]];
    g_ncl[ng] = ncl;
    g_npieces[ng] = np_;
    if (np_ == 1) {
      gfit[ng] = fits[r];
    } else {
      double* x = (double*)malloc(sizeof(double) * 4 * ncl);
      double *y = x + ncl, *z = x + 2 * ncl, *al = x + 3 * ncl;
      int m = 0;
      for (int64_t t = r; t >= 0; t = link[t])
        for (int64_t q = cnt[t]; q < cnt[t + 1]; q++) {
          int64_t X, Y, Z;
          orc_coords(in, &cl[lst[q]], &X, &Y, &Z);
          x[m] = (double)X * u; y[m] = (double)Y * u; z[m] = (double)Z * u;
          al[m] = sector_alpha(cl[lst[q]].sector);
          m++;
        }
      orc_fit_points_xs(P, ncl, x, y, z, al, &gfit[ng]);
      free(x);
    }
    ng++;
  }
  free(cnt); free(lst); free(fill); free(sec); free(exit_side); free(entry_side); free(row_in);
  free(row_out); free(z_in); free(z_out); free(bb); free(ba); free(bb2); free(ba2); free(ib); free(ia); free(prev);
  return ng;
}

/* ------------------------------------------------------------ 9b. looper legs
 * Follows the library's definition of joining the legs of a looping track
 * within one sector (the paper, section "Hardware and data flow", names the
 * full TPC tracking on the EPN GPUs; a track whose circle lies inside the TPC
 * crosses a sector once per turn, on the same transverse path each time, and
 * steps 5-8 find every crossing as a track of its own):
 *   - a step-8 track can loop when the circle through its fitted point and
 *     direction (at the reference x) with the curvature of |q/pT| + 3 sigma
 *     (sigma from the fit's covariance scaled as below) lies within
 *     loop_radius of the beam axis: |centre| + 1/|k| <= loop_radius, the
 *     centre being (x - snp/k, y + cos(phi)/k) in the sector frame (k the
 *     signed curvature); a short leg's q/pT is too uncertain for the fitted
 *     circle alone to tell;
 *   - tracks A < B of one sector are a candidate pair when both loop, neither
 *     fit is flagged and their q/pT have the same sign (successive turns cross
 *     the sector in the same direction, so their fits share orientation);
 *   - each fit's covariance is scaled by max(1, chi2/ndf) of that fit (the
 *     measurement errors the fit assumes understate the scatter of clusters
 *     that overlap, which loopers' clusters often do);
 *   - both states are carried to the larger of the two reference x (one of
 *     them moves, with its covariance); there the turn count is m = the
 *     integer nearest (ties away from zero) to (zeta_B - zeta_A) / S, with
 *     S = tgl_A 2 pi / |k_A| the zeta advance of one turn; the pair is a
 *     candidate only for 1 <= |m| <= max_turns and tgl_A, tgl_B of one sign
 *     (so that along every link zeta advances in the direction of the one
 *     sign of tgl that the legs of a chain share, and chains cannot close);
 *   - A's state is advanced by m turns (zeta + m S; the rest of the state is
 *     that of the same transverse point one turn on), d = s_B - that, and
 *     chi2 = d^T (J C_A J^T + C_B)^-1 d with J the identity plus the zeta
 *     row's m 2 pi / |k_A| (tgl) and -m S / (q/pT)_A (q/pT) entries; the pair
 *     is accepted when chi2 <= chi2_cut;
 *   - an accepted pair is directed from the leg of lower zeta along the fitted
 *     motion to the other: A -> B when m > 0, B -> A when m < 0;
 *   - every track's next leg is its outgoing accepted pair of least |m|, then
 *     least chi2, then lowest index; its previous leg likewise over the
 *     incoming pairs; A -> B links when B is A's next and A is B's previous.
 * Chains of links are the turns of one looper in that sector. */
typedef struct {
  double chi2_cut;         /* 30 */
  double loop_radius_cm;   /* 275: the 250 cm outer field cage + 10 % */
  int32_t max_turns;       /* 4 */
  int32_t pad;
} orc_loop_params;

/* State and covariance of a fit carried to x_out, the covariance scaled by
 * max(1, chi2/ndf); returns 1 if the transport stops. */
static int carry_fit(const orc_params* P, const orc_fit* f, double x_out, double* s, double* C) {
  double F[25];
  for (int i = 0; i < 5; i++) s[i] = f->par[i];
  unpack_cov(f->cov, C);
  const double q = f->ndf > 0 ? f->chi2 / (double)f->ndf : 1.0;
  if (q > 1.0)
    for (int i = 0; i < 25; i++) C[i] *= q;
  if (x_out == f->x) return 0;
  double out[5];
  if (orc_transport(P, s, x_out - f->x, out, F)) return 1;
  for (int i = 0; i < 5; i++) s[i] = out[i];
  sandwich(F, C);
  return 0;
}

/* Farthest distance from the beam axis of the circle through f's fitted
 * point and direction with |q/pT| raised by 3 sigma; -1 if undefined. */
static double loop_reach(const orc_params* P, const orc_fit* f) {
  const double q = f->ndf > 0 && f->chi2 > (double)f->ndf ? f->chi2 / (double)f->ndf : 1.0;
  const double sq = sqrt(f->cov[14] * q);
  const double qpt = f->par[4] + (f->par[4] < 0.0 ? -3.0 : 3.0) * sq;
  const double k = kfac(P) * qpt;
  const double sn = f->par[2];
  if (f->par[4] == 0.0 || k == 0.0 || !(fabs(sn) < 1.0)) return -1.0;
  const double cs = sqrt(1.0 - sn * sn);
  const double xc = f->x - sn / k, yc = f->par[0] + cs / k;
  return sqrt(xc * xc + yc * yc) + 1.0 / fabs(k);
}

/* 1 if the track f can loop within radius r_out. */
int orc_loops(const orc_params* P, const orc_fit* f, double r_out) {
  const double r = loop_reach(P, f);
  return r >= 0.0 && r <= r_out;
}

/* chi2 of B against A advanced by m turns (states and covariances at one x;
 * turn the transverse arc of a turn, S the zeta advance of one). */
static double turns_chi2(const double* sa, const double* CA_in, const double* sb, const double* CB, double turn,
                         double S, int m) {
  double J[25], CA[25], d[5];
  for (int i = 0; i < 25; i++) { J[i] = 0.0; CA[i] = CA_in[i]; }
  for (int i = 0; i < 5; i++) J[i * 5 + i] = 1.0;
  J[1 * 5 + 3] = m * turn;
  J[1 * 5 + 4] = -m * S / sa[4];
  sandwich(J, CA);
  for (int i = 0; i < 5; i++) d[i] = sb[i] - sa[i];
  d[1] -= m * S;
  for (int i = 0; i < 25; i++) CA[i] += CB[i];
  return chi2_spd(CA, d);
}

/* Matching chi2 of legs A and B and their signed turn count *m (A's turns to
 * reach B); -1 when the pair is not a candidate (transport stops, no advance
 * per turn, tgl of opposite signs, or |m| outside 1..max_turns). */
/* As orc_loop_pair, with the unrounded turn count r and the chi2 with the
 * other integer nearest r (the turn count had r rounded the other way; -1 if
 * that is 0 or out of range) for the borderline test. */
double orc_loop_pair_r(const orc_params* P, const orc_loop_params* LP, const orc_fit* A, const orc_fit* B, int* m_out,
                       double* r_out, double* alt_out) {
  const double two_pi = 2.0 * 3.14159265358979323846;
  const double xr = A->x > B->x ? A->x : B->x;
  double sa[5], sb[5], CA[25], CB[25];
  *m_out = 0;
  if (carry_fit(P, A, xr, sa, CA) || carry_fit(P, B, xr, sb, CB)) return -1.0;
  const double k = kfac(P) * sa[4];
  if (k == 0.0) return -1.0;
  const double turn = two_pi / fabs(k);
  const double S = sa[3] * turn;
  if (S == 0.0) return -1.0;
  const double r = (sb[1] - sa[1]) / S;
  if (r_out) *r_out = r;
  if (alt_out) *alt_out = -1.0;
  if (!(sa[3] * sb[3] > 0.0)) return -1.0;
  if (!(fabs(r) < (double)LP->max_turns + 1.0)) return -1.0;
  const int m = (int)(r < 0.0 ? -floor(-r + 0.5) : floor(r + 0.5));
  if (alt_out) {
    /* the other integer nearest r */
    const int ma = (double)m > r ? m - 1 : m + 1;
    if (ma != 0 && abs(ma) <= LP->max_turns) *alt_out = turns_chi2(sa, CA, sb, CB, turn, S, ma);
  }
  if (m == 0 || abs(m) > LP->max_turns) return -1.0;
  *m_out = m;
  return turns_chi2(sa, CA, sb, CB, turn, S, m);
}

double orc_loop_pair(const orc_params* P, const orc_loop_params* LP, const orc_fit* A, const orc_fit* B, int* m_out) {
  return orc_loop_pair_r(P, LP, A, B, m_out, NULL, NULL);
}

/* Ordering key of a candidate (turns |m|, chi2, index): 1 if (m1, c1, i1)
 * comes before (m2, c2, i2). */
static int loop_before(int m1, double c1, int32_t i1, int m2, double c2, int32_t i2) {
  if (m1 != m2) return m1 < m2;
  if (c1 != c2) return c1 < c2;
  return i1 < i2;
}

/* Looper-leg join of the step-8 tracks (fits[nt], cl2trk over n clusters):
 * next[t] / prev[t] = the linked following / preceding leg or -1;
 * next_chi2[t] = the chi2 of the link to next[t] or -1; borderline[t] = 1
 * when a decision about t is within 1 % of flipping: t's looping reach within
 * 1 % of loop_radius; a pair of t whose chi2 lies within 1 % of the cut; a
 * pair of t whose (zeta_B - zeta_A) / S lies within 0.01 of a half-integer
 * (the turn count's rounding, or the range bound max_turns + 1/2) while its
 * chi2 with either neighbouring turn count is at most 1.01 cut; or t's two
 * best candidates in one direction with equal |m| and chi2 within 1 % of each
 * other.  Returns the number of links. */
int64_t orc_join_loopers(const orc_input* in, const orc_params* P, const orc_loop_params* LP, const orc_cluster* cl,
                         int64_t n, const int32_t* cl2trk, int64_t nt, const orc_fit* fits, int32_t* next,
                         int32_t* prev, double* next_chi2, int8_t* borderline) {
  (void)in;   /* the geometry plays no part: the fits carry the reference x */
  int32_t* sec = (int32_t*)malloc(sizeof(int32_t) * (nt + 1));
  int8_t* loops = (int8_t*)malloc((size_t)nt + 1);
  for (int64_t t = 0; t < nt; t++) sec[t] = -1;
  for (int64_t i = 0; i < n; i++) if (cl2trk[i] >= 0 && sec[cl2trk[i]] < 0) sec[cl2trk[i]] = cl[i].sector;
  for (int64_t t = 0; t < nt; t++) borderline[t] = 0;
  for (int64_t t = 0; t < nt; t++) {
    loops[t] = 0;
    if (sec[t] < 0 || fits[t].flags) continue;
    const double reach = loop_reach(P, &fits[t]);
    if (reach < 0.0) continue;
    loops[t] = reach <= LP->loop_radius_cm;
    if (fabs(reach - LP->loop_radius_cm) <= 0.01 * LP->loop_radius_cm) borderline[t] = 1;
  }
  /* per track and direction (0 next, 1 prev): best and runner-up (m, chi2, index) */
  int* bm = (int*)malloc(sizeof(int) * 4 * (nt + 1));
  double* bc = (double*)malloc(sizeof(double) * 4 * (nt + 1));
  int32_t* bi = (int32_t*)malloc(sizeof(int32_t) * 4 * (nt + 1));
  for (int64_t q = 0; q < 4 * nt; q++) { bm[q] = 0; bc[q] = -1.0; bi[q] = -1; }
  for (int64_t a = 0; a < nt; a++) {
    if (!loops[a]) continue;
    for (int64_t b = a + 1; b < nt; b++) {
      if (!loops[b] || sec[b] != sec[a] || (fits[a].par[4] > 0.0) != (fits[b].par[4] > 0.0)) continue;
      int m;
      double r = 0.0, alt = -1.0;
      const double c2 = orc_loop_pair_r(P, LP, &fits[a], &fits[b], &m, &r, &alt);
      const double fr = fabs(r) - floor(fabs(r));
      if (fabs(fr - 0.5) <= 0.01 &&
          ((c2 >= 0.0 && c2 <= 1.01 * LP->chi2_cut) || (alt >= 0.0 && alt <= 1.01 * LP->chi2_cut)))
        borderline[a] = borderline[b] = 1;
      if (c2 < 0.0) continue;
      if (fabs(c2 - LP->chi2_cut) <= 0.01 * LP->chi2_cut) borderline[a] = borderline[b] = 1;
      if (c2 > LP->chi2_cut) continue;
      const int am = m < 0 ? -m : m;
      const int64_t f = m > 0 ? a : b, g = m > 0 ? b : a;
      /* f's outgoing (slot 0) gains g; g's incoming (slot 1) gains f */
      const int64_t who[2] = {f, g};
      const int32_t other[2] = {(int32_t)g, (int32_t)f};
      for (int dir = 0; dir < 2; dir++) {
        const int64_t q = 4 * who[dir] + 2 * dir;   /* q: best, q + 1: runner-up */
        if (bi[q] < 0 || loop_before(am, c2, other[dir], bm[q], bc[q], bi[q])) {
          bm[q + 1] = bm[q]; bc[q + 1] = bc[q]; bi[q + 1] = bi[q];
          bm[q] = am; bc[q] = c2; bi[q] = other[dir];
        } else if (bi[q + 1] < 0 || loop_before(am, c2, other[dir], bm[q + 1], bc[q + 1], bi[q + 1])) {
          bm[q + 1] = am; bc[q + 1] = c2; bi[q + 1] = other[dir];
        }
      }
    }
  }
  for (int64_t t = 0; t < nt; t++) {
    next[t] = prev[t] = -1;
    next_chi2[t] = -1.0;
    for (int dir = 0; dir < 2; dir++) {
      const int64_t q = 4 * t + 2 * dir;
      if (bi[q + 1] >= 0 && bm[q + 1] == bm[q] && bc[q + 1] - bc[q] <= 0.01 * (bc[q] > 1.0 ? bc[q] : 1.0))
        borderline[t] = 1;
    }
  }
  int64_t links = 0;
  for (int64_t f = 0; f < nt; f++) {
    const int32_t g = bi[4 * f];
    if (g >= 0 && bi[4 * (int64_t)g + 2] == f) {
      next[f] = g;
      prev[g] = (int32_t)f;
      next_chi2[f] = bc[4 * f];
      links++;
    }
  }
  free(sec); free(loops); free(bm); free(bc); free(bi);
  return links;
}

/* ------------------------------------------------------------ 10. track-model compression
 * The paper gives online tracking as the way to compress TPC data ("Hardware
 * and data flow": the reconstruction runs online to reduce the data); this is
 * the library's definition of that compression of the clusters on tracks:
 *   - the track model is the step-8 fit: parameters p at x0 (the innermost
 *     cluster) carried along the exact helix from row to row (the predicted
 *     state only, no measurement updates), clusters taken innermost first;
 *   - a cluster's residuals are its measured (y, zeta) minus the prediction at
 *     its row; codes = rint(residual / step) (ties away from zero) for steps
 *     step_y, step_z;
 *   - a cluster is coded if both |codes| <= 127, otherwise escaped (kept raw);
 *     clusters after a failed transport are escaped;
 *   - decoding: prediction + code * step; the coded position is within step/2.
 * Output per cluster: status 0 (not on a track), 1 (coded), 2 (escaped);
 * q_y, q_z (may be NULL; test output): the residuals in steps before rounding,
 * NaN where no prediction was made. */
typedef struct {
  double step_y;   /* 0.0125 cm (1/32 pad) */
  double step_z;   /* 0.015625 cm (1/32 time bin) */
} orc_cmp_params;

int64_t orc_compress(const orc_input* in, const orc_params* P, const orc_cmp_params* CP, const orc_cluster* cl,
                     int64_t n, const int32_t* cl2trk, int64_t nt, const orc_fit* fits, int8_t* code_y,
                     int8_t* code_z, uint8_t* status, double* q_y, double* q_z) {
  const double u = 7.8125e-4;
  for (int64_t i = 0; i < n; i++) { code_y[i] = 0; code_z[i] = 0; status[i] = 0; }
  if (q_y) for (int64_t i = 0; i < n; i++) q_y[i] = q_z[i] = NAN;
  int64_t* cnt = (int64_t*)calloc((size_t)nt + 1, sizeof(int64_t));
  for (int64_t i = 0; i < n; i++) if (cl2trk[i] >= 0) cnt[cl2trk[i] + 1]++;
  for (int64_t t = 0; t < nt; t++) cnt[t + 1] += cnt[t];
  int64_t* lst = (int64_t*)malloc(sizeof(int64_t) * (cnt[nt] + 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (nt + 1));
  memcpy(fill, cnt, sizeof(int64_t) * nt);
  for (int64_t i = 0; i < n; i++) if (cl2trk[i] >= 0) lst[fill[cl2trk[i]]++] = i;
  int64_t coded = 0;
  for (int64_t t = 0; t < nt; t++) {
    double s[5], x = fits[t].x;
    for (int k = 0; k < 5; k++) s[k] = fits[t].par[k];
    int ok = 1;
    for (int64_t q = cnt[t]; q < cnt[t + 1]; q++) {
      const int64_t c = lst[q];
      int64_t X, Y, Z;
      orc_coords(in, &cl[c], &X, &Y, &Z);
      const double xc = (double)X * u;
      if (ok && xc != x) {
        double ns[5];
        if (orc_transport(P, s, xc - x, ns, NULL)) ok = 0;
        else { memcpy(s, ns, sizeof(ns)); x = xc; }
      }
      if (!ok) { status[c] = 2; continue; }
      const double ry = ((double)Y * u - s[0]) / CP->step_y, rz = ((double)Z * u - s[1]) / CP->step_z;
      if (q_y) { q_y[c] = ry; q_z[c] = rz; }
      const double cy = round(ry), cz = round(rz);
      if (fabs(cy) <= 127.0 && fabs(cz) <= 127.0) {
        code_y[c] = (int8_t)cy;
        code_z[c] = (int8_t)cz;
        status[c] = 1;
        coded++;
      } else {
        status[c] = 2;
      }
    }
  }
  free(cnt); free(lst); free(fill);
  return coded;
}

/* ------------------------------------------------------------ 10c. entropy coding of the codes
 * The library's definition of a bit stream for the step-10 codes (the size the
 * step reaches; the paper gives compression as the reason for online
 * tracking, "Hardware and data flow"):
 *   - symbols: code + 128 of the y and z codes of the coded clusters
 *     (status 1), one alphabet of 256 per component;
 *   - per component, Huffman code lengths from the symbol counts: the leaves
 *     (symbols with a count) ordered by (count, symbol) form queue A, new
 *     nodes join queue B in creation order; each merge takes the lighter of
 *     the two queue heads twice (a leaf before a node of equal weight), and a
 *     leaf's length is its depth (a single symbol gets length 1).  If a
 *     length exceeds 24, every count c becomes (c + 1) / 2 and the lengths
 *     are built again;
 *   - canonical codewords: symbols ordered by (length, symbol), the first
 *     gets 0, each next (previous + 1) << (length - previous length);
 *   - the stream: for each coded cluster in index order its y codeword then
 *     its z codeword, most significant bit first; stream bit b is bit
 *     31 - b % 32 of 32-bit word b / 32; the last word is zero-padded. */
#define ORC_MAX_CODE_LEN 24

/* Huffman lengths of one 256-symbol alphabet (count 0: length 0). */
static void huff_lengths(const uint64_t* count_in, uint8_t* len) {
  uint64_t c[256];
  for (int i = 0; i < 256; i++) c[i] = count_in[i];
  for (;;) {
    int leaves[256], n = 0;
    for (int i = 0; i < 256; i++) { len[i] = 0; if (c[i]) leaves[n++] = i; }
    if (n == 0) return;
    if (n == 1) { len[leaves[0]] = 1; return; }
    /* queue A: leaves by (count, symbol), insertion sort */
    for (int i = 1; i < n; i++)
      for (int j = i; j > 0 && (c[leaves[j]] < c[leaves[j - 1]] ||
                                (c[leaves[j]] == c[leaves[j - 1]] && leaves[j] < leaves[j - 1])); j--) {
        int t = leaves[j]; leaves[j] = leaves[j - 1]; leaves[j - 1] = t;
      }
    /* nodes 0..255 are the leaves (by symbol), 256.. the merged ones */
    int parent[512];
    uint64_t w[512];
    for (int i = 0; i < 512; i++) parent[i] = -1;
    for (int i = 0; i < 256; i++) w[i] = c[i];
    int qa = 0, qb = 256, nb = 256;   /* heads of A (index into leaves) and B (node id); next node id */
    for (int m = 0; m < n - 1; m++) {
      int pick[2];
      for (int k = 0; k < 2; k++) {
        int take_a;
        if (qa >= n) take_a = 0;
        else if (qb >= nb) take_a = 1;
        else take_a = w[leaves[qa]] <= w[qb];
        pick[k] = take_a ? leaves[qa++] : qb++;
      }
      w[nb] = w[pick[0]] + w[pick[1]];
      parent[pick[0]] = parent[pick[1]] = nb;
      nb++;
    }
    int maxlen = 0;
    for (int i = 0; i < n; i++) {
      int d = 0;
      for (int x = leaves[i]; parent[x] >= 0; x = parent[x]) d++;
      len[leaves[i]] = (uint8_t)(d > 255 ? 255 : d);
      if (d > maxlen) maxlen = d;
    }
    if (maxlen <= ORC_MAX_CODE_LEN) return;
    for (int i = 0; i < 256; i++) if (c[i]) c[i] = (c[i] + 1) / 2;
  }
}

/* Canonical codewords from the lengths. */
static void huff_codes(const uint8_t* len, uint32_t* code) {
  uint32_t next = 0;
  int prev_len = 0, first = 1;
  for (int l = 1; l <= ORC_MAX_CODE_LEN; l++)
    for (int s = 0; s < 256; s++) {
      if (len[s] != l) continue;
      if (first) { next = 0; first = 0; }
      else next = (next + 1) << (l - prev_len);
      code[s] = next;
      prev_len = l;
    }
}

/* Encode the codes of n clusters.  len_out[512]: the lengths of the y then
 * the z alphabet; words (may be NULL) receives the stream if it holds
 * cap_words words.  Returns the stream's length in bits. */
int64_t orc_entropy_encode(int64_t n, const int8_t* code_y, const int8_t* code_z, const uint8_t* status,
                           uint8_t* len_out, uint32_t* words, int64_t cap_words) {
  uint64_t hist[2][256];
  memset(hist, 0, sizeof(hist));
  for (int64_t i = 0; i < n; i++) {
    if (status[i] != 1) continue;
    hist[0][code_y[i] + 128]++;
    hist[1][code_z[i] + 128]++;
  }
  uint32_t code[2][256];
  memset(code, 0, sizeof(code));
  for (int k = 0; k < 2; k++) {
    huff_lengths(hist[k], len_out + 256 * k);
    huff_codes(len_out + 256 * k, code[k]);
  }
  int64_t nbits = 0;
  for (int64_t i = 0; i < n; i++)
    if (status[i] == 1) nbits += len_out[code_y[i] + 128] + len_out[256 + code_z[i] + 128];
  if (words && (nbits + 31) / 32 <= cap_words) {
    for (int64_t k = 0; k < (nbits + 31) / 32; k++) words[k] = 0;
    int64_t b = 0;
    for (int64_t i = 0; i < n; i++) {
      if (status[i] != 1) continue;
      for (int comp = 0; comp < 2; comp++) {
        const int sym = (comp ? code_z[i] : code_y[i]) + 128;
        const int l = len_out[256 * comp + sym];
        const uint32_t cw = code[comp][sym];
        for (int j = l - 1; j >= 0; j--, b++)
          if ((cw >> j) & 1u) words[b / 32] |= 1u << (31 - b % 32);
      }
    }
  }
  return nbits;
}

/* ------------------------------------------------------------ 11. drift calibration
 * The paper lists calibration among the EPNs' tasks ("Hardware and data flow");
 * this is the library's definition of a drift-velocity / T0 calibration from
 * tracks of a collision whose vertex lies on the beam axis at z = 0:
 *   - per step-8 track with >= 20 clusters and no flag, its state is carried
 *     along the exact helix from its reference x to x = 0 (the beam axis); it
 *     is used if |y| there is below 3 cm;
 *   - the time bin of the vertex, t_v = zeta(x = 0) / (zeta per time bin):
 *     its most populated whole bin b* (tracks with floor(t_v) = b, lowest b on
 *     ties) locates it; the mean over the tracks within 3 bins of b* + 0.5,
 *     then over those within 1.5 bins of that mean, estimates it;
 *   - with a known collision time t0 and drift length L, the drift velocity is
 *     off by eps = (L / zeta_per_bin) / (t_v - t0) - 1 (the vertex's charge
 *     drifts the full length); with a known drift velocity, t0 = t_v - L /
 *     zeta_per_bin. */
int64_t orc_calibrate_drift(const orc_params* P, const orc_fit* fits, const int32_t* ncl, int64_t nt,
                            double zeta_per_bin, double* t_vertex, double* tv_track, uint8_t* used) {
  for (int64_t t = 0; t < nt; t++) {
    used[t] = 0;
    tv_track[t] = 0.0;
    if (ncl[t] < 20 || fits[t].flags) continue;
    double s[5], out[5];
    for (int k = 0; k < 5; k++) s[k] = fits[t].par[k];
    if (orc_transport(P, s, -fits[t].x, out, NULL)) continue;
    if (fabs(out[0]) >= 3.0) continue;
    tv_track[t] = out[1] / zeta_per_bin;
    used[t] = 1;
  }
  /* mode of floor(t_v) over [0, nbins) */
  const int64_t nbins = 1 << 20;
  int64_t* h = (int64_t*)calloc((size_t)nbins, sizeof(int64_t));
  for (int64_t t = 0; t < nt; t++)
    if (used[t] && tv_track[t] >= 0.0 && tv_track[t] < (double)nbins) h[(int64_t)floor(tv_track[t])]++;
  int64_t best = -1;
  for (int64_t b = 0; b < nbins; b++)
    if (h[b] > 0 && (best < 0 || h[b] > h[best])) best = b;
  free(h);
  if (best < 0) { *t_vertex = 0.0; return 0; }
  double centre = (double)best + 0.5;
  const double win[2] = {3.0, 1.5};
  int64_t nu = 0;
  for (int pass = 0; pass < 2; pass++) {
    double sum = 0.0;
    int64_t cnt = 0;
    for (int64_t t = 0; t < nt; t++)
      if (used[t] && fabs(tv_track[t] - centre) <= win[pass]) { sum += tv_track[t]; cnt++; }
    if (cnt == 0) { *t_vertex = 0.0; return 0; }
    centre = sum / (double)cnt;
    nu = cnt;
  }
  *t_vertex = centre;
  return nu;
}
