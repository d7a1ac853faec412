/*
 * tpcgen.c — seeded synthetic TPC timeframe generator.
 *
 * Input module shared by the tests, the benchmark and the smoke check.  It
 * simulates helical tracks from the vertex in a solenoidal field, deposits a 2D
 * Gaussian charge cloud per pad-row crossing (Landau-distributed amplitude),
 * adds Gaussian pixel noise, digitises to 10-bit ADCs, applies the
 * zero-suppression threshold and writes the ZS pages of the library's input
 * format.  Zero suppression itself happens upstream of the EPN in the paper
 * (section "Hardware and data flow": ZS in the FPGA user logic of the readout),
 * which is why the encoder lives here, with the input, and not in the
 * reconstruction.  Nothing here decodes pages, finds clusters or fits tracks.
 *
 * Determinism: every random number comes from a xoshiro256** stream seeded by
 * splitmix64 over (seed, purpose, index...), so the output does not depend on
 * the number of threads.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ZS_MAGIC 0x5A53u
#define FRAG 256
#define HALO 3

typedef struct {
  uint64_t seed;
  int32_t n_sectors;
  int32_t n_rows;
  const int32_t* npads;
  const int32_t* row_x;        /* units of 0.05 cm */
  int32_t n_time_bins;
  int32_t n_collisions;
  const double* coll_t0;       /* time bin at which drift from the central electrode starts */
  const int32_t* coll_ntracks; /* tracks per collision, loopers included */
  double looper_frac;
  double pt_min, pt_mean_excess;
  double looper_pt_min, looper_pt_max;
  double eta_min, eta_max;
  double phi_min, phi_max;
  double bz;
  double drift_length;
  double bin_cm;
  double outer_radius;
  double sigma_pad, sigma_time;
  double landau_mpv, landau_xi, amp_cap;
  double noise_sigma;
  int32_t zs_threshold;
  int32_t max_turns;
  int32_t want_labels;
  int32_t n_threads;
} tpcgen_config;

typedef struct {
  double pt, phi, eta, t0;
  int32_t charge, collision, looper, n_hits;
} tpcgen_track;

typedef struct {
  double pad, time;
  float amp;
  int32_t sector, row, track, leg;
} tpcgen_hit;

typedef struct {
  uint8_t* pages;
  uint64_t pages_bytes;
  uint64_t* page_offsets;
  int64_t n_pages;
  int64_t n_digits;
  int32_t* digit_labels;
  int64_t n_tracks;
  tpcgen_track* tracks;
  int64_t n_hits;
  tpcgen_hit* hits;
} tpcgen_result;

/* ---------------------------------------------------------------- RNG */
static inline uint64_t splitmix64(uint64_t* x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
typedef struct { uint64_t s[4]; } rng_t;
static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static inline uint64_t rng_next(rng_t* r) {
  uint64_t* s = r->s;
  uint64_t res = rotl(s[1] * 5, 7) * 9, t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3]; s[2] ^= t; s[3] = rotl(s[3], 45);
  return res;
}
static void rng_seed(rng_t* r, uint64_t seed, uint64_t a, uint64_t b, uint64_t c) {
  uint64_t x = seed ^ (a * 0xD1B54A32D192ED03ull) ^ (b * 0xABC98388FB8FAC03ull) ^ (c * 0x8CB92BA72F3D8DD7ull);
  for (int i = 0; i < 4; i++) r->s[i] = splitmix64(&x);
}
/* uniform in (0, 1) */
static inline double rng_u(rng_t* r) { return ((rng_next(r) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
static inline double rng_normal(rng_t* r) {
  double u1 = rng_u(r), u2 = rng_u(r);
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}
/* standard normal conditioned on x >= a (a > 0): Marsaglia's 1964 tail method */
static inline double rng_normal_tail(rng_t* r, double a) {
  for (;;) {
    double x = sqrt(a * a - 2.0 * log(rng_u(r)));
    if (rng_u(r) * x <= a) return x;
  }
}
/* Landau-like amplitude: alpha = 1, beta = 1 stable variate by Chambers,
 * Mallows and Stuck (1976), shifted so that its mode sits at mpv. */
#define STABLE11_MODE (-0.42931451)
static inline double rng_landau(rng_t* r, double mpv, double xi) {
  const double hp = 1.5707963267948966;
  double w = 3.141592653589793 * (rng_u(r) - 0.5);
  double e = -log(rng_u(r));
  double x = (1.0 / hp) * ((hp + w) * tan(w) - log(hp * e * cos(w) / (hp + w)));
  return mpv + xi * (x - STABLE11_MODE);
}

/* ---------------------------------------------------------------- hits */
typedef struct {
  tpcgen_hit* v;
  int64_t n, cap;
} hitvec;
static void hv_push(hitvec* h, tpcgen_hit x) {
  if (h->n == h->cap) {
    h->cap = h->cap ? 2 * h->cap : 256;
    h->v = (tpcgen_hit*)realloc(h->v, (size_t)h->cap * sizeof(tpcgen_hit));
  }
  h->v[h->n++] = x;
}

static int hit_cmp_s(const void* a, const void* b) {
  double sa = ((const double*)a)[0], sb = ((const double*)b)[0];
  return (sa > sb) - (sa < sb);
}

/* All pad-row crossings of one track, in order of arc length. */
static void track_hits(const tpcgen_config* c, const tpcgen_track* tr, int32_t tid, hitvec* out) {
  const double PI = 3.141592653589793;
  double R = 100.0 * tr->pt / (0.299792458 * c->bz);
  double om = -(double)tr->charge / R; /* dphi/ds */
  double tl = sinh(tr->eta);
  double period = 2.0 * PI * R;
  double s_exit = 1e300;
  if (2.0 * R > c->outer_radius) s_exit = 2.0 * R * asin(c->outer_radius / (2.0 * R));
  int side_c = tl < 0.0;
  /* collect (s, sector, row, pad, time, branch) then sort by s */
  typedef struct { double s, pad, time; int32_t sector, row, leg; } cand;
  cand* cv = NULL;
  int64_t nc = 0, capc = 0;
  for (int s = 0; s < c->n_sectors; s++) {
    int is_c = (s >= 18);
    if (c->n_sectors > 1 && is_c != side_c) continue;
    if (c->n_sectors == 1 && side_c) continue;
    double alpha = ((s % 18) + 0.5) * (20.0 * PI / 180.0);
    double pl0 = tr->phi - alpha;
    double sp0 = sin(pl0), cp0 = cos(pl0);
    for (int r = 0; r < c->n_rows; r++) {
      double X = c->row_x[r] * 0.05;
      double v = sp0 + om * X;
      if (v < -1.0 || v > 1.0) continue;
      double as = asin(v);
      for (int br = 0; br < 2; br++) {
        double th = br == 0 ? as : PI - as;
        double sb = fmod((th - pl0) / om, period);
        if (sb <= 0.0) sb += period;
        double yl = (cp0 - cos(th)) / om;
        int np = c->npads[r];
        double pc = yl / 0.4 + 0.5 * (np - 1);
        if (pc < -0.5 || pc >= np - 0.5) continue;
        for (int m = 0; m < c->max_turns; m++) {
          double sa = sb + m * period;
          if (sa >= s_exit) break;
          double z = sa * tl;
          if (fabs(z) >= c->drift_length) break;
          double tc = tr->t0 + (c->drift_length - fabs(z)) / c->bin_cm;
          if (tc < -0.5 || tc >= c->n_time_bins - 0.5) continue;
          if (nc == capc) {
            capc = capc ? 2 * capc : 128;
            cv = (cand*)realloc(cv, (size_t)capc * sizeof(cand));
          }
          cv[nc].s = sa; cv[nc].pad = pc; cv[nc].time = tc;
          cv[nc].sector = s; cv[nc].row = r; cv[nc].leg = m;
          nc++;
        }
      }
    }
  }
  qsort(cv, (size_t)nc, sizeof(cand), hit_cmp_s);
  for (int64_t i = 0; i < nc; i++) {
    tpcgen_hit h;
    h.pad = cv[i].pad; h.time = cv[i].time; h.amp = 0.f;
    h.sector = cv[i].sector; h.row = cv[i].row; h.track = tid; h.leg = cv[i].leg;
    hv_push(out, h);
  }
  free(cv);
}

/* ---------------------------------------------------------------- pages */
typedef struct {
  uint8_t* b;
  size_t n, cap;
} bytevec;
static void bv_reserve(bytevec* v, size_t extra) {
  if (v->n + extra > v->cap) {
    size_t nc = v->cap ? v->cap : 4096;
    while (nc < v->n + extra) nc *= 2;
    v->b = (uint8_t*)realloc(v->b, nc);
    v->cap = nc;
  }
}
static inline void put16(uint8_t* p, uint16_t x) { p[0] = (uint8_t)x; p[1] = (uint8_t)(x >> 8); }
static inline void put32(uint8_t* p, uint32_t x) {
  p[0] = (uint8_t)x; p[1] = (uint8_t)(x >> 8); p[2] = (uint8_t)(x >> 16); p[3] = (uint8_t)(x >> 24);
}

/* Encode one window (fragment f of a row) from the digitised plane adc[t][p]. */
static void encode_page(bytevec* out, const uint16_t* adc, int np, int T, int f, int sector, int row,
                        int thr, const int32_t* lab_plane, int32_t** labs, int64_t* nlabs, int64_t* labcap,
                        uint8_t* scratch_e, uint8_t* scratch_r, uint16_t* scratch_q) {
  int t0 = f * FRAG, t1 = t0 + FRAG;
  if (t1 > T) t1 = T;
  int ne = 0, nr = 0, nd = 0;
  int lo_tb = 0, lo_r = 0, lo_d = 0, hi_tb = -1, hi_r = 0, hi_d = 0;
  for (int t = t0; t < t1; t++) {
    int tt = t - t0;
    const uint16_t* rowp = adc + (size_t)t * np;
    int runs_here = 0;
    int p = 0;
    if (tt >= FRAG - HALO && hi_tb < 0) { hi_tb = ne; hi_r = nr; hi_d = nd; }
    while (p < np) {
      if (rowp[p] < thr) { p++; continue; }
      int ps = p;
      while (p < np && rowp[p] >= thr) {
        scratch_q[nd] = rowp[p];
        if (labs) {
          if (*nlabs == *labcap) {
            *labcap = *labcap ? 2 * *labcap : 4096;
            *labs = (int32_t*)realloc(*labs, (size_t)*labcap * sizeof(int32_t));
          }
          (*labs)[(*nlabs)++] = lab_plane[(size_t)t * np + p];
        }
        nd++; p++;
      }
      scratch_r[2 * nr] = (uint8_t)ps;
      scratch_r[2 * nr + 1] = (uint8_t)(p - ps);
      nr++;
      runs_here++;
    }
    if (runs_here) {
      scratch_e[2 * ne] = (uint8_t)tt;
      scratch_e[2 * ne + 1] = (uint8_t)runs_here;
      ne++;
    }
    if (tt == HALO - 1) { lo_tb = ne; lo_r = nr; lo_d = nd; }
  }
  if (t1 - t0 < HALO) { lo_tb = ne; lo_r = nr; lo_d = nd; }
  if (hi_tb < 0) { hi_tb = ne; hi_r = nr; hi_d = nd; }
  size_t body = 32 + 2 * (size_t)ne + 2 * (size_t)nr;
  body = (body + 3) & ~(size_t)3;
  size_t nw = ((size_t)nd + 2) / 3;
  size_t len = body + 4 * nw;
  len = (len + 15) & ~(size_t)15;
  bv_reserve(out, len);
  uint8_t* pg = out->b + out->n;
  memset(pg, 0, len);
  put32(pg + 0, (uint32_t)len);
  put16(pg + 4, (uint16_t)ne);
  put16(pg + 6, (uint16_t)nr);
  put16(pg + 8, (uint16_t)nd);
  pg[10] = (uint8_t)sector; pg[11] = (uint8_t)row;
  put16(pg + 12, (uint16_t)f);
  put16(pg + 14, ZS_MAGIC);
  put16(pg + 16, (uint16_t)lo_tb); put16(pg + 18, (uint16_t)lo_r); put16(pg + 20, (uint16_t)lo_d);
  put16(pg + 22, (uint16_t)hi_tb); put16(pg + 24, (uint16_t)hi_r); put16(pg + 26, (uint16_t)hi_d);
  memcpy(pg + 32, scratch_e, 2 * (size_t)ne);
  memcpy(pg + 32 + 2 * ne, scratch_r, 2 * (size_t)nr);
  for (size_t w = 0; w < nw; w++) {
    uint32_t word = 0;
    for (int k = 0; k < 3; k++) {
      size_t d = 3 * w + k;
      if (d < (size_t)nd) word |= (uint32_t)(scratch_q[d] & 1023u) << (10 * k);
    }
    put32(pg + body + 4 * w, word);
  }
  out->n += len;
}

/* ---------------------------------------------------------------- main */
typedef struct {
  bytevec pages;
  int32_t* labs;
  int64_t nlabs, labcap;
  int64_t ndig;
  uint64_t* page_len; /* per fragment */
} rowout;

int tpcgen_generate(const tpcgen_config* c, tpcgen_result** res_out) {
  const double PI = 3.141592653589793;
  if (!c || !res_out || c->n_rows <= 0 || c->n_sectors <= 0 || c->n_time_bins <= 0) return -1;
  for (int r = 0; r < c->n_rows; r++)
    if (c->npads[r] < 3 || c->npads[r] > 255) return -1;
#ifdef _OPENMP
  if (c->n_threads > 0) omp_set_num_threads(c->n_threads);
#endif
  /* ---- tracks */
  int64_t ntr = 0;
  for (int k = 0; k < c->n_collisions; k++) ntr += c->coll_ntracks[k];
  tpcgen_track* tracks = (tpcgen_track*)calloc((size_t)(ntr ? ntr : 1), sizeof(tpcgen_track));
  {
    int64_t i = 0;
    for (int k = 0; k < c->n_collisions; k++) {
      rng_t r;
      rng_seed(&r, c->seed, 1, (uint64_t)k, 0);
      int n = c->coll_ntracks[k];
      int nl = (int)floor(n * c->looper_frac + 0.5);
      for (int j = 0; j < n; j++, i++) {
        tpcgen_track* t = &tracks[i];
        t->collision = k;
        t->t0 = c->coll_t0[k];
        t->looper = j >= n - nl;
        t->charge = rng_u(&r) < 0.5 ? -1 : 1;
        t->phi = c->phi_min + (c->phi_max - c->phi_min) * rng_u(&r);
        t->eta = c->eta_min + (c->eta_max - c->eta_min) * rng_u(&r);
        if (t->looper)
          t->pt = c->looper_pt_min + (c->looper_pt_max - c->looper_pt_min) * rng_u(&r);
        else
          t->pt = c->pt_min - c->pt_mean_excess * log(rng_u(&r));
        t->n_hits = 0;
      }
    }
  }
  /* ---- hits per track (parallel), then amplitudes per track stream */
  hitvec* th = (hitvec*)calloc((size_t)(ntr ? ntr : 1), sizeof(hitvec));
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < ntr; i++) {
    track_hits(c, &tracks[i], (int32_t)i, &th[i]);
    rng_t r;
    rng_seed(&r, c->seed, 2, (uint64_t)i, 0);
    for (int64_t j = 0; j < th[i].n; j++) {
      double a = rng_landau(&r, c->landau_mpv, c->landau_xi);
      if (a > c->amp_cap) a = c->amp_cap;
      if (a < 1.0) a = 1.0;
      th[i].v[j].amp = (float)a;
    }
    tracks[i].n_hits = (int32_t)th[i].n;
  }
  /* ---- bucket hits by (sector, row), stable in track order */
  int64_t nsr = (int64_t)c->n_sectors * c->n_rows;
  int64_t* bstart = (int64_t*)calloc((size_t)nsr + 1, sizeof(int64_t));
  int64_t nh = 0;
  for (int64_t i = 0; i < ntr; i++)
    for (int64_t j = 0; j < th[i].n; j++) {
      bstart[(int64_t)th[i].v[j].sector * c->n_rows + th[i].v[j].row + 1]++;
      nh++;
    }
  for (int64_t b = 0; b < nsr; b++) bstart[b + 1] += bstart[b];
  tpcgen_hit* hits = (tpcgen_hit*)malloc((size_t)(nh ? nh : 1) * sizeof(tpcgen_hit));
  {
    int64_t* fill = (int64_t*)malloc((size_t)nsr * sizeof(int64_t));
    memcpy(fill, bstart, (size_t)nsr * sizeof(int64_t));
    for (int64_t i = 0; i < ntr; i++) {
      for (int64_t j = 0; j < th[i].n; j++) {
        int64_t b = (int64_t)th[i].v[j].sector * c->n_rows + th[i].v[j].row;
        hits[fill[b]++] = th[i].v[j];
      }
      free(th[i].v);
    }
    free(fill);
  }
  free(th);
  /* ---- per (sector, row): deposit, noise, digitise, encode */
  int T = c->n_time_bins;
  int nfrag = (T + FRAG - 1) / FRAG;
  int npmax = 0;
  for (int r = 0; r < c->n_rows; r++) if (c->npads[r] > npmax) npmax = c->npads[r];
  rowout* ro = (rowout*)calloc((size_t)nsr, sizeof(rowout));
  const double two_pi_sp_st = 2.0 * PI * c->sigma_pad * c->sigma_time;
  const double a_tail = (c->zs_threshold - 0.5) / c->noise_sigma;
  const double p_tail = 0.5 * erfc(a_tail / sqrt(2.0));
  const double log1mp = log1p(-p_tail);
#pragma omp parallel
  {
    size_t plane_n = (size_t)T * npmax;
    float* sig = (float*)malloc(plane_n * sizeof(float));
    float* best = c->want_labels ? (float*)malloc(plane_n * sizeof(float)) : NULL;
    int32_t* lab = c->want_labels ? (int32_t*)malloc(plane_n * sizeof(int32_t)) : NULL;
    uint16_t* adc = (uint16_t*)malloc(plane_n * sizeof(uint16_t));
    uint8_t* se = (uint8_t*)malloc(2 * FRAG);
    uint8_t* sr = (uint8_t*)malloc(2 * (size_t)FRAG * 128);
    uint16_t* sq = (uint16_t*)malloc(sizeof(uint16_t) * (size_t)FRAG * 256);
#pragma omp for schedule(dynamic, 1)
    for (int64_t b = 0; b < nsr; b++) {
      int s = (int)(b / c->n_rows), r = (int)(b % c->n_rows);
      int np = c->npads[r];
      size_t n = (size_t)T * np;
      memset(sig, 0, n * sizeof(float));
      if (lab) {
        memset(best, 0, n * sizeof(float));
        for (size_t i = 0; i < n; i++) lab[i] = -1;
      }
      for (int64_t h = bstart[b]; h < bstart[b + 1]; h++) {
        const tpcgen_hit* hh = &hits[h];
        int p0 = (int)floor(hh->pad - 3.0), p1 = (int)ceil(hh->pad + 3.0);
        int q0 = (int)floor(hh->time - 4.0), q1 = (int)ceil(hh->time + 4.0);
        if (p0 < 0) p0 = 0;
        if (p1 > np - 1) p1 = np - 1;
        if (q0 < 0) q0 = 0;
        if (q1 > T - 1) q1 = T - 1;
        double fp[16], ft[16];
        const double isq2 = 0.7071067811865476;
        for (int p = p0; p <= p1; p++)
          fp[p - p0] = 0.5 * (erfc(-(p + 0.5 - hh->pad) / c->sigma_pad * isq2) -
                              erfc(-(p - 0.5 - hh->pad) / c->sigma_pad * isq2));
        for (int t = q0; t <= q1; t++)
          ft[t - q0] = 0.5 * (erfc(-(t + 0.5 - hh->time) / c->sigma_time * isq2) -
                              erfc(-(t - 0.5 - hh->time) / c->sigma_time * isq2));
        double A = hh->amp * two_pi_sp_st;
        for (int t = q0; t <= q1; t++)
          for (int p = p0; p <= p1; p++) {
            float w = (float)(A * fp[p - p0] * ft[t - q0]);
            size_t i = (size_t)t * np + p;
            sig[i] += w;
            if (lab && w > best[i]) { best[i] = w; lab[i] = hh->track; }
          }
      }
      /* digitise: explicit noise where there is signal, tail sampling elsewhere */
      rng_t rs, rt;
      rng_seed(&rs, c->seed, 3, (uint64_t)s, (uint64_t)r);
      rng_seed(&rt, c->seed, 4, (uint64_t)s, (uint64_t)r);
      for (size_t i = 0; i < n; i++) {
        if (sig[i] > 0.f) {
          double v = rint(sig[i] + c->noise_sigma * rng_normal(&rs));
          if (v < 0) v = 0;
          if (v > 1023) v = 1023;
          adc[i] = (uint16_t)v;
        } else {
          adc[i] = 0;
        }
      }
      if (p_tail > 0.0) {
        size_t i = 0;
        for (;;) {
          double g = floor(log(rng_u(&rt)) / log1mp);
          if (g > (double)n) break;
          i += (size_t)g;
          if (i >= n) break;
          double v = rint(c->noise_sigma * rng_normal_tail(&rt, a_tail));
          if (v > 1023) v = 1023;
          if (sig[i] <= 0.f) {
            adc[i] = (uint16_t)v;
            if (lab) lab[i] = -1;
          }
          i++;
        }
      }
      rowout* o = &ro[b];
      o->page_len = (uint64_t*)malloc((size_t)nfrag * sizeof(uint64_t));
      for (int f = 0; f < nfrag; f++) {
        size_t before = o->pages.n;
        int64_t nl0 = o->nlabs;
        encode_page(&o->pages, adc, np, T, f, s, r, c->zs_threshold, lab, lab ? &o->labs : NULL,
                    &o->nlabs, &o->labcap, se, sr, sq);
        o->page_len[f] = o->pages.n - before;
        (void)nl0;
      }
      /* digits of this row: count from the labels or from the plane */
      int64_t nd = 0;
      for (size_t i = 0; i < n; i++) nd += adc[i] >= c->zs_threshold;
      o->ndig = nd;
    }
    free(sig); free(best); free(lab); free(adc); free(se); free(sr); free(sq);
  }
  /* ---- concatenate */
  tpcgen_result* res = (tpcgen_result*)calloc(1, sizeof(tpcgen_result));
  uint64_t total = 0;
  int64_t ndig = 0, nlab = 0;
  for (int64_t b = 0; b < nsr; b++) { total += ro[b].pages.n; ndig += ro[b].ndig; nlab += ro[b].nlabs; }
  res->pages = (uint8_t*)malloc(total ? total : 16);
  res->pages_bytes = total;
  res->n_pages = nsr * nfrag;
  res->page_offsets = (uint64_t*)malloc((size_t)res->n_pages * sizeof(uint64_t));
  res->n_digits = ndig;
  if (c->want_labels) res->digit_labels = (int32_t*)malloc((size_t)(nlab ? nlab : 1) * sizeof(int32_t));
  uint64_t off = 0;
  int64_t lo = 0;
  for (int64_t b = 0; b < nsr; b++) {
    memcpy(res->pages + off, ro[b].pages.b, ro[b].pages.n);
    uint64_t o2 = off;
    for (int f = 0; f < nfrag; f++) {
      res->page_offsets[b * nfrag + f] = o2;
      o2 += ro[b].page_len[f];
    }
    off += ro[b].pages.n;
    if (c->want_labels && ro[b].nlabs) {
      memcpy(res->digit_labels + lo, ro[b].labs, (size_t)ro[b].nlabs * sizeof(int32_t));
      lo += ro[b].nlabs;
    }
    free(ro[b].pages.b); free(ro[b].labs); free(ro[b].page_len);
  }
  free(ro);
  free(bstart);
  res->n_tracks = ntr;
  res->tracks = tracks;
  res->n_hits = nh;
  res->hits = hits;
  *res_out = res;
  return 0;
}

void tpcgen_free(tpcgen_result* r) {
  if (!r) return;
  free(r->pages); free(r->page_offsets); free(r->digit_labels); free(r->tracks); free(r->hits);
  free(r);
}

/* Landau amplitudes alone, for checking the sampler. */
void tpcgen_sample_landau(uint64_t seed, int64_t n, double mpv, double xi, double* out) {
  rng_t r;
  rng_seed(&r, seed, 9, 0, 0);
  for (int64_t i = 0; i < n; i++) out[i] = rng_landau(&r, mpv, xi);
}
