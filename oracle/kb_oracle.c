/*
 * kb_oracle.c -- plain, slow, FP64 CPU oracle for the KBMOD shift-and-stack search with
 * the in-line sigma-G lightcurve clip (Smotherman et al. 2021, "Sifting Through the Static",
 * arXiv 2109.03296).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg may load this library.  It shares no code, header, table or constant with the CUDA path.
 *
 * Every function follows the definition it cites, in the order the paper states it, with no
 * blocking, fusion or pruning: every (start pixel, trajectory) pair is evaluated in full.
 * Floating point is FP64 throughout, except the three FP32 operations of the canonical track
 * rounding (kbo_track_offsets), which are part of the definition of an integer-pixel track.
 * Build with -ffp-contract=off so that no multiply-add is fused.
 *
 * Readings of points the paper leaves open (listed with their reasons in the design notes):
 *   R0  psi_t = (I_t w_t) correlated with P_t, phi_t = w_t correlated with P_t^2, w = 1/var;
 *       zero weight outside the image and at masked pixels, no edge renormalisation;
 *       psi = phi = 0 at a masked pixel.
 *   R1  track offset = floor(fl32(fl32(vx) * fl32(t_t - t_0)) + 0.5f), round half up.
 *   R2  percentiles: linear interpolation between order statistics (Hyndman-Fan type 7).
 *   R3  the clipped lightcurve is the flux psi_t/phi_t (clip_on = 0) or the per-epoch
 *       likelihood psi_t/sqrt(phi_t) (clip_on = 1).
 *   R4  keep iff  median - n sigma_G <= a_t <= median + n sigma_G  (inclusive).
 *   R5  per-pixel top-K ordered by L' descending, ties by lower trajectory index.
 *   R7  sigma_G = C (x_hi - x_lo) with C = 1 / (sqrt2 (erfinv(2 q_hi - 1) - erfinv(2 q_lo - 1))),
 *       i.e. Eq. 3 solved for sigma_G (Eq. 4 as printed drops the sqrt2 of Eq. 3).
 *   R8  threshold and top-K act on the clipped L'.
 *   R9  an epoch is valid iff its track position is inside the image and phi > 0 there
 *       (both psi and phi finite); a trajectory needs at least min_obs valid epochs.
 *   R12 stamps use all valid epochs, or only kept ones when a keep mask is given.
 *   R13 bilinear sampling: pixel centres at integer coordinates, cell = floor of the position.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KBO_MAX_T 4096

/* ---------------------------------------------------------------------------------------- */
/* Small helpers                                                                            */
/* ---------------------------------------------------------------------------------------- */

static int cmp_double(const void* a, const void* b) {
  double x = *(const double*)a, y = *(const double*)b;
  return (x > y) - (x < y);
}

/* erf^{-1}(y) for |y| < 1 by bisection on the C99 libm erf: erf is strictly increasing, so
 * 200 halvings of [-6, 6] pin the root to the last bit of a double. */
double kbo_erfinv(double y) {
  if (!(y > -1.0 && y < 1.0)) return NAN;
  double lo = -6.0, hi = 6.0;
  for (int i = 0; i < 200; ++i) {
    double mid = 0.5 * (lo + hi);
    if (erf(mid) < y) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* Coefficient C of sigma_G = C (x_hi - x_lo): Section 3.1, Eqs. 2-5, with the sqrt2 of Eq. 3. */
double kbo_sigma_g_coeff(double q_lo, double q_hi) {
  return 1.0 / (sqrt(2.0) * (kbo_erfinv(2.0 * q_hi - 1.0) - kbo_erfinv(2.0 * q_lo - 1.0)));
}

/* Percentile of n ascending values by linear interpolation between order statistics (R2). */
double kbo_percentile_sorted(const double* s, int n, double q) {
  double h = (double)(n - 1) * q;
  int lo = (int)floor(h);
  if (lo < 0) lo = 0;
  if (lo > n - 1) lo = n - 1;
  int hi = lo + 1 < n ? lo + 1 : n - 1;
  return s[lo] + (h - (double)lo) * (s[hi] - s[lo]);
}

/* sigma-G clip of one lightcurve (Section 3.1: reject every point not within +-n sigma_G of the
 * median).  a[0..n) are the lightcurve values; keep[i] is set to 1 for kept points.  Returns the
 * number kept.  med/sg (nullable) receive the median and sigma_G. */
int kbo_sigma_g_clip(const double* a, int n, double q_lo, double q_mid, double q_hi,
                     double n_sigma, uint8_t* keep, double* med, double* sg) {
  if (n <= 0) return 0;
  double* s = (double*)malloc(sizeof(double) * (size_t)n);
  memcpy(s, a, sizeof(double) * (size_t)n);
  qsort(s, (size_t)n, sizeof(double), cmp_double);
  double x_lo = kbo_percentile_sorted(s, n, q_lo);
  double x_mid = kbo_percentile_sorted(s, n, q_mid);
  double x_hi = kbo_percentile_sorted(s, n, q_hi);
  free(s);
  double sigma_g = kbo_sigma_g_coeff(q_lo, q_hi) * (x_hi - x_lo);
  double lower = x_mid - n_sigma * sigma_g, upper = x_mid + n_sigma * sigma_g;
  int kept = 0;
  for (int i = 0; i < n; ++i) {
    keep[i] = (uint8_t)(a[i] >= lower && a[i] <= upper);
    kept += keep[i];
  }
  if (med) *med = x_mid;
  if (sg) *sg = sigma_g;
  return kept;
}

/* ---------------------------------------------------------------------------------------- */
/* Track offsets (R1)                                                                       */
/* ---------------------------------------------------------------------------------------- */

static int32_t track_offset(float v, double t, double t0) {
  float dt = (float)(t - t0);
  float d = v * dt;         /* one IEEE single multiply */
  float e = d + 0.5f;       /* one IEEE single add */
  return (int32_t)floorf(e);
}

void kbo_track_offsets(const double* times, int T, const float* vx, const float* vy, int n,
                       int32_t* offx, int32_t* offy) {
  for (int j = 0; j < n; ++j)
    for (int t = 0; t < T; ++t) {
      offx[(size_t)j * T + t] = track_offset(vx[j], times[t], times[0]);
      offy[(size_t)j * T + t] = track_offset(vy[j], times[t], times[0]);
    }
}

/* ---------------------------------------------------------------------------------------- */
/* psi / phi likelihood images (Section 3, R0)                                               */
/* ---------------------------------------------------------------------------------------- */

static int pixel_masked(const float* img, const float* var, const uint8_t* mask, size_t i) {
  if (mask && mask[i]) return 1;
  double v = var[i], x = img[i];
  if (!isfinite(v) || v <= 0.0) return 1;
  if (!isfinite(x)) return 1;
  return 0;
}

void kbo_psi_phi(const float* img, const float* var, const uint8_t* mask, const float* psf,
                 int T, int H, int W, int k, double* psi, double* phi) {
  int r = k / 2;
  size_t hw = (size_t)H * W;
#pragma omp parallel for collapse(2) schedule(static)
  for (int t = 0; t < T; ++t)
    for (int y = 0; y < H; ++y) {
      const float* P = psf + (size_t)t * k * k;
      size_t base = (size_t)t * hw;
      for (int x = 0; x < W; ++x) {
        size_t o = base + (size_t)y * W + x;
        if (pixel_masked(img, var, mask, o)) { psi[o] = 0.0; phi[o] = 0.0; continue; }
        double s_psi = 0.0, s_phi = 0.0;
        for (int uy = -r; uy <= r; ++uy) {
          int yy = y + uy;
          if (yy < 0 || yy >= H) continue;
          for (int ux = -r; ux <= r; ++ux) {
            int xx = x + ux;
            if (xx < 0 || xx >= W) continue;
            size_t i = base + (size_t)yy * W + xx;
            if (pixel_masked(img, var, mask, i)) continue;
            double w = 1.0 / (double)var[i];
            double p = (double)P[(uy + r) * k + (ux + r)];
            s_psi += w * (double)img[i] * p;
            s_phi += w * p * p;
          }
        }
        psi[o] = s_psi;
        phi[o] = s_phi;
      }
    }
}

/* psi/phi at a list of sample pixels only (t, y, x triples), for full-size spot checks; a triple
 * outside [0,T) x [0,H) x [0,W) gets NaN. */
void kbo_psi_phi_at(const float* img, const float* var, const uint8_t* mask, const float* psf,
                    int T, int H, int W, int k, const int32_t* tyx, int n, double* psi,
                    double* phi) {
  int r = k / 2;
  size_t hw = (size_t)H * W;
#pragma omp parallel for schedule(static)
  for (int s = 0; s < n; ++s) {
    int t = tyx[3 * s], y = tyx[3 * s + 1], x = tyx[3 * s + 2];
    if (t < 0 || t >= T || y < 0 || y >= H || x < 0 || x >= W) {
      psi[s] = NAN;
      phi[s] = NAN;
      continue;
    }
    const float* P = psf + (size_t)t * k * k;
    size_t base = (size_t)t * hw;
    size_t o = base + (size_t)y * W + x;
    if (pixel_masked(img, var, mask, o)) { psi[s] = 0.0; phi[s] = 0.0; continue; }
    double s_psi = 0.0, s_phi = 0.0;
    for (int uy = -r; uy <= r; ++uy) {
      int yy = y + uy;
      if (yy < 0 || yy >= H) continue;
      for (int ux = -r; ux <= r; ++ux) {
        int xx = x + ux;
        if (xx < 0 || xx >= W) continue;
        size_t i = base + (size_t)yy * W + xx;
        if (pixel_masked(img, var, mask, i)) continue;
        double w = 1.0 / (double)var[i];
        double p = (double)P[(uy + r) * k + (ux + r)];
        s_psi += w * (double)img[i] * p;
        s_phi += w * p * p;
      }
    }
    psi[s] = s_psi;
    phi[s] = s_phi;
  }
}

/* ---------------------------------------------------------------------------------------- */
/* One trajectory: gather, clip, clipped sums (Section 3 nu = Psi/sqrt(Phi); Section 3.1 clip  */
/* and recomputed sum LH'; Section 3.2 clip before selection)                               */
/* ---------------------------------------------------------------------------------------- */

typedef struct {
  double lh, flux;
  int nvalid, nkept;
  uint32_t mask[KBO_MAX_T / 32];
  int ok; /* 1 if the trajectory is eligible for selection (before the L' threshold) */
} traj_result;

static void eval_traj(const double* psi, const double* phi, int T, int H, int W, int x0, int y0,
                      const int32_t* ox, const int32_t* oy, int min_obs, int clip, double q_lo,
                      double q_mid, double q_hi, double n_sigma, int clip_on, traj_result* res,
                      double* buf_psi, double* buf_phi, double* buf_a, int* buf_t,
                      uint8_t* buf_keep) {
  size_t hw = (size_t)H * W;
  int n = 0;
  for (int t = 0; t < T; ++t) {
    int x = x0 + ox[t], y = y0 + oy[t];
    if (x < 0 || x >= W || y < 0 || y >= H) continue;
    size_t i = (size_t)t * hw + (size_t)y * W + x;
    double p = psi[i], f = phi[i];
    if (!(f > 0.0) || !isfinite(p) || !isfinite(f)) continue;
    buf_psi[n] = p;
    buf_phi[n] = f;
    buf_a[n] = clip_on ? p / sqrt(f) : p / f;
    buf_t[n] = t;
    ++n;
  }
  memset(res, 0, sizeof(*res));
  res->nvalid = n;
  if (n < min_obs || n == 0) return;
  if (clip) {
    kbo_sigma_g_clip(buf_a, n, q_lo, q_mid, q_hi, n_sigma, buf_keep, NULL, NULL);
  } else {
    for (int i = 0; i < n; ++i) buf_keep[i] = 1;
  }
  double s_psi = 0.0, s_phi = 0.0;
  int nk = 0;
  for (int i = 0; i < n; ++i) {
    if (!buf_keep[i]) continue;
    s_psi += buf_psi[i];
    s_phi += buf_phi[i];
    res->mask[buf_t[i] >> 5] |= 1u << (buf_t[i] & 31);
    ++nk;
  }
  res->nkept = nk;
  if (nk == 0 || !(s_phi > 0.0)) return;
  res->lh = s_psi / sqrt(s_phi);
  res->flux = s_psi / s_phi;
  res->ok = 1;
}

/* Evaluate one integer-pixel trajectory (the single-trajectory variant of Section 4.1). */
int kbo_eval_one(const double* psi, const double* phi, const double* times, int T, int H, int W,
                 int x0, int y0, float vx, float vy, int min_obs, int clip, double q_lo,
                 double q_mid, double q_hi, double n_sigma, int clip_on, double* lh,
                 double* flux, int32_t* nvalid, int32_t* nkept, uint32_t* mask) {
  if (T <= 0 || T > KBO_MAX_T) return -1;
  int32_t ox[KBO_MAX_T], oy[KBO_MAX_T];
  kbo_track_offsets(times, T, &vx, &vy, 1, ox, oy);
  double bp[KBO_MAX_T], bf[KBO_MAX_T], ba[KBO_MAX_T];
  int bt[KBO_MAX_T];
  uint8_t bk[KBO_MAX_T];
  traj_result r;
  eval_traj(psi, phi, T, H, W, x0, y0, ox, oy, min_obs, clip, q_lo, q_mid, q_hi, n_sigma,
            clip_on, &r, bp, bf, ba, bt, bk);
  *lh = r.ok ? r.lh : NAN;
  *flux = r.ok ? r.flux : NAN;
  *nvalid = r.nvalid;
  *nkept = r.nkept;
  int mw = (T + 31) / 32;
  for (int w = 0; w < mw; ++w) mask[w] = r.mask[w];
  return r.ok;
}

/* How close one integer-pixel trajectory's clipped lightcurve comes to a clip bound (reading
 * R6): the smallest |a_t - (median -+ n sigma_G)| over its valid epochs, in units of
 * max(sigma_G, |median|, 1e-30).  Float32 and FP64 evaluations can take different keep
 * decisions only for an epoch within rounding of a bound; R6 accepts either decision where this
 * margin is at most 1e-5.  Returns +inf when the clip is off or the trajectory has fewer than
 * max(min_obs, 1) valid epochs (no clip decision is taken). */
double kbo_clip_margin(const double* psi, const double* phi, const double* times, int T, int H,
                       int W, int x0, int y0, float vx, float vy, int min_obs, int clip,
                       double q_lo, double q_mid, double q_hi, double n_sigma, int clip_on) {
  if (T <= 0 || T > KBO_MAX_T || !clip) return INFINITY;
  int32_t ox[KBO_MAX_T], oy[KBO_MAX_T];
  kbo_track_offsets(times, T, &vx, &vy, 1, ox, oy);
  double a[KBO_MAX_T];
  uint8_t keep[KBO_MAX_T];
  size_t hw = (size_t)H * W;
  int n = 0;
  for (int t = 0; t < T; ++t) {
    const int px = x0 + ox[t], py = y0 + oy[t];
    if (px < 0 || py < 0 || px >= W || py >= H) continue;   /* off the image: not valid */
    const double pv = psi[(size_t)t * hw + (size_t)py * W + px];
    const double fv = phi[(size_t)t * hw + (size_t)py * W + px];
    if (!(fv > 0.0 && isfinite(fv) && isfinite(pv))) continue;   /* R9 validity */
    a[n++] = clip_on ? pv / sqrt(fv) : pv / fv;
  }
  if (n == 0 || n < min_obs) return INFINITY;
  double med = 0.0, sg = 0.0;
  kbo_sigma_g_clip(a, n, q_lo, q_mid, q_hi, n_sigma, keep, &med, &sg);
  double lower = med - n_sigma * sg, upper = med + n_sigma * sg;
  double scale = fmax(fmax(sg, fabs(med)), 1e-30);
  double m = INFINITY;
  for (int i = 0; i < n; ++i) {
    double d = fmin(fabs(a[i] - lower), fabs(a[i] - upper));
    if (d < m) m = d;
  }
  return m / scale;
}

/* Candidate counts per stage over every (start pixel, trajectory) pair of a window (the stages
 * Fig. 3 counts): out[0] pairs with at least max(min_obs, 1) valid epochs; out[1] pairs whose
 * clipped L' is defined and reaches lh_min; out[2], out[3] the sums of n_kept and n_valid over
 * the out[1] pairs.  Each pair is evaluated in full as in kbo_search. */
int kbo_stage_counts(const double* psi, const double* phi, const double* times, int T, int H,
                     int W, const float* vx, const float* vy, int n_traj, double lh_min,
                     int min_obs, int clip, double q_lo, double q_mid, double q_hi,
                     double n_sigma, int clip_on, int x_lo, int x_hi, int y_lo, int y_hi,
                     unsigned long long* out) {
  if (T <= 0 || T > KBO_MAX_T || n_traj < 0) return -1;
  if (x_lo < 0 || x_hi > W || y_lo < 0 || y_hi > H || x_lo > x_hi || y_lo > y_hi) return -1;
  int32_t* ox = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_traj * T + 4);
  int32_t* oy = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_traj * T + 4);
  kbo_track_offsets(times, T, vx, vy, n_traj, ox, oy);
  int ww = x_hi - x_lo;
  int npix = ww * (y_hi - y_lo);
  unsigned long long c_valid = 0, c_pass = 0, c_kept = 0, c_nvalid = 0;
#pragma omp parallel reduction(+ : c_valid, c_pass, c_kept, c_nvalid)
  {
    double* bp = (double*)malloc(sizeof(double) * T);
    double* bf = (double*)malloc(sizeof(double) * T);
    double* ba = (double*)malloc(sizeof(double) * T);
    int* bt = (int*)malloc(sizeof(int) * T);
    uint8_t* bk = (uint8_t*)malloc((size_t)T);
#pragma omp for schedule(dynamic, 1)
    for (int p = 0; p < npix; ++p) {
      const int sx = x_lo + p % ww, sy = y_lo + p / ww;   /* start pixel */
      for (int j = 0; j < n_traj; ++j) {
        traj_result r;
        eval_traj(psi, phi, T, H, W, sx, sy, ox + (size_t)j * T, oy + (size_t)j * T, min_obs,
                  clip, q_lo, q_mid, q_hi, n_sigma, clip_on, &r, bp, bf, ba, bt, bk);
        if (r.nvalid > 0 && r.nvalid >= min_obs) ++c_valid;
        if (r.ok && r.lh >= lh_min) {
          ++c_pass;
          c_kept += (unsigned long long)r.nkept;
          c_nvalid += (unsigned long long)r.nvalid;
        }
      }
    }
    free(bp);
    free(bf);
    free(ba);
    free(bt);
    free(bk);
  }
  free(ox);
  free(oy);
  out[0] = c_valid;
  out[1] = c_pass;
  out[2] = c_kept;
  out[3] = c_nvalid;
  return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Exhaustive search + threshold + per-pixel top-K (Section 3, 3.1, 3.2; R5, R8)             */
/* ---------------------------------------------------------------------------------------- */

/* Outputs are [npix][K] for the start-pixel window [x_lo,x_hi) x [y_lo,y_hi), row-major,
 * with masks [npix][K][ceil(T/32)].  Empty slots: idx -1, lh -inf, flux 0, counts 0, mask 0. */
int kbo_search(const double* psi, const double* phi, const double* times, int T, int H, int W,
               const float* vx, const float* vy, int n_traj, int K, double lh_min, int min_obs,
               int clip, double q_lo, double q_mid, double q_hi, double n_sigma, int clip_on,
               int x_lo, int x_hi, int y_lo, int y_hi, double* out_lh, double* out_flux,
               int32_t* out_idx, int32_t* out_nvalid, int32_t* out_nkept, uint32_t* out_mask) {
  if (T <= 0 || T > KBO_MAX_T || K <= 0 || n_traj < 0) return -1;
  if (x_lo < 0 || x_hi > W || y_lo < 0 || y_hi > H || x_lo > x_hi || y_lo > y_hi) return -1;
  int mw = (T + 31) / 32;
  int32_t* ox = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_traj * T + 4);
  int32_t* oy = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_traj * T + 4);
  kbo_track_offsets(times, T, vx, vy, n_traj, ox, oy);
  int ww = x_hi - x_lo;
  int npix = ww * (y_hi - y_lo);
  for (size_t i = 0; i < (size_t)npix * K; ++i) {
    out_lh[i] = -INFINITY;
    out_flux[i] = 0.0;
    out_idx[i] = -1;
    out_nvalid[i] = 0;
    out_nkept[i] = 0;
  }
  memset(out_mask, 0, sizeof(uint32_t) * (size_t)npix * K * mw);

#pragma omp parallel
  {
    double* bp = (double*)malloc(sizeof(double) * T);
    double* bf = (double*)malloc(sizeof(double) * T);
    double* ba = (double*)malloc(sizeof(double) * T);
    int* bt = (int*)malloc(sizeof(int) * T);
    uint8_t* bk = (uint8_t*)malloc((size_t)T);
#pragma omp for schedule(dynamic, 1)
    for (int p = 0; p < npix; ++p) {
      int x0 = x_lo + p % ww, y0 = y_lo + p / ww;
      double* lh = out_lh + (size_t)p * K;
      double* fl = out_flux + (size_t)p * K;
      int32_t* ix = out_idx + (size_t)p * K;
      int32_t* nv = out_nvalid + (size_t)p * K;
      int32_t* nk = out_nkept + (size_t)p * K;
      uint32_t* mk = out_mask + (size_t)p * K * mw;
      for (int j = 0; j < n_traj; ++j) {
        traj_result r;
        eval_traj(psi, phi, T, H, W, x0, y0, ox + (size_t)j * T, oy + (size_t)j * T, min_obs,
                  clip, q_lo, q_mid, q_hi, n_sigma, clip_on, &r, bp, bf, ba, bt, bk);
        if (!r.ok || !(r.lh >= lh_min)) continue;
        /* insertion into the ordered list: position of the first slot ranked below (lh, j) */
        int s = 0;
        while (s < K && ix[s] >= 0 && (lh[s] > r.lh || (lh[s] == r.lh && ix[s] < j))) ++s;
        if (s >= K) continue;
        for (int m = K - 1; m > s; --m) {
          lh[m] = lh[m - 1];
          fl[m] = fl[m - 1];
          ix[m] = ix[m - 1];
          nv[m] = nv[m - 1];
          nk[m] = nk[m - 1];
          memcpy(mk + (size_t)m * mw, mk + (size_t)(m - 1) * mw, sizeof(uint32_t) * mw);
        }
        lh[s] = r.lh;
        fl[s] = r.flux;
        ix[s] = j;
        nv[s] = r.nvalid;
        nk[s] = r.nkept;
        memcpy(mk + (size_t)s * mw, r.mask, sizeof(uint32_t) * mw);
      }
    }
    free(bp);
    free(bf);
    free(ba);
    free(bt);
    free(bk);
  }
  free(ox);
  free(oy);
  return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Coadded postage stamps (Section 3.3: per-pixel median along the trajectory; also the mean) */
/* ---------------------------------------------------------------------------------------- */

int kbo_stamps(const float* img, const float* var, const uint8_t* mask, const double* times,
               int T, int H, int W, const int32_t* x0, const int32_t* y0, const float* vx,
               const float* vy, const uint32_t* keep_mask, int n, int radius, double* out_mean,
               double* out_median) {
  if (T <= 0 || T > KBO_MAX_T || radius < 0) return -1;
  int side = 2 * radius + 1;
  int mw = (T + 31) / 32;
  size_t hw = (size_t)H * W;
#pragma omp parallel
  {
    double* vals = (double*)malloc(sizeof(double) * T);
    int32_t ox[KBO_MAX_T], oy[KBO_MAX_T];
#pragma omp for schedule(dynamic, 1)
    for (int c = 0; c < n; ++c) {
      kbo_track_offsets(times, T, vx + c, vy + c, 1, ox, oy);
      for (int sy = -radius; sy <= radius; ++sy)
        for (int sx = -radius; sx <= radius; ++sx) {
          int m = 0;
          for (int t = 0; t < T; ++t) {
            if (keep_mask && !((keep_mask[(size_t)c * mw + (t >> 5)] >> (t & 31)) & 1u)) continue;
            int x = x0[c] + ox[t] + sx, y = y0[c] + oy[t] + sy;
            if (x < 0 || x >= W || y < 0 || y >= H) continue;
            size_t i = (size_t)t * hw + (size_t)y * W + x;
            if (pixel_masked(img, var, mask, i)) continue;
            vals[m++] = (double)img[i];
          }
          size_t o = (size_t)c * side * side + (size_t)(sy + radius) * side + (sx + radius);
          if (m == 0) { out_mean[o] = NAN; out_median[o] = NAN; continue; }
          double s = 0.0;
          for (int i = 0; i < m; ++i) s += vals[i];
          out_mean[o] = s / m;
          qsort(vals, (size_t)m, sizeof(double), cmp_double);
          out_median[o] = (m & 1) ? vals[m / 2] : 0.5 * (vals[m / 2 - 1] + vals[m / 2]);
        }
    }
    free(vals);
  }
  return 0;
}

/* ---------------------------------------------------------------------------------------- */
/* Sub-pixel trajectory likelihood and its gradient (refinement off the velocity grid)       */
/* ---------------------------------------------------------------------------------------- */

/* Bilinear sample of image plane t at real position (x, y) with pixel centres at integers
 * (R13: the cell is floor(x), floor(y)).  Outside taps contribute zero.  Also returns
 * d/dx and d/dy of the sample (piecewise-linear derivative). */
static double bilinear(const double* plane, int H, int W, double x, double y, double* dx,
                       double* dy) {
  double fx = floor(x), fy = floor(y);
  int ix = (int)fx, iy = (int)fy;
  double ax = x - fx, ay = y - fy;
  double v00 = 0, v01 = 0, v10 = 0, v11 = 0;
  if (iy >= 0 && iy < H && ix >= 0 && ix < W) v00 = plane[(size_t)iy * W + ix];
  if (iy >= 0 && iy < H && ix + 1 >= 0 && ix + 1 < W) v01 = plane[(size_t)iy * W + ix + 1];
  if (iy + 1 >= 0 && iy + 1 < H && ix >= 0 && ix < W) v10 = plane[(size_t)(iy + 1) * W + ix];
  if (iy + 1 >= 0 && iy + 1 < H && ix + 1 >= 0 && ix + 1 < W)
    v11 = plane[(size_t)(iy + 1) * W + ix + 1];
  double top = v00 + ax * (v01 - v00), bot = v10 + ax * (v11 - v10);
  if (dx) *dx = (1.0 - ay) * (v01 - v00) + ay * (v11 - v10);
  if (dy) *dy = bot - top;
  return top + ay * (bot - top);
}

/* L = Psi/sqrt(Phi) and alpha = Psi/Phi over the epochs set in keep (fixed mask), with
 * Psi = sum_t psi_t(x0 + vx dt_t, y0 + vy dt_t) and Phi likewise, dt_t = t_t - t_0 in FP64.
 * grad (nullable) receives dL/d(x0, y0, vx, vy).  Returns 0, or -1 if Phi <= 0. */
int kbo_traj_eval_subpixel(const double* psi, const double* phi, const double* times, int T,
                           int H, int W, const uint32_t* keep, double x0, double y0, double vx,
                           double vy, double* lh, double* flux, double* grad) {
  size_t hw = (size_t)H * W;
  double Ps = 0, Ph = 0;
  double dPs[4] = {0, 0, 0, 0}, dPh[4] = {0, 0, 0, 0};
  for (int t = 0; t < T; ++t) {
    if (!((keep[t >> 5] >> (t & 31)) & 1u)) continue;
    double dt = times[t] - times[0];
    double x = x0 + vx * dt, y = y0 + vy * dt;
    double gpx, gpy, gfx, gfy;
    double p = bilinear(psi + (size_t)t * hw, H, W, x, y, &gpx, &gpy);
    double f = bilinear(phi + (size_t)t * hw, H, W, x, y, &gfx, &gfy);
    Ps += p;
    Ph += f;
    dPs[0] += gpx; dPs[1] += gpy; dPs[2] += gpx * dt; dPs[3] += gpy * dt;
    dPh[0] += gfx; dPh[1] += gfy; dPh[2] += gfx * dt; dPh[3] += gfy * dt;
  }
  if (!(Ph > 0.0)) { *lh = NAN; *flux = NAN; return -1; }
  *lh = Ps / sqrt(Ph);
  *flux = Ps / Ph;
  if (grad) {
    double dL_dPs = 1.0 / sqrt(Ph);
    double dL_dPh = -0.5 * Ps / (Ph * sqrt(Ph));
    for (int i = 0; i < 4; ++i) grad[i] = dL_dPs * dPs[i] + dL_dPh * dPh[i];
  }
  return 0;
}

/* Vector-Jacobian product of the sub-pixel evaluation: given upstream weights gL on L and gA on
 * alpha = Psi/Phi, adds to grad_params[4] (nullable) the values gL dL/dp + gA dalpha/dp for
 * p = (x0, y0, vx, vy), and to the dense [T][H][W] arrays grad_psi, grad_phi (nullable) the
 * weights of every pixel: L and alpha depend on a pixel only through Psi or Phi, each a sum of
 * bilinear taps (R13), so a tap of weight w on kept epoch t receives cPsi w (psi) or cPhi w (phi)
 * with cPsi = gL/sqrt(Phi) + gA/Phi and cPhi = -gL Psi/(2 Phi^{3/2}) - gA Psi/Phi^2.
 * Taps outside the image get nothing.  Returns -1 (nothing added) if Phi <= 0. */
int kbo_traj_vjp(const double* psi, const double* phi, const double* times, int T, int H, int W,
                 const uint32_t* keep, double x0, double y0, double vx, double vy, double gL,
                 double gA, double* grad_params, double* grad_psi, double* grad_phi) {
  size_t hw = (size_t)H * W;
  double Ps = 0, Ph = 0;
  double dPs[4] = {0, 0, 0, 0}, dPh[4] = {0, 0, 0, 0};
  for (int t = 0; t < T; ++t) {
    if (!((keep[t >> 5] >> (t & 31)) & 1u)) continue;
    double dt = times[t] - times[0];
    double x = x0 + vx * dt, y = y0 + vy * dt;
    double gpx, gpy, gfx, gfy;
    Ps += bilinear(psi + (size_t)t * hw, H, W, x, y, &gpx, &gpy);
    Ph += bilinear(phi + (size_t)t * hw, H, W, x, y, &gfx, &gfy);
    dPs[0] += gpx; dPs[1] += gpy; dPs[2] += gpx * dt; dPs[3] += gpy * dt;
    dPh[0] += gfx; dPh[1] += gfy; dPh[2] += gfx * dt; dPh[3] += gfy * dt;
  }
  if (!(Ph > 0.0)) return -1;
  double cPs = gL / sqrt(Ph) + gA / Ph;
  double cPh = -0.5 * gL * Ps / (Ph * sqrt(Ph)) - gA * Ps / (Ph * Ph);
  if (grad_params)
    for (int i = 0; i < 4; ++i) grad_params[i] += cPs * dPs[i] + cPh * dPh[i];
  if (!grad_psi && !grad_phi) return 0;
  for (int t = 0; t < T; ++t) {
    if (!((keep[t >> 5] >> (t & 31)) & 1u)) continue;
    double dt = times[t] - times[0];
    double x = x0 + vx * dt, y = y0 + vy * dt;
    double fx = floor(x), fy = floor(y);
    int ix = (int)fx, iy = (int)fy;
    double ax = x - fx, ay = y - fy;
    for (int k = 0; k < 4; ++k) {
      int xx = ix + (k & 1), yy = iy + (k >> 1);
      if (xx < 0 || xx >= W || yy < 0 || yy >= H) continue;
      double w = ((k & 1) ? ax : 1.0 - ax) * ((k >> 1) ? ay : 1.0 - ay);
      size_t i = (size_t)t * hw + (size_t)yy * W + xx;
      if (grad_psi) grad_psi[i] += cPs * w;
      if (grad_phi) grad_phi[i] += cPh * w;
    }
  }
  return 0;
}

/* Gradient ascent on the sub-pixel likelihood L(x0, y0, vx, vy) with Adam (Kingma & Ba 2015:
 * m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2, step lr * mhat / (sqrt(vhat) + eps) with
 * mhat = m/(1-b1^k), vhat = v/(1-b2^k)), learning rate lr_pos for (x0, y0) and lr_vel for
 * (vx, vy); the kept mask stays fixed.  params [4] are updated in place.  Each of the n_steps
 * steps evaluates L and its gradient at the current params and moves them; the final L and alpha
 * are those at the returned params.  If Phi <= 0 at some evaluation the ascent stops there,
 * params keep their values, lh and flux are NaN and -1 is returned. */
int kbo_refine_adam(const double* psi, const double* phi, const double* times, int T, int H,
                    int W, const uint32_t* keep, double* params, int n_steps, double lr_pos,
                    double lr_vel, double b1, double b2, double eps, double* lh, double* flux) {
  double m[4] = {0, 0, 0, 0}, v[4] = {0, 0, 0, 0};
  double b1k = 1.0, b2k = 1.0;
  for (int k = 1; k <= n_steps; ++k) {
    double L, fl, g[4];
    if (kbo_traj_eval_subpixel(psi, phi, times, T, H, W, keep, params[0], params[1], params[2],
                               params[3], &L, &fl, g)) {
      *lh = NAN; *flux = NAN;
      return -1;
    }
    b1k *= b1;
    b2k *= b2;
    for (int i = 0; i < 4; ++i) {
      m[i] = b1 * m[i] + (1.0 - b1) * g[i];
      v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
      double mh = m[i] / (1.0 - b1k), vh = v[i] / (1.0 - b2k);
      double lr = i < 2 ? lr_pos : lr_vel;
      params[i] += lr * mh / (sqrt(vh) + eps);  /* ascent */
    }
  }
  return kbo_traj_eval_subpixel(psi, phi, times, T, H, W, keep, params[0], params[1], params[2],
                                params[3], lh, flux, NULL);
}

/* ---------------------------------------------------------------------------------------- */
/* Central moments of a coadded stamp (Section 3.3)                                          */
/* ---------------------------------------------------------------------------------------- */

/* Moments of stamp S (side = 2r+1, row-major) about its centre, the trajectory's position
 * (R17): with dy = row - r, dx = col - r, NaN pixels (no contributing epoch) left out, and the
 * weights w = S - min S (the smallest non-NaN pixel, so every weight is >= 0):
 *   out[0] = sum w,  out[1] = x = sum dx w / sum w,  out[2] = y = sum dy w / sum w,
 *   out[3] = xy = sum dx dy w / sum w,  out[4] = xx = sum dx^2 w / sum w,
 *   out[5] = yy = sum dy^2 w / sum w.
 * Returns 1 if the stamp passes the filter: sum w > 0 and |x| < lim[0], |y| < lim[1],
 * |xy| < lim[2], xx < lim[3], yy < lim[4] (strict), else 0. */
int kbo_stamp_moments(const double* S, int r, const double* lim, double* out) {
  int side = 2 * r + 1;
  double lo = INFINITY;
  for (int i = 0; i < side * side; ++i)
    if (!isnan(S[i]) && S[i] < lo) lo = S[i];
  double m0 = 0, mx = 0, my = 0, mxy = 0, mxx = 0, myy = 0;
  for (int row = 0; row < side; ++row) {
    for (int col = 0; col < side; ++col) {
      double v = S[row * side + col];
      if (isnan(v)) continue;
      double w = v - lo;
      double dx = col - r, dy = row - r;
      m0 += w;
      mx += dx * w;
      my += dy * w;
      mxy += dx * dy * w;
      mxx += dx * dx * w;
      myy += dy * dy * w;
    }
  }
  out[0] = m0;
  out[1] = mx / m0;
  out[2] = my / m0;
  out[3] = mxy / m0;
  out[4] = mxx / m0;
  out[5] = myy / m0;
  if (!(m0 > 0.0)) return 0;
  return fabs(out[1]) < lim[0] && fabs(out[2]) < lim[1] && fabs(out[3]) < lim[2] &&
         out[4] < lim[3] && out[5] < lim[4];
}

/* ---------------------------------------------------------------------------------------- */
/* Clustering of candidates (Fig. 3 caption names it; reading R19)                          */
/* ---------------------------------------------------------------------------------------- */

/* Greedy de-duplication in priority order (index 0 first): candidate i (start (x0, y0), velocity
 * (vx, vy)) is a duplicate of j when their positions agree within r at the first epoch and at
 * t0 + dt (the last epoch): |p_i - p_j| <= r at both, with p(dt) = (x0 + vx dt, y0 + vy dt).
 * Walking the candidates in order, i is kept unless it duplicates an already kept j; rep[i] is i
 * when kept, else the first (lowest-index) kept j it duplicates.  valid (nullable): candidates
 * with valid[i] == 0 take no part (keep 0, rep -1), nor do candidates whose start pixel lies
 * outside 0 .. 2^20 - 1 on either axis (the placeholders of empty survivor slots). */
static int kbo_dup(const int32_t* x0, const int32_t* y0, const float* vx, const float* vy,
                   int i, int j, double dt, double r2) {
  double dx0 = (double)x0[i] - (double)x0[j], dy0 = (double)y0[i] - (double)y0[j];
  if (dx0 * dx0 + dy0 * dy0 > r2) return 0;
  double xi = (double)x0[i] + (double)vx[i] * dt, yi = (double)y0[i] + (double)vy[i] * dt;
  double xj = (double)x0[j] + (double)vx[j] * dt, yj = (double)y0[j] + (double)vy[j] * dt;
  double dx1 = xi - xj, dy1 = yi - yj;
  return dx1 * dx1 + dy1 * dy1 <= r2;
}

void kbo_cluster(const int32_t* x0, const int32_t* y0, const float* vx, const float* vy,
                 const uint8_t* valid, int n, double dt, double r, uint8_t* keep, int32_t* rep) {
  double r2 = r * r;
  for (int i = 0; i < n; ++i) {
    keep[i] = 0;
    rep[i] = -1;
    if (valid && !valid[i]) continue;
    if (x0[i] < 0 || x0[i] >= (1 << 20) || y0[i] < 0 || y0[i] >= (1 << 20)) continue;
    int found = -1;
    for (int j = 0; j < i && found < 0; ++j)
      if (keep[j] && kbo_dup(x0, y0, vx, vy, i, j, dt, r2)) found = j;
    if (found < 0) {
      keep[i] = 1;
      rep[i] = i;
    } else {
      rep[i] = found;
    }
  }
}

/* Thread count of the OpenMP loops (timing of the CPU baseline). */
void kbo_set_threads(int n) { omp_set_num_threads(n > 0 ? n : 1); }
int kbo_get_threads(void) { return omp_get_max_threads(); }
