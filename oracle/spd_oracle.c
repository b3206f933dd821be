/*
 * spd_oracle.c -- CPU FP64 oracle for single-pulse detection by boxcar filters
 * (Adamek & Armour, "Single Pulse Detection Algorithms for Real-time Fast Radio
 * Burst Searches using GPUs", arXiv:1910.08324).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or call
 * this file; only the test-suite, the smoke check and the bench's CPU-baseline
 * leg use it.  It shares no code, header, table or constant generator with the
 * CUDA library: every grid, sum and bound below is re-derived from the paper.
 *
 * Everything is plain, slow and in double precision.  Each function names the
 * passage of the paper it follows.
 *
 * Contents
 *   grids      spdo_grid_exhaustive / spdo_grid_boxdit(_iters) / spdo_grid_igrid
 *              (Sec. 2.2.1 parameters B and L_s; Alg. 1 and the BoxDIT width
 *              formula of Sec. 3.1, with one L^i_max per iteration or the
 *              same for all; Sec. 3.2 layers, Eq. boxcarsize, Table 1)
 *   O1         spdo_search: the definition, Eq. boxcar + Eq. SNRlong (+ Eq.
 *              whitenoise), Y = max over the grid (Eq. MSD03), for every start
 *   O2         spdo_boxdit_steps(_iters): Alg. 1 run literally (boxcars on the
 *              decimated series x^i extended from X^{i-1}, shifted decimation)
 *              spdo_igrid_steps: Sec. 3.2 run literally (binary tree of shifted
 *              decimated layers, depth extensions from ancestor layers)
 *   bounds     spdo_rsnr_bounds: Appendix A, Eq. RSNRmax and Eq. RSNRmin
 *   pulse      spdo_pulse_rsnr: Appendix A, Eq. RSNR (coverage d_s) for one
 *              rectangular pulse, maximised over every eligible boxcar
 *   peaks      spdo_candidates: threshold + local-maximum rule (the paper's
 *              peak-finding step of Sec. 4.5 is not defined in the paper; the
 *              rule used here is the one stated in the function's comment)
 *   noise      spdo_msd_levels / spdo_msd_table: mean and standard deviation
 *              with iterated outlier rejection at power-of-two decimations,
 *              interpolated to every width (Sec. 4.5, "Calculation of mean and
 *              standard deviation"; the interpolation rule is a reading)
 *
 * Conventions shared with the test-suite (readings of the paper):
 *   - A boxcar is indexed by its first sample (Eq. boxcar is forward looking).
 *   - Width L is evaluated at start s iff s mod L_s(L) == 0 and s + L <= nt
 *     (the paper does not define series ends; nothing is padded).
 *   - Y[s] is the maximum SNR over eligible widths; W[s] is the index, in the
 *     ascending width table, of the smallest width reaching it (strict '>'
 *     while widths are visited in increasing order).
 *   - Iterations stop at the first width >= S_end ("nearest longer", Sec. 3).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define SPDO_EXPORT __attribute__((visibility("default")))

/* ------------------------------------------------------------------------ */
/* Grids                                                                     */
/* ------------------------------------------------------------------------ */

/* Ideal SPD (Sec. 3.1, first paragraph): every width 1..lmax at every sample. */
SPDO_EXPORT int32_t spdo_grid_exhaustive(int32_t lmax, int32_t *L, int32_t *Ls,
                                         int32_t cap) {
  if (lmax < 1) return -1;
  if (lmax > cap) return -2;
  for (int32_t w = 1; w <= lmax; ++w) {
    L[w - 1] = w;
    Ls[w - 1] = 1;
  }
  return lmax;
}

/*
 * BoxDIT grid (Alg. 1 and the width formula of Sec. 3.1), decimation D = 2.
 * Iteration i computes, on x^i, the widths
 *     L = L^{i-1}_MAX + D^i * m,   m = 1 .. L^i_max,
 * at every point of x^i, i.e. at every D^i-th sample of x^0 (L_s = D^i), and
 *     L^i_MAX = L^{i-1}_MAX + D^i * L^i_max,   L^{-1}_MAX = 0.
 * L^i_max may differ from iteration to iteration (Sec. 3.1, discussion of
 * BoxDIT's single implementation): iteration i uses k[i], and iterations past
 * the list repeat its last entry.  Each L^i_max must be even (divisible by D).
 * Iterations continue until a width >= s_end has been produced, which is the
 * last width kept.  If n_iter > 0 exactly n_iter full iterations are produced
 * instead (the paper's BD-8 footnote counts iterations this way).
 */
SPDO_EXPORT int32_t spdo_grid_boxdit_iters(const int32_t *k, int32_t nk, int32_t s_end,
                                           int32_t n_iter, int32_t *L, int32_t *Ls,
                                           int32_t cap) {
  if (nk < 1 || s_end < 1) return -1;
  for (int32_t i = 0; i < nk; ++i)
    if (k[i] < 2 || (k[i] % 2) != 0) return -1;
  int32_t n = 0;
  int64_t lmax_cum = 0; /* L^{i-1}_MAX */
  int64_t Di = 1;       /* D^i */
  for (int32_t i = 0;; ++i) {
    if (n_iter > 0 && i >= n_iter) return n;
    const int32_t ki = k[i < nk ? i : nk - 1];
    for (int32_t m = 1; m <= ki; ++m) {
      int64_t w = lmax_cum + Di * m;
      if (w > 2147483647LL) return -3;
      if (n >= cap) return -2;
      L[n] = (int32_t)w;
      Ls[n] = (int32_t)Di;
      ++n;
      if (n_iter <= 0 && w >= s_end) return n;
    }
    lmax_cum += Di * ki;
    Di *= 2;
    if (Di > (1LL << 30)) return -3;
  }
}

/* The same with one L^i_max = k for every iteration (BD-k of Sec. 4). */
SPDO_EXPORT int32_t spdo_grid_boxdit(int32_t k, int32_t s_end, int32_t n_iter,
                                     int32_t *L, int32_t *Ls, int32_t cap) {
  return spdo_grid_boxdit_iters(&k, 1, s_end, n_iter, L, Ls, cap);
}

/*
 * IGRID grid (Sec. 3.2).  With P layers per step the boxcar separation at step
 * i is L_s = 2^i / P (never below one sample).  The widths of step i are those
 * of Eq. boxcarsize read through Table 1: starting from 2^i, depth d adds the
 * widths 2^i + m * 2^(i-d), m = 0 .. 2^d - 1 (all of them lie in [2^i, 2^(i+1))
 * as the text states); at steps i < d the increment cannot go below one
 * sample, so every width of [2^i, 2^(i+1)) is produced.  d = 0, P = 1 is the
 * plain DIT of Alg. 3 (widths 2^i at separation 2^i).
 */
SPDO_EXPORT int32_t spdo_grid_igrid(int32_t d, int32_t P, int32_t s_end, int32_t *L,
                                    int32_t *Ls, int32_t cap) {
  if (d < 0 || P < 1 || (P & (P - 1)) != 0 || s_end < 1) return -1;
  if (P < (1 << d)) return -1; /* separation must divide the width increment */
  int32_t n = 0;
  for (int32_t i = 0; i < 31; ++i) {
    int64_t base = 1LL << i;
    int64_t sep = base / P;
    if (sep < 1) sep = 1;
    int64_t inc = (i >= d) ? (base >> d) : 1;
    int64_t count = (i >= d) ? (1LL << d) : base; /* number of widths at this step */
    for (int64_t m = 0; m < count; ++m) {
      int64_t w = base + m * inc;
      if (n >= cap) return -2;
      L[n] = (int32_t)w;
      Ls[n] = (int32_t)sep;
      ++n;
      if (w >= s_end) return n;
    }
  }
  return -3;
}

/* ------------------------------------------------------------------------ */
/* O1: the definition                                                        */
/* ------------------------------------------------------------------------ */

/*
 * For each DM row r and each start s:
 *   X_L[s] = sum_{j<L} x[s+j]                        (Eq. boxcar)
 *   SNR_L[s] = (X_L[s] - mu_L) / sigma_L             (Eq. SNRlong)
 *   white noise: mu_L = L mu_r, sigma_L = sqrt(L) sigma_r   (Eq. whitenoise)
 *   table noise: mu_L, sigma_L given per row and width index
 *   Y[s] = max over eligible grid widths (Eq. MSD03, all iterations combined)
 * The grid (L[], Ls[]) must be sorted by increasing L.  Y2[s] receives the
 * largest SNR among the other eligible widths (-HUGE_VAL if there is none), so
 * that callers can tell when the best width is decided by a near-tie.
 * literal != 0 sums every boxcar sample by sample; otherwise X_L[s] is taken as
 * the difference of two running totals of x (the same sum, in FP64).
 * Outputs are dense [ndm][nt].
 */
SPDO_EXPORT int32_t spdo_search(const double *x, int64_t ndm, int64_t nt, int64_t ld,
                                const int32_t *L, const int32_t *Ls, int32_t n,
                                int32_t noise_mode, const double *mu,
                                const double *sigma, int32_t literal,
                                int32_t nthreads, double *Y, int32_t *W, double *Y2) {
  if (ndm < 0 || nt < 1 || ld < nt || n < 1) return -1;
  for (int32_t g = 1; g < n; ++g)
    if (L[g] <= L[g - 1]) return -1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#else
  (void)nthreads;
#endif
  int32_t err = 0;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < ndm; ++r) {
    const double *xr = x + r * ld;
    double *run = NULL;
    if (!literal) {
      run = (double *)malloc((size_t)(nt + 1) * sizeof(double));
      if (!run) {
#pragma omp atomic write
        err = -4;
        continue;
      }
      run[0] = 0.0;
      for (int64_t t = 0; t < nt; ++t) run[t + 1] = run[t] + xr[t];
    }
    for (int64_t s = 0; s < nt; ++s) {
      double best = -HUGE_VAL, second = -HUGE_VAL;
      int32_t widx = -1;
      for (int32_t g = 0; g < n; ++g) {
        int64_t w = L[g];
        if (s % Ls[g] != 0 || s + w > nt) continue;
        double X;
        if (literal) {
          X = 0.0;
          for (int64_t j = 0; j < w; ++j) X += xr[s + j];
        } else {
          X = run[s + w] - run[s];
        }
        double muL, sigL;
        if (noise_mode == 0) {
          muL = (double)w * mu[r];
          sigL = sqrt((double)w) * sigma[r];
        } else {
          muL = mu[r * n + g];
          sigL = sigma[r * n + g];
        }
        double snr = (X - muL) / sigL;
        if (snr > best) {
          second = best;
          best = snr;
          widx = g;
        } else if (snr > second) {
          second = snr;
        }
      }
      Y[r * nt + s] = best;
      W[r * nt + s] = widx;
      if (Y2) Y2[r * nt + s] = second;
    }
    free(run);
  }
  return err;
}

/* ------------------------------------------------------------------------ */
/* O2: the paper's BoxDIT, step by step                                      */
/* ------------------------------------------------------------------------ */

/*
 * Alg. 1 for one row, D = 2, L^i_max = k = kl[i] (the last entry of kl
 * repeats for later iterations):
 *   - iteration i holds x^i (length len_i) and X^{i-1} at every D^i-th sample
 *     (X^{-1} = 0, L^{-1}_MAX = 0);
 *   - Boxcars(): for every point n of x^i and m = 1..k,
 *         X_L[s] = X^{i-1}[s] + sum_{j<m} x^i[n+j],  s = n D^i,
 *         L = L^{i-1}_MAX + D^i m               (the two formulas of Sec. 3.1)
 *     and X^i[s] is the sum for m = k;
 *   - Decimate(): x^{i+1}[n - k/D] = sum_{j<D} x^i[D n + j] for n - k/D >= 0
 *     (the shifted decimation of Sec. 3.1);
 *   - L^i_MAX = L^{i-1}_MAX + D^i k.
 * A sum exists only if every x^i sample it needs exists; that is exactly
 * s + L <= nt.  Stops after the first width >= s_end, or after n_iter full
 * iterations if n_iter > 0.  Y/Wlen are combined over iterations per start
 * (max SNR, smallest width on ties); Wlen holds the width itself.
 * White noise per row (mu[r], sigma[r]).
 */
static void boxdit_row(const double *x0, int64_t nt, const int32_t *kl, int32_t nk,
                       int32_t s_end, int32_t n_iter, double mu, double sigma, double *Y,
                       int32_t *Wlen) {
  for (int64_t s = 0; s < nt; ++s) {
    Y[s] = -HUGE_VAL;
    Wlen[s] = 0;
  }
  int64_t len = nt;
  double *xi = (double *)malloc((size_t)nt * sizeof(double));
  double *Xprev = (double *)calloc((size_t)nt, sizeof(double)); /* X^{i-1}[n D^i] at index n */
  double *Xcur = (double *)calloc((size_t)nt, sizeof(double));
  memcpy(xi, x0, (size_t)nt * sizeof(double));
  int64_t lmax_cum = 0, Di = 1;
  int done = 0;
  for (int32_t i = 0; !done; ++i) {
    if (n_iter > 0 && i >= n_iter) break;
    const int32_t k = kl[i < nk ? i : nk - 1]; /* L^i_max */
    /* Boxcars() */
    for (int64_t nn = 0; nn < len; ++nn) {
      int64_t s = nn * Di;
      double acc = Xprev[nn];
      for (int32_t m = 1; m <= k; ++m) {
        int64_t w = lmax_cum + Di * m;
        if (nn + m - 1 >= len) break; /* x^i[n+m-1] does not exist */
        acc += xi[nn + m - 1];
        double snr = (acc - (double)w * mu) / (sqrt((double)w) * sigma);
        if (snr > Y[s]) {
          Y[s] = snr;
          Wlen[s] = (int32_t)w;
        }
        if (n_iter <= 0 && w >= s_end) break;
      }
      if (nn + k - 1 < len) Xcur[nn] = acc; /* X^i at this point (only needed if complete) */
    }
    /* did this iteration reach s_end? */
    if (n_iter <= 0) {
      for (int32_t m = 1; m <= k; ++m)
        if (lmax_cum + Di * m >= s_end) done = 1;
    }
    if (done) break;
    /* Decimate(): x^{i+1}[n - k/2] = x^i[2n] + x^i[2n+1] */
    int64_t half = k / 2;
    int64_t newlen = 0;
    for (int64_t nn = half;; ++nn) {
      if (2 * nn + 1 >= len) break;
      xi[nn - half] = xi[2 * nn] + xi[2 * nn + 1];
      newlen = nn - half + 1;
    }
    /* X^i is needed at every 2nd point of x^i for the next iteration */
    for (int64_t nn = 0; 2 * nn < len; ++nn) Xprev[nn] = Xcur[2 * nn];
    len = newlen;
    lmax_cum += Di * k;
    Di *= 2;
    if (len <= 0) break;
  }
  free(xi);
  free(Xprev);
  free(Xcur);
}

SPDO_EXPORT int32_t spdo_boxdit_steps_iters(const double *x, int64_t ndm, int64_t nt,
                                            int64_t ld, const int32_t *k, int32_t nk,
                                            int32_t s_end, int32_t n_iter, const double *mu,
                                            const double *sigma, double *Y, int32_t *Wlen) {
  if (nk < 1 || nt < 1 || ld < nt) return -1;
  for (int32_t i = 0; i < nk; ++i)
    if (k[i] < 2 || (k[i] % 2) != 0) return -1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < ndm; ++r)
    boxdit_row(x + r * ld, nt, k, nk, s_end, n_iter, mu[r], sigma[r], Y + r * nt,
               Wlen + r * nt);
  return 0;
}

SPDO_EXPORT int32_t spdo_boxdit_steps(const double *x, int64_t ndm, int64_t nt,
                                      int64_t ld, int32_t k, int32_t s_end,
                                      int32_t n_iter, const double *mu,
                                      const double *sigma, double *Y, int32_t *Wlen) {
  return spdo_boxdit_steps_iters(x, ndm, nt, ld, &k, 1, s_end, n_iter, mu, sigma, Y, Wlen);
}

/* ------------------------------------------------------------------------ */
/* O2: the paper's IGRID, step by step                                       */
/* ------------------------------------------------------------------------ */

/*
 * Sec. 3.2 for one row.  A layer x^i_h is the series decimated i times with
 * shift h: x^i_h[n] = sum of the 2^i samples of x^0 starting at h + n 2^i.
 * Step 0 is x^0_0 = x.  A parent x^i_h gives two children
 *     x^{i+1}_h[n]       = x^i_h[2n]   + x^i_h[2n+1]
 *     x^{i+1}_{h+2^i}[n] = x^i_h[2n+1] + x^i_h[2n+2]
 * and step i keeps the layers whose shifts are multiples of L_s = 2^i/P (at
 * least 1), i.e. P layers once 2^i >= P.  At step i every sample of every kept
 * layer is a boxcar of width 2^i starting at h + n 2^i; depth d extends it by
 * pieces 2^(i-1), 2^(i-2), ... 2^(i-d) taken from the ancestor layers
 * x^{i-1}, ..., x^{i-d} that start right where the sum so far ends (Eq.
 * boxcarsize with a_k in {0,1}, Table 1).  Every width 2^i + sum a_k 2^(i-k)
 * is evaluated; at steps i < d only pieces of at least one sample exist.
 * The step producing the first width >= s_end is the last one, and within it
 * no width above that one is used.  White noise per row.
 */
typedef struct {
  int64_t shift;
  int64_t len;
  double *v;
} layer_t;

static const layer_t *find_layer(const layer_t *ls, int nl, int64_t shift) {
  for (int a = 0; a < nl; ++a)
    if (ls[a].shift == shift) return &ls[a];
  return NULL;
}

static void igrid_row(const double *x0, int64_t nt, int32_t d, int32_t P,
                      int32_t s_end, double mu, double sigma, double *Y,
                      int32_t *Wlen) {
  for (int64_t s = 0; s < nt; ++s) {
    Y[s] = -HUGE_VAL;
    Wlen[s] = 0;
  }
  enum { MAXSTEP = 32 };
  layer_t *steps[MAXSTEP];
  int nls[MAXSTEP];
  memset(steps, 0, sizeof(steps));
  memset(nls, 0, sizeof(nls));
  /* step 0 */
  steps[0] = (layer_t *)malloc(sizeof(layer_t));
  steps[0][0].shift = 0;
  steps[0][0].len = nt;
  steps[0][0].v = (double *)malloc((size_t)nt * sizeof(double));
  memcpy(steps[0][0].v, x0, (size_t)nt * sizeof(double));
  nls[0] = 1;
  int last = 0;
  for (int32_t i = 0; i < MAXSTEP; ++i) {
    int64_t b = 1LL << i;
    /* evaluate the boxcars of step i */
    int dd = (i < d) ? i : d;
    int64_t nvar = 1LL << dd;
    int stop_here = 0;
    for (int a = 0; a < nls[i]; ++a) {
      const layer_t *ly = &steps[i][a];
      for (int64_t n = 0; n < ly->len; ++n) {
        int64_t s = ly->shift + n * b;
        for (int64_t v = 0; v < nvar; ++v) {
          /* bits of v (most significant first) are a_1 .. a_dd */
          int64_t w = b;
          double acc = ly->v[n];
          int ok = 1;
          for (int kk = 1; kk <= dd && ok; ++kk) {
            int abit = (int)((v >> (dd - kk)) & 1);
            if (!abit) continue;
            int64_t piece = b >> kk;
            int64_t pstart = s + w;
            const layer_t *anc = find_layer(steps[i - kk], nls[i - kk], pstart % piece);
            if (!anc) {
              ok = 0;
              break;
            }
            int64_t pi = (pstart - anc->shift) / piece;
            if (pi >= anc->len) {
              ok = 0;
              break;
            }
            acc += anc->v[pi];
            w += piece;
          }
          if (!ok) continue;
          if (w > b && (w - (b >> dd)) >= s_end) continue; /* beyond the nearest longer width */
          double snr = (acc - (double)w * mu) / (sqrt((double)w) * sigma);
          if (snr > Y[s] || (snr == Y[s] && w < Wlen[s])) {
            Y[s] = snr;
            Wlen[s] = (int32_t)w;
          }
        }
      }
    }
    /* does this step produce a width >= s_end? (its widths are b + m b/2^dd) */
    for (int64_t v = 0; v < nvar; ++v)
      if (b + v * (b >> dd) >= s_end) stop_here = 1;
    last = i;
    if (stop_here || i + 1 >= MAXSTEP) break;
    /* children for step i+1 */
    int64_t sep_next = (2 * b) / P;
    if (sep_next < 1) sep_next = 1;
    steps[i + 1] = (layer_t *)calloc((size_t)(2 * nls[i]), sizeof(layer_t));
    int nc = 0;
    for (int a = 0; a < nls[i]; ++a) {
      const layer_t *par = &steps[i][a];
      for (int child = 0; child < 2; ++child) {
        int64_t sh = par->shift + child * b;
        if (sh % sep_next != 0) continue;
        int64_t clen = 0;
        double *cv = (double *)malloc((size_t)(par->len / 2 + 1) * sizeof(double));
        for (int64_t n = 0;; ++n) {
          int64_t i0 = 2 * n + child;
          if (i0 + 1 >= par->len) break;
          cv[n] = par->v[i0] + par->v[i0 + 1];
          clen = n + 1;
        }
        steps[i + 1][nc].shift = sh;
        steps[i + 1][nc].len = clen;
        steps[i + 1][nc].v = cv;
        ++nc;
      }
    }
    nls[i + 1] = nc;
    if (nc == 0) break;
  }
  for (int i = 0; i <= last + 1 && i < MAXSTEP; ++i) {
    if (!steps[i]) continue;
    for (int a = 0; a < nls[i]; ++a) free(steps[i][a].v);
    free(steps[i]);
  }
}

SPDO_EXPORT int32_t spdo_igrid_steps(const double *x, int64_t ndm, int64_t nt, int64_t ld,
                                     int32_t d, int32_t P, int32_t s_end,
                                     const double *mu, const double *sigma, double *Y,
                                     int32_t *Wlen) {
  if (d < 0 || P < 1 || (P & (P - 1)) != 0 || P < (1 << d) || nt < 1 || ld < nt)
    return -1;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t r = 0; r < ndm; ++r)
    igrid_row(x + r * ld, nt, d, P, s_end, mu[r], sigma[r], Y + r * nt, Wlen + r * nt);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Appendix A: signal-loss bounds                                            */
/* ------------------------------------------------------------------------ */

/*
 * Best case (Appendix A, "Best detection case"):
 *   RSNRbar_max(S;L) = sqrt(S/L) C if S < L, sqrt(L/S) C if S >= L
 *   RSNR_max(S) = max over the width set               (Eq. RSNRmax)
 * Worst case (Appendix A, "Worst detection case"), per width L with its L_s:
 *   S <= L - L_s           : sqrt(S/L) C
 *   L - L_s < S < L        : d< C / sqrt(L S),  d< = S - floor((S - L + L_s)/2)  (Eq. ds_wc1)
 *   L <= S < L + L_s       : d> C / sqrt(L S),  d> = L - floor((L + L_s - S)/2)  (Eq. ds_wc2)
 *   S >= L + L_s           : sqrt(L/S) C
 *   RSNR_min(S) = max over the width set               (Eq. RSNRmin)
 */
SPDO_EXPORT void spdo_rsnr_bounds(const int32_t *L, const int32_t *Ls, int32_t n,
                                  int32_t S, double C, double *rmax, double *rmin) {
  double bmax = 0.0, bmin = 0.0;
  for (int32_t g = 0; g < n; ++g) {
    double l = (double)L[g], ls = (double)Ls[g], s = (double)S;
    double vmax = (S < L[g]) ? sqrt(s / l) * C : sqrt(l / s) * C;
    double vmin;
    if (S <= L[g] - Ls[g]) {
      vmin = sqrt(s / l) * C;
    } else if (S < L[g]) {
      double ds = s - floor((s - l + ls) / 2.0);
      vmin = ds * C / sqrt(l * s);
    } else if (S < L[g] + Ls[g]) {
      double ds = l - floor((l + ls - s) / 2.0);
      vmin = ds * C / sqrt(l * s);
    } else {
      vmin = sqrt(l / s) * C;
    }
    if (vmax > bmax) bmax = vmax;
    if (vmin > bmin) bmin = vmin;
  }
  *rmax = bmax;
  *rmin = bmin;
}

/*
 * Recovered SNR of one noise-free rectangular pulse of width S and amplitude
 * C/sqrt(S) (Eq. amplitudenormalization) starting at sample t, with white-noise
 * normalisation mu = 0, sigma = 1 (Sec. 2.1).  A boxcar [s, s+L) covers
 * d_s = |[s,s+L) intersect [t,t+S)| samples and gives d_s C / sqrt(L S)
 * (Eq. RSNR).  Every eligible start s (s mod L_s == 0, 0 <= s, s + L <= nt) of
 * every width is tried; the best value is returned and *bestL receives the
 * smallest width reaching it (0 if none).  The eligible starts whose boxcar
 * can touch the pulse are enumerated one by one.
 */
SPDO_EXPORT double spdo_pulse_rsnr(const int32_t *L, const int32_t *Ls, int32_t n,
                                   int64_t nt, int32_t S, int64_t t, double C,
                                   int32_t *bestL) {
  double best = -HUGE_VAL;
  int32_t bl = 0;
  for (int32_t g = 0; g < n; ++g) {
    int64_t l = L[g], ls = Ls[g];
    int64_t lo = t - l + 1;
    if (lo < 0) lo = 0;
    lo = ((lo + ls - 1) / ls) * ls;
    double bw = 0.0;
    for (int64_t s = lo; s < t + S; s += ls) {
      if (s + l > nt) break;
      int64_t a = s > t ? s : t;
      int64_t b = (s + l) < (t + S) ? (s + l) : (t + S);
      int64_t cov = b - a;
      if (cov < 0) cov = 0;
      double v = (double)cov * C / sqrt((double)l * (double)S);
      if (v > bw) bw = v;
    }
    if (bw > best) {
      best = bw;
      bl = (int32_t)l;
    }
  }
  if (bestL) *bestL = bl;
  return best;
}

/*
 * The measurement of Sec. 4.1: one series per pulse shift, the highest RSNR of
 * each series, then the maximum and minimum over the shifts (RSNR_max/min as
 * measured) and their mean.  The pulse starts at t0 + shift, shift = 0 ..
 * n_shift-1, where t0 is a multiple of every separation in the grid and at least
 * the largest width, and the series is long enough for every boxcar that can
 * touch the pulse.
 */
SPDO_EXPORT void spdo_sliding(const int32_t *L, const int32_t *Ls, int32_t n, int32_t S,
                              int64_t n_shift, double C, double *rmax, double *rmin,
                              double *rmean) {
  int64_t maxL = 1, maxLs = 1;
  for (int32_t g = 0; g < n; ++g) {
    if (L[g] > maxL) maxL = L[g];
    if (Ls[g] > maxLs) maxLs = Ls[g];
  }
  int64_t t0 = ((maxL + maxLs - 1) / maxLs) * maxLs;
  int64_t nt = t0 + n_shift + S + maxL + 1;
  /*
   * No boxcar of width L can give more than min(S, L) C / sqrt(L S) (its
   * coverage is at most min(S, L)).  Widths are visited from the largest such
   * bound down and a width is skipped once its bound cannot beat the best value
   * found so far; this changes the running time only, never the result.
   */
  int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  double *ub = (double *)malloc((size_t)n * sizeof(double));
  for (int32_t g = 0; g < n; ++g) {
    double l = (double)L[g], sv = (double)S;
    ub[g] = (l < sv ? l : sv) * C / sqrt(l * sv);
    order[g] = g;
  }
  for (int32_t a = 1; a < n; ++a) { /* insertion sort, descending bound */
    int32_t v = order[a];
    int32_t b = a - 1;
    while (b >= 0 && ub[order[b]] < ub[v]) {
      order[b + 1] = order[b];
      --b;
    }
    order[b + 1] = v;
  }
  double hi = -HUGE_VAL, lo = HUGE_VAL, sum = 0.0;
  for (int64_t sh = 0; sh < n_shift; ++sh) {
    int64_t t = t0 + sh;
    double best = -HUGE_VAL;
    for (int32_t a = 0; a < n; ++a) {
      int32_t g = order[a];
      if (ub[g] <= best) break;
      double v = spdo_pulse_rsnr(L + g, Ls + g, 1, nt, S, t, C, NULL);
      if (v > best) best = v;
    }
    if (best > hi) hi = best;
    if (best < lo) lo = best;
    sum += best;
  }
  free(order);
  free(ub);
  *rmax = hi;
  *rmin = lo;
  *rmean = sum / (double)n_shift;
}

/* ------------------------------------------------------------------------ */
/* Candidate selection                                                       */
/* ------------------------------------------------------------------------ */

/*
 * The paper selects candidates "using a peak-finding algorithm" (Sec. 4.5)
 * without defining it.  Rule used here: start s of row r is a candidate iff
 *   Y[s] >= thr, Y[s] > Y[s'] for every s - R <= s' < s, and
 *   Y[s] >= Y[s'] for every s < s' <= s + R   (s' inside the row),
 * so the leftmost sample of a plateau wins; R = 0 is a plain threshold.
 * Records come out ordered by (row, start); at most cap are written and the
 * total number is returned.  Y, W are dense [ndm][nt].
 */
SPDO_EXPORT int64_t spdo_candidates(const double *Y, const int32_t *W, int64_t ndm,
                                    int64_t nt, double thr, int32_t R, int64_t *out_row,
                                    int64_t *out_start, int32_t *out_w,
                                    double *out_snr, int64_t cap) {
  int64_t cnt = 0;
  for (int64_t r = 0; r < ndm; ++r) {
    const double *yr = Y + r * nt;
    for (int64_t s = 0; s < nt; ++s) {
      double v = yr[s];
      if (!(v >= thr)) continue;
      int ok = 1;
      for (int64_t q = s - R; q < s && ok; ++q)
        if (q >= 0 && !(v > yr[q])) ok = 0;
      for (int64_t q = s + 1; q <= s + R && ok; ++q)
        if (q < nt && !(v >= yr[q])) ok = 0;
      if (!ok) continue;
      if (cnt < cap) {
        out_row[cnt] = r;
        out_start[cnt] = s;
        out_w[cnt] = W ? W[r * nt + s] : -1;
        out_snr[cnt] = v;
      }
      ++cnt;
    }
  }
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* Noise statistics (Sec. 4.5, calculation of mean and standard deviation)   */
/* ------------------------------------------------------------------------ */

/*
 * Mean and standard deviation of the base-level noise of every row, at the
 * decimations 2^k, k = 0..nlev-1 (Sec. 4.5: the deviation is computed only for
 * boxcars whose width is a power of two, i.e. for the series decimated in time).
 *
 * Level k of a row is the series of sums of its complete, non-overlapping
 * blocks of 2^k samples.  For each level separately (the paper's point-wise
 * outlier rejection, repeated until convergence):
 *   included = every value of the level
 *   for pass = 0 .. max_passes-1:
 *     n, mean, sd = count, mean and standard deviation of the included values
 *                   (population form, sum of squared deviations over n)
 *     stop if thr <= 0 (no rejection) or pass == max_passes-1
 *     next = values with |v - mean| <= thr * sd
 *     stop if |next| == n (the next pass would keep as many values)
 *     included = next
 * mu, sigma, cnt: [ndm][nlev] outputs; a level without values gets n = 0 and
 * mean = sd = 0.  Plain two-pass sums in FP64 (the paper's streaming Chan et al.
 * update is a faster way to the same two numbers).
 */
SPDO_EXPORT int spdo_msd_levels(const double *x, int64_t ndm, int64_t nt, int64_t ld,
                                int32_t nlev, double thr, int32_t max_passes, double *mu,
                                double *sigma, int64_t *cnt) {
  if (ndm < 0 || nt < 0 || ld < nt || nlev < 1 || nlev > 40 || max_passes < 1) return -1;
  int rc = 0;
#pragma omp parallel for schedule(dynamic)
  for (int64_t r = 0; r < ndm; ++r) {
    const double *xr = x + r * ld;
    for (int32_t k = 0; k < nlev; ++k) {
      const int64_t B = (int64_t)1 << k;
      const int64_t nv = nt / B;
      double m = 0.0, sd = 0.0;
      int64_t n = 0;
      double *v = nv > 0 ? (double *)malloc(sizeof(double) * (size_t)nv) : NULL;
      char *inc = nv > 0 ? (char *)malloc((size_t)nv) : NULL;
      if (nv > 0 && (!v || !inc)) {
        rc = -2;
        free(v);
        free(inc);
        continue;
      }
      for (int64_t i = 0; i < nv; ++i) {
        double a = 0.0;
        for (int64_t j = 0; j < B; ++j) a += xr[i * B + j];
        v[i] = a;
        inc[i] = 1;
      }
      for (int32_t pass = 0; pass < max_passes && nv > 0; ++pass) {
        double s1 = 0.0;
        n = 0;
        for (int64_t i = 0; i < nv; ++i)
          if (inc[i]) {
            s1 += v[i];
            ++n;
          }
        m = n > 0 ? s1 / (double)n : 0.0;
        double s2 = 0.0;
        for (int64_t i = 0; i < nv; ++i)
          if (inc[i]) s2 += (v[i] - m) * (v[i] - m);
        sd = n > 0 ? sqrt(s2 / (double)n) : 0.0;
        if (!(thr > 0.0) || pass == max_passes - 1) break;
        int64_t nn = 0;
        for (int64_t i = 0; i < nv; ++i) nn += fabs(v[i] - m) <= thr * sd ? 1 : 0;
        if (nn == n) break;
        for (int64_t i = 0; i < nv; ++i) inc[i] = fabs(v[i] - m) <= thr * sd ? 1 : 0;
      }
      mu[r * nlev + k] = m;
      sigma[r * nlev + k] = sd;
      cnt[r * nlev + k] = n;
      free(v);
      free(inc);
    }
  }
  return rc;
}

/*
 * Mean and deviation of every width of a grid from the level statistics of
 * spdo_msd_levels (Sec. 4.5: values for widths between powers of two are
 * interpolated; the paper does not say how).  Reading used here: the per-sample
 * mean m_k = mu_k / 2^k and the white-normalised deviation rho_k =
 * sigma_k / sqrt(2^k) are interpolated linearly in log2(L) between the levels
 * a = floor(log2 L) and a + 1, then mu_L = L m, sigma_L = sqrt(L) rho.  White
 * noise (rho constant) therefore follows Eq. whitenoise exactly, and a width
 * that is a power of two gets its level's values.  A level is usable when it
 * has at least 2 values; widths beyond the last usable level h keep m_h and
 * rho_h (white extrapolation).  tmu, tsig: [ndm][nw].
 */
SPDO_EXPORT int spdo_msd_table(const double *mu, const double *sigma, const int64_t *cnt,
                               int64_t ndm, int32_t nlev, const int32_t *L, int32_t nw,
                               double *tmu, double *tsig) {
  if (ndm < 0 || nlev < 1 || nw < 0) return -1;
  for (int64_t r = 0; r < ndm; ++r) {
    const double *m = mu + r * nlev, *s = sigma + r * nlev;
    const int64_t *c = cnt + r * nlev;
    int h = -1;
    while (h + 1 < nlev && c[h + 1] >= 2) ++h;
    for (int32_t w = 0; w < nw; ++w) {
      const double Lw = (double)L[w];
      double mm, rr;
      if (h < 0) {
        mm = 0.0;
        rr = 0.0;
      } else {
        const double lg = log2(Lw);
        int a = (int)floor(lg);
        if (a >= h) {
          mm = m[h] / ldexp(1.0, h);
          rr = s[h] / sqrt(ldexp(1.0, h));
        } else {
          const double f = lg - (double)a;
          const double ma = m[a] / ldexp(1.0, a), mb = m[a + 1] / ldexp(1.0, a + 1);
          const double ra = s[a] / sqrt(ldexp(1.0, a)), rb = s[a + 1] / sqrt(ldexp(1.0, a + 1));
          mm = ma + f * (mb - ma);
          rr = ra + f * (rb - ra);
        }
      }
      tmu[r * nw + w] = Lw * mm;
      tsig[r * nw + w] = sqrt(Lw) * rr;
    }
  }
  return 0;
}
