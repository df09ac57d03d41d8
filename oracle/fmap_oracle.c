/*
 * Plain FP64 CPU oracle of the transient F-statistic map.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library; the product path never
 * does.  It shares no code, header or table with the CUDA library.
 *
 * What it computes (Keitel & Ashton, arXiv:1805.05652):
 *   - windows, Sec. 2 Eq. (winrect) and Eq. (winexp);
 *   - windowed sums of the atoms, Sec. 2 (the text after Eq. F_xMx and after
 *     Eq. Fmn: A, B, C, Fa, Fb are partial sums of the atoms), with the
 *     antenna-matrix sums weighted by the square of the window and the
 *     projections Fa, Fb weighted by the window itself, because the signal
 *     model of Sec. 2 is h = w(t) h_CW;
 *   - D = A B - C^2 and F from Eq. (F_FaFb); the map stores 2F;
 *   - the F-map grid t0_m = t0_min + m dt0, tau_n = tau_min + n dtau, Eq. (Fmn);
 *   - windows that run past the data end are truncated, not dropped (App. A,
 *     the "non-embedded" convention);
 *   - the max-2F detection statistic (Sec. 4.3) and a log Bayes factor
 *     marginalised over (t0, tau) (Sec. 2 Eq. F_OSG: e^F is proportional to
 *     the odds; App. A names the marginalisation step).
 *
 * Readings where the paper is silent (each is tested and documented):
 *   - an atom is evaluated at its SFT start t; it is inside the window when
 *     t0 <= t and t + T_sft <= t0 + L (L = tau, or 3 tau for exp, Eq.
 *     winexp's cut; exp lengths floor(c tau / 8) for other cuts c given in
 *     eighths of tau).  The literal reading t in [t0, t0 + L] is available
 *     with inclusive = 1;
 *   - a cell with fewer than 2 atoms (Sec. 4.1) or D <= 0 is invalid: 2F = 0
 *     and it is left out of max, argmax and the Bayes factor;
 *   - logB = ln( (1/N_valid) sum_valid e^{F_mn} ) + log_prior_const;
 *   - argmax ties go to the lowest linear index m * N_tau + n.
 *
 * Grid array g (int64[12 + ...]): t0_min, dt0, n_t0, tau_min, dtau, n_tau,
 * t_sft, window (0 rect, 1 exp, 2 table), inclusive (0 / 1), exp / table cut
 * in eighths of tau (0: 24, i.e. 3 tau), explicit axes (0 / 1), number of
 * window-table samples (window 2).  With explicit axes the t0 values and then
 * the tau values follow (a non-uniform grid; t0_min, dt0, tau_min and dtau are
 * then unused); otherwise t0_m = t0_min + m dt0 and tau_n = tau_min + n dtau
 * (Eq. Fmn).  A table window's samples follow last, each the IEEE bit
 * pattern of a float32 value in an int64.
 * Atom layout: t[N] ascending (the direct mode accepts any order);
 * antenna [3][N] (a^2, b^2, ab) shared by all templates, or [T][3][N];
 * fafb [T][4][N] (Re Fa, Im Fa, Re Fb, Im Fb).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { G_T0MIN, G_DT0, G_NT0, G_TAUMIN, G_DTAU, G_NTAU, G_TSFT, G_WIN, G_INCL, G_CUT, G_AXES,
       G_NTAB, G_VALUES };

/* Grid values t0_m and tau_n (Eq. Fmn, or the explicit axes). */
static int64_t t0_at(const int64_t* g, int64_t m) {
  return g[G_AXES] ? g[G_VALUES + m] : g[G_T0MIN] + m * g[G_DT0];
}
static int64_t tau_at(const int64_t* g, int64_t n) {
  return g[G_AXES] ? g[G_VALUES + g[G_NT0] + n] : g[G_TAUMIN] + n * g[G_DTAU];
}

static void set_threads(int n_threads) {
#ifdef _OPENMP
  if (n_threads > 0) omp_set_num_threads(n_threads);
#else
  (void)n_threads;
#endif
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Window weight of Eq. (winrect) / (winexp); 0 outside the window. */
static int inside_window(const int64_t* g, int64_t t, int64_t t0, int64_t tau) {
  const int64_t cut8 = g[G_CUT] > 0 ? g[G_CUT] : 24;
  int64_t len = (g[G_WIN] == 0) ? tau : cut8 * tau / 8;
  if (t < t0) return 0;
  if (g[G_INCL]) return t <= t0 + len;
  return t + g[G_TSFT] <= t0 + len;
}

/* Sample k of a table window (float32 bits stored in the grid array). */
static double table_sample(const int64_t* g, int64_t k) {
  const int64_t* tab = g + G_VALUES + (g[G_AXES] ? g[G_NT0] + g[G_NTAU] : 0);
  uint32_t bits = (uint32_t)tab[k];
  float v;
  memcpy(&v, &bits, sizeof v);
  return (double)v;
}

/* Generic window: the samples w_k at x_k = k X / (n - 1), X = cut / 8, joined
 * linearly; 0 past X. */
static double table_weight(const int64_t* g, int64_t t, int64_t t0, int64_t tau) {
  const int64_t n = g[G_NTAB];
  const int64_t cut8 = g[G_CUT] > 0 ? g[G_CUT] : 24;
  const double u = (double)(t - t0) * ((double)(n - 1) * 8.0 / ((double)cut8 * (double)tau));
  const double k = floor(u);
  if (k >= (double)(n - 1)) return k > (double)(n - 1) ? 0.0 : table_sample(g, n - 1);
  const int64_t i = (int64_t)k;
  const double w0 = table_sample(g, i), w1 = table_sample(g, i + 1);
  return w0 + (u - k) * (w1 - w0);
}

static double window_weight(const int64_t* g, int64_t t, int64_t t0, int64_t tau) {
  if (!inside_window(g, t, t0, tau)) return 0.0;
  if (g[G_WIN] == 0) return 1.0;
  if (g[G_WIN] == 2) return table_weight(g, t, t0, tau);
  return exp(-(double)(t - t0) / (double)tau);
}

/* 2F from the windowed sums, Eq. (F_FaFb) times two. */
double oracle_twoF_from_sums(double A, double B, double C, double fa_re, double fa_im,
                             double fb_re, double fb_im, int32_t count, int32_t* valid) {
  double D = A * B - C * C;
  if (count < 2 || !(D > 0.0)) {
    *valid = 0;
    return 0.0;
  }
  double F = (B * (fa_re * fa_re + fa_im * fa_im) + A * (fb_re * fb_re + fb_im * fb_im) -
              2.0 * C * (fa_re * fb_re + fa_im * fb_im)) / D;
  *valid = 1;
  return 2.0 * F;
}

/* Direct definition of the sums of one cell: loop over every atom. */
static void cell_sums_direct(const int64_t* g, int n_sft, const int64_t* t, const double* ant,
                             const double* x, int64_t t0, int64_t tau, double s[7],
                             int32_t* count) {
  for (int k = 0; k < 7; ++k) s[k] = 0.0;
  int32_t c = 0;
  for (int a = 0; a < n_sft; ++a) {
    if (!inside_window(g, t[a], t0, tau)) continue;
    double w = window_weight(g, t[a], t0, tau);
    double w2 = w * w;
    s[0] += w2 * ant[a];
    s[1] += w2 * ant[n_sft + a];
    s[2] += w2 * ant[2 * n_sft + a];
    s[3] += w * x[a];
    s[4] += w * x[n_sft + a];
    s[5] += w * x[2 * n_sft + a];
    s[6] += w * x[3 * n_sft + a];
    ++c;
  }
  *count = c;
}

/* sums[T][n_t0][n_tau][7] = A, B, C, Re Fa, Im Fa, Re Fb, Im Fb; counts[n_t0][n_tau]. */
int oracle_sums(const int64_t* g, int n_sft, const int64_t* t, int n_templates,
                int shared_antenna, const double* antenna, const double* fafb, double* sums,
                int32_t* counts, int n_threads) {
  set_threads(n_threads);
  const int64_t n_t0 = g[G_NT0], n_tau = g[G_NTAU];
  const int64_t cells = n_t0 * n_tau;
#pragma omp parallel for collapse(2) schedule(dynamic, 4)
  for (int64_t j = 0; j < n_templates; ++j) {
    for (int64_t m = 0; m < n_t0; ++m) {
      const double* ant = shared_antenna ? antenna : antenna + j * 3 * (int64_t)n_sft;
      const double* x = fafb + j * 4 * (int64_t)n_sft;
      int64_t t0 = t0_at(g, m);
      for (int64_t n = 0; n < n_tau; ++n) {
        int64_t tau = tau_at(g, n);
        int32_t c;
        double* s = sums + ((j * cells) + m * n_tau + n) * 7;
        cell_sums_direct(g, n_sft, t, ant, x, t0, tau, s, &c);
        if (j == 0 && counts) counts[m * n_tau + n] = c;
      }
    }
  }
  return 0;
}

/* First atom index with t[a] >= t0 (t ascending). */
static int first_at_or_after(int n_sft, const int64_t* t, int64_t t0) {
  int lo = 0, hi = n_sft;
  while (lo < hi) {
    int mid = lo + (hi - lo) / 2;
    if (t[mid] < t0) lo = mid + 1; else hi = mid;
  }
  return lo;
}

/*
 * The F-map.  mode 0: direct definition per cell (every atom visited);
 * mode 1: the paper's per-row algorithms in FP64 -- rect: for each t0 row,
 * running sums extended atom by atom as tau grows (Sec. 3, rectangular case;
 * needs dtau > 0); exp: each cell sums its own window's atoms (Sec. 3,
 * exponential case).  map2F[T][n_t0][n_tau], valid[T][n_t0][n_tau],
 * counts[n_t0][n_tau] (nullable).
 */
int oracle_fmap(int mode, const int64_t* g, int n_sft, const int64_t* t, int n_templates,
                int shared_antenna, const double* antenna, const double* fafb, double* map2F,
                uint8_t* valid, int32_t* counts, int n_threads) {
  set_threads(n_threads);
  const int64_t n_t0 = g[G_NT0], n_tau = g[G_NTAU];
  const int64_t cells = n_t0 * n_tau;
  if (mode == 1 && g[G_WIN] == 0 && n_tau > 1 && tau_at(g, 1) <= tau_at(g, 0)) return -1;
  int err = 0;
#pragma omp parallel
  {
    double* acc = (double*)malloc(sizeof(double) * 4 * (size_t)(n_templates > 0 ? n_templates : 1));
    if (!acc) {
#pragma omp atomic write
      err = -2;
    }
#pragma omp for collapse(2) schedule(dynamic, 2)
    for (int64_t j = 0; j < (mode == 1 && g[G_WIN] == 1 ? 1 : n_templates); ++j) {
      for (int64_t m = 0; m < n_t0; ++m) {
        if (!acc) continue;
        int64_t t0 = t0_at(g, m);
        if (mode == 0) {
          const double* ant = shared_antenna ? antenna : antenna + j * 3 * (int64_t)n_sft;
          const double* x = fafb + j * 4 * (int64_t)n_sft;
          for (int64_t n = 0; n < n_tau; ++n) {
            int64_t tau = tau_at(g, n);
            double s[7];
            int32_t c, v;
            cell_sums_direct(g, n_sft, t, ant, x, t0, tau, s, &c);
            int64_t o = j * cells + m * n_tau + n;
            map2F[o] = oracle_twoF_from_sums(s[0], s[1], s[2], s[3], s[4], s[5], s[6], c, &v);
            valid[o] = (uint8_t)v;
            if (j == 0 && counts) counts[m * n_tau + n] = c;
          }
        } else if (g[G_WIN] == 0) {
          /* rectangular: running partial sums over tau for this t0 row */
          const double* ant = shared_antenna ? antenna : antenna + j * 3 * (int64_t)n_sft;
          const double* x = fafb + j * 4 * (int64_t)n_sft;
          int a = first_at_or_after(n_sft, t, t0);
          double s[7] = {0, 0, 0, 0, 0, 0, 0};
          int32_t c = 0;
          for (int64_t n = 0; n < n_tau; ++n) {
            int64_t tau = tau_at(g, n);
            while (a < n_sft && inside_window(g, t[a], t0, tau)) {
              s[0] += ant[a];
              s[1] += ant[n_sft + a];
              s[2] += ant[2 * n_sft + a];
              s[3] += x[a];
              s[4] += x[n_sft + a];
              s[5] += x[2 * n_sft + a];
              s[6] += x[3 * n_sft + a];
              ++c;
              ++a;
            }
            int32_t v;
            int64_t o = j * cells + m * n_tau + n;
            map2F[o] = oracle_twoF_from_sums(s[0], s[1], s[2], s[3], s[4], s[5], s[6], c, &v);
            valid[o] = (uint8_t)v;
            if (j == 0 && counts) counts[m * n_tau + n] = c;
          }
        } else {
          /* exponential or table window: each cell sums its own window; the weights of a
           * cell are shared by all templates */
          int a0 = first_at_or_after(n_sft, t, t0);
          for (int64_t n = 0; n < n_tau; ++n) {
            int64_t tau = tau_at(g, n);
            double sa[3] = {0, 0, 0};
            for (int k = 0; k < 4 * n_templates; ++k) acc[k] = 0.0;
            int32_t c = 0;
            for (int a = a0; a < n_sft && inside_window(g, t[a], t0, tau); ++a) {
              double w = window_weight(g, t[a], t0, tau);
              double w2 = w * w;
              if (shared_antenna) {
                sa[0] += w2 * antenna[a];
                sa[1] += w2 * antenna[n_sft + a];
                sa[2] += w2 * antenna[2 * n_sft + a];
              }
              for (int jj = 0; jj < n_templates; ++jj) {
                const double* x = fafb + (int64_t)jj * 4 * n_sft;
                acc[4 * jj + 0] += w * x[a];
                acc[4 * jj + 1] += w * x[n_sft + a];
                acc[4 * jj + 2] += w * x[2 * n_sft + a];
                acc[4 * jj + 3] += w * x[3 * n_sft + a];
              }
              ++c;
            }
            for (int jj = 0; jj < n_templates; ++jj) {
              double A = sa[0], B = sa[1], C = sa[2];
              if (!shared_antenna) {
                const double* ant = antenna + (int64_t)jj * 3 * n_sft;
                A = B = C = 0.0;
                for (int a = a0; a < n_sft && inside_window(g, t[a], t0, tau); ++a) {
                  double w = window_weight(g, t[a], t0, tau);
                  A += w * w * ant[a];
                  B += w * w * ant[n_sft + a];
                  C += w * w * ant[2 * n_sft + a];
                }
              }
              int32_t v;
              int64_t o = jj * cells + m * n_tau + n;
              map2F[o] = oracle_twoF_from_sums(A, B, C, acc[4 * jj], acc[4 * jj + 1],
                                               acc[4 * jj + 2], acc[4 * jj + 3], c, &v);
              valid[o] = (uint8_t)v;
            }
            if (counts) counts[m * n_tau + n] = c;
          }
        }
      }
    }
    free(acc);
  }
  return err;
}

/*
 * Selected cells by the direct definition: cell_idx[k] = (template, m, n).
 * out2F[k], valid[k], counts[k]; sums_out[k][7] when non-null.
 */
int oracle_cells(const int64_t* g, int n_sft, const int64_t* t, int n_templates,
                 int shared_antenna, const double* antenna, const double* fafb, int64_t n_cells,
                 const int64_t* cell_idx, double* out2F, uint8_t* valid, int32_t* counts,
                 double* sums_out, int n_threads) {
  set_threads(n_threads);
  int err = 0;
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t k = 0; k < n_cells; ++k) {
    int64_t j = cell_idx[3 * k], m = cell_idx[3 * k + 1], n = cell_idx[3 * k + 2];
    if (j < 0 || j >= n_templates || m < 0 || m >= g[G_NT0] || n < 0 || n >= g[G_NTAU]) {
#pragma omp atomic write
      err = -1;
      continue;
    }
    const double* ant = shared_antenna ? antenna : antenna + j * 3 * (int64_t)n_sft;
    const double* x = fafb + j * 4 * (int64_t)n_sft;
    int64_t t0 = t0_at(g, m);
    int64_t tau = tau_at(g, n);
    double s[7];
    int32_t c, v;
    cell_sums_direct(g, n_sft, t, ant, x, t0, tau, s, &c);
    out2F[k] = oracle_twoF_from_sums(s[0], s[1], s[2], s[3], s[4], s[5], s[6], c, &v);
    valid[k] = (uint8_t)v;
    if (counts) counts[k] = c;
    if (sums_out)
      for (int q = 0; q < 7; ++q) sums_out[7 * k + q] = s[q];
  }
  return err;
}

/*
 * Per-template reductions of a map: max 2F over valid cells, its argmax
 * (lowest linear index on ties), N_valid and
 * logB = ln( (1/N_valid) sum_valid e^{2F/2} ) + log_prior_const, evaluated as
 * F_max + ln sum e^{F - F_max} - ln N_valid.  N_valid = 0 gives max2F = 0,
 * m = n = -1 and logB = NaN.
 */
int oracle_summary(int n_templates, int64_t n_t0, int64_t n_tau, const double* map2F,
                   const uint8_t* valid, double log_prior_const, double* max2F, int32_t* am,
                   int32_t* an, double* logB, int64_t* n_valid) {
  const int64_t cells = n_t0 * n_tau;
  for (int j = 0; j < n_templates; ++j) {
    const double* f = map2F + (int64_t)j * cells;
    const uint8_t* v = valid + (int64_t)j * cells;
    double best = -INFINITY;
    int64_t arg = -1, nv = 0;
    for (int64_t c = 0; c < cells; ++c) {
      if (!v[c]) continue;
      ++nv;
      if (f[c] > best) {
        best = f[c];
        arg = c;
      }
    }
    n_valid[j] = nv;
    if (nv == 0) {
      max2F[j] = 0.0;
      am[j] = an[j] = -1;
      logB[j] = NAN;
      continue;
    }
    double Fmax = 0.5 * best, s = 0.0;
    for (int64_t c = 0; c < cells; ++c)
      if (v[c]) s += exp(0.5 * f[c] - Fmax);
    max2F[j] = best;
    am[j] = (int32_t)(arg / n_tau);
    an[j] = (int32_t)(arg % n_tau);
    logB[j] = Fmax + log(s) - log((double)nv) + log_prior_const;
  }
  return 0;
}
