/*
 * ch_oracle.c -- plain, slow, single-threaded FP64 reference of the Cahn-Hilliard
 * ensemble time-stepper.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this
 * file; only the test-suite, the smoke check and the CPU-baseline leg of the benchmark
 * do.  It shares no code, header, table or constant generator with the CUDA library.
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared (see oracle/build.py), so every
 * product below is rounded on its own (no fused multiply-add).
 *
 * What it computes (paper: O Naraigh & Gloster, "A large-scale statistical study of the
 * coarsening rate in models of Ostwald-Ripening"):
 *   - the Cahn-Hilliard equation with constant mobility, Sec. 1 Eq. (3):
 *         dC/dt = lap(C^3 - C - gamma lap C),  periodic square domain [0,L)^2;
 *   - the free energy and its time derivative, Sec. 1 Eq. (4), with the bulk term
 *     1/4 (C^2-1)^2 (the prefactor that makes Eq. (4)'s dF/dt the derivative of F for
 *     the flux of Eq. (3));
 *   - the coarsening rate beta = -(t/F) dF/dt, Sec. 1 Eq. (6), and its time average
 *     over a window [t1, T], Sec. 3.3 Eq. (42) (the paper's beta_0 estimate,
 *     applied to the CH ensembles in Sec. 4.2, Table 4);
 *   - statistics of beta across an ensemble: the moments of Sec. 3.3 Eqs. (41a,b) per
 *     sample time, histograms (the empirical p_beta(b, t) of Sec. 1 Eq. (7)), the window
 *     mean of mu_1 (Eq. (42)) and the slope k of the least-squares line mu_2 = k t;
 *   - the grid-refinement error E_n of Appendix A (2 x 2 restriction, L1 distance);
 *   - Model 1, the mean-field droplet population of Secs. 2-3 (Eqs. (13), (14), (31),
 *     (33), (36), (38), (39)), integrated by the Dormand-Prince 5(4) pair.
 * The discretisation (Sec. 4.1 names only a semi-implicit ADI finite-difference method
 * with periodic boundaries) is read as the delta-form approximate factorisation
 *     (I + s D_x^4)(I + s D_y^4)(C^{n+1} - C^n) = dt * lap_h( C^3 - C - gamma lap_h C )^n,
 *     s = gamma*dt,  D^4 = (D^2)^2,  lap_h the 5-point Laplacian,
 * i.e. the nonlinear and cross terms explicit and gamma*lap^2 implicit per direction.
 * Each implicit factor is a cyclic, constant, symmetric pentadiagonal system per grid
 * line; this file solves it by Gaussian elimination of the bordered band (no pivoting:
 * the matrix is symmetric positive definite).  Every step is written in the order the
 * scheme states it; no blocking, fusion or reordering.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_OK 0
#define OR_EINVAL (-1)
#define OR_ENOMEM (-2)

/* ------------------------------------------------------------------------------ */
/* SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable pseudorandom number     */
/* generators", OOPSLA 2014).  The generator keeps a 64-bit state, adds the odd       */
/* constant 0x9e3779b97f4a7c15 before each draw and returns a bijective mix of the   */
/* new state, so the k-th draw (k = 0, 1, ...) of a stream started from `seed` is    */
/* mix(seed + (k+1) * 0x9e3779b97f4a7c15): a counter-based generator.                 */
/* ------------------------------------------------------------------------------ */
static uint64_t or_sm64_mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

uint64_t or_splitmix64(uint64_t seed, uint64_t k) {
  uint64_t state = seed;
  state += (k + 1ULL) * 0x9e3779b97f4a7c15ULL;
  return or_sm64_mix(state);
}

/* Uniform u in [0,1): the top 53 bits of the draw times 2^-53 (exact in FP64). */
double or_uniform(uint64_t seed, uint64_t k) {
  return (double)(or_splitmix64(seed, k) >> 11) * (1.0 / 9007199254740992.0);
}

/*
 * Initial field: C = C0 + 0.1 * (2u - 1), u i.i.d. uniform, one draw per grid point,
 * draw index k = counter_base + j*nx + i (row-major, x fastest).  This is the
 * "mean + uniform noise" construction of Sec. 4.1 with the noise amplitude +-0.1 about
 * a chosen mean C0 (the paper's two mixtures are C0 = 0.45 and C0 = 0.5 read off its
 * formulas; here C0 is an input).
 */
void or_initial_field(int nx, int ny, double C0, uint64_t seed, uint64_t counter_base,
                      double* C) {
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      uint64_t k = counter_base + (uint64_t)j * (uint64_t)nx + (uint64_t)i;
      double u = or_uniform(seed, k);
      double noise = 0.1 * (2.0 * u - 1.0);
      C[(size_t)j * nx + i] = C0 + noise;
    }
}

/* ------------------------------------------------------------------------------ */
/* 5-point periodic Laplacian:                                                        */
/*   lap_h v = (v[i+1] + v[i-1] - 2 v[i]) / hx^2 + (v[j+1] + v[j-1] - 2 v[j]) / hy^2  */
/* ------------------------------------------------------------------------------ */
static double or_lap_at(const double* v, int nx, int ny, double hx, double hy, int i, int j) {
  int ip = (i + 1) % nx, im = (i + nx - 1) % nx;
  int jp = (j + 1) % ny, jm = (j + ny - 1) % ny;
  double c = v[(size_t)j * nx + i];
  double dxx = (v[(size_t)j * nx + ip] + v[(size_t)j * nx + im] - 2.0 * c) / (hx * hx);
  double dyy = (v[(size_t)jp * nx + i] + v[(size_t)jm * nx + i] - 2.0 * c) / (hy * hy);
  return dxx + dyy;
}

void or_laplacian(int nx, int ny, double hx, double hy, const double* v, double* out) {
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) out[(size_t)j * nx + i] = or_lap_at(v, nx, ny, hx, hy, i, j);
}

/*
 * Chemical potential and explicit right-hand side of the delta form:
 *   f  = C^3 - C                   (derivative of the bulk energy 1/4 (C^2-1)^2)
 *   mu = f - gamma lap_h C         (the bracket of Eq. (3))
 *   R  = dt lap_h mu               (explicit update; the implicit part is solved below)
 */
void or_rhs(int nx, int ny, double hx, double hy, double gamma, double dt, const double* C,
            double* mu, double* R) {
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      size_t p = (size_t)j * nx + i;
      double c = C[p];
      double f = c * c * c - c;
      mu[p] = f - gamma * or_lap_at(C, nx, ny, hx, hy, i, j);
    }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) R[(size_t)j * nx + i] = dt * or_lap_at(mu, nx, ny, hx, hy, i, j);
}

/* ------------------------------------------------------------------------------ */
/* Cyclic pentadiagonal solve  A x = r,  A = I + s (D^2)^2  on a periodic line of n   */
/* points (D^2 the unit-spacing second difference, s already divided by h^4):        */
/* A[i][i] = 1 + 6s, A[i][i+-1] = -4s, A[i][i+-2] = s, indices mod n.  Needs n >= 5 so */
/* the +-1 and +-2 offsets never alias.                                               */
/*                                                                                    */
/* Method: split the unknowns into the first m = n-2 ("band") and the last two        */
/* ("border").  In block form [[B, E], [F, G]] with B the non-cyclic pentadiagonal    */
/* band, E, F the corner couplings and G the 2x2 corner block.  Gaussian elimination  */
/* of B without pivoting is applied to [E | r_B]; the 2x2 Schur complement            */
/* G - F B^-1 E gives the border unknowns, back-substitution the rest.  This is plain */
/* Gaussian elimination of A in natural order with the fill confined to the last two */
/* rows and columns.                                                                  */
/* ------------------------------------------------------------------------------ */
static double or_penta_coef(int n, double s, int i, int j) {
  int d = ((j - i) % n + n) % n;
  if (d == 0) return 1.0 + 6.0 * s;
  if (d == 1 || d == n - 1) return -4.0 * s;
  if (d == 2 || d == n - 2) return s;
  return 0.0;
}

int or_cyclic_penta_solve(int n, double s, const double* r, double* x) {
  if (n < 5) return OR_EINVAL;
  int m = n - 2;
  /* band[i][2 + (j - i)] holds B[i][j] for |j - i| <= 2 */
  double* band = (double*)calloc((size_t)m * 5, sizeof(double));
  double* rhs = (double*)calloc((size_t)m * 3, sizeof(double)); /* columns: E0, E1, r_B */
  if (!band || !rhs) {
    free(band);
    free(rhs);
    return OR_ENOMEM;
  }
  for (int i = 0; i < m; ++i) {
    for (int d = -2; d <= 2; ++d) {
      int j = i + d;
      if (j >= 0 && j < m) band[(size_t)i * 5 + 2 + d] = or_penta_coef(n, s, i, j);
    }
    rhs[(size_t)i * 3 + 0] = or_penta_coef(n, s, i, m);
    rhs[(size_t)i * 3 + 1] = or_penta_coef(n, s, i, m + 1);
    rhs[(size_t)i * 3 + 2] = r[i];
  }
  /* forward elimination (no pivoting) */
  for (int k = 0; k < m; ++k) {
    double piv = band[(size_t)k * 5 + 2];
    for (int i = k + 1; i <= k + 2 && i < m; ++i) {
      double l = band[(size_t)i * 5 + 2 + (k - i)] / piv;
      for (int j = k; j <= k + 2 && j < m; ++j)
        band[(size_t)i * 5 + 2 + (j - i)] -= l * band[(size_t)k * 5 + 2 + (j - k)];
      for (int c = 0; c < 3; ++c) rhs[(size_t)i * 3 + c] -= l * rhs[(size_t)k * 3 + c];
    }
  }
  /* back substitution: Y = B^-1 [E0 E1 r_B] */
  for (int i = m - 1; i >= 0; --i) {
    for (int c = 0; c < 3; ++c) {
      double acc = rhs[(size_t)i * 3 + c];
      for (int j = i + 1; j <= i + 2 && j < m; ++j) acc -= band[(size_t)i * 5 + 2 + (j - i)] * rhs[(size_t)j * 3 + c];
      rhs[(size_t)i * 3 + c] = acc / band[(size_t)i * 5 + 2];
    }
  }
  /* Schur complement S = G - F Y[:,0:2], t = r_C - F Y[:,2] */
  double S[2][2], t[2];
  for (int a = 0; a < 2; ++a) {
    for (int b = 0; b < 2; ++b) {
      double acc = or_penta_coef(n, s, m + a, m + b);
      for (int j = 0; j < m; ++j) acc -= or_penta_coef(n, s, m + a, j) * rhs[(size_t)j * 3 + b];
      S[a][b] = acc;
    }
    double acc = r[m + a];
    for (int j = 0; j < m; ++j) acc -= or_penta_coef(n, s, m + a, j) * rhs[(size_t)j * 3 + 2];
    t[a] = acc;
  }
  double det = S[0][0] * S[1][1] - S[0][1] * S[1][0];
  double xm0 = (t[0] * S[1][1] - S[0][1] * t[1]) / det;
  double xm1 = (S[0][0] * t[1] - S[1][0] * t[0]) / det;
  x[m] = xm0;
  x[m + 1] = xm1;
  for (int i = 0; i < m; ++i)
    x[i] = rhs[(size_t)i * 3 + 2] - rhs[(size_t)i * 3 + 0] * xm0 - rhs[(size_t)i * 3 + 1] * xm1;
  free(band);
  free(rhs);
  return OR_OK;
}

/* ------------------------------------------------------------------------------ */
/* Observables (Eq. (4) discretised; read at C^n and the mu^n of the same step):      */
/*   F_h    = hx hy sum [ 1/4 (C^2-1)^2 + 1/2 gamma ((D+x C)^2 + (D+y C)^2) ]         */
/*   dFdt_h = -hx hy sum [ (D+x mu)^2 + (D+y mu)^2 ]                                  */
/* with forward differences D+x v = (v[i+1]-v[i])/hx (periodic).  Summation in        */
/* row-major order.                                                                   */
/* ------------------------------------------------------------------------------ */
void or_observables(int nx, int ny, double hx, double hy, double gamma, const double* C,
                    const double* mu, double* F, double* dFdt) {
  double sF = 0.0, sD = 0.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      int ip = (i + 1) % nx, jp = (j + 1) % ny;
      size_t p = (size_t)j * nx + i;
      double c = C[p];
      double cx = (C[(size_t)j * nx + ip] - c) / hx;
      double cy = (C[(size_t)jp * nx + i] - c) / hy;
      double w = c * c - 1.0;
      sF += 0.25 * w * w + 0.5 * gamma * (cx * cx + cy * cy);
      double mx = (mu[(size_t)j * nx + ip] - mu[p]) / hx;
      double my = (mu[(size_t)jp * nx + i] - mu[p]) / hy;
      sD += mx * mx + my * my;
    }
  *F = hx * hy * sF;
  *dFdt = -(hx * hy * sD);
}

/* Coarsening rate, Eq. (6): beta = -(t/F) dF/dt, t = n dt measured from t = 0. */
double or_beta(double t, double F, double dFdt) { return -(t / F) * dFdt; }

/* ------------------------------------------------------------------------------ */
/* One time step of the delta-form factorised scheme on one member (in place):       */
/*   1. mu, R from C^n (or_rhs);                                                      */
/*   2. W  = A_x^-1 R  on every row   (A_x = I + s_x D_x^4,  s_x = gamma dt / hx^4); */
/*   3. dC = A_y^-1 W  on every column (s_y = gamma dt / hy^4);                       */
/*   4. C^{n+1} = C^n + dC.                                                           */
/* If obs != NULL, obs[0..1] receive F_h and dFdt_h of C^n (before the update).       */
/* ------------------------------------------------------------------------------ */
int or_step(int nx, int ny, double L, double gamma, double dt, double* C, double* obs) {
  if (nx < 5 || ny < 5) return OR_EINVAL;
  double hx = L / nx, hy = L / ny;
  double sx = gamma * dt / (hx * hx * hx * hx);
  double sy = gamma * dt / (hy * hy * hy * hy);
  size_t np = (size_t)nx * ny;
  int nmax = nx > ny ? nx : ny;
  double* mu = (double*)malloc(np * sizeof(double));
  double* R = (double*)malloc(np * sizeof(double));
  double* lin = (double*)malloc((size_t)nmax * sizeof(double));
  double* lout = (double*)malloc((size_t)nmax * sizeof(double));
  int rc = OR_OK;
  if (!mu || !R || !lin || !lout) {
    rc = OR_ENOMEM;
    goto done;
  }
  or_rhs(nx, ny, hx, hy, gamma, dt, C, mu, R);
  if (obs) or_observables(nx, ny, hx, hy, gamma, C, mu, &obs[0], &obs[1]);
  /* rows: R -> W (stored back into R) */
  for (int j = 0; j < ny; ++j) {
    for (int i = 0; i < nx; ++i) lin[i] = R[(size_t)j * nx + i];
    rc = or_cyclic_penta_solve(nx, sx, lin, lout);
    if (rc) goto done;
    for (int i = 0; i < nx; ++i) R[(size_t)j * nx + i] = lout[i];
  }
  /* columns: W -> dC, then C += dC */
  for (int i = 0; i < nx; ++i) {
    for (int j = 0; j < ny; ++j) lin[j] = R[(size_t)j * nx + i];
    rc = or_cyclic_penta_solve(ny, sy, lin, lout);
    if (rc) goto done;
    for (int j = 0; j < ny; ++j) C[(size_t)j * nx + i] = C[(size_t)j * nx + i] + lout[j];
  }
done:
  free(mu);
  free(R);
  free(lin);
  free(lout);
  return rc;
}

/* Observables of the current field without stepping (F_h, dFdt_h at C). */
int or_field_observables(int nx, int ny, double L, double gamma, const double* C, double* F,
                         double* dFdt) {
  if (nx < 5 || ny < 5) return OR_EINVAL;
  double hx = L / nx, hy = L / ny;
  size_t np = (size_t)nx * ny;
  double* mu = (double*)malloc(np * sizeof(double));
  double* R = (double*)malloc(np * sizeof(double));
  if (!mu || !R) {
    free(mu);
    free(R);
    return OR_ENOMEM;
  }
  or_rhs(nx, ny, hx, hy, gamma, 1.0, C, mu, R);
  or_observables(nx, ny, hx, hy, gamma, C, mu, F, dFdt);
  free(mu);
  free(R);
  return OR_OK;
}

/*
 * A run of one member from step index n0 for nsteps steps.  On every step index n with
 * n % every == 0 a sample (t_n, F_h, dFdt_h, beta) is taken from C^n before that step's
 * update and appended to `series` (4 doubles per sample, capacity max_samples).  Samples
 * with t_n >= t1 are added to the running time average of beta (rectangle rule over the
 * samples, the discrete form of Eq. (42)): *beta_sum += beta, *beta_count += 1.
 */
int or_run(int nx, int ny, double L, double gamma, double dt, double* C, int64_t n0,
           int64_t nsteps, int every, double t1, double* series, int64_t max_samples,
           int64_t* nsamples, double* beta_sum, int64_t* beta_count) {
  if (every < 1) return OR_EINVAL;
  int64_t ns = 0;
  for (int64_t n = n0; n < n0 + nsteps; ++n) {
    int take = (n % every) == 0;
    double obs[2];
    int rc = or_step(nx, ny, L, gamma, dt, C, take ? obs : NULL);
    if (rc) return rc;
    if (take) {
      double t = (double)n * dt;
      double beta = or_beta(t, obs[0], obs[1]);
      if (series && ns < max_samples) {
        series[ns * 4 + 0] = t;
        series[ns * 4 + 1] = obs[0];
        series[ns * 4 + 2] = obs[1];
        series[ns * 4 + 3] = beta;
      }
      ++ns;
      if (t >= t1) {
        *beta_sum += beta;
        *beta_count += 1;
      }
    }
  }
  if (nsamples) *nsamples = ns;
  return OR_OK;
}

/* ------------------------------------------------------------------------------ */
/* Ensemble statistics of beta across the M runs of one ensemble.                   */
/* beta[j * ld + s] is run j's beta at sample s (j < M, s < T); every run is sampled */
/* at the same times.  A non-finite value (a diverged run) is left out of sample s's */
/* statistics, and the count of values used is reported.                             */
/* ------------------------------------------------------------------------------ */

/*
 * Moments across the ensemble per sample time, Sec. 3.3 Eqs. (41a,b) (applied to the
 * Cahn-Hilliard ensembles in Secs. 4.2-4.3):
 *     mu_1 = (1/M) sum_j beta_j,    mu_p = (1/M) sum_j (beta_j - mu_1)^p,  p = 2, 3, 4,
 * with M the number of finite values.  out[s * 5 + 0] = that count, out[s * 5 + p] = mu_p
 * (NaN when the count is 0).
 */
void or_beta_moments(int64_t M, int64_t T, int64_t ld, const double* beta, double* out) {
  for (int64_t s = 0; s < T; ++s) {
    int64_t count = 0;
    double sum = 0.0;
    for (int64_t j = 0; j < M; ++j) {
      double b = beta[j * ld + s];
      if (isfinite(b)) {
        sum += b;
        count += 1;
      }
    }
    double mu1 = count > 0 ? sum / (double)count : NAN;
    double c2 = 0.0, c3 = 0.0, c4 = 0.0;
    for (int64_t j = 0; j < M; ++j) {
      double b = beta[j * ld + s];
      if (isfinite(b)) {
        double d = b - mu1;
        c2 += d * d;
        c3 += d * d * d;
        c4 += d * d * d * d;
      }
    }
    out[s * 5 + 0] = (double)count;
    out[s * 5 + 1] = mu1;
    out[s * 5 + 2] = count > 0 ? c2 / (double)count : NAN;
    out[s * 5 + 3] = count > 0 ? c3 / (double)count : NAN;
    out[s * 5 + 4] = count > 0 ? c4 / (double)count : NAN;
  }
}

/*
 * Histogram of beta across the ensemble per sample time, the empirical form of
 * p_beta(b, t), Sec. 1 Eq. (7).  Bin width w = (hi - lo) / nbins; a finite value b < lo
 * counts in out[s][0]; otherwise k = floor((b - lo) / w) selects out[s][k + 1] when
 * k < nbins, else out[s][nbins + 1].  Non-finite values are not counted.
 * out is T x (nbins + 2).  Returns OR_EINVAL unless lo < hi (finite) and nbins >= 1.
 */
int or_beta_histogram(int64_t M, int64_t T, int64_t ld, const double* beta, double lo, double hi,
                      int nbins, int64_t* out) {
  if (!(isfinite(lo) && isfinite(hi) && lo < hi) || nbins < 1) return OR_EINVAL;
  double w = (hi - lo) / (double)nbins;
  for (int64_t s = 0; s < T; ++s) {
    int64_t* row = out + s * (int64_t)(nbins + 2);
    for (int k = 0; k < nbins + 2; ++k) row[k] = 0;
    for (int64_t j = 0; j < M; ++j) {
      double b = beta[j * ld + s];
      if (!isfinite(b)) continue;
      if (b < lo) {
        row[0] += 1;
        continue;
      }
      double k = floor((b - lo) / w);
      if (k < (double)nbins)
        row[(int64_t)k + 1] += 1;
      else
        row[nbins + 1] += 1;
    }
  }
  return OR_OK;
}

/*
 * Trend statistics of the moment series (t[s], mu1[s], mu2[s]), s < T, t increasing.
 *   out[0]: the window estimate of beta_0, Sec. 3.3 Eq. (42):
 *           (1/(t_b - t_a)) * integral of mu_1 over the samples with t1 <= t <= t2,
 *           the integral by the trapezoid rule between consecutive such samples, t_a and
 *           t_b the first and last of them (t_b - t_a = t2 - t1 when samples fall on both
 *           ends of the window); NaN with fewer than two samples in the window.
 *   out[1]: k of the least-squares fit mu_2 = k t (a line through the origin), Sec. 3.3
 *           and Sec. 4.2 Table 4, over the samples with tf1 <= t <= tf2:
 *           k minimises sum (mu_2 - k t)^2, i.e. k = sum(t mu_2) / sum(t^2); NaN when that
 *           denominator is 0.
 *   out[2], out[3]: the numbers of samples in the two windows.
 */
void or_beta_trend(int64_t T, const double* t, const double* mu1, const double* mu2, double t1,
                   double t2, double tf1, double tf2, double* out) {
  double integral = 0.0, ta = 0.0, tb = 0.0;
  int64_t nw = 0;
  for (int64_t s = 0; s < T; ++s) {
    if (t[s] >= t1 && t[s] <= t2) {
      if (nw == 0) ta = t[s];
      tb = t[s];
      nw += 1;
      if (s + 1 < T && t[s + 1] >= t1 && t[s + 1] <= t2)
        integral += 0.5 * (t[s + 1] - t[s]) * (mu1[s] + mu1[s + 1]);
    }
  }
  double stm = 0.0, stt = 0.0;
  int64_t nf = 0;
  for (int64_t s = 0; s < T; ++s) {
    if (t[s] >= tf1 && t[s] <= tf2) {
      stm += t[s] * mu2[s];
      stt += t[s] * t[s];
      nf += 1;
    }
  }
  out[0] = nw >= 2 ? integral / (tb - ta) : NAN;
  out[1] = stt > 0.0 ? stm / stt : NAN;
  out[2] = (double)nw;
  out[3] = (double)nf;
}

/* ------------------------------------------------------------------------------ */
/* Grid-refinement error, Appendix A: the L1 distance between a field on an n-grid   */
/* and the same run on the n/2-grid, the fine field restricted by averaging 2 x 2    */
/* blocks.  Grid points are taken at cell centres, so fine points (2i, 2j),          */
/* (2i+1, 2j), (2i, 2j+1), (2i+1, 2j+1) surround coarse point (i, j) symmetrically.   */
/* ------------------------------------------------------------------------------ */

/*
 * E = (1/|Omega|) sum_{i,j} | 1/4 [f(2i,2j) + f(2i+1,2j) + f(2i,2j+1) + f(2i+1,2j+1)]
 *                             - c(i,j) | dx_c dy_c
 *   = mean over the coarse points of |restricted fine - coarse|,
 * fine[j * nx + i] on nx x ny points (both even), coarse[j * (nx/2) + i] on nx/2 x ny/2.
 * Returns NAN unless nx and ny are even and >= 2.
 */
double or_refinement_error(int nx, int ny, const double* fine, const double* coarse) {
  if (nx < 2 || ny < 2 || nx % 2 || ny % 2) return NAN;
  int mx = nx / 2, my = ny / 2;
  double sum = 0.0;
  for (int j = 0; j < my; ++j) {
    for (int i = 0; i < mx; ++i) {
      double r = 0.25 * (fine[(size_t)(2 * j) * nx + 2 * i] + fine[(size_t)(2 * j) * nx + 2 * i + 1] +
                         fine[(size_t)(2 * j + 1) * nx + 2 * i] + fine[(size_t)(2 * j + 1) * nx + 2 * i + 1]);
      sum += fabs(r - coarse[(size_t)j * mx + i]);
    }
  }
  return sum / ((double)mx * (double)my);
}

/* ------------------------------------------------------------------------------ */
/* Model 1: a population of N droplets under mean-field (LSW-type) dynamics.          */
/*   dR_i/dt = H(R_i + eps) (-1/R_i^2 + u/R_i),   Sec. 2.1 Eq. (13), regularised as  */
/*                                                 in Sec. 3.1 Eq. (39);              */
/*   u = sum_i H(R_i) / sum_i H(R_i) R_i,          Sec. 2.1 Eq. (14);                 */
/* H(s) = 1 for s > 0, else 0.  Observables (Sec. 2.4): F = 1/2 sum H(R_i) R_i^2      */
/* (Eq. (31) with the volume constraint met), dF/dt = -sum H(R_i)/R_i (1 - u R_i)^2   */
/* (Eq. (33)), beta = -(t/F) dF/dt (Eq. (36)).  Start: R_i(0) = r_i (Eq. (38)).       */
/* Time stepping: the Dormand-Prince 5(4) Runge-Kutta pair (J. R. Dormand and P. J.   */
/* Prince, J. Comput. Appl. Math. 6 (1980) 19-26), the method of Matlab's ODE45 that  */
/* the paper names, on the whole N-vector with one step size.                         */
/* ------------------------------------------------------------------------------ */

/* Right-hand side of the droplet system at radii R: out_i = dR_i/dt; *u_out = u. */
static void or_drop_rhs(int N, const double* R, double eps, double* out, double* u_out) {
  double alive = 0.0, sum_r = 0.0;
  for (int i = 0; i < N; ++i) {
    if (R[i] > 0.0) {
      alive += 1.0;
      sum_r += R[i];
    }
  }
  double u = sum_r > 0.0 ? alive / sum_r : 0.0;
  for (int i = 0; i < N; ++i) out[i] = (R[i] + eps > 0.0) ? (-1.0 / (R[i] * R[i]) + u / R[i]) : 0.0;
  if (u_out) *u_out = u;
}

/* F, dF/dt and the number of droplets with R > 0 (Eqs. (31), (33)). */
void or_drop_observables(int N, const double* R, double* F, double* dFdt, double* alive) {
  double cnt = 0.0, sum_r = 0.0;
  for (int i = 0; i < N; ++i) {
    if (R[i] > 0.0) {
      cnt += 1.0;
      sum_r += R[i];
    }
  }
  double u = sum_r > 0.0 ? cnt / sum_r : 0.0;
  double f = 0.0, d = 0.0;
  for (int i = 0; i < N; ++i) {
    if (R[i] > 0.0) {
      f += 0.5 * R[i] * R[i];
      double g = 1.0 - u * R[i];
      d += g * g / R[i];
    }
  }
  *F = f;
  *dFdt = -d;
  *alive = cnt;
}

/* The Dormand-Prince tableau: nodes c, stage weights a (lower triangle, row s holds the
 * weights of stages 1..s-1 for stage s), the fifth-order weights b (= row 7 of a) and the
 * embedded fourth-order weights bs. */
static const double OR_DP_C[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
static const double OR_DP_A[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
static const double OR_DP_BS[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0,
                                   -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};

/*
 * One Dormand-Prince step of size h from y (n components) for a right-hand side f:
 * k[0] must hold f(y) on entry (first-same-as-last); on return ynew holds the
 * fifth-order solution, k[6] = f(ynew), and err[i] = ynew_i - (fourth-order solution)_i.
 * k is 7 x n scratch, ys n scratch.
 */
typedef void (*or_rhs_fn)(int n, const double* y, double eps, double* out, double* u_out);

static void or_dp_step(int n, const double* y, double h, double eps, or_rhs_fn f, double* k, double* ys,
                       double* ynew, double* err) {
  for (int s = 1; s < 7; ++s) {
    for (int i = 0; i < n; ++i) {
      double acc = 0.0;
      for (int j = 0; j < s; ++j) acc += OR_DP_A[s][j] * k[(size_t)j * n + i];
      ys[i] = y[i] + h * acc;
    }
    f(n, ys, eps, k + (size_t)s * n, NULL);
  }
  /* stage 7 is evaluated at the fifth-order solution itself (row 7 of a = b) */
  for (int i = 0; i < n; ++i) {
    ynew[i] = ys[i];
    double lo = 0.0;
    for (int j = 0; j < 7; ++j) lo += OR_DP_BS[j] * k[(size_t)j * n + i];
    err[i] = ynew[i] - (y[i] + h * lo);
  }
}

/*
 * Integrate a droplet population from t = 0 to t_end.  R (n values) holds R(0) on entry
 * and R(t_end) on return.  Step control (adaptive when rtol > 0): a step of size h is
 * accepted when the scaled error norm
 *     err = sqrt( (1/n) sum_i ( e_i / (atol + rtol * max(|R_i|, |Rnew_i|)) )^2 ) <= 1,
 * and the next size is h * min(5, max(0.2, 0.9 err^(-1/5))) (at most h after a rejection;
 * 5 h when err = 0); the first try is h0.  With rtol <= 0 every step has size h0 (fixed
 * steps).  Steps are shortened to land exactly on each sample time ts[0 .. ns) (increasing,
 * within [0, t_end]); at each, the sample (t, F, dF/dt, beta, alive) is written to
 * series[5 s ..].  stats[0] = accepted steps, stats[1] = rejected steps.
 * Returns OR_OK, OR_EINVAL (bad arguments; more than max_steps steps; h below 1e-300).
 */
int or_drop_run(int n, double* R, double t_end, int ns, const double* ts, double rtol, double atol, double h0,
                double eps, int64_t max_steps, double* series, int64_t* stats) {
  if (n < 1 || !(t_end >= 0.0) || !(h0 > 0.0) || ns < 0 || max_steps < 1) return OR_EINVAL;
  double* k = (double*)malloc(sizeof(double) * 7 * (size_t)n);
  double* ys = (double*)malloc(sizeof(double) * (size_t)n);
  double* ynew = (double*)malloc(sizeof(double) * (size_t)n);
  double* err = (double*)malloc(sizeof(double) * (size_t)n);
  if (!k || !ys || !ynew || !err) {
    free(k); free(ys); free(ynew); free(err);
    return OR_ENOMEM;
  }
  int rc = OR_OK;
  double t = 0.0, h = h0;
  int next = 0;
  int64_t acc = 0, rej = 0;
  or_drop_rhs(n, R, eps, k, NULL);
  for (;;) {
    while (next < ns && ts[next] <= t) { /* samples due at the current time */
      double F, D, alive;
      or_drop_observables(n, R, &F, &D, &alive);
      double* row = series + 5 * (size_t)next;
      row[0] = t;
      row[1] = F;
      row[2] = D;
      row[3] = or_beta(t, F, D);
      row[4] = alive;
      ++next;
    }
    if (t >= t_end) break;
    if (acc + rej >= max_steps || !(h > 1e-300)) {
      rc = OR_EINVAL;
      break;
    }
    double target = next < ns && ts[next] < t_end ? ts[next] : t_end;
    int lands = h >= target - t;
    double hs = lands ? target - t : h;
    or_dp_step(n, R, hs, eps, or_drop_rhs, k, ys, ynew, err);
    double e2 = 0.0;
    for (int i = 0; i < n; ++i) {
      double sc = atol + rtol * fmax(fabs(R[i]), fabs(ynew[i]));
      double q = err[i] / sc;
      e2 += q * q;
    }
    double en = rtol > 0.0 ? sqrt(e2 / (double)n) : 0.0;
    int accept = rtol <= 0.0 || en <= 1.0;
    if (accept) {
      memcpy(R, ynew, sizeof(double) * (size_t)n);
      memcpy(k, k + (size_t)6 * n, sizeof(double) * (size_t)n);
      t = lands ? target : t + hs;
      ++acc;
    } else {
      ++rej;
    }
    if (rtol > 0.0) {
      double fac = en > 0.0 ? 0.9 * pow(en, -0.2) : 5.0;
      fac = fmin(5.0, fmax(0.2, fac));
      if (!accept) fac = fmin(fac, 1.0);
      h = hs * fac;
    }
  }
  stats[0] = acc;
  stats[1] = rej;
  free(k); free(ys); free(ynew); free(err);
  return rc;
}

/* One Dormand-Prince step of the scalar test equation y' = g(t) = t^p (time-only right-hand
 * side) from (t, y) with step h: returns the fifth-order value, *err = fifth - fourth. */
double or_dp_poly_step(int p, double t, double y, double h, double* err) {
  double k[7];
  for (int s = 0; s < 7; ++s) k[s] = pow(t + OR_DP_C[s] * h, (double)p);
  double hi = 0.0, lo = 0.0;
  for (int j = 0; j < 6; ++j) hi += OR_DP_A[6][j] * k[j];
  for (int j = 0; j < 7; ++j) lo += OR_DP_BS[j] * k[j];
  *err = h * (hi - lo);
  return y + h * hi;
}

/* One Dormand-Prince step of the linear test equation y' = lam y from y with step h:
 * returns the fifth-order value, *err = fifth - fourth. */
double or_dp_lin_step(double lam, double y, double h, double* err) {
  double k[7], ys = y;
  k[0] = lam * y;
  for (int s = 1; s < 7; ++s) {
    double acc = 0.0;
    for (int j = 0; j < s; ++j) acc += OR_DP_A[s][j] * k[j];
    ys = y + h * acc;
    k[s] = lam * ys;
  }
  double lo = 0.0;
  for (int j = 0; j < 7; ++j) lo += OR_DP_BS[j] * k[j];
  *err = ys - (y + h * lo);
  return ys;
}
