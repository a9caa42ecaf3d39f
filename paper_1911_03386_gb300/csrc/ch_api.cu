// ch_api.cu -- host side of libch: the C ABI declared in include/ch.h.
//
// A handle owns one set of device buffers (see ch_internal.h), a stream, the FP64
// constants of every member and captured CUDA graphs of a fixed number of steps.
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "ch.h"
#include "ch_handle.h"
#include "ch_internal.h"

namespace chk {
// Error text for ch_last_error() from other translation units of the library.
void record_error(const char* msg);
}

namespace {
thread_local std::string g_last_error;
}  // namespace

namespace chh {

int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  return fail(CH_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define CH_CUDA(call, what)                      \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return cuda_fail(e_, what); \
  } while (0)

constexpr size_t kSmemMax = 227 * 1024;  // dynamic shared memory per CTA on sm_103a
constexpr double kPrerollTol64 = 1e-17;    // FP64 pre-roll: max |(M^K)_ij| (relative state error)
// FP32 members with max(s_x, s_y) above this keep their field as the pair hi + lo
// (compensated update): the delta-form factor damps the high diagonal modes by only
// ~1/(4s) per step, so the rounding of an FP32 field would accumulate there; at s = 13.8
// (256^2) the plain FP32 field reproduces the FP64 <beta> within one standard error, at
// s = 882 (1024^2) it does not.
constexpr double kCompS = 16.0;
constexpr int kGraphSteps = 16;

// ---------------------------------------------------------------------------------------
// Spectral factor of the cyclic pentadiagonal operator I + s D^4 (stencil
// [s, -4s, 1+6s, -4s, s], symbol 1 + s (z - 2 + 1/z)^2):
//   I + s D^4 = c Q Q^T,  q(z) = 1 - p1 z - p2 z^2 = (1 - a z)(1 - conj(a) z),  |a| < 1.
// The zeros of the symbol solve z^2 - w z + 1 = 0 with w = 2 +- i/sqrt(s); a is the root
// inside the unit circle (a = 2 / (w + sqrt(w^2 - 4)) on the larger-modulus branch), so
// p1 = 2 Re a, p2 = -|a|^2, c = s / |a|^2.  The three coefficient equations
//   c (1 + p1^2 + p2^2) = 1 + 6s,  c (p1 p2 - p1) = -4s,  -c p2 = s
// are then polished by Newton's method in FP64.
// ---------------------------------------------------------------------------------------
bool spectral_factor(double s, double* c, double* p1, double* p2) {
  const double a0 = 1.0 + 6.0 * s, a1 = -4.0 * s, a2 = s;
  const std::complex<double> w(2.0, 1.0 / std::sqrt(s));
  const std::complex<double> disc = std::sqrt(w * w - 4.0);
  const std::complex<double> den = std::abs(w + disc) >= std::abs(w - disc) ? w + disc : w - disc;
  const std::complex<double> a = 2.0 / den;
  double q1 = 2.0 * a.real(), q2 = -std::norm(a), cc = s / std::norm(a);
  for (int it = 0; it < 4; ++it) {
    const double f0 = cc * (1.0 + q1 * q1 + q2 * q2) - a0;
    const double f1 = cc * (q1 * q2 - q1) - a1;
    const double f2 = -cc * q2 - a2;
    // Jacobian rows d(f0, f1, f2)/d(c, p1, p2)
    const double J[3][3] = {{1.0 + q1 * q1 + q2 * q2, 2.0 * cc * q1, 2.0 * cc * q2},
                            {q1 * q2 - q1, cc * (q2 - 1.0), cc * q1},
                            {-q2, 0.0, -cc}};
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (!(std::fabs(det) > 0.0)) break;
    const double f[3] = {f0, f1, f2};
    double dx[3];
    for (int k = 0; k < 3; ++k) {  // Cramer's rule
      double M[3][3];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = (j == k) ? f[i] : J[i][j];
      dx[k] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1]) - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0]) +
               M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) /
              det;
    }
    cc -= dx[0];
    q1 -= dx[1];
    q2 -= dx[2];
  }
  if (!std::isfinite(cc) || !(cc > 0.0) || !std::isfinite(q1) || !std::isfinite(q2)) return false;
  // roots of q outside the unit circle: |a|^2 = -p2 < 1
  if (!(-q2 < 1.0) || !(-q2 > 0.0)) return false;
  const double r0 = cc * (1.0 + q1 * q1 + q2 * q2) - a0;
  const double r1 = cc * (q1 * q2 - q1) - a1;
  const double r2 = -cc * q2 - a2;
  if (!(std::fabs(r0) <= 1e-13 * a0 && std::fabs(r1) <= 1e-13 * a0 && std::fabs(r2) <= 1e-13 * a0)) return false;
  *c = cc;
  *p1 = q1;
  *p2 = q2;
  return true;
}

// Smallest K with max |(M^K)_ij| <= tol for the companion matrix M = [[p1, p2], [1, 0]]:
// a recurrence pre-rolled over K points from a zero state then carries a state error
// below tol relative to the line's largest value.
int preroll_length(double p1, double p2, double tol) {
  double m00 = 1, m01 = 0, m10 = 0, m11 = 1;
  for (int k = 1; k <= 4000000; ++k) {
    const double n00 = p1 * m00 + p2 * m10, n01 = p1 * m01 + p2 * m11;
    m10 = m00;
    m11 = m01;
    m00 = n00;
    m01 = n01;
    const double mx = std::fmax(std::fmax(std::fabs(m00), std::fabs(m01)), std::fmax(std::fabs(m10), std::fabs(m11)));
    if (mx <= tol) return k;
  }
  return -1;
}

// Leading points of an FP64 pre-roll of K points that may run in FP32 (multiple of 16).
// The FP32 part's local error per step is at most 2^-24 (3 + g (3 + |p1| + |p2|)) R: the
// input truncated to FP32 (2^-23 R), the coefficients rounded to FP32 acting on a state of
// at most g R, and two FMA roundings of values up to (1 + |p2| g) R and g R, where
// g = sum_k |(M^k)_00| bounds |y| / R.  Summed through the recurrence the state error is at
// most g2 = sum_k ||M^k||_inf times that, and the FP64 points after it multiply it by
// M^(K - head).  Returns the largest head with ||M^(K - head)||_inf E <= tol R.
int preroll_head_length(double p1, double p2, int K, double tol) {
  double m00 = 1, m01 = 0, m10 = 0, m11 = 1, g = 0, g2 = 0;
  std::vector<double> norms;  // ||M^k||_inf, k = 0 .. K
  for (int k = 0; k <= 4000000; ++k) {
    const double ninf = std::fmax(std::fabs(m00) + std::fabs(m01), std::fabs(m10) + std::fabs(m11));
    if (k <= K) norms.push_back(ninf);
    g += std::fabs(m00);
    g2 += ninf;
    if (ninf <= 1e-30 && k >= K) break;
    const double n00 = p1 * m00 + p2 * m10, n01 = p1 * m01 + p2 * m11;
    m10 = m00;
    m11 = m01;
    m00 = n00;
    m01 = n01;
  }
  const double E = g2 * std::ldexp(1.0, -24) * (3.0 + g * (3.0 + std::fabs(p1) + std::fabs(p2)));
  int tail = 0;  // smallest number of FP64 points that damps E below tol
  while (tail <= K && norms[tail] * E > tol) ++tail;
  if (tail > K) return 0;
  return (K - tail) / 16 * 16;
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// 2x2 row-major matrix product c = a b.
static void mat2_mul(const double* a, const double* b, double* c) {
  const double r0 = a[0] * b[0] + a[1] * b[2], r1 = a[0] * b[1] + a[1] * b[3];
  const double r2 = a[2] * b[0] + a[3] * b[2], r3 = a[2] * b[1] + a[3] * b[3];
  c[0] = r0;
  c[1] = r1;
  c[2] = r2;
  c[3] = r3;
}

// Scan tables of the segment row sweep (S points per lane, G lanes, n = S G) for the
// companion matrix M = [[p1, p2], [1, 0]]; products of M in FP64.
void seg_tables(double p1, double p2, int S, int G, chk::SegTable* t) {
  std::memset(t, 0, sizeof *t);
  if (G > 64) G = 64;  // callers keep G <= 64 (B holds 64 segment powers)
  const double M[4] = {p1, p2, 1.0, 0.0};
  double MS[4] = {1.0, 0.0, 0.0, 1.0};
  for (int k = 0; k < S; ++k) mat2_mul(M, MS, MS);
  double Ad[4] = {MS[0], MS[1], MS[2], MS[3]};
  for (int d = 0; d < 5 && (1 << d) < G; ++d) {
    std::memcpy(t->A[d], Ad, sizeof Ad);
    mat2_mul(Ad, Ad, Ad);
  }
  double Bl[4] = {1.0, 0.0, 0.0, 1.0};
  for (int l = 0; l < G; ++l) {
    std::memcpy(t->B[l], Bl, sizeof Bl);
    mat2_mul(Bl, MS, Bl);
  }
  // Bl = M^(S G) = M^n;  P = (I - M^n)^-1
  const double a = 1.0 - Bl[0], b = -Bl[1], c = -Bl[2], d = 1.0 - Bl[3];
  const double det = a * d - b * c;
  t->P[0] = d / det;
  t->P[1] = -b / det;
  t->P[2] = -c / det;
  t->P[3] = a / det;
  for (int i = 0; i < 20; ++i) (&t->Af[0][0])[i] = (float)(&t->A[0][0])[i];
  for (int i = 0; i < 256; ++i) (&t->Bf[0][0])[i] = (float)(&t->B[0][0])[i];
  for (int i = 0; i < 4; ++i) t->Pf[i] = (float)t->P[i];
}

// Closed-form segment responses of the recurrence y_i = r_i + p1 y_{i-1} + p2 y_{i-2} over
// S <= 32 points (see SegTable::Hf), computed in FP64 and rounded to FP32.
void seg_responses(double p1, double p2, int S, chk::SegTable* t) {
  double h[2][32], g[2][32], k[2][32];
  for (int j = 0; j < 2; ++j) {
    // forward homogeneous response to (y_-1, y_-2) = e_j
    double y1 = j == 0 ? 1.0 : 0.0, y2 = j == 0 ? 0.0 : 1.0;
    for (int i = 0; i < S; ++i) {
      const double yi = p1 * y1 + p2 * y2;
      h[j][i] = yi;
      y2 = y1;
      y1 = yi;
    }
    // its backward pass from a zero state
    double x1 = 0.0, x2 = 0.0;
    for (int i = S - 1; i >= 0; --i) {
      const double xi = h[j][i] + p1 * x1 + p2 * x2;
      g[j][i] = xi;
      x2 = x1;
      x1 = xi;
    }
    // backward homogeneous response to (x_S, x_S+1) = e_j
    x1 = j == 0 ? 1.0 : 0.0;
    x2 = j == 0 ? 0.0 : 1.0;
    for (int i = S - 1; i >= 0; --i) {
      const double xi = p1 * x1 + p2 * x2;
      k[j][i] = xi;
      x2 = x1;
      x1 = xi;
    }
  }
  for (int u = 0; u < 32; ++u) {
    const bool in = u < S;
    t->Hf[u][0] = in ? (float)g[0][u] : 0.f;
    t->Hf[u][1] = in ? (float)g[1][u] : 0.f;
    t->Hf[u][2] = in ? (float)k[0][u] : 0.f;
    t->Hf[u][3] = in ? (float)k[1][u] : 0.f;
  }
}

bool is_pow2_upto32(int g) { return g >= 1 && g <= 32 && (g & (g - 1)) == 0; }

}  // namespace chh

void chk::record_error(const char* msg) { g_last_error = msg; }


namespace chh {

void drop_graph(ch_ensemble* h) {
  if (h->graph) cudaGraphExecDestroy(h->graph);
  h->graph = nullptr;
  h->graph_steps = 0;
}

void free_device(ch_ensemble* h) {
  drop_graph(h);
  cudaFree(h->C);
  cudaFree(h->W);
  cudaFree(h->dmp);
  cudaFree(h->dms);
  cudaFree(h->dseg);
  cudaFree(h->dsegy);
  cudaFree(h->dcst);
  cudaFree(h->drt);
  cudaFree(h->dst);
  cudaFree(h->dct);
  cudaFree(h->dres);
  cudaFree(h->dpart);
  cudaFree(h->dseries);
  cudaFree(h->dobs);
  h->C = h->W = nullptr;
  h->dmp = nullptr;
  h->dms = nullptr;
  h->dseg = h->dsegy = nullptr;
  h->dcst = nullptr;
  h->cap_cst = 0;
  h->drt = h->dst = h->dct = h->dres = nullptr;
  h->cap_rt = h->cap_st = h->cap_ct = h->cap_part = h->cap_res = 0;
  h->dpart = nullptr;
  h->dseries = h->dobs = nullptr;
}

int validate_desc(const ch_member_desc& d, int k) {
  char buf[160];
  if (d.nx < 5 || d.ny < 5) {
    snprintf(buf, sizeof buf, "member %d: nx=%d ny=%d, both must be >= 5", k, d.nx, d.ny);
    return fail(CH_EINVAL, buf);
  }
  if ((int64_t)d.nx * d.ny > (int64_t)1 << 30) {
    snprintf(buf, sizeof buf, "member %d: nx*ny too large", k);
    return fail(CH_EINVAL, buf);
  }
  if (!finite_pos(d.L) || !finite_pos(d.gamma) || !finite_pos(d.dt)) {
    snprintf(buf, sizeof buf, "member %d: L, gamma and dt must be finite and > 0", k);
    return fail(CH_EINVAL, buf);
  }
  if (!std::isfinite(d.C0)) {
    snprintf(buf, sizeof buf, "member %d: C0 is not finite", k);
    return fail(CH_EINVAL, buf);
  }
  return CH_OK;
}

// Constants of one member (all computed in FP64).
int fill_params(const ch_member_desc& d, int precision, MemberParams* p) {
  std::memset(p, 0, sizeof *p);
  p->nx = d.nx;
  p->ny = d.ny;
  p->L = d.L;
  p->hx = d.L / d.nx;
  p->hy = d.L / d.ny;
  p->gamma = d.gamma;
  p->dt = d.dt;
  p->C0 = d.C0;
  p->seed = d.seed;
  p->counter_base = d.counter_base;
  const double hx2 = p->hx * p->hx, hy2 = p->hy * p->hy;
  p->a = 1.0 - 2.0 * d.gamma / hx2 - 2.0 * d.gamma / hy2;
  p->bx = d.gamma / hx2;
  p->by = d.gamma / hy2;
  p->rho = hx2 / hy2;
  p->w0 = -2.0 * (1.0 + p->rho);
  const double sigma = d.gamma * d.dt;
  const double sx = sigma / (hx2 * hx2), sy = sigma / (hy2 * hy2);
  if (!spectral_factor(sx, &p->cx, &p->p1x, &p->p2x) || !spectral_factor(sy, &p->cy, &p->p1y, &p->p2y))
    return fail(CH_EINVAL, "factorisation of I + s D^4 did not converge (s out of range)");
  const double tol = precision == CH_FP64 ? kPrerollTol64 : 1e-8;
  p->kx = preroll_length(p->p1x, p->p2x, tol);
  p->ky = preroll_length(p->p1y, p->p2y, tol);
  if (p->kx < 0 || p->ky < 0) return fail(CH_EINVAL, "decay of I + s D^4 too slow (s out of range)");
  p->kappa = d.dt / (hx2 * p->cx * p->cy);
  p->fa = (float)p->a;
  p->fbx = (float)p->bx;
  p->fby = (float)p->by;
  p->frho = (float)p->rho;
  p->fw0 = (float)p->w0;
  p->fp1x = (float)p->p1x;
  p->fp2x = (float)p->p2x;
  p->fp1y = (float)p->p1y;
  p->fp2y = (float)p->p2y;
  p->fkappa = (float)p->kappa;
  p->comp = precision == CH_FP32 && std::max(sx, sy) > kCompS ? 1 : 0;
  p->lo_offset = -1;
  p->every = 1;
  p->t1 = 0.0;
  return CH_OK;
}

// C tile (nr+4 rows, dense pitch when rows move in 16-byte pieces) + mu tile (nr+2 rows,
// pitch nx+1) + the FP64 reduction buffer; R' and the row sweep reuse the C tile's memory.
size_t rows_smem_bytes(int nr, int nx, size_t elt, int threads) {
  const int lc = (nx * (int)elt) % 16 == 0 ? nx : nx + 1;
  const size_t c_region = std::max((size_t)(nr + 4) * lc, (size_t)nr * (nx + 1));
  size_t b = (c_region + (size_t)(nr + 2) * (nx + 1)) * elt;
  b = (b + 15) & ~(size_t)15;
  return b + (size_t)2 * (threads / 32) * sizeof(double);
}

// Segment form: C tile buffer(s) (nr+4 rows, dense pitch; two when the kernel is
// persistent) + mu tile (nr+2 rows, 16 bytes of padding after every segment of S) + 24
// scan constants and the sample flag (28 elements) + the FP64 reduction buffer; tile
// sizes rounded to 4 elements.
size_t seg_ctile(int nr, int nx) { return ((size_t)(nr + 4) * nx + 3) / 4 * 4; }
size_t seg_mtile(int nr, int nx, int S, size_t elt) {
  return ((size_t)(nr + 2) * ((size_t)nx + (16 / elt) * (size_t)(nx / S)) + 3) / 4 * 4;
}
size_t seg_smem_bytes(size_t ccap, size_t mcap, int nbuf, size_t elt, int threads) {
  size_t b = ((size_t)nbuf * ccap + mcap + 28) * elt;
  b = (b + 15) & ~(size_t)15;
  return b + (size_t)2 * (threads / 32) * sizeof(double);
}
size_t rows_seg_smem_bytes(int nr, int nx, int S, size_t elt, int threads, int nbuf) {
  return seg_smem_bytes(seg_ctile(nr, nx), seg_mtile(nr, nx, S, elt), nbuf, elt, threads);
}

// Stencil block: C (nr+4) x (nc+4), mu (nr+2) x (nc+2), then the FP64 reduction buffer.
size_t blk_smem_bytes(int nr, int nc, size_t elt, int threads) {
  size_t b = ((size_t)(nr + 4) * (nc + 4) + (size_t)(nr + 2) * (nc + 2)) * elt;
  b = (b + 15) & ~(size_t)15;
  return b + (size_t)2 * (threads / 32) * sizeof(double);
}

size_t sweep_smem_bytes(int nr, int nx, size_t elt) { return (size_t)nr * (nx + 1) * elt; }

// W panel swept in place + C panel, twice when double-buffered
size_t cols_panel_elems(int nc, int ny) { return (size_t)ny * (nc + 1); }
size_t cols_smem_bytes(int nc, int ny, size_t elt, bool persist) {
  return (size_t)(persist ? 4 : 2) * cols_panel_elems(nc, ny) * elt;
}

int round_warps(int t) { return ((t + 31) / 32) * 32; }

// Tiles and launch shapes from the tuning request (fields <= 0 take the defaults of the
// precision: FP64 split form with one thread per line, FP32 fused form with chunked
// sweeps).  Band heights and panel widths shrink per member until they fit the shared
// memory; a member's tiles depend only on its size, the precision and the tuning.
int build_tiles(ch_ensemble* h, const ch_tuning& t) {
  const bool f64 = h->precision == CH_FP64;
  const int split = t.split >= 0 ? (t.split ? 1 : 0) : (f64 ? 1 : 0);
  const int threads = t.threads > 0 ? t.threads : (f64 ? 512 : 256);
  if (threads % 32 || threads > 512) return fail(CH_EINVAL, "threads must be a multiple of 32, at most 512");
  const int want_br = t.rows_band > 0 ? t.rows_band : (f64 ? 16 : 32);
  const int want_br_seg = t.rows_band > 0 ? t.rows_band : 16;
  const int want_bs = t.sweep_band > 0 ? t.sweep_band : 32;
  const int want_bc = t.cols_panel > 0 ? t.cols_panel : 32;
  if (t.sweep_band > 512 || want_bc * std::max(1, t.cols_p) > threads || want_br * std::max(1, t.rows_p) > threads)
    return fail(CH_EINVAL, "band/panel times threads per line exceeds the CTA size");
  // streaming sweeps: split form (rows and columns), or in the fused form for the columns
  // of members outside the segment column form; default on for CH_FP64
  const int stream = t.stream >= 0 ? (t.stream ? 1 : 0) : (f64 ? 1 : 0);
  const bool persist = t.persist > 0 && (t.persist & 1);
  const bool seg_persist = t.persist > 0 && (t.persist & 2) != 0;
  const int max_wp = f64 ? 16 : 32;

  // Kernel class of each member, from its own size and the tuning only (a run's arithmetic
  // must not depend on the other members): segment-form rows with S = 16 or 32 points per
  // lane (nx / S lanes per row, a power of two <= 32) or chunked sweeps; segment-form
  // columns with S = 32 or 16 rows per warp (ny / S warps) or panels / streaming.
  auto row_fits = [&](const MemberParams& p, int S) {
    return p.nx % S == 0 && is_pow2_upto32(p.nx / S) && (p.nx * (int)h->elt) % 16 == 0;
  };
  // segment columns: ny / S segments in one CTA (at most max_wp warps) or over a pair of
  // CTAs of a cluster (at most 2 max_wp)
  auto col_fits = [&](const MemberParams& p, int S) {
    const int wp = p.ny / S;
    return p.ny % S == 0 && wp >= 1 && (wp & (wp - 1)) == 0 && wp <= 2 * max_wp;
  };
  auto col_pair = [&](const MemberParams& p, int S) { return p.ny / S > max_wp; };
  // transposed-block rows: nx = 32 nw, nw <= 16
  auto rowT_fits = [&](const MemberParams& p) { return p.nx % 32 == 0 && p.nx / 32 <= 16; };
  auto row_class = [&](const MemberParams& p) {  // 1: transposed-block, 16 / 32: segment, 0: chunked
    if (split || t.row_seg < 0) return 0;
    if (t.row_seg > 0) return t.row_seg;
    return row_fits(p, 16) ? 16 : row_fits(p, 32) ? 32 : 0;
  };
  // split form: segment-form row sweep (rowseg_kernel) for FP32 members that fit, or for
  // every member with an explicit S; the pre-rolled sweeps otherwise (FP64 default: one
  // thread per line costs fewer FP64 operations)
  auto sweep_class = [&](const MemberParams& p) {
    if (!split || t.row_seg < 0 || t.row_seg == 1) return 0;
    if (t.row_seg > 1) return t.row_seg;
    if (f64) return 0;
    return row_fits(p, 16) ? 16 : row_fits(p, 32) ? 32 : 0;
  };
  auto col_class = [&](const MemberParams& p) {
    if (t.col_seg < 0 || (t.col_seg == 0 && f64 && split)) return 0;
    if (t.col_seg > 0) return t.col_seg;
    for (int pass = 0; pass < 2; ++pass)  // one CTA per panel first, then CTA pairs
      for (int S : {32, 16})
        if (col_fits(p, S) && col_pair(p, S) == (pass == 1)) return S;
    return 0;
  };
  // class index of a segment-form member's columns: S = 16, 32 in one CTA, then over pairs
  auto col_index = [&](const MemberParams& p, int S) { return (S == 32 ? 1 : 0) + (col_pair(p, S) ? 2 : 0); };
  // cluster-resident form (FP32): nx = 128 or 256, ny = 32 Q with Q <= 8 CTAs per cluster.
  // By default not for compensated 256-wide members: their C, lo and mu/W tiles take 118 KB
  // of shared memory, one CTA per SM, and the tiled kernels step them faster
  auto resident = [&](const MemberParams& p) {
    const bool fits = (p.nx == 128 || p.nx == 256) && p.ny % 32 == 0 && p.ny >= 32 && p.ny <= 256;
    return !f64 && fits && (t.resident == 1 || (t.resident == 0 && !(p.comp && p.nx == 256)));
  };
  // rows per CTA of a resident member: 64 (one 512-thread CTA per SM, half the CTAs per
  // member) for 256-column members whose ny is a multiple of 64 when asked for, else 32
  auto resident_rows = [&](const MemberParams& p) {
    return (t.resident_rows == 64 && p.nx == 256 && p.ny % 64 == 0) ? 64 : 32;
  };
  int cwarps[4] = {8, 8, max_wp, max_wp};  // warps per CTA of each class
  for (int k = 0; k < h->m; ++k) {
    if (!h->has(k) || resident(h->hp[k])) continue;
    const MemberParams& p = h->hp[k];
    if (t.row_seg == 1 && !split && !rowT_fits(p))
      return fail(CH_EINVAL, "row_seg 1: some member's nx is not 32 times at most 16");
    if (t.row_seg > 1 && !row_fits(p, t.row_seg))
      return fail(CH_EINVAL, "row_seg: some member's nx is not S times a power of two <= 32");
    if (t.col_seg > 0 && !col_fits(p, t.col_seg))
      return fail(CH_EINVAL, "col_seg: some member's ny is not S times a power of two <= 64 (<= 32 for FP64)");
    const int cc = col_class(p);
    if (cc && !col_pair(p, cc)) cwarps[col_index(p, cc)] = std::max(cwarps[col_index(p, cc)], p.ny / cc);
  }

  std::vector<Tile> rts[3], csts[4], sts[3], ct;  // rows: S = 16, S = 32, chunked; columns: 4 classes
  std::vector<Tile> rcl[chk::kResClasses];        // cluster-resident members by class
  std::vector<Tile> rtb;                          // stencil blocks of long rows (last)
  std::vector<Tile> rtT[17];                   // rows, transposed-block form, by nw
  chk::LaunchShape sh{};
  sh.split = split;
  sh.stream = stream;
  sh.rows_threads = threads;
  sh.cols_threads = threads;
  sh.sweep_threads = 0;
  int64_t part = 0;
  for (int k = 0; k < h->m; ++k) {
    MemberParams& p = h->hp[k];
    if (!h->has(k)) {
      p.nbands = 0;
      p.partial_base = part;
      continue;
    }
    if (resident(p)) {
      // one tile per member; one partial slot per CTA of its cluster.  Scan tables: rows
      // of 16 segments of nx / 16 points, columns of ny / (nx / 8) segments of nx / 8 (the
      // same for both CTA heights)
      const int nr = resident_rows(p), Q = p.ny / nr;
      rcl[chk::res_class(p.nx, nr, p.comp, Q)].push_back(Tile{k, 0, p.ny, 0, 0, 0});
      p.seg_g = p.row_t = p.col_s = 0;
      p.kx32 = 0;
      p.nbands = Q;
      p.partial_base = part;
      part += Q;
      seg_tables(p.p1x, p.p2x, p.nx / 16, 16, &h->hseg[k]);
      seg_tables(p.p1y, p.p2y, p.nx / 8, p.ny / (p.nx / 8), &h->hsegy[k]);
      seg_responses(p.p1y, p.p2y, p.nx / 8, &h->hsegy[k]);
      continue;
    }
    const int rc = row_class(p), cc = col_class(p), ri = rc == 16 ? 0 : rc == 32 ? 1 : 2;
    const int sc = sweep_class(p), si = sc == 16 ? 0 : sc == 32 ? 1 : 2;
    const bool seg = rc > 1;
    int br = std::min(p.ny, rc == 1 ? 32 : seg ? want_br_seg : want_br);
    auto row_bytes = [&](int nr) {
      return seg ? rows_seg_smem_bytes(nr, p.nx, rc, h->elt, threads, seg_persist ? 2 : 1)
                 : rows_smem_bytes(nr, p.nx, h->elt, threads);
    };
    // FP64 split form: rows too long for a band of the requested height run the stencil in
    // blocks of br rows x kBlockCols columns
    const bool blk = split && f64 && row_bytes(br) > kSmemMax;
    while (!blk && rc != 1 && br > 1 && row_bytes(br) > kSmemMax) br = (br + 1) / 2;
    // segment form without an explicit band: at least two CTAs per SM (wide rows)
    if (seg && t.rows_band <= 0)
      while (br > 4 && row_bytes(br) > kSmemMax / 2) br = (br + 1) / 2;
    if (!blk && rc != 1 && row_bytes(br) > kSmemMax) return fail(CH_EINVAL, "row too long for shared memory");
    p.seg_g = seg ? p.nx / rc : sc ? p.nx / sc : 0;
    p.row_t = rc == 1 ? p.nx / 32 : 0;
    p.col_s = cc;
    if (rc == 1) seg_tables(p.p1x, p.p2x, 32, p.nx / 32, &h->hseg[k]);
    if (sc) seg_tables(p.p1x, p.p2x, sc, p.nx / sc, &h->hseg[k]);
    if (seg) {
      seg_tables(p.p1x, p.p2x, rc, p.seg_g, &h->hseg[k]);
      sh.seg_ccap[ri] = std::max(sh.seg_ccap[ri], (int)seg_ctile(br, p.nx));
      sh.seg_mcap[ri] = std::max(sh.seg_mcap[ri], (int)seg_mtile(br, p.nx, rc, h->elt));
    }
    // FP32 heads of the FP64 streaming row sweeps' pre-rolls.  (The column stream with heads
    // measured slower: 0.299 against 0.259 ms at 256 x 256^2, so its pre-rolls stay FP64.)
    p.kx32 = f64 && stream && t.preroll_head >= 0 ? preroll_head_length(p.p1x, p.p2x, p.kx, kPrerollTol64) : 0;
    p.rows_p = t.rows_p > 0 ? t.rows_p : (f64 ? 1 : std::max(1, std::min(threads / br, p.nx / 64)));
    if (br * p.rows_p > threads) p.rows_p = std::max(1, threads / br);
    int bs = stream ? std::min(p.ny, 32) : std::min(p.ny, want_bs);
    while (bs > 1 && !stream && sweep_smem_bytes(bs, p.nx, h->elt) > kSmemMax) bs = (bs + 1) / 2;
    int bc = stream ? std::min(p.nx, 32) : std::min(p.nx, want_bc);
    if (!cc) {
      while (bc > 1 && !stream && cols_smem_bytes(bc + 3, p.ny, h->elt, persist) > kSmemMax) bc = (bc + 1) / 2;
      if (!stream && cols_smem_bytes(bc + 3, p.ny, h->elt, persist) > kSmemMax)
        return fail(CH_EINVAL, "column too long for shared memory");
    }
    p.cols_p = t.cols_p > 0 ? t.cols_p : (f64 ? 1 : std::max(1, std::min(threads / bc, p.ny / 64)));
    if (bc * p.cols_p > threads) p.cols_p = std::max(1, threads / bc);
    int b = 0;
    std::vector<Tile>& rdst = rc == 1 ? rtT[p.nx / 32] : rts[ri];
    if (blk) {
      const int nc = std::min(p.nx, chk::kBlockCols);
      while (br > 1 && blk_smem_bytes(br, nc, h->elt, threads) > kSmemMax) br = (br + 1) / 2;
      for (int j0 = 0; j0 < p.ny; j0 += br)
        for (int x0 = 0; x0 < p.nx; x0 += nc, ++b)
          rtb.push_back(Tile{k, j0, std::min(br, p.ny - j0), b, x0, std::min(nc, p.nx - x0)});
      sh.blk_smem = std::max(sh.blk_smem, blk_smem_bytes(br, nc, h->elt, threads));
    } else {
      for (int j0 = 0; j0 < p.ny; j0 += br, ++b) rdst.push_back(Tile{k, j0, std::min(br, p.ny - j0), b});
    }
    p.nbands = b;
    p.partial_base = part;
    part += b;
    if (split && sc) {
      // segment-form sweep: one row per lane group, two rounds per CTA
      const int rows = 2 * (std::min(threads, 256) / 32) * (32 / (p.nx / sc));
      int q = 0;
      for (int j0 = 0; j0 < p.ny; j0 += rows, ++q) sts[si].push_back(Tile{k, j0, std::min(rows, p.ny - j0), q});
    } else if (split) {
      int q = 0;
      for (int j0 = 0; j0 < p.ny; j0 += bs, ++q) sts[2].push_back(Tile{k, j0, std::min(bs, p.ny - j0), q});
      if (!stream) {
        sh.sweep_smem = std::max(sh.sweep_smem, sweep_smem_bytes(bs, p.nx, h->elt));
        sh.sweep_threads = std::max(sh.sweep_threads, std::max(128, round_warps(bs)));
      }
    }
    if (cc) {
      const int ci = col_index(p, cc), wp = p.ny / cc;
      const int width = ci >= 2 ? 32 : 32 * (cwarps[ci] / wp);  // pairs: one 32-column panel
      seg_tables(p.p1y, p.p2y, cc, wp, &h->hsegy[k]);
      int q = 0;
      for (int i0 = 0; i0 < p.nx; i0 += width, ++q) csts[ci].push_back(Tile{k, i0, std::min(width, p.nx - i0), q});
    } else {
      int q = 0;
      for (int i0 = 0; i0 < p.nx; i0 += bc, ++q) ct.push_back(Tile{k, i0, std::min(bc, p.nx - i0), q});
      if (!stream) sh.cols_panel_cap = std::max(sh.cols_panel_cap, (int)cols_panel_elems(bc, p.ny));
    }
    if (!blk) sh.rows_smem = std::max(sh.rows_smem, rows_smem_bytes(br, p.nx, h->elt, threads));
  }
  // Panel buffers start on 16-byte boundaries (the 16-byte copies need it): round the
  // panel capacity to 4 elements and size the shared memory from the rounded capacity.
  sh.cols_panel_cap = (sh.cols_panel_cap + 3) / 4 * 4;
  if (!stream) sh.cols_smem = (size_t)(persist ? 4 : 2) * sh.cols_panel_cap * h->elt;
  sh.cols_persist = persist ? 1 : 0;
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (!stream && !ct.empty()) {
    const int per_sm = chk::cols_blocks_per_sm(h->precision, sh.cols_persist, threads, sh.cols_smem);
    sh.cols_grid = std::max(1, sms * std::max(1, per_sm));
  }
  if (sh.sweep_threads > 512) return fail(CH_EINVAL, "row-sweep band above 512 rows");
  // segment-form rows: shared memory and persistent grid per class (the largest C tile and
  // mu tile of a class may come from different members)
  sh.seg_persist = seg_persist ? 1 : 0;
  for (int c = 0; c < 2; ++c) {
    sh.rt_seg[c] = (int)rts[c].size();
    if (rts[c].empty()) continue;
    const int nbuf = seg_persist ? 2 : 1;
    sh.seg_smem[c] = seg_smem_bytes(sh.seg_ccap[c], sh.seg_mcap[c], nbuf, h->elt, threads);
    if (sh.seg_smem[c] > kSmemMax) return fail(CH_EINVAL, "segment row tiles of the mixed members exceed shared memory");
    if (seg_persist) {
      const int per_sm = chk::seg_blocks_per_sm(h->precision, c ? 32 : 16, std::min(threads, 256), sh.seg_smem[c]);
      sh.seg_grid[c] = std::max(1, sms * std::max(1, per_sm));
    }
  }
  for (int c = 0; c < 4; ++c) {
    sh.cst_n[c] = (int)csts[c].size();
    sh.colseg_threads[c] = 32 * cwarps[c];
    sh.colseg_smem[c] = (size_t)2 * 2 * 32 * cwarps[c] * h->elt;
  }
  std::vector<Tile> rt, cst, st;
  for (int c = 0; c < 2; ++c) sh.st_seg[c] = (int)sts[c].size();
  for (int c = 0; c < 3; ++c) st.insert(st.end(), sts[c].begin(), sts[c].end());
  for (int nw = 1; nw <= 16; ++nw) {
    sh.rtT_n[nw] = (int)rtT[nw].size();
    rt.insert(rt.end(), rtT[nw].begin(), rtT[nw].end());
  }
  for (int c = 0; c < 3; ++c) rt.insert(rt.end(), rts[c].begin(), rts[c].end());
  sh.rt_blk = (int)rtb.size();
  rt.insert(rt.end(), rtb.begin(), rtb.end());
  for (int c = 0; c < 4; ++c) cst.insert(cst.end(), csts[c].begin(), csts[c].end());
  std::vector<Tile> rest;
  for (int c = 0; c < chk::kResClasses; ++c) {
    sh.res_n[c] = (int)rcl[c].size();
    rest.insert(rest.end(), rcl[c].begin(), rcl[c].end());
  }
  sh.n_row_tiles = (int)rt.size();
  sh.n_sweep_tiles = (int)st.size();
  sh.n_col_tiles = (int)ct.size();
  h->rest.swap(rest);
  h->rt.swap(rt);
  h->st.swap(st);
  h->ct.swap(ct);
  h->cst.swap(cst);
  h->shape = sh;
  h->total_bands = part;
  h->tuning = t;
  return CH_OK;
}

// (Re)allocate the device tile tables and partial slots for the current tiles, upload
// them and the member parameters.  The caller has synchronised the stream.
int upload_tiles(ch_ensemble* h) {
  auto ensure = [&](void** p, size_t& cap, size_t need, size_t elt) -> cudaError_t {
    need = std::max<size_t>(need, 1);
    if (need <= cap) return cudaSuccess;
    cudaFree(*p);
    *p = nullptr;
    cap = 0;
    cudaError_t e = chk::dev_malloc(p, need * elt);
    if (e == cudaSuccess) cap = need;
    return e;
  };
  cudaError_t e;
  if ((e = ensure((void**)&h->drt, h->cap_rt, h->rt.size(), sizeof(Tile))) != cudaSuccess ||
      (e = ensure((void**)&h->dst, h->cap_st, h->st.size(), sizeof(Tile))) != cudaSuccess ||
      (e = ensure((void**)&h->dct, h->cap_ct, h->ct.size(), sizeof(Tile))) != cudaSuccess ||
      (e = ensure((void**)&h->dcst, h->cap_cst, h->cst.size(), sizeof(Tile))) != cudaSuccess ||
      (e = ensure((void**)&h->dres, h->cap_res, h->rest.size(), sizeof(Tile))) != cudaSuccess ||
      (e = ensure((void**)&h->dpart, h->cap_part, (size_t)h->total_bands, sizeof(double2))) != cudaSuccess) {
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? CH_ENOMEM : CH_ECUDA, std::string("tile tables: ") + cudaGetErrorString(e));
  }
  CH_CUDA(cudaMemcpyAsync(h->drt, h->rt.data(), sizeof(Tile) * h->rt.size(), cudaMemcpyHostToDevice, h->stream), "tiles");
  if (!h->st.empty())
    CH_CUDA(cudaMemcpyAsync(h->dst, h->st.data(), sizeof(Tile) * h->st.size(), cudaMemcpyHostToDevice, h->stream), "tiles");
  CH_CUDA(cudaMemcpyAsync(h->dct, h->ct.data(), sizeof(Tile) * h->ct.size(), cudaMemcpyHostToDevice, h->stream), "tiles");
  CH_CUDA(cudaMemsetAsync(h->dpart, 0, sizeof(double2) * std::max<int64_t>(h->total_bands, 1), h->stream), "partials");
  CH_CUDA(cudaMemcpyAsync(h->dmp, h->hp.data(), sizeof(MemberParams) * h->m, cudaMemcpyHostToDevice, h->stream),
          "upload member parameters");
  int n_rowT = 0;
  for (int nw = 1; nw <= 16; ++nw) n_rowT += h->shape.rtT_n[nw];
  if (!h->rest.empty())
    CH_CUDA(cudaMemcpyAsync(h->dres, h->rest.data(), sizeof(Tile) * h->rest.size(), cudaMemcpyHostToDevice, h->stream),
            "tiles");
  if (h->shape.rt_seg[0] + h->shape.rt_seg[1] + h->shape.st_seg[0] + h->shape.st_seg[1] + n_rowT + h->rest.size())
    CH_CUDA(cudaMemcpyAsync(h->dseg, h->hseg.data(), sizeof(chk::SegTable) * h->m, cudaMemcpyHostToDevice, h->stream),
            "upload scan tables");
  if (!h->cst.empty())
    CH_CUDA(cudaMemcpyAsync(h->dcst, h->cst.data(), sizeof(Tile) * h->cst.size(), cudaMemcpyHostToDevice, h->stream),
            "tiles");
  if (!h->cst.empty() || !h->rest.empty()) {
    CH_CUDA(cudaMemcpyAsync(h->dsegy, h->hsegy.data(), sizeof(chk::SegTable) * h->m, cudaMemcpyHostToDevice,
                            h->stream),
            "upload scan tables");
  }
  CH_CUDA(cudaStreamSynchronize(h->stream), "upload tiles");
  return CH_OK;
}

int upload_params(ch_ensemble* h) {
  CH_CUDA(cudaMemcpyAsync(h->dmp, h->hp.data(), sizeof(MemberParams) * h->m, cudaMemcpyHostToDevice, h->stream),
          "upload member parameters");
  return CH_OK;
}

int reset_state(ch_ensemble* h) {
  CH_CUDA(chk::launch_init_fields(h->view(), h->precision, h->max_points, h->stream), "initial fields");
  CH_CUDA(cudaMemcpyAsync(h->dms, h->hs0.data(), sizeof(MemberState) * h->m, cudaMemcpyHostToDevice, h->stream),
          "reset member state");
  if (h->dseries && h->series_cap > 0)
    CH_CUDA(cudaMemsetAsync(h->dseries, 0, sizeof(double) * 4 * h->series_cap * h->m, h->stream), "clear series");
  return CH_OK;
}

int create_common(int m, const ch_member_desc* d, int precision, ch_handle* out) {
  if (!out) return fail(CH_EINVAL, "out is NULL");
  *out = nullptr;
  if (m < 1 || !d) return fail(CH_EINVAL, "need m >= 1 members");
  if (precision != CH_FP64 && precision != CH_FP32) return fail(CH_EINVAL, "precision must be CH_FP64 or CH_FP32");
  for (int k = 0; k < m; ++k) {
    int rc = validate_desc(d[k], k);
    if (rc) return rc;
  }
  ch_ensemble* h = new ch_ensemble();
  h->precision = precision;
  h->m = m;
  h->elt = precision == CH_FP64 ? sizeof(double) : sizeof(float);
  cudaGetDevice(&h->device);
  h->hp.resize(m);
  h->hseg.resize(m);
  h->hsegy.resize(m);
  int64_t off = 0;
  for (int k = 0; k < m; ++k) {
    int rc = fill_params(d[k], precision, &h->hp[k]);
    if (rc) {
      delete h;
      return rc;
    }
    h->hp[k].offset = off;
    const int64_t np = (int64_t)d[k].nx * d[k].ny;
    // keep every member's field 16-byte aligned
    off += (np + 3) & ~(int64_t)3;
    h->max_points = std::max(h->max_points, np);
  }
  h->total_points = off;
  // lo blocks of compensated members follow the fields in C
  for (int k = 0; k < m; ++k)
    if (h->hp[k].comp) {
      h->hp[k].lo_offset = off;
      off += ((int64_t)d[k].nx * d[k].ny + 3) & ~(int64_t)3;
    }
  h->c_points = off;
  int rc = build_tiles(h, default_tuning());
  if (rc) {
    delete h;
    return rc;
  }
  h->hs0.assign(m, MemberState{});
  for (auto& s : h->hs0) s.remaining = chk::kUnbounded;

  cudaError_t e = cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "cudaStreamCreate");
  }
  h->stream = h->own;
  auto alloc = [&](void** p, size_t bytes) -> cudaError_t { return chk::dev_malloc(p, bytes == 0 ? 16 : bytes); };
  if ((e = alloc(&h->C, h->elt * h->c_points)) != cudaSuccess ||
      (e = alloc(&h->W, h->elt * h->total_points)) != cudaSuccess ||
      (e = alloc((void**)&h->dmp, sizeof(MemberParams) * m)) != cudaSuccess ||
      (e = alloc((void**)&h->dms, sizeof(MemberState) * m)) != cudaSuccess ||
      (e = alloc((void**)&h->dseg, sizeof(chk::SegTable) * m)) != cudaSuccess ||
      (e = alloc((void**)&h->dsegy, sizeof(chk::SegTable) * m)) != cudaSuccess ||
      (e = alloc((void**)&h->dobs, sizeof(double) * 3 * m)) != cudaSuccess) {
    free_device(h);
    cudaStreamDestroy(h->own);
    delete h;
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? CH_ENOMEM : CH_ECUDA,
                std::string("device allocation: ") + cudaGetErrorString(e));
  }
  if ((e = chk::set_kernel_smem_limits(precision)) != cudaSuccess ||
      (e = cudaMemsetAsync(h->W, 0, h->elt * h->total_points, h->stream)) != cudaSuccess) {
    int r = cuda_fail(e, "handle set-up");
    ch_destroy(h);
    return r;
  }
  if ((rc = upload_tiles(h)) || (rc = reset_state(h))) {
    ch_destroy(h);
    return rc;
  }
  if ((e = cudaStreamSynchronize(h->stream)) != cudaSuccess) {
    int r = cuda_fail(e, "handle set-up");
    ch_destroy(h);
    return r;
  }
  *out = h;
  return CH_OK;
}

int check_handle(ch_handle h) { return h ? CH_OK : fail(CH_EINVAL, "handle is NULL"); }

int check_member(ch_handle h, int member) {
  if (!h) return fail(CH_EINVAL, "handle is NULL");
  if (member < 0 || member >= h->m) return fail(CH_EINVAL, "member index out of range");
  return CH_OK;
}

// n single steps of the tiled kernels (every member outside the cluster-resident form).
int launch_tiled_direct(ch_ensemble* h, int64_t n) {
  const chk::DevView v = h->view();
  if (h->shape.n_row_tiles == 0) return CH_OK;
  for (int64_t i = 0; i < n; ++i) {
    cudaError_t e = chk::launch_step(v, h->precision, h->shape, h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "step launch");
  }
  return CH_OK;
}

void free_aux(ch_ensemble* h) {
  for (int i = 0; i < ch_ensemble::kAux; ++i) {
    if (h->aux[i]) cudaStreamDestroy(h->aux[i]);
    if (h->aux_done[i]) cudaEventDestroy(h->aux_done[i]);
    h->aux[i] = nullptr;
    h->aux_done[i] = nullptr;
  }
  if (h->fork) cudaEventDestroy(h->fork);
  h->fork = nullptr;
  h->aux_used = 0;
}

// The auxiliary streams and their events, created on first use.
int ensure_aux(ch_ensemble* h) {
  if (h->fork) return CH_OK;
  for (int i = 0; i < ch_ensemble::kAux; ++i) {
    CH_CUDA(cudaStreamCreateWithFlags(&h->aux[i], cudaStreamNonBlocking), "auxiliary stream");
    CH_CUDA(cudaEventCreateWithFlags(&h->aux_done[i], cudaEventDisableTiming), "auxiliary event");
  }
  CH_CUDA(cudaEventCreateWithFlags(&h->fork, cudaEventDisableTiming), "fork event");
  return CH_OK;
}

int fork_resident(ch_ensemble* h, int64_t n) {
  h->aux_used = 0;
  const int nc = chk::resident_classes(h->shape);
  if (nc == 0 || n <= 0) return CH_OK;
  if (nc == 1 && h->shape.n_row_tiles == 0) {  // nothing to overlap with
    CH_CUDA(chk::launch_resident(h->view(), h->precision, h->shape, n, &h->stream, 1), "resident step launch");
    return CH_OK;
  }
  if (int rc = ensure_aux(h)) return rc;
  const int na = std::min(nc, (int)ch_ensemble::kAux);
  CH_CUDA(cudaEventRecord(h->fork, h->stream), "fork");
  for (int i = 0; i < na; ++i) CH_CUDA(cudaStreamWaitEvent(h->aux[i], h->fork, 0), "fork");
  CH_CUDA(chk::launch_resident(h->view(), h->precision, h->shape, n, h->aux, na), "resident step launch");
  for (int i = 0; i < na; ++i) CH_CUDA(cudaEventRecord(h->aux_done[i], h->aux[i]), "join");
  h->aux_used = na;
  return CH_OK;
}

int join_resident(ch_ensemble* h) {
  for (int i = 0; i < h->aux_used; ++i) CH_CUDA(cudaStreamWaitEvent(h->stream, h->aux_done[i], 0), "join");
  h->aux_used = 0;
  return CH_OK;
}

int launch_steps_direct(ch_ensemble* h, int64_t n) {
  if (int rc = fork_resident(h, n)) return rc;
  if (int rc = launch_tiled_direct(h, n)) return rc;
  return join_resident(h);
}

int ensure_graph(ch_ensemble* h) {
  if (h->graph) return CH_OK;
  const int n = kGraphSteps;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "begin graph capture");
  const chk::DevView v = h->view();
  cudaError_t le = cudaSuccess;
  for (int i = 0; i < n && le == cudaSuccess; ++i) le = chk::launch_step(v, h->precision, h->shape, h->stream);
  e = cudaStreamEndCapture(h->stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(le, "step launch during capture");
  }
  if (e != cudaSuccess) return cuda_fail(e, "end graph capture");
  e = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    h->graph = nullptr;
    return cuda_fail(e, "graph instantiate");
  }
  h->graph_steps = n;
  return CH_OK;
}

int copy_out(ch_ensemble* h, void* dst, const void* src, size_t bytes, const char* what) {
  CH_CUDA(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, h->stream), what);
  CH_CUDA(cudaStreamSynchronize(h->stream), what);
  return CH_OK;
}

int read_states(ch_ensemble* h, std::vector<MemberState>& s) {
  s.resize(h->m);
  return copy_out(h, s.data(), h->dms, sizeof(MemberState) * h->m, "read member state");
}

ch_tuning default_tuning() {
  ch_tuning t;
  t.split = -1;
  t.rows_band = t.rows_p = t.sweep_band = t.cols_panel = t.cols_p = t.threads = 0;
  t.stream = -1;
  t.persist = -1;
  t.row_seg = 0;
  t.col_seg = 0;
  t.resident = 0;
  t.resident_rows = 0;
  t.preroll_head = 0;
  return t;
}

}  // namespace chh

using namespace chh;

extern "C" {

int ch_create_ensemble(int nx, int ny, double L, double gamma, double dt, int m, const double* C0, uint64_t seed,
                       int precision, ch_handle* out) {
  if (m < 1 || !C0) return fail(CH_EINVAL, "need m >= 1 and a C0 array");
  std::vector<ch_member_desc> d(m);
  for (int k = 0; k < m; ++k) {
    d[k].nx = nx;
    d[k].ny = ny;
    d[k].L = L;
    d[k].gamma = gamma;
    d[k].dt = dt;
    d[k].C0 = C0[k];
    d[k].seed = seed;
    d[k].counter_base = (uint64_t)k * (uint64_t)nx * (uint64_t)ny;
  }
  return create_common(m, d.data(), precision, out);
}

int ch_create_batch(int m, const ch_member_desc* d, int precision, ch_handle* out) {
  return create_common(m, d, precision, out);
}

void ch_destroy(ch_handle h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_device(h);
  free_aux(h);
  if (h->own) cudaStreamDestroy(h->own);
  delete h;
}

int ch_set_stream(ch_handle h, void* cuda_stream) {
  if (int rc = check_handle(h)) return rc;
  CH_CUDA(cudaStreamSynchronize(h->stream), "synchronise before stream switch");
  drop_graph(h);
  h->stream = cuda_stream ? static_cast<cudaStream_t>(cuda_stream) : h->own;
  h->external_stream = cuda_stream != nullptr;
  return CH_OK;
}

int ch_set_sampling(ch_handle h, int every, double t1, int64_t capacity) {
  if (int rc = check_handle(h)) return rc;
  if (every < 1 || capacity < 0 || !std::isfinite(t1)) return fail(CH_EINVAL, "every >= 1, capacity >= 0, finite t1");
  if (capacity > 0 && (double)capacity * h->m * 4 * sizeof(double) > 64.0 * (1ull << 30))
    return fail(CH_EINVAL, "series capacity too large");
  CH_CUDA(cudaStreamSynchronize(h->stream), "synchronise");
  if (capacity != h->series_cap) {
    cudaFree(h->dseries);
    h->dseries = nullptr;
    h->series_cap = 0;
    if (capacity > 0) {
      cudaError_t e = chk::dev_malloc(&h->dseries, sizeof(double) * 4 * capacity * h->m);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(CH_ENOMEM, "series allocation");
      }
    }
    h->series_cap = capacity;
  }
  h->every = every;
  h->t1 = t1;
  for (auto& p : h->hp) {
    p.every = every;
    p.t1 = t1;
    p.series_cap = capacity;
  }
  if (int rc = upload_params(h)) return rc;
  // clear samples and averages, keep fields and step indices
  std::vector<MemberState> s;
  if (int rc = read_states(h, s)) return rc;
  for (auto& x : s) {
    x.nsamples = 0;
    x.beta_count = 0;
    x.beta_sum = 0.0;
  }
  CH_CUDA(cudaMemcpyAsync(h->dms, s.data(), sizeof(MemberState) * h->m, cudaMemcpyHostToDevice, h->stream),
          "write member state");
  if (h->dseries) CH_CUDA(cudaMemsetAsync(h->dseries, 0, sizeof(double) * 4 * capacity * h->m, h->stream), "clear series");
  drop_graph(h);  // graphs hold the old DevView (series pointer)
  CH_CUDA(cudaStreamSynchronize(h->stream), "synchronise");
  return CH_OK;
}

int ch_step(ch_handle h, int64_t nsteps) {
  if (int rc = check_handle(h)) return rc;
  if (nsteps < 0) return fail(CH_EINVAL, "nsteps must be >= 0");
  // The legacy default stream cannot be captured: launch directly there.
  const bool can_graph = h->stream != nullptr && h->stream != cudaStreamLegacy && h->stream != cudaStreamPerThread;
  CH_CUDA(chk::inject_nan(h->C, h->precision, h->hp.data(), h->m, h->stream), "injected NaN");
  // cluster-resident members on their own streams (launches of many steps each), beside
  // the other members' single steps on the handle's stream, replayed from a captured graph
  // where possible; the handle's stream then waits for both
  if (int rc = fork_resident(h, nsteps)) return rc;
  if (h->shape.n_row_tiles > 0) {
    int64_t left = nsteps;
    if (can_graph && left >= kGraphSteps) {
      if (int rc = ensure_graph(h)) return rc;
      while (left >= h->graph_steps) {
        CH_CUDA(cudaGraphLaunch(h->graph, h->stream), "graph launch");
        left -= h->graph_steps;
      }
    }
    if (int rc = launch_tiled_direct(h, left)) return rc;
  }
  return join_resident(h);
}

int ch_synchronize(ch_handle h) {
  if (int rc = check_handle(h)) return rc;
  CH_CUDA(cudaStreamSynchronize(h->stream), "synchronise");
  return CH_OK;
}

int ch_observables(ch_handle h, double* F, double* dFdt, double* beta) {
  if (int rc = check_handle(h)) return rc;
  CH_CUDA(chk::launch_observe(h->view(), h->precision, h->shape, h->stream), "observe launch");
  std::vector<double> o(3 * (size_t)h->m);
  if (int rc = copy_out(h, o.data(), h->dobs, sizeof(double) * o.size(), "read observables")) return rc;
  bool bad = false;
  for (int k = 0; k < h->m; ++k) {
    if (F) F[k] = o[3 * k];
    if (dFdt) dFdt[k] = o[3 * k + 1];
    if (beta) beta[k] = o[3 * k + 2];
    if (!std::isfinite(o[3 * k]) || !std::isfinite(o[3 * k + 1])) bad = true;
  }
  if (bad) return fail(CH_ENONFINITE, "a member's F or dF/dt is not finite (the run diverged)");
  return CH_OK;
}

int ch_beta_avg(ch_handle h, double* avg, int64_t* count) {
  if (int rc = check_handle(h)) return rc;
  std::vector<MemberState> s;
  if (int rc = read_states(h, s)) return rc;
  for (int k = 0; k < h->m; ++k) {
    if (avg) avg[k] = s[k].beta_count ? s[k].beta_sum / (double)s[k].beta_count : NAN;
    if (count) count[k] = s[k].beta_count;
  }
  return CH_OK;
}

int ch_series(ch_handle h, int member, double* out, int64_t cap, int64_t* n) {
  if (int rc = check_member(h, member)) return rc;
  if (cap < 0 || (cap > 0 && !out)) return fail(CH_EINVAL, "bad output buffer");
  std::vector<MemberState> s;
  if (int rc = read_states(h, s)) return rc;
  const int64_t have = std::min<int64_t>(s[member].nsamples, h->series_cap);
  const int64_t take = std::min<int64_t>(have, cap);
  if (take > 0) {
    std::vector<double> ring(4 * (size_t)h->series_cap);
    if (int rc = copy_out(h, ring.data(), h->dseries + (size_t)member * 4 * h->series_cap,
                          sizeof(double) * ring.size(), "read series"))
      return rc;
    const int64_t first = s[member].nsamples - have;  // oldest kept sample number
    for (int64_t i = 0; i < take; ++i) {
      const int64_t slot = (first + i) % h->series_cap;
      std::memcpy(out + 4 * i, ring.data() + 4 * slot, 4 * sizeof(double));
    }
  }
  if (n) *n = take;
  return CH_OK;
}

}  // extern "C"

namespace chh {
// Member k's field as FP64 values (FP32: hi, plus lo for compensated members).
int read_member_field(ch_ensemble* h, int k, double* out) {
  const MemberParams& p = h->hp[k];
  const int64_t np = (int64_t)p.nx * p.ny;
  if (h->precision == CH_FP64)
    return copy_out(h, out, static_cast<double*>(h->C) + p.offset, sizeof(double) * np, "read field");
  std::vector<float> tmp(np), lo;
  if (int rc = copy_out(h, tmp.data(), static_cast<float*>(h->C) + p.offset, sizeof(float) * np, "read field")) return rc;
  if (p.comp) {
    lo.resize(np);
    if (int rc = copy_out(h, lo.data(), static_cast<float*>(h->C) + p.lo_offset, sizeof(float) * np, "read field"))
      return rc;
  }
  for (int64_t i = 0; i < np; ++i) out[i] = p.comp ? (double)tmp[i] + (double)lo[i] : (double)tmp[i];
  return CH_OK;
}

// Member k's field from FP64 values (FP32: rounded to hi, the remainder to lo for
// compensated members).  Synchronises.
int write_member_field(ch_ensemble* h, int k, const double* in) {
  const MemberParams& p = h->hp[k];
  const int64_t np = (int64_t)p.nx * p.ny;
  if (h->precision == CH_FP64) {
    CH_CUDA(cudaMemcpyAsync(static_cast<double*>(h->C) + p.offset, in, sizeof(double) * np, cudaMemcpyHostToDevice,
                            h->stream),
            "write field");
  } else {
    std::vector<float> hi(np), lo(p.comp ? np : 0);
    for (int64_t i = 0; i < np; ++i) {
      hi[i] = (float)in[i];
      if (p.comp) lo[i] = (float)(in[i] - (double)hi[i]);
    }
    CH_CUDA(cudaMemcpyAsync(static_cast<float*>(h->C) + p.offset, hi.data(), sizeof(float) * np,
                            cudaMemcpyHostToDevice, h->stream),
            "write field");
    if (p.comp)
      CH_CUDA(cudaMemcpyAsync(static_cast<float*>(h->C) + p.lo_offset, lo.data(), sizeof(float) * np,
                              cudaMemcpyHostToDevice, h->stream),
              "write field");
  }
  CH_CUDA(cudaStreamSynchronize(h->stream), "write field");
  return CH_OK;
}
}  // namespace chh

extern "C" {

int ch_get_field(ch_handle h, int member, double* out) {
  if (int rc = check_member(h, member)) return rc;
  if (!out) return fail(CH_EINVAL, "out is NULL");
  return read_member_field(h, member, out);
}

int ch_set_field(ch_handle h, int member, const double* in) {
  if (int rc = check_member(h, member)) return rc;
  if (!in) return fail(CH_EINVAL, "in is NULL");
  const MemberParams& p = h->hp[member];
  const int64_t np = (int64_t)p.nx * p.ny;
  for (int64_t i = 0; i < np; ++i)
    if (!std::isfinite(in[i])) return fail(CH_EINVAL, "field value is not finite");
  return write_member_field(h, member, in);
}

int ch_set_fields(ch_handle h, const double* in) {
  if (int rc = check_handle(h)) return rc;
  if (!in) return fail(CH_EINVAL, "in is NULL");
  int64_t src = 0;
  for (int k = 0; k < h->m; ++k) {
    const MemberParams& p = h->hp[k];
    const int64_t np = (int64_t)p.nx * p.ny;
    if (h->precision == CH_FP64) {
      CH_CUDA(cudaMemcpyAsync(static_cast<double*>(h->C) + p.offset, in + src, sizeof(double) * np,
                              cudaMemcpyHostToDevice, h->stream),
              "write fields");
    } else if (int rc = write_member_field(h, k, in + src)) {
      return rc;
    }
    src += np;
  }
  CH_CUDA(cudaStreamSynchronize(h->stream), "write fields");
  return CH_OK;
}

int ch_get_fields(ch_handle h, double* out) {
  if (int rc = check_handle(h)) return rc;
  if (!out) return fail(CH_EINVAL, "out is NULL");
  int64_t dst = 0;
  for (int k = 0; k < h->m; ++k) {
    const MemberParams& p = h->hp[k];
    const int64_t np = (int64_t)p.nx * p.ny;
    if (h->precision == CH_FP64) {
      CH_CUDA(cudaMemcpyAsync(out + dst, static_cast<double*>(h->C) + p.offset, sizeof(double) * np,
                              cudaMemcpyDeviceToHost, h->stream),
              "read fields");
    } else if (int rc = read_member_field(h, k, out + dst)) {
      return rc;
    }
    dst += np;
  }
  CH_CUDA(cudaStreamSynchronize(h->stream), "read fields");
  return CH_OK;
}

int ch_launch_phase(ch_handle h, int phase) {
  if (int rc = check_handle(h)) return rc;
  if (phase < 0 || phase > 2) return fail(CH_EINVAL, "phase must be 0, 1 or 2");
  CH_CUDA(chk::launch_phase(h->view(), h->precision, phase, h->shape, h->stream), "phase launch");
  return CH_OK;
}

int ch_set_tuning(ch_handle h, const ch_tuning* t) {
  if (int rc = check_handle(h)) return rc;
  const ch_tuning req = t ? *t : default_tuning();
  if (req.rows_band < 0 || req.rows_p < 0 || req.sweep_band < 0 || req.cols_panel < 0 || req.cols_p < 0 ||
      req.threads < 0 || req.split < -1 || req.split > 1 || req.stream < -1 || req.stream > 1 || req.persist < -1 ||
      req.persist > 3)
    return fail(CH_EINVAL, "tuning fields must be >= 0 (split, stream: -1, 0 or 1; persist: -1 .. 3)");
  if (req.row_seg != -1 && req.row_seg != 0 && req.row_seg != 1 && req.row_seg != 16 && req.row_seg != 32)
    return fail(CH_EINVAL, "row_seg must be -1, 0, 1, 16 or 32");
  if (req.col_seg != -1 && req.col_seg != 0 && req.col_seg != 16 && req.col_seg != 32)
    return fail(CH_EINVAL, "col_seg must be -1, 0, 16 or 32");
  if (req.resident < -1 || req.resident > 1) return fail(CH_EINVAL, "resident must be -1, 0 or 1");
  if (req.resident_rows != 0 && req.resident_rows != 32 && req.resident_rows != 64)
    return fail(CH_EINVAL, "resident_rows must be 0, 32 or 64");
  if (req.preroll_head < -1 || req.preroll_head > 0) return fail(CH_EINVAL, "preroll_head must be -1 or 0");
  CH_CUDA(cudaStreamSynchronize(h->stream), "synchronise");
  const std::vector<MemberParams> saved = h->hp;
  const ch_tuning old = h->tuning;
  if (int rc = build_tiles(h, req)) {
    h->hp = saved;
    build_tiles(h, old);
    return rc;
  }
  drop_graph(h);
  return upload_tiles(h);
}

int ch_get_tuning(ch_handle h, ch_tuning* t) {
  if (int rc = check_handle(h)) return rc;
  if (!t) return fail(CH_EINVAL, "t is NULL");
  // the shape in effect, with per-member values of member 0
  t->split = h->shape.split;
  t->rows_band = h->rt.empty() ? 0 : h->rt[0].count;
  t->rows_p = h->hp[0].rows_p;
  t->sweep_band = h->st.empty() ? 0 : h->st[0].count;
  t->cols_panel = h->ct.empty() ? 0 : h->ct[0].count;
  t->cols_p = h->hp[0].cols_p;
  t->threads = h->shape.rows_threads;
  t->stream = h->shape.stream;
  t->persist = h->shape.cols_persist | (h->shape.seg_persist << 1);
  // kernel classes of member 0
  t->row_seg = h->hp[0].row_t ? 1 : (h->hp[0].seg_g ? h->hp[0].nx / h->hp[0].seg_g : (h->shape.split ? 0 : -1));
  t->col_seg = h->hp[0].col_s ? h->hp[0].col_s : -1;
  t->resident = h->rest.empty() ? -1 : 1;
  t->resident_rows = 0;
  t->preroll_head = h->tuning.preroll_head < 0 ? -1 : 0;
  for (const Tile& r : h->rest)
    if (r.member == 0) {  // member 0 runs in the resident form
      t->row_seg = t->col_seg = 0;
      t->resident_rows = h->hp[0].nbands > 0 ? h->hp[0].ny / h->hp[0].nbands : 32;
    }
  return CH_OK;
}

int ch_get_step(ch_handle h, int member, int64_t* n) {
  if (int rc = check_member(h, member)) return rc;
  if (!n) return fail(CH_EINVAL, "n is NULL");
  MemberState s;
  if (int rc = copy_out(h, &s, h->dms + member, sizeof s, "read step")) return rc;
  *n = s.step;
  return CH_OK;
}

int ch_reset(ch_handle h) {
  if (int rc = check_handle(h)) return rc;
  if (int rc = reset_state(h)) return rc;
  CH_CUDA(cudaStreamSynchronize(h->stream), "reset");
  return CH_OK;
}

int ch_num_members(ch_handle h, int* m) {
  if (int rc = check_handle(h)) return rc;
  if (m) *m = h->m;
  return CH_OK;
}

int ch_member_shape(ch_handle h, int member, int* nx, int* ny) {
  if (int rc = check_member(h, member)) return rc;
  if (nx) *nx = h->hp[member].nx;
  if (ny) *ny = h->hp[member].ny;
  return CH_OK;
}

int ch_debug_row_solve(ch_handle h, int member, double* out) {
  if (int rc = check_member(h, member)) return rc;
  if (!out) return fail(CH_EINVAL, "out is NULL");
  for (const Tile& r : h->rest)
    if (r.member == member)
      return fail(CH_EINVAL, "member runs in the cluster-resident form: its row solve has no phase of its own "
                             "(set_tuning resident = -1 to use the tiled kernels)");
  // phases 0 and 1 only touch W, the band partials and the members' active flags
  CH_CUDA(chk::launch_phase(h->view(), h->precision, 0, h->shape, h->stream), "row phase");
  CH_CUDA(chk::launch_phase(h->view(), h->precision, 1, h->shape, h->stream), "row phase");
  const MemberParams& p = h->hp[member];
  const int64_t np = (int64_t)p.nx * p.ny;
  const double scale = p.dt / (p.hx * p.hx * p.cx);
  if (h->precision == CH_FP64) {
    if (int rc = copy_out(h, out, static_cast<double*>(h->W) + p.offset, sizeof(double) * np, "read W")) return rc;
    for (int64_t i = 0; i < np; ++i) out[i] *= scale;
    return CH_OK;
  }
  std::vector<float> tmp(np);
  if (int rc = copy_out(h, tmp.data(), static_cast<float*>(h->W) + p.offset, sizeof(float) * np, "read W")) return rc;
  for (int64_t i = 0; i < np; ++i) out[i] = (double)tmp[i] * scale;
  return CH_OK;
}

// Checkpoint file: "CHCKPT01", int32 precision, int32 m, m x (int32 nx, int32 ny),
// int64 series_cap, fields (elt * c_points bytes: the fields, then the lo blocks of
// compensated FP32 members), MemberState[m], series ring.
int ch_save(ch_handle h, const char* path) {
  if (int rc = check_handle(h)) return rc;
  if (!path) return fail(CH_EINVAL, "path is NULL");
  std::vector<unsigned char> fields(h->elt * h->c_points);
  if (int rc = copy_out(h, fields.data(), h->C, fields.size(), "read fields")) return rc;
  std::vector<MemberState> s;
  if (int rc = read_states(h, s)) return rc;
  std::vector<double> series(4 * (size_t)h->series_cap * h->m);
  if (!series.empty())
    if (int rc = copy_out(h, series.data(), h->dseries, sizeof(double) * series.size(), "read series")) return rc;
  FILE* f = fopen(path, "wb");
  if (!f) return fail(CH_EINVAL, std::string("cannot open ") + path);
  bool ok = fwrite("CHCKPT01", 1, 8, f) == 8;
  int32_t hdr[2] = {h->precision, h->m};
  ok = ok && fwrite(hdr, sizeof hdr, 1, f) == 1;
  for (int k = 0; k < h->m && ok; ++k) {
    int32_t sh[2] = {h->hp[k].nx, h->hp[k].ny};
    ok = fwrite(sh, sizeof sh, 1, f) == 1;
  }
  int64_t cap = h->series_cap;
  ok = ok && fwrite(&cap, sizeof cap, 1, f) == 1;
  ok = ok && fwrite(fields.data(), 1, fields.size(), f) == fields.size();
  ok = ok && fwrite(s.data(), sizeof(MemberState), s.size(), f) == s.size();
  if (!series.empty()) ok = ok && fwrite(series.data(), sizeof(double), series.size(), f) == series.size();
  ok = (fclose(f) == 0) && ok;
  return ok ? CH_OK : fail(CH_EINVAL, std::string("write failed: ") + path);
}

int ch_load(ch_handle h, const char* path) {
  if (int rc = check_handle(h)) return rc;
  if (!path) return fail(CH_EINVAL, "path is NULL");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(CH_EINVAL, std::string("cannot open ") + path);
  char magic[8];
  int32_t hdr[2];
  bool ok = fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "CHCKPT01", 8) == 0;
  ok = ok && fread(hdr, sizeof hdr, 1, f) == 1 && hdr[0] == h->precision && hdr[1] == h->m;
  for (int k = 0; k < h->m && ok; ++k) {
    int32_t sh[2];
    ok = fread(sh, sizeof sh, 1, f) == 1 && sh[0] == h->hp[k].nx && sh[1] == h->hp[k].ny;
  }
  int64_t cap = -1;
  ok = ok && fread(&cap, sizeof cap, 1, f) == 1 && cap == h->series_cap;
  std::vector<unsigned char> fields(h->elt * h->c_points);
  std::vector<MemberState> s(h->m);
  std::vector<double> series(4 * (size_t)h->series_cap * h->m);
  ok = ok && fread(fields.data(), 1, fields.size(), f) == fields.size();
  ok = ok && fread(s.data(), sizeof(MemberState), s.size(), f) == s.size();
  if (!series.empty()) ok = ok && fread(series.data(), sizeof(double), series.size(), f) == series.size();
  fclose(f);
  if (!ok) return fail(CH_EINVAL, "checkpoint does not match this handle (members, precision or sampling)");
  CH_CUDA(cudaMemcpyAsync(h->C, fields.data(), fields.size(), cudaMemcpyHostToDevice, h->stream), "write fields");
  CH_CUDA(cudaMemcpyAsync(h->dms, s.data(), sizeof(MemberState) * s.size(), cudaMemcpyHostToDevice, h->stream),
          "write state");
  if (!series.empty())
    CH_CUDA(cudaMemcpyAsync(h->dseries, series.data(), sizeof(double) * series.size(), cudaMemcpyHostToDevice, h->stream),
            "write series");
  CH_CUDA(cudaStreamSynchronize(h->stream), "load");
  return CH_OK;
}

int ch_penta_factor(double s, int precision, double* c, double* p1, double* p2, int* K) {
  if (!finite_pos(s)) return fail(CH_EINVAL, "s must be finite and > 0");
  if (precision != CH_FP64 && precision != CH_FP32) return fail(CH_EINVAL, "bad precision");
  double cc, q1, q2;
  if (!spectral_factor(s, &cc, &q1, &q2)) return fail(CH_EINVAL, "factorisation did not converge");
  const int k = preroll_length(q1, q2, precision == CH_FP64 ? kPrerollTol64 : 1e-8);
  if (k < 0) return fail(CH_EINVAL, "decay too slow");
  if (c) *c = cc;
  if (p1) *p1 = q1;
  if (p2) *p2 = q2;
  if (K) *K = k;
  return CH_OK;
}

int ch_preroll_head(double s, int* K, int* head) {
  if (!finite_pos(s)) return fail(CH_EINVAL, "s must be finite and > 0");
  double cc, q1, q2;
  if (!spectral_factor(s, &cc, &q1, &q2)) return fail(CH_EINVAL, "factorisation did not converge");
  const int k = preroll_length(q1, q2, kPrerollTol64);
  if (k < 0) return fail(CH_EINVAL, "decay too slow");
  if (K) *K = k;
  if (head) *head = preroll_head_length(q1, q2, k, kPrerollTol64);
  return CH_OK;
}

int ch_seg_tables(double s, int seg, int groups, double* out) {
  if (!finite_pos(s)) return fail(CH_EINVAL, "s must be finite and > 0");
  if (seg < 1 || !is_pow2_upto32(groups)) return fail(CH_EINVAL, "seg >= 1 and groups a power of two in [1, 32]");
  if (!out) return fail(CH_EINVAL, "out is NULL");
  double cc, q1, q2;
  if (!spectral_factor(s, &cc, &q1, &q2)) return fail(CH_EINVAL, "factorisation did not converge");
  chk::SegTable t;
  seg_tables(q1, q2, seg, groups, &t);
  std::memcpy(out, &t.A[0][0], sizeof t.A);
  std::memcpy(out + 20, &t.B[0][0], 32 * 4 * sizeof(double));  // groups <= 32
  std::memcpy(out + 148, t.P, sizeof t.P);
  return CH_OK;
}

const char* ch_last_error(void) { return g_last_error.c_str(); }

const char* ch_version(void) { return "ch 0.1 sm_103a"; }

}  // extern "C"
