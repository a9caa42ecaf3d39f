// ch_stats.cu -- ensemble statistics of sampled beta series on the device.
//
// The paper's ensemble analysis (Sec. 3.3 Eqs. (41a,b) and (42), applied to the
// Cahn-Hilliard ensembles in Secs. 4.2-4.3, Tables 4-5) works on the coarsening rate
// beta_j(t) of M runs sampled at common times:
//   - moments across the runs per sample time: mu_1 = mean, mu_p = mean of (beta - mu_1)^p;
//   - the empirical distribution p_beta(b, t) of Sec. 1 Eq. (7), as a histogram per time;
//   - the window estimate of beta_0 (time mean of mu_1 over [t1, t2], Eq. (42)) and the
//     slope k of the least-squares line mu_2 = k t through the origin.
// Values that are not finite (a run that diverged) are left out of a sample's statistics.
//
// Layout.  A series set is read through a strided view: run j's sample s lives at
//   base[off_j + slot(s) * sstride + component],  slot(s) = (first + s) mod ring,
// which covers both a dense beta[M][ld] array (sstride 1, ring = T) and the handle's
// series rings (records of 4 doubles t, F, dF/dt, beta; ring = the sampling capacity).
//
// Kernels.  A CTA owns 32 consecutive sample times (one per lane) and its 8 warps split
// the runs, so for a fixed run a warp reads 32 consecutive samples (one coalesced row of a
// dense array; one 32-byte record each in a series ring, which also holds t, so the
// sampling-time check costs no extra DRAM sector).  The moments take two passes over the
// runs (mean, then central sums), both in FP64; the second pass re-reads from L2.  The
// histogram counts in shared memory with atomics and writes each time's row once.  The
// trend statistics are one CTA over the moments table.
//
// Also here: the grid-refinement error E_n of Appendix A (the mean L1 distance between a
// field restricted by 2 x 2 block means and the same run on the grid of half the points
// per axis), one CTA per coarse row and a second CTA over the row values.
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "ch.h"
#include "ch_handle.h"

namespace chs {

constexpr int kLanes = 32;    // sample times per CTA
constexpr int kWarps = 8;     // warps splitting the runs
constexpr int kThreads = kLanes * kWarps;
constexpr int kPad = kLanes + 1;  // shared histogram row stride (bank-conflict free both ways)

struct View {
  const double* base;
  const int64_t* moff;  // [M] element offset of run j (nullptr: j * mstride)
  int64_t mstride;
  int64_t sstride;      // elements between consecutive slots
  int64_t ring;         // slots (sample s is in slot (first + s) mod ring)
  int64_t first;
  int bc;               // component of beta within a slot
  int tc;               // component of t within a slot, < 0: t from tv[s]
  const double* tv;
  int64_t M, T;
};

__device__ __forceinline__ int64_t slot_offset(const View& v, int64_t s) {
  int64_t q = v.first + s;
  if (q >= v.ring) q %= v.ring;
  return q * v.sstride;
}

__device__ __forceinline__ int64_t run_offset(const View& v, int64_t j) {
  return v.moff ? v.moff[j] : j * v.mstride;
}

// Row s of out (6 doubles): t, count, mu_1 .. mu_4.  *mismatch |= 1 when a run's t differs
// from run 0's at the same sample (series views only).
__global__ void __launch_bounds__(kThreads) moments_kernel(View v, double* __restrict__ out,
                                                           int* __restrict__ mismatch) {
  __shared__ double rs[4][kWarps][kLanes];
  __shared__ int64_t rc[kWarps][kLanes];
  __shared__ double mean_s[kLanes];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t s = (int64_t)blockIdx.x * kLanes + lane;
  const bool on = s < v.T;
  const int64_t so = on ? slot_offset(v, s) : 0;
  double t0 = 0.0;
  if (on) t0 = v.tc < 0 ? v.tv[s] : v.base[run_offset(v, 0) + so + v.tc];

  double sum = 0.0;
  int64_t cnt = 0;
  int bad = 0;
  if (on) {
    for (int64_t j = w; j < v.M; j += kWarps) {
      const int64_t o = run_offset(v, j) + so;
      const double b = v.base[o + v.bc];
      if (v.tc >= 0 && v.base[o + v.tc] != t0) bad = 1;
      if (isfinite(b)) {
        sum += b;
        ++cnt;
      }
    }
  }
  if (bad && mismatch) atomicOr(mismatch, 1);
  rs[0][w][lane] = sum;
  rc[w][lane] = cnt;
  __syncthreads();
  if (w == 0) {
    double a = 0.0;
    int64_t c = 0;
    for (int k = 0; k < kWarps; ++k) {
      a += rs[0][k][lane];
      c += rc[k][lane];
    }
    mean_s[lane] = c > 0 ? a / (double)c : __longlong_as_double(0x7ff8000000000000LL);
    rc[0][lane] = c;
  }
  __syncthreads();
  const double mu1 = mean_s[lane];
  double c2 = 0.0, c3 = 0.0, c4 = 0.0;
  if (on) {
    for (int64_t j = w; j < v.M; j += kWarps) {
      const double b = v.base[run_offset(v, j) + so + v.bc];
      if (isfinite(b)) {
        const double d = b - mu1;
        const double d2 = d * d;
        c2 += d2;
        c3 += d2 * d;
        c4 += d2 * d2;
      }
    }
  }
  rs[1][w][lane] = c2;
  rs[2][w][lane] = c3;
  rs[3][w][lane] = c4;
  __syncthreads();
  if (w == 0 && on) {
    double a2 = 0.0, a3 = 0.0, a4 = 0.0;
    for (int k = 0; k < kWarps; ++k) {
      a2 += rs[1][k][lane];
      a3 += rs[2][k][lane];
      a4 += rs[3][k][lane];
    }
    const int64_t c = rc[0][lane];
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    double* o = out + s * CH_MOMENTS;
    o[0] = t0;
    o[1] = (double)c;
    o[2] = mu1;
    o[3] = c > 0 ? a2 / (double)c : nan;
    o[4] = c > 0 ? a3 / (double)c : nan;
    o[5] = c > 0 ? a4 / (double)c : nan;
  }
}

// Row s of out (nbins + 2 counts): below lo, the bins, at or above the end of the last bin.
__global__ void __launch_bounds__(kThreads) histogram_kernel(View v, double lo, double w, int nbins,
                                                             int64_t* __restrict__ out) {
  extern __shared__ int hist[];  // [nbins + 2][kPad]
  const int nb2 = nbins + 2;
  for (int i = threadIdx.x; i < nb2 * kPad; i += kThreads) hist[i] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const int64_t s = (int64_t)blockIdx.x * kLanes + lane;
  if (s < v.T) {
    const int64_t so = slot_offset(v, s);
    for (int64_t j = wp; j < v.M; j += kWarps) {
      const double b = v.base[run_offset(v, j) + so + v.bc];
      if (!isfinite(b)) continue;
      int bin;
      if (b < lo) {
        bin = 0;
      } else {
        const double k = floor((b - lo) / w);
        bin = k < (double)nbins ? (int)k + 1 : nbins + 1;
      }
      atomicAdd(&hist[bin * kPad + lane], 1);
    }
  }
  __syncthreads();
  // time-major output: consecutive threads write consecutive bins of one sample time
  const int64_t s0 = (int64_t)blockIdx.x * kLanes;
  for (int i = threadIdx.x; i < nb2 * kLanes; i += kThreads) {
    const int l = i / nb2, bin = i - l * nb2;
    if (s0 + l < v.T) out[(s0 + l) * nb2 + bin] = hist[bin * kPad + l];
  }
}

// out[0] window mean of mu_1 (trapezoid over consecutive samples in [t1, t2], divided by the
// span of those samples), out[1] k = sum t mu_2 / sum t^2 over [tf1, tf2], out[2..3] counts.
__global__ void __launch_bounds__(kThreads) trend_kernel(const double* __restrict__ mom, int64_t T, double t1,
                                                         double t2, double tf1, double tf2,
                                                         double* __restrict__ out) {
  __shared__ double rd[3][kThreads];
  __shared__ int64_t ri[4][kThreads];
  double integral = 0.0, stm = 0.0, stt = 0.0;
  int64_t nw = 0, nf = 0, smin = INT64_MAX, smax = -1;
  for (int64_t s = threadIdx.x; s < T; s += kThreads) {
    const double* r = mom + s * CH_MOMENTS;
    const double t = r[0];
    if (t >= t1 && t <= t2) {
      ++nw;
      smin = s < smin ? s : smin;
      smax = s > smax ? s : smax;
      if (s + 1 < T) {
        const double tn = r[CH_MOMENTS];
        if (tn >= t1 && tn <= t2) integral += 0.5 * (tn - t) * (r[2] + r[CH_MOMENTS + 2]);
      }
    }
    if (t >= tf1 && t <= tf2) {
      stm += t * r[3];
      stt += t * t;
      ++nf;
    }
  }
  const int i = threadIdx.x;
  rd[0][i] = integral;
  rd[1][i] = stm;
  rd[2][i] = stt;
  ri[0][i] = nw;
  ri[1][i] = nf;
  ri[2][i] = smin;
  ri[3][i] = smax;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (i < h) {
      rd[0][i] += rd[0][i + h];
      rd[1][i] += rd[1][i + h];
      rd[2][i] += rd[2][i + h];
      ri[0][i] += ri[0][i + h];
      ri[1][i] += ri[1][i + h];
      ri[2][i] = ri[2][i + h] < ri[2][i] ? ri[2][i + h] : ri[2][i];
      ri[3][i] = ri[3][i + h] > ri[3][i] ? ri[3][i + h] : ri[3][i];
    }
    __syncthreads();
  }
  if (i == 0) {
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    const int64_t n_w = ri[0][0];
    out[0] = n_w >= 2 ? rd[0][0] / (mom[ri[3][0] * CH_MOMENTS] - mom[ri[2][0] * CH_MOMENTS]) : nan;
    out[1] = rd[2][0] > 0.0 ? rd[1][0] / rd[2][0] : nan;
    out[2] = (double)n_w;
    out[3] = (double)ri[1][0];
  }
}

// row[j] = mean over coarse row j of |1/4 (f(2i,2j) + f(2i+1,2j) + f(2i,2j+1) + f(2i+1,2j+1)) - c(i,j)|.
__global__ void __launch_bounds__(kThreads) refine_rows_kernel(const double* __restrict__ fine,
                                                               const double* __restrict__ coarse, int nx,
                                                               double* __restrict__ row) {
  __shared__ double red[kThreads];
  const int j = blockIdx.x, mx = nx / 2;
  const double* f0 = fine + (size_t)(2 * j) * nx;
  const double* f1 = f0 + nx;
  const double* c = coarse + (size_t)j * mx;
  double sum = 0.0;
  for (int i = threadIdx.x; i < mx; i += kThreads) {
    const double r = 0.25 * (f0[2 * i] + f0[2 * i + 1] + f1[2 * i] + f1[2 * i + 1]);
    sum += fabs(r - c[i]);
  }
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) row[j] = red[0] / (double)mx;
}

// out[0] = mean of row[0 .. my).
__global__ void __launch_bounds__(kThreads) refine_total_kernel(const double* __restrict__ row, int my,
                                                                double* __restrict__ out) {
  __shared__ double red[kThreads];
  double sum = 0.0;
  for (int j = threadIdx.x; j < my; j += kThreads) sum += row[j];
  red[threadIdx.x] = sum;
  __syncthreads();
  for (int h = kThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = red[0] / (double)my;
}

// out: 1 + ny/2 doubles (E, then the row means).
cudaError_t launch_refinement(const double* fine, const double* coarse, int nx, int ny, double* out,
                              cudaStream_t st) {
  refine_rows_kernel<<<ny / 2, kThreads, 0, st>>>(fine, coarse, nx, out + 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  refine_total_kernel<<<1, kThreads, 0, st>>>(out + 1, ny / 2, out);
  return cudaGetLastError();
}

bool refine_sizes_ok(int nx, int ny) { return nx >= 2 && ny >= 2 && nx % 2 == 0 && ny % 2 == 0; }

size_t histogram_smem(int nbins) { return sizeof(int) * (size_t)(nbins + 2) * kPad; }

cudaError_t launch_moments(const View& v, double* out, int* mismatch, cudaStream_t st) {
  if (v.T <= 0) return cudaSuccess;
  moments_kernel<<<(unsigned)((v.T + kLanes - 1) / kLanes), kThreads, 0, st>>>(v, out, mismatch);
  return cudaGetLastError();
}

cudaError_t launch_histogram(const View& v, double lo, double hi, int nbins, int64_t* out, cudaStream_t st) {
  if (v.T <= 0) return cudaSuccess;
  const size_t smem = histogram_smem(nbins);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(histogram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const double w = (hi - lo) / (double)nbins;
  histogram_kernel<<<(unsigned)((v.T + kLanes - 1) / kLanes), kThreads, smem, st>>>(v, lo, w, nbins, out);
  return cudaGetLastError();
}

cudaError_t launch_trend(const double* mom, int64_t T, double t1, double t2, double tf1, double tf2, double* out,
                         cudaStream_t st) {
  trend_kernel<<<1, kThreads, 0, st>>>(mom, T, t1, t2, tf1, tf2, out);
  return cudaGetLastError();
}

View dense_view(const double* t, const double* beta, int64_t M, int64_t T, int64_t ld) {
  View v{};
  v.base = beta;
  v.moff = nullptr;
  v.mstride = ld;
  v.sstride = 1;
  v.ring = T > 0 ? T : 1;
  v.first = 0;
  v.bc = 0;
  v.tc = -1;
  v.tv = t;
  v.M = M;
  v.T = T;
  return v;
}

bool dense_args_ok(const double* beta, int64_t M, int64_t T, int64_t ld) {
  return M >= 1 && T >= 0 && ld >= T && (T == 0 || beta);
}

bool bins_ok(double lo, double hi, int nbins) {
  return std::isfinite(lo) && std::isfinite(hi) && lo < hi && nbins >= 1 && nbins <= CH_MAX_BINS;
}

// Device scratch of one handle-level statistics call (freed on scope exit).
struct Scratch {
  std::vector<void*> p;
  ~Scratch() {
    for (void* q : p) cudaFree(q);
  }
  template <class T>
  cudaError_t get(T** out, size_t count) {
    void* q = nullptr;
    cudaError_t e = chk::dev_malloc(&q, sizeof(T) * (count > 0 ? count : 1));
    if (e != cudaSuccess) {
      cudaGetLastError();
      return e;
    }
    p.push_back(q);
    *out = static_cast<T*>(q);
    return cudaSuccess;
  }
};

// View of the sampled series of the selected runs over the samples all of them hold.
int series_view(ch_ensemble* h, const int* members, int count, Scratch& sc, View* v) {
  if (int rc = chh::check_handle(h)) return rc;
  std::vector<int> list;
  if (!members) {
    for (int k = 0; k < h->m; ++k)
      if (h->has(k)) list.push_back(k);
  } else {
    if (count < 1) return chh::fail(CH_EINVAL, "count >= 1 members");
    for (int i = 0; i < count; ++i) {
      const int k = members[i];
      if (k < 0 || k >= h->m || !h->has(k)) return chh::fail(CH_EINVAL, "member index out of range");
      list.push_back(k);
    }
  }
  if (list.empty()) return chh::fail(CH_EINVAL, "no members");
  if (h->series_cap <= 0 || !h->dseries)
    return chh::fail(CH_EINVAL, "no series kept (ch_set_sampling with capacity > 0)");
  for (int k : list)
    if (h->hp[k].dt != h->hp[list[0]].dt || h->hp[k].every != h->hp[list[0]].every)
      return chh::fail(CH_EINVAL, "members are sampled at different times (dt or sampling period differ)");
  std::vector<MemberState> s;
  if (int rc = chh::read_states(h, s)) return rc;
  int64_t hi = INT64_MAX, first = 0;
  for (int k : list) {
    const int64_t ns = s[k].nsamples;
    hi = ns < hi ? ns : hi;
    const int64_t kept = ns < h->series_cap ? ns : h->series_cap;
    first = ns - kept > first ? ns - kept : first;
  }
  const int64_t T = hi > first ? hi - first : 0;
  std::vector<int64_t> off(list.size());
  for (size_t j = 0; j < list.size(); ++j) off[j] = (int64_t)list[j] * 4 * h->series_cap;
  int64_t* doff = nullptr;
  if (cudaError_t e = sc.get(&doff, off.size())) return chh::cuda_fail(e, "statistics scratch");
  CH_CHECK_CUDA(cudaMemcpyAsync(doff, off.data(), sizeof(int64_t) * off.size(), cudaMemcpyHostToDevice, h->stream),
                "statistics offsets");
  View w{};
  w.base = h->dseries;
  w.moff = doff;
  w.mstride = 0;
  w.sstride = 4;
  w.ring = h->series_cap;
  w.first = first;
  w.bc = 3;
  w.tc = 0;
  w.tv = nullptr;
  w.M = (int64_t)list.size();
  w.T = T;
  *v = w;
  return CH_OK;
}

// Moments of the selected runs into a device table (and the sampling-time check).
int series_moments(ch_ensemble* h, const View& v, Scratch& sc, double** dmom) {
  int* dflag = nullptr;
  if (cudaError_t e = sc.get(dmom, (size_t)v.T * CH_MOMENTS)) return chh::cuda_fail(e, "statistics scratch");
  if (cudaError_t e = sc.get(&dflag, 1)) return chh::cuda_fail(e, "statistics scratch");
  CH_CHECK_CUDA(cudaMemsetAsync(dflag, 0, sizeof(int), h->stream), "statistics flag");
  CH_CHECK_CUDA(launch_moments(v, *dmom, dflag, h->stream), "moments kernel");
  int flag = 0;
  if (int rc = chh::copy_out(h, &flag, dflag, sizeof(int), "statistics flag")) return rc;
  if (flag) return chh::fail(CH_EINVAL, "members were sampled at different times");
  return CH_OK;
}

}  // namespace chs

extern "C" {

int ch_stats_moments(const double* t, const double* beta, int64_t members, int64_t samples, int64_t ld,
                     double* out, void* stream) {
  if (!chs::dense_args_ok(beta, members, samples, ld) || (samples > 0 && (!t || !out)))
    return chh::fail(CH_EINVAL, "members >= 1, samples >= 0, ld >= samples, non-NULL arrays");
  const chs::View v = chs::dense_view(t, beta, members, samples, ld);
  CH_CHECK_CUDA(chs::launch_moments(v, out, nullptr, static_cast<cudaStream_t>(stream)), "moments kernel");
  return CH_OK;
}

int ch_stats_histogram(const double* beta, int64_t members, int64_t samples, int64_t ld, double lo, double hi,
                       int nbins, int64_t* out, void* stream) {
  if (!chs::dense_args_ok(beta, members, samples, ld) || (samples > 0 && !out))
    return chh::fail(CH_EINVAL, "members >= 1, samples >= 0, ld >= samples, non-NULL arrays");
  if (!chs::bins_ok(lo, hi, nbins)) return chh::fail(CH_EINVAL, "finite lo < hi, 1 <= nbins <= CH_MAX_BINS");
  const chs::View v = chs::dense_view(nullptr, beta, members, samples, ld);
  CH_CHECK_CUDA(chs::launch_histogram(v, lo, hi, nbins, out, static_cast<cudaStream_t>(stream)), "histogram kernel");
  return CH_OK;
}

int ch_stats_trend(const double* moments, int64_t samples, double t1, double t2, double tf1, double tf2,
                   double* out, void* stream) {
  if (samples < 0 || (samples > 0 && !moments) || !out) return chh::fail(CH_EINVAL, "samples >= 0, non-NULL arrays");
  CH_CHECK_CUDA(chs::launch_trend(moments, samples, t1, t2, tf1, tf2, out, static_cast<cudaStream_t>(stream)),
                "trend kernel");
  return CH_OK;
}

int ch_ensemble_moments(ch_handle h, const int* members, int count, double* out, int64_t cap, int64_t* n) {
  if (cap < 0 || (cap > 0 && !out)) return chh::fail(CH_EINVAL, "bad output buffer");
  chs::Scratch sc;
  chs::View v;
  if (int rc = chs::series_view(h, members, count, sc, &v)) return rc;
  double* dmom = nullptr;
  if (int rc = chs::series_moments(h, v, sc, &dmom)) return rc;
  const int64_t take = v.T < cap ? v.T : cap;
  if (take > 0)
    if (int rc = chh::copy_out(h, out, dmom, sizeof(double) * CH_MOMENTS * take, "read moments")) return rc;
  if (n) *n = take;
  return CH_OK;
}

int ch_ensemble_histogram(ch_handle h, const int* members, int count, double lo, double hi, int nbins,
                          int64_t* out, int64_t cap, int64_t* n) {
  if (cap < 0 || (cap > 0 && !out)) return chh::fail(CH_EINVAL, "bad output buffer");
  if (!chs::bins_ok(lo, hi, nbins)) return chh::fail(CH_EINVAL, "finite lo < hi, 1 <= nbins <= CH_MAX_BINS");
  chs::Scratch sc;
  chs::View v;
  if (int rc = chs::series_view(h, members, count, sc, &v)) return rc;
  double* dmom = nullptr;
  if (int rc = chs::series_moments(h, v, sc, &dmom)) return rc;  // checks the sampling times
  const int64_t take = v.T < cap ? v.T : cap;
  if (take > 0) {
    v.T = take;
    int64_t* dh = nullptr;
    if (cudaError_t e = sc.get(&dh, (size_t)take * (nbins + 2))) return chh::cuda_fail(e, "statistics scratch");
    CH_CHECK_CUDA(chs::launch_histogram(v, lo, hi, nbins, dh, h->stream), "histogram kernel");
    if (int rc = chh::copy_out(h, out, dh, sizeof(int64_t) * (size_t)take * (nbins + 2), "read histogram"))
      return rc;
  }
  if (n) *n = take;
  return CH_OK;
}

int ch_refinement_error(const double* fine, const double* coarse, int nx, int ny, double* out, void* stream) {
  if (!chs::refine_sizes_ok(nx, ny) || !fine || !coarse || !out)
    return chh::fail(CH_EINVAL, "nx, ny even and >= 2, non-NULL arrays");
  CH_CHECK_CUDA(chs::launch_refinement(fine, coarse, nx, ny, out, static_cast<cudaStream_t>(stream)),
                "refinement kernels");
  return CH_OK;
}

int ch_ensemble_refinement_error(ch_handle fine, int fine_member, ch_handle coarse, int coarse_member,
                                 double* out) {
  if (int rc = chh::check_handle(fine)) return rc;
  if (int rc = chh::check_handle(coarse)) return rc;
  if (!out) return chh::fail(CH_EINVAL, "out is NULL");
  if (fine_member < 0 || fine_member >= fine->m || !fine->has(fine_member) || coarse_member < 0 ||
      coarse_member >= coarse->m || !coarse->has(coarse_member))
    return chh::fail(CH_EINVAL, "member index out of range");
  if (fine->precision != CH_FP64 || coarse->precision != CH_FP64)
    return chh::fail(CH_EINVAL, "the refinement error compares FP64 fields");
  const MemberParams& pf = fine->hp[fine_member];
  const MemberParams& pc = coarse->hp[coarse_member];
  if (!chs::refine_sizes_ok(pf.nx, pf.ny) || pc.nx * 2 != pf.nx || pc.ny * 2 != pf.ny)
    return chh::fail(CH_EINVAL, "the coarse member must have half the points of the fine member per axis");
  CH_CHECK_CUDA(cudaStreamSynchronize(coarse->stream), "synchronise the coarse handle");
  chs::Scratch sc;
  double* dout = nullptr;
  if (cudaError_t e = sc.get(&dout, 1 + (size_t)pf.ny / 2)) return chh::cuda_fail(e, "refinement scratch");
  const double* f = static_cast<const double*>(fine->C) + pf.offset;
  const double* c = static_cast<const double*>(coarse->C) + pc.offset;
  CH_CHECK_CUDA(chs::launch_refinement(f, c, pf.nx, pf.ny, dout, fine->stream), "refinement kernels");
  return chh::copy_out(fine, out, dout, sizeof(double), "read refinement error");
}

int ch_ensemble_trend(ch_handle h, const int* members, int count, double t1, double t2, double tf1, double tf2,
                      double* out) {
  if (!out) return chh::fail(CH_EINVAL, "out is NULL");
  chs::Scratch sc;
  chs::View v;
  if (int rc = chs::series_view(h, members, count, sc, &v)) return rc;
  double* dmom = nullptr;
  if (int rc = chs::series_moments(h, v, sc, &dmom)) return rc;
  double* dout = nullptr;
  if (cudaError_t e = sc.get(&dout, 4)) return chh::cuda_fail(e, "statistics scratch");
  CH_CHECK_CUDA(chs::launch_trend(dmom, v.T, t1, t2, tf1, tf2, dout, h->stream), "trend kernel");
  return chh::copy_out(h, out, dout, sizeof(double) * 4, "read trend");
}

}  // extern "C"
