// ch_droplets.cu -- Model 1 of the paper: ensembles of mean-field droplet populations.
//
// Each population of N droplets evolves by
//   dR_i/dt = H(R_i + eps) (-1/R_i^2 + u/R_i),   u = sum H(R_i) / sum H(R_i) R_i,
// (Sec. 2.1 Eqs. (13)-(14), regularised as in Sec. 3.1 Eq. (39); H(s) = 1 for s > 0), from
// R_i(0) = r_i (Eq. (38)), with F = 1/2 sum H(R_i) R_i^2, dF/dt = -sum H(R_i)/R_i (1 - u R_i)^2
// and beta = -(t/F) dF/dt sampled at given times (Sec. 2.4 Eqs. (31), (33), (36)).  The
// paper integrates with Matlab's ODE45; here every population runs the same Dormand-Prince
// 5(4) pair (J. R. Dormand and P. J. Prince, J. Comput. Appl. Math. 6 (1980) 19-26) with
// its own adaptive step size.
//
// Design: one CTA per population, for the whole run (one launch for the ensemble).  A
// thread owns positions i = tid, tid + blockDim, ...; the stage vectors k_1..k_7 and the
// stage values live in a per-population slice of global memory that stays in L2, and
// between compactions every thread touches only its own positions, so the only
// synchronisation is the block reductions: u at each of the 6 stages of a step, the
// error norm, and the observables on sample steps.  Reductions run in a fixed order
// (per-thread sums, then a shuffle tree, then warps in order): deterministic.  Every
// thread takes the same accept / reject decision from the same reduced value.
//
// Active set: a droplet with R + eps <= 0 has stopped for good (H(R + eps) = 0), counts
// in neither u nor the observables and adds nothing to the error norm, so at every sample
// time and every 256 accepted steps the population is compacted: the droplets that still
// evolve move, in order, to the front of the working arrays (a block-wide scan), and the
// stopped ones are written to their place in the output.  A step then costs in proportion
// to the droplets still evolving (about a tenth of them by t = 4 from uniform radii).
// The error norm still divides by the full N.  On GB300 the work is FP64-pipe bound
// (divisions above all), so the right-hand side takes one division, q = 1/R, and forms
// q (u - q) = -1/R^2 + u/R.
//
// Working set: a population of up to kSmemDroplets droplets keeps its working arrays (R,
// k_1..k_7, stage values, indices: 80 bytes a droplet) in shared memory, where a stage's
// loads, stores and reductions cost tens of cycles instead of an L2 round trip each;
// larger populations keep them in global memory (L2-resident).  The code is the same for
// both (generic pointers).
//
// The step loop is bounded by max_steps; a population that reaches it, or whose step
// size underflows, stops with a status code.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include <cuda_runtime.h>

#include "ch.h"
#include "ch_handle.h"

namespace chd {

constexpr int kMaxThreads = 1024;
constexpr int kBytesPerDroplet = 9 * 8 + 2 * 4;             // R, k_1..k_7, stage value; two indices
constexpr int kSmemDroplets = (227 * 1024 - 1024) / kBytesPerDroplet;  // 2892

// Dormand-Prince nodes and weights (row s: weights of stages 1..s-1 for stage s; row 7 is
// the fifth-order solution), and the embedded fourth-order weights.
__constant__ double kA[7][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0},
    {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0},
    {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0},
    {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0}};
__constant__ double kBs[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0, -92097.0 / 339200.0,
                              187.0 / 2100.0, 1.0 / 40.0};

struct View {
  int N;
  double* R;        // [M][N] radii (in: start, out: at t_end), original order
  double* Rc;       // [M][N] working radii of the active set (compacted order)
  int* idx;         // [M][N] original index of each active position
  int* idx2;        // [M][N] scratch of the compaction
  double* K;        // [M][7][N] stage derivatives (active positions)
  double* Y;        // [M][N] stage values (after stage 7: the fifth-order solution)
  const double* ts; // [ns] sample times
  int ns;
  double t_end, rtol, atol, h0, eps;
  int64_t max_steps;
  double* series;   // [M][ns][5] t, F, dF/dt, beta, live droplets
  int64_t* stats;   // [M][3] accepted, rejected, status (0 ok, 1 step limit, 2 step underflow)
  int smem;         // 1: working arrays in dynamic shared memory (N <= kSmemDroplets)
};

// Sum of two values over the CTA, returned to every thread (fixed order).
__device__ __forceinline__ double2 block_sum(double a, double b, double2* red) {
  const unsigned full = 0xffffffffu;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(full, a, o);
    b += __shfl_down_sync(full, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  __syncthreads();  // red is free (previous readers done)
  if (lane == 0) red[warp] = make_double2(a, b);
  __syncthreads();
  double2 s = make_double2(0.0, 0.0);
  for (int w = 0; w < nw; ++w) {
    s.x += red[w].x;
    s.y += red[w].y;
  }
  return s;
}

// u of the radii y (each thread sums its own droplets).
__device__ __forceinline__ double mean_field(const double* y, int N, double2* red) {
  double cnt = 0.0, sum = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double r = y[i];
    if (r > 0.0) {
      cnt += 1.0;
      sum += r;
    }
  }
  const double2 s = block_sum(cnt, sum, red);
  return s.y > 0.0 ? s.x / s.y : 0.0;
}

__device__ __forceinline__ double rhs(double r, double u, double eps) {
  if (!(r + eps > 0.0)) return 0.0;
  const double q = 1.0 / r;
  return q * (u - q);
}

// Moves the active positions whose droplet still evolves (R + eps > 0) to the front of
// Rc / K0 / idx, keeping their order, and writes the others to Rout at their original
// index.  Rt, Kt, it: scratch of n entries.  Returns the new active count (all threads).
__device__ int compact(double* Rc, double* K0, int* idx, double* Rt, double* Kt, int* it, double* Rout, int n,
                       double eps, int* wsum) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int base = 0;
  for (int c0 = 0; c0 < n; c0 += blockDim.x) {
    const int i = c0 + threadIdx.x;
    const bool in = i < n;
    const double r = in ? Rc[i] : 0.0;
    const bool keep = in && (r + eps > 0.0);
    if (in && !keep) Rout[idx[i]] = r;
    const unsigned b = __ballot_sync(full, keep);
    const int before = __popc(b & ((1u << lane) - 1u));
    __syncthreads();  // wsum free
    if (lane == 0) wsum[w] = __popc(b);
    __syncthreads();
    int off = 0, tot = 0;
    for (int k = 0; k < nw; ++k) {
      const int x = wsum[k];
      off += k < w ? x : 0;
      tot += x;
    }
    if (keep) {
      const int o = base + off + before;
      Rt[o] = r;
      Kt[o] = K0[i];
      it[o] = idx[i];
    }
    base += tot;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < base; i += blockDim.x) {
    Rc[i] = Rt[i];
    K0[i] = Kt[i];
    idx[i] = it[i];
  }
  __syncthreads();
  return base;
}

__device__ void sample(const double* R, int N, double t, double* row, double2* red) {
  double cnt = 0.0, sum = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double r = R[i];
    if (r > 0.0) {
      cnt += 1.0;
      sum += r;
    }
  }
  const double2 cs = block_sum(cnt, sum, red);
  const double u = cs.y > 0.0 ? cs.x / cs.y : 0.0;
  double f = 0.0, d = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const double r = R[i];
    if (r > 0.0) {
      f += 0.5 * r * r;
      const double g = 1.0 - u * r;
      d += g * g / r;
    }
  }
  const double2 fd = block_sum(f, d, red);
  if (threadIdx.x == 0) {
    row[0] = t;
    row[1] = fd.x;
    row[2] = -fd.y;
    row[3] = -(t / fd.x) * (-fd.y);
    row[4] = cs.x;
  }
}

__global__ void __launch_bounds__(kMaxThreads) drop_kernel(View v) {
  __shared__ double2 red[kMaxThreads / 32];
  __shared__ int wsum[kMaxThreads / 32];
  __shared__ double s_ctl[2];  // accept flag, next step size (written by thread 0)
  extern __shared__ __align__(16) double dsm[];
  const int m = blockIdx.x, N = v.N;
  double* Rout = v.R + (size_t)m * N;
  double *R, *K, *Y;
  int *idx, *idx2;
  if (v.smem) {
    R = dsm;
    K = R + N;
    Y = K + 7 * (size_t)N;
    idx = reinterpret_cast<int*>(Y + N);
    idx2 = idx + N;
  } else {
    R = v.Rc + (size_t)m * N;
    K = v.K + (size_t)m * 7 * N;
    Y = v.Y + (size_t)m * N;
    idx = v.idx + (size_t)m * N;
    idx2 = v.idx2 + (size_t)m * N;
  }
  double* series = v.series ? v.series + (size_t)m * v.ns * 5 : nullptr;
  const double eps = v.eps, rtol = v.rtol, atol = v.atol;

  // active set = every droplet, k_1 = f(R)
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    R[i] = Rout[i];
    idx[i] = i;
  }
  int n = N;
  {
    const double u = mean_field(R, n, red);
    for (int i = threadIdx.x; i < n; i += blockDim.x) K[i] = rhs(R[i], u, eps);
  }
  double t = 0.0, h = v.h0;
  int next = 0, status = 0;
  int64_t acc = 0, rej = 0;
  bool tidy = true;
  for (;;) {
    while (next < v.ns && v.ts[next] <= t) {
      if (series) sample(R, n, t, series + (size_t)next * 5, red);
      ++next;
      tidy = true;
    }
    if (tidy) {
      n = compact(R, K, idx, K + N, K + 2 * (size_t)N, idx2, Rout, n, eps, wsum);
      tidy = false;
    }
    if (t >= v.t_end) break;
    if (acc + rej >= v.max_steps) {
      status = 1;
      break;
    }
    if (!(h > 1e-300)) {
      status = 2;
      break;
    }
    const double target = (next < v.ns && v.ts[next] < v.t_end) ? v.ts[next] : v.t_end;
    const bool lands = h >= target - t;
    const double hs = lands ? target - t : h;
    // stages 2..7; stage 7 is evaluated at the fifth-order solution
    for (int s = 1; s < 7; ++s) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double a = 0.0;
        for (int j = 0; j < s; ++j) a += kA[s][j] * K[(size_t)j * N + i];
        Y[i] = R[i] + hs * a;
      }
      const double u = mean_field(Y, n, red);  // reads only this thread's droplets, then reduces
      double* Ks = K + (size_t)s * N;
      for (int i = threadIdx.x; i < n; i += blockDim.x) Ks[i] = rhs(Y[i], u, eps);
    }
    // scaled error norm of (fifth - fourth) order solutions (stopped droplets add 0)
    double e2 = 0.0;
    if (rtol > 0.0) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double lo = 0.0;
        for (int j = 0; j < 7; ++j) lo += kBs[j] * K[(size_t)j * N + i];
        const double yn = Y[i], y0 = R[i];
        const double e = yn - (y0 + hs * lo);
        const double q = e / (atol + rtol * fmax(fabs(y0), fabs(yn)));
        e2 += q * q;
      }
    }
    // the step controller runs on one thread (pow and sqrt are long FP64 sequences) and
    // its decision is broadcast through shared memory
    const double e2sum = rtol > 0.0 ? block_sum(e2, 0.0, red).x : 0.0;
    if (threadIdx.x == 0) {
      const double en = rtol > 0.0 ? sqrt(e2sum / (double)N) : 0.0;
      const bool ok = rtol <= 0.0 || en <= 1.0;
      double hn = h;
      if (rtol > 0.0) {
        double fac = en > 0.0 ? 0.9 * pow(en, -0.2) : 5.0;
        fac = fmin(5.0, fmax(0.2, fac));
        if (!ok) fac = fmin(fac, 1.0);
        hn = hs * fac;
      }
      s_ctl[0] = ok ? 1.0 : 0.0;
      s_ctl[1] = hn;
    }
    __syncthreads();
    const bool accept = s_ctl[0] != 0.0;
    h = s_ctl[1];
    if (accept) {
      const double* K7 = K + (size_t)6 * N;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        R[i] = Y[i];
        K[i] = K7[i];
      }
      t = lands ? target : t + hs;
      ++acc;
      if ((acc & 255) == 0) tidy = true;
    } else {
      ++rej;
    }
  }
  for (int i = threadIdx.x; i < n; i += blockDim.x) Rout[idx[i]] = R[i];
  if (threadIdx.x == 0) {
    v.stats[3 * m + 0] = acc;
    v.stats[3 * m + 1] = rej;
    v.stats[3 * m + 2] = status;
  }
}

}  // namespace chd

extern "C" {

int ch_droplets_run(int M, int N, double* R, double t_end, int nsamples, const double* t_samples, double rtol,
                    double atol, double h0, double eps, int64_t max_steps, double* series, int64_t* steps,
                    void* stream) {
  if (M < 1 || N < 1 || !R || !(t_end >= 0.0) || !std::isfinite(t_end) || nsamples < 0 ||
      (nsamples > 0 && !t_samples) || !(h0 > 0.0) || !std::isfinite(rtol) || !(atol > 0.0) || !(eps >= 0.0) ||
      max_steps < 1)
    return chh::fail(CH_EINVAL, "M, N >= 1, finite t_end >= 0, h0 > 0, atol > 0, eps >= 0, max_steps >= 1");
  for (int s = 0; s < nsamples; ++s)
    if (!std::isfinite(t_samples[s]) || (s > 0 && !(t_samples[s] > t_samples[s - 1])))
      return chh::fail(CH_EINVAL, "sample times must be finite and increasing");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t nR = (size_t)M * N;
  std::vector<void*> bufs;
  auto cleanup = [&]() {
    for (void* p : bufs) cudaFree(p);
  };
  auto get = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (chk::dev_malloc(&p, bytes > 0 ? bytes : 1) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    bufs.push_back(p);
    return p;
  };
  chd::View v{};
  v.N = N;
  v.R = static_cast<double*>(get(sizeof(double) * nR));
  v.Rc = static_cast<double*>(get(sizeof(double) * nR));
  v.idx = static_cast<int*>(get(sizeof(int) * nR));
  v.idx2 = static_cast<int*>(get(sizeof(int) * nR));
  v.K = static_cast<double*>(get(sizeof(double) * 7 * nR));
  v.Y = static_cast<double*>(get(sizeof(double) * nR));
  double* dts = static_cast<double*>(get(sizeof(double) * (size_t)nsamples));
  v.series = static_cast<double*>(get(sizeof(double) * 5 * (size_t)M * nsamples));
  v.stats = static_cast<int64_t*>(get(sizeof(int64_t) * 3 * (size_t)M));
  if (!v.R || !v.Rc || !v.idx || !v.idx2 || !v.K || !v.Y || !dts || !v.series || !v.stats) {
    cleanup();
    return chh::fail(CH_ENOMEM, "droplet buffers");
  }
  v.ts = dts;
  v.ns = nsamples;
  v.t_end = t_end;
  v.rtol = rtol;
  v.atol = atol;
  v.h0 = h0;
  v.eps = eps;
  v.max_steps = max_steps;
  cudaError_t e = cudaMemcpyAsync(v.R, R, sizeof(double) * nR, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nsamples > 0)
    e = cudaMemcpyAsync(dts, t_samples, sizeof(double) * nsamples, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nsamples > 0)
    e = cudaMemsetAsync(v.series, 0xff, sizeof(double) * 5 * (size_t)M * nsamples, st);  // NaN until sampled
  if (e == cudaSuccess) {
    const int threads = N >= chd::kMaxThreads ? chd::kMaxThreads : ((N + 31) / 32) * 32;
    v.smem = N <= chd::kSmemDroplets ? 1 : 0;
    const size_t smem = v.smem ? (size_t)N * chd::kBytesPerDroplet : 0;
    if (smem > 48 * 1024)
      e = cudaFuncSetAttribute(chd::drop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
      chd::drop_kernel<<<M, threads, smem, st>>>(v);
      e = cudaGetLastError();
    }
  }
  std::vector<int64_t> hst(3 * (size_t)M);
  if (e == cudaSuccess) e = cudaMemcpyAsync(R, v.R, sizeof(double) * nR, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && series && nsamples > 0)
    e = cudaMemcpyAsync(series, v.series, sizeof(double) * 5 * (size_t)M * nsamples, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hst.data(), v.stats, sizeof(int64_t) * 3 * M, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) return chh::cuda_fail(e, "droplet run");
  if (steps) std::copy(hst.begin(), hst.end(), steps);
  for (int m = 0; m < M; ++m)
    if (hst[3 * (size_t)m + 2] != 0)
      return chh::fail(CH_EINVAL, hst[3 * (size_t)m + 2] == 1 ? "a population reached max_steps"
                                                              : "a population's step size underflowed");
  return CH_OK;
}

}  // extern "C"
