// ch_kernels.cu -- sm_103a kernels of one Cahn-Hilliard step (delta-form factorised ADI).
//
// One step of every member is two launches:
//   rows_kernel  (one CTA per band of rows of one member)
//     C rows j0-2 .. j0+nr+1  --(smem)-->  mu = C^3 - C - gamma lap_h C  on rows j0-1..j0+nr
//     [sample steps] FP64 partial sums of the F and dF/dt densities (Sec. 1 Eq. (4))
//     R' = scaled dt lap_h mu (the 13-point explicit right-hand side, Sec. 1 Eq. (3))
//     row sweep  W' = Q_x^-T Q_x^-1 R'  (cyclic, pre-rolled second-order recurrences)
//     W' rows --> global scratch W
//   cols_kernel  (one CTA per panel of columns of one member)
//     W' panel --(smem)--> column sweep  Z = Q_y^-T Q_y^-1 W'  -->  C += kappa Z
//     [panel 0] finalise the member's sample (F, dF/dt, beta, window average) and
//     advance its step counter.
//
// The cyclic solve.  I + s D^4 (stencil [s, -4s, 1+6s, -4s, s], periodic) factors as
// c Q Q^T with Q the circulant of q(z) = 1 - p1 z - p2 z^2 whose roots lie outside the
// unit circle (spectral factorisation; the host computes p1, p2, c in FP64 as the fixed
// point of the band LDL^T recurrences).  Q y = r is the periodic recurrence
//     y_i = r_i + p1 y_{i-1} + p2 y_{i-2}      (i mod n),
// Q^T x = y the same recurrence run backwards.  Its impulse response decays like
// |root|^-k, so the periodic solution at i equals the recurrence started from a zero
// state K points before i (cyclically, wrapping as many times as needed when K > n) up
// to a relative error below the precision's unit round-off; the host picks K from the
// powers of the companion matrix.  A thread that owns the chunk [c0, c1) of a line
// therefore needs nothing from the other threads: it pre-rolls over the K points before
// c0 (forward) or after c1 (backward).  This costs 2 FMA per point per pass plus 2K per
// chunk, against ~9 FMA per point for a band LDL^T + Woodbury corner correction, which
// matters because the FP64 path is bound by the FP64 pipe on GB300.
#include <cstdint>
#include <cuda_runtime.h>

#include "ch_internal.h"

namespace chk {
namespace {

// -------------------------------------------------------------------------------------
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) evaluated as a counter-based generator:
// draw k of the stream seeded with `seed` is mix(seed + (k + 1) * golden_gamma).
// -------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t sm64_draw(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1ull) * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void init_fields_kernel(DevView v) {
  for (int m = blockIdx.y; m < v.m; m += gridDim.y) {
    const MemberParams& P = v.mp[m];
    const int64_t npts = (int64_t)P.nx * P.ny;
    T* C = static_cast<T*>(v.C) + P.offset;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < npts;
         p += (int64_t)gridDim.x * blockDim.x) {
      // u = top 53 bits * 2^-53 (exact); C = C0 + 0.1 (2u - 1) with every operation
      // rounded on its own (no contraction): the FP64 field is bit-identical to its
      // definition.
      const double u = (double)(sm64_draw(P.seed, P.counter_base + (uint64_t)p) >> 11) *
                       (1.0 / 9007199254740992.0);
      const double noise = __dmul_rn(0.1, __dsub_rn(__dmul_rn(2.0, u), 1.0));
      C[p] = (T)__dadd_rn(P.C0, noise);
    }
  }
}

// Fixed-order block reduction of two FP64 sums (deterministic for a given block size).
__device__ __forceinline__ void block_sum2(double& a, double& b, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    red[2 * warp] = a;
    red[2 * warp + 1] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sa = 0.0, sb = 0.0;
    for (int w = 0; w < nw; ++w) {
      sa += red[2 * w];
      sb += red[2 * w + 1];
    }
    a = sa;
    b = sb;
  }
}

// FP64 chemical potential at (row r of the C tile, column i) from the stored field, used by
// the FP32 form's observables so that dF/dt is the FP64 functional of the FP32 field.
template <typename T>
__device__ __forceinline__ double mu64_at(const T* Cs, int ld, int r, int i, int nx, double a, double bx,
                                          double by) {
  const T* c0 = Cs + (size_t)r * ld;
  const int ie = (i + 1 == nx) ? 0 : i + 1;
  const int iw = (i == 0) ? nx - 1 : i - 1;
  const double c = (double)c0[i];
  return c * (c * c - a) - bx * ((double)c0[ie] + (double)c0[iw]) - by * ((double)c0[i + ld] + (double)c0[i - ld]);
}

__device__ __forceinline__ int wrap_index(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

// Forward recurrence y_i = r_i + p1 y_{i-1} + p2 y_{i-2} on the chunk [c0, c1) of a
// periodic line of n points stored with element stride `es` starting at `in`; the state
// is pre-rolled from zero over the K points before c0 (cyclically).
template <typename T>
__device__ __forceinline__ void sweep_forward(const T* __restrict__ in, T* __restrict__ out,
                                              int es, int n, int c0, int c1, int K, T p1, T p2) {
  T y1 = T(0), y2 = T(0);
  int k = wrap_index(c0 - K, n);
  for (int q = 0; q < K; ++q) {
    const T y = fma(p1, y1, fma(p2, y2, in[k * es]));
    y2 = y1;
    y1 = y;
    if (++k == n) k = 0;
  }
  for (int i = c0; i < c1; ++i) {
    const T y = fma(p1, y1, fma(p2, y2, in[i * es]));
    out[i * es] = y;
    y2 = y1;
    y1 = y;
  }
}

// Backward recurrence x_i = y_i + p1 x_{i+1} + p2 x_{i+2} on [c0, c1), pre-rolled over the
// K points after c1 (cyclically).
template <typename T>
__device__ __forceinline__ void sweep_backward(const T* __restrict__ in, T* __restrict__ out,
                                               int es, int n, int c0, int c1, int K, T p1, T p2) {
  T x1 = T(0), x2 = T(0);
  int k = wrap_index(c1 - 1 + K, n);
  for (int q = 0; q < K; ++q) {
    const T x = fma(p1, x1, fma(p2, x2, in[k * es]));
    x2 = x1;
    x1 = x;
    if (--k < 0) k = n - 1;
  }
  for (int i = c1 - 1; i >= c0; --i) {
    const T x = fma(p1, x1, fma(p2, x2, in[i * es]));
    out[i * es] = x;
    x2 = x1;
    x1 = x;
  }
}

// -------------------------------------------------------------------------------------
// Row kernel: stencil + observables + row sweep for a band of rows of one member.
// Shared memory: Cs = (nr+4) rows of C (halo 2), Ms = (nr+2) rows of mu, row pitch nx+1,
// then a small FP64 reduction buffer.  Cs is reused for R' and then for W', Ms for the
// forward-sweep output.
// -------------------------------------------------------------------------------------
template <typename T, bool OBS_ONLY>
__global__ void __launch_bounds__(512) rows_kernel(DevView v) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tile tl = v.row_tiles[blockIdx.x];
  const MemberParams& P = v.mp[tl.member];
  MemberState* st = v.ms + tl.member;
  bool sample = true;
  if (!OBS_ONLY) {
    const bool active = st->remaining > 0;
    if (tl.index == 0 && threadIdx.x == 0) st->active = active ? 1 : 0;
    if (!active) return;
    sample = (st->step % P.every) == 0;
  }
  const int nx = P.nx, ny = P.ny, j0 = tl.start, nr = tl.count;
  const int ld = nx + 1;
  T* Cs = reinterpret_cast<T*>(smem);
  T* Ms = Cs + (size_t)(nr + 4) * ld;
  double* red = reinterpret_cast<double*>(
      smem + ((((size_t)(2 * nr + 6) * ld * sizeof(T)) + 15) & ~(size_t)15));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

  // 1. C rows j0-2 .. j0+nr+1 (periodic in j), one warp per row, coalesced.
  {
    const T* __restrict__ C = static_cast<const T*>(v.C) + P.offset;
    for (int r = warp; r < nr + 4; r += nwarps) {
      int j = j0 - 2 + r;
      if (j < 0) j += ny;
      if (j >= ny) j -= ny;
      const T* src = C + (int64_t)j * nx;
      T* dst = Cs + (size_t)r * ld;
      for (int i = lane; i < nx; i += 32) dst[i] = src[i];
    }
  }
  __syncthreads();

  // 2. mu on rows j0-1 .. j0+nr  (Ms row r <-> Cs row r+1).
  {
    const T a = (T)P.a, bx = (T)P.bx, by = (T)P.by;
    for (int r = warp; r < nr + 2; r += nwarps) {
      const T* c0 = Cs + (size_t)(r + 1) * ld;
      const T* cm = c0 - ld;
      const T* cp = c0 + ld;
      T* mrow = Ms + (size_t)r * ld;
      for (int i = lane; i < nx; i += 32) {
        const int ie = (i + 1 == nx) ? 0 : i + 1;
        const int iw = (i == 0) ? nx - 1 : i - 1;
        const T c = c0[i];
        const T u = c * fma(c, c, -a);
        mrow[i] = fma(-by, cp[i] + cm[i], fma(-bx, c0[ie] + c0[iw], u));
      }
    }
  }
  __syncthreads();

  // 3. Sample steps: FP64 partial sums of the F and dF/dt densities over the band's rows.
  if (sample) {
    double sF = 0.0, sD = 0.0;
    const double hxi = 1.0 / P.hx, hyi = 1.0 / P.hy, hg = 0.5 * P.gamma;
    for (int r = warp; r < nr; r += nwarps) {
      const T* c0 = Cs + (size_t)(r + 2) * ld;
      const T* cp = c0 + ld;
      const T* m0 = Ms + (size_t)(r + 1) * ld;
      const T* mp = m0 + ld;
      for (int i = lane; i < nx; i += 32) {
        const int ie = (i + 1 == nx) ? 0 : i + 1;
        const double c = (double)c0[i];
        const double gx = ((double)c0[ie] - c) * hxi;
        const double gy = ((double)cp[i] - c) * hyi;
        const double w = c * c - 1.0;
        sF += 0.25 * w * w + hg * (gx * gx + gy * gy);
        double mu, mue, mun;
        if (sizeof(T) == sizeof(double)) {
          mu = (double)m0[i];
          mue = (double)m0[ie];
          mun = (double)mp[i];
        } else {
          mu = mu64_at(Cs, ld, r + 2, i, nx, P.a, P.bx, P.by);
          mue = mu64_at(Cs, ld, r + 2, ie, nx, P.a, P.bx, P.by);
          mun = mu64_at(Cs, ld, r + 3, i, nx, P.a, P.bx, P.by);
        }
        const double mx = (mue - mu) * hxi;
        const double my = (mun - mu) * hyi;
        sD += mx * mx + my * my;
      }
    }
    block_sum2(sF, sD, red);
    if (threadIdx.x == 0) v.partials[P.partial_base + tl.index] = make_double2(sF, sD);
    __syncthreads();
  }
  if (OBS_ONLY) return;

  // 4. R' = (mu_e + mu_w) + rho (mu_n + mu_s) + w0 mu on rows j0 .. j0+nr-1 -> Cs rows 0..
  {
    const T rho = (T)P.rho, w0 = (T)P.w0;
    for (int r = warp; r < nr; r += nwarps) {
      const T* m0 = Ms + (size_t)(r + 1) * ld;
      const T* mm = m0 - ld;
      const T* mp = m0 + ld;
      T* out = Cs + (size_t)r * ld;
      for (int i = lane; i < nx; i += 32) {
        const int ie = (i + 1 == nx) ? 0 : i + 1;
        const int iw = (i == 0) ? nx - 1 : i - 1;
        out[i] = fma(w0, m0[i], fma(rho, mp[i] + mm[i], m0[ie] + m0[iw]));
      }
    }
  }
  __syncthreads();

  // 5. Row sweep: sweep_p threads per row, each owning a chunk of the row.
  const int sweep_p = P.rows_p;
  const int nsweep = nr * sweep_p;
  const int chunk = (nx + sweep_p - 1) / sweep_p;
  const int row = threadIdx.x % nr;
  const int c0 = (threadIdx.x / nr) * chunk;
  const int c1 = min(nx, c0 + chunk);
  const bool sweeper = threadIdx.x < nsweep && c0 < c1;
  const T p1 = (T)P.p1x, p2 = (T)P.p2x;
  if (sweeper) sweep_forward<T>(Cs + (size_t)row * ld, Ms + (size_t)row * ld, 1, nx, c0, c1, P.kx, p1, p2);
  __syncthreads();
  if (sweeper) sweep_backward<T>(Ms + (size_t)row * ld, Cs + (size_t)row * ld, 1, nx, c0, c1, P.kx, p1, p2);
  __syncthreads();

  // 6. W' rows -> global scratch.
  {
    T* __restrict__ W = static_cast<T*>(v.W) + P.offset;
    for (int r = warp; r < nr; r += nwarps) {
      const T* src = Cs + (size_t)r * ld;
      T* dst = W + (int64_t)(j0 + r) * nx;
      for (int i = lane; i < nx; i += 32) dst[i] = src[i];
    }
  }
}

// -------------------------------------------------------------------------------------
// Column kernel: column sweep and update for a panel of columns of one member.
// Shared memory: Ws and Ys, ny rows of nc+1 elements each.
// -------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) cols_kernel(DevView v) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tile tl = v.col_tiles[blockIdx.x];
  MemberState* st = v.ms + tl.member;
  if (!st->active) return;
  const MemberParams& P = v.mp[tl.member];
  const int nx = P.nx, ny = P.ny, i0 = tl.start, nc = tl.count;
  const int ldc = nc + 1;
  T* Ws = reinterpret_cast<T*>(smem);
  T* Ys = Ws + (size_t)ny * ldc;

  {
    const T* __restrict__ W = static_cast<const T*>(v.W) + P.offset;
    for (int idx = threadIdx.x; idx < ny * nc; idx += blockDim.x) {
      const int j = idx / nc, c = idx - j * nc;
      Ws[(size_t)j * ldc + c] = W[(int64_t)j * nx + i0 + c];
    }
  }
  __syncthreads();

  const int sweep_p = P.cols_p;
  const int nsweep = nc * sweep_p;
  const int chunk = (ny + sweep_p - 1) / sweep_p;
  const int col = threadIdx.x % nc;
  const int c0 = (threadIdx.x / nc) * chunk;
  const int c1 = min(ny, c0 + chunk);
  const bool sweeper = threadIdx.x < nsweep && c0 < c1;
  const T p1 = (T)P.p1y, p2 = (T)P.p2y;
  if (sweeper) sweep_forward<T>(Ws + col, Ys + col, ldc, ny, c0, c1, P.ky, p1, p2);
  __syncthreads();
  if (sweeper) sweep_backward<T>(Ys + col, Ws + col, ldc, ny, c0, c1, P.ky, p1, p2);
  __syncthreads();

  {
    T* __restrict__ C = static_cast<T*>(v.C) + P.offset;
    const T kap = (T)P.kappa;
    for (int idx = threadIdx.x; idx < ny * nc; idx += blockDim.x) {
      const int j = idx / nc, c = idx - j * nc;
      const int64_t g = (int64_t)j * nx + i0 + c;
      C[g] = fma(kap, Ws[(size_t)j * ldc + c], C[g]);
    }
  }

  // Panel 0 finalises the member's sample of this step (partials written by the row
  // kernel of the same step) and advances the member's step counter.  No other CTA of
  // this launch reads or writes the member's state.
  if (tl.index == 0 && threadIdx.x == 0) {
    const int64_t n = st->step;
    if (n % P.every == 0) {
      double sF = 0.0, sD = 0.0;
      for (int b = 0; b < P.nbands; ++b) {
        const double2 pr = v.partials[P.partial_base + b];
        sF += pr.x;
        sD += pr.y;
      }
      const double hh = P.hx * P.hy;
      const double F = hh * sF;
      const double dFdt = -(hh * sD);
      const double t = (double)n * P.dt;
      const double beta = -(t / F) * dFdt;
      st->F = F;
      st->dFdt = dFdt;
      st->beta = beta;
      if (!isfinite(F) || !isfinite(dFdt)) st->nonfinite = 1;
      if (P.series_cap > 0) {
        double* s = v.series + ((size_t)tl.member * P.series_cap + (size_t)(st->nsamples % P.series_cap)) * 4;
        s[0] = t;
        s[1] = F;
        s[2] = dFdt;
        s[3] = beta;
      }
      st->nsamples += 1;
      if (t >= P.t1) {
        st->beta_sum += beta;
        st->beta_count += 1;
      }
    }
    st->step = n + 1;
    if (st->remaining != kUnbounded) st->remaining -= 1;
  }
}

// F, dF/dt, beta of the current fields (one thread per member) for ch_observables.
__global__ void obs_finalize_kernel(DevView v) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= v.m) return;
  const MemberParams& P = v.mp[m];
  double sF = 0.0, sD = 0.0;
  for (int b = 0; b < P.nbands; ++b) {
    const double2 pr = v.partials[P.partial_base + b];
    sF += pr.x;
    sD += pr.y;
  }
  const double hh = P.hx * P.hy;
  const double F = hh * sF;
  const double dFdt = -(hh * sD);
  const double t = (double)v.ms[m].step * P.dt;
  v.obs_now[3 * m + 0] = F;
  v.obs_now[3 * m + 1] = dFdt;
  v.obs_now[3 * m + 2] = -(t / F) * dFdt;
}

template <typename T>
cudaError_t step_impl(const DevView& v, int n_row_tiles, int n_col_tiles, const LaunchShape& sh,
                      cudaStream_t st) {
  rows_kernel<T, false><<<n_row_tiles, sh.rows_threads, sh.rows_smem, st>>>(v);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  cols_kernel<T><<<n_col_tiles, sh.cols_threads, sh.cols_smem, st>>>(v);
  return cudaGetLastError();
}

template <typename T>
cudaError_t phase_impl(const DevView& v, int phase, int n_tiles, const LaunchShape& sh, cudaStream_t st) {
  if (phase == 0)
    rows_kernel<T, false><<<n_tiles, sh.rows_threads, sh.rows_smem, st>>>(v);
  else
    cols_kernel<T><<<n_tiles, sh.cols_threads, sh.cols_smem, st>>>(v);
  return cudaGetLastError();
}

template <typename T>
cudaError_t observe_impl(const DevView& v, int n_row_tiles, const LaunchShape& sh, cudaStream_t st) {
  rows_kernel<T, true><<<n_row_tiles, sh.rows_threads, sh.rows_smem, st>>>(v);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  obs_finalize_kernel<<<(v.m + 127) / 128, 128, 0, st>>>(v);
  return cudaGetLastError();
}

}  // namespace

cudaError_t set_kernel_smem_limits(int precision, size_t rows_smem, size_t cols_smem) {
  cudaError_t e;
  if (precision == 0) {
    e = cudaFuncSetAttribute(rows_kernel<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(rows_kernel<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(cols_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cols_smem);
  }
  e = cudaFuncSetAttribute(rows_kernel<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(rows_kernel<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)rows_smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(cols_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cols_smem);
}

cudaError_t launch_init_fields(const DevView& v, int precision, int64_t max_points, cudaStream_t st) {
  int64_t blocks = (max_points + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  dim3 grid((unsigned)blocks, (unsigned)(v.m < 65535 ? v.m : 65535));
  if (precision == 0)
    init_fields_kernel<double><<<grid, 256, 0, st>>>(v);
  else
    init_fields_kernel<float><<<grid, 256, 0, st>>>(v);
  return cudaGetLastError();
}

cudaError_t launch_step(const DevView& v, int precision, int n_row_tiles, int n_col_tiles,
                        const LaunchShape& sh, cudaStream_t st) {
  return precision == 0 ? step_impl<double>(v, n_row_tiles, n_col_tiles, sh, st)
                        : step_impl<float>(v, n_row_tiles, n_col_tiles, sh, st);
}

cudaError_t launch_phase(const DevView& v, int precision, int phase, int n_tiles, const LaunchShape& sh,
                         cudaStream_t st) {
  return precision == 0 ? phase_impl<double>(v, phase, n_tiles, sh, st) : phase_impl<float>(v, phase, n_tiles, sh, st);
}

cudaError_t launch_observe(const DevView& v, int precision, int n_row_tiles, const LaunchShape& sh,
                           cudaStream_t st) {
  return precision == 0 ? observe_impl<double>(v, n_row_tiles, sh, st)
                        : observe_impl<float>(v, n_row_tiles, sh, st);
}

}  // namespace chk
