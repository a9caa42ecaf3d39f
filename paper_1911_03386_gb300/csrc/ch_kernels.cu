// ch_kernels.cu -- sm_103a kernels of one Cahn-Hilliard step (delta-form factorised ADI).
//
// A step of every member is one of two launch sequences (chosen per handle):
//
//   fused   rows_kernel   C rows (+2 halo) --smem--> mu --> R' --> row sweep --> W
//           cols_kernel   W panel --smem--> column sweep --> C += kappa Z
//   split   stencil_kernel   C rows (+2 halo) --smem--> mu --> R' --> W (global)
//           rowsweep_kernel  W rows --smem--> row sweep in place --> W
//           cols_kernel      as above
//
// rows_kernel keeps R' on chip (5 words of traffic per point and step: read C, write W,
// read W, read C, write C), the bandwidth-lean form used for FP32.  The split form moves
// two more words (R' written and read back) but lets every thread of the stencil kernel
// do FP64 work and lets the row sweeps run as many full warps of independent recurrences
// per SM: the form used for FP64, which is bound by GB300's FP64 pipe (2 DFMA per SM per
// clock), not by HBM.
//
//   mu = C^3 - C - gamma lap_h C = C (C^2 - a) - bx (Ce + Cw) - by (Cn + Cs)
//   R' = (mu_e + mu_w) + rho (mu_n + mu_s) + w0 mu       (R = dt lap_h mu = dt/hx^2 R')
//
// On sample steps the stencil phase also writes FP64 partial sums of the F and dF/dt
// densities (Sec. 1 Eq. (4)) per row band, and the column kernel's panel-0 CTA of each
// member reduces them in fixed order into F, dF/dt, beta (Eq. (6)) and the beta window
// average, then advances the member's step counter.
//
// The cyclic solve.  I + s D^4 (stencil [s, -4s, 1+6s, -4s, s], periodic) factors as
// c Q Q^T with Q the circulant of q(z) = 1 - p1 z - p2 z^2 whose roots lie outside the
// unit circle (spectral factorisation, computed on the host in FP64).  Q y = r is the
// periodic recurrence
//     y_i = r_i + p1 y_{i-1} + p2 y_{i-2}      (i mod n),
// Q^T x = y the same recurrence run backwards.  Its impulse response decays like
// |root|^-k, so the periodic solution at i equals the recurrence started from a zero
// state K points before i (cyclically, wrapping as many times as needed when K > n) up
// to a relative error below the precision's unit round-off; the host picks K from the
// powers of the companion matrix.  A thread that owns the chunk [c0, c1) of a line
// therefore needs nothing from the other threads: it pre-rolls over the K points before
// c0 (forward) or after c1 (backward).  This costs 2 FMA per point per pass plus 2K per
// chunk, against ~9 FMA per point for a band LDL^T + Woodbury corner correction.  With
// one chunk per line the sweep can run in place (the pre-roll reads precede every write
// they depend on).
//
// Segment form (rows_seg_kernel).  Since K grows like s^(1/4) ~ n, pre-rolled chunks
// cost (1 + K p / n) passes for p chunks per line.  The segment form holds a row in the
// registers of G = n / S lanes (S consecutive points each) and solves each recurrence
// exactly: a pass from a zero state over every segment gives its end state e_l; an
// inclusive scan across the lanes (Kogge-Stone, log2 G shuffle steps with the constant
// matrices M^(S 2^d), M = [[p1, p2], [1, 0]]) gives the state Y_l after segment l of a
// line started from zero; the periodic start state is x0 = (I - M^n)^-1 Y_{G-1}, lane l
// starts from M^(S l) x0 + Y_{l-1}, and a second pass over the segment produces the
// solution.  Two passes per recurrence whatever K, no shared-memory sweep traffic, no
// barrier inside the sweep.
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
__global__ void init_fields_kernel(DevView v, const int* list, int count) {
  for (int q = blockIdx.y; q < count; q += gridDim.y) {
    const int m = list ? list[q] : q;
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
      const double c = __dadd_rn(P.C0, noise);
      C[p] = (T)c;
      if (sizeof(T) == 4 && P.comp)  // lo part: the exact remainder of the FP64 value
        static_cast<T*>(v.C)[P.lo_offset + p] = (T)__dsub_rn(c, (double)(T)c);
    }
  }
}

// -------------------------------------------------------------------------------------
// Asynchronous global -> shared copies (cp.async, element-sized), so that a CTA has all
// of its tile's loads in flight at once.
// -------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void cp_async_elem(T* smem_dst, const T* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  if (sizeof(T) == 8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem_src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem_src) : "memory");
}

// Rows of a field can be moved in 16-byte pieces when a row is a whole number of them
// (member bases are 16-byte aligned); tiles then use the dense pitch nx.
template <typename T>
__device__ __forceinline__ bool rows_vec_ok(int nx) {
  return (nx * (int)sizeof(T)) % 16 == 0;
}

// Pitch of a C tile: dense when rows move in 16-byte pieces, else nx + 1.
template <typename T>
__device__ __forceinline__ int ctile_pitch(int nx) {
  return rows_vec_ok<T>(nx) ? nx : nx + 1;
}

// Rows j_first .. j_first+nrows-1 (periodic in j) of an ny x nx field -> shared rows of
// pitch ld, one warp per row; 16-byte copies when rows_vec_ok (then ld must be nx).  The
// caller waits (cp_async_wait_all + __syncthreads).
template <typename T>
__device__ __forceinline__ void load_rows_async(T* dst, int ld, const T* __restrict__ field, int nx, int ny,
                                                int j_first, int nrows) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int r = warp; r < nrows; r += nwarps) {
    int j = j_first + r;
    if (j < 0) j += ny;
    if (j >= ny) j -= ny;
    const T* src = field + (int64_t)j * nx;
    T* d = dst + (size_t)r * ld;
    if (rows_vec_ok<T>(nx) && ld == nx) {
      const int nv = nx * (int)sizeof(T) / 16;
      for (int q = lane; q < nv; q += 32)
        cp_async16(reinterpret_cast<char*>(d) + 16 * q, reinterpret_cast<const char*>(src) + 16 * q);
    } else {
      for (int i = lane; i < nx; i += 32) cp_async_elem(d + i, src + i);
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
                                          double by) {  // ld: C tile pitch
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

// Whole-line sweep in place by one thread, written for instruction economy: the pre-roll
// walks contiguous segments (no per-point wrap test) and every pass runs in batches of 8
// whose loads are issued before the batch's dependent FMAs.  The recurrences are the ones
// stated at the top of this file (forward over the K points before the line start, then
// the line; backward over the K points after its end, then the line).
template <typename T>
__device__ __forceinline__ void seg_forward(const T* line, int es, int begin, int end, T p1, T p2, T& a, T& b) {
  int i = begin;
  for (; i + 8 <= end; i += 8) {
    T r[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) r[u] = line[(i + u) * es];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const T y = fma(p1, a, fma(p2, b, r[u]));
      b = a;
      a = y;
    }
  }
  for (; i < end; ++i) {
    const T y = fma(p1, a, fma(p2, b, line[i * es]));
    b = a;
    a = y;
  }
}

template <typename T>
__device__ __forceinline__ void seg_backward(const T* line, int es, int hi, int lo, T p1, T p2, T& a, T& b) {
  int i = hi;  // walks hi, hi-1, ..., lo
  for (; i - 8 >= lo - 1; i -= 8) {
    T r[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) r[u] = line[(i - u) * es];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const T y = fma(p1, a, fma(p2, b, r[u]));
      b = a;
      a = y;
    }
  }
  for (; i >= lo; --i) {
    const T y = fma(p1, a, fma(p2, b, line[i * es]));
    b = a;
    a = y;
  }
}

template <typename T>
__device__ __forceinline__ void line_sweep_inplace(T* line, int es, int n, int K, T p1, T p2) {
  // forward pre-roll over indices -K .. -1 (mod n), in increasing order
  T a = T(0), b = T(0);
  for (int rem = K, idx = wrap_index(-K, n); rem > 0;) {
    const int seg = min(rem, n - idx);
    seg_forward<T>(line, es, idx, idx + seg, p1, p2, a, b);
    rem -= seg;
    idx = 0;
  }
  // forward pass in place
  int i = 0;
  for (; i + 8 <= n; i += 8) {
    T r[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) r[u] = line[(i + u) * es];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const T y = fma(p1, a, fma(p2, b, r[u]));
      line[(i + u) * es] = y;
      b = a;
      a = y;
    }
  }
  for (; i < n; ++i) {
    const T y = fma(p1, a, fma(p2, b, line[i * es]));
    line[i * es] = y;
    b = a;
    a = y;
  }
  // backward pre-roll over indices n-1+K .. n (mod n), in decreasing order
  a = T(0);
  b = T(0);
  for (int rem = K, idx = wrap_index(n - 1 + K, n); rem > 0;) {
    const int seg = min(rem, idx + 1);
    seg_backward<T>(line, es, idx, idx - seg + 1, p1, p2, a, b);
    rem -= seg;
    idx = n - 1;
  }
  // backward pass in place
  i = n - 1;
  for (; i - 8 >= -1; i -= 8) {
    T r[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) r[u] = line[(i - u) * es];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const T x = fma(p1, a, fma(p2, b, r[u]));
      line[(i - u) * es] = x;
      b = a;
      a = x;
    }
  }
  for (; i >= 0; --i) {
    const T x = fma(p1, a, fma(p2, b, line[i * es]));
    line[i * es] = x;
    b = a;
    a = x;
  }
}

// Chunked in-place sweep of a line shared by several threads, lean form: thread owns
// [c0, c1) (active = it owns a non-empty chunk).  Each pass pre-rolls first (contiguous
// segments, reads only), then after a CTA barrier runs its chunk in place in batches of
// 8 with the loads issued ahead.  Every thread of the CTA must call it (it contains
// __syncthreads).
template <typename T>
__device__ __forceinline__ void chunk_sweep_inplace(T* line, int es, int n, int c0, int c1, int K, T p1, T p2,
                                                    bool active) {
  T a = T(0), b = T(0);
  if (active) {
    for (int rem = K, idx = wrap_index(c0 - K, n); rem > 0;) {
      const int seg = min(rem, n - idx);
      seg_forward<T>(line, es, idx, idx + seg, p1, p2, a, b);
      rem -= seg;
      idx = 0;
    }
  }
  __syncthreads();
  if (active) {
    int i = c0;
    for (; i + 8 <= c1; i += 8) {
      T r[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) r[u] = line[(i + u) * es];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const T y = fma(p1, a, fma(p2, b, r[u]));
        line[(i + u) * es] = y;
        b = a;
        a = y;
      }
    }
    for (; i < c1; ++i) {
      const T y = fma(p1, a, fma(p2, b, line[i * es]));
      line[i * es] = y;
      b = a;
      a = y;
    }
  }
  __syncthreads();
  a = T(0);
  b = T(0);
  if (active) {
    for (int rem = K, idx = wrap_index(c1 - 1 + K, n); rem > 0;) {
      const int seg = min(rem, idx + 1);
      seg_backward<T>(line, es, idx, idx - seg + 1, p1, p2, a, b);
      rem -= seg;
      idx = n - 1;
    }
  }
  __syncthreads();
  if (active) {
    int i = c1 - 1;
    for (; i - 8 >= c0 - 1; i -= 8) {
      T r[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) r[u] = line[(i - u) * es];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const T x = fma(p1, a, fma(p2, b, r[u]));
        line[(i - u) * es] = x;
        b = a;
        a = x;
      }
    }
    for (; i >= c0; --i) {
      const T x = fma(p1, a, fma(p2, b, line[i * es]));
      line[i * es] = x;
      b = a;
      a = x;
    }
  }
}

// mu on nrows rows: Ms row r (pitch lm) <- C tile row r+1 (pitch lc; rows r .. r+2 read).
template <typename T>
__device__ __forceinline__ void compute_mu(const T* Cs, int lc, T* Ms, int lm, int nx, int nrows, T a, T bx, T by) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int r = warp; r < nrows; r += nwarps) {
    const T* c0 = Cs + (size_t)(r + 1) * lc;
    const T* cm = c0 - lc;
    const T* cp = c0 + lc;
    T* mrow = Ms + (size_t)r * lm;
    for (int i = lane; i < nx; i += 32) {
      const int ie = (i + 1 == nx) ? 0 : i + 1;
      const int iw = (i == 0) ? nx - 1 : i - 1;
      const T c = c0[i];
      const T u = c * fma(c, c, -a);
      mrow[i] = fma(-by, cp[i] + cm[i], fma(-bx, c0[ie] + c0[iw], u));
    }
  }
}

// FP32 form: FP64 partial sums of the F and dF/dt densities over the band's nr rows (C
// tile rows 2..nr+1) with mu recomputed in FP64 from the stored field once per point.  A
// warp walks a strip of rows down a chunk of 31 columns, carrying three C rows and two mu
// rows in registers; lane 31 holds the column after the chunk, so east neighbours come
// from the next lane.  Fixed work split and order: deterministic.
template <typename T>
__device__ void band_partials_mu64(const DevView& v, const Tile& tl, int nx, int nr, const MemberParams& P,
                                   double2* slot, double* red) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const double a = P.a, bx = P.bx, by = P.by;
  // the stored field in FP64 (hi + lo for compensated members), read from global memory:
  // band row q of the tile is field row j0 - 2 + q (periodic)
  const T* Hg = static_cast<const T*>(v.C) + P.offset;
  const T* Lg = P.comp ? static_cast<const T*>(v.C) + P.lo_offset : nullptr;
  const int ny = P.ny;
  // field row of band row q (q from -1 to nr + 3, j0 - 3 .. j0 + nr + 1): one wrap at most
  auto at = [&](int q, int ii) {
    int j = tl.start - 2 + q;
    j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
    const int64_t k = (int64_t)j * nx + ii;
    return Lg ? (double)Hg[k] + (double)Lg[k] : (double)Hg[k];
  };
  const int nchunk = (nx + 30) / 31;
  const int nstrip = max(1, nwarps / nchunk);
  const int hs = (nr + nstrip - 1) / nstrip;
  // unscaled sums: (C^2 - 1)^2, (D+x C)^2, (D+y C)^2, (D+x mu)^2, (D+y mu)^2 (the grid
  // spacings and prefactors are applied once per thread at the end)
  double sw = 0.0, sdx = 0.0, sdy = 0.0, smx = 0.0, smy = 0.0;
  for (int item = warp; item < nchunk * nstrip; item += nwarps) {
    const int k = item % nchunk, r0 = (item / nchunk) * hs, r1 = min(nr, r0 + hs);
    if (r0 >= r1) continue;
    const int i = (31 * k + lane) % nx;
    const bool own = lane < 31 && 31 * k + lane < nx;
    const int iw = i == 0 ? nx - 1 : i - 1, ie = i + 1 == nx ? 0 : i + 1;
    // C at tile row q in FP64, and its west / east neighbours (shuffles inside the chunk)
    auto cload = [&](int q) { return at(q, i); };
    auto mu_row = [&](int q, double cq, double cdn, double cup) {
      double w = __shfl_up_sync(full, cq, 1), e = __shfl_down_sync(full, cq, 1);
      if (lane == 0) w = at(q, iw);
      if (lane == 31) e = at(q, ie);
      return cq * (cq * cq - a) - bx * (e + w) - by * (cup + cdn);
    };
    const int q0 = r0 + 2;
    double cm = cload(q0 - 1), c0 = cload(q0), c1 = cload(q0 + 1), c2 = cload(q0 + 2);
    double mu0 = mu_row(q0, c0, cm, c1);
    double mu1 = mu_row(q0 + 1, c1, c0, c2);
    for (int r = r0; r < r1; ++r) {
      const double ce = __shfl_down_sync(full, c0, 1);
      const double mue = __shfl_down_sync(full, mu0, 1);
      if (own) {
        const double w = c0 * c0 - 1.0, gx = ce - c0, gy = c1 - c0, mx = mue - mu0, my = mu1 - mu0;
        sw += w * w;
        sdx += gx * gx;
        sdy += gy * gy;
        smx += mx * mx;
        smy += my * my;
      }
      if (r + 1 < r1) {  // advance: row q+3 enters, mu of row q+2
        const double c3 = cload(r + 5);
        const double mu2 = mu_row(r + 4, c2, c1, c3);
        c0 = c1;
        c1 = c2;
        c2 = c3;
        mu0 = mu1;
        mu1 = mu2;
      }
    }
  }
  const double hxi2 = 1.0 / (P.hx * P.hx), hyi2 = 1.0 / (P.hy * P.hy);
  double sF = 0.25 * sw + 0.5 * P.gamma * (hxi2 * sdx + hyi2 * sdy);
  double sD = hxi2 * smx + hyi2 * smy;
  block_sum2(sF, sD, red);
  if (threadIdx.x == 0) *slot = make_double2(sF, sD);
}

// FP64 partial sums of the F and dF/dt densities over the band's nr rows (C tile rows
// 2..nr+1, mu rows 1..nr), reduced in fixed order; thread 0 stores them.
template <typename T>
__device__ __forceinline__ void band_partials(const DevView& v, const Tile& tl, const T* Cs, int lc, const T* Ms,
                                              int lm, int nx, int nr, const MemberParams& P, double2* slot,
                                              double* red, int seg = 0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  if (sizeof(T) == sizeof(float)) {
    band_partials_mu64<T>(v, tl, nx, nr, P, slot, red);
    return;
  }
  double sF = 0.0, sD = 0.0;
  const double hxi = 1.0 / P.hx, hyi = 1.0 / P.hy, hg = 0.5 * P.gamma;
  for (int r = warp; r < nr; r += nwarps) {
    const T* c0 = Cs + (size_t)(r + 2) * lc;
    const T* cp = c0 + lc;
    const T* m0 = Ms + (size_t)(r + 1) * lm;
    const T* mp = m0 + lm;
    for (int i = lane; i < nx; i += 32) {
      const int ie = (i + 1 == nx) ? 0 : i + 1;
      const double c = (double)c0[i];
      const double gx = ((double)c0[ie] - c) * hxi;
      const double gy = ((double)cp[i] - c) * hyi;
      const double w = c * c - 1.0;
      sF += 0.25 * w * w + hg * (gx * gx + gy * gy);
      double mu, mue, mun;
      if (sizeof(T) == sizeof(double)) {
        // mu tile index of point i (segment form: 16 bytes of padding per segment)
        const int pi = seg ? i + (16 / (int)sizeof(T)) * (i / seg) : i;
        const int pe = seg ? ie + (16 / (int)sizeof(T)) * (ie / seg) : ie;
        mu = (double)m0[pi];
        mue = (double)m0[pe];
        mun = (double)mp[pi];
      } else {
        mu = mu64_at(Cs, lc, r + 2, i, nx, P.a, P.bx, P.by);
        mue = mu64_at(Cs, lc, r + 2, ie, nx, P.a, P.bx, P.by);
        mun = mu64_at(Cs, lc, r + 3, i, nx, P.a, P.bx, P.by);
      }
      const double mx = (mue - mu) * hxi;
      const double my = (mun - mu) * hyi;
      sD += mx * mx + my * my;
    }
  }
  block_sum2(sF, sD, red);
  if (threadIdx.x == 0) *slot = make_double2(sF, sD);
}

// R' of one grid point from the mu tile (row pointer m0 = band row r + 1).
template <typename T>
__device__ __forceinline__ T rprime_at(const T* m0, int ld, int i, int nx, T rho, T w0) {
  const int ie = (i + 1 == nx) ? 0 : i + 1;
  const int iw = (i == 0) ? nx - 1 : i - 1;
  return fma(w0, m0[i], fma(rho, m0[i + ld] + m0[i - ld], m0[ie] + m0[iw]));
}

// Active flag and sample decision of a stencil-phase CTA.
__device__ __forceinline__ bool stencil_prologue(const Tile& tl, MemberState* st, const MemberParams& P, bool& sample) {
  const bool active = st->remaining > 0;
  if (tl.index == 0 && threadIdx.x == 0) st->active = active ? 1 : 0;
  sample = (st->step % P.every) == 0;
  return active;
}

__device__ __forceinline__ double* red_buffer(unsigned char* smem, size_t tile_bytes) {
  return reinterpret_cast<double*>(smem + ((tile_bytes + 15) & ~(size_t)15));
}

// The sample itself from the member's summed partials (sF, sD): F, dF/dt, beta, the series
// ring and the window average; then the step counter and horizon advance.
__device__ __forceinline__ void finalize_sums(const DevView& v, int member, MemberState* st, const MemberParams& P,
                                              double sF, double sD) {
  const int64_t n = st->step;
  if (n % P.every == 0) {
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
      double* s = v.series + ((size_t)member * P.series_cap + (size_t)(st->nsamples % P.series_cap)) * 4;
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

// Sample finalisation of one member (called once per member and step by the column phase,
// after the stencil phase wrote the band partials): the partials summed in band order, then
// finalize_sums.
__device__ __forceinline__ void finalize_sample(const DevView& v, int member, MemberState* st, const MemberParams& P) {
  double sF = 0.0, sD = 0.0;
  if (st->step % P.every == 0) {
    for (int b = 0; b < P.nbands; ++b) {
      const double2 pr = v.partials[P.partial_base + b];
      sF += pr.x;
      sD += pr.y;
    }
  }
  finalize_sums(v, member, st, P, sF, sD);
}

// -------------------------------------------------------------------------------------
// Fused row kernel: stencil + observables + row sweep for a band of rows of one member.
// Shared memory: Cs = (nr+4) rows of C (halo 2), Ms = (nr+2) rows of mu, pitch nx+1, then
// the FP64 reduction buffer.  Cs is reused for R' and then for W', Ms for the forward
// sweep output.
// -------------------------------------------------------------------------------------
template <typename T, bool OBS_ONLY>
__global__ void __launch_bounds__(512) rows_kernel(DevView v, int tile_base) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tile tl = v.row_tiles[tile_base + blockIdx.x];
  const MemberParams& P = v.mp[tl.member];
  MemberState* st = v.ms + tl.member;
  bool sample = true;
  if (!OBS_ONLY && !stencil_prologue(tl, st, P, sample)) return;
  const int nx = P.nx, ny = P.ny, j0 = tl.start, nr = tl.count;
  const int lc = ctile_pitch<T>(nx), lm = nx + 1, lr = nx + 1;
  // R' and the row sweep reuse the C tile's memory (pitch lr) once mu is known
  const size_t c_region = max((size_t)(nr + 4) * lc, (size_t)nr * lr);
  T* Cs = reinterpret_cast<T*>(smem);
  T* Ms = Cs + c_region;
  T* Rs = Cs;
  double* red = red_buffer(smem, (c_region + (size_t)(nr + 2) * lm) * sizeof(T));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

  load_rows_async<T>(Cs, lc, static_cast<const T*>(v.C) + P.offset, nx, ny, j0 - 2, nr + 4);
  cp_async_wait_all();
  __syncthreads();
  compute_mu<T>(Cs, lc, Ms, lm, nx, nr + 2, (T)P.a, (T)P.bx, (T)P.by);
  __syncthreads();
  if (sample) {
    band_partials<T>(v, tl, Cs, lc, Ms, lm, nx, nr, P, v.partials + P.partial_base + tl.index, red);
    __syncthreads();
  }
  if (OBS_ONLY) return;

  {
    const T rho = (T)P.rho, w0 = (T)P.w0;
    for (int r = warp; r < nr; r += nwarps) {
      const T* m0 = Ms + (size_t)(r + 1) * lm;
      T* out = Rs + (size_t)r * lr;
      for (int i = lane; i < nx; i += 32) out[i] = rprime_at<T>(m0, lm, i, nx, rho, w0);
    }
  }
  __syncthreads();

  // Row sweep: rows_p threads per row, each owning a chunk of the row.
  const int sweep_p = P.rows_p;
  const int nsweep = nr * sweep_p;
  const int chunk = (nx + sweep_p - 1) / sweep_p;
  const int row = threadIdx.x % nr;
  const int c0 = (threadIdx.x / nr) * chunk;
  const int c1 = min(nx, c0 + chunk);
  const bool sweeper = threadIdx.x < nsweep && c0 < c1;
  const T p1 = (T)P.p1x, p2 = (T)P.p2x;
  if (sweep_p == 1) {
    if (sweeper) line_sweep_inplace<T>(Rs + (size_t)row * lr, 1, nx, P.kx, p1, p2);
  } else {
    chunk_sweep_inplace<T>(Rs + (size_t)row * lr, 1, nx, c0, c1, P.kx, p1, p2, sweeper);
  }
  __syncthreads();

  {
    T* __restrict__ W = static_cast<T*>(v.W) + P.offset;
    for (int r = warp; r < nr; r += nwarps) {
      const T* src = Rs + (size_t)r * lr;
      T* dst = W + (int64_t)(j0 + r) * nx;
      for (int i = lane; i < nx; i += 32) dst[i] = src[i];
    }
  }
}

// -------------------------------------------------------------------------------------
// Segment form of the fused row kernel (see the top of this file).
// -------------------------------------------------------------------------------------
constexpr unsigned kFull = 0xffffffffu;

// Padding after every segment of the mu tile: 16 bytes, so that the 16-byte segment reads
// of 8 consecutive lanes fall in distinct banks.
template <typename T>
__device__ __forceinline__ constexpr int seg_pad() { return 16 / (int)sizeof(T); }

template <typename T, int S>
__device__ __forceinline__ int seg_addr(int i) { return i + seg_pad<T>() * (i / S); }

// A member constant in the kernel's precision (FP32 kernels read the pre-rounded copy).
template <typename T>
__device__ __forceinline__ T pick(double d, float f);
template <>
__device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float pick<float>(double, float f) { return f; }

// C update of one point, C <- C + kappa z.  For compensated FP32 members the field is the
// pair hi + lo (lo at the same index of the member's lo block): Fast2Sum (|hi| >= |d|)
// keeps the rounding error of the new hi in lo, so the rounding of the stored field does
// not accumulate in the weakly damped modes.  lo is null otherwise.
template <typename T>
__device__ __forceinline__ T c_update(T c, T kap, T z, T* lo) {
  if (sizeof(T) == 4 && lo) {
    const T d = kap * z + *lo;
    const T s = c + d;
    *lo = d - (s - c);
    return s;
  }
  return fma(kap, z, c);
}

// The lo block of member P at element index i of its field, or null (plain update).
template <typename T>
__device__ __forceinline__ T* lo_ptr(const DevView& v, const MemberParams& P, int64_t i) {
  return (sizeof(T) == 4 && P.comp) ? static_cast<T*>(v.C) + P.lo_offset + i : nullptr;
}

// 4 consecutive elements (16-byte aligned for float, 32-byte for double).
__device__ __forceinline__ void ld4(const float* p, float* v) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  v[0] = q.x;
  v[1] = q.y;
  v[2] = q.z;
  v[3] = q.w;
}
__device__ __forceinline__ void ld4(const double* p, double* v) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, const float* v) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* p, const double* v) {
  *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2*>(p + 2) = make_double2(v[2], v[3]);
}

// One recurrence over a row held as segments: y (S values of this lane) in, solution out.
// REV = false: y_i = r_i + p1 y_{i-1} + p2 y_{i-2} (increasing i); REV = true: the same
// recurrence for decreasing i.  G lanes (a power of two, lg = log2 G) hold the row, lane
// l the points [l S, l S + S); Ks = the scan constants A[0..4] (M^(S 2^d)) then P
// ((I - M^n)^-1); B = M^(S pos), pos = the lane's place in the recurrence's order.  Every
// lane of the warp must call it (full-warp shuffles, width G).
template <typename T, int S, int R, bool REV>
__device__ __forceinline__ void seg_sweep(T (&y)[R][S], T p1, T p2, int l, int G, int lg, const T* Ks,
                                          const T (&B)[4]) {
  // R rows at once, each stage interleaved over the rows (independent chains)
  T a[R], b[R];
#pragma unroll
  for (int t = 0; t < R; ++t) a[t] = b[t] = T(0);
#pragma unroll
  for (int k = 0; k < S; ++k) {
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const T v = fma(p1, a[t], fma(p2, b[t], y[t][REV ? S - 1 - k : k]));
      b[t] = a[t];
      a[t] = v;
    }
  }
  const int pos = REV ? G - 1 - l : l;
#pragma unroll
  for (int d = 0; d < 5; ++d) {
    if (d < lg) {
      const int delta = 1 << d;
      T A[4];
      ld4(Ks + 4 * d, A);
#pragma unroll
      for (int t = 0; t < R; ++t) {
        const T ya = REV ? __shfl_down_sync(kFull, a[t], delta, G) : __shfl_up_sync(kFull, a[t], delta, G);
        const T yb = REV ? __shfl_down_sync(kFull, b[t], delta, G) : __shfl_up_sync(kFull, b[t], delta, G);
        if (pos >= delta) {
          const T na = fma(A[0], ya, fma(A[1], yb, a[t]));
          b[t] = fma(A[2], ya, fma(A[3], yb, b[t]));
          a[t] = na;
        }
      }
    }
  }
  const int last = REV ? 0 : G - 1;
  T Pm[4];
  ld4(Ks + 20, Pm);
#pragma unroll
  for (int t = 0; t < R; ++t) {
    const T Ea = __shfl_sync(kFull, a[t], last, G), Eb = __shfl_sync(kFull, b[t], last, G);
    const T xa = fma(Pm[0], Ea, Pm[1] * Eb), xb = fma(Pm[2], Ea, Pm[3] * Eb);
    T pa = REV ? __shfl_down_sync(kFull, a[t], 1, G) : __shfl_up_sync(kFull, a[t], 1, G);
    T pb = REV ? __shfl_down_sync(kFull, b[t], 1, G) : __shfl_up_sync(kFull, b[t], 1, G);
    if (pos == 0) {
      pa = T(0);
      pb = T(0);
    }
    a[t] = fma(B[0], xa, fma(B[1], xb, pa));
    b[t] = fma(B[2], xa, fma(B[3], xb, pb));
  }
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const int u = REV ? S - 1 - k : k;
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const T v = fma(p1, a[t], fma(p2, b[t], y[t][u]));
      y[t][u] = v;
      b[t] = a[t];
      a[t] = v;
    }
  }
}

// Segment-form row work of one band (tile tl of member P) whose C rows j0-2 .. j0+nr+1
// are in Cs (dense pitch nx): mu tile Ms (nr+2 rows, pitch nx + 16 bytes per segment), the
// sample partials, then R' in registers, the forward and backward recurrences and W
// stored with 16-byte writes.  Ks holds the member's 24 scan constants.  mu is computed 4
// points per thread from 16-byte tile reads; each row is then taken by a group of G lanes.
// Called by every thread of the CTA; contains barriers.
template <typename T, int S>
__device__ __forceinline__ void seg_tile(const DevView& v, const Tile& tl, const MemberParams& P, const T* Cs, T* Ms,
                                         const T* Ks, double* red, bool sample) {
  const int nx = P.nx, j0 = tl.start, nr = tl.count;
  const int lmp = nx + seg_pad<T>() * (nx / S);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

  // mu tile: Ms row r <- C tile row r + 1, 4 points per thread; a row's chunks are taken
  // by cs consecutive lanes (cs = min(32, nx/4), a power of two), the chunk neighbours
  // coming from the adjacent lanes except at the ends of a lane run.
  {
    const T a = pick<T>(P.a, P.fa), bx = pick<T>(P.bx, P.fbx), by = pick<T>(P.by, P.fby);
    const int nq = nx >> 2;
    const int cs = nq < 32 ? nq : 32;
    const int rpp = 32 / cs;
    const int sub = lane / cs, ql = lane - sub * cs;
    for (int rb = warp * rpp; rb < nr + 2; rb += nwarps * rpp) {
      const int r = rb + sub;
      const bool rv = r < nr + 2;
      const int rr = rv ? r : nr + 1;
      const T* c0 = Cs + (size_t)(rr + 1) * nx;
      T* mrow = Ms + (size_t)rr * lmp;
      for (int q0 = 0; q0 < nq; q0 += cs) {
        const int i = (q0 + ql) << 2;
        T c[4], n[4], so[4];
        ld4(c0 + i, c);
        ld4(c0 - nx + i, n);
        ld4(c0 + nx + i, so);
        T w = __shfl_up_sync(kFull, c[3], 1);
        T e = __shfl_down_sync(kFull, c[0], 1);
        if (ql == 0) w = c0[i == 0 ? nx - 1 : i - 1];
        if (ql == cs - 1) e = c0[i + 4 == nx ? 0 : i + 4];
        T out[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const T ce = k < 3 ? c[k + 1] : e;
          const T cw = k > 0 ? c[k - 1] : w;
          const T u = c[k] * fma(c[k], c[k], -a);
          out[k] = fma(-by, so[k] + n[k], fma(-bx, ce + cw, u));
        }
        if (rv) st4(mrow + seg_addr<T, S>(i), out);
      }
    }
  }
  __syncthreads();
  if (sample) {
    band_partials<T>(v, tl, Cs, nx, Ms, lmp, nx, nr, P, v.partials + P.partial_base + tl.index, red, S);
    __syncthreads();
  }

  // rows: G lanes per row, groups of one warp take rows round-robin
  const SegTable& tab = v.seg[tl.member];
  const int G = P.seg_g;
  const int lg = __ffs(G) - 1;
  const int gpw = 32 / G, ngroups = nwarps * gpw;
  const int l = lane & (G - 1), grp = warp * gpw + (lane >> lg);
  T Bf[4], Bb[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    Bf[k] = pick<T>(tab.B[l][k], tab.Bf[l][k]);
    Bb[k] = pick<T>(tab.B[G - 1 - l][k], tab.Bf[G - 1 - l][k]);
  }
  const T p1 = pick<T>(P.p1x, P.fp1x), p2 = pick<T>(P.p2x, P.fp2x), rho = pick<T>(P.rho, P.frho),
          w0 = pick<T>(P.w0, P.fw0);
  T* __restrict__ W = static_cast<T*>(v.W) + P.offset;
  // FP32 with 16-point segments: two rows per group, their chains interleaved
  constexpr int R = 1;  // rows per group (2 measured slower: fewer CTAs per SM)
  const int rounds = (nr + R * ngroups - 1) / (R * ngroups);
  for (int k = 0; k < rounds; ++k) {
    T m[R][S];
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int r = (k * ngroups + grp) * R + t;
      const T* mrow = Ms + (size_t)((r < nr ? r : nr - 1) + 1) * lmp + l * (S + seg_pad<T>());
#pragma unroll
      for (int c = 0; c < S / 4; ++c) ld4(mrow + 4 * c, &m[t][4 * c]);
      const T left = __shfl_sync(kFull, m[t][S - 1], (l + G - 1) & (G - 1), G);
      const T right = __shfl_sync(kFull, m[t][0], (l + 1) & (G - 1), G);
      T prev = left;
#pragma unroll
      for (int c = 0; c < S / 4; ++c) {
        T up[4], dn[4];
        ld4(mrow - lmp + 4 * c, up);
        ld4(mrow + lmp + 4 * c, dn);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int u = 4 * c + q;
          const T cur = m[t][u];
          const T e = u + 1 < S ? m[t][u + 1] : right;
          m[t][u] = fma(w0, cur, fma(rho, dn[q] + up[q], e + prev));
          prev = cur;
        }
      }
    }
    seg_sweep<T, S, R, false>(m, p1, p2, l, G, lg, Ks, Bf);
    seg_sweep<T, S, R, true>(m, p1, p2, l, G, lg, Ks, Bb);
#pragma unroll
    for (int t = 0; t < R; ++t) {
      const int r = (k * ngroups + grp) * R + t;
      if (r < nr) {
        T* dst = W + (int64_t)(j0 + r) * nx + l * S;
#pragma unroll
        for (int c = 0; c < S / 4; ++c) st4(dst + 4 * c, &m[t][4 * c]);
      }
    }
  }
}

// -------------------------------------------------------------------------------------
// Fused row kernel, transposed-block form: a band of up to 32 rows (j0 .. j0+31) of one
// member with nx = 32 nw (nw <= 16); warp w owns the columns [32 w, 32 w + 32).  With
// lane = column the stencil walks down the band (C as coalesced 128-byte row pieces
// straight from HBM, x neighbours by shuffles, y neighbours in registers); the warp's
// 32 x 32 block of R' is then transposed through shared memory so that lane = row, each
// lane runs the row recurrences over its 32 columns, and the nw segments of a row are
// joined through shared memory (local pass, sequential combination of the segment end
// states, periodic start state, second pass).  W goes back through the transpose and out
// as coalesced row pieces.  On sample steps the FP64 F and dF/dt densities are summed
// with backward differences (the periodic sums are the same).
// -------------------------------------------------------------------------------------
template <typename T, bool REV>
__device__ __forceinline__ void rowT_pass(T (&x)[32], T p1, T p2, const SegTable& tab, T* xs, int warp, int lane,
                                          int nw) {
  T a = T(0), b = T(0);
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const T t = fma(p1, a, fma(p2, b, x[REV ? 31 - k : k]));
    b = a;
    a = t;
  }
  xs[2 * (warp * 32 + lane)] = a;
  xs[2 * (warp * 32 + lane) + 1] = b;
  __syncthreads();
  const T A0 = pick<T>(tab.A[0][0], tab.Af[0][0]), A1 = pick<T>(tab.A[0][1], tab.Af[0][1]);
  const T A2 = pick<T>(tab.A[0][2], tab.Af[0][2]), A3 = pick<T>(tab.A[0][3], tab.Af[0][3]);
  const int pos = REV ? nw - 1 - warp : warp;
  T ya = T(0), yb = T(0), pa = T(0), pb = T(0);
  for (int k = 0; k < nw; ++k) {
    const int w = REV ? nw - 1 - k : k;
    const T ea = xs[2 * (w * 32 + lane)], eb = xs[2 * (w * 32 + lane) + 1];
    const T na = fma(A0, ya, fma(A1, yb, ea));
    yb = fma(A2, ya, fma(A3, yb, eb));
    ya = na;
    if (k + 1 == pos) {
      pa = ya;
      pb = yb;
    }
  }
  const T P0 = pick<T>(tab.P[0], tab.Pf[0]), P1 = pick<T>(tab.P[1], tab.Pf[1]);
  const T P2 = pick<T>(tab.P[2], tab.Pf[2]), P3 = pick<T>(tab.P[3], tab.Pf[3]);
  const T xa = fma(P0, ya, P1 * yb), xb = fma(P2, ya, P3 * yb);
  const T B0 = pick<T>(tab.B[pos][0], tab.Bf[pos][0]), B1 = pick<T>(tab.B[pos][1], tab.Bf[pos][1]);
  const T B2 = pick<T>(tab.B[pos][2], tab.Bf[pos][2]), B3 = pick<T>(tab.B[pos][3], tab.Bf[pos][3]);
  a = fma(B0, xa, fma(B1, xb, pa));
  b = fma(B2, xa, fma(B3, xb, pb));
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    const int u = REV ? 31 - k : k;
    const T t = fma(p1, a, fma(p2, b, x[u]));
    x[u] = t;
    b = a;
    a = t;
  }
}

// Sample step of rowsT_kernel: FP64 partial sums of the F and dF/dt densities of the band
// rows at column i, mu recomputed in FP64 from the stored field, backward differences
// (the periodic sums equal those of forward differences); a second walk down the band.
template <typename T>
__device__ __noinline__ void rowT_partials(const DevView& v, const Tile& tl, const MemberParams& P, const T* Cm,
                                           double* red, int i, int iw, int ie, int lane) {
  const unsigned full = 0xffffffffu;
  const int nx = P.nx, ny = P.ny, nr = tl.count;
  const double a = P.a, bx = P.bx, by = P.by;
  const int iww = iw == 0 ? nx - 1 : iw - 1;
  const int64_t dlo = P.comp ? P.lo_offset - P.offset : 0;  // lo block relative to hi
  auto val = [&](const T* r, int ii) { return P.comp ? (double)r[ii] + (double)r[dlo + ii] : (double)r[ii]; };
  int jn = tl.start - 2;
  if (jn < 0) jn += ny;
  const T* r0 = Cm + (int64_t)jn * nx;
  if (++jn == ny) jn = 0;
  const T* r1 = Cm + (int64_t)jn * nx;
  double sw = 0.0, sdx = 0.0, sdy = 0.0, smx = 0.0, smy = 0.0, mu_prev = 0.0;
  for (int q = 0; q <= nr; ++q) {  // mu rows j0-1 .. j0+nr-1
    if (++jn == ny) jn = 0;
    const T* r2 = Cm + (int64_t)jn * nx;
    const double cd = val(r1, i), cs = val(r0, i), cn = val(r2, i);
    double w = __shfl_up_sync(full, cd, 1), e = __shfl_down_sync(full, cd, 1);
    if (lane == 0) w = val(r1, iw);
    if (lane == 31) e = val(r1, ie);
    const double mu = cd * (cd * cd - a) - bx * (e + w) - by * (cn + cs);
    double muw = __shfl_up_sync(full, mu, 1);
    if (lane == 0) muw = w * (w * w - a) - bx * (cd + val(r1, iww)) - by * (val(r2, iw) + val(r0, iw));
    if (q >= 1) {
      const double gx = cd - w, gy = cd - cs, wv = cd * cd - 1.0, mx = mu - muw, my = mu - mu_prev;
      sw += wv * wv;
      sdx += gx * gx;
      sdy += gy * gy;
      smx += mx * mx;
      smy += my * my;
    }
    mu_prev = mu;
    r0 = r1;
    r1 = r2;
  }
  const double hxi2 = 1.0 / (P.hx * P.hx), hyi2 = 1.0 / (P.hy * P.hy);
  double sF = 0.25 * sw + 0.5 * P.gamma * (hxi2 * sdx + hyi2 * sdy);
  double sD = hxi2 * smx + hyi2 * smy;
  block_sum2(sF, sD, red);
  if (threadIdx.x == 0) v.partials[P.partial_base + tl.index] = make_double2(sF, sD);
}

// Shared memory (elements of T): nw transpose tiles of 32 x 33, the mu edge columns
// (nw x 2 x 34), the segment end states (2 directions x nw x 64), then the FP64
// reduction buffer.
template <typename T>
__global__ void __launch_bounds__(512) rowsT_kernel(DevView v, int tile_base) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned full = 0xffffffffu;
  const Tile tl = v.row_tiles[tile_base + blockIdx.x];
  const MemberParams& P = v.mp[tl.member];
  MemberState* st = v.ms + tl.member;
  if (st->remaining <= 0) {
    if (tl.index == 0 && threadIdx.x == 0) st->active = 0;
    return;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nx = P.nx, ny = P.ny, j0 = tl.start, nr = tl.count;
  T* tile = reinterpret_cast<T*>(smem) + warp * 32 * 33;
  T* edge = reinterpret_cast<T*>(smem) + nw * 32 * 33;  // [w][side][34]: C halo columns, then mu edges
  T* xch = edge + nw * 68;                              // [dir][w][32][2]
  double* red = red_buffer(smem, ((size_t)nw * 32 * 33 + nw * 68 + 2 * nw * 64) * sizeof(T));
  int smp = 0;
  if (lane == 0) smp = (st->step % P.every) == 0;
  smp = __shfl_sync(full, smp, 0);
  if (threadIdx.x == 0 && tl.index == 0) st->active = 1;

  const int i = 32 * warp + lane;
  const int iw = i == 0 ? nx - 1 : i - 1, ie = i + 1 == nx ? 0 : i + 1;
  const T* __restrict__ Cm = static_cast<const T*>(v.C) + P.offset;
  // the 36 rows j0-2 .. j0+33 (periodic in j) at column i, all loads issued before use;
  // the halo columns of this warp's block (left of lane 0, right of lane 31) for rows
  // j0-1 .. j0+32 go through shared memory, 68 loads spread over the lanes
  int jb = j0 - 2;
  if (jb < 0) jb += ny;
  T m[36];
  {
    int jn = jb;
#pragma unroll
    for (int q = 0; q < 36; ++q) {
      m[q] = Cm[(int64_t)jn * nx + i];
      if (++jn == ny) jn = 0;
    }
    T* halo = edge + warp * 68;
    const int hl = 32 * warp == 0 ? nx - 1 : 32 * warp - 1, hr = 32 * warp + 32 == nx ? 0 : 32 * warp + 32;
    for (int k = lane; k < 68; k += 32) {
      const int q = k < 34 ? k : k - 34;
      const int j = (jb + 1 + q) % ny;
      halo[k] = Cm[(int64_t)j * nx + (k < 34 ? hl : hr)];
    }
    __syncwarp();
    const T a = pick<T>(P.a, P.fa), bx = pick<T>(P.bx, P.fbx), by = pick<T>(P.by, P.fby);
    // mu of row j0-1+q into m[q] (in place: row q of C is not needed after it)
#pragma unroll
    for (int q = 0; q < 34; ++q) {
      const T c1 = m[q + 1];
      T w = __shfl_up_sync(full, c1, 1), e = __shfl_down_sync(full, c1, 1);
      if (lane == 0) w = halo[q];
      if (lane == 31) e = halo[34 + q];
      m[q] = fma(-by, m[q + 2] + m[q], fma(-bx, e + w, c1 * fma(c1, c1, -a)));
    }
    __syncwarp();
    if (lane == 0 || lane == 31) {
#pragma unroll
      for (int q = 0; q < 34; ++q) halo[(lane == 31) * 34 + q] = m[q];
    }
  }
  __syncthreads();
  // R' in place: m[q] <- R' of band row q (mu rows q, q+1, q+2)
  {
    const T rho = pick<T>(P.rho, P.frho), w0 = pick<T>(P.w0, P.fw0);
    const T* eleft = edge + (((warp + nw - 1) % nw) * 2 + 1) * 34;  // lane 31 of the warp on the left
    const T* eright = edge + (((warp + 1) % nw) * 2) * 34;          // lane 0 of the warp on the right
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      T w = __shfl_up_sync(full, m[q + 1], 1), e = __shfl_down_sync(full, m[q + 1], 1);
      if (lane == 0) w = eleft[q + 1];
      if (lane == 31) e = eright[q + 1];
      m[q] = fma(w0, m[q + 1], fma(rho, m[q + 2] + m[q], e + w));
    }
  }
  // transpose: lane r takes band row r's 32 columns of this warp
#pragma unroll
  for (int q = 0; q < 32; ++q) tile[q * 33 + lane] = m[q];
  __syncwarp();
  T x[32];
#pragma unroll
  for (int c = 0; c < 32; ++c) x[c] = tile[lane * 33 + c];
  const SegTable& tab = v.seg[tl.member];
  const T p1 = pick<T>(P.p1x, P.fp1x), p2 = pick<T>(P.p2x, P.fp2x);
  rowT_pass<T, false>(x, p1, p2, tab, xch, warp, lane, nw);
  rowT_pass<T, true>(x, p1, p2, tab, xch + nw * 64, warp, lane, nw);
  // transpose back and store W as row pieces
#pragma unroll
  for (int c = 0; c < 32; ++c) tile[lane * 33 + c] = x[c];
  __syncwarp();
  T* __restrict__ Wm = static_cast<T*>(v.W) + P.offset + i;
  for (int q = 0; q < nr; ++q) Wm[(int64_t)(j0 + q) * nx] = tile[q * 33 + lane];
  if (smp) rowT_partials<T>(v, tl, P, Cm, red, i, iw, ie, lane);
}

// Next tile at or after t (stride gridDim.x) whose member still steps; tiles of finished
// members are skipped, their band-0 CTA clearing the member's active flag.
__device__ __forceinline__ int next_active_tile(const DevView& v, int base, int t, int ntiles) {
  while (t < ntiles) {
    const Tile tl = v.row_tiles[base + t];
    MemberState* st = v.ms + tl.member;
    if (st->remaining > 0) return t;
    if (tl.index == 0 && threadIdx.x == 0) st->active = 0;
    t += gridDim.x;
  }
  return t;
}

// Per-tile set-up by the CTA: thread 0 marks the member active and decides the sample,
// threads 0..23 load the scan constants (visible after the caller's barrier).
template <typename T>
__device__ __forceinline__ void seg_tile_setup(const DevView& v, const Tile& tl, const MemberParams& P, T* Ks,
                                               int* s_sample) {
  if (threadIdx.x == 0) {
    MemberState* st = v.ms + tl.member;
    if (tl.index == 0) st->active = 1;
    *s_sample = (st->step % P.every) == 0;
  }
  if (threadIdx.x < 24) {
    const SegTable& tab = v.seg[tl.member];
    Ks[threadIdx.x] = threadIdx.x < 20
                          ? pick<T>(tab.A[threadIdx.x >> 2][threadIdx.x & 3], tab.Af[threadIdx.x >> 2][threadIdx.x & 3])
                          : pick<T>(tab.P[threadIdx.x - 20], tab.Pf[threadIdx.x - 20]);
  }
}

// Fused row kernel, segment form (nx = G S, G a power of two <= 32, rows in 16-byte
// pieces; at most 256 threads).  Shared memory: C tile buffer(s) of ccap elements (two
// when PERSIST), the mu tile (mcap elements), the 24 scan constants and the sample flag
// (28 T), then the FP64 reduction buffer.  PERSIST: a CTA walks the tiles blockIdx.x,
// + gridDim.x, ... and copies the next tile's C band while it computes the current one.
template <typename T, int S, bool PERSIST>
__global__ void __launch_bounds__(256) rows_seg_kernel(DevView v, int base, int ntiles, int ccap, int mcap) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* Cbuf = reinterpret_cast<T*>(smem);
  T* Ms = Cbuf + (size_t)(PERSIST ? 2 : 1) * ccap;
  T* Ks = Ms + mcap;
  int* s_sample = reinterpret_cast<int*>(Ks + 24);
  double* red = red_buffer(smem, ((size_t)(PERSIST ? 2 : 1) * ccap + mcap + 28) * sizeof(T));
  auto issue = [&](int t, T* dst) {
    const Tile tl = v.row_tiles[base + t];
    const MemberParams& P = v.mp[tl.member];
    load_rows_async<T>(dst, P.nx, static_cast<const T*>(v.C) + P.offset, P.nx, P.ny, tl.start - 2, tl.count + 4);
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  int t = next_active_tile(v, base, blockIdx.x, PERSIST ? ntiles : blockIdx.x + 1);
  if (t >= ntiles || (!PERSIST && t != (int)blockIdx.x)) return;
  issue(t, Cbuf);
  int cur = 0;
  while (t < ntiles) {
    const int nt = PERSIST ? next_active_tile(v, base, t + gridDim.x, ntiles) : ntiles;
    if (PERSIST && nt < ntiles) {
      issue(nt, Cbuf + (size_t)(cur ^ 1) * ccap);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    const Tile tl = v.row_tiles[base + t];
    const MemberParams& P = v.mp[tl.member];
    seg_tile_setup<T>(v, tl, P, Ks, s_sample);
    __syncthreads();
    seg_tile<T, S>(v, tl, P, Cbuf + (size_t)cur * ccap, Ms, Ks, red, *s_sample != 0);
    __syncthreads();  // the mu tile, constants and this C buffer are free again
    t = nt;
    cur ^= 1;
  }
}

// -------------------------------------------------------------------------------------
// Split form, kernel 1: stencil + observables of a band, R' written to the W scratch.
// -------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) stencil_kernel(DevView v, int tile_base) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tile tl = v.row_tiles[tile_base + blockIdx.x];
  const MemberParams& P = v.mp[tl.member];
  MemberState* st = v.ms + tl.member;
  bool sample = true;
  if (!stencil_prologue(tl, st, P, sample)) return;
  const int nx = P.nx, ny = P.ny, j0 = tl.start, nr = tl.count;
  const int lc = ctile_pitch<T>(nx), lm = nx + 1;
  T* Cs = reinterpret_cast<T*>(smem);
  T* Ms = Cs + (size_t)(nr + 4) * lc;
  double* red = red_buffer(smem, ((size_t)(nr + 4) * lc + (size_t)(nr + 2) * lm) * sizeof(T));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;

  load_rows_async<T>(Cs, lc, static_cast<const T*>(v.C) + P.offset, nx, ny, j0 - 2, nr + 4);
  cp_async_wait_all();
  __syncthreads();
  compute_mu<T>(Cs, lc, Ms, lm, nx, nr + 2, (T)P.a, (T)P.bx, (T)P.by);
  __syncthreads();
  if (sample) band_partials<T>(v, tl, Cs, lc, Ms, lm, nx, nr, P, v.partials + P.partial_base + tl.index, red);

  T* __restrict__ W = static_cast<T*>(v.W) + P.offset;
  const T rho = (T)P.rho, w0 = (T)P.w0;
  for (int r = warp; r < nr; r += nwarps) {
    const T* m0 = Ms + (size_t)(r + 1) * lm;
    T* dst = W + (int64_t)(j0 + r) * nx;
    for (int i = lane; i < nx; i += 32) dst[i] = rprime_at<T>(m0, lm, i, nx, rho, w0);
  }
}

// -------------------------------------------------------------------------------------
// Split form, kernel 1 for rows too long for a shared-memory band (FP64): the same
// stencil on a block of nr rows x nc columns.  C is staged with a 2-point halo on every
// side (periodic, both axes), mu on a 1-point halo; mu and R' are formed in exactly the
// operation order of compute_mu and rprime_at, so W equals the whole-row kernel's bit for
// bit.  Each block writes its own partial slot (index = band x blocks per band + block).
// OBS: observables of the current field only (partials, no W, no step state), the block
// counterpart of rows_kernel<T, true> for ch_observables.
// Shared memory: Cs (nr+4) x (nc+4), Ms (nr+2) x (nc+2), then the FP64 reduction buffer.
// -------------------------------------------------------------------------------------
template <typename T, bool OBS>
__global__ void __launch_bounds__(512) stencil_block_kernel(DevView v, int tile_base) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tile tl = v.row_tiles[tile_base + blockIdx.x];
  const MemberParams& P = v.mp[tl.member];
  MemberState* st = v.ms + tl.member;
  bool sample = true;
  if (!OBS && !stencil_prologue(tl, st, P, sample)) return;
  const int nx = P.nx, ny = P.ny, j0 = tl.start, nr = tl.count, i0 = tl.x0, nc = tl.xn;
  const int lc = nc + 4, lm = nc + 2;
  T* Cs = reinterpret_cast<T*>(smem);
  T* Ms = Cs + (size_t)(nr + 4) * lc;
  double* red = red_buffer(smem, ((size_t)(nr + 4) * lc + (size_t)(nr + 2) * lm) * sizeof(T));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const T* Cg = static_cast<const T*>(v.C) + P.offset;
  // rows j0-2 .. j0+nr+1 and columns i0-2 .. i0+nc+1, one wrap at most (nx, ny >= 5)
  for (int r = warp; r < nr + 4; r += nwarps) {
    int j = j0 - 2 + r;
    j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
    const T* src = Cg + (int64_t)j * nx;
    T* dst = Cs + (size_t)r * lc;
    for (int c = lane; c < lc; c += 32) {
      int i = i0 - 2 + c;
      i = i < 0 ? i + nx : (i >= nx ? i - nx : i);
      dst[c] = src[i];
    }
  }
  __syncthreads();
  const T a = (T)P.a, bx = (T)P.bx, by = (T)P.by;
  for (int r = warp; r < nr + 2; r += nwarps) {
    const T* c0 = Cs + (size_t)(r + 1) * lc + 1;
    const T* cm = c0 - lc;
    const T* cp = c0 + lc;
    T* mrow = Ms + (size_t)r * lm;
    for (int c = lane; c < nc + 2; c += 32) {
      const T x = c0[c];
      const T u = x * fma(x, x, -a);
      mrow[c] = fma(-by, cp[c] + cm[c], fma(-bx, c0[c + 1] + c0[c - 1], u));
    }
  }
  __syncthreads();
  if (sample) {
    double sF = 0.0, sD = 0.0;
    const double hxi = 1.0 / P.hx, hyi = 1.0 / P.hy, hg = 0.5 * P.gamma;
    for (int r = warp; r < nr; r += nwarps) {
      const T* c0 = Cs + (size_t)(r + 2) * lc + 2;
      const T* m0 = Ms + (size_t)(r + 1) * lm + 1;
      for (int c = lane; c < nc; c += 32) {
        const double x = (double)c0[c];
        const double gx = ((double)c0[c + 1] - x) * hxi;
        const double gy = ((double)c0[c + lc] - x) * hyi;
        const double w = x * x - 1.0;
        sF += 0.25 * w * w + hg * (gx * gx + gy * gy);
        const double mu = (double)m0[c];
        const double mx = ((double)m0[c + 1] - mu) * hxi;
        const double my = ((double)m0[c + lm] - mu) * hyi;
        sD += mx * mx + my * my;
      }
    }
    block_sum2(sF, sD, red);
    if (threadIdx.x == 0) v.partials[P.partial_base + tl.index] = make_double2(sF, sD);
  }
  if (OBS) return;
  T* __restrict__ W = static_cast<T*>(v.W) + P.offset;
  const T rho = (T)P.rho, w0 = (T)P.w0;
  for (int r = warp; r < nr; r += nwarps) {
    const T* m0 = Ms + (size_t)(r + 1) * lm + 1;
    T* dst = W + (int64_t)(j0 + r) * nx + i0;
    for (int c = lane; c < nc; c += 32)
      dst[c] = fma(w0, m0[c], fma(rho, m0[c + lm] + m0[c - lm], m0[c + 1] + m0[c - 1]));
  }
}

// -------------------------------------------------------------------------------------
// Split form, kernel 2: row sweep of a band of rows, one thread per row, in place in
// shared memory (pitch nx+1).
// -------------------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(512) rowsweep_kernel(DevView v, int tile_base) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tile tl = v.sweep_tiles[tile_base + blockIdx.x];
  if (!v.ms[tl.member].active) return;
  const MemberParams& P = v.mp[tl.member];
  const int nx = P.nx, j0 = tl.start, nr = tl.count;
  const int ld = nx + 1;
  T* Bs = reinterpret_cast<T*>(smem);
  T* W = static_cast<T*>(v.W) + P.offset;
  load_rows_async<T>(Bs, ld, W, nx, P.ny, j0, nr);
  cp_async_wait_all();
  __syncthreads();
  if (threadIdx.x < nr) line_sweep_inplace<T>(Bs + (size_t)threadIdx.x * ld, 1, nx, P.kx, (T)P.p1x, (T)P.p2x);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int r = warp; r < nr; r += nwarps) {
    const T* src = Bs + (size_t)r * ld;
    T* dst = W + (int64_t)(j0 + r) * nx;
    for (int i = lane; i < nx; i += 32) dst[i] = src[i];
  }
}

// -------------------------------------------------------------------------------------
// Split form, kernel 2, segment form: the row recurrences of R' (held in W) for a band of
// rows, each row in the registers of G = nx / S lanes (S consecutive points per lane,
// 16-byte loads and stores straight from HBM), solved by segment scans (top of this
// file); W' written back in place.  No shared-memory tiles, one barrier at set-up.
// -------------------------------------------------------------------------------------
template <typename T, int S>
__global__ void __launch_bounds__(256) rowseg_kernel(DevView v, int tile_base) {
  __shared__ __align__(16) T Ks[24];
  const Tile tl = v.sweep_tiles[tile_base + blockIdx.x];
  if (!v.ms[tl.member].active) return;
  const MemberParams& P = v.mp[tl.member];
  const SegTable& tab = v.seg[tl.member];
  if (threadIdx.x < 24)
    Ks[threadIdx.x] = threadIdx.x < 20
                          ? pick<T>(tab.A[threadIdx.x >> 2][threadIdx.x & 3], tab.Af[threadIdx.x >> 2][threadIdx.x & 3])
                          : pick<T>(tab.P[threadIdx.x - 20], tab.Pf[threadIdx.x - 20]);
  __syncthreads();
  const int nx = P.nx, j0 = tl.start, nr = tl.count;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int G = P.seg_g;
  const int lg = __ffs(G) - 1;
  const int gpw = 32 / G, ngroups = nwarps * gpw;
  const int l = lane & (G - 1), grp = warp * gpw + (lane >> lg);
  T Bf[4], Bb[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    Bf[k] = pick<T>(tab.B[l][k], tab.Bf[l][k]);
    Bb[k] = pick<T>(tab.B[G - 1 - l][k], tab.Bf[G - 1 - l][k]);
  }
  const T p1 = pick<T>(P.p1x, P.fp1x), p2 = pick<T>(P.p2x, P.fp2x);
  T* __restrict__ W = static_cast<T*>(v.W) + P.offset;
  const int rounds = (nr + ngroups - 1) / ngroups;
  for (int k = 0; k < rounds; ++k) {
    const int r = k * ngroups + grp;
    T* row = W + (int64_t)(j0 + (r < nr ? r : nr - 1)) * nx + l * S;
    T m[1][S];
#pragma unroll
    for (int c = 0; c < S / 4; ++c) ld4(row + 4 * c, &m[0][4 * c]);
    seg_sweep<T, S, 1, false>(m, p1, p2, l, G, lg, Ks, Bf);
    seg_sweep<T, S, 1, true>(m, p1, p2, l, G, lg, Ks, Bb);
    if (r < nr) {
#pragma unroll
      for (int c = 0; c < S / 4; ++c) st4(row + 4 * c, &m[0][4 * c]);
    }
  }
}

// -------------------------------------------------------------------------------------
// Column kernel: column sweep and update for panels of columns.
// Shared memory per buffer: Ws (the W panel, swept in place) and Cs (the C panel), ny rows
// of nc+1 elements each; cols_p threads per column.  With PERSIST, a CTA walks the panels
// blockIdx.x, blockIdx.x + gridDim.x, ... with two buffers: the next panel's W and C are
// copied in (cp.async) while the current one is swept and written back, so every CTA keeps
// memory traffic in flight through its compute phases.  Without PERSIST each CTA takes one
// panel.  panel_cap: elements of one panel buffer (max over members of ny * (nc + 1)).
// -------------------------------------------------------------------------------------
// Panels move in 16-byte pieces (dense pitch nc) when the panel's rows are 16-byte aligned
// whole pieces; otherwise element by element with pitch nc + 1.
template <typename T>
__device__ __forceinline__ bool panel_vec_ok(int nx, int i0, int nc) {
  return (nx * (int)sizeof(T)) % 16 == 0 && (i0 * (int)sizeof(T)) % 16 == 0 && (nc * (int)sizeof(T)) % 16 == 0;
}

template <typename T>
__device__ __forceinline__ void cols_issue(const DevView& v, int tile, T* Ws, T* Cs) {
  const Tile tl = v.col_tiles[tile];
  if (!v.ms[tl.member].active) return;
  const MemberParams& P = v.mp[tl.member];
  const int nx = P.nx, ny = P.ny, i0 = tl.start, nc = tl.count;
  const T* W = static_cast<const T*>(v.W) + P.offset + i0;
  const T* C = static_cast<const T*>(v.C) + P.offset + i0;
  if (panel_vec_ok<T>(nx, i0, nc)) {
    const int nv = nc * (int)sizeof(T) / 16;  // 16-byte pieces per panel row
    const int tv = threadIdx.x % nv, ty = threadIdx.x / nv, ry = blockDim.x / nv;
    if (ty >= ry) return;
    for (int j = ty; j < ny; j += ry) {
      cp_async16(reinterpret_cast<char*>(Ws + (size_t)j * nc) + 16 * tv,
                 reinterpret_cast<const char*>(W + (int64_t)j * nx) + 16 * tv);
      cp_async16(reinterpret_cast<char*>(Cs + (size_t)j * nc) + 16 * tv,
                 reinterpret_cast<const char*>(C + (int64_t)j * nx) + 16 * tv);
    }
    return;
  }
  const int ldc = nc + 1;
  const int tx = threadIdx.x % nc, ty = threadIdx.x / nc, ry = blockDim.x / nc;
  if (ty >= ry) return;
  for (int j = ty; j < ny; j += ry) {
    cp_async_elem(Ws + (size_t)j * ldc + tx, W + (int64_t)j * nx + tx);
    cp_async_elem(Cs + (size_t)j * ldc + tx, C + (int64_t)j * nx + tx);
  }
}

template <typename T, bool PERSIST>
__global__ void __launch_bounds__(512) cols_kernel(DevView v, int ntiles, int panel_cap) {
  extern __shared__ __align__(16) unsigned char smem[];
  T* buf[2];
  buf[0] = reinterpret_cast<T*>(smem);
  buf[1] = buf[0] + 2 * (size_t)panel_cap;
  int tile = blockIdx.x;
  if (tile >= ntiles) return;
  cols_issue<T>(v, tile, buf[0], buf[0] + panel_cap);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  for (int it = 0; tile < ntiles; ++it) {
    const int next = tile + gridDim.x;
    T* Ws = buf[PERSIST ? (it & 1) : 0];
    T* Cs = Ws + panel_cap;
    if (PERSIST && next < ntiles) {
      T* Wn = buf[(it + 1) & 1];
      cols_issue<T>(v, next, Wn, Wn + panel_cap);
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 1;\n" ::: "memory");
    __syncthreads();
    const Tile tl = v.col_tiles[tile];
    MemberState* st = v.ms + tl.member;
    if (st->active) {
      const MemberParams& P = v.mp[tl.member];
      const int nx = P.nx, ny = P.ny, i0 = tl.start, nc = tl.count;
      const bool vec = panel_vec_ok<T>(nx, i0, nc);
      const int ldc = vec ? nc : nc + 1;
      const int sweep_p = P.cols_p;
      const int nsweep = nc * sweep_p;
      const int chunk = (ny + sweep_p - 1) / sweep_p;
      const int col = threadIdx.x % nc;
      const int c0 = (threadIdx.x / nc) * chunk;
      const int c1 = min(ny, c0 + chunk);
      const bool sweeper = threadIdx.x < nsweep && c0 < c1;
      const T p1 = (T)P.p1y, p2 = (T)P.p2y;
      if (sweep_p == 1) {
        if (sweeper) line_sweep_inplace<T>(Ws + col, ldc, ny, P.ky, p1, p2);
      } else {
        chunk_sweep_inplace<T>(Ws + col, ldc, ny, c0, c1, P.ky, p1, p2, sweeper);
      }
      __syncthreads();
      T* __restrict__ C = static_cast<T*>(v.C) + P.offset;
      T* const Lb = lo_ptr<T>(v, P, 0);  // lo block of compensated members, else null
      const T kap = (T)P.kappa;
      if (vec) {
        // 16-byte pieces: 4 floats or 2 doubles per thread and row
        constexpr int E = 16 / sizeof(T);
        const int nv = nc / E;
        const int tv = threadIdx.x % nv, ty = threadIdx.x / nv, ry = blockDim.x / nv;
        if (ty < ry)
          for (int j = ty; j < ny; j += ry) {
            const T* w = Ws + (size_t)j * nc + E * tv;
            const T* c = Cs + (size_t)j * nc + E * tv;
            T* g = C + (int64_t)j * nx + i0 + E * tv;
            if (E == 4) {
              T* lo = Lb ? Lb + (int64_t)j * nx + i0 + E * tv : nullptr;
              float4 o;
              o.x = (float)c_update<T>(c[0], kap, w[0], lo);
              o.y = (float)c_update<T>(c[1], kap, w[1], lo ? lo + 1 : nullptr);
              o.z = (float)c_update<T>(c[2], kap, w[2], lo ? lo + 2 : nullptr);
              o.w = (float)c_update<T>(c[3], kap, w[3], lo ? lo + 3 : nullptr);
              *reinterpret_cast<float4*>(g) = o;
            } else {
              double2 o;
              o.x = (double)fma(kap, w[0], c[0]);
              o.y = (double)fma(kap, w[1], c[1]);
              *reinterpret_cast<double2*>(g) = o;
            }
          }
      } else {
        const int tx = threadIdx.x % nc, ty = threadIdx.x / nc, ry = blockDim.x / nc;
        if (ty < ry)
          for (int j = ty; j < ny; j += ry)
            C[(int64_t)j * nx + i0 + tx] = c_update<T>(Cs[(size_t)j * ldc + tx], kap, Ws[(size_t)j * ldc + tx],
                                                       Lb ? Lb + (int64_t)j * nx + i0 + tx : nullptr);
      }
      // Panel 0 finalises the member's sample of this step (partials written by the
      // stencil phase of the same step) and advances the member's step counter.  No other
      // CTA of this launch reads or writes the member's state.
      if (tl.index == 0 && threadIdx.x == 0) finalize_sample(v, tl.member, st, P);
    }
    __syncthreads();  // the buffer is refilled two panels later
    if (!PERSIST) break;
    tile = next;
  }
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// -------------------------------------------------------------------------------------
// Column kernel, segment form (fused form).  A CTA takes up to 32 * ppc columns of one
// member (ppc panels of 32); each panel's columns are split into wp = ny / S segments of S
// rows, one warp per segment and one lane per column, so every access to W and C is a
// coalesced row piece of the panel and the S values of a lane stay in registers.  Each
// recurrence runs as a pass from a zero state over the segment, an exchange of the
// segments' end states through shared memory, the sequential combination over the wp
// segments (Y_w = M^S Y_{w-1} + e_w), the periodic start state x0 = (I - M^ny)^-1 Y_{wp-1},
// and a second pass from M^(S w) x0 + Y_{w-1}.  Then C += kappa Z row piece by row piece.
// -------------------------------------------------------------------------------------
template <typename T, int S, bool REV>
__device__ __forceinline__ void colseg_pass(T (&y)[S], T p1, T p2, const SegTable& tab, T* xs, int warp, int lane,
                                            int wseg, int wp, int pbase) {
  T a = T(0), b = T(0);
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const T t = fma(p1, a, fma(p2, b, y[REV ? S - 1 - k : k]));
    b = a;
    a = t;
  }
  xs[2 * (warp * 32 + lane)] = a;
  xs[2 * (warp * 32 + lane) + 1] = b;
  __syncthreads();
  // sequential combination over the panel's segments in the recurrence's order
  const T A0 = pick<T>(tab.A[0][0], tab.Af[0][0]), A1 = pick<T>(tab.A[0][1], tab.Af[0][1]);
  const T A2 = pick<T>(tab.A[0][2], tab.Af[0][2]), A3 = pick<T>(tab.A[0][3], tab.Af[0][3]);
  const int pos = REV ? wp - 1 - wseg : wseg;
  T ya = T(0), yb = T(0), pa = T(0), pb = T(0);
  for (int k = 0; k < wp; ++k) {
    const int w = pbase + (REV ? wp - 1 - k : k);
    const T ea = xs[2 * (w * 32 + lane)], eb = xs[2 * (w * 32 + lane) + 1];
    const T na = fma(A0, ya, fma(A1, yb, ea));
    yb = fma(A2, ya, fma(A3, yb, eb));
    ya = na;
    if (k + 1 == pos) {
      pa = ya;
      pb = yb;
    }
  }
  const T P0 = pick<T>(tab.P[0], tab.Pf[0]), P1 = pick<T>(tab.P[1], tab.Pf[1]);
  const T P2 = pick<T>(tab.P[2], tab.Pf[2]), P3 = pick<T>(tab.P[3], tab.Pf[3]);
  const T xa = fma(P0, ya, P1 * yb), xb = fma(P2, ya, P3 * yb);
  const T B0 = pick<T>(tab.B[pos][0], tab.Bf[pos][0]), B1 = pick<T>(tab.B[pos][1], tab.Bf[pos][1]);
  const T B2 = pick<T>(tab.B[pos][2], tab.Bf[pos][2]), B3 = pick<T>(tab.B[pos][3], tab.Bf[pos][3]);
  a = fma(B0, xa, fma(B1, xb, pa));
  b = fma(B2, xa, fma(B3, xb, pb));
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const int u = REV ? S - 1 - k : k;
    const T t = fma(p1, a, fma(p2, b, y[u]));
    y[u] = t;
    b = a;
    a = t;
  }
}

template <typename T, int S>
__global__ void __launch_bounds__(sizeof(T) == 4 ? 1024 : 512) colseg_kernel(DevView v, int tile_base) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tile tl = v.colseg_tiles[tile_base + blockIdx.x];
  MemberState* st = v.ms + tl.member;
  if (!st->active) return;
  const MemberParams& P = v.mp[tl.member];
  const SegTable& tab = v.segy[tl.member];
  const int nx = P.nx, ny = P.ny;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int wp = ny / S;
  const int sg = warp / wp, wseg = warp - sg * wp, pbase = sg * wp;
  const int cl = 32 * sg + lane;                      // column within the tile
  const bool cv = sg < nwarps / wp && cl < tl.count;  // this lane owns a column
  const int col = tl.start + (cv ? cl : 0);
  T* xf = reinterpret_cast<T*>(smem);
  T* xb = xf + 2 * 32 * nwarps;
  const T* __restrict__ Wg = static_cast<const T*>(v.W) + P.offset + (int64_t)wseg * S * nx + col;
  T y[S];
#pragma unroll
  for (int u = 0; u < S; ++u) y[u] = cv ? Wg[(int64_t)u * nx] : T(0);
  const T p1 = pick<T>(P.p1y, P.fp1y), p2 = pick<T>(P.p2y, P.fp2y);
  colseg_pass<T, S, false>(y, p1, p2, tab, xf, warp, lane, wseg, wp, pbase);
  colseg_pass<T, S, true>(y, p1, p2, tab, xb, warp, lane, wseg, wp, pbase);
  if (cv) {
    const T kap = pick<T>(P.kappa, P.fkappa);
    const int64_t base = (int64_t)wseg * S * nx + col;
    T* __restrict__ Cg = static_cast<T*>(v.C) + P.offset + base;
    T* const Lg = lo_ptr<T>(v, P, base);  // lo part of compensated members, else null
    if (Lg) {
#pragma unroll
      for (int u0 = 0; u0 < S; u0 += 4) {  // hi and lo of 4 rows in flight, then the pair update
        T c[4], lo[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          c[u] = Cg[(int64_t)(u0 + u) * nx];
          lo[u] = Lg[(int64_t)(u0 + u) * nx];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          Cg[(int64_t)(u0 + u) * nx] = c_update<T>(c[u], kap, y[u0 + u], &lo[u]);
          Lg[(int64_t)(u0 + u) * nx] = lo[u];
        }
      }
    } else {
#pragma unroll
      for (int u0 = 0; u0 < S; u0 += 8) {  // 8 loads in flight, few extra registers
        T c[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) c[u] = Cg[(int64_t)(u0 + u) * nx];
#pragma unroll
        for (int u = 0; u < 8; ++u) Cg[(int64_t)(u0 + u) * nx] = fma(kap, y[u0 + u], c[u]);
      }
    }
  }
  // The first tile of the member finalises its sample of this step and advances its step
  // counter (no other CTA of this launch touches the member's state).
  if (tl.index == 0 && threadIdx.x == 0) finalize_sample(v, tl.member, st, P);
}

// -------------------------------------------------------------------------------------
// Column kernel, segment form over a cluster of two CTAs: columns taller than one CTA's
// warps can hold (FP64: more than 16 segments of S rows, FP32: more than 32) split their
// wp = ny / S segments over the pair; each CTA writes its warps' segment end states to its
// own shared memory and the combination reads the partner's through distributed shared
// memory (mapa + ld.shared::cluster) after a cluster barrier.  One 32-column panel per pair.
// -------------------------------------------------------------------------------------
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\nbarrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Shared-memory address of p in CTA `rank` of the cluster.
__device__ __forceinline__ unsigned peer_addr(const void* p, unsigned rank) {
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  unsigned r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}

__device__ __forceinline__ float ld_peer(unsigned addr, float) {
  float x;
  asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(x) : "r"(addr) : "memory");
  return x;
}
__device__ __forceinline__ double ld_peer(unsigned addr, double) {
  double x;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(x) : "r"(addr) : "memory");
  return x;
}

template <typename T, int S, bool REV>
__device__ __forceinline__ void colseg2_pass(T (&y)[S], T p1, T p2, const SegTable& tab, T* xs, int warp, int lane,
                                             int nw, unsigned rank) {
  const int wp = 2 * nw, wseg = (int)rank * nw + warp;
  T a = T(0), b = T(0);
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const T t = fma(p1, a, fma(p2, b, y[REV ? S - 1 - k : k]));
    b = a;
    a = t;
  }
  xs[2 * (warp * 32 + lane)] = a;
  xs[2 * (warp * 32 + lane) + 1] = b;
  cluster_sync();
  const unsigned peer = peer_addr(xs, rank ^ 1u);  // the partner's end-state buffer
  const T A0 = pick<T>(tab.A[0][0], tab.Af[0][0]), A1 = pick<T>(tab.A[0][1], tab.Af[0][1]);
  const T A2 = pick<T>(tab.A[0][2], tab.Af[0][2]), A3 = pick<T>(tab.A[0][3], tab.Af[0][3]);
  const int pos = REV ? wp - 1 - wseg : wseg;
  T ya = T(0), yb = T(0), pa = T(0), pb = T(0);
  for (int k = 0; k < wp; ++k) {
    const int w = REV ? wp - 1 - k : k;  // segment in recurrence order
    const int ow = w % nw;
    T ea, eb;
    if ((unsigned)(w / nw) == rank) {
      ea = xs[2 * (ow * 32 + lane)];
      eb = xs[2 * (ow * 32 + lane) + 1];
    } else {
      ea = ld_peer(peer + (unsigned)(2 * (ow * 32 + lane)) * (unsigned)sizeof(T), T(0));
      eb = ld_peer(peer + (unsigned)(2 * (ow * 32 + lane) + 1) * (unsigned)sizeof(T), T(0));
    }
    const T na = fma(A0, ya, fma(A1, yb, ea));
    yb = fma(A2, ya, fma(A3, yb, eb));
    ya = na;
    if (k + 1 == pos) {
      pa = ya;
      pb = yb;
    }
  }
  const T P0 = pick<T>(tab.P[0], tab.Pf[0]), P1 = pick<T>(tab.P[1], tab.Pf[1]);
  const T P2 = pick<T>(tab.P[2], tab.Pf[2]), P3 = pick<T>(tab.P[3], tab.Pf[3]);
  const T xa = fma(P0, ya, P1 * yb), xb = fma(P2, ya, P3 * yb);
  const T B0 = pick<T>(tab.B[pos][0], tab.Bf[pos][0]), B1 = pick<T>(tab.B[pos][1], tab.Bf[pos][1]);
  const T B2 = pick<T>(tab.B[pos][2], tab.Bf[pos][2]), B3 = pick<T>(tab.B[pos][3], tab.Bf[pos][3]);
  a = fma(B0, xa, fma(B1, xb, pa));
  b = fma(B2, xa, fma(B3, xb, pb));
#pragma unroll
  for (int k = 0; k < S; ++k) {
    const int u = REV ? S - 1 - k : k;
    const T t = fma(p1, a, fma(p2, b, y[u]));
    y[u] = t;
    b = a;
    a = t;
  }
}

template <typename T, int S>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(sizeof(T) == 4 ? 1024 : 512)
    colseg2_kernel(DevView v, int tile_base) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tile tl = v.colseg_tiles[tile_base + blockIdx.x / 2];  // both CTAs of a pair: one tile
  MemberState* st = v.ms + tl.member;
  if (!st->active) return;  // taken by both CTAs of the pair alike
  const unsigned rank = cluster_rank();
  const MemberParams& P = v.mp[tl.member];
  const SegTable& tab = v.segy[tl.member];
  const int nx = P.nx;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int wseg = (int)rank * nw + warp;
  const bool cv = lane < tl.count;
  const int col = tl.start + (cv ? lane : 0);
  T* xf = reinterpret_cast<T*>(smem);
  T* xb = xf + 2 * 32 * nw;
  const T* __restrict__ Wg = static_cast<const T*>(v.W) + P.offset + (int64_t)wseg * S * nx + col;
  T y[S];
#pragma unroll
  for (int u = 0; u < S; ++u) y[u] = cv ? Wg[(int64_t)u * nx] : T(0);
  const T p1 = pick<T>(P.p1y, P.fp1y), p2 = pick<T>(P.p2y, P.fp2y);
  colseg2_pass<T, S, false>(y, p1, p2, tab, xf, warp, lane, nw, rank);
  colseg2_pass<T, S, true>(y, p1, p2, tab, xb, warp, lane, nw, rank);
  if (cv) {
    const T kap = pick<T>(P.kappa, P.fkappa);
    const int64_t base = (int64_t)wseg * S * nx + col;
    T* __restrict__ Cg = static_cast<T*>(v.C) + P.offset + base;
    T* const Lg = lo_ptr<T>(v, P, base);
#pragma unroll
    for (int u0 = 0; u0 < S; u0 += 4) {
      T c[4], lo[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        c[u] = Cg[(int64_t)(u0 + u) * nx];
        lo[u] = Lg ? Lg[(int64_t)(u0 + u) * nx] : T(0);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        Cg[(int64_t)(u0 + u) * nx] = c_update<T>(c[u], kap, y[u0 + u], Lg ? &lo[u] : nullptr);
        if (Lg) Lg[(int64_t)(u0 + u) * nx] = lo[u];
      }
    }
  }
  if (tl.index == 0 && rank == 0 && threadIdx.x == 0) finalize_sample(v, tl.member, st, P);
  cluster_sync();  // the partner may still read this CTA's end states
}

// -------------------------------------------------------------------------------------
// Cluster-resident form (FP32).  A member with nx = 128 or 256 and ny = NR Q keeps its whole
// field in the shared memory of a cluster of Q CTAs for a chunk of steps: CTA q holds rows
// NR q .. NR q + NR - 1 (NR = 32, Q <= 8; or NR = 64 for nx = 256, Q <= 4) plus two halo rows
// on each side, so HBM sees one load and one store of the field per launch instead of five
// words per point and step.  One step:
//   mu      NR + 2 rows (own rows and one halo row each side) from the C tile, 4 points per
//           thread, into the mu/W tile;
//   rows    R' in registers, both row recurrences as segment scans across 16 lanes per
//           row (S = nx / 16 points per lane), W back into the mu/W tile;
//   columns a thread owns SC = nx / 8 rows of one column: the forward recurrence from a
//           zero state over its W, then the backward recurrence from a zero state over that
//           result; both end states go to shared memory, and after the step's only cluster
//           barrier every thread combines the end states of all segments of its column in
//           recurrence order (read through distributed shared memory), which gives every
//           segment's forward start state s_k and backward start state t_k.  The solution
//           is then closed-form, x = G0(F0(W)) + g s_k + k t_k with the segment responses
//           g, k (SegTable::Hf), except the two first and two last rows of a segment, which
//           are taken from the combination (t_{k-1}, and the first two backward steps from
//           t_k over s_{k+1}).  Every CTA computes the same s_k, t_k with the same
//           operations, so it updates its halo rows -- its neighbours' boundary rows --
//           itself, bit for bit as the neighbours update them: no halo exchange.
// The end states are double-buffered by step parity (a CTA may start the next step while
// others still read this step's).  Sample steps add the FP64 partial sums of the F and
// dF/dt densities (mu recomputed in FP64 from the stored field, as in the other FP32
// kernels); rank 0 sums the CTAs' partials in rank order and finalises the sample.  mu and
// R' are formed in the operation order of the segment-form kernels.
// -------------------------------------------------------------------------------------
// NR rows of the field per CTA (32 or 64) with 8 NR threads: every thread owns 2 rows in the
// row phase and NX / 8 rows of one column in the column phase.  NR = 32: two CTAs per SM (the
// register and shared-memory budgets of a plain 256-column CTA); NR = 64: one CTA of 512
// threads per SM, half as many CTAs per member.

__device__ __forceinline__ unsigned cluster_size() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
  return r;
}

// Four FP32 values from distributed shared memory.  No memory clobber: the loads of a
// combination are issued back to back and wait only where their values are used (the
// cluster barrier before them carries the ordering).
__device__ __forceinline__ float4 ld_peer4(unsigned addr) {
  float4 x;
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(x.x), "=f"(x.y), "=f"(x.z), "=f"(x.w)
               : "r"(addr));
  return x;
}

__device__ __forceinline__ void st_peer2d(unsigned addr, double2 x) {
  asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(addr), "d"(x.x), "d"(x.y) : "memory");
}

// Element (r, i) of the mu/W tile (pitch NX floats).  The 16-byte quad of column i is
// XOR-ed with bits 3..5 of its quad index: the row phase's 16-byte reads of 16 lanes S
// points apart, the mu phase's consecutive quads and the column phase's consecutive
// columns all fall in distinct banks.
template <int NX>
__device__ __forceinline__ int res_swz(int r, int i) {
  const int q = i >> 2;
  return r * NX + (((q ^ ((q >> 3) & 7)) << 2) | (i & 3));
}

// 2 x 2 matrix (row-major, 4 floats) times a state.
__device__ __forceinline__ float2 mat2v(const float* A, float2 v) {
  return make_float2(fmaf(A[0], v.x, A[1] * v.y), fmaf(A[2], v.x, A[3] * v.y));
}
__device__ __forceinline__ float2 mat2v_add(const float* A, float2 v, float2 w) {
  return make_float2(fmaf(A[0], v.x, fmaf(A[1], v.y, w.x)), fmaf(A[2], v.x, fmaf(A[3], v.y, w.y)));
}

// FP64 partial sums of the F and dF/dt densities over the CTA's own rows (C tile rows
// 2 .. 33; hi + lo for compensated members), mu recomputed in FP64 from the stored field.
// Thread = column i of a block of 32 NX / 256 rows, walking down with three field rows in
// registers; x neighbours by shuffles (lanes hold consecutive columns), the ends of a warp's
// run loaded.  Fixed work split and order.  Result in thread 0.
template <int NX, int NR, bool COMP>
__device__ __forceinline__ void res_partials(const float* Ct, const float* Lt, const MemberParams& P, double* red,
                                             double& sF, double& sD) {
  constexpr int RB = NX / 8;  // rows per thread (NR NX points over 8 NR threads)
  const int lane = threadIdx.x & 31;
  const int i = threadIdx.x % NX, r0 = (threadIdx.x / NX) * RB;
  const int ie = i + 1 == NX ? 0 : i + 1, iw = i == 0 ? NX - 1 : i - 1, iee = ie + 1 == NX ? 0 : ie + 1;
  const double a = P.a, bx = P.bx, by = P.by;
  auto at = [&](int r, int ii) {  // own row r (-2 .. 33) at column ii, in FP64
    const int k = (r + 2) * NX + ii;
    return COMP ? (double)Ct[k] + (double)Lt[k] : (double)Ct[k];
  };
  auto mu_of = [&](double c, double e, double w, double n, double s) {
    return c * (c * c - a) - bx * (e + w) - by * (n + s);
  };
  // west / east neighbours of the field at row r (value cv of this lane's column)
  auto nbrs = [&](double cv, int r, double& w, double& e) {
    w = __shfl_up_sync(kFull, cv, 1);
    e = __shfl_down_sync(kFull, cv, 1);
    if (lane == 0) w = at(r, iw);
    if (lane == 31) e = at(r, ie);
  };
  double sw = 0.0, sdx = 0.0, sdy = 0.0, smx = 0.0, smy = 0.0;
  double cm = at(r0 - 1, i), c0 = at(r0, i), c1 = at(r0 + 1, i);
  double w0, e0;
  nbrs(c0, r0, w0, e0);
  double mu0 = mu_of(c0, e0, w0, c1, cm);
  for (int r = r0; r < r0 + RB; ++r) {
    const double c2 = at(r + 2, i);
    double w1, e1;
    nbrs(c1, r + 1, w1, e1);
    const double mu1 = mu_of(c1, e1, w1, c2, c0);
    double mue = __shfl_down_sync(kFull, mu0, 1);
    if (lane == 31) mue = mu_of(e0, at(r, iee), c0, at(r + 1, ie), at(r - 1, ie));
    const double w = c0 * c0 - 1.0, gx = e0 - c0, gy = c1 - c0, mx = mue - mu0, my = mu1 - mu0;
    sw += w * w;
    sdx += gx * gx;
    sdy += gy * gy;
    smx += mx * mx;
    smy += my * my;
    cm = c0;
    c0 = c1;
    c1 = c2;
    e0 = e1;
    mu0 = mu1;
  }
  (void)cm;
  const double hxi2 = 1.0 / (P.hx * P.hx), hyi2 = 1.0 / (P.hy * P.hy);
  sF = 0.25 * sw + 0.5 * P.gamma * (hxi2 * sdx + hyi2 * sdy);
  sD = hxi2 * smx + hyi2 * smy;
  block_sum2(sF, sD, red);
}

// Shared memory of the resident kernel (bytes): C tile (and lo tile), mu/W tile, the
// column end states (two step parities), the scan tables, the FP64 reduction buffer, the
// per-rank partial slots (two step parities) and the member's state (rank 0).
constexpr int kResConsts = 288;  // row A, P (24); column A, P (8); row B (16 x 4); column B (16 x 4); H (32 x 4)
__host__ __device__ constexpr size_t res_smem_bytes(int nx, int nr, bool comp) {
  return (size_t)((comp ? 2 : 1) * (nr + 4) + (nr + 2)) * nx * sizeof(float) +
         (size_t)2 * 8 * nr * sizeof(float4) + kResConsts * sizeof(float) + (size_t)(nr / 2) * sizeof(double) +
         16 * sizeof(double2) + (sizeof(MemberState) + 15) / 16 * 16;
}

template <int NX, int NR, bool COMP, bool OBS>
__global__ void __launch_bounds__(8 * NR, NR == 32 ? 2 : 1) res_kernel(DevView v, int tile_base, int64_t nsteps) {
  constexpr int TH = 8 * NR;      // threads per CTA
  constexpr int S = NX / 16;      // row points per lane
  constexpr int SC = NX / 8;      // column points per thread
  constexpr int NSEG = NR / SC;   // column segments per CTA
  constexpr int KMAX = 256 / SC;  // column segments at most (ny <= 256)
  constexpr int NQ = NX / 4;      // 16-byte quads per row
  constexpr int CT = NR + 4, MT = NR + 2;
  extern __shared__ __align__(16) unsigned char smem[];
  float* Ct = reinterpret_cast<float*>(smem);
  float* Lt = Ct + CT * NX;
  float* Mw = Lt + (COMP ? CT * NX : 0);
  float4* xs = reinterpret_cast<float4*>(Mw + MT * NX);  // [2][TH]
  float* Ks = reinterpret_cast<float*>(xs + 2 * TH);       // see kResConsts
  double* red = reinterpret_cast<double*>(Ks + kResConsts);  // 2 per warp
  double2* part = reinterpret_cast<double2*>(red + NR / 2);  // [2][8]: by step parity, then rank
  MemberState* lst = reinterpret_cast<MemberState*>(part + 16);

  const unsigned Q = cluster_size(), rank = cluster_rank();
  const Tile tl = v.res_tiles[tile_base + blockIdx.x / Q];
  const int m = tl.member;
  const MemberParams& P = v.mp[m];
  MemberState* st = v.ms + m;
  const int ny = P.ny, j0 = (int)rank * NR;
  const int tid = threadIdx.x, lane = tid & 31;
  float* __restrict__ Cg = static_cast<float*>(v.C) + P.offset;
  float* __restrict__ Lg = COMP ? static_cast<float*>(v.C) + P.lo_offset : nullptr;

  // the steps of this launch, read before any CTA of the cluster changes the state (rank 0
  // writes it back only at the end)
  const int64_t n0 = st->step, rem = st->remaining;
  const int64_t nrun = OBS ? 0 : (rem < nsteps ? rem : nsteps);
  if (!OBS && nrun <= 0) return;  // the same decision in every CTA of the cluster

  // C (and lo) rows j0 - 2 .. j0 + 33, periodic
  for (int k = tid; k < CT * NQ; k += TH) {
    const int r = k / NQ, q = k - r * NQ;
    int j = j0 - 2 + r;
    j = j < 0 ? j + ny : (j >= ny ? j - ny : j);
    reinterpret_cast<float4*>(Ct + r * NX)[q] = reinterpret_cast<const float4*>(Cg + (int64_t)j * NX)[q];
    if (COMP) reinterpret_cast<float4*>(Lt + r * NX)[q] = reinterpret_cast<const float4*>(Lg + (int64_t)j * NX)[q];
  }
  if (OBS) {
    __syncthreads();
    double sF, sD;
    res_partials<NX, NR, COMP>(Ct, Lt, P, red, sF, sD);
    if (tid == 0) v.partials[P.partial_base + rank] = make_double2(sF, sD);
    return;
  }
  // column phase: column c, rows g SC .. g SC + SC - 1 of this CTA = segment gs of ns
  const int c = tid % NX, g = tid / NX;
  const int ns = (int)Q * NSEG, gs = (int)rank * NSEG + g;
  {
    const SegTable& tx = v.seg[m];
    const SegTable& ty = v.segy[m];
    for (int k = tid; k < kResConsts; k += TH) {
      float x = 0.f;
      if (k < 20)
        x = tx.Af[k >> 2][k & 3];
      else if (k < 24)
        x = tx.Pf[k - 20];
      else if (k < 28)
        x = ty.Af[0][k - 24];
      else if (k < 32)
        x = ty.Pf[k - 28];
      else if (k < 96)
        x = tx.Bf[(k - 32) >> 2][k & 3];
      else if (k < 160)
        x = (k - 96) >> 2 < ns ? ty.Bf[(k - 96) >> 2][k & 3] : 0.f;
      else
        x = ty.Hf[(k - 160) >> 2][k & 3];
      Ks[k] = x;
    }
  }
  const float* KB = Ks + 32;   // row start-state matrices M^(S l), l = 0 .. 15
  const float* KC = Ks + 96;   // column powers M^(SC k), k = 0 .. ns - 1
  const float* KH = Ks + 160;  // column segment responses (g1, g2, k1, k2) per row
  // row phase: 16 lanes per row, rows grp and grp + NR / 2
  const int l = tid & 15, grp = tid >> 4;
  const float a = P.fa, bx = P.fbx, by = P.fby, rho = P.frho, w0 = P.fw0;
  const float p1x = P.fp1x, p2x = P.fp2x, p1y = P.fp1y, p2y = P.fp2y, kap = P.fkappa;
  // the member's state lives in shared memory of rank 0 for the launch
  const bool keeper = rank == 0 && tid == 0;
  if (keeper) *lst = *st;
  cluster_sync();  // every CTA of the cluster runs and has its tile and constants

  for (int64_t s = 0; s < nrun; ++s) {
    const bool sample = ((n0 + s) % P.every) == 0;
    if (sample) {
      double sF, sD;
      res_partials<NX, NR, COMP>(Ct, Lt, P, red, sF, sD);
      if (tid == 0) st_peer2d(peer_addr(part + 8 * (s & 1) + rank, 0), make_double2(sF, sD));
    }
    // mu of own rows -1 .. 32 (tile row r + 1 of C) into mu/W tile row r
    {
      const int q = tid % NQ;
      for (int r = tid / NQ; r < MT; r += TH / NQ) {  // warp-uniform (NQ >= 32)
        const float* c0 = Ct + (r + 1) * NX;
        float cc[4], nn[4], so[4];
        ld4(c0 + 4 * q, cc);
        ld4(c0 - NX + 4 * q, nn);
        ld4(c0 + NX + 4 * q, so);
        float w = __shfl_up_sync(kFull, cc[3], 1), e = __shfl_down_sync(kFull, cc[0], 1);
        if (lane == 0) w = c0[q == 0 ? NX - 1 : 4 * q - 1];
        if (lane == 31) e = c0[q == NQ - 1 ? 0 : 4 * q + 4];
        float out[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const float ce = k < 3 ? cc[k + 1] : e;
          const float cw = k > 0 ? cc[k - 1] : w;
          const float u = cc[k] * fmaf(cc[k], cc[k], -a);
          out[k] = fmaf(-by, so[k] + nn[k], fmaf(-bx, ce + cw, u));
        }
        st4(Mw + res_swz<NX>(r, 4 * q), out);
      }
    }
    __syncthreads();
    // R' and the row recurrences of own rows grp, grp + NR / 2 (mu/W tile rows + 1)
    {
      float y[2][S];
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        const int r = grp + (NR / 2) * t + 1;
#pragma unroll
        for (int k = 0; k < S / 4; ++k) ld4(Mw + res_swz<NX>(r, l * S + 4 * k), &y[t][4 * k]);
        const float left = __shfl_sync(kFull, y[t][S - 1], (l + 15) & 15, 16);
        const float right = __shfl_sync(kFull, y[t][0], (l + 1) & 15, 16);
        float prv = left;
#pragma unroll
        for (int k = 0; k < S / 4; ++k) {
          float up[4], dn[4];
          ld4(Mw + res_swz<NX>(r - 1, l * S + 4 * k), up);
          ld4(Mw + res_swz<NX>(r + 1, l * S + 4 * k), dn);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int u = 4 * k + q;
            const float cur = y[t][u];
            const float e = u + 1 < S ? y[t][u + 1] : right;
            y[t][u] = fmaf(w0, cur, fmaf(rho, dn[q] + up[q], e + prv));
            prv = cur;
          }
        }
      }
      {
        float B[4];
        ld4(KB + 4 * l, B);
        seg_sweep<float, S, 2, false>(y, p1x, p2x, l, 16, 4, Ks, B);
        ld4(KB + 4 * (15 - l), B);
        seg_sweep<float, S, 2, true>(y, p1x, p2x, l, 16, 4, Ks, B);
      }
      __syncthreads();  // every mu read of this step is done: W replaces mu
#pragma unroll
      for (int t = 0; t < 2; ++t)
#pragma unroll
        for (int k = 0; k < S / 4; ++k) st4(Mw + res_swz<NX>(grp + (NR / 2) * t + 1, l * S + 4 * k), &y[t][4 * k]);
    }
    __syncthreads();
    // columns
    {
      float4* xsb = xs + (s & 1) * TH;
      float y[SC];
#pragma unroll
      for (int u = 0; u < SC; ++u) y[u] = Mw[res_swz<NX>(g * SC + u + 1, c)];
      // forward recurrence from a zero state, then the backward one over its result
      float fa = 0.f, fb = 0.f;
#pragma unroll
      for (int u = 0; u < SC; ++u) {
        const float t = fmaf(p1y, fa, fmaf(p2y, fb, y[u]));
        y[u] = t;
        fb = fa;
        fa = t;
      }
      float ba = 0.f, bb = 0.f;
#pragma unroll
      for (int u = SC - 1; u >= 0; --u) {
        const float t = fmaf(p1y, ba, fmaf(p2y, bb, y[u]));
        y[u] = t;
        bb = ba;
        ba = t;
      }
      xsb[tid] = make_float4(fa, fb, ba, bb);  // (y_SC-1, y_SC-2), (x_0, x_1)
      cluster_sync();
      if (keeper) {
        // the sample (partials of every CTA, summed in rank order) and the step counter
        double sF = 0.0, sD = 0.0;
        if (sample)
          for (unsigned k = 0; k < Q; ++k) {
            sF += part[8 * (s & 1) + k].x;
            sD += part[8 * (s & 1) + k].y;
          }
        finalize_sums(v, m, lst, P, sF, sD);
      }
      // the end states of the column's ns segments (k in recurrence order of the forward
      // pass), then the combination -- the same operations in every thread of the column
      float4 E[KMAX];
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        if (k < ns) {
          const unsigned owner = (unsigned)(k / NSEG);
          const int slot = (k - (int)owner * NSEG) * NX + c;
          E[k] = owner == rank ? xsb[slot] : ld_peer4(peer_addr(xsb + slot, owner));
        }
      }
      const float* A = Ks + 24;  // M^SC: one segment, either direction
      const float* PP = Ks + 28; // (I - M^ny)^-1
      const float Eb[4] = {KH[0], KH[1], KH[4], KH[5]};  // (x_0, x_1) per unit start state s
      // forward: the total from zero, the periodic start x0, then s_k = M^(SC k) x0 + Y_k-1;
      // backward end states with their true start: e_k + Eb s_k (kept in E[k].z, .w)
      float2 Y = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < KMAX; ++k)
        if (k < ns) Y = mat2v_add(A, Y, make_float2(E[k].x, E[k].y));
      const float2 x0 = mat2v(PP, Y);
      float2 s_own = x0, s_next = x0;
      Y = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < KMAX; ++k) {
        if (k < ns) {
          const float2 sk = mat2v_add(KC + 4 * k, x0, Y);
          if (k == gs) s_own = sk;
          if (k == (gs + 1 == ns ? 0 : gs + 1)) s_next = sk;
          const float2 eb = mat2v_add(Eb, sk, make_float2(E[k].z, E[k].w));
          E[k].z = eb.x;
          E[k].w = eb.y;
          Y = mat2v_add(A, Y, make_float2(E[k].x, E[k].y));
        }
      }
      // backward, segments from the last: the total, the periodic start of the last
      // segment, then t_k = M^(SC (ns-1-k)) t_last + Z_k+1
      // (k runs down from KMAX - 1 so that E is indexed by constants and stays in registers)
      float2 Z = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = KMAX - 1; k >= 0; --k)
        if (k < ns) Z = mat2v_add(A, Z, make_float2(E[k].z, E[k].w));
      const float2 tl0 = mat2v(PP, Z);
      float2 t_own = tl0, t_prev = tl0;
      Z = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = KMAX - 1; k >= 0; --k) {
        if (k < ns) {
          const float2 tk = mat2v_add(KC + 4 * (ns - 1 - k), tl0, Z);
          if (k == gs) t_own = tk;
          if (k == (gs == 0 ? ns - 1 : gs - 1)) t_prev = tk;
          Z = mat2v_add(A, Z, make_float2(E[k].z, E[k].w));
        }
      }
      // the solution of this segment: closed form inside, the combination at its ends
#pragma unroll
      for (int u = 2; u < SC - 2; ++u) {
        float H[4];
        ld4(KH + 4 * u, H);
        y[u] = fmaf(H[3], t_own.y, fmaf(H[2], t_own.x, fmaf(H[1], s_own.y, fmaf(H[0], s_own.x, y[u]))));
      }
      y[0] = t_prev.x;
      y[1] = t_prev.y;
      y[SC - 1] = fmaf(p1y, t_own.x, fmaf(p2y, t_own.y, s_next.x));
      y[SC - 2] = fmaf(p1y, y[SC - 1], fmaf(p2y, t_own.x, s_next.y));
#pragma unroll
      for (int u = 0; u < SC; ++u) {
        const int k = (g * SC + u + 2) * NX + c;
        Ct[k] = c_update<float>(Ct[k], kap, y[u], COMP ? Lt + k : nullptr);
      }
      // halo rows: the previous segment's last two rows (above the first segment of this
      // CTA) and the next segment's first two rows (below the last), as their owners
      // compute them
      if (g == 0) {
        const float h1 = fmaf(p1y, t_prev.x, fmaf(p2y, t_prev.y, s_own.x));
        const float h0 = fmaf(p1y, h1, fmaf(p2y, t_prev.x, s_own.y));
        Ct[NX + c] = c_update<float>(Ct[NX + c], kap, h1, COMP ? Lt + NX + c : nullptr);
        Ct[c] = c_update<float>(Ct[c], kap, h0, COMP ? Lt + c : nullptr);
      }
      if (g == NSEG - 1) {
        const int k34 = (NR + 2) * NX + c, k35 = k34 + NX;
        Ct[k34] = c_update<float>(Ct[k34], kap, t_own.x, COMP ? Lt + k34 : nullptr);
        Ct[k35] = c_update<float>(Ct[k35], kap, t_own.y, COMP ? Lt + k35 : nullptr);
      }
    }
    __syncthreads();
  }
  cluster_sync();  // no CTA leaves while others may still read its end states
  if (keeper) *st = *lst;
  // own rows back to HBM
  for (int k = tid; k < NR * NQ; k += TH) {
    const int r = k / NQ, q = k - r * NQ;
    reinterpret_cast<float4*>(Cg + (int64_t)(j0 + r) * NX)[q] = reinterpret_cast<const float4*>(Ct + (r + 2) * NX)[q];
    if (COMP)
      reinterpret_cast<float4*>(Lg + (int64_t)(j0 + r) * NX)[q] = reinterpret_cast<const float4*>(Lt + (r + 2) * NX)[q];
  }
}

// -------------------------------------------------------------------------------------
// Streaming sweeps (split form).  Lines are not held on chip: each warp owns 32 lines (one
// per lane) and streams them, so the number of recurrences in flight per SM is bounded by
// registers rather than by shared memory.  The intermediate y of the two-pass solve lives
// in the W scratch (in place: W holds R' -> y -> W' in the row sweep, W' -> y in the
// column sweep).  Pre-roll reads of a pass always precede that pass's writes to the same
// elements: the forward pass pre-rolls over the line's end and writes front to back; the
// backward pass pre-rolls over the line's start and writes back to front.
// -------------------------------------------------------------------------------------
constexpr int kStreamWarps = 4;  // register budget of the streaming sweeps: launch bounds of 4 warps
// Warps per CTA of the streaming sweeps (at most kStreamWarps).  One: the SMs then hold
// whole-warp shares of the lines (256 x 256^2: 2048 warps over 152 SMs, 13 or 14 each),
// where 4-warp CTAs left some SMs 16 warps and others 12; measured 0.192 / 0.242 ms per
// row / column launch against 0.212 / 0.260 with 4-warp CTAs.
constexpr int kStreamCta = 1;


// shared memory of rowstream_kernel: per warp two 32 x (CW+1) tiles, CW = 32 floats / 16 doubles
constexpr size_t rowstream_smem_bytes(size_t elt) {
  return (size_t)kStreamCta * 2 * 32 * ((elt == 8 ? 16 : 32) + 1) * elt;
}

// Binary64 -> binary32 with the significand truncated, from the two formats' fields (IEEE
// 754: binary64 = sign, 11-bit exponent biased by 1023, 52-bit fraction; binary32 = sign,
// 8-bit exponent biased by 127, 23-bit fraction): the exponent is rebiased by 896 and the
// top 23 fraction bits kept, so the relative error is below 2^-23.  |x| < 2^-126 gives a
// signed zero, |x| >= 2^128 (and NaN) a signed infinity.  Integer operations only: the
// FP32 heads of the FP64 pre-rolls leave the FP64 pipe to the FP64 part.
__device__ __forceinline__ float f32_trunc(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned mag = hi & 0x7fffffffu, sign = hi & 0x80000000u;
  const unsigned body = __funnelshift_l(lo, mag - (896u << 20), 3);  // (exp - 896) << 23 | fraction >> 29
  const unsigned bits = mag < (897u << 20) ? sign : (mag >= (1151u << 20) ? (sign | 0x7f800000u) : (sign | body));
  return __uint_as_float(bits);
}

// Sequence position q of a pass -> column/row index: positions 0..K-1 are the pre-roll,
// K..K+n-1 the line itself.  Forward: pre-roll over indices -K..-1 (mod n), then 0..n-1.
// Backward: pre-roll over n-1+K..n (mod n), then n-1..0.
__device__ __forceinline__ int fwd_index(int q, int K, int n) { return q < K ? wrap_index(q - K, n) : q - K; }
__device__ __forceinline__ int bwd_index(int q, int K, int n) {
  return q < K ? wrap_index(n - 1 + K - q, n) : n - 1 - (q - K);
}

// Column sweep + update, one thread per column, straight from global memory (a warp reads
// 32 consecutive elements of a row per access).  Tiles: 32-column groups; kStreamCta
// groups per CTA.
template <typename T>
__global__ void __launch_bounds__(32 * kStreamWarps) colstream_kernel(DevView v, int ntiles, int tile_base) {
  const int wt = blockIdx.x * kStreamCta + (threadIdx.x >> 5);
  if (wt >= ntiles) return;
  const Tile tl = v.col_tiles[tile_base + wt];
  MemberState* st = v.ms + tl.member;
  if (!st->active) return;
  const MemberParams& P = v.mp[tl.member];
  const int lane = threadIdx.x & 31;
  const int nx = P.nx, ny = P.ny, K = P.ky;
  if (lane < tl.count) {
    T* Wc = static_cast<T*>(v.W) + P.offset + tl.start + lane;
    T* Cc = static_cast<T*>(v.C) + P.offset + tl.start + lane;
    const T p1 = (T)P.p1y, p2 = (T)P.p2y, kap = (T)P.kappa;
    T* const Lc = lo_ptr<T>(v, P, tl.start + lane);  // lo column of compensated members, else null
    constexpr int kUnroll = 8;  // loads issued ahead of the recurrence
    const int len = K + ny;
    // forward: y_j = W'_j + p1 y_{j-1} + p2 y_{j-2}; y written over W'
    T y1 = T(0), y2 = T(0);
    for (int q0 = 0; q0 < len; q0 += kUnroll) {
      T r[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u)
        if (q0 + u < len) r[u] = Wc[(int64_t)fwd_index(q0 + u, K, ny) * nx];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (q0 + u < len) {
          const T y = fma(p1, y1, fma(p2, y2, r[u]));
          y2 = y1;
          y1 = y;
          if (q0 + u >= K) Wc[(int64_t)(q0 + u - K) * nx] = y;
        }
      }
    }
    // backward: x_j = y_j + p1 x_{j+1} + p2 x_{j+2};  C_j += kappa x_j
    T x1 = T(0), x2 = T(0);
    for (int q0 = 0; q0 < len; q0 += kUnroll) {
      T r[kUnroll], c[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (q0 + u < len) {
          const int j = bwd_index(q0 + u, K, ny);
          r[u] = Wc[(int64_t)j * nx];
          if (q0 + u >= K) c[u] = Cc[(int64_t)j * nx];
        }
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (q0 + u < len) {
          const T x = fma(p1, x1, fma(p2, x2, r[u]));
          x2 = x1;
          x1 = x;
          if (q0 + u >= K) {
            const int64_t jj = ny - 1 - (q0 + u - K);
            Cc[jj * nx] = c_update<T>(c[u], kap, x, Lc ? Lc + jj * nx : nullptr);
          }
        }
      }
    }
  }
  if (tl.index == 0 && lane == 0) finalize_sample(v, tl.member, st, P);
}

// Row sweep, one thread per row, streaming CW-column chunks of the warp's 32 rows through
// a double-buffered shared tile (pitch CW+1, conflict-free for the cp.async fill and for
// the per-thread walk).  CW = 32 floats or 16 doubles, so the tiles of a 4-warp CTA take
// about 34 KB in both precisions and the whole launch fits the SMs in one wave.
// Tiles: 32-row groups.
template <typename T>
struct StreamChunk {
  static constexpr int CW = sizeof(T) == 8 ? 16 : 32;
};

template <typename T>
__global__ void __launch_bounds__(32 * kStreamWarps) rowstream_kernel(DevView v, int ntiles, int tile_base) {
  constexpr int CW = StreamChunk<T>::CW;
  constexpr int RPI = 32 / CW;  // rows covered by one warp-wide copy instruction
  extern __shared__ __align__(16) unsigned char smem[];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wt = blockIdx.x * kStreamCta + w;
  if (wt >= ntiles) return;
  const Tile tl = v.sweep_tiles[tile_base + wt];
  if (!v.ms[tl.member].active) return;
  const MemberParams& P = v.mp[tl.member];
  const int nx = P.nx, K = P.kx, nr = tl.count;
  T* Wb = static_cast<T*>(v.W) + P.offset + (int64_t)tl.start * nx;
  const T p1 = (T)P.p1x, p2 = (T)P.p2x;
  const float fp1 = P.fp1x, fp2 = P.fp2x;
  const int kh = sizeof(T) == 8 ? P.kx32 : 0;  // FP32 head of each pre-roll: chunks 0 .. kh/CW - 1
  const int len = K + nx;
  const int nchunks = (len + CW - 1) / CW;
  // this warp's two 32 x (CW+1) buffers
  T (*buf)[32][CW + 1] =
      reinterpret_cast<T (*)[32][CW + 1]>(reinterpret_cast<T*>(smem) + (size_t)w * 2 * 32 * (CW + 1));
  const int cl = lane % CW, rsub = lane / CW;  // copy geometry: column cl of rows rsub, rsub + RPI, ...
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      // the backward pass reads (through cp.async) what other lanes stored in the forward pass
      __threadfence_block();
      __syncwarp();
    }
    auto issue = [&](int ch, int b) {
      const int q = ch * CW + cl;
      if (q < len) {
        const int col = pass == 0 ? fwd_index(q, K, nx) : bwd_index(q, K, nx);
        for (int r = rsub; r < nr; r += RPI) cp_async_elem(&buf[b][r][cl], Wb + (int64_t)r * nx + col);
      }
      asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    issue(0, 0);
    T s1 = T(0), s2 = T(0);
    float f1 = 0.f, f2 = 0.f;
    for (int ch = 0; ch < nchunks; ++ch) {
      const int b = ch & 1;
      if (ch + 1 < nchunks) {
        issue(ch + 1, b ^ 1);
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
      } else {
        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
      }
      __syncwarp();
      const int qbase = ch * CW;
      const int cnt = min(CW, len - qbase);
      if (lane < nr) {
        T* row = buf[b][lane];
        if (qbase + CW <= kh) {
          if constexpr (sizeof(T) == 8) {  // FP32 head: nothing of it is stored
            float vals[CW];
#pragma unroll
            for (int u = 0; u < CW; ++u) vals[u] = f32_trunc(row[u]);
#pragma unroll
            for (int u = 0; u < CW; ++u) {
              const float val = fmaf(fp1, f1, fmaf(fp2, f2, vals[u]));
              f2 = f1;
              f1 = val;
            }
            if (qbase + CW == kh) {
              s1 = (T)f1;
              s2 = (T)f2;
            }
          }
        } else if (cnt == CW) {
          T vals[CW];
#pragma unroll
          for (int u = 0; u < CW; ++u) vals[u] = row[u];
#pragma unroll
          for (int u = 0; u < CW; ++u) {
            const T val = fma(p1, s1, fma(p2, s2, vals[u]));
            s2 = s1;
            s1 = val;
            row[u] = val;
          }
        } else {
          for (int u = 0; u < cnt; ++u) {
            const T val = fma(p1, s1, fma(p2, s2, row[u]));
            s2 = s1;
            s1 = val;
            row[u] = val;
          }
        }
      }
      __syncwarp();
      // write back the positions that belong to the line itself (not the pre-roll)
      const int q = qbase + cl;
      if (q < len && q >= K) {
        const int col = pass == 0 ? q - K : nx - 1 - (q - K);
        for (int r = rsub; r < nr; r += RPI) Wb[(int64_t)r * nx + col] = buf[b][r][cl];
      }
      __syncwarp();
    }
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

// Dynamic shared memory of rowsT_kernel with nw warps.
template <typename T>
size_t rowT_smem_bytes(int nw) {
  size_t b = ((size_t)nw * 32 * 33 + (size_t)nw * 68 + (size_t)2 * nw * 64) * sizeof(T);
  b = (b + 15) & ~(size_t)15;
  return b + (size_t)2 * nw * sizeof(double);
}

template <typename T>
void seg_launch(const DevView& v, const LaunchShape& sh, cudaStream_t st) {
  const int threads = min(sh.rows_threads, 256);
  int base = 0;
  for (int nw = 1; nw <= 16; ++nw) {
    if (sh.rtT_n[nw] > 0) rowsT_kernel<T><<<sh.rtT_n[nw], 32 * nw, rowT_smem_bytes<T>(nw), st>>>(v, base);
    base += sh.rtT_n[nw];
  }
  for (int c = 0; c < 2; ++c) {
    const int n = sh.rt_seg[c];
    if (n > 0) {
      const int grid = sh.seg_persist ? min(n, sh.seg_grid[c]) : n;
      const size_t sm = sh.seg_smem[c];
      const int cc = sh.seg_ccap[c], mc = sh.seg_mcap[c];
      if (c == 0) {
        if (sh.seg_persist)
          rows_seg_kernel<T, 16, true><<<grid, threads, sm, st>>>(v, base, n, cc, mc);
        else
          rows_seg_kernel<T, 16, false><<<grid, threads, sm, st>>>(v, base, n, cc, mc);
      } else {
        if (sh.seg_persist)
          rows_seg_kernel<T, 32, true><<<grid, threads, sm, st>>>(v, base, n, cc, mc);
        else
          rows_seg_kernel<T, 32, false><<<grid, threads, sm, st>>>(v, base, n, cc, mc);
      }
    }
    base += n;
  }
  if (sh.n_row_tiles > base)
    rows_kernel<T, false><<<sh.n_row_tiles - base, sh.rows_threads, sh.rows_smem, st>>>(v, base);
}

template <typename T>
void colseg_launch(const DevView& v, const LaunchShape& sh, cudaStream_t st) {
  // column tiles ordered by class: S = 16, S = 32 (one CTA per tile), then S = 16, S = 32
  // over CTA pairs (two CTAs per tile)
  int base = 0;
  if (sh.cst_n[0] > 0) colseg_kernel<T, 16><<<sh.cst_n[0], sh.colseg_threads[0], sh.colseg_smem[0], st>>>(v, base);
  base += sh.cst_n[0];
  if (sh.cst_n[1] > 0) colseg_kernel<T, 32><<<sh.cst_n[1], sh.colseg_threads[1], sh.colseg_smem[1], st>>>(v, base);
  base += sh.cst_n[1];
  if (sh.cst_n[2] > 0)
    colseg2_kernel<T, 16><<<2 * sh.cst_n[2], sh.colseg_threads[2], sh.colseg_smem[2], st>>>(v, base);
  base += sh.cst_n[2];
  if (sh.cst_n[3] > 0)
    colseg2_kernel<T, 32><<<2 * sh.cst_n[3], sh.colseg_threads[3], sh.colseg_smem[3], st>>>(v, base);
}

template <typename T>
cudaError_t phase_impl(const DevView& v, int phase, const LaunchShape& sh, cudaStream_t st) {
  if (sh.n_row_tiles == 0) return cudaSuccess;  // no member present
  switch (phase) {
    case 0:
      if (sh.split) {
        const int whole = sh.n_row_tiles - sh.rt_blk;
        if (whole > 0) stencil_kernel<T><<<whole, sh.rows_threads, sh.rows_smem, st>>>(v, 0);
        if (sh.rt_blk > 0) {
          if (sizeof(T) != sizeof(double)) return cudaErrorInvalidValue;  // FP64 only
          stencil_block_kernel<T, false><<<sh.rt_blk, sh.rows_threads, sh.blk_smem, st>>>(v, whole);
        }
      } else
        seg_launch<T>(v, sh, st);
      break;
    case 1: {
      if (!sh.split) return cudaSuccess;
      // segment-form members first (sweep tiles ordered S = 16, S = 32, others)
      const int threads = min(sh.rows_threads, 256);
      if (sh.st_seg[0] > 0) rowseg_kernel<T, 16><<<sh.st_seg[0], threads, 0, st>>>(v, 0);
      if (sh.st_seg[1] > 0) rowseg_kernel<T, 32><<<sh.st_seg[1], threads, 0, st>>>(v, sh.st_seg[0]);
      const int base = sh.st_seg[0] + sh.st_seg[1], rest = sh.n_sweep_tiles - base;
      if (rest <= 0) break;
      if (sh.stream)
        rowstream_kernel<T><<<(rest + kStreamCta - 1) / kStreamCta, 32 * kStreamCta,
                              rowstream_smem_bytes(sizeof(T)), st>>>(v, rest, base);
      else
        rowsweep_kernel<T><<<rest, sh.sweep_threads, sh.sweep_smem, st>>>(v, base);
      break;
    }
    default:
      colseg_launch<T>(v, sh, st);
      if (sh.n_col_tiles == 0)
        break;
      else if (sh.stream)
        colstream_kernel<T><<<(sh.n_col_tiles + kStreamCta - 1) / kStreamCta, 32 * kStreamCta, 0, st>>>(
            v, sh.n_col_tiles, 0);
      else if (sh.cols_persist)
        cols_kernel<T, true><<<min(sh.n_col_tiles, sh.cols_grid), sh.cols_threads, sh.cols_smem, st>>>(
            v, sh.n_col_tiles, sh.cols_panel_cap);
      else
        cols_kernel<T, false><<<sh.n_col_tiles, sh.cols_threads, sh.cols_smem, st>>>(v, sh.n_col_tiles,
                                                                                      sh.cols_panel_cap);
  }
  return cudaGetLastError();
}

// One launch of the resident kernel over the n tiles of one class (clusters of Q CTAs).
template <int NX, int NR, bool COMP, bool OBS>
cudaError_t res_launch(const DevView& v, int base, int n, int Q, int64_t nsteps, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(n * Q), 1, 1);
  cfg.blockDim = dim3(8 * NR, 1, 1);
  cfg.dynamicSmemBytes = res_smem_bytes(NX, NR, COMP);
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)Q;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, res_kernel<NX, NR, COMP, OBS>, v, base, nsteps);
}

template <bool OBS>
cudaError_t res_all(const DevView& v, const LaunchShape& sh, int64_t nsteps, cudaStream_t st) {
  int base = 0;
  for (int ci = 0; ci < kResClasses; ++ci) {
    const int n = sh.res_n[ci];
    if (n <= 0) continue;
    const int Q = ci % 8 + 1;
    const bool comp = (ci / 8) & 1;
    const int form = ci / 16;  // 0: 128 columns, 32 rows; 1: 256 columns, 32 rows; 2: 256, 64
    cudaError_t e;
    if (form == 2)
      e = comp ? res_launch<256, 64, true, OBS>(v, base, n, Q, nsteps, st)
               : res_launch<256, 64, false, OBS>(v, base, n, Q, nsteps, st);
    else if (form == 1)
      e = comp ? res_launch<256, 32, true, OBS>(v, base, n, Q, nsteps, st)
               : res_launch<256, 32, false, OBS>(v, base, n, Q, nsteps, st);
    else
      e = comp ? res_launch<128, 32, true, OBS>(v, base, n, Q, nsteps, st)
               : res_launch<128, 32, false, OBS>(v, base, n, Q, nsteps, st);
    if (e != cudaSuccess) return e;
    base += n;
  }
  return cudaSuccess;
}

template <int NX, int NR, bool COMP>
cudaError_t res_smem_limit() {
  const int b = (int)res_smem_bytes(NX, NR, COMP);
  cudaError_t e = cudaFuncSetAttribute(res_kernel<NX, NR, COMP, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(res_kernel<NX, NR, COMP, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
}

template <typename T>
cudaError_t step_impl(const DevView& v, const LaunchShape& sh, cudaStream_t st) {
  for (int ph = 0; ph < 3; ++ph) {
    cudaError_t e = phase_impl<T>(v, ph, sh, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t observe_impl(const DevView& v, const LaunchShape& sh, cudaStream_t st) {
  // whole-row tiles through the observe mode of rows_kernel, stencil blocks of long rows
  // (last in the list) through the observe mode of stencil_block_kernel
  const int whole = sh.n_row_tiles - sh.rt_blk;
  if (whole > 0) rows_kernel<T, true><<<whole, sh.rows_threads, sh.rows_smem, st>>>(v, 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (sh.rt_blk > 0) {
    if (sizeof(T) != sizeof(double)) return cudaErrorInvalidValue;  // FP64 only
    stencil_block_kernel<T, true><<<sh.rt_blk, sh.rows_threads, sh.blk_smem, st>>>(v, whole);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (sizeof(T) == sizeof(float) && (e = res_all<true>(v, sh, 0, st)) != cudaSuccess) return e;
  obs_finalize_kernel<<<(v.m + 127) / 128, 128, 0, st>>>(v);
  return cudaGetLastError();
}

template <typename T>
cudaError_t smem_limits_impl() {
  const int limit = 227 * 1024;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(rows_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(rows_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(stencil_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(stencil_block_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(stencil_block_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(rowsT_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(rows_seg_kernel<T, 16, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(rows_seg_kernel<T, 32, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(rows_seg_kernel<T, 16, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(rows_seg_kernel<T, 32, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) !=
      cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(rowsweep_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) != cudaSuccess)
    return e;

  if ((e = cudaFuncSetAttribute(rowstream_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(cols_kernel<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(cols_kernel<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
}

}  // namespace

cudaError_t set_kernel_smem_limits(int precision) {
  if (precision == 0) return smem_limits_impl<double>();
  cudaError_t e;
  if ((e = smem_limits_impl<float>()) != cudaSuccess || (e = res_smem_limit<128, 32, false>()) != cudaSuccess ||
      (e = res_smem_limit<128, 32, true>()) != cudaSuccess || (e = res_smem_limit<256, 32, false>()) != cudaSuccess ||
      (e = res_smem_limit<256, 32, true>()) != cudaSuccess || (e = res_smem_limit<256, 64, false>()) != cudaSuccess)
    return e;
  return res_smem_limit<256, 64, true>();
}

size_t resident_smem_bytes(int nx, int nr, int comp) { return res_smem_bytes(nx, nr, comp != 0); }

cudaError_t launch_resident(const DevView& v, int precision, const LaunchShape& sh, int64_t nsteps,
                            const cudaStream_t* streams, int nstreams) {
  if (precision == 0 || nsteps <= 0) return cudaSuccess;
  // the classes present, each on its own stream (round robin)
  int base = 0, j = 0;
  for (int ci = 0; ci < kResClasses; ++ci) {
    const int n = sh.res_n[ci];
    if (n <= 0) continue;
    LaunchShape one{};
    one.res_n[ci] = n;
    const DevView vc = [&] {
      DevView w = v;
      w.res_tiles = v.res_tiles + base;
      return w;
    }();
    const cudaStream_t st = streams[j++ % nstreams];
    for (int64_t done = 0; done < nsteps; done += kResChunk) {
      const int64_t k = nsteps - done < kResChunk ? nsteps - done : kResChunk;
      cudaError_t e = res_all<false>(vc, one, k, st);
      if (e != cudaSuccess) return e;
    }
    base += n;
  }
  return cudaSuccess;
}

int resident_classes(const LaunchShape& sh) {
  int c = 0;
  for (int ci = 0; ci < kResClasses; ++ci) c += sh.res_n[ci] > 0;
  return c;
}

cudaError_t launch_init_members(const DevView& v, int precision, const int* list, int count, int64_t max_points,
                                cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  int64_t blocks = (max_points + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  dim3 grid((unsigned)blocks, (unsigned)(count < 65535 ? count : 65535));
  if (precision == 0)
    init_fields_kernel<double><<<grid, 256, 0, st>>>(v, list, count);
  else
    init_fields_kernel<float><<<grid, 256, 0, st>>>(v, list, count);
  return cudaGetLastError();
}

cudaError_t launch_init_fields(const DevView& v, int precision, int64_t max_points, cudaStream_t st) {
  return launch_init_members(v, precision, nullptr, v.m, max_points, st);
}

cudaError_t launch_step(const DevView& v, int precision, const LaunchShape& sh, cudaStream_t st) {
  return precision == 0 ? step_impl<double>(v, sh, st) : step_impl<float>(v, sh, st);
}

cudaError_t launch_phase(const DevView& v, int precision, int phase, const LaunchShape& sh, cudaStream_t st) {
  return precision == 0 ? phase_impl<double>(v, phase, sh, st) : phase_impl<float>(v, phase, sh, st);
}

cudaError_t launch_observe(const DevView& v, int precision, const LaunchShape& sh, cudaStream_t st) {
  return precision == 0 ? observe_impl<double>(v, sh, st) : observe_impl<float>(v, sh, st);
}

int seg_blocks_per_sm(int precision, int seg, int threads, size_t smem) {
  int n = 0;
  cudaError_t e;
  if (precision == 0)
    e = seg == 16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rows_seg_kernel<double, 16, true>, threads, smem)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rows_seg_kernel<double, 32, true>, threads, smem);
  else
    e = seg == 16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rows_seg_kernel<float, 16, true>, threads, smem)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, rows_seg_kernel<float, 32, true>, threads, smem);
  return e == cudaSuccess ? n : 0;
}

int cols_blocks_per_sm(int precision, int persist, int threads, size_t smem) {
  int n = 0;
  cudaError_t e;
  if (precision == 0)
    e = persist ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cols_kernel<double, true>, threads, smem)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cols_kernel<double, false>, threads, smem);
  else
    e = persist ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cols_kernel<float, true>, threads, smem)
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, cols_kernel<float, false>, threads, smem);
  return e == cudaSuccess ? n : 0;
}

}  // namespace chk
