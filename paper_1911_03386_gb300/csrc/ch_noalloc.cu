// ch_noalloc.cu -- ch_step_field_noalloc: an FP64 Cahn-Hilliard step on a caller-owned
// device field that allocates no device memory (and, when it succeeds, no host memory).
//
// Some callers cannot call cudaMalloc: code embedded in a host framework that owns all
// device memory through its own pool (a stray cudaMalloc bypasses its accounting and can
// fail once the pool has reserved the free memory), real-time loops where an allocation's
// implicit synchronisation and unbounded latency are not allowed after start-up, and
// processes whose device-memory budget is fixed when they start.  ch_create_ensemble
// allocates a handle's buffers, so those callers use this entry point instead: they pass
// the field (input and output, on the device), and the one intermediate the step needs --
// the row-solve result W, nx*ny doubles -- lives in the file-scope array below, which
// exists on every GPU that loads the library from load until process exit.
//
// The kernels are the same two phases as a handle's step (13-point stencil + row sweep,
// then column sweep + update; see ch_kernels.cu) without observables or step counters,
// with the member constants passed by value instead of from device tables.
#include <cstdint>
#include <cstdio>

#include <cuda_runtime.h>

#include "ch.h"

namespace chk {
void record_error(const char* msg);  // ch_api.cu
}

namespace {

// Largest grid the allocation-free step accepts: 1024 x 1024 points (8 MiB of FP64).
constexpr int64_t kNoAllocMaxPoints = (int64_t)1 << 20;

// The scratch.  In host code this name is only a stand-in for the device array: host code
// must use the address returned by cudaGetSymbolAddress, never the name itself.
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocMaxPoints];

constexpr size_t kSmemMax = 227 * 1024;
constexpr int kThreads = 256;

struct StepConsts {
  int nx, ny;
  int kx, ky;      // pre-roll lengths of the x / y recurrences
  int br, bc;      // rows per row-kernel CTA, columns per column-kernel CTA
  double a, bx, by, rho, w0;
  double p1x, p2x, p1y, p2y;
  double kappa;
};

__device__ __forceinline__ int na_wrap(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

__device__ __forceinline__ void na_forward(const double* in, double* out, int es, int n, int K, double p1, double p2) {
  double y1 = 0.0, y2 = 0.0;
  int k = na_wrap(-K, n);
  for (int q = 0; q < K; ++q) {
    const double y = fma(p1, y1, fma(p2, y2, in[k * es]));
    y2 = y1;
    y1 = y;
    if (++k == n) k = 0;
  }
  for (int i = 0; i < n; ++i) {
    const double y = fma(p1, y1, fma(p2, y2, in[i * es]));
    out[i * es] = y;
    y2 = y1;
    y1 = y;
  }
}

__device__ __forceinline__ void na_backward(const double* in, double* out, int es, int n, int K, double p1, double p2) {
  double x1 = 0.0, x2 = 0.0;
  int k = na_wrap(n - 1 + K, n);
  for (int q = 0; q < K; ++q) {
    const double x = fma(p1, x1, fma(p2, x2, in[k * es]));
    x2 = x1;
    x1 = x;
    if (--k < 0) k = n - 1;
  }
  for (int i = n - 1; i >= 0; --i) {
    const double x = fma(p1, x1, fma(p2, x2, in[i * es]));
    out[i * es] = x;
    x2 = x1;
    x1 = x;
  }
}

// Phase 1: rows j0 .. j0+br-1 of C -> mu -> R' -> row sweep -> W (scratch).
__global__ void __launch_bounds__(kThreads) noalloc_rows(const double* __restrict__ C, double* __restrict__ W,
                                                         StepConsts P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nx = P.nx, ny = P.ny;
  const int j0 = blockIdx.x * P.br;
  const int nr = min(P.br, ny - j0);
  const int ld = nx + 1;
  double* Cs = reinterpret_cast<double*>(smem);
  double* Ms = Cs + (size_t)(nr + 4) * ld;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int r = warp; r < nr + 4; r += nwarps) {
    int j = j0 - 2 + r;
    if (j < 0) j += ny;
    if (j >= ny) j -= ny;
    for (int i = lane; i < nx; i += 32) Cs[(size_t)r * ld + i] = C[(int64_t)j * nx + i];
  }
  __syncthreads();
  for (int r = warp; r < nr + 2; r += nwarps) {
    const double* c0 = Cs + (size_t)(r + 1) * ld;
    for (int i = lane; i < nx; i += 32) {
      const int ie = (i + 1 == nx) ? 0 : i + 1, iw = (i == 0) ? nx - 1 : i - 1;
      const double c = c0[i];
      const double u = c * fma(c, c, -P.a);
      Ms[(size_t)r * ld + i] = fma(-P.by, c0[i + ld] + c0[i - ld], fma(-P.bx, c0[ie] + c0[iw], u));
    }
  }
  __syncthreads();
  for (int r = warp; r < nr; r += nwarps) {
    const double* m0 = Ms + (size_t)(r + 1) * ld;
    for (int i = lane; i < nx; i += 32) {
      const int ie = (i + 1 == nx) ? 0 : i + 1, iw = (i == 0) ? nx - 1 : i - 1;
      Cs[(size_t)r * ld + i] = fma(P.w0, m0[i], fma(P.rho, m0[i + ld] + m0[i - ld], m0[ie] + m0[iw]));
    }
  }
  __syncthreads();
  if (threadIdx.x < nr) na_forward(Cs + (size_t)threadIdx.x * ld, Ms + (size_t)threadIdx.x * ld, 1, nx, P.kx, P.p1x, P.p2x);
  __syncthreads();
  if (threadIdx.x < nr) na_backward(Ms + (size_t)threadIdx.x * ld, Cs + (size_t)threadIdx.x * ld, 1, nx, P.kx, P.p1x, P.p2x);
  __syncthreads();
  for (int r = warp; r < nr; r += nwarps)
    for (int i = lane; i < nx; i += 32) W[(int64_t)(j0 + r) * nx + i] = Cs[(size_t)r * ld + i];
}

// Phase 2: columns i0 .. i0+bc-1: W (scratch) -> column sweep -> C += kappa Z.
__global__ void __launch_bounds__(kThreads) noalloc_cols(double* __restrict__ C, const double* __restrict__ W,
                                                         StepConsts P) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int nx = P.nx, ny = P.ny;
  const int i0 = blockIdx.x * P.bc;
  const int nc = min(P.bc, nx - i0);
  const int ldc = nc + 1;
  double* Ws = reinterpret_cast<double*>(smem);
  double* Ys = Ws + (size_t)ny * ldc;
  for (int idx = threadIdx.x; idx < ny * nc; idx += blockDim.x) {
    const int j = idx / nc, c = idx - j * nc;
    Ws[(size_t)j * ldc + c] = W[(int64_t)j * nx + i0 + c];
  }
  __syncthreads();
  if (threadIdx.x < nc) na_forward(Ws + threadIdx.x, Ys + threadIdx.x, ldc, ny, P.ky, P.p1y, P.p2y);
  __syncthreads();
  if (threadIdx.x < nc) na_backward(Ys + threadIdx.x, Ws + threadIdx.x, ldc, ny, P.ky, P.p1y, P.p2y);
  __syncthreads();
  for (int idx = threadIdx.x; idx < ny * nc; idx += blockDim.x) {
    const int j = idx / nc, c = idx - j * nc;
    const int64_t g = (int64_t)j * nx + i0 + c;
    C[g] = fma(P.kappa, Ws[(size_t)j * ldc + c], C[g]);
  }
}

int na_fail(int code, const char* msg) {
  chk::record_error(msg);  // text for ch_last_error(); only on failure
  return code;
}

// Device address of the scratch in the current context, and the kernels' shared-memory
// limit, set up on every call.  Neither allocates.  The address belongs to the module as
// loaded in the current context, so it is not cached: after a device reset, or when the
// caller switches to another context of the same device, the module is loaded again at
// another address, and a cached pointer would then point at freed or unmapped memory.
cudaError_t scratch_address(double** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(noalloc_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(noalloc_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemMax);
  if (e != cudaSuccess) return e;
  *out = static_cast<double*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" int ch_step_field_noalloc(double* C, int nx, int ny, double L, double gamma, double dt, int64_t nsteps,
                                     void* stream) {
  if (!C || nx < 5 || ny < 5 || nsteps < 0) return na_fail(CH_EINVAL, "bad field pointer, size or step count");
  if ((int64_t)nx * ny > kNoAllocMaxPoints)
    return na_fail(CH_EINVAL, "ch_step_field_noalloc: nx*ny exceeds the 1048576-point (1024x1024) scratch limit");
  if (!(L > 0.0) || !(gamma > 0.0) || !(dt > 0.0) || !(L < 1e300) || !(gamma < 1e300) || !(dt < 1e300))
    return na_fail(CH_EINVAL, "L, gamma and dt must be finite and > 0");
  StepConsts P;
  P.nx = nx;
  P.ny = ny;
  const double hx = L / nx, hy = L / ny, hx2 = hx * hx, hy2 = hy * hy;
  P.a = 1.0 - 2.0 * gamma / hx2 - 2.0 * gamma / hy2;
  P.bx = gamma / hx2;
  P.by = gamma / hy2;
  P.rho = hx2 / hy2;
  P.w0 = -2.0 * (1.0 + P.rho);
  const double sigma = gamma * dt;
  double cx, cy;
  if (ch_penta_factor(sigma / (hx2 * hx2), CH_FP64, &cx, &P.p1x, &P.p2x, &P.kx) != CH_OK ||
      ch_penta_factor(sigma / (hy2 * hy2), CH_FP64, &cy, &P.p1y, &P.p2y, &P.ky) != CH_OK)
    return na_fail(CH_EINVAL, "implicit factor out of range");
  P.kappa = dt / (hx2 * cx * cy);
  // band height and panel width that fit the shared memory (same rule as the handles)
  int br = ny < 16 ? ny : 16;
  while (br > 1 && (size_t)(2 * br + 6) * (nx + 1) * sizeof(double) > kSmemMax) br = (br + 1) / 2;
  int bc = nx < 16 ? nx : 16;
  while (bc > 1 && (size_t)2 * ny * (bc + 1) * sizeof(double) > kSmemMax) bc = (bc + 1) / 2;
  const size_t rows_smem = (size_t)(2 * br + 6) * (nx + 1) * sizeof(double);
  const size_t cols_smem = (size_t)2 * ny * (bc + 1) * sizeof(double);
  if (rows_smem > kSmemMax || cols_smem > kSmemMax) return na_fail(CH_EINVAL, "grid line too long");
  P.br = br;
  P.bc = bc;
  double* W = nullptr;
  if (scratch_address(&W) != cudaSuccess) return na_fail(CH_ECUDA, "scratch set-up failed");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int row_blocks = (ny + br - 1) / br, col_blocks = (nx + bc - 1) / bc;
  // Launch errors are read with cudaPeekAtLastError, which leaves the error state as it
  // is for the caller.  A failure here returns with the steps before it already enqueued.
  for (int64_t s = 0; s < nsteps; ++s) {
    noalloc_rows<<<row_blocks, kThreads, rows_smem, st>>>(C, W, P);
    noalloc_cols<<<col_blocks, kThreads, cols_smem, st>>>(C, W, P);
    if (cudaPeekAtLastError() != cudaSuccess) return na_fail(CH_ECUDA, "ch_step_field_noalloc: launch failed");
  }
  return CH_OK;
}
