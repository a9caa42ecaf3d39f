// ch_internal.h -- data layout shared by the CUDA kernels and the host side of libch.
//
// Device memory of one handle (all owned by the handle):
//   C, W        field and row-solve scratch, one contiguous ny x nx block per member at
//               MemberParams::offset (elements), FP64 or FP32 by the handle's precision;
//   members     MemberParams[m]   constants of each run (read-only after creation);
//   state       MemberState[m]    step index, horizon, sampling accumulators;
//   row_tiles   Tile[]            one CTA of the stencil (or fused row) kernel per band of rows;
//   sweep_tiles Tile[]            one CTA of the row-sweep kernel per band (split form);
//   col_tiles   Tile[]            one CTA of the column kernel per tile (a column panel);
//   partials    double2[]         FP64 (sum F density, sum dF/dt density) per row band;
//   series      double[m][cap][4] ring of (t, F, dF/dt, beta) samples per member.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace chk {

constexpr int64_t kUnbounded = INT64_MAX;

constexpr int kBlockCols = 256;  // columns of a stencil block (long rows, FP64 split form)

struct MemberParams {
  int64_t offset;        // first element of the member's field in C and W
  int nx, ny;
  int kx, ky;            // pre-roll lengths of the x / y recurrences (see ch_kernels.cu)
  int kx32;              // FP64 streaming row sweeps: leading pre-roll points run in FP32 (0: none)
  int nbands;            // row tiles of this member = partial slots per sample
  int rows_p, cols_p;    // threads per line in the row / column sweep
  int seg_g;             // segment form of the row sweep: lanes per row (nx / S), 0 = chunked
  int col_s;             // segment form of the column kernel: rows per warp S, 0 = panels / streaming
  int row_t;             // transposed-block form of the row kernel: nw = nx / 32 warps, 0 = other forms
  int every;             // sampling period in steps
  int64_t partial_base;  // first partial slot
  int64_t series_cap;    // samples kept per member (ring)
  double L, hx, hy, gamma, dt;
  // chemical potential  mu = C (C^2 - a) - bx (Ce + Cw) - by (Cn + Cs)
  double a, bx, by;
  // scaled explicit right-hand side  R' = (mu_e + mu_w) + rho (mu_n + mu_s) + w0 mu,
  // R = dt lap_h mu = (dt / hx^2) R'
  double rho, w0;
  // spectral factor of the cyclic pentadiagonal operator  I + s D^4 = c Q Q^T,
  // Q y = r  <=>  y_i = r_i + p1 y_{i-1} + p2 y_{i-2}   (indices mod n)
  double p1x, p2x, cx;
  double p1y, p2y, cy;
  // C^{n+1} = C^n + kappa Z,  Z = Q_y^-T Q_y^-1 Q_x^-T Q_x^-1 R',  kappa = dt/(hx^2 cx cy)
  double kappa;
  double t1;             // start of the beta time-average window
  double C0;
  uint64_t seed, counter_base;
  // the constants above rounded to FP32, for the FP32 kernels
  float fa, fbx, fby, frho, fw0, fp1x, fp2x, fp1y, fp2y, fkappa;
  // FP32 form at large s: the field is the unevaluated pair hi + lo of FP32 values (hi in
  // C at offset, lo in C at lo_offset); the update keeps the rounding error of hi in lo
  int comp;              // 1: compensated update (lo_offset valid)
  int64_t lo_offset;     // first element of the lo part in C, -1 if none
};

// Scan tables of the segment form of the row sweep (S points per lane, G lanes per row),
// for the companion matrix M = [[p1, p2], [1, 0]] of the recurrence, 2x2 row-major:
// A[d] = M^(S 2^d) (scan steps), B[l] = M^(S l) (start state of lane l from the periodic
// start state), P = (I - M^nx)^-1 (periodic start state from the scan total).
struct SegTable {
  double A[5][4];
  double B[64][4];       // up to 64 segments: columns over a CTA pair (rows use at most 32)
  double P[4];
  float Af[5][4];        // the same rounded to FP32
  float Bf[64][4];
  float Pf[4];
  // Closed-form responses of one segment of S <= 32 points (cluster-resident column
  // kernel), FP32: Hf[u] = (g1_u, g2_u, k1_u, k2_u) where, on a segment with start states
  // s = (y_-1, y_-2) of the forward and t = (x_S, x_S+1) of the backward recurrence,
  // x_u = G0(F0(r))_u + g1_u s_0 + g2_u s_1 + k1_u t_0 + k2_u t_1 (F0, G0: the forward and
  // backward recurrences from zero states; g = G0 of the forward homogeneous responses,
  // k = the backward homogeneous responses).
  float Hf[32][4];
};

struct MemberState {
  int64_t step;          // index n of the current field C^n
  int64_t remaining;     // steps still to run (kUnbounded: no horizon)
  int active;            // written by the row kernel: member steps in this launch pair
  int nonfinite;         // set once F or dF/dt is not finite
  int64_t nsamples;      // samples taken since the last reset
  int64_t beta_count;
  double beta_sum;
  double F, dFdt, beta;  // last sample
};

struct Tile {
  int member;
  int start;             // first row (row tiles) or first column (column tiles)
  int count;             // rows / columns in the tile
  int index;             // band / panel number within the member
  int x0, xn;            // stencil blocks of long rows: first column and width (else 0, 0)
};

struct DevView {
  void* C;
  void* W;
  const MemberParams* mp;
  MemberState* ms;
  const Tile* row_tiles;
  const Tile* sweep_tiles;
  const Tile* col_tiles;
  double2* partials;
  double* series;
  double* obs_now;       // [m][3] F, dF/dt, beta of ch_observables
  const SegTable* seg;   // [m] scan tables (segment form of the row sweep)
  const SegTable* segy;  // [m] scan tables of the y recurrence (segment form of the column kernel)
  const Tile* colseg_tiles;  // CTAs of the segment-form column kernel
  const Tile* res_tiles;     // one per member of the cluster-resident form (FP32)
  int m;
};

// Cluster-resident form (FP32): a member with nx = 128 or 256 and ny = NR Q (NR = 32 rows per
// CTA, Q = 1 .. 8; or NR = 64, nx = 256, Q = 1 .. 4) is stepped by a cluster of Q CTAs that
// keep its field in shared memory for a whole chunk of steps.  Its tiles are ordered by
// class (form, compensated, Q) with form 0: nx = 128, NR = 32; 1: nx = 256, NR = 32;
// 2: nx = 256, NR = 64 -- class index = (form * 2 + comp) * 8 + Q - 1.
constexpr int kResClasses = 48;
constexpr int64_t kResChunk = 4096;  // steps per launch of the resident kernel
inline int res_class(int nx, int nr, int comp, int Q) {
  const int form = nx == 128 ? 0 : (nr == 32 ? 1 : 2);
  return (form * 2 + (comp ? 1 : 0)) * 8 + Q - 1;
}

// Launch shapes chosen on the host per handle (see ch_api.cu).
struct LaunchShape {
  int split;             // 1: stencil_kernel + rowsweep_kernel, 0: fused rows_kernel
  int stream;            // 1 (split only): rowstream_kernel + colstream_kernel, 32-line tiles
  int n_row_tiles, n_sweep_tiles, n_col_tiles;
  int rows_threads;      // threads per stencil / fused CTA
  size_t rows_smem;      // dynamic shared memory (max over tiles)
  int sweep_threads;
  size_t sweep_smem;
  int cols_threads;
  size_t cols_smem;
  int cols_persist;      // 1: cols_kernel walks panels with double-buffered copies
  int cols_grid;         // CTAs of the persistent column kernel (SMs x resident CTAs)
  int cols_panel_cap;    // elements of one panel buffer
  // Row tiles are ordered by kernel class: first the transposed-block form (32-row bands),
  // grouped by nw = nx / 32 (rtT_n[nw] tiles for nw = 1 .. 16), then the segment form
  // with S = 16 (rt_seg[0] tiles) and S = 32 (rt_seg[1]), then the chunked form.
  int rtT_n[17];
  int rt_seg[2];
  // split form, FP64: members whose rows do not fit a shared-memory band run the stencil in
  // blocks of rows x kBlockCols columns (stencil_block_kernel); their rt_blk tiles come last
  int rt_blk;
  size_t blk_smem;
  // split form: sweep tiles ordered S = 16 (st_seg[0]), S = 32 (st_seg[1]) segment-form
  // members (rowseg_kernel), then the others
  int st_seg[2];
  int seg_persist;       // 1: the segment row kernel walks its tiles with a double-buffered C band
  int seg_grid[2];       // CTAs of the persistent segment row kernel
  int seg_ccap[2], seg_mcap[2];  // elements of one C tile buffer / of the mu tile (max over the class)
  size_t seg_smem[2];    // dynamic shared memory of the segment-form row kernel
  // Column tiles of the segment form: cst_n[0] with S = 16, cst_n[1] with S = 32 (one CTA
  // per tile), then cst_n[2], cst_n[3] with S = 16, 32 over CTA pairs (tall columns).
  int cst_n[4];
  int colseg_threads[4];
  size_t colseg_smem[4];
  // cluster-resident members (FP32): tiles per class (see res_class)
  int res_n[kResClasses];
};

// Host-side fault injection (ch_fault.cu; armed by ch_set_fault or CH_FAULT).
enum { kFaultNone = 0, kFaultAlloc = 1, kFaultNan = 2, kFaultTimeout = 3 };
// Every device allocation of the library goes through here: an armed alloc fault makes
// the N-th one report cudaErrorMemoryAllocation without allocating.
cudaError_t dev_malloc(void** p, size_t bytes);
template <class T>
cudaError_t dev_malloc(T** p, size_t bytes) {
  return dev_malloc(reinterpret_cast<void**>(p), bytes);
}
// 1 (and the fault's argument) if a fault of this kind is armed, disarming it.
int take_fault(int kind, int64_t* arg);
// An armed nan fault writes a NaN into the first grid point of member arg (host-to-device
// copy on st); mp: the host copy of the member constants.
cudaError_t inject_nan(void* C, int precision, const MemberParams* mp, int m, cudaStream_t st);
// An armed timeout fault stalls the calling host thread for its milliseconds.
void stall_if_armed();

// Kernel launchers (ch_kernels.cu).  Each returns the launch status.
cudaError_t launch_init_fields(const DevView& v, int precision, int64_t max_points, cudaStream_t st);
// Initial fields of the members listed in `list` (device array of count member indices).
cudaError_t launch_init_members(const DevView& v, int precision, const int* list, int count, int64_t max_points,
                                cudaStream_t st);
// One step = phases 0 (stencil or fused rows), 1 (row sweep, split form only), 2 (columns).
cudaError_t launch_step(const DevView& v, int precision, const LaunchShape& sh, cudaStream_t st);
cudaError_t launch_phase(const DevView& v, int precision, int phase, const LaunchShape& sh, cudaStream_t st);
cudaError_t launch_observe(const DevView& v, int precision, const LaunchShape& sh, cudaStream_t st);
// nsteps steps of every cluster-resident member (no-op when there are none), in launches
// of at most kResChunk steps; each class present goes to streams[i % nstreams].
cudaError_t launch_resident(const DevView& v, int precision, const LaunchShape& sh, int64_t nsteps,
                            const cudaStream_t* streams, int nstreams);
// Number of resident classes present in a launch shape.
int resident_classes(const LaunchShape& sh);
// Dynamic shared memory of the cluster-resident kernel for rows of nx floats, nr per CTA.
size_t resident_smem_bytes(int nx, int nr, int comp);
cudaError_t set_kernel_smem_limits(int precision);
// Resident CTAs per SM of the column kernel for a launch shape (0 on error).
int cols_blocks_per_sm(int precision, int persist, int threads, size_t smem);
// Resident CTAs per SM of the persistent segment row kernel (0 on error).
int seg_blocks_per_sm(int precision, int seg, int threads, size_t smem);

}  // namespace chk
