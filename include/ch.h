/*
 * ch.h -- C ABI of the GB300 Cahn-Hilliard ensemble engine (libch.so).
 *
 * The engine time-steps ensembles of independent periodic 2-D Cahn-Hilliard runs
 *     dC/dt = lap(C^3 - C - gamma lap C)                      (paper Sec. 1, Eq. (3))
 * and accumulates, per run, the free energy F and dF/dt       (Sec. 1, Eq. (4)),
 * the coarsening rate beta = -(t/F) dF/dt                     (Sec. 1, Eq. (6))
 * and the time average of beta over a window [t1, T]          (Sec. 3.3, Eq. (42); the
 * window [20, 100] of Sec. 4.2, Table 4).  The paper (Sec. 4.1) runs M = 1024 such
 * simulations with "semi-implicit ADI finite differences, periodic in both directions";
 * this library's scheme is the delta-form approximate factorisation
 *     (I + s D_x^4)(I + s D_y^4)(C^{n+1} - C^n) = dt lap_h(C^3 - C - gamma lap_h C)^n,
 *     s = gamma dt,  D^4 = (D^2)^2,  lap_h the 5-point Laplacian, h = L/n per axis,
 * so one step is a 13-point explicit stencil followed by cyclic pentadiagonal solves
 * along every row and then every column.
 *
 * Conventions
 *  - All functions return CH_OK (0) on success or a negative CH_E* code; a message for
 *    the last failure on the calling host thread is in ch_last_error().
 *  - Fields are row-major ny x nx arrays, x fastest: C[j*nx + i] is at (i*L/nx, j*L/ny).
 *  - Host pointers are caller-owned and only read/written during the call.  The library
 *    allocates and owns all device memory of a handle (released by ch_destroy).
 *  - A handle is not thread-safe: use one handle per host thread.  Work is enqueued on the
 *    handle's CUDA stream (its own by default, or the caller's via ch_set_stream); calls
 *    that return host data synchronise that stream only.
 *  - Precision: CH_FP64 keeps fields and all arithmetic in FP64.  CH_FP32 keeps fields,
 *    the stencil and the sweeps in FP32 (sweep coefficients computed in FP64, rounded
 *    once), while the F / dF/dt reductions, beta and its time average stay in FP64.
 */
#ifndef CH_H_
#define CH_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define CH_OK 0
#define CH_PENDING 1         /* ch_poll: request not finished yet */
#define CH_EINVAL (-1)       /* invalid argument (sizes, NULL pointers, non-finite values) */
#define CH_ENOMEM (-2)       /* device or host allocation failed, or over the HBM budget */
#define CH_ECUDA (-3)        /* a CUDA runtime call failed (message in ch_last_error) */
#define CH_ENONFINITE (-4)   /* a run's F or dF/dt became NaN/Inf (the run has diverged) */
#define CH_ETIMEOUT (-5)     /* a bounded wait ran out */
#define CH_EBUSY (-6)        /* the serving queue is full */
#define CH_ENOTFOUND (-7)    /* unknown request id */

/* Precision forms. */
#define CH_FP64 0
#define CH_FP32 1

typedef struct ch_ensemble* ch_handle;

/*
 * One member of an uneven batch: an independent run on its own nx x ny periodic grid
 * over [0,L)^2 with interface parameter gamma and step dt.  The initial field is
 *     C = C0 + 0.1 (2u - 1),  u = top 53 bits of SplitMix64 draw k times 2^-53,
 *     k = counter_base + j*nx + i,   SplitMix64 stream seeded with `seed`
 * (the uniform-noise initial condition of Sec. 4.1 about the mean C0; SplitMix64 as
 * published by Steele, Lea & Flood, OOPSLA 2014).
 */
typedef struct {
  int nx, ny;              /* grid points per axis, each >= 5 */
  double L;                /* domain edge, > 0 */
  double gamma;            /* > 0 */
  double dt;               /* > 0 */
  double C0;               /* mean of the initial field, finite */
  uint64_t seed;
  uint64_t counter_base;
} ch_member_desc;

/*
 * Create an ensemble of m members sharing nx, ny, L, gamma, dt (Sec. 4.1, Table 3: one
 * ensemble = M runs of one size).  Member k starts from C0[k] + noise, with draws
 * counter_base = k*nx*ny of the stream `seed`.  C0 is host memory of length m (read
 * during the call only).  precision is CH_FP64 or CH_FP32.  Sampling defaults to every
 * step with the beta window starting at t1 = 0 (see ch_set_sampling).
 * Errors: CH_EINVAL (nx or ny < 5, m < 1, L/gamma/dt not > 0, non-finite C0, bad
 * precision, NULL out), CH_ENOMEM, CH_ECUDA.
 */
int ch_create_ensemble(int nx, int ny, double L, double gamma, double dt, int m,
                       const double* C0, uint64_t seed, int precision, ch_handle* out);

/*
 * Create an uneven batch: m members of differing sizes and parameters (d: host array of
 * length m), stepped together by the same kernels in one launch per phase.
 * Errors as ch_create_ensemble, per member.
 */
int ch_create_batch(int m, const ch_member_desc* d, int precision, ch_handle* out);

/* Release every device and host resource of h (NULL is ignored).  Synchronises first. */
void ch_destroy(ch_handle h);

/*
 * Run all further work of h on the caller's CUDA stream (a cudaStream_t passed as void*;
 * NULL restores the handle's own stream).  Captured step graphs are discarded.
 */
int ch_set_stream(ch_handle h, void* cuda_stream);

/*
 * Sampling of the observables (Sec. 1 Eqs. (4), (6)): on every step index n with
 * n % every == 0, F_h, dF_h/dt and beta = -(t_n/F_h) dF_h/dt, t_n = n dt, are taken
 * from C^n (before that step's update) and appended to the member's series ring of
 * `capacity` samples (0: keep none).  Samples with t_n >= t1 enter the running time
 * average of beta (rectangle rule, the discrete form of Sec. 3.3 Eq. (42)).
 * Resets the series and the averages.  Errors: CH_EINVAL (every < 1, capacity < 0,
 * t1 not finite).
 */
int ch_set_sampling(ch_handle h, int every, double t1, int64_t capacity);

/*
 * Advance every member by nsteps >= 0 steps (asynchronous on the handle's stream; the
 * launches are replayed from captured CUDA graphs).  Errors: CH_EINVAL, CH_ECUDA.
 */
int ch_step(ch_handle h, int64_t nsteps);

/* Wait for the handle's stream.  Errors: CH_ECUDA. */
int ch_synchronize(ch_handle h);

/*
 * F_h, dF_h/dt and beta of the current fields, one value per member (host arrays of
 * length m, any of them may be NULL).  Discretisation of Eq. (4) with forward
 * differences:  F_h = hx hy sum[1/4 (C^2-1)^2 + gamma/2 ((D+x C)^2 + (D+y C)^2)],
 * dF_h/dt = -hx hy sum[(D+x mu)^2 + (D+y mu)^2], mu = C^3 - C - gamma lap_h C;
 * beta = -(t/F) dF/dt at t = n dt (Eq. (6)).  Synchronises the stream.
 * Errors: CH_ENONFINITE if any member's field is not finite, CH_ECUDA.
 */
int ch_observables(ch_handle h, double* F, double* dFdt, double* beta);

/*
 * Per-member running time average of beta over the samples with t >= t1 (host arrays of
 * length m; either may be NULL): avg[k] = sum / count (NaN when count is 0).
 * Synchronises the stream.
 */
int ch_beta_avg(ch_handle h, double* avg, int64_t* count);

/*
 * Copy member k's series to out (host, 4 doubles per sample: t, F, dF/dt, beta), oldest
 * first, at most cap samples; *n receives the number written.  Synchronises.
 */
int ch_series(ch_handle h, int member, double* out, int64_t cap, int64_t* n);

/* Copy member k's current field to out (host, ny*nx doubles; FP32 fields are widened). */
int ch_get_field(ch_handle h, int member, double* out);

/*
 * Overwrite member k's field with in (host, ny*nx doubles; rounded to FP32 in the FP32
 * form).  Does not change the step index.  Synchronises.
 */
int ch_set_field(ch_handle h, int member, const double* in);

/*
 * Bulk transfer of every member's field: `in` / `out` hold the members in order, member
 * k as ny_k*nx_k doubles (total = sum of nx*ny).  With page-locked host buffers the FP64
 * copies are asynchronous DMA; FP32 fields are converted on the host.  Synchronises.
 */
int ch_set_fields(ch_handle h, const double* in);
int ch_get_fields(ch_handle h, double* out);

/*
 * Launch one phase of a step for every member, on the handle's stream: phase 0 = the
 * 13-point stencil (observables on sample steps), fused with the row sweep in the fused
 * form; phase 1 = the row sweep in the split form (nothing in the fused form); phase 2 =
 * the column kernel (column sweep, update, sample finalisation, step counter).  Phases 0,
 * 1, 2 in order are exactly one ch_step(h, 1) of every member outside the cluster-resident
 * form (ch_tuning.resident), whose members the phases leave unchanged; they exist
 * separately so callers can time each kernel with events on the stream.
 * Errors: CH_EINVAL (phase), CH_ECUDA.
 */
int ch_launch_phase(ch_handle h, int phase);

/*
 * Launch shape of a handle's kernels (no effect on results beyond round-off order within
 * a line's recurrence chunks; every choice is checked by the parity tests).  Fields <= 0
 * (split: -1) take the precision's default.
 *   split       1: stencil and row sweep as separate kernels (default for CH_FP64: all
 *               threads of the stencil kernel do FP64 work, the sweeps run as many
 *               independent recurrences per SM); 0: one fused row kernel (default for
 *               CH_FP32: R' stays on chip, 5 words of traffic per point and step).
 *   rows_band   rows per stencil / fused CTA (default 16 FP64, 32 FP32).
 *   rows_p      fused form: threads per row in the row sweep (chunks pre-rolled alone).
 *   sweep_band  split form: rows (one thread each) per row-sweep CTA (default 32).
 *   cols_panel  columns per column CTA (default 32).
 *   cols_p      threads per column (default 1 FP64; FP32 chosen from ny).
 *   threads     threads per stencil / fused / column CTA, multiple of 32, <= 512
 *               (default 512 FP64, 256 FP32).
 *   stream      1 = streaming sweeps (a warp streams 32 lines through small
 *               double-buffered tiles or straight from global memory, the pass
 *               intermediate kept in the scratch field), so recurrences in flight are not
 *               limited by shared memory: rows and columns in the split form, the columns
 *               of members outside the segment column form in the fused form; 0 = whole
 *               lines resident in shared memory (sweep_band, cols_panel, cols_p apply).
 *               Default: 1 for CH_FP64, 0 for CH_FP32.
 *   persist     bit 0: the column kernel runs one CTA per resident slot and walks its
 *               panels with double-buffered copies (the next panel loads while the current
 *               one is swept); bit 1: the same for the segment-form row kernel (the next
 *               band's C rows load while the current band is computed).  0 = one CTA per
 *               panel / band (default).
 *   row_seg     fused form: segment form of the row sweep with S = row_seg points per
 *               lane (16 or 32): a row is held in registers by nx/S lanes and every
 *               recurrence runs as a local pass, a scan of the segment end states across
 *               the lanes and a second pass from the exact start state (no pre-roll;
 *               rows_p does not apply).  Needs nx/S to be a power of two <= 32 for every
 *               member.  0 = automatic (16 if every member fits, else 32 if every member
 *               fits, else the chunked sweep); -1 = chunked sweep.  1 = transposed-block
 *               form (nx = 32 nw, nw <= 16): a warp takes 32 columns of a 32-row band, runs
 *               the stencil with lane = column straight from HBM, transposes its 32 x 32
 *               block of R' through shared memory and runs the row recurrences with lane =
 *               row, joining the nw segments of a row through shared memory (explicit
 *               only).  Kernel classes are chosen per member (automatic: segment S = 16,
 *               else S = 32, else chunked), so a run's arithmetic does not depend on the
 *               other members; an explicit value applies to every member.
 *   col_seg     segment form of the column kernel with S = col_seg rows per warp (16 or
 *               32): lanes take adjacent columns, a column's ny/S segments sit in ny/S
 *               warps, W and C move as coalesced row pieces straight between registers
 *               and HBM, and each recurrence is a local pass, a combination of the segment
 *               end states through shared memory and a second pass (no pre-roll, no
 *               panels in shared memory).  Up to 32 segments (16 for CH_FP64) sit in one
 *               CTA; taller columns (up to 64 / 32 segments) are split over the two CTAs
 *               of a thread-block cluster, which exchange their segment end states through
 *               distributed shared memory.  Needs ny/S to be a power of two within those
 *               limits for every member.  0 = automatic, per member: S = 32 in one CTA,
 *               else S = 16 in one CTA, else S = 32, else 16 over a CTA pair, else panels
 *               or streaming (CH_FP64 split form: streaming for every member); -1 = panels
 *               or streaming.
 *   resident    cluster-resident form of CH_FP32 members with nx = 128 or 256 and
 *               ny = 32 Q, Q = 1 .. 8: the member's field stays in the shared memory of a
 *               cluster of Q CTAs (32 rows each, two halo rows per side) for a launch of
 *               up to 4096 steps; the row recurrences are segment scans across 16 lanes
 *               per row, the column recurrences combine their segment end states through
 *               distributed shared memory, and neighbouring CTAs exchange halo rows by
 *               remote shared-memory stores.  HBM then moves the field once per launch
 *               instead of five words per point and step.  The phase launches
 *               (ch_launch_phase, ch_debug_row_solve) do not touch such members.
 *               0 = on for every member that fits except compensated members 256 wide
 *               (their tiles need 118 KB of shared memory per CTA, one CTA per SM, and
 *               the tiled kernels are faster there) (default); 1 = on for every member
 *               that fits; -1 = off.
 *   resident_rows  rows of a resident member per CTA: 32 (clusters of ny/32 CTAs of 256
 *               threads, two per SM) or 64 (256-column members with ny a multiple of 64:
 *               clusters of ny/64 CTAs of 512 threads, one per SM, half the CTAs per
 *               member); 0 = default.
 *   preroll_head  FP64 streaming row sweeps (stream): the leading points of every row
 *               pre-roll run in FP32 from the zero state and the rest in FP64 from it; the
 *               FP64 part is long enough that the FP32 part's rounding reaches the line
 *               damped below the pre-roll's own 1e-17 tolerance (ch_preroll_head), so the
 *               FP64 pipe does fewer operations for the same result to FP64 round-off.
 *               0 = on (default); -1 = every pre-roll point in FP64.
 * Bands and panels shrink per member to fit 227 KB of shared memory.  Captured step
 * graphs are discarded.  Errors: CH_EINVAL (negative fields, products above the CTA
 * size, lines too long for shared memory, a row_seg that some member's nx does not fit).
 */
typedef struct {
  int split;
  int rows_band;
  int rows_p;
  int sweep_band;
  int cols_panel;
  int cols_p;
  int threads;
  int stream;
  int persist;
  int row_seg;
  int col_seg;
  int resident;
  int resident_rows;
  int preroll_head;
} ch_tuning;
int ch_set_tuning(ch_handle h, const ch_tuning* t); /* NULL restores the defaults */
int ch_get_tuning(ch_handle h, ch_tuning* t);       /* shape in effect (member 0's values) */

/* Step index n of member k (t = n dt). */
int ch_get_step(ch_handle h, int member, int64_t* n);

/* Regenerate every initial field, set the step index to 0 and clear samples/averages. */
int ch_reset(ch_handle h);

/* Number of members; per-member grid size (either pointer may be NULL). */
int ch_num_members(ch_handle h, int* m);
int ch_member_shape(ch_handle h, int member, int* nx, int* ny);

/*
 * Row-solve output of the current fields, for testing the row phase on its own: runs the
 * stencil and row-sweep phases (not the column phase; fields, step indices and samples
 * are unchanged) and copies member k's W = (I + s D_x^4)^-1 R, R = dt lap_h mu, into out
 * (host, ny*nx doubles).  Synchronises.
 */
int ch_debug_row_solve(ch_handle h, int member, double* out);

/*
 * Checkpoint / resume: write or read every field, step index, sample series and
 * average accumulator of h to/from the file at path (the resumed run continues
 * bit-identically).  ch_load needs a handle created with the same members and precision.
 * Errors: CH_EINVAL (mismatch), CH_ECUDA, CH_ENOMEM.
 */
int ch_save(ch_handle h, const char* path);
int ch_load(ch_handle h, const char* path);

/*
 * Host-side constants of one implicit factor, no GPU work: for the cyclic pentadiagonal
 * operator I + s D^4 (stencil [s, -4s, 1+6s, -4s, s], s = gamma dt / h^4 > 0) returns
 * c, p1, p2 with  I + s D^4 = c Q Q^T,  Q y = r  <=>  y_i = r_i + p1 y_{i-1} + p2 y_{i-2}
 * (indices mod n), and the pre-roll length K after which a recurrence started from a zero
 * state agrees with the periodic solution to the precision's round-off (CH_FP64 or
 * CH_FP32).  These are the coefficients the sweeps use (Sec. 4.1: each ADI direction is
 * a batch of pentadiagonal solves).  Any output pointer may be NULL.
 * Errors: CH_EINVAL (s not finite or <= 0, bad precision, no convergence).
 */
int ch_penta_factor(double s, int precision, double* c, double* p1, double* p2, int* K);

/*
 * Host-side split of an FP64 pre-roll, no GPU work: for the recurrence of
 * ch_penta_factor(s, CH_FP64) (companion matrix M = [[p1, p2], [1, 0]], pre-roll length K)
 * returns in *head the number of leading pre-roll points that the FP64 streaming row
 * sweeps run in FP32 (ch_tuning.preroll_head).  The FP32 part starts from the zero state
 * with its inputs truncated to FP32 and FP32 coefficients; its state error is at most
 *   E = g2 2^-24 (3 + g (3 + |p1| + |p2|)) R,
 * R the line's largest input, g = sum_k |(M^k)_00| (the impulse response's l1 norm) and
 * g2 = sum_k ||M^k||_inf; the K - head FP64 points that follow multiply it by M^(K - head).
 * head is the largest multiple of 16 with ||M^(K - head)||_inf E <= 1e-17 R, the
 * tolerance K itself is chosen for, or 0.  Either output pointer may be NULL.
 * Errors: CH_EINVAL (s as in ch_penta_factor).
 */
int ch_preroll_head(double s, int* K, int* head);

/*
 * Host-side scan tables of the segment form of the row sweep (ch_tuning.row_seg), no GPU
 * work: for the recurrence y_i = r_i + p1 y_{i-1} + p2 y_{i-2} on a periodic line of
 * n = seg * groups points split into `groups` segments of `seg` points, with companion
 * matrix M = [[p1, p2], [1, 0]] acting on the state (y_i, y_{i-1}), writes 152 doubles to
 * out (host memory, caller-owned), each 2x2 matrix row-major:
 *   out[0..19]    M^(seg 2^d), d = 0..4          (steps of the scan over the segments)
 *   out[20..147]  M^(seg l),   l = 0..31          (start state of segment l from x0)
 *   out[148..151] (I - M^n)^-1                     (periodic start state x0)
 * Entries for d >= log2(groups) or l >= groups are zero.  p1, p2 are those of
 * ch_penta_factor(s).  Errors: CH_EINVAL (s as in ch_penta_factor, seg < 1, groups not a
 * power of two in [1, 32], out NULL).
 */
int ch_seg_tables(double s, int seg, int groups, double* out);

/*
 * Allocation-free step (the paper has no counterpart; this is a deployment aid).
 * Advance one FP64 field C -- ny*nx doubles in device memory, row-major, owned by the
 * caller, read and overwritten in place -- by nsteps steps of the same scheme as
 * ch_step (grid nx x ny over [0,L)^2, gamma, dt), enqueued on `stream` (a cudaStream_t,
 * NULL for the legacy default stream).  No observables or step counters are kept.
 *
 * For callers that cannot call cudaMalloc: code inside a host framework that owns all
 * device memory through its own pool allocator, real-time loops that forbid an
 * allocation's synchronisation and latency after start-up, and processes whose device
 * memory budget is fixed at start.  The call allocates no device memory (on success it
 * touches no host heap either): its one intermediate, the row-solve result W, lives in a
 * static device array of 1,048,576 doubles (8 MiB) that every GPU loading libch holds
 * until the process exits.  So nx*ny must be <= 1,048,576 (e.g. 1024 x 1024); larger
 * grids are rejected with CH_EINVAL and a message in ch_last_error().
 *
 * Every call looks up the array's device address in the current context
 * (cudaGetSymbolAddress, which allocates nothing) and sets the kernels' shared-memory
 * limits, so a device reset or a switch to another context between calls is safe.  The
 * first call on a device also loads the library's kernels there: make it before any
 * stream capture on that device.  All calls on a device share the array, which keeps
 * the last call's contents; every step overwrites all of W before reading it, so
 * nothing needs clearing.  Calls whose work overlaps on the GPU (other streams, other
 * host threads) race on the array: serialise them.
 * Errors: CH_EINVAL (NULL C, nx or ny < 5, nx*ny above the limit, L/gamma/dt not finite
 * and > 0, nsteps < 0), CH_ECUDA (set-up or launch failed).  Launch errors are read
 * without clearing the CUDA error state, so an error the caller left pending also gives
 * CH_ECUDA (and stays pending).  After CH_ECUDA the field may have advanced by fewer than
 * nsteps steps: the steps enqueued before the failure still run.
 */
int ch_step_field_noalloc(double* C, int nx, int ny, double L, double gamma, double dt, int64_t nsteps,
                          void* stream);

/* ------------------------------------------------------------------------------------ */
/* Ensemble statistics of beta, computed on the device from sampled series.               */
/*                                                                                        */
/* The paper's analysis of an ensemble (Sec. 3.3 Eqs. (41a,b), (42); Secs. 4.2-4.3,        */
/* Tables 4-5) works on beta_j(t) of M runs sampled at common times.  A value that is not */
/* finite (a diverged run) is left out of its sample's statistics, and the number of      */
/* values used is reported.  The dense forms take device arrays and are asynchronous on  */
/* `stream` (a cudaStream_t, NULL = legacy default stream); the ensemble forms read a     */
/* handle's series rings and return host arrays.                                          */
/* ------------------------------------------------------------------------------------ */

#define CH_MOMENTS 6      /* doubles per row of a moments table */
#define CH_MAX_BINS 1024  /* largest histogram bin count */

/*
 * Moments across the runs per sample time, Eqs. (41a,b).  beta[j * ld + s] is run j's
 * beta at sample s (members runs, samples times, ld >= samples), t[s] the sample times
 * (device arrays).  Row s of out (device, samples x CH_MOMENTS) = t_s, the count c_s of
 * finite values, mu_1 = (1/c_s) sum beta, and mu_p = (1/c_s) sum (beta - mu_1)^p for
 * p = 2, 3, 4 (NaN when c_s = 0), all in FP64.  Errors: CH_EINVAL (members < 1,
 * samples < 0, ld < samples, a NULL array with samples > 0), CH_ECUDA.
 */
int ch_stats_moments(const double* t, const double* beta, int64_t members, int64_t samples, int64_t ld,
                     double* out, void* stream);

/*
 * Histogram per sample time: the empirical distribution p_beta(b, t) of Sec. 1 Eq. (7).
 * Row s of out (device, samples x (nbins + 2) counts) = the values below lo, then nbins
 * bins of width w = (hi - lo) / nbins (value b >= lo goes to bin floor((b - lo) / w),
 * both operations in FP64 with round-to-nearest division), then the values past the
 * last bin.  beta as in ch_stats_moments.  Errors: CH_EINVAL (as ch_stats_moments;
 * lo < hi finite, 1 <= nbins <= CH_MAX_BINS), CH_ECUDA.
 */
int ch_stats_histogram(const double* beta, int64_t members, int64_t samples, int64_t ld, double lo, double hi,
                       int nbins, int64_t* out, void* stream);

/*
 * Trend statistics of a moments table (device, samples rows, t increasing):
 *   out[0]  the window estimate of beta_0, Eq. (42): the integral of mu_1 by the trapezoid
 *           rule between consecutive samples with t1 <= t <= t2, divided by the time
 *           between the first and the last of them (NaN with fewer than two);
 *   out[1]  k of the least-squares line mu_2 = k t through the origin (Sec. 3.3, Sec. 4.2
 *           Table 4) over the samples with tf1 <= t <= tf2: sum t mu_2 / sum t^2 (NaN
 *           when no sample has t != 0);
 *   out[2], out[3]  the numbers of samples in the two windows.
 * out: device, 4 doubles.  Errors: CH_EINVAL (samples < 0, NULL arrays), CH_ECUDA.
 */
int ch_stats_trend(const double* moments, int64_t samples, double t1, double t2, double tf1, double tf2,
                   double* out, void* stream);

/*
 * The same three statistics over a handle's series (ch_set_sampling with capacity > 0)
 * for the runs members[0 .. count) (host array of member indices; NULL = every member,
 * count ignored), on the samples that all of them still hold, oldest first.  The runs
 * must share dt and the sampling period and hold their samples at equal times (checked
 * on the device); else CH_EINVAL.  out is host memory: cap rows of CH_MOMENTS doubles or
 * of nbins + 2 counts (*n receives the rows written), or 4 doubles for the trend.
 * Synchronise the stream.  Errors: CH_EINVAL, CH_ENOMEM, CH_ECUDA.
 */
int ch_ensemble_moments(ch_handle h, const int* members, int count, double* out, int64_t cap, int64_t* n);
int ch_ensemble_histogram(ch_handle h, const int* members, int count, double lo, double hi, int nbins,
                          int64_t* out, int64_t cap, int64_t* n);
int ch_ensemble_trend(ch_handle h, const int* members, int count, double t1, double t2, double tf1, double tf2,
                      double* out);

/*
 * Grid-refinement error of Appendix A: E = (1/|Omega|) sum over the coarse points of
 * |restricted fine - coarse| dx_c dy_c, the fine field restricted by the mean of each
 * 2 x 2 block: fine points (2i, 2j), (2i+1, 2j), (2i, 2j+1), (2i+1, 2j+1) against coarse
 * point (i, j), which is their centre when both grids sample cell centres.  fine is an
 * nx x ny FP64 device array (row-major, x fastest; nx, ny even), coarse nx/2 x ny/2.
 * out (device, 1 + ny/2 doubles) receives E, then the mean over each coarse row.
 * Asynchronous on `stream`.  Errors: CH_EINVAL (odd or < 2 sizes, NULL arrays), CH_ECUDA.
 */
int ch_refinement_error(const double* fine, const double* coarse, int nx, int ny, double* out, void* stream);

/*
 * The same between member fine_member of handle `fine` and member coarse_member of handle
 * `coarse` (both FP64; the coarse member has half the points per axis).  Waits for the
 * coarse handle's stream, runs on the fine handle's stream and writes E to *out (host).
 * Errors: CH_EINVAL (handles, members, precision or sizes), CH_ENOMEM, CH_ECUDA.
 */
int ch_ensemble_refinement_error(ch_handle fine, int fine_member, ch_handle coarse, int coarse_member,
                                 double* out);

/* ------------------------------------------------------------------------------------ */
/* Model 1: ensembles of mean-field droplet populations (Secs. 2-3).                      */
/* ------------------------------------------------------------------------------------ */

/*
 * Integrate M populations of N droplets each from t = 0 to t_end on the device:
 *   dR_i/dt = H(R_i + eps) (-1/R_i^2 + u/R_i),  u = sum H(R_i) / sum H(R_i) R_i
 * (Sec. 2.1 Eqs. (13)-(14), regularised as in Sec. 3.1 Eq. (39); H(s) = 1 for s > 0, else
 * 0), each population with its own Dormand-Prince 5(4) step size.  A step of size h is
 * accepted when sqrt((1/N) sum_i (e_i / (atol + rtol max(|R_i|, |Rnew_i|)))^2) <= 1 (e the
 * fifth- minus fourth-order solution); the next size is h min(5, max(0.2, 0.9 err^(-1/5)))
 * (at most h after a rejection); the first try is h0.  rtol <= 0: fixed steps of h0.
 * Steps are shortened to land on every sample time, where (t, F, dF/dt, beta, live
 * droplets) is recorded, F = 1/2 sum H(R_i) R_i^2, dF/dt = -sum H(R_i)/R_i (1 - u R_i)^2,
 * beta = -(t/F) dF/dt (Sec. 2.4 Eqs. (31), (33), (36)).
 *   R          host, M x N (population-major): radii at t = 0 in, at t_end out
 *   t_samples  host, nsamples increasing times (those above t_end are never reached)
 *   series     host, M x nsamples x 5 doubles, or NULL; unreached samples are NaN
 *   steps      host, M x 3 (accepted, rejected, status 0 ok / 1 step limit / 2 step
 *              underflow), or NULL
 * All buffers are the caller's; the call allocates device scratch (10 M N doubles, 2 M N
 * ints) and
 * synchronises `stream` (a cudaStream_t, NULL = legacy default stream).
 * Errors: CH_EINVAL (arguments; a population reached max_steps steps or its step size
 * underflowed, with R and steps still written), CH_ENOMEM, CH_ECUDA.
 */
int ch_droplets_run(int M, int N, double* R, double t_end, int nsamples, const double* t_samples, double rtol,
                    double atol, double h0, double eps, int64_t max_steps, double* series, int64_t* steps,
                    void* stream);

/* ------------------------------------------------------------------------------------ */
/* Serving: a stream of single-run requests with continuous batching.                    */
/*                                                                                        */
/* The paper (Sec. 4.1) ran its ensembles as M separate processes sharing the GPUs        */
/* through CUDA MPS.  A server instead keeps every admitted run on the device and steps   */
/* all of them together (the kernels of ch_create_batch): requests that arrive while      */
/* others run are admitted as soon as a member slot and room for their fields in the HBM  */
/* budget free up (FIFO), and each run retires the step its horizon ends.  A run's result */
/* depends only on its own request (same result alone and in any mix).  A worker thread  */
/* inside the library drives the GPU; the calls below never block on GPU work except     */
/* ch_server_wait.                                                                        */
/* ------------------------------------------------------------------------------------ */
typedef struct ch_server_s* ch_server;

typedef struct {
  int nx, ny;          /* grid, each >= 5 */
  double L, gamma, dt; /* > 0 */
  double C0;           /* mean of the initial field (C0 + 0.1(2u-1), SplitMix64 stream `seed`) */
  uint64_t seed;
  int64_t nsteps;      /* horizon, >= 1 */
  int every;           /* sampling period for the beta average (0: 100) */
  double t1;           /* beta window start (< 0: 0.2 * nsteps * dt) */
  double* field_out;   /* optional host buffer, ny*nx doubles, for the final field; caller-
                          owned, must stay valid until the request is polled */
} ch_request;

typedef struct {
  int64_t steps;       /* steps run (= nsteps) */
  double F, dFdt, beta;/* observables of the final field (Eqs. (4), (6)) at t = nsteps dt */
  double beta_avg;     /* time average of the sampled beta over t >= t1 (Eq. (42)) */
  int64_t beta_count;
  int nonfinite;       /* the run diverged */
  double t_queued_s;   /* submit -> admitted */
  double t_run_s;      /* admitted -> result ready */
  double t_total_s;    /* submit -> result ready (time-to-result) */
} ch_result;

typedef struct {
  int64_t submitted, completed, running, queued, max_running;
  int64_t member_steps, grid_point_steps, chunks;
  double busy_s, wall_s;           /* worker time with runs present; time since creation */
  size_t arena_bytes, arena_peak_bytes;
} ch_server_stats_t;

/*
 * Create a server of one precision whose runs' fields fit in hbm_budget_bytes of device
 * memory (two arenas: fields and row-solve scratch, allocated now) with at most
 * max_members runs in flight.  Errors: CH_EINVAL, CH_ENOMEM, CH_ECUDA.
 */
int ch_server_create(size_t hbm_budget_bytes, int precision, int max_members, ch_server* out);
/* Queue a request (non-blocking); *id identifies it.  Errors: CH_EINVAL (bad request),
 * CH_ENOMEM (larger than the whole budget), CH_EBUSY (queue full), or the server's error. */
int ch_submit(ch_server s, const ch_request* r, uint64_t* id);
/* CH_PENDING while queued or running; CH_OK with *out filled once finished (the request is
 * then forgotten); CH_ENONFINITE if the run diverged; CH_ENOTFOUND for unknown ids. */
int ch_poll(ch_server s, uint64_t id, ch_result* out);
/* ch_poll after waiting up to timeout_s seconds for the result; CH_ETIMEOUT if not ready. */
int ch_server_wait(ch_server s, uint64_t id, double timeout_s, ch_result* out);
int ch_server_stats(ch_server s, ch_server_stats_t* out);
/* Stop the worker (runs in flight are abandoned) and release everything. */
void ch_server_destroy(ch_server s);

/*
 * Measured fused multiply-add throughput (a measurement aid; the paper has no
 * counterpart).  Enqueues on `stream` one kernel of `blocks` CTAs x `threads` threads
 * (a multiple of 32, at most 1024) in which every thread runs 8 independent chains of
 * 16 x iters FMAs in FP64 (precision CH_FP64) or FP32 (CH_FP32), with no memory traffic,
 * and sets *flops (host) to the floating-point operations it performs (2 per FMA).  The
 * caller times it (e.g. with CUDA events on `stream`) to get the pipe's peak rate.  `sink`
 * is a device double the kernel never writes in practice (it keeps the work live).
 * Errors: CH_EINVAL (shape, iters < 1, NULL pointer, precision), CH_ECUDA (launch).
 */
int ch_fma_peak(int precision, int blocks, int threads, int64_t iters, double* sink, void* stream, double* flops);

/*
 * Host-side fault injection, for testing callers' error handling (the paper has no
 * counterpart).  Arms one fault, process-wide, that fires once:
 *   "alloc[:N]"     the N-th device allocation of the library from now (default the next)
 *                   reports failure without allocating: the call that made it returns
 *                   CH_ENOMEM, releases what it had allocated and leaves no handle;
 *   "nan[:M]"       the next ch_step first writes a NaN into the first grid point of
 *                   member M (default 0) of its handle with a host-to-device copy; the
 *                   member's next sample (and ch_observables) reports CH_ENONFINITE;
 *   "timeout[:MS]"  the next chunk of a server's worker thread starts MS milliseconds
 *                   late (default 2000): ch_server_wait with a shorter timeout returns
 *                   CH_ETIMEOUT, a later wait the result;
 *   "none", "" or NULL disarms.
 * The environment variable CH_FAULT, read at the library's first allocation or first
 * ch_set_fault, arms the same specs.  No fault touches device code: nothing faults, traps
 * or hangs a GPU.  Errors: CH_EINVAL (malformed spec).
 */
int ch_set_fault(const char* spec);

/* Message of the last failure on this host thread ("" if none). */
const char* ch_last_error(void);

/* Library build id, e.g. "ch 0.1 sm_103a". */
const char* ch_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CH_H_ */
