/*
 * libttice -- incremental tensor-train decomposition (TT-ICE / TT-ICE*) on one GB300 GPU.
 *
 * The operation is the increment update of Algorithm 1 (TT-ICE) and Algorithm 2 (TT-ICE*) of
 * "An Incremental Tensor Train Decomposition Algorithm" (arXiv 2211.12487): a batch of b new
 * observations, each a d-way tensor of shape n_1 x ... x n_d, is projected onto the left-orthonormal
 * cores U_1..U_d of the accumulation; every core whose residual exceeds its share of the error
 * tolerance is expanded with just enough orthonormal residual directions (Eqs. 9-11), and the
 * coefficients of the batch are appended to the growing last core (Eq. 13).
 *
 * Conventions shared by every entry point
 *  - Memory: pointers documented "device" are CUDA device pointers; "host" pointers are ordinary
 *    host memory.  The caller owns every buffer it passes; the library owns the cores.
 *  - Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls on
 *    one handle must be issued from one host thread at a time; work is ordered on the given stream.
 *  - Layout of an increment: b observations, observation-major, each observation in C order
 *    (n_d fastest), i.e. a contiguous array of shape (b, n_1, ..., n_d).
 *  - Core layout (Eq. 3): U_i is the (r_{i-1} n_i) x r_i unfolding of core G_i with row index
 *    a*n_i + k for G_i[a, k, :] (rank index slower than the mode index).
 *  - Errors: every function returns 0 (TTICE_OK) or a negative TTICE_E* code; ttice_strerror()
 *    names it.  Nothing traps on the device: device-detected failures set a sticky status that the
 *    next synchronising call returns.  A failing ttice_update leaves the decomposition exactly as it
 *    was before the call (cores, ranks and last core are rolled back).
 */
#ifndef TTICE_H
#define TTICE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TTICE_OK 0
#define TTICE_EINVAL (-1)     /* bad argument (null pointer, size, mode) */
#define TTICE_ENOMEM (-2)     /* device allocation failed */
#define TTICE_ECAPACITY (-3)  /* a rank would exceed its capacity (see ttice_reserve_rank) */
#define TTICE_ENONFINITE (-4) /* the increment holds NaN or Inf */
#define TTICE_ETIMEOUT (-5)   /* an iterative device solve hit its iteration limit */
#define TTICE_ECUDA (-6)      /* a CUDA runtime call failed */
#define TTICE_EINTERNAL (-7)

/* Skip test before any core update (Sec. 4.3, last heuristic). */
#define TTICE_SKIP_NONE 0  /* never skip: plain TT-ICE behaviour */
#define TTICE_SKIP_EXACT 1 /* skip iff the batch relative error (Eq. 20) <= eps (default) */
#define TTICE_SKIP_MEAN 2  /* the paper's surrogate: skip iff mean_j eps_Y(j) <= eps */

/* Relaxed tolerance for the selected observations (Sec. 4.3, subselection). */
#define TTICE_EPSUPD_EXACT 0  /* Eq. 18 (default) */
#define TTICE_EPSUPD_APPROX 1 /* Eq. 19, count-weighted */

/* Arithmetic of the path.  In every mode the cores are stored in FP64 and the rank decision (the
 * Ritz values it reads), the re-orthogonalisation of new directions (CGS2, Cholesky-QR) and all
 * norms and thresholds are FP64. */
#define TTICE_FP64 0 /* FP64 everywhere: the plain FP64 GPU TT-ICE */
#define TTICE_FP32 1 /* FP32 projections and residuals, Gram as FP32 products summed in FP64, FP32
                        eigen-solve candidates + FP64 Rayleigh-Ritz.  The projections of the chain
                        (every stage whose unfolding has >= 32 columns per observation, a multiple of
                        4) run on the tensor cores in TF32 with each operand split into a TF32 head
                        and tail (three products, FP32 accuracy), their residual norms by Pythagoras;
                        large re-orthogonalisations (CGS work m r k >= 4e9) run their two CGS passes
                        on the tensor cores the same way, and their Cholesky-QR too once m k^2 >=
                        5e8 (column norms in FP64).  The coupling they leave is the tensor core's
                        FP32 summation error, ~2^-23 of the products' magnitudes per 8-term MMA:
                        ~1e-9 for delocalised columns at m ~ 5e4, up to ~1e-7 for short or
                        localised ones (FP64: ~1e-15). */
#define TTICE_TF32 2 /* as TTICE_FP32, but the projections of the large stages of the chain (Eq. 6,
                        Eq. 12: r_{i-1} n_i >= 256 rows and >= 65536 entries per observation) and
                        their new rows take one TF32 product (heads only, FP32 accumulation) instead
                        of three; small stages, the first pass's kernel for n_1 <= 128, the
                        residuals of updated cores, the Grams, the re-orthogonalisation and the
                        eigen-solve keep the TTICE_FP32 arithmetic.  Error budget: 1/16 of each
                        increment's eps^2 ||Y||^2 is reserved for the TF32 rounding (2^-11 relative
                        per operand): every decision of Algorithm 2 (skip test, subselection,
                        eps_upd, per-core thresholds) runs at eps sqrt(15/16), so the reported
                        errors and the coefficients may be off by that share before Theorem 1's
                        bound eps ||Y|| is at risk.  The share holds where the rounding averages
                        out (measured: 5.5e-5 ||y||^2 per observation on a 480p video stream) but not
                        on every input (6.6e-4 ||y||^2 on a 64^3 x 4 flow stream with localised core
                        columns: within the share from eps = 0.1); TTICE_FP32 has no such limit. */
#define TTICE_BF16 3 /* reserved (tensor-core projections): ttice_create returns TTICE_EINVAL */
#define TTICE_SPLIT_BF16 4 /* reserved (split-BF16 projections): ttice_create returns TTICE_EINVAL */

/* Element type of increments passed to ttice_update / ttice_project, and of reconstructions. */
#define TTICE_F32 0
#define TTICE_F64 1

typedef struct ttice_s* ttice_t;

typedef struct {
  int skip_mode;        /* TTICE_SKIP_*, default TTICE_SKIP_EXACT */
  int subselect;        /* 0/1: update only with observations whose eps_Y(j) > eps (Eq. 17), default 1 */
  int eps_upd_mode;     /* TTICE_EPSUPD_*, default TTICE_EPSUPD_EXACT */
  double occupancy_tau; /* core i is left alone iff r_i/(r_{i-1} n_i) >= tau (Eq. 16), default 1.0 */
  int precision;        /* TTICE_FP64 .. TTICE_SPLIT_BF16, default TTICE_FP64 */
  int input_dtype;      /* TTICE_F32 or TTICE_F64 */
} ttice_heuristics;

typedef struct {
  int64_t max_batch;   /* largest b passed to update/project (default 32) */
  int64_t max_rank;    /* capacity of every TT-rank r_1..r_d (default 512; also capped at the
                          product of the leading mode sizes) */
  int64_t obs_reserve; /* initial capacity of the last core in observations (grows by doubling) */
} ttice_capacity;

typedef struct {
  int32_t skipped;        /* 1 if the core update was skipped (error already <= eps) */
  int32_t n_selected;     /* |D|, observations used to update the cores (Eq. 17) */
  double rel_err_before;  /* batch relative error against the cores before the update (Eq. 20) */
  double eps_upd;         /* Eq. 18/19 (NaN when skipped) */
  double eps_core;        /* per-core truncation threshold eps_upd ||D|| / sqrt(d) */
  int64_t ranks[18];      /* r_0 .. r_d after the update (d <= 16), r_{d+1} = 1 */
  int32_t new_dirs[16];   /* directions appended to each core U_1..U_d */
  int64_t n_obs;          /* observations stored in the last core */
  int64_t core_elems;     /* sum_i r_{i-1} n_i r_i over U_1..U_d plus r_d * n_obs (Eq. 22 denominator) */
  int32_t eig_sweep_limit; /* eigen-solves of this update that stopped at their sweep limit */
  int32_t eig_sweeps;      /* block-Jacobi sweeps spent by the eigen-solves of this update */
  int32_t krylov_solves;   /* eigen-solves of this update done by the certified block-Krylov path */
  int32_t krylov_fallbacks; /* ... that fell back to the full Jacobi solve */
} ttice_update_stats;

/* Fill defaults. */
void ttice_default_heuristics(ttice_heuristics* h);
void ttice_default_capacity(ttice_capacity* c);

/* Create an empty decomposition (all ranks 0, Sec. 5 init read as TT-ICE from empty cores, which
 * equals TT-SVD of the first increment).  dims: host array of d mode sizes (1 <= d <= 16);
 * eps: relative error bound eps_des in (0, 1) (Problem 1, Corollary 1).  h and cap may be NULL for
 * defaults.  Allocates every core at capacity on the current CUDA device. */
int ttice_create(const int64_t* dims, int d, double eps, const ttice_heuristics* h,
                 const ttice_capacity* cap, ttice_t* out);

/* One TT-ICE* increment (Algorithm 2; with skip_mode NONE, subselect 0 and tau > 1 exactly
 * Algorithm 1).  Y: device, `batch` observations of input_dtype, layout above; must stay valid
 * until the call returns (the call synchronises `stream` at its decision points).  On success the
 * batch is appended to the last core as observations n_obs .. n_obs+batch-1. */
int ttice_update(ttice_t h, const void* Y, int64_t batch, void* stream);

/* Sequential projection of `batch` observations onto U_1..U_d without changing the state
 * (Algorithm 2 "project"; the relative prediction error of Sec. 5.1).  Y: device, input_dtype.
 * coeffs: device, batch x r_d FP64, row j = coefficients of observation j (may be NULL).
 * rel_err: device, batch FP64 relative errors eps_Y(j) of Eq. 17 (may be NULL).  Asynchronous. */
int ttice_project(ttice_t h, const void* Y, int64_t batch, double* coeffs, double* rel_err,
                  void* stream);

/* Current TT-ranks r_0 .. r_d, r_{d+1}=1 into ranks (host, d+2 entries). */
int ttice_ranks(ttice_t h, int64_t* ranks);

/* Reconstruct stored observations first .. first+count-1 (Eq. 14): out is a device array of
 * count observations in the increment layout, element type out_dtype (TTICE_F32/F64), at least
 * count * n_1 ... n_d elements.  Any count works (ranges above 65535 observations run in chunks).
 * Its two intermediate buffers come from cudaMallocAsync on `stream`.  Asynchronous. */
int ttice_reconstruct(ttice_t h, int64_t first, int64_t count, void* out, int out_dtype,
                      void* stream);

/* Shape and placement of h: *d = number of modes, dims[0..d) = n_1..n_d (room for 16), *device =
 * the CUDA device its buffers live on (the current device at ttice_create / ttice_open).  Any
 * argument may be NULL.  Host only. */
int ttice_info(ttice_t h, int* d, int64_t* dims, int* device);

/* Statistics of the last update. */
int ttice_stats(ttice_t h, ttice_update_stats* st);

/* Copy core U_i (1 <= i <= d) to host as a row-major (r_{i-1} n_i) x r_i FP64 matrix; rows/cols
 * receive its shape.  host may be NULL to query the shape.  Synchronous. */
int ttice_get_core(ttice_t h, int i, double* host, int64_t* rows, int64_t* cols);

/* Copy the last core (Eq. 13) to host as a row-major n_obs x r_d FP64 matrix (row j = coefficients
 * of observation j, zero-extended).  host may be NULL to query the shape.  Synchronous. */
int ttice_get_last_core(ttice_t h, double* host, int64_t* n_obs, int64_t* rd);

/* Replace the whole state with host data: ranks r_0..r_d (d+1 entries, r_0 = 1), cores[i] a
 * row-major (r_i n_{i+1}) x r_{i+1} FP64 matrix for i = 0..d-1, last: n_obs x r_d row-major.
 * Used to resume from stored cores (the cores are the compressed format) and by lockstep tests. */
int ttice_load(ttice_t h, const int64_t* ranks, const double* const* cores, const double* last,
               int64_t n_obs);

/* Capacity.  The method itself bounds no rank: each update appends as many directions as the
 * residual needs (Eq. 9, Eq. 10), so a rank can outgrow the capacity chosen at ttice_create.  An
 * update that would do so returns TTICE_ECAPACITY and leaves the decomposition as it was;
 * ttice_capacity_miss names the rank and the size it needed, ttice_reserve_rank raises that rank's
 * capacity, and the update can then be repeated.  (The library's own solver limit, a Gram side
 * above 4608, also returns TTICE_ECAPACITY, with *k = 0.) */

/* Rank capacities cap_0 .. cap_d (host, d+1 entries, cap_0 = 1). */
int ttice_capacities(ttice_t h, int64_t* caps);

/* Device memory held by h in bytes (cores at capacity, work buffers, last core). */
int ttice_device_bytes(ttice_t h, int64_t* bytes);

/* Device bytes that ttice_create(dims, d, *, h, cap) would allocate, with the rank capacities
 * caps[1..d] (host, d+1 entries; NULL: the default rule cap_i = min(max_rank, cap_{i-1} n_{i-1})),
 * computed by the creation code itself without allocating anything and without a GPU.  What
 * admission by projected memory needs; equal to ttice_device_bytes of the created handle. */
int ttice_projected_bytes(const int64_t* dims, int d, const ttice_heuristics* h, const ttice_capacity* cap,
                          const int64_t* caps, int64_t* bytes);

/* After an update that returned TTICE_ECAPACITY: *k = the rank index (1 <= k <= d) whose capacity
 * it needed to exceed and *need = the rank r_k it needed; *k = 0 otherwise (also after a successful
 * update). */
int ttice_capacity_miss(ttice_t h, int* k, int64_t* need);

/* Raise the capacity of rank r_k (1 <= k <= d) to at least cap (clipped to cap_{k-1} n_k, the
 * largest rank the unfolding allows).  Re-allocates the cores and work buffers that the capacity
 * sizes on the current device and moves the decomposition into them, device to device; ranks, cores,
 * last core and statistics are unchanged.  No work of h may be in flight (a failed ttice_update has
 * already finished its work when it returns); work of other handles is neither waited for nor
 * ordered against.  A capacity already at least cap is a no-op.  On TTICE_ENOMEM the handle is
 * left unchanged. */
int ttice_reserve_rank(ttice_t h, int k, int64_t cap);

/* Checkpoint / resume.  The cores are the compressed form of the accumulation (Sec. 5.3): a
 * checkpoint file holds the decomposition and what is needed to continue it, nothing else.  Layout,
 * all values little-endian, no padding:
 *   char[8] "TTICECK1" | int32 version = 1 | int32 d | int64 n_1..n_d | float64 eps |
 *   int32 skip_mode | int32 subselect | int32 eps_upd_mode | float64 occupancy_tau |
 *   int32 precision | int32 input_dtype | int64 r_0..r_d | int64 n_obs |
 *   U_1..U_d, each row-major (r_{i-1} n_i) x r_i float64 | last core, row-major n_obs x r_d float64 |
 *   uint64 FNV-1a (64-bit) of every preceding byte.
 * Readers reject a wrong magic or version, shapes that violate r_0 = 1 and r_i <= r_{i-1} n_i, a
 * checksum mismatch, a short file and trailing bytes, with TTICE_EINVAL. */

/* Write a checkpoint from host data (cores and last core as in ttice_load).  Host only. */
int ttice_checkpoint_write(const char* path, int d, const int64_t* dims, double eps,
                           const ttice_heuristics* heur, const int64_t* ranks,
                           const double* const* cores, const double* last, int64_t n_obs);

/* Read a checkpoint into host memory.  With cores == NULL only the header is read (d, dims[<=16],
 * eps, heur, ranks[d+1], n_obs), to size the buffers; then call again with cores[i] holding
 * (r_i n_{i+1}) x r_{i+1} doubles and last n_obs x r_d doubles.  Host only. */
int ttice_checkpoint_read(const char* path, int* d, int64_t* dims, double* eps, ttice_heuristics* heur,
                          int64_t* ranks, int64_t* n_obs, double* const* cores, double* last);

/* Save the state of h (synchronous; no work of h may be in flight). */
int ttice_save(ttice_t h, const char* path);

/* Create a handle on the current device from a checkpoint: its mode sizes, eps and heuristics, and
 * its decomposition; `cap` (NULL: defaults) sets the batch size and the capacities, each rank's
 * capacity being raised to at least its saved rank.  Updates then continue the stream. */
int ttice_open(const char* path, const ttice_capacity* cap, ttice_t* out);

/* Device-time profile of ttice_update, by phase of Algorithm 2.  Times come from CUDA events
 * recorded on the update's stream around each phase; bytes and flops are the algorithmic amounts
 * (what the method must read, write and compute for the sizes involved, not what the kernels
 * happen to move).  Phases:
 *   0 first pass over the increment, stage 1 (U_1^T Y_1, residual norms, ||y||^2; Eq. 6, Eq. 17)
 *   1 first pass, stages 2..d (Eq. 12 chain with residual norms)
 *   2 residual of the selected observations against a core (Algorithm 2, R_i)
 *   3 residual Gram matrix (Eq. 9 via R R^T or R^T R)
 *   4 truncated eigen-solve, refinement and rank rule (Eq. 5 / Eq. 9)
 *   5 CGS2, normalisation, sign and append (Eq. 10)
 *   6 projection of the selected observations onto the updated core (D_{i+1}, Eq. 12)
 *   7 final projection of the whole batch onto the updated cores and append (Eq. 13) */
#define TTICE_NPHASES 8
typedef struct {
  double ms[TTICE_NPHASES];
  double bytes[TTICE_NPHASES];
  double flops[TTICE_NPHASES];
  int64_t count[TTICE_NPHASES];
  int64_t updates;
} ttice_profile;

/* Enable (1) or disable (0) phase profiling of h; enabling also clears the accumulated profile. */
int ttice_profile_enable(ttice_t h, int on);
/* Accumulated profile since the last enable.  Host struct. */
int ttice_profile_read(ttice_t h, ttice_profile* out);
/* Kernel launches issued by this library in this process so far. */
int64_t ttice_kernel_launches(void);

/* Allocation-free variant of ttice_reconstruct (the paper has no counterpart: this is a service of
 * the library).  For callers that cannot allocate device memory when they reconstruct -- code being
 * captured into a CUDA graph that must hold no allocation nodes, real-time loops that cannot wait on
 * the allocator, or processes whose device memory is reserved in advance -- it computes the same
 * reconstruction as ttice_reconstruct (same arguments, same output) without calling cudaMalloc,
 * cudaFree or any allocating routine.  Its intermediates live in one fixed array of device memory
 * inside the library: two buffers of TTICE_NOALLOC_MAX_ELEMS doubles (64 MiB in all), which every
 * GPU that loads the library holds until the process exits.
 *  - Limit: count * (n_1 ... n_d) must not exceed TTICE_NOALLOC_MAX_ELEMS (and count <= 65535);
 *    larger requests return TTICE_EINVAL without doing any work.
 *  - The first call on a device looks up the array's device address with that device current (the
 *    caller's current device); make that first call before any stream capture.  The address is kept
 *    for the life of the process: after cudaDeviceReset on that device (which also ends every
 *    handle there) the entry point must not be called again in this process.
 *  - All calls share the array.  Calls whose work overlaps on the GPU (different streams, or
 *    different handles, at the same time) race on it: serialise them.
 *  - Asynchronous on `stream`, like ttice_reconstruct. */
#define TTICE_NOALLOC_MAX_ELEMS (4LL * 1024 * 1024)
int ttice_reconstruct_noalloc(ttice_t h, int64_t first, int64_t count, void* out, int out_dtype,
                              void* stream);

/* Free h.  Synchronises the device first (cudaFree would as well), so no work of h may be left
 * running; work of other handles is waited for too. */
void ttice_destroy(ttice_t h);
const char* ttice_strerror(int code);
/* Name of the CUDA runtime error behind the last TTICE_ECUDA or TTICE_ENOMEM that a call returned
 * to the calling thread ("cudaSuccess" if none). */
const char* ttice_last_cuda_error(void);

/* Test hook for the out-of-memory paths (failures are injected on the host, never provoked on the
 * device): the n-th device allocation of the library from now on (process-wide) fails with
 * TTICE_ENOMEM as if the device were full, and ttice_last_cuda_error names
 * cudaErrorMemoryAllocation.  n <= 0 disarms it. */
void ttice_test_fail_alloc(int64_t n);

/* Test hooks of the tensor-core kernels (host-side settings; nothing here faults a GPU):
 *  - ttice_test_wait_limit_ns: the time limit of every bounded wait inside the tensor-core kernels
 *    (0 restores the default of 2 s).  A wait that runs out makes the kernel leave cleanly and the
 *    update return TTICE_ETIMEOUT with the decomposition as it was.
 *  - ttice_test_drop_copy: the next tensor-core projection launch issues no copy for chunk `chunk`
 *    of its first thread block, so that the consumers' bounded wait runs out (-1 disarms).
 *  - ttice_test_tc_cgs_min: the CGS work m r k from which the mixed path runs the re-orthogonalisation
 *    of new directions (CGS2, and CholQR2 from the smaller of this and m k^2 = 5e8) on the tensor
 *    cores, and the transposed projection of stages with few columns per observation from the smaller
 *    of this and m r b L = 2e8 (0: whenever the shapes allow; negative: the defaults). */
void ttice_test_wait_limit_ns(uint64_t ns);
void ttice_test_drop_copy(int64_t chunk);
void ttice_test_tc_cgs_min(double flops);

#ifdef __cplusplus
}
#endif
#endif /* TTICE_H */
