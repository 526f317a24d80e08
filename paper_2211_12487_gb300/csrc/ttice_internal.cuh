// Internal declarations of libttice: device views, kernel launchers and the handle layout.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "ttice.h"

#include <atomic>

namespace ttice {

constexpr int kMaxD = 16;

// Element counts of a decomposition's arrays: core i holds r_i n_{i+1} r_{i+1} elements (0-based,
// i = 0..d-1) and the last core n_obs r_d.  Every product and the running total are checked for
// int64 overflow, and the total must stay below INT64_MAX / 8 so that its byte count fits too.
// Returns false on overflow or a negative size; core_elems (d entries), last_elems and total may be
// null.
inline bool checked_shape_elems(int d, const int64_t* dims, const int64_t* ranks, int64_t n_obs,
                                int64_t* core_elems, int64_t* last_elems, int64_t* total) {
  int64_t t = 0;
  for (int i = 0; i < d; ++i) {
    int64_t a = 0, e = 0;
    if (dims[i] < 0 || ranks[i] < 0 || ranks[i + 1] < 0) return false;
    if (__builtin_mul_overflow(ranks[i], dims[i], &a) || __builtin_mul_overflow(a, ranks[i + 1], &e) ||
        __builtin_add_overflow(t, e, &t))
      return false;
    if (core_elems) core_elems[i] = e;
  }
  int64_t l = 0;
  if (n_obs < 0 || __builtin_mul_overflow(n_obs, ranks[d], &l) || __builtin_add_overflow(t, l, &t))
    return false;
  if (t > INT64_MAX / 8) return false;
  if (last_elems) *last_elems = l;
  if (total) *total = t;
  return true;
}

// Count of kernel launches issued by this library (process-wide), for launch accounting.
extern std::atomic<long long> g_kernel_launches;
inline void note_launch() { g_kernel_launches.fetch_add(1, std::memory_order_relaxed); }

// A strided matrix view with a two-level batch index: batch z -> (z1, z2) = (z / bdiv, z % bdiv),
// element (row, col) of batch z at p + z1*bs1 + z2*bs2 + row*rs + col*cs (element units).
struct View {
  const void* p = nullptr;
  int64_t rs = 0, cs = 0, bs1 = 0, bs2 = 0;
};

// C(z) = alpha * A(z) * B(z) + beta * X(z), M x N, inner dimension K.
struct GemmArgs {
  int64_t M = 0, N = 0, K = 0;
  View A, B, X;
  void* C = nullptr;
  int64_t c_rs = 0, c_cs = 0, c_bs1 = 0, c_bs2 = 0;
  double alpha = 1.0, beta = 0.0;
  int nbatch = 1, bdiv = 1;
  int atomic = 0;         // add into C with atomics (C zeroed by the caller); allows split-K
  int store = 1;          // write C at all
  double* norm = nullptr; // optional: += sum of squares of the C(z) entries into norm[z1]
  int norm_rows = 0;      // with norm: accumulate per output row instead (norm[row])
  int allow_splitk = 0;   // with atomic: split K across CTAs when the tile grid is small
  int64_t c_zero_elems = 0;  // without atomic: C spans this many elements from C; if the tile grid
                             // is small, zero them and split K with atomic adds instead of stores
  int sym = 0;  // C is a symmetric Gram (c_cs = 1, leading dimension c_rs): only its upper triangle
                // is formed and mirrored.  1: one M x M matrix (every batch adds into it);
                // 2: batch zb is the block (zb / bdiv, zb % bdiv) of size M x N of a larger one
};

template <typename TA, typename TB, typename TX, typename TC, typename ACC>
cudaError_t gemm(const GemmArgs& g, cudaStream_t st);

// Symmetric eigen-solve by cyclic two-sided Jacobi with round-robin parallel ordering.
// G: FP64 s x s (leading dimension ldg, symmetric).  Works in T.  On return w[0..s) holds the
// eigenvalues in descending order and V (s x s, column-major, ld s) the matching eigenvectors.
// work: device scratch of 2*s*(s+1) T (eigenvector iterate, and the matrix when it does not fit in
// shared memory).
// status (device int): set to 1 if the sweep limit was hit.
template <typename T>
cudaError_t jacobi_eig(const double* G, int64_t ldg, int s, T* w, T* V, T* work, int* status,
                       cudaStream_t st);

// Multi-CTA block Jacobi (see bjacobi.cu): same outputs as jacobi_eig.  work: block_jacobi_work<T>(s)
// elements; fro: device double[3] scratch (the Frobenius and off-diagonal norms the stopping rule
// reads); flags: device int[5] ([2] = sweeps, [3] = 1 if the sweep limit was hit while rotations
// were still significant, [4] = internal).
template <typename T>
int64_t block_jacobi_work(int s);
template <typename T>
cudaError_t block_jacobi_eig(const double* G, int64_t ldg, int s, T* w, T* V, T* work, double* fro,
                             int* flags, int max_sweeps, cudaStream_t st);

// Device-side decision of Algorithm 2 (skip test, subselection, eps_upd, per-core threshold).
struct Decision {
  int skip;
  int nsel;
  double batch_err;   // Eq. 20
  double ynorm2;      // ||Y||^2
  double dnorm2;      // ||D||^2
  double eps_upd;     // Eq. 18 / 19
  double eps_c;       // eps_upd ||D|| / sqrt(d)
  int nonfinite;
};

// rho2s: squared residuals per TT stage and observation (stage-major, nst x b)
cudaError_t launch_decision(const double* rho2s, int nst, const double* y2, int b, double eps, int d,
                            int skip_mode, int subselect, int eps_upd_mode, Decision* dec,
                            int* sel, cudaStream_t st);

// Rank rule of the delta-truncated SVD (Eq. 5 / Eq. 9) on Ritz values theta[0..K) (descending).
// full: theta holds every eigenvalue of the Gram (tail summed directly from the smallest);
// otherwise tail(r) = trace - sum_{j<r} theta_j.  Writes out[0] = r (or -1 if K too small),
// out[1] = status.  max_new = m - r_i (directions available), cap_new = capacity left.
cudaError_t launch_rank_rule(const double* theta, int K, int full, const double* trace,
                             const double* eps_c, int max_new, int* out, cudaStream_t st);

// K1 (k1.cu): fused first pass of stage 1 -- W = U_1^T Y_1, ||y||^2 and ||Y_1 - U_1 W||^2 per
// observation in one read of the increment.  Supported for n_1 <= 32 and 1 <= r_1 <= 32.
template <typename TY, typename T>
bool k1_supported(int n1, int r);
// part: device scratch of 2 * (4*152 + b) doubles (per-CTA partial sums).
template <typename TY, typename T>
cudaError_t launch_k1(const TY* Y, int b, int64_t L, int n1, int r, const T* U, int64_t ldu, T* W,
                      double* y2, double* rho2, double* part, cudaStream_t st);
cudaError_t launch_k1_reduce(const double* part, int b, int64_t per_obs, double* y2, double* rho2,
                             cudaStream_t st);

// K1 with TMA staging (k1_tma.cu), FP32 increments: same outputs as launch_k1; status (device int)
// becomes nonzero if a tile copy never completed within the bounded wait.
bool k1_tma_supported(const void* Y, int64_t L, int n1, int r);
// part: device scratch of 2 * b * ceil(L / 256) doubles (per-tile partial sums).
template <typename T>
cudaError_t launch_k1_tma(const float* Y, int b, int64_t L, int n1, int r, const T* U, int64_t ldu,
                          T* W, double* y2, double* rho2, double* part, int* status, cudaStream_t st);

// K1 on the tensor cores (k1_tc.cu), FP32 increments and FP32 cores: the same outputs as
// launch_k1_tma (y2 == nullptr: projection only), with the projection as TF32 tcgen05 MMAs on a
// three-product hi/lo split (FP32 accuracy) and the residual norm as ||y||^2 - ||w||^2.  Supported for
// n_1 <= 128 and 1 <= r_1 <= 64.  part: k1_tc_part_elems(b, L) doubles.  status becomes nonzero if a
// wait of the kernel expired.
bool k1_tc_supported(const void* Y, int64_t L, int n1, int r);
int64_t k1_tc_part_elems(int b, int64_t L);
cudaError_t launch_k1_tc(const float* Y, int b, int64_t L, int n1, int r, const float* U, int64_t ldu,
                         float* W, double* y2, double* rho2, double* part, int* status, cudaStream_t st);

// Projection of a batch onto a core on the tensor cores (tc_proj.cu): W(z) = U^T X(z) for b
// observations, X(z) m x L row-major FP32 (16-byte aligned, L % 4 == 0, L >= 32), U given as its
// TF32 head/tail pair Uh, Ul (column-major, ld ldhl % 32 == 0, hlcols columns allocated, zero beyond
// the core), W(z) r x L row-major.  With x2 and/or rho2 (device, b doubles each): x2[z] = ||X(z)||^2,
// rho2[z] = ||X(z)||^2 - ||W(z)||^2 (clamped to [0, x2]).  part: tc_proj_part_elems(b, L, r, m) doubles.
// ws: tc_ws_elems floats of workspace for splitting K (may be null).
// status becomes nonzero if a wait of the kernel expired.
bool tc_proj_supported(const void* X, int64_t L, int64_t m, int r, int64_t ldhl);
int64_t tc_proj_part_elems(int b, int64_t L, int64_t r, int64_t m);
constexpr int64_t tc_ws_elems = 16LL << 20;
cudaError_t launch_tc_proj(const float* X, int b, int64_t L, int64_t m, int r, const float* Uh, const float* Ul,
                           int64_t ldhl, int64_t hlcols, float* W, double* x2, double* rho2, double* part,
                           float* ws, int* status, cudaStream_t st, int nprod = 3);
// General product on the tensor cores (the same kernel): D[n][l] = sum_k B(k, n) A(k, l) for
// n < r (N), l < L (M, per observation), k < K, each operand split into TF32 head and tail (three
// products, FP32 accuracy; the main product summed in registers over 64-long K segments), or with
// nprod = 1 the heads alone (one TF32 product, FP32 accumulation).
//   A, one of: raw FP32 X (x != nullptr): A(k, l) of observation z = x[z x_obs + k ldx + l]
//              (16-byte aligned; ldx, x_obs multiples of 4; b observations), split by converter warps;
//              or pre-split (ah != nullptr): A(k, l) = ah[l lda + k] + al[l lda + k] (lda % 32 == 0,
//              la_alloc rows allocated, zero beyond the operand; b = 1), copied by TMA.
//   B: pre-split, B(k, n) = bh[n ldb + k] + bl[n ldb + k] (ldb % 32 == 0, nb_alloc columns allocated,
//      zero beyond the operand), copied by TMA.
//   Store of D[n][l] of observation z at o = z o_obs + n ldn + l ldl, by `mode`: 0 float out[o] = D
//   (with x2 / rho2 as for launch_tc_proj), 1 double out[o] -= D, 2 float out[o], out2[o] = TF32
//   head and tail of D, 3 double out[o] = D, 4 float out[o] = in[(n / in_lz) in_obs + (n % in_lz)
//   in_ldn + l in_ldl] - D (a residual whose input has its own layout).
struct TcGemm {
  const float* x = nullptr;
  int64_t ldx = 0, x_obs = 0;
  const float* ah = nullptr;
  const float* al = nullptr;
  int64_t lda = 0, la_alloc = 0;
  int64_t L = 0;
  int b = 1;
  int64_t K = 0;
  const float* bh = nullptr;
  const float* bl = nullptr;
  int64_t ldb = 0, nb_alloc = 0;
  int r = 0;
  int mode = 0;
  int nprod = 3;  // 3: split operands (FP32 accuracy); 1: one TF32 product
  void* out = nullptr;
  void* out2 = nullptr;
  int64_t o_obs = 0, ldn = 0, ldl = 1;
  const float* in = nullptr;
  int64_t in_lz = 1, in_obs = 0, in_ldn = 0, in_ldl = 0;
  double* x2 = nullptr;
  double* rho2 = nullptr;
  double* part = nullptr;
  int* status = nullptr;
  // optional workspace (floats) for splitting K when the output alone cannot fill the GPU (mode 0 in
  // the chain layout o_obs = r L, ldn = L, ldl = 1): partial products, then a summing pass
  float* ws = nullptr;
  int64_t ws_elems = 0;
  // optional device flag: the product runs only if *run_if != 0 (decided by earlier kernels on the
  // stream, so the host need not synchronise)
  const int* run_if = nullptr;
};
cudaError_t launch_tc_gemm(const TcGemm& g, cudaStream_t st);
// flag = 1 if some column j < k of P (FP64, column j at P + j ld, r entries) has norm > thr (flag is
// only ever raised: the caller zeroes it)
cudaError_t launch_cols_above(const double* P, int64_t r, int k, int64_t ld, double thr, int* flag,
                              cudaStream_t st);
// Transposing split of b observations of W (r x L, row-major): row z L + l of hi / lo (ld_out >= r)
// holds the TF32 head / tail of W[z][:][l], zero up to the next multiple of 32.
cudaError_t launch_split_tf32_transpose(const float* W, int b, int64_t r, int64_t L, float* hi, float* lo,
                                        int64_t ld_out, cudaStream_t st);
// TF32 head/tail split of FP32 columns [c0, c1) (ld_in rows, zero up to the next multiple of 32
// within ld_out) into hi, lo (ld_out).
cudaError_t launch_split_tf32(const float* in, int64_t ld_in, int64_t c0, int64_t c1, float* hi, float* lo,
                              int64_t ld_out, cudaStream_t st);
// The same from FP64 columns (rows [0, rows), zero up to the next multiple of 32): head = tf32(x),
// tail = tf32(x - head) computed in FP64; f32 (optional, ld_out) receives the FP32 rounding of x and
// sumsq (optional, zeroed by the caller) gains the FP64 sum of squares of each column c at sumsq[c - c0].
cudaError_t launch_split_tf32_f64(const double* in, int64_t ld_in, int64_t rows, int64_t c0, int64_t c1, float* hi,
                                  float* lo, int64_t ld_out, cudaStream_t st, float* f32 = nullptr,
                                  double* sumsq = nullptr);
// W[z][n][l] = P[(z L + l) k + n] (FP64 -> FP32) for b observations, n < k, l < L; w2[z] (optional,
// zeroed by the caller) gains the sum of squares of observation z.
cudaError_t launch_scatter_stage(const double* P, int b, int64_t k, int64_t L, float* W, double* w2,
                                 cudaStream_t st);
// rho2[z] += x2[z] - w2[z], z < b
cudaError_t launch_pythagoras(const double* x2, const double* w2, int b, double* rho2, cudaStream_t st);
// TF32 head / tail of I - Rinv (k x k, column-major), transposed into rows of ld (the B operand of a
// product X (I - Rinv)); zero outside the k x k corner of the ld x ld block.
cudaError_t launch_eye_minus_split(const double* Rinv, int k, float* hi, float* lo, int ld, cudaStream_t st,
                                   const int* run_if = nullptr);
// Near-orthonormal columns (S = V^T V = I + E, ||E||_F <= 1e-4): the same operand for the symmetric
// orthonormalisation V S^{-1/2} = V - V F, F = I - S^{-1/2} = E/2 - 3 E^2/8 + 5 E^3/16 (the next
// term, 35 E^4/128, is below 3e-17), formed in FP32 from E (FP64 S - I, diagonal from diag) in one
// CTA.  Otherwise *fallback is set to 1 and the operand is left alone (for the Cholesky route).
cudaError_t launch_lowdin_split(const double* S, int k, const double* diag, float* hi, float* lo, int ld,
                                int* fallback, cudaStream_t st);
// Bounded-wait limit of the tensor-core kernels (0 restores the default of 2 s), and a test hook:
// the next tc_proj launch issues no copy for chunk `chunk` of its first CTA, so that the consumers'
// bounded wait runs out.
void tc_set_wait_ns(unsigned long long ns);
void tc_drop_next_copy(long long chunk);

// Misc kernels.
cudaError_t launch_fill(double* p, int64_t n, double v, cudaStream_t st);
// n pseudo-random values in [-1, 1) (splitmix64 of seed + index)
cudaError_t launch_fill_random(float* p, int64_t n, uint64_t seed, cudaStream_t st);
template <typename TI, typename TO>
cudaError_t launch_cast(const TI* in, TO* out, int64_t n, cudaStream_t st);
template <typename T>
cudaError_t launch_gather_obs(const T* Y, T* out, const int* sel, int nsel, int64_t N,
                              cudaStream_t st);
// Stage outputs of a core that gained k columns: out[z] (r0 + k rows of L) = src[sel[z]] (r0 rows of
// L; sel == nullptr: src[z]) followed by add[z] (k rows of L), for z < nobs.
template <typename T>
cudaError_t launch_expand_stage(const T* src, const int* sel, int64_t r0, const T* add, int64_t k, int64_t L,
                                int nobs, T* out, cudaStream_t st);
template <typename T>
cudaError_t launch_sum_squares(const T* x, int b, int64_t N, double* out, cudaStream_t st);
// diag sum of an FP64 s x s matrix into *out
cudaError_t launch_trace(const double* G, int64_t ldg, int s, double* out, cudaStream_t st);
// canonical sign of the k columns of V (m x k, ld): sign[c] = -1 if the column's largest-|.| entry
// (lowest index on ties) is negative, else 1.  part: scratch of 128 k doubles.
cudaError_t launch_canonical_sign(const double* V, int64_t m, int k, int64_t ld, double* part, double* sign,
                                  cudaStream_t st);
// Cholesky-QR step support: given S = V^T V (k x k, FP64, ld k), overwrite Rinv (k x k, ld k) with
// the inverse of the upper Cholesky factor (S = R^T R).  One CTA.  *status is set to 1 if S is not
// positive definite (left as it is otherwise).
// diag (optional, k entries) replaces the diagonal of S; run_if (optional device flag): the kernel
// does nothing unless *run_if != 0.
cudaError_t launch_chol_inv(const double* S, int k, double* Rinv, int* status, cudaStream_t st,
                            const double* diag = nullptr, const int* run_if = nullptr);
// Block-Krylov basis Q (s x 8 nblk, FP32, nblk in 2..8) of the Gram G and H = Q^T G Q
// (8 nblk x 8 nblk, FP64, ld 8 nblk) in one thread-block cluster (krylov.cu).  G32: s x s FP32
// scratch (used when a CTA's rows of G do not fit in shared memory); *lost is set if a block lost
// rank.  start: X_0 (s x 8, column-major) or nullptr for a fixed pseudo-random block.  Requires
// s >= 64.
cudaError_t launch_krylov(const double* G, float* G32, int64_t s, int nblk, float* Q, double* H,
                          int* lost, uint64_t seed, const float* start, cudaStream_t st);
// scale column j of V (m x k, ld) by 1/sqrt(theta[j])
cudaError_t launch_scale_cols_rsqrt(double* V, int64_t m, int k, int64_t ld, const double* theta,
                                    cudaStream_t st);
// copy an m x k column-major block (ld_in) into U columns [c0, c0+k) (ld_out), with FP32 mirror,
// column c multiplied by sign[c] (optional)
cudaError_t launch_copy_cols(const double* in, int64_t ld_in, int64_t m, int k, double* out,
                             int64_t ld_out, float* mirror, cudaStream_t st, const double* sign = nullptr);
// append b coefficient vectors (b x r, row-major) to the last core rows [n0, n0+b) (ld cap)
cudaError_t launch_append_last(const double* coef, int b, int r, double* last, int64_t n0,
                               int64_t ld, cudaStream_t st);
template <typename TC>
cudaError_t launch_append_last_t(const TC* coef, int b, int r, double* last, int64_t n0, int64_t ld,
                                 cudaStream_t st);
// out[j] = sum_i V[j*ld + i]^2 for the k columns of an m x k column-major matrix
cudaError_t launch_col_norms(const double* V, int64_t m, int k, int64_t ld, double* out,
                             cudaStream_t st);
// res[j] = ||GQ[:,j] - theta[j] Q[:,j]|| for j < k (column-major, ld s)
cudaError_t launch_ritz_residual(const double* GQ, const double* Q, const double* theta, int64_t s,
                                 int k, double* res, cudaStream_t st);
// rel[j] = sqrt(sum_i rho2s[i b + j] / y2[j]) (0 when y2 = 0); rho2s stage-major, nst x b
cudaError_t launch_rel_err(const double* rho2s, int nst, const double* y2, int b, double* rel,
                           cudaStream_t st);
// gather top-K eigenvector columns of a float/double s x s column-major matrix into FP64 Q (s x K)
template <typename T>
cudaError_t launch_to_f64(const T* in, int64_t n, double* out, cudaStream_t st);

}  // namespace ttice

#define TT_CUDA(x)                               \
  do {                                           \
    cudaError_t e__ = (x);                       \
    if (e__ != cudaSuccess) return e__;          \
  } while (0)
