// Symmetric eigen-solve of residual Gram matrices (the truncated SVD of Eq. 9 via G = R R^T) and the
// rank rule of the delta-truncated SVD (Eq. 5).
//
// jacobi_eig: cyclic two-sided Jacobi (Golub & Van Loan, Sec. 8.5) with the round-robin ("circle")
// ordering, so that the s/2 rotations of one round act on disjoint index pairs and are applied in
// parallel: all rotation angles of a round are computed from the matrix before the round, then the
// rows of the rotated pairs are combined, then the columns (A <- J^T A J with J block diagonal), and
// the eigenvector matrix is updated (V <- V J).  One CTA of 1024 threads; the working matrix lives in
// shared memory when it fits, otherwise in global scratch.  A rotation is skipped when
// |a_pq| <= eps_T sqrt(|a_pp a_qq|); sweeps stop when a sweep performs no rotation or after a fixed
// sweep limit (reported through `status`, never by spinning).
#include <algorithm>
#include <cfloat>
#include <mutex>

#include "ttice_internal.cuh"

namespace ttice {
namespace {

template <typename T> struct Lim;
template <> struct Lim<float> { static __device__ float eps() { return FLT_EPSILON; } };
template <> struct Lim<double> { static __device__ double eps() { return DBL_EPSILON; } };

constexpr int kMaxSweeps = 40;
constexpr int kEigThreads = 1024;
constexpr size_t kEigSmemMax = 200 * 1024;  // dynamic shared memory cap of jacobi_kernel

template <typename T>
__global__ void __launch_bounds__(kEigThreads) jacobi_kernel(const double* G, int64_t ldg, int s,
                                                             T* w, T* Vout, T* work, int* status,
                                                             int use_smem) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T rc[512], rsn[512];
  __shared__ int rp[512], rq[512];
  __shared__ int nrot;
  const int lda = s + 1;
  T* A = use_smem ? reinterpret_cast<T*>(smem_raw) : work;
  T* V = work + (use_smem ? 0 : (int64_t)s * lda);  // s x s column-major, ld s
  const int tid = threadIdx.x, nt = blockDim.x;

  __shared__ double red[33];
  __shared__ int stall;
  __shared__ double prev_off;
  double fro = 0.0;
  for (int64_t e = tid; e < (int64_t)s * s; e += nt) {
    const int i = (int)(e / s), j = (int)(e % s);
    const double g = G[i * ldg + j];
    fro += g * g;
    A[i * lda + j] = (T)g;
    V[(int64_t)j * s + i] = (i == j) ? T(1) : T(0);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  if ((tid & 31) == 0) red[tid >> 5] = fro;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < nt / 32; ++w) t += red[w];
    red[0] = sqrt(t);
  }
  __syncthreads();
  // Off-diagonal entries below eps_T ||A||_F are at the rounding level of the working precision:
  // rotating them moves no eigenvalue beyond that level.  Rotations at that level regenerate noise of
  // the same size, so the sweeps also stop once the off-diagonal norm has stagnated (see below).
  const T floor_abs = (T)((double)Lim<T>::eps() * red[0]);
  __syncthreads();

  const int np = (s + 1) & ~1;  // players, with a dummy when s is odd
  const int npairs = np / 2;
  const T teps = Lim<T>::eps();
  int sweep = 0;
  for (; sweep < kMaxSweeps; ++sweep) {
    if (tid == 0) nrot = 0;
    __syncthreads();
    for (int round = 0; round < np - 1; ++round) {
      for (int k = tid; k < npairs; k += nt) {
        int p, q;
        if (k == 0) { p = round; q = np - 1; }
        else { p = (round + k) % (np - 1); q = (round - k + (np - 1)) % (np - 1); }
        if (p > q) { int t = p; p = q; q = t; }
        T c = T(1), sn = T(0);
        if (q < s) {
          const T apq = A[p * lda + q];
          const T app = A[p * lda + p], aqq = A[q * lda + q];
          if (fabs(apq) > floor_abs && fabs(apq) > teps * sqrt(fabs(app * aqq))) {
            const T tau = (aqq - app) / (T(2) * apq);
            const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
            c = T(1) / sqrt(T(1) + t * t);
            sn = t * c;
            atomicAdd(&nrot, 1);
          }
        }
        rc[k] = c; rsn[k] = sn; rp[k] = p; rq[k] = (q < s) ? q : -1;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int64_t e = tid; e < (int64_t)npairs * s; e += nt) {
        const int k = (int)(e / s), j = (int)(e % s);
        const int q = rq[k];
        if (q < 0 || rsn[k] == T(0)) continue;
        const int p = rp[k];
        const T c = rc[k], sn = rsn[k];
        const T ap = A[p * lda + j], aq = A[q * lda + j];
        A[p * lda + j] = c * ap - sn * aq;
        A[q * lda + j] = sn * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, and V <- V J
      for (int64_t e = tid; e < (int64_t)npairs * s; e += nt) {
        const int k = (int)(e / s), i = (int)(e % s);
        const int q = rq[k];
        if (q < 0 || rsn[k] == T(0)) continue;
        const int p = rp[k];
        const T c = rc[k], sn = rsn[k];
        const T ap = A[i * lda + p], aq = A[i * lda + q];
        A[i * lda + p] = c * ap - sn * aq;
        A[i * lda + q] = sn * ap + c * aq;
        const T vp = V[(int64_t)p * s + i], vq = V[(int64_t)q * s + i];
        V[(int64_t)p * s + i] = c * vp - sn * vq;
        V[(int64_t)q * s + i] = sn * vp + c * vq;
      }
      __syncthreads();
    }
    __syncthreads();
    if (nrot == 0) break;
    // off-diagonal norm after this sweep: Jacobi converges quadratically, so a sweep that does not
    // at least quarter it is rotating rounding noise -- stop there
    double off = 0.0;
    for (int64_t e = tid; e < (int64_t)s * s; e += nt) {
      const int i = (int)(e / s), j = (int)(e % s);
      if (i != j) { const double a = (double)A[i * lda + j]; off += a * a; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
    __syncthreads();
    if ((tid & 31) == 0) red[1 + (tid >> 5)] = off;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < nt / 32; ++w) t += red[1 + w];
      stall = (sweep > 0 && t > 0.25 * prev_off) ? 1 : 0;
      prev_off = t;
    }
    __syncthreads();
    if (stall) break;
  }
  if (tid == 0 && status) *status = (sweep >= kMaxSweeps) ? 1 : 0;
  // sort by descending eigenvalue (ties by index) and write outputs
  for (int i = tid; i < s; i += nt) {
    const T di = A[i * lda + i];
    int rank = 0;
    for (int j = 0; j < s; ++j) {
      const T dj = A[j * lda + j];
      rank += (dj > di) || (dj == di && j < i);
    }
    w[rank] = di;
    for (int r = 0; r < s; ++r) Vout[(int64_t)rank * s + r] = V[(int64_t)i * s + r];
  }
}

__global__ void rank_rule_kernel(const double* theta, int K, int full, const double* trace,
                                 const double* eps_c, int max_new, int* out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double tol = *eps_c;
  int r = -1;
  if (full) {
    // tail(r) = sum_{j >= r} theta_j, accumulated from the smallest (negative Ritz values are 0)
    double tail = 0.0;
    // find the smallest r with sqrt(tail(r)) <= tol: scan r from K down to 0
    int best = K;
    for (int j = K - 1; j >= 0; --j) {
      tail += fmax(theta[j], 0.0);
      if (sqrt(tail) <= tol) best = j;
      else break;
    }
    r = best;
  } else {
    double acc = 0.0;
    const double tr = *trace;
    if (sqrt(fmax(tr, 0.0)) <= tol) r = 0;
    for (int j = 0; j < K && r < 0; ++j) {
      acc += fmax(theta[j], 0.0);
      if (sqrt(fmax(tr - acc, 0.0)) <= tol) r = j + 1;
    }
  }
  if (r > max_new) r = max_new;
  out[0] = r;
}

// Inverse of the upper Cholesky factor of an SPD k x k matrix (column-major, ld k), one CTA.
__global__ void chol_inv_kernel(const double* S, int k, double* Rinv, int* status) {
  extern __shared__ double sm[];
  double* R = sm;          // k x k, column-major
  double* Ri = sm + k * k; // k x k
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < k * k; e += nt) { R[e] = S[e]; Ri[e] = 0.0; }
  __syncthreads();
  __shared__ int bad;
  if (tid == 0) bad = 0;
  __syncthreads();
  // right-looking Cholesky, upper factor: S = R^T R
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      double d = R[j + j * k];
      if (!(d > 0.0)) { bad = 1; d = 1.0; }
      R[j + j * k] = sqrt(d);
    }
    __syncthreads();
    const double rjj = R[j + j * k];
    for (int c = j + 1 + tid; c < k; c += nt) R[j + c * k] /= rjj;
    __syncthreads();
    for (int e = tid; e < (k - j - 1) * (k - j - 1); e += nt) {
      const int a = j + 1 + e / (k - j - 1), c = j + 1 + e % (k - j - 1);
      if (c >= a) R[a + c * k] -= R[j + a * k] * R[j + c * k];
    }
    __syncthreads();
  }
  // invert the upper triangular R column by column (each thread one column of Ri)
  for (int c = tid; c < k; c += nt) {
    for (int i = c; i >= 0; --i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int l = i + 1; l <= c; ++l) v -= R[i + l * k] * Ri[l + c * k];
      Ri[i + c * k] = v / R[i + i * k];
    }
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += nt) {
    const int i = e % k, c = e / k;
    Rinv[e] = (i <= c) ? Ri[e] : 0.0;
  }
  if (tid == 0 && status) *status = bad;
}

}  // namespace

template <typename T>
cudaError_t jacobi_eig(const double* G, int64_t ldg, int s, T* w, T* V, T* work, int* status,
                       cudaStream_t st) {
  if (s <= 0) return cudaSuccess;
  if (s > 1024) return cudaErrorInvalidValue;
  const size_t need = (size_t)s * (s + 1) * sizeof(T);
  const int use_smem = need <= kEigSmemMax;
  const size_t smem = use_smem ? need : 0;
  // The attribute is raised once, to the largest size any call uses, so that concurrent calls from
  // several host threads never race a smaller setting against a launch that needs more.
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(jacobi_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kEigSmemMax);
  });
  TT_CUDA(attr_err);
  // threads: about four rotation-update items per thread per phase, so that small problems do not
  // pay for 1024-thread barriers
  const int npairs = (s + 1) / 2;
  int threads = (int)std::min<int64_t>(kEigThreads, std::max<int64_t>(64, ((int64_t)npairs * s / 4 + 31) / 32 * 32));
  note_launch();
  jacobi_kernel<T><<<1, threads, smem, st>>>(G, ldg, s, w, V, work, status, use_smem);
  return cudaGetLastError();
}

template cudaError_t jacobi_eig<float>(const double*, int64_t, int, float*, float*, float*, int*,
                                       cudaStream_t);
template cudaError_t jacobi_eig<double>(const double*, int64_t, int, double*, double*, double*,
                                        int*, cudaStream_t);

cudaError_t launch_rank_rule(const double* theta, int K, int full, const double* trace,
                             const double* eps_c, int max_new, int* out, cudaStream_t st) {
  note_launch();
  rank_rule_kernel<<<1, 32, 0, st>>>(theta, K, full, trace, eps_c, max_new, out);
  return cudaGetLastError();
}

cudaError_t launch_chol_inv(const double* S, int k, double* Rinv, int* status, cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  if (k > 112) return cudaErrorInvalidValue;
  const size_t smem = 2 * (size_t)k * k * sizeof(double);
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(chol_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(2 * 112 * 112 * sizeof(double)));
  });
  TT_CUDA(attr_err);
  note_launch();
  chol_inv_kernel<<<1, 256, smem, st>>>(S, k, Rinv, status);
  return cudaGetLastError();
}

}  // namespace ttice
