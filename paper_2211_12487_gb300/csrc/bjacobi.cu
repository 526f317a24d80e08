// Multi-CTA block Jacobi eigen-solver for the residual Gram matrices of Eq. 9 (s up to 1024).
//
// Two-sided cyclic block Jacobi (Golub & Van Loan, Sec. 8.5, block variant): the matrix is split
// into nb blocks of BS rows/columns; the block pairs (I, J) of one round come from the round-robin
// ordering on block indices, so the nb/2 pairs of a round are disjoint.  One round is three kernels:
//   solve: one CTA per pair loads the 2BS x 2BS submatrix A[I u J, I u J] into shared memory and
//          applies one cyclic sweep of scalar Jacobi rotations to it, accumulating the orthogonal
//          Q (2BS x 2BS) of the sweep;
//   rows:  A[I u J, :] <- Q^T A[I u J, :] for every pair (disjoint row sets), tiled over columns;
//   cols:  A[:, I u J] <- A[:, I u J] Q and V[:, I u J] <- V[:, I u J] Q, tiled over rows.
// A sweep is nb-1 rounds; a flag raised by any significant rotation keeps the next sweep alive, and
// a sweep that leaves the off-diagonal norm at the working precision's rounding level without
// halving it ends the solve too (rotations of rounding noise would otherwise run to the sweep cap);
// every kernel returns at once after the solve has ended, so a fixed launch sequence costs almost
// nothing once converged.  Padding to nb*BS adds zero rows/columns, which no rotation touches (their
// off-diagonal entries are exactly zero), so the first s coordinates carry the eigenpairs.
#include <algorithm>
#include <cfloat>

#include "ttice_internal.cuh"

namespace ttice {
namespace {

template <typename T> struct BJ;
template <> struct BJ<float> {
  static constexpr int BS = 16;
  static __device__ float eps() { return FLT_EPSILON; }
};
template <> struct BJ<double> {
  static constexpr int BS = 16;
  static __device__ double eps() { return DBL_EPSILON; }
};

constexpr int kTile = 64;
constexpr int kThreads = 256;

__device__ __forceinline__ void circle_pair(int players, int round, int k, int* p, int* q) {
  int a, b;
  if (k == 0) { a = round; b = players - 1; }
  else { a = (round + k) % (players - 1); b = (round - k + (players - 1)) % (players - 1); }
  *p = a < b ? a : b;
  *q = a < b ? b : a;
}

template <typename T>
__global__ void bj_init(const double* G, int64_t ldg, int s, int sp, T* A, T* V, double* fro,
                        int* flags) {
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)sp * sp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / sp), j = (int)(e % sp);
    double g = (i < s && j < s) ? G[i * ldg + j] : 0.0;
    acc += g * g;
    A[e] = (T)g;
    V[(int64_t)j * sp + i] = (i == j) ? T(1) : T(0);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(fro, acc);
  if (blockIdx.x == 0 && threadIdx.x == 0) { flags[0] = 0; flags[1] = 0; flags[2] = 0; }
}

// One CTA per block pair, one warp per rotation: the 2BS x 2BS subproblem lives in shared memory;
// in each of the 2BS-1 rounds of a cyclic sweep, lane 0 of warp k computes the rotation of pair k
// (broadcast by a shuffle), the warp combines the two rows of its pair, the CTA synchronises, the
// warp combines the two columns (of S and of the accumulated Q), and the CTA synchronises again.
template <typename T>
__global__ void __launch_bounds__(32 * BJ<T>::BS) bj_solve(const T* A, int sp, int nb, int round,
                                                           T* Qb, const double* fro, int* flags) {
  constexpr int BS = BJ<T>::BS, N2 = 2 * BS;
  static_assert(N2 == 32, "one lane per row/column element");
  if (flags[1]) return;
  __shared__ T S[N2][N2 + 1];
  __shared__ T Q[N2][N2 + 1];
  int bi, bj;
  circle_pair(nb, round, blockIdx.x, &bi, &bj);
  const int tid = threadIdx.x, k = tid >> 5, lane = tid & 31;
  auto gidx = [&](int a) { return a < BS ? bi * BS + a : bj * BS + (a - BS); };
  for (int e = tid; e < N2 * N2; e += 32 * BS) {
    const int a = e / N2, b = e % N2;
    S[a][b] = A[(int64_t)gidx(a) * sp + gidx(b)];
    Q[a][b] = (a == b) ? T(1) : T(0);
  }
  __syncthreads();
  const T teps = BJ<T>::eps();
  const T floor_abs = (T)((double)teps * sqrt(*fro));  // rounding level, see jacobi_kernel
  int any = 0;
  for (int round2 = 0; round2 < N2 - 1; ++round2) {
    int p, q;
    circle_pair(N2, round2, k, &p, &q);
    T c = T(1), sn = T(0);
    if (lane == 0) {
      const T apq = S[p][q], app = S[p][p], aqq = S[q][q];
      if (fabs(apq) > floor_abs && fabs(apq) > teps * sqrt(fabs(app * aqq))) {
        const T tau = (aqq - app) / (T(2) * apq);
        const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
        c = T(1) / sqrt(T(1) + t * t);
        sn = t * c;
        any = 1;
      }
    }
    c = __shfl_sync(0xffffffffu, c, 0);
    sn = __shfl_sync(0xffffffffu, sn, 0);
    if (sn != T(0)) {  // rows p, q of S
      const T xp = S[p][lane], xq = S[q][lane];
      S[p][lane] = c * xp - sn * xq;
      S[q][lane] = sn * xp + c * xq;
    }
    __syncthreads();
    if (sn != T(0)) {  // columns p, q of S and of Q
      const T xp = S[lane][p], xq = S[lane][q];
      S[lane][p] = c * xp - sn * xq;
      S[lane][q] = sn * xp + c * xq;
      const T vp = Q[lane][p], vq = Q[lane][q];
      Q[lane][p] = c * vp - sn * vq;
      Q[lane][q] = sn * vp + c * vq;
    }
    __syncthreads();
  }
  T* Qo = Qb + (int64_t)blockIdx.x * N2 * N2;
  for (int e = tid; e < N2 * N2; e += 32 * BS) Qo[e] = Q[e / N2][e % N2];
  if (__syncthreads_or(any) && tid == 0) atomicOr(flags, 1);
}

// A[I u J, tile] <- Q^T A[I u J, tile]
template <typename T>
__global__ void __launch_bounds__(kThreads) bj_rows(T* A, int sp, int nb, int round, const T* Qb,
                                                    const int* flags) {
  constexpr int BS = BJ<T>::BS, N2 = 2 * BS;
  if (flags[1]) return;
  __shared__ T Q[N2][N2 + 1];
  __shared__ T X[N2][kTile + 1];
  int bi, bj;
  circle_pair(nb, round, blockIdx.x, &bi, &bj);
  const int c0 = blockIdx.y * kTile;
  const int tid = threadIdx.x;
  const T* Qi = Qb + (int64_t)blockIdx.x * N2 * N2;
  auto gidx = [&](int a) { return a < BS ? bi * BS + a : bj * BS + (a - BS); };
  for (int e = tid; e < N2 * N2; e += kThreads) Q[e / N2][e % N2] = Qi[e];
  for (int e = tid; e < N2 * kTile; e += kThreads) {
    const int a = e / kTile, c = e % kTile;
    X[a][c] = (c0 + c < sp) ? A[(int64_t)gidx(a) * sp + c0 + c] : T(0);
  }
  __syncthreads();
  for (int e = tid; e < N2 * kTile; e += kThreads) {
    const int a = e / kTile, c = e % kTile;
    if (c0 + c >= sp) continue;
    T acc = T(0);
#pragma unroll 8
    for (int b = 0; b < N2; ++b) acc = fma(Q[b][a], X[b][c], acc);
    A[(int64_t)gidx(a) * sp + c0 + c] = acc;
  }
}

// A[tile, I u J] <- A[tile, I u J] Q ; V[tile, I u J] <- V[tile, I u J] Q (V column-major)
template <typename T>
__global__ void __launch_bounds__(kThreads) bj_cols(T* A, T* V, int sp, int nb, int round,
                                                    const T* Qb, const int* flags) {
  constexpr int BS = BJ<T>::BS, N2 = 2 * BS;
  if (flags[1]) return;
  __shared__ T Q[N2][N2 + 1];
  __shared__ T X[kTile][N2 + 1];  // the A tile, then the V tile (both as [row][pair column])
  int bi, bj;
  circle_pair(nb, round, blockIdx.x, &bi, &bj);
  const int r0 = blockIdx.y * kTile;
  const int tid = threadIdx.x;
  const T* Qi = Qb + (int64_t)blockIdx.x * N2 * N2;
  auto gidx = [&](int a) { return a < BS ? bi * BS + a : bj * BS + (a - BS); };
  for (int e = tid; e < N2 * N2; e += kThreads) Q[e / N2][e % N2] = Qi[e];
  for (int e = tid; e < kTile * N2; e += kThreads) {
    const int i = e / N2, a = e % N2;
    X[i][a] = (r0 + i < sp) ? A[(int64_t)(r0 + i) * sp + gidx(a)] : T(0);
  }
  __syncthreads();
  for (int e = tid; e < kTile * N2; e += kThreads) {
    const int i = e / N2, a = e % N2;
    if (r0 + i >= sp) continue;
    T acc = T(0);
#pragma unroll 8
    for (int b = 0; b < N2; ++b) acc = fma(X[i][b], Q[b][a], acc);
    A[(int64_t)(r0 + i) * sp + gidx(a)] = acc;
  }
  __syncthreads();
  for (int e = tid; e < N2 * kTile; e += kThreads) {
    const int a = e / kTile, i = e % kTile;
    X[i][a] = (r0 + i < sp) ? V[(int64_t)gidx(a) * sp + r0 + i] : T(0);
  }
  __syncthreads();
  for (int e = tid; e < N2 * kTile; e += kThreads) {
    const int a = e / kTile, i = e % kTile;
    if (r0 + i >= sp) continue;
    T acc = T(0);
#pragma unroll 8
    for (int b = 0; b < N2; ++b) acc = fma(X[i][b], Q[b][a], acc);
    V[(int64_t)gidx(a) * sp + r0 + i] = acc;
  }
}

// Squared off-diagonal norm of A after a sweep, accumulated into *off.
template <typename T>
__global__ void bj_offnorm(const T* A, int sp, double* off, const int* flags) {
  if (flags[1]) return;
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)sp * sp;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(e / sp), j = (int)(e % sp);
    if (i != j) { const double a = (double)A[e]; acc += a * a; }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(off, acc);
}

// End of a sweep.  norms: [0] ||A||_F^2, [1] off-diagonal^2 after this sweep (reset here), [2] after
// the previous sweep.  The solve has converged when a sweep rotated nothing, or when the
// off-diagonal norm is at the rounding level of T (below 64 sqrt(s) eps_T ||A||_F) and the sweep
// did not halve it: the rotations left are rotating rounding noise (the rule of jacobi_kernel).
template <typename T>
__global__ void bj_sweep_end(int* flags, int max_sweeps, double* norms, int s) {
  if (flags[1]) return;
  const double gate = 64.0 * sqrt((double)s) * (double)BJ<T>::eps() * sqrt(norms[0]);
  const bool stalled = flags[2] >= 1 && norms[1] > 0.25 * norms[2] && norms[1] <= gate * gate;
  flags[2] += 1;
  if (flags[0] == 0 || stalled) flags[1] = 1;
  else if (flags[2] >= max_sweeps) flags[3] = 1;  // sweep limit reached while still rotating
  flags[0] = 0;
  norms[2] = norms[1];
  norms[1] = 0.0;
}

// eigenvalues = diag(A)[0..s), sorted descending (ties by index); eigenvectors follow.
template <typename T>
__global__ void bj_finish(const T* A, const T* V, int sp, int s, T* w, T* Vout) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < s; i += gridDim.x * blockDim.x) {
    const T di = A[(int64_t)i * sp + i];
    int rank = 0;
    for (int j = 0; j < s; ++j) {
      const T dj = A[(int64_t)j * sp + j];
      rank += (dj > di) || (dj == di && j < i);
    }
    w[rank] = di;
    const T* src = V + (int64_t)i * sp;
    T* dst = Vout + (int64_t)rank * s;
    for (int r = 0; r < s; ++r) dst[r] = src[r];
  }
}

}  // namespace

template <typename T>
int64_t block_jacobi_work(int s) {
  constexpr int BS = BJ<T>::BS, N2 = 2 * BS;
  int nb = (s + BS - 1) / BS;
  nb += nb & 1;
  const int64_t sp = (int64_t)nb * BS;
  return 2 * sp * sp + (int64_t)(nb / 2) * N2 * N2 + 16;
}

template <typename T>
cudaError_t block_jacobi_eig(const double* G, int64_t ldg, int s, T* w, T* Vout, T* work,
                             double* fro, int* flags, int max_sweeps, cudaStream_t st) {
  constexpr int BS = BJ<T>::BS, N2 = 2 * BS;
  if (s <= 0) return cudaSuccess;
  int nb = (s + BS - 1) / BS;
  nb += nb & 1;
  if (nb < 2) nb = 2;
  const int sp = nb * BS;
  T* A = work;
  T* V = work + (int64_t)sp * sp;
  T* Qb = V + (int64_t)sp * sp;
  const int npairs = nb / 2;
  TT_CUDA(cudaMemsetAsync(fro, 0, 3 * sizeof(double), st));
  TT_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), st));
  {
    int64_t n = (int64_t)sp * sp;
    int grid = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 8);
    note_launch();
    bj_init<T><<<grid, kThreads, 0, st>>>(G, ldg, s, sp, A, V, fro, flags);
  }
  const int tiles = (sp + kTile - 1) / kTile;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    for (int round = 0; round < nb - 1; ++round) {
      note_launch();
      bj_solve<T><<<npairs, 32 * BS, 0, st>>>(A, sp, nb, round, Qb, fro, flags);
      note_launch();
      bj_rows<T><<<dim3(npairs, tiles), kThreads, 0, st>>>(A, sp, nb, round, Qb, flags);
      note_launch();
      bj_cols<T><<<dim3(npairs, tiles), kThreads, 0, st>>>(A, V, sp, nb, round, Qb, flags);
    }
    {
      const int64_t n = (int64_t)sp * sp;
      const int grid = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 2);
      note_launch();
      bj_offnorm<T><<<grid, kThreads, 0, st>>>(A, sp, fro + 1, flags);
    }
    note_launch();
    bj_sweep_end<T><<<1, 1, 0, st>>>(flags, max_sweeps, fro, s);
  }
  note_launch();
  bj_finish<T><<<(s + 127) / 128, 128, 0, st>>>(A, V, sp, s, w, Vout);
  (void)N2;
  return cudaGetLastError();
}

template int64_t block_jacobi_work<float>(int);
template int64_t block_jacobi_work<double>(int);
template cudaError_t block_jacobi_eig<float>(const double*, int64_t, int, float*, float*, float*,
                                             double*, int*, int, cudaStream_t);
template cudaError_t block_jacobi_eig<double>(const double*, int64_t, int, double*, double*,
                                              double*, double*, int*, int, cudaStream_t);

}  // namespace ttice
