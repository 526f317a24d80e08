// Multi-CTA block Jacobi eigen-solver for the residual Gram matrices of Eq. 9 (s up to 4608; blocks
// of BS = 32 in FP32, 16 in FP64).
//
// Two-sided cyclic block Jacobi (Golub & Van Loan, Sec. 8.5, block variant): the matrix is split
// into nb blocks of BS rows/columns; the block pairs (I, J) of one round come from the round-robin
// ordering on block indices, so the nb/2 pairs of a round are disjoint.  One round is three kernels:
//   solve:    one CTA per pair loads the 2BS x 2BS submatrix A[I u J, I u J] into shared memory and
//             applies one cyclic sweep of scalar Jacobi rotations to it, accumulating the orthogonal
//             Q (2BS x 2BS) of the sweep;
//   update A: A_out[P_a, P_b] = Q_a^T A_in[P_a, P_b] Q_b for every pair of index sets (one 2BS x 2BS
//             block per CTA; A is double-buffered, so rows and columns are combined in one pass);
//   update V: V[:, P_a] <- V[:, P_a] Q_a in 64-row tiles.
// The next round's solve needs only A, so the V update of a round runs on a second branch of the
// graph, beside the next round's solve and A update (the Q factors alternate between two buffers,
// and a solve waits for the V update that read its buffer two rounds before).
// A sweep is nb-1 rounds; a flag raised by any significant rotation keeps the next sweep alive.  A
// sweep that leaves the off-diagonal norm at the rounding level of the working precision ends the
// solve (below sqrt(s) eps_T ||A||_F, the level of the FP rounding of A itself; or below 64 times
// that without halving it, when the rotations are turning rounding noise); every kernel returns at
// once after the solve has ended, so a fixed launch sequence costs almost nothing once converged.
// Two sweeps of launches are captured once into a CUDA graph and replayed.  Padding to nb*BS adds
// zero rows/columns, which no rotation touches (their off-diagonal entries are exactly zero), so
// the first s coordinates carry the eigenpairs.
#include <algorithm>
#include <cfloat>
#include <map>
#include <mutex>
#include <tuple>
#include <type_traits>

#include "ttice_internal.cuh"

namespace ttice {
namespace {

template <typename T> struct BJ;
template <> struct BJ<float> {
  static constexpr int BS = 32;  // 64 x 64 sub-problems: half the rounds per sweep of BS = 16
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
  constexpr int BS = BJ<T>::BS, N2 = 2 * BS, EL = N2 / 32;  // elements of a row / column per lane
  static_assert(N2 % 32 == 0, "whole warps per row / column");
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
        // t = sgn(tau) / (|tau| + sqrt(1 + tau^2)), tau = (a_qq - a_pp) / (2 a_pq), multiplied
        // through by |2 a_pq|: one hypot, one division, one reciprocal square root
        const T th = aqq - app, ph = T(2) * apq;
        const bool pos = (th == T(0)) || ((th > T(0)) == (ph > T(0)));
        const T mag = fabs(ph) / (fabs(th) + hypot(th, ph));
        const T t = pos ? mag : -mag;
        c = rsqrt(T(1) + t * t);
        sn = t * c;
        any = 1;
      }
    }
    c = __shfl_sync(0xffffffffu, c, 0);
    sn = __shfl_sync(0xffffffffu, sn, 0);
    if (sn != T(0)) {  // rows p, q of S
#pragma unroll
      for (int h = 0; h < EL; ++h) {
        const int x = lane + 32 * h;
        const T xp = S[p][x], xq = S[q][x];
        S[p][x] = c * xp - sn * xq;
        S[q][x] = sn * xp + c * xq;
      }
    }
    __syncthreads();
    if (sn != T(0)) {  // columns p, q of S and of Q
#pragma unroll
      for (int h = 0; h < EL; ++h) {
        const int x = lane + 32 * h;
        const T xp = S[x][p], xq = S[x][q];
        S[x][p] = c * xp - sn * xq;
        S[x][q] = sn * xp + c * xq;
        const T vp = Q[x][p], vq = Q[x][q];
        Q[x][p] = c * vp - sn * vq;
        Q[x][q] = sn * vp + c * vq;
      }
    }
    __syncthreads();
  }
  T* Qo = Qb + (int64_t)blockIdx.x * N2 * N2;
  for (int e = tid; e < N2 * N2; e += 32 * BS) Qo[e] = Q[e / N2][e % N2];
  if (__syncthreads_or(any) && tid == 0) atomicOr(flags, 1);
}

// One round's update of A and V with the pairs' orthogonal factors Q (2BS x 2BS each):
//   A_out[P_a, P_b] = Q_a^T A_in[P_a, P_b] Q_b  for every pair of index sets P_a = I_a u J_a, and
//   V[:, P_a] <- V[:, P_a] Q_a                  (in place: the column sets are disjoint).
// part 0: one CTA per A block on or above the diagonal (each block above it also writes its mirror,
// so A stays exactly symmetric); part 1: one CTA per 64-row tile of V and pair.
// The products are register-tiled: the 256 threads form a 16 x 16 grid and each computes an R x R
// (A block, R = 2BS / 16) or 4 x R (V tile) piece of the result from rows of the shared-memory
// operands, so that a shared-memory load feeds R fused multiply-adds instead of one.
template <typename T>
__global__ void __launch_bounds__(kThreads) bj_update(const T* Ain, T* Aout, T* V, int sp, int nb, int round,
                                                      const T* Qb, const int* flags, int part) {
  constexpr int BS = BJ<T>::BS, N2 = 2 * BS, R = N2 / 16, RV = kTile / 16, LD = N2 + 4;
  constexpr int LDX = (N2 > kTile ? N2 : kTile) + 4;  // X holds N2 x N2 (A block) or N2 x kTile (V)
  constexpr int VEC = 16 / (int)sizeof(T);
  using Vec = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
  static_assert(BS % VEC == 0 && LD % VEC == 0 && LDX % VEC == 0, "16-byte aligned rows");
  static_assert(N2 % 16 == 0 && kThreads == 256, "16 x 16 thread grid");
  if (flags[1]) return;
  // dynamic shared memory: Qa, Qc (N2 rows of LD) and X (N2 rows of LDX)
  extern __shared__ __align__(16) unsigned char bj_smem[];
  T* Qa = reinterpret_cast<T*>(bj_smem);
  T* Qc = Qa + N2 * LD;
  T* X = Qc + N2 * LD;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  if (part == 0) {
    // block index -> (a, b), a <= b, column by column of the upper triangle: b (b + 1) / 2 + a
    const int64_t q = blockIdx.x;
    int b = (int)((sqrt(8.0 * (double)q + 1.0) - 1.0) * 0.5);
    while ((int64_t)b * (b + 1) / 2 > q) --b;
    while ((int64_t)(b + 1) * (b + 2) / 2 <= q) ++b;
    const int a = (int)(q - (int64_t)b * (b + 1) / 2);
    int ai, aj, bi, bj;
    circle_pair(nb, round, a, &ai, &aj);
    circle_pair(nb, round, b, &bi, &bj);
    auto ga = [&](int t) { return t < BS ? ai * BS + t : aj * BS + (t - BS); };
    auto gb = [&](int t) { return t < BS ? bi * BS + t : bj * BS + (t - BS); };
    const T* Qa_g = Qb + (int64_t)a * N2 * N2;
    const T* Qb_g = Qb + (int64_t)b * N2 * N2;
    // 16-byte loads and stores (VEC elements), several in flight per thread: the loads come from L2
    // and would otherwise be exposed one by one
#pragma unroll 4
    for (int e = tid * VEC; e < N2 * N2; e += kThreads * VEC) {
      const int r = e / N2, c = e % N2;  // c is a multiple of VEC: within one half of the pair
      *reinterpret_cast<Vec*>(Qa + r * LD + c) = *reinterpret_cast<const Vec*>(Qa_g + e);
      *reinterpret_cast<Vec*>(Qc + r * LD + c) = *reinterpret_cast<const Vec*>(Qb_g + e);
      *reinterpret_cast<Vec*>(X + r * LDX + c) = *reinterpret_cast<const Vec*>(Ain + (int64_t)ga(r) * sp + gb(c));
    }
    __syncthreads();
    // M = Qa^T X: M[r][c] = sum_k Qa[k][r] X[k][c], rows r = R ty + i, columns c = R tx + j
    T m[R][R];
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) m[i][j] = T(0);
#pragma unroll 4
    for (int k = 0; k < N2; ++k) {
      T av[R], bv[R];
#pragma unroll
      for (int i = 0; i < R; ++i) av[i] = Qa[k * LD + R * ty + i];
#pragma unroll
      for (int j = 0; j < R; ++j) bv[j] = X[k * LDX + R * tx + j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) m[i][j] = fma(av[i], bv[j], m[i][j]);
    }
    __syncthreads();
    // M transposed into X: X[c][r] = M[r][c], so that the second product reads rows again
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) X[(R * tx + j) * LDX + R * ty + i] = m[i][j];
    __syncthreads();
    // O = M Qc: O[r][c] = sum_k M[r][k] Qc[k][c] = sum_k X[k][r] Qc[k][c]
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) m[i][j] = T(0);
#pragma unroll 4
    for (int k = 0; k < N2; ++k) {
      T av[R], bv[R];
#pragma unroll
      for (int i = 0; i < R; ++i) av[i] = X[k * LDX + R * ty + i];
#pragma unroll
      for (int j = 0; j < R; ++j) bv[j] = Qc[k * LD + R * tx + j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) m[i][j] = fma(av[i], bv[j], m[i][j]);
    }
    // O through shared memory (X, row-major), so that the stores to A are whole 16-byte vectors of
    // consecutive columns (stored straight from the registers, a warp's store would touch 16-32
    // rows at once)
    __syncthreads();
#pragma unroll
    for (int i = 0; i < R; ++i)
#pragma unroll
      for (int j = 0; j < R; ++j) X[(R * ty + i) * LDX + R * tx + j] = m[i][j];
    __syncthreads();
#pragma unroll 4
    for (int e = tid * VEC; e < N2 * N2; e += kThreads * VEC) {  // A_out[P_a(r)][P_b(c .. c + VEC)]
      const int r = e / N2, c = e % N2;  // c is a multiple of VEC: within one half of the pair
      *reinterpret_cast<Vec*>(Aout + (int64_t)ga(r) * sp + gb(c)) = *reinterpret_cast<const Vec*>(X + r * LDX + c);
    }
    if (a != b) {
#pragma unroll 4
      for (int e = tid * VEC; e < N2 * N2; e += kThreads * VEC) {  // the mirror: A_out[P_b(c)][P_a(r ..)]
        const int c = e / N2, r = e % N2;
        Vec w;
        T* wq = reinterpret_cast<T*>(&w);
#pragma unroll
        for (int q = 0; q < VEC; ++q) wq[q] = X[(r + q) * LDX + c];
        *reinterpret_cast<Vec*>(Aout + (int64_t)gb(c) * sp + ga(r)) = w;
      }
    }
    return;
  }
  // V tile: rows [r0, r0 + kTile) of the columns P_a; X[c][i] = V[r0 + i][P_a(c)] (V column-major)
  const int64_t vt = blockIdx.x;
  const int tiles = (sp + kTile - 1) / kTile;
  const int a = (int)(vt / tiles), r0 = (int)(vt % tiles) * kTile;
  int ai, aj;
  circle_pair(nb, round, a, &ai, &aj);
  auto ga = [&](int t) { return t < BS ? ai * BS + t : aj * BS + (t - BS); };
  const T* Qa_g = Qb + (int64_t)a * N2 * N2;
#pragma unroll 4
  for (int e = tid * VEC; e < N2 * N2; e += kThreads * VEC)
    *reinterpret_cast<Vec*>(Qa + (e / N2) * LD + e % N2) = *reinterpret_cast<const Vec*>(Qa_g + e);
#pragma unroll 4
  for (int e = tid * VEC; e < N2 * kTile; e += kThreads * VEC) {
    const int c = e / kTile, i = e % kTile;  // sp is a multiple of 32: a vector is all in or all out
    Vec v;
    if (r0 + i < sp) v = *reinterpret_cast<const Vec*>(V + (int64_t)ga(c) * sp + r0 + i);
    else v = Vec{};
    *reinterpret_cast<Vec*>(X + c * LDX + i) = v;
  }
  __syncthreads();
  // Vnew[i][c] = sum_k X[k][i] Qa[k][c]: rows i = RV ty + u, columns c = R tx + j
  T v[RV][R];
#pragma unroll
  for (int u = 0; u < RV; ++u)
#pragma unroll
    for (int j = 0; j < R; ++j) v[u][j] = T(0);
#pragma unroll 4
  for (int k = 0; k < N2; ++k) {
    T av[RV], bv[R];
#pragma unroll
    for (int u = 0; u < RV; ++u) av[u] = X[k * LDX + RV * ty + u];
#pragma unroll
    for (int j = 0; j < R; ++j) bv[j] = Qa[k * LD + R * tx + j];
#pragma unroll
    for (int u = 0; u < RV; ++u)
#pragma unroll
      for (int j = 0; j < R; ++j) v[u][j] = fma(av[u], bv[j], v[u][j]);
  }
  // the tile back through shared memory (X, the input's layout) as whole 16-byte vectors of rows
  __syncthreads();
#pragma unroll
  for (int u = 0; u < RV; ++u)
#pragma unroll
    for (int j = 0; j < R; ++j) X[(R * tx + j) * LDX + RV * ty + u] = v[u][j];
  __syncthreads();
#pragma unroll 4
  for (int e = tid * VEC; e < N2 * kTile; e += kThreads * VEC) {
    const int c = e / kTile, i = e % kTile;  // sp is a multiple of 32: a vector is all in or all out
    if (r0 + i < sp) *reinterpret_cast<Vec*>(V + (int64_t)ga(c) * sp + r0 + i) = *reinterpret_cast<const Vec*>(X + c * LDX + i);
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
// the previous sweep.  The solve has converged when a sweep rotated nothing; when the off-diagonal
// norm is below sqrt(s) eps_T ||A||_F, the size of the rounding of A's own entries in T (what is
// left is not resolved by the working precision: another sweep would only turn it); or when it is
// below 64 times that and the sweep did not halve it (rotations of rounding noise, the rule of
// jacobi_kernel).
// `cur` is the buffer (0 or 1) that holds A after this sweep; it is recorded in flags[4] when the
// solve ends here, since the launches after that return at once and swap nothing.
template <typename T>
__global__ void bj_sweep_end(int* flags, int max_sweeps, double* norms, int s, int cur) {
  if (flags[1]) return;
  const double floor2 = (double)s * (double)BJ<T>::eps() * (double)BJ<T>::eps() * norms[0];
  const double gate = 64.0 * sqrt(floor2);
  const bool stalled = (flags[2] >= 1 && norms[1] > 0.25 * norms[2] && norms[1] <= gate * gate) ||
                       norms[1] <= floor2;
  flags[2] += 1;
  flags[4] = cur;
  if (flags[0] == 0 || stalled) flags[1] = 1;
  else if (flags[2] >= max_sweeps) { flags[3] = 1; flags[1] = 1; }  // sweep limit reached while still rotating
  flags[0] = 0;
  norms[2] = norms[1];
  norms[1] = 0.0;
}

// eigenvalues = diag(A)[0..s), sorted descending (ties by index); eigenvectors follow.  A is the
// buffer flags[4] names.  One CTA per eigenpair i (kFinishThreads threads): its rank among the
// diagonal entries, counted by the whole CTA, then its vector copied with consecutive threads on
// consecutive entries.
constexpr int kFinishThreads = 128;
template <typename T>
__global__ void __launch_bounds__(kFinishThreads) bj_finish(const T* A0, const T* A1, const T* V, int sp, int s,
                                                            T* w, T* Vout, const int* flags) {
  const T* A = flags[4] ? A1 : A0;
  const int i = blockIdx.x;
  const T di = A[(int64_t)i * sp + i];
  int cnt = 0;
  for (int j = threadIdx.x; j < s; j += kFinishThreads) {
    const T dj = A[(int64_t)j * sp + j];
    cnt += (dj > di) || (dj == di && j < i);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  __shared__ int part[kFinishThreads / 32];
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = cnt;
  __syncthreads();
  int rank = 0;
#pragma unroll
  for (int k = 0; k < kFinishThreads / 32; ++k) rank += part[k];
  if (threadIdx.x == 0) w[rank] = di;
  const T* src = V + (int64_t)i * sp;
  T* dst = Vout + (int64_t)rank * s;
  for (int r = threadIdx.x; r < s; r += kFinishThreads) dst[r] = src[r];
}

}  // namespace

template <typename T>
int64_t block_jacobi_work(int s) {
  constexpr int BS = BJ<T>::BS, N2 = 2 * BS;
  int nb = (s + BS - 1) / BS;
  nb += nb & 1;
  const int64_t sp = (int64_t)nb * BS;
  return 3 * sp * sp + 2 * (int64_t)(nb / 2) * N2 * N2 + 16;  // A twice, V, Q of two rounds
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
  T* A0 = work;                       // A, double-buffered: each round reads one, writes the other
  T* A1 = work + (int64_t)sp * sp;
  T* V = A1 + (int64_t)sp * sp;
  const int npairs = nb / 2;
  T* Qbuf[2] = {V + (int64_t)sp * sp, V + (int64_t)sp * sp + (int64_t)npairs * N2 * N2};
  TT_CUDA(cudaMemsetAsync(fro, 0, 3 * sizeof(double), st));
  TT_CUDA(cudaMemsetAsync(flags, 0, 5 * sizeof(int), st));
  {
    int64_t n = (int64_t)sp * sp;
    int grid = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 8);
    note_launch();
    bj_init<T><<<grid, kThreads, 0, st>>>(G, ldg, s, sp, A0, V, fro, flags);
  }
  const int tiles = (sp + kTile - 1) / kTile;
  const int64_t a_ctas = (int64_t)npairs * (npairs + 1) / 2, v_ctas = (int64_t)npairs * tiles;
  const size_t upd_smem = ((size_t)2 * N2 * (N2 + 4) + (size_t)N2 * ((N2 > kTile ? N2 : kTile) + 4)) * sizeof(T);
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [&] {
    attr_err = cudaFuncSetAttribute(bj_update<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)upd_smem);
  });
  TT_CUDA(attr_err);
  // Two sweeps of rounds (the buffer parities repeat after two, since a sweep has nb - 1 rounds, an
  // odd count) are captured once into a CUDA graph per (buffers, size) and replayed until the sweep
  // cap; every kernel returns at once after the solve has ended.  Capture goes to private streams
  // of the calling thread (the main branch cs, the V branch cv): nothing runs there, the graph is
  // launched on st.  Edges: solve(g) -> V update(g) -> V update(g + 1) on cv; V update(g) ->
  // solve(g + 2), which overwrites its Q buffer; the last V update of a sweep -> the sweep's end
  // test, which may end the solve (a V update still to start would then skip its rotations).
  auto enqueue_two_sweeps = [&](cudaStream_t cs, cudaStream_t cv, cudaEvent_t ev_q, cudaEvent_t* ev_v) -> cudaError_t {
    int cur = 0, g = 0;
    for (int sweep = 0; sweep < 2; ++sweep) {
      for (int round = 0; round < nb - 1; ++round, ++g) {
        T* Ain = cur ? A1 : A0;
        T* Aout = cur ? A0 : A1;
        T* Qb = Qbuf[g & 1];
        if (g >= 2) TT_CUDA(cudaStreamWaitEvent(cs, ev_v[g & 1], 0));
        bj_solve<T><<<npairs, 32 * BS, 0, cs>>>(Ain, sp, nb, round, Qb, fro, flags);
        TT_CUDA(cudaEventRecord(ev_q, cs));
        bj_update<T><<<(unsigned)a_ctas, kThreads, upd_smem, cs>>>(Ain, Aout, V, sp, nb, round, Qb, flags, 0);
        TT_CUDA(cudaStreamWaitEvent(cv, ev_q, 0));
        bj_update<T><<<(unsigned)v_ctas, kThreads, upd_smem, cv>>>(Ain, Aout, V, sp, nb, round, Qb, flags, 1);
        TT_CUDA(cudaEventRecord(ev_v[g & 1], cv));
        cur ^= 1;
      }
      const int64_t n = (int64_t)sp * sp;
      const int grid = (int)std::min<int64_t>((n + kThreads - 1) / kThreads, 152 * 2);
      bj_offnorm<T><<<grid, kThreads, 0, cs>>>(cur ? A1 : A0, sp, fro + 1, flags);
      TT_CUDA(cudaStreamWaitEvent(cs, ev_v[(g - 1) & 1], 0));
      bj_sweep_end<T><<<1, 1, 0, cs>>>(flags, max_sweeps, fro, s, cur);
    }
    return cudaGetLastError();
  };
  using Key = std::tuple<const void*, const void*, const void*, int, int>;
  static std::mutex mu;
  static std::map<Key, cudaGraphExec_t> cache;
  const Key key{work, fro, flags, s, max_sweeps};
  cudaGraphExec_t exec = nullptr;
  {
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) exec = it->second;
  }
  if (!exec) {
    thread_local cudaStream_t cs = nullptr, cv = nullptr;
    thread_local cudaEvent_t ev_q = nullptr, ev_v[2] = {nullptr, nullptr};
    if (!cs) TT_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    if (!cv) TT_CUDA(cudaStreamCreateWithFlags(&cv, cudaStreamNonBlocking));
    if (!ev_q) TT_CUDA(cudaEventCreateWithFlags(&ev_q, cudaEventDisableTiming));
    for (cudaEvent_t& e : ev_v)
      if (!e) TT_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    TT_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    const cudaError_t ee = enqueue_two_sweeps(cs, cv, ev_q, ev_v);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (ee != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      return ee;
    }
    if (ce != cudaSuccess) return ce;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) return ie;
    std::lock_guard<std::mutex> lock(mu);
    if (cache.size() >= 512) {  // bound the cache: drop everything (graphs are cheap to rebuild)
      for (auto& kv : cache) cudaGraphExecDestroy(kv.second);
      cache.clear();
    }
    cache[key] = exec;
  }
  const int per_graph = 2 * (3 * (nb - 1) + 2);  // kernels in one replay
  for (int g = 0; g < (max_sweeps + 1) / 2; ++g) {
    for (int k = 0; k < per_graph; ++k) note_launch();
    TT_CUDA(cudaGraphLaunch(exec, st));
  }
  note_launch();
  bj_finish<T><<<s, kFinishThreads, 0, st>>>(A0, A1, V, sp, s, w, Vout, flags);
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
