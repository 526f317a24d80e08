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

#include "jacobi_rot.cuh"
#include "ttice_internal.cuh"

namespace ttice {
namespace {

using jrot::block_after;
using jrot::diag_after;
using jrot::make_rotation;
using jrot::rr_pair;
using jrot::rr_pair_of;

template <typename T> struct Lim;
template <> struct Lim<float> { static __device__ float eps() { return FLT_EPSILON; } };
template <> struct Lim<double> { static __device__ double eps() { return DBL_EPSILON; } };

// sweep caps: quadratic convergence reaches the working precision in well under these; what
// remains beyond them is rotation of rounding noise
template <typename T> struct SweepCap;
template <> struct SweepCap<float> { static constexpr int value = 14; };
template <> struct SweepCap<double> { static constexpr int value = 30; };
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
  const double off_gate = 64.0 * sqrt((double)s) * (double)Lim<T>::eps() * red[0];
  __syncthreads();

  const int np = (s + 1) & ~1;  // players, with a dummy when s is odd
  const int npairs = np / 2;
  const T teps = Lim<T>::eps();
  int sweep = 0;
  for (; sweep < SweepCap<T>::value; ++sweep) {
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
    // off-diagonal norm after this sweep.  Early sweeps may shrink it by as little as ~0.6; once it
    // is down at the rounding level (below off_gate) a sweep that does not halve it is rotating
    // rounding noise -- stop there
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
      stall = (sweep > 0 && t > 0.25 * prev_off && t <= off_gate * off_gate) ? 1 : 0;
      prev_off = t;
    }
    __syncthreads();
    if (stall) break;
  }
  if (tid == 0 && status) *status = (sweep >= SweepCap<T>::value) ? 1 : 0;
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

// ---- small problems (s <= 128): everything in shared memory, one barrier per round ----
//
// The same cyclic Jacobi method and round-robin ordering as above, arranged so that a round needs a
// single barrier.  Each thread owns one 2x2 block (pair i rows, pair j columns) of the round: it
// forms R_i B R_j^T from the matrix before the round (A_in) into a second buffer (A_out), writing the
// mirrored block too, and applies rotation i to the V entries of rows {p_j, q_j}, which no other
// thread touches in that round.  The rotations of the next round are computed in the same phase by
// re-forming, from A_in, the three entries of each next pair that this round produces (with the same
// helper functions, so they agree with what is written), which removes the barrier between the
// angle computation and the update.
constexpr int kSmallEigMax = 128;

template <typename T>
__global__ void __launch_bounds__(kEigThreads) jacobi_small_kernel(const double* G, int64_t ldg, int s,
                                                                   T* w, T* Vout, int* status) {
  constexpr int NP = kSmallEigMax / 2;   // most pairs of a round
  constexpr int NA = NP * (NP + 1) / 2;  // most 2x2 blocks with i <= j
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T rc[2][NP], rs[2][NP], rt[2][NP];  // rotation of each pair: c, s, t = s / c
  __shared__ int rpq[2][NP];                     // the pair itself: p | q << 16
  __shared__ unsigned short ij_tab[NA];          // i << 8 | j of the blocks a thread owns
  __shared__ double red[33];
  __shared__ int rotated, stop;
  __shared__ double prev_off;
  const int lda = s + 1;
  T* Ain = reinterpret_cast<T*>(smem_raw);
  T* Aout = Ain + (int64_t)s * lda;
  T* V = Aout + (int64_t)s * lda;  // s x s column-major, ld s
  const int tid = threadIdx.x, nt = blockDim.x;

  double fro = 0.0;
  for (int e = tid; e < s * s; e += nt) {
    const int i = e / s, j = e - i * s;
    const double g = G[i * ldg + j];
    fro += g * g;
    Ain[i * lda + j] = (T)g;
    V[j * s + i] = (i == j) ? T(1) : T(0);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(0xffffffffu, fro, o);
  if ((tid & 31) == 0) red[tid >> 5] = fro;
  const int np = (s + 1) & ~1;
  const int m = np - 1;
  const int npairs = np / 2;
  const int nA = npairs * (npairs + 1) / 2;
  for (int t = tid; t < nA; t += nt) {
    int i = 0, off = 0;
    while (off + (npairs - i) <= t) { off += npairs - i; ++i; }
    ij_tab[t] = (unsigned short)((i << 8) | (i + (t - off)));
  }
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < nt / 32; ++q) t += red[q];
    red[32] = sqrt(t);
    rotated = 0;
    stop = 0;
  }
  __syncthreads();
  const T floor_abs = (T)((double)Lim<T>::eps() * red[32]);
  const double off_gate = 64.0 * sqrt((double)s) * (double)Lim<T>::eps() * red[32];
  int cur = 0;
  for (int k = tid; k < npairs; k += nt) {
    int p, q;
    rr_pair<T>(k, 0, m, p, q);
    T c = T(1), sn = T(0), t = T(0);
    if (q < s) make_rotation(Ain[p * lda + p], Ain[q * lda + q], Ain[p * lda + q], floor_abs, c, sn, t);
    rc[0][k] = c; rs[0][k] = sn; rt[0][k] = t;
    rpq[0][k] = p | (q << 16);
  }
  __syncthreads();
  // The last warp computes the next round's angles while the others update A and V, so a round's
  // critical path is the longer of the two, not their sum.  V items: (pair i, row x), rows fastest
  // so that a warp touches consecutive words.
  const int nwork = nt - 32;
  const bool angle_warp = tid >= nwork;
  const int vi0 = angle_warp ? npairs : tid / s, vx0 = angle_warp ? 0 : tid - (tid / s) * s;
  const int vdi = nwork / s, vdx = nwork - vdi * s;

  int sweep = 0;
  for (; sweep < SweepCap<T>::value; ++sweep) {
    for (int round = 0; round < m; ++round) {
      // A <- J^T A J, one 2x2 block (and its mirror) per item, from Ain into Aout
      for (int t = angle_warp ? nA : tid; t < nA; t += nwork) {
        const int ij = ij_tab[t];
        const int i = ij >> 8, j = ij & 255;
        const int pqi = rpq[cur][i];
        const int pi = pqi & 0xffff, qi = pqi >> 16;
        const T si = rs[cur][i];
        if (i == j) {
          if (qi < s) {
            const T app = Ain[pi * lda + pi], aqq = Ain[qi * lda + qi], apq = Ain[pi * lda + qi];
            if (si != T(0)) {
              const T tt = rt[cur][i];
              Aout[pi * lda + pi] = diag_after(app, tt, apq, true);
              Aout[qi * lda + qi] = diag_after(aqq, tt, apq, false);
              Aout[pi * lda + qi] = T(0);
              Aout[qi * lda + pi] = T(0);
              rotated = 1;
            } else {
              Aout[pi * lda + pi] = app;
              Aout[qi * lda + qi] = aqq;
              Aout[pi * lda + qi] = apq;
              Aout[qi * lda + pi] = apq;
            }
          } else {
            Aout[pi * lda + pi] = Ain[pi * lda + pi];
          }
        } else {
          const int pqj = rpq[cur][j];
          const int pj = pqj & 0xffff, qj = pqj >> 16;
          T o[4];
          block_after(Ain, lda, s, pi, qi, pj, qj, rc[cur][i], si, rc[cur][j], rs[cur][j], o);
          Aout[pi * lda + pj] = o[0];
          Aout[pj * lda + pi] = o[0];
          if (qj < s) { Aout[pi * lda + qj] = o[1]; Aout[qj * lda + pi] = o[1]; }
          if (qi < s) { Aout[qi * lda + pj] = o[2]; Aout[pj * lda + qi] = o[2]; }
          if (qi < s && qj < s) { Aout[qi * lda + qj] = o[3]; Aout[qj * lda + qi] = o[3]; }
        }
      }
      // V <- V J, in place: item (i, x) owns V[x, p_i] and V[x, q_i]
      for (int i = vi0, x = vx0; i < npairs;) {
        const T si = rs[cur][i];
        if (si != T(0)) {  // a rotation implies q_i < s
          const int pqi = rpq[cur][i];
          const int pi = pqi & 0xffff, qi = pqi >> 16;
          const T ci = rc[cur][i];
          const T vp = V[pi * s + x], vq = V[qi * s + x];
          V[pi * s + x] = fma(ci, vp, -(si * vq));
          V[qi * s + x] = fma(si, vp, ci * vq);
        }
        x += vdx;
        i += vdi;
        if (x >= s) { x -= s; ++i; }
      }
      // pairs and angles of the next round, from the entries this round produces
      const int rn = (round + 1 == m) ? 0 : round + 1;
      for (int k = angle_warp ? tid - nwork : npairs; k < npairs; k += 32) {
        int p, q;
        rr_pair<T>(k, rn, m, p, q);
        T c = T(1), sn = T(0), t = T(0);
        if (q < s) {
          const int a = rr_pair_of(p, round, m), b = rr_pair_of(q, round, m);
          const int pqa = rpq[cur][a], pqb = rpq[cur][b];
          const int pa = pqa & 0xffff, qa = pqa >> 16, pb = pqb & 0xffff, qb = pqb >> 16;
          T app = Ain[p * lda + p], aqq = Ain[q * lda + q];
          if (rs[cur][a] != T(0)) app = diag_after(app, rt[cur][a], Ain[pa * lda + qa], p == pa);
          if (rs[cur][b] != T(0)) aqq = diag_after(aqq, rt[cur][b], Ain[pb * lda + qb], q == pb);
          T apq;
          if (a == b) {  // only when s <= 2: the same pair again
            apq = (rs[cur][a] != T(0)) ? T(0) : Ain[p * lda + q];
          } else {
            const bool alo = a < b;
            const int lo = alo ? a : b, hi = alo ? b : a;
            const int pl = alo ? pa : pb, ql = alo ? qa : qb, ph = alo ? pb : pa, qh = alo ? qb : qa;
            T o[4];
            block_after(Ain, lda, s, pl, ql, ph, qh, rc[cur][lo], rs[cur][lo], rc[cur][hi], rs[cur][hi], o);
            const int xl = alo ? p : q, xh = alo ? q : p;  // entry (xl, xh) of the block
            apq = (xl == pl) ? ((xh == ph) ? o[0] : o[1]) : ((xh == ph) ? o[2] : o[3]);
          }
          make_rotation(app, aqq, apq, floor_abs, c, sn, t);
        }
        rc[cur ^ 1][k] = c; rs[cur ^ 1][k] = sn; rt[cur ^ 1][k] = t;
        rpq[cur ^ 1][k] = p | (q << 16);
      }
      __syncthreads();
      cur ^= 1;
      T* tmp = Ain; Ain = Aout; Aout = tmp;
    }
    // stop when a sweep rotated nothing, or when the off-diagonal norm is at the rounding level
    // (below off_gate) and the sweep did not halve it: what is left is rounding noise
    double off = 0.0;
    for (int e = tid; e < s * s; e += nt) {
      const int i = e / s, j = e - i * s;
      if (i != j) { const double a = (double)Ain[i * lda + j]; off += a * a; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) off += __shfl_xor_sync(0xffffffffu, off, o);
    if ((tid & 31) == 0) red[tid >> 5] = off;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int q = 0; q < nt / 32; ++q) t += red[q];
      stop = (rotated == 0) || (sweep > 0 && t > 0.25 * prev_off && t <= off_gate * off_gate);
      prev_off = t;
      rotated = 0;
    }
    __syncthreads();
    if (stop) break;
  }
  if (tid == 0 && status) *status = (sweep >= SweepCap<T>::value) ? 1 : 0;
  for (int i = tid; i < s; i += nt) {
    const T di = Ain[i * lda + i];
    int rank = 0;
    for (int j = 0; j < s; ++j) {
      const T dj = Ain[j * lda + j];
      rank += (dj > di) || (dj == di && j < i);
    }
    w[rank] = di;
    for (int r = 0; r < s; ++r) Vout[(int64_t)rank * s + r] = V[i * s + r];
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
__global__ void chol_inv_kernel(const double* S, int k, const double* diag, double* Rinv, int* status,
                                const int* run_if) {
  if (run_if && *run_if == 0) return;
  extern __shared__ double sm[];
  double* R = sm;          // k x k, column-major
  double* Ri = sm + k * k; // k x k
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < k * k; e += nt) {
    R[e] = (diag && e % (k + 1) == 0) ? diag[e / (k + 1)] : S[e];
    Ri[e] = 0.0;
  }
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
  // invert the upper triangular R column by column (each thread one column of Ri), multiplying by
  // the reciprocal diagonal (k FP64 divisions in parallel instead of k^2/2 on the critical path)
  __shared__ double dinv[112];
  for (int i = tid; i < k; i += nt) dinv[i] = 1.0 / R[i + i * k];
  __syncthreads();
  for (int c = tid; c < k; c += nt) {
    for (int i = c; i >= 0; --i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int l = i + 1; l <= c; ++l) v = fma(-R[i + l * k], Ri[l + c * k], v);
      Ri[i + c * k] = v * dinv[i];
    }
  }
  __syncthreads();
  for (int e = tid; e < k * k; e += nt) {
    const int i = e % k, c = e / k;
    Rinv[e] = (i <= c) ? Ri[e] : 0.0;
  }
  if (tid == 0 && status && bad) *status = 1;  // sticky: a caller may check several factorisations at once
}

}  // namespace


template <typename T>
cudaError_t jacobi_eig(const double* G, int64_t ldg, int s, T* w, T* V, T* work, int* status,
                       cudaStream_t st) {
  if (s <= 0) return cudaSuccess;
  if (s > 1024) return cudaErrorInvalidValue;
  const size_t small_need = (2 * (size_t)s * (s + 1) + (size_t)s * s) * sizeof(T);
  if (s <= kSmallEigMax && small_need <= kEigSmemMax) {
    static std::once_flag once_small;
    static cudaError_t small_err = cudaSuccess;
    std::call_once(once_small, [] {
      small_err = cudaFuncSetAttribute(jacobi_small_kernel<T>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEigSmemMax);
    });
    TT_CUDA(small_err);
    const int npairs = (s + 1) / 2;
    const int threads = std::min(kEigThreads, std::max(64, (npairs * npairs + 31) / 32 * 32));
    note_launch();
    jacobi_small_kernel<T><<<1, threads, small_need, st>>>(G, ldg, s, w, V, status);
    return cudaGetLastError();
  }
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

cudaError_t launch_chol_inv(const double* S, int k, double* Rinv, int* status, cudaStream_t st,
                            const double* diag, const int* run_if) {
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
  chol_inv_kernel<<<1, 256, smem, st>>>(S, k, diag, Rinv, status, run_if);
  return cudaGetLastError();
}

}  // namespace ttice
