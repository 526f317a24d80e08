// Rotation helpers of the cyclic two-sided Jacobi method (Golub & Van Loan, Sec. 8.5) with the
// round-robin ("circle") ordering, arranged for one barrier per round: each thread forms whole 2x2
// blocks R_i B R_j^T of a round from the matrix before it, and the angles of the next round are
// re-formed from the same inputs by the same functions (so they agree with what is written).
// Used by the one-CTA solver (eig.cu).
#pragma once

#include <cfloat>

namespace ttice {
namespace jrot {

template <typename T> struct Eps;
template <> struct Eps<float> { static __device__ __forceinline__ float value() { return FLT_EPSILON; } };
template <> struct Eps<double> { static __device__ __forceinline__ double value() { return DBL_EPSILON; } };

template <typename T>
__device__ __forceinline__ void rr_pair(int k, int r, int m, int& p, int& q) {
  // (r + k) mod m and (r - k) mod m for 0 <= r, k < m, without an integer division
  if (k == 0) { p = r; q = m; }
  else {
    p = r + k; if (p >= m) p -= m;
    q = r - k; if (q < 0) q += m;
  }
  if (p > q) { const int t = p; p = q; q = t; }
}

// pair index of player x in round r (inverse of rr_pair); m = players - 1
__device__ __forceinline__ int rr_pair_of(int x, int r, int m) {
  if (x == m || x == r) return 0;
  int k = x - r;
  if (k < 0) k += m;
  return (2 * k <= m) ? k : m - k;
}

// The rotation that zeroes a_pq: t = sgn(tau) / (|tau| + sqrt(1 + tau^2)) with
// tau = (a_qq - a_pp) / (2 a_pq), evaluated as sgn(tau) |2 a_pq| / (|a_qq - a_pp| + hypot(.)) (the
// same value multiplied through by |2 a_pq|: one hypot, one division and one reciprocal square root
// instead of three square roots and three divisions, which matters for FP64 at 1/64 rate).
template <typename T>
__device__ __forceinline__ void make_rotation(T app, T aqq, T apq, T floor_abs, T& c, T& sn, T& t) {
  c = T(1); sn = T(0); t = T(0);
  if (fabs(apq) > floor_abs && fabs(apq) > Eps<T>::value() * sqrt(fabs(app * aqq))) {
    const T th = aqq - app, ph = T(2) * apq;
    const bool pos = (th == T(0)) || ((th > T(0)) == (ph > T(0)));  // tau >= 0
    const T mag = fabs(ph) / (fabs(th) + hypot(th, ph));
    t = pos ? mag : -mag;
    c = rsqrt(T(1) + t * t);
    sn = t * c;
  }
}

// new diagonal entries of a rotated pair: a_pp - t a_pq and a_qq + t a_pq (a_pq becomes 0)
template <typename T>
__device__ __forceinline__ T diag_after(T a, T t, T apq, bool is_p) {
  return is_p ? fma(-t, apq, a) : fma(t, apq, a);
}

// R_i B R_j^T of one 2x2 block, R = [[c, -s], [s, c]]; entries of rows/columns that are the dummy
// player are zero in B and never read from the result
template <typename T>
__device__ __forceinline__ void block_after(const T* A, int lda, int s, int pi, int qi, int pj, int qj,
                                            T ci, T si, T cj, T sj, T o[4]) {
  const bool ri = qi < s, rj = qj < s;
  const T b00 = A[pi * lda + pj];
  const T b01 = rj ? A[pi * lda + qj] : T(0);
  const T b10 = ri ? A[qi * lda + pj] : T(0);
  const T b11 = (ri && rj) ? A[qi * lda + qj] : T(0);
  const T m00 = fma(ci, b00, -(si * b10)), m01 = fma(ci, b01, -(si * b11));
  const T m10 = fma(si, b00, ci * b10), m11 = fma(si, b01, ci * b11);
  o[0] = fma(cj, m00, -(sj * m01));
  o[1] = fma(sj, m00, cj * m01);
  o[2] = fma(cj, m10, -(sj * m11));
  o[3] = fma(sj, m10, cj * m11);
}


}  // namespace jrot
}  // namespace ttice
