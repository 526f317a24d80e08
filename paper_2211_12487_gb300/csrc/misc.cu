// Small device kernels of the update: the decision of Algorithm 2 (skip test, subselection, relaxed
// tolerance, per-core threshold), norms, gathers, sign canonicalisation and core / last-core appends.
#include <algorithm>
#include <cmath>

#include "ttice_internal.cuh"

namespace ttice {

std::atomic<long long> g_kernel_launches{0};

namespace {

constexpr int kThreads = 256;
constexpr unsigned kSignSlices = 64;  // row slices per column of the canonical-sign search

inline unsigned grid_for(int64_t n, int per = kThreads) {
  int64_t g = (n + per - 1) / per;
  if (g > 152 * 32) g = 152 * 32;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// Algorithm 2: per-observation relative errors (Eq. 17), skip test (Eq. 20 or the mean surrogate),
// subselection D = {j : eps_Y(j) > eps}, eps_upd (Eq. 18 or 19), eps = eps_upd ||D|| / sqrt(d).
// One thread: b is small and the order of the FP64 sums is fixed (ascending j).  rho2 holds the
// squared residual of every observation per TT stage (stage-major, nst x b); rho2(j) is their sum,
// taken in ascending stage order (the orthogonal decomposition of ||y_j - ~y_j||^2).
__global__ void decision_kernel(const double* rho2s, int nst, const double* y2, int b, double eps,
                                int d, int skip_mode, int subselect, int eps_upd_mode, Decision* dec,
                                int* sel) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  auto rho2 = [&](int j) {
    double v = 0.0;
    for (int i = 0; i < nst; ++i) v += rho2s[(int64_t)i * b + j];
    return v;
  };
  Decision D;
  double ynorm2 = 0.0, rsum = 0.0, relsum = 0.0;
  int nonfinite = 0;
  for (int j = 0; j < b; ++j) {
    ynorm2 += y2[j];
    const double rj = rho2(j);
    rsum += rj;
    const double rel = y2[j] > 0.0 ? sqrt(rj / y2[j]) : 0.0;
    relsum += rel;
    if (!isfinite(y2[j]) || !isfinite(rj)) nonfinite = 1;
  }
  D.nonfinite = nonfinite;
  D.ynorm2 = ynorm2;
  D.batch_err = ynorm2 > 0.0 ? sqrt(rsum / ynorm2) : 0.0;
  int skip = 0;
  if (skip_mode == TTICE_SKIP_EXACT) skip = D.batch_err <= eps;
  else if (skip_mode == TTICE_SKIP_MEAN) skip = (relsum / b) <= eps;
  D.skip = skip;
  D.nsel = 0;
  D.dnorm2 = 0.0;
  D.eps_upd = NAN;
  D.eps_c = NAN;
  if (!skip) {
    double rest_rho2 = 0.0, rest_rel = 0.0;
    int nsel = 0;
    for (int j = 0; j < b; ++j) {
      const double rj = rho2(j);
      const double rel = y2[j] > 0.0 ? sqrt(rj / y2[j]) : 0.0;
      if (!subselect || rel > eps) {
        sel[nsel++] = j;
        D.dnorm2 += y2[j];
      } else {
        rest_rho2 += rj;
        rest_rel += rel;
      }
    }
    D.nsel = nsel;
    if (nsel > 0) {
      double eps_upd;
      if (nsel == b) eps_upd = eps;
      else if (eps_upd_mode == TTICE_EPSUPD_EXACT) {
        const double t = eps * sqrt(ynorm2);
        const double num = t * t - rest_rho2;
        eps_upd = sqrt(fmax(num, 0.0) / D.dnorm2);
      } else {
        eps_upd = fmax((eps * b - rest_rel) / nsel, 0.0);
      }
      D.eps_upd = eps_upd;
      D.eps_c = eps_upd * sqrt(D.dnorm2) / sqrt((double)d);
    }
  }
  *dec = D;
}

// Pseudo-random start vectors in [-1, 1): splitmix64 of (seed, index).
__global__ void fill_random_kernel(float* p, int64_t n, uint64_t seed) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    p[i] = (float)((double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
  }
}

__global__ void fill_kernel(double* p, int64_t n, double v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

template <typename TI, typename TO>
__global__ void cast_kernel(const TI* in, TO* out, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}

template <typename T>
__global__ void gather_obs_kernel(const T* Y, T* out, const int* sel, int nsel, int64_t N) {
  const int j = blockIdx.y;
  const T* src = Y + (int64_t)sel[j] * N;
  T* dst = out + (int64_t)j * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = src[i];
}

template <typename T>
__global__ void expand_stage_kernel(const T* src, const int* sel, int64_t r0, const T* add, int64_t k, int64_t L,
                                    T* out) {
  const int z = blockIdx.y;
  const int64_t no = r0 * L, nn = (r0 + k) * L;
  const T* s = src + (int64_t)(sel ? sel[z] : z) * no;
  const T* a = add + (int64_t)z * k * L;
  T* d = out + (int64_t)z * nn;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nn; e += (int64_t)gridDim.x * blockDim.x)
    d[e] = e < no ? s[e] : a[e - no];
}

template <typename T>
__global__ void sum_squares_kernel(const T* x, int64_t N, double* out) {
  const int j = blockIdx.y;
  const T* p = x + (int64_t)j * N;
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = (double)p[i];
    s = fma(v, v, s);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    atomicAdd(out + j, t);
  }
}

__global__ void trace_kernel(const double* G, int64_t ldg, int s, double* out) {
  double t = 0.0;
  for (int i = threadIdx.x; i < s; i += blockDim.x) t += G[i * ldg + i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) a += red[w];
    *out = a;
  }
}

// one CTA per column: index of the largest |v| (lowest index on ties), flip the column if negative
// Canonical sign, step 1: per column c and row slice blockIdx.x, the largest |V| and its lowest index
// into part[(c nb + slice) 2 + {0, 1}].
__global__ void sign_partial_kernel(const double* V, int64_t m, int64_t ld, double* part) {
  const int c = blockIdx.y, nb = gridDim.x;
  const double* v = V + (int64_t)c * ld;
  double best = -1.0;
  int64_t bi = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m; i += (int64_t)nb * blockDim.x) {
    const double a = fabs(v[i]);
    if (a > best) { best = a; bi = i; }
  }
  __shared__ double sb[kThreads];
  __shared__ int64_t si[kThreads];
  sb[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const double b2 = sb[threadIdx.x + o];
      const int64_t i2 = si[threadIdx.x + o];
      if (b2 > sb[threadIdx.x] || (b2 == sb[threadIdx.x] && i2 < si[threadIdx.x])) {
        sb[threadIdx.x] = b2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[((int64_t)c * nb + blockIdx.x) * 2] = sb[0];
    part[((int64_t)c * nb + blockIdx.x) * 2 + 1] = (double)si[0];
  }
}

// Step 2: sign[c] = -1 if the column's largest-|.| entry (lowest index on ties) is negative, else 1.
__global__ void sign_finish_kernel(const double* V, int64_t ld, const double* part, int nb, double* sign) {
  const int c = blockIdx.x;
  if (threadIdx.x != 0) return;
  double best = -1.0, bi = 0.0;
  for (int j = 0; j < nb; ++j) {
    const double b2 = part[((int64_t)c * nb + j) * 2], i2 = part[((int64_t)c * nb + j) * 2 + 1];
    if (b2 > best || (b2 == best && i2 < bi)) { best = b2; bi = i2; }
  }
  sign[c] = (best >= 0.0 && V[(int64_t)c * ld + (int64_t)bi] < 0.0) ? -1.0 : 1.0;
}

__global__ void scale_cols_rsqrt_kernel(double* V, int64_t m, int64_t ld, const double* theta) {
  const int c = blockIdx.y;
  const double s = 1.0 / sqrt(theta[c]);
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x)
    V[c * ld + i] *= s;
}

__global__ void copy_cols_kernel(const double* in, int64_t ld_in, int64_t m, double* out,
                                 int64_t ld_out, float* mirror, const double* sign) {
  const int c = blockIdx.y;
  const double sg = sign ? sign[c] : 1.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < m;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = sg * in[c * ld_in + i];
    out[c * ld_out + i] = v;
    if (mirror) mirror[c * ld_out + i] = (float)v;
  }
}

template <typename TC>
__global__ void append_last_kernel(const TC* coef, int b, int r, double* last, int64_t n0,
                                   int64_t ld) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < b * r; e += gridDim.x * blockDim.x) {
    const int j = e / r, a = e % r;
    last[(n0 + j) * ld + a] = (double)coef[e];
  }
}

__global__ void col_norms_kernel(const double* V, int64_t m, int64_t ld, double* out) {
  const double* v = V + (int64_t)blockIdx.x * ld;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) s = fma(v[i], v[i], s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ double red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    out[blockIdx.x] = t;
  }
}

// Deterministic pseudo-random numbers in [-1, 1) (splitmix64 of seed + index): start blocks of the
// Krylov eigen-solver; the solver's result does not depend on them once converged.
// res[j] = || GQ[:, j] - theta[j] Q[:, j] ||  (Ritz residual norms), one CTA per column.
__global__ void ritz_residual_kernel(const double* GQ, const double* Q, const double* theta,
                                     int64_t s, double* res) {
  const int j = blockIdx.x;
  const double th = theta[j];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < s; i += blockDim.x) {
    const double e = GQ[(int64_t)j * s + i] - th * Q[(int64_t)j * s + i];
    a = fma(e, e, a);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  __shared__ double red[kThreads / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = a;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    res[j] = sqrt(t);
  }
}

__global__ void rel_err_kernel(const double* rho2s, int nst, const double* y2, int b, double* rel) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= b) return;
  double r = 0.0;
  for (int i = 0; i < nst; ++i) r += rho2s[(int64_t)i * b + j];
  rel[j] = y2[j] > 0.0 ? sqrt(r / y2[j]) : 0.0;
}

}  // namespace

cudaError_t launch_decision(const double* rho2s, int nst, const double* y2, int b, double eps, int d,
                            int skip_mode, int subselect, int eps_upd_mode, Decision* dec,
                            int* sel, cudaStream_t st) {
  note_launch();
  decision_kernel<<<1, 32, 0, st>>>(rho2s, nst, y2, b, eps, d, skip_mode, subselect, eps_upd_mode,
                                    dec, sel);
  return cudaGetLastError();
}

cudaError_t launch_fill_random(float* p, int64_t n, uint64_t seed, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  note_launch();
  fill_random_kernel<<<grid_for(n), kThreads, 0, st>>>(p, n, seed);
  return cudaGetLastError();
}

cudaError_t launch_fill(double* p, int64_t n, double v, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  note_launch();
  fill_kernel<<<grid_for(n), kThreads, 0, st>>>(p, n, v);
  return cudaGetLastError();
}

template <typename TI, typename TO>
cudaError_t launch_cast(const TI* in, TO* out, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  note_launch();
  cast_kernel<TI, TO><<<grid_for(n), kThreads, 0, st>>>(in, out, n);
  return cudaGetLastError();
}
template cudaError_t launch_cast<double, float>(const double*, float*, int64_t, cudaStream_t);
template cudaError_t launch_cast<float, double>(const float*, double*, int64_t, cudaStream_t);
template cudaError_t launch_cast<double, double>(const double*, double*, int64_t, cudaStream_t);
template cudaError_t launch_cast<float, float>(const float*, float*, int64_t, cudaStream_t);

template <typename T>
cudaError_t launch_gather_obs(const T* Y, T* out, const int* sel, int nsel, int64_t N,
                              cudaStream_t st) {
  if (nsel <= 0 || N <= 0) return cudaSuccess;
  dim3 grid(std::min<unsigned>(grid_for(N), 1024u), (unsigned)nsel);
  note_launch();
  gather_obs_kernel<T><<<grid, kThreads, 0, st>>>(Y, out, sel, nsel, N);
  return cudaGetLastError();
}
template cudaError_t launch_gather_obs<float>(const float*, float*, const int*, int, int64_t,
                                              cudaStream_t);
template cudaError_t launch_gather_obs<double>(const double*, double*, const int*, int, int64_t,
                                               cudaStream_t);

template <typename T>
cudaError_t launch_expand_stage(const T* src, const int* sel, int64_t r0, const T* add, int64_t k, int64_t L,
                                int nobs, T* out, cudaStream_t st) {
  const int64_t nn = (r0 + k) * L;
  if (nobs <= 0 || nn <= 0) return cudaSuccess;
  dim3 grid(std::min<unsigned>(grid_for(nn), 1024u), (unsigned)nobs);
  note_launch();
  expand_stage_kernel<T><<<grid, kThreads, 0, st>>>(src, sel, r0, add, k, L, out);
  return cudaGetLastError();
}
template cudaError_t launch_expand_stage<float>(const float*, const int*, int64_t, const float*, int64_t, int64_t,
                                                int, float*, cudaStream_t);
template cudaError_t launch_expand_stage<double>(const double*, const int*, int64_t, const double*, int64_t,
                                                 int64_t, int, double*, cudaStream_t);

template <typename T>
cudaError_t launch_sum_squares(const T* x, int b, int64_t N, double* out, cudaStream_t st) {
  if (b <= 0 || N <= 0) return cudaSuccess;
  dim3 grid(std::min<unsigned>(grid_for(N), 256u), (unsigned)b);
  note_launch();
  sum_squares_kernel<T><<<grid, kThreads, 0, st>>>(x, N, out);
  return cudaGetLastError();
}
template cudaError_t launch_sum_squares<float>(const float*, int, int64_t, double*, cudaStream_t);
template cudaError_t launch_sum_squares<double>(const double*, int, int64_t, double*, cudaStream_t);

cudaError_t launch_trace(const double* G, int64_t ldg, int s, double* out, cudaStream_t st) {
  note_launch();
  trace_kernel<<<1, 1024, 0, st>>>(G, ldg, s, out);
  return cudaGetLastError();
}

cudaError_t launch_canonical_sign(const double* V, int64_t m, int k, int64_t ld, double* part, double* sign,
                                  cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  const unsigned nb = std::max<unsigned>(1u, std::min<unsigned>(grid_for(m), kSignSlices));
  note_launch();
  sign_partial_kernel<<<dim3(nb, (unsigned)k), kThreads, 0, st>>>(V, m, ld, part);
  TT_CUDA(cudaGetLastError());
  note_launch();
  sign_finish_kernel<<<k, 32, 0, st>>>(V, ld, part, (int)nb, sign);
  return cudaGetLastError();
}

cudaError_t launch_scale_cols_rsqrt(double* V, int64_t m, int k, int64_t ld, const double* theta,
                                    cudaStream_t st) {
  if (k <= 0 || m <= 0) return cudaSuccess;
  dim3 grid(std::min<unsigned>(grid_for(m), 64u), (unsigned)k);
  note_launch();
  scale_cols_rsqrt_kernel<<<grid, kThreads, 0, st>>>(V, m, ld, theta);
  return cudaGetLastError();
}

cudaError_t launch_copy_cols(const double* in, int64_t ld_in, int64_t m, int k, double* out,
                             int64_t ld_out, float* mirror, cudaStream_t st, const double* sign) {
  if (k <= 0 || m <= 0) return cudaSuccess;
  dim3 grid(std::min<unsigned>(grid_for(m), 64u), (unsigned)k);
  note_launch();
  copy_cols_kernel<<<grid, kThreads, 0, st>>>(in, ld_in, m, out, ld_out, mirror, sign);
  return cudaGetLastError();
}

template <typename TC>
cudaError_t launch_append_last_t(const TC* coef, int b, int r, double* last, int64_t n0, int64_t ld,
                                 cudaStream_t st) {
  if (b <= 0 || r <= 0) return cudaSuccess;
  note_launch();
  append_last_kernel<TC><<<grid_for((int64_t)b * r), kThreads, 0, st>>>(coef, b, r, last, n0, ld);
  return cudaGetLastError();
}
template cudaError_t launch_append_last_t<float>(const float*, int, int, double*, int64_t, int64_t,
                                                 cudaStream_t);
template cudaError_t launch_append_last_t<double>(const double*, int, int, double*, int64_t,
                                                  int64_t, cudaStream_t);

cudaError_t launch_append_last(const double* coef, int b, int r, double* last, int64_t n0,
                               int64_t ld, cudaStream_t st) {
  return launch_append_last_t<double>(coef, b, r, last, n0, ld, st);
}

cudaError_t launch_col_norms(const double* V, int64_t m, int k, int64_t ld, double* out,
                             cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  note_launch();
  col_norms_kernel<<<k, kThreads, 0, st>>>(V, m, ld, out);
  return cudaGetLastError();
}

cudaError_t launch_ritz_residual(const double* GQ, const double* Q, const double* theta, int64_t s,
                                 int k, double* res, cudaStream_t st) {
  if (k <= 0) return cudaSuccess;
  note_launch();
  ritz_residual_kernel<<<k, kThreads, 0, st>>>(GQ, Q, theta, s, res);
  return cudaGetLastError();
}

cudaError_t launch_rel_err(const double* rho2s, int nst, const double* y2, int b, double* rel,
                           cudaStream_t st) {
  if (b <= 0) return cudaSuccess;
  note_launch();
  rel_err_kernel<<<(b + 127) / 128, 128, 0, st>>>(rho2s, nst, y2, b, rel);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_to_f64(const T* in, int64_t n, double* out, cudaStream_t st) {
  return launch_cast<T, double>(in, out, n, st);
}
template cudaError_t launch_to_f64<float>(const float*, int64_t, double*, cudaStream_t);
template cudaError_t launch_to_f64<double>(const double*, int64_t, double*, cudaStream_t);

}  // namespace ttice
