// K1: the first pass over an increment, stage 1 (Eq. 6 and Eq. 17 of Algorithm 2), fused.
//
// For every observation z and every column l of its n_1 x L_1 unfolding Y_1(z) (L_1 = n_2 ... n_d):
//   w = U_1^T y            (r_1 coefficients, written to W(z) in the stage layout a*L_1 + l),
//   e = y - U_1 w           (direct residual, never formed in memory),
//   ||y||^2 and ||e||^2      accumulated per observation in FP64.
// This is the only pass that reads the whole increment from HBM, so it is written as a streaming
// kernel: one column per thread, the n_1 loads of a column coalesced across the warp (consecutive
// threads read consecutive l), U_1 held in shared memory in both orders so that the projection and
// the back-projection read it with 16-byte broadcast loads, per-thread FP64 partial norms reduced by
// warp shuffles and written as one partial per CTA, summed per observation in a fixed order.  The grid is a multiple of the SM count (persistent,
// grid-stride over columns).  Precision T is the arithmetic of the projection (FP32 on the mixed
// paths, FP64 on the FP64 path); the norms are always accumulated in FP64.
#include <algorithm>

#include "ttice_internal.cuh"

namespace ttice {
namespace {

constexpr int kK1Threads = 256;

template <typename TY, typename T, int N1, int RM>
__global__ void __launch_bounds__(kK1Threads) k1_kernel(const TY* __restrict__ Y, int64_t L, int n1,
                                                        int r, const T* __restrict__ U, int64_t ldu,
                                                        T* __restrict__ W, double* part,
                                                        int64_t blocks_per_obs) {
  // Ua[a][k] = U(k, a) (k fastest) for the projection, Uk[k][a] for the back-projection.
  __shared__ __align__(16) T Ua[RM][N1];
  __shared__ __align__(16) T Uk[N1][RM];
  for (int e = threadIdx.x; e < RM * N1; e += blockDim.x) {
    const int a = e / N1, k = e % N1;
    const T v = (a < r && k < n1) ? U[(int64_t)a * ldu + k] : T(0);
    Ua[a][k] = v;
    Uk[k][a] = v;
  }
  __syncthreads();
  const int z = blockIdx.y;
  const TY* Yz = Y + (int64_t)z * n1 * L;
  T* Wz = W + (int64_t)z * r * L;
  double sy = 0.0, se = 0.0;
  for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < L;
       l += blocks_per_obs * blockDim.x) {
    T y[N1];
#pragma unroll
    for (int k = 0; k < N1; ++k) y[k] = (k < n1) ? (T)__ldcs(Yz + (int64_t)k * L + l) : T(0);
    T w[RM];
#pragma unroll
    for (int a = 0; a < RM; ++a) {
      T acc = T(0);
#pragma unroll
      for (int k = 0; k < N1; ++k) acc = fma(Ua[a][k], y[k], acc);
      w[a] = acc;
    }
#pragma unroll
    for (int a = 0; a < RM; ++a)
      if (a < r) Wz[(int64_t)a * L + l] = w[a];
#pragma unroll
    for (int k = 0; k < N1; ++k) {
      T acc = y[k];
#pragma unroll
      for (int a = 0; a < RM; ++a) acc = fma(-Uk[k][a], w[a], acc);
      const double e = (double)acc, yy = (double)y[k];
      se = fma(e, e, se);
      sy = fma(yy, yy, sy);
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sy += __shfl_xor_sync(0xffffffffu, sy, o);
    se += __shfl_xor_sync(0xffffffffu, se, o);
  }
  __shared__ double red[2][kK1Threads / 32];
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = sy;
    red[1][threadIdx.x >> 5] = se;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < kK1Threads / 32; ++w) { a += red[0][w]; c += red[1][w]; }
    double* pz = part + 2 * ((int64_t)z * blocks_per_obs + blockIdx.x);
    pz[0] = a;
    pz[1] = c;
  }
}

}  // namespace

// Per-observation sums of the K1 partials (fixed order, so the result does not depend on how the
// partials were scheduled): y2[z] += sum_j part[z][j][0], rho2[z] += sum_j part[z][j][1].
__global__ void k1_reduce_kernel(const double* part, int64_t per_obs, double* y2, double* rho2) {
  const int z = blockIdx.x;
  const double* p = part + 2 * (int64_t)z * per_obs;
  __shared__ double sa[256], sc[256];
  double a = 0.0, c = 0.0;
  for (int64_t j = threadIdx.x; j < per_obs; j += blockDim.x) { a += p[2 * j]; c += p[2 * j + 1]; }
  sa[threadIdx.x] = a;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) { sa[threadIdx.x] += sa[threadIdx.x + o]; sc[threadIdx.x] += sc[threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { y2[z] += sa[0]; rho2[z] += sc[0]; }
}

cudaError_t launch_k1_reduce(const double* part, int b, int64_t per_obs, double* y2, double* rho2,
                             cudaStream_t st) {
  note_launch();
  k1_reduce_kernel<<<b, 256, 0, st>>>(part, per_obs, y2, rho2);
  return cudaGetLastError();
}

namespace {


template <typename TY, typename T, int N1, int RM>
cudaError_t run_k1(const TY* Y, int b, int64_t L, int n1, int r, const T* U, int64_t ldu, T* W,
                   double* y2, double* rho2, double* part, cudaStream_t st) {
  // persistent grid: about four CTAs per SM in total, split over the observations
  int64_t per_obs = (4 * 152 + b - 1) / b;
  per_obs = std::max<int64_t>(1, std::min<int64_t>(per_obs, (L + kK1Threads - 1) / kK1Threads));
  dim3 grid((unsigned)per_obs, (unsigned)b);
  note_launch();
  k1_kernel<TY, T, N1, RM><<<grid, kK1Threads, 0, st>>>(Y, L, n1, r, U, ldu, W, part, per_obs);
  TT_CUDA(cudaGetLastError());
  return launch_k1_reduce(part, b, per_obs, y2, rho2, st);
}

}  // namespace

template <typename TY, typename T>
bool k1_supported(int n1, int r) {
  return n1 <= 32 && r <= 32 && r >= 1;
}

template <typename TY, typename T>
cudaError_t launch_k1(const TY* Y, int b, int64_t L, int n1, int r, const T* U, int64_t ldu, T* W,
                      double* y2, double* rho2, double* part, cudaStream_t st) {
  if (n1 <= 8 && r <= 8) return run_k1<TY, T, 8, 8>(Y, b, L, n1, r, U, ldu, W, y2, rho2, part, st);
  if (n1 <= 16 && r <= 16) return run_k1<TY, T, 16, 16>(Y, b, L, n1, r, U, ldu, W, y2, rho2, part, st);
  if (n1 <= 32 && r <= 16) return run_k1<TY, T, 32, 16>(Y, b, L, n1, r, U, ldu, W, y2, rho2, part, st);
  if (n1 <= 32 && r <= 24) return run_k1<TY, T, 32, 24>(Y, b, L, n1, r, U, ldu, W, y2, rho2, part, st);
  if (n1 <= 32 && r <= 32) return run_k1<TY, T, 32, 32>(Y, b, L, n1, r, U, ldu, W, y2, rho2, part, st);
  return cudaErrorInvalidValue;
}

#define TT_K1_INST(TY, T)                                                                          \
  template bool k1_supported<TY, T>(int, int);                                                      \
  template cudaError_t launch_k1<TY, T>(const TY*, int, int64_t, int, int, const T*, int64_t, T*, \
                                        double*, double*, double*, cudaStream_t);
TT_K1_INST(float, float)
TT_K1_INST(double, float)
TT_K1_INST(float, double)
TT_K1_INST(double, double)

}  // namespace ttice
