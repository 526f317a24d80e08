// K1 with TMA staging: the first pass over an FP32 increment, stage 1 (Eq. 6, Eq. 17), fused.
//
// The increment is viewed as a 2-D tensor of (b * n_1) rows by L_1 columns (row z*n_1 + k holds
// mode-1 index k of observation z).  The grid is persistent (a multiple of the SM count); each CTA
// walks tiles of n_1 x 256 columns of one observation.  Thread 0 keeps kStages tiles in flight with
// cp.async.bulk.tensor (TMA) into shared memory, each completing on its own mbarrier; the CTA waits
// on the barrier of the current stage, every thread takes one column of the tile from shared memory,
// accumulates w = U_1^T y in registers (U_1 broadcast from shared memory, 16-byte loads), writes w,
// forms the direct residual e = y - U_1 w and the FP64 sums ||y||^2, ||e||^2 (one partial per tile,
// summed per observation afterwards in a fixed order), and the stage is
// refilled with the tile kStages ahead once the CTA has finished reading it.  Every mbarrier wait
// is bounded: on expiry the kernel records the failure in `status`, waits (bounded again) for its
// own copies still in flight, and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "ttice_internal.cuh"

namespace ttice {
namespace {

constexpr int kTileL = 256;
constexpr int kStages = 2;
constexpr int kThreads = kTileL;         // one column per thread
constexpr long long kSpinLimit = 1LL << 24;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n"
      "}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

template <typename T, int N1, int RM, bool NORMS>
__global__ void __launch_bounds__(kThreads) k1_tma_kernel(const __grid_constant__ CUtensorMap tmap,
                                                          int n1, int r, int64_t L, int b,
                                                          const T* __restrict__ U, int64_t ldu,
                                                          T* __restrict__ W, double* part,
                                                          int* status) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // stage buffers (kStages x N1 x kTileL floats), placed on a 128-byte boundary for the TMA writes
  float* tiles = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  __shared__ __align__(16) T Uk[N1][RM];               // Uk[k][a] = U_1(k, a)
  __shared__ __align__(8) uint64_t full[kStages];
  __shared__ double red[2][kThreads / 32];
  const int tid = threadIdx.x;
  for (int e = tid; e < N1 * RM; e += kThreads) {
    const int k = e / RM, a = e % RM;
    Uk[k][a] = (a < r && k < n1) ? U[(int64_t)a * ldu + k] : T(0);
  }
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) mbar_init(&full[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();

  const int64_t tiles_per_obs = (L + kTileL - 1) / kTileL;
  const int64_t ntiles = tiles_per_obs * b;
  const uint32_t tile_bytes = (uint32_t)n1 * kTileL * sizeof(float);
  auto issue = [&](int64_t t, int s) {
    const int z = (int)(t / tiles_per_obs);
    const int x = (int)((t % tiles_per_obs) * kTileL);
    mbar_expect_tx(&full[s], tile_bytes);
    tma_load_2d(tiles + (size_t)s * N1 * kTileL, &tmap, x, z * n1, &full[s]);
  };
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      const int64_t t = blockIdx.x + (int64_t)s * gridDim.x;
      if (t < ntiles) issue(t, s);
    }
  }

  __shared__ int stage_ok;
  int it = 0;
  bool failed = false;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int s = it % kStages;
    const uint32_t parity = (uint32_t)((it / kStages) & 1);
    // One thread waits (bounded) and the outcome is shared, so that the whole CTA takes the same
    // branch; then every thread observes the completed phase (acquiring the tile's bytes).
    if (tid == 0) stage_ok = mbar_wait_bounded(&full[s], parity) ? 1 : 0;
    __syncthreads();
    if (!stage_ok) { failed = true; break; }
    mbar_try_wait(&full[s], parity);
    const float* tile = tiles + (size_t)s * N1 * kTileL;
    const int z = (int)(t / tiles_per_obs);
    const int64_t l = (t % tiles_per_obs) * kTileL + tid;
    T w[RM];
#pragma unroll
    for (int a = 0; a < RM; ++a) w[a] = T(0);
    // squares of one column are summed in T (n_1 <= 32 terms), columns are combined in FP64
    T sy_c = T(0);
#pragma unroll
    for (int k = 0; k < N1; ++k) {
      if (k < n1) {
        const T y = (T)tile[k * kTileL + tid];
        sy_c = fma(y, y, sy_c);
#pragma unroll
        for (int a = 0; a < RM; ++a) w[a] = fma(Uk[k][a], y, w[a]);
      }
    }
    if (l < L) {
      T* Wz = W + (int64_t)z * r * L + l;
#pragma unroll
      for (int a = 0; a < RM; ++a)
        if (a < r) Wz[(int64_t)a * L] = w[a];
    }
    if constexpr (!NORMS) {
      __syncthreads();  // every thread is done reading stage s
      if (tid == 0) {
        const int64_t tn = t + (int64_t)kStages * gridDim.x;
        if (tn < ntiles) issue(tn, s);
      }
      continue;
    }
    // back-projection with one independent accumulator per row k (e_k = y_k - sum_a U(k,a) w_a)
    T e[N1];
#pragma unroll
    for (int k = 0; k < N1; ++k) e[k] = (k < n1) ? (T)tile[k * kTileL + tid] : T(0);
#pragma unroll
    for (int a = 0; a < RM; ++a) {
#pragma unroll
      for (int k = 0; k < N1; ++k) e[k] = fma(-Uk[k][a], w[a], e[k]);
    }
    T se_c = T(0);
#pragma unroll
    for (int k = 0; k < N1; ++k)
      if (k < n1) se_c = fma(e[k], e[k], se_c);
    double sy = (double)sy_c, se = (double)se_c;
    // per-tile reduction of the two norms, one FP64 atomic each per tile
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      se += __shfl_xor_sync(0xffffffffu, se, o);
    }
    if ((tid & 31) == 0) { red[0][tid >> 5] = sy; red[1][tid >> 5] = se; }
    __syncthreads();  // also: every thread is done reading stage s
    if (tid == 0) {
      double a = 0.0, c = 0.0;
      for (int q = 0; q < kThreads / 32; ++q) { a += red[0][q]; c += red[1][q]; }
      part[2 * t] = a;
      part[2 * t + 1] = c;
      const int64_t tn = t + (int64_t)kStages * gridDim.x;
      if (tn < ntiles) issue(tn, s);
    }
  }
  if (failed && tid == 0) {
    atomicOr(status, 1);
    // drain: wait (bounded) for the copies this CTA still has in flight before leaving
    for (int j = 0; j < kStages; ++j) {
      const int itj = it + j;
      const int64_t t = blockIdx.x + (int64_t)itj * gridDim.x;
      if (t >= ntiles) break;
      mbar_wait_bounded(&full[itj % kStages], (uint32_t)((itj / kStages) & 1));
    }
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

template <typename T, int N1, int RM, bool NORMS>
cudaError_t run(const float* Y, int b, int64_t L, int n1, int r, const T* U, int64_t ldu, T* W,
                double* y2, double* rho2, double* part, int* status, cudaStream_t st) {
  auto enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t gdim[2] = {(cuuint64_t)L, (cuuint64_t)b * n1};
  const cuuint64_t gstride[1] = {(cuuint64_t)L * sizeof(float)};
  const cuuint32_t box[2] = {(cuuint32_t)kTileL, (cuuint32_t)n1};
  const cuuint32_t estride[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(Y), gdim, gstride, box,
          estride, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const size_t smem = (size_t)kStages * N1 * kTileL * sizeof(float) + 128;
  // one-time set-up per instantiation: shared-memory attribute, occupancy and SM count
  static std::once_flag once;
  static cudaError_t setup_err = cudaSuccess;
  static int per_sm = 1, sms = 152;
  std::call_once(once, [smem] {
    setup_err = cudaFuncSetAttribute(k1_tma_kernel<T, N1, RM, NORMS>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (setup_err == cudaSuccess)
      setup_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k1_tma_kernel<T, N1, RM, NORMS>,
                                                                kThreads, smem);
    int dev = 0;
    if (setup_err == cudaSuccess) setup_err = cudaGetDevice(&dev);
    if (setup_err == cudaSuccess)
      setup_err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  });
  TT_CUDA(setup_err);
  const int64_t ntiles = ((L + kTileL - 1) / kTileL) * b;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((int64_t)sms * std::max(per_sm, 1), ntiles));
  note_launch();
  k1_tma_kernel<T, N1, RM, NORMS><<<(unsigned)grid, kThreads, smem, st>>>(map, n1, r, L, b, U, ldu,
                                                                           W, part, status);
  TT_CUDA(cudaGetLastError());
  if constexpr (NORMS) return launch_k1_reduce(part, b, (L + kTileL - 1) / kTileL, y2, rho2, st);
  return cudaSuccess;
}

}  // namespace

bool k1_tma_supported(const void* Y, int64_t L, int n1, int r) {
  return encode_fn() != nullptr && (reinterpret_cast<uintptr_t>(Y) % 16) == 0 && (L % 4) == 0 &&
         L < (1LL << 31) && n1 >= 1 && n1 <= 32 && r >= 1 && r <= 32;
}

template <typename T>
cudaError_t launch_k1_tma(const float* Y, int b, int64_t L, int n1, int r, const T* U, int64_t ldu,
                          T* W, double* y2, double* rho2, double* part, int* status, cudaStream_t st) {
  // y2 == nullptr: projection only (no residual, no norms)
  const bool nrm = y2 != nullptr;
#define TT_K1_CASE(N1_, RM_)                                                                   \
  return nrm ? run<T, N1_, RM_, true>(Y, b, L, n1, r, U, ldu, W, y2, rho2, part, status, st)  \
             : run<T, N1_, RM_, false>(Y, b, L, n1, r, U, ldu, W, y2, rho2, part, status, st)
  if (n1 <= 8 && r <= 8) TT_K1_CASE(8, 8);
  if (n1 <= 16 && r <= 16) TT_K1_CASE(16, 16);
  if (n1 <= 24 && r <= 16) TT_K1_CASE(24, 16);
  if (n1 <= 24 && r <= 24) TT_K1_CASE(24, 24);
  if (n1 <= 32 && r <= 16) TT_K1_CASE(32, 16);
  if (n1 <= 32 && r <= 32) TT_K1_CASE(32, 32);
#undef TT_K1_CASE
  return cudaErrorInvalidValue;
}

template cudaError_t launch_k1_tma<float>(const float*, int, int64_t, int, int, const float*,
                                          int64_t, float*, double*, double*, double*, int*,
                                          cudaStream_t);
template cudaError_t launch_k1_tma<double>(const float*, int, int64_t, int, int, const double*,
                                           int64_t, double*, double*, double*, double*, int*,
                                           cudaStream_t);

}  // namespace ttice
