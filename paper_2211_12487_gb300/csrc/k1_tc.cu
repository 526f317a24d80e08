// K1 on the tensor cores: the first pass over an FP32 increment, stage 1 (Eq. 6, Eq. 17), with the
// projection W = U_1^T Y_1 as tcgen05 MMAs.
//
// Arithmetic.  TF32 keeps 10 mantissa bits, which would perturb W by ~1e-3 relative and, through
// the later stages, the rank decisions.  Each operand x is therefore split into x_hi = tf32(x) and
// x_lo = x - x_hi (exact in FP32) and the product is taken as A_hi B_hi + A_lo B_hi + A_hi B_lo (the
// dropped A_lo B_lo is ~2^-22 relative), accumulated in FP32 in tensor memory: W to FP32 accuracy.
// The residual norm of each column uses the orthogonality of U_1 (Pythagoras): ||y - U_1 w||^2 =
// ||y||^2 - ||w||^2, the two sums taken per column in FP32 (at most 32 and 64 terms) and combined
// in FP64.  That is exact for an orthonormal U_1; in FP32 it carries ~1e-7 ||y||^2 of rounding per
// column, which the per-observation sum averages, against the ~1e-6 relative of a direct FP32
// residual.
//
// Shapes.  The MMA is D[128 x N] += A[128 x 8] B[8 x N] with M = 128 columns of the increment (one
// tile), K = 8 mode-1 rows per instruction, N = r_1 rounded up to 16 (at most 64).  Mode 1 is staged
// in chunks of 32 rows (one 128-byte swizzle row of TF32); n_1 <= 128 gives at most four chunks,
// rows beyond n_1 are zero.
//
// Roles (6 warps, one persistent CTA per SM):
//   warp 4, one lane:  TMA loads of raw 32 x 128 FP32 chunks (row-major, no swizzle; n_1 rounded up
//                      to 8 rows when n_1 < 32) into a ring;
//   warps 0-3:         each thread owns one column of the tile: it reads its 32 values of a chunk,
//                      writes x_hi and x_lo into the K-major, 128-byte-swizzled A operand (one row
//                      per column) and sums y^2; after the last chunk it reads its row of the
//                      accumulator from tensor memory (w), stores w, and forms ||y||^2 - ||w||^2;
//   warp 5:            allocates tensor memory; one lane issues the MMAs of each chunk and commits
//                      them to the barriers that free the A slot and, per tile, publish the
//                      accumulator (two accumulators, so the MMAs of tile t+1 overlap the epilogue
//                      of tile t).
// U_1 (hi and lo) is staged once per CTA as the K-major B operand.  Every wait is bounded in time;
// on expiry the waiting thread raises a CTA-wide abort flag, every role leaves its loop, the MMA
// warp waits for its issued MMAs, the producer for its copies in flight, tensor memory is freed
// and `status` records the failure.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "ttice_internal.cuh"

namespace ttice {
namespace {

constexpr int kTile = 128;        // columns per tile (MMA M)
constexpr int kChunk = 32;        // mode-1 rows per staged chunk
constexpr int kMaxChunks = 4;     // n_1 <= 128
constexpr int kRawStages = 4;     // TMA ring
constexpr int kAStages = 2;       // A-operand ring
constexpr int kConvWarps = 4;
constexpr int kThreads = (kConvWarps + 2) * 32;
constexpr int kProducerWarp = kConvWarps, kMmaWarp = kConvWarps + 1;
constexpr int kAccCols = 64;      // tensor-memory columns per accumulator
constexpr uint32_t kTmemCols = 2 * kAccCols;
constexpr uint32_t kRawBytes = kChunk * kTile * 4;   // 16 KB
constexpr uint32_t kABytes = kTile * kChunk * 4;     // 16 KB: 128 rows x 128 B
constexpr unsigned long long kWaitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
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
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of `bar` with the given parity to complete, for at most about kWaitNs; gives up
// early once another thread has raised *abort, and raises it on expiry.  The clock is first read
// after 128 unsuccessful polls, so a wait on a completed phase costs one try_wait.
__device__ __forceinline__ bool wait_bounded(uint64_t* bar, uint32_t parity, volatile int* abort) {
  unsigned long long t0 = 0;
  for (uint32_t i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 127u) == 127u) {
      if (*abort) return false;
      const unsigned long long t = now_ns();
      if (t0 == 0) {
        t0 = t;
      } else if (t - t0 > kWaitNs) {
        *abort = 1;
        return false;
      }
    }
  }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
// MMA K steps (8 rows each) of chunk c that reach a row below n_1
__device__ __forceinline__ int chunk_ksteps(int n1, int c) {
  const int rows = n1 - c * kChunk;
  return rows >= kChunk ? kChunk / 8 : (rows + 7) / 8;
}
// Shared-memory matrix descriptor of a K-major operand with the 128-byte swizzle: rows of 128 bytes
// (32 TF32 values of K), groups of 8 rows 1024 bytes apart.  `addr` is the first row's address plus
// the byte offset of the K step inside the 128-byte row.
__device__ __forceinline__ uint64_t kmajor_sw128_desc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFFu);         // start address
  d |= (uint64_t)1 << 16;                          // leading byte offset (unused for this layout)
  d |= (uint64_t)((1024u >> 4) & 0x3FFFu) << 32;   // stride byte offset: next group of 8 rows
  d |= (uint64_t)1 << 46;                          // descriptor version
  d |= (uint64_t)2 << 61;                          // 128-byte swizzle
  return d;
}
// Instruction descriptor of tcgen05.mma kind::tf32: D FP32, A and B TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t tf32_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n"
      " .reg .pred p;\n"
      " setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
      "}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 16 consecutive accumulator columns of this thread's lane
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15},"
      " [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

template <int RP, bool NORMS>
__global__ void __launch_bounds__(kThreads, 1)
    k1_tc_kernel(const __grid_constant__ CUtensorMap tmap, int n1, int box_rows, int r, int64_t L,
                 int b, const float* __restrict__ U, int64_t ldu, float* __restrict__ W, double* part,
                 int* status) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nch = (n1 + kChunk - 1) / kChunk;
  unsigned char* raw = base;                                  // kRawStages x 16 KB
  unsigned char* a_hi = raw + kRawStages * kRawBytes;         // kAStages x 16 KB
  unsigned char* a_lo = a_hi + kAStages * kABytes;            // kAStages x 16 KB
  unsigned char* u_hi = a_lo + kAStages * kABytes;            // nch x RP rows x 128 B
  unsigned char* u_lo = u_hi + (size_t)nch * RP * 128;

  __shared__ __align__(8) uint64_t raw_full[kRawStages], raw_empty[kRawStages];
  __shared__ __align__(8) uint64_t a_full[kAStages], a_empty[kAStages];
  __shared__ __align__(8) uint64_t acc_full[2], acc_empty[2], mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;

  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;

  // U_1 as the K-major B operand: row a (N index) holds U_1(k, a) for the 32 k of a chunk, 16-byte
  // unit j (k = 4j..4j+3) at position j ^ (a % 8) of the row.
  for (int u = tid; u < nch * RP * 8; u += kThreads) {
    const int c = u / (RP * 8), a = (u / 8) % RP, j = u % 8;
    float4 hi, lo;
    float* ph = &hi.x;
    float* pl = &lo.x;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int k = c * kChunk + 4 * j + e;
      const float x = (a < r && k < n1) ? U[(int64_t)a * ldu + k] : 0.0f;
      ph[e] = tf32_hi(x);
      pl[e] = x - ph[e];
    }
    const size_t off = ((size_t)c * RP + a) * 128 + (size_t)((j ^ (a & 7)) << 4);
    *reinterpret_cast<float4*>(u_hi + off) = hi;
    *reinterpret_cast<float4*>(u_lo + off) = lo;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  if (tid == 0) {
    for (int s = 0; s < kRawStages; ++s) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_empty[s], kConvWarps);
    }
    for (int q = 0; q < kAStages; ++q) {
      mbar_init(&a_full[q], kConvWarps);
      mbar_init(&a_empty[q], 1);
    }
    for (int q = 0; q < 2; ++q) {
      mbar_init(&acc_full[q], 1);
      mbar_init(&acc_empty[q], kConvWarps);
    }
    mbar_init(&mma_done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (wid == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    tc_fence_before();
  }
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  const int64_t tpo = (L + kTile - 1) / kTile;  // tiles per observation
  const int64_t ntiles = tpo * b;

  if (wid == kProducerWarp) {
    if (lane == 0) {
      int64_t g = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int z = (int)(t / tpo);
        const int x = (int)((t % tpo) * kTile);
        for (int c = 0; c < nch; ++c, ++g) {
          const int s = (int)(g % kRawStages);
          if (g >= kRawStages &&
              !wait_bounded(&raw_empty[s], (uint32_t)(((g / kRawStages) - 1) & 1), &abort_flag)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&raw_full[s], (uint32_t)box_rows * kTile * 4);
          tma_load_2d(smem_u32(raw + (size_t)s * kRawBytes), &tmap, x, z * n1 + c * kChunk, &raw_full[s]);
        }
      }
      // the copies of the last kRawStages loads may still be in flight (on an abort): wait for them
      for (int64_t j = g > kRawStages ? g - kRawStages : 0; j < g; ++j) {
        const unsigned long long t0 = now_ns();
        while (!mbar_try_wait(&raw_full[j % kRawStages], (uint32_t)((j / kRawStages) & 1)) &&
               now_ns() - t0 < kWaitNs) {
        }
      }
    }
  } else if (wid == kMmaWarp) {
    if (lane == 0) {
      constexpr uint32_t idesc = tf32_idesc(kTile, RP);
      int64_t g = 0;
      int it = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++it) {
        const int acc = it & 1;
        if (it >= 2 && !wait_bounded(&acc_empty[acc], (uint32_t)(((it >> 1) - 1) & 1), &abort_flag)) break;
        tc_fence_after();
        const uint32_t d = tmem + (uint32_t)(acc * kAccCols);
        for (int c = 0; c < nch; ++c, ++g) {
          const int q = (int)(g % kAStages);
          if (!wait_bounded(&a_full[q], (uint32_t)((g / kAStages) & 1), &abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ah = smem_u32(a_hi + (size_t)q * kABytes), al = smem_u32(a_lo + (size_t)q * kABytes);
          const uint32_t bh = smem_u32(u_hi + (size_t)c * RP * 128), bl = smem_u32(u_lo + (size_t)c * RP * 128);
          const int nk = chunk_ksteps(n1, c);
#pragma unroll
          for (int kk = 0; kk < kChunk / 8; ++kk) {
            if (kk >= nk) break;
            const uint32_t ko = (uint32_t)kk * 32;  // 8 TF32 values of K
            mma_tf32(d, kmajor_sw128_desc(ah + ko), kmajor_sw128_desc(bh + ko), idesc, (c | kk) != 0);
            mma_tf32(d, kmajor_sw128_desc(al + ko), kmajor_sw128_desc(bh + ko), idesc, 1);
            mma_tf32(d, kmajor_sw128_desc(ah + ko), kmajor_sw128_desc(bl + ko), idesc, 1);
          }
          mma_commit(&a_empty[q]);  // frees the A slot once these MMAs have read it
        }
        if (ok) mma_commit(&acc_full[acc]);
      }
      // every MMA issued has completed before tensor memory is released
      mma_commit(&mma_done);
      const unsigned long long t0 = now_ns();
      while (!mbar_try_wait(&mma_done, 0) && now_ns() - t0 < kWaitNs) {
      }
    }
  } else {
    // converters and epilogue: thread tid owns column tid of every tile.  The epilogue of tile t
    // runs after the conversion of tile t+1, so that the MMAs of tile t overlap that conversion.
    int64_t g = 0;
    int it = 0;
    int64_t t_prev = -1;
    float y2_prev = 0.0f;
    for (int64_t t = blockIdx.x;; t += gridDim.x, ++it) {
      const bool conv = t < ntiles;
      float y2 = 0.0f;  // ||y||^2 of this column (at most 128 terms)
      bool ok = true;
      for (int c = 0; conv && c < nch; ++c, ++g) {
        const int s = (int)(g % kRawStages), q = (int)(g % kAStages);
        bool got = wait_bounded(&raw_full[s], (uint32_t)((g / kRawStages) & 1), &abort_flag);
        if (got && g >= kAStages)
          got = wait_bounded(&a_empty[q], (uint32_t)(((g / kAStages) - 1) & 1), &abort_flag);
        if (!__all_sync(0xffffffffu, got)) {  // the warp takes one branch (aligned tcgen05 loads below)
          ok = false;
          break;
        }
        const float* rw = reinterpret_cast<const float*>(raw + (size_t)s * kRawBytes);
        unsigned char* ah = a_hi + (size_t)q * kABytes + (size_t)tid * 128;
        unsigned char* al = a_lo + (size_t)q * kABytes + (size_t)tid * 128;
        const int units = 2 * chunk_ksteps(n1, c);  // 16-byte units the MMAs of this chunk read
#pragma unroll
        for (int j = 0; j < kChunk / 4; ++j) {
          if (j < units) {
            float4 hi, lo;
            float* ph = &hi.x;
            float* pl = &lo.x;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int kk = 4 * j + e;
              const float y = (c * kChunk + kk < n1) ? rw[kk * kTile + tid] : 0.0f;
              y2 = fmaf(y, y, y2);
              ph[e] = tf32_hi(y);
              pl[e] = y - ph[e];
            }
            const int off = (j ^ (tid & 7)) << 4;
            *reinterpret_cast<float4*>(ah + off) = hi;
            *reinterpret_cast<float4*>(al + off) = lo;
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&a_full[q]);
          mbar_arrive(&raw_empty[s]);
        }
      }
      if (!ok) break;
      if (t_prev >= 0) {
        // epilogue of the previous tile (iteration it - 1)
        const int ip = it - 1, acc = ip & 1;
        if (!__all_sync(0xffffffffu, wait_bounded(&acc_full[acc], (uint32_t)((ip >> 1) & 1), &abort_flag)))
          break;
        tc_fence_after();
        float w[RP];
        const uint32_t taddr = tmem + ((uint32_t)(wid * 32) << 16) + (uint32_t)(acc * kAccCols);
#pragma unroll
        for (int j = 0; j < RP / 16; ++j) tmem_ld16(taddr + (uint32_t)(16 * j), w + 16 * j);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[acc]);
        float ws = 0.0f;
#pragma unroll
        for (int a = 0; a < RP; ++a)
          if (a < r) ws = fmaf(w[a], w[a], ws);
        const int zp = (int)(t_prev / tpo);
        const int64_t lp = (t_prev % tpo) * kTile + tid;
        if (lp < L) {
          float* Wz = W + (int64_t)zp * r * L + lp;
#pragma unroll
          for (int a = 0; a < RP; ++a)
            if (a < r) Wz[(int64_t)a * L] = w[a];
        }
        if constexpr (NORMS) {
          // the difference of two FP32 sums of one column is exact to their own rounding
          float sy = y2_prev, se = y2_prev - ws;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            sy += __shfl_xor_sync(0xffffffffu, sy, o);
            se += __shfl_xor_sync(0xffffffffu, se, o);
          }
          if (lane == 0) {
            part[(t_prev * kConvWarps + wid) * 2] = (double)sy;
            part[(t_prev * kConvWarps + wid) * 2 + 1] = (double)se;
          }
        }
      }
      if (!conv) break;
      t_prev = t;
      y2_prev = y2;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (wid == kMmaWarp) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols)
                 : "memory");
  }
  if (tid == 0 && abort_flag) atomicOr(status, 1);
}

// ||y||^2 and ||y - U_1 w||^2 per observation from the per-tile, per-warp partial sums, added in a
// fixed order; the residual is clamped at zero (the Pythagorean difference can round below it when
// U_1 spans the observation).
__global__ void k1_tc_reduce_kernel(const double* part, int64_t per_obs, double* y2, double* rho2) {
  const int z = blockIdx.x;
  double a = 0.0, c = 0.0;
  for (int64_t i = threadIdx.x; i < per_obs; i += blockDim.x) {
    a += part[((int64_t)z * per_obs + i) * 2];
    c += part[((int64_t)z * per_obs + i) * 2 + 1];
  }
  __shared__ double sa[256], sc[256];
  sa[threadIdx.x] = a;
  sc[threadIdx.x] = c;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      sa[threadIdx.x] += sa[threadIdx.x + o];
      sc[threadIdx.x] += sc[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    y2[z] = sa[0];
    rho2[z] = fmin(fmax(sc[0], 0.0), sa[0]);
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

size_t smem_bytes(int nch, int rp) {
  return (size_t)kRawStages * kRawBytes + 2 * (size_t)kAStages * kABytes + 2 * (size_t)nch * rp * 128 + 1024;
}

template <int RP, bool NORMS>
cudaError_t run(const float* Y, int b, int64_t L, int n1, int r, const float* U, int64_t ldu, float* W,
                double* y2, double* rho2, double* part, int* status, cudaStream_t st) {
  auto enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  CUtensorMap map;
  const cuuint64_t gdim[2] = {(cuuint64_t)L, (cuuint64_t)b * n1};
  const cuuint64_t gstride[1] = {(cuuint64_t)L * sizeof(float)};
  // rows per copy: a whole chunk, or n_1 rounded up to 8 when one chunk covers mode 1
  const int box_rows = n1 >= kChunk ? kChunk : (n1 + 7) / 8 * 8;
  const cuuint32_t box[2] = {(cuuint32_t)kTile, (cuuint32_t)box_rows};
  const cuuint32_t estride[2] = {1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(Y), gdim, gstride, box, estride,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  const int nch = (n1 + kChunk - 1) / kChunk;
  const size_t smem = smem_bytes(nch, RP);
  static std::once_flag once;
  static cudaError_t setup_err = cudaSuccess;
  static int sms = 148;
  std::call_once(once, [] {
    setup_err = cudaFuncSetAttribute(k1_tc_kernel<RP, NORMS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_bytes(kMaxChunks, RP));
    int dev = 0;
    if (setup_err == cudaSuccess) setup_err = cudaGetDevice(&dev);
    if (setup_err == cudaSuccess) setup_err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  });
  TT_CUDA(setup_err);
  const int64_t ntiles = ((L + kTile - 1) / kTile) * b;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(sms, ntiles));
  note_launch();
  k1_tc_kernel<RP, NORMS><<<(unsigned)grid, kThreads, smem, st>>>(map, n1, box_rows, r, L, b, U, ldu, W,
                                                                   part, status);
  TT_CUDA(cudaGetLastError());
  if constexpr (NORMS) {
    note_launch();
    k1_tc_reduce_kernel<<<b, 256, 0, st>>>(part, ((L + kTile - 1) / kTile) * kConvWarps, y2, rho2);
    TT_CUDA(cudaGetLastError());
  }
  return cudaSuccess;
}

}  // namespace

bool k1_tc_supported(const void* Y, int64_t L, int n1, int r) {
  return encode_fn() != nullptr && (reinterpret_cast<uintptr_t>(Y) % 16) == 0 && (L % 4) == 0 &&
         L < (1LL << 31) && n1 >= 1 && n1 <= kMaxChunks * kChunk && r >= 1 && r <= kAccCols;
}

int64_t k1_tc_part_elems(int b, int64_t L) { return 2 * (int64_t)b * ((L + kTile - 1) / kTile) * kConvWarps; }

cudaError_t launch_k1_tc(const float* Y, int b, int64_t L, int n1, int r, const float* U, int64_t ldu,
                         float* W, double* y2, double* rho2, double* part, int* status, cudaStream_t st) {
  const bool nrm = y2 != nullptr;
#define TT_K1TC_CASE(RP_)                                                                 \
  return nrm ? run<RP_, true>(Y, b, L, n1, r, U, ldu, W, y2, rho2, part, status, st)      \
             : run<RP_, false>(Y, b, L, n1, r, U, ldu, W, y2, rho2, part, status, st)
  if (r <= 16) TT_K1TC_CASE(16);
  if (r <= 32) TT_K1TC_CASE(32);
  if (r <= 48) TT_K1TC_CASE(48);
  if (r <= 64) TT_K1TC_CASE(64);
#undef TT_K1TC_CASE
  return cudaErrorInvalidValue;
}

}  // namespace ttice
