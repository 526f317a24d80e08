// Generic strided, batched SIMT GEMM used by the FP64 path and by the small contractions of every
// path: projections U_i^T Y_i (Eq. 12), back-projections and residuals (Eq. 6), residual Gram
// matrices (Eq. 9 via R R^T), CGS2 projections (Eq. 10) and reconstructions (Eq. 14).
//
// Tiles of BM x BN outputs, BK-deep K slices staged in shared memory (converted to the accumulator
// type on load), TM x TN outputs per thread.  Loads follow whichever operand stride is 1, so both
// K-contiguous and M/N-contiguous operands are read coalesced.  The epilogue forms
// alpha*acc + beta*X, optionally accumulates the squared entries per batch (FP64 atomics), and either
// stores or atomically adds into C (the latter enables split-K and reductions over a batch index).
#include <algorithm>

#include "ttice_internal.cuh"

namespace ttice {
namespace {

template <typename T>
__device__ __forceinline__ T ld_elem(const void* p, int64_t off) {
  return static_cast<const T*>(p)[off];
}

template <typename TA, typename TB, typename TX, typename TC, typename ACC, int BM, int BN, int BK,
          int TM, int TN>
__global__ void __launch_bounds__((BM / TM) * (BN / TN)) gemm_kernel(GemmArgs g, int ksplit, int64_t kchunk) {
  constexpr int NT = (BM / TM) * (BN / TN);  // threads: one per TM x TN block of outputs
  static_assert(NT % 32 == 0 && NT <= 256, "whole warps, at most 256 threads");
  __shared__ ACC As[BK][BM + 1];
  __shared__ ACC Bs[BK][BN + 1];
  const int z = blockIdx.z;
  const int zb = z / ksplit, zk = z % ksplit;
  const int z1 = zb / g.bdiv, z2 = zb % g.bdiv;
  const int64_t aoff = z1 * g.A.bs1 + z2 * g.A.bs2;
  const int64_t boff = z1 * g.B.bs1 + z2 * g.B.bs2;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  const int64_t kbeg = zk * kchunk;
  const int64_t kend = min(g.K, kbeg + kchunk);
  const int tid = threadIdx.x;
  const int tx = tid % (BN / TN), ty = tid / (BN / TN);
  // symmetric Gram: global row/column offsets of this batch's block; tiles wholly below the
  // diagonal are left to the mirror writes of their transposes
  const int64_t sym_r = (g.sym == 2) ? (int64_t)z1 * g.M : 0, sym_c = (g.sym == 2) ? (int64_t)z2 * g.N : 0;
  if (g.sym && sym_r + m0 > sym_c + n0 + BN - 1) return;
  const bool a_kfast = (g.A.cs == 1);
  const bool b_nfast = (g.B.cs == 1);

  // FP32 products accumulated into FP64 every kMixSlabs K-slabs when the output is FP64
  constexpr bool kMix = sizeof(ACC) == 4 && sizeof(TC) == 8;
  constexpr int kMixSlabs = 4;
  ACC acc[TM][TN];
  double acc64[kMix ? TM : 1][kMix ? TN : 1];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = ACC(0);
  if constexpr (kMix) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc64[i][j] = 0.0;
  }
  int slab = 0;

  // register double buffering: the next K-slab is loaded from global memory while the current one
  // is multiplied out of shared memory
  constexpr int NA = (BM * BK + NT - 1) / NT, NB = (BN * BK + NT - 1) / NT;
  ACC ra[NA], rb[NB];
  auto load_slab = [&](int64_t k0) {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int e = tid + q * NT;
      ACC v = ACC(0);
      if (e < BM * BK) {
        int mm, kk;
        if (a_kfast) { mm = e / BK; kk = e % BK; } else { mm = e % BM; kk = e / BM; }
        const int64_t gm = m0 + mm, gk = k0 + kk;
        if (gm < g.M && gk < kend) v = (ACC)ld_elem<TA>(g.A.p, aoff + gm * g.A.rs + gk * g.A.cs);
      }
      ra[q] = v;
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int e = tid + q * NT;
      ACC v = ACC(0);
      if (e < BN * BK) {
        int nn, kk;
        if (b_nfast) { nn = e % BN; kk = e / BN; } else { nn = e / BK; kk = e % BK; }
        const int64_t gn = n0 + nn, gk = k0 + kk;
        if (gn < g.N && gk < kend) v = (ACC)ld_elem<TB>(g.B.p, boff + gk * g.B.rs + gn * g.B.cs);
      }
      rb[q] = v;
    }
  };
  auto store_slab = [&]() {
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const int e = tid + q * NT;
      if (e < BM * BK) {
        int mm, kk;
        if (a_kfast) { mm = e / BK; kk = e % BK; } else { mm = e % BM; kk = e / BM; }
        As[kk][mm] = ra[q];
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int e = tid + q * NT;
      if (e < BN * BK) {
        int nn, kk;
        if (b_nfast) { nn = e % BN; kk = e / BN; } else { nn = e / BK; kk = e % BK; }
        Bs[kk][nn] = rb[q];
      }
    }
  };
  if (kbeg < kend) {
    load_slab(kbeg);
    store_slab();
  }
  __syncthreads();
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    const bool more = k0 + BK < kend;
    if (more) load_slab(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      ACC a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + i * (BM / TM)];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bs[kk][tx + j * (BN / TN)];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
    if (more) {
      store_slab();
      __syncthreads();
    }
    if constexpr (kMix) {
      if (++slab == kMixSlabs) {
        slab = 0;
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TN; ++j) { acc64[i][j] += (double)acc[i][j]; acc[i][j] = ACC(0); }
      }
    }
  }
  if constexpr (kMix) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc64[i][j] += (double)acc[i][j];
  }

  // squared outputs: summed per thread in the accumulator type (at most TM*TN terms), then in FP64
  ACC ss_t = ACC(0);
  ACC rowss[TM];
#pragma unroll
  for (int i = 0; i < TM; ++i) rowss[i] = ACC(0);
  TC* C = static_cast<TC*>(g.C);
  const int64_t coff = z1 * g.c_bs1 + z2 * g.c_bs2;
  const int64_t xoff = z1 * g.X.bs1 + z2 * g.X.bs2;
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int64_t gm = m0 + ty + i * (BM / TM);
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int64_t gn = n0 + tx + j * (BN / TN);
      if (gm < g.M && gn < g.N) {
        double v;
        if constexpr (kMix) v = g.alpha * acc64[i][j];
        else v = g.alpha * (double)acc[i][j];
        if (g.X.p) v += g.beta * (double)ld_elem<TX>(g.X.p, xoff + gm * g.X.rs + gn * g.X.cs);
        const TC cv = (TC)v;
        if (g.norm) {
          const ACC q = (ACC)cv;
          ss_t = fma(q, q, ss_t);
          rowss[i] = fma(q, q, rowss[i]);
        }
        if (g.store && g.sym) {
          const int64_t R = sym_r + gm, Cc = sym_c + gn;  // position in the symmetric matrix
          if (R <= Cc) {
            TC* dst = C + R * g.c_rs + Cc;
            if (g.atomic) atomicAdd(dst, cv);
            else *dst = cv;
            if (R < Cc) {
              TC* mir = C + Cc * g.c_rs + R;
              if (g.atomic) atomicAdd(mir, cv);
              else *mir = cv;
            }
          }
        } else if (g.store) {
          TC* dst = C + coff + gm * g.c_rs + gn * g.c_cs;
          if (g.atomic) atomicAdd(dst, cv);
          else *dst = cv;
        }
      }
    }
  }
  if (g.norm && g.norm_rows) {
    // reduce each tile row over the BN/TN threads that share it, then one atomic per row per CTA
    __shared__ double rsum[BM];
    for (int i = tid; i < BM; i += NT) rsum[i] = 0.0;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < TM; ++i)
      if (rowss[i] != ACC(0)) atomicAdd(&rsum[ty + i * (BM / TM)], (double)rowss[i]);
    __syncthreads();
    for (int i = tid; i < BM; i += NT) {
      const int64_t gm = m0 + i;
      if (gm < g.M && rsum[i] != 0.0) atomicAdd(g.norm + gm, rsum[i]);
    }
  } else if (g.norm) {
    double ss = (double)ss_t;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if ((tid & 31) == 0 && ss != 0.0) atomicAdd(g.norm + z1, ss);
  }
}

template <typename TA, typename TB, typename TX, typename TC, typename ACC, int BM, int BN, int BK,
          int TM, int TN>
cudaError_t run(const GemmArgs& g, cudaStream_t st) {
  constexpr int NT = (BM / TM) * (BN / TN);
  const int64_t gx = (g.N + BN - 1) / BN, gy = (g.M + BM - 1) / BM;
  int ksplit = 1;
  int64_t kchunk = g.K > 0 ? g.K : 1;
  const bool zero_split = !g.atomic && g.store && g.c_zero_elems > 0 && !g.X.p && !g.norm;
  if ((g.atomic && g.allow_splitk && !g.X.p && !g.norm) || zero_split) {
    const int64_t tiles = gx * gy * g.nbatch;
    const int64_t target = 2 * 152;
    if (tiles < target && g.K > 4 * BK) {
      int64_t want = (target + tiles - 1) / tiles;
      int64_t maxs = (g.K + 4 * BK - 1) / (4 * BK);
      ksplit = (int)std::min<int64_t>(std::min<int64_t>(want, maxs), 4096);
      kchunk = (g.K + ksplit - 1) / ksplit;
      kchunk = (kchunk + BK - 1) / BK * BK;
      ksplit = (int)((g.K + kchunk - 1) / kchunk);
    }
  }
  if (gx == 0 || gy == 0 || g.nbatch == 0) return cudaSuccess;
  if (gy > 65535 || (int64_t)g.nbatch * ksplit > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)gx, (unsigned)gy, (unsigned)(g.nbatch * ksplit));
  if (zero_split && ksplit > 1) {
    // a plain-store output split over K: zero it, then every K-chunk adds its part
    const cudaError_t e = cudaMemsetAsync(g.C, 0, (size_t)g.c_zero_elems * sizeof(TC), st);
    if (e != cudaSuccess) return e;
    GemmArgs ga = g;
    ga.atomic = 1;
    note_launch();
    gemm_kernel<TA, TB, TX, TC, ACC, BM, BN, BK, TM, TN><<<grid, NT, 0, st>>>(ga, ksplit, kchunk);
    return cudaGetLastError();
  }
  note_launch();
  gemm_kernel<TA, TB, TX, TC, ACC, BM, BN, BK, TM, TN><<<grid, NT, 0, st>>>(g, ksplit, kchunk);
  return cudaGetLastError();
}

}  // namespace

template <typename TA, typename TB, typename TX, typename TC, typename ACC>
cudaError_t gemm(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.nbatch <= 0) return cudaSuccess;
  if (g.M <= 16 && g.N <= 16) return run<TA, TB, TX, TC, ACC, 16, 16, 16, 1, 1>(g, st);
  if (g.M <= 32 && g.N <= 32) return run<TA, TB, TX, TC, ACC, 32, 32, 16, 2, 2>(g, st);
  if (g.M <= 16) return run<TA, TB, TX, TC, ACC, 16, 256, 16, 2, 8>(g, st);
  if (g.M <= 32) return run<TA, TB, TX, TC, ACC, 32, 128, 16, 4, 4>(g, st);
  // a few columns (new directions, last stages): narrow tiles, no padding of N, many CTAs (which
  // matters most for FP64, at 1/64 of the FP32 rate per SM)
  if (g.N <= 4) return run<TA, TB, TX, TC, ACC, 32, 4, 16, 1, 1>(g, st);
  if (g.N <= 16 && g.M <= 4096) return run<TA, TB, TX, TC, ACC, 32, 16, 16, 2, 1>(g, st);
  if (g.N <= 16) return run<TA, TB, TX, TC, ACC, 256, 16, 16, 8, 2>(g, st);
  return run<TA, TB, TX, TC, ACC, 64, 64, 16, 4, 4>(g, st);
}

#define TT_GEMM_INST(TA, TB, TX, TC, ACC) \
  template cudaError_t gemm<TA, TB, TX, TC, ACC>(const GemmArgs&, cudaStream_t);

// FP64 path
TT_GEMM_INST(double, double, double, double, double)
TT_GEMM_INST(double, float, float, double, double)
TT_GEMM_INST(double, double, float, double, double)
TT_GEMM_INST(double, float, double, double, double)
// FP32 projections
TT_GEMM_INST(float, float, float, float, float)
TT_GEMM_INST(float, double, double, float, float)
TT_GEMM_INST(float, float, double, float, float)
TT_GEMM_INST(float, double, float, float, float)
// Gram of FP32 residuals: FP64 accumulation of exact FP64 products, or FP32 products with FP64
// accumulation across K-slabs
TT_GEMM_INST(float, float, float, double, double)
TT_GEMM_INST(float, float, float, double, float)
TT_GEMM_INST(float, float, double, double, float)
TT_GEMM_INST(float, double, double, double, double)
TT_GEMM_INST(float, double, double, double, float)
// reconstruction into FP32 outputs
TT_GEMM_INST(double, double, double, float, double)

}  // namespace ttice
