// Block-Krylov basis of a residual Gram matrix in one cooperative launch (the candidate step of the
// mixed-precision truncated eigen-solve of Eq. 9; the FP64 Rayleigh-Ritz step and its certification
// follow on the host side).
//
// Q = [X_0, ..., X_7] (s x 64, column-major, ld s): X_0 a fixed pseudo-random block, X_i = G X_{i-1}
// projected out of the earlier blocks twice (block classical Gram-Schmidt, CGS2) and orthonormalised
// by Cholesky-QR applied twice; then H = Q^T G Q (64 x 64, FP64 output).  G is the FP64 Gram; the
// kernel keeps an FP32 copy (products and per-CTA sums in FP32, cross-CTA sums in FP64).
//
// Layout of the work: P CTAs, CTA c owns the rows [c nr, (c+1) nr) of every basis column, so every
// update of the basis is row-local.  Each reduction over rows (the projections Q^T X_i, the block
// Grams X_i^T X_i, H) writes one partial per CTA into a ping-pong buffer; after a grid barrier every
// CTA sums the P partials itself, in CTA order, so all CTAs hold bit-identical sums (and apply the
// same Cholesky factor) and the result does not depend on scheduling.  G X_{i-1} stages X_{i-1} in
// shared memory and reads G rows from L2.
//
// Grid barriers are bounded: a CTA that waits longer than kSpinLimit polls (or sees the error flag
// another CTA raised) sets the flag and returns; the host reports TTICE_ETIMEOUT.  The launch is
// cooperative, so all CTAs are resident.
#include <algorithm>
#include <mutex>

#include "ttice_internal.cuh"

namespace ttice {
namespace {

constexpr int kKT = 256;          // threads per CTA
constexpr int kKW = kKT / 32;     // warps per CTA
constexpr int kBP = 8;            // block width
constexpr int kNBk = 8;           // blocks
constexpr int kKB = kBP * kNBk;   // basis size
constexpr int kNQ = kBP * (kBP + 1) / 2;
constexpr int kSlot = kKB * kKB;  // floats per CTA in a partial buffer (the largest partial is H's)
constexpr int kMaxP = 128;
constexpr long long kSpinLimit = 1ll << 22;

__device__ __forceinline__ double hash_uniform(uint64_t seed, int64_t i) {
  // splitmix64 of (seed, index), mapped to [-1, 1)
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// Sense-free counting barrier over the whole grid.  sync[0] = arrivals, sync[1] = generation,
// sync[2] = error flag.  Returns false (in every thread of the CTA) on timeout or error.
__device__ bool grid_barrier(unsigned int* sync, unsigned int nblocks) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = sync + 1;
    volatile int* verr = reinterpret_cast<volatile int*>(sync + 2);
    int ok = 1;
    const unsigned int g = *vgen;
    __threadfence();
    if (atomicAdd(sync, 1u) == nblocks - 1) {
      atomicExch(sync, 0u);
      __threadfence();
      atomicAdd(sync + 1, 1u);
    } else {
      long long it = 0;
      while (*vgen == g) {
        if (*verr != 0) { ok = 0; break; }
        if (++it > kSpinLimit) { atomicExch(reinterpret_cast<int*>(sync + 2), 1); ok = 0; break; }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*verr != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

struct Rows {
  int r0, r1;
};

// Cholesky-QR twice of the block columns [col0, col0 + kBP) restricted to this CTA's rows, with the
// block Gram summed over all CTAs.  Rtot (8 x 8, row-major, upper) receives R2 R1, the factor with
// X_before = X_after Rtot.  Returns false if a barrier failed.
__device__ bool block_cholqr2(float* Q, int s, int col0, Rows rw, float* part, int& pp, unsigned int* sync,
                              int* lost, float* wsum, double* S, float* Rt, float* Rid, float* R1,
                              float* Rtot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const unsigned int P = gridDim.x;
  auto qi = [](int a, int b) { return a * kBP - a * (a + 1) / 2 + b; };
  for (int pass = 0; pass < 2; ++pass) {
    float acc[kNQ];
#pragma unroll
    for (int q = 0; q < kNQ; ++q) acc[q] = 0.f;
    for (int r = rw.r0 + tid; r < rw.r1; r += kKT) {
      float x[kBP];
#pragma unroll
      for (int a = 0; a < kBP; ++a) x[a] = Q[(int64_t)(col0 + a) * s + r];
#pragma unroll
      for (int a = 0; a < kBP; ++a)
#pragma unroll
        for (int b = a; b < kBP; ++b) acc[qi(a, b)] = fmaf(x[a], x[b], acc[qi(a, b)]);
    }
#pragma unroll
    for (int q = 0; q < kNQ; ++q) {
      float v = acc[q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (lane == 0) wsum[warp * kNQ + q] = v;
    }
    __syncthreads();
    float* mine = part + ((int64_t)pp * P + blockIdx.x) * kSlot;
    if (tid < kNQ) {
      float v = 0.f;
      for (int w = 0; w < kKW; ++w) v += wsum[w * kNQ + tid];
      mine[tid] = v;
    }
    if (!grid_barrier(sync, P)) return false;
    const float* all = part + (int64_t)pp * P * kSlot;
    pp ^= 1;
    if (tid < kNQ) {
      double v = 0.0;
      for (unsigned int c = 0; c < P; ++c) v += (double)__ldcg(all + (int64_t)c * kSlot + tid);
      int a = 0;
      while (tid >= qi(a, kBP)) ++a;
      S[a * kBP + (tid - qi(a, 0))] = v;
    }
    __syncthreads();
    if (warp == 0) {
      // right-looking Cholesky, lane c keeps column c of the upper triangle
      double col[kBP];
#pragma unroll
      for (int k = 0; k < kBP; ++k) col[k] = (lane < kBP && k <= lane) ? S[k * kBP + lane] : 0.0;
      int bad = 0;
      double my_inv = 0.0;
#pragma unroll
      for (int j = 0; j < kBP; ++j) {
        double d = __shfl_sync(0xffffffffu, col[j], j);
        if (!(d > 0.0)) { bad = 1; d = 1.0; }
        const double rjj = sqrt(d), inv = 1.0 / rjj;
        if (lane == j) { col[j] = rjj; my_inv = inv; }
        else if (lane > j) col[j] *= inv;
#pragma unroll
        for (int k = j + 1; k < kBP; ++k) {
          const double rjk = __shfl_sync(0xffffffffu, col[j], k);
          if (lane >= k && lane < kBP) col[k] = fma(-rjk, col[j], col[k]);
        }
      }
      if (lane < kBP) {
#pragma unroll
        for (int k = 0; k < kBP; ++k) Rt[k * kBP + lane] = (k <= lane) ? (float)col[k] : 0.f;
        Rid[lane] = (float)my_inv;
      }
      if (lane == 0 && bad && blockIdx.x == 0) atomicOr(lost, 1);
    }
    __syncthreads();
    if (pass == 0) {
      if (tid < kBP * kBP) R1[tid] = Rt[tid];
    } else if (tid < kBP * kBP) {
      const int i = tid / kBP, j = tid % kBP;  // (R2 R1)_ij, both upper triangular
      float v = 0.f;
      for (int k = i; k <= j; ++k) v = fmaf(Rt[i * kBP + k], R1[k * kBP + j], v);
      Rtot[tid] = v;
    }
    for (int r = rw.r0 + tid; r < rw.r1; r += kKT) {
      float x[kBP];
#pragma unroll
      for (int a = 0; a < kBP; ++a) x[a] = Q[(int64_t)(col0 + a) * s + r];
#pragma unroll
      for (int c = 0; c < kBP; ++c) {
        float v = x[c];
#pragma unroll
        for (int a = 0; a < c; ++a) v = fmaf(-x[a], Rt[a * kBP + c], v);
        x[c] = v * Rid[c];
      }
#pragma unroll
      for (int c = 0; c < kBP; ++c) Q[(int64_t)(col0 + c) * s + r] = x[c];
    }
    __syncthreads();
  }
  return true;
}

// Y[rl, a] = sum_k G[r0 + rl, k] X[k, a] for this CTA's rows (X staged in xs, s x kBP column-major),
// four rows per warp so that every staged X value feeds four rows.  G rows come from the shared slab
// (ld gld) or from the FP32 copy in global memory.  out(rl, a, v) stores the result.
template <typename Out>
__device__ void g_times_block(const float* gbase, int64_t gld, const float* xs, int s, int nloc, Out out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int rb = warp * 4; rb < nloc; rb += kKW * 4) {
    float acc[4][kBP];
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int a = 0; a < kBP; ++a) acc[t][a] = 0.f;
    const float* g[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) g[t] = gbase + (int64_t)min(rb + t, nloc - 1) * gld;
#pragma unroll 2
    for (int k = lane; k < s; k += 32) {
      float x[kBP];
#pragma unroll
      for (int a = 0; a < kBP; ++a) x[a] = xs[a * s + k];
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const float gv = g[t][k];
#pragma unroll
        for (int a = 0; a < kBP; ++a) acc[t][a] = fmaf(gv, x[a], acc[t][a]);
      }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t)
#pragma unroll
      for (int a = 0; a < kBP; ++a) {
        float v = acc[t][a];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        acc[t][a] = v;
      }
    if (lane == 0) {
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (rb + t < nloc) {
#pragma unroll
          for (int a = 0; a < kBP; ++a) out(rb + t, a, acc[t][a]);
        }
    }
  }
}

// gslab != 0: this CTA's rows of G are kept in shared memory (ld s + 4) for the whole kernel;
// otherwise they are streamed from the FP32 copy G32 (written here, read only by the same CTA).
__global__ void __launch_bounds__(kKT) krylov_kernel(const double* G, float* G32, int s, float* Q,
                                                     float* part, double* H, unsigned int* sync,
                                                     int* lost, uint64_t seed, int gslab) {
  extern __shared__ __align__(16) float sm[];
  __shared__ float wsum[kKW * kNQ];
  __shared__ double S[kBP * kBP];
  __shared__ float Rt[kBP * kBP], Rid[kBP], R1[kBP * kBP], Rtot[kBP * kBP];
  __shared__ float T[(kKB - kBP) * kBP], Ttot[kKB * kBP];
  const int tid = threadIdx.x;
  const unsigned int P = gridDim.x;
  const int nr = (s + (int)P - 1) / (int)P;
  Rows rw;
  rw.r0 = min(s, (int)blockIdx.x * nr);
  rw.r1 = min(s, rw.r0 + nr);
  const int nloc = rw.r1 - rw.r0;
  int pp = 0;
  float* xs = sm;                          // s x kBP staging of the previous block
  float* gs = sm + (int64_t)s * kBP;       // nr x (s + 4) slab of G rows (gslab)
  const int64_t gld = gslab ? (int64_t)s + 4 : (int64_t)s;
  const float* gbase = gslab ? gs : G32 + (int64_t)rw.r0 * s;
  const bool writer = blockIdx.x == 0;     // every CTA holds the same coefficients; CTA 0 writes H

  // FP32 rows of G; this CTA's rows of the start block
  for (int64_t e = tid; e < (int64_t)nloc * s; e += kKT) {
    const int rl = (int)(e / s), k = (int)(e - (int64_t)rl * s);
    const float v = (float)G[(int64_t)(rw.r0 + rl) * s + k];
    if (gslab) gs[rl * gld + k] = v;
    else G32[(int64_t)(rw.r0 + rl) * s + k] = v;
  }
  for (int e = tid; e < nloc * kBP; e += kKT) {
    const int r = rw.r0 + e % nloc, a = e / nloc;
    const int64_t i = (int64_t)a * s + r;
    Q[i] = (float)hash_uniform(seed, i);
  }
  if (writer)
    for (int e = tid; e < kKB * kKB; e += kKT) H[e] = 0.0;
  __syncthreads();
  if (!block_cholqr2(Q, s, 0, rw, part, pp, sync, lost, wsum, S, Rt, Rid, R1, Rtot)) return;

  for (int blk = 1; blk <= kNBk; ++blk) {
    // every CTA's rows of X_{blk-1} are final
    if (!grid_barrier(sync, P)) return;
    const int cprev = (blk - 1) * kBP, ccur = blk * kBP;
    for (int e = tid; e < s * kBP; e += kKT) {
      const int a = e / s, k = e - a * s;
      xs[e] = __ldcg(Q + (int64_t)(cprev + a) * s + k);
    }
    __syncthreads();
    if (blk == kNBk) {
      // last block column of H: X_j^T (G X_7) for every block j, from an explicit G X_7
      float* gx = xs + (int64_t)s * kBP;  // nloc x kBP after the staging (gslab: reuse the tail)
      if (gslab) gx = gs + (int64_t)nr * gld;
      g_times_block(gbase, gld, xs, s, nloc, [&](int rl, int a, float v) { gx[rl * kBP + a] = v; });
      __syncthreads();
      float* mine = part + ((int64_t)pp * P + blockIdx.x) * kSlot;
      for (int e = tid; e < kKB * kBP; e += kKT) {
        const int a = e / kBP, j = e - a * kBP;
        const float* qa = Q + (int64_t)a * s + rw.r0;
        float v = 0.f;
        for (int rl = 0; rl < nloc; ++rl) v = fmaf(qa[rl], gx[rl * kBP + j], v);
        mine[e] = v;
      }
      if (!grid_barrier(sync, P)) return;
      if (writer) {
        const float* all = part + (int64_t)pp * P * kSlot;
        for (int e = tid; e < kKB * kBP; e += kKT) {
          const int a = e / kBP, j = e - a * kBP;
          double v = 0.0;
          for (unsigned int c = 0; c < P; ++c) v += (double)__ldcg(all + (int64_t)c * kSlot + e);
          const int col = cprev + j;
          if (a < cprev) { H[a * kKB + col] = v; H[col * kKB + a] = v; }
          else Ttot[(a - cprev) * kBP + j] = (float)v;
        }
        __syncthreads();
        for (int e = tid; e < kBP * kBP; e += kKT) {  // symmetrised diagonal block
          const int a = e / kBP, j = e - a * kBP;
          H[(cprev + a) * kKB + cprev + j] = 0.5 * ((double)Ttot[a * kBP + j] + (double)Ttot[j * kBP + a]);
        }
      }
      break;
    }
    // X_blk = G X_{blk-1} on this CTA's rows
    g_times_block(gbase, gld, xs, s, nloc, [&](int rl, int a, float v) {
      Q[(int64_t)(ccur + a) * s + rw.r0 + rl] = v;
    });
    __syncthreads();
    // X_blk -= Q_prev (Q_prev^T X_blk), twice; Ttot accumulates the two coefficient blocks
    const int nq = ccur;
    for (int e = tid; e < nq * kBP; e += kKT) Ttot[e] = 0.f;
    for (int pass = 0; pass < 2; ++pass) {
      float* mine = part + ((int64_t)pp * P + blockIdx.x) * kSlot;
      for (int e = tid; e < nq * kBP; e += kKT) {
        const int a = e / kBP, j = e - a * kBP;
        const float* qa = Q + (int64_t)a * s + rw.r0;
        const float* xj = Q + (int64_t)(ccur + j) * s + rw.r0;
        float v = 0.f;
        for (int rl = 0; rl < nloc; ++rl) v = fmaf(qa[rl], xj[rl], v);
        mine[e] = v;
      }
      if (!grid_barrier(sync, P)) return;
      const float* all = part + (int64_t)pp * P * kSlot;
      pp ^= 1;
      for (int e = tid; e < nq * kBP; e += kKT) {
        double v = 0.0;
        for (unsigned int c = 0; c < P; ++c) v += (double)__ldcg(all + (int64_t)c * kSlot + e);
        T[e] = (float)v;
        Ttot[e] += (float)v;
      }
      __syncthreads();
      for (int e = tid; e < nloc * kBP; e += kKT) {
        const int j = e / nloc, r = rw.r0 + (e - j * nloc);
        float v = Q[(int64_t)(ccur + j) * s + r];
        for (int a = 0; a < nq; ++a) v = fmaf(-Q[(int64_t)a * s + r], T[a * kBP + j], v);
        Q[(int64_t)(ccur + j) * s + r] = v;
      }
      __syncthreads();
    }
    if (!block_cholqr2(Q, s, ccur, rw, part, pp, sync, lost, wsum, S, Rt, Rid, R1, Rtot)) return;
    // block column blk-1 of H (G X_{blk-1} = Q_prev Ttot + X_blk Rtot): rows of the earlier blocks from
    // Ttot (diagonal block symmetrised), block blk from Rtot, zero below
    if (writer) {
      for (int e = tid; e < nq * kBP; e += kKT) {
        const int a = e / kBP, j = e - a * kBP;
        const int col = cprev + j;
        if (a < cprev) {
          H[a * kKB + col] = (double)Ttot[e];
          H[col * kKB + a] = (double)Ttot[e];
        } else {
          const int aa = a - cprev;
          H[a * kKB + col] = 0.5 * ((double)Ttot[e] + (double)Ttot[(cprev + j) * kBP + aa]);
        }
      }
      for (int e = tid; e < kBP * kBP; e += kKT) {
        const int a = e / kBP, j = e - a * kBP;  // X_blk^T G X_{blk-1} = Rtot
        H[(ccur + a) * kKB + cprev + j] = (double)Rtot[e];
        H[(cprev + j) * kKB + ccur + a] = (double)Rtot[e];
      }
    }
  }
}

int krylov_ctas(int s) { return std::min(kMaxP, std::max(4, (s + 31) / 32)); }

// launch shape: P CTAs and whether the G slab fits in shared memory (with the block staging and
// the explicit G X_7 rows)
struct KrylovShape {
  int P;
  int gslab;
  size_t smem;
};

KrylovShape krylov_shape(int s) {
  constexpr size_t kCap = 200 * 1024 / sizeof(float);
  KrylovShape k;
  const size_t stage = (size_t)s * kBP;
  for (int P = krylov_ctas(s); P <= kMaxP; ++P) {
    const size_t nr = (size_t)(s + P - 1) / P;
    const size_t need = stage + nr * ((size_t)s + 4) + nr * kBP;
    if (need <= kCap) {
      k.P = P; k.gslab = 1; k.smem = need * sizeof(float);
      return k;
    }
  }
  k.P = krylov_ctas(s);
  const size_t nr = (size_t)(s + k.P - 1) / k.P;
  k.gslab = 0;
  k.smem = (stage + nr * kBP) * sizeof(float);
  return k;
}

}  // namespace

int64_t krylov_part_floats() { return 2ll * kMaxP * kSlot; }

cudaError_t launch_krylov(const double* G, float* G32, int64_t s, float* Q, float* part, double* H,
                          unsigned int* sync, int* lost, uint64_t seed, cudaStream_t st) {
  static_assert(kKB == 64, "the caller's buffers hold a 64-vector basis");
  if (s < kKB) return cudaErrorInvalidValue;
  const KrylovShape ks = krylov_shape((int)s);
  if (ks.smem > 200 * 1024) return cudaErrorInvalidValue;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  static int max_resident = 0;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(krylov_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    int dev = 0, sms = 0, per_sm = 0;
    if (attr_err == cudaSuccess) attr_err = cudaGetDevice(&dev);
    if (attr_err == cudaSuccess) attr_err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (attr_err == cudaSuccess)
      attr_err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, krylov_kernel, kKT, 200 * 1024);
    max_resident = sms * per_sm;
  });
  TT_CUDA(attr_err);
  if (ks.P > max_resident) return cudaErrorCooperativeLaunchTooLarge;
  TT_CUDA(cudaMemsetAsync(sync, 0, 3 * sizeof(unsigned int), st));
  int si = (int)s, slab = ks.gslab;
  void* args[] = {(void*)&G, (void*)&G32, (void*)&si, (void*)&Q, (void*)&part, (void*)&H,
                  (void*)&sync, (void*)&lost, (void*)&seed, (void*)&slab};
  note_launch();
  return cudaLaunchCooperativeKernel((const void*)krylov_kernel, dim3(ks.P), dim3(kKT), args, ks.smem, st);
}

}  // namespace ttice
