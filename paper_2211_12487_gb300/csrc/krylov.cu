// Block-Krylov basis of a residual Gram matrix in one thread-block cluster (the candidate step of
// the mixed-precision truncated eigen-solve of Eq. 9; the FP64 Rayleigh-Ritz step and its
// certification follow on the host side).
//
// Q = [X_0, ..., X_{nblk-1}] (s x 8 nblk, column-major, ld s; nblk <= 8): X_0 a given start block (a
// restart from earlier Ritz vectors) or a fixed pseudo-random one, X_i = G X_{i-1}
// projected out of the earlier blocks twice (block classical Gram-Schmidt, CGS2) and orthonormalised
// by Cholesky-QR applied twice; H = Q^T G Q (8 nblk x 8 nblk, FP64).  Products and per-CTA sums in FP32,
// sums across CTAs in FP64.
//
// One cluster of C CTAs (16 where the device allows it, else 8), all on one GPC: CTA c owns the rows
// [c nr, (c+1) nr) of every basis column and keeps them in shared memory, so every update of the
// basis is local.  Reductions over rows (the projections Q^T X_i, the block Grams, H's last block
// column) write one partial per CTA into shared memory; after a cluster barrier every CTA reads the C
// partials through distributed shared memory and sums them in rank order, so all CTAs hold
// bit-identical sums (and apply the same Cholesky factor).  G X_{i-1} reads X_{i-1} from the owners'
// shared memory in chunks, and the CTA's rows of G from shared memory when they fit (else from an
// FP32 copy in global memory that only this CTA reads).
//
// H needs no G Q product: with G X_c = Q_{<=c} Ttot + X_{c+1} Rtot (the two CGS2 coefficient blocks
// summed, and R2 R1 of the two Cholesky-QR passes), block column c of H is Ttot over the earlier
// blocks (its diagonal block symmetrised), Rtot below it, and zero further down (the block-Lanczos
// structure).  Only the last block column uses an explicit G X_{nblk-1}.
//
// Cluster barriers are hardware barriers; the kernel has no spin loop and no early exit.
#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

#include "ttice_internal.cuh"

namespace cg = cooperative_groups;

namespace ttice {
namespace {

constexpr int kKT = 256;          // threads per CTA
constexpr int kKW = kKT / 32;     // warps per CTA
constexpr int kBP = 8;            // block width
constexpr int kNBk = 8;           // blocks
constexpr int kKB = kBP * kNBk;   // basis size
constexpr int kNQ = kBP * (kBP + 1) / 2;
constexpr int kPartMax = kKB * kBP;  // the largest per-CTA partial (H's last block column)
constexpr int kChunk = 1024;         // rows of X_{i-1} staged at a time
constexpr size_t kSmemCap = 208 * 1024;

__device__ __forceinline__ double hash_uniform(uint64_t seed, int64_t i) {
  // splitmix64 of (seed, index), mapped to [-1, 1)
  uint64_t z = seed + 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z = z ^ (z >> 31);
  return (double)(z >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

__host__ __device__ inline int krylov_ldq(int nr) { return nr | 1; }

// This CTA's rows [r0, r0 + nloc) of the basis: q[col * ldq + rl] (odd ldq: conflict-free columns).
struct Loc {
  int r0, nloc, nr, ldq;
  float* q;
};

// Sum over the cluster's CTAs of entries [0, n) of the partial buffer `part` (same offset in every
// CTA's shared memory), in rank order, in FP64.  put(e, v) is called by the thread that owns e.
template <typename F>
__device__ void cluster_sum(cg::cluster_group& cl, float* part, int n, F put) {
  const unsigned int C = cl.num_blocks();
  for (int e = threadIdx.x; e < n; e += kKT) {
    double v = 0.0;
#pragma unroll 4
    for (unsigned int c = 0; c < C; ++c) v += (double)cl.map_shared_rank(part, c)[e];
    put(e, v);
  }
}

__device__ __forceinline__ int packed_upper(int a, int b) { return a * kBP - a * (a + 1) / 2 + b; }

// Block Gram X^T X of the block columns [col0, col0 + kBP) over this CTA's rows, packed upper
// triangle (kNQ entries), written to out[0 .. kNQ) by threads 0 .. kNQ-1.
__device__ void local_block_gram(Loc L, int col0, float* wsum, float* out) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float acc[kNQ];
#pragma unroll
  for (int q = 0; q < kNQ; ++q) acc[q] = 0.f;
  for (int rl = tid; rl < L.nloc; rl += kKT) {
    float x[kBP];
#pragma unroll
    for (int a = 0; a < kBP; ++a) x[a] = L.q[(col0 + a) * L.ldq + rl];
#pragma unroll
    for (int a = 0; a < kBP; ++a)
#pragma unroll
      for (int b = a; b < kBP; ++b) acc[packed_upper(a, b)] = fmaf(x[a], x[b], acc[packed_upper(a, b)]);
  }
#pragma unroll
  for (int q = 0; q < kNQ; ++q) {
    float v = acc[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) wsum[warp * kNQ + q] = v;
  }
  __syncthreads();
  if (tid < kNQ) {
    float v = 0.f;
    for (int w = 0; w < kKW; ++w) v += wsum[w * kNQ + tid];
    out[tid] = v;
  }
}

// Cholesky-QR twice of the block columns [col0, col0 + kBP) of the local rows, with the block Gram
// summed over the cluster.  Rtot (8 x 8, row-major, upper) receives R2 R1, the factor with
// X_before = X_after Rtot.  With gram_ready the first pass takes its Gram from S (upper triangle,
// S[a * kBP + b], a <= b) instead of forming and summing it.
__device__ void block_cholqr2(cg::cluster_group& cl, Loc L, int col0, float* part2, int& pp, int* lost,
                              float* wsum, double* S, float* Rt, float* Rid, float* R1, float* Rtot,
                              bool gram_ready) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto qi = [](int a, int b) { return packed_upper(a, b); };
  for (int pass = 0; pass < 2; ++pass) {
    if (!(pass == 0 && gram_ready)) {
      float* mine = part2 + pp * kPartMax;
      local_block_gram(L, col0, wsum, mine);
      cl.sync();
      cluster_sum(cl, mine, kNQ, [&](int e, double v) {
        int a = 0;
        while (e >= qi(a, kBP)) ++a;
        S[a * kBP + (e - qi(a, 0))] = v;
      });
      pp ^= 1;
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
      if (lane == 0 && bad && cl.block_rank() == 0) atomicOr(lost, 1);
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
    for (int rl = tid; rl < L.nloc; rl += kKT) {
      float x[kBP];
#pragma unroll
      for (int a = 0; a < kBP; ++a) x[a] = L.q[(col0 + a) * L.ldq + rl];
#pragma unroll
      for (int c = 0; c < kBP; ++c) {
        float v = x[c];
#pragma unroll
        for (int a = 0; a < c; ++a) v = fmaf(-x[a], Rt[a * kBP + c], v);
        x[c] = v * Rid[c];
      }
#pragma unroll
      for (int c = 0; c < kBP; ++c) L.q[(col0 + c) * L.ldq + rl] = x[c];
    }
    __syncthreads();
  }
}

// out[a * ldo + rl] = sum_k G[r0 + rl, k] X[k, a] for this CTA's rows, with X = the block columns
// [cprev, cprev + kBP) of the basis, read from the owners' shared memory in chunks of kChunk rows.
// Four rows per warp, so that every staged X value feeds four rows.
__device__ void g_times_block(cg::cluster_group& cl, Loc L, int s, int cprev, const float* gbase, int64_t gld,
                              float* xs, float* out, int ldo) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int e = tid; e < L.nloc * kBP; e += kKT) {
    const int a = e / L.nloc, rl = e - a * L.nloc;
    out[a * ldo + rl] = 0.f;
  }
  for (int k0 = 0; k0 < s; k0 += kChunk) {
    const int kc = min(kChunk, s - k0);
    __syncthreads();
    for (int e = tid; e < kc * kBP; e += kKT) {
      const int a = e / kc, k = e - a * kc;
      const int row = k0 + k, owner = row / L.nr;
      const float* rq = cl.map_shared_rank(L.q, (unsigned int)owner);
      xs[a * kc + k] = rq[(cprev + a) * L.ldq + (row - owner * L.nr)];
    }
    __syncthreads();
    for (int rb = warp * 4; rb < L.nloc; rb += kKW * 4) {
      float acc[4][kBP];
#pragma unroll
      for (int t = 0; t < 4; ++t)
#pragma unroll
        for (int a = 0; a < kBP; ++a) acc[t][a] = 0.f;
      const float* g[4];
#pragma unroll
      for (int t = 0; t < 4; ++t) g[t] = gbase + (int64_t)min(rb + t, L.nloc - 1) * gld + k0;
#pragma unroll 2
      for (int k = lane; k < kc; k += 32) {
        float x[kBP];
#pragma unroll
        for (int a = 0; a < kBP; ++a) x[a] = xs[a * kc + k];
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
          if (rb + t < L.nloc) {
#pragma unroll
            for (int a = 0; a < kBP; ++a) out[a * ldo + rb + t] += acc[t][a];
          }
      }
    }
  }
  __syncthreads();
}

// Shared memory (floats): xs min(s, kChunk)*kBP | q kKB*ldq | gx kBP*ldq | part 2*kPartMax |
// gslab nr*(s+4)
struct KrylovShape {
  int C;
  int nr;
  int gslab;
  size_t smem;
};

size_t krylov_base_floats(int s, int nr) {
  const int kc = s < kChunk ? s : kChunk;
  return (size_t)kc * kBP + (size_t)(kKB + kBP) * krylov_ldq(nr) + 2 * (size_t)kPartMax;
}

// nblk (1 .. kNBk) blocks: a basis of kk = nblk kBP vectors and H of kk x kk (row-major, ld kk).
// X_0 is start (s x kBP, column-major, ld s) when given, else the pseudo-random block of `seed`.
__global__ void __launch_bounds__(kKT) krylov_kernel(const double* G, float* G32, int s, float* Q,
                                                     double* H, int* lost, uint64_t seed, int gslab,
                                                     int nblk, const float* start) {
  extern __shared__ __align__(16) float sm[];
  __shared__ float wsum[kKW * kNQ];
  __shared__ double S[kBP * kBP];
  __shared__ float Rt[kBP * kBP], Rid[kBP], R1[kBP * kBP], Rtot[kBP * kBP];
  __shared__ float T[(kKB - kBP) * kBP], Ttot[kKB * kBP];
  __shared__ double Td[(kKB - kBP) * kBP], Sp[kNQ];  // second-pass coefficients, Gram before it
  cg::cluster_group cl = cg::this_cluster();
  const int tid = threadIdx.x;
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  Loc L;
  L.nr = (s + C - 1) / C;
  L.r0 = min(s, rank * L.nr);
  L.nloc = min(s, L.r0 + L.nr) - L.r0;
  L.ldq = krylov_ldq(L.nr);
  const int kcmax = min(s, kChunk);
  float* xs = sm;                                   // kChunk x kBP staging
  L.q = xs + (size_t)kcmax * kBP;                   // kKB x ldq local rows of Q
  float* gx = L.q + (size_t)kKB * L.ldq;            // kBP x ldq local rows of G X_7
  float* part2 = gx + (size_t)kBP * L.ldq;          // 2 x kPartMax partial sums (ping-pong)
  float* gs = part2 + 2 * kPartMax;                 // nr x (s + 4) rows of G (gslab)
  const int nloc = L.nloc;
  int pp = 0;
  const int64_t gld = gslab ? (int64_t)s + 4 : (int64_t)s;
  const float* gbase = gslab ? gs : G32 + (int64_t)L.r0 * s;
  const bool writer = rank == 0;  // every CTA holds the same coefficients; rank 0 writes H
  const int kk = nblk * kBP;      // basis size; H is kk x kk with leading dimension kk

  // FP32 rows of G; this CTA's rows of the start block
  for (int64_t e = tid; e < (int64_t)nloc * s; e += kKT) {
    const int rl = (int)(e / s), k = (int)(e - (int64_t)rl * s);
    const float v = (float)G[(int64_t)(L.r0 + rl) * s + k];
    if (gslab) gs[rl * gld + k] = v;
    else G32[(int64_t)(L.r0 + rl) * s + k] = v;
  }
  for (int e = tid; e < nloc * kBP; e += kKT) {
    const int a = e / nloc, rl = e - a * nloc;
    const int64_t i = (int64_t)a * s + L.r0 + rl;
    L.q[a * L.ldq + rl] = start ? start[i] : (float)hash_uniform(seed, i);
  }
  if (writer)
    for (int e = tid; e < kk * kk; e += kKT) H[e] = 0.0;
  __syncthreads();
  block_cholqr2(cl, L, 0, part2, pp, lost, wsum, S, Rt, Rid, R1, Rtot, false);

  for (int blk = 1; blk <= nblk; ++blk) {
    cl.sync();  // every CTA's rows of X_{blk-1} are final
    const int cprev = (blk - 1) * kBP, ccur = blk * kBP;
    if (blk == nblk) {
      // last block column of H: X_j^T (G X_last) for every block j, from an explicit G X_last
      g_times_block(cl, L, s, cprev, gbase, gld, xs, gx, L.ldq);
      float* mine = part2 + pp * kPartMax;
      for (int e = tid; e < kk * kBP; e += kKT) {
        const int a = e / kBP, j = e - a * kBP;
        const float* qa = L.q + a * L.ldq;
        const float* gj = gx + j * L.ldq;
        float v = 0.f;
        for (int rl = 0; rl < nloc; ++rl) v = fmaf(qa[rl], gj[rl], v);
        mine[e] = v;
      }
      cl.sync();
      if (writer) {
        cluster_sum(cl, mine, kk * kBP, [&](int e, double v) {
          const int a = e / kBP, j = e - a * kBP;
          const int col = cprev + j;
          if (a < cprev) { H[a * kk + col] = v; H[col * kk + a] = v; }
          else Ttot[(a - cprev) * kBP + j] = (float)v;
        });
        __syncthreads();
        for (int e = tid; e < kBP * kBP; e += kKT) {  // symmetrised diagonal block
          const int a = e / kBP, j = e - a * kBP;
          H[(cprev + a) * kk + cprev + j] = 0.5 * ((double)Ttot[a * kBP + j] + (double)Ttot[j * kBP + a]);
        }
      }
      break;
    }
    // X_blk = G X_{blk-1} on this CTA's rows
    g_times_block(cl, L, s, cprev, gbase, gld, xs, L.q + ccur * L.ldq, L.ldq);
    // X_blk -= Q_prev (Q_prev^T X_blk), twice; Ttot accumulates the two coefficient blocks.  The
    // second pass's sum also carries the block Gram of X_blk before that pass, from which the Gram
    // after it follows exactly (Q_prev orthonormal): X''^T X'' = X'^T X' - T2^T T2.  T2 is the
    // second pass's small correction, so the difference loses nothing, and the first Cholesky-QR
    // pass needs no sum of its own.
    const int nq = ccur;
    for (int e = tid; e < nq * kBP; e += kKT) Ttot[e] = 0.f;
    for (int pass = 0; pass < 2; ++pass) {
      float* mine = part2 + pp * kPartMax;
      for (int e = tid; e < nq * kBP; e += kKT) {
        const int a = e / kBP, j = e - a * kBP;
        const float* qa = L.q + a * L.ldq;
        const float* xj = L.q + (ccur + j) * L.ldq;
        float v = 0.f;
        for (int rl = 0; rl < nloc; ++rl) v = fmaf(qa[rl], xj[rl], v);
        mine[e] = v;
      }
      if (pass == 1) local_block_gram(L, ccur, wsum, mine + nq * kBP);
      cl.sync();
      cluster_sum(cl, mine, nq * kBP + (pass == 1 ? kNQ : 0), [&](int e, double v) {
        if (e < nq * kBP) {
          T[e] = (float)v;
          Ttot[e] += (float)v;
          Td[e] = v;
        } else {
          Sp[e - nq * kBP] = v;
        }
      });
      pp ^= 1;
      __syncthreads();
      if (pass == 1 && tid < kNQ) {
        int a = 0;
        while (tid >= packed_upper(a, kBP)) ++a;
        const int b = tid - packed_upper(a, 0);
        double v = Sp[tid];
        for (int c = 0; c < nq; ++c) v -= Td[c * kBP + a] * Td[c * kBP + b];
        S[a * kBP + b] = v;
      }
      for (int e = tid; e < nloc * kBP; e += kKT) {
        const int j = e / nloc, rl = e - j * nloc;
        float v = L.q[(ccur + j) * L.ldq + rl];
        for (int a = 0; a < nq; ++a) v = fmaf(-L.q[a * L.ldq + rl], T[a * kBP + j], v);
        L.q[(ccur + j) * L.ldq + rl] = v;
      }
      __syncthreads();
    }
    block_cholqr2(cl, L, ccur, part2, pp, lost, wsum, S, Rt, Rid, R1, Rtot, true);
    // block column blk-1 of H (G X_{blk-1} = Q_prev Ttot + X_blk Rtot): rows of the earlier blocks from
    // Ttot (diagonal block symmetrised), block blk from Rtot, zero below
    if (writer) {
      for (int e = tid; e < nq * kBP; e += kKT) {
        const int a = e / kBP, j = e - a * kBP;
        const int col = cprev + j;
        if (a < cprev) {
          H[a * kk + col] = (double)Ttot[e];
          H[col * kk + a] = (double)Ttot[e];
        } else {
          const int aa = a - cprev;
          H[a * kk + col] = 0.5 * ((double)Ttot[e] + (double)Ttot[(cprev + j) * kBP + aa]);
        }
      }
      for (int e = tid; e < kBP * kBP; e += kKT) {
        const int a = e / kBP, j = e - a * kBP;  // X_blk^T G X_{blk-1} = Rtot
        H[(ccur + a) * kk + cprev + j] = (double)Rtot[e];
        H[(cprev + j) * kk + ccur + a] = (double)Rtot[e];
      }
    }
  }
  // the basis for the host; no CTA leaves while another may still read its shared memory
  for (int e = tid; e < nloc * kk; e += kKT) {
    const int a = e / nloc, rl = e - a * nloc;
    Q[(int64_t)a * s + L.r0 + rl] = L.q[a * L.ldq + rl];
  }
  cl.sync();
}

KrylovShape krylov_shape(int s, int C) {
  KrylovShape k;
  k.C = C;
  k.nr = (s + C - 1) / C;
  const size_t base = krylov_base_floats(s, k.nr);
  const size_t slab = (size_t)k.nr * ((size_t)s + 4);
  k.gslab = (base + slab) * sizeof(float) <= kSmemCap;
  k.smem = (base + (k.gslab ? slab : 0)) * sizeof(float);
  return k;
}

}  // namespace

cudaError_t launch_krylov(const double* G, float* G32, int64_t s, int nblk, float* Q, double* H,
                          int* lost, uint64_t seed, const float* start, cudaStream_t st) {
  static_assert(kKB == 64, "the caller's buffers hold up to a 64-vector basis");
  if (s < kKB || nblk < 2 || nblk > kNBk) return cudaErrorInvalidValue;
  // cluster size: 16 CTAs where the device allows that many (non-portable), else 8
  static std::once_flag once;
  static cudaError_t setup_err = cudaSuccess;
  static int cluster = 8;
  std::call_once(once, [] {
    setup_err = cudaFuncSetAttribute(krylov_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemCap);
    if (setup_err != cudaSuccess) return;
    if (cudaFuncSetAttribute(krylov_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 16;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(kKT);
      cfg.dynamicSmemBytes = kSmemCap;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int n = 0;
      if (cudaOccupancyMaxActiveClusters(&n, krylov_kernel, &cfg) == cudaSuccess && n >= 1) cluster = 16;
    }
    (void)cudaGetLastError();  // a refused query leaves no error behind
  });
  TT_CUDA(setup_err);
  const KrylovShape ks = krylov_shape((int)s, cluster);
  if (ks.smem > kSmemCap) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)ks.C;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)ks.C);
  cfg.blockDim = dim3(kKT);
  cfg.dynamicSmemBytes = ks.smem;
  cfg.stream = st;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  note_launch();
  return cudaLaunchKernelEx(&cfg, krylov_kernel, G, G32, (int)s, Q, H, lost, seed, ks.gslab, nblk, start);
}

}  // namespace ttice
