// Projection of a batch onto a core on the tensor cores: W(z) = U^T X(z) for every observation z of
// a stage of the chain (Eq. 6 for stage 1, Eq. 12 for the later stages), with the per-observation
// norms of the input and of the projection, whose difference is the stage's squared residual
// ||X(z) - U W(z)||^2 = ||X(z)||^2 - ||W(z)||^2 for an orthonormal U (Pythagoras).
//
// Shapes.  X(z) is m x L, row-major (the stage-i unfolding, L columns per observation, observation-
// major); U is m x r, column-major; W(z) is r x L, row-major.  One work item is a tile of 128
// consecutive columns of one observation (the MMA's M, one tensor-memory lane per column) against
// one N tile of NT output rows (MMA N, 64 or 128); K = m runs in chunks of 32 rows (one 128-byte
// swizzle row of TF32).
//
// Arithmetic.  Each operand is split into a TF32 head and a TF32 tail (x_hi = tf32(x), x_lo =
// tf32(x - x_hi), both rounded to nearest, so the MMA reads them exactly; x_hi + x_lo carries
// ~2^-22 relative error), and each K step issues A_hi B_hi into a main accumulator and A_lo B_hi +
// A_hi B_lo into a cross accumulator (the dropped tail product is ~2^-22 relative), FP32 in tensor
// memory.  Every add into a tensor-memory accumulator carries a rounding biased towards zero (about
// half an ulp, measured through the per-observation residuals), so the main accumulator adds K in
// 32-long segments (4 adds; one segment when K <= 256) that the epilogue sums into FP32 registers
// with round-to-nearest, from a ring of segment accumulators so that the MMAs run ahead of the
// epilogue; the cross products, ~2^-11 of the main ones, keep one accumulator per item.  W is then
// at FP32 accuracy up to that bias, which grows like sqrt(K / 32) ulps (~3e-6 relative at K = 2e4);
// the Pythagorean residual ||X||^2 - ||W||^2 inherits it multiplied by ||X||^2 / ||R||^2.  With
// nprod = 1 (the TF32 mode of the path) only A_hi B_hi is taken: no tail operands are copied or
// written and the cross accumulator stays unused, so W carries the TF32 rounding of both operands
// (2^-11 relative each, unbiased).  The
// head/tail pair of U is kept in global memory next to the core (ttice_s::Uh, Ul) and copied
// straight into the 128-byte-swizzled K-major B operand by TMA; X is staged raw by TMA and split by
// converter warps, which write the K-major A operand.
//
// Roles (14 warps, one persistent CTA per SM):
//   warps 0-3  converters: thread = tile column; split 32 values per chunk into the A operand and
//              sum x^2 of the column;
//   warps 4-11 epilogue: thread = tensor-memory lane = tile column, two warps per lane quarter, each
//              holding half of the N tile in registers: add every segment's main accumulator, then
//              the cross accumulator, store W and sum w^2;
//   warp 12    one lane issues the TMA copies (X chunk, U head and tail chunk);
//   warp 13    allocates tensor memory; one lane issues the MMAs, committing each chunk to the
//              barriers that free its A and B slots, and each segment to its accumulator's barrier
//              (a ring of 6 main and 2 cross accumulators at N = 64, 3 and 1 at N = 128).
// Every wait is bounded in time (the limit is a launch argument); on expiry the waiting thread
// raises a CTA-wide abort flag, every role leaves its loop, the MMA lane waits for the MMAs it
// issued and the producer for its copies in flight, tensor memory is freed and `status` records the
// failure.
#include <algorithm>
#include <mutex>

#include "tc_common.cuh"
#include "ttice_internal.cuh"

namespace ttice {
namespace {

using namespace tc;

constexpr int kTile = 128;   // columns per item (MMA M)
constexpr int kChunk = 32;   // K rows per staged chunk
constexpr int kConvWarps = 4, kEpiWarps = 8;  // epilogue: two warps per 32-lane quarter, half the N tile each
constexpr int kProducerWarp = kConvWarps + kEpiWarps, kMmaWarp = kProducerWarp + 1;
constexpr int kThreads = (kMmaWarp + 1) * 32;
constexpr uint32_t kRawBytes = kChunk * kTile * 4;  // 16 KB
constexpr uint32_t kABytes = kTile * kChunk * 4;    // 16 KB per half (head or tail)
// ring depths of the main-accumulator segments and of the per-item cross accumulator in tensor
// memory (SEGB + CB accumulators of NT columns <= 512)
// With the converters (raw A), the A operand lives in tensor memory: its a stages of 64 columns
// (head at +0, tail at +32, one K value per column) follow the accumulators.
template <int NT, bool APRE>
struct Tm;
template <>
struct Tm<64, true> { static constexpr int segb = 6, cb = 2; };
template <>
struct Tm<128, true> { static constexpr int segb = 3, cb = 1; };
template <>
struct Tm<64, false> { static constexpr int segb = 4, cb = 2; };
template <>
struct Tm<128, false> { static constexpr int segb = 2, cb = 1; };

// ring depths per N tile (dynamic shared memory stays within 227 KB): raw X chunks, A stages (in
// shared memory with a pre-split A, in tensor memory otherwise), B chunks
template <int NT, bool APRE>
struct Cfg;
template <>
struct Cfg<64, true> { static constexpr int raw = 1, a = 4, b = 6; };
template <>
struct Cfg<128, true> { static constexpr int raw = 1, a = 3, b = 4; };
template <>
struct Cfg<64, false> { static constexpr int raw = 6, a = 2, b = 8; };
template <>
struct Cfg<128, false> { static constexpr int raw = 4, a = 2, b = 5; };

template <int NT, bool APRE>
constexpr size_t smem_bytes() {
  return (APRE ? 0 : (size_t)Cfg<NT, APRE>::raw * kRawBytes) +
         (APRE ? 2 * (size_t)Cfg<NT, APRE>::a * kABytes : 0) + 2 * (size_t)Cfg<NT, APRE>::b * NT * 128 + 1024;
}

// Store of the result D[n][l] (n: output row, the MMA's N; l: the item's column, the MMA's M):
enum StoreMode {
  kStoreF32 = 0,  // out (float) = D, with the optional norm partials
  kSubF64 = 1,    // out (double) -= D
  kSplitF32 = 2,  // out, out2 (float) = TF32 head and tail of D (the operand form of a later product)
  kStoreF64 = 3,  // out (double) = D
  kResidF32 = 4,  // out (float) = in - D, in (float) read at its own layout (a residual)
  kAddF64 = 5     // out (double) += D atomically (K may be split: the splits add into one output)
};

struct ProjArgs {
  int64_t L, m;    // columns per observation (MMA M extent), K
  int r, b, nj, tpo, nch;
  // narrow layout (L <= 64 dividing 128): a tile holds opt = 128 / L whole observations, lane
  // o L + l = column l of observation t opt + o; b counts tiles then, nb the observations
  int narrow, opt, nb;
  // split K: item q of an nsplit-fold launch covers chunks [ks cps, min(nch, (ks + 1) cps)) of
  // K, ks = q / (b tpo nj), and stores its partial D at out + ks ws_stride (kStoreF32 only)
  int nsplit, cps;
  int seglen;  // chunks per main-accumulator segment
  int tfast;   // item order: column tiles fastest (else observations, then N tiles)
  int64_t ws_stride, px_stride;  // partial D and x^2 partials of one K split
  int mode;
  int nprod;  // 3: head x head + the two tail products; 1: head x head only
  void* out;
  void* out2;
  int64_t o_obs, ldn, ldl;  // element (n, l) of observation z at z * o_obs + n * ldn + l * ldl
  const float* in;          // kResidF32: in[(n / in_lz) in_obs + (n % in_lz) in_ldn + l in_ldl]
  int64_t in_lz, in_obs, in_ldn, in_ldl;
  // norm partials, contiguous per observation: wide layout x [obs][tile][conv warp], w [obs][tile][N
  // tile][epilogue warp]; narrow layout x [obs][xs], w [obs][N tile][half][xs], xs = max(1, L / 32)
  double* part_x;
  double* part_w;
  int* status;
  const int* run_if;  // the kernel returns at once unless *run_if != 0 (nullptr: always runs)
  unsigned long long wait_ns;
  long long drop_chunk;  // test hook: CTA 0 issues no copy for its chunk of this index (-1: none)
};

// Item q -> (observation z, column tile t, N tile j, K split ks), observations fastest: the CTAs
// running at one time share a few N tiles of B across all observations, so each B tile streams
// from HBM about once and its other readers hit L2 (with N tiles fastest, every observation would
// re-read all of B: 32x the core's bytes on the 1080p stream's third core).
// With a pre-split A operand (one observation, several A tiles), A tiles go fastest instead: the
// running CTAs then share each B tile across all A tiles.
__device__ __forceinline__ void decode_item(int64_t q, const ProjArgs& a, int* z, int* t, int* j, int* ks) {
  if (a.tfast) {
    *t = (int)(q % a.tpo);
    *z = (int)((q / a.tpo) % a.b);
    *j = (int)((q / ((int64_t)a.tpo * a.b)) % a.nj);
  } else {
    *z = (int)(q % a.b);
    *j = (int)((q / a.b) % a.nj);
    *t = (int)((q / ((int64_t)a.b * a.nj)) % a.tpo);
  }
  *ks = (int)(q / ((int64_t)a.b * a.nj * a.tpo));
}

// APRE: the A operand (rows = the items' columns, K contiguous) is given pre-split as TF32 head /
// tail arrays and copied by TMA straight into the A slots (xmap / xlmap are their maps); otherwise
// xmap describes the raw FP32 X and the converter warps build the A slots.
template <int NT, bool APRE>
__global__ void __launch_bounds__(kThreads, 1)
    tc_proj_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap xlmap,
                   const __grid_constant__ CUtensorMap uhmap, const __grid_constant__ CUtensorMap ulmap,
                   const ProjArgs a) {
  if (a.run_if && *a.run_if == 0) return;  // every thread reads the same flag before any barrier
  constexpr int RAW = Cfg<NT, APRE>::raw, AST = Cfg<NT, APRE>::a, BST = Cfg<NT, APRE>::b;
  constexpr uint32_t kBBytes = NT * 128;  // one half of a B chunk: NT rows of 128 bytes
  // tensor memory: main-accumulator segments at [0, SEGB NT), cross accumulators at
  // [SEGB NT, (SEGB + CB) NT), and (raw A) the A stages after them, 64 columns each
  constexpr int SEGB = Tm<NT, APRE>::segb, CB = Tm<NT, APRE>::cb;
  constexpr uint32_t kTmemCols = 512;
  constexpr uint32_t kACol = (uint32_t)((SEGB + CB) * NT);
  static_assert(APRE || kACol + 64 * AST <= kTmemCols, "tensor memory holds accumulators and A stages");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* raw = base;  // raw X chunks (raw A only)
  unsigned char* a_hi = raw + (APRE ? 0 : RAW * kRawBytes);  // A stages (pre-split A only)
  unsigned char* a_lo = a_hi + (APRE ? AST * kABytes : 0);
  unsigned char* b_hi = a_lo + (APRE ? AST * kABytes : 0);
  unsigned char* b_lo = b_hi + BST * kBBytes;

  __shared__ __align__(8) uint64_t raw_full[RAW], raw_empty[RAW];
  __shared__ __align__(8) uint64_t a_full[AST], a_empty[AST];
  __shared__ __align__(8) uint64_t b_full[BST], b_empty[BST];
  __shared__ __align__(8) uint64_t seg_full[SEGB], seg_empty[SEGB], cross_empty[CB], mma_done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, wid = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int s = 0; s < RAW; ++s) {
      mbar_init(&raw_full[s], 1);
      mbar_init(&raw_empty[s], kConvWarps);
    }
    for (int s = 0; s < AST; ++s) {
      mbar_init(&a_full[s], APRE ? 1 : kConvWarps);
      mbar_init(&a_empty[s], 1);
    }
    for (int s = 0; s < BST; ++s) {
      mbar_init(&b_full[s], 1);
      mbar_init(&b_empty[s], 1);
    }
    for (int s = 0; s < SEGB; ++s) {
      mbar_init(&seg_full[s], 1);
      mbar_init(&seg_empty[s], kEpiWarps);
    }
    for (int s = 0; s < CB; ++s) mbar_init(&cross_empty[s], kEpiWarps);
    mbar_init(&mma_done, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (wid == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    fence_before();
  }
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  const int64_t nitems = (int64_t)a.nsplit * a.b * a.tpo * a.nj;
  const unsigned long long lim = a.wait_ns;

  if (wid == kProducerWarp) {
    if (lane == 0) {
      int64_t g = 0;
      bool ok = true;
      for (int64_t q = blockIdx.x; q < nitems && ok; q += gridDim.x) {
        int z, t, j, ks;
        decode_item(q, a, &z, &t, &j, &ks);
        const int c_lo = ks * a.cps, c_hi = min(a.nch, c_lo + a.cps);
        for (int c = c_lo; c < c_hi; ++c, ++g) {
          const int s = (int)(g % RAW), sb = (int)(g % BST), qa = (int)(g % AST);
          if constexpr (APRE) {
            if (g >= AST && !wait_bounded(&a_empty[qa], (uint32_t)(((g / AST) - 1) & 1), &abort_flag, lim)) {
              ok = false;
              break;
            }
            if (!(blockIdx.x == 0 && g == a.drop_chunk)) {
              mbar_expect_tx(&a_full[qa], (a.nprod == 3 ? 2 : 1) * kABytes);
              tma_load_2d(smem_u32(a_hi + (size_t)qa * kABytes), &xmap, c * kChunk, t * kTile, &a_full[qa]);
              if (a.nprod == 3)
                tma_load_2d(smem_u32(a_lo + (size_t)qa * kABytes), &xlmap, c * kChunk, t * kTile, &a_full[qa]);
            }
          } else {
            if (g >= RAW && !wait_bounded(&raw_empty[s], (uint32_t)(((g / RAW) - 1) & 1), &abort_flag, lim)) {
              ok = false;
              break;
            }
            if (!(blockIdx.x == 0 && g == a.drop_chunk)) {
              mbar_expect_tx(&raw_full[s], kRawBytes);
              if (a.narrow)
                tma_load_3d(smem_u32(raw + (size_t)s * kRawBytes), &xmap, 0, c * kChunk, z * a.opt, &raw_full[s]);
              else
                tma_load_3d(smem_u32(raw + (size_t)s * kRawBytes), &xmap, t * kTile, c * kChunk, z, &raw_full[s]);
            }
          }
          if (g >= BST && !wait_bounded(&b_empty[sb], (uint32_t)(((g / BST) - 1) & 1), &abort_flag, lim)) {
            ok = false;
            ++g;
            break;
          }
          mbar_expect_tx(&b_full[sb], (a.nprod == 3 ? 2 : 1) * kBBytes);
          tma_load_2d(smem_u32(b_hi + (size_t)sb * kBBytes), &uhmap, c * kChunk, j * NT, &b_full[sb]);
          if (a.nprod == 3)
            tma_load_2d(smem_u32(b_lo + (size_t)sb * kBBytes), &ulmap, c * kChunk, j * NT, &b_full[sb]);
        }
      }
      // copies of the last ring slots may still be in flight (on an abort): wait for them
      if constexpr (APRE) {
        for (int64_t k = g > AST ? g - AST : 0; k < g; ++k)
          wait_drain(&a_full[k % AST], (uint32_t)((k / AST) & 1), lim);
      } else {
        for (int64_t k = g > RAW ? g - RAW : 0; k < g; ++k)
          wait_drain(&raw_full[k % RAW], (uint32_t)((k / RAW) & 1), lim);
      }
      for (int64_t k = g > BST ? g - BST : 0; k < g; ++k)
        wait_drain(&b_full[k % BST], (uint32_t)((k / BST) & 1), lim);
    }
  } else if (wid == kMmaWarp) {
    if (lane == 0) {
      int64_t g = 0, sg = 0;  // chunks and segments issued
      int it = 0;
      bool ok = true;
      for (int64_t q = blockIdx.x; q < nitems && ok; q += gridDim.x, ++it) {
        int z, t, j, ks;
        decode_item(q, a, &z, &t, &j, &ks);
        const int c_lo = ks * a.cps, c_hi = min(a.nch, c_lo + a.cps);
        const int nN = min(NT, (a.r - j * NT + 15) / 16 * 16);  // MMA N of this item
        const uint32_t idesc = tf32_idesc(kTile, nN);
        const int cbi = it % CB;
        if (it >= CB && !wait_bounded(&cross_empty[cbi], (uint32_t)(((it / CB) - 1) & 1), &abort_flag, lim)) break;
        const uint32_t dc = tmem + (uint32_t)((SEGB + cbi) * NT);
        uint32_t d = 0;
        for (int c = c_lo; c < c_hi; ++c, ++g) {
          const int cs = (c - c_lo) % a.seglen;  // chunk within its segment
          if (cs == 0) {
            const int p = (int)(sg % SEGB);
            if (sg >= SEGB && !wait_bounded(&seg_empty[p], (uint32_t)(((sg / SEGB) - 1) & 1), &abort_flag, lim)) {
              ok = false;
              break;
            }
            fence_after();
            d = tmem + (uint32_t)(p * NT);
          }
          const int qa = (int)(g % AST), sb = (int)(g % BST);
          if (!wait_bounded(&a_full[qa], (uint32_t)((g / AST) & 1), &abort_flag, lim) ||
              !wait_bounded(&b_full[sb], (uint32_t)((g / BST) & 1), &abort_flag, lim)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t bh = smem_u32(b_hi + (size_t)sb * kBBytes), bl = smem_u32(b_lo + (size_t)sb * kBBytes);
          const int64_t rows = a.m - (int64_t)c * kChunk;
          const int nk = rows >= kChunk ? kChunk / 8 : (int)((rows + 7) / 8);
          if constexpr (APRE) {
            const uint32_t ah = smem_u32(a_hi + (size_t)qa * kABytes), al = smem_u32(a_lo + (size_t)qa * kABytes);
#pragma unroll
            for (int kk = 0; kk < kChunk / 8; ++kk) {
              if (kk >= nk) break;
              const uint32_t ko = (uint32_t)kk * 32;  // 8 TF32 values of K
              // head x head into the segment's main accumulator; the two tail products (~2^-11 of it)
              // into the item's cross accumulator
              mma_tf32(d, kmajor_sw128_desc(ah + ko), kmajor_sw128_desc(bh + ko), idesc, (cs | kk) != 0);
              if (a.nprod == 3) {
                mma_tf32(dc, kmajor_sw128_desc(al + ko), kmajor_sw128_desc(bh + ko), idesc, ((c - c_lo) | kk) != 0);
                mma_tf32(dc, kmajor_sw128_desc(ah + ko), kmajor_sw128_desc(bl + ko), idesc, 1);
              }
            }
          } else {
            const uint32_t at = tmem + kACol + 64u * (uint32_t)qa;  // head; tail 32 columns on
#pragma unroll
            for (int kk = 0; kk < kChunk / 8; ++kk) {
              if (kk >= nk) break;
              const uint32_t ko = (uint32_t)kk * 32;
              mma_tf32_ta(d, at + 8u * kk, kmajor_sw128_desc(bh + ko), idesc, (cs | kk) != 0);
              if (a.nprod == 3) {
                mma_tf32_ta(dc, at + 32u + 8u * kk, kmajor_sw128_desc(bh + ko), idesc, ((c - c_lo) | kk) != 0);
                mma_tf32_ta(dc, at + 8u * kk, kmajor_sw128_desc(bl + ko), idesc, 1);
              }
            }
          }
          mma_commit(&a_empty[qa]);  // these slots are free once the MMAs above have read them
          mma_commit(&b_empty[sb]);
          if (cs == a.seglen - 1 || c == c_hi - 1) {
            mma_commit(&seg_full[sg % SEGB]);  // the segment (and, after the last one, the cross sum) is done
            ++sg;
          }
        }
      }
      // every MMA issued has completed before tensor memory is released
      mma_commit(&mma_done);
      wait_drain(&mma_done, 0, lim);
    }
  } else if (wid < kConvWarps) {
    if constexpr (!APRE) {  // with a pre-split A operand the A slots are filled by TMA
    // converters: thread tid owns column tid of the item's tile
    int64_t g = 0;
    for (int64_t q = blockIdx.x; q < nitems; q += gridDim.x) {
      int z, t, j, ks;
      decode_item(q, a, &z, &t, &j, &ks);
      const int c_lo = ks * a.cps, c_hi = min(a.nch, c_lo + a.cps);
      double* part_x = a.part_x ? a.part_x + (int64_t)ks * a.px_stride : nullptr;
      float x2 = 0.0f;
      bool ok = true;
      for (int c = c_lo; c < c_hi; ++c, ++g) {
        const int s = (int)(g % RAW), qa = (int)(g % AST);
        bool got = wait_bounded(&raw_full[s], (uint32_t)((g / RAW) & 1), &abort_flag, lim);
        if (got && g >= AST) got = wait_bounded(&a_empty[qa], (uint32_t)(((g / AST) - 1) & 1), &abort_flag, lim);
        if (!__all_sync(0xffffffffu, got)) {
          ok = false;
          break;
        }
        const float* rw = reinterpret_cast<const float*>(raw + (size_t)s * kRawBytes);
        // the raw chunk: [k][128 columns] (wide) or [observation][k][L] (narrow)
        const int rbase = a.narrow ? (tid / (int)a.L) * kChunk * (int)a.L + tid % (int)a.L : tid;
        const int rstep = a.narrow ? (int)a.L : kTile;
        const int64_t rows = a.m - (int64_t)c * kChunk;
        const int kv = rows >= kChunk ? kChunk : (int)rows;  // rows of K in this chunk
        // this thread's row of A (tensor-memory lane tid): 32 K values, head and tail (the tail itself
        // rounded to TF32: the MMA reads it exactly), zero past the chunk's rows
        uint32_t hv[kChunk], lv[kChunk];
#pragma unroll
        for (int kk = 0; kk < kChunk; ++kk) {
          const float y = kk < kv ? rw[rbase + kk * rstep] : 0.0f;
          x2 = fmaf(y, y, x2);
          const float hy = tf32_hi(y);
          hv[kk] = __float_as_uint(hy);
          lv[kk] = __float_as_uint(tf32_hi(y - hy));
        }
        const uint32_t at = tmem + ((uint32_t)(wid * 32) << 16) + kACol + 64u * (uint32_t)qa;
        tmem_st32(at, hv);
        if (a.nprod == 3) tmem_st32(at + 32u, lv);
        tmem_wait_st();
        fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&a_full[qa]);
          mbar_arrive(&raw_empty[s]);
        }
      }
      if (!ok) break;
      if (part_x && j == 0) {
        double s = (double)x2;
        if (a.narrow) {  // sum over the lanes of one observation (aligned groups of min(L, 32))
          const int gsz = min((int)a.L, 32);
          for (int o = 1; o < gsz; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          const int ob = tid / (int)a.L, l = tid % (int)a.L, zz = z * a.opt + ob;
          const int xs = max(1, (int)a.L / 32);
          if (ob < a.opt && zz < a.nb && (l & 31) == 0) part_x[(int64_t)zz * xs + l / 32] = s;
        } else {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (lane == 0) part_x[((int64_t)z * a.tpo + t) * kConvWarps + wid] = s;
        }
      }
    }
    }
  } else if (wid < kProducerWarp) {
    // epilogue: thread = tensor-memory lane = tile column, one half of the item's N tile per warp.
    // The main accumulator of each segment is added into NT/2 FP32 registers (round-to-nearest),
    // then the item's cross accumulator; the result is stored as W and its squares summed.
    constexpr int H = NT / 2;
    const int ew = wid - kConvWarps, qd = ew & 3, hf = ew >> 2;  // lane quarter, half of the N tile
    int64_t sg = 0;
    int it = 0;
    bool ok = true;
    for (int64_t q = blockIdx.x; q < nitems && ok; q += gridDim.x, ++it) {
      int z, t, j, ks;
      decode_item(q, a, &z, &t, &j, &ks);
      const int c_lo = ks * a.cps, c_hi = min(a.nch, c_lo + a.cps);
      const int nseg = (c_hi - c_lo + a.seglen - 1) / a.seglen;
      const int nN = min(NT, (a.r - j * NT + 15) / 16 * 16);
      const int c0 = hf * H;  // first column of this warp's half
      float run[H];
#pragma unroll
      for (int e = 0; e < H; ++e) run[e] = 0.0f;
      const uint32_t lanes = (uint32_t)(qd * 32) << 16;
      // add the accumulator at column offset `col` of tensor memory into run (two 16-column loads in
      // flight per wait)
      auto take = [&](uint32_t col) {
        const uint32_t taddr = tmem + lanes + col + (uint32_t)c0;
#pragma unroll
        for (int pc = 0; pc < H / 16; pc += 2) {
          if (c0 + pc * 16 < nN) {
            float v[32];
            tmem_ld16(taddr + (uint32_t)(16 * pc), v);
            if (pc + 1 < H / 16) tmem_ld16(taddr + (uint32_t)(16 * (pc + 1)), v + 16);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 32; ++e)
              if (pc * 16 + e < H) run[pc * 16 + e] += v[e];
          }
        }
      };
      for (int s = 0; s < nseg; ++s, ++sg) {
        const int p = (int)(sg % SEGB);
        if (!__all_sync(0xffffffffu, wait_bounded(&seg_full[p], (uint32_t)((sg / SEGB) & 1), &abort_flag, lim))) {
          ok = false;
          break;
        }
        fence_after();
        take((uint32_t)(p * NT));
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&seg_empty[p]);
      }
      if (!ok) break;
      {  // the item's cross sum (complete with its last segment; unused with one product)
        const int cbi = it % CB;
        if (a.nprod == 3) take((uint32_t)((SEGB + cbi) * NT));
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&cross_empty[cbi]);
      }
      const int cl = qd * 32 + lane;  // the tile column of this lane
      const int ob = a.narrow ? cl / (int)a.L : 0;
      const int64_t zl = a.narrow ? (int64_t)z * a.opt + ob : z;           // its observation
      const int64_t l = a.narrow ? cl % (int)a.L : (int64_t)t * kTile + cl;  // its column there
      const bool lane_ok = !a.narrow || (ob < a.opt && zl < a.nb);
      const int64_t base = zl * a.o_obs + l * a.ldl + ks * a.ws_stride;
      float w2 = 0.0f;
#pragma unroll
      for (int e = 0; e < H; ++e) {
        const int ai = j * NT + c0 + e;
        if (c0 + e < nN && ai < a.r) {
          const float v = run[e];
          w2 = fmaf(v, v, w2);
          if (l < a.L && lane_ok) {
            const int64_t o = base + (int64_t)ai * a.ldn;
            if (a.mode == kStoreF32) {
              static_cast<float*>(a.out)[o] = v;
            } else if (a.mode == kSubF64) {
              static_cast<double*>(a.out)[o] -= (double)v;
            } else if (a.mode == kStoreF64) {
              static_cast<double*>(a.out)[o] = (double)v;
            } else if (a.mode == kAddF64) {
              atomicAdd(static_cast<double*>(a.out) + o, (double)v);
            } else if (a.mode == kResidF32) {
              const int64_t zi = ai / a.in_lz;
              static_cast<float*>(a.out)[o] =
                  a.in[zi * a.in_obs + (ai - zi * a.in_lz) * a.in_ldn + l * a.in_ldl] - v;
            } else {
              const float hv = tf32_hi(v);
              static_cast<float*>(a.out)[o] = hv;
              static_cast<float*>(a.out2)[o] = tf32_hi(v - hv);
            }
          }
        }
      }
      if (a.part_w) {
        double s = (double)w2;
        if (a.narrow) {
          const int gsz = min((int)a.L, 32);
          for (int o = 1; o < gsz; o <<= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          const int xs = max(1, (int)a.L / 32);
          if (lane_ok && (l & 31) == 0) a.part_w[(zl * a.nj + j) * 2 * xs + (int64_t)hf * xs + l / 32] = s;
        } else {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
          if (lane == 0) a.part_w[(((int64_t)z * a.tpo + t) * a.nj + j) * kEpiWarps + ew] = s;
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  if (wid == kMmaWarp) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
  if (tid == 0 && abort_flag) atomicOr(a.status, 1);
}

// Per observation: ||X(z)||^2 and ||X(z)||^2 - ||W(z)||^2 (clamped to [0, ||X(z)||^2]: the difference
// of the two FP32-accurate sums can round below zero when U spans the observation), summed in a
// fixed order.
__global__ void tc_proj_reduce_kernel(const double* part_x, const double* part_w, int64_t xper, int64_t wper,
                                      double* x2_out, double* rho2_out) {
  const int z = blockIdx.x;
  double sx = 0.0, sw = 0.0;
  for (int64_t i = threadIdx.x; i < xper; i += blockDim.x) sx += part_x[(int64_t)z * xper + i];
  for (int64_t i = threadIdx.x; i < wper; i += blockDim.x) sw += part_w[(int64_t)z * wper + i];
  __shared__ double ax[256], aw[256];
  ax[threadIdx.x] = sx;
  aw[threadIdx.x] = sw;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      ax[threadIdx.x] += ax[threadIdx.x + o];
      aw[threadIdx.x] += aw[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (x2_out) x2_out[z] = ax[0];
    if (rho2_out) rho2_out[z] = fmin(fmax(ax[0] - aw[0], 0.0), ax[0]);
  }
}

// After a split-K launch: W = sum over the splits of the partial products (block of o_obs elements
// per observation), w^2 of the sum, x^2 summed over splits and slots, rho2 = x^2 - w^2 (clamped).
__global__ void tc_splitk_reduce_kernel(const float* ws, int nsplit, int64_t ws_stride, int64_t o_obs, float* W,
                                        const double* part_x, int64_t px_stride, int64_t xper, double* x2_out,
                                        double* rho2_out) {
  const int z = blockIdx.x;
  double w2 = 0.0, sx = 0.0;
  for (int64_t e = threadIdx.x; e < o_obs; e += blockDim.x) {
    float acc = 0.0f;
    for (int k = 0; k < nsplit; ++k) acc += ws[k * ws_stride + z * o_obs + e];
    W[z * o_obs + e] = acc;
    w2 += (double)acc * acc;
  }
  if (part_x)
    for (int64_t i = threadIdx.x; i < (int64_t)nsplit * xper; i += blockDim.x)
      sx += part_x[(i / xper) * px_stride + z * xper + i % xper];
  __shared__ double aw[256], ax[256];
  aw[threadIdx.x] = w2;
  ax[threadIdx.x] = sx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      aw[threadIdx.x] += aw[threadIdx.x + o];
      ax[threadIdx.x] += ax[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (x2_out) x2_out[z] = ax[0];
    if (rho2_out) rho2_out[z] = fmin(fmax(ax[0] - aw[0], 0.0), ax[0]);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) == cudaSuccess &&
        qr == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    cudaGetLastError();
  });
  return fn;
}

int pick_nt(int r) { return r <= 64 ? 64 : 128; }

std::atomic<unsigned long long> g_wait_ns{2000000000ull};
std::atomic<long long> g_drop_chunk{-1};

// Observations of fewer than 128 columns are packed 128 / L to a tile when L divides 128 (L >= 4).
bool narrow_layout(const TcGemm& g) { return g.ah == nullptr && g.L <= 64 && g.L >= 4 && kTile % g.L == 0; }

bool encode_2d(CUtensorMap* map, const float* p, int64_t inner, int64_t outer, int64_t ld, uint32_t box_inner,
               uint32_t box_outer, bool sw128) {
  const cuuint64_t gdim[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t gstride[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {box_inner, box_outer};
  const cuuint32_t es[2] = {1, 1};
  return encode_fn()(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(p), gdim, gstride, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, sw128 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int NT, bool APRE>
cudaError_t run(const TcGemm& g, cudaStream_t st) {
  if (!encode_fn()) return cudaErrorNotSupported;
  CUtensorMap xmap, xlmap, uhmap, ulmap;
  if constexpr (APRE) {
    if (!encode_2d(&xmap, g.ah, g.lda, g.la_alloc, g.lda, kChunk, kTile, true) ||
        !encode_2d(&xlmap, g.al, g.lda, g.la_alloc, g.lda, kChunk, kTile, true))
      return cudaErrorInvalidValue;
  } else {
    const cuuint64_t gdim[3] = {(cuuint64_t)g.L, (cuuint64_t)g.K, (cuuint64_t)g.b};
    const cuuint64_t gstride[2] = {(cuuint64_t)g.ldx * 4, (cuuint64_t)g.x_obs * 4};
    const bool nar = narrow_layout(g);
    const cuuint32_t box[3] = {nar ? (cuuint32_t)g.L : (cuuint32_t)kTile, (cuuint32_t)kChunk,
                               nar ? (cuuint32_t)(kTile / g.L) : 1u};
    const cuuint32_t es[3] = {1, 1, 1};
    if (encode_fn()(&xmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(g.x), gdim, gstride, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
    xlmap = xmap;  // unused
  }
  if (!encode_2d(&uhmap, g.bh, g.ldb, g.nb_alloc, g.ldb, kChunk, NT, true) ||
      !encode_2d(&ulmap, g.bl, g.ldb, g.nb_alloc, g.ldb, kChunk, NT, true))
    return cudaErrorInvalidValue;
  static std::once_flag once;
  static cudaError_t setup_err = cudaSuccess;
  static int sms = 148;
  std::call_once(once, [] {
    setup_err = cudaFuncSetAttribute(tc_proj_kernel<NT, APRE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem_bytes<NT, APRE>());
    int dev = 0;
    if (setup_err == cudaSuccess) setup_err = cudaGetDevice(&dev);
    if (setup_err == cudaSuccess) setup_err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  });
  TT_CUDA(setup_err);
  ProjArgs a;
  a.L = g.L;
  a.m = g.K;
  a.r = g.r;
  a.narrow = !APRE && narrow_layout(g);
  a.opt = a.narrow ? (int)(kTile / g.L) : 1;
  a.nb = APRE ? 1 : g.b;
  a.b = a.narrow ? (a.nb + a.opt - 1) / a.opt : a.nb;
  a.nj = (g.r + NT - 1) / NT;
  a.tpo = a.narrow ? 1 : (int)((g.L + kTile - 1) / kTile);
  a.tfast = APRE ? 1 : 0;
  a.nch = (int)((g.K + kChunk - 1) / kChunk);
  a.mode = g.mode;
  a.nprod = g.nprod == 1 ? 1 : 3;
  a.out = g.out;
  a.out2 = g.out2;
  a.o_obs = g.o_obs;
  a.ldn = g.ldn;
  a.ldl = g.ldl;
  a.in = g.in;
  a.in_lz = g.in_lz > 0 ? g.in_lz : 1;
  a.in_obs = g.in_obs;
  a.in_ldn = g.in_ldn;
  a.in_ldl = g.in_ldl;
  const bool norms = !APRE && (g.x2 != nullptr || g.rho2 != nullptr);
  // split K when the output is too small to fill the GPU (few, tall contractions): chain layout only
  const int64_t items1 = (int64_t)a.b * a.tpo * a.nj, wsz = (int64_t)a.nb * g.r * g.L;
  a.nsplit = 1;
  if (!APRE && g.mode == kStoreF32 && g.ws && g.o_obs == (int64_t)g.r * g.L && g.ldn == g.L && g.ldl == 1 &&
      items1 < sms && a.nch >= 8) {
    int64_t ns = std::min<int64_t>((2 * sms + items1 - 1) / items1, a.nch / 4);
    ns = std::min<int64_t>(ns, g.ws_elems / std::max<int64_t>(wsz, 1));
    if (ns >= 2) a.nsplit = (int)ns;
  }
  if (g.mode == kAddF64 && items1 < sms && a.nch >= 8) {  // the splits add into the output directly
    const int64_t ns = std::min<int64_t>((2 * sms + items1 - 1) / items1, a.nch / 4);
    if (ns >= 2) a.nsplit = (int)ns;
  }
  a.cps = (a.nch + a.nsplit - 1) / a.nsplit;
  a.nsplit = (a.nch + a.cps - 1) / a.cps;  // every split has at least one chunk
  // one segment for a short K range (<= 256: its rounding bias is a few ulps); beyond, 32-long
  // segments where residual norms are taken by Pythagoras (which amplifies the bias by
  // ||x||^2 / ||R||^2), 64-long ones elsewhere (half the promotions, ~1.4e-7 relative bias)
  a.seglen = a.cps <= 8 ? a.cps : (norms ? 1 : 2);
  const bool ws_split = a.nsplit > 1 && g.mode != kAddF64;
  a.ws_stride = ws_split ? wsz : 0;
  if (ws_split) a.out = g.ws;
  a.part_x = norms ? g.part : nullptr;
  const int64_t xs = std::max<int64_t>(1, g.L / 32);
  const int64_t xper = a.narrow ? xs : (int64_t)a.tpo * kConvWarps;
  const int64_t wper = a.narrow ? (int64_t)a.nj * 2 * xs : (int64_t)a.tpo * a.nj * kEpiWarps;
  a.px_stride = (int64_t)a.nb * xper;
  a.part_w = norms && a.nsplit == 1 ? g.part + (int64_t)a.nsplit * a.nb * xper : nullptr;
  a.status = g.status;
  if (g.run_if && (ws_split || norms)) return cudaErrorInvalidValue;  // no follow-up pass checks the flag
  a.run_if = g.run_if;
  a.wait_ns = g_wait_ns.load();
  a.drop_chunk = g_drop_chunk.exchange(-1);
  const int64_t nitems = (int64_t)a.nsplit * items1;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(sms, nitems));
  note_launch();
  tc_proj_kernel<NT, APRE><<<(unsigned)grid, kThreads, smem_bytes<NT, APRE>(), st>>>(xmap, xlmap, uhmap, ulmap, a);
  TT_CUDA(cudaGetLastError());
  if (ws_split) {
    note_launch();
    tc_splitk_reduce_kernel<<<a.nb, 256, 0, st>>>(g.ws, a.nsplit, wsz, (int64_t)g.r * g.L, static_cast<float*>(g.out),
                                                 a.part_x, a.px_stride, xper, g.x2, g.rho2);
    TT_CUDA(cudaGetLastError());
  } else if (norms) {
    note_launch();
    tc_proj_reduce_kernel<<<a.nb, 256, 0, st>>>(a.part_x, a.part_w, xper, wper, g.x2, g.rho2);
    TT_CUDA(cudaGetLastError());
  }
  return cudaSuccess;
}

}  // namespace

bool tc_proj_supported(const void* X, int64_t L, int64_t m, int r, int64_t ldhl) {
  // columns per observation: >= 32 (a tile per 128 of them) or a divisor of 128 (observations packed)
  const bool shape_ok = L >= 32 || (L >= 4 && kTile % L == 0);
  return encode_fn() != nullptr && (reinterpret_cast<uintptr_t>(X) % 16) == 0 && (L % 4) == 0 && shape_ok &&
         L < (1LL << 31) && m >= 1 && m < (1LL << 31) && r >= 1 && (ldhl % 32) == 0;
}

int64_t tc_proj_part_elems(int b, int64_t L, int64_t r, int64_t m) {
  const int64_t tpo = (L + kTile - 1) / kTile;
  const int64_t nj = (r + 63) / 64;  // the most N tiles any tile width gives
  const int64_t nch = (m + kChunk - 1) / kChunk;  // the most K splits (x^2 partials per split)
  return (int64_t)b * tpo * (kConvWarps + nj * kEpiWarps) + (int64_t)b * std::max<int64_t>(2, tpo * kConvWarps) * (nch / 4 + 1);
}

cudaError_t launch_tc_gemm(const TcGemm& g, cudaStream_t st) {
  if (g.L < 1 || g.K < 1 || g.r < 1 || g.b < 1) return cudaSuccess;
  const bool pre = g.ah != nullptr;
  if (pick_nt(g.r) == 64) return pre ? run<64, true>(g, st) : run<64, false>(g, st);
  return pre ? run<128, true>(g, st) : run<128, false>(g, st);
}

cudaError_t launch_tc_proj(const float* X, int b, int64_t L, int64_t m, int r, const float* Uh, const float* Ul,
                           int64_t ldhl, int64_t hlcols, float* W, double* x2, double* rho2, double* part,
                           float* ws, int* status, cudaStream_t st, int nprod) {
  TcGemm g;
  g.x = X;
  g.ldx = L;
  g.x_obs = m * L;
  g.L = L;
  g.b = b;
  g.K = m;
  g.bh = Uh;
  g.bl = Ul;
  g.ldb = ldhl;
  g.nb_alloc = hlcols;
  g.r = r;
  g.mode = kStoreF32;
  g.out = W;
  g.o_obs = (int64_t)r * L;
  g.ldn = L;
  g.ldl = 1;
  g.x2 = x2;
  g.rho2 = rho2;
  g.part = part;
  g.status = status;
  g.ws = ws;
  g.ws_elems = ws ? tc_ws_elems : 0;
  g.nprod = nprod;
  return launch_tc_gemm(g, st);
}

void tc_set_wait_ns(unsigned long long ns) { g_wait_ns.store(ns ? ns : 2000000000ull); }
void tc_drop_next_copy(long long chunk) { g_drop_chunk.store(chunk); }

// Head / tail split of FP32 core columns [c0, c1) (all ld_in rows) into the TF32 pair the tensor
// cores read (ld_out rows each; rows beyond ld_in are left as they are).
__global__ void split_tf32_kernel(const float* in, int64_t ld_in, int64_t c0, int64_t c1, float* hi, float* lo,
                                  int64_t ld_out) {
  const int64_t rows = min((ld_in + 31) / 32 * 32, ld_out);  // the last K chunk is zero past the column
  for (int64_t c = c0 + blockIdx.y; c < c1; c += gridDim.y)
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows; i += (int64_t)gridDim.x * blockDim.x) {
      const float x = i < ld_in ? in[c * ld_in + i] : 0.0f;
      const float h = tf32_hi(x);
      hi[c * ld_out + i] = h;
      lo[c * ld_out + i] = tf32_hi(x - h);
    }
}

__global__ void split_tf32_f64_kernel(const double* in, int64_t ld_in, int64_t rows, int64_t c0, int64_t c1,
                                      float* hi, float* lo, int64_t ld_out, float* f32, double* sumsq) {
  __shared__ double red[8];
  const int64_t rows32 = (rows + 31) / 32 * 32;  // the last K chunk is zero past the operand
  for (int64_t c = c0 + blockIdx.y; c < c1; c += gridDim.y) {
    double q = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < rows32; i += (int64_t)gridDim.x * blockDim.x) {
      const double x = i < rows ? in[c * ld_in + i] : 0.0;
      const float h = tf32_hi((float)x);
      hi[c * ld_out + i] = h;
      lo[c * ld_out + i] = tf32_hi((float)(x - (double)h));
      if (f32) f32[c * ld_out + i] = (float)x;
      q = fma(x, x, q);
    }
    if (sumsq) {  // block sum, one atomic per block and column
      for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = q;
      __syncthreads();
      if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
        atomicAdd(sumsq + (c - c0), t);
      }
      __syncthreads();
    }
  }
}

cudaError_t launch_split_tf32_f64(const double* in, int64_t ld_in, int64_t rows, int64_t c0, int64_t c1, float* hi,
                                  float* lo, int64_t ld_out, cudaStream_t st, float* f32, double* sumsq) {
  if (c1 <= c0 || rows <= 0) return cudaSuccess;
  const int64_t bx = std::min<int64_t>((rows + 255) / 256, 64);
  const int64_t by = std::min<int64_t>(c1 - c0, 1024);
  note_launch();
  split_tf32_f64_kernel<<<dim3((unsigned)bx, (unsigned)by), 256, 0, st>>>(in, ld_in, rows, c0, c1, hi, lo, ld_out,
                                                                            f32, sumsq);
  return cudaGetLastError();
}

// B operand of Vn (I - R^{-1}): row j, entry l = TF32 head / tail of delta_lj - Rinv[l + j k] (Rinv
// k x k column-major); the ld x ld block is zero outside the k x k corner.
__global__ void eye_minus_split_kernel(const double* Rinv, int k, float* hi, float* lo, int ld, const int* run_if) {
  if (run_if && *run_if == 0) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ld * ld; e += gridDim.x * blockDim.x) {
    const int j = e / ld, l = e % ld;
    const double f = (j < k && l < k) ? (l == j ? 1.0 : 0.0) - Rinv[l + (int64_t)j * k] : 0.0;
    const float h = tf32_hi((float)f);
    hi[e] = h;
    lo[e] = tf32_hi((float)(f - (double)h));
  }
}

cudaError_t launch_eye_minus_split(const double* Rinv, int k, float* hi, float* lo, int ld, cudaStream_t st,
                                   const int* run_if) {
  if (k <= 0 || k > ld) return cudaErrorInvalidValue;
  note_launch();
  eye_minus_split_kernel<<<(ld * ld + 255) / 256, 256, 0, st>>>(Rinv, k, hi, lo, ld, run_if);
  return cudaGetLastError();
}

constexpr int kLowdinThreads = 1024;
constexpr int kLowdinMax = 112;  // largest k (two k x k FP32 matrices in shared memory)

__global__ void __launch_bounds__(kLowdinThreads)
    lowdin_split_kernel(const double* S, int k, const double* diag, float* hi, float* lo, int ld, int* fallback) {
  extern __shared__ float lw[];
  float* E = lw;           // E[l][j], l-major rows of k
  float* E2 = lw + k * k;  // E^2
  __shared__ double red[kLowdinThreads / 32];
  __shared__ int small;
  const int tid = threadIdx.x, kk = k * k;
  double q = 0.0;
  for (int e = tid; e < kk; e += kLowdinThreads) {
    const int l = e / k, j = e % k;
    const double v = (l == j) ? (diag ? diag[j] : S[(int64_t)j * k + j]) - 1.0 : S[(int64_t)j * k + l];
    E[e] = (float)v;
    q = fma(v, v, q);
  }
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  if ((tid & 31) == 0) red[tid >> 5] = q;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < kLowdinThreads / 32; ++w) t += red[w];
    small = t <= 1e-8;  // ||E||_F <= 1e-4 (NaN fails too)
    if (!small) *fallback = 1;
  }
  __syncthreads();
  if (!small) return;
  for (int e = tid; e < kk; e += kLowdinThreads) {  // E^2
    const int l = e / k, j = e % k;
    float v = 0.0f;
    for (int m = 0; m < k; ++m) v = fmaf(E[l * k + m], E[m * k + j], v);
    E2[e] = v;
  }
  __syncthreads();
  for (int e = tid; e < ld * ld; e += kLowdinThreads) {  // F = E/2 - 3 E^2/8 + 5 E^3/16, row j of B
    const int j = e / ld, l = e % ld;
    float f = 0.0f;
    if (j < k && l < k) {
      float e3 = 0.0f;
      for (int m = 0; m < k; ++m) e3 = fmaf(E2[l * k + m], E[m * k + j], e3);
      f = 0.5f * E[l * k + j] - 0.375f * E2[l * k + j] + 0.3125f * e3;
    }
    const float h = tf32_hi(f);
    hi[e] = h;
    lo[e] = tf32_hi(f - h);
  }
}

cudaError_t launch_lowdin_split(const double* S, int k, const double* diag, float* hi, float* lo, int ld,
                                int* fallback, cudaStream_t st) {
  if (k <= 0 || k > ld || k > kLowdinMax) return cudaErrorInvalidValue;
  static std::once_flag once;
  static cudaError_t attr_err = cudaSuccess;
  std::call_once(once, [] {
    attr_err = cudaFuncSetAttribute(lowdin_split_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)(2 * kLowdinMax * kLowdinMax * sizeof(float)));
  });
  TT_CUDA(attr_err);
  note_launch();
  lowdin_split_kernel<<<1, kLowdinThreads, 2 * (size_t)k * k * sizeof(float), st>>>(S, k, diag, hi, lo, ld, fallback);
  return cudaGetLastError();
}

// W (b observations of r x L, row-major, observation-major) -> its transpose split: row n = z L + l
// of hi / lo holds W[z][0..r)[l] (ld_out >= r, zero up to the next multiple of 32).  32 x 32 tiles
// through shared memory, so that both the reads (along l) and the writes (along r) are coalesced.
__global__ void split_tf32_transpose_kernel(const float* W, int64_t r, int64_t L, float* hi, float* lo,
                                            int64_t ld_out) {
  __shared__ float tile[32][33];
  const int64_t z = blockIdx.z;
  const int64_t a0 = (int64_t)blockIdx.y * 32, l0 = (int64_t)blockIdx.x * 32;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8 threads
  for (int k = ty; k < 32; k += 8) {
    const int64_t a = a0 + k, l = l0 + tx;
    tile[k][tx] = (a < r && l < L) ? W[z * r * L + a * L + l] : 0.0f;
  }
  __syncthreads();
  const int64_t r32 = (r + 31) / 32 * 32;
  for (int k = ty; k < 32; k += 8) {
    const int64_t l = l0 + k, a = a0 + tx;
    if (l < L && a < r32) {
      const float x = tile[tx][k];
      const float h = tf32_hi(x);
      const int64_t o = (z * L + l) * ld_out + a;
      hi[o] = h;
      lo[o] = tf32_hi(x - h);
    }
  }
}

cudaError_t launch_split_tf32_transpose(const float* W, int b, int64_t r, int64_t L, float* hi, float* lo,
                                        int64_t ld_out, cudaStream_t st) {
  if (b <= 0 || r <= 0 || L <= 0) return cudaSuccess;
  const dim3 grid((unsigned)((L + 31) / 32), (unsigned)((r + 31) / 32), (unsigned)b);
  note_launch();
  split_tf32_transpose_kernel<<<grid, dim3(32, 8), 0, st>>>(W, r, L, hi, lo, ld_out);
  return cudaGetLastError();
}

// Stage outputs from the FP64 sums of a transposed projection: W[z][n][l] = P[(z L + l) k + n] for
// n < k, l < L; w2[z] (optional) gains the squares.
__global__ void scatter_stage_kernel(const double* P, int64_t k, int64_t L, float* W, double* w2) {
  __shared__ double red[8];
  const int64_t z = blockIdx.y, per = k * L;
  double q = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t n = e / L, l = e - n * L;
    const double v = P[(z * L + l) * k + n];
    W[z * per + e] = (float)v;
    q = fma(v, v, q);
  }
  if (w2) {
    for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = q;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
      atomicAdd(w2 + z, t);
    }
  }
}

__global__ void pythagoras_kernel(const double* x2, const double* w2, int b, double* rho2) {
  const int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z < b) rho2[z] += x2[z] - w2[z];
}

__global__ void cols_above_kernel(const double* P, int64_t r, int64_t ld, double thr2, int* flag) {
  __shared__ double red[8];
  const double* p = P + (int64_t)blockIdx.x * ld;
  double q = 0.0;
  for (int64_t a = threadIdx.x; a < r; a += blockDim.x) q = fma(p[a], p[a], q);
  for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = q;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    if (!(t <= thr2)) atomicExch(flag, 1);  // also raised by NaN
  }
}

cudaError_t launch_cols_above(const double* P, int64_t r, int k, int64_t ld, double thr, int* flag,
                              cudaStream_t st) {
  if (k <= 0 || r <= 0) return cudaSuccess;
  note_launch();
  cols_above_kernel<<<k, 256, 0, st>>>(P, r, ld, thr * thr, flag);
  return cudaGetLastError();
}

cudaError_t launch_scatter_stage(const double* P, int b, int64_t k, int64_t L, float* W, double* w2,
                                 cudaStream_t st) {
  const int64_t per = k * L;
  if (b <= 0 || per <= 0) return cudaSuccess;
  const unsigned bx = (unsigned)std::min<int64_t>((per + 255) / 256, 256);
  note_launch();
  scatter_stage_kernel<<<dim3(bx, (unsigned)b), 256, 0, st>>>(P, k, L, W, w2);
  return cudaGetLastError();
}

cudaError_t launch_pythagoras(const double* x2, const double* w2, int b, double* rho2, cudaStream_t st) {
  if (b <= 0) return cudaSuccess;
  note_launch();
  pythagoras_kernel<<<(b + 255) / 256, 256, 0, st>>>(x2, w2, b, rho2);
  return cudaGetLastError();
}

cudaError_t launch_split_tf32(const float* in, int64_t ld_in, int64_t c0, int64_t c1, float* hi, float* lo,
                              int64_t ld_out, cudaStream_t st) {
  if (c1 <= c0 || ld_in <= 0) return cudaSuccess;
  const int64_t bx = std::min<int64_t>((ld_in + 255) / 256, 64);
  const int64_t by = std::min<int64_t>(c1 - c0, 1024);
  note_launch();
  split_tf32_kernel<<<dim3((unsigned)bx, (unsigned)by), 256, 0, st>>>(in, ld_in, c0, c1, hi, lo, ld_out);
  return cudaGetLastError();
}

}  // namespace ttice
