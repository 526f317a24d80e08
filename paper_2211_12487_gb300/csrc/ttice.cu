// libttice host side: the handle, the C-ABI entry points and the orchestration of one TT-ICE*
// increment (Algorithm 2) over the device kernels.
//
// Device state of a handle (all zero-initialised, so the padding of Eq. 11 is implicit):
//   U[i]   core i (0-based; the paper's U_{i+1}) as a column-major (cap_i n_i) x cap_{i+1} FP64 array.
//          Only the leading (r_i n_i) x r_{i+1} block is non-zero; appending a column (Eq. 10) writes
//          the next column, growing r_i appends zero rows at the bottom of U[i+1] for free.
//   Uf[i]  FP32 mirror of U[i] (used by the FP32 projections).
//   last   the last core (Eq. 13): row j = the r_d coefficients of observation j (ld cap_d), with the
//          implicit zero extension of Theorem 2.
// Stage buffers hold the chain of projections Y_{i+1} = reshape(U_i^T Y_i) (Eq. 12) observation-
// major: observation z, row a, column l at z*(r_{i+1} L_i) + a*L_i + l, which is also the (r_{i+1}
// n_{i+1}) x L_{i+1} unfolding consumed by the next stage.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "ttice_internal.cuh"

using namespace ttice;

// TTICE_TF32: the share of each increment's squared error bound (eps^2 ||Y||^2) reserved for the
// error of its one-product TF32 projections.  Every decision of Algorithm 2 (skip, subselection,
// eps_upd, the per-core thresholds) runs at eps sqrt(1 - kTf32Share), so the projections may move
// the squared errors they report, and the reconstruction through the coefficients they produce,
// by kTf32Share eps^2 ||Y||^2 before the bound eps ||Y|| of Theorem 1 can be exceeded.
// What the TF32 rounding (2^-11 relative per operand, unbiased) does to a Pythagorean residual
// ||x||^2 - ||U~^T x~||^2: the rounded core U~ is orthonormal only to ~2^-11 / sqrt(3 m) per column
// (m = r_{i-1} n_i rows), which moves ||w||^2 by about twice that times the energy along the column;
// and the rounded input x~ moves it by ~2^-11 ||x||^2 / sqrt(the entries holding its energy).  Both
// average out only on large stages, so a stage takes one product only from kTf32MinRows rows and
// kTf32MinEntries entries per observation (a few 1e-5 ||y||^2 per stage where the core's columns
// and the input's energy are spread); the small stages,
// the first pass's kernel, the residuals of the updated cores, the Grams, the re-orthogonalisation
// and the eigen-solve keep the split products.  The rule does not bound the effect for every input:
// columns of a core concentrated on few rows (2^-11 per column however large m is) or stage inputs
// whose energy sits in few entries keep it near 2^-11.  Measured with the rule in FP64 (numpy,
// TF32 operands rounded to nearest): up to 5.5e-5 ||y||^2 per observation on the 480p video stream
// (0.5% of eps^2 at eps = 0.1), up to 6.6e-4 ||y||^2 on the 64^3 x 4 flow stream (26% of eps^2 at
// eps = 0.05, 6.6% at eps = 0.1), where the cores' columns are localised.
constexpr double kTf32Share = 1.0 / 16.0;
constexpr int64_t kTf32MinRows = 256, kTf32MinEntries = 65536;

struct ttice_s {
  int d = 0;
  int device = 0;  // CUDA device the handle's buffers live on (current at creation)
  int64_t n[kMaxD] = {};
  int64_t L[kMaxD] = {};  // L[i] = n[i+1] * ... * n[d-1]
  int64_t N = 0;
  double eps = 0.0;
  ttice_heuristics h{};
  ttice_capacity capc{};
  int64_t cap[kMaxD + 1] = {};  // rank capacities, cap[0] = 1
  int64_t ldu[kMaxD] = {};      // rows of the U[i] allocation = cap[i] * n[i]
  int64_t r[kMaxD + 1] = {};    // ranks r_0..r_d (host mirror), r[0] = 1
  int last_new[kMaxD] = {};      // directions each core gained in its last truncation (sizes solver choice)
  double* U[kMaxD] = {};
  float* Uf[kMaxD] = {};
  // TF32 head / tail split of Uf for the tensor-core projections (mixed path): column-major, leading
  // dimension ldhl[i] (ldu rounded up to 32), hlcols[i] columns (cap rounded up to 256), zero beyond
  // the core; kept equal to split(Uf) column by column wherever Uf changes
  float* Uh[kMaxD] = {};
  float* Ul[kMaxD] = {};
  int64_t ldhl[kMaxD] = {};
  int64_t hlcols[kMaxD] = {};
  double* last = nullptr;
  int64_t last_cap = 0;  // observations
  int64_t n_obs = 0;
  int wt_bytes = 8;  // working type of stage buffers: 8 (FP64 path) or 4
  // tensor-core products of the large stage projections and new rows: 3 (split operands, FP32
  // accuracy) or 1 (TTICE_TF32: one TF32 product)
  int nprod = 3;
  // tolerance of the decisions (skip test, subselection, eps_upd, per-core thresholds): eps, or in
  // the TF32 mode eps sqrt(1 - kTf32Share), the rest of eps^2 left to the projection error
  double eps_dec = 0.0;
  // workspace
  void* stage[kMaxD] = {};
  void* dstage[kMaxD] = {};
  void* dgather = nullptr;
  void* Rbuf = nullptr;
  int64_t s_max = 0;
  double* G = nullptr;
  float* w32 = nullptr;
  float* V32 = nullptr;
  double* w64 = nullptr;
  double* V64 = nullptr;
  double* work64 = nullptr;
  double* bjw64 = nullptr;  // block Jacobi scratch (FP64 path)
  float* bjw32 = nullptr;   // block Jacobi scratch (FP32 eigenvectors of the mixed paths)
  double* fro = nullptr;
  int* bjflags = nullptr;
  double* Q = nullptr;   // s_max x kRR
  double* Q2 = nullptr;  // s_max x kRR
  double* GQ = nullptr;  // s_max x kRR
  double* Ssm = nullptr; // kRR x kRR
  double* Rinv = nullptr;
  double* H = nullptr;
  double* Z = nullptr;   // kRR x kRR eigenvectors
  double* theta = nullptr;
  float* G32 = nullptr;   // FP32 copy of the Gram for the Krylov solver
  // block Krylov with its basis in global memory (large Grams): basis (s x kBigK), G times it, two
  // s x kBigP work blocks, CGS coefficients (kBigK x kBigP), and the projected matrix (kBigK^2, FP64)
  float* BQ = nullptr;
  float* BGQ = nullptr;
  float* BY = nullptr;
  float* BY2 = nullptr;
  float* BC = nullptr;
  double* BH = nullptr;
  float* KQ = nullptr;    // block-Krylov basis, s_max x kKry
  float* kstart = nullptr;  // start block of a restarted Krylov solve, s_max x kKryP
  double* KV = nullptr;   // s_max x kKryP (start block), also kKry x kKry eigenvectors of H
  double* res = nullptr;  // Ritz residual norms
  double* h_dbl = nullptr;  // pinned host scratch
  double* Ebuf = nullptr;  // R V for a column-side Gram (m x s)
  int64_t max_ms = 0;
  double* Vn = nullptr;  // new directions, max_m x kRR
  const double* dir_src = nullptr;    // eigen / Ritz vectors of the current truncated SVD (s x K)
  const double* dir_scale = nullptr;  // their eigenvalues (column-side Grams: 1/sqrt scaling)
  bool dir_left = true;
  int64_t dir_s = 0;
  double* Vn2 = nullptr;
  double* P = nullptr;   // cap x kRR projections for CGS2
  // tensor-core CGS of the mixed path: TF32 head / tail of the new directions (ldv x kRR, ldv = max_m
  // rounded up to 32) and of their projections on the core (ldp x kRR, ldp = largest capacity
  // rounded up to 32)
  float* Vnh = nullptr;
  float* Vnl = nullptr;
  // mixed path: a block of up to kb[i] new directions of core i re-orthogonalised against the core's
  // earlier columns at once (VB, m x kb FP64, its TF32 head / tail at ld ldv) with its projections
  // (PB, FP64, and their split at ld ldp); kb[i] = 0 where the block would not fit kVBudget
  double* VB = nullptr;
  float* VBh = nullptr;
  float* VBl = nullptr;
  double* PB = nullptr;
  float* PBh = nullptr;
  float* PBl = nullptr;
  int kb[kMaxD] = {};
  float* Fh = nullptr;  // TF32 head / tail of I - R^{-1} of a tensor-core CholQR pass (kRR x kRR)
  float* Fl = nullptr;
  double* dsq = nullptr;  // FP64 squared column norms of the chunk (the Gram's diagonal), kRR
  double* sgn = nullptr;       // canonical sign of each new column (kRR)
  double* sgn_part = nullptr;  // its per-slice partial maxima (128 kRR)
  // tensor-core residual of the mixed path: the transposed TF32 split of U_i^T D_i (rows n = z L + l,
  // ld ldwt) and the TF32 split of the residual for its Gram; rlay = layout of the residual in Rbuf:
  // 0 the stage layout [z][i][l], 1 R^T (row n holds the m entries of column n), 2 R row-major
  // (row i holds the c = nsel L entries)
  float* WTh = nullptr;
  float* WTl = nullptr;
  float* Rh = nullptr;
  float* Rl = nullptr;
  int rlay = 0;
  int64_t wt_elems = 0, rs_elems = 0;  // sizes of WTh / WTl and of Rh / Rl (floats each)
  float* tcws = nullptr;  // split-K workspace of the tensor-core projections (tc_ws_elems floats)
  float* Ph = nullptr;
  float* Pl = nullptr;
  int64_t ldv = 0, ldp = 0;
  int64_t max_m = 0;
  double* rho2 = nullptr;    // squared residual per TT stage and observation (stage-major, d x b)
  double* h_rho2 = nullptr;  // pinned copy (first pass of an update)
  double* y2 = nullptr;
  double* rn2 = nullptr;    // per-observation ||R_i(z)||^2 of the residual being truncated
  double* h_rn2 = nullptr;  // pinned copy
  double* part = nullptr;  // per-CTA / per-tile partial norms of the first pass
  double* trace = nullptr;
  Decision* dec = nullptr;
  int* sel = nullptr;
  int* ibuf = nullptr;  // [0] rank, [1] eig status, [2] chol status, [3] nonfinite
  Decision* h_dec = nullptr;  // pinned
  int* h_sel = nullptr;       // pinned
  int* h_int = nullptr;       // pinned
  float* h_w32 = nullptr;     // pinned, s_max
  ttice_update_stats stats{};
  int64_t dev_bytes = 0;  // device memory held by this handle
  int miss_k = 0;         // rank index k whose capacity the last failed update needed to exceed (0: none)
  int64_t miss_need = 0;  // ... and the rank it needed
  // phase profiling
  bool prof_on = false;
  bool nvtx_open = false;  // a phase's NVTX range is open on this handle
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<std::pair<int, size_t>> marks;  // (phase, index of the start event; end = +1)
  ttice_profile prof{};
};

namespace {

enum Phase {
  PH_K1 = 0, PH_CHAIN = 1, PH_RESID = 2, PH_GRAM = 3, PH_EIG = 4, PH_ORTH = 5, PH_DPROJ = 6,
  PH_FINAL = 7
};

cudaEvent_t next_event(ttice_s* h) {
  if (h->ev_used == h->ev_pool.size()) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    h->ev_pool.push_back(e);
  }
  return h->ev_pool[h->ev_used++];
}

// Record the start of a phase and add its algorithmic bytes / flops.
// NVTX ranges name the phases on the host thread for profilers (ncu --nvtx --nvtx-include
// "ttice:eig/", nsys); they cost nothing measurable when no tool is attached.  At most one is open
// per handle: a phase closes the one an error path may have left open.
const char* const kPhaseNames[] = {"ttice:first_pass", "ttice:chain",      "ttice:residual",
                                   "ttice:gram",       "ttice:eig",        "ttice:orth_append",
                                   "ttice:d_project",  "ttice:final"};
void nvtx_close(ttice_s* h) {
  if (h->nvtx_open) {
    nvtxRangePop();
    h->nvtx_open = false;
  }
}
void ph_begin(ttice_s* h, int ph, cudaStream_t st, double bytes, double flops) {
  nvtx_close(h);
  nvtxRangePushA(kPhaseNames[ph]);
  h->nvtx_open = true;
  if (!h->prof_on) return;
  h->marks.push_back({ph, h->ev_used});
  cudaEventRecord(next_event(h), st);
  h->prof.bytes[ph] += bytes;
  h->prof.flops[ph] += flops;
  h->prof.count[ph] += 1;
}
void ph_end(ttice_s* h, cudaStream_t st) {
  nvtx_close(h);
  if (!h->prof_on) return;
  cudaEventRecord(next_event(h), st);
}
// After the stream has been synchronised: fold the recorded event pairs into the profile.
void ph_collect(ttice_s* h) {
  if (!h->prof_on) return;
  for (auto& m : h->marks) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev_pool[m.second], h->ev_pool[m.second + 1]) == cudaSuccess)
      h->prof.ms[m.first] += ms;
  }
  h->marks.clear();
  h->ev_used = 0;
}

constexpr int kRR = 96;         // largest Rayleigh-Ritz subspace
constexpr int kRRFast = 90;     // largest whose FP64 Jacobi runs in one CTA's shared memory
constexpr int kDirectEig = 32;  // Gram matrices up to this size are diagonalised in FP64 directly
constexpr int kDirectEig32 = 96;  // mixed path: FP32 Jacobi in one CTA up to this size
constexpr int kMaxEig = 4608;  // largest Gram side (128^3 x 4 flow: 33 x 128 = 4224)
constexpr int kMaxSweeps64 = 15;  // block Jacobi sweep limits (quadratic convergence needs ~6-10)
constexpr int kMaxSweeps32 = 12;
constexpr int kKryP = 8;         // block size of the Krylov eigen-solver
constexpr int kKryBlocks = 8;    // blocks: a basis of kKry = 64 vectors
constexpr int kKry = kKryP * kKryBlocks;
constexpr int kKrylovMin = 96;   // mixed path: Gram matrices above this size try the Krylov solver first
// Mixed path, Gram sides from kBigKrylovMin: a block Krylov basis of kBigK vectors in global memory
// (blocks of kBigP) is tried first.  Flat residual spectra (noise) have leading eigenvalues a few
// 1e-3 apart, which a 64-vector basis cannot resolve; 96 blocks of 8 certify the leading ~30 pairs
// of a 3840-sided Marchenko-Pastur spectrum to ~1e-14 in exact arithmetic.
constexpr int kBigP = 8;
constexpr int kBigBlocks = 96;
constexpr int kBigK = kBigP * kBigBlocks;
constexpr int kBigKrylovMin = 1024;
// Mixed path: new directions of a core are re-orthogonalised against its earlier columns in blocks
// of up to kBlockDirs (one pass over the core per block instead of per 96-column chunk), where the
// block's m x kb FP64 array stays within kVBudget doubles.
constexpr int64_t kBlockDirs = 768;
constexpr int64_t kVBudget = int64_t(64) << 20;
constexpr int64_t kMaxGridZ = 65535;  // batch (grid z) limit of one contraction launch

// The CUDA error behind the last TTICE_ECUDA returned to this thread (ttice_last_cuda_error).
thread_local cudaError_t g_last_cuda_error = cudaSuccess;

int cu(cudaError_t e) {
  if (e == cudaSuccess) return TTICE_OK;
  g_last_cuda_error = e;
  return TTICE_ECUDA;
}
#define TT_TRY(...)                      \
  do {                                   \
    int rc__ = (__VA_ARGS__);            \
    if (rc__ != TTICE_OK) return rc__;   \
  } while (0)
#define TT_CU(...) TT_TRY(cu(__VA_ARGS__))

// Device allocations made while a handle is being built are added to *g_alloc_sink.
thread_local int64_t* g_alloc_sink = nullptr;
// Dry run (ttice_projected_bytes): allocations are counted but not made, the pointers stay null.
thread_local bool g_dry_run = false;
// Test hook (ttice_test_fail_alloc): the allocation that takes this count from 1 to 0 fails.
std::atomic<long long> g_fail_alloc{0};

// A non-blocking stream private to the calling thread for the library's own set-up copies and
// fills (zeroing new buffers, moving cores to grown buffers), synchronised on its own: building or
// growing one handle never waits for, nor orders against, work that other threads have in flight.
cudaStream_t setup_stream() {
  thread_local cudaStream_t s = nullptr;
  if (!s && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    s = nullptr;
  }
  return s;
}

template <typename T>
int dalloc(T** p, int64_t count) {
  *p = nullptr;
  if (count <= 0) return TTICE_OK;
  if (g_dry_run) {
    if (g_alloc_sink) *g_alloc_sink += count * (int64_t)sizeof(T);
    return TTICE_OK;
  }
  if (g_fail_alloc.load(std::memory_order_relaxed) > 0 && g_fail_alloc.fetch_sub(1) == 1) {
    g_last_cuda_error = cudaErrorMemoryAllocation;  // injected: as if the device were full
    return TTICE_ENOMEM;
  }
  const cudaError_t me = cudaMalloc((void**)p, (size_t)count * sizeof(T));
  if (me != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    g_last_cuda_error = me;
    return TTICE_ENOMEM;
  }
  if (g_alloc_sink) *g_alloc_sink += count * (int64_t)sizeof(T);
  cudaStream_t fs = setup_stream();
  if (!fs) return cu(cudaErrorNotReady);
  TT_TRY(cu(cudaMemsetAsync(*p, 0, (size_t)count * sizeof(T), fs)));
  return cu(cudaStreamSynchronize(fs));
}
int dalloc_bytes(void** p, int64_t bytes) {
  return dalloc<unsigned char>(reinterpret_cast<unsigned char**>(p), bytes);
}

void free_all(ttice_s* h) {
  for (int i = 0; i < kMaxD; ++i) {
    cudaFree(h->U[i]); cudaFree(h->Uf[i]); cudaFree(h->stage[i]); cudaFree(h->dstage[i]);
    cudaFree(h->Uh[i]); cudaFree(h->Ul[i]);
  }
  void* ptrs[] = {h->G32, h->BQ, h->BGQ, h->BY, h->BY2, h->BC, h->BH, h->KQ, h->kstart, h->KV, h->res,
                  h->bjw64, h->bjw32, h->fro, h->bjflags,
                  h->last, h->dgather, h->Rbuf, h->G, h->w32, h->V32, h->w64, h->V64,
                  h->work64, h->Q, h->Q2, h->GQ, h->Ssm, h->Rinv, h->H, h->Z, h->theta, h->Vn,
                  h->Vn2, h->Ebuf, h->P, h->Vnh, h->Vnl, h->Fh, h->Fl, h->VB, h->VBh, h->VBl, h->PB, h->PBh, h->PBl, h->dsq, h->sgn, h->sgn_part, h->Ph, h->Pl, h->WTh, h->WTl, h->Rh, h->Rl, h->tcws, h->part, h->rho2, h->y2, h->rn2, h->trace, h->dec, h->sel, h->ibuf};
  for (void* p : ptrs) cudaFree(p);
  cudaFreeHost(h->h_dec); cudaFreeHost(h->h_sel); cudaFreeHost(h->h_int); cudaFreeHost(h->h_w32); cudaFreeHost(h->h_dbl);
  cudaFreeHost(h->h_rn2);
  cudaFreeHost(h->h_rho2);
}

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// ---------------------------------------------------------------- GEMM helpers
// W(z) = U_i^T X(z) for every observation z: M = r_{i+1}, K = m_i, N = L_i.
template <typename TU, typename TX, typename TW>
int proj(const TU* Ui, int64_t ldu, const TX* X, int64_t m, int64_t L, int64_t rnext, int b, TW* W,
         cudaStream_t st) {
  GemmArgs g;
  g.M = rnext; g.N = L; g.K = m;
  g.A.p = Ui; g.A.rs = ldu; g.A.cs = 1;
  g.B.p = X; g.B.rs = L; g.B.cs = 1; g.B.bs1 = m * L;
  g.C = W; g.c_rs = L; g.c_cs = 1; g.c_bs1 = rnext * L;
  g.nbatch = b;
  g.c_zero_elems = (int64_t)b * rnext * L;  // short-and-wide outputs (large m_i) split over K
  using ACC = typename std::conditional<sizeof(TW) == 8, double, float>::type;
  return cu(gemm<TU, TX, TX, TW, ACC>(g, st));
}

// R(z) = X(z) - U_i W(z); norm[z] += ||R(z)||^2; R stored iff R != nullptr.
template <typename TU, typename TW, typename TX, typename TR>
int resid(const TU* Ui, int64_t ldu, const TW* W, const TX* X, int64_t m, int64_t L, int64_t rnext,
          int b, TR* R, double* norm, cudaStream_t st) {
  GemmArgs g;
  g.M = m; g.N = L; g.K = rnext;
  g.A.p = Ui; g.A.rs = 1; g.A.cs = ldu;
  g.B.p = W; g.B.rs = L; g.B.cs = 1; g.B.bs1 = rnext * L;
  g.X.p = X; g.X.rs = L; g.X.cs = 1; g.X.bs1 = m * L;
  g.alpha = -1.0; g.beta = 1.0;
  g.C = R; g.c_rs = L; g.c_cs = 1; g.c_bs1 = m * L;
  g.store = R != nullptr;
  g.norm = norm;
  g.nbatch = b;
  using ACC = typename std::conditional<sizeof(TW) == 8, double, float>::type;
  return cu(gemm<TU, TW, TX, TR, ACC>(g, st));
}

template <typename T>
int sumsq(const T* X, int b, int64_t n, double* out, cudaStream_t st) {
  return cu(launch_sum_squares<T>(X, b, n, out, st));
}

// Stage i of the mixed path on the tensor cores: FP32 stage input X (the increment for i = 0, a stage
// buffer otherwise) in a layout the projection kernel takes.
bool tc_stage(const ttice_s* h, int i, const void* X) {
  return h->Uh[i] != nullptr && h->r[i + 1] > 0 &&
         tc_proj_supported(X, h->L[i], h->r[i] * h->n[i], (int)h->r[i + 1], h->ldhl[i]);
}
// Products of stage i's projection on the tensor cores: one in the TF32 mode on a large stage, else
// the three of the split operands.
int stage_nprod(const ttice_s* h, int i) {
  const int64_t m = h->r[i] * h->n[i];
  return (h->nprod == 1 && m >= kTf32MinRows && m * h->L[i] >= kTf32MinEntries) ? 1 : 3;
}
int tc_project(ttice_s* h, int i, const void* X, int b, void* W, double* x2, double* rho2, cudaStream_t st) {
  return cu(launch_tc_proj(static_cast<const float*>(X), b, h->L[i], h->r[i] * h->n[i], (int)h->r[i + 1], h->Uh[i],
                           h->Ul[i], h->ldhl[i], h->hlcols[i], static_cast<float*>(W), x2, rho2, h->part, h->tcws,
                           h->ibuf + 5, st, stage_nprod(h, i)));
}

// Stages of the mixed path whose unfolding has too few or unaligned columns per observation for the
// projection kernel's tile layouts (L_i not a multiple of 4: the 1080p view's last core has L = 3):
// the stage input transposed and split (rows z L + l, K = its m rows), against columns [r0, r0 + k)
// of U_i's split on the tensor cores with FP64 sums across K splits (the output, k x b L, cannot fill
// the GPU by itself), then scattered to the stage layout [z][n][l] in FP32.  With rho2:
// rho2[z] += ||X_z||^2 - ||W_z||^2.
constexpr double kTcStageTMin = 2e8;  // m k b L below which the SIMT GEMM is as fast
// Mixed path: the CGS work m r k above which its two passes run on the tensor cores (the FP64
// products would take more than a few milliseconds at GB300's FP64 rate).
constexpr double kTcCgsMin = 4e9;
std::atomic<double> g_tc_cgs_min{kTcCgsMin};  // ttice_test_tc_cgs_min (0 forces the tensor-core forms)
bool tc_stage_t_ok(const ttice_s* h, int i, int b, int64_t k) {
  const int64_t m = h->r[i] * h->n[i], L = h->L[i], ldm = (m + 31) / 32 * 32;
  return h->Uh[i] != nullptr && k > 0 && m >= 32 && (m + 31) / 32 <= 65535 && b * L * ldm <= h->rs_elems &&
         b * L * k <= h->max_ms && (double)m * k * b * L >= std::min(kTcStageTMin, g_tc_cgs_min.load());
}
int tc_project_t(ttice_s* h, int i, const float* X, int b, int64_t r0, int k, float* W, double* rho2,
                 cudaStream_t st) {
  const int64_t m = h->r[i] * h->n[i], L = h->L[i], ldm = (m + 31) / 32 * 32;
  double* P = h->Ebuf;  // b L x k
  TT_CU(launch_split_tf32_transpose(X, b, m, L, h->Rh, h->Rl, ldm, st));
  TT_CU(cudaMemsetAsync(P, 0, (size_t)b * L * k * sizeof(double), st));
  TcGemm g;  // P[z L + l][n] = sum_a X[z][a][l] U[a][r0 + n]
  g.ah = h->Rh; g.al = h->Rl; g.lda = ldm; g.la_alloc = b * L;
  g.L = b * L; g.K = m;
  g.bh = h->Uh[i] + r0 * h->ldhl[i]; g.bl = h->Ul[i] + r0 * h->ldhl[i]; g.ldb = h->ldhl[i];
  g.nb_alloc = h->hlcols[i] - r0;
  g.r = k;
  g.mode = 5; g.out = P; g.ldn = 1; g.ldl = k;
  g.status = h->ibuf + 5;
  g.nprod = stage_nprod(h, i);
  TT_CU(launch_tc_gemm(g, st));
  if (rho2) {
    TT_CU(cudaMemsetAsync(h->part, 0, 2 * (size_t)b * sizeof(double), st));
    TT_TRY(sumsq<float>(X, b, m * L, h->part, st));
  }
  TT_CU(launch_scatter_stage(P, b, k, L, W, rho2 ? h->part + b : nullptr, st));
  if (rho2) TT_CU(launch_pythagoras(h->part, h->part + b, b, rho2, st));
  return TTICE_OK;
}

// ---------------------------------------------------------------- chain projection
// Project b observations of X0 (stage-0 layout) through U_1..U_d into `bufs`; with `errors`,
// rho2[i b + z] = ||R_i(z)||^2 for every stage i (their sum over i is ||y_z - ~y_z||^2, the orthogonal
// decomposition) and y2[z] = ||y_z||^2.  Without `errors`, `first` > 0 starts at stage `first` from
// the stage output already in bufs[first - 1].
template <typename WT, typename TY>
int chain(ttice_s* h, const TY* X0, int b, void** bufs, bool errors, cudaStream_t st, int first = 0) {
  if (errors) first = 0;
  const WT* Xw = first > 0 ? static_cast<const WT*>(bufs[first - 1]) : nullptr;
  const double sw = sizeof(WT), sy = sizeof(TY);
  // stage 1 of the mixed path on the tensor cores (FP32 increment and cores): the dedicated first-pass
  // kernel where it applies (n_1 <= 128, r_1 <= 64: K is a few chunks, and the projection kernel's
  // per-item pipeline would dominate; measured 0.30 against 0.57 ms on a 537 MB flow batch), else the
  // projection kernel
  const bool k1_fits = sizeof(TY) == 4 && sizeof(WT) == 4 && first == 0 && h->r[1] > 0 &&
                       k1_tc_supported(X0, h->L[0], (int)h->n[0], (int)h->r[1]);
  const bool tc0 = sizeof(TY) == 4 && sizeof(WT) == 4 && first == 0 && !k1_fits && tc_stage(h, 0, X0);
  const bool tc_k1 = !tc0 && sizeof(TY) == 4 && sizeof(WT) == 4 && first == 0 && h->r[1] > 0 &&
                     k1_tc_supported(X0, h->L[0], (int)h->n[0], (int)h->r[1]);
  const bool fused_k1 =
      errors && h->r[1] > 0 && (tc0 || tc_k1 || k1_supported<TY, WT>((int)h->n[0], (int)h->r[1]));
  if (errors) {
    TT_CU(cudaMemsetAsync(h->rho2, 0, (size_t)h->d * b * sizeof(double), st));
    TT_CU(cudaMemsetAsync(h->y2, 0, b * sizeof(double), st));
    TT_CU(cudaMemsetAsync(h->ibuf + 5, 0, sizeof(int), st));
    const double N = (double)h->N, r1 = (double)h->r[1];
    ph_begin(h, PH_K1, st, b * (sy * N + sw * r1 * h->L[0]), b * (4.0 * N * r1 + 4.0 * N));
    if (!fused_k1) TT_TRY(sumsq<TY>(X0, b, h->N, h->y2, st));
  } else {
    double by = first > 0 ? sw * b * (double)h->r[first] * h->L[first - 1] : sy * b * h->N, fl = 0.0;
    for (int i = first; i < h->d; ++i) {
      const double out = (double)b * h->r[i + 1] * h->L[i];
      by += sw * out * (i + 1 < h->d ? 2.0 : 1.0);
      fl += 2.0 * b * (double)h->r[i] * h->n[i] * h->L[i] * h->r[i + 1];
    }
    ph_begin(h, PH_FINAL, st, by, fl);
  }
  for (int i = first; i < h->d; ++i) {
    const int64_t m = h->r[i] * h->n[i], rn = h->r[i + 1], L = h->L[i];
    WT* W = static_cast<WT*>(bufs[i]);
    if (errors && i == 1) {
      ph_end(h, st);
      double by = 0.0, fl = 0.0;
      for (int j = 1; j < h->d; ++j) {
        const double mj = (double)h->r[j] * h->n[j];
        by += sw * b * (mj * h->L[j] + (double)h->r[j + 1] * h->L[j]);
        // the projection, and on the FP64 path the back-projection of the direct residual too (the
        // mixed path takes the residual norm by Pythagoras)
        fl += (double)b * h->L[j] * ((sizeof(WT) == 4 ? 2.0 : 4.0) * mj * h->r[j + 1] + 2.0 * mj);
      }
      ph_begin(h, PH_CHAIN, st, by, fl);
    }
    if (rn == 0 || m == 0) {
      // nothing is represented from here on: the whole remaining stage is residual
      if (errors && m > 0) {
        if (i == 0) TT_TRY(sumsq<TY>(X0, b, m * L, h->rho2, st));
        else TT_TRY(sumsq<WT>(Xw, b, m * L, h->rho2 + (int64_t)i * b, st));
      }
      // zero the coefficients of the remaining stages
      for (int j = i; j < h->d; ++j) {
        const int64_t sz = (int64_t)b * h->r[j + 1] * h->L[j];
        if (sz > 0) TT_CU(cudaMemsetAsync(bufs[j], 0, sz * sizeof(WT), st));
      }
      ph_end(h, st);
      return TTICE_OK;
    }
    const WT* Ui = (sizeof(WT) == 8) ? reinterpret_cast<const WT*>(h->U[i])
                                     : reinterpret_cast<const WT*>(h->Uf[i]);
    if (i == 0 && tc0) {
      TT_TRY(tc_project(h, 0, X0, b, W, errors ? h->y2 : nullptr, errors ? h->rho2 : nullptr, st));
    } else if (i == 0 && tc_k1) {
      TT_CU(launch_k1_tc(reinterpret_cast<const float*>(X0), b, L, (int)m, (int)rn,
                         reinterpret_cast<const float*>(Ui), h->ldu[i], reinterpret_cast<float*>(W),
                         errors ? h->y2 : nullptr, errors ? h->rho2 : nullptr, h->part, h->ibuf + 5, st));
    } else if (i == 0 && fused_k1) {
      if constexpr (sizeof(TY) == 4) {
        if (k1_tma_supported(X0, L, (int)m, (int)rn)) {
          TT_CU((launch_k1_tma<WT>(reinterpret_cast<const float*>(X0), b, L, (int)m, (int)rn, Ui,
                                   h->ldu[i], W, h->y2, h->rho2, h->part, h->ibuf + 5, st)));
        } else {
          TT_CU((launch_k1<TY, WT>(X0, b, L, (int)m, (int)rn, Ui, h->ldu[i], W, h->y2, h->rho2, h->part, st)));
        }
      } else {
        TT_CU((launch_k1<TY, WT>(X0, b, L, (int)m, (int)rn, Ui, h->ldu[i], W, h->y2, h->rho2, h->part, st)));
      }
    } else if (i == 0 && !errors && sizeof(TY) == 4 && k1_tma_supported(X0, L, (int)m, (int)rn)) {
      TT_CU((launch_k1_tma<WT>(reinterpret_cast<const float*>(X0), b, L, (int)m, (int)rn, Ui,
                               h->ldu[i], W, nullptr, nullptr, nullptr, h->ibuf + 5, st)));
    } else if (i == 0) {
      TT_TRY(proj<WT, TY, WT>(Ui, h->ldu[i], X0, m, L, rn, b, W, st));
      if (errors) TT_TRY((resid<WT, WT, TY, WT>(Ui, h->ldu[i], W, X0, m, L, rn, b, nullptr, h->rho2, st)));
    } else if (sizeof(WT) == 4 && tc_stage(h, i, Xw)) {
      // Pythagorean residual per observation: ||X_i||^2 - ||U_i^T X_i||^2
      TT_TRY(tc_project(h, i, Xw, b, W, nullptr, errors ? h->rho2 + (int64_t)i * b : nullptr, st));
    } else if (sizeof(WT) == 4 && tc_stage_t_ok(h, i, b, rn)) {
      TT_TRY(tc_project_t(h, i, reinterpret_cast<const float*>(Xw), b, 0, (int)rn, reinterpret_cast<float*>(W),
                          errors ? h->rho2 + (int64_t)i * b : nullptr, st));
    } else {
      TT_TRY(proj<WT, WT, WT>(Ui, h->ldu[i], Xw, m, L, rn, b, W, st));
      if (errors)
        TT_TRY((resid<WT, WT, WT, WT>(Ui, h->ldu[i], W, Xw, m, L, rn, b, nullptr, h->rho2 + (int64_t)i * b, st)));
    }
    Xw = W;
  }
  ph_end(h, st);
  return TTICE_OK;
}

int sync_read(ttice_s* h, cudaStream_t st) {
  TT_CU(cudaStreamSynchronize(st));
  return TTICE_OK;
}

// FP64 Rayleigh-Ritz on the K candidate vectors in h->Q (s x K): orthonormalise them (CholQR2),
// form H = Q^T G Q, diagonalise it (FP64 Jacobi), apply the rank rule to the Ritz values
// (tail = trace - sum theta, Eq. 5) and leave the Ritz vectors in h->Q2 and values in h->theta.
int rayleigh_ritz(ttice_s* h, int64_t s, int K, const double* d_eps, int max_new, cudaStream_t st) {
  // CholQR2: orthonormalise Q in FP64
  for (int pass = 0; pass < 2; ++pass) {
    TT_CU(cudaMemsetAsync(h->Ssm, 0, (size_t)K * K * sizeof(double), st));
    GemmArgs g;  // S = Q^T Q
    g.M = K; g.N = K; g.K = s; g.atomic = 1; g.allow_splitk = 1;
    g.A.p = h->Q; g.A.rs = s; g.A.cs = 1;
    g.B.p = h->Q; g.B.rs = 1; g.B.cs = s;
    g.C = h->Ssm; g.c_rs = 1; g.c_cs = K;
    TT_CU((gemm<double, double, double, double, double>(g, st)));
    TT_CU(launch_chol_inv(h->Ssm, K, h->Rinv, h->ibuf + 2, st));
    GemmArgs q;  // Q2 = Q Rinv
    q.M = s; q.N = K; q.K = K;
    q.A.p = h->Q; q.A.rs = 1; q.A.cs = s;
    q.B.p = h->Rinv; q.B.rs = 1; q.B.cs = K;
    q.C = h->Q2; q.c_rs = 1; q.c_cs = s;
    TT_CU((gemm<double, double, double, double, double>(q, st)));
    std::swap(h->Q, h->Q2);
  }
  {  // GQ = G Q ; H = Q^T GQ
    GemmArgs g;
    g.M = s; g.N = K; g.K = s; g.atomic = 1; g.allow_splitk = 1;
    g.A.p = h->G; g.A.rs = s; g.A.cs = 1;
    g.B.p = h->Q; g.B.rs = 1; g.B.cs = s;
    g.C = h->GQ; g.c_rs = 1; g.c_cs = s;
    TT_CU(cudaMemsetAsync(h->GQ, 0, (size_t)s * K * sizeof(double), st));
    TT_CU((gemm<double, double, double, double, double>(g, st)));
    TT_CU(cudaMemsetAsync(h->H, 0, (size_t)K * K * sizeof(double), st));
    GemmArgs hh;
    hh.M = K; hh.N = K; hh.K = s; hh.atomic = 1; hh.allow_splitk = 1;
    hh.A.p = h->Q; hh.A.rs = s; hh.A.cs = 1;
    hh.B.p = h->GQ; hh.B.rs = 1; hh.B.cs = s;
    hh.C = h->H; hh.c_rs = K; hh.c_cs = 1;
    TT_CU((gemm<double, double, double, double, double>(hh, st)));
  }
  TT_CU(jacobi_eig<double>(h->H, K, K, h->theta, h->Z, h->work64, h->ibuf + 1, st));
  TT_CU(launch_rank_rule(h->theta, K, K == s, h->trace, d_eps, max_new, h->ibuf, st));
  {  // Ritz vectors Q2 = Q Z
    GemmArgs g;
    g.M = s; g.N = K; g.K = K;
    g.A.p = h->Q; g.A.rs = 1; g.A.cs = s;
    g.B.p = h->Z; g.B.rs = 1; g.B.cs = K;
    g.C = h->Q2; g.c_rs = 1; g.c_cs = s;
    TT_CU((gemm<double, double, double, double, double>(g, st)));
  }
  return TTICE_OK;
}

// Candidate eigenvectors for the leading part of the Gram G (s x s) from a block Krylov subspace
// built in FP32 (an FP32 copy of G) by one thread-block cluster: X_0 = orth(random s x p),
// X_i = orth((I - Q Q^T) G X_{i-1}) (CGS2 against the basis Q = [X_0 .. X_{i-1}]), kKryBlocks
// blocks, and H = Q^T G Q (FP32 products, FP64 accumulation across CTAs).  H is diagonalised by FP32
// Jacobi and its leading K eigenvectors, mapped back to R^s in FP64, are left in h->Q for the FP64
// Rayleigh-Ritz step, which alone decides the rank.
// *K_out = 0 when the subspace is too small for the tolerance.
int krylov_candidates(ttice_s* h, int64_t s, double eps_c, int nblk, const float* start, int* K_out,
                       cudaStream_t st) {
  *K_out = 0;
  float* Qb = h->KQ;
  const int k = nblk * kKryP;
  TT_CU(cudaMemsetAsync(h->ibuf + 6, 0, sizeof(int), st));
  TT_CU(launch_krylov(h->G, h->G32, s, nblk, Qb, h->H, h->ibuf + 6, 0x5eedull + (uint64_t)s, start, st));
  TT_CU(cudaMemsetAsync(h->bjflags, 0, 4 * sizeof(int), st));
  TT_CU(jacobi_eig<float>(h->H, k, k, h->w32, h->V32, h->bjw32, h->bjflags + 3, st));
  TT_CU(cudaMemcpyAsync(h->h_w32, h->w32, k * sizeof(float), cudaMemcpyDeviceToHost, st));
  TT_CU(cudaMemcpyAsync(h->h_dbl, h->trace, sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_CU(cudaMemcpyAsync(h->h_int + 6, h->ibuf + 6, sizeof(int), cudaMemcpyDeviceToHost, st));
  ph_end(h, st);
  TT_TRY(sync_read(h, st));
  ph_begin(h, PH_EIG, st, 0.0, 0.0);
  if (h->h_int[6]) return TTICE_OK;  // the Krylov blocks lost rank: leave it to the full solver
  // leading part needed: smallest r with trace - sum_{j<r} theta_j <= eps^2 (sizes the RR step)
  const double tr = h->h_dbl[0];
  double acc = 0.0;
  int r32 = -1;
  if (std::sqrt(std::max(tr, 0.0)) <= eps_c) r32 = 0;
  for (int j = 0; j < k && r32 < 0; ++j) {
    acc += std::max((double)h->h_w32[j], 0.0);
    if (std::sqrt(std::max(tr - acc, 0.0)) <= eps_c) r32 = j + 1;
  }
  if (r32 < 0 || r32 + 8 > k - 8) return TTICE_OK;  // subspace too small: full solver
  const int K = std::min(k, r32 + 8);
  // candidates Q = Q_krylov V[:, :K] in FP64
  TT_CU(launch_to_f64<float>(h->V32, (int64_t)k * K, h->KV, st));
  GemmArgs c;
  c.M = s; c.N = K; c.K = k;
  c.A.p = Qb; c.A.rs = 1; c.A.cs = s;
  c.B.p = h->KV; c.B.rs = 1; c.B.cs = k;
  c.C = h->Q; c.c_rs = 1; c.c_cs = s;
  TT_CU((gemm<float, double, double, double, double>(c, st)));
  *K_out = K;
  return TTICE_OK;
}

// Large Grams (s >= kBigKrylovMin, mixed path): block Krylov with the basis in global memory, FP32
// products.  X_0 pseudo-random; X_i = G X_{i-1} projected out of the earlier blocks twice (CGS2) and
// orthonormalised by Cholesky-QR twice; H = Q^T G Q in FP64 sums, diagonalised by FP32 Jacobi; the
// leading Ritz vectors the rank rule needs (plus 8) become the FP64 candidates h->Q of the
// Rayleigh-Ritz step.  *K_out = 0 when the blocks lost rank or the subspace is too small.
int krylov_big_candidates(ttice_s* h, int64_t s, double eps_c, int* K_out, cudaStream_t st) {
  *K_out = 0;
  const int P = kBigP, k = kBigK;
  float* Q = h->BQ;
  TT_CU((launch_cast<double, float>(h->G, h->G32, s * s, st)));
  TT_CU(cudaMemsetAsync(h->ibuf + 6, 0, sizeof(int), st));
  TT_CU(launch_fill_random(h->BY, s * P, 0x5eedull + (uint64_t)s, st));
  for (int i = 0; i < kBigBlocks; ++i) {
    const int64_t q0 = (int64_t)i * P;  // columns of the basis so far
    if (i > 0) {
      GemmArgs y;  // Y = G X_{i-1}
      y.M = s; y.N = P; y.K = s;
      y.A.p = h->G32; y.A.rs = s; y.A.cs = 1;
      y.B.p = Q + (q0 - P) * s; y.B.rs = 1; y.B.cs = s;
      y.C = h->BY; y.c_rs = 1; y.c_cs = s;
      TT_CU((gemm<float, float, float, float, float>(y, st)));
      for (int pass = 0; pass < 2; ++pass) {
        TT_CU(cudaMemsetAsync(h->BC, 0, (size_t)q0 * P * sizeof(float), st));
        GemmArgs c;  // C = Q^T Y
        c.M = q0; c.N = P; c.K = s; c.atomic = 1; c.allow_splitk = 1;
        c.A.p = Q; c.A.rs = s; c.A.cs = 1;
        c.B.p = h->BY; c.B.rs = 1; c.B.cs = s;
        c.C = h->BC; c.c_rs = 1; c.c_cs = q0;
        TT_CU((gemm<float, float, float, float, float>(c, st)));
        GemmArgs u;  // Y -= Q C
        u.M = s; u.N = P; u.K = q0;
        u.A.p = Q; u.A.rs = 1; u.A.cs = s;
        u.B.p = h->BC; u.B.rs = 1; u.B.cs = q0;
        u.X.p = h->BY; u.X.rs = 1; u.X.cs = s;
        u.alpha = -1.0; u.beta = 1.0;
        u.C = h->BY; u.c_rs = 1; u.c_cs = s;
        TT_CU((gemm<float, float, float, float, float>(u, st)));
      }
    }
    for (int pass = 0; pass < 2; ++pass) {  // CholQR2 of the block into the basis
      const float* src = pass == 0 ? h->BY : h->BY2;
      float* dst = pass == 0 ? h->BY2 : Q + q0 * s;
      TT_CU(cudaMemsetAsync(h->Ssm, 0, (size_t)P * P * sizeof(double), st));
      GemmArgs g;  // S = Y^T Y
      g.M = P; g.N = P; g.K = s; g.atomic = 1; g.allow_splitk = 1;
      g.A.p = src; g.A.rs = s; g.A.cs = 1;
      g.B.p = src; g.B.rs = 1; g.B.cs = s;
      g.C = h->Ssm; g.c_rs = 1; g.c_cs = P;
      TT_CU((gemm<float, float, float, double, double>(g, st)));
      TT_CU(launch_chol_inv(h->Ssm, P, h->Rinv, h->ibuf + 6, st));
      GemmArgs q;  // Y Rinv
      q.M = s; q.N = P; q.K = P;
      q.A.p = src; q.A.rs = 1; q.A.cs = s;
      q.B.p = h->Rinv; q.B.rs = 1; q.B.cs = P;
      q.C = dst; q.c_rs = 1; q.c_cs = s;
      TT_CU((gemm<float, double, float, float, float>(q, st)));
    }
  }
  {  // H = Q^T (G Q)
    GemmArgs g;
    g.M = s; g.N = k; g.K = s;
    g.A.p = h->G32; g.A.rs = s; g.A.cs = 1;
    g.B.p = Q; g.B.rs = 1; g.B.cs = s;
    g.C = h->BGQ; g.c_rs = 1; g.c_cs = s;
    TT_CU((gemm<float, float, float, float, float>(g, st)));
    TT_CU(cudaMemsetAsync(h->BH, 0, (size_t)k * k * sizeof(double), st));
    GemmArgs hh;
    hh.M = k; hh.N = k; hh.K = s; hh.atomic = 1; hh.allow_splitk = 1;
    hh.A.p = Q; hh.A.rs = s; hh.A.cs = 1;
    hh.B.p = h->BGQ; hh.B.rs = 1; hh.B.cs = s;
    hh.C = h->BH; hh.c_rs = 1; hh.c_cs = k;
    TT_CU((gemm<float, float, float, double, double>(hh, st)));
  }
  TT_CU(block_jacobi_eig<float>(h->BH, k, k, h->w32, h->V32, h->bjw32, h->fro, h->bjflags, kMaxSweeps32, st));
  TT_CU(cudaMemcpyAsync(h->h_w32, h->w32, k * sizeof(float), cudaMemcpyDeviceToHost, st));
  TT_CU(cudaMemcpyAsync(h->h_dbl, h->trace, sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_CU(cudaMemcpyAsync(h->h_int + 6, h->ibuf + 6, sizeof(int), cudaMemcpyDeviceToHost, st));
  TT_CU(cudaMemcpyAsync(h->h_int + 8, h->bjflags, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  ph_end(h, st);
  TT_TRY(sync_read(h, st));
  ph_begin(h, PH_EIG, st, 0.0, 0.0);
  if (h->prof_on) h->prof.flops[PH_EIG] += 8.0 * (double)k * k * k * h->h_int[10];
  if (h->h_int[6]) return TTICE_OK;  // the blocks lost rank: leave it to the full solver
  const double tr = h->h_dbl[0];
  double acc = 0.0;
  int r32 = -1;
  if (std::sqrt(std::max(tr, 0.0)) <= eps_c) r32 = 0;
  for (int j = 0; j < k && r32 < 0; ++j) {
    acc += std::max((double)h->h_w32[j], 0.0);
    if (std::sqrt(std::max(tr - acc, 0.0)) <= eps_c) r32 = j + 1;
  }
  if (r32 < 0 || r32 + 8 > kRR) return TTICE_OK;  // more than one Rayleigh-Ritz problem: full solver
  const int K = r32 + 8;
  GemmArgs c;  // candidates Q V[:, :K] in FP64
  c.M = s; c.N = K; c.K = k;
  c.A.p = Q; c.A.rs = 1; c.A.cs = s;
  c.B.p = h->V32; c.B.rs = 1; c.B.cs = k;
  c.C = h->Q; c.c_rs = 1; c.c_cs = s;
  TT_CU((gemm<float, float, float, double, double>(c, st)));
  *K_out = K;
  return TTICE_OK;
}

// After rayleigh_ritz: accept the Krylov result iff every Ritz pair the rank rule used has a
// residual ||G z - theta z|| <= 1e-6 theta_1, i.e. the Ritz values are converged far below the
// truncation threshold (errors are second order in the residual).  The rule at rank rR reads
// theta_1 .. theta_rR only (tail(rR) <= eps^2 < tail(rR - 1)), and those are also the directions
// appended, so the leading rR pairs are checked.
int krylov_certify(ttice_s* h, int64_t s, int K, bool* ok, cudaStream_t st) {
  *ok = false;
  // G z_j for all K Ritz vectors z = Q Z: (G Q) Z from the G Q the Rayleigh-Ritz step formed, an
  // s x K x K product instead of s x s x K (the two differ by FP64 rounding); their residuals are
  // read together with the rank the rule chose, in one host round trip
  GemmArgs g;
  g.M = s; g.N = K; g.K = K;
  g.A.p = h->GQ; g.A.rs = 1; g.A.cs = s;
  g.B.p = h->Z; g.B.rs = 1; g.B.cs = K;
  g.C = h->Vn2; g.c_rs = 1; g.c_cs = s;
  TT_CU((gemm<double, double, double, double, double>(g, st)));
  TT_CU(launch_ritz_residual(h->Vn2, h->Q2, h->theta, s, K, h->res, st));
  TT_CU(cudaMemcpyAsync(h->h_int, h->ibuf, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  TT_CU(cudaMemcpyAsync(h->h_dbl, h->res, K * sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_CU(cudaMemcpyAsync(h->h_dbl + 128, h->theta, sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_TRY(sync_read(h, st));
  const int rR = h->h_int[0];
  if (rR < 0) return TTICE_OK;
  // rR = 0 is decided by the trace alone (no Ritz value enters it)
  if (rR == 0) { *ok = true; return TTICE_OK; }
  const int jm = std::min(rR, K);
  const double tol = 1e-6 * std::max(h->h_dbl[128], 0.0);
  bool good = true;
  for (int j = 0; j < jm; ++j) good = good && (h->h_dbl[j] <= tol);
  *ok = good;
  return TTICE_OK;
}

// After krylov_certify turned a Krylov result down (some Ritz pair the rule used has a residual above
// 1e-6 theta_1, as in flat spectra whose leading eigenvalues lie 1e-3 apart): accept the rank
// decision itself when its margin exceeds what the residuals allow.  With Ritz values theta_j and
// Ritz vectors Z (the rule's leading rR) and residual matrix G Z - Z Theta of Frobenius norm rho,
// G - E (||E|| <= 2 rho) has span(Z) as an invariant subspace, so the leading eigenvalues of G
// exceed the matching Ritz values by at most 2 rho each (Weyl), given that the Krylov space holds the
// leading eigenvectors (a random start).  The rule's
// rank rR has Ritz tail(rR) <= eps^2, which bounds the true tail of the appended directions exactly
// (their captured energy is the sum of their Ritz values); the true rank is rR as well when
// tail(rR - 1) - 2 rho (rR - 1) > eps^2.  Reads the residuals krylov_certify left in h->h_dbl.
int krylov_margin_ok(ttice_s* h, int K, double eps_c, bool* ok, cudaStream_t st) {
  *ok = false;
  const int rR = h->h_int[0];
  if (rR <= 0 || rR > K) return TTICE_OK;
  TT_CU(cudaMemcpyAsync(h->h_dbl + 130, h->theta, K * sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_CU(cudaMemcpyAsync(h->h_dbl + 250, h->trace, sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_TRY(sync_read(h, st));
  double rho2 = 0.0;
  for (int j = 0; j < rR; ++j) rho2 += h->h_dbl[j] * h->h_dbl[j];
  const double tr = h->h_dbl[250];
  double tail = tr;  // tail(rR - 1) from the Ritz values
  for (int j = 0; j < rR - 1; ++j) tail -= h->h_dbl[130 + j];
  const double slack = 2.0 * std::sqrt(rho2) * (rR - 1) + 1e-12 * std::fabs(tr);
  *ok = tail - slack > eps_c * eps_c;
  return TTICE_OK;
}

// Energy of R along each eigenvector of its Gram held in h->V64 (s x s, a complete basis),
// measured on R itself (||q_j^T R||^2 or ||R v_j||^2) into h->theta, so that the truncation tail
// does not inherit the squared rounding of the Gram matrix.  The basis is complete, so these
// energies sum to ||R||^2 and the tail is summed directly.
template <typename WT>
int measure_energies(ttice_s* h, const WT* R, int64_t m, int64_t L, int nsel, int64_t s, bool left,
                     cudaStream_t st) {
  double* e = h->theta;
  TT_CU(cudaMemsetAsync(e, 0, s * sizeof(double), st));
  // FP64 path: FP64 products of FP64 residuals.  Mixed path (FP32 residual): FP32 products of the
  // FP32 residual and the FP32 eigenvectors, accumulated in FP64 (the residual itself carries FP32
  // rounding, so FP64 products would add no accuracy and cost 64x on GB300).
  using VT = WT;
  const VT* V = (sizeof(WT) == 8) ? reinterpret_cast<const VT*>(h->V64) : reinterpret_cast<const VT*>(h->V32);
  using ACC = typename std::conditional<sizeof(WT) == 8, double, float>::type;
  const int64_t c = L * nsel;
  if (left) {
    GemmArgs g;  // E = V^T R, row norms
    g.M = s; g.N = L; g.K = m;
    g.A.p = V; g.A.rs = s; g.A.cs = 1;
    g.B.p = R; g.B.rs = L; g.B.cs = 1; g.B.bs1 = m * L;
    if (h->rlay == 2) { g.N = c; g.B.rs = c; g.B.bs1 = 0; }  // row-major R: one m x c matrix
    g.store = 0; g.norm = e; g.norm_rows = 1;
    g.nbatch = h->rlay == 2 ? 1 : nsel;
    TT_CU((gemm<VT, WT, double, double, ACC>(g, st)));
  } else if (sizeof(WT) == 4 && h->rlay == 1 && h->Rh && s * ((s + 31) / 32 * 32) <= h->rs_elems) {
    // E = R V (m x s) on the tensor cores: R^T (rows n, the m entries of column n of R) as the
    // A operand, the split FP32 eigenvectors as the B operand; then the column norms
    const int64_t lds = (s + 31) / 32 * 32;
    TT_CU(launch_split_tf32(reinterpret_cast<const float*>(V), s, 0, s, h->Rh, h->Rl, lds, st));
    TcGemm g;
    g.x = reinterpret_cast<const float*>(R); g.ldx = m; g.x_obs = m * c; g.b = 1;
    g.L = m; g.K = c;
    g.bh = h->Rh; g.bl = h->Rl; g.ldb = lds; g.nb_alloc = s;
    g.r = (int)s;
    g.mode = 3; g.out = h->Ebuf; g.ldn = m; g.ldl = 1;
    g.status = h->ibuf + 5;
    TT_CU(launch_tc_gemm(g, st));
    TT_CU(launch_col_norms(h->Ebuf, m, (int)s, m, e, st));
  } else {
    TT_CU(cudaMemsetAsync(h->Ebuf, 0, (size_t)m * s * sizeof(double), st));
    GemmArgs g;  // E = R V (m x s), column norms
    g.M = m; g.N = s; g.K = L; g.atomic = 1; g.allow_splitk = 1;
    g.A.p = R; g.A.rs = L; g.A.cs = 1; g.A.bs1 = m * L;
    g.B.p = V; g.B.rs = 1; g.B.cs = s; g.B.bs1 = L;
    if (h->rlay == 1) { g.K = c; g.A.rs = 1; g.A.cs = m; g.A.bs1 = 0; g.B.bs1 = 0; }  // R^T storage
    g.C = h->Ebuf; g.c_rs = 1; g.c_cs = m;
    g.nbatch = h->rlay == 1 ? 1 : nsel;
    TT_CU((gemm<WT, VT, double, double, ACC>(g, st)));
    TT_CU(launch_col_norms(h->Ebuf, m, (int)s, m, e, st));
  }
  return TTICE_OK;
}

// Mixed path: residual work m r c above which R_i = D_i - U_i W runs on the tensor cores.
constexpr double kTcResidMin = 2e8;

// R = D - U_i W for the nsel selected observations on the tensor cores (D: FP32, stage layout; W =
// U_i^T D, FP32, stage layout): the transposed split of W is the B operand, the FP32 mirror of U_i
// the A operand (lanes = rows of R), and the epilogue subtracts from D.  R is written as R^T (for a
// column-side Gram, c < m) or row-major (row side), the layouts the Gram's pre-split operands need.
bool tc_resid_ok(const ttice_s* h, int i, int64_t m, int64_t L, int nsel, int64_t ri) {
  const int64_t c = L * nsel;
  return h->Uh[i] != nullptr && ri > 0 && m >= 32 && m % 4 == 0 && h->ldu[i] % 4 == 0 &&
         (m > c || c % 4 == 0) && (double)m * ri * c >= kTcResidMin;
}
int tc_resid(ttice_s* h, int i, const float* D, const float* W, int64_t m, int64_t L, int nsel, int64_t ri,
             float* R, cudaStream_t st) {
  const int64_t c = L * nsel, ldwt = (ri + 31) / 32 * 32;
  TT_CU(launch_split_tf32_transpose(W, nsel, ri, L, h->WTh, h->WTl, ldwt, st));
  TcGemm g;
  g.x = h->Uf[i]; g.ldx = h->ldu[i]; g.x_obs = h->ldu[i] * ri; g.b = 1;
  g.L = m; g.K = ri;
  g.bh = h->WTh; g.bl = h->WTl; g.ldb = ldwt; g.nb_alloc = c;
  g.r = (int)c;
  g.mode = 4; g.out = R;
  g.in = D; g.in_lz = L; g.in_obs = m * L; g.in_ldn = 1; g.in_ldl = L;
  const bool left = m <= c;
  if (left) { g.ldn = 1; g.ldl = c; }  // row i of R: the c columns
  else { g.ldn = m; g.ldl = 1; }       // row n of R^T: the m entries of column n
  g.status = h->ibuf + 5;
  TT_CU(launch_tc_gemm(g, st));
  h->rlay = left ? 2 : 1;
  return TTICE_OK;
}

// ---------------------------------------------------------------- truncated SVD of one residual
// Residual R (observation-major blocks, m x L each, nsel blocks) -> new directions Vn (m x rR,
// column-major, ld m), rR returned through *rR_out.
template <typename WT>
int truncated_dirs(ttice_s* h, int core, const WT* R, int64_t m, int64_t L, int nsel, double eps_c,
                   int max_new, int* rR_out, cudaStream_t st) {
  const int64_t c = L * nsel;
  const bool left = m <= c;  // Gram on the row side (R R^T) or the column side (R^T R)
  const int64_t s = left ? m : c;
  if (s > kMaxEig) return TTICE_ECAPACITY;
  // Gram (FP64 accumulation)
  ph_begin(h, PH_GRAM, st, (double)sizeof(WT) * m * c + 8.0 * s * s, 2.0 * (double)s * s * (left ? c : m));
  if (h->rlay != 0) {
    // residual from the tensor cores (R^T or row-major R): the Gram as a product of two pre-split
    // operands on the tensor cores, every row of the residual against every other (both triangles)
    const int64_t kdim = h->rlay == 1 ? m : c, ld32 = (kdim + 31) / 32 * 32;
    TT_CU(launch_split_tf32(reinterpret_cast<const float*>(R), kdim, 0, s, h->Rh, h->Rl, ld32, st));
    TcGemm g;
    g.ah = h->Rh; g.al = h->Rl; g.lda = ld32; g.la_alloc = s;
    g.L = s; g.K = kdim;
    g.bh = h->Rh; g.bl = h->Rl; g.ldb = ld32; g.nb_alloc = s;
    g.r = (int)s;
    g.mode = 5; g.out = h->G; g.ldn = s; g.ldl = 1;  // FP64 sums; K split when s is small and K long
    g.status = h->ibuf + 5;
    TT_CU(cudaMemsetAsync(h->G, 0, (size_t)s * s * sizeof(double), st));
    TT_CU(launch_tc_gemm(g, st));
  } else {
  TT_CU(cudaMemsetAsync(h->G, 0, (size_t)s * s * sizeof(double), st));
  {
    GemmArgs g;
    g.atomic = 1; g.allow_splitk = 1;
    g.C = h->G;
    // symmetric: only the upper triangle of G is formed (and mirrored)
    if (left) {
      g.M = m; g.N = m; g.K = L;
      g.A.p = R; g.A.rs = L; g.A.cs = 1; g.A.bs1 = m * L;
      g.B.p = R; g.B.rs = 1; g.B.cs = L; g.B.bs1 = m * L;
      g.c_rs = s; g.c_cs = 1;
      g.nbatch = nsel;
      g.sym = 1;
    } else {
      g.M = L; g.N = L; g.K = m;
      g.A.p = R; g.A.rs = 1; g.A.cs = L; g.A.bs1 = m * L;
      g.B.p = R; g.B.rs = L; g.B.cs = 1; g.B.bs2 = m * L;
      g.c_rs = s; g.c_cs = 1; g.c_bs1 = L * s; g.c_bs2 = L;
      g.nbatch = nsel * nsel; g.bdiv = nsel;
      g.sym = 2;
    }
    if constexpr (sizeof(WT) == 8) TT_CU((gemm<WT, WT, WT, double, double>(g, st)));
    else TT_CU((gemm<WT, WT, WT, double, float>(g, st)));  // FP32 products, FP64 accumulation
  }
  }
  TT_CU(launch_trace(h->G, s, (int)s, h->trace, st));
  ph_end(h, st);
  ph_begin(h, PH_EIG, st, 0.0, 0.0);
  const double* d_eps = &h->dec->eps_c;  // the per-core threshold decided on the device
  TT_CU(cudaMemsetAsync(h->ibuf, 0, 4 * sizeof(int), st));

  const double* Vdir = nullptr;  // s x K Ritz / eigen vectors (column-major, ld s)
  const double* thet = nullptr;
  int K = 0;
  bool rr_on_jacobi = false;  // mixed path: rank decided by Rayleigh-Ritz on the FP32 Jacobi basis
  if (sizeof(WT) == 8) {
    // FP64 eigen-solve: one CTA for small Gram matrices, the multi-CTA block Jacobi otherwise.
    if (s <= kDirectEig) {
      TT_CU(jacobi_eig<double>(h->G, s, (int)s, h->w64, h->V64, h->work64, h->ibuf + 1, st));
    } else {
      TT_CU(block_jacobi_eig<double>(h->G, s, (int)s, h->w64, h->V64, h->bjw64, h->fro, h->bjflags,
                                     kMaxSweeps64, st));
      TT_CU(cudaMemcpyAsync(h->ibuf + 1, h->bjflags + 3, sizeof(int), cudaMemcpyDeviceToDevice, st));
      TT_CU(cudaMemcpyAsync(h->ibuf + 3, h->bjflags + 2, sizeof(int), cudaMemcpyDeviceToDevice, st));
    }
    TT_TRY((measure_energies<WT>(h, R, m, L, nsel, s, left, st)));
    double* e = h->theta;
    TT_CU(launch_rank_rule(e, (int)s, 1, h->trace, d_eps, max_new, h->ibuf, st));
    Vdir = h->V64; thet = h->w64; K = (int)s;
  } else {
    bool have = false, big = false;
    // a 64-vector basis cannot do better; a core that last gained more directions than one Rayleigh-
    // Ritz problem holds most likely needs the full solver again (the basis would be built in vain)
    const bool try_big = s >= kBigKrylovMin && h->BQ && h->last_new[core] <= kRR - 8;
    if (try_big) {
      int Kk = 0;
      TT_TRY(krylov_big_candidates(h, s, eps_c, &Kk, st));
      if (Kk > 0) {
        TT_TRY(rayleigh_ritz(h, s, Kk, d_eps, max_new, st));
        bool ok = false;
        TT_TRY(krylov_certify(h, s, Kk, &ok, st));
        if (!ok) TT_TRY(krylov_margin_ok(h, Kk, eps_c, &ok, st));
        if (ok) { have = true; K = Kk; h->stats.krylov_solves += 1; }
      }
      if (!have) h->stats.krylov_fallbacks += 1;
    }
    if (!have && !try_big && s > kKrylovMin && !(s >= kBigKrylovMin && h->last_new[core] > kRR - 8)) {
      // block Krylov candidates + FP64 Rayleigh-Ritz, kept only if certified: a 32-vector basis
      // first (enough for a few new directions, and an 8x smaller Ritz problem), then 64 — restarted
      // from the first attempt's leading Ritz vectors when it got as far as Rayleigh-Ritz, and from a
      // fresh block if that restart fails too (well-converged start vectors span a nearly invariant
      // subspace, so the restarted recurrence can break down)
      bool restart = false, restarted = false;
      for (int attempt = 0; attempt < 3; ++attempt) {
        const int nblk = attempt == 0 ? kKryBlocks / 2 : kKryBlocks;
        if (attempt == 2 && !restarted) break;
        const bool from_ritz = attempt == 1 && restart;
        int Kk = 0;
        TT_TRY(krylov_candidates(h, s, eps_c, nblk, from_ritz ? h->kstart : nullptr, &Kk, st));
        restarted = restarted || from_ritz;
        if (Kk > 0) {
          TT_TRY(rayleigh_ritz(h, s, Kk, d_eps, max_new, st));
          bool ok = false;
          TT_TRY(krylov_certify(h, s, Kk, &ok, st));
          if (ok) { have = true; K = Kk; h->stats.krylov_solves += 1; break; }
          if (attempt == 0 && Kk >= kKryP) {  // Ritz vectors h->Q2 (s x Kk, FP64): the leading 8 seed the retry
            TT_CU((launch_cast<double, float>(h->Q2, h->kstart, s * kKryP, st)));
            restart = true;
          }
        }
      }
      if (!have) h->stats.krylov_fallbacks += 1;
    }
    if (!have) {
    // FP32 Jacobi (one CTA for small matrices, block Jacobi otherwise) for approximate
    // eigenvectors, then FP64 Rayleigh-Ritz on the leading K of them.
    if (s <= kDirectEig32) {
      TT_CU(cudaMemsetAsync(h->bjflags, 0, 4 * sizeof(int), st));
      TT_CU(jacobi_eig<float>(h->G, s, (int)s, h->w32, h->V32, h->bjw32, h->bjflags + 3, st));
    } else {
      TT_CU(block_jacobi_eig<float>(h->G, s, (int)s, h->w32, h->V32, h->bjw32, h->fro, h->bjflags,
                                    kMaxSweeps32, st));
    }
    TT_CU(cudaMemcpyAsync(h->h_w32, h->w32, s * sizeof(float), cudaMemcpyDeviceToHost, st));
    TT_CU(cudaMemcpyAsync(h->h_int + 8, h->bjflags, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    ph_end(h, st);
    TT_TRY(sync_read(h, st));
    h->stats.eig_sweeps += h->h_int[10];
    if (h->prof_on) h->prof.flops[PH_EIG] += 8.0 * (double)s * s * s * h->h_int[10];  // A and V rotations
    if (h->h_int[11]) h->stats.eig_sweep_limit += 1;
    ph_begin(h, PH_EIG, st, 0.0, 0.0);
    // size of the Rayleigh-Ritz subspace from the FP32 spectrum (only sizes a buffer; the rank
    // itself is decided below from FP64 Ritz values)
    double tail = 0.0;
    int r32 = (int)s;
    for (int j = (int)s - 1; j >= 0; --j) {
      tail += std::max((double)h->h_w32[j], 0.0);
      if (std::sqrt(tail) <= eps_c) r32 = j; else break;
    }
    K = std::min<int>((int)s, std::min(r32 + 8, kRR));
    if (r32 + 8 > kRRFast) {
      // more directions than a fast Rayleigh-Ritz problem holds (above 90 its FP64 Jacobi leaves
      // shared memory and takes ~8 ms): use the whole FP32 eigenbasis, promoted to FP64, with the
      // energy of R along each vector measured on R itself (complete basis, so the truncation tail is
      // a direct sum, as on the FP64 path)
      TT_CU(launch_to_f64<float>(h->V32, s * s, h->V64, st));
      TT_CU(launch_to_f64<float>(h->w32, s, h->w64, st));
      TT_TRY((measure_energies<WT>(h, R, m, L, nsel, s, left, st)));
      TT_CU(launch_rank_rule(h->theta, (int)s, 1, h->trace, d_eps, max_new, h->ibuf, st));
      Vdir = h->V64; thet = h->theta; K = (int)s;
      have = true;
      big = true;
    }
    if (!big) TT_CU(launch_to_f64<float>(h->V32, s * K, h->Q, st));
    if (!big) TT_TRY(rayleigh_ritz(h, s, K, d_eps, max_new, st));
    rr_on_jacobi = !big;
    }
    if (!big) { Vdir = h->Q2; thet = h->theta; }
  }
  TT_CU(cudaMemcpyAsync(h->h_int, h->ibuf, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
  ph_end(h, st);
  TT_TRY(sync_read(h, st));
  int rR = h->h_int[0];
  if (h->h_int[1] != 0) h->stats.eig_sweep_limit += 1;  // unconverged sweeps: energies are still measured
  if (sizeof(WT) == 8 && s > kDirectEig) {
    h->stats.eig_sweeps += h->h_int[3];
    if (h->prof_on) h->prof.flops[PH_EIG] += 8.0 * (double)s * s * s * h->h_int[3];
  }
  if (rR < 0 && rr_on_jacobi) {
    // the FP32 spectrum placed the rank more than 8 below what the FP64 Ritz values need: decide on
    // the complete FP32 eigenbasis instead, with the energies measured on R (as for a rank beyond
    // one Rayleigh-Ritz problem)
    ph_begin(h, PH_EIG, st, 0.0, 0.0);
    TT_CU(launch_to_f64<float>(h->V32, s * s, h->V64, st));
    TT_TRY((measure_energies<WT>(h, R, m, L, nsel, s, left, st)));
    TT_CU(launch_rank_rule(h->theta, (int)s, 1, h->trace, d_eps, max_new, h->ibuf, st));
    TT_CU(cudaMemcpyAsync(h->h_int, h->ibuf, 4 * sizeof(int), cudaMemcpyDeviceToHost, st));
    ph_end(h, st);
    TT_TRY(sync_read(h, st));
    rR = h->h_int[0];
    Vdir = h->V64;
    thet = h->theta;
  }
  if (rR < 0) return TTICE_ECAPACITY;  // no subspace holds the tolerance (not reached in practice)
  *rR_out = rR;
  h->last_new[core] = rR;
  if (rR == 0) return TTICE_OK;
  h->dir_src = Vdir;
  h->dir_scale = thet;
  h->dir_left = left;
  h->dir_s = s;
  return TTICE_OK;
}

// New directions c0 .. c0+k-1 of the current truncated SVD into Vn (m x k): the leading
// eigenvectors themselves for a row-side Gram, u_j = R v_j / sqrt(theta_j) for a column-side one.
template <typename WT>
int build_dirs(ttice_s* h, const WT* R, int64_t m, int64_t L, int nsel, int c0, int k,
               cudaStream_t st, double* dst = nullptr) {
  double* Vn = dst ? dst : h->Vn;  // m x k, ld m
  const int64_t s = h->dir_s;
  const double* Vdir = h->dir_src + (int64_t)c0 * s;
  if (h->dir_left) {
    TT_CU(cudaMemcpy2DAsync(Vn, m * sizeof(double), Vdir, s * sizeof(double), m * sizeof(double),
                            k, cudaMemcpyDeviceToDevice, st));
  } else if (sizeof(WT) == 4 && h->rlay == 1 && h->WTh && ((s + 31) / 32 * 32) * k <= h->wt_elems) {
    // u_j = R v_j on the tensor cores: R^T as the A operand, the split eigenvectors as B
    const int64_t lds = (s + 31) / 32 * 32, c = L * nsel;
    TT_CU(launch_split_tf32_f64(Vdir, s, s, 0, k, h->WTh, h->WTl, lds, st));
    TcGemm g;
    g.x = reinterpret_cast<const float*>(R); g.ldx = m; g.x_obs = m * c; g.b = 1;
    g.L = m; g.K = c;
    g.bh = h->WTh; g.bl = h->WTl; g.ldb = lds; g.nb_alloc = k;
    g.r = k;
    g.mode = 3; g.out = Vn; g.ldn = m; g.ldl = 1;
    g.status = h->ibuf + 5;
    TT_CU(launch_tc_gemm(g, st));
    TT_CU(launch_scale_cols_rsqrt(Vn, m, k, m, h->dir_scale + c0, st));
  } else {
    TT_CU(cudaMemsetAsync(Vn, 0, (size_t)m * k * sizeof(double), st));
    GemmArgs g;
    g.M = m; g.N = k; g.K = L; g.atomic = 1; g.allow_splitk = 1;
    g.A.p = R; g.A.rs = L; g.A.cs = 1; g.A.bs1 = m * L;
    g.B.p = Vdir; g.B.rs = 1; g.B.cs = s; g.B.bs1 = L;
    if (h->rlay == 1) { g.K = L * nsel; g.A.rs = 1; g.A.cs = m; g.A.bs1 = 0; g.B.bs1 = 0; }  // R^T storage
    g.C = Vn; g.c_rs = 1; g.c_cs = m;
    g.nbatch = h->rlay == 1 ? 1 : nsel;
    // mixed path: FP32 products of the FP32 residual (FP64 accumulation); the directions are
    // re-orthogonalised against the core and among themselves afterwards
    using BACC = typename std::conditional<sizeof(WT) == 8, double, float>::type;
    TT_CU((gemm<WT, double, double, double, BACC>(g, st)));
    TT_CU(launch_scale_cols_rsqrt(Vn, m, k, m, h->dir_scale + c0, st));
  }
  return TTICE_OK;
}


// Operands of a tensor-core CGS pass: the directions V (FP64, m x k, ld m) with their TF32 head /
// tail (ld ldv, valloc columns allocated) and the projections P (FP64, ncols x k) with theirs (ld
// ldp, palloc columns).
struct CgsWs {
  double* V;
  float* Vh;
  float* Vl;
  int64_t ldv, valloc;
  double* P;
  float* Ph;
  float* Pl;
  int64_t ldp, palloc;
};
CgsWs chunk_ws(ttice_s* h) { return {h->Vn, h->Vnh, h->Vnl, h->ldv, kRR, h->P, h->Ph, h->Pl, h->ldp, kRR}; }

// One CGS pass of V (m x k, FP64, column-major) against columns [c0, c0 + ncols) of U[core] on the
// tensor cores: P = U^T V from the TF32 head / tail splits of V (from FP64) and of U (three products,
// FP32 accuracy, short K segments summed in registers, K splits in FP64), stored as the head / tail
// of P, then V -= U P with U from its FP32 mirror, subtracted in FP64.  P is small (the coupling left
// by an explicit residual), so the FP32-accurate products leave a coupling of ~2^-22 |P| after the
// pass; the floor is the FP32 rounding of the tensor-core sums, ~1e-9 of unit vectors for K in the
// tens of thousands.
int cgs_pass_tc(ttice_s* h, int core, int64_t m, int k, int64_t c0, int64_t ncols, const CgsWs& w, cudaStream_t st,
                const int* run_if = nullptr) {
  const int64_t r = ncols;
  TT_CU(launch_split_tf32_f64(w.V, m, m, 0, k, w.Vh, w.Vl, w.ldv, st));
  // P[a][j] = sum_i U[i][c0 + a] V[i][j]: A rows j (K = i), B rows a (K = i); summed in FP64 as P^T
  // (row j at P + j r), K split across CTAs when the output is small (few rows of U, tall columns),
  // then split into the TF32 head / tail that the product below reads as its B operand (rows j, K = a)
  TT_CU(cudaMemsetAsync(w.P, 0, (size_t)r * k * sizeof(double), st));
  TcGemm a;
  a.ah = w.Vh; a.al = w.Vl; a.lda = w.ldv; a.la_alloc = w.valloc;
  a.L = k; a.K = m;
  a.bh = h->Uh[core] + c0 * h->ldhl[core]; a.bl = h->Ul[core] + c0 * h->ldhl[core]; a.ldb = h->ldhl[core];
  a.nb_alloc = h->hlcols[core] - c0;
  a.r = (int)r;
  a.mode = 5; a.out = w.P; a.ldn = 1; a.ldl = r;
  a.status = h->ibuf + 5;
  a.run_if = run_if;
  TT_CU(launch_tc_gemm(a, st));
  TT_CU(launch_split_tf32_f64(w.P, r, r, 0, k, w.Ph, w.Pl, w.ldp, st));
  TcGemm b;  // V[i][j] -= sum_a U[i][c0 + a] P[a][j]: A = U (K = a rows, i contiguous), B rows j (K = a)
  b.x = h->Uf[core] + c0 * h->ldu[core]; b.ldx = h->ldu[core]; b.x_obs = h->ldu[core] * r; b.b = 1;
  b.L = m; b.K = r;
  b.bh = w.Ph; b.bl = w.Pl; b.ldb = w.ldp; b.nb_alloc = w.palloc;
  b.r = k;
  b.mode = 1; b.out = w.V; b.ldn = m; b.ldl = 1;
  b.status = h->ibuf + 5;
  b.run_if = run_if;
  TT_CU(launch_tc_gemm(b, st));
  return TTICE_OK;
}

// Coupling |U^T v| above which the tensor-core CGS runs its second pass.  One pass leaves ~2^-22 of
// the coupling it removes plus the floor of the FP32 sums; directions built from an explicit
// residual start near 1e-6, so the second pass only matters for inputs far from orthogonal.
constexpr double kCgsRepeat = 1.0 / 1024;

// Tensor-core CGS of w.V against columns [c0, c0 + ncols) of U[core]: one pass, and a second one only
// where the first met a coupling above kCgsRepeat (decided on the device).
int cgs_tc(ttice_s* h, int core, int64_t m, int k, int64_t c0, int64_t ncols, const CgsWs& w, cudaStream_t st) {
  if (ncols <= 0) return TTICE_OK;
  TT_TRY(cgs_pass_tc(h, core, m, k, c0, ncols, w, st));
  TT_CU(cudaMemsetAsync(h->ibuf + 7, 0, sizeof(int), st));
  TT_CU(launch_cols_above(w.P, ncols, k, ncols, kCgsRepeat, h->ibuf + 7, st));
  return cgs_pass_tc(h, core, m, k, c0, ncols, w, st, h->ibuf + 7);  // runs only if the flag was raised
}

// Mixed path: the CholQR work m k^2 from which a chunk's Cholesky-QR runs on the tensor cores (with
// the CGS on them): its FP64 form costs 8 m k^2 flops, milliseconds at GB300's FP64 rate from here.
constexpr double kTcCholMin = 1e8;

// One CholQR pass of Vn (m x k, FP64) on the tensor cores: the off-diagonal of S = Vn^T Vn from the
// TF32 head / tail of Vn (three products, FP32 segment sums, the K splits added in FP64), its
// diagonal summed in FP64 (the tensor core's FP32 sums of positive terms carry a rounding bias of
// ~1e-7 that would be left in the column norms), then Vn <- Vn T written as Vn - Vn (I - T): the
// product on the tensor cores from the FP32 rounding of Vn, the subtraction in FP64.  T = S^{-1/2}
// (the symmetric orthonormalisation, from a series in E = S - I) when ||E||_F <= 1e-4, as it is for
// unit-scaled directions already orthogonal to the core; otherwise T = R^{-1} with S = R^T R in FP64
// (the Cholesky-QR step).  I - T is small, so the product's FP32 accuracy costs ~2^-22 of it; the
// floor is the FP32 rounding of the off-diagonal sums, as in the tensor-core CGS.
int cholqr_pass_tc(ttice_s* h, int64_t m, int k, cudaStream_t st) {
  float* Vf = reinterpret_cast<float*>(h->Vn2);  // FP32 Vn at ld ldv (ldv k floats fit: m >= 32)
  TT_CU(cudaMemsetAsync(h->dsq, 0, (size_t)k * sizeof(double), st));
  TT_CU(launch_split_tf32_f64(h->Vn, m, m, 0, k, h->Vnh, h->Vnl, h->ldv, st, Vf, h->dsq));
  TT_CU(cudaMemsetAsync(h->Ssm, 0, (size_t)k * k * sizeof(double), st));
  TcGemm g;  // S[a][j] = sum_i Vn[i][a] Vn[i][j]: A and B both the split of Vn (K = i)
  g.ah = h->Vnh; g.al = h->Vnl; g.lda = h->ldv; g.la_alloc = kRR;
  g.L = k; g.K = m;
  g.bh = h->Vnh; g.bl = h->Vnl; g.ldb = h->ldv; g.nb_alloc = kRR;
  g.r = k;
  g.mode = 5; g.out = h->Ssm; g.ldn = k; g.ldl = 1;
  g.status = h->ibuf + 5;
  TT_CU(launch_tc_gemm(g, st));
  // near-orthonormal chunk (the usual case): the symmetric orthonormalisation from a short series in
  // E = S - I, with no FP64 factorisation; otherwise (flag raised on the device) Cholesky in FP64
  TT_CU(cudaMemsetAsync(h->ibuf + 8, 0, sizeof(int), st));
  TT_CU(launch_lowdin_split(h->Ssm, k, h->dsq, h->Fh, h->Fl, kRR, h->ibuf + 8, st));
  TT_CU(launch_chol_inv(h->Ssm, k, h->Rinv, h->ibuf + 2, st, h->dsq, h->ibuf + 8));
  TT_CU(launch_eye_minus_split(h->Rinv, k, h->Fh, h->Fl, kRR, st, h->ibuf + 8));
  TcGemm q;  // Vn[i][j] -= sum_l Vn[i][l] F[l][j]: A = FP32 Vn (i contiguous, K = l), B rows j (K = l)
  q.x = Vf; q.ldx = h->ldv; q.x_obs = h->ldv * k; q.b = 1;
  q.L = m; q.K = k;
  q.bh = h->Fh; q.bl = h->Fl; q.ldb = kRR; q.nb_alloc = kRR;
  q.r = k;
  q.mode = 1; q.out = h->Vn; q.ldn = m; q.ldl = 1;
  q.status = h->ibuf + 5;
  TT_CU(launch_tc_gemm(q, st));
  return TTICE_OK;
}

// CGS2 of the new directions Vn (m x k) against U[core] (m x r), CholQR2 among themselves,
// canonical sign, and append as columns r..r+k-1 of U[core] (Eq. 10).  On the tensor cores the
// second CGS pass runs only when the first met a coupling above kCgsRepeat (a device flag).
// cgs_from > 0 (with `blocked`, tensor-core path only): the chunk was already re-orthogonalised
// against columns [0, cgs_from) together with the rest of its block, and only [cgs_from, r) remain.
int orthonormalize_append(ttice_s* h, int core, int64_t m, int k, cudaStream_t st, int64_t cgs_from = 0,
                          bool blocked = false) {
  const int64_t r = h->r[core + 1];
  double* U = h->U[core];
  const int64_t ld = h->ldu[core];
  const bool tc = blocked || (h->Uh[core] && r > 0 && m >= 32 && ld % 4 == 0 &&
                              (double)m * r * k >= g_tc_cgs_min.load());
  if (tc) TT_TRY(cgs_tc(h, core, m, k, cgs_from, r - cgs_from, chunk_ws(h), st));
  for (int pass = 0; pass < 2 && r > 0 && !tc; ++pass) {
    GemmArgs a;  // P = U^T Vn  (r x k, column-major ld r)
    a.M = r; a.N = k; a.K = m; a.atomic = 1; a.allow_splitk = 1;
    a.A.p = U; a.A.rs = ld; a.A.cs = 1;
    a.B.p = h->Vn; a.B.rs = 1; a.B.cs = m;
    a.C = h->P; a.c_rs = 1; a.c_cs = r;
    TT_CU(cudaMemsetAsync(h->P, 0, (size_t)r * k * sizeof(double), st));
    TT_CU((gemm<double, double, double, double, double>(a, st)));
    GemmArgs b;  // Vn = Vn - U P
    b.M = m; b.N = k; b.K = r;
    b.A.p = U; b.A.rs = 1; b.A.cs = ld;
    b.B.p = h->P; b.B.rs = 1; b.B.cs = r;
    b.X.p = h->Vn; b.X.rs = 1; b.X.cs = m;
    b.alpha = -1.0; b.beta = 1.0;
    b.C = h->Vn; b.c_rs = 1; b.c_cs = m;
    TT_CU((gemm<double, double, double, double, double>(b, st)));
  }
  const bool tc_chol = tc && (double)m * k * k >= std::min(kTcCholMin, g_tc_cgs_min.load());
  for (int pass = 0; pass < 2 && tc_chol; ++pass) TT_TRY(cholqr_pass_tc(h, m, k, st));
  for (int pass = 0; pass < 2 && !tc_chol; ++pass) {
    TT_CU(cudaMemsetAsync(h->Ssm, 0, (size_t)k * k * sizeof(double), st));
    GemmArgs g;  // S = Vn^T Vn
    g.M = k; g.N = k; g.K = m; g.atomic = 1; g.allow_splitk = 1;
    g.A.p = h->Vn; g.A.rs = m; g.A.cs = 1;
    g.B.p = h->Vn; g.B.rs = 1; g.B.cs = m;
    g.C = h->Ssm; g.c_rs = 1; g.c_cs = k;
    TT_CU((gemm<double, double, double, double, double>(g, st)));
    TT_CU(launch_chol_inv(h->Ssm, k, h->Rinv, h->ibuf + 2, st));
    GemmArgs q;  // Vn2 = Vn Rinv
    q.M = m; q.N = k; q.K = k;
    q.A.p = h->Vn; q.A.rs = 1; q.A.cs = m;
    q.B.p = h->Rinv; q.B.rs = 1; q.B.cs = k;
    q.C = h->Vn2; q.c_rs = 1; q.c_cs = m;
    TT_CU((gemm<double, double, double, double, double>(q, st)));
    std::swap(h->Vn, h->Vn2);
  }
  TT_CU(launch_canonical_sign(h->Vn, m, k, m, h->sgn_part, h->sgn, st));
  TT_CU(launch_copy_cols(h->Vn, m, m, k, U + r * ld, ld, h->Uf[core] ? h->Uf[core] + r * ld : nullptr,
                         st, h->sgn));
  if (h->Uh[core])
    TT_CU(launch_split_tf32(h->Uf[core], ld, r, r + k, h->Uh[core], h->Ul[core], h->ldhl[core], st));
  return TTICE_OK;
}

int grow_last(ttice_s* h, int64_t need) {
  if (need <= h->last_cap) return TTICE_OK;
  int64_t nc = std::max<int64_t>(h->last_cap * 2, need);
  double* p = nullptr;
  int64_t* sink = g_alloc_sink;  // counted below, as the net change
  g_alloc_sink = nullptr;
  const int arc = dalloc<double>(&p, nc * h->cap[h->d]);
  g_alloc_sink = sink;
  TT_TRY(arc);
  if (h->last) {
    cudaStream_t fs = setup_stream();
    int rc = fs ? cu(cudaMemcpyAsync(p, h->last, (size_t)h->last_cap * h->cap[h->d] * sizeof(double),
                                     cudaMemcpyDeviceToDevice, fs))
                : cu(cudaErrorNotReady);
    if (rc == TTICE_OK) rc = cu(cudaStreamSynchronize(fs));
    if (rc != TTICE_OK) {
      cudaFree(p);
      return rc;
    }
    cudaFree(h->last);
  }
  h->dev_bytes += (nc - h->last_cap) * h->cap[h->d] * (int64_t)sizeof(double);
  h->last = p;
  h->last_cap = nc;
  return TTICE_OK;
}

void fill_stats(ttice_s* h) {
  for (int i = 0; i <= h->d; ++i) h->stats.ranks[i] = h->r[i];
  h->stats.ranks[h->d + 1] = 1;
  h->stats.n_obs = h->n_obs;
  int64_t e = 0;
  for (int i = 0; i < h->d; ++i) e += h->r[i] * h->n[i] * h->r[i + 1];
  e += h->r[h->d] * h->n_obs;
  h->stats.core_elems = e;
}

// Undo the rank growth of a failed update: zero the appended columns (which also removes every
// entry they had in padded rows) and restore the ranks.
void rollback(ttice_s* h, const int64_t* r_old, cudaStream_t st) {
  for (int i = 0; i < h->d; ++i) {
    if (h->r[i + 1] > r_old[i + 1]) {
      const int64_t ld = h->ldu[i];
      const size_t bytes = (size_t)(h->r[i + 1] - r_old[i + 1]) * ld;
      cudaMemsetAsync(h->U[i] + r_old[i + 1] * ld, 0, bytes * sizeof(double), st);
      if (h->Uf[i]) cudaMemsetAsync(h->Uf[i] + r_old[i + 1] * ld, 0, bytes * sizeof(float), st);
      if (h->Uh[i]) {
        const size_t hb = (size_t)(h->r[i + 1] - r_old[i + 1]) * h->ldhl[i] * sizeof(float);
        cudaMemsetAsync(h->Uh[i] + r_old[i + 1] * h->ldhl[i], 0, hb, st);
        cudaMemsetAsync(h->Ul[i] + r_old[i + 1] * h->ldhl[i], 0, hb, st);
      }
    }
  }
  for (int i = 0; i <= h->d; ++i) h->r[i] = r_old[i];
  cudaStreamSynchronize(st);
}

// Rows [r0, r0 + k) of the stage output U_i^T X for nobs observations of the stage input X (the
// columns core i appended), into out (nobs x k x L_i).
template <typename WT, typename TY>
int new_rows(ttice_s* h, int i, const void* X, int nobs, int64_t r0, int k, WT* out, cudaStream_t st) {
  const int64_t m = h->r[i] * h->n[i], L = h->L[i];
  if (sizeof(WT) == 4 && h->Uh[i] && (i > 0 || sizeof(TY) == 4) && tc_proj_supported(X, L, m, k, h->ldhl[i]))
    return cu(launch_tc_proj(static_cast<const float*>(X), nobs, L, m, k, h->Uh[i] + r0 * h->ldhl[i],
                             h->Ul[i] + r0 * h->ldhl[i], h->ldhl[i], h->hlcols[i] - r0, reinterpret_cast<float*>(out),
                             nullptr, nullptr, h->part, h->tcws, h->ibuf + 5, st, stage_nprod(h, i)));
  if (sizeof(WT) == 4 && i > 0 && tc_stage_t_ok(h, i, nobs, k))
    return tc_project_t(h, i, static_cast<const float*>(X), nobs, r0, k, reinterpret_cast<float*>(out), nullptr, st);
  const WT* Ui = ((sizeof(WT) == 8) ? reinterpret_cast<const WT*>(h->U[i]) : reinterpret_cast<const WT*>(h->Uf[i])) +
                 r0 * h->ldu[i];
  if (i == 0) return proj<WT, TY, WT>(Ui, h->ldu[i], static_cast<const TY*>(X), m, L, k, nobs, out, st);
  return proj<WT, WT, WT>(Ui, h->ldu[i], static_cast<const WT*>(X), m, L, k, nobs, out, st);
}

template <typename WT, typename TY>
int update_impl(ttice_s* h, const TY* Y, int b, cudaStream_t st) {
  nvtx_close(h);
  h->miss_k = 0;
  h->miss_need = 0;
  TT_TRY(grow_last(h, h->n_obs + b));
  void** S1 = h->stage;
  TT_TRY((chain<WT, TY>(h, Y, b, S1, true, st)));
  TT_CU(launch_decision(h->rho2, h->d, h->y2, b, h->eps_dec, h->d, h->h.skip_mode, h->h.subselect,
                        h->h.eps_upd_mode, h->dec, h->sel, st));
  TT_CU(cudaMemcpyAsync(h->h_dec, h->dec, sizeof(Decision), cudaMemcpyDeviceToHost, st));
  TT_CU(cudaMemcpyAsync(h->h_sel, h->sel, b * sizeof(int), cudaMemcpyDeviceToHost, st));
  TT_CU(cudaMemcpyAsync(h->h_int + 5, h->ibuf + 5, sizeof(int), cudaMemcpyDeviceToHost, st));
  TT_CU(cudaMemcpyAsync(h->h_rho2, h->rho2, (size_t)h->d * b * sizeof(double), cudaMemcpyDeviceToHost, st));
  TT_TRY(sync_read(h, st));
  const Decision dec = *h->h_dec;
  if (h->h_int[5]) return TTICE_ETIMEOUT;  // a staged copy of the first pass never completed
  if (dec.nonfinite) return TTICE_ENONFINITE;
  std::memset(&h->stats, 0, sizeof(h->stats));
  h->stats.skipped = dec.skip;
  h->stats.n_selected = dec.nsel;
  h->stats.rel_err_before = dec.batch_err;
  h->stats.eps_upd = dec.eps_upd;
  h->stats.eps_core = dec.eps_c;

  if (!dec.skip && dec.nsel > 0) {
    int64_t r_old[kMaxD + 1];
    std::memcpy(r_old, h->r, sizeof(r_old));
    const int nsel = dec.nsel;
    const TY* D0 = Y;
    if (nsel < b) {
      TT_CU(launch_gather_obs<TY>(Y, static_cast<TY*>(h->dgather), h->sel, nsel, h->N, st));
      D0 = static_cast<const TY*>(h->dgather);
    }
    const WT* X = nullptr;  // stage input for i >= 1
    // While no core has grown in this update, D_i and U_i^T D_i of the selected observations are
    // exactly what the first pass computed (same cores, same inputs): its stage outputs and per-stage
    // residual norms are reused instead of recomputed.
    bool pristine = true;
    int first_grown = h->d;  // first core that gained directions
    int rc = TTICE_OK;
    for (int i = 0; i < h->d && rc == TTICE_OK; ++i) {
      const int64_t m = h->r[i] * h->n[i], L = h->L[i];
      const int64_t ri = h->r[i + 1];
      int grew = 0;
      // U_i^T D_i of the selected observations is the first pass's, also after earlier cores grew:
      // D_i then gained the rows of the new rank indices, where U_i is zero (padded)
      const WT* Wp = nullptr;
      if (ri > 0 && m > 0) {
        if (nsel == b) {
          Wp = static_cast<const WT*>(S1[i]);
        } else {
          WT* g = static_cast<WT*>(h->dstage[i]);
          rc = cu(launch_gather_obs<WT>(static_cast<const WT*>(S1[i]), g, h->sel, nsel, ri * L, st));
          if (rc != TTICE_OK) break;
          Wp = g;
        }
      }
      const TY* D0i = D0;
      const WT* Xi = X;
      if (m > 0 && !((double)ri >= h->h.occupancy_tau * (double)m)) {
        WT* R = static_cast<WT*>(h->Rbuf);
        const WT* Ui = (sizeof(WT) == 8) ? reinterpret_cast<const WT*>(h->U[i])
                                         : reinterpret_cast<const WT*>(h->Uf[i]);
        {
          const double sx = (i == 0) ? sizeof(TY) : sizeof(WT), sw = sizeof(WT);
          ph_begin(h, PH_RESID, st, nsel * (sx * m * L + sw * m * L + 2.0 * sw * ri * L),
                   2.0 * nsel * (double)m * L * ri);  // R = D - U W, with W the first pass's
        }
        bool small = false;  // ||R_i||_F <= eps_c: the rank rule gives 0 without any eigenvalue
        h->rlay = 0;
        // mixed path, FP32 stage input: the residual on the tensor cores
        const void* Din = i == 0 ? static_cast<const void*>(D0i) : static_cast<const void*>(Xi);
        const bool tcr = sizeof(WT) == 4 && (i > 0 || sizeof(TY) == 4) && tc_resid_ok(h, i, m, L, nsel, ri);
        if (ri > 0 && pristine) {
          double t = 0.0;
          for (int z = 0; z < nsel; ++z) t += h->h_rho2[(int64_t)i * b + h->h_sel[z]];
          small = std::sqrt(t) <= dec.eps_c;
          if (!small && tcr) {
            rc = tc_resid(h, i, static_cast<const float*>(Din), reinterpret_cast<const float*>(Wp), m, L, nsel, ri,
                          reinterpret_cast<float*>(R), st);
          } else if (!small) {
            if (i == 0) rc = resid<WT, WT, TY, WT>(Ui, h->ldu[i], Wp, D0i, m, L, ri, nsel, R, nullptr, st);
            else rc = resid<WT, WT, WT, WT>(Ui, h->ldu[i], Wp, Xi, m, L, ri, nsel, R, nullptr, st);
          }
        } else if (ri > 0) {
          // an earlier core grew: the residual D_i - U_i Wp now also holds D_i's new rows, and its
          // norm is summed from the explicit residual
          rc = cu(cudaMemsetAsync(h->rn2, 0, nsel * sizeof(double), st));
          if (rc == TTICE_OK && tcr) {
            rc = tc_resid(h, i, static_cast<const float*>(Din), reinterpret_cast<const float*>(Wp), m, L, nsel, ri,
                          reinterpret_cast<float*>(R), st);
            if (rc == TTICE_OK) rc = sumsq<WT>(R, 1, m * L * nsel, h->rn2, st);
          } else if (rc == TTICE_OK) {
            if (i == 0) rc = resid<WT, WT, TY, WT>(Ui, h->ldu[i], Wp, D0i, m, L, ri, nsel, R, h->rn2, st);
            else rc = resid<WT, WT, WT, WT>(Ui, h->ldu[i], Wp, Xi, m, L, ri, nsel, R, h->rn2, st);
          }
          if (rc == TTICE_OK) rc = cu(cudaMemcpyAsync(h->h_rn2, h->rn2, nsel * sizeof(double),
                                                      cudaMemcpyDeviceToHost, st));
          if (rc == TTICE_OK) rc = sync_read(h, st);
          if (rc == TTICE_OK) {
            double t = 0.0;
            for (int z = 0; z < nsel; ++z) t += h->h_rn2[z];
            small = std::sqrt(t) <= dec.eps_c;
          }
        } else {
          if (i == 0) rc = cu(launch_cast<TY, WT>(D0i, R, (int64_t)nsel * m * L, st));
          else rc = cu(cudaMemcpyAsync(R, Xi, (size_t)nsel * m * L * sizeof(WT), cudaMemcpyDeviceToDevice, st));
        }
        ph_end(h, st);
        if (rc != TTICE_OK) break;
        const int max_new = (int)(m - ri);
        int rR = 0;
        // Eq. 5 at r = 0: the tail is ||R_i||_F^2 itself, so no direction is needed and the Gram and
        // its eigen-solve are skipped
        if (!small) rc = truncated_dirs<WT>(h, i, R, m, L, nsel, dec.eps_c, max_new, &rR, st);
        if (rc != TTICE_OK) break;
        if (rR > 0) {
          if (ri + rR > h->cap[i + 1]) {
            h->miss_k = i + 1;
            h->miss_need = ri + rR;
            rc = TTICE_ECAPACITY;
            break;
          }
          // append in chunks of at most kRR directions; each chunk is re-orthogonalised against the
          // core including the chunks already appended (block CGS2).  Mixed path, many directions
          // and a large core: blocks of up to kb[i] directions are first re-orthogonalised against
          // the core's earlier columns together (one pass over the core per block), then each chunk
          // only against the chunks of its block already appended.
          const bool blocked = sizeof(WT) == 4 && h->kb[i] > 0 && rR > kRR && h->Uh[i] && m >= 32 &&
                               h->ldu[i] % 4 == 0 && (double)m * ri * rR >= g_tc_cgs_min.load();
          const int kblk = blocked ? h->kb[i] : rR;
          for (int b0 = 0; b0 < rR && rc == TTICE_OK; b0 += kblk) {
            const int kbb = std::min(kblk, rR - b0);
            const int64_t r_blk = h->r[i + 1];  // columns before this block
            if (blocked) {
              const int64_t ldvb = (h->ldu[i] + 31) / 32 * 32, ldpb = (h->cap[i + 1] + 31) / 32 * 32;
              const CgsWs w{h->VB, h->VBh, h->VBl, ldvb, h->kb[i], h->PB, h->PBh, h->PBl, ldpb, h->kb[i]};
              ph_begin(h, PH_ORTH, st, 8.0 * m * (2.0 * r_blk + 2.0 * kbb), 12.0 * m * r_blk * kbb);
              rc = build_dirs<WT>(h, R, m, L, nsel, b0, kbb, st, h->VB);
              if (rc == TTICE_OK) rc = cgs_tc(h, i, m, kbb, 0, r_blk, w, st);
              ph_end(h, st);
            }
            for (int c0 = 0; c0 < kbb && rc == TTICE_OK; c0 += kRR) {
              const int kc = std::min(kRR, kbb - c0);
              const int64_t rcur = h->r[i + 1];
              ph_begin(h, PH_ORTH, st, 8.0 * m * (2.0 * rcur + 3.0 * kc),
                       8.0 * m * rcur * kc + 8.0 * m * (double)kc * kc);
              if (blocked) {
                rc = cu(cudaMemcpyAsync(h->Vn, h->VB + (int64_t)c0 * m, (size_t)m * kc * sizeof(double),
                                        cudaMemcpyDeviceToDevice, st));
                if (rc == TTICE_OK) rc = orthonormalize_append(h, i, m, kc, st, r_blk, true);
              } else {
                rc = build_dirs<WT>(h, R, m, L, nsel, b0 + c0, kc, st);
                if (rc == TTICE_OK) rc = orthonormalize_append(h, i, m, kc, st);
              }
              ph_end(h, st);
              if (rc == TTICE_OK) h->r[i + 1] = rcur + kc;
            }
          }
          if (rc != TTICE_OK) break;
          grew = rR;
        }
      }
      h->stats.new_dirs[i] = grew;
      if (grew > 0 && first_grown == h->d) first_grown = i;
      if (grew > 0) pristine = false;
      // D_{i+1} = reshape(U_i^T D_i) with the updated core: the first pass's Wp followed by the rows of
      // the appended columns, U_i[:, ri:rn]^T D_i.  Formed also for the last TT core when every
      // observation was selected: those are then the coefficients of the updated decomposition.
      const int64_t rn = h->r[i + 1];
      if (m == 0 || rn == 0) break;  // nothing flows to the next cores
      if (grew == 0) {
        if (i + 1 < h->d) X = Wp;  // U_i is unchanged on every row of D_i
        continue;
      }
      if (i + 1 == h->d && nsel < b) break;
      {
        const double sx = (i == 0) ? sizeof(TY) : sizeof(WT);
        ph_begin(h, PH_DPROJ, st, nsel * (sx * m * L + sizeof(WT) * ((double)rn + grew) * L),
                 2.0 * nsel * (double)m * L * grew);
      }
      WT* add = static_cast<WT*>(h->Rbuf);  // the residual is no longer needed
      WT* Wn = static_cast<WT*>(h->dstage[i]);
      const void* Din = i == 0 ? static_cast<const void*>(D0i) : static_cast<const void*>(Xi);
      rc = new_rows<WT, TY>(h, i, Din, nsel, ri, grew, add, st);
      if (rc == TTICE_OK)
        rc = cu(launch_expand_stage<WT>(static_cast<const WT*>(S1[i]), nsel < b ? h->sel : nullptr, ri, add, grew, L,
                                        nsel, Wn, st));
      ph_end(h, st);
      X = Wn;
    }
    if (rc != TTICE_OK) {
      rollback(h, r_old, st);
      h->marks.clear();
      h->ev_used = 0;
      return rc;
    }
    // project every observation onto the updated cores (Algorithm 2, last two steps): the stage
    // outputs of cores that did not grow are the first pass's (the rows their inputs gained meet zero
    // rows of the core), those of cores that grew gain the rows of their new columns.  With every
    // observation selected, these are the D projections formed above.
    for (int i = first_grown; i < h->d; ++i) {
      const int grew = h->stats.new_dirs[i];
      if (grew == 0) continue;
      const int64_t m = h->r[i] * h->n[i], L = h->L[i], r0 = h->r[i + 1] - grew;
      if (nsel < b) {
        ph_begin(h, PH_FINAL, st, b * (sizeof(WT) * (double)m * L + sizeof(WT) * (2.0 * r0 + grew) * L),
                 2.0 * b * (double)m * L * grew);
        WT* add = static_cast<WT*>(h->Rbuf);
        const void* Xin = i == 0 ? static_cast<const void*>(Y) : S1[i - 1];
        TT_TRY((new_rows<WT, TY>(h, i, Xin, b, r0, grew, add, st)));
        TT_CU(launch_expand_stage<WT>(static_cast<const WT*>(S1[i]), nullptr, r0, add, grew, L, b,
                                      static_cast<WT*>(h->dstage[i]), st));
        ph_end(h, st);
      }
      std::swap(h->stage[i], h->dstage[i]);
    }
  }
  const int rd = (int)h->r[h->d];
  TT_CU(launch_append_last_t<WT>(static_cast<const WT*>(S1[h->d - 1]), b, rd, h->last, h->n_obs,
                                 h->cap[h->d], st));
  TT_CU(cudaMemcpyAsync(h->h_int + 5, h->ibuf + 5, sizeof(int), cudaMemcpyDeviceToHost, st));
  TT_TRY(sync_read(h, st));
  if (h->h_int[5]) return TTICE_ETIMEOUT;  // a staged copy of a projection pass never completed
  h->n_obs += b;
  fill_stats(h);
  ph_collect(h);
  if (h->prof_on) h->prof.updates += 1;
  return TTICE_OK;
}

template <typename WT, typename TY>
int project_impl(ttice_s* h, const TY* Y, int b, double* coeffs, double* rel, cudaStream_t st) {
  nvtx_close(h);
  TT_TRY((chain<WT, TY>(h, Y, b, h->stage, rel != nullptr, st)));
  const int rd = (int)h->r[h->d];
  if (coeffs && rd > 0) TT_CU((launch_cast<WT, double>(static_cast<const WT*>(h->stage[h->d - 1]), coeffs, (int64_t)b * rd, st)));
  if (rel) TT_CU(launch_rel_err(h->rho2, h->d, h->y2, b, rel, st));
  return TTICE_OK;
}

}  // namespace

// ================================================================== C ABI
extern "C" {

void ttice_default_heuristics(ttice_heuristics* h) {
  if (!h) return;
  h->skip_mode = TTICE_SKIP_EXACT;
  h->subselect = 1;
  h->eps_upd_mode = TTICE_EPSUPD_EXACT;
  h->occupancy_tau = 1.0;
  h->precision = TTICE_FP64;
  h->input_dtype = TTICE_F32;
}

void ttice_default_capacity(ttice_capacity* c) {
  if (!c) return;
  c->max_batch = 32;
  c->max_rank = 512;
  c->obs_reserve = 1024;
}

const char* ttice_strerror(int code) {
  switch (code) {
    case TTICE_OK: return "ok";
    case TTICE_EINVAL: return "invalid argument";
    case TTICE_ENOMEM: return "device allocation failed";
    case TTICE_ECAPACITY: return "rank capacity or solver limit exceeded";
    case TTICE_ENONFINITE: return "increment contains NaN or Inf";
    case TTICE_ETIMEOUT: return "iterative device solve hit its iteration limit";
    case TTICE_ECUDA: return "CUDA runtime error";
    default: return "internal error";
  }
}

const char* ttice_last_cuda_error(void) { return cudaGetErrorName(g_last_cuda_error); }

void ttice_test_fail_alloc(int64_t n) { g_fail_alloc.store(n > 0 ? n : 0); }

void ttice_test_wait_limit_ns(uint64_t ns) { tc_set_wait_ns(ns); }

void ttice_test_drop_copy(int64_t chunk) { tc_drop_next_copy(chunk); }

void ttice_test_tc_cgs_min(double flops) { g_tc_cgs_min.store(flops < 0.0 ? kTcCgsMin : flops); }

}  // extern "C"

namespace {

// Build a handle.  caps (host, d+1 entries, caps[0] ignored) overrides the rank capacities of the
// default rule cap_i = min(max_rank, cap_{i-1} n_{i-1}); each is still clipped to cap_{i-1} n_{i-1}.
int create_handle(const int64_t* dims, int d, double eps, const ttice_heuristics* hp,
                  const ttice_capacity* cp, const int64_t* caps, ttice_t* out) {
  if (!dims || !out || d < 1 || d > kMaxD || !(eps > 0.0) || !(eps < 1.0)) return TTICE_EINVAL;
  *out = nullptr;
  ttice_s* h = new (std::nothrow) ttice_s();
  if (!h) return TTICE_ENOMEM;
  ttice_default_heuristics(&h->h);
  ttice_default_capacity(&h->capc);
  if (hp) h->h = *hp;
  if (cp) h->capc = *cp;
  if (h->h.precision != TTICE_FP64 && h->h.precision != TTICE_FP32 && h->h.precision != TTICE_TF32) {
    delete h;
    return TTICE_EINVAL;
  }
  if (h->h.input_dtype != TTICE_F32 && h->h.input_dtype != TTICE_F64) { delete h; return TTICE_EINVAL; }
  if (h->capc.max_batch < 1 || h->capc.max_rank < 1) { delete h; return TTICE_EINVAL; }
  h->d = d;
  h->eps = eps;
  h->nprod = h->h.precision == TTICE_TF32 ? 1 : 3;
  h->eps_dec = h->h.precision == TTICE_TF32 ? eps * std::sqrt(1.0 - kTf32Share) : eps;
  h->N = 1;
  // the current device (without one, the first allocation below fails and reports why)
  if (!g_dry_run && cudaGetDevice(&h->device) != cudaSuccess) { cudaGetLastError(); h->device = 0; }
  for (int i = 0; i < d; ++i) {
    if (dims[i] < 1) { delete h; return TTICE_EINVAL; }
    h->n[i] = dims[i];
    h->N *= dims[i];
  }
  for (int i = 0; i < d; ++i) {
    int64_t l = 1;
    for (int j = i + 1; j < d; ++j) l *= h->n[j];
    h->L[i] = l;
  }
  h->cap[0] = 1;
  h->r[0] = 1;
  for (int i = 1; i <= d; ++i) {
    const int64_t want = caps ? caps[i] : h->capc.max_rank;
    if (want < 1) { delete h; return TTICE_EINVAL; }
    h->cap[i] = std::min<int64_t>(want, h->cap[i - 1] * h->n[i - 1]);
  }
  g_alloc_sink = &h->dev_bytes;
  h->wt_bytes = (h->h.precision == TTICE_FP64) ? 8 : 4;
  const int64_t B = h->capc.max_batch;
  int rc = TTICE_OK;
  int64_t max_mL = 0;
  for (int i = 0; i < d && rc == TTICE_OK; ++i) {
    h->ldu[i] = h->cap[i] * h->n[i];
    h->max_m = std::max(h->max_m, h->ldu[i]);
    rc = dalloc<double>(&h->U[i], h->ldu[i] * h->cap[i + 1]);
    if (rc == TTICE_OK && h->wt_bytes == 4) rc = dalloc<float>(&h->Uf[i], h->ldu[i] * h->cap[i + 1]);
    if (h->wt_bytes == 4) {
      h->ldhl[i] = (h->ldu[i] + 31) / 32 * 32;
      h->hlcols[i] = (h->cap[i + 1] + 255) / 256 * 256;
      if (rc == TTICE_OK) rc = dalloc<float>(&h->Uh[i], h->ldhl[i] * h->hlcols[i]);
      if (rc == TTICE_OK) rc = dalloc<float>(&h->Ul[i], h->ldhl[i] * h->hlcols[i]);
    }
    const int64_t st_elems = B * h->cap[i + 1] * h->L[i];
    if (rc == TTICE_OK) rc = dalloc_bytes(&h->stage[i], st_elems * h->wt_bytes);
    if (rc == TTICE_OK) rc = dalloc_bytes(&h->dstage[i], st_elems * h->wt_bytes);
    max_mL = std::max(max_mL, h->ldu[i] * h->L[i]);
    h->s_max = std::max(h->s_max, std::min<int64_t>(h->ldu[i], h->L[i] * B));
    h->max_ms = std::max(h->max_ms, h->ldu[i] * std::min<int64_t>({h->ldu[i], h->L[i] * B, (int64_t)kMaxEig}));
  }
  h->s_max = std::min<int64_t>(h->s_max, kMaxEig);
  const int64_t s = std::max<int64_t>(h->s_max, 1);
  const int in_bytes = h->h.input_dtype == TTICE_F32 ? 4 : 8;
  if (rc == TTICE_OK) rc = dalloc_bytes(&h->dgather, B * h->N * in_bytes);
  if (rc == TTICE_OK) rc = dalloc_bytes(&h->Rbuf, B * max_mL * h->wt_bytes);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->G, s * s);
  if (rc == TTICE_OK) rc = dalloc<float>(&h->w32, s);
  if (rc == TTICE_OK) rc = dalloc<float>(&h->V32, s * s);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->w64, std::max<int64_t>(s, kRR));
  if (rc == TTICE_OK) rc = dalloc<double>(&h->V64, std::max<int64_t>(s * s, (int64_t)kRR * kRR));  // both paths
  if (rc == TTICE_OK) rc = dalloc<double>(&h->work64, 2 * std::max<int64_t>(s, kRR) * (std::max<int64_t>(s, kRR) + 1));
  if (rc == TTICE_OK && h->wt_bytes == 8) rc = dalloc<double>(&h->bjw64, block_jacobi_work<double>((int)s));
  if (rc == TTICE_OK && h->wt_bytes == 4) rc = dalloc<float>(&h->bjw32, block_jacobi_work<float>((int)s));
  if (rc == TTICE_OK) rc = dalloc<double>(&h->fro, 3);  // ||A||^2, off-norm^2 now and one sweep back
  if (rc == TTICE_OK) rc = dalloc<int>(&h->bjflags, 8);
  if (rc == TTICE_OK && h->wt_bytes == 4) rc = dalloc<float>(&h->G32, s * s);
  if (h->wt_bytes == 4 && s >= kBigKrylovMin) {
    if (rc == TTICE_OK) rc = dalloc<float>(&h->BQ, s * kBigK);
    if (rc == TTICE_OK) rc = dalloc<float>(&h->BGQ, s * kBigK);
    if (rc == TTICE_OK) rc = dalloc<float>(&h->BY, s * kBigP);
    if (rc == TTICE_OK) rc = dalloc<float>(&h->BY2, s * kBigP);
    if (rc == TTICE_OK) rc = dalloc<float>(&h->BC, (int64_t)kBigK * kBigP);
    if (rc == TTICE_OK) rc = dalloc<double>(&h->BH, (int64_t)kBigK * kBigK);
  }
  if (rc == TTICE_OK) rc = dalloc<float>(&h->KQ, s * kKry);
  if (rc == TTICE_OK) rc = dalloc<float>(&h->kstart, s * kKryP);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->KV, std::max<int64_t>(s * kKryP, kKry * kKry));
  if (rc == TTICE_OK) rc = dalloc<double>(&h->res, kRR);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->Q, s * kRR);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->Q2, s * kRR);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->GQ, s * kRR);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->Ssm, kRR * kRR);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->Rinv, kRR * kRR);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->H, kRR * kRR);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->Z, kRR * kRR);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->theta, std::max<int64_t>(s, kRR) + 8);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->Ebuf, std::max<int64_t>(h->max_ms, 1));
  if (rc == TTICE_OK) rc = dalloc<double>(&h->Vn, h->max_m * kRR);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->Vn2, h->max_m * kRR);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->sgn, kRR);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->sgn_part, 128 * kRR);
  int64_t maxcap = 1;
  for (int i = 1; i <= d; ++i) maxcap = std::max(maxcap, h->cap[i]);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->P, maxcap * kRR);
  if (h->wt_bytes == 4) {
    h->ldv = (h->max_m + 31) / 32 * 32;
    h->ldp = (maxcap + 31) / 32 * 32;
    if (rc == TTICE_OK) rc = dalloc<float>(&h->Vnh, h->ldv * kRR);
    if (rc == TTICE_OK) rc = dalloc<float>(&h->Vnl, h->ldv * kRR);
    if (rc == TTICE_OK) rc = dalloc<float>(&h->Fh, kRR * kRR);
    if (rc == TTICE_OK) rc = dalloc<float>(&h->Fl, kRR * kRR);
    if (rc == TTICE_OK) rc = dalloc<double>(&h->dsq, kRR);
    if (rc == TTICE_OK) rc = dalloc<float>(&h->Ph, h->ldp * kRR);
    if (rc == TTICE_OK) rc = dalloc<float>(&h->Pl, h->ldp * kRR);
    int64_t vb = 0, pb = 0, vbs = 0, pbs = 0;
    for (int i = 0; i < d; ++i) {
      const int64_t k = std::min<int64_t>(kBlockDirs, kVBudget / std::max<int64_t>(h->ldu[i], 1) / 32 * 32);
      h->kb[i] = k >= 2 * kRR && h->cap[i + 1] > kRR ? (int)k : 0;
      if (!h->kb[i]) continue;
      vb = std::max(vb, h->ldu[i] * h->kb[i]);
      pb = std::max(pb, h->cap[i + 1] * h->kb[i]);
      vbs = std::max(vbs, (h->ldu[i] + 31) / 32 * 32 * h->kb[i]);     // split of V at ld rounded to 32
      pbs = std::max(pbs, (h->cap[i + 1] + 31) / 32 * 32 * h->kb[i]);  // split of P likewise
    }
    if (vb > 0) {
      if (rc == TTICE_OK) rc = dalloc<double>(&h->VB, vb);
      if (rc == TTICE_OK) rc = dalloc<float>(&h->VBh, vbs);
      if (rc == TTICE_OK) rc = dalloc<float>(&h->VBl, vbs);
      if (rc == TTICE_OK) rc = dalloc<double>(&h->PB, pb);
      if (rc == TTICE_OK) rc = dalloc<float>(&h->PBh, pbs);
      if (rc == TTICE_OK) rc = dalloc<float>(&h->PBl, pbs);
    }
    int64_t wt = 0, rs = 0;
    for (int i = 0; i < d; ++i) {
      const int64_t c = B * h->L[i], mi = h->ldu[i];
      wt = std::max(wt, c * ((h->cap[i + 1] + 31) / 32 * 32));
      rs = std::max(rs, std::max(c * ((mi + 31) / 32 * 32), mi * ((c + 31) / 32 * 32)));
    }
    h->wt_elems = wt;
    h->rs_elems = rs;
    if (rc == TTICE_OK) rc = dalloc<float>(&h->WTh, wt);
    if (rc == TTICE_OK) rc = dalloc<float>(&h->WTl, wt);
    if (rc == TTICE_OK) rc = dalloc<float>(&h->Rh, rs);
    if (rc == TTICE_OK) rc = dalloc<float>(&h->Rl, rs);
    if (rc == TTICE_OK) rc = dalloc<float>(&h->tcws, tc_ws_elems);
  }
  int64_t part_elems = std::max<int64_t>(2 * std::max<int64_t>(4 * 152 + B, B * ((h->L[0] + 255) / 256)),
                                         k1_tc_part_elems((int)B, h->L[0]));
  if (h->wt_bytes == 4)
    for (int i = 0; i < d; ++i)
      part_elems = std::max(part_elems, tc_proj_part_elems((int)B, h->L[i], h->cap[i + 1], h->ldu[i]));
  if (rc == TTICE_OK) rc = dalloc<double>(&h->part, part_elems);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->rho2, (int64_t)h->d * B);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->rn2, B);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->y2, B);
  if (rc == TTICE_OK) rc = dalloc<double>(&h->trace, 1);
  if (rc == TTICE_OK) rc = dalloc<Decision>(&h->dec, 1);
  if (rc == TTICE_OK) rc = dalloc<int>(&h->sel, B);
  if (rc == TTICE_OK) rc = dalloc<int>(&h->ibuf, 16);
  if (rc == TTICE_OK && !g_dry_run && cudaMallocHost((void**)&h->h_dec, sizeof(Decision)) != cudaSuccess) rc = TTICE_ENOMEM;
  if (rc == TTICE_OK && !g_dry_run && cudaMallocHost((void**)&h->h_sel, B * sizeof(int)) != cudaSuccess) rc = TTICE_ENOMEM;
  if (rc == TTICE_OK && !g_dry_run && cudaMallocHost((void**)&h->h_int, 16 * sizeof(int)) != cudaSuccess) rc = TTICE_ENOMEM;
  if (rc == TTICE_OK && !g_dry_run && cudaMallocHost((void**)&h->h_w32, s * sizeof(float)) != cudaSuccess) rc = TTICE_ENOMEM;
  if (rc == TTICE_OK && !g_dry_run && cudaMallocHost((void**)&h->h_dbl, 256 * sizeof(double)) != cudaSuccess) rc = TTICE_ENOMEM;
  if (rc == TTICE_OK && !g_dry_run && cudaMallocHost((void**)&h->h_rn2, B * sizeof(double)) != cudaSuccess) rc = TTICE_ENOMEM;
  if (rc == TTICE_OK && !g_dry_run && cudaMallocHost((void**)&h->h_rho2, (size_t)h->d * B * sizeof(double)) != cudaSuccess)
    rc = TTICE_ENOMEM;
  if (rc == TTICE_OK) rc = grow_last(h, std::max<int64_t>(h->capc.obs_reserve, 1));
  g_alloc_sink = nullptr;
  if (rc != TTICE_OK) {
    free_all(h);
    delete h;
    return rc;
  }
  fill_stats(h);
  *out = h;
  return TTICE_OK;
}

}  // namespace

extern "C" {

int ttice_create(const int64_t* dims, int d, double eps, const ttice_heuristics* hp,
                 const ttice_capacity* cp, ttice_t* out) {
  return create_handle(dims, d, eps, hp, cp, nullptr, out);
}

int ttice_capacities(ttice_t h, int64_t* caps) {
  if (!h || !caps) return TTICE_EINVAL;
  for (int i = 0; i <= h->d; ++i) caps[i] = h->cap[i];
  return TTICE_OK;
}

int ttice_device_bytes(ttice_t h, int64_t* bytes) {
  if (!h || !bytes) return TTICE_EINVAL;
  *bytes = h->dev_bytes;
  return TTICE_OK;
}

int ttice_projected_bytes(const int64_t* dims, int d, const ttice_heuristics* hp, const ttice_capacity* cp,
                          const int64_t* caps, int64_t* bytes) {
  if (!bytes) return TTICE_EINVAL;
  *bytes = 0;
  ttice_t h = nullptr;
  g_dry_run = true;
  const int rc = create_handle(dims, d, 0.5, hp, cp, caps, &h);
  g_dry_run = false;
  if (rc != TTICE_OK) return rc;
  *bytes = h->dev_bytes;
  delete h;  // a dry run holds no device or pinned memory
  return TTICE_OK;
}

int ttice_capacity_miss(ttice_t h, int* k, int64_t* need) {
  if (!h || !k || !need) return TTICE_EINVAL;
  *k = h->miss_k;
  *need = h->miss_need;
  return TTICE_OK;
}

int ttice_reserve_rank(ttice_t h, int k, int64_t cap) {
  if (!h || k < 1 || k > h->d || cap < 1) return TTICE_EINVAL;
  const int64_t want = std::min<int64_t>(cap, h->cap[k - 1] * h->n[k - 1]);
  if (want <= h->cap[k]) return TTICE_OK;
  int64_t caps[kMaxD + 1];
  for (int i = 0; i <= h->d; ++i) caps[i] = h->cap[i];
  caps[k] = want;
  ttice_capacity c = h->capc;
  c.obs_reserve = std::max<int64_t>(h->last_cap, 1);
  int64_t dims[kMaxD];
  for (int i = 0; i < h->d; ++i) dims[i] = h->n[i];
  ttice_t g = nullptr;
  TT_TRY(create_handle(dims, h->d, h->eps, &h->h, &c, caps, &g));
  // the decomposition: the leading (r_i n_i) x r_{i+1} block of every core (its row and column
  // layout does not depend on the capacities, only the leading dimension does) and the last core
  cudaStream_t fs = setup_stream();
  int rc = fs ? TTICE_OK : cu(cudaErrorNotReady);
  for (int i = 0; i < h->d && rc == TTICE_OK; ++i) {
    const int64_t rows = h->r[i] * h->n[i], cols = h->r[i + 1];
    if (rows == 0 || cols == 0) continue;
    rc = cu(cudaMemcpy2DAsync(g->U[i], g->ldu[i] * sizeof(double), h->U[i], h->ldu[i] * sizeof(double),
                              rows * sizeof(double), cols, cudaMemcpyDeviceToDevice, fs));
    if (rc == TTICE_OK && h->Uf[i])
      rc = cu(cudaMemcpy2DAsync(g->Uf[i], g->ldu[i] * sizeof(float), h->Uf[i], h->ldu[i] * sizeof(float),
                                rows * sizeof(float), cols, cudaMemcpyDeviceToDevice, fs));
    for (int hl = 0; hl < 2 && rc == TTICE_OK && h->Uh[i]; ++hl)
      rc = cu(cudaMemcpy2DAsync(hl ? g->Ul[i] : g->Uh[i], g->ldhl[i] * sizeof(float), hl ? h->Ul[i] : h->Uh[i],
                                h->ldhl[i] * sizeof(float), rows * sizeof(float), cols, cudaMemcpyDeviceToDevice, fs));
  }
  const int64_t rd = h->r[h->d];
  if (rc == TTICE_OK && h->n_obs > 0 && rd > 0)
    rc = cu(cudaMemcpy2DAsync(g->last, g->cap[g->d] * sizeof(double), h->last, h->cap[h->d] * sizeof(double),
                              rd * sizeof(double), h->n_obs, cudaMemcpyDeviceToDevice, fs));
  if (rc == TTICE_OK) rc = cu(cudaStreamSynchronize(fs));
  if (rc != TTICE_OK) {
    cudaGetLastError();
    free_all(g);
    delete g;
    return rc;
  }
  for (int i = 0; i <= h->d; ++i) g->r[i] = h->r[i];
  for (int i = 0; i < h->d; ++i) g->last_new[i] = h->last_new[i];
  g->n_obs = h->n_obs;
  g->stats = h->stats;
  g->prof_on = h->prof_on;
  g->prof = h->prof;
  std::swap(g->ev_pool, h->ev_pool);
  std::swap(*h, *g);  // h now holds the new buffers, g the old ones
  free_all(g);
  delete g;
  fill_stats(h);
  return TTICE_OK;
}

void ttice_destroy(ttice_t h) {
  if (!h) return;
  cudaDeviceSynchronize();
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  free_all(h);
  delete h;
}

int ttice_update(ttice_t h, const void* Y, int64_t batch, void* stream) {
  if (!h || !Y || batch < 1 || batch > h->capc.max_batch) return TTICE_EINVAL;
  cudaStream_t st = S(stream);
  const int b = (int)batch;
  if (h->wt_bytes == 8) {
    if (h->h.input_dtype == TTICE_F32) return update_impl<double, float>(h, (const float*)Y, b, st);
    return update_impl<double, double>(h, (const double*)Y, b, st);
  }
  if (h->h.input_dtype == TTICE_F32) return update_impl<float, float>(h, (const float*)Y, b, st);
  return update_impl<float, double>(h, (const double*)Y, b, st);
}

int ttice_project(ttice_t h, const void* Y, int64_t batch, double* coeffs, double* rel_err,
                  void* stream) {
  if (!h || !Y || batch < 1 || batch > h->capc.max_batch) return TTICE_EINVAL;
  cudaStream_t st = S(stream);
  const int b = (int)batch;
  if (h->wt_bytes == 8) {
    if (h->h.input_dtype == TTICE_F32) return project_impl<double, float>(h, (const float*)Y, b, coeffs, rel_err, st);
    return project_impl<double, double>(h, (const double*)Y, b, coeffs, rel_err, st);
  }
  if (h->h.input_dtype == TTICE_F32) return project_impl<float, float>(h, (const float*)Y, b, coeffs, rel_err, st);
  return project_impl<float, double>(h, (const double*)Y, b, coeffs, rel_err, st);
}

int ttice_ranks(ttice_t h, int64_t* ranks) {
  if (!h || !ranks) return TTICE_EINVAL;
  for (int i = 0; i <= h->d; ++i) ranks[i] = h->r[i];
  ranks[h->d + 1] = 1;
  return TTICE_OK;
}

int ttice_stats(ttice_t h, ttice_update_stats* st) {
  if (!h || !st) return TTICE_EINVAL;
  *st = h->stats;
  return TTICE_OK;
}

int ttice_reconstruct(ttice_t h, int64_t first, int64_t count, void* out, int out_dtype,
                      void* stream) {
  if (!h || !out || first < 0 || count < 1 || first + count > h->n_obs) return TTICE_EINVAL;
  if (out_dtype != TTICE_F32 && out_dtype != TTICE_F64) return TTICE_EINVAL;
  cudaStream_t st = S(stream);
  const int d = h->d;
  const int64_t rd = h->r[d];
  const size_t esize = out_dtype == TTICE_F32 ? 4 : 8;
  if (rd == 0) return cu(cudaMemsetAsync(out, 0, (size_t)count * h->N * esize, st));
  // observations are a grid dimension of the contractions (at most 65535 per launch): long ranges
  // are reconstructed in chunks through the same two intermediate buffers
  const int64_t chunk = std::min<int64_t>(count, kMaxGridZ);
  double *bufA = nullptr, *bufB = nullptr;
  if (d > 1) {
    if (cudaMallocAsync((void**)&bufA, (size_t)chunk * h->N * sizeof(double), st) != cudaSuccess) return TTICE_ENOMEM;
    if (cudaMallocAsync((void**)&bufB, (size_t)chunk * h->N * sizeof(double), st) != cudaSuccess) {
      cudaFreeAsync(bufA, st);
      return TTICE_ENOMEM;
    }
  }
  double* bufs[2] = {bufA, bufB};
  int rc = TTICE_OK;
  for (int64_t c0 = 0; c0 < count && rc == TTICE_OK; c0 += chunk) {
    const int64_t cnt = std::min(chunk, count - c0);
    void* outc = static_cast<char*>(out) + (size_t)c0 * h->N * esize;
    // X (per observation r_{i+1} x rest) -> U_i X (per observation (r_i n_i) x rest)
    const double* X = h->last + (first + c0) * h->cap[d];
    int64_t x_bs = h->cap[d];  // observation stride of X
    int64_t rest = 1;
    for (int i = d - 1; i >= 0 && rc == TTICE_OK; --i) {
      const int64_t m = h->r[i] * h->n[i], rn = h->r[i + 1];
      GemmArgs g;
      g.M = m; g.N = rest; g.K = rn;
      g.A.p = h->U[i]; g.A.rs = 1; g.A.cs = h->ldu[i];
      g.B.p = X; g.B.rs = rest; g.B.cs = 1; g.B.bs1 = x_bs;
      g.nbatch = (int)cnt;
      g.c_rs = rest; g.c_cs = 1; g.c_bs1 = m * rest;
      if (i == 0) {
        g.C = outc;
        if (out_dtype == TTICE_F64) rc = cu(gemm<double, double, double, double, double>(g, st));
        else rc = cu(gemm<double, double, double, float, double>(g, st));
      } else {
        double* dst = bufs[i & 1];
        g.C = dst;
        rc = cu(gemm<double, double, double, double, double>(g, st));
        X = dst;
        x_bs = m * rest;
      }
      rest *= h->n[i];
    }
  }
  if (bufA) cudaFreeAsync(bufA, st);
  if (bufB) cudaFreeAsync(bufB, st);
  return rc;
}

int ttice_info(ttice_t h, int* d, int64_t* dims, int* device) {
  if (!h) return TTICE_EINVAL;
  if (d) *d = h->d;
  if (dims)
    for (int i = 0; i < h->d; ++i) dims[i] = h->n[i];
  if (device) *device = h->device;
  return TTICE_OK;
}

int ttice_get_core(ttice_t h, int i, double* host, int64_t* rows, int64_t* cols) {
  if (!h || i < 1 || i > h->d) return TTICE_EINVAL;
  const int c = i - 1;
  const int64_t m = h->r[c] * h->n[c], r = h->r[c + 1];
  if (rows) *rows = m;
  if (cols) *cols = r;
  if (!host || m == 0 || r == 0) return TTICE_OK;
  std::vector<double> tmp((size_t)m * r);
  if (cudaMemcpy2D(tmp.data(), m * sizeof(double), h->U[c], h->ldu[c] * sizeof(double),
                   m * sizeof(double), r, cudaMemcpyDeviceToHost) != cudaSuccess)
    return TTICE_ECUDA;
  for (int64_t a = 0; a < m; ++a)
    for (int64_t b = 0; b < r; ++b) host[a * r + b] = tmp[b * m + a];
  return TTICE_OK;
}

int ttice_get_last_core(ttice_t h, double* host, int64_t* n_obs, int64_t* rd) {
  if (!h) return TTICE_EINVAL;
  const int64_t r = h->r[h->d];
  if (n_obs) *n_obs = h->n_obs;
  if (rd) *rd = r;
  if (!host || h->n_obs == 0 || r == 0) return TTICE_OK;
  if (cudaMemcpy2D(host, r * sizeof(double), h->last, h->cap[h->d] * sizeof(double),
                   r * sizeof(double), h->n_obs, cudaMemcpyDeviceToHost) != cudaSuccess)
    return TTICE_ECUDA;
  return TTICE_OK;
}

int ttice_profile_enable(ttice_t h, int on) {
  if (!h) return TTICE_EINVAL;
  h->prof_on = on != 0;
  std::memset(&h->prof, 0, sizeof(h->prof));
  h->marks.clear();
  h->ev_used = 0;
  return TTICE_OK;
}

int ttice_profile_read(ttice_t h, ttice_profile* out) {
  if (!h || !out) return TTICE_EINVAL;
  *out = h->prof;
  return TTICE_OK;
}

int64_t ttice_kernel_launches(void) { return g_kernel_launches.load(); }

int ttice_load(ttice_t h, const int64_t* ranks, const double* const* cores, const double* last,
               int64_t n_obs) {
  if (!h || !ranks || ranks[0] != 1 || n_obs < 0 || (n_obs > 0 && !last)) return TTICE_EINVAL;
  int64_t last_elems = 0;  // the last core at capacity width must be addressable
  if (__builtin_mul_overflow(n_obs, h->cap[h->d], &last_elems) || last_elems > INT64_MAX / 8) return TTICE_EINVAL;
  for (int i = 1; i <= h->d; ++i) {
    if (ranks[i] < 0 || ranks[i] > h->cap[i] || ranks[i] > ranks[i - 1] * h->n[i - 1]) return TTICE_ECAPACITY;
    if (ranks[i] > 0 && !cores[i - 1]) return TTICE_EINVAL;
  }
  TT_TRY(grow_last(h, std::max<int64_t>(n_obs, 1)));
  for (int i = 0; i < h->d; ++i) {
    const int64_t ld = h->ldu[i], m = ranks[i] * h->n[i], r = ranks[i + 1];
    std::vector<double> colmajor((size_t)ld * h->cap[i + 1], 0.0);
    for (int64_t a = 0; a < m; ++a)
      for (int64_t b = 0; b < r; ++b) colmajor[b * ld + a] = cores[i][a * r + b];
    TT_CU(cudaMemcpy(h->U[i], colmajor.data(), colmajor.size() * sizeof(double), cudaMemcpyHostToDevice));
    if (h->Uf[i]) {
      std::vector<float> f(colmajor.begin(), colmajor.end());
      TT_CU(cudaMemcpy(h->Uf[i], f.data(), f.size() * sizeof(float), cudaMemcpyHostToDevice));
    }
    if (h->Uh[i]) {
      TT_CU(launch_split_tf32(h->Uf[i], ld, 0, h->cap[i + 1], h->Uh[i], h->Ul[i], h->ldhl[i], nullptr));
      TT_CU(cudaStreamSynchronize(nullptr));
    }
  }
  const int64_t capd = h->cap[h->d];
  std::vector<double> lc((size_t)h->last_cap * capd, 0.0);
  for (int64_t j = 0; j < n_obs; ++j)
    for (int64_t a = 0; a < ranks[h->d]; ++a) lc[j * capd + a] = last[j * ranks[h->d] + a];
  TT_CU(cudaMemcpy(h->last, lc.data(), lc.size() * sizeof(double), cudaMemcpyHostToDevice));
  for (int i = 0; i <= h->d; ++i) h->r[i] = ranks[i];
  h->n_obs = n_obs;
  fill_stats(h);
  return TTICE_OK;
}

}  // extern "C"

namespace {
int save_impl(ttice_t h, const char* path);
int open_impl(const char* path, const ttice_capacity* cp, ttice_t* out);
}  // namespace

extern "C" {

// Checkpoints build host copies of the cores: an allocation failure there is reported, not thrown
// across the C ABI.
int ttice_save(ttice_t h, const char* path) {
  if (!h || !path) return TTICE_EINVAL;
  try {
    return save_impl(h, path);
  } catch (const std::bad_alloc&) {
    return TTICE_ENOMEM;
  }
}

int ttice_open(const char* path, const ttice_capacity* cp, ttice_t* out) {
  if (!path || !out) return TTICE_EINVAL;
  *out = nullptr;
  try {
    return open_impl(path, cp, out);
  } catch (const std::bad_alloc&) {
    return TTICE_ENOMEM;
  }
}

}  // extern "C"

namespace {

int save_impl(ttice_t h, const char* path) {
  const int d = h->d;
  std::vector<std::vector<double>> cores(d);
  std::vector<const double*> ptrs(d, nullptr);
  for (int i = 1; i <= d; ++i) {
    int64_t rows = 0, cols = 0;
    TT_TRY(ttice_get_core(h, i, nullptr, &rows, &cols));
    cores[i - 1].resize((size_t)(rows * cols));
    if (rows * cols > 0) TT_TRY(ttice_get_core(h, i, cores[i - 1].data(), &rows, &cols));
    ptrs[i - 1] = cores[i - 1].data();
  }
  int64_t n_obs = 0, rd = 0;
  TT_TRY(ttice_get_last_core(h, nullptr, &n_obs, &rd));
  std::vector<double> last((size_t)(n_obs * rd));
  if (!last.empty()) TT_TRY(ttice_get_last_core(h, last.data(), &n_obs, &rd));
  int64_t ranks[kMaxD + 1];
  for (int i = 0; i <= d; ++i) ranks[i] = h->r[i];
  return ttice_checkpoint_write(path, d, h->n, h->eps, &h->h, ranks, ptrs.data(), last.data(), n_obs);
}

int open_impl(const char* path, const ttice_capacity* cp, ttice_t* out) {
  int d = 0;
  int64_t dims[kMaxD], ranks[kMaxD + 1], n_obs = 0;
  double eps = 0.0;
  ttice_heuristics heur{};
  TT_TRY(ttice_checkpoint_read(path, &d, dims, &eps, &heur, ranks, &n_obs, nullptr, nullptr));
  std::vector<std::vector<double>> cores(d);
  std::vector<double*> ptrs(d);
  std::vector<const double*> cptrs(d);
  for (int i = 0; i < d; ++i) {
    cores[i].resize((size_t)(ranks[i] * dims[i] * ranks[i + 1]) + 1);
    ptrs[i] = cores[i].data();
    cptrs[i] = cores[i].data();
  }
  std::vector<double> last((size_t)(n_obs * ranks[d]) + 1);
  TT_TRY(ttice_checkpoint_read(path, &d, dims, &eps, &heur, ranks, &n_obs, ptrs.data(), last.data()));
  ttice_capacity c;
  ttice_default_capacity(&c);
  if (cp) c = *cp;
  c.obs_reserve = std::max<int64_t>(c.obs_reserve, n_obs);
  int64_t caps[kMaxD + 1];
  caps[0] = 1;
  for (int i = 1; i <= d; ++i) caps[i] = std::max<int64_t>(c.max_rank, std::max<int64_t>(ranks[i], 1));
  ttice_t h = nullptr;
  TT_TRY(create_handle(dims, d, eps, &heur, &c, caps, &h));
  const int rc = ttice_load(h, ranks, cptrs.data(), last.data(), n_obs);
  if (rc != TTICE_OK) {
    ttice_destroy(h);
    return rc;
  }
  *out = h;
  return TTICE_OK;
}

}  // namespace

// ================================================================== allocation-free reconstruction
// ttice_reconstruct obtains its two intermediate buffers from cudaMallocAsync on every call.  Some
// callers cannot allocate device memory at the point where they need a reconstruction: code running
// under a CUDA-graph capture that must not contain allocation nodes, real-time loops that forbid the
// allocator's latency and possible synchronisation, or processes whose device memory is carved up
// in advance by another runtime.  ttice_reconstruct_noalloc computes exactly the same chain of
// contractions but keeps the intermediates in a fixed array of device memory that belongs to this
// library: kNoAllocElems doubles per buffer, two buffers (64 MiB in total), held by every GPU that
// loads the library until the process exits.
namespace {

constexpr int64_t kNoAllocElems = TTICE_NOALLOC_MAX_ELEMS;
static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocElems];

// Host code may not use g_noalloc_scratch directly (on the host it is only a stand-in symbol, not a
// device address).  Its device address is looked up once per device, with that device current, and
// cached; the first call on a device therefore does this lookup.
double* noalloc_scratch_for_current_device(int* err) {
  static std::mutex mu;
  static double* addr[64] = {};
  static bool done[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) { *err = TTICE_ECUDA; return nullptr; }
  std::lock_guard<std::mutex> lock(mu);
  if (!done[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess) {
      cudaGetLastError();
      *err = TTICE_ECUDA;
      return nullptr;
    }
    addr[dev] = static_cast<double*>(p);
    done[dev] = true;
  }
  *err = TTICE_OK;
  return addr[dev];
}

}  // namespace

extern "C" int ttice_reconstruct_noalloc(ttice_t h, int64_t first, int64_t count, void* out,
                                         int out_dtype, void* stream) {
  if (!h || !out || first < 0 || count < 1 || first + count > h->n_obs) return TTICE_EINVAL;
  if (out_dtype != TTICE_F32 && out_dtype != TTICE_F64) return TTICE_EINVAL;
  if (count > 65535 || count * h->N > kNoAllocElems) return TTICE_EINVAL;  // beyond the fixed scratch
  int err = TTICE_OK;
  double* scratch = noalloc_scratch_for_current_device(&err);
  if (err != TTICE_OK) return err;
  cudaStream_t st = S(stream);
  const int d = h->d;
  if (h->r[d] == 0) {
    return cu(cudaMemsetAsync(out, 0, (size_t)count * h->N * (out_dtype == TTICE_F32 ? 4 : 8), st));
  }
  // Every element of an intermediate is written before it is read (plain stores, no accumulation),
  // so the contents left by an earlier call never need clearing.
  double* bufs[2] = {scratch, scratch + kNoAllocElems};
  const double* X = h->last + first * h->cap[d];
  int64_t x_bs = h->cap[d];
  int64_t rest = 1;
  for (int i = d - 1; i >= 0; --i) {
    const int64_t m = h->r[i] * h->n[i], rn = h->r[i + 1];
    GemmArgs g;
    g.M = m; g.N = rest; g.K = rn;
    g.A.p = h->U[i]; g.A.rs = 1; g.A.cs = h->ldu[i];
    g.B.p = X; g.B.rs = rest; g.B.cs = 1; g.B.bs1 = x_bs;
    g.nbatch = (int)count;
    g.c_rs = rest; g.c_cs = 1; g.c_bs1 = m * rest;
    int rc;
    if (i == 0) {
      g.C = out;
      if (out_dtype == TTICE_F64) rc = cu(gemm<double, double, double, double, double>(g, st));
      else rc = cu(gemm<double, double, double, float, double>(g, st));
    } else {
      double* dst = bufs[i & 1];
      g.C = dst;
      rc = cu(gemm<double, double, double, double, double>(g, st));
      X = dst;
      x_bs = m * rest;
    }
    if (rc != TTICE_OK) return rc;
    rest *= h->n[i];
  }
  return TTICE_OK;
}
