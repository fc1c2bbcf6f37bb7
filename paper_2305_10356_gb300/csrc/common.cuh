// Internal declarations shared by the translation units of libofsc (not part of the C ABI).
#pragma once

// Checked build (-DOFSC_DEBUG=1): the direction product checks every column index and row range
// before it uses them, records the first violation instead of making the access, and the calls
// that run it return OFSC_ERR_INVALID_ARG naming it.
#ifndef OFSC_DEBUG
#define OFSC_DEBUG 0
#endif

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/ofsc.h"
#include "spmm_dir.cuh"

namespace ofsc {

constexpr int kNumSMs = 152;  // GB300: 2 dies x 76 SMs
constexpr int kMaxK = 128;    // widest padded feature block handled by the kernels

// Last-error message of the calling host thread.
void set_error(const char* fmt, ...);
void clear_error();

// Records `st` with a message and returns it.
ofsc_status fail(ofsc_status st, const char* fmt, ...);

// Maps a CUDA error to OFSC_ERR_CUDA / OFSC_ERR_OOM and records it.
ofsc_status cuda_fail(cudaError_t e, const char* what);

// Device memory of the library: cudaMalloc / cudaFree, or the caller's allocator when one is set
// (ofsc_set_allocator). A block is always freed by the allocator that made it; freeing through a
// caller's allocator synchronises the device first, so no queued kernel still uses the block.
cudaError_t dev_alloc_bytes(void** p, size_t bytes);
cudaError_t dev_free(void* p);
template <class T>
inline cudaError_t dev_alloc(T** p, size_t bytes) {
  return dev_alloc_bytes(reinterpret_cast<void**>(p), bytes);
}
// An NVTX range over a host phase of a call (no cost without an attached tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// A call's scratch block, freed when the call returns (both frees wait for the device's queued work).
struct DevBuf {
  void* p = nullptr;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { dev_free(p); }
};

#define OFSC_CUDA(call)                                        \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return ::ofsc::cuda_fail(e_, #call); \
  } while (0)

#define OFSC_LAUNCH_CHECK(what)                                 \
  do {                                                          \
    cudaError_t e_ = cudaGetLastError();                        \
    if (e_ != cudaSuccess) return ::ofsc::cuda_fail(e_, what);  \
  } while (0)

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Lanes per row in the sparse product (4 values per lane) and the index of its partition.
inline int spmm_lanes(int kp) {
  int l = 2;
  while (l * 4 < kp) l *= 2;
  return l;
}
inline int spmm_lanes_index(int lanes) {
  return lanes <= 2 ? 0 : lanes <= 4 ? 1 : lanes <= 8 ? 2 : lanes <= 16 ? 3 : 4;
}
// Lane groups of the sparse product: about 512 nonzeros each, between 1 and 4 blocks per SM.
// Warps of the direction product (one row at a time per warp): about kRowNnz nonzeros each, at
// least OFSC_ROW_MIN_WARPS_PER_SM per SM (a small graph takes few SMs, leaving the rest to other
// problems' kernels in a batch) and at most kRowMaxWarps, in blocks of kRowWarpsPerBlock warps. Blocks of one warp retire as soon as their warp is done, so the
// hardware balances the load warp by warp (blocks of eight warps, held by their slowest warp,
// measured 22-29% slower on the 2M-node, k = 128 graph). A warp takes a hub row whole, so a warp's
// share must stay well above the largest degree. The macros exist for tuning builds.
#ifndef OFSC_ROW_WPB
#define OFSC_ROW_WPB 1
#endif
#ifndef OFSC_ROW_NNZ
#define OFSC_ROW_NNZ 256
#endif
#ifndef OFSC_ROW_MAX_WARPS_PER_SM
#define OFSC_ROW_MAX_WARPS_PER_SM 32
#endif
#ifndef OFSC_ROW_MIN_WARPS_PER_SM
#define OFSC_ROW_MIN_WARPS_PER_SM 4
#endif
constexpr int kRowPart = 5;
constexpr int kRowWarpsPerBlock = OFSC_ROW_WPB;
constexpr int kRowNnz = OFSC_ROW_NNZ;
constexpr int kRowMaxWarps = OFSC_ROW_MAX_WARPS_PER_SM * kNumSMs;
inline int row_warps(int64_t nnz) {
  int64_t w = nnz / kRowNnz;
  if (w < OFSC_ROW_MIN_WARPS_PER_SM * kNumSMs) w = OFSC_ROW_MIN_WARPS_PER_SM * kNumSMs;
  if (w > kRowMaxWarps) w = kRowMaxWarps;
  return (int)ceil_div(w, kRowWarpsPerBlock) * kRowWarpsPerBlock;
}
// Per-block partial sums of the sparse product's dots are folded to at most this many rows, in a
// fixed order, before the line-search solve reads them.
constexpr int kDotsRows = 64;
// Blocks of the V pass (each writes one row of diag(V^T G) partials).
constexpr int kVpassMaxBlocks = 8 * kNumSMs;
inline int spmm_groups(int64_t nnz, int lpr) {
  const int64_t gpb = 256 / lpr;
  int64_t g = nnz / 512;
  if (g < kNumSMs * gpb) g = kNumSMs * gpb;
  if (g > 4 * kNumSMs * gpb) g = 4 * kNumSMs * gpb;
  return (int)ceil_div(g, gpb) * (int)gpb;
}

// Device control block of one ofsc_iterate / ofsc_objective_grad call.
struct Ctrl {
  int it;          // updates X <- X + V diag(alpha) applied so far
  int done;        // 1 once the loop must stop (every kernel returns early)
  int converged;   // 1 if ||G_t|| <= tol ||G_0||
  int status;      // OFSC_OK or OFSC_ERR_NONFINITE
  int maxit;
  int trace_cap;
  int k;           // real (unpadded) columns
  int restart;     // 1: the optional CG restart (beta_j = 0 where v_j . g_j >= 0); 0: Algorithm 2
  int vscale_exp;  // columns of V are stored scaled once |V_j| exceeds 2^vscale_exp ||G_0||
  int withhold;    // test hook: the tensor-core direction pass's converters withhold their arrivals
  long long spin_limit;  // polls per bounded mbarrier wait (0: the compiled default)
  double tol;
  double g0;       // ||G_0||_F
  double gnorm;    // ||G_t||_F of the last direction pass
  double rel;      // gnorm / g0
  double f;        // objective at X_t
  double normA2;   // ||A||_F^2
  double trB;      // tr(X^T A X) of the current X (carried for the f1 objective)
  int dots_blocks; // blocks of the last sparse product that wrote dot partials
  int near_tol;    // 1 once ||G_t|| <= tol ||G_0|| was seen on an update whose AX came from the
                   // recurrence: the host then makes every later update exact, and only an exact
                   // update may stop the run
};


// Device workspace of the iteration for one padded width kp, cached on the graph handle.
struct Workspace {
  int64_t n = 0;
  int kp = 0;
  int gather = 0;
  float* X = nullptr;   // n x kp, working copy of the block (zero padded)
  float* Y = nullptr;   // A X
  float* V = nullptr;   // search direction
  float* W = nullptr;   // A V
  float* G = nullptr;   // direction g(X) of the last pass (G_{t-1} while G_t is formed)
  void* Vh = nullptr;   // D^-1/2 V, FP32 or BF16: the block gathered by the sparse product
  double* gram_part = nullptr;  // [gram_gy][6][kp*kp] per-row-group partial Grams
  double* gram = nullptr;       // [6][kp*kp] reduced Grams R, P, Q, B, E, C
  float* Rn = nullptr;          // kp*kp: X^T X for the next direction pass
  float* Bn = nullptr;          // kp*kp: X^T A X for the next direction pass
  double* R64 = nullptr;        // kp*kp: X^T X of the current X (exact recurrence, FP64)
  double* B64 = nullptr;        // kp*kp: X^T A X of the current X (f2 methods)
  double* dots = nullptr;       // [spmm blocks][2][kp]: partial diag(V^T AV), diag(V^T AX)
  float* part_tc = nullptr;     // tensor-core Gram partials (sized for kp > 64, or when a call
  size_t part_tc_bytes = 0;     // forces the tensor-core Grams at a smaller kp)
  CUtensorMap vh_map[2];        // TMA maps over Vh as FP32 [0] and BF16 [1] (gather4 rows)
  bool vh_map_ok[2] = {false, false};
  float* alpha = nullptr;       // kp
  float* beta = nullptr;        // kp
  double* alpha64 = nullptr;    // kp
  double* beta64 = nullptr;     // kp
  // Extended exponent range of the direction: the stored FP32 V holds V_true diag(1 / vscale) with
  // vscale a power of two per column (1 unless V_true outgrows 2^vscale_exp ||G_0||), so beta products
  // that FP64 represents cannot overflow FP32 storage; vinv = 1 / vscale in FP32 for the V pass.
  double* vscale = nullptr;     // kp
  float* vinv = nullptr;        // kp
  double* colpart = nullptr;    // [row_blocks][5][kp]
  double* dE = nullptr;         // kp: diag(V^T AX) (f1 methods)
  void* bimg = nullptr;         // kp = 128: B operand images of the f2 tensor-core direction pass
  int64_t* carry_row = nullptr; // [kRowMaxWarps][2]: split rows of the merge-path product
  float* carry = nullptr;       // [kRowMaxWarps][2][kp]: their partial sums
  double* solve = nullptr;      // line-search scratch: per-block trace partials, diagonals, cubics
  Ctrl* ctrl = nullptr;
  Ctrl* ctrl_host = nullptr;    // pinned
  int gram_gy = 0;
  int row_blocks = 0;
  size_t bytes = 0;
  std::vector<cudaEvent_t> events;  // pool for the optional per-phase timing
  int64_t launches = 0;             // kernels launched by the current call
};

}  // namespace ofsc

// The CG state between calls (ofsc_state_create): V_{t-1}, G_{t-1} (n x kp FP32), V's column
// scales (kp), V_{t-1}^T V_{t-1} (kp x kp), the run's update count t (0: empty), ||G_0|| and the
// method that made it.
struct ofsc_state {
  int64_t n = 0;
  int k = 0, kp = 0, method = -1, device = 0;
  int64_t t = 0;
  double g0 = 0.0;
  float* V = nullptr;
  float* G = nullptr;
  double* vscale = nullptr;
  double* Q = nullptr;
};

struct ofsc_graph {
  int64_t n = 0;
  int64_t m_in = 0;
  int64_t nnz = 0;
  int64_t n_selfloops = 0;
  int64_t n_duplicates = 0;
  int64_t n_isolated = 0;
  int weighted = 0;
  double normA2 = 0.0;
  int device = 0;
  // The direction product's shape chosen by ofsc_autotune for one padded width and gather storage:
  // gathers in flight per lane (0: the kernel's default); the row partition is bnd[kRowPart].
  // Merge-path shares of the direction product's warps (mp[2 groups + 2], recomputed with the row
  // partition) and the longest row's nonzeros: rows longer than a warp's share use them.
  int64_t* mp = nullptr;
  int64_t max_row = 0;
  int dir_tuned_kp = 0;
  int dir_tuned_bf16 = 0;
  int dir_slots = 0;
  int dir_mp = 0;  // 1: merge path timed faster, -1: whole rows, 0: untuned
  int64_t* row_ptr = nullptr;  // [n+1]
  int32_t* col = nullptr;      // [nnz]
  float* val = nullptr;        // [nnz] or null
  float* dinv = nullptr;       // [n]  D^-1/2 in FP32
  double* deg = nullptr;       // [n]
  // nnz-balanced row ranges of the sparse product's lane groups, one partition per group width
  // (2, 4, 8, 16, 32 lanes): bnd[i] has groups[i] + 1 entries
  // bnd[5]: warps of the direction product (one row at a time per warp, kRowWarpsPerBlock warps
  // per block)
  int64_t* bnd[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  int groups[6] = {0, 0, 0, 0, 0, 0};
  ofsc::Workspace ws;
  cudaStream_t stream = nullptr;  // this graph's stream in ofsc_iterate_batched (created on first use)
  // opts.overlap_gram: the stream the Grams V^T X, V^T V run on beside the direction product, and
  // the events that fork it from and join it to the update's stream (created on first use)
  cudaStream_t side = nullptr;
  cudaEvent_t side_fork = nullptr, side_join = nullptr;
};

namespace ofsc {
void workspace_free(Workspace& ws);

// Arguments of one tensor-core Gram launch (csrc/gram_tc.cu): L^T R_b over all rows.
struct GramTcArgs {
  int64_t n;             // rows
  int ld;                // row stride of every block, in floats (multiple of 4, rows 16-byte aligned)
  int k;                 // features read (<= 128); features k..127 count as zero
  int nr;                // right blocks (1..4)
  const float* L;        // left block
  const float* R[4];     // right blocks
  int lslot;             // index b with R[b] == L (its tiles serve as the A operand), or -1
  int64_t rows_per_cta;  // multiple of 32
  float* part;           // [ctas][nr][128][128] FP32 partials
  Ctrl* ctrl;            // status / stop flag (may be null only with ignore_done = 1)
  int ignore_done;
  int use_ws;            // allow the warp-specialised TMA kernel (L one of R, nr <= 2; own segments)
};
// Arguments of the direction pass (k_direction in csrc/iterate.cu, k_direction_tc in
// csrc/direction_tc.cu).
struct RowArgs {
  int64_t n;
  int kp;
  float* X;
  float* Y;
  const float* V;
  const float* W;
  float* G;
  const float* Rn;
  const float* Bn;
  const float* alpha;
  double* colpart;  // [gridDim.x][6][kp]: sums of G^2, (G - G_prev) G, G_prev^2, G AX, V_prev AX, V_prev G
  Ctrl* ctrl;
  int update;
  int need_vy;      // read V_{t-1} for the V_prev AX sums even without an update
  int eval;         // no previous G (objective/gradient evaluation and the final report)
  int ignore_done;
  void* bimg;       // f2 tensor-core pass: 256 KB for the B operand images of X^T A X and X^T X
};

// Arguments of the TMA-gather sparse product (csrc/spmm_tma.cu): out = -base - D^-1/2 S Vh.
struct TmaSpmmArgs {
  int64_t n;
  int kp;
  const int64_t* row_ptr;
  const int32_t* col;
  const float* val;
  const float* dinv;
  const int64_t* bnd;   // [groups + 1] row ranges, one per warp
  int groups;
  const float* base;    // V
  float* out;           // AV
  double* dots;         // [groups / 4][kp] partials of diag(V^T AV)
  Ctrl* ctrl;
};
bool spmm_tma_supported(int kp);
int spmm_tma_groups_per_block();
ofsc_status spmm_tma_encode(const void* vh, int64_t n, int kp, bool bf16, CUtensorMap* map);
// 2-D tensor map over a row-major FP32 block (rows x cols, row stride ld values): boxes of box_cols
// x box_rows values with the 128-byte swizzle (box_cols <= 32), zero fill outside the block.
ofsc_status tma_encode_f32_sw128(const float* base, int64_t rows, int cols, int ld, int box_cols, int box_rows,
                                 CUtensorMap* map);
cudaError_t spmm_tma_launch(const CUtensorMap& map, const TmaSpmmArgs& a, bool bf16, bool weighted, cudaStream_t s);

// Direction pass of OFM-f1 / TriOFM-f1 at padded k = 128 with the kp x kp product on the tensor
// cores (csrc/direction_tc.cu); *nblk receives the rows of column-sum partials written.
bool direction_tc_supported(int method, int kp);
cudaError_t direction_tc_launch(int method, const RowArgs& a, cudaStream_t s, int* nblk);

// Edge-weight gradient of f1 / f2 (csrc/wgrad.cu).
struct WgradArgs {
  int64_t n;
  int kp;
  int which;             // 1: f1, 2: f2
  const float* X;        // [n][kp]
  const float* AX;       // [n][kp]
  const double* R64;     // X^T X (f2)
  const int64_t* row_ptr;
  const int32_t* col;
  const float* val;      // weighted S (or null)
  const float* dinv;
  float* r;              // [n] scratch
  float* Z;              // [n][kp] scratch (f2)
  int64_t m;
  const int32_t* src;
  const int32_t* dst;
  float* grad;           // [m]
  int* bad;              // set when an endpoint is out of range
};
// Y = A X = -X - D^-1/2 S D^-1/2 X for an n x kp FP32 row block (kp a multiple of 8, rows 16-byte
// aligned); scratch: n x kp FP32 (receives D^-1/2 X). Queued on s; no control block.
cudaError_t apply_A(ofsc_graph* g, int kp, const float* X, float* Y, float* scratch, cudaStream_t s);
// Replaces the direction product's row partition (bnd[kRowPart]) with `warps` nnz-balanced row
// ranges; synchronises s.
ofsc_status set_row_partition(ofsc_graph* g, int warps, cudaStream_t s);
cudaError_t wgrad_launch(const WgradArgs& w, cudaStream_t s);

// Rayleigh-Ritz algebra of csrc/ritz.cu (k x k FP64; work holds [4][kp][kp] doubles).
cudaError_t ritz_prepare_launch(const double* R64, const double* B64, int k, int kp, double* work, float* Rn,
                                double* lam, double* sums, Ctrl* ctrl, cudaStream_t s);
cudaError_t ritz_relerr_launch(const double* GtG, const double* work, int k, int kp, const double* sums, double* out,
                               cudaStream_t s);

int64_t gram_tc_rows_per_cta(int64_t n, int nr);
size_t gram_tc_part_bytes(int64_t n, int nr, int64_t rows_per_cta);
cudaError_t gram_tc_launch(GramTcArgs a, const int* slot, int kp, double* gram, cudaStream_t s);
cudaError_t gram_tc_launch_ld(GramTcArgs a, const int* slot, int kout, int ld_out, int64_t kk_stride,
                              double* gram, cudaStream_t s);
}
