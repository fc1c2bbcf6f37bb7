// Algorithm 2 on the device: the direction pass, the sparse product with its fused epilogue, the
// k x k Gram reductions and the FP64 exact line search (Sec. 3.2), driven by ofsc_iterate.
//
// Per update t (the paper's steps 7-11, Sec. 4) the device runs:
//   direction pass  X += V diag(alpha), AX += AV diag(alpha)   (previous update, fused)
//                   G = g(X) from AX and the k x k blocks X^T X, X^T A X       (Eqs. (5),(7),(10),(12))
//                   column sums for beta and ||G||
//   beta            beta_i = sum (G - G_prev) G / sum G_prev^2, stop test        (Algorithm 2)
//   V pass          V = -G + V diag(beta), Vh = D^-1/2 V (FP32 or BF16)
//   sparse product  AV = -V - D^-1/2 S Vh by gathering rows of Vh, with diag(V^T AV), diag(V^T G)
//   Grams           V^T X, V^T V (and V^T AX, V^T AV for f2)                     (Sec. 3.3)
//   line search     cubic coefficients, real roots, alpha; X^T X and X^T A X of the next X
// AX is carried by the recurrence AX_{t+1} = AX_t + AV_t diag(alpha_t), exact in exact arithmetic
// since A is linear; it is recomputed from X every y_refresh updates and at the end. AV itself
// is computed from V every update: a recurrence for it would multiply its rounding error by the
// column-wise beta, which is not bounded by 1.
#include <cuda_bf16.h>
#include <stdarg.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "group.cuh"
#include "cubic.cuh"

namespace ofsc {
namespace {
// Columns of the stored direction are rescaled once |V_j| exceeds 2^kDefaultVscaleExp ||G_0||.
constexpr int kDefaultVscaleExp = 20;
}  // namespace
}  // namespace ofsc

namespace ofsc {
namespace {

enum { M_OFM_F1 = 0, M_TRI_F1 = 1, M_OFM_F2 = 2, M_TRI_F2 = 3 };
constexpr int kPairs = 6;
enum { G_R = 0, G_P = 1, G_Q = 2, G_B = 3, G_E = 4, G_C = 5 };
constexpr int kRowThreads = 256;
constexpr int kMaxRowBlocks = 8 * kNumSMs;
constexpr int kGramChunk = 32;    // rows staged in shared memory per Gram step

__device__ __forceinline__ bool is_tri(int method) { return method == M_TRI_F1 || method == M_TRI_F2; }
__device__ __forceinline__ bool is_f2(int method) { return method >= M_OFM_F2; }

// ------------------------------------------------------------------------------------------
// Setup kernels
// ------------------------------------------------------------------------------------------

__global__ void k_init_ctrl(Ctrl* c, double tol, int maxit, int k, double normA2, int trace_cap, int restart = 0,
                            int vscale_exp = kDefaultVscaleExp, long long spin_limit = 0, int withhold = 0) {
  c->it = 0;
  c->restart = restart;
  c->vscale_exp = vscale_exp;
  c->spin_limit = spin_limit;
  c->withhold = withhold;
  c->done = 0;
  c->converged = 0;
  c->status = OFSC_OK;
  c->maxit = maxit;
  c->trace_cap = trace_cap;
  c->k = k;
  c->tol = tol;
  c->g0 = 0.0;
  c->gnorm = 0.0;
  c->rel = 1.0;
  c->f = 0.0;
  c->normA2 = normA2;
  c->trB = 0.0;
  c->dots_blocks = 0;
  c->near_tol = 0;
}

__global__ void k_pad_in(int64_t n, int k, int kp, const float* __restrict__ src,
                         float* __restrict__ dst, Ctrl* ctrl) {
  int bad = 0;
  const int64_t total = n * kp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t l = i / kp;
    int c = (int)(i - l * kp);
    float x = c < k ? src[l * k + c] : 0.0f;
    if (!isfinite(x)) bad = 1;
    dst[i] = x;
  }
  if (bad) {
    ctrl->status = OFSC_ERR_NONFINITE;
    ctrl->done = 1;
  }
}

__global__ void k_pad_out(int64_t n, int k, int kp, const float* __restrict__ src, float* __restrict__ dst) {
  const int64_t total = n * k;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t l = i / k;
    int c = (int)(i - l * k);
    dst[i] = src[l * kp + c];
  }
}

// X += V diag(alpha) without touching AX (the refresh recomputes AX from X afterwards).
__global__ void k_update_x(int64_t n, int kp, float* __restrict__ X, const float* __restrict__ V,
                           const float* __restrict__ alpha, Ctrl* ctrl) {
  if (ctrl->done) return;
  const int64_t total = n * kp;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    int c = (int)(i % kp);
    X[i] = fmaf(alpha[c], V[i], X[i]);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->it += 1;
}

// ------------------------------------------------------------------------------------------
// Sparse product Y = A M with A = -I - D^-1/2 S D^-1/2, fused epilogues
// ------------------------------------------------------------------------------------------


__device__ __forceinline__ void fma4(float4& acc, float w, const float4& v) {
  acc.x = fmaf(w, v.x, acc.x);
  acc.y = fmaf(w, v.y, acc.y);
  acc.z = fmaf(w, v.z, acc.z);
  acc.w = fmaf(w, v.w, acc.w);
}

// AX = -X - D^-1/2 S D^-1/2 X row by row, the exact product behind the objective, the gradient
// and the periodic refresh of the AX recurrence (each gathered row is scaled by its own D^-1/2
// entry and edge weight). A group of LANES lanes owns a contiguous range of rows holding about
// nnz / groups nonzeros; lane q holds columns [4q, 4q + 4). For each row the group loads up to
// LANES column indices at once and keeps 8 row gathers in flight per lane.
template <int LANES, bool WEIGHTED>
__global__ void __launch_bounds__(256, 2) k_spmm(SpmmArgs a) {
  if (!a.ignore_done && a.ctrl->done) return;
  constexpr int GPB = 256 / LANES;
  const int lane = threadIdx.x % LANES;
  const int grp = threadIdx.x / LANES;
  const unsigned mask = LANES == 32 ? 0xffffffffu : (((1u << LANES) - 1u) << ((threadIdx.x & 31) / LANES * LANES));
  const int c = lane * 4;
  const bool active = c < a.kp;
  const int gid = blockIdx.x * GPB + grp;
  if (gid >= a.groups) return;
  const float* X = (const float*)a.gather;
  const int64_t ra = a.bnd[gid], rb = a.bnd[gid + 1];
  int64_t p1 = ra < rb ? a.row_ptr[ra] : 0;
  for (int64_t l = ra; l < rb; ++l) {
    const int64_t p0 = p1;
    p1 = a.row_ptr[l + 1];
    const int64_t o = l * a.kp + c;
    float4 base = make_float4(0.f, 0.f, 0.f, 0.f);
    if (active) base = *(const float4*)(a.base + o);
    const float s = a.dinv[l];
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t pb = p0; pb < p1; pb += LANES) {
      const int cnt = (int)min((int64_t)LANES, p1 - pb);
      int jj = 0;
      float ww = 0.0f;
      if (lane < cnt) {
        jj = __ldg(a.col + pb + lane);
        ww = (WEIGHTED ? __ldg(a.val + pb + lane) : 1.0f) * __ldg(a.dinv + jj);
      }
      int q = 0;
      for (; q + 8 <= cnt; q += 8) {
        float4 v[8];
        float w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int j = __shfl_sync(mask, jj, q + u, LANES);
          w[u] = __shfl_sync(mask, ww, q + u, LANES);
          if (active) v[u] = __ldg((const float4*)(X + (int64_t)j * a.kp + c));
        }
        if (active) {
#pragma unroll
          for (int u = 0; u < 8; ++u) fma4(acc, w[u], v[u]);
        }
      }
      for (; q < cnt; ++q) {
        const int j = __shfl_sync(mask, jj, q, LANES);
        const float w = __shfl_sync(mask, ww, q, LANES);
        if (active) fma4(acc, w, __ldg((const float4*)(X + (int64_t)j * a.kp + c)));
      }
    }
    if (!active) continue;
    *(float4*)(a.out + o) = make_float4(-fmaf(s, acc.x, base.x), -fmaf(s, acc.y, base.y),
                                        -fmaf(s, acc.z, base.z), -fmaf(s, acc.w, base.w));
  }
}

// Xh = D^-1/2 X (FP32), the gathered block of the exact AX product.
__global__ void k_scale_rows(int64_t n, int kp, const float* __restrict__ X, const float* __restrict__ dinv,
                             float* __restrict__ Xh, const Ctrl* ctrl, int ignore_done) {
  if (!ignore_done && ctrl->done) return;
  const int64_t total = n * kp / 4;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = i * 4;
    const float s = dinv[e / kp];
    const float4 x = *(const float4*)(X + e);
    *(float4*)(Xh + e) = make_float4(s * x.x, s * x.y, s * x.z, s * x.w);
  }
}

// Folds the per-block partials of diag(V^T AV) (pw: nw rows of kp) and of diag(V^T G) (pg: ng
// rows) into gridDim.x rows of out[r][2][kp]: row r sums the blocks [r nb / R, (r + 1) nb / R) of
// each source in order, so the result does not depend on scheduling.
struct DotsFoldArgs {
  const double* pw;
  const double* pg;
  double* out;
  const Ctrl* ctrl;
  int nw, ng, kp;
};

__device__ __forceinline__ void dots_fold_body(const DotsFoldArgs& a, const VBlock vb) {
  const double* __restrict__ pw = a.pw;
  const double* __restrict__ pg = a.pg;
  double* __restrict__ out = a.out;
  const int nw = a.nw, ng = a.ng, kp = a.kp;
  if (a.ctrl->done) return;
  // 2 kp <= blockDim.x columns; blockDim.x / (2 kp) lane groups split this block's rows and are
  // combined in group order
  __shared__ double red[256];
  const int r = vb.x, R = vb.gx, width = 2 * kp, groups = blockDim.x / width;
  const int t = threadIdx.x % width, l = threadIdx.x / width;
  if (l < groups) {
    const int which = t / kp, j = t % kp;
    const double* p = which ? pg : pw;
    const int nb = which ? ng : nw;
    const int b0 = (int)((int64_t)r * nb / R), b1 = (int)((int64_t)(r + 1) * nb / R);
    double sum = 0.0;
    for (int b = b0 + l; b < b1; b += groups) sum += p[(int64_t)b * kp + j];
    red[l * width + t] = sum;
  }
  __syncthreads();
  if (threadIdx.x < width) {
    double sum = 0.0;
    for (int g = 0; g < groups; ++g) sum += red[g * width + threadIdx.x];
    out[(int64_t)r * width + threadIdx.x] = sum;
  }
}

__global__ void k_dots_fold(const __grid_constant__ DotsFoldArgs a) { dots_fold_body(a, hw_block()); }

__global__ void k_dots_fold_g(const __grid_constant__ GroupParams<DotsFoldArgs> p) {
  VBlock vb;
  const DotsFoldArgs& a = group_find(p, &vb);
  dots_fold_body(a, vb);
}

// V_t = -G_t + V_{t-1} diag(beta) (V_0 = -G_0), stored as V_t diag(1 / s_t) (column scales s_t from
// k_beta: the FP32 coefficients are vinv = 1 / s_t and beta s_{t-1} / s_t), its gather copy
// Vh = D^-1/2 V_t (FP32 or BF16) and
// per-block partial sums of diag(V_t^T G_t), the derivative of every line-search polynomial at
// alpha = 0. LPN lanes cover a row (four columns each, fixed per thread), 256 / LPN rows per
// block step; each thread sums its columns over its rows, and the block adds its row groups in
// order in FP64 into dots_g[blockIdx.x][kp].
struct VpassArgs {
  int64_t n;
  const float* G;
  float* V;
  void* Vh;
  const float* dinv;
  const float* beta;
  const float* vinv;
  double* dots_g;
  Ctrl* ctrl;
  int kp, first;
};

template <int LPN, bool BF16>
__device__ __forceinline__ void vpass_body(const VpassArgs& a, const VBlock vb) {
  const int64_t n = a.n;
  const int kp = a.kp, first = a.first;
  const float* __restrict__ G = a.G;
  float* __restrict__ V = a.V;
  void* __restrict__ Vh = a.Vh;
  const float* __restrict__ dinv = a.dinv;
  const float* __restrict__ beta = a.beta;
  const float* __restrict__ vinv = a.vinv;
  double* __restrict__ dots_g = a.dots_g;
  if (a.ctrl->done) return;
  constexpr int RPB = 256 / LPN;
  constexpr int W = 4 * LPN;
  __shared__ float red[RPB * W];
  const int lane = threadIdx.x % LPN, rg = threadIdx.x / LPN;
  const int c = lane * 4;
  const bool active = c < kp;
  float4 b = make_float4(0.f, 0.f, 0.f, 0.f), acc = b, iv = make_float4(1.f, 1.f, 1.f, 1.f);
  if (active && !first) {
    b = *(const float4*)(beta + c);
    iv = *(const float4*)(vinv + c);  // powers of two: exact
  }
  if (active) {
    for (int64_t row = (int64_t)vb.x * RPB + rg; row < n; row += (int64_t)vb.gx * RPB) {
      const int64_t e = row * kp + c;
      const float4 g = *(const float4*)(G + e);
      float4 v = make_float4(-g.x * iv.x, -g.y * iv.y, -g.z * iv.z, -g.w * iv.w);
      if (!first) {
        const float4 vp = *(const float4*)(V + e);
        v.x = fmaf(b.x, vp.x, v.x);
        v.y = fmaf(b.y, vp.y, v.y);
        v.z = fmaf(b.z, vp.z, v.z);
        v.w = fmaf(b.w, vp.w, v.w);
      }
      *(float4*)(V + e) = v;
      acc.x = fmaf(v.x, g.x, acc.x);
      acc.y = fmaf(v.y, g.y, acc.y);
      acc.z = fmaf(v.z, g.z, acc.z);
      acc.w = fmaf(v.w, g.w, acc.w);
      const float s = dinv[row];
      if (BF16) {
        __nv_bfloat162 h0 = __floats2bfloat162_rn(s * v.x, s * v.y);
        __nv_bfloat162 h1 = __floats2bfloat162_rn(s * v.z, s * v.w);
        uint2 u;
        u.x = *reinterpret_cast<uint32_t*>(&h0);
        u.y = *reinterpret_cast<uint32_t*>(&h1);
        *(uint2*)((__nv_bfloat16*)Vh + e) = u;
      } else {
        *(float4*)((float*)Vh + e) = make_float4(s * v.x, s * v.y, s * v.z, s * v.w);
      }
    }
  }
  *(float4*)(red + rg * W + c) = acc;
  __syncthreads();
  for (int j = threadIdx.x; j < kp; j += blockDim.x) {
    double sum = 0.0;
    for (int r = 0; r < RPB; ++r) sum += (double)red[r * W + j];
    dots_g[(int64_t)vb.x * kp + j] = sum;
  }
}

template <int LPN, bool BF16>
__global__ void __launch_bounds__(256) k_vpass(const __grid_constant__ VpassArgs a) {
  vpass_body<LPN, BF16>(a, hw_block());
}

template <int LPN, bool BF16>
__global__ void __launch_bounds__(256) k_vpass_g(const __grid_constant__ GroupParams<VpassArgs> p) {
  VBlock vb;
  const VpassArgs& a = group_find(p, &vb);
  vpass_body<LPN, BF16>(a, vb);
}

// ------------------------------------------------------------------------------------------
// Direction pass: optional update, G = g(X), column sums for beta
// ------------------------------------------------------------------------------------------


// Warp-batched direction pass. A warp owns S = 32 / (KPMAX / 4) row slots of KPB rows each;
// lane q of a slot holds columns [4q, 4q + 4) of its rows in registers. The rows are staged in a
// warp-private shared buffer so every lane can read x_m (and y_m) as a broadcast, while the
// k x k block (triu-masked for TriOFM) stays resident in shared memory. All global loads of a
// batch are issued before any arithmetic, so each warp keeps up to 5 * KPB 16-byte loads in
// flight. Column sums (for beta and ||G||) go to per-block partials in a fixed order.
#ifndef OFSC_DIR_KPB
#define OFSC_DIR_KPB 8
#endif
#ifndef OFSC_DIR_MINB
#define OFSC_DIR_MINB 1
#endif
constexpr int kKPB = OFSC_DIR_KPB;  // rows per slot per batch
constexpr int kColSums = 6;  // column sums of the direction pass

template <int KPMAX, bool F2>
struct DirShape {
  static constexpr int LPR = KPMAX / 4;       // lanes per row
  static constexpr int S = 32 / LPR;          // row slots per warp
  static constexpr int ROWS = S * kKPB;       // rows per warp batch
  static constexpr int SSTR = kKPB * KPMAX + 4;  // floats per slot in the stage (bank offset)
  static constexpr int NSTAGE = F2 ? 2 : 1;
  static constexpr size_t kk_floats = (size_t)KPMAX * KPMAX * (F2 ? 2 : 1);
  static constexpr size_t stage_floats = (size_t)(kRowThreads / 32) * S * SSTR * NSTAGE;
  static constexpr size_t red_doubles = (size_t)(kRowThreads / 32) * S * kColSums * KPMAX;
  static constexpr size_t bytes() {
    return kk_floats * 4 + (stage_floats * 4 > red_doubles * 8 ? stage_floats * 4 : red_doubles * 8);
  }
};

template <int METHOD, int KPMAX>
__global__ void __launch_bounds__(kRowThreads, OFSC_DIR_MINB) k_direction(RowArgs a) {
#define OFSC_VB_X blockIdx.x
#define OFSC_VB_GX gridDim.x
#include "direction_body.inc"
#undef OFSC_VB_X
#undef OFSC_VB_GX
}

// The same pass for every graph of a batch in one launch (see group.cuh).
template <int METHOD, int KPMAX>
__global__ void __launch_bounds__(kRowThreads, OFSC_DIR_MINB) k_direction_g(const __grid_constant__ GroupParams<RowArgs> p) {
  VBlock vb;
  const RowArgs& a = group_find(p, &vb);
#define OFSC_VB_X ((unsigned)vb.x)
#define OFSC_VB_GX ((unsigned)vb.gx)
#include "direction_body.inc"
#undef OFSC_VB_X
#undef OFSC_VB_GX
}

// ------------------------------------------------------------------------------------------
// beta and the stop test (one block)
// ------------------------------------------------------------------------------------------

// Folds nb rows of width values into gridDim.x rows: row r sums the rows [r nb / R, (r + 1) nb / R)
// in order (a fixed shape, so the sums do not depend on scheduling).
struct FoldArgs {
  const double* part;
  double* out;
  const Ctrl* ctrl;
  int nb, width, ignore_done;
};

__device__ __forceinline__ void fold_rows_body(const FoldArgs& a, const VBlock vb) {
  const double* __restrict__ part = a.part;
  double* __restrict__ out = a.out;
  const int nb = a.nb, width = a.width;
  if (!a.ignore_done && a.ctrl->done) return;
  const int r = vb.x, R = vb.gx;
  const int b0 = (int)((int64_t)r * nb / R), b1 = (int)((int64_t)(r + 1) * nb / R);
  for (int t = threadIdx.x; t < width; t += blockDim.x) {
    double sum = 0.0;
#pragma unroll 8
    for (int b = b0; b < b1; ++b) sum += part[(int64_t)b * width + t];
    out[(int64_t)r * width + t] = sum;
  }
}

__global__ void k_fold_rows(const __grid_constant__ FoldArgs a) { fold_rows_body(a, hw_block()); }

__global__ void k_fold_rows_g(const __grid_constant__ GroupParams<FoldArgs> p) {
  VBlock vb;
  const FoldArgs& a = group_find(p, &vb);
  fold_rows_body(a, vb);
}

// stop_ok: this update's G came from an exact AX, so meeting tol may stop the run; on an update
// whose AX came from the recurrence, meeting tol only sets near_tol (the host then schedules an
// exact update), so a run never stops on a recurrence value.
// beta (FP32, for the V pass) is the stored-direction coefficient beta_true s_{t-1} / s_t with s the
// column scales (vscale, updated here in place; vinv = 1 / s_t); beta64 is Algorithm 2's beta.
// qprev: the Gram V_{t-1}^T V_{t-1} of the stored previous direction (its diagonal bounds |V_t|).
struct BetaArgs {
  const double* colpart;
  float* beta;
  double* beta64;
  double* dE;
  Ctrl* ctrl;
  double* vscale;
  float* vinv;
  const double* qprev;
  int nblk, kp, first, eval, stop_ok;
};

// One block (the grouped twin runs one block per problem).
__device__ __forceinline__ void beta_body(const BetaArgs& a) {
  const double* __restrict__ colpart = a.colpart;
  float* beta = a.beta;
  double* beta64 = a.beta64;
  double* dE = a.dE;
  Ctrl* ctrl = a.ctrl;
  double* vscale = a.vscale;
  float* vinv = a.vinv;
  const double* __restrict__ qprev = a.qprev;
  const int nblk = a.nblk, kp = a.kp, first = a.first, eval = a.eval, stop_ok = a.stop_ok;
  if (!eval && ctrl->done) return;
  __shared__ double sh[256];
  __shared__ double lanes[256 * kColSums];  // [lane group][kColSums][kp]
  const int j = threadIdx.x;
  // the blocks' rows are split over 256 / kp lane groups, then combined in group order
  {
    const int ng = 256 / kp, c = j % kp, l = j / kp;
    if (l < ng) {
      double acc[kColSums] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
      for (int b = l; b < nblk; b += ng) {
        const double* p = colpart + (int64_t)b * kColSums * kp;
#pragma unroll
        for (int q = 0; q < kColSums; ++q) acc[q] += p[q * kp + c];
      }
#pragma unroll
      for (int q = 0; q < kColSums; ++q) lanes[(l * kColSums + q) * kp + c] = acc[q];
    }
  }
  __syncthreads();
  // the lane groups in group order, one thread per (sum, column): spread over the warps, as an
  // FP64 add chain in one warp per column would hold one sub-partition's FP64 unit for all of it
  __shared__ double tot[kColSums * kMaxK];  // [kColSums][kp]
  for (int t = j; t < kColSums * kp; t += 256) {
    const int q = t / kp, c = t % kp;
    double acc = 0.0;
    for (int l = 0; l < 256 / kp; ++l) acc += lanes[(l * kColSums + q) * kp + c];
    tot[t] = acc;
  }
  __syncthreads();
  double gg = 0.0, num = 0.0, den = 0.0, gy = 0.0, vy = 0.0, vg = 0.0;
  if (j < kp) {
    gg = tot[j];
    num = tot[kp + j];
    den = tot[2 * kp + j];
    gy = tot[3 * kp + j];
    vy = tot[4 * kp + j];
    vg = tot[5 * kp + j];
  }
  sh[j] = gg;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (j < s) sh[j] += sh[j + s];
    __syncthreads();
  }
  const double gnorm = sqrt(sh[0]);
  if (eval) {
    if (j == 0) {
      ctrl->gnorm = gnorm;
      ctrl->rel = ctrl->g0 > 0.0 ? gnorm / ctrl->g0 : 0.0;
    }
    return;
  }
  __shared__ int stop;
  if (j == 0) {
    stop = 0;
    ctrl->gnorm = gnorm;
    if (!isfinite(gnorm)) {
      ctrl->status = OFSC_ERR_NONFINITE;
      stop = 1;
    } else if (first) {
      ctrl->g0 = gnorm;
      ctrl->rel = gnorm > 0.0 ? 1.0 : 0.0;
      if (gnorm == 0.0) {
        ctrl->converged = 1;
        stop = 1;
      } else if (ctrl->maxit <= 0) {
        stop = 1;
      }
    } else {
      const double rel = gnorm / ctrl->g0;
      ctrl->rel = rel;
      if (rel <= ctrl->tol && stop_ok) {
        ctrl->converged = 1;
        stop = 1;
      } else if (rel <= ctrl->tol) {
        ctrl->near_tol = 1;
        if (ctrl->it >= ctrl->maxit) stop = 1;
      } else if (ctrl->it >= ctrl->maxit) {
        stop = 1;
      }
    }
    if (stop) ctrl->done = 1;
  }
  __syncthreads();
  if (j < kp) {
    double b = 0.0;
    if (!first && den != 0.0) b = num / den;
    const double s_old = first ? 1.0 : vscale[j];
    // the optional restart (not in Algorithm 2): a column whose new direction would not descend,
    // -|g_j|^2 + beta_j v_prev,j^T g_j >= 0, takes beta_j = 0
    if (ctrl->restart && -gg + b * s_old * vg >= 0.0) b = 0.0;
    // column scale of V_t: |V_t,j| <= |G_t,j| + |beta_j| s_old |Vs_{t-1,j}| = mu; s_t = 1 while
    // mu <= 2^vscale_exp ||G_0||, else the power of two that brings the stored column back under it
    // (scaling by powers of two is exact, so the stored values carry the same bits of V)
    double s_new = 1.0, inv_s = 1.0;  // 1 / s_new, exact for a power of two (no FP64 division)
    if (!first) {
      const double mu = sqrt(gg) + fabs(b) * s_old * sqrt(fmax(qprev[(int64_t)j * kp + j], 0.0));
      const double ref = ldexp(ctrl->g0, ctrl->vscale_exp);
      if (mu > ref && ref > 0.0 && isfinite(mu)) {
        int e = 0;
        frexp(mu / ref, &e);  // mu / ref in [2^(e-1), 2^e)
        s_new = ldexp(1.0, e);
        inv_s = ldexp(1.0, -e);
      }
    }
    vscale[j] = s_new;
    vinv[j] = (float)inv_s;
    beta[j] = (float)(b * s_old * inv_s);
    beta64[j] = b;
    // diag(V_t^T AX_t) with V_t = -G_t + V_{t-1} diag(beta): -diag(G^T AX) + beta diag(V_prev^T AX)
    if (dE) dE[j] = first ? -gy : -gy + b * s_old * vy;
  }
}

__global__ void k_beta(const __grid_constant__ BetaArgs a) { beta_body(a); }

__global__ void k_beta_g(const __grid_constant__ GroupParams<BetaArgs> p) {
  VBlock vb;
  const BetaArgs& a = group_find(p, &vb);
  beta_body(a);
}

// ------------------------------------------------------------------------------------------
// Grams L^T R over all rows: per row-group partials with compensated FP32 accumulation
// ------------------------------------------------------------------------------------------

struct GramPairs {
  const float* L[kPairs];
  const float* R[kPairs];
  int slot[kPairs];  // output slot (G_R ... G_C)
};

struct GramArgs {
  int64_t n;
  int kp;
  int npairs;
  int nt;            // tiles per dimension
  int64_t rows_per_group;
  GramPairs pairs;
  double* part;      // [gridDim.y][kPairs][kp*kp]
  Ctrl* ctrl;
  int ignore_done;
};

template <int M>
struct VecT;
template <>
struct VecT<1> {
  using T = float;
  static __device__ __forceinline__ void get(const float* p, float* o) { o[0] = p[0]; }
};
template <>
struct VecT<2> {
  static __device__ __forceinline__ void get(const float* p, float* o) {
    float2 v = *(const float2*)p;
    o[0] = v.x;
    o[1] = v.y;
  }
};
template <>
struct VecT<4> {
  static __device__ __forceinline__ void get(const float* p, float* o) {
    float4 v = *(const float4*)p;
    o[0] = v.x;
    o[1] = v.y;
    o[2] = v.z;
    o[3] = v.w;
  }
};

// 256 threads as 16 x 16; tile T x T with T = 16 M; thread (tx, ty) owns rows ty*M.., cols tx*M..
// Each 32-row chunk is staged in shared memory; the next chunk's float4 loads are issued into
// registers before the current chunk's FMAs, so global latency overlaps the arithmetic.
template <int M>
__device__ __forceinline__ void gram_body(const GramArgs& a, const VBlock vb) {
  if (!a.ignore_done && a.ctrl->done) return;
  constexpr int T = 16 * M;
  constexpr int NV = kGramChunk * T / 4;          // float4 per operand per chunk
  constexpr int V4 = (NV + 255) / 256;            // per thread
  __shared__ __align__(16) float Ls[kGramChunk][T];
  __shared__ __align__(16) float Rs[kGramChunk][T];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int nt2 = a.nt * a.nt;
  const int pair = vb.x / nt2;
  const int tile = vb.x % nt2;
  const int i0 = (tile / a.nt) * T, j0 = (tile % a.nt) * T;
  const float* __restrict__ L = a.pairs.L[pair];
  const float* __restrict__ R = a.pairs.R[pair];
  const int64_t r0 = (int64_t)vb.y * a.rows_per_group;
  const int64_t r1 = min(a.n, r0 + a.rows_per_group);
  float s[M][M], cmp[M][M];
#pragma unroll
  for (int u = 0; u < M; ++u)
#pragma unroll
    for (int v = 0; v < M; ++v) s[u][v] = cmp[u][v] = 0.0f;
  float4 pl[V4], pr[V4];
  auto fetch = [&](int64_t rb) {
#pragma unroll
    for (int q = 0; q < V4; ++q) {
      const int i = (tid + q * 256) * 4;
      const int r = i / T, cc = i % T;
      const int64_t l = rb + r;
      const bool ok = l < r1 && (tid + q * 256) < NV;
      pl[q] = (ok && i0 + cc < a.kp) ? *(const float4*)(L + l * a.kp + i0 + cc) : make_float4(0.f, 0.f, 0.f, 0.f);
      pr[q] = (ok && j0 + cc < a.kp) ? *(const float4*)(R + l * a.kp + j0 + cc) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  if (r0 < r1) fetch(r0);
  for (int64_t rb = r0; rb < r1; rb += kGramChunk) {
#pragma unroll
    for (int q = 0; q < V4; ++q) {
      const int i = (tid + q * 256) * 4;
      if (tid + q * 256 < NV) {
        *(float4*)(&Ls[i / T][i % T]) = pl[q];
        *(float4*)(&Rs[i / T][i % T]) = pr[q];
      }
    }
    __syncthreads();
    if (rb + kGramChunk < r1) fetch(rb + kGramChunk);
    float acc[M][M];
#pragma unroll
    for (int u = 0; u < M; ++u)
#pragma unroll
      for (int v = 0; v < M; ++v) acc[u][v] = 0.0f;
#pragma unroll 8
    for (int r = 0; r < kGramChunk; ++r) {
      float av[M], bv[M];
      VecT<M>::get(&Ls[r][ty * M], av);
      VecT<M>::get(&Rs[r][tx * M], bv);
#pragma unroll
      for (int u = 0; u < M; ++u)
#pragma unroll
        for (int v = 0; v < M; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
    // Kahan-compensated running sum of the chunk partials
#pragma unroll
    for (int u = 0; u < M; ++u)
#pragma unroll
      for (int v = 0; v < M; ++v) {
        const float y = acc[u][v] - cmp[u][v];
        const float t = s[u][v] + y;
        cmp[u][v] = (t - s[u][v]) - y;
        s[u][v] = t;
      }
    __syncthreads();
  }
  double* out = a.part + ((int64_t)vb.y * kPairs + a.pairs.slot[pair]) * a.kp * a.kp;
#pragma unroll
  for (int u = 0; u < M; ++u)
#pragma unroll
    for (int v = 0; v < M; ++v) {
      const int i = i0 + ty * M + u, j = j0 + tx * M + v;
      if (i < a.kp && j < a.kp) out[i * a.kp + j] = (double)s[u][v] - (double)cmp[u][v];
    }
}

template <int M>
__global__ void __launch_bounds__(256) k_gram(const __grid_constant__ GramArgs a) { gram_body<M>(a, hw_block()); }

template <int M>
__global__ void __launch_bounds__(256) k_gram_g(const __grid_constant__ GroupParams<GramArgs> p) {
  VBlock vb;
  const GramArgs& a = group_find(p, &vb);
  gram_body<M>(a, vb);
}

// Blocks of 32 consecutive entries (one slot each, as kp^2 is a multiple of 64): warp w sums the
// row groups w, w + 8, ... (coalesced, one entry per lane); the eight warp sums are added in warp
// order.
struct GramReduceArgs {
  const double* part;
  double* gram;
  Ctrl* ctrl;
  int gy, kp, slot_mask, ignore_done;
};

__device__ __forceinline__ void gram_reduce_body(const GramReduceArgs& a, const VBlock vb) {
  const double* __restrict__ part = a.part;
  double* __restrict__ gram = a.gram;
  const int gy = a.gy, kp = a.kp, slot_mask = a.slot_mask;
  if (!a.ignore_done && a.ctrl->done) return;
  __shared__ double ws[8][32];
  const int kk = kp * kp, lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int base = vb.x * 32; base < kPairs * kk; base += vb.gx * 32) {
    if (!((slot_mask >> (base / kk)) & 1)) continue;  // uniform over the block
    const int i = base + lane;
    double s = 0.0;
    for (int b = warp; b < gy; b += 8) s += part[(int64_t)b * kPairs * kk + i];
    ws[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
      double t = 0.0;
      for (int w = 0; w < 8; ++w) t += ws[w][lane];
      gram[i] = t;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256) k_gram_reduce(const __grid_constant__ GramReduceArgs a) {
  gram_reduce_body(a, hw_block());
}

__global__ void __launch_bounds__(256) k_gram_reduce_g(const __grid_constant__ GroupParams<GramReduceArgs> p) {
  VBlock vb;
  const GramReduceArgs& a = group_find(p, &vb);
  gram_reduce_body(a, vb);
}

// ------------------------------------------------------------------------------------------
// FP64 line search (one block): cubic coefficients, real roots, alpha, next X^T X and X^T AX
// ------------------------------------------------------------------------------------------


// Sum over the 256 threads of each of NV <= 16 values, every thread receiving the totals. Value
// q is summed by warp q mod 8: lane l adds the values of threads l, l + 32, ..., l + 224 in that
// order, then the lanes are added pairwise (offsets 16, 8, 4, 2, 1). A fixed order, so the sums
// repeat bit for bit. On GB300 an FP64 warp instruction occupies its sub-partition's FP64 unit for
// tens of cycles, so the cost is the number of FP64 instructions on the busiest sub-partition:
// about 3,800 cycles for 15 values, against 14,000 for a pairwise tree over the threads, whose
// last levels run in one warp.
template <int NV>
__device__ void block_sum(double (&v)[NV], double* sh) {
  static_assert(NV <= 16, "two values per warp");
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int q = 0; q < NV; ++q) sh[q * 256 + tid] = v[q];
  __syncthreads();
  double t[2] = {0.0, 0.0};
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int q = w + 8 * u;
    if (q < NV) {
      double s = sh[q * 256 + lane];
#pragma unroll
      for (int i = 1; i < 8; ++i) s += sh[q * 256 + lane + 32 * i];
      t[u] = s;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (w + 8 * u < NV) t[u] += __shfl_down_sync(0xffffffffu, t[u], off);
  __syncthreads();  // every thread has read its rows before the totals are written over them
  if (lane == 0) {
#pragma unroll
    for (int u = 0; u < 2; ++u)
      if (w + 8 * u < NV) sh[(w + 8 * u) * 256] = t[u];
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NV; ++q) v[q] = sh[q * 256];
  __syncthreads();
}

constexpr int kSolveBlocks = 128;  // most blocks of the trace and update passes (>= kMaxK)

// Blocks of the trace and update passes: one per 256 k x k entries, at least 8.
inline int solve_blocks(int kp) { return std::max(8, std::min(kSolveBlocks, (kp * kp + 255) / 256)); }
constexpr int kSolveSums = 16;     // per-block partial sums of the trace pass

struct SolveArgs {
  const double* gram;  // [6][kp*kp]: V^T X (P), V^T V (Q); f2 methods also V^T AX (E), V^T AV (C)
  const double* dots;  // [dots_blocks][2][kp] partials of diag(V^T AV), diag(V^T G)
  int dots_blocks;
  const double* dE;    // f1 methods: diag(V^T AX) from the direction pass and beta (objective only)
  double* R64;         // X^T X of X_t on entry, of X_{t+1} on exit
  double* B64;         // X^T A X likewise (f2 methods)
  int kp;
  int k;
  int method;
  float* Rn;
  float* Bn;
  float* alpha;
  double* alpha64;
  const double* beta64;
  double* trace;
  Ctrl* ctrl;
  double alpha0;  // > 0: fixed step for update 0 instead of the line search
  double* part;   // scratch: [kSolveBlocks][kSolveSums] trace partials, [kp][4] diagonals, [kp][4] cubics
  int tblocks;    // blocks of the trace pass (rows of trace partials)
  const double* vscale;  // column scales s of the stored V: the Grams and dots are of V diag(1/s)
};

// C = V^T A V and B = X^T A X are symmetric; the recurrences leave rounding asymmetry.
#define SYM(M, i, j) (0.5 * ((M)[(i) * kp + (j)] + (M)[(j) * kp + (i)]))
// The Grams of the stored direction Vs = V diag(1/s) scaled back to V (row index = column of V):
// P = V^T X, E = V^T AX carry s_i; Q = V^T V, C = V^T AV carry s_i s_j (s = 1: the stored values).
#define PS(i, j) (sc[i] * P[(i) * kp + (j)])
#define ES(i, j) (sc[i] * E[(i) * kp + (j)])
#define QS(i, j) (sc[i] * sc[j] * Q[(i) * kp + (j)])
#define CS(i, j) (sc[i] * sc[j] * SYM(C, i, j))

// Line search, pass 1 of 3 (nb = solve_blocks(kp) blocks). Block b: the diagonals diag(V^T AV), diag(V^T AX)
// and diag(V^T G) of columns b, b + nb, ...; for TriOFM their cubics alone (Eqs. (16)/(18) before the
// prefix sum); and its slice of the k x k traces that make up f(X_t) and the OFM cubic (Eq. (15)).
// Per-block partial sums go to a.part in a fixed order. Partial layout (v[0..14]):
//   v[0..2]   tr B, ||R||_F^2, tr(R B)                         (objective)
//   v[3..8]   tr(QQ), tr(QP), tr(PP), tr(PP^T), tr(QR), tr(PR)  (OFM-f1 cubic)
//   v[3..13]  tr(QC) ... tr(RE), tr C, tr E                     (OFM-f2 cubic)
__device__ __forceinline__ void solve_traces_body(const SolveArgs& a, const VBlock vb) {
  if (a.ctrl->done) return;
  __shared__ double sh[15 * 256];
  const int kp = a.kp, kk = kp * kp, tid = threadIdx.x, b = vb.x, nb = vb.gx;
  const bool f2 = is_f2(a.method), tri = is_tri(a.method);
  const double* P = a.gram + G_P * kk;
  const double* Q = a.gram + G_Q * kk;
  const double* E = a.gram + G_E * kk;
  const double* C = a.gram + G_C * kk;
  const double* R = a.R64;
  const double* B = a.B64;
  const double* sc = a.vscale;
  double* diag = a.part + kSolveBlocks * kSolveSums;  // [kp][4]: dC, dE, dG
  double* coef = diag + 4 * kp;                       // [kp][4]: cubic of column j alone
  for (int j = b; j < kp; j += nb) {
    double s2[2] = {0.0, 0.0};
    for (int r = tid; r < a.dots_blocks; r += 256) {
      s2[0] += a.dots[(int64_t)r * 2 * kp + j];
      s2[1] += a.dots[(int64_t)r * 2 * kp + kp + j];
    }
    block_sum<2>(s2, sh);
    // The constant term of every cubic is the derivative along V at alpha = 0, i.e. diag(V^T G)
    // (with the 1/4 of Eq. (15) for OFM-f1): summing v.g directly avoids the cancellation in
    // tr(V^T AX) + tr(V^T X X^T X) near a fixed point, where AX = -X X^T X.
    const double dC = f2 ? CS(j, j) : sc[j] * sc[j] * s2[0];
    const double dE = f2 ? ES(j, j) : a.dE[j];
    const double dG = sc[j] * s2[1];
    if (tid == 0) {
      diag[4 * j + 0] = dC;
      diag[4 * j + 1] = dE;
      diag[4 * j + 2] = dG;
    }
    if (tri) {
      // Column j of g(X + aV) depends on columns 1..j only, so its term of the prefix cubic is
      // v_j^T g(X + aV)_j, a sum over m <= j of products of two polynomials in a.
      double d[3] = {0.0, 0.0, 0.0};  // a^1, a^2, a^3
      for (int m = tid; m <= j; m += 256) {
        if (a.method == M_TRI_F1) {
          // (P_jm + a Q_jm)(R_mj + a (P_jm + P_mj) + a^2 Q_mj)
          const double x0 = PS(j, m), x1 = QS(j, m);
          const double y0 = R[m * kp + j], y1 = PS(j, m) + PS(m, j), y2 = QS(m, j);
          d[0] += x0 * y1 + x1 * y0;
          d[1] += x0 * y2 + x1 * y1;
          d[2] += x1 * y2;
        } else {
          // -(E_jm + a C_jm)(R_mj + a (P_jm + P_mj) + a^2 Q_mj)
          const double x0 = ES(j, m), x1 = CS(j, m);
          const double y0 = R[m * kp + j], y1 = PS(j, m) + PS(m, j), y2 = QS(m, j);
          // -(P_jm + a Q_jm)(B_mj + a (E_jm + E_mj) + a^2 C_mj)
          const double u0 = PS(j, m), u1 = QS(j, m);
          const double w0 = SYM(B, m, j), w1 = ES(j, m) + ES(m, j), w2 = CS(m, j);
          d[0] -= x0 * y1 + x1 * y0 + u0 * w1 + u1 * w0;
          d[1] -= x0 * y2 + x1 * y1 + u0 * w2 + u1 * w1;
          d[2] -= x1 * y2 + u1 * w2;
        }
      }
      block_sum<3>(d, sh);
      if (tid == 0) {
        coef[4 * j + 0] = d[2];
        coef[4 * j + 1] = d[1];
        coef[4 * j + 2] = d[0] + (a.method == M_TRI_F1 ? dC : 2.0 * dC);
        coef[4 * j + 3] = dG;  // v_j^T g_j at a = 0
      }
    }
  }
  double v[15];
#pragma unroll
  for (int q = 0; q < 15; ++q) v[q] = 0.0;
  for (int i = b * 256 + tid; i < kk; i += nb * 256) {
    const int r = i / kp, c = i % kp, it = c * kp + r;
    const double rr = R[i];
    v[1] += rr * rr;
    if (f2) {
      v[2] += rr * SYM(B, c, r);
      if (r == c) v[0] += B[i];
    }
    if (tri) continue;
    const double q = QS(r, c), p = PS(r, c);
    if (a.method == M_OFM_F1) {
      const double pt = PS(c, r);
      v[3] += q * QS(c, r);
      v[4] += q * pt;
      v[5] += p * pt;
      v[6] += p * p;
      v[7] += q * R[it];
      v[8] += p * R[it];
    } else {
      const double e = ES(r, c), et = ES(c, r), cji = CS(c, r), bji = SYM(B, c, r);
      v[3] += q * cji;      // tr(Q C)
      v[4] += p * cji;      // tr(P C)
      v[5] += q * et;       // tr(Q E)
      v[6] += p * e;        // tr(P E^T)
      v[7] += p * et;       // tr(P E)
      v[8] += q * bji;      // tr(Q B)
      v[9] += rr * cji;     // tr(R C)
      v[10] += p * bji;     // tr(P B)
      v[11] += rr * et;     // tr(R E)
      if (r == c) {
        v[12] += CS(r, r);
        v[13] += e;
      }
    }
  }
  block_sum<15>(v, sh);
  if (tid == 0) {
#pragma unroll
    for (int q = 0; q < 15; ++q) a.part[b * kSolveSums + q] = v[q];
  }
}

__global__ void __launch_bounds__(256) k_solve_traces(const __grid_constant__ SolveArgs a) { solve_traces_body(a, hw_block()); }

__global__ void __launch_bounds__(256) k_solve_traces_g(const __grid_constant__ GroupParams<SolveArgs> p) {
  VBlock vb;
  const SolveArgs& a = group_find(p, &vb);
  solve_traces_body(a, vb);
}

// Line search, pass 2 of 3 (one block): f(X_t), the cubic coefficients and their roots, i.e. the
// step(s) alpha, written to a.alpha / a.alpha64; also the objective, the trace record and the
// running tr(X^T AX) of the f1 methods.
__device__ __forceinline__ void solve_body(const SolveArgs& a, const VBlock vb) {
  if (a.ctrl->done) return;
  __shared__ double sh[15 * 256];
  __shared__ double coef[kMaxK][4];
  __shared__ double al[kMaxK];
  __shared__ int bad;
  const int kp = a.kp, k = a.k, tid = threadIdx.x;
  const bool f2 = is_f2(a.method);
  const double* diag = a.part + kSolveBlocks * kSolveSums;
  if (tid == 0) bad = 0;
  double v[15];
#pragma unroll
  for (int q = 0; q < 15; ++q) v[q] = tid < a.tblocks ? a.part[tid * kSolveSums + q] : 0.0;
  if (tid < kp) {
    if (f2) {
      v[14] += diag[4 * tid + 2];  // tr(V^T G)
    } else {
      v[9] += diag[4 * tid + 0];   // tr(V^T AV)
      v[10] += diag[4 * tid + 2];  // tr(V^T G)
    }
  }
  block_sum<15>(v, sh);  // also orders bad = 0 before its use
  // objective at X_t: f1 = ||A||^2 + 2 tr B + ||R||^2, f2 = 2 tr B - tr(R B)
  const double trB = f2 ? v[0] : a.ctrl->trB;
  const double f = f2 ? 2.0 * trB - v[2] : a.ctrl->normA2 + 2.0 * trB + v[1];

  if (!is_tri(a.method)) {
    double c3, c2, c1, c0;
    if (a.method == M_OFM_F1) {
      // (1/4) d/dalpha f1(X + alpha V) = tr(V^T A (X + aV)) + tr(V^T Z Z^T Z), Z = X + aV
      c3 = v[3];
      c2 = 3.0 * v[4];
      c1 = v[9] + v[5] + v[6] + v[7];
      c0 = 0.25 * v[10];  // = tr(E) + tr(P R) with G = grad f1 = 4 (AX + X X^T X)
    } else {
      // d/dalpha f2 = tr(V^T (4 A Z - 2 Z Z^T A Z - 2 A Z Z^T Z)), Z = X + aV
      c3 = -4.0 * v[3];
      c2 = -6.0 * (v[4] + v[5]);
      c1 = 2.0 * (2.0 * v[12] - 2.0 * v[6] - 2.0 * v[7] - v[8] - v[9]);
      c0 = v[14];  // = 2 tr(2E - P B - R E) = tr(V^T grad f2)
    }
    // warp 0 solves the cubic, its three real roots (if it has three) in lanes 0-2 at once (FP64
    // issue is scarce: 8 warps solving it would cost 8x)
    if (tid < 32) {
      int b = 0;
      const double st = pick_step_warp(c3, c2, c1, c0, &b);
      if (tid == 0) {
        bad |= b;
        al[0] = st;
      }
    }
    __syncthreads();
    const double st = al[0];
    __syncthreads();
    for (int j = tid; j < kp; j += 256) al[j] = j < k ? st : 0.0;
  } else {
    // prefix sums over columns of the per-column cubics (Hillis-Steele, kp <= 256 threads)
    const double* cg = diag + 4 * kp;
    if (tid < kp)
      for (int q = 0; q < 4; ++q) coef[tid][q] = cg[4 * tid + q];
    __syncthreads();
    for (int off = 1; off < kp; off <<= 1) {
      double t4[4] = {0.0, 0.0, 0.0, 0.0};
      if (tid < kp && tid >= off)
        for (int q = 0; q < 4; ++q) t4[q] = coef[tid - off][q];
      __syncthreads();
      if (tid < kp)
        for (int q = 0; q < 4; ++q) coef[tid][q] += t4[q];
      __syncthreads();
    }
    if (tid < kp) {
      int b = 0;
      al[tid] = tid < k ? pick_step(coef[tid][0], coef[tid][1], coef[tid][2], coef[tid][3], &b) : 0.0;
      if (b) bad = 1;
    }
  }
  __syncthreads();
  if (a.alpha0 > 0.0 && a.ctrl->it == 0) {
    for (int j = tid; j < kp; j += 256) al[j] = j < k ? a.alpha0 : 0.0;
    __syncthreads();
  }
  for (int j = tid; j < kp; j += 256) {
    a.alpha[j] = (float)(al[j] * a.vscale[j]);  // the step along the stored direction V diag(1/s)
    a.alpha64[j] = al[j];
  }
  if (!f2) {  // tr(X'^T AX') = tr B + 2 sum al_j E_jj + sum al_j^2 C_jj
    double t1[1] = {0.0};
    for (int j = tid; j < kp; j += 256) t1[0] += 2.0 * al[j] * diag[4 * j + 1] + al[j] * al[j] * diag[4 * j + 0];
    block_sum<1>(t1, sh);
    if (tid == 0) a.ctrl->trB = trB + t1[0];
  }
  const int t = a.ctrl->it;
  if (a.trace && t < a.ctrl->trace_cap) {
    double* rec = a.trace + (int64_t)t * (3 + 2 * k);
    if (tid == 0) {
      rec[0] = t;
      rec[1] = a.ctrl->rel;
      rec[2] = f;
    }
    for (int j = tid; j < k; j += 256) {
      rec[3 + j] = al[j];
      rec[3 + k + j] = a.beta64[j];
    }
  }
  __syncthreads();
  if (tid == 0) {
    a.ctrl->f = f;
    if (bad) {
      a.ctrl->status = OFSC_ERR_NONFINITE;
      a.ctrl->done = 1;
    }
  }
}

__global__ void __launch_bounds__(256) k_solve(const __grid_constant__ SolveArgs a) { solve_body(a, hw_block()); }

__global__ void __launch_bounds__(256) k_solve_g(const __grid_constant__ GroupParams<SolveArgs> p) {
  VBlock vb;
  const SolveArgs& a = group_find(p, &vb);
  solve_body(a, vb);
}

// Line search, pass 3 of 3 (solve_blocks(kp) blocks): X' = X + V diag(al), AX' = AX + AV diag(al) give
//   X'^T X'  = R + diag(al) P + P^T diag(al) + diag(al) Q diag(al)
//   X'^T AX' = B + E^T diag(al) + diag(al) E + diag(al) C diag(al)
// element by element in FP64 (each element read and written by one thread, so in place).
__device__ __forceinline__ void solve_update_body(const SolveArgs& a, const VBlock vb) {
  if (a.ctrl->done) return;
  __shared__ double al[kMaxK];
  const int kp = a.kp, kk = kp * kp, tid = threadIdx.x;
  const bool f2 = is_f2(a.method);
  const double* P = a.gram + G_P * kk;
  const double* Q = a.gram + G_Q * kk;
  const double* E = a.gram + G_E * kk;
  const double* C = a.gram + G_C * kk;
  const double* sc = a.vscale;
  for (int j = tid; j < kp; j += 256) al[j] = a.alpha64[j];
  __syncthreads();
  for (int i = vb.x * 256 + tid; i < kk; i += vb.gx * 256) {
    const int r = i / kp, c = i % kp;
    const double ar = al[r], ac = al[c];
    const double rn = a.R64[i] + ar * PS(r, c) + PS(c, r) * ac + ar * QS(r, c) * ac;
    a.R64[i] = rn;
    a.Rn[i] = (float)rn;
    if (f2) {
      const double bn = a.B64[i] + ES(c, r) * ac + ar * ES(r, c) + ar * CS(r, c) * ac;
      a.B64[i] = bn;
      a.Bn[i] = (float)bn;
    }
  }
}

__global__ void __launch_bounds__(256) k_solve_update(const __grid_constant__ SolveArgs a) { solve_update_body(a, hw_block()); }

__global__ void __launch_bounds__(256) k_solve_update_g(const __grid_constant__ GroupParams<SolveArgs> p) {
  VBlock vb;
  const SolveArgs& a = group_find(p, &vb);
  solve_update_body(a, vb);
}
#undef SYM
#undef PS
#undef ES
#undef QS
#undef CS

// Exact refresh: X^T X and X^T AX of the current X from their Grams; objective of X.
__global__ void k_set_rb(const double* __restrict__ gram, int kp, int objective, float* Rn, float* Bn,
                         double* R64, double* B64, Ctrl* ctrl, int ignore_done) {
  if (!ignore_done && ctrl->done) return;
  __shared__ double sh[3 * 256];
  const int kk = kp * kp, tid = threadIdx.x;
  const double* R = gram + G_R * kk;
  const double* B = gram + G_B * kk;
  double fv[3] = {0.0, 0.0, 0.0};
  for (int i = tid; i < kk; i += 256) {
    const int r = i / kp, c = i % kp;
    const double b = 0.5 * (B[i] + B[c * kp + r]);
    Rn[i] = (float)R[i];
    Bn[i] = (float)b;
    if (R64) {
      R64[i] = R[i];
      B64[i] = b;
    }
    fv[1] += R[i] * R[i];
    fv[2] += R[i] * b;
    if (r == c) fv[0] += B[i];
  }
  block_sum<3>(fv, sh);
  if (tid == 0) {
    ctrl->trB = fv[0];
    ctrl->f = objective == 2 ? 2.0 * fv[0] - fv[2] : ctrl->normA2 + 2.0 * fv[0] + fv[1];
  }
}

}  // namespace
}  // namespace ofsc

// ==========================================================================================
// Host side
// ==========================================================================================

namespace ofsc {
namespace {

constexpr int kGramTargetBlocks = 4 * kNumSMs;

thread_local int64_t g_launches = 0;  // kernels launched by the current call on this thread

// The direction product, counted among the call's launches; slots > 0: a tuned shape.
int spmm_dir(const SpmmArgs& a, bool weighted, bool bf16, int slots, cudaStream_t s) {
  g_launches += a.mp ? 2 : 1;  // the merge-path form adds the fixup of split rows
  return launch_spmm_dir(a, weighted, bf16, slots, s);
}

// Checked builds: a recorded out-of-range access of the direction product makes the call fail
// (its results are not meaningful), whatever else it returned; release builds return st.
ofsc_status bounds_checked(ofsc_status st, const char* who) {
  unsigned long long code = 0;
  const cudaError_t e = spmm_dir_take_bounds(&code);
  if (e != cudaSuccess) return cuda_fail(e, "bounds check");
  if (code == 0) return st;
  const unsigned kind = (unsigned)(code >> 60);
  long long v = (long long)(code & ((1ull << 60) - 1));
  if (v & (1ll << 59)) v -= (1ll << 60);  // sign of a negative column index
  return fail(OFSC_ERR_INVALID_ARG, "%s: bounds check: %s %lld", who,
              kind == 1 ? "column index outside [0, n):" : "row or nonzero range outside the CSR, warp", v);
}

// Whether the direction product runs on the merge-path shares: forced on or off by `setting`
// (> 0, < 0); else the form ofsc_autotune timed faster for this padded width and gather storage;
// else on graphs of at least 2^23 stored entries, where equal shares of rows + nonzeros balance
// the rows' epilogues as well as the gathers and the fixup's launch is negligible (2M-node
// DC-SBM, 60.6M entries: 2.26 -> 2.12 ms per BF16 product); else when the longest row holds at
// least 1024 nonzeros and more than four warps' shares (the warp that takes it whole then runs a
// chain of at least 128 dependent gather steps, several times as long as the other warps').
bool use_merge_path(const ofsc_graph* g, int setting, int kp, bool bf16) {
  if (g->mp == nullptr || g->nnz <= 0 || g->groups[kRowPart] <= 0) return false;
  if (setting != 0) return setting > 0;
  if (g->dir_mp != 0 && g->dir_tuned_kp == kp && g->dir_tuned_bf16 == (bf16 ? 1 : 0)) return g->dir_mp > 0;
  if (g->nnz >= (int64_t(1) << 23)) return true;
  return g->max_row >= 1024 && g->max_row * g->groups[kRowPart] > 4 * g->nnz;
}

// The gathers in flight per lane that ofsc_autotune chose for this padded width and gather storage
// (0, the kernel's default, for any other).
int tuned_slots(const ofsc_graph* g, int kp, bool bf16) {
  return (g->dir_tuned_kp == kp && g->dir_tuned_bf16 == (bf16 ? 1 : 0)) ? g->dir_slots : 0;
}

int gram_m_for(int kp) { return kp <= 16 ? 1 : kp <= 32 ? 2 : 4; }
int gram_nt_for(int kp) { return (int)ceil_div(kp, 16 * gram_m_for(kp)); }

// Row groups of a Gram launch with `npairs` pairs: about kGramTargetBlocks blocks in total.
int64_t gram_rows_per_group(int64_t n, int kp, int npairs, int* gy) {
  const int nt = gram_nt_for(kp);
  int64_t want = ceil_div(kGramTargetBlocks, (int64_t)npairs * nt * nt);
  int64_t maxg = ceil_div(n > 0 ? n : 1, kGramChunk);
  if (want > maxg) want = maxg;
  if (want < 1) want = 1;
  int64_t rpg = ceil_div(n > 0 ? n : 1, want);
  rpg = ceil_div(rpg, kGramChunk) * kGramChunk;
  *gy = (int)ceil_div(n > 0 ? n : 1, rpg);
  return rpg;
}

// Optional per-phase device timing: CUDA events around launches on the call's stream.
struct Prof {
  Workspace& ws;
  ofsc_profile* out;
  cudaStream_t s;
  size_t used = 0;
  std::vector<int> phases;
  cudaEvent_t next() {
    if (used == ws.events.size()) {
      cudaEvent_t e = nullptr;
      cudaEventCreate(&e);
      ws.events.push_back(e);
    }
    return ws.events[used++];
  }
  void begin(int ph) {
    if (!out) return;
    phases.push_back(ph);
    cudaEventRecord(next(), s);
  }
  void end() {
    if (out) cudaEventRecord(next(), s);
  }
  // Adds the recorded intervals to `out` (waits for the last event) and recycles the events.
  void collect() {
    if (!out || phases.empty()) return;
    cudaEventSynchronize(ws.events[used - 1]);
    for (size_t i = 0; i < phases.size(); ++i) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, ws.events[2 * i], ws.events[2 * i + 1]) == cudaSuccess) {
        out->ms[phases[i]] += ms;
        out->launches[phases[i]] += 1;
      }
    }
    phases.clear();
    used = 0;
  }
};

template <int LANES>
void launch_spmm_l(const SpmmArgs& a, bool weighted, cudaStream_t s) {
  ++g_launches;
  const int grid = a.groups / (256 / LANES);
  if (weighted) k_spmm<LANES, true><<<grid, 256, 0, s>>>(a);
  else k_spmm<LANES, false><<<grid, 256, 0, s>>>(a);
}

// AX for the row block in a.gather (= a.base), on the lane-group partition of a.kp.
void launch_spmm(const SpmmArgs& a, bool weighted, cudaStream_t s) {
  if (a.n <= 0) return;
  switch (spmm_lanes(a.kp)) {
    case 2: launch_spmm_l<2>(a, weighted, s); break;
    case 4: launch_spmm_l<4>(a, weighted, s); break;
    case 8: launch_spmm_l<8>(a, weighted, s); break;
    case 16: launch_spmm_l<16>(a, weighted, s); break;
    default: launch_spmm_l<32>(a, weighted, s); break;
  }
}

void launch_vpass(int lpn, bool bf16, int grid, cudaStream_t s, int64_t n, int kp, const float* G, float* V, void* Vh,
                  const float* dinv, const float* beta, const float* vinv, int first, double* dots_g, Ctrl* ctrl) {
  VpassArgs a{};
  a.n = n;
  a.kp = kp;
  a.G = G;
  a.V = V;
  a.Vh = Vh;
  a.dinv = dinv;
  a.beta = beta;
  a.vinv = vinv;
  a.first = first;
  a.dots_g = dots_g;
  a.ctrl = ctrl;
#define OFSC_VPASS(L)                                                       \
  case L:                                                                  \
    if (bf16) {                                                            \
      OFSC_GROUPABLE((k_vpass<L, true>), (k_vpass_g<L, true>), VpassArgs);   \
      k_vpass<L, true><<<grid, 256, 0, s>>>(a);                             \
    } else {                                                               \
      OFSC_GROUPABLE((k_vpass<L, false>), (k_vpass_g<L, false>), VpassArgs); \
      k_vpass<L, false><<<grid, 256, 0, s>>>(a);                            \
    }                                                                      \
    break;
  switch (lpn) {
    OFSC_VPASS(2)
    OFSC_VPASS(4)
    OFSC_VPASS(8)
    OFSC_VPASS(16)
    default:
      OFSC_VPASS(32)
  }
#undef OFSC_VPASS
}

int kpmax_for(int kp) { return kp <= 16 ? 16 : kp <= 32 ? 32 : kp <= 64 ? 64 : 128; }

template <int METHOD, int KPMAX>
cudaError_t launch_direction_t(const RowArgs& a, cudaStream_t s, int* nblk_out) {
  using Sh = DirShape<KPMAX, (METHOD >= M_OFM_F2)>;
  static int blocks_per_sm = 0;
  const size_t smem = Sh::bytes();
  if (blocks_per_sm == 0) {
    cudaError_t e = cudaFuncSetAttribute(k_direction<METHOD, KPMAX>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_direction<METHOD, KPMAX>, kRowThreads, smem);
    if (e != cudaSuccess) return e;
    blocks_per_sm = nb > 0 ? nb : 1;
  }
  const int64_t warps_needed = ceil_div(a.n, (int64_t)Sh::ROWS);
  int grid = (int)std::min<int64_t>(ceil_div(warps_needed, kRowThreads / 32), (int64_t)blocks_per_sm * kNumSMs);
  if (grid > kMaxRowBlocks) grid = kMaxRowBlocks;
  if (grid < 1) grid = 1;
  OFSC_GROUPABLE((k_direction<METHOD, KPMAX>), (k_direction_g<METHOD, KPMAX>), RowArgs);
  k_direction<METHOD, KPMAX><<<grid, kRowThreads, smem, s>>>(a);
  ++g_launches;
  *nblk_out = grid;
  return cudaGetLastError();
}

template <int METHOD>
cudaError_t launch_direction_m(const RowArgs& a, cudaStream_t s, int* nblk) {
  switch (kpmax_for(a.kp)) {
    case 16: return launch_direction_t<METHOD, 16>(a, s, nblk);
    case 32: return launch_direction_t<METHOD, 32>(a, s, nblk);
    case 64: return launch_direction_t<METHOD, 64>(a, s, nblk);
    default: return launch_direction_t<METHOD, 128>(a, s, nblk);
  }
}

cudaError_t launch_rowpass(int method, const RowArgs& a, cudaStream_t s, int* nblk) {
  switch (method) {
    case M_OFM_F1: return launch_direction_m<M_OFM_F1>(a, s, nblk);
    case M_TRI_F1: return launch_direction_m<M_TRI_F1>(a, s, nblk);
    case M_OFM_F2: return launch_direction_m<M_OFM_F2>(a, s, nblk);
    default: return launch_direction_m<M_TRI_F2>(a, s, nblk);
  }
}

cudaError_t launch_gram(Workspace& ws, const GramPairs& pairs, int npairs, int slot_mask,
                        int ignore_done, cudaStream_t s, Prof* prof = nullptr) {
  GramArgs a;
  a.n = ws.n;
  a.kp = ws.kp;
  a.npairs = npairs;
  a.nt = gram_nt_for(ws.kp);
  int gy = 1;
  a.rows_per_group = gram_rows_per_group(ws.n, ws.kp, npairs, &gy);
  if (gy > ws.gram_gy) {  // the workspace holds ws.gram_gy row groups: fewer, larger ones
    a.rows_per_group = ceil_div(ceil_div(ws.n, (int64_t)ws.gram_gy), (int64_t)kGramChunk) * kGramChunk;
    gy = (int)ceil_div(ws.n, a.rows_per_group);
  }
  a.pairs = pairs;
  a.part = ws.gram_part;
  a.ctrl = ws.ctrl;
  a.ignore_done = ignore_done;
  dim3 grid(npairs * a.nt * a.nt, gy);
  if (prof) prof->begin(OFSC_PHASE_GRAM);
  switch (gram_m_for(ws.kp)) {
    case 1:
      OFSC_GROUPABLE(k_gram<1>, k_gram_g<1>, GramArgs);
      k_gram<1><<<grid, 256, 0, s>>>(a);
      break;
    case 2:
      OFSC_GROUPABLE(k_gram<2>, k_gram_g<2>, GramArgs);
      k_gram<2><<<grid, 256, 0, s>>>(a);
      break;
    default:
      OFSC_GROUPABLE(k_gram<4>, k_gram_g<4>, GramArgs);
      k_gram<4><<<grid, 256, 0, s>>>(a);
      break;
  }
  if (prof) {
    prof->end();
    prof->begin(OFSC_PHASE_GRAM_REDUCE);
  }
  const int total = kPairs * ws.kp * ws.kp;
  GramReduceArgs ra{};
  ra.part = ws.gram_part;
  ra.gy = gy;
  ra.kp = ws.kp;
  ra.slot_mask = slot_mask;
  ra.gram = ws.gram;
  ra.ctrl = ws.ctrl;
  ra.ignore_done = ignore_done;
  OFSC_GROUPABLE(k_gram_reduce, k_gram_reduce_g, GramReduceArgs);
  k_gram_reduce<<<(int)std::min<int64_t>(ceil_div(total, 32), 8 * kNumSMs), 256, 0, s>>>(ra);
  if (prof) prof->end();
  g_launches += 2;
  return cudaGetLastError();
}

// Bytes of the tensor-core Gram partials for n rows (two or four right blocks per launch).
size_t gram_tc_part_need(int64_t n) {
  return std::max(gram_tc_part_bytes(n, 2, gram_tc_rows_per_cta(n, 2)),
                  gram_tc_part_bytes(n, 4, gram_tc_rows_per_cta(n, 4)));
}

ofsc_status ensure_workspace(ofsc_graph* g, int kp) {
  Workspace& ws = g->ws;
  if (ws.kp == kp && ws.n == g->n && ws.X) return OFSC_OK;
  workspace_free(ws);
  const int64_t n = g->n;
  const size_t blk = (size_t)(n > 0 ? n : 1) * kp * sizeof(float);
  int gy1 = 1, gy2 = 1;
  gram_rows_per_group(n, kp, kPairs, &gy1);
  gram_rows_per_group(n, kp, 2, &gy2);
  const int gy = std::max(gy1, gy2);
  const size_t kk = (size_t)kp * kp;
  ws.n = n;
  ws.kp = kp;
  ws.gram_gy = gy;
  ws.row_blocks = kMaxRowBlocks;
  struct {
    void** p;
    size_t bytes;
  } items[] = {
      {(void**)&ws.X, blk},
      {(void**)&ws.Y, blk},
      {(void**)&ws.V, blk},
      {(void**)&ws.W, blk},
      {(void**)&ws.G, blk},
      {(void**)&ws.Vh, blk},
      {(void**)&ws.gram_part, (size_t)gy * kPairs * kk * sizeof(double)},
      {(void**)&ws.gram, kPairs * kk * sizeof(double)},
      {(void**)&ws.Rn, kk * sizeof(float)},
      {(void**)&ws.Bn, kk * sizeof(float)},
      {(void**)&ws.R64, kk * sizeof(double)},
      {(void**)&ws.B64, kk * sizeof(double)},
      {(void**)&ws.dots, (size_t)((kRowMaxWarps + kRowWarpsPerBlock) + kVpassMaxBlocks + 2 * kDotsRows) * kp * sizeof(double)},
      {(void**)&ws.part_tc, kp > 64 ? gram_tc_part_need(n) : (size_t)16},
      {(void**)&ws.alpha, kp * sizeof(float)},
      {(void**)&ws.beta, kp * sizeof(float)},
      {(void**)&ws.alpha64, kp * sizeof(double)},
      {(void**)&ws.beta64, kp * sizeof(double)},
      {(void**)&ws.vscale, kp * sizeof(double)},
      {(void**)&ws.vinv, kp * sizeof(float)},
      {(void**)&ws.colpart, (size_t)(kMaxRowBlocks + kDotsRows) * kColSums * kp * sizeof(double)},
      {(void**)&ws.dE, (size_t)kp * sizeof(double)},
      {(void**)&ws.bimg, kp == 128 ? (size_t)(4 * 4 * 128 * 32 * 4) : (size_t)16},
      {(void**)&ws.carry_row, (size_t)kRowMaxWarps * 2 * sizeof(int64_t)},
      {(void**)&ws.carry, (size_t)kRowMaxWarps * 2 * kp * sizeof(float)},
      {(void**)&ws.solve, (size_t)(kSolveBlocks * kSolveSums + 8 * kp) * sizeof(double)},
      {(void**)&ws.ctrl, sizeof(Ctrl)},
  };
  size_t total = 0;
  for (auto& it : items) {
    cudaError_t e = dev_alloc(it.p, it.bytes);
    if (e != cudaSuccess) {
      workspace_free(ws);
      return cuda_fail(e, "workspace cudaMalloc");
    }
    total += it.bytes;
  }
  cudaError_t e = cudaMallocHost((void**)&ws.ctrl_host, sizeof(Ctrl));
  if (e != cudaSuccess) {
    workspace_free(ws);
    return cuda_fail(e, "cudaMallocHost");
  }
  ws.part_tc_bytes = kp > 64 ? gram_tc_part_need(n) : (size_t)16;
  ws.bytes = total;
  return OFSC_OK;
}

// The tensor-core Gram partials for a call that forces the tensor-core Grams at kp <= 64 (the
// workspace holds them only for kp > 64): grown once, kept with the workspace.
ofsc_status ensure_part_tc(Workspace& ws) {
  const size_t need = gram_tc_part_need(ws.n);
  if (ws.part_tc_bytes >= need) return OFSC_OK;
  float* p = nullptr;
  cudaError_t e = dev_alloc(&p, need);
  if (e != cudaSuccess) return cuda_fail(e, "tensor-core Gram partials");
  dev_free(ws.part_tc);  // synchronises with any queued use of the old buffer
  ws.bytes += need - ws.part_tc_bytes;
  ws.part_tc = p;
  ws.part_tc_bytes = need;
  return OFSC_OK;
}

struct Runner {
  ofsc_graph* g;
  Workspace& ws;
  cudaStream_t s;
  int method;
  bool bf16;
  Prof& prof;
  bool tc = false;   // Grams on the tensor cores
  bool tc_dir = true;  // with tc: the direction pass on the tensor cores too (padded k = 128)
  bool mp = false;     // the direction product on the merge-path shares (rows longer than a share)
  bool tma = false;  // sparse product with TMA gather4
  // with a side stream: V^T X and V^T V run there, beside the direction product (set by the
  // caller when it may, i.e. not under per-phase timing)
  cudaStream_t side = nullptr;
  cudaEvent_t side_fork = nullptr, side_join = nullptr;

  // L^T R_b for b < nr into the gram slots, on the tensor cores or the CUDA cores, on stream `on`
  // (the update's stream when null)
  cudaError_t grams(const float* L, const float* const* R, int nr, const int* slots, int ignore_done,
                    bool timed, cudaStream_t on = nullptr) {
    if (on == nullptr) on = s;
    if (tc) {
      GramTcArgs t{};
      t.n = ws.n;
      t.ld = ws.kp;
      t.k = ws.kp;
      t.nr = nr;
      t.L = L;
      t.lslot = -1;
      for (int b = 0; b < nr; ++b) {
        t.R[b] = R[b];
        if (R[b] == L && t.lslot < 0) t.lslot = b;
      }
      t.rows_per_cta = gram_tc_rows_per_cta(ws.n, nr);
      t.part = ws.part_tc;
      t.use_ws = 1;
      t.ctrl = ws.ctrl;
      t.ignore_done = ignore_done;
      if (timed) prof.begin(OFSC_PHASE_GRAM);
      cudaError_t e = gram_tc_launch(t, slots, ws.kp, ws.gram, on);
      if (timed) prof.end();
      g_launches += 3;
      return e;
    }
    GramPairs p{};
    int mask = 0;
    for (int b = 0; b < nr; ++b) {
      p.L[b] = L;
      p.R[b] = R[b];
      p.slot[b] = slots[b];
      mask |= 1 << slots[b];
    }
    return launch_gram(ws, p, nr, mask, ignore_done, on, timed ? &prof : nullptr);
  }

  SpmmArgs spmm_base() const {
    SpmmArgs a{};
    a.n = ws.n;
    a.kp = ws.kp;
    a.row_ptr = g->row_ptr;
    a.col = g->col;
    a.val = g->val;
    a.dinv = g->dinv;
    const int pi = spmm_lanes_index(spmm_lanes(ws.kp));
    a.bnd = g->bnd[pi];
    a.groups = g->groups[pi];
    a.ctrl = ws.ctrl;
    return a;
  }

  // The warp-per-row product's arguments on the direction partition, merge-path when chosen.
  void dir_partition(SpmmArgs& a) const {
    a.bnd = g->bnd[kRowPart];
    a.groups = g->groups[kRowPart];
    if (mp) {
      a.mp = g->mp;
      a.carry_row = ws.carry_row;
      a.carry = ws.carry;
    }
  }

  // AX from X exactly, then X^T X and X^T AX; Rn, Bn and f of `objective` from them.
  // (The gather copy Vh of the current direction is dead here: the next V pass rewrites it, so
  // it holds D^-1/2 X for the warp-per-row product.)
  cudaError_t refresh(int objective, int ignore_done) {
    prof.begin(OFSC_PHASE_REFRESH);
    float* Xh = (float*)ws.Vh;
    k_scale_rows<<<(int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ws.n * ws.kp / 4, 256), 8 * kNumSMs)), 256, 0,
                   s>>>(ws.n, ws.kp, ws.X, g->dinv, Xh, ws.ctrl, ignore_done);
    ++g_launches;
    SpmmArgs a = spmm_base();
    dir_partition(a);
    a.gather = Xh;
    a.base = ws.X;
    a.out = ws.Y;
    a.ignore_done = ignore_done;
    spmm_dir(a, g->weighted != 0, false, 0, s);
    const float* R[2] = {ws.X, ws.Y};
    const int slots[2] = {G_R, G_B};
    cudaError_t e = grams(ws.X, R, 2, slots, ignore_done, false);
    if (e != cudaSuccess) return e;
    k_set_rb<<<1, 256, 0, s>>>(ws.gram, ws.kp, objective, ws.Rn, ws.Bn, ws.R64, ws.B64, ws.ctrl,
                               ignore_done);
    ++g_launches;
    prof.end();
    return cudaGetLastError();
  }

  cudaError_t rowpass(int dir_method, int update, int eval, int ignore_done, int* nblk, int need_vy = 0) {
    RowArgs r{};
    r.n = ws.n;
    r.kp = ws.kp;
    r.X = ws.X;
    r.Y = ws.Y;
    r.V = ws.V;
    r.W = ws.W;
    r.G = ws.G;
    r.Rn = ws.Rn;
    r.Bn = ws.Bn;
    r.alpha = ws.alpha;
    r.colpart = ws.colpart;
    r.ctrl = ws.ctrl;
    r.update = update;
    r.need_vy = need_vy;
    r.eval = eval;
    r.ignore_done = ignore_done;
    r.bimg = ws.bimg;
    prof.begin(OFSC_PHASE_DIRECTION);
    cudaError_t e;
    if (tc && tc_dir && direction_tc_supported(dir_method, ws.kp)) {
      e = direction_tc_launch(dir_method, r, s, nblk);
      g_launches += dir_method >= M_OFM_F2 ? 2 : 1;  // the f2 pass formats its B images first
    } else {
      e = launch_rowpass(dir_method, r, s, nblk);
    }
    prof.end();
    return e;
  }

  // beta, the stop test and the objective's diagonal term from the direction pass's column sums,
  // folded to kDotsRows rows first (eval: only the gradient norm)
  void beta(int nblk, int first, int eval, int stop_ok = 1) {
    const double* cp = ws.colpart;
    if (nblk > kDotsRows) {
      double* folded = ws.colpart + (size_t)kMaxRowBlocks * kColSums * ws.kp;
      FoldArgs fa{};
      fa.part = ws.colpart;
      fa.nb = nblk;
      fa.width = kColSums * ws.kp;
      fa.out = folded;
      fa.ctrl = ws.ctrl;
      fa.ignore_done = eval;
      OFSC_GROUPABLE(k_fold_rows, k_fold_rows_g, FoldArgs);
      k_fold_rows<<<kDotsRows, 256, 0, s>>>(fa);
      ++g_launches;
      cp = folded;
      nblk = kDotsRows;
    }
    BetaArgs ba{};
    ba.colpart = cp;
    ba.nblk = nblk;
    ba.kp = ws.kp;
    ba.beta = ws.beta;
    ba.beta64 = ws.beta64;
    ba.dE = eval ? nullptr : ws.dE;
    ba.ctrl = ws.ctrl;
    ba.first = first;
    ba.eval = eval;
    ba.stop_ok = stop_ok;
    ba.vscale = ws.vscale;
    ba.vinv = ws.vinv;
    ba.qprev = ws.gram + G_Q * (size_t)ws.kp * ws.kp;
    OFSC_GROUPABLE(k_beta, k_beta_g, BetaArgs);
    k_beta<<<1, 256, 0, s>>>(ba);
    ++g_launches;
  }

  cudaError_t direction_and_linesearch(int first, const ofsc_opts& o, int k, double alpha0) {
    const bool f2 = method >= M_OFM_F2;
    // Partials of diag(V^T AV) (sparse product) and diag(V^T G) (V pass) in ws.dots, then their
    // fold into kDotsRows rows of [2][kp] for the solve.
    double* dots_w = ws.dots;
    double* dots_g = ws.dots + (size_t)(kRowMaxWarps + kRowWarpsPerBlock) * ws.kp;
    double* folded = dots_g + (size_t)kVpassMaxBlocks * ws.kp;
    // V_t = -G_t + V_{t-1} diag(beta) and Vh = D^-1/2 V_t for the gather
    prof.begin(OFSC_PHASE_OTHER);
    const int lpn = spmm_lanes(ws.kp);
    const int vgrid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(ws.n, 256 / lpn), kVpassMaxBlocks));
    launch_vpass(lpn, bf16, vgrid, s, ws.n, ws.kp, ws.G, ws.V, ws.Vh, g->dinv, ws.beta, ws.vinv, first, dots_g,
                 ws.ctrl);
    ++g_launches;
    prof.end();
    // V^T X and V^T V for every method; V^T AX and V^T AV in full for the f2 methods. The first
    // two need only V and X, so with a side stream they run beside the sparse product.
    const float* Rs[4] = {ws.X, ws.V, ws.Y, ws.W};
    const int slots[4] = {G_P, G_Q, G_E, G_C};
    const bool overlap = side != nullptr && (!f2 || tc);
    if (overlap) {
      cudaError_t e = cudaEventRecord(side_fork, s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(side, side_fork, 0);
      if (e == cudaSuccess) e = grams(ws.V, Rs, 2, slots, 0, false, side);
      if (e == cudaSuccess) e = cudaEventRecord(side_join, side);
      if (e != cudaSuccess) return e;
    }
    // AV_t exactly (one sparse product), with diag(V^T AV)
    SpmmArgs a = spmm_base();
    a.gather = ws.Vh;
    a.base = ws.V;
    a.out = ws.W;
    a.dots = dots_w;
    int dots_blocks = 0;
    prof.begin(OFSC_PHASE_SPMM);
    if (tma) {
      TmaSpmmArgs t{};
      t.n = ws.n;
      t.kp = ws.kp;
      t.row_ptr = g->row_ptr;
      t.col = g->col;
      t.val = g->val;
      t.dinv = g->dinv;
      const int pi = spmm_lanes_index(32);
      t.bnd = g->bnd[pi];
      t.groups = g->groups[pi];
      t.base = ws.V;
      t.out = ws.W;
      t.dots = dots_w;
      t.ctrl = ws.ctrl;
      cudaError_t e = spmm_tma_launch(ws.vh_map[bf16 ? 1 : 0], t, bf16, g->weighted != 0, s);
      if (e != cudaSuccess) return e;
      ++g_launches;
      dots_blocks = t.groups / spmm_tma_groups_per_block();
    } else {
      dir_partition(a);
      dots_blocks = spmm_dir(a, g->weighted != 0, bf16, tuned_slots(g, ws.kp, bf16), s);
    }
    DotsFoldArgs df{};
    df.pw = dots_w;
    df.nw = dots_blocks;
    df.pg = dots_g;
    df.ng = vgrid;
    df.kp = ws.kp;
    df.out = folded;
    df.ctrl = ws.ctrl;
    OFSC_GROUPABLE(k_dots_fold, k_dots_fold_g, DotsFoldArgs);
    k_dots_fold<<<kDotsRows, 256, 0, s>>>(df);
    ++g_launches;
    prof.end();
    cudaError_t e;
    if (overlap) {
      // join first: the f2 launch (V; AX, AV) reuses the partials buffer of the side launch
      e = cudaStreamWaitEvent(s, side_join, 0);
      if (e == cudaSuccess && f2) e = grams(ws.V, Rs + 2, 2, slots + 2, 0, true);
    } else if (tc && f2) {
      // two warp-specialised launches: (V; X, V), then (V; AX, AV) with V staged on its own
      e = grams(ws.V, Rs, 2, slots, 0, true);
      if (e == cudaSuccess) e = grams(ws.V, Rs + 2, 2, slots + 2, 0, true);
    } else {
      e = grams(ws.V, Rs, f2 ? 4 : 2, slots, 0, true);
    }
    if (e != cudaSuccess) return e;
    SolveArgs sa{};
    sa.gram = ws.gram;
    sa.dots = folded;
    sa.dots_blocks = kDotsRows;
    sa.dE = ws.dE;
    sa.R64 = ws.R64;
    sa.B64 = ws.B64;
    sa.kp = ws.kp;
    sa.k = k;
    sa.method = method;
    sa.Rn = ws.Rn;
    sa.Bn = ws.Bn;
    sa.alpha = ws.alpha;
    sa.alpha64 = ws.alpha64;
    sa.beta64 = ws.beta64;
    sa.trace = o.trace;
    sa.ctrl = ws.ctrl;
    sa.alpha0 = alpha0;
    sa.part = ws.solve;
    sa.tblocks = solve_blocks(ws.kp);
    sa.vscale = ws.vscale;
    prof.begin(OFSC_PHASE_LINESEARCH);
    OFSC_GROUPABLE(k_solve_traces, k_solve_traces_g, SolveArgs);
    OFSC_GROUPABLE(k_solve, k_solve_g, SolveArgs);
    OFSC_GROUPABLE(k_solve_update, k_solve_update_g, SolveArgs);
    k_solve_traces<<<sa.tblocks, 256, 0, s>>>(sa);
    k_solve<<<1, 256, 0, s>>>(sa);
    k_solve_update<<<sa.tblocks, 256, 0, s>>>(sa);
    g_launches += 3;
    prof.end();
    return cudaGetLastError();
  }
};

int grid_elems(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 8 * kNumSMs)); }

ofsc_status finish(Workspace& ws, cudaStream_t s, Ctrl* out) {
  OFSC_CUDA(cudaMemcpyAsync(ws.ctrl_host, ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  OFSC_CUDA(cudaStreamSynchronize(s));
  *out = *ws.ctrl_host;
  return OFSC_OK;
}

}  // namespace

cudaError_t apply_A(ofsc_graph* g, int kp, const float* X, float* Y, float* scratch, cudaStream_t s) {
  if (g->n == 0) return cudaSuccess;
  k_scale_rows<<<(int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(g->n * kp / 4, 256), 8 * kNumSMs)), 256, 0, s>>>(
      g->n, kp, X, g->dinv, scratch, nullptr, 1);
  SpmmArgs a{};
  a.n = g->n;
  a.kp = kp;
  a.row_ptr = g->row_ptr;
  a.col = g->col;
  a.val = g->val;
  a.dinv = g->dinv;
  a.bnd = g->bnd[kRowPart];
  a.groups = g->groups[kRowPart];
  a.gather = scratch;
  a.base = X;
  a.out = Y;
  a.ignore_done = 1;
  spmm_dir(a, g->weighted != 0, false, 0, s);
  return cudaGetLastError();
}

}  // namespace ofsc

using namespace ofsc;

extern "C" ofsc_status ofsc_objective_grad(ofsc_graph* g, int32_t objective, int32_t k, const float* X,
                                           double* f_out, float* G_out, void* stream_) {
  clear_error();
  if (!g) return fail(OFSC_ERR_INVALID_ARG, "ofsc_objective_grad: graph is NULL");
  if (objective != OFSC_F1 && objective != OFSC_F2)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_objective_grad: objective must be OFSC_F1 or OFSC_F2");
  if (k < 1 || k > kMaxK) return fail(OFSC_ERR_INVALID_ARG, "ofsc_objective_grad: k=%d outside [1, %d]", k, kMaxK);
  if (g->n > 0 && !X) return fail(OFSC_ERR_INVALID_ARG, "ofsc_objective_grad: X is NULL");
  cudaStream_t s = (cudaStream_t)stream_;
  const int kp = round_up(k, 8);
  ofsc_status st = ensure_workspace(g, kp);
  if (st != OFSC_OK) return st;
  Workspace& ws = g->ws;
  const int method = objective == OFSC_F1 ? M_OFM_F1 : M_OFM_F2;
  Prof prof{ws, nullptr, s};
  Runner run{g, ws, s, method, false, prof};
  run.mp = use_merge_path(g, 0, kp, false);
  // a single evaluation, on the CUDA cores at every k: the Grams as FP32 products summed in FP64,
  // and the direction pass in plain FP32. The iteration's tensor-core engines accumulate in FP32
  // tensor memory, which at N = 2M biases the diagonal of X^T X by a few 1e-6 (512-row segments,
  // rounding toward zero), and grad f = 4 (AX + X X^T X) cancels its two terms to 1.5e-5 of its
  // largest entry there.
  run.tc = false;
  run.tc_dir = false;
  k_init_ctrl<<<1, 1, 0, s>>>(ws.ctrl, 0.0, 0, k, g->normA2, 0);
  ++g_launches;
  OFSC_LAUNCH_CHECK("k_init_ctrl");
  Ctrl c{};
  if (g->n > 0) {
    k_pad_in<<<grid_elems(g->n * kp), 256, 0, s>>>(g->n, k, kp, X, ws.X, ws.ctrl);
    ++g_launches;
    OFSC_LAUNCH_CHECK("k_pad_in");
    OFSC_CUDA(run.refresh(objective, 0));
    int nblk = 0;
    OFSC_CUDA(run.rowpass(method, 0, 1, 0, &nblk));
    if (G_out) {
      k_pad_out<<<grid_elems(g->n * k), 256, 0, s>>>(g->n, k, kp, ws.G, G_out);
      ++g_launches;
      OFSC_LAUNCH_CHECK("k_pad_out");
    }
    st = finish(ws, s, &c);
    if (st != OFSC_OK) return st;
    st = bounds_checked(OFSC_OK, "ofsc_objective_grad");
    if (st != OFSC_OK) return st;
  } else {
    c.f = objective == OFSC_F1 ? 0.0 : 0.0;
  }
  if (c.status == OFSC_ERR_TIMEOUT) return fail(c.status, "ofsc_objective_grad: a bounded tensor-core wait timed out");
  if (c.status != OFSC_OK) return fail(c.status, "ofsc_objective_grad: non-finite value in X");
  if (!std::isfinite(c.f)) return fail(OFSC_ERR_NONFINITE, "ofsc_objective_grad: non-finite objective");
  if (f_out) *f_out = c.f;
  return OFSC_OK;
}

extern "C" ofsc_status ofsc_weight_grad(ofsc_graph* g, int32_t objective, int32_t k, const float* X, int64_t m,
                                        const int32_t* src, const int32_t* dst, float* grad, void* stream_) {
  clear_error();
  if (!g) return fail(OFSC_ERR_INVALID_ARG, "ofsc_weight_grad: graph is NULL");
  if (objective != OFSC_F1 && objective != OFSC_F2)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_weight_grad: objective must be OFSC_F1 or OFSC_F2");
  if (k < 1 || k > kMaxK) return fail(OFSC_ERR_INVALID_ARG, "ofsc_weight_grad: k=%d outside [1, %d]", k, kMaxK);
  if (!g->weighted) return fail(OFSC_ERR_INVALID_ARG, "ofsc_weight_grad: the graph was built without edge weights");
  if (m < 0 || (m > 0 && (!src || !dst || !grad)) || (g->n > 0 && !X))
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_weight_grad: bad edge arrays or NULL X");
  cudaStream_t s = (cudaStream_t)stream_;
  const int kp = round_up(k, 8);
  ofsc_status st = ensure_workspace(g, kp);
  if (st != OFSC_OK) return st;
  Workspace& ws = g->ws;
  Prof prof{ws, nullptr, s};
  Runner run{g, ws, s, objective == OFSC_F1 ? M_OFM_F1 : M_OFM_F2, false, prof};
  run.mp = use_merge_path(g, 0, kp, false);
  run.tc = false;  // a single evaluation: the CUDA-core Grams (FP64 sums), as ofsc_objective_grad
  DevBuf sbuf;
  OFSC_CUDA(dev_alloc(&sbuf.p, (size_t)(g->n + 1) * sizeof(float) + 16));
  void* scratch = sbuf.p;
  int* bad = (int*)scratch;
  float* r = (float*)((char*)scratch + 16);
  cudaMemsetAsync(bad, 0, sizeof(int), s);
  k_init_ctrl<<<1, 1, 0, s>>>(ws.ctrl, 0.0, 0, k, g->normA2, 0);
  cudaError_t e = cudaSuccess;
  if (g->n > 0) {
    k_pad_in<<<grid_elems(g->n * kp), 256, 0, s>>>(g->n, k, kp, X, ws.X, ws.ctrl);
    e = run.refresh(objective, 0);  // A X and X^T X
  }
  if (e == cudaSuccess) {
    WgradArgs w{};
    w.n = g->n;
    w.kp = kp;
    w.which = objective;
    w.X = ws.X;
    w.AX = ws.Y;
    w.R64 = ws.R64;
    w.row_ptr = g->row_ptr;
    w.col = g->col;
    w.val = g->val;
    w.dinv = g->dinv;
    w.r = r;
    w.Z = ws.W;
    w.m = m;
    w.src = src;
    w.dst = dst;
    w.grad = grad;
    w.bad = bad;
    e = wgrad_launch(w, s);
  }
  int hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "ofsc_weight_grad");
  Ctrl c{};
  st = finish(ws, s, &c);
  if (st != OFSC_OK) return st;
  if (hbad) return fail(OFSC_ERR_INVALID_ARG, "ofsc_weight_grad: an edge endpoint is outside [0, n)");
  if (c.status != OFSC_OK) return fail(c.status, "ofsc_weight_grad: failed (status %d)", c.status);
  return OFSC_OK;
}

extern "C" ofsc_status ofsc_rayleigh_ritz(ofsc_graph* g, int32_t k, const float* X, double* ritz, double* relerr,
                                          void* stream_) {
  clear_error();
  if (!g) return fail(OFSC_ERR_INVALID_ARG, "ofsc_rayleigh_ritz: graph is NULL");
  if (k < 1 || k > kMaxK) return fail(OFSC_ERR_INVALID_ARG, "ofsc_rayleigh_ritz: k=%d outside [1, %d]", k, kMaxK);
  if (!ritz || !relerr || (g->n > 0 && !X)) return fail(OFSC_ERR_INVALID_ARG, "ofsc_rayleigh_ritz: NULL pointer");
  if (g->n < k) return fail(OFSC_ERR_INVALID_ARG, "ofsc_rayleigh_ritz: n=%lld < k=%d", (long long)g->n, k);
  cudaStream_t s = (cudaStream_t)stream_;
  const int kp = round_up(k, 8);
  ofsc_status st = ensure_workspace(g, kp);
  if (st != OFSC_OK) return st;
  Workspace& ws = g->ws;
  Prof prof{ws, nullptr, s};
  Runner run{g, ws, s, M_OFM_F1, false, prof};
  run.mp = use_merge_path(g, 0, kp, false);
  run.tc = false;  // a single evaluation: the CUDA-core Grams (FP64 sums), as ofsc_objective_grad
  DevBuf wbuf;
  OFSC_CUDA(dev_alloc(&wbuf.p, (4 * (size_t)kp * kp + 2) * sizeof(double)));
  double* work = (double*)wbuf.p;
  double* sums = work + 4 * (size_t)kp * kp;
  double* out = sums + 1;
  k_init_ctrl<<<1, 1, 0, s>>>(ws.ctrl, 0.0, 0, k, g->normA2, 0);
  k_pad_in<<<grid_elems(g->n * kp), 256, 0, s>>>(g->n, k, kp, X, ws.X, ws.ctrl);
  cudaError_t e = run.refresh(1, 0);  // A X, X^T X (R64), X^T A X (B64)
  if (e == cudaSuccess) e = ritz_prepare_launch(ws.R64, ws.B64, k, kp, work, ws.Rn, ritz, sums, ws.ctrl, s);
  int nblk = 0;
  // G = 4 (A X + X Rn) = 4 E with Rn = -(X^T X)^-1 X^T A X (the OFM-f1 row pass, evaluation form)
  if (e == cudaSuccess) e = run.rowpass(M_OFM_F1, 0, 1, 0, &nblk);
  if (e == cudaSuccess) {
    const float* Rs[1] = {ws.G};
    const int slots[1] = {G_E};
    e = run.grams(ws.G, Rs, 1, slots, 0, false);
  }
  if (e == cudaSuccess) e = ritz_relerr_launch(ws.gram + (size_t)G_E * kp * kp, work, k, kp, sums, out, s);
  double h = 0.0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, out, sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "ofsc_rayleigh_ritz");
  Ctrl c{};
  st = finish(ws, s, &c);
  if (st != OFSC_OK) return st;
  if (c.status == OFSC_ERR_INVALID_ARG) return fail(c.status, "ofsc_rayleigh_ritz: X^T X is not positive definite");
  if (c.status != OFSC_OK) return fail(c.status, "ofsc_rayleigh_ritz: failed (status %d)", c.status);
  if (!std::isfinite(h)) return fail(OFSC_ERR_NONFINITE, "ofsc_rayleigh_ritz: non-finite relerr");
  *relerr = h;
  return OFSC_OK;
}

namespace ofsc {
namespace {

// Argument checks shared by the single and batched entry points (no launches).
ofsc_status check_iterate_args(const ofsc_graph* g, int32_t method, int32_t k, const float* X, double tol,
                               int32_t maxit, const ofsc_opts& o, const char* who) {
  if (!g) return fail(OFSC_ERR_INVALID_ARG, "%s: graph is NULL", who);
  if (method < OFSC_OFM_F1 || method > OFSC_TRI_F2) return fail(OFSC_ERR_INVALID_ARG, "%s: unknown method %d", who, method);
  if (k < 1 || k > kMaxK) return fail(OFSC_ERR_INVALID_ARG, "%s: k=%d outside [1, %d]", who, k, kMaxK);
  if (maxit < 0) return fail(OFSC_ERR_INVALID_ARG, "%s: maxit < 0", who);
  if (!(tol == tol)) return fail(OFSC_ERR_INVALID_ARG, "%s: tol is NaN", who);
  if (g->n > 0 && !X) return fail(OFSC_ERR_INVALID_ARG, "%s: X is NULL", who);
  if (o.gather != OFSC_GATHER_FP32 && o.gather != OFSC_GATHER_BF16)
    return fail(OFSC_ERR_INVALID_ARG, "%s: unknown gather mode %d", who, o.gather);
  if (o.trace && o.trace_cap < 0) return fail(OFSC_ERR_INVALID_ARG, "%s: trace_cap < 0", who);
  if (o.gram_engine < OFSC_GRAM_AUTO || o.gram_engine > OFSC_GRAM_TC)
    return fail(OFSC_ERR_INVALID_ARG, "%s: unknown gram_engine %d", who, o.gram_engine);
  if (o.spmm_engine < OFSC_SPMM_AUTO || o.spmm_engine > OFSC_SPMM_TMA)
    return fail(OFSC_ERR_INVALID_ARG, "%s: unknown spmm_engine %d", who, o.spmm_engine);
  if (o.cg_restart != 0 && o.cg_restart != 1)
    return fail(OFSC_ERR_INVALID_ARG, "%s: cg_restart must be 0 or 1", who);
  if (!(o.refine_tol >= 0.0)) return fail(OFSC_ERR_INVALID_ARG, "%s: refine_tol must be >= 0", who);
  if (!(o.exact_tail == o.exact_tail)) return fail(OFSC_ERR_INVALID_ARG, "%s: exact_tail is NaN", who);
  if (o.vscale_exp < -60 || o.vscale_exp > 60)
    return fail(OFSC_ERR_INVALID_ARG, "%s: vscale_exp outside [-60, 60]", who);
  if (o.spin_limit < 0) return fail(OFSC_ERR_INVALID_ARG, "%s: spin_limit < 0", who);
  if (o.withhold_arrivals != 0 && o.withhold_arrivals != 1)
    return fail(OFSC_ERR_INVALID_ARG, "%s: withhold_arrivals must be 0 or 1", who);
  if (o.merge_path < -1 || o.merge_path > 1) return fail(OFSC_ERR_INVALID_ARG, "%s: merge_path must be -1, 0 or 1", who);
  if (o.group_launches < 0 || o.group_launches > 64)
    return fail(OFSC_ERR_INVALID_ARG, "%s: group_launches must be in [0, 64]", who);
  if (o.overlap_gram < -1 || o.overlap_gram > 1)
    return fail(OFSC_ERR_INVALID_ARG, "%s: overlap_gram must be -1, 0 or 1", who);
  const int kp = round_up(k, 8);
  const bool tc = o.gram_engine == OFSC_GRAM_TC || (o.gram_engine == OFSC_GRAM_AUTO && kp > 64);
  if (tc && kp > 128) return fail(OFSC_ERR_INVALID_ARG, "%s: tensor-core Grams need k <= 128", who);
  if (o.spmm_engine == OFSC_SPMM_TMA && !spmm_tma_supported(kp))
    return fail(OFSC_ERR_INVALID_ARG, "%s: the TMA sparse product needs a padded k of 64 or 128", who);
  return OFSC_OK;
}

// One graph's run of Algorithm 2 on one stream: setup, the update of iteration t (no host reads),
// and the final report. ofsc_iterate drives one Job; ofsc_iterate_batched drives many in lockstep.
struct Job {
  ofsc_graph* g;
  int method, k, kp, objective, maxit, y_refresh;
  float* X;
  double tol;
  ofsc_opts o;
  cudaStream_t s;
  Prof prof;
  Runner run;
  int64_t launches = 0;  // kernels launched for this graph
  // FP32 refinement sweep of a BF16-gather run: pending until a host check reads
  // ||G_t|| <= refine_tol ||G_0||; refined_at is the update from which gathers are FP32 (-1: never)
  bool refine_pending = false;
  int refined_at = -1;
  // Exact tail (opts.exact_tail > 0, or 1e3 tol by default): once a host check reads
  // ||G_t|| <= exact_tail ||G_0||, every
  // later update is exact; exact_at is the first such update. Independently, tol met on an update
  // whose AX came from the recurrence (near_tol) makes the update after the next host check exact,
  // and only exact updates may stop the run.
  double exact_tail;
  bool exact = false;
  int exact_at = -1;
  int forced_refresh = -1;
  // opts.state: the CG state to resume (resume: it holds a run) and to leave for the next call
  ofsc_state* cg = nullptr;
  bool resume = false;

  Job(ofsc_graph* g_, int method_, int k_, float* X_, double tol_, int maxit_, const ofsc_opts& o_, cudaStream_t s_)
      : g(g_), method(method_), k(k_), kp(round_up(k_, 8)),
        objective((method_ == OFSC_OFM_F1 || method_ == OFSC_TRI_F1) ? 1 : 2), maxit(maxit_),
        y_refresh(o_.y_refresh > 0 ? o_.y_refresh : 32), X(X_), tol(tol_), o(o_), s(s_),
        prof{g_->ws, o_.profile, s_}, run{g_, g_->ws, s_, method_, o_.gather == OFSC_GATHER_BF16, prof},
        refine_pending(o_.gather == OFSC_GATHER_BF16 && o_.refine_tol > 0.0),
        exact_tail(o_.exact_tail > 0.0 ? o_.exact_tail : (o_.exact_tail == 0.0 && tol_ > 0.0 ? 1e3 * tol_ : 0.0)) {}

  // Host check after update t: copies done, rel (and it) from the control block; the caller
  // synchronises the stream before calling checked().
  cudaError_t queue_check(cudaStream_t on) {
    return cudaMemcpyAsync(g->ws.ctrl_host, g->ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, on);
  }
  // After the copy of queue_check has landed: switches a pending BF16 run to FP32 gathers once the
  // relative direction norm has reached refine_tol (from update t + 1 on). Returns done.
  bool checked(int t) {
    const Ctrl& c = *g->ws.ctrl_host;
    if (refine_pending && !c.done && c.status == OFSC_OK && c.rel <= o.refine_tol) {
      refine_pending = false;
      run.bf16 = false;
      refined_at = t + 1;
    }
    if (!exact && exact_tail > 0.0 && !c.done && c.status == OFSC_OK && c.rel <= exact_tail) {
      exact = true;
      exact_at = t + 1;
    }
    if (c.near_tol && !c.done && c.status == OFSC_OK) forced_refresh = t + 1;
    return c.done != 0;
  }

  // Workspace, engines and TMA maps; call before any launch (allocates, so never under capture).
  // alone: the call runs this graph only.
  ofsc_status prepare(bool alone) {
    cg = o.state;
    if (cg) {
      int dev = 0;
      cudaGetDevice(&dev);
      if (cg->n != g->n || cg->k != k || cg->kp != kp || cg->device != dev)
        return fail(OFSC_ERR_INVALID_ARG, "opts.state: made for n=%lld, k=%d on device %d, not n=%lld, k=%d on %d",
                    (long long)cg->n, cg->k, cg->device, (long long)g->n, k, dev);
      if (cg->t > 0 && cg->method != method)
        return fail(OFSC_ERR_INVALID_ARG, "opts.state: holds a run of method %d, not %d", cg->method, method);
      resume = cg->t > 0;
    }
    ofsc_status st = ensure_workspace(g, kp);
    if (st != OFSC_OK) return st;
    Workspace& ws = g->ws;
    run.tc = o.gram_engine == OFSC_GRAM_TC || (o.gram_engine == OFSC_GRAM_AUTO && kp > 64);
    run.tma = o.spmm_engine == OFSC_SPMM_TMA;
    run.mp = use_merge_path(g, o.merge_path, kp, run.bf16);
    if (run.tc) {
      st = ensure_part_tc(ws);
      if (st != OFSC_OK) return st;
    }
    // The Grams V^T X, V^T V beside the direction product: when asked for, and by default for a
    // call on one graph whose N x kp blocks are small (n kp <= 2^23: V and X together take at
    // most 64 MB, half the L2), where the two kernels share idle SMs rather than HBM bandwidth.
    // At n kp = 2^28 (2M x 128) the overlap measured 14% slower per update, at n kp <= 2.4M from
    // 4% to 8% faster. A batch already overlaps its graphs' streams.
    const bool overlap =
        o.overlap_gram > 0 || (o.overlap_gram == 0 && alone && (int64_t)g->n * kp <= (int64_t(1) << 23));
    if (overlap && o.group_launches == 0 && !o.profile) {
      if (!g->side) OFSC_CUDA(cudaStreamCreateWithFlags(&g->side, cudaStreamNonBlocking));
      if (!g->side_fork) OFSC_CUDA(cudaEventCreateWithFlags(&g->side_fork, cudaEventDisableTiming));
      if (!g->side_join) OFSC_CUDA(cudaEventCreateWithFlags(&g->side_join, cudaEventDisableTiming));
      run.side = g->side;
      run.side_fork = g->side_fork;
      run.side_join = g->side_join;
    }
    if (run.tma) {
      const int mi = run.bf16 ? 1 : 0;
      if (!ws.vh_map_ok[mi]) {
        st = spmm_tma_encode(ws.Vh, ws.n, kp, run.bf16, &ws.vh_map[mi]);
        if (st != OFSC_OK) return st;
        ws.vh_map_ok[mi] = true;
      }
    }
    return OFSC_OK;
  }

  // Control block, padded copy of X_0, exact AX_0 with X^T X and X^T AX.
  ofsc_status start() {
    NvtxRange nv("start: exact AX");
    const int64_t l0 = g_launches;
    Workspace& ws = g->ws;
    k_init_ctrl<<<1, 1, 0, s>>>(ws.ctrl, tol, maxit, k, g->normA2, o.trace ? o.trace_cap : 0, o.cg_restart ? 1 : 0,
                                o.vscale_exp != 0 ? o.vscale_exp : kDefaultVscaleExp, (long long)o.spin_limit,
                                o.withhold_arrivals ? 1 : 0);
    ++g_launches;
    OFSC_LAUNCH_CHECK("k_init_ctrl");
    k_pad_in<<<grid_elems(g->n * kp), 256, 0, s>>>(g->n, k, kp, X, ws.X, ws.ctrl);
    ++g_launches;
    OFSC_LAUNCH_CHECK("k_pad_in");
    OFSC_CUDA(run.refresh(objective, 0));
    if (resume) {  // the saved run: V_{t-1}, G_{t-1}, V's scales, V_{t-1}^T V_{t-1}, ||G_0||
      const size_t blk = (size_t)g->n * kp * sizeof(float);
      OFSC_CUDA(cudaMemcpyAsync(ws.V, cg->V, blk, cudaMemcpyDeviceToDevice, s));
      OFSC_CUDA(cudaMemcpyAsync(ws.G, cg->G, blk, cudaMemcpyDeviceToDevice, s));
      OFSC_CUDA(cudaMemcpyAsync(ws.vscale, cg->vscale, (size_t)kp * sizeof(double), cudaMemcpyDeviceToDevice, s));
      OFSC_CUDA(cudaMemcpyAsync(ws.gram + G_Q * (size_t)kp * kp, cg->Q, (size_t)kp * kp * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
      OFSC_CUDA(cudaMemcpyAsync(&ws.ctrl->g0, &cg->g0, sizeof(double), cudaMemcpyHostToDevice, s));
    }
    launches += g_launches - l0;
    return OFSC_OK;
  }

  // Before the final update overwrites them: G_{t-1}, V's scales and V_{t-1}^T V_{t-1} into the
  // CG state (V_{t-1} itself is kept by keep_state once the call has ended).
  cudaError_t save_before_final() {
    Workspace& ws = g->ws;
    const size_t blk = (size_t)g->n * kp * sizeof(float);
    cudaError_t e = cudaMemcpyAsync(cg->G, ws.G, blk, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cg->vscale, ws.vscale, (size_t)kp * sizeof(double), cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(cg->Q, ws.gram + G_Q * (size_t)kp * kp, (size_t)kp * kp * sizeof(double),
                          cudaMemcpyDeviceToDevice, s);
    return e;
  }

  // After the final report (c: the control block it read): a run that performed all maxit > 0
  // updates without stopping leaves its state (t grows by maxit); any other leaves it empty.
  cudaError_t keep_state(const Ctrl& c) {
    if (!cg) return cudaSuccess;
    if (maxit > 0 && c.status == OFSC_OK && !c.converged && c.it == maxit) {
      cudaError_t e = cudaMemcpyAsync(cg->V, g->ws.V, (size_t)g->n * kp * sizeof(float), cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) {
        cg->t = 0;
        return e;
      }
      cg->t += maxit;
      cg->g0 = c.g0;
      cg->method = method;
    } else if (maxit > 0 || c.status != OFSC_OK) {
      cg->t = 0;
    }
    return cudaSuccess;
  }

  // Iteration t: G_t (with the update of X_t fused in, or an exact refresh of AX every y_refresh
  // updates), beta and the stop test, and for t < maxit the direction and the line search.
  // Depends on t only through t == 0, t == maxit and the refresh schedule.
  ofsc_status update(int t) {
    NvtxRange nv(is_refresh(t) ? "update (exact refresh)" : "update");
    const int64_t l0 = g_launches;
    Workspace& ws = g->ws;
    int nblk = 0;
    if (cg && t == maxit && maxit > 0) OFSC_CUDA(save_before_final());
    if (t == 0 && resume) {
      // update t of the saved run: G from start()'s exact AX, beta against the saved G_{t-1}
      OFSC_CUDA(run.rowpass(method, 0, 0, 0, &nblk, 1));
      prof.begin(OFSC_PHASE_BETA);
      run.beta(nblk, 0, 0, 1);
      prof.end();
      OFSC_LAUNCH_CHECK("k_beta");
      if (t < maxit) OFSC_CUDA(run.direction_and_linesearch(0, o, k, 0.0));
      launches += g_launches - l0;
      return OFSC_OK;
    }
    if (is_refresh(t)) {
      prof.begin(OFSC_PHASE_OTHER);
      k_update_x<<<grid_elems(g->n * kp), 256, 0, s>>>(g->n, kp, ws.X, ws.V, ws.alpha, ws.ctrl);
      ++g_launches;
      prof.end();
      OFSC_LAUNCH_CHECK("k_update_x");
      OFSC_CUDA(run.refresh(objective, 0));
      OFSC_CUDA(run.rowpass(method, 0, 0, 0, &nblk, 1));
    } else {
      // t = 0 has no previous direction: evaluation mode skips the G_{t-1} read
      OFSC_CUDA(run.rowpass(method, t > 0 ? 1 : 0, t == 0 ? 1 : 0, 0, &nblk));
    }
    prof.begin(OFSC_PHASE_BETA);
    // t = 0 follows the exact AX of start(); a refresh update is exact as well
    run.beta(nblk, t == 0 ? 1 : 0, 0, (t == 0 || is_refresh(t)) ? 1 : 0);
    prof.end();
    OFSC_LAUNCH_CHECK("k_beta");
    if (t < maxit) OFSC_CUDA(run.direction_and_linesearch(t == 0 ? 1 : 0, o, k, t == 0 ? o.alpha0 : 0.0));
    launches += g_launches - l0;
    return OFSC_OK;
  }

  // exact: every update from here on recomputes AX, X^T X and X^T AX (the exact tail)
  bool is_refresh(int t) const { return t > 0 && (exact || t == forced_refresh || (t % y_refresh) == 0); }
  // The launches of update(t) are the same for every t with plain(t) true.
  bool plain(int t) const { return t > 0 && t < maxit && !is_refresh(t); }

  // Final report, queued: from an exact AX when the run has no error status (read by the caller
  // into `c` after a stream synchronisation), then the unpadded X.
  ofsc_status report(const Ctrl& c) {
    NvtxRange nv("report");
    const int64_t l0 = g_launches;
    Workspace& ws = g->ws;
    if (c.status == OFSC_OK) {
      OFSC_CUDA(run.refresh(objective, 1));
      int nblk = 0;
      OFSC_CUDA(run.rowpass(method, 0, 1, 1, &nblk));
      run.beta(nblk, 0, 1);
      OFSC_LAUNCH_CHECK("k_beta(eval)");
    }
    k_pad_out<<<grid_elems(g->n * k), 256, 0, s>>>(g->n, k, kp, ws.X, X);
    ++g_launches;
    OFSC_LAUNCH_CHECK("k_pad_out");
    OFSC_CUDA(cudaMemcpyAsync(ws.ctrl_host, ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
    launches += g_launches - l0;
    return OFSC_OK;
  }

  // After the stream has drained: the result from the control block copied by report().
  ofsc_status result(ofsc_result* out) const {
    const Ctrl& c = *g->ws.ctrl_host;
    ofsc_status rs = c.status != OFSC_OK ? c.status : (c.converged ? OFSC_OK : OFSC_ERR_NOT_CONVERGED);
    if (out) {
      out->iterations = c.it;
      out->status = rs;
      out->rel_dir_norm = c.rel;
      out->g0_norm = c.g0;
      out->f = c.f;
      out->kernel_launches = launches;
      out->refined_at = refined_at;
      out->exact_at = exact_at;
    }
    return rs;
  }
};

ofsc_status iterate_lockstep(int32_t count, ofsc_graph* const* graphs, int32_t method, const int32_t* ks,
                             float* const* Xs, double tol, int32_t maxit, const ofsc_opts& o, ofsc_result* outs,
                             cudaStream_t caller, const char* who);

ofsc_status result_error(ofsc_status rs, const char* who) {
  if (rs == OFSC_ERR_NONFINITE) return fail(rs, "%s: non-finite value in X0 or in the iteration", who);
  if (rs == OFSC_ERR_TIMEOUT) return fail(rs, "%s: a bounded tensor-core wait timed out", who);
  return rs;
}

}  // namespace
}  // namespace ofsc

extern "C" ofsc_status ofsc_iterate(ofsc_graph* g, int32_t method, int32_t k, float* X, double tol,
                                    int32_t maxit, const ofsc_opts* opts, ofsc_result* out, void* stream_) {
  clear_error();
  NvtxRange nv("ofsc_iterate");
  ofsc_opts o{};
  if (opts) o = *opts;
  ofsc_status st = check_iterate_args(g, method, k, X, tol, maxit, o, "ofsc_iterate");
  if (st != OFSC_OK) return st;
  const int check_every = o.check_every > 0 ? o.check_every : 16;
  cudaStream_t s = (cudaStream_t)stream_;
  if (out) *out = ofsc_result{0, OFSC_OK, 0.0, 0.0, 0.0, 0, -1, -1};
  if (g->n == 0) return OFSC_OK;
  if (!o.profile && o.direct_launch == 0) {
    // replay the repeating updates from a captured CUDA graph (the same launches, so the same bits)
    ofsc_graph* gs[1] = {g};
    const int32_t kk[1] = {k};
    float* xs[1] = {X};
    return bounds_checked(iterate_lockstep(1, gs, method, kk, xs, tol, maxit, o, out, s, "ofsc_iterate"),
                          "ofsc_iterate");
  }
  Job job(g, method, k, X, tol, maxit, o, s);
  st = job.prepare(true);
  if (st != OFSC_OK) return st;
  g_launches = 0;
  st = job.start();
  if (st != OFSC_OK) return st;
  Workspace& ws = g->ws;
  for (int t = 0; t <= maxit; ++t) {
    st = job.update(t);
    if (st != OFSC_OK) return st;
    if (t == maxit) break;
    if ((t + 1) % check_every == 0) {
      OFSC_CUDA(job.queue_check(s));
      OFSC_CUDA(cudaStreamSynchronize(s));
      job.prof.collect();
      if (job.checked(t)) break;
    }
  }
  Ctrl c{};
  st = finish(ws, s, &c);
  job.prof.collect();
  if (st != OFSC_OK) return st;
  st = job.report(c);
  if (st != OFSC_OK) return st;
  OFSC_CUDA(job.keep_state(c));
  OFSC_CUDA(cudaStreamSynchronize(s));
  job.prof.collect();
  return bounds_checked(result_error(job.result(out), "ofsc_iterate"), "ofsc_iterate");
}

// ==========================================================================================
// ofsc_autotune: the row-partition granularity of the direction product, chosen by timing.
// ==========================================================================================

extern "C" ofsc_status ofsc_autotune(ofsc_graph* g, int32_t k, int32_t gather, int32_t* warps_out,
                                     int32_t* slots_out, int32_t* merge_out, double* ms_out,
                                     void* stream_) {
  clear_error();
  NvtxRange nv("ofsc_autotune");
  if (!g) return fail(OFSC_ERR_INVALID_ARG, "ofsc_autotune: graph is NULL");
  if (k < 1 || k > kMaxK) return fail(OFSC_ERR_INVALID_ARG, "ofsc_autotune: k=%d outside [1, %d]", k, kMaxK);
  if (gather != OFSC_GATHER_FP32 && gather != OFSC_GATHER_BF16)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_autotune: unknown gather mode %d", gather);
  cudaStream_t s = (cudaStream_t)stream_;
  const int kp = round_up(k, 8);
  const bool bf16 = gather == OFSC_GATHER_BF16;
  if (g->n == 0 || g->nnz == 0) {
    if (warps_out) *warps_out = g->groups[kRowPart];
    if (slots_out) *slots_out = dir_default_slots(kp, bf16, g->weighted != 0);
    if (merge_out) *merge_out = 0;
    if (ms_out) *ms_out = 0.0;
    return OFSC_OK;
  }
  ofsc_status st = ensure_workspace(g, kp);
  if (st != OFSC_OK) return st;
  Workspace& ws = g->ws;
  // timing depends on the access pattern only: zero blocks
  OFSC_CUDA(cudaMemsetAsync(ws.V, 0, (size_t)g->n * kp * sizeof(float), s));
  OFSC_CUDA(cudaMemsetAsync(ws.Vh, 0, (size_t)g->n * kp * sizeof(float), s));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  OFSC_CUDA(cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(ce, "ofsc_autotune: cudaEventCreate");
  }
  struct Ev {
    cudaEvent_t a, b;
    ~Ev() {
      cudaEventDestroy(a);
      cudaEventDestroy(b);
    }
  } ev{e0, e1};
  const int min_wps = OFSC_ROW_MIN_WARPS_PER_SM, max_wps = OFSC_ROW_MAX_WARPS_PER_SM;
  int opts[4];
  const int nopt = dir_slot_options(kp, bf16, opts);
  int best_w = 0, best_u = 0;
  bool best_mp = false;
  float best_ms = 0.0f;
  for (int wps = min_wps; wps <= max_wps; wps *= 2) {
    const int W = wps * kNumSMs;
    if (wps > min_wps && (int64_t)W * 16 > g->nnz) break;  // at least 16 nonzeros per warp
    st = set_row_partition(g, W, s);
    if (st != OFSC_OK) return st;
    SpmmArgs a{};
    a.n = g->n;
    a.kp = kp;
    a.row_ptr = g->row_ptr;
    a.col = g->col;
    a.val = g->val;
    a.dinv = g->dinv;
    a.bnd = g->bnd[kRowPart];
    a.groups = g->groups[kRowPart];
    a.gather = ws.Vh;
    a.base = ws.V;
    a.out = ws.W;
    a.dots = ws.dots;
    a.ctrl = ws.ctrl;
    a.ignore_done = 1;
    // the whole-row shapes, then (option index nopt) the merge-path split with the default slots
    for (int oi = 0; oi <= nopt; ++oi) {
      const bool mp = oi == nopt;
      if (mp && g->nnz == 0) break;
      const int u = mp ? 0 : opts[oi];
      if (mp) {
        a.mp = g->mp;  // set_row_partition recomputed the shares for W warps
        a.carry_row = ws.carry_row;
        a.carry = ws.carry;
      }
      launch_spmm_dir(a, g->weighted != 0, bf16, u, s);  // warm
      OFSC_CUDA(cudaEventRecord(e0, s));
      for (int r = 0; r < 3; ++r) launch_spmm_dir(a, g->weighted != 0, bf16, u, s);
      OFSC_CUDA(cudaEventRecord(e1, s));
      OFSC_CUDA(cudaEventSynchronize(e1));
      OFSC_LAUNCH_CHECK("ofsc_autotune: direction product");
      float ms = 0.0f;
      OFSC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      ms /= 3.0f;
      if (best_w == 0 || ms < best_ms) {
        best_w = W;
        best_u = mp ? dir_default_slots(kp, bf16, g->weighted != 0) : u;
        best_mp = mp;
        best_ms = ms;
      }
    }
  }
  if (g->groups[kRowPart] != best_w) {
    st = set_row_partition(g, best_w, s);
    if (st != OFSC_OK) return st;
  }
  g->dir_tuned_kp = kp;
  g->dir_tuned_bf16 = bf16 ? 1 : 0;
  g->dir_slots = best_mp ? 0 : best_u;
  g->dir_mp = best_mp ? 1 : -1;
  if (warps_out) *warps_out = best_w;
  if (slots_out) *slots_out = best_u;
  if (merge_out) *merge_out = best_mp ? 1 : 0;
  if (ms_out) *ms_out = best_ms;
  return OFSC_OK;
}

// ==========================================================================================
// ofsc_iterate_batched: Algorithm 2 on many independent graphs at once.
//
// Each graph runs on a stream of its own (owned by its handle), forked from the caller's stream,
// so the kernels of small graphs share the SMs. The graphs advance in lockstep: iteration t of
// every graph is queued before iteration t + 1 of any. The updates whose launches do not depend
// on t (not the first, not a refresh of AX, not the last) are captured once, for all graphs, into
// one CUDA graph (a branch per graph) and replayed; a graph that has stopped keeps its branch,
// whose kernels return at once on its control block's stop flag, as they do between the host's
// flag reads in ofsc_iterate. So every graph gets the same launches, in the same order on its
// stream, as ofsc_iterate would give it, and the same bits.
// ==========================================================================================

namespace ofsc {
namespace {

struct BatchEvents {
  std::vector<cudaEvent_t> ev;
  ~BatchEvents() {
    for (cudaEvent_t e : ev) cudaEventDestroy(e);
  }
  cudaError_t make(size_t n) {
    ev.assign(n, nullptr);
    for (auto& e : ev) {
      cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
      if (r != cudaSuccess) return r;
    }
    return cudaSuccess;
  }
};

// Orders every job stream after `main` (fork) or `main` after every job stream (join).
cudaError_t fork_jobs(cudaStream_t main, std::vector<std::unique_ptr<Job>>& jobs, cudaEvent_t e) {
  cudaError_t r = cudaEventRecord(e, main);
  for (auto& j : jobs)
    if (r == cudaSuccess) r = cudaStreamWaitEvent(j->s, e, 0);
  return r;
}
cudaError_t join_jobs(cudaStream_t main, std::vector<std::unique_ptr<Job>>& jobs, const std::vector<cudaEvent_t>& e) {
  cudaError_t r = cudaSuccess;
  for (size_t i = 0; i < jobs.size() && r == cudaSuccess; ++i) {
    r = cudaEventRecord(e[i], jobs[i]->s);
    if (r == cudaSuccess) r = cudaStreamWaitEvent(main, e[i], 0);
  }
  return r;
}

struct HubStream {
  cudaStream_t s = nullptr;
  ~HubStream() {
    if (s) cudaStreamDestroy(s);
  }
};

struct GraphExec {
  cudaGraphExec_t exec = nullptr;
  ~GraphExec() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

}  // namespace
}  // namespace ofsc

namespace ofsc {
namespace {

// The lockstep driver of ofsc_iterate_batched, and of ofsc_iterate when it replays: arguments
// already checked, outs already cleared. Updates whose launches repeat for every problem are
// captured once into a CUDA graph and replayed (unless o.direct_launch); a trace is allowed for
// one problem (its records are written by a kernel at the device-side update index).
ofsc_status iterate_lockstep(int32_t count, ofsc_graph* const* graphs, int32_t method, const int32_t* ks,
                             float* const* Xs, double tol, int32_t maxit, const ofsc_opts& o, ofsc_result* outs,
                             cudaStream_t caller, const char* who) {
  NvtxRange nv("lockstep iteration");
  const int check_every = o.check_every > 0 ? o.check_every : 16;
  std::vector<std::unique_ptr<Job>> jobs;
  std::vector<int> slot;  // job index -> position in the caller's arrays
  for (int i = 0; i < count; ++i) {
    ofsc_graph* g = graphs[i];
    if (g->n == 0) continue;
    if (!g->stream) OFSC_CUDA(cudaStreamCreateWithFlags(&g->stream, cudaStreamNonBlocking));
    jobs.emplace_back(new Job(g, method, ks[i], Xs[i], tol, maxit, o, g->stream));
    slot.push_back(i);
  }
  if (jobs.empty()) return OFSC_OK;
  for (auto& j : jobs) {
    ofsc_status st = j->prepare(jobs.size() == 1);
    if (st != OFSC_OK) return st;
  }
  BatchEvents ev;
  OFSC_CUDA(ev.make(jobs.size() + 1));
  const std::vector<cudaEvent_t> jev(ev.ev.begin() + 1, ev.ev.end());
  cudaEvent_t fev = ev.ev[0];
  const bool replay = o.direct_launch == 0;
  // A hub stream of this call orders the graphs' streams (the caller's stream may be the legacy
  // default stream, on which no capture can start): caller -> hub -> graphs -> hub -> caller.
  HubStream hub;
  OFSC_CUDA(cudaStreamCreateWithFlags(&hub.s, cudaStreamNonBlocking));
  cudaStream_t main = hub.s;
  OFSC_CUDA(cudaEventRecord(fev, caller));
  OFSC_CUDA(cudaStreamWaitEvent(main, fev, 0));

  OFSC_CUDA(fork_jobs(main, jobs, fev));
  for (auto& j : jobs) {
    ofsc_status st = j->start();
    if (st != OFSC_OK) return st;
  }
  GraphExec plain;                  // one plain update of every graph
  std::vector<int64_t> plain_launches(jobs.size(), 0);
  const bool group = o.group_launches > 0;
  const int lanes = o.group_launches;
  bool forked = true;               // job streams are ordered after main and main not after them
  for (int t = 0; t <= maxit; ++t) {
    bool all_plain = true;
    for (auto& j : jobs) all_plain = all_plain && j->plain(t);
    if (replay && all_plain) {
      if (forked) {
        OFSC_CUDA(join_jobs(main, jobs, jev));
        forked = false;
      }
      if (!plain.exec) {
        // capture: main forks into one branch per graph and joins them again
        OFSC_CUDA(cudaStreamBeginCapture(main, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = fork_jobs(main, jobs, fev);
        ofsc_status st = OFSC_OK;
        for (size_t i = 0; i < jobs.size() && ce == cudaSuccess && st == OFSC_OK; ++i) {
          const int64_t l0 = jobs[i]->launches;
          st = jobs[i]->update(t);
          plain_launches[i] = jobs[i]->launches - l0;
          jobs[i]->launches = l0;  // counted when the graph runs
        }
        if (ce == cudaSuccess && st == OFSC_OK) ce = join_jobs(main, jobs, jev);
        cudaGraph_t graph = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(main, &graph);
        if (st != OFSC_OK) {
          if (graph) cudaGraphDestroy(graph);
          return st;
        }
        if (ce == cudaSuccess) ce = ee;
        // one launch per kernel of the update over every graph's blocks (the captured graph is
        // one chain per graph); kept as captured if it holds a node the rewrite does not know
        cudaGraph_t grouped = nullptr;
        int grouped_launches = 0;
        if (ce == cudaSuccess && group) {
          const cudaError_t ge = regroup_chains(graph, lanes, &grouped, &grouped_launches);
          if (ge != cudaSuccess) {
            (void)cudaGetLastError();
            grouped = nullptr;
          }
        }
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&plain.exec, grouped ? grouped : graph, 0);
        if (grouped) {
          cudaGraphDestroy(grouped);
          // a grouped launch serving several graphs is counted once, for the first of them
          for (size_t i = 0; i < jobs.size(); ++i) plain_launches[i] = i == 0 ? grouped_launches : 0;
        }
        if (graph) cudaGraphDestroy(graph);
        OFSC_CUDA(ce);
      }
      OFSC_CUDA(cudaGraphLaunch(plain.exec, main));
      for (size_t i = 0; i < jobs.size(); ++i) jobs[i]->launches += plain_launches[i];
    } else {
      if (!forked) {
        OFSC_CUDA(fork_jobs(main, jobs, fev));
        forked = true;
      }
      for (auto& j : jobs) {
        ofsc_status st = j->update(t);
        if (st != OFSC_OK) return st;
      }
    }
    if (t == maxit) break;
    if ((t + 1) % check_every == 0) {
      if (forked) {
        OFSC_CUDA(join_jobs(main, jobs, jev));
        forked = false;
      }
      for (auto& j : jobs) OFSC_CUDA(j->queue_check(main));
      OFSC_CUDA(cudaStreamSynchronize(main));
      bool all = true, switched = false;
      for (auto& j : jobs) {
        const bool was = j->run.bf16;
        all = j->checked(t) && all;
        switched = switched || (was != j->run.bf16);
      }
      if (all) break;
      // a job that moved to FP32 gathers launches other kernels: capture the plain update again
      // (a job in its exact tail is never plain, so the batch launches directly from then on)
      if (switched && plain.exec) {
        cudaGraphExecDestroy(plain.exec);
        plain.exec = nullptr;
      }
    }
  }
  // final reports: read every control block, then queue the exact evaluations together
  if (forked) OFSC_CUDA(join_jobs(main, jobs, jev));
  for (auto& j : jobs)
    OFSC_CUDA(cudaMemcpyAsync(j->g->ws.ctrl_host, j->g->ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, main));
  OFSC_CUDA(cudaStreamSynchronize(main));
  OFSC_CUDA(fork_jobs(main, jobs, fev));
  for (auto& j : jobs) {
    const Ctrl c = *j->g->ws.ctrl_host;
    ofsc_status st = j->report(c);
    if (st != OFSC_OK) return st;
    OFSC_CUDA(j->keep_state(c));
  }
  OFSC_CUDA(join_jobs(main, jobs, jev));
  OFSC_CUDA(cudaEventRecord(fev, main));
  OFSC_CUDA(cudaStreamWaitEvent(caller, fev, 0));
  OFSC_CUDA(cudaStreamSynchronize(main));
  ofsc_status worst = OFSC_OK;
  for (size_t i = 0; i < jobs.size(); ++i) {
    const ofsc_status rs = jobs[i]->result(outs ? &outs[slot[i]] : nullptr);
    if (rs != OFSC_OK && (worst == OFSC_OK || worst == OFSC_ERR_NOT_CONVERGED)) worst = rs;
  }
  return result_error(worst, who);
}

}  // namespace
}  // namespace ofsc

extern "C" ofsc_status ofsc_iterate_batched(int32_t count, ofsc_graph* const* graphs, int32_t method,
                                            const int32_t* ks, float* const* Xs, double tol, int32_t maxit,
                                            const ofsc_opts* opts, ofsc_result* outs, void* stream_) {
  clear_error();
  if (count < 0) return fail(OFSC_ERR_INVALID_ARG, "ofsc_iterate_batched: count < 0");
  if (count > 0 && (!graphs || !ks || !Xs)) return fail(OFSC_ERR_INVALID_ARG, "ofsc_iterate_batched: NULL array");
  ofsc_opts o{};
  if (opts) o = *opts;
  if (o.trace || o.profile)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_iterate_batched: opts.trace and opts.profile must be NULL");
  if (opts && opts->state)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_iterate_batched: opts.state must be NULL (one state per call)");
  for (int i = 0; i < count; ++i) {
    ofsc_status st = check_iterate_args(graphs[i], method, ks[i], Xs[i], tol, maxit, o, "ofsc_iterate_batched");
    if (st != OFSC_OK) return st;
    for (int j = 0; j < i; ++j)
      if (graphs[j] == graphs[i]) return fail(OFSC_ERR_INVALID_ARG, "ofsc_iterate_batched: graph %d repeats graph %d", i, j);
  }
  if (outs)
    for (int i = 0; i < count; ++i) outs[i] = ofsc_result{0, OFSC_OK, 0.0, 0.0, 0.0, 0, -1, -1};
  return bounds_checked(iterate_lockstep(count, graphs, method, ks, Xs, tol, maxit, o, outs, (cudaStream_t)stream_,
                                         "ofsc_iterate_batched"),
                        "ofsc_iterate_batched");
}

// ==========================================================================================
// ofsc_objective_grad_noalloc: the objective and gradient with no device allocation.
//
// Some callers must not allocate device memory while they run: a process whose device memory is
// already reserved by another allocator (a framework's caching pool) would see cudaMalloc fail,
// and latency-bound loops cannot afford the driver call and the implicit synchronisation that
// cudaMalloc/cudaFree bring. This variant takes all of its temporary storage from one
// file-scope static device array instead of the graph handle's workspace.
//
// Limits: n * kp <= 2^20 (kp = k rounded up to a multiple of 8, k <= 128); the array holds
// kNoAllocBytes (about 30 MiB) on every GPU that loads the library, until the process exits.
// The first call on a device looks the array's address up (cudaGetSymbolAddress) with that
// device current; make that first call before any stream capture. The address is cached per
// device for the life of the process: after a cudaDeviceReset of a device, this entry point must
// not be called on it again. The graph must live on the current device. Every call shares the one
// array and it keeps the last call's contents, so calls that overlap on the GPU (other streams,
// other host threads) race; order them. Nothing read by a call depends on earlier contents: the
// control block, the padded copy of X and every partial sum are written before they are read.
// ==========================================================================================

namespace ofsc {
namespace {

constexpr int64_t kNoAllocMaxBlock = int64_t(1) << 20;  // n * kp elements
constexpr int kNoAllocGramGroups = 8;                    // row groups of the Gram partials
constexpr size_t kNoAllocAlign = 256;
constexpr size_t al256(size_t b) { return (b + kNoAllocAlign - 1) / kNoAllocAlign * kNoAllocAlign; }
constexpr size_t kNoAllocCtrl = al256(sizeof(Ctrl));
constexpr size_t kNoAllocBlockBytes = al256((size_t)kNoAllocMaxBlock * sizeof(float));
constexpr size_t kNoAllocGramPart = al256((size_t)kNoAllocGramGroups * kPairs * kMaxK * kMaxK * sizeof(double));
constexpr size_t kNoAllocGram = al256((size_t)kPairs * kMaxK * kMaxK * sizeof(double));
constexpr size_t kNoAllocKK = al256((size_t)kMaxK * kMaxK * sizeof(float));
constexpr size_t kNoAllocColpart = al256((size_t)kMaxRowBlocks * kColSums * kMaxK * sizeof(double));
constexpr size_t kNoAllocBytes = kNoAllocCtrl + 4 * kNoAllocBlockBytes + kNoAllocGramPart +
                                 kNoAllocGram + 2 * kNoAllocKK + kNoAllocColpart;

}  // namespace
}  // namespace ofsc

static __device__ __align__(256) unsigned char g_noalloc_scratch[ofsc::kNoAllocBytes];

namespace ofsc {
namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device `dev` (looked up once per device; the
// cached address belongs to that device's primary context, so it does not survive a
// cudaDeviceReset of the device).
ofsc_status noalloc_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_objective_grad_noalloc: device %d not supported", dev);
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
    g_noalloc_ptr[dev] = p;
  }
  *out = g_noalloc_ptr[dev];
  return OFSC_OK;
}

}  // namespace
}  // namespace ofsc

extern "C" ofsc_status ofsc_objective_grad_noalloc(const ofsc_graph* gc, int32_t objective, int32_t k,
                                                   const float* X, double* f_out, float* G_out,
                                                   void* stream_) {
  clear_error();
  if (!gc) return fail(OFSC_ERR_INVALID_ARG, "ofsc_objective_grad_noalloc: graph is NULL");
  if (objective != OFSC_F1 && objective != OFSC_F2)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_objective_grad_noalloc: objective must be OFSC_F1 or OFSC_F2");
  if (k < 1 || k > kMaxK)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_objective_grad_noalloc: k=%d outside [1, %d]", k, kMaxK);
  const int kp = round_up(k, 8);
  if (gc->n * kp > kNoAllocMaxBlock)
    return fail(OFSC_ERR_INVALID_ARG,
                "ofsc_objective_grad_noalloc: n * kp = %lld exceeds the static scratch limit of %lld "
                "elements (use ofsc_objective_grad)", (long long)(gc->n * kp), (long long)kNoAllocMaxBlock);
  if (gc->n > 0 && !X) return fail(OFSC_ERR_INVALID_ARG, "ofsc_objective_grad_noalloc: X is NULL");
  cudaStream_t s = (cudaStream_t)stream_;
  if (gc->n == 0) {
    if (f_out) *f_out = 0.0;
    return OFSC_OK;
  }
  int dev = 0;
  OFSC_CUDA(cudaGetDevice(&dev));
  if (dev != gc->device)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_objective_grad_noalloc: the current device is %d, the graph's is %d",
                dev, gc->device);
  void* base = nullptr;
  ofsc_status st = noalloc_scratch(dev, &base);
  if (st != OFSC_OK) return st;
  unsigned char* p = (unsigned char*)base;
  Workspace ws;  // views into the static array; owns nothing
  ws.n = gc->n;
  ws.kp = kp;
  ws.ctrl = (Ctrl*)p;
  p += kNoAllocCtrl;
  ws.X = (float*)p;
  p += kNoAllocBlockBytes;
  ws.Y = (float*)p;
  p += kNoAllocBlockBytes;
  ws.G = (float*)p;
  p += kNoAllocBlockBytes;
  ws.Vh = p;
  p += kNoAllocBlockBytes;
  ws.gram_part = (double*)p;
  p += kNoAllocGramPart;
  ws.gram = (double*)p;
  p += kNoAllocGram;
  ws.Rn = (float*)p;
  p += kNoAllocKK;
  ws.Bn = (float*)p;
  p += kNoAllocKK;
  ws.colpart = (double*)p;

  ofsc_graph* g = const_cast<ofsc_graph*>(gc);  // read only: the CSR and D^-1/2
  const int method = objective == OFSC_F1 ? M_OFM_F1 : M_OFM_F2;
  Prof prof{ws, nullptr, s};
  Runner run{g, ws, s, method, false, prof};
  k_init_ctrl<<<1, 1, 0, s>>>(ws.ctrl, 0.0, 0, k, g->normA2, 0);
  k_pad_in<<<grid_elems(g->n * kp), 256, 0, s>>>(g->n, k, kp, X, ws.X, ws.ctrl);
  OFSC_LAUNCH_CHECK("noalloc: k_pad_in");
  // A X exactly, then X^T X and X^T A X with at most kNoAllocGramGroups row groups
  SpmmArgs a = run.spmm_base();
  a.gather = ws.X;
  a.base = ws.X;
  a.out = ws.Y;
  launch_spmm(a, g->weighted != 0, s);
  GramArgs ga;
  ga.n = ws.n;
  ga.kp = kp;
  ga.npairs = 2;
  ga.nt = gram_nt_for(kp);
  ga.pairs = GramPairs{};
  ga.pairs.L[0] = ws.X; ga.pairs.R[0] = ws.X; ga.pairs.slot[0] = G_R;
  ga.pairs.L[1] = ws.X; ga.pairs.R[1] = ws.Y; ga.pairs.slot[1] = G_B;
  int64_t rpg = ceil_div(ceil_div(ws.n, kNoAllocGramGroups), kGramChunk) * kGramChunk;
  const int gy = (int)ceil_div(ws.n, rpg);
  ga.rows_per_group = rpg;
  ga.part = ws.gram_part;
  ga.ctrl = ws.ctrl;
  ga.ignore_done = 0;
  dim3 grid(2 * ga.nt * ga.nt, gy);
  switch (gram_m_for(kp)) {
    case 1: k_gram<1><<<grid, 256, 0, s>>>(ga); break;
    case 2: k_gram<2><<<grid, 256, 0, s>>>(ga); break;
    default: k_gram<4><<<grid, 256, 0, s>>>(ga); break;
  }
  GramReduceArgs ra{};
  ra.part = ws.gram_part;
  ra.gy = gy;
  ra.kp = kp;
  ra.slot_mask = (1 << G_R) | (1 << G_B);
  ra.gram = ws.gram;
  ra.ctrl = ws.ctrl;
  ra.ignore_done = 0;
  k_gram_reduce<<<(int)std::min<int64_t>(ceil_div(kPairs * kp * kp, 32), 8 * kNumSMs), 256, 0, s>>>(ra);
  k_set_rb<<<1, 256, 0, s>>>(ws.gram, kp, objective, ws.Rn, ws.Bn, nullptr, nullptr, ws.ctrl, 0);
  OFSC_LAUNCH_CHECK("noalloc: refresh");
  int nblk = 0;
  OFSC_CUDA(run.rowpass(method, 0, 1, 0, &nblk));
  if (G_out) {
    k_pad_out<<<grid_elems(g->n * k), 256, 0, s>>>(g->n, k, kp, ws.G, G_out);
    OFSC_LAUNCH_CHECK("noalloc: k_pad_out");
  }
  Ctrl c{};
  OFSC_CUDA(cudaMemcpyAsync(&c, ws.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s));
  OFSC_CUDA(cudaStreamSynchronize(s));
  if (c.status != OFSC_OK) return fail(c.status, "ofsc_objective_grad_noalloc: non-finite value in X");
  if (!std::isfinite(c.f)) return fail(OFSC_ERR_NONFINITE, "ofsc_objective_grad_noalloc: non-finite objective");
  if (f_out) *f_out = c.f;
  return OFSC_OK;
}

// ==========================================================================================
// The CG state between calls (opts.state): create, free, and its host image (a checkpoint).
// ==========================================================================================

namespace {

struct StateHeader {
  uint64_t magic;  // "OFSCSTAT"
  int64_t n, t;
  int32_t k, kp, method, reserved;
  double g0;
};
constexpr uint64_t kStateMagic = 0x5441545343534f46ull;

int64_t state_bytes(const ofsc_state* st) {
  return (int64_t)sizeof(StateHeader) + 2 * st->n * st->kp * (int64_t)sizeof(float) +
         ((int64_t)st->kp + (int64_t)st->kp * st->kp) * (int64_t)sizeof(double);
}

}  // namespace

extern "C" ofsc_status ofsc_state_create(const ofsc_graph* g, int32_t k, ofsc_state** out) {
  clear_error();
  if (!out) return fail(OFSC_ERR_INVALID_ARG, "ofsc_state_create: out is NULL");
  *out = nullptr;
  if (!g) return fail(OFSC_ERR_INVALID_ARG, "ofsc_state_create: graph is NULL");
  if (k < 1 || k > kMaxK) return fail(OFSC_ERR_INVALID_ARG, "ofsc_state_create: k=%d outside [1, %d]", k, kMaxK);
  ofsc_state* st = new ofsc_state();
  st->n = g->n;
  st->k = k;
  st->kp = round_up(k, 8);
  cudaGetDevice(&st->device);
  const size_t blk = (size_t)std::max<int64_t>(g->n, 1) * st->kp * sizeof(float);
  cudaError_t e = dev_alloc(&st->V, blk);
  if (e == cudaSuccess) e = dev_alloc(&st->G, blk);
  if (e == cudaSuccess) e = dev_alloc(&st->vscale, (size_t)st->kp * sizeof(double));
  if (e == cudaSuccess) e = dev_alloc(&st->Q, (size_t)st->kp * st->kp * sizeof(double));
  if (e != cudaSuccess) {
    ofsc_state_free(st);
    return cuda_fail(e, "ofsc_state_create");
  }
  *out = st;
  return OFSC_OK;
}

extern "C" ofsc_status ofsc_state_free(ofsc_state* st) {
  clear_error();
  if (!st) return OFSC_OK;
  dev_free(st->V);
  dev_free(st->G);
  dev_free(st->vscale);
  dev_free(st->Q);
  delete st;
  return OFSC_OK;
}

extern "C" ofsc_status ofsc_state_info(const ofsc_state* st, int64_t* t_out, int64_t* bytes_out) {
  clear_error();
  if (!st) return fail(OFSC_ERR_INVALID_ARG, "ofsc_state_info: state is NULL");
  if (t_out) *t_out = st->t;
  if (bytes_out) *bytes_out = state_bytes(st);
  return OFSC_OK;
}

extern "C" ofsc_status ofsc_state_save(const ofsc_state* st, void* host, int64_t bytes, void* stream_) {
  clear_error();
  if (!st || !host) return fail(OFSC_ERR_INVALID_ARG, "ofsc_state_save: NULL argument");
  if (bytes != state_bytes(st))
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_state_save: %lld bytes, the image takes %lld", (long long)bytes,
                (long long)state_bytes(st));
  cudaStream_t s = (cudaStream_t)stream_;
  StateHeader h{kStateMagic, st->n, st->t, st->k, st->kp, st->method, 0, st->g0};
  unsigned char* p = (unsigned char*)host;
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  const size_t blk = (size_t)st->n * st->kp * sizeof(float);
  OFSC_CUDA(cudaMemcpyAsync(p, st->V, blk, cudaMemcpyDeviceToHost, s));
  OFSC_CUDA(cudaMemcpyAsync(p + blk, st->G, blk, cudaMemcpyDeviceToHost, s));
  OFSC_CUDA(cudaMemcpyAsync(p + 2 * blk, st->vscale, (size_t)st->kp * sizeof(double), cudaMemcpyDeviceToHost, s));
  OFSC_CUDA(cudaMemcpyAsync(p + 2 * blk + st->kp * sizeof(double), st->Q, (size_t)st->kp * st->kp * sizeof(double),
                            cudaMemcpyDeviceToHost, s));
  OFSC_CUDA(cudaStreamSynchronize(s));
  return OFSC_OK;
}

extern "C" ofsc_status ofsc_state_load(ofsc_state* st, const void* host, int64_t bytes, void* stream_) {
  clear_error();
  if (!st || !host) return fail(OFSC_ERR_INVALID_ARG, "ofsc_state_load: NULL argument");
  if (bytes != state_bytes(st))
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_state_load: %lld bytes, the image takes %lld", (long long)bytes,
                (long long)state_bytes(st));
  StateHeader h;
  std::memcpy(&h, host, sizeof(h));
  if (h.magic != kStateMagic || h.n != st->n || h.k != st->k || h.kp != st->kp || h.t < 0 ||
      (h.t > 0 && (h.method < OFSC_OFM_F1 || h.method > OFSC_TRI_F2)))
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_state_load: not a state image for n=%lld, k=%d", (long long)st->n, st->k);
  cudaStream_t s = (cudaStream_t)stream_;
  const unsigned char* p = (const unsigned char*)host + sizeof(h);
  const size_t blk = (size_t)st->n * st->kp * sizeof(float);
  OFSC_CUDA(cudaMemcpyAsync(st->V, p, blk, cudaMemcpyHostToDevice, s));
  OFSC_CUDA(cudaMemcpyAsync(st->G, p + blk, blk, cudaMemcpyHostToDevice, s));
  OFSC_CUDA(cudaMemcpyAsync(st->vscale, p + 2 * blk, (size_t)st->kp * sizeof(double), cudaMemcpyHostToDevice, s));
  OFSC_CUDA(cudaMemcpyAsync(st->Q, p + 2 * blk + st->kp * sizeof(double), (size_t)st->kp * st->kp * sizeof(double),
                            cudaMemcpyHostToDevice, s));
  OFSC_CUDA(cudaStreamSynchronize(s));
  st->t = h.t;
  st->method = h.method;
  st->g0 = h.g0;
  return OFSC_OK;
}
