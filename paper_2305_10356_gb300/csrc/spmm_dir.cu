// The direction product of one update of Algorithm 2 (the sparse product of Sec. 3.3):
// W = A V = -V - D^-1/2 S D^-1/2 V with A = L - 2I (Eq. (1)), gathering Vh = D^-1/2 V.
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "group.cuh"

namespace ofsc {
namespace {

#if OFSC_DEBUG
// Checked build: the first out-of-range access the direction product met, (kind << 60) | value
// (kind 1: a column index outside [0, n), value the index; kind 2: a warp's row or nonzero range
// outside the CSR, value the warp), 0 if none. Read and cleared by spmm_dir_take_bounds.
__device__ unsigned long long g_bounds_bad = 0ull;
__device__ __forceinline__ void bounds_bad(unsigned kind, long long value) {
  atomicCAS(&g_bounds_bad, 0ull, ((unsigned long long)kind << 60) | ((unsigned long long)value & ((1ull << 60) - 1)));
}
#endif

#ifndef OFSC_ROW_U32
#define OFSC_ROW_U32 8  // gathers in flight per lane when a warp covers a row of 128 columns
#endif
#ifndef OFSC_ROW_WARPS_F32
#define OFSC_ROW_WARPS_F32 32  // resident warps per SM the registers must allow (FP32 slots)
#endif
#ifndef OFSC_ROW_U16_BF16
#define OFSC_ROW_U16_BF16 6  // gathers in flight per lane for 16-byte BF16 slots (128 columns)
#endif
// Weighted graphs load an FP32 value beside every column index: fewer slots keep them in the
// same 64 registers without spilling.
#ifndef OFSC_ROW_U32_W
#define OFSC_ROW_U32_W 8
#endif
#ifndef OFSC_ROW_U16_BF16_W
#define OFSC_ROW_U16_BF16_W 6
#endif
#ifndef OFSC_ROW_WARPS_BF16
#define OFSC_ROW_WARPS_BF16 32  // resident warps per SM the registers must allow (BF16 slots)
#endif


// W = A V = -V - D^-1/2 S Vh for a direction V (or AX from Xh = D^-1/2 X), with the fused
// per-block partial sums of diag(V^T AV). A warp owns a contiguous, nnz-balanced range of rows
// and takes one row at a time, so its control flow is uniform: LPN lanes per nonzero hold four
// columns each, NPI = 32 / LPN nonzeros are gathered side by side and U of those slots per lane
// are in flight together (STEP = U NPI <= 32 nonzeros per step; a short row's last step is
// predicated, not split). The STEP column indices of a step are loaded one per lane and handed
// out by shuffle; those of the next step (at a row end, of the next row) are loaded while the
// current gathers are in flight, and a row's epilogue operands (its row of V, its D^-1/2 entry)
// are loaded with the gathers of its last step (staging them through shared memory with cp.async
// measured 12% slower). Each lane sums its slots in nonzero order; the NPI partial sums of a row
// are combined by an xor-shuffle butterfly, which leaves the same bits in every lane (for LPN = 32
// the sum is in plain nonzero order). Each warp writes its own row of partials (no block-wide
// barrier, so a block is never held by its slowest warp's reduction); k_dots_fold folds them.
// One gathered slot of VPL consecutive values of a row of Vh, kept raw (FP32: float4; BF16: 8
// values in a uint4) until it is accumulated, so a slot in flight costs four registers.
template <int VPL, bool BF16>
struct Slot;
template <>
struct Slot<4, false> {
  using Raw = float4;
  static __device__ __forceinline__ Raw load(const void* p, int64_t row, int kp, int c) {
    return __ldg((const float4*)((const float*)p + row * kp + c));
  }
  static __device__ __forceinline__ Raw zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ void fma(float* acc, float w, const Raw& r) {
    acc[0] = fmaf(w, r.x, acc[0]);
    acc[1] = fmaf(w, r.y, acc[1]);
    acc[2] = fmaf(w, r.z, acc[2]);
    acc[3] = fmaf(w, r.w, acc[3]);
  }
};
template <>
struct Slot<8, true> {
  using Raw = uint4;
  static __device__ __forceinline__ Raw load(const void* p, int64_t row, int kp, int c) {
    return __ldg((const uint4*)((const __nv_bfloat16*)p + row * kp + c));
  }
  static __device__ __forceinline__ Raw zero() { return make_uint4(0u, 0u, 0u, 0u); }
  static __device__ __forceinline__ void fma(float* acc, float w, const Raw& r) {
    const uint32_t u[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (w == 1.0f) {  // binary S (a compile-time 1): add each BF16 half straight into FP32
        // add.f32.bf16 widens exactly and rounds once, the same bits as widening then fmaf(1, x,
        // acc), without the shift and mask that unpacking takes per value
        float lo_acc = acc[2 * i], hi_acc = acc[2 * i + 1];
        asm("{ .reg .b16 lo, hi;\n mov.b32 {lo, hi}, %2;\n add.rn.f32.bf16 %0, lo, %0;\n"
            " add.rn.f32.bf16 %1, hi, %1;\n}"
            : "+f"(lo_acc), "+f"(hi_acc)
            : "r"(u[i]));
        acc[2 * i] = lo_acc;
        acc[2 * i + 1] = hi_acc;
        continue;
      }
      const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u[i]));
      acc[2 * i] = fmaf(w, f.x, acc[2 * i]);
      acc[2 * i + 1] = fmaf(w, f.y, acc[2 * i + 1]);
    }
  }
};

// Slots in flight per lane: FP32 rows use 4 values per lane, BF16 rows 8 (16-byte loads), so a
// warp holds twice as many BF16 rows in flight in the same registers.
template <int LPN, int VPL, bool WEIGHTED>
__host__ __device__ constexpr int dir_slots() {
  return VPL == 4 ? (LPN == 32 ? (WEIGHTED ? OFSC_ROW_U32_W : OFSC_ROW_U32) : LPN == 16 ? 4 : 2)
                  : (LPN == 16 ? (WEIGHTED ? OFSC_ROW_U16_BF16_W : OFSC_ROW_U16_BF16) : LPN == 8 ? 4 : 2);
}

// UU: gathers in flight per lane (0: the default of dir_slots; other values are the shapes the
// autotuner may pick). MP: the warps take the merge-path shares a.mp (a long row can span warps;
// the partial sums of a row a warp does not both start and finish go to a.carry).
#define OFSC_DIR_BOUNDS \
  __launch_bounds__(32 * kRowWarpsPerBlock, (VPL == 4 ? OFSC_ROW_WARPS_F32 : OFSC_ROW_WARPS_BF16) / kRowWarpsPerBlock)

template <int LPN, int VPL, bool WEIGHTED, bool BF16, bool DOTS, int UU, bool MP>
__global__ void OFSC_DIR_BOUNDS k_spmm_dir(SpmmArgs a) {
#define OFSC_VB_X blockIdx.x
#include "spmm_dir_body.inc"
#undef OFSC_VB_X
}

// The same product for every graph of a batch in one launch (see group.cuh).
template <int LPN, int VPL, bool WEIGHTED, bool BF16, bool DOTS, int UU, bool MP>
__global__ void OFSC_DIR_BOUNDS k_spmm_dir_g(const __grid_constant__ GroupParams<SpmmArgs> p) {
  VBlock vb;
  const SpmmArgs& a = group_find(p, &vb);
#define OFSC_VB_X ((unsigned)vb.x)
#include "spmm_dir_body.inc"
#undef OFSC_VB_X
}
#undef OFSC_DIR_BOUNDS

// Rows split across warps by the merge-path shares: the warp that starts a row and leaves it
// unfinished adds, in warp order, its partial sums and those of the following warps up to the one
// that finishes the row, then writes W = -V - D^-1/2 (sum) for the row and adds the row's share of
// diag(V^T AV) to its own row of dots partials. One warp per warp of the product, four columns
// per lane (kp <= 128).
__device__ __forceinline__ void spmm_fixup_body(const SpmmArgs& a, const VBlock vb) {
  if (!a.ignore_done && a.ctrl->done) return;
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)vb.x * 8 + (threadIdx.x >> 5);
  if (w >= a.groups) return;
  const int64_t r = a.carry_row[2 * w + 1];
  if (r < 0) return;  // no row that this warp started and left unfinished
  const int c = lane * 4;
  const bool active = c < a.kp;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (active) acc = *(const float4*)(a.carry + (2 * w + 1) * a.kp + c);
  for (int64_t w2 = w + 1; w2 < a.groups; ++w2) {
    const bool mid = a.carry_row[2 * w2 + 1] == -(r + 2);  // a share inside the row
    const int64_t slot = mid ? 2 * w2 + 1 : 2 * w2;
    if (!mid && a.carry_row[2 * w2] != r) break;
    if (active) {
      const float4 v = *(const float4*)(a.carry + slot * a.kp + c);
      acc = make_float4(acc.x + v.x, acc.y + v.y, acc.z + v.z, acc.w + v.w);
    }
    if (!mid) break;  // the warp that finishes the row
  }
  if (!active) return;
  const float sr = a.dinv[r];
  const float4 b = *(const float4*)(a.base + r * a.kp + c);
  const float4 o = make_float4(-fmaf(sr, acc.x, b.x), -fmaf(sr, acc.y, b.y), -fmaf(sr, acc.z, b.z),
                               -fmaf(sr, acc.w, b.w));
  *(float4*)(a.out + r * a.kp + c) = o;
  if (a.dots) {
    double* d = a.dots + w * a.kp + c;
    d[0] += (double)b.x * (double)o.x;
    d[1] += (double)b.y * (double)o.y;
    d[2] += (double)b.z * (double)o.z;
    d[3] += (double)b.w * (double)o.w;
  }
}

__global__ void __launch_bounds__(256) k_spmm_fixup(const __grid_constant__ SpmmArgs a) { spmm_fixup_body(a, hw_block()); }

__global__ void __launch_bounds__(256) k_spmm_fixup_g(const __grid_constant__ GroupParams<SpmmArgs> p) {
  VBlock vb;
  const SpmmArgs& a = group_find(p, &vb);
  spmm_fixup_body(a, vb);
}

// mp[w] = first row and mp[warps + 1 + w] = first nonzero of warp w's share of the merged list of
// row ends and nonzeros: the point (i, d - i) of diagonal d = w (n + nnz) / warps, with i the
// number of rows whose end, row_ptr[i + 1] + i in merged order, lies before d.
__global__ void k_merge_partition(int64_t n, const int64_t* __restrict__ row_ptr, int warps, int64_t* __restrict__ mp) {
  const int64_t total = n + row_ptr[n];
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w <= warps; w += gridDim.x * blockDim.x) {
    const int64_t d = total * w / warps;
    int64_t lo = 0, hi = n;  // first i in [0, n] with row_ptr[i + 1] + i >= d (i = n if none)
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (row_ptr[mid + 1] + mid < d) lo = mid + 1;
      else hi = mid;
    }
    mp[w] = lo;
    mp[warps + 1 + w] = d - lo;
  }
}

__global__ void k_max_row(int64_t n, const int64_t* __restrict__ row_ptr, unsigned long long* out) {
  unsigned long long m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)(row_ptr[i + 1] - row_ptr[i]));
  for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(out, m);
}

template <int LPN, int VPL, bool WEIGHTED, bool BF16, bool DOTS, int UU, bool MP>
void launch_dir_u(const SpmmArgs& a, cudaStream_t s) {
  if (DOTS) {  // the iteration's product (the one a replayed update holds) can run grouped
    OFSC_GROUPABLE((k_spmm_dir<LPN, VPL, WEIGHTED, BF16, DOTS, UU, MP>),
                   (k_spmm_dir_g<LPN, VPL, WEIGHTED, BF16, DOTS, UU, MP>), SpmmArgs);
    if (MP) OFSC_GROUPABLE(k_spmm_fixup, k_spmm_fixup_g, SpmmArgs);
  }
  k_spmm_dir<LPN, VPL, WEIGHTED, BF16, DOTS, UU, MP><<<a.groups / kRowWarpsPerBlock, 32 * kRowWarpsPerBlock, 0, s>>>(a);
  if (MP) k_spmm_fixup<<<(a.groups + 7) / 8, 256, 0, s>>>(a);
}

// A tuned number of slots in flight (u = 2, 4, 6, 8) only for the product with dots (the direction
// product of the iteration); u must keep u * 32 / LPN <= 32 nonzeros per step, else the default.
// The merge-path form (a.mp set) takes the default number of slots.
template <int LPN, int VPL, bool WEIGHTED, bool BF16>
void launch_dir_w(const SpmmArgs& a, bool dots, int u, cudaStream_t s) {
  constexpr int NPI = 32 / LPN;
  if (a.mp) {
    if (dots) launch_dir_u<LPN, VPL, WEIGHTED, BF16, true, 0, true>(a, s);
    else launch_dir_u<LPN, VPL, WEIGHTED, BF16, false, 0, true>(a, s);
    return;
  }
  if (!dots) return launch_dir_u<LPN, VPL, WEIGHTED, BF16, false, 0, false>(a, s);
  if (u == 2) return launch_dir_u<LPN, VPL, WEIGHTED, BF16, true, 2, false>(a, s);
  if constexpr (4 * NPI <= 32)
    if (u == 4) return launch_dir_u<LPN, VPL, WEIGHTED, BF16, true, 4, false>(a, s);
  if constexpr (6 * NPI <= 32)
    if (u == 6) return launch_dir_u<LPN, VPL, WEIGHTED, BF16, true, 6, false>(a, s);
  if constexpr (8 * NPI <= 32)
    if (u == 8) return launch_dir_u<LPN, VPL, WEIGHTED, BF16, true, 8, false>(a, s);
  launch_dir_u<LPN, VPL, WEIGHTED, BF16, true, 0, false>(a, s);
}

template <int LPN, int VPL, bool BF16>
void launch_dir_l(const SpmmArgs& a, bool weighted, int u, cudaStream_t s) {
  const bool dots = a.dots != nullptr;
  if (weighted) launch_dir_w<LPN, VPL, true, BF16>(a, dots, u, s);
  else launch_dir_w<LPN, VPL, false, BF16>(a, dots, u, s);
}

template <int LPN, int VPL>
int default_slots(bool weighted) {
  return weighted ? dir_slots<LPN, VPL, true>() : dir_slots<LPN, VPL, false>();
}

}  // namespace

// Lanes per nonzero of the direction product: rows of kp values, VPL per lane, a power of two
// of at least 2.
int dir_lanes(int kp, int vpl) {
  int l = 2;
  while (l * vpl < kp) l *= 2;
  return l;
}

int dir_default_slots(int kp, bool bf16, bool weighted) {
  if (bf16) {
    switch (dir_lanes(kp, 8)) {
      case 2: return default_slots<2, 8>(weighted);
      case 4: return default_slots<4, 8>(weighted);
      case 8: return default_slots<8, 8>(weighted);
      default: return default_slots<16, 8>(weighted);
    }
  }
  switch (dir_lanes(kp, 4)) {
    case 2: return default_slots<2, 4>(weighted);
    case 4: return default_slots<4, 4>(weighted);
    case 8: return default_slots<8, 4>(weighted);
    case 16: return default_slots<16, 4>(weighted);
    default: return default_slots<32, 4>(weighted);
  }
}

int dir_slot_options(int kp, bool bf16, int* out) {
  const int lpn = dir_lanes(kp, bf16 ? 8 : 4), npi = 32 / lpn;
  int n = 0;
  for (int u = 2; u <= 8; u += 2)
    if (u * npi <= 32) out[n++] = u;
  return n;
}

cudaError_t merge_partition(int64_t n, const int64_t* row_ptr, int warps, int64_t* mp, cudaStream_t s) {
  k_merge_partition<<<(warps + 256) / 256, 256, 0, s>>>(n, row_ptr, warps, mp);
  return cudaGetLastError();
}

cudaError_t max_row_length(int64_t n, const int64_t* row_ptr, unsigned long long* max_row, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4 * kNumSMs);
  k_max_row<<<(int)blocks, 256, 0, s>>>(n, row_ptr, max_row);
  return cudaGetLastError();
}

cudaError_t spmm_dir_take_bounds(unsigned long long* code) {
  *code = 0;
#if OFSC_DEBUG
  cudaError_t e = cudaMemcpyFromSymbol(code, g_bounds_bad, sizeof(*code));
  if (e == cudaSuccess && *code) {
    const unsigned long long zero = 0;
    e = cudaMemcpyToSymbol(g_bounds_bad, &zero, sizeof(zero));
  }
  return e;
#else
  return cudaSuccess;
#endif
}

int launch_spmm_dir(const SpmmArgs& a, bool weighted, bool bf16, int slots, cudaStream_t s) {
  if (bf16) {
    switch (dir_lanes(a.kp, 8)) {
      case 2: launch_dir_l<2, 8, true>(a, weighted, slots, s); break;
      case 4: launch_dir_l<4, 8, true>(a, weighted, slots, s); break;
      case 8: launch_dir_l<8, 8, true>(a, weighted, slots, s); break;
      default: launch_dir_l<16, 8, true>(a, weighted, slots, s); break;
    }
  } else {
    switch (dir_lanes(a.kp, 4)) {
      case 2: launch_dir_l<2, 4, false>(a, weighted, slots, s); break;
      case 4: launch_dir_l<4, 4, false>(a, weighted, slots, s); break;
      case 8: launch_dir_l<8, 4, false>(a, weighted, slots, s); break;
      case 16: launch_dir_l<16, 4, false>(a, weighted, slots, s); break;
      default: launch_dir_l<32, 4, false>(a, weighted, slots, s); break;
    }
  }
  return a.groups;
}

}  // namespace ofsc
