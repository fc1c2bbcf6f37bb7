// AV = -V - D^-1/2 S (D^-1/2 V) (the sparse product of Sec. 3.3) with the rows of D^-1/2 V
// gathered by the tensor memory accelerator (cp.async.bulk.tensor ... tile::gather4).
//
// Each warp owns a contiguous, nnz-balanced range of rows and streams its nonzeros four at a
// time: lane 0 issues one gather4 per 4 nonzeros (4 rows of k values, BF16 or FP32) into a ring of
// shared-memory slots, each with its own mbarrier, kTmaStages slots ahead of the consumer. All 32
// lanes then read their k/32 columns of the 4 rows from shared memory and accumulate them into
// the current row; when the stream passes a row's end the warp writes AV for that row and adds
// its terms of diag(V^T AV) to its partial sums. Deep memory-level parallelism therefore
// costs no registers. Every mbarrier wait is bounded (OFSC_ERR_TIMEOUT on expiry).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"

namespace ofsc {
namespace {

constexpr int kTmaWarps = 4;
constexpr int kTmaStages = 8;
constexpr long long kTmaSpin = 1ll << 22;

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool bar_wait(uint64_t* bar, uint32_t parity, long long limit) {
  const uint32_t addr = smem_addr(bar);
  for (long long it = 0; it < limit; ++it) {
    uint32_t ok;
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n"
        "}\n"
        : "=r"(ok)
        : "r"(addr), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

template <int CPL, bool BF16>
struct RowSlice;  // one lane's CPL consecutive values of a row in shared memory, as FP32
template <>
struct RowSlice<4, true> {
  static __device__ __forceinline__ void fma(const unsigned char* row, int lane, float w, float* acc) {
    const uint2 u = *(const uint2*)(row + lane * 8);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
    const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
    acc[0] = fmaf(w, a.x, acc[0]);
    acc[1] = fmaf(w, a.y, acc[1]);
    acc[2] = fmaf(w, b.x, acc[2]);
    acc[3] = fmaf(w, b.y, acc[3]);
  }
};
template <>
struct RowSlice<4, false> {
  static __device__ __forceinline__ void fma(const unsigned char* row, int lane, float w, float* acc) {
    const float4 v = *(const float4*)(row + lane * 16);
    acc[0] = fmaf(w, v.x, acc[0]);
    acc[1] = fmaf(w, v.y, acc[1]);
    acc[2] = fmaf(w, v.z, acc[2]);
    acc[3] = fmaf(w, v.w, acc[3]);
  }
};
template <>
struct RowSlice<2, true> {
  static __device__ __forceinline__ void fma(const unsigned char* row, int lane, float w, float* acc) {
    const uint32_t u = *(const uint32_t*)(row + lane * 4);
    const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u));
    acc[0] = fmaf(w, a.x, acc[0]);
    acc[1] = fmaf(w, a.y, acc[1]);
  }
};
template <>
struct RowSlice<2, false> {
  static __device__ __forceinline__ void fma(const unsigned char* row, int lane, float w, float* acc) {
    const float2 v = *(const float2*)(row + lane * 8);
    acc[0] = fmaf(w, v.x, acc[0]);
    acc[1] = fmaf(w, v.y, acc[1]);
  }
};

template <int CPL>
__device__ __forceinline__ void ldg_cpl(const float* p, float* o) {
  if constexpr (CPL == 4) {
    const float4 v = *(const float4*)p;
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
  } else {
    const float2 v = *(const float2*)p;
    o[0] = v.x; o[1] = v.y;
  }
}

template <int CPL>
__device__ __forceinline__ void stg_cpl(float* p, const float* v) {
  if constexpr (CPL == 4) *(float4*)p = make_float4(v[0], v[1], v[2], v[3]);
  else *(float2*)p = make_float2(v[0], v[1]);
}

template <int CPL, bool BF16, bool WEIGHTED>
__global__ void __launch_bounds__(kTmaWarps * 32) k_spmm_tma(const __grid_constant__ CUtensorMap tmap, TmaSpmmArgs a) {
  if (a.ctrl->done) return;
  const long long lim = a.ctrl->spin_limit > 0 ? a.ctrl->spin_limit : kTmaSpin;
  constexpr int KP = CPL * 32;
  constexpr int ROWB = KP * (BF16 ? 2 : 4);
  constexpr int SLOT = 4 * ROWB;
  extern __shared__ unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[kTmaWarps][kTmaStages];
  __shared__ float dred[kTmaWarps][KP];
  __shared__ int abort_flag;
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  unsigned char* ring = base + (size_t)warp * kTmaStages * SLOT;
  uint64_t* bar = bars[warp];
  if (threadIdx.x == 0) abort_flag = 0;
  if (lane == 0) {
    for (int s = 0; s < kTmaStages; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&bar[s])), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();

  float dcw[CPL];
#pragma unroll
  for (int u = 0; u < CPL; ++u) dcw[u] = 0.f;
  const int c = lane * CPL;
  const int gid = blockIdx.x * kTmaWarps + warp;
  bool ok = true;
  if (gid < a.groups) {
    const int64_t ra = a.bnd[gid], rb = a.bnd[gid + 1];
    if (ra < rb) {
      const int64_t z0 = a.row_ptr[ra], z1 = a.row_ptr[rb];
      const int64_t nst = (z1 - z0 + 3) / 4;  // stages of 4 nonzeros
      // producer: column indices in windows of 32 nonzeros (the next window is loaded ahead)
      int64_t pw = -1;
      int cw_cur = 0, cw_next = 0;
      auto load_win = [&](int64_t w) -> int {
        const int64_t i = z0 + w * 32 + lane;
        return i < z1 ? __ldg(a.col + i) : 0;
      };
      auto issue = [&](int64_t s) {
        const int64_t w = (4 * s) >> 5;
        if (w != pw) {
          if (w == pw + 1 && pw >= 0) cw_cur = cw_next;
          else cw_cur = load_win(w);
          cw_next = load_win(w + 1);
          pw = w;
        }
        const int o = (int)((4 * s) & 31);
        const int j0 = __shfl_sync(0xffffffffu, cw_cur, o);
        const int j1 = __shfl_sync(0xffffffffu, cw_cur, o + 1);
        const int j2 = __shfl_sync(0xffffffffu, cw_cur, o + 2);
        const int j3 = __shfl_sync(0xffffffffu, cw_cur, o + 3);
        if (lane == 0) {
          const int slot = (int)(s % kTmaStages);
          const uint32_t b = smem_addr(&bar[slot]);
          asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(SLOT) : "memory");
          asm volatile(
              "cp.async.bulk.tensor.2d.shared::cta.global.tile::gather4.mbarrier::complete_tx::bytes "
              "[%0], [%1, {%2, %3, %4, %5, %6}], [%7];" ::"r"(smem_addr(ring + slot * SLOT)),
              "l"(&tmap), "r"(0), "r"(j0), "r"(j1), "r"(j2), "r"(j3), "r"(b)
              : "memory");
        }
      };
      // consumer state: current row, its end (window of row pointers), epilogue operands
      int64_t r = ra, wbase = ra;
      int64_t wreg = (ra + 1 + lane <= rb) ? a.row_ptr[ra + 1 + lane] : z1;
      auto row_end = [&](int64_t row) -> int64_t {
        if (row - wbase >= 32) {
          wbase = row;
          wreg = (row + 1 + lane <= rb) ? a.row_ptr[row + 1 + lane] : z1;
        }
        return __shfl_sync(0xffffffffu, wreg, (int)(row - wbase));
      };
      int64_t rend = row_end(r);
      float acc[CPL], ev[CPL];
      float es = 0.f;
      auto load_epi = [&](int64_t row) {
        es = a.dinv[row];
        const int64_t o = row * KP + c;
        ldg_cpl<CPL>(a.base + o, ev);
      };
      auto finish = [&]() {
        const int64_t o = r * KP + c;
        float w[CPL];
#pragma unroll
        for (int u = 0; u < CPL; ++u) {
          w[u] = -fmaf(es, acc[u], ev[u]);
          dcw[u] = fmaf(ev[u], w[u], dcw[u]);
          acc[u] = 0.f;
        }
        stg_cpl<CPL>(a.out + o, w);
        ++r;
        if (r < rb) {
          rend = row_end(r);
          load_epi(r);
        }
      };
#pragma unroll
      for (int u = 0; u < CPL; ++u) acc[u] = 0.f;
      load_epi(r);
      const int64_t pre = nst < kTmaStages ? nst : kTmaStages;
      for (int64_t s = 0; s < pre; ++s) issue(s);
      int64_t s = 0;
      for (; s < nst; ++s) {
        const int slot = (int)(s % kTmaStages);
        if (!bar_wait(&bar[slot], (uint32_t)((s / kTmaStages) & 1), lim)) {
          ok = false;
          break;
        }
        const unsigned char* rows = ring + slot * SLOT;
        const int64_t zs = z0 + 4 * s;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t zq = zs + q;
          if (zq >= z1) break;
          while (zq >= rend) finish();  // the stream crossed into the next row
          const float wq = WEIGHTED ? __ldg(a.val + zq) : 1.0f;
          RowSlice<CPL, BF16>::fma(rows + q * ROWB, lane, wq, acc);
        }
        __syncwarp();
        if (s + kTmaStages < nst) issue(s + kTmaStages);
      }
      if (ok) {
        while (r < rb) finish();  // the last row and any empty rows after it
      } else {
        // stop consuming, but let the copies already issued land (bounded) before the CTA exits
        const int64_t last = (s + kTmaStages < nst) ? s + kTmaStages : nst;
        for (int64_t t = s + 1; t < last; ++t)
          bar_wait(&bar[t % kTmaStages], (uint32_t)((t / kTmaStages) & 1), lim);
      }
    }
  }
  if (!ok) abort_flag = 1;
  // per-block partials of diag(V^T AV): warps in order, then columns
#pragma unroll
  for (int u = 0; u < CPL; ++u) dred[warp][c + u] = dcw[u];
  __syncthreads();
  for (int j = threadIdx.x; j < KP; j += blockDim.x) {
    double sum = 0.0;
    for (int w = 0; w < kTmaWarps; ++w) sum += (double)dred[w][j];
    a.dots[(int64_t)blockIdx.x * KP + j] = sum;
  }
  if (threadIdx.x == 0 && abort_flag) {
    a.ctrl->status = OFSC_ERR_TIMEOUT;
    a.ctrl->done = 1;
  }
}

std::mutex g_encode_mu;
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;

template <int CPL, bool BF16, bool W>
cudaError_t launch_t(const CUtensorMap& map, const TmaSpmmArgs& a, cudaStream_t s) {
  constexpr int SLOT = 4 * CPL * 32 * (BF16 ? 2 : 4);
  const size_t smem = (size_t)kTmaWarps * kTmaStages * SLOT + 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_spmm_tma<CPL, BF16, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const int grid = a.groups / kTmaWarps;
  k_spmm_tma<CPL, BF16, W><<<grid, kTmaWarps * 32, smem, s>>>(map, a);
  return cudaGetLastError();
}

}  // namespace

bool spmm_tma_supported(int kp) { return kp == 64 || kp == 128; }

int spmm_tma_groups_per_block() { return kTmaWarps; }

// cuTensorMapEncodeTiled from the driver, looked up once.
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  std::lock_guard<std::mutex> lock(g_encode_mu);
  if (!g_encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e == cudaSuccess && q == cudaDriverEntryPointSuccess && fn) g_encode = (PFN_cuTensorMapEncodeTiled_v12000)fn;
  }
  return g_encode;
}

// Tensor map over the n x kp block `vh` (FP32 or BF16), one row per box: the gather4 layout.
ofsc_status spmm_tma_encode(const void* vh, int64_t n, int kp, bool bf16, CUtensorMap* map) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return fail(OFSC_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  const cuuint64_t dims[2] = {(cuuint64_t)kp, (cuuint64_t)(n > 0 ? n : 1)};
  const cuuint64_t strides[1] = {(cuuint64_t)kp * (bf16 ? 2 : 4)};
  const cuuint32_t box[2] = {(cuuint32_t)kp, 1};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   const_cast<void*>(vh), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(OFSC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return OFSC_OK;
}

ofsc_status tma_encode_f32_sw128(const float* base, int64_t rows, int cols, int ld, int box_cols, int box_rows,
                                 CUtensorMap* map) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return fail(OFSC_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  if (box_cols * 4 > 128 || ((uintptr_t)base & 15) || (ld & 3))
    return fail(OFSC_ERR_INVALID_ARG, "tensor map: box wider than the 128-byte swizzle or misaligned block");
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)(rows > 0 ? rows : 1)};
  const cuuint64_t strides[1] = {(cuuint64_t)ld * 4};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(OFSC_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return OFSC_OK;
}

cudaError_t spmm_tma_launch(const CUtensorMap& map, const TmaSpmmArgs& a, bool bf16, bool weighted, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  const int key = (a.kp == 128 ? 4 : 0) + (bf16 ? 2 : 0) + (weighted ? 1 : 0);
  switch (key) {
    case 0: return launch_t<2, false, false>(map, a, s);
    case 1: return launch_t<2, false, true>(map, a, s);
    case 2: return launch_t<2, true, false>(map, a, s);
    case 3: return launch_t<2, true, true>(map, a, s);
    case 4: return launch_t<4, false, false>(map, a, s);
    case 5: return launch_t<4, false, true>(map, a, s);
    case 6: return launch_t<4, true, false>(map, a, s);
    default: return launch_t<4, true, true>(map, a, s);
  }
}

}  // namespace ofsc
