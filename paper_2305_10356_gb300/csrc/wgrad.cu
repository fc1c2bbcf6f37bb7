// Gradient of the objectives with respect to the edge weights of S (the differentiable form of
// Eqs. (2) and (3)). With A_hat = D^-1/2 S D^-1/2, A = -I - A_hat and Gamma = df/dA_hat,
//   Gamma = 2 (I + A_hat - X X^T)   (f1),     Gamma = -X (2I - X^T X) X^T   (f2),
// a listing of the pair {a, b}, a != b, moves S_ab = S_ba and the degrees d_a, d_b, so
//   df/dw = 2 Gamma_ab / sqrt(d_a d_b) - r_a / d_a - r_b / d_b,   r_a = sum_j Gamma_aj A_hat_aj,
// with r_a = 2 (sum_j A_hat_aj^2 - x_a . (A_hat X)_a) for f1 and -(M x_a) . (A_hat X)_a for f2
// (M = 2I - X^T X, A_hat X = -(A X + X)). One warp per node forms r (and M x for f2); one warp per
// listed edge looks up S_ab in its CSR row and forms the k-dot of Gamma_ab (an SDDMM).
#include "common.cuh"

namespace ofsc {
namespace {

constexpr int kWgThreads = 256;

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Per node a: r[a]; for f2 also Z[a] = M x_a. X, AX: [n][kp] FP32; R64: X^T X (FP64, kp x kp).
__global__ void __launch_bounds__(kWgThreads) k_wgrad_nodes(int64_t n, int kp, int which, const float* __restrict__ X,
                                                            const float* __restrict__ AX, const int64_t* __restrict__ row_ptr,
                                                            const int32_t* __restrict__ col, const float* __restrict__ val,
                                                            const float* __restrict__ dinv, const double* __restrict__ R64,
                                                            float* __restrict__ r, float* __restrict__ Z) {
  extern __shared__ float Ms[];  // [kp][kp], M = 2I - X^T X (f2)
  if (which == 2) {
    for (int e = threadIdx.x; e < kp * kp; e += blockDim.x)
      Ms[e] = (float)((e / kp == e % kp ? 2.0 : 0.0) - R64[e]);
    __syncthreads();
  }
  const int lane = threadIdx.x & 31;
  const int c = lane * 4;
  const bool act = c < kp;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t a = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); a < n; a += warps) {
    float4 x = make_float4(0.f, 0.f, 0.f, 0.f), y = x;
    if (act) {
      x = *(const float4*)(X + a * kp + c);
      y = *(const float4*)(AX + a * kp + c);
    }
    const float4 h = make_float4(-(y.x + x.x), -(y.y + x.y), -(y.z + x.z), -(y.w + x.w));  // (A_hat X)_a
    float ra;
    if (which == 1) {
      const float sa = dinv[a];
      float sq = 0.0f;
      for (int64_t p = row_ptr[a] + lane; p < row_ptr[a + 1]; p += 32) {
        const float ah = (val ? val[p] : 1.0f) * sa * dinv[col[p]];
        sq = fmaf(ah, ah, sq);
      }
      const float dot = warp_sum(x.x * h.x + x.y * h.y + x.z * h.z + x.w * h.w);
      ra = 2.0f * (warp_sum(sq) - dot);
    } else {
      float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int m = 0; m < kp; ++m) {
        const float xv = (m & 3) == 0 ? x.x : (m & 3) == 1 ? x.y : (m & 3) == 2 ? x.z : x.w;
        const float xm = __shfl_sync(0xffffffffu, xv, m >> 2);
        if (act) {
          const float4 mr = *(const float4*)(Ms + m * kp + c);
          z.x = fmaf(xm, mr.x, z.x);
          z.y = fmaf(xm, mr.y, z.y);
          z.z = fmaf(xm, mr.z, z.z);
          z.w = fmaf(xm, mr.w, z.w);
        }
      }
      if (act) *(float4*)(Z + a * kp + c) = z;
      ra = -warp_sum(z.x * h.x + z.y * h.y + z.z * h.z + z.w * h.w);
    }
    if (lane == 0) r[a] = ra;
  }
}

// Per listed edge e = (a, b): df/dw_e (0 for a self-loop). Indices outside [0, n) write 0 and set
// *bad.
__global__ void __launch_bounds__(kWgThreads) k_wgrad_edges(int64_t m, int64_t n, const int32_t* __restrict__ src,
                                                            const int32_t* __restrict__ dst, int kp, int which,
                                                            const float* __restrict__ X, const float* __restrict__ Z,
                                                            const float* __restrict__ r, const int64_t* __restrict__ row_ptr,
                                                            const int32_t* __restrict__ col, const float* __restrict__ val,
                                                            const float* __restrict__ dinv, float* __restrict__ grad,
                                                            int* bad) {
  const int lane = threadIdx.x & 31;
  const int c = lane * 4;
  const bool act = c < kp;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t e = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); e < m; e += warps) {
    const int a = src[e], b = dst[e];
    if (a < 0 || b < 0 || a >= n || b >= n) {
      if (lane == 0) {
        grad[e] = 0.0f;
        *bad = 1;
      }
      continue;
    }
    if (a == b) {
      if (lane == 0) grad[e] = 0.0f;
      continue;
    }
    // S_ab: binary search for b among row a's ascending columns (lane 0), then broadcast
    float sab = 0.0f;
    if (lane == 0) {
      int64_t lo = row_ptr[a], hi = row_ptr[a + 1];
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (col[mid] < b) lo = mid + 1;
        else hi = mid;
      }
      if (lo < row_ptr[a + 1] && col[lo] == b) sab = val ? val[lo] : 1.0f;
    }
    sab = __shfl_sync(0xffffffffu, sab, 0);
    float4 xa = make_float4(0.f, 0.f, 0.f, 0.f), ob = xa;
    if (act) {
      xa = *(const float4*)(X + (int64_t)a * kp + c);
      ob = *(const float4*)((which == 1 ? X : Z) + (int64_t)b * kp + c);
    }
    const float dot = warp_sum(xa.x * ob.x + xa.y * ob.y + xa.z * ob.z + xa.w * ob.w);
    if (lane == 0) {
      const float sa = dinv[a], sb = dinv[b];
      const float ah = sab * sa * sb;
      const float gam = which == 1 ? 2.0f * (ah - dot) : -dot;
      grad[e] = 2.0f * gam * sa * sb - r[a] * sa * sa - r[b] * sb * sb;
    }
  }
}

}  // namespace

cudaError_t wgrad_launch(const WgradArgs& w, cudaStream_t s) {
  const int grid_n = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(w.n, kWgThreads / 32), 8 * kNumSMs));
  const size_t smem = w.which == 2 ? (size_t)w.kp * w.kp * sizeof(float) : 0;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_nodes, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 128 * 4);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (w.n > 0)
    k_wgrad_nodes<<<grid_n, kWgThreads, smem, s>>>(w.n, w.kp, w.which, w.X, w.AX, w.row_ptr, w.col, w.val, w.dinv,
                                                   w.R64, w.r, w.Z);
  const int grid_e = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(w.m, kWgThreads / 32), 32 * kNumSMs));
  if (w.m > 0)
    k_wgrad_edges<<<grid_e, kWgThreads, 0, s>>>(w.m, w.n, w.src, w.dst, w.kp, w.which, w.X, w.Z, w.r, w.row_ptr, w.col,
                                                w.val, w.dinv, w.grad, w.bad);
  return cudaGetLastError();
}

}  // namespace ofsc
