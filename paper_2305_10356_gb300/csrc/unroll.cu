// Gradient of f1 (Eq. (2)) after T unrolled updates of OFM-f1 (Algorithm 2 with the exact line
// search of Eq. (15)) with respect to the starting block X_0, by reverse accumulation with
// checkpoints.
//
// Forward, per update t (the iteration as Algorithm 2 states it, A X recomputed every update):
//   G_t = 4 (A X_t + X_t X_t^T X_t)                                      (Eq. (5))
//   beta_t,j = <G_t - G_{t-1}, G_t>_j / |G_{t-1},j|^2, 0 for a zero denominator;   V_0 = -G_0
//   V_t = -G_t + V_{t-1} diag(beta_t)
//   alpha_t = the chosen real root of p(a) = <V_t, A Z + Z Z^T Z>, Z = X_t + a V_t (Eq. (15))
//   X_{t+1} = X_t + alpha_t V_t
// Reverse, with H(Z)[U] = A U + U Z^T Z + Z (U^T Z + Z^T U) the Hessian of f1/4 applied to U:
//   alpha by the implicit-function theorem: c = -<Xbar_{t+1}, V_t> / <V_t, H(X_{t+1})[V_t]>,
//     Xbar_t = Xbar_{t+1} + c H(X_{t+1})[V_t],
//     Vbar_t += alpha Xbar_{t+1} + c (G_{t+1}/4 + alpha H(X_{t+1})[V_t]);
//   beta through its quotient (held at 0 where a zero denominator set it):
//     bbar_j = <Vbar_t, V_{t-1}>_j, nbar = bbar/den, dbar = -bbar beta/den,
//     Gbar_t = Gcarry - Vbar_t + nbar (2 G_t - G_{t-1}),  Gcarry <- -nbar G_t + 2 dbar G_{t-1},
//     Vbar_{t-1} = Vbar_t diag(beta_t);
//   G_t through its Hessian: Xbar_t += 4 H(X_t)[Gbar_t].
// The forward keeps X_t, V_{t-1}, G_{t-1} at the start of every segment of `ckpt` updates and the
// reverse sweep recomputes one segment at a time. Row blocks are n x kp FP32 (kp = k rounded up to
// a multiple of 8, zero columns inert); k x k products come from the tensor-core Grams (FP64
// results); per-column sums are FP64.
#include <algorithm>
#include <array>
#include <cmath>
#include <initializer_list>
#include <utility>
#include <vector>

#include "common.cuh"
#include "cubic.cuh"

namespace ofsc {
namespace {

constexpr int kUrThreads = 256;
constexpr int kUrDotBlocks = 2 * kNumSMs;

// out = sum_i coef_i (.) in_i + sum_j in_j M_j, coef_i = scale_i * (*dscale_i) * cscale_i[c].
struct RowTerm {
  const float* in;
  double scale;
  const double* dscale;  // device scalar or nullptr
  const double* cscale;  // device [kp] or nullptr
};
struct MixArgs {
  int64_t n;
  int kp;
  float* out;
  int nt;
  RowTerm t[5];
  int nm;
  const float* min[2];
  const float* M[2];  // FP32 [kp][kp]
};

// One thread covers four columns of one row; a block covers 1024 / kp rows per pass. The matrix
// factors and the block's rows of their left operands sit in shared memory. `out` may be the
// input of an elementwise term (each element is read and written by one thread).
__global__ void __launch_bounds__(kUrThreads) k_rowmix(MixArgs a) {
  extern __shared__ float sm[];
  const int kp = a.kp, tpr = kp / 4, rpi = kUrThreads / tpr;
  float* Ms = sm;                         // [nm][kp][kp]
  float* stage = sm + a.nm * kp * kp;     // [nm][rpi][kp]
  for (int j = 0; j < a.nm; ++j)
    for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) Ms[j * kp * kp + e] = a.M[j][e];
  const int lr = threadIdx.x / tpr, c = (threadIdx.x % tpr) * 4;
  const bool lane_ok = lr < rpi;
  float4 coef[5];
  for (int i = 0; i < a.nt; ++i) {
    const double s = a.t[i].scale * (a.t[i].dscale ? *a.t[i].dscale : 1.0);
    double cs[4] = {1.0, 1.0, 1.0, 1.0};
    if (a.t[i].cscale && lane_ok)
      for (int q = 0; q < 4; ++q) cs[q] = a.t[i].cscale[c + q];
    coef[i] = make_float4((float)(s * cs[0]), (float)(s * cs[1]), (float)(s * cs[2]), (float)(s * cs[3]));
  }
  __syncthreads();
  for (int64_t base = (int64_t)blockIdx.x * rpi; base < a.n; base += (int64_t)gridDim.x * rpi) {
    if (a.nm > 0) {
      for (int j = 0; j < a.nm; ++j)
        for (int e = threadIdx.x; e < rpi * kp; e += blockDim.x) {
          const int64_t r = base + e / kp;
          stage[j * rpi * kp + e] = r < a.n ? a.min[j][r * kp + e % kp] : 0.0f;
        }
      __syncthreads();
    }
    const int64_t r = base + lr;
    if (lane_ok && r < a.n) {
      float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
      for (int i = 0; i < a.nt; ++i) {
        const float4 v = *(const float4*)(a.t[i].in + r * kp + c);
        acc.x = fmaf(coef[i].x, v.x, acc.x);
        acc.y = fmaf(coef[i].y, v.y, acc.y);
        acc.z = fmaf(coef[i].z, v.z, acc.z);
        acc.w = fmaf(coef[i].w, v.w, acc.w);
      }
      for (int j = 0; j < a.nm; ++j) {
        const float* row = stage + j * rpi * kp + lr * kp;
        const float* M = Ms + j * kp * kp;
        for (int m = 0; m < kp; ++m) {
          const float x = row[m];
          const float4 mv = *(const float4*)(M + m * kp + c);
          acc.x = fmaf(x, mv.x, acc.x);
          acc.y = fmaf(x, mv.y, acc.y);
          acc.z = fmaf(x, mv.z, acc.z);
          acc.w = fmaf(x, mv.w, acc.w);
        }
      }
      *(float4*)(a.out + r * kp + c) = acc;
    }
    if (a.nm > 0) __syncthreads();
  }
}

// Per-column FP64 sums of (a_p - a2_p) (.) b_p for p < np (a2_p may be null): per-block partials
// [gridDim.x][np][kp], folded by k_colfold in block order.
struct DotArgs {
  int64_t n;
  int kp;
  int np;
  const float* a[4];
  const float* a2[4];
  const float* b[4];
  double* part;
};

__global__ void __launch_bounds__(kUrThreads) k_coldots(DotArgs d) {
  __shared__ double red[4 * 1024];  // [np][rpi][kp]: rpi * kp = 1024
  const int kp = d.kp, tpr = kp / 4, rpi = kUrThreads / tpr;
  const int lr = threadIdx.x / tpr, c = (threadIdx.x % tpr) * 4;
  const bool lane_ok = lr < rpi;
  double acc[4][4];
  for (int p = 0; p < 4; ++p)
    for (int q = 0; q < 4; ++q) acc[p][q] = 0.0;
  if (lane_ok)
    for (int64_t r = (int64_t)blockIdx.x * rpi + lr; r < d.n; r += (int64_t)gridDim.x * rpi) {
      for (int p = 0; p < d.np; ++p) {
        float4 x = *(const float4*)(d.a[p] + r * kp + c);
        if (d.a2[p]) {
          const float4 y = *(const float4*)(d.a2[p] + r * kp + c);
          x = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
        }
        const float4 z = *(const float4*)(d.b[p] + r * kp + c);
        acc[p][0] += (double)x.x * z.x;
        acc[p][1] += (double)x.y * z.y;
        acc[p][2] += (double)x.z * z.z;
        acc[p][3] += (double)x.w * z.w;
      }
    }
  if (lane_ok)
    for (int p = 0; p < d.np; ++p)
      for (int q = 0; q < 4; ++q) red[(p * rpi + lr) * kp + c + q] = acc[p][q];
  __syncthreads();
  for (int e = threadIdx.x; e < d.np * kp; e += blockDim.x) {
    const int p = e / kp, cc = e % kp;
    double s = 0.0;
    for (int l = 0; l < rpi; ++l) s += red[(p * rpi + l) * kp + cc];
    d.part[((int64_t)blockIdx.x * d.np + p) * kp + cc] = s;
  }
}

__global__ void k_colfold(const double* __restrict__ part, int nb, int width, double* __restrict__ out) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < width; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * width + e];
    out[e] = s;
  }
}

// M = s (A + A^T) (sym) or s A, FP64 [kp][kp] -> FP32.
__global__ void k_mat(const double* __restrict__ A, int kp, double s, int sym, float* __restrict__ M) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < kp * kp; e += gridDim.x * blockDim.x) {
    const int i = e / kp, j = e % kp;
    M[e] = (float)(s * (sym ? A[e] + A[j * kp + i] : A[e]));
  }
}

__device__ double ur_block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

// beta_t of Algorithm 2 from the column sums [gg | (G_t - G_{t-1}).G_t | den | v_{t-1}.G_t], and
// whether beta_t carries a derivative (live: a nonzero denominator).
__global__ void k_ur_beta(const double* __restrict__ s, int kp, double* beta, double* den_out, int* live) {
  for (int j = threadIdx.x; j < kp; j += blockDim.x) {
    const double num = s[kp + j], den = s[2 * kp + j];
    const double b = den != 0.0 ? num / den : 0.0;
    const int lv = den != 0.0;
    beta[j] = b;
    den_out[j] = den;
    live[j] = lv;
  }
}

// alpha_t from the Grams P = V^T X, Q = V^T V, R = X^T X and the column sums diag(V^T AV),
// diag(V^T G): the cubic of Eq. (15) (as printed, one quarter of d/da f1) and its chosen root.
__global__ void k_ur_alpha(const double* __restrict__ P, const double* __restrict__ Q, const double* __restrict__ R,
                           const double* __restrict__ dd, int kp, double* alpha, int* bad) {
  __shared__ double sh[kUrThreads];
  const int kk = kp * kp;
  double t0 = 0, t1 = 0, t2 = 0, t3 = 0, t4 = 0;
  for (int i = threadIdx.x; i < kk; i += blockDim.x) {
    const int r = i / kp, c = i % kp, it = c * kp + r;
    t0 += Q[i] * Q[it];
    t1 += Q[i] * P[it];
    t2 += P[i] * P[it] + P[i] * P[i] + Q[i] * R[it];
  }
  for (int j = threadIdx.x; j < kp; j += blockDim.x) {
    t3 += dd[j];
    t4 += dd[kp + j];
  }
  t0 = ur_block_sum(t0, sh);
  t1 = ur_block_sum(t1, sh);
  t2 = ur_block_sum(t2, sh);
  t3 = ur_block_sum(t3, sh);
  t4 = ur_block_sum(t4, sh);
  if (threadIdx.x == 0) {
    int b = 0;
    const double a = pick_step(t0, 3.0 * t1, t3 + t2, 0.25 * t4, &b);
    *alpha = a;
    if (b) *bad = 1;
  }
}

// c = -<Xbar, V> / <V, H1> and the coefficients {alpha, c/4, c alpha, c} of the V and X updates.
__global__ void k_ur_adj_alpha(const double* __restrict__ s, int kp, const double* __restrict__ alpha,
                               double* coef, int* bad) {
  __shared__ double sh[kUrThreads];
  double a = 0.0, p = 0.0;
  for (int j = threadIdx.x; j < kp; j += blockDim.x) {
    a += s[j];
    p += s[kp + j];
  }
  a = ur_block_sum(a, sh);
  p = ur_block_sum(p, sh);
  if (threadIdx.x == 0) {
    double c = 0.0;
    if (p != 0.0 && isfinite(p) && isfinite(a)) c = -a / p;
    else if (a != 0.0) *bad = 1;
    coef[0] = *alpha;
    coef[1] = 0.25 * c;
    coef[2] = c * *alpha;
    coef[3] = c;
  }
}

// nbar = bbar / den, dbar = -bbar beta / den on live columns, 0 elsewhere.
__global__ void k_ur_adj_beta(const double* __restrict__ bbar, const double* __restrict__ beta,
                              const double* __restrict__ den, const int* __restrict__ live, int kp, double* nbar,
                              double* dbar) {
  for (int j = threadIdx.x; j < kp; j += blockDim.x) {
    const bool lv = live[j] != 0;
    nbar[j] = lv ? bbar[j] / den[j] : 0.0;
    dbar[j] = lv ? -bbar[j] * beta[j] / den[j] : 0.0;
  }
}

// f1 = ||A||^2 + 2 tr(X^T AX) + ||X^T X||_F^2 from diag(X^T AX) and R = X^T X.
__global__ void k_ur_loss(const double* __restrict__ xax, const double* __restrict__ R, int kp, double normA2,
                          double* f) {
  __shared__ double sh[kUrThreads];
  double a = 0.0, r = 0.0;
  for (int j = threadIdx.x; j < kp; j += blockDim.x) a += xax[j];
  for (int i = threadIdx.x; i < kp * kp; i += blockDim.x) r += R[i] * R[i];
  a = ur_block_sum(a, sh);
  r = ur_block_sum(r, sh);
  if (threadIdx.x == 0) *f = normA2 + 2.0 * a + r;
}

__global__ void k_ur_pad(int64_t n, int k, int kp, const float* __restrict__ src, float* __restrict__ dst, int in) {
  const int64_t total = n * kp;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / kp;
    const int c = (int)(e % kp);
    if (in) dst[e] = c < k ? src[r * k + c] : 0.0f;
    else if (c < k) dst[r * k + c] = src[e];
  }
}

// Edge-weight derivative, step part: for every stored entry p = (a, b) of S,
//   Gam[p] += w1 (Gbar_a . X_b + Gbar_b . X_a) + w2 c (V_a . X1_b + V_b . X1_a),
// i.e. Gamma = dL/dA_hat = -dL/dA symmetrised, with dL/dA += 4 Gbar_t X_t^T (from G_t) and
// c V_t X_{t+1}^T (from alpha_t). A warp owns a row; groups of gs lanes take one entry each.
__global__ void __launch_bounds__(kUrThreads) k_ur_sddmm(int64_t n, int kp, const int64_t* __restrict__ row_ptr,
                                                        const int32_t* __restrict__ col, const float* __restrict__ Gb,
                                                        const float* __restrict__ Xt, const float* __restrict__ Vt,
                                                        const float* __restrict__ X1, const double* __restrict__ cptr,
                                                        float w1, float w2, float* __restrict__ gam) {
  const int lane = threadIdx.x & 31;
  int gs = 1;
  while (gs * 4 < kp) gs *= 2;
  const int per = 32 / gs, gl = lane % gs, grp = lane / gs, c = gl * 4;
  const bool act = c < kp;
  const float w2c = w2 * (float)*cptr;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t a = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); a < n; a += warps) {
    float4 ga = make_float4(0.f, 0.f, 0.f, 0.f), xa = ga, va = ga, x1a = ga;
    if (act) {
      ga = *(const float4*)(Gb + a * kp + c);
      xa = *(const float4*)(Xt + a * kp + c);
      va = *(const float4*)(Vt + a * kp + c);
      x1a = *(const float4*)(X1 + a * kp + c);
    }
    const int64_t beg = row_ptr[a], end = row_ptr[a + 1];
    for (int64_t base = beg; base < end; base += per) {
      const int64_t p = base + grp;
      float s1 = 0.0f, s2 = 0.0f;
      if (p < end && act) {
        const int64_t b = col[p];
        const float4 xb = *(const float4*)(Xt + b * kp + c);
        const float4 gb = *(const float4*)(Gb + b * kp + c);
        const float4 vb = *(const float4*)(Vt + b * kp + c);
        const float4 x1b = *(const float4*)(X1 + b * kp + c);
        s1 = ga.x * xb.x + ga.y * xb.y + ga.z * xb.z + ga.w * xb.w + gb.x * xa.x + gb.y * xa.y + gb.z * xa.z + gb.w * xa.w;
        s2 = va.x * x1b.x + va.y * x1b.y + va.z * x1b.z + va.w * x1b.w + vb.x * x1a.x + vb.y * x1a.y + vb.z * x1a.z +
             vb.w * x1a.w;
      }
      for (int off = gs / 2; off > 0; off >>= 1) {
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
        s2 += __shfl_xor_sync(0xffffffffu, s2, off);
      }
      if (gl == 0 && p < end) gam[p] += w1 * s1 + w2c * s2;
    }
  }
}

// r_a = sum over row a of Gam[p] A_hat_p (A_hat_p = S_p D^-1/2_a D^-1/2_b).
__global__ void k_ur_wnodes(int64_t n, const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const float* __restrict__ val, const float* __restrict__ dinv, const float* __restrict__ gam,
                            float* __restrict__ r) {
  for (int64_t a = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; a < n; a += (int64_t)gridDim.x * blockDim.x) {
    float acc = 0.0f;
    const float sa = dinv[a];
    for (int64_t p = row_ptr[a]; p < row_ptr[a + 1]; ++p) acc += gam[p] * (val ? val[p] : 1.0f) * sa * dinv[col[p]];
    r[a] = acc;
  }
}

// grad[e] += 2 Gam_ab / sqrt(d_a d_b) - r_a / d_a - r_b / d_b for every listed edge with a != b
// inside [0, n) (the others were set by the direct term).
__global__ void k_ur_wedges(int64_t m, int64_t n, const int32_t* __restrict__ src, const int32_t* __restrict__ dst,
                            const int64_t* __restrict__ row_ptr, const int32_t* __restrict__ col,
                            const float* __restrict__ dinv, const float* __restrict__ gam, const float* __restrict__ r,
                            float* __restrict__ grad) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
    const int a = src[e], b = dst[e];
    if (a < 0 || b < 0 || a >= n || b >= n || a == b) continue;
    int64_t lo = row_ptr[a], hi = row_ptr[a + 1];
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (col[mid] < b) lo = mid + 1;
      else hi = mid;
    }
    if (lo >= row_ptr[a + 1] || col[lo] != b) continue;
    const float sa = dinv[a], sb = dinv[b];
    grad[e] += 2.0f * gam[lo] * sa * sb - r[a] * sa * sa - r[b] * sb * sb;
  }
}

int elem_grid(int64_t total) { return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(total, 256), 8 * kNumSMs)); }

struct Engine {
  ofsc_graph* g;
  int64_t n;
  int kp;
  cudaStream_t s;
  std::vector<void*> owned;
  // scratch
  float *AX = nullptr, *gat = nullptr, *H = nullptr, *M0 = nullptr, *M1 = nullptr;
  double *gram = nullptr, *part = nullptr, *sums = nullptr, *coef = nullptr, *nbar = nullptr, *dbar = nullptr,
         *fdev = nullptr;
  int* bad = nullptr;
  size_t blk() const { return (size_t)n * kp * sizeof(float); }

  cudaError_t alloc(void** p, size_t bytes) {
    cudaError_t e = dev_alloc(p, bytes);
    if (e == cudaSuccess) owned.push_back(*p);
    return e;
  }
  ~Engine() {
    for (void* p : owned) dev_free(p);
  }
  cudaError_t init() {
    const size_t kk = (size_t)kp * kp;
    cudaError_t e;
    if ((e = alloc((void**)&AX, blk())) != cudaSuccess) return e;
    if ((e = alloc((void**)&gat, blk())) != cudaSuccess) return e;
    if ((e = alloc((void**)&H, blk())) != cudaSuccess) return e;
    if ((e = alloc((void**)&M0, kk * sizeof(float))) != cudaSuccess) return e;
    if ((e = alloc((void**)&M1, kk * sizeof(float))) != cudaSuccess) return e;
    if ((e = alloc((void**)&gram, 3 * kk * sizeof(double))) != cudaSuccess) return e;  // 2 Gram slots + X^T X
    if ((e = alloc((void**)&part, (size_t)kUrDotBlocks * 4 * kp * sizeof(double))) != cudaSuccess) return e;
    if ((e = alloc((void**)&sums, 4 * (size_t)kp * sizeof(double))) != cudaSuccess) return e;
    if ((e = alloc((void**)&coef, 8 * sizeof(double))) != cudaSuccess) return e;
    if ((e = alloc((void**)&nbar, (size_t)kp * sizeof(double))) != cudaSuccess) return e;
    if ((e = alloc((void**)&dbar, (size_t)kp * sizeof(double))) != cudaSuccess) return e;
    if ((e = alloc((void**)&fdev, sizeof(double))) != cudaSuccess) return e;
    if ((e = alloc((void**)&bad, sizeof(int))) != cudaSuccess) return e;
    return cudaMemsetAsync(bad, 0, sizeof(int), s);
  }

  cudaError_t mix(float* out, std::initializer_list<RowTerm> terms, std::initializer_list<std::pair<const float*, const float*>> mats) {
    MixArgs a{};
    a.n = n;
    a.kp = kp;
    a.out = out;
    for (const RowTerm& t : terms) a.t[a.nt++] = t;
    for (const auto& m : mats) {
      a.min[a.nm] = m.first;
      a.M[a.nm] = m.second;
      ++a.nm;
    }
    const int rpi = kUrThreads / (kp / 4);
    const size_t smem = ((size_t)a.nm * kp * kp + (size_t)a.nm * rpi * kp) * sizeof(float);
    static bool attr = false;
    if (!attr) {
      cudaError_t e = cudaFuncSetAttribute(k_rowmix, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)((2 * 128 * 128 + 2 * 1024) * sizeof(float)));
      if (e != cudaSuccess) return e;
      attr = true;
    }
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, rpi), 2 * kNumSMs));
    k_rowmix<<<grid, kUrThreads, smem, s>>>(a);
    return cudaGetLastError();
  }

  // column sums of (a_p - a2_p) (.) b_p into sums[p][kp]
  cudaError_t dots(std::initializer_list<std::array<const float*, 3>> pairs) {
    DotArgs d{};
    d.n = n;
    d.kp = kp;
    for (const auto& p : pairs) {
      d.a[d.np] = p[0];
      d.a2[d.np] = p[1];
      d.b[d.np] = p[2];
      ++d.np;
    }
    d.part = part;
    const int rpi = kUrThreads / (kp / 4);
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(n, rpi), kUrDotBlocks));
    k_coldots<<<grid, kUrThreads, 0, s>>>(d);
    k_colfold<<<ceil_div(d.np * kp, 256), 256, 0, s>>>(part, grid, d.np * kp, sums);
    return cudaGetLastError();
  }

  // gram[b] = L^T R_b (FP64 kp x kp), b < nr <= 2, on the tensor cores; synchronises the stream.
  // Explicit rows per CTA select the kernel that stages rows with bounds-checked plain loads
  // (any kp), about two CTAs per SM.
  ofsc_status grams(const float* L, const float* R0, const float* R1) {
    const float* R[2] = {R0, R1};
    const int64_t rpb = std::max<int64_t>(1, ceil_div(ceil_div(n, 2 * kNumSMs), (int64_t)32)) * 32;
    return ofsc_gram(n, kp, kp, L, R1 ? 2 : 1, R, rpb, gram, s);
  }

  cudaError_t mat(const double* A, double sc, int sym, float* M) {
    k_mat<<<ceil_div(kp * kp, 256), 256, 0, s>>>(A, kp, sc, sym, M);
    return cudaGetLastError();
  }

  // G = 4 (A X + X X^T X); leaves AX in this->AX and X^T X in gram[0]
  ofsc_status grad_f1(const float* X, float* G) {
    OFSC_CUDA(apply_A(g, kp, X, AX, gat, s));
    ofsc_status st = grams(X, X, nullptr);
    if (st != OFSC_OK) return st;
    OFSC_CUDA(mat(gram, 4.0, 0, M0));
    OFSC_CUDA(mix(G, {{AX, 4.0, nullptr, nullptr}}, {{X, M0}}));
    return OFSC_OK;
  }
};

// Per-update scalars kept for the whole run.
struct Scalars {
  double* alpha;  // [T]
  double* beta;   // [T][kp]
  double* den;    // [T][kp]
  int* live;      // [T][kp]
};

// Update t from X_t (and V_{t-1}, G_{t-1} for t > 0): G_t, V_t, AV_t, alpha_t, beta_t, X_{t+1}.
ofsc_status forward_step(Engine& E, const Scalars& sc, int t, const float* Xt, const float* Vp, const float* Gp,
                         float* Gt, float* Vt, float* AVt, float* Xn) {
  const int kp = E.kp;
  ofsc_status st = E.grad_f1(Xt, Gt);
  if (st != OFSC_OK) return st;
  double* beta = sc.beta + (size_t)t * kp;
  if (t > 0) {
    OFSC_CUDA(E.dots({{{Gt, nullptr, Gt}}, {{Gt, Gp, Gt}}, {{Gp, nullptr, Gp}}, {{Vp, nullptr, Gt}}}));
    k_ur_beta<<<1, 128, 0, E.s>>>(E.sums, kp, beta, sc.den + (size_t)t * kp, sc.live + (size_t)t * kp);
    OFSC_CUDA(E.mix(Vt, {{Gt, -1.0, nullptr, nullptr}, {Vp, 1.0, nullptr, beta}}, {}));
  } else {
    OFSC_CUDA(cudaMemsetAsync(beta, 0, kp * sizeof(double), E.s));
    OFSC_CUDA(cudaMemsetAsync(sc.den + 0, 0, kp * sizeof(double), E.s));
    OFSC_CUDA(cudaMemsetAsync(sc.live + 0, 0, kp * sizeof(int), E.s));
    OFSC_CUDA(E.mix(Vt, {{Gt, -1.0, nullptr, nullptr}}, {}));
  }
  OFSC_CUDA(apply_A(E.g, kp, Vt, AVt, E.gat, E.s));
  // R = X^T X is still in gram[0] from grad_f1; keep it apart from the next Grams
  double* R = E.gram + 2 * (size_t)kp * kp;  // the third slot
  OFSC_CUDA(cudaMemcpyAsync(R, E.gram, (size_t)kp * kp * sizeof(double), cudaMemcpyDeviceToDevice, E.s));
  st = E.grams(Vt, Xt, Vt);  // P = V^T X, Q = V^T V
  if (st != OFSC_OK) return st;
  OFSC_CUDA(E.dots({{{Vt, nullptr, AVt}}, {{Vt, nullptr, Gt}}}));
  k_ur_alpha<<<1, kUrThreads, 0, E.s>>>(E.gram, E.gram + (size_t)kp * kp, R, E.sums, kp, sc.alpha + t, E.bad);
  OFSC_CUDA(E.mix(Xn, {{Xt, 1.0, nullptr, nullptr}, {Vt, 1.0, sc.alpha + t, nullptr}}, {}));
  return OFSC_OK;
}

}  // namespace
}  // namespace ofsc

using namespace ofsc;

extern "C" ofsc_status ofsc_unrolled_grad(ofsc_graph* g, int32_t k, const float* X0, int32_t T, int32_t ckpt,
                                          int64_t m, const int32_t* src, const int32_t* dst, double* f_out,
                                          float* grad, float* grad_w, void* stream_) {
  clear_error();
  if (!g) return fail(OFSC_ERR_INVALID_ARG, "ofsc_unrolled_grad: graph is NULL");
  if (k < 1 || k > kMaxK) return fail(OFSC_ERR_INVALID_ARG, "ofsc_unrolled_grad: k=%d outside [1, %d]", k, kMaxK);
  if (T < 0 || T > 4096) return fail(OFSC_ERR_INVALID_ARG, "ofsc_unrolled_grad: T=%d outside [0, 4096]", T);
  if (ckpt < 0) return fail(OFSC_ERR_INVALID_ARG, "ofsc_unrolled_grad: ckpt < 0");
  if (g->n > 0 && !X0) return fail(OFSC_ERR_INVALID_ARG, "ofsc_unrolled_grad: X0 is NULL");
  if (grad_w) {
    if (!g->weighted) return fail(OFSC_ERR_INVALID_ARG, "ofsc_unrolled_grad: grad_w needs a graph built with weights");
    if (m < 0 || (m > 0 && (!src || !dst))) return fail(OFSC_ERR_INVALID_ARG, "ofsc_unrolled_grad: bad edge arrays");
  }
  cudaStream_t s = (cudaStream_t)stream_;
  const int kp = round_up(k, 8);
  const int S = T == 0 ? 1 : std::min<int>(ckpt > 0 ? ckpt : 5, T);
  const int nseg = T == 0 ? 0 : (T + S - 1) / S;
  if (g->n == 0) {
    if (f_out) *f_out = g->normA2;
    if (grad_w && m > 0) OFSC_CUDA(cudaMemsetAsync(grad_w, 0, (size_t)m * sizeof(float), s));
    OFSC_CUDA(cudaStreamSynchronize(s));
    return OFSC_OK;
  }
  Engine E{g, g->n, kp, s};
  OFSC_CUDA(E.init());
  // segment storage: X_[0..S], V_[-1..S-1], G_[-1..S], AV_[0..S-1]; checkpoints per segment
  std::vector<float*> Xs(S + 1), Vs(S + 1), Gs(S + 2), AVs(S), ckX(nseg), ckV(nseg), ckG(nseg);
  for (auto* v : {&Xs, &Vs, &Gs, &AVs})
    for (float*& p : *v) OFSC_CUDA(E.alloc((void**)&p, E.blk()));
  for (int q = 1; q < nseg; ++q) {
    OFSC_CUDA(E.alloc((void**)&ckX[q], E.blk()));
    OFSC_CUDA(E.alloc((void**)&ckV[q], E.blk()));
    OFSC_CUDA(E.alloc((void**)&ckG[q], E.blk()));
  }
  float *X0p = nullptr, *Xbar = nullptr, *Vbar = nullptr, *Gcarry = nullptr, *Gbar = nullptr, *Gnext = nullptr;
  for (float** p : {&X0p, &Xbar, &Vbar, &Gcarry, &Gbar, &Gnext}) OFSC_CUDA(E.alloc((void**)p, E.blk()));
  Scalars sc{};
  const int Tn = T > 0 ? T : 1;
  OFSC_CUDA(E.alloc((void**)&sc.alpha, Tn * sizeof(double)));
  OFSC_CUDA(E.alloc((void**)&sc.beta, (size_t)Tn * kp * sizeof(double)));
  OFSC_CUDA(E.alloc((void**)&sc.den, (size_t)Tn * kp * sizeof(double)));
  OFSC_CUDA(E.alloc((void**)&sc.live, (size_t)Tn * kp * sizeof(int)));
  float *gam = nullptr, *rnode = nullptr;
  int* wbad = nullptr;  // a listed endpoint outside [0, n)
  if (grad_w) {
    OFSC_CUDA(E.alloc((void**)&gam, std::max<int64_t>(1, g->nnz) * sizeof(float)));
    OFSC_CUDA(E.alloc((void**)&rnode, (size_t)g->n * sizeof(float)));
    OFSC_CUDA(E.alloc((void**)&wbad, sizeof(int)));
    OFSC_CUDA(cudaMemsetAsync(gam, 0, std::max<int64_t>(1, g->nnz) * sizeof(float), s));
    OFSC_CUDA(cudaMemsetAsync(wbad, 0, sizeof(int), s));
  }
  k_ur_pad<<<elem_grid(g->n * kp), 256, 0, s>>>(g->n, k, kp, X0, X0p, 1);
  OFSC_LAUNCH_CHECK("k_ur_pad");

  // Forward sweep: keep X_t, V_{t-1}, G_{t-1} at each segment start; rotate the rest.
  auto V_ = [&](int i) { return Vs[i + 1]; };  // i = -1 .. S-1
  auto G_ = [&](int i) { return Gs[i + 1]; };  // i = -1 .. S
  OFSC_CUDA(cudaMemcpyAsync(Xs[0], X0p, E.blk(), cudaMemcpyDeviceToDevice, s));
  ofsc_status st;
  for (int q = 0; q < nseg; ++q) {
    const int t0 = q * S, t1 = std::min(T, t0 + S);
    if (q > 0) {
      OFSC_CUDA(cudaMemcpyAsync(ckX[q], Xs[0], E.blk(), cudaMemcpyDeviceToDevice, s));
      OFSC_CUDA(cudaMemcpyAsync(ckV[q], V_(-1), E.blk(), cudaMemcpyDeviceToDevice, s));
      OFSC_CUDA(cudaMemcpyAsync(ckG[q], G_(-1), E.blk(), cudaMemcpyDeviceToDevice, s));
    }
    for (int t = t0; t < t1; ++t) {
      const int i = t - t0;
      st = forward_step(E, sc, t, Xs[i], V_(i - 1), G_(i - 1), G_(i), V_(i), AVs[i], Xs[i + 1]);
      if (st != OFSC_OK) return st;
    }
    // the last update's V, G become the next segment's "previous"; its X_{t1} the next start
    const int len = t1 - t0;
    OFSC_CUDA(cudaMemcpyAsync(V_(-1), V_(len - 1), E.blk(), cudaMemcpyDeviceToDevice, s));
    OFSC_CUDA(cudaMemcpyAsync(G_(-1), G_(len - 1), E.blk(), cudaMemcpyDeviceToDevice, s));
    OFSC_CUDA(cudaMemcpyAsync(Xs[0], Xs[len], E.blk(), cudaMemcpyDeviceToDevice, s));
  }
  // Loss at X_T (in Xs[0]) and its gradient G_T, the adjoint Xbar_T
  st = E.grad_f1(Xs[0], Xbar);
  if (st != OFSC_OK) return st;
  OFSC_CUDA(E.dots({{{Xs[0], nullptr, E.AX}}}));
  k_ur_loss<<<1, kUrThreads, 0, s>>>(E.sums, E.gram, kp, g->normA2, E.fdev);
  if (grad_w) {  // f1(X_T) itself: the weight gradient at fixed X_T
    WgradArgs w{};
    w.n = g->n;
    w.kp = kp;
    w.which = 1;
    w.X = Xs[0];
    w.AX = E.AX;
    w.R64 = E.gram;
    w.row_ptr = g->row_ptr;
    w.col = g->col;
    w.val = g->val;
    w.dinv = g->dinv;
    w.r = rnode;
    w.Z = E.H;
    w.m = m;
    w.src = src;
    w.dst = dst;
    w.grad = grad_w;
    w.bad = wbad;
    OFSC_CUDA(wgrad_launch(w, s));
  }
  OFSC_CUDA(cudaMemcpyAsync(Gnext, Xbar, E.blk(), cudaMemcpyDeviceToDevice, s));
  OFSC_CUDA(cudaMemsetAsync(Vbar, 0, E.blk(), s));
  OFSC_CUDA(cudaMemsetAsync(Gcarry, 0, E.blk(), s));

  // Reverse sweep, one recomputed segment at a time
  for (int q = nseg - 1; q >= 0; --q) {
    const int t0 = q * S, t1 = std::min(T, t0 + S), len = t1 - t0;
    if (q > 0) {
      OFSC_CUDA(cudaMemcpyAsync(Xs[0], ckX[q], E.blk(), cudaMemcpyDeviceToDevice, s));
      OFSC_CUDA(cudaMemcpyAsync(V_(-1), ckV[q], E.blk(), cudaMemcpyDeviceToDevice, s));
      OFSC_CUDA(cudaMemcpyAsync(G_(-1), ckG[q], E.blk(), cudaMemcpyDeviceToDevice, s));
    } else {
      OFSC_CUDA(cudaMemcpyAsync(Xs[0], X0p, E.blk(), cudaMemcpyDeviceToDevice, s));
    }
    for (int t = t0; t < t1; ++t) {
      const int i = t - t0;
      st = forward_step(E, sc, t, Xs[i], V_(i - 1), G_(i - 1), G_(i), V_(i), AVs[i], Xs[i + 1]);
      if (st != OFSC_OK) return st;
    }
    for (int t = t1 - 1; t >= t0; --t) {
      const int i = t - t0;
      const float *Xt = Xs[i], *X1 = Xs[i + 1], *Vt = V_(i), *AVt = AVs[i], *Gt = G_(i);
      const float* G1 = i + 1 < len ? G_(i + 1) : Gnext;
      // alpha_t: H1 = H(X_{t+1})[V_t] into E.H
      st = E.grams(X1, X1, Vt);  // R1 = X1^T X1, B1 = X1^T V
      if (st != OFSC_OK) return st;
      OFSC_CUDA(E.mat(E.gram, 1.0, 0, E.M0));
      OFSC_CUDA(E.mat(E.gram + (size_t)kp * kp, 1.0, 1, E.M1));
      OFSC_CUDA(E.mix(E.H, {{AVt, 1.0, nullptr, nullptr}}, {{Vt, E.M0}, {X1, E.M1}}));
      OFSC_CUDA(E.dots({{{Xbar, nullptr, Vt}}, {{Vt, nullptr, E.H}}}));
      k_ur_adj_alpha<<<1, kUrThreads, 0, s>>>(E.sums, kp, sc.alpha + t, E.coef, E.bad);
      OFSC_CUDA(E.mix(Vbar, {{Vbar, 1.0, nullptr, nullptr}, {Xbar, 1.0, E.coef + 0, nullptr},
                             {G1, 1.0, E.coef + 1, nullptr}, {E.H, 1.0, E.coef + 2, nullptr}}, {}));
      OFSC_CUDA(E.mix(Xbar, {{Xbar, 1.0, nullptr, nullptr}, {E.H, 1.0, E.coef + 3, nullptr}}, {}));
      // beta_t
      if (t > 0) {
        const float *Gp = G_(i - 1), *Vp = V_(i - 1);
        OFSC_CUDA(E.dots({{{Vbar, nullptr, Vp}}}));
        const size_t o = (size_t)t * kp;
        k_ur_adj_beta<<<1, 128, 0, s>>>(E.sums, sc.beta + o, sc.den + o, sc.live + o, kp, E.nbar, E.dbar);
        OFSC_CUDA(E.mix(Gbar, {{Gcarry, 1.0, nullptr, nullptr}, {Vbar, -1.0, nullptr, nullptr},
                               {Gt, 2.0, nullptr, E.nbar}, {Gp, -1.0, nullptr, E.nbar}}, {}));
        OFSC_CUDA(E.mix(Gcarry, {{Gt, -1.0, nullptr, E.nbar}, {Gp, 2.0, nullptr, E.dbar}}, {}));
        OFSC_CUDA(E.mix(Vbar, {{Vbar, 1.0, nullptr, sc.beta + o}}, {}));
      } else {
        OFSC_CUDA(E.mix(Gbar, {{Gcarry, 1.0, nullptr, nullptr}, {Vbar, -1.0, nullptr, nullptr}}, {}));
      }
      if (grad_w) {
        k_ur_sddmm<<<(int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(g->n, kUrThreads / 32), 16 * kNumSMs)),
                     kUrThreads, 0, s>>>(g->n, kp, g->row_ptr, g->col, Gbar, Xt, Vt, X1, E.coef + 3, -2.0f, -0.5f, gam);
        OFSC_LAUNCH_CHECK("k_ur_sddmm");
      }
      // G_t: Xbar += 4 H(X_t)[Gbar]
      OFSC_CUDA(apply_A(g, kp, Gbar, E.H, E.gat, s));
      st = E.grams(Xt, Xt, Gbar);  // R_t, B = X_t^T Gbar
      if (st != OFSC_OK) return st;
      OFSC_CUDA(E.mat(E.gram, 4.0, 0, E.M0));
      OFSC_CUDA(E.mat(E.gram + (size_t)kp * kp, 4.0, 1, E.M1));
      OFSC_CUDA(E.mix(Xbar, {{Xbar, 1.0, nullptr, nullptr}, {E.H, 4.0, nullptr, nullptr}}, {{Gbar, E.M0}, {Xt, E.M1}}));
    }
    OFSC_CUDA(cudaMemcpyAsync(Gnext, G_(0), E.blk(), cudaMemcpyDeviceToDevice, s));
  }
  if (grad) {
    k_ur_pad<<<elem_grid(g->n * kp), 256, 0, s>>>(g->n, k, kp, Xbar, grad, 0);
    OFSC_LAUNCH_CHECK("k_ur_pad");
  }
  if (grad_w && T > 0) {
    k_ur_wnodes<<<elem_grid(g->n), 256, 0, s>>>(g->n, g->row_ptr, g->col, g->val, g->dinv, gam, rnode);
    if (m > 0) k_ur_wedges<<<elem_grid(m), 256, 0, s>>>(m, g->n, src, dst, g->row_ptr, g->col, g->dinv, gam, rnode, grad_w);
    OFSC_LAUNCH_CHECK("k_ur_wedges");
  }
  double f = 0.0;
  int bad = 0, hwbad = 0;
  OFSC_CUDA(cudaMemcpyAsync(&f, E.fdev, sizeof(double), cudaMemcpyDeviceToHost, s));
  OFSC_CUDA(cudaMemcpyAsync(&bad, E.bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (wbad) OFSC_CUDA(cudaMemcpyAsync(&hwbad, wbad, sizeof(int), cudaMemcpyDeviceToHost, s));
  OFSC_CUDA(cudaStreamSynchronize(s));
  if (f_out) *f_out = f;
  if (hwbad) return fail(OFSC_ERR_INVALID_ARG, "ofsc_unrolled_grad: an edge endpoint is outside [0, n)");
  if (bad || !std::isfinite(f))
    return fail(OFSC_ERR_NONFINITE, "ofsc_unrolled_grad: non-finite value or a vanishing curvature along a direction");
  return OFSC_OK;
}
