// Algorithm 1, steps 3-4: row normalisation and Euclidean K-means (K-means++ seeding, Lloyd).
//
// K-means++ (Arthur and Vassilvitskii 2007) draws its uniforms from Philox-4x32-10 (Salmon,
// Moraes, Dror and Shaw, SC'11): draw c of run r is word 0 of Philox(ctr = {c, r, 0, 0},
// key = {seed_lo, seed_hi}) divided by 2^32. Every reduction here has a fixed order, so a seed
// gives the same labels on every run.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

namespace ofsc {
namespace {

__device__ __forceinline__ void philox_round(uint32_t& c0, uint32_t& c1, uint32_t& c2, uint32_t& c3,
                                             uint32_t k0, uint32_t k1) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t hi0 = __umulhi(M0, c0), lo0 = M0 * c0;
  const uint32_t hi1 = __umulhi(M1, c2), lo1 = M1 * c2;
  const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
  c0 = n0;
  c1 = lo1;
  c2 = n2;
  c3 = lo0;
}

__device__ double philox_uniform(uint64_t seed, uint32_t run, uint32_t draw) {
  uint32_t c0 = draw, c1 = run, c2 = 0, c3 = 0;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    philox_round(c0, c1, c2, c3, k0, k1);
  }
  return (double)c0 * (1.0 / 4294967296.0);
}

// ---------------------------------------------------------------------------------------------
// Row normalisation: one warp per row, FP32 sum of squares
// ---------------------------------------------------------------------------------------------
__global__ void k_row_normalize(int64_t n, int k, float* __restrict__ X) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t l = warp; l < n; l += nwarps) {
    float* row = X + l * k;
    float ss = 0.0f;
    for (int j = lane; j < k; j += 32) ss = fmaf(row[j], row[j], ss);
    for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
    if (ss > 0.0f) {
      const float nr = sqrtf(ss);
      for (int j = lane; j < k; j += 32) row[j] = row[j] / nr;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// K-means++ seeding
// ---------------------------------------------------------------------------------------------

// D2[i] = min(D2[i], ||x_i - x_c||^2) with c = *centre (first: D2 = the distance itself).
__global__ void k_seed_dist(int64_t n, int d, const float* __restrict__ X, const int64_t* __restrict__ centre,
                            double* __restrict__ D2, int first) {
  const int64_t c = *centre;
  const float* xc = X + c * d;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float* xi = X + i * d;
    float s = 0.0f;
    for (int j = 0; j < d; ++j) {
      const float t = xi[j] - xc[j];
      s = fmaf(t, t, s);
    }
    const double v = (double)s;
    D2[i] = first ? v : fmin(D2[i], v);
  }
}

constexpr int kSumBlocks = 512;

// bsum[b] = sum of D2 over the contiguous chunk of block b (fixed tree order).
__global__ void __launch_bounds__(256) k_chunk_sum(int64_t n, int64_t chunk, const double* __restrict__ D2,
                                                   double* __restrict__ bsum) {
  __shared__ double sh[256];
  const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += 256) s += D2[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = sh[0];
}

// One thread: the first index whose running sum of D2 exceeds u * total (or floor(u n) when the
// total is 0); the running sum goes chunk by chunk, then element by element inside the chunk.
__global__ void k_seed_pick(int64_t n, int64_t chunk, int nblk, const double* __restrict__ D2,
                            const double* __restrict__ bsum, uint64_t seed, int run, int draw,
                            int64_t* __restrict__ centre) {
  const double u = philox_uniform(seed, (uint32_t)run, (uint32_t)draw);
  double total = 0.0;
  for (int b = 0; b < nblk; ++b) total += bsum[b];
  int64_t j;
  if (draw == 0 || !(total > 0.0)) {
    j = (int64_t)(u * (double)n);
  } else {
    const double target = u * total;
    double run_sum = 0.0;
    int b = 0;
    for (; b < nblk - 1; ++b) {
      if (run_sum + bsum[b] > target) break;
      run_sum += bsum[b];
    }
    const int64_t i0 = b * chunk, i1 = min(n, i0 + chunk);
    j = i1 - 1;
    for (int64_t i = i0; i < i1; ++i) {
      run_sum += D2[i];
      if (run_sum > target) {
        j = i;
        break;
      }
    }
  }
  if (j > n - 1) j = n - 1;
  if (j < 0) j = 0;
  *centre = j;
}

__global__ void k_copy_centroid(int d, const float* __restrict__ X, const int64_t* __restrict__ centre,
                                float* __restrict__ mu) {
  const int64_t c = *centre;
  for (int j = threadIdx.x; j < d; j += blockDim.x) mu[j] = X[c * d + j];
}

// ---------------------------------------------------------------------------------------------
// Lloyd iterations
// ---------------------------------------------------------------------------------------------

// Nearest centroid of every row (ties: lowest index); dist = its squared distance (FP32).
// Centroids live in shared memory; a warp stages 32 rows (row stride d + 1, conflict-free).
__global__ void __launch_bounds__(256) k_assign(int64_t n, int d, int C, const float* __restrict__ X,
                                                const float* __restrict__ mu, int32_t* __restrict__ labels,
                                                float* __restrict__ dist, int* __restrict__ changed,
                                                int check) {
  extern __shared__ float sm[];
  float* mus = sm;                      // C * d
  float* xs = sm + C * d;               // 8 warps * 32 * (d + 1)
  for (int i = threadIdx.x; i < C * d; i += blockDim.x) mus[i] = mu[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* xw = xs + warp * 32 * (d + 1);
  int my_changed = 0;
  const int64_t nbatches = (n + 31) / 32;
  for (int64_t bt = blockIdx.x * 8 + warp; bt < nbatches; bt += (int64_t)gridDim.x * 8) {
    const int64_t r0 = bt * 32;
    const int rows = (int)min((int64_t)32, n - r0);
    for (int i = lane; i < rows * d; i += 32) {
      const int r = i / d, j = i % d;
      xw[r * (d + 1) + j] = X[(r0 + r) * d + j];
    }
    __syncwarp();
    if (lane < rows) {
      const float* x = xw + lane * (d + 1);
      float best = 0.0f;
      int bc = 0;
      for (int c = 0; c < C; ++c) {
        const float* m = mus + c * d;
        float s = 0.0f;
        for (int j = 0; j < d; ++j) {
          const float t = x[j] - m[j];
          s = fmaf(t, t, s);
        }
        if (c == 0 || s < best) {
          best = s;
          bc = c;
        }
      }
      const int64_t i = r0 + lane;
      if (check && labels[i] != bc) my_changed = 1;
      labels[i] = bc;
      dist[i] = best;
    }
    __syncwarp();
  }
  if (check) {
    for (int o = 16; o > 0; o >>= 1) my_changed |= __shfl_xor_sync(0xffffffffu, my_changed, o);
    if (lane == 0 && my_changed) atomicOr(changed, 1);
  }
}

// Per-chunk centroid sums: block b adds its rows in index order (deterministic), threads over dims.
__global__ void k_centroid_part(int64_t n, int d, int C, int64_t chunk, const float* __restrict__ X,
                                const int32_t* __restrict__ labels, float* __restrict__ part,
                                int* __restrict__ cpart) {
  extern __shared__ float acc[];       // C * d
  int* cnt = (int*)(acc + C * d);      // C
  for (int i = threadIdx.x; i < C * d; i += blockDim.x) acc[i] = 0.0f;
  for (int i = threadIdx.x; i < C; i += blockDim.x) cnt[i] = 0;
  __syncthreads();
  const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  for (int64_t i = i0; i < i1; ++i) {
    const int c = labels[i];
    for (int j = threadIdx.x; j < d; j += blockDim.x) acc[c * d + j] += X[i * d + j];
    if (threadIdx.x == 0) cnt[c] += 1;
  }
  __syncthreads();
  float* out = part + (int64_t)blockIdx.x * C * d;
  for (int i = threadIdx.x; i < C * d; i += blockDim.x) out[i] = acc[i];
  for (int i = threadIdx.x; i < C; i += blockDim.x) cpart[blockIdx.x * C + i] = cnt[i];
}

// mu[c] = (sum over chunks in order, FP64) / count; empty clusters keep their slot for the host.
__global__ void k_centroid_final(int d, int C, int nblk, const float* __restrict__ part,
                                 const int* __restrict__ cpart, float* __restrict__ mu,
                                 int* __restrict__ counts) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < C * d; i += gridDim.x * blockDim.x) {
    const int c = i / d;
    double s = 0.0;
    int cntc = 0;
    for (int b = 0; b < nblk; ++b) {
      s += (double)part[(int64_t)b * C * d + i];
      cntc += cpart[b * C + c];
    }
    if (cntc > 0) mu[i] = (float)(s / cntc);
    if (i % d == 0) counts[c] = cntc;
  }
}

// Farthest row from its own centroid among rows not yet taken (ties: lowest index); one block
// per chunk, then one block over the chunk winners.
__global__ void __launch_bounds__(256) k_farthest_part(int64_t n, int64_t chunk, const float* __restrict__ dist,
                                                       const unsigned char* __restrict__ taken,
                                                       float* __restrict__ bval, int64_t* __restrict__ bidx) {
  __shared__ float sv[256];
  __shared__ int64_t si[256];
  const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  float best = -1.0f;
  int64_t bi = -1;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += 256) {
    const float v = taken[i] ? -1.0f : dist[i];
    if (v > best) {
      best = v;
      bi = i;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      const float v2 = sv[threadIdx.x + o];
      const int64_t i2 = si[threadIdx.x + o];
      if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 >= 0 && (si[threadIdx.x] < 0 || i2 < si[threadIdx.x]))) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bval[blockIdx.x] = sv[0];
    bidx[blockIdx.x] = si[0];
  }
}

__global__ void k_farthest_final(int nblk, int d, const float* __restrict__ bval, const int64_t* __restrict__ bidx,
                                 const float* __restrict__ X, unsigned char* __restrict__ taken,
                                 float* __restrict__ mu_c) {
  __shared__ int64_t win;
  if (threadIdx.x == 0) {
    float best = -2.0f;
    int64_t bi = 0;
    for (int b = 0; b < nblk; ++b) {
      if (bidx[b] >= 0 && (bval[b] > best || (bval[b] == best && bidx[b] < bi))) {
        best = bval[b];
        bi = bidx[b];
      }
    }
    win = bi;
    taken[bi] = 1;
  }
  __syncthreads();
  for (int j = threadIdx.x; j < d; j += blockDim.x) mu_c[j] = X[win * d + j];
}

__global__ void __launch_bounds__(256) k_dist_sum(int64_t n, int64_t chunk, const float* __restrict__ dist,
                                                  double* __restrict__ bsum) {
  __shared__ double sh[256];
  const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += 256) s += (double)dist[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) bsum[blockIdx.x] = sh[0];
}

struct Buffers {
  std::vector<void*> ptrs;
  ~Buffers() {
    for (void* p : ptrs) dev_free(p);
  }
  template <typename T>
  cudaError_t alloc(T** p, size_t count) {
    cudaError_t e = dev_alloc((void**)p, (count > 0 ? count : 1) * sizeof(T));
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
};

int grid_for(int64_t items, int per_block = 256) {
  return (int)std::max<int64_t>(1, std::min<int64_t>(ceil_div(items, per_block), 8 * kNumSMs));
}

}  // namespace
}  // namespace ofsc

using namespace ofsc;

extern "C" ofsc_status ofsc_row_normalize(int64_t n, int32_t k, float* X, void* stream) {
  clear_error();
  if (n < 0 || k < 1) return fail(OFSC_ERR_INVALID_ARG, "ofsc_row_normalize: bad n=%lld k=%d", (long long)n, k);
  if (n == 0) return OFSC_OK;
  if (!X) return fail(OFSC_ERR_INVALID_ARG, "ofsc_row_normalize: X is NULL");
  k_row_normalize<<<grid_for(n * 32), 256, 0, (cudaStream_t)stream>>>(n, k, X);
  OFSC_LAUNCH_CHECK("k_row_normalize");
  return OFSC_OK;
}

extern "C" ofsc_status ofsc_kmeans(int64_t n, int32_t d, const float* X, int32_t C, uint64_t seed,
                                   int32_t n_init, int32_t maxit, int32_t* labels, double* inertia,
                                   void* stream_) {
  clear_error();
  if (n < 1 || d < 1 || C < 1 || C > n || n_init < 1 || maxit < 1)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_kmeans: bad sizes (n=%lld d=%d C=%d n_init=%d maxit=%d)",
                (long long)n, d, C, n_init, maxit);
  if (!X || !labels) return fail(OFSC_ERR_INVALID_ARG, "ofsc_kmeans: NULL pointer");
  const size_t assign_smem = ((size_t)C * d + 8 * 32 * (size_t)(d + 1)) * sizeof(float);
  const size_t part_smem = (size_t)C * d * sizeof(float) + C * sizeof(int);
  if (assign_smem > 200 * 1024 || part_smem > 200 * 1024)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_kmeans: n_clusters * d too large (%d x %d)", C, d);
  cudaStream_t s = (cudaStream_t)stream_;
  OFSC_CUDA(cudaFuncSetAttribute(k_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  OFSC_CUDA(cudaFuncSetAttribute(k_centroid_part, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));

  const int nblk = (int)std::min<int64_t>(kSumBlocks, ceil_div(n, 256));
  const int64_t chunk = ceil_div(n, nblk);
  const int cblk = (int)std::min<int64_t>(2 * kNumSMs, ceil_div(n, 512));
  const int64_t cchunk = ceil_div(n, cblk);

  Buffers b;
  double *D2, *bsum;
  int64_t *centre, *fidx;
  float *mu, *dist, *part, *fval;
  int32_t* lab;
  int *cpart, *counts, *changed;
  unsigned char* taken;
  OFSC_CUDA(b.alloc(&D2, n));
  OFSC_CUDA(b.alloc(&bsum, kSumBlocks));
  OFSC_CUDA(b.alloc(&centre, 1));
  OFSC_CUDA(b.alloc(&fidx, kSumBlocks));
  OFSC_CUDA(b.alloc(&fval, kSumBlocks));
  OFSC_CUDA(b.alloc(&mu, (size_t)C * d));
  OFSC_CUDA(b.alloc(&dist, n));
  OFSC_CUDA(b.alloc(&part, (size_t)cblk * C * d));
  OFSC_CUDA(b.alloc(&lab, n));
  OFSC_CUDA(b.alloc(&cpart, (size_t)cblk * C));
  OFSC_CUDA(b.alloc(&counts, C));
  OFSC_CUDA(b.alloc(&changed, 1));
  OFSC_CUDA(b.alloc(&taken, n));
  std::vector<int> h_counts(C);
  std::vector<double> h_bsum(kSumBlocks);
  int h_changed = 0;
  double best_inertia = INFINITY;
  const int agrid = (int)std::min<int64_t>(ceil_div(ceil_div(n, 32), 8), 2 * kNumSMs);

  for (int run = 0; run < n_init; ++run) {
    // K-means++ seeding
    for (int c = 0; c < C; ++c) {
      if (c > 0) {
        k_chunk_sum<<<nblk, 256, 0, s>>>(n, chunk, D2, bsum);
      }
      k_seed_pick<<<1, 1, 0, s>>>(n, chunk, nblk, D2, bsum, seed, run, c, centre);
      k_copy_centroid<<<1, 128, 0, s>>>(d, X, centre, mu + (size_t)c * d);
      if (c + 1 < C) k_seed_dist<<<grid_for(n), 256, 0, s>>>(n, d, X, centre, D2, c == 0 ? 1 : 0);
    }
    OFSC_LAUNCH_CHECK("k-means++ seeding");
    // Lloyd
    for (int it = 0; it < maxit; ++it) {
      OFSC_CUDA(cudaMemsetAsync(changed, 0, sizeof(int), s));
      k_assign<<<agrid, 256, assign_smem, s>>>(n, d, C, X, mu, lab, dist, changed, it > 0 ? 1 : 0);
      OFSC_LAUNCH_CHECK("k_assign");
      if (it > 0) {
        OFSC_CUDA(cudaMemcpyAsync(&h_changed, changed, sizeof(int), cudaMemcpyDeviceToHost, s));
        OFSC_CUDA(cudaStreamSynchronize(s));
        if (!h_changed) break;
      }
      k_centroid_part<<<cblk, 128, part_smem, s>>>(n, d, C, cchunk, X, lab, part, cpart);
      k_centroid_final<<<grid_for((int64_t)C * d), 256, 0, s>>>(d, C, cblk, part, cpart, mu, counts);
      OFSC_LAUNCH_CHECK("centroid update");
      OFSC_CUDA(cudaMemcpyAsync(h_counts.data(), counts, C * sizeof(int), cudaMemcpyDeviceToHost, s));
      OFSC_CUDA(cudaStreamSynchronize(s));
      bool any_empty = false;
      for (int c = 0; c < C; ++c) any_empty |= (h_counts[c] == 0);
      if (any_empty) {
        OFSC_CUDA(cudaMemsetAsync(taken, 0, n, s));
        for (int c = 0; c < C; ++c) {
          if (h_counts[c] != 0) continue;
          k_farthest_part<<<nblk, 256, 0, s>>>(n, chunk, dist, taken, fval, fidx);
          k_farthest_final<<<1, 128, 0, s>>>(nblk, d, fval, fidx, X, taken, mu + (size_t)c * d);
        }
        OFSC_LAUNCH_CHECK("empty clusters");
      }
    }
    k_assign<<<agrid, 256, assign_smem, s>>>(n, d, C, X, mu, lab, dist, changed, 0);
    k_dist_sum<<<nblk, 256, 0, s>>>(n, chunk, dist, bsum);
    OFSC_LAUNCH_CHECK("final assignment");
    OFSC_CUDA(cudaMemcpyAsync(h_bsum.data(), bsum, nblk * sizeof(double), cudaMemcpyDeviceToHost, s));
    OFSC_CUDA(cudaStreamSynchronize(s));
    double tot = 0.0;
    for (int i = 0; i < nblk; ++i) tot += h_bsum[i];
    if (run == 0 || tot < best_inertia) {
      best_inertia = tot;
      OFSC_CUDA(cudaMemcpyAsync(labels, lab, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
    }
  }
  OFSC_CUDA(cudaStreamSynchronize(s));
  if (inertia) *inertia = best_inertia;
  return OFSC_OK;
}
