// ofsc_graph_build: S, D and D^-1/2 of Eq. (1) from an undirected edge list, on the device.
//
// Each input edge {u, v} with u != v contributes the directed entries (u, v) and (v, u). The
// entries are keyed by (row, col), sorted with a stable radix sort, and equal keys are merged:
// a binary S keeps one entry of weight 1, a weighted S sums the FP32 weights of the merged
// entries in FP64 (in input order, which the stable sort preserves) and rounds once to FP32.
// Degrees are integer counts (binary) or FP64 sums in column order (weighted); D^-1/2 is
// (float)(1.0 / sqrt(D_ii)) in IEEE FP64, 0 for isolated nodes.
#include <cub/cub.cuh>

#include "common.cuh"

namespace ofsc {
namespace {

__global__ void k_validate(int64_t m, int64_t n, const int32_t* __restrict__ src,
                           const int32_t* __restrict__ dst, const float* __restrict__ w,
                           int* __restrict__ flags, unsigned long long* __restrict__ loops) {
  unsigned long long my_loops = 0;
  int bad = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    int32_t u = src[e], v = dst[e];
    if (u < 0 || v < 0 || u >= n || v >= n) bad |= 1;
    if (w) {
      float x = w[e];
      if (!(isfinite(x) && x > 0.0f)) bad |= 2;
    }
    my_loops += (u == v);
  }
  if (bad) atomicOr(flags, bad);
  for (int o = 16; o > 0; o >>= 1) my_loops += __shfl_down_sync(0xffffffffu, my_loops, o);
  if ((threadIdx.x & 31) == 0 && my_loops) atomicAdd(loops, my_loops);
}

// keys[e] = (u << bits) | v for e < m and (v << bits) | u for m <= e < 2m; a self-loop gets the
// sentinel key n << bits, which sorts after every valid key.
__global__ void k_make_keys(int64_t m, int64_t n, int bits, const int32_t* __restrict__ src,
                            const int32_t* __restrict__ dst, const float* __restrict__ w,
                            uint64_t* __restrict__ keys, float* __restrict__ vals) {
  const uint64_t sentinel = (uint64_t)n << bits;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < m;
       e += (int64_t)gridDim.x * blockDim.x) {
    uint64_t u = (uint32_t)src[e], v = (uint32_t)dst[e];
    bool loop = (u == v);
    keys[e] = loop ? sentinel : ((u << bits) | v);
    keys[m + e] = loop ? sentinel : ((v << bits) | u);
    if (vals) {
      vals[e] = w[e];
      vals[m + e] = w[e];
    }
  }
}

__global__ void k_heads(int64_t nvalid, const uint64_t* __restrict__ keys, int64_t* __restrict__ head) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvalid;
       i += (int64_t)gridDim.x * blockDim.x)
    head[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1 : 0;
}

// Unique entry u = idx[i] - 1 for each head i: column, row, merged weight.
__global__ void k_scatter(int64_t nvalid, int bits, const uint64_t* __restrict__ keys,
                          const float* __restrict__ vals, const int64_t* __restrict__ idx,
                          int32_t* __restrict__ col, int32_t* __restrict__ row_of,
                          float* __restrict__ val) {
  const uint64_t mask = (1ull << bits) - 1ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nvalid;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = keys[i];
    if (i > 0 && keys[i - 1] == key) continue;
    int64_t u = idx[i] - 1;
    col[u] = (int32_t)(key & mask);
    row_of[u] = (int32_t)(key >> bits);
    if (vals) {
      double s = 0.0;
      for (int64_t j = i; j < nvalid && keys[j] == key; ++j) s += (double)vals[j];
      val[u] = (float)s;
    }
  }
}

__global__ void k_row_ptr(int64_t nnz, int64_t n, const int32_t* __restrict__ row_of,
                          int64_t* __restrict__ row_ptr) {
  for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < nnz;
       u += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = row_of[u];
    int64_t prev = (u == 0) ? -1 : (int64_t)row_of[u - 1];
    for (int64_t q = prev + 1; q <= r; ++q) row_ptr[q] = u;
    if (u == nnz - 1)
      for (int64_t q = r + 1; q <= n; ++q) row_ptr[q] = nnz;
  }
}

__global__ void k_degree(int64_t n, const int64_t* __restrict__ row_ptr, const float* __restrict__ val,
                         double* __restrict__ deg, float* __restrict__ dinv, double* __restrict__ dinv64,
                         unsigned long long* __restrict__ isolated) {
  unsigned long long iso = 0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    int64_t p0 = row_ptr[r], p1 = row_ptr[r + 1];
    double d;
    if (val) {
      d = 0.0;
      for (int64_t p = p0; p < p1; ++p) d += (double)val[p];
    } else {
      d = (double)(p1 - p0);
    }
    deg[r] = d;
    const double s64 = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    dinv64[r] = s64;
    dinv[r] = (float)s64;
    iso += (d == 0.0);
  }
  for (int o = 16; o > 0; o >>= 1) iso += __shfl_down_sync(0xffffffffu, iso, o);
  if ((threadIdx.x & 31) == 0 && iso) atomicAdd(isolated, iso);
}

// Per-block partial of sum_ij (s_i S_ij s_j)^2 with s = 1/sqrt(D) in FP64; fixed block order.
constexpr int kNormBlocks = 256;
__global__ void __launch_bounds__(256) k_normA_part(int64_t n, const int64_t* __restrict__ row_ptr,
                                                    const int32_t* __restrict__ col,
                                                    const float* __restrict__ val,
                                                    const double* __restrict__ dinv64,
                                                    double* __restrict__ part) {
  double acc = 0.0;
  for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
       r += (int64_t)gridDim.x * blockDim.x) {
    const double sr = dinv64[r];
    if (sr == 0.0) continue;
    for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) {
      const double a = sr * (val ? (double)val[p] : 1.0) * dinv64[col[p]];
      acc += a * a;
    }
  }
  __shared__ double sh[256];
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// bnd[g] = first row whose row pointer is >= g * nnz / groups (bnd[groups] = n).
__global__ void k_partition(int64_t n, const int64_t* __restrict__ row_ptr, int groups, int64_t* __restrict__ bnd) {
  const int64_t nnz = row_ptr[n];
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g <= groups; g += gridDim.x * blockDim.x) {
    if (g == 0 || g == groups) {
      bnd[g] = g == 0 ? 0 : n;
      continue;
    }
    const int64_t target = nnz * (int64_t)g / groups;  // nnz < 2^31, g < 2^17: no overflow
    int64_t lo = 0, hi = n;  // first r in [0, n] with row_ptr[r] >= target
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (row_ptr[mid] < target) lo = mid + 1;
      else hi = mid;
    }
    bnd[g] = lo;
  }
}

int bit_length(uint64_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

int grid_for(int64_t items, int threads = 256) {
  int64_t g = ceil_div(items > 0 ? items : 1, threads);
  return (int)(g < 8 * kNumSMs ? g : 8 * kNumSMs);
}

struct Scratch {
  void* p[12] = {};
  ~Scratch() {
    for (void* q : p) dev_free(q);
  }
};

}  // namespace

ofsc_status set_row_partition(ofsc_graph* g, int warps, cudaStream_t s) {
  if (warps < 1 || warps > kRowMaxWarps) return fail(OFSC_ERR_INVALID_ARG, "row partition: %d warps", warps);
  int64_t* nb = nullptr;
  int64_t* nmp = nullptr;
  OFSC_CUDA(dev_alloc(&nb, (size_t)(warps + 1) * sizeof(int64_t)));
  cudaError_t e = dev_alloc(&nmp, (size_t)(2 * warps + 2) * sizeof(int64_t));
  if (e == cudaSuccess) {
    k_partition<<<grid_for(warps + 1), 256, 0, s>>>(g->n, g->row_ptr, warps, nb);
    e = cudaGetLastError();
  }
  // the merge-path shares follow the same warp count (the product reads mp[0 .. 2 warps + 1])
  if (e == cudaSuccess) e = merge_partition(g->n, g->row_ptr, warps, nmp, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    dev_free(nb);
    dev_free(nmp);
    return cuda_fail(e, "row partition");
  }
  dev_free(g->bnd[kRowPart]);  // synchronises with any queued use of the old ranges
  dev_free(g->mp);
  g->bnd[kRowPart] = nb;
  g->mp = nmp;
  g->groups[kRowPart] = warps;
  return OFSC_OK;
}

}  // namespace ofsc

using namespace ofsc;

extern "C" ofsc_status ofsc_graph_build(int64_t n, int64_t m, const int32_t* src, const int32_t* dst,
                                        const float* w, uint32_t flags, void* stream_,
                                        ofsc_graph** out) {
  clear_error();
  NvtxRange nv("ofsc_graph_build");
  if (!out) return fail(OFSC_ERR_INVALID_ARG, "ofsc_graph_build: out is NULL");
  *out = nullptr;
  if (n < 0 || n >= (int64_t(1) << 31))
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_graph_build: n=%lld outside [0, 2^31)", (long long)n);
  // m < 2^30 keeps the 2 m directed entries within the int item count of CUB's radix sort (the
  // paper's largest graph, 970M stored nonzeros, is 485M listed edges)
  if (m < 0 || m >= (int64_t(1) << 30))
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_graph_build: m=%lld outside [0, 2^30)", (long long)m);
  if (flags != 0) return fail(OFSC_ERR_INVALID_ARG, "ofsc_graph_build: flags must be 0");
  if (m > 0 && (!src || !dst)) return fail(OFSC_ERR_INVALID_ARG, "ofsc_graph_build: src/dst NULL");
  cudaStream_t stream = (cudaStream_t)stream_;

  ofsc_graph* g = new ofsc_graph();
  cudaGetDevice(&g->device);
  g->n = n;
  g->m_in = m;
  g->weighted = (w != nullptr);
  struct Guard {
    ofsc_graph*& g;
    bool keep = false;
    ~Guard() {
      if (!keep) ofsc_graph_free(g);
    }
  } guard{g};

  Scratch sc;
  int* d_flags = nullptr;
  unsigned long long* d_counts = nullptr;  // [0] self-loops, [1] isolated
  OFSC_CUDA(dev_alloc(&d_flags, sizeof(int)));
  sc.p[0] = d_flags;
  OFSC_CUDA(dev_alloc(&d_counts, 2 * sizeof(unsigned long long)));
  sc.p[1] = d_counts;
  OFSC_CUDA(cudaMemsetAsync(d_flags, 0, sizeof(int), stream));
  OFSC_CUDA(cudaMemsetAsync(d_counts, 0, 2 * sizeof(unsigned long long), stream));

  OFSC_CUDA(dev_alloc(&g->row_ptr, (n + 1) * sizeof(int64_t)));
  OFSC_CUDA(dev_alloc(&g->dinv, (n > 0 ? n : 1) * sizeof(float)));
  OFSC_CUDA(dev_alloc(&g->deg, (n > 0 ? n : 1) * sizeof(double)));

  int64_t nvalid = 0, nnz = 0;
  unsigned long long h_counts[2] = {0, 0};
  if (m > 0) {
    k_validate<<<grid_for(m), 256, 0, stream>>>(m, n, src, dst, w, d_flags, d_counts);
    OFSC_LAUNCH_CHECK("k_validate");
    int h_flags = 0;
    OFSC_CUDA(cudaMemcpyAsync(&h_flags, d_flags, sizeof(int), cudaMemcpyDeviceToHost, stream));
    OFSC_CUDA(cudaMemcpyAsync(h_counts, d_counts, sizeof(h_counts), cudaMemcpyDeviceToHost, stream));
    OFSC_CUDA(cudaStreamSynchronize(stream));
    if (h_flags & 1) return fail(OFSC_ERR_INVALID_ARG, "ofsc_graph_build: node id outside [0, n)");
    if (h_flags & 2) return fail(OFSC_ERR_INVALID_ARG, "ofsc_graph_build: weight not finite or <= 0");
    nvalid = 2 * (m - (int64_t)h_counts[0]);
  }
  g->n_selfloops = (int64_t)h_counts[0];

  const int bits = bit_length((uint64_t)(n > 1 ? n - 1 : 1));
  const int end_bit = bits + bit_length((uint64_t)n);
  if (m > 0) {
    const int64_t m2 = 2 * m;
    uint64_t *keys_a = nullptr, *keys_b = nullptr;
    float *vals_a = nullptr, *vals_b = nullptr;
    OFSC_CUDA(dev_alloc(&keys_a, m2 * sizeof(uint64_t)));
    sc.p[2] = keys_a;
    OFSC_CUDA(dev_alloc(&keys_b, m2 * sizeof(uint64_t)));
    sc.p[3] = keys_b;
    if (w) {
      OFSC_CUDA(dev_alloc(&vals_a, m2 * sizeof(float)));
      sc.p[4] = vals_a;
      OFSC_CUDA(dev_alloc(&vals_b, m2 * sizeof(float)));
      sc.p[5] = vals_b;
    }
    k_make_keys<<<grid_for(m), 256, 0, stream>>>(m, n, bits, src, dst, w, keys_a, vals_a);
    OFSC_LAUNCH_CHECK("k_make_keys");
    cub::DoubleBuffer<uint64_t> kb(keys_a, keys_b);
    cub::DoubleBuffer<float> vb(vals_a, vals_b);
    size_t temp = 0;
    if (w)
      OFSC_CUDA(cub::DeviceRadixSort::SortPairs(nullptr, temp, kb, vb, (int)m2, 0, end_bit, stream));
    else
      OFSC_CUDA(cub::DeviceRadixSort::SortKeys(nullptr, temp, kb, (int)m2, 0, end_bit, stream));
    void* d_temp = nullptr;
    OFSC_CUDA(dev_alloc(&d_temp, temp > 0 ? temp : 1));
    sc.p[6] = d_temp;
    if (w)
      OFSC_CUDA(cub::DeviceRadixSort::SortPairs(d_temp, temp, kb, vb, (int)m2, 0, end_bit, stream));
    else
      OFSC_CUDA(cub::DeviceRadixSort::SortKeys(d_temp, temp, kb, (int)m2, 0, end_bit, stream));
    const uint64_t* keys = kb.Current();
    const float* vals = w ? vb.Current() : nullptr;

    if (nvalid > 0) {
      int64_t* head = nullptr;
      OFSC_CUDA(dev_alloc(&head, nvalid * sizeof(int64_t)));
      sc.p[7] = head;
      k_heads<<<grid_for(nvalid), 256, 0, stream>>>(nvalid, keys, head);
      OFSC_LAUNCH_CHECK("k_heads");
      size_t temp2 = 0;
      OFSC_CUDA(cub::DeviceScan::InclusiveSum(nullptr, temp2, head, head, (int)nvalid, stream));
      void* d_temp2 = nullptr;
      OFSC_CUDA(dev_alloc(&d_temp2, temp2 > 0 ? temp2 : 1));
      sc.p[8] = d_temp2;
      OFSC_CUDA(cub::DeviceScan::InclusiveSum(d_temp2, temp2, head, head, (int)nvalid, stream));
      OFSC_CUDA(cudaMemcpyAsync(&nnz, head + nvalid - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, stream));
      OFSC_CUDA(cudaStreamSynchronize(stream));
      OFSC_CUDA(dev_alloc(&g->col, nnz * sizeof(int32_t)));
      if (w) OFSC_CUDA(dev_alloc(&g->val, nnz * sizeof(float)));
      int32_t* row_of = nullptr;
      OFSC_CUDA(dev_alloc(&row_of, nnz * sizeof(int32_t)));
      sc.p[9] = row_of;
      k_scatter<<<grid_for(nvalid), 256, 0, stream>>>(nvalid, bits, keys, vals, head, g->col,
                                                       row_of, g->val);
      OFSC_LAUNCH_CHECK("k_scatter");
      k_row_ptr<<<grid_for(nnz), 256, 0, stream>>>(nnz, n, row_of, g->row_ptr);
      OFSC_LAUNCH_CHECK("k_row_ptr");
    }
  }
  if (nnz == 0) OFSC_CUDA(cudaMemsetAsync(g->row_ptr, 0, (n + 1) * sizeof(int64_t), stream));
  g->nnz = nnz;
  g->n_duplicates = nvalid - nnz;

  double normA2 = (double)n;
  if (n > 0) {
    double* dinv64 = nullptr;
    OFSC_CUDA(dev_alloc(&dinv64, n * sizeof(double)));
    sc.p[11] = dinv64;
    k_degree<<<grid_for(n), 256, 0, stream>>>(n, g->row_ptr, g->val, g->deg, g->dinv, dinv64, d_counts + 1);
    OFSC_LAUNCH_CHECK("k_degree");
    double* part = nullptr;
    OFSC_CUDA(dev_alloc(&part, kNormBlocks * sizeof(double)));
    sc.p[10] = part;
    k_normA_part<<<kNormBlocks, 256, 0, stream>>>(n, g->row_ptr, g->col, g->val, dinv64, part);
    OFSC_LAUNCH_CHECK("k_normA_part");
    double h_part[kNormBlocks];
    OFSC_CUDA(cudaMemcpyAsync(h_part, part, sizeof(h_part), cudaMemcpyDeviceToHost, stream));
    OFSC_CUDA(cudaMemcpyAsync(h_counts, d_counts, sizeof(h_counts), cudaMemcpyDeviceToHost, stream));
    OFSC_CUDA(cudaStreamSynchronize(stream));
    for (int b = 0; b < kNormBlocks; ++b) normA2 += h_part[b];
    g->n_isolated = (int64_t)h_counts[1];
  }
  g->normA2 = normA2;
  for (int i = 0; i < 6; ++i) {
    g->groups[i] = i == kRowPart ? row_warps(nnz) : spmm_groups(nnz, 2 << i);
    OFSC_CUDA(dev_alloc(&g->bnd[i], (g->groups[i] + 1) * sizeof(int64_t)));
    k_partition<<<grid_for(g->groups[i] + 1), 256, 0, stream>>>(n, g->row_ptr, g->groups[i], g->bnd[i]);
    OFSC_LAUNCH_CHECK("k_partition");
  }
  // the merge-path shares of the direction product's warps, and the longest row
  OFSC_CUDA(dev_alloc(&g->mp, (size_t)(2 * g->groups[kRowPart] + 2) * sizeof(int64_t)));
  OFSC_CUDA(merge_partition(n, g->row_ptr, g->groups[kRowPart], g->mp, stream));
  unsigned long long* d_max = (unsigned long long*)d_counts;  // the counts were read above
  OFSC_CUDA(cudaMemsetAsync(d_max, 0, sizeof(unsigned long long), stream));
  OFSC_CUDA(max_row_length(n, g->row_ptr, d_max, stream));
  unsigned long long h_max = 0;
  OFSC_CUDA(cudaMemcpyAsync(&h_max, d_max, sizeof(h_max), cudaMemcpyDeviceToHost, stream));
  OFSC_CUDA(cudaStreamSynchronize(stream));
  g->max_row = (int64_t)h_max;
  guard.keep = true;
  *out = g;
  return OFSC_OK;
}
