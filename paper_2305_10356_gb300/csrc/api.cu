// Error state, the library's device allocator (cudaMalloc or the caller's), graph-handle accessors
// and release.
#include <stdarg.h>

#include <mutex>
#include <unordered_map>

#include "common.cuh"

namespace ofsc {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

void clear_error() { g_last_error.clear(); }

ofsc_status fail(ofsc_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

ofsc_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // allocation failures are not sticky; clear them
    return OFSC_ERR_OOM;
  }
  return OFSC_ERR_CUDA;
}

namespace {
struct Allocator {
  ofsc_alloc_fn alloc = nullptr;
  ofsc_free_fn free = nullptr;
  void* user = nullptr;
};
std::mutex g_alloc_mu;
Allocator g_alloc;                                      // the current one (alloc == NULL: cudaMalloc)
std::unordered_map<void*, Allocator> g_alloc_owner;    // blocks made by a caller's allocator
}  // namespace

cudaError_t dev_alloc_bytes(void** p, size_t bytes) {
  *p = nullptr;
  Allocator a;
  {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    a = g_alloc;
  }
  if (!a.alloc) return cudaMalloc(p, bytes);
  void* q = a.alloc(bytes, a.user);
  if (!q) return cudaErrorMemoryAllocation;
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  g_alloc_owner[q] = a;
  *p = q;
  return cudaSuccess;
}

cudaError_t dev_free(void* p) {
  if (!p) return cudaSuccess;
  Allocator a;
  {
    std::lock_guard<std::mutex> lock(g_alloc_mu);
    auto it = g_alloc_owner.find(p);
    if (it == g_alloc_owner.end()) return cudaFree(p);
    a = it->second;
    g_alloc_owner.erase(it);
  }
  // the caller's allocator may hand the block out again at once: no queued kernel may still use it
  const cudaError_t e = cudaDeviceSynchronize();
  a.free(p, a.user);
  return e;
}

void workspace_free(Workspace& ws) {
  dev_free(ws.X);
  dev_free(ws.Y);
  dev_free(ws.V);
  dev_free(ws.W);
  dev_free(ws.G);
  dev_free(ws.Vh);
  dev_free(ws.gram_part);
  dev_free(ws.gram);
  dev_free(ws.Rn);
  dev_free(ws.Bn);
  dev_free(ws.R64);
  dev_free(ws.B64);
  dev_free(ws.dots);
  dev_free(ws.part_tc);
  dev_free(ws.alpha);
  dev_free(ws.beta);
  dev_free(ws.alpha64);
  dev_free(ws.beta64);
  dev_free(ws.vscale);
  dev_free(ws.vinv);
  dev_free(ws.colpart);
  dev_free(ws.dE);
  dev_free(ws.bimg);
  dev_free(ws.carry_row);
  dev_free(ws.carry);
  dev_free(ws.solve);
  dev_free(ws.ctrl);
  if (ws.ctrl_host) cudaFreeHost(ws.ctrl_host);
  for (cudaEvent_t e : ws.events) cudaEventDestroy(e);
  ws = Workspace();
}

}  // namespace ofsc

extern "C" {

const char* ofsc_last_error(void) { return ofsc::g_last_error.c_str(); }

int32_t ofsc_version(void) { return 100; }

ofsc_status ofsc_graph_free(ofsc_graph* g) {
  if (!g) return OFSC_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(g->device);
  ofsc::workspace_free(g->ws);
  ofsc::dev_free(g->row_ptr);
  ofsc::dev_free(g->col);
  ofsc::dev_free(g->val);
  ofsc::dev_free(g->dinv);
  ofsc::dev_free(g->deg);
  for (int i = 0; i < 6; ++i) ofsc::dev_free(g->bnd[i]);
  ofsc::dev_free(g->mp);
  if (g->stream) cudaStreamDestroy(g->stream);
  if (g->side) cudaStreamDestroy(g->side);
  if (g->side_fork) cudaEventDestroy(g->side_fork);
  if (g->side_join) cudaEventDestroy(g->side_join);
  cudaSetDevice(prev);
  delete g;
  return OFSC_OK;
}

ofsc_status ofsc_graph_get_info(const ofsc_graph* g, ofsc_graph_info* info) {
  if (!g || !info) return ofsc::fail(OFSC_ERR_INVALID_ARG, "ofsc_graph_get_info: NULL argument");
  info->n = g->n;
  info->m_in = g->m_in;
  info->nnz = g->nnz;
  info->n_selfloops = g->n_selfloops;
  info->n_duplicates = g->n_duplicates;
  info->n_isolated = g->n_isolated;
  info->weighted = g->weighted;
  info->normA_fro2 = g->normA2;
  return OFSC_OK;
}

ofsc_status ofsc_graph_csr(const ofsc_graph* g, const int64_t** row_ptr, const int32_t** col,
                           const float** val, const float** dinv, const double** deg) {
  if (!g) return ofsc::fail(OFSC_ERR_INVALID_ARG, "ofsc_graph_csr: NULL graph");
  if (row_ptr) *row_ptr = g->row_ptr;
  if (col) *col = g->col;
  if (val) *val = g->val;
  if (dinv) *dinv = g->dinv;
  if (deg) *deg = g->deg;
  return OFSC_OK;
}

}  // extern "C"

extern "C" ofsc_status ofsc_set_allocator(ofsc_alloc_fn alloc, ofsc_free_fn free_fn, void* user) {
  using namespace ofsc;
  clear_error();
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_set_allocator: give both functions or neither");
  std::lock_guard<std::mutex> lock(g_alloc_mu);
  g_alloc = Allocator{alloc, free_fn, user};
  return OFSC_OK;
}
