// Error state, graph-handle accessors and release.
#include <stdarg.h>

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

void workspace_free(Workspace& ws) {
  cudaFree(ws.X);
  cudaFree(ws.Y);
  cudaFree(ws.V);
  cudaFree(ws.W);
  cudaFree(ws.G);
  cudaFree(ws.Vh);
  cudaFree(ws.gram_part);
  cudaFree(ws.gram);
  cudaFree(ws.Rn);
  cudaFree(ws.Bn);
  cudaFree(ws.R64);
  cudaFree(ws.B64);
  cudaFree(ws.dots);
  cudaFree(ws.part_tc);
  cudaFree(ws.alpha);
  cudaFree(ws.beta);
  cudaFree(ws.alpha64);
  cudaFree(ws.beta64);
  cudaFree(ws.vscale);
  cudaFree(ws.vinv);
  cudaFree(ws.colpart);
  cudaFree(ws.dE);
  cudaFree(ws.solve);
  cudaFree(ws.ctrl);
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
  cudaFree(g->row_ptr);
  cudaFree(g->col);
  cudaFree(g->val);
  cudaFree(g->dinv);
  cudaFree(g->deg);
  for (int i = 0; i < 6; ++i) cudaFree(g->bnd[i]);
  if (g->stream) cudaStreamDestroy(g->stream);
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
