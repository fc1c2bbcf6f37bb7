// Registry of grouped twins and the rewrite of a captured batch update into grouped launches.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "group.cuh"

namespace ofsc {

namespace {

struct Twin {
  const void* grouped;
  GroupLayout layout;
};

std::mutex g_group_mu;
std::unordered_map<const void*, Twin>& twins() {
  static std::unordered_map<const void*, Twin> m;
  return m;
}

bool group_lookup(const void* plain, Twin* out) {
  std::lock_guard<std::mutex> lock(g_group_mu);
  auto it = twins().find(plain);
  if (it == twins().end()) return false;
  *out = it->second;
  return true;
}

// One node of a chain, read from the captured graph.
struct Item {
  cudaGraphNode_t node;
  cudaGraphNodeType type;
  cudaKernelNodeParams kp;  // kernel nodes
  Twin twin;                // kernel nodes with a registered twin (twin.grouped != nullptr)
};

struct GroupKey {
  int lane;
  const void* grouped;
  unsigned bx, by, bz;
  size_t smem;
  bool operator<(const GroupKey& o) const {
    if (lane != o.lane) return lane < o.lane;
    if (grouped != o.grouped) return grouped < o.grouped;
    if (bx != o.bx) return bx < o.bx;
    if (by != o.by) return by < o.by;
    if (bz != o.bz) return bz < o.bz;
    return smem < o.smem;
  }
};

bool groupable(const Item& it) {
  return it.type == cudaGraphNodeTypeKernel && it.twin.grouped != nullptr && it.kp.gridDim.z == 1 &&
         it.kp.kernelParams != nullptr && it.kp.extra == nullptr;
}

// Copies a memset, memcpy or kernel node into `out` after `deps`.
cudaError_t copy_node(const Item& it, cudaGraph_t out, const std::vector<cudaGraphNode_t>& deps,
                      cudaGraphNode_t* added) {
  const cudaGraphNode_t* d = deps.empty() ? nullptr : deps.data();
  switch (it.type) {
    case cudaGraphNodeTypeKernel:
      return cudaGraphAddKernelNode(added, out, d, deps.size(), &it.kp);
    case cudaGraphNodeTypeMemset: {
      cudaMemsetParams p{};
      cudaError_t e = cudaGraphMemsetNodeGetParams(it.node, &p);
      if (e != cudaSuccess) return e;
      return cudaGraphAddMemsetNode(added, out, d, deps.size(), &p);
    }
    case cudaGraphNodeTypeMemcpy: {
      cudaMemcpy3DParms p{};
      cudaError_t e = cudaGraphMemcpyNodeGetParams(it.node, &p);
      if (e != cudaSuccess) return e;
      return cudaGraphAddMemcpyNode(added, out, d, deps.size(), &p);
    }
    case cudaGraphNodeTypeEmpty:
      return cudaGraphAddEmptyNode(added, out, d, deps.size());
    default:
      return cudaErrorNotSupported;
  }
}

}  // namespace

bool group_register(const void* plain, const void* grouped, const GroupLayout& layout) {
  std::lock_guard<std::mutex> lock(g_group_mu);
  twins()[plain] = Twin{grouped, layout};
  return true;
}

cudaError_t regroup_chains(cudaGraph_t captured, int lanes, cudaGraph_t* out, int* launches_out) {
  *out = nullptr;
  size_t n = 0;
  cudaError_t e = cudaGraphGetNodes(captured, nullptr, &n);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> nodes(n);
  if (n > 0) {
    e = cudaGraphGetNodes(captured, nodes.data(), &n);
    if (e != cudaSuccess) return e;
  }
  // the chains: every node has at most one dependency and one dependent
  std::unordered_map<cudaGraphNode_t, cudaGraphNode_t> next;
  std::vector<cudaGraphNode_t> roots;
  for (cudaGraphNode_t nd : nodes) {
    size_t nin = 0, nout = 0;
    e = cudaGraphNodeGetDependencies(nd, nullptr, nullptr, &nin);
    if (e == cudaSuccess) e = cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nout);
    if (e != cudaSuccess) return e;
    if (nin > 1 || nout > 1) return cudaErrorNotSupported;
    if (nin == 0) roots.push_back(nd);
    if (nout == 1) {
      cudaGraphNode_t d = nullptr;
      size_t one = 1;
      e = cudaGraphNodeGetDependentNodes(nd, &d, nullptr, &one);
      if (e != cudaSuccess) return e;
      next[nd] = d;
    }
  }
  // chains in the order of their first nodes in the graph's node list (a stable order)
  std::vector<std::vector<Item>> chains;
  size_t seen = 0;
  for (cudaGraphNode_t r : roots) {
    std::vector<Item> ch;
    for (cudaGraphNode_t nd = r; nd != nullptr;) {
      Item it{};
      it.node = nd;
      e = cudaGraphNodeGetType(nd, &it.type);
      if (e != cudaSuccess) return e;
      if (it.type == cudaGraphNodeTypeKernel) {
        e = cudaGraphKernelNodeGetParams(nd, &it.kp);
        if (e != cudaSuccess) return e;
        // a node copied through its parameters loses its launch attributes: take only nodes
        // without a cluster shape or a cooperative launch
        cudaLaunchAttributeValue v{};
        e = cudaGraphKernelNodeGetAttribute(nd, cudaLaunchAttributeClusterDimension, &v);
        if (e != cudaSuccess) return e;
        if ((uint64_t)v.clusterDim.x * v.clusterDim.y * v.clusterDim.z > 1) return cudaErrorNotSupported;
        v = cudaLaunchAttributeValue{};
        e = cudaGraphKernelNodeGetAttribute(nd, cudaLaunchAttributeCooperative, &v);
        if (e != cudaSuccess) return e;
        if (v.cooperative != 0) return cudaErrorNotSupported;
        Twin t{};
        if (group_lookup(it.kp.func, &t)) it.twin = t;
      }
      ch.push_back(it);
      auto f = next.find(nd);
      nd = f == next.end() ? nullptr : f->second;
    }
    seen += ch.size();
    chains.push_back(std::move(ch));
  }
  if (seen != n) return cudaErrorNotSupported;
  // lanes: the chains, largest first (blocks over all their launches), dealt out in snake order
  // so that every lane holds a similar share of the work
  std::vector<int64_t> work(chains.size(), 0);
  for (size_t c = 0; c < chains.size(); ++c)
    for (const Item& it : chains[c])
      if (it.type == cudaGraphNodeTypeKernel)
        work[c] += (int64_t)it.kp.gridDim.x * it.kp.gridDim.y * it.kp.gridDim.z * it.kp.blockDim.x;
  std::vector<size_t> order(chains.size());
  for (size_t c = 0; c < order.size(); ++c) order[c] = c;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return work[a] > work[b]; });
  if (lanes < 1) lanes = 1;
  std::vector<int> lane_of(chains.size(), 0);
  for (size_t i = 0; i < order.size(); ++i) {
    const size_t round = i / (size_t)lanes, r = i % (size_t)lanes;
    lane_of[order[i]] = (int)(round % 2 == 0 ? r : (size_t)lanes - 1 - r);
  }

  cudaGraph_t g = nullptr;
  e = cudaGraphCreate(&g, 0);
  if (e != cudaSuccess) return e;
  std::vector<size_t> pos(chains.size(), 0);
  std::vector<cudaGraphNode_t> last(chains.size(), nullptr);
  int launches = 0;
  auto fail = [&](cudaError_t err) {
    cudaGraphDestroy(g);
    return err;
  };
  while (true) {
    // non-groupable heads first, each copied as it is
    bool any = false, copied = false;
    for (size_t c = 0; c < chains.size(); ++c) {
      while (pos[c] < chains[c].size() && !groupable(chains[c][pos[c]])) {
        const Item& it = chains[c][pos[c]];
        std::vector<cudaGraphNode_t> deps;
        if (last[c]) deps.push_back(last[c]);
        cudaGraphNode_t added = nullptr;
        e = copy_node(it, g, deps, &added);
        if (e != cudaSuccess) return fail(e);
        if (it.type == cudaGraphNodeTypeKernel) ++launches;
        last[c] = added;
        ++pos[c];
        copied = true;
      }
      any = any || pos[c] < chains[c].size();
    }
    if (!any) break;
    if (copied) continue;
    // every remaining head is groupable: group the most common kernel and shape among them
    // (per lane; lanes advance independently, their launches overlap on the device)
    std::map<GroupKey, std::vector<size_t>> by_key;
    for (size_t c = 0; c < chains.size(); ++c) {
      if (pos[c] >= chains[c].size()) continue;
      const Item& it = chains[c][pos[c]];
      by_key[GroupKey{lane_of[c], it.twin.grouped, it.kp.blockDim.x, it.kp.blockDim.y, it.kp.blockDim.z,
                      (size_t)it.kp.sharedMemBytes}].push_back(c);
    }
    auto best = by_key.begin();
    for (auto it = by_key.begin(); it != by_key.end(); ++it)
      if (it->second.size() > best->second.size() ||
          (it->second.size() == best->second.size() && it->second.front() < best->second.front()))
        best = it;
    // the largest problems' blocks first, so that they start first and the launch's tail is short
    std::vector<size_t> members = best->second;
    std::stable_sort(members.begin(), members.end(), [&](size_t a, size_t b) {
      const Item& x = chains[a][pos[a]];
      const Item& y = chains[b][pos[b]];
      return (int64_t)x.kp.gridDim.x * x.kp.gridDim.y > (int64_t)y.kp.gridDim.x * y.kp.gridDim.y;
    });
    const Item& first = chains[members[0]][pos[members[0]]];
    const GroupLayout& L = first.twin.layout;
    if (first.kp.sharedMemBytes > 48 * 1024) {
      e = cudaFuncSetAttribute(first.twin.grouped, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)first.kp.sharedMemBytes);
      if (e != cudaSuccess) return fail(e);
    }
    // kGroupMax problems per launch: the work list is the launch's parameter block
    for (size_t m0 = 0; m0 < members.size(); m0 += (size_t)kGroupMax) {
      const int cnt = (int)std::min<size_t>((size_t)kGroupMax, members.size() - m0);
      std::vector<unsigned char> params(L.bytes, 0);
      int* start = reinterpret_cast<int*>(params.data() + L.off_start);
      int* gridx = reinterpret_cast<int*>(params.data() + L.off_gridx);
      std::memcpy(params.data(), &cnt, sizeof(int));  // count is the first member
      int total = 0;
      std::vector<cudaGraphNode_t> deps;
      for (int i = 0; i < cnt; ++i) {
        const size_t c = members[m0 + i];
        const Item& it = chains[c][pos[c]];
        std::memcpy(params.data() + L.off_args + (size_t)i * L.arg_bytes, it.kp.kernelParams[0], L.arg_bytes);
        const int64_t blocks = (int64_t)it.kp.gridDim.x * it.kp.gridDim.y;
        if ((int64_t)total + blocks > 0x7fffffff) return fail(cudaErrorNotSupported);
        start[i] = total;
        gridx[i] = (int)it.kp.gridDim.x;
        total += (int)blocks;
        if (last[c]) deps.push_back(last[c]);
      }
      start[cnt] = total;
      void* kparams[1] = {params.data()};
      cudaKernelNodeParams p{};
      p.func = const_cast<void*>(first.twin.grouped);
      p.gridDim = dim3((unsigned)total, 1, 1);
      p.blockDim = first.kp.blockDim;
      p.sharedMemBytes = first.kp.sharedMemBytes;
      p.kernelParams = kparams;
      std::sort(deps.begin(), deps.end());
      deps.erase(std::unique(deps.begin(), deps.end()), deps.end());
      cudaGraphNode_t added = nullptr;
      e = cudaGraphAddKernelNode(&added, g, deps.empty() ? nullptr : deps.data(), deps.size(), &p);
      if (e != cudaSuccess) return fail(e);
      ++launches;
      for (int i = 0; i < cnt; ++i) {
        last[members[m0 + i]] = added;
        ++pos[members[m0 + i]];
      }
    }
  }
  *out = g;
  if (launches_out) *launches_out = launches;
  return cudaSuccess;
}

}  // namespace ofsc
