// Grouped launches: one launch runs the same kernel body for several independent problems (the
// graphs of a batch), each with its own argument block and its own grid. The blocks of all the
// problems are laid end to end over blockIdx.x: this flattened (problem, block) work list lets one
// launch per kernel of an update cover many problems, while every problem's blocks see the block
// indices and grid of its own launch, so its arithmetic is that of its own launch bit for bit.
//
// A kernel that can run grouped has its body compiled twice: in the plain __global__ kernel, which
// takes the argument struct, and in a grouped __global__ twin, which takes a GroupParams holding up
// to kGroupMax problems' argument structs and finds its own. The work list travels in the twin's
// kernel parameters (read-only parameter space, read through the constant cache, never aliased by
// the body's stores). The twins are registered against the plain kernels (group_register), so a
// captured update can be rewritten into grouped launches (regroup_chains).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

namespace ofsc {

// A block's place in the launch the body was written for.
struct VBlock {
  int x, y;    // blockIdx.x, blockIdx.y
  int gx, gy;  // gridDim.x, gridDim.y
};

__device__ __forceinline__ VBlock hw_block() {
  return VBlock{(int)blockIdx.x, (int)blockIdx.y, (int)gridDim.x, (int)gridDim.y};
}

// Problems per grouped launch (a lane with more takes several launches).
constexpr int kGroupMax = 32;

// The work list of one grouped launch, passed by value as its kernel parameter.
template <class A>
struct GroupParams {
  int count;
  int start[kGroupMax + 1];  // first flattened block of each problem, then the total
  int gridx[kGroupMax];      // grid.x of each problem's own launch (grid.y = blocks / grid.x)
  A args[kGroupMax];         // each problem's argument struct
};

// This block's problem (binary search over `start`) and its place in that problem's launch.
template <class A>
__device__ __forceinline__ const A& group_find(const GroupParams<A>& p, VBlock* vb) {
  const int b = (int)blockIdx.x;
  int lo = 0, hi = p.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.start[mid] <= b) lo = mid;
    else hi = mid - 1;
  }
  const int local = b - p.start[lo];
  const int gx = p.gridx[lo];
  vb->x = local % gx;
  vb->y = local / gx;
  vb->gx = gx;
  vb->gy = (p.start[lo + 1] - p.start[lo]) / gx;
  return p.args[lo];
}

// Host-side layout of GroupParams<A>, so that the rewrite can fill one for any registered kernel.
struct GroupLayout {
  size_t bytes;      // sizeof(GroupParams<A>)
  size_t off_start;  // offsetof(..., start)
  size_t off_gridx;  // offsetof(..., gridx)
  size_t off_args;   // offsetof(..., args)
  size_t arg_bytes;  // sizeof(A), also the stride of args
};

template <class A>
GroupLayout group_layout() {
  return GroupLayout{sizeof(GroupParams<A>), offsetof(GroupParams<A>, start), offsetof(GroupParams<A>, gridx),
                     offsetof(GroupParams<A>, args), sizeof(A)};
}

// Registers `grouped` (a kernel taking one GroupParams<A>) as the twin of `plain` (a kernel taking
// one A). Thread-safe; returns true (for one-time static initialisers).
bool group_register(const void* plain, const void* grouped, const GroupLayout& layout);

// Registers a plain kernel's twin once, at the first launch through the enclosing code (wrap a
// template-id with commas in parentheses).
#define OFSC_GROUPABLE(plain, grouped, Args)                                                          \
  do {                                                                                                 \
    static const bool ofsc_registered_ = ::ofsc::group_register(                                       \
        (const void*)(plain), (const void*)(grouped), ::ofsc::group_layout<Args>());                  \
    (void)ofsc_registered_;                                                                            \
  } while (0)

// From `captured`, a graph made of independent chains (one per problem: the same update of
// independent problems, captured on one stream each), builds `*out`: each chain's nodes keep
// their order, and at each step the chains whose next node launches the same registered kernel
// with the same block shape and shared memory share grouped launches (up to kGroupMax problems
// each), the largest problems' blocks first. The chains are dealt into `lanes` lanes of similar
// work (largest first, snake order) and grouped only within a lane: a grouped launch waits for the
// previous launch of every problem it serves, so separate lanes let one lane's short single-block
// steps (beta, the cubic's solve) overlap another lane's sparse products. Kernels without a twin,
// memsets and copies are copied as they are. Fails with cudaErrorNotSupported on any other node,
// on a kernel node with a cluster shape or a cooperative launch, or on a graph that is not a set
// of chains (the caller then keeps `captured`). `launches_out` (nullable) receives the kernel
// nodes of `*out`.
cudaError_t regroup_chains(cudaGraph_t captured, int lanes, cudaGraph_t* out, int* launches_out);

}  // namespace ofsc
