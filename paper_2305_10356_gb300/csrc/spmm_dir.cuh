// Arguments and entry points of the sparse products W = A V (the direction product, spmm_dir.cu)
// and A X, with A = L - 2I = -I - D^-1/2 S D^-1/2 (Eq. (1)).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ofsc {

struct Ctrl;

// Operands of the two sparse products: the direction product W = A V (k_spmm_dir, gathering
// Vh = D^-1/2 V) and the exact AX = A X (k_spmm, gathering X and scaling by D^-1/2 per nonzero).
struct SpmmArgs {
  int64_t n;
  int kp;
  const int64_t* row_ptr;
  const int32_t* col;
  const float* val;
  const float* dinv;
  const int64_t* bnd;  // [groups + 1]: contiguous, nnz-balanced row ranges of the lane groups / warps
  int groups;
  const void* gather;  // direction: Vh = D^-1/2 V (FP32 or BF16); AX: X
  const float* base;   // direction: V; AX: X  (the row block M in A M = -M - D^-1/2 S D^-1/2 M)
  float* out;          // direction: W = AV; AX: AX
  double* dots;        // direction with dots: [blocks][kp] partials of diag(V^T AV)
  Ctrl* ctrl;
  int ignore_done;
  // Merge-path split (k_spmm_dir only; NULL: the row ranges of bnd): mp[0 .. groups] are the first
  // rows and mp[groups + 1 .. 2 groups + 1] the first nonzeros of the warps' equal shares of the
  // rows + nonzeros, so a long row can span warps. A warp's partial sums of a row it does not
  // finish, or did not start, go to carry (row ids in carry_row: [warp][2], -1 none; slot 0 the
  // row the warp finishes, slot 1 the row it leaves unfinished, as r if it started it, else
  // -(r + 2)), and k_spmm_fixup adds them in warp order and writes those rows.
  const int64_t* mp;
  int64_t* carry_row;  // [groups][2]
  float* carry;        // [groups][2][kp]
};

// The direction product (spmm_dir.cu): lanes per nonzero for rows of kp values with vpl values per
// lane; the default and the candidate numbers of gathers in flight per lane; the launch (slots 0:
// the default), returning the rows of dots partials it writes (one per warp).
int dir_lanes(int kp, int vpl);
int dir_default_slots(int kp, bool bf16, bool weighted);
int dir_slot_options(int kp, bool bf16, int* out);
int launch_spmm_dir(const SpmmArgs& a, bool weighted, bool bf16, int slots, cudaStream_t s);
// The merge-path partition of `warps` warps over the rows + nonzeros of row_ptr into mp[2 warps + 2],
// and the largest row (nonzeros) into *max_row (device int64, atomically maximised: zero it first).
cudaError_t merge_partition(int64_t n, const int64_t* row_ptr, int warps, int64_t* mp, cudaStream_t s);
cudaError_t max_row_length(int64_t n, const int64_t* row_ptr, unsigned long long* max_row, cudaStream_t s);
// Checked builds (OFSC_DEBUG): the first out-of-range access the direction product recorded since
// the last call, (kind << 60) | value, or 0, and clears it (synchronous: call after the stream
// has drained). Release builds: always 0.
cudaError_t spmm_dir_take_bounds(unsigned long long* code);

}  // namespace ofsc
