// Gram blocks L^T R_b over all N rows on the 5th-generation tensor cores (tcgen05, kind::tf32).
//
// These are the k x k dot products of Sec. 3.3 (V^T X, V^T V, V^T AX, V^T AV, X^T X, X^T AX): dense
// contractions over the N rows with k <= 128 features. One CTA owns a contiguous range of rows:
//   * 4 warps load 32 rows of every block into registers (the next chunk is in flight while the
//     tensor cores work on the current one), split each FP32 value x into tf32 hi = rna(x) and
//     lo = rna(x - hi), and store hi and lo transposed (feature-major, rows contiguous) in the
//     K-major, 128-byte-swizzled shared-memory layout that tcgen05.mma reads;
//   * one thread issues, per 8-row K step, D += Ahi*Bhi + Ahi*Blo + Alo*Bhi (3-term TF32 split,
//     about FP32 accuracy) with D (128 features x 128 nr columns, FP32) in tensor memory, and
//     commits the batch to an mbarrier;
//   * at the end of the range, tcgen05.ld moves D to registers and the CTA writes an FP32
//     partial; a second kernel sums the partials over CTAs in a fixed order in FP64.
// Every wait on the mbarrier is bounded: on expiry the CTA records OFSC_ERR_TIMEOUT, stops
// issuing, frees its tensor memory and returns.
#include <algorithm>

#include "tcgen05.cuh"

namespace ofsc {
namespace {

constexpr int kTcThreads = 128;

}  // namespace

namespace {

template <int NR, bool SEPARATE_L>
__global__ void __launch_bounds__(kTcThreads, 1) k_gram_tc(GramTcArgs a) {
  if (!a.ignore_done && a.ctrl->done) return;
  const long long lim = spin_limit_of(a.ctrl);
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  constexpr int NT = NR + (SEPARATE_L ? 1 : 0);   // staged blocks
  constexpr uint32_t NCOLS = NR * kTcM <= 128 ? 128 : NR * kTcM <= 256 ? 256 : 512;
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* hi = base;                        // NT tiles: R_0..R_{NR-1} [, L]
  unsigned char* lo = base + NT * kTcTile;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lidx = SEPARATE_L ? NR : a.lslot;      // tile index of the A operand
  const float* src[NT];
#pragma unroll
  for (int b = 0; b < NR; ++b) src[b] = a.R[b];
  if (SEPARATE_L) src[NT - 1] = a.L;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(NCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    abort_flag = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t r1 = min(a.n, r0 + a.rows_per_cta);
  const int64_t nchunks = r1 > r0 ? (r1 - r0 + kTcRows - 1) / kTcRows : 0;
  const int f0 = warp * 32;  // this warp's 32 features; lane = chunk row
  float4 buf[NT][8];

  auto fetch = [&](int64_t c) {
    const int64_t row = r0 + c * kTcRows + lane;
    const bool rok = row < r1;
#pragma unroll
    for (int b = 0; b < NT; ++b)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int f = f0 + 4 * i;
        buf[b][i] = (rok && f < a.k) ? *(const float4*)(src[b] + row * a.ld + f) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
  };
  auto stage = [&]() {
#pragma unroll
    for (int b = 0; b < NT; ++b)
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float v[4] = {buf[b][i].x, buf[b][i].y, buf[b][i].z, buf[b][i].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int f = f0 + 4 * i + q;
          const uint32_t h = tf32_rna(v[q]);
          const uint32_t l = tf32_rna(v[q] - __uint_as_float(h));
          const uint32_t off = (uint32_t)b * kTcTile + tile_off(f, lane);
          *(uint32_t*)(hi + off) = h;
          *(uint32_t*)(lo + off) = l;
        }
      }
  };

  uint32_t phase = 0;
  if (nchunks > 0) fetch(0);
  for (int64_t c = 0; c < nchunks; ++c) {
    if (c > 0) {  // the tensor cores must be done reading the tiles before they are rewritten
      if (!mbar_wait(&bar, phase, lim)) abort_flag = 1;
      phase ^= 1;
    }
    __syncthreads();
    if (abort_flag) break;
    stage();
    asm volatile("fence.proxy.async.shared::cta;");  // generic-proxy stores -> tensor-core reads
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t hs = smem_u32(hi), ls = smem_u32(lo);
#pragma unroll
      for (int s = 0; s < kTcRows / 8; ++s) {  // K steps of 8 rows (32 bytes)
        const uint64_t ahi = sw128_desc(hs + lidx * kTcTile + s * 32);
        const uint64_t alo = sw128_desc(ls + lidx * kTcTile + s * 32);
#pragma unroll
        for (int h = 0; h < (NR + 1) / 2; ++h) {  // N = 256 covers right blocks 2h, 2h + 1
          const int ncol = (2 * h + 1 < NR) ? 256 : 128;
          const uint32_t id = tf32_idesc(ncol);
          const uint32_t d = tmem + (uint32_t)(h * 256);
          const uint64_t bhi = sw128_desc(hs + 2 * h * kTcTile + s * 32);
          const uint64_t blo = sw128_desc(ls + 2 * h * kTcTile + s * 32);
          mma_tf32(d, ahi, bhi, id, (c > 0 || s > 0) ? 1u : 0u);
          mma_tf32(d, ahi, blo, id, 1u);
          mma_tf32(d, alo, bhi, id, 1u);
        }
      }
      mma_commit(&bar);
    }
    if (c + 1 < nchunks) fetch(c + 1);  // next chunk's loads overlap the tensor-core work
  }
  bool ok = !abort_flag;
  if (nchunks > 0 && ok) {
    ok = mbar_wait(&bar, phase, lim);
    if (!ok) abort_flag = 1;
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  float* out = a.part + (int64_t)blockIdx.x * NR * kTcM * kTcM;
  const int fi = warp * 32 + lane;  // TMEM lane = feature of L
  if (!abort_flag && nchunks > 0) {
#pragma unroll 1
    for (int c0 = 0; c0 < NR * kTcM; c0 += 32) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
          "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
            "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
            "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
            "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;");
      const int b = c0 / kTcM, j0 = c0 % kTcM;
      float4* dst = (float4*)(out + ((int64_t)b * kTcM + fi) * kTcM + j0);
#pragma unroll
      for (int q = 0; q < 8; ++q)
        dst[q] = make_float4(__uint_as_float(r[4 * q]), __uint_as_float(r[4 * q + 1]),
                             __uint_as_float(r[4 * q + 2]), __uint_as_float(r[4 * q + 3]));
    }
  } else {
    for (int j = 0; j < NR * kTcM; j += 4) {
      const int b = j / kTcM, jj = j % kTcM;
      *(float4*)(out + ((int64_t)b * kTcM + fi) * kTcM + jj) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  if (abort_flag && tid == 0) {
    a.ctrl->status = OFSC_ERR_TIMEOUT;
    a.ctrl->done = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
}

// ------------------------------------------------------------------------------------------
// Warp-specialised Grams for one or two right blocks when the left block is one of them (the
// Grams of every update). One CTA per SM walks a contiguous range of rows in 32-row chunks, and
// no stage waits for another unless a ring is full:
//   * warp 4 (one thread) loads the raw FP32 chunk of every block with TMA, four boxes of 32 rows
//     x 32 features, 128-byte swizzle, into a ring of kWsRaw stages;
//   * warps 0-3 convert a raw chunk into the tf32 hi/lo K-major tiles of a ring of kWsTile stages
//     (warp w owns features 32w..32w+31, lane = feature; the swizzle keeps both the row reads and
//     the 16-byte feature-line writes free of bank conflicts);
//   * warp 5 (one thread) issues each chunk's MMAs as k_gram_tc does, then commits them to free
//     the tile stage and, at a segment end, to hand the accumulator over.
// Accuracy: the tensor cores accumulate a segment of kWsSegRows rows in FP32 in tensor memory
// (columns [0, 128 NR)); its error grows linearly with the rows it holds. At every segment end
// warps 0-3 (TMEM lanes 32w..32w+31 are warp w's) add the segment into a running FP32 total kept
// in columns [128 NR, 256 NR) with round-to-nearest adds, so a CTA's result carries the error of
// one short segment plus about one rounding per segment. The total is written once per CTA and
// the partials are reduced by k_gram_tc_reduce1/2. Every wait is bounded: on expiry the CTA
// records OFSC_ERR_TIMEOUT, every role stops, the TMA copies and MMAs already issued are waited
// for (bounded), and the tensor memory is freed.
#ifndef OFSC_WS_RAW
#define OFSC_WS_RAW 3
#endif
#ifndef OFSC_WS_SEG
#define OFSC_WS_SEG 512
#endif
constexpr int kWsRaw = OFSC_WS_RAW;
constexpr int kWsTile = 2;
constexpr int kWsThreads = 192;
constexpr int kWsBox = 32 * 128;  // one TMA box: 32 rows x 32 FP32 features
constexpr int64_t kWsSegRows = OFSC_WS_SEG;

// SEPL: the left block is staged and converted as a block of its own after the NR right blocks
// (the left block is not one of them); the three blocks of NR = 2 then take a raw ring of two stages
// and one tile stage (193 KB).
template <int NR, bool SEPL>
struct WsShape {
  static constexpr int NB = NR + (SEPL ? 1 : 0);   // blocks staged per chunk
  static constexpr int RAWS = SEPL ? 2 : kWsRaw;    // raw ring stages
  static constexpr int TILES = SEPL ? 1 : kWsTile;  // tile ring stages
  static constexpr int RAW = NB * 4 * kWsBox;       // one raw stage: four boxes per block
  static constexpr int TILE = NB * kTcTile;         // the hi (or lo) tiles of one stage
  static constexpr size_t bytes() { return (size_t)RAWS * RAW + (size_t)TILES * 2 * TILE + 1024; }
};

struct WsArgs {
  int64_t n;
  int lslot;
  int64_t rows_per_cta;  // multiple of 32
  int64_t seg_rows;      // multiple of 32
  float* part;           // [ctas][nr][128][128]
  Ctrl* ctrl;
  int ignore_done;
};

template <int NR, bool SEPL>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_gram_tc_ws(const __grid_constant__ CUtensorMap m0, const __grid_constant__ CUtensorMap m1,
                 const __grid_constant__ CUtensorMap ml, WsArgs a) {
  if (!a.ignore_done && a.ctrl->done) return;
  const long long lim = spin_limit_of(a.ctrl);
  using Sh = WsShape<NR, SEPL>;
  constexpr int RAWS = Sh::RAWS, TILES = Sh::TILES;
  const int atile = SEPL ? NR : a.lslot;  // the tile of the left block (the A operand)
  constexpr uint32_t NCOLS = NR == 1 ? 256 : 512;  // segment accumulator, then the running total
  constexpr uint32_t TOT = NR * kTcM;               // first column of the total
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t raw_full[kWsRaw], raw_empty[kWsRaw], tile_full[kWsTile], tile_empty[kWsTile];
  __shared__ uint64_t acc_full, acc_empty;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* raw = base;                      // [kWsRaw][NR][4 boxes]
  unsigned char* hi = base + RAWS * Sh::RAW;    // [kWsTile][NR tiles]
  unsigned char* lo = hi + TILES * Sh::TILE;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (warp == 5) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(NCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < RAWS; ++st) {
      mbar_init(&raw_full[st], 1);
      mbar_init(&raw_empty[st], 4);
    }
    for (int tt = 0; tt < TILES; ++tt) {
      mbar_init(&tile_full[tt], 4);
      mbar_init(&tile_empty[tt], 1);
    }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, 4);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  const int64_t r0 = (int64_t)blockIdx.x * a.rows_per_cta;
  const int64_t r1 = min(a.n, r0 + a.rows_per_cta);
  const int64_t nchunks = r1 > r0 ? (r1 - r0 + 31) / 32 : 0;
  const int64_t cps = a.seg_rows / 32;  // chunks per segment
  auto seg_last = [&](int64_t c) { return (c + 1) % cps == 0 || c + 1 == nchunks; };

  if (warp == 4) {
    if (lane == 0) {  // producer
      int64_t c = 0;
      for (; c < nchunks; ++c) {
        const int st = (int)(c % RAWS);
        if (c >= RAWS && !ws_wait(&raw_empty[st], (uint32_t)((c / RAWS - 1) & 1), &abort_flag, lim)) break;
        mbar_expect_tx(&raw_full[st], (uint32_t)Sh::RAW);
        const int y = (int)(r0 + c * 32);
        unsigned char* dst = raw + st * Sh::RAW;
#pragma unroll
        for (int b = 0; b < Sh::NB; ++b)
#pragma unroll
          for (int fb = 0; fb < 4; ++fb)
            tma_load_box(dst + (b * 4 + fb) * kWsBox, b == NR ? &ml : (b ? &m1 : &m0), fb * 32, y, &raw_full[st]);
      }
      // the copies already issued must land before the CTA may exit
      for (int64_t d = c > RAWS ? c - RAWS : 0; d < c; ++d) mbar_wait(&raw_full[d % RAWS], (uint32_t)((d / RAWS) & 1), lim);
    }
  } else if (warp == 5) {
    if (lane == 0) {  // MMA issuer
      int64_t c = 0;
      for (; c < nchunks; ++c) {
        const int tt = (int)(c % TILES);
        const int64_t seg = c / cps;
        const bool first = c % cps == 0;
        if (!ws_wait(&tile_full[tt], (uint32_t)((c / TILES) & 1), &abort_flag, lim)) break;
        if (first && seg > 0 && !ws_wait(&acc_empty, (uint32_t)((seg - 1) & 1), &abort_flag, lim)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t hs = smem_u32(hi + tt * Sh::TILE), ls = smem_u32(lo + tt * Sh::TILE);
#pragma unroll
        for (int s = 0; s < 4; ++s) {  // K steps of 8 rows (32 bytes)
          const uint64_t ahi = sw128_desc(hs + atile * kTcTile + s * 32);
          const uint64_t alo = sw128_desc(ls + atile * kTcTile + s * 32);
#pragma unroll
          for (int h = 0; h < (NR + 1) / 2; ++h) {
            const int ncol = (2 * h + 1 < NR) ? 256 : 128;
            const uint32_t id = tf32_idesc(ncol);
            const uint32_t d = tmem + (uint32_t)(h * 256);
            const uint64_t bhi = sw128_desc(hs + 2 * h * kTcTile + s * 32);
            const uint64_t blo = sw128_desc(ls + 2 * h * kTcTile + s * 32);
            mma_tf32(d, ahi, bhi, id, (!first || s > 0) ? 1u : 0u);
            mma_tf32(d, ahi, blo, id, 1u);
            mma_tf32(d, alo, bhi, id, 1u);
          }
        }
        mma_commit(&tile_empty[tt]);
        if (seg_last(c)) mma_commit(&acc_full);
      }
      // the MMAs already issued must finish before the tensor memory is released
      if (c > 0) mbar_wait(&tile_empty[(c - 1) % TILES], (uint32_t)(((c - 1) / TILES) & 1), lim);
    }
  } else {  // warps 0-3: convert, and drain at segment ends
    const int fb = warp;
    const int fi = warp * 32 + lane;  // TMEM lane = feature of the left block
    int64_t c = 0;
    for (; c < nchunks; ++c) {
      const int st = (int)(c % RAWS), tt = (int)(c % TILES);
      if (!ws_wait(&raw_full[st], (uint32_t)((c / RAWS) & 1), &abort_flag, lim)) break;
      if (c >= TILES && !ws_wait(&tile_empty[tt], (uint32_t)((c / TILES - 1) & 1), &abort_flag, lim)) break;
      // lane = feature fb*32 + lane; four consecutive rows per step: four 4-byte reads from the
      // swizzled row lines (one line per read, all lanes distinct words) and one 16-byte store per
      // tile into the feature's K-major line (each group of 8 lanes hits 8 distinct 16-byte banks)
#pragma unroll
      for (int b = 0; b < Sh::NB; ++b) {
        const unsigned char* box = raw + st * Sh::RAW + (b * 4 + fb) * kWsBox + (lane & 3) * 4;
        unsigned char* dh = hi + tt * Sh::TILE + b * kTcTile;
        unsigned char* dl = lo + tt * Sh::TILE + b * kTcTile;
#pragma unroll
        for (int rg = 0; rg < 8; ++rg) {
          uint32_t h[4];
          float l[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int r = 4 * rg + i;
            const float x = *(const float*)(box + r * 128 + ((((lane >> 2) ^ r) & 7) << 4));
            h[i] = tf32_round(x);
            l[i] = x - __uint_as_float(h[i]);  // exact
          }
          const uint32_t off = tile_off(fi, 4 * rg);
          *(uint4*)(dh + off) = make_uint4(h[0], h[1], h[2], h[3]);
          *(float4*)(dl + off) = make_float4(l[0], l[1], l[2], l[3]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;");  // generic-proxy stores -> tensor-core reads
      __syncwarp();
      if (lane == 0) {
        mbar_arrive(&raw_empty[st]);
        mbar_arrive(&tile_full[tt]);
      }
      if (seg_last(c)) {
        const int64_t seg = c / cps;
        if (!ws_wait(&acc_full, (uint32_t)(seg & 1), &abort_flag, lim)) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t lanes = (uint32_t)(warp * 32) << 16;
#pragma unroll 1
        for (uint32_t c0 = 0; c0 < TOT; c0 += 32) {
          uint32_t d[32], t[32];
          tmem_ld32(tmem + lanes + c0, d);
          if (seg > 0) tmem_ld32(tmem + lanes + TOT + c0, t);
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int q = 0; q < 32; ++q)
            t[q] = seg > 0 ? __float_as_uint(__uint_as_float(t[q]) + __uint_as_float(d[q])) : d[q];
          tmem_st32(tmem + lanes + TOT + c0, t);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty);
      }
    }
    // the CTA's total into its partial (zero if it had no rows)
    float* out = a.part + (int64_t)blockIdx.x * NR * kTcM * kTcM;
    if (nchunks > 0 && !abort_flag) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
      for (uint32_t c0 = 0; c0 < TOT; c0 += 32) {
        uint32_t t[32];
        tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + TOT + c0, t);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        const int b = (int)(c0 / kTcM), j0 = (int)(c0 % kTcM);
        float4* dst = (float4*)(out + ((int64_t)b * kTcM + fi) * kTcM + j0);
#pragma unroll
        for (int q = 0; q < 8; ++q)
          dst[q] = make_float4(__uint_as_float(t[4 * q]), __uint_as_float(t[4 * q + 1]), __uint_as_float(t[4 * q + 2]),
                               __uint_as_float(t[4 * q + 3]));
      }
    } else {
      for (int j = 0; j < NR * kTcM; j += 4) {
        const int b = j / kTcM, jj = j % kTcM;
        *(float4*)(out + ((int64_t)b * kTcM + fi) * kTcM + jj) = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (abort_flag && tid == 0) {
    a.ctrl->status = OFSC_ERR_TIMEOUT;
    a.ctrl->done = 1;
  }
  if (warp == 5) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS));
}

// The per-CTA FP32 partials are summed in FP64 in two fixed-order levels: level 1 adds groups of
// kRedGroup consecutive CTAs (all groups and elements in parallel), level 2 adds the groups in
// order. The result does not depend on scheduling.
constexpr int kRedGroup = 32;

__global__ void k_gram_tc_reduce1(const float* __restrict__ part, int nctas, int total, double* __restrict__ lvl1,
                                  const Ctrl* ctrl, int ignore_done) {
  if (ctrl && !ignore_done && ctrl->done) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  const int g = blockIdx.y;
  const int c0 = g * kRedGroup, c1 = min(nctas, c0 + kRedGroup);
  double s = 0.0;
  for (int c = c0; c < c1; ++c) s += (double)part[(int64_t)c * total + t];
  lvl1[(int64_t)g * total + t] = s;
}

// gram[slot[b] * kk_stride + i * ld_out + j] = sum over groups, in order, of lvl1[g][b][i][j], for
// i, j < kout.
__global__ void k_gram_tc_reduce2(const double* __restrict__ lvl1, int ngroups, int nr, int kout, int ld_out,
                                  int64_t kk_stride, int s0, int s1, int s2, int s3, double* __restrict__ gram,
                                  const Ctrl* ctrl, int ignore_done) {
  if (ctrl && !ignore_done && ctrl->done) return;
  const int slot[4] = {s0, s1, s2, s3};
  const int total = nr * kout * kout;
  const int64_t stride = (int64_t)nr * kTcM * kTcM;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int b = t / (kout * kout), ij = t % (kout * kout), i = ij / kout, j = ij % kout;
    const int64_t e = ((int64_t)b * kTcM + i) * kTcM + j;
    double s = 0.0;
    for (int g = 0; g < ngroups; ++g) s += lvl1[g * stride + e];
    gram[(int64_t)slot[b] * kk_stride + (int64_t)i * ld_out + j] = s;
  }
}

template <int NR, bool SEP>
cudaError_t launch_t(const GramTcArgs& a, int grid, cudaStream_t s) {
  constexpr int NT = NR + (SEP ? 1 : 0);
  // Two tile sets (hi, lo) plus alignment slack; at least 100 KB so that at most two CTAs share
  // an SM, which keeps the tensor-memory columns they allocate within the 512 available.
  size_t smem = (size_t)NT * 2 * kTcTile + 1024;
  if (smem < 100 * 1024) smem = 100 * 1024;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_gram_tc<NR, SEP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_gram_tc<NR, SEP><<<grid, kTcThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

// Rows accumulated in one tensor-memory segment. The FP32 accumulation on the tensor cores loses
// about 2e-8 relative per accumulated product block (measured: the error grows linearly with the
// segment: 2e-6 at 256 rows, 1.4e-5 at 2048, 1e-3 at 131072), so segments are kept short and
// summed in FP64 afterwards: 8 CTAs per SM for up to two right blocks, 4 for more.
int64_t gram_tc_rows_per_cta(int64_t n, int nr) {
  const int64_t ctas = nr <= 2 ? 8 * kNumSMs : 4 * kNumSMs;
  int64_t rpc = (n + ctas - 1) / ctas;
  rpc = (rpc + kTcRows - 1) / kTcRows * kTcRows;
  return rpc < kTcRows ? kTcRows : rpc;
}

// Bytes of the partials buffer: the FP32 per-CTA partials, then the FP64 level-1 sums.
static size_t part_floats_bytes(int64_t ctas, int nr) {
  const size_t b = (size_t)(ctas > 0 ? ctas : 1) * nr * kTcM * kTcM * sizeof(float);
  return (b + 255) / 256 * 256;
}

// Row ranges of the warp-specialised kernel: one CTA per SM, each split into segments of
// kWsSegRows rows; returns the CTAs and sets the rows per CTA and the segments per CTA.
static int64_t ws_layout(int64_t n, int64_t* rpc) {
  int64_t r = (n + kNumSMs - 1) / kNumSMs;
  r = std::max<int64_t>(32, (r + 31) / 32 * 32);
  *rpc = r;
  return (n + r - 1) / r;
}

static size_t parts_bytes(int64_t parts, int nr) {
  const int64_t groups = (std::max<int64_t>(parts, 1) + kRedGroup - 1) / kRedGroup;
  return part_floats_bytes(parts, nr) + (size_t)groups * nr * kTcM * kTcM * sizeof(double);
}

size_t gram_tc_part_bytes(int64_t n, int nr, int64_t rows_per_cta) {
  const int64_t ctas = (n + rows_per_cta - 1) / rows_per_cta;
  int64_t rpc;
  const int64_t ws_ctas = ws_layout(n, &rpc);
  return std::max(parts_bytes(ctas, nr), parts_bytes(ws_ctas, nr));
}

// Launches the partial Grams and their FP64 reduction into gram[slot][kp][kp].
cudaError_t gram_tc_launch(GramTcArgs a, const int* slot, int kp, double* gram, cudaStream_t s) {
  return gram_tc_launch_ld(a, slot, kp, kp, (int64_t)kp * kp, gram, s);
}

template <int NR, bool SEPL>
cudaError_t launch_ws(const CUtensorMap& m0, const CUtensorMap& m1, const CUtensorMap& ml, const WsArgs& w,
                      int grid, cudaStream_t s) {
  const size_t smem = WsShape<NR, SEPL>::bytes();
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_gram_tc_ws<NR, SEPL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_gram_tc_ws<NR, SEPL><<<grid, kWsThreads, smem, s>>>(m0, m1, ml, w);
  return cudaGetLastError();
}

cudaError_t gram_tc_launch_ld(GramTcArgs a, const int* slot, int kout, int ld_out, int64_t kk_stride,
                              double* gram, cudaStream_t s) {
  if (a.n <= 0) return cudaSuccess;
  int grid = (int)((a.n + a.rows_per_cta - 1) / a.rows_per_cta);
  const bool sep = a.lslot < 0;
  cudaError_t e = cudaSuccess;
  if (a.use_ws && (sep ? a.nr == 2 : a.nr <= 2)) {
    WsArgs w{};
    const int64_t ctas = ws_layout(a.n, &w.rows_per_cta);
    w.n = a.n;
    w.lslot = a.lslot;
    w.seg_rows = kWsSegRows;
    w.part = a.part;
    w.ctrl = a.ctrl;
    w.ignore_done = a.ignore_done;
    CUtensorMap m0, m1;
    if (tma_encode_f32_sw128(a.R[0], a.n, a.k, a.ld, 32, 32, &m0) != OFSC_OK) return cudaErrorInvalidValue;
    if (a.nr > 1 && tma_encode_f32_sw128(a.R[1], a.n, a.k, a.ld, 32, 32, &m1) != OFSC_OK) return cudaErrorInvalidValue;
    if (a.nr == 1) m1 = m0;
    CUtensorMap ml = m0;
    if (sep && tma_encode_f32_sw128(a.L, a.n, a.k, a.ld, 32, 32, &ml) != OFSC_OK) return cudaErrorInvalidValue;
    e = sep ? launch_ws<2, true>(m0, m1, ml, w, (int)ctas, s)
            : (a.nr == 1 ? launch_ws<1, false>(m0, m1, ml, w, (int)ctas, s)
                         : launch_ws<2, false>(m0, m1, ml, w, (int)ctas, s));
    grid = (int)ctas;  // partials to reduce
  } else {
  switch (a.nr * 2 + (sep ? 1 : 0)) {
    case 2: e = launch_t<1, false>(a, grid, s); break;
    case 3: e = launch_t<1, true>(a, grid, s); break;
    case 4: e = launch_t<2, false>(a, grid, s); break;
    case 5: e = launch_t<2, true>(a, grid, s); break;
    case 6: e = launch_t<3, false>(a, grid, s); break;
    case 7: e = launch_t<3, true>(a, grid, s); break;
    case 8: e = launch_t<4, false>(a, grid, s); break;
    default: e = launch_t<4, true>(a, grid, s); break;
  }
  }
  if (e != cudaSuccess) return e;
  const int total_p = a.nr * kTcM * kTcM;
  const int ngroups = (grid + kRedGroup - 1) / kRedGroup;
  double* lvl1 = (double*)((char*)a.part + part_floats_bytes(grid, a.nr));
  k_gram_tc_reduce1<<<dim3((total_p + 255) / 256, ngroups), 256, 0, s>>>(a.part, grid, total_p, lvl1, a.ctrl,
                                                                          a.ignore_done);
  const int total = a.nr * kout * kout;
  const int rgrid = (int)std::min<int64_t>((total + 255) / 256, 4 * kNumSMs);
  k_gram_tc_reduce2<<<rgrid, 256, 0, s>>>(lvl1, ngroups, a.nr, kout, ld_out, kk_stride, slot[0],
                                          a.nr > 1 ? slot[1] : 0, a.nr > 2 ? slot[2] : 0, a.nr > 3 ? slot[3] : 0,
                                          gram, a.ctrl, a.ignore_done);
  return cudaGetLastError();
}

}  // namespace ofsc

using namespace ofsc;

extern "C" ofsc_status ofsc_gram(int64_t n, int32_t k, int32_t ld, const float* L, int32_t nr,
                                 const float* const* R, int64_t rows_per_block, double* out, void* stream_) {
  clear_error();
  if (n < 0 || k < 1 || k > 128 || ld < k || (ld & 3) || nr < 1 || nr > 4)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_gram: bad sizes (n=%lld k=%d ld=%d nr=%d)", (long long)n, k, ld, nr);
  if (!R || !out || (n > 0 && !L)) return fail(OFSC_ERR_INVALID_ARG, "ofsc_gram: NULL pointer");
  if (((uintptr_t)L & 15) != 0) return fail(OFSC_ERR_INVALID_ARG, "ofsc_gram: L not 16-byte aligned");
  GramTcArgs a{};
  a.n = n;
  a.ld = ld;
  a.k = k;
  a.nr = nr;
  a.L = L;
  a.lslot = -1;
  for (int b = 0; b < nr; ++b) {
    if (n > 0 && (!R[b] || ((uintptr_t)R[b] & 15) != 0))
      return fail(OFSC_ERR_INVALID_ARG, "ofsc_gram: R[%d] NULL or not 16-byte aligned", b);
    a.R[b] = R[b];
    if (R[b] == L && a.lslot < 0) a.lslot = b;
  }
  if (rows_per_block < 0 || (rows_per_block % kTcRows) != 0)
    return fail(OFSC_ERR_INVALID_ARG, "ofsc_gram: rows_per_block must be a non-negative multiple of %d", kTcRows);
  a.rows_per_cta = rows_per_block > 0 ? rows_per_block : gram_tc_rows_per_cta(n, nr);
  a.use_ws = rows_per_block == 0;
  cudaStream_t s = (cudaStream_t)stream_;
  if (n == 0) {
    OFSC_CUDA(cudaMemsetAsync(out, 0, (size_t)nr * k * k * sizeof(double), s));
    return OFSC_OK;
  }
  const size_t pbytes = gram_tc_part_bytes(n, nr, a.rows_per_cta);
  DevBuf pbuf, cbuf;
  OFSC_CUDA(dev_alloc(&pbuf.p, pbytes));
  OFSC_CUDA(dev_alloc(&cbuf.p, sizeof(Ctrl)));
  void* part = pbuf.p;
  Ctrl* ctrl = (Ctrl*)cbuf.p;
  cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), s);
  a.part = (float*)part;
  a.ctrl = ctrl;
  const int slot[4] = {0, 1, 2, 3};
  cudaError_t e = gram_tc_launch_ld(a, slot, k, k, (int64_t)k * k, out, s);
  Ctrl h{};
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return cuda_fail(e, "ofsc_gram");
  OFSC_CUDA(cudaStreamSynchronize(s));
  if (h.status == OFSC_ERR_TIMEOUT) return fail(OFSC_ERR_TIMEOUT, "ofsc_gram: tensor-core wait timed out");
  return OFSC_OK;
}
