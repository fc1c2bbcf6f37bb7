// The direction pass of OFM-f1 (Eq. (5)) and TriOFM-f1 (Eq. (7)) at padded k = 128 with the
// N x 128 by 128 x 128 product on the 5th-generation tensor cores. Per 128-row tile:
//   X_new = X + V diag(alpha),  AX_new = AX + AV diag(alpha)      (the previous update)
//   P = X_new R' (R' = X^T X, or triu(X^T X) for TriOFM)           (tcgen05 kind::tf32, 3 terms)
//   G = 4 (AX_new + P) (OFM-f1) or AX_new + P (TriOFM-f1)
// and the six column sums of the SIMT k_direction (G^2, (G - G_prev) G, G_prev^2, G AX,
// V_prev AX, V_prev G). One CTA per SM walks its tiles:
//   * warps 0-3 (converters) form X_new in 32-feature chunks with coalesced row loads, store it,
//     and write its tf32 hi/lo parts straight into K-major 128-byte-swizzled shared tiles (eight
//     lanes cover a row's 128-byte chunk, so the 16-byte stores are conflict-free), a ring of two
//     chunk stages;
//   * warp 8 (one thread) issues per chunk D += Ahi R'hi + Ahi R'lo + Alo R'hi into one of two
//     128-column tensor-memory accumulators (R' hi/lo stay in shared memory, built at the start);
//   * warps 4-7 (epilogue; TMEM lanes 32(w-4)..) move P out with tcgen05.ld, turn it back into
//     row layout through a swizzled 4 KB staging tile per warp, then stream AX, AV, V and G_prev
//     with coalesced loads, write AX_new and G, and add the column sums into per-warp shared
//     accumulators after a two-step shuffle over the warp's four row groups.
// Every mbarrier wait is bounded: on expiry the CTA records OFSC_ERR_TIMEOUT, every role stops,
// the MMAs already issued are waited for (bounded) and the tensor memory is freed.
#include "tcgen05.cuh"

namespace ofsc {
namespace {

constexpr int kDtThreads = 288;           // converters 0-3, epilogue 4-7, MMA 8
constexpr int kDtStages = 2;              // A chunk stages
constexpr int kDtChunk = 128 * 32 * 4;    // one A chunk: 128 rows x 32 features, FP32 (16 KB)
constexpr int kDtB = 4 * kTcTile;         // R' as B: 128 x 128 (64 KB per hi or lo)
constexpr int kDtSums = 6;
constexpr size_t kDtSmem = 2 * (size_t)kDtB + (size_t)kDtStages * 2 * kDtChunk + 4 * 32 * 32 * 4 +
                           4 * (size_t)kDtSums * 128 * 4 + 1024;

template <bool TRI>
__global__ void __launch_bounds__(kDtThreads, 1) k_direction_tc(RowArgs a) {
  if (!a.ignore_done && a.ctrl->done) return;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t a_full[kDtStages], a_empty[kDtStages], d_full[2], d_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* bhi = base;
  unsigned char* blo = base + kDtB;
  unsigned char* ahi = base + 2 * kDtB;          // [stage]
  unsigned char* alo = ahi + kDtStages * kDtChunk;
  float* pst = (float*)(alo + kDtStages * kDtChunk);  // [4 warps][32 rows][32 columns], swizzled
  float* csum = pst + 4 * 32 * 32;                    // [4 warps][6][128]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int KP = 128;
  float* __restrict__ Xp = a.X;
  float* __restrict__ Yp = a.Y;
  const float* __restrict__ Vp = a.V;
  const float* __restrict__ Wp = a.W;
  float* __restrict__ Gp = a.G;
  const long long lim = spin_limit_of(a.ctrl);
  // test hook (opts.withhold_arrivals): the converters never signal a full stage, so the MMA
  // warp's first bounded wait runs out before any MMA is issued (no copy or MMA in flight)
  const bool withhold = a.ctrl->withhold != 0;

  if (warp == 8) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < kDtStages; ++st) {
      mbar_init(&a_full[st], 4);
      mbar_init(&a_empty[st], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&d_full[b], 1);
      mbar_init(&d_empty[b], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    if (a.update && blockIdx.x == 0) a.ctrl->it += 1;
  }
  // R' as the B operand (N = output feature, K = input feature): element (n, k) = R'[k][n]
  for (int e = tid; e < KP * KP; e += blockDim.x) {
    const int n = e >> 7, k = e & 127;
    const float v = (TRI && k > n) ? 0.0f : a.Rn[k * KP + n];
    const uint32_t h = tf32_round(v);
    const uint32_t off = (uint32_t)(k >> 5) * kTcTile + tile_off(n, k & 31);
    *(uint32_t*)(bhi + off) = h;
    *(float*)(blo + off) = v - __uint_as_float(h);
  }
  for (int e = tid; e < 4 * kDtSums * KP; e += blockDim.x) csum[e] = 0.0f;
  asm volatile("fence.proxy.async.shared::cta;");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  const int64_t ntiles = (a.n + 127) / 128;
  const int64_t nt = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (warp < 4) {  // converters: X_new chunks into the A stages
    const int j = lane & 7;
    bool ok = true;
    for (int64_t i = 0; i < nt && ok; ++i) {
      const int64_t row0 = (blockIdx.x + i * gridDim.x) * 128;
      for (int kc = 0; kc < 4; ++kc) {
        const int64_t u = i * 4 + kc;
        const int st = (int)(u % kDtStages);
        if (u >= kDtStages && !ws_wait(&a_empty[st], (uint32_t)((u / kDtStages - 1) & 1), &abort_flag, lim)) {
          ok = false;
          break;
        }
        const int f = kc * 32 + 4 * j;
        float4 al = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a.update) al = *(const float4*)(a.alpha + f);
        unsigned char* dh = ahi + st * kDtChunk;
        unsigned char* dl = alo + st * kDtChunk;
        // every global load of the chunk before any store or arithmetic
        float4 xs[8], vs[8];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
          const int64_t row = row0 + warp * 32 + rr * 4 + (lane >> 3);
          const int64_t o = row * KP + f;
          xs[rr] = row < a.n ? *(const float4*)(Xp + o) : make_float4(0.f, 0.f, 0.f, 0.f);
          vs[rr] = (a.update && row < a.n) ? *(const float4*)(Vp + o) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
          const int r = warp * 32 + rr * 4 + (lane >> 3);  // tile row
          const int64_t row = row0 + r;
          float4 x = xs[rr];
          if (a.update) {
            const float4 v = vs[rr];
            x = make_float4(fmaf(al.x, v.x, x.x), fmaf(al.y, v.y, x.y), fmaf(al.z, v.z, x.z), fmaf(al.w, v.w, x.w));
            if (row < a.n) *(float4*)(Xp + row * KP + f) = x;
          }
          const uint32_t h0 = tf32_round(x.x), h1 = tf32_round(x.y), h2 = tf32_round(x.z), h3 = tf32_round(x.w);
          const uint32_t off = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
          *(uint4*)(dh + off) = make_uint4(h0, h1, h2, h3);
          *(float4*)(dl + off) = make_float4(x.x - __uint_as_float(h0), x.y - __uint_as_float(h1),
                                             x.z - __uint_as_float(h2), x.w - __uint_as_float(h3));
        }
        asm volatile("fence.proxy.async.shared::cta;");  // generic-proxy stores -> tensor-core reads
        __syncwarp();
        if (lane == 0 && !withhold) mbar_arrive(&a_full[st]);
      }
    }
  } else if (warp < 8) {  // epilogue
    const int ew = warp - 4;
    const int j = lane & 7, rs = lane >> 3;
    float* ps = pst + ew * 32 * 32;
    float* cs = csum + ew * kDtSums * KP;
    for (int64_t i = 0; i < nt; ++i) {
      const int buf = (int)(i & 1);
      if (!ws_wait(&d_full[buf], (uint32_t)((i >> 1) & 1), &abort_flag, lim)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int64_t row0 = (blockIdx.x + i * gridDim.x) * 128 + ew * 32;
      for (int cc = 0; cc < 4; ++cc) {
        uint32_t p[32];
        tmem_ld32(tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(buf * 128 + cc * 32), p);
        asm volatile("tcgen05.wait::ld.sync.aligned;");
        // thread = row (lane); chunk q of the row's 32 columns at position q ^ (row & 7)
#pragma unroll
        for (int q = 0; q < 8; ++q)
          *(float4*)(ps + lane * 32 + ((q ^ (lane & 7)) << 2)) =
              make_float4(__uint_as_float(p[4 * q]), __uint_as_float(p[4 * q + 1]), __uint_as_float(p[4 * q + 2]),
                          __uint_as_float(p[4 * q + 3]));
        __syncwarp();
        const int c = cc * 32 + 4 * j;
        float4 al = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a.update) al = *(const float4*)(a.alpha + c);
        float s[kDtSums][4];
#pragma unroll
        for (int w = 0; w < kDtSums; ++w) s[w][0] = s[w][1] = s[w][2] = s[w][3] = 0.0f;
        // two halves of four rows: every global load of a half before any store or arithmetic
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          float4 ys[4], ws[4], vs[4], gs[4];
#pragma unroll
          for (int r4 = 0; r4 < 4; ++r4) {
            const int64_t row = row0 + (hh * 4 + r4) * 4 + rs;
            const int64_t o = row * KP + c;
            const bool in = row < a.n;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            ys[r4] = in ? *(const float4*)(Yp + o) : z;
            ws[r4] = (in && a.update) ? *(const float4*)(Wp + o) : z;
            vs[r4] = (in && (a.update || a.need_vy)) ? *(const float4*)(Vp + o) : z;
            gs[r4] = (in && !a.eval) ? *(const float4*)(Gp + o) : z;
          }
#pragma unroll
          for (int r4 = 0; r4 < 4; ++r4) {
            const int rl = (hh * 4 + r4) * 4 + rs;  // the warp's local row
            const int64_t row = row0 + rl;
            if (row >= a.n) continue;
            const float4 pv = *(const float4*)(ps + rl * 32 + ((j ^ (rl & 7)) << 2));
            const int64_t o = row * KP + c;
            float4 y = ys[r4];
            if (a.update) {
              const float4 w = ws[r4];
              y = make_float4(fmaf(al.x, w.x, y.x), fmaf(al.y, w.y, y.y), fmaf(al.z, w.z, y.z), fmaf(al.w, w.w, y.w));
              *(float4*)(Yp + o) = y;
            }
            const float4 v = vs[r4], gp = gs[r4];
            const float yv[4] = {y.x, y.y, y.z, y.w}, pp[4] = {pv.x, pv.y, pv.z, pv.w};
            const float vv[4] = {v.x, v.y, v.z, v.w}, gpv[4] = {gp.x, gp.y, gp.z, gp.w};
            float g[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              g[q] = TRI ? yv[q] + pp[q] : 4.0f * (yv[q] + pp[q]);
              s[0][q] = fmaf(g[q], g[q], s[0][q]);
              s[1][q] = fmaf(g[q] - gpv[q], g[q], s[1][q]);
              s[2][q] = fmaf(gpv[q], gpv[q], s[2][q]);
              s[3][q] = fmaf(g[q], yv[q], s[3][q]);
              s[4][q] = fmaf(vv[q], yv[q], s[4][q]);
              s[5][q] = fmaf(vv[q], g[q], s[5][q]);
            }
            *(float4*)(Gp + o) = make_float4(g[0], g[1], g[2], g[3]);
          }
        }
        __syncwarp();  // the staging tile is rewritten by the next chunk
        // the four row groups (lanes j, j + 8, j + 16, j + 24) in a fixed order
#pragma unroll
        for (int w = 0; w < kDtSums; ++w)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            s[w][q] += __shfl_xor_sync(0xffffffffu, s[w][q], 8);
            s[w][q] += __shfl_xor_sync(0xffffffffu, s[w][q], 16);
          }
        if (lane < 8) {
#pragma unroll
          for (int w = 0; w < kDtSums; ++w)
#pragma unroll
            for (int q = 0; q < 4; ++q) cs[w * KP + c + q] += s[w][q];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&d_empty[buf]);
    }
  } else if (lane == 0) {  // warp 8: the MMAs
    const uint32_t idesc = tf32_idesc(128);
    int64_t issued = 0;  // chunks whose MMAs were committed
    bool ok = true;
    for (int64_t i = 0; i < nt && ok; ++i) {
      const int buf = (int)(i & 1);
      if (i >= 2 && !ws_wait(&d_empty[buf], (uint32_t)((i / 2 - 1) & 1), &abort_flag, lim)) break;
      for (int kc = 0; kc < 4; ++kc) {
        const int64_t u = i * 4 + kc;
        const int st = (int)(u % kDtStages);
        if (!ws_wait(&a_full[st], (uint32_t)((u / kDtStages) & 1), &abort_flag, lim)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t as_hi = smem_u32(ahi + st * kDtChunk), as_lo = smem_u32(alo + st * kDtChunk);
        const uint32_t bs_hi = smem_u32(bhi) + kc * kTcTile, bs_lo = smem_u32(blo) + kc * kTcTile;
        const uint32_t d = tmem + (uint32_t)(buf * 128);
#pragma unroll
        for (int s = 0; s < 4; ++s) {  // K steps of 8 features (32 bytes)
          const uint64_t a_h = sw128_desc(as_hi + s * 32), a_l = sw128_desc(as_lo + s * 32);
          const uint64_t b_h = sw128_desc(bs_hi + s * 32), b_l = sw128_desc(bs_lo + s * 32);
          mma_tf32(d, a_h, b_h, idesc, (kc > 0 || s > 0) ? 1u : 0u);
          mma_tf32(d, a_h, b_l, idesc, 1u);
          mma_tf32(d, a_l, b_h, idesc, 1u);
        }
        mma_commit(&a_empty[st]);
        issued = u + 1;
        if (kc == 3) mma_commit(&d_full[buf]);
      }
    }
    // the MMAs already issued must finish before the tensor memory is released
    if (issued > 0) mbar_wait(&a_empty[(issued - 1) % kDtStages], (uint32_t)(((issued - 1) / kDtStages) & 1), lim);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  // per-block column sums in a fixed order (epilogue warps 0..3)
  for (int t = tid; t < kDtSums * KP; t += blockDim.x) {
    double sum = 0.0;
    for (int ew = 0; ew < 4; ++ew) sum += (double)csum[ew * kDtSums * KP + t];
    a.colpart[(int64_t)blockIdx.x * kDtSums * KP + t] = sum;
  }
  if (abort_flag && tid == 0) {
    a.ctrl->status = OFSC_ERR_TIMEOUT;
    a.ctrl->done = 1;
  }
  if (warp == 8) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

// ------------------------------------------------------------------------------------------
// The direction pass of OFM-f2 (Eq. (10)) and TriOFM-f2 (Eq. (12)) at padded k = 128 on the tensor
// cores. Per 128-row tile, with X_new = X + V diag(alpha) and AX_new = AX + AV diag(alpha):
//   P = X_new B' + AX_new R'  (B' = X^T A X, R' = X^T X, or their upper triangles for TriOFM)
//   G = 4 AX_new - 2 P (OFM-f2) or 2 AX_new - P (TriOFM-f2)
// as one K = 256 product (tcgen05 kind::tf32, 3-term hi/lo split per factor), and the six column
// sums of the f1 pass. The hi/lo images of B' and R' (256 KB) do not fit beside the A stages, so
// k_f2_bimage writes them once per update to global memory in the tiles' swizzled layout and the
// MMA thread streams each 32-row K chunk in with one bulk copy (B' and R' halves in two buffers,
// so one half reloads while the other half's MMAs run):
//   * warps 0-3 form X_new, warps 4-7 AX_new, 32-feature chunks of 128 rows, into tf32 hi/lo
//     K-major 128-byte-swizzled tiles of a ring of two stages (warps 0-3 also store X_new);
//   * warp 12 (one thread) copies the B chunks and issues Dx += Xhi B'hi + Xhi B'lo + Xlo B'hi and
//     Dy += Yhi R'hi + Yhi R'lo + Ylo R'hi into two 128-column tensor-memory accumulators (of a
//     pair of such, 512 columns): each FP32 accumulator then takes as many MMA updates as the f1
//     pass's, which keeps the accumulation rounding at the f1 pass's size;
//   * warps 8-11 read P = Dx + Dy with tcgen05.ld, recompute and store AX_new from AX and AV (their second
//     reads, mostly from L2), form G and the column sums as the f1 pass does.
// Every wait is bounded; on expiry the CTA records OFSC_ERR_TIMEOUT, stops every role, waits
// (bounded) for the copies and MMAs it issued and frees its tensor memory.
constexpr int kD2Threads = 416;                       // converters 0-7, epilogue 8-11, MMA 12
constexpr int kD2Stage = 4 * kTcTile;                 // X hi, X lo, AX hi, AX lo of one chunk
constexpr int kD2Half = 2 * kTcTile;                  // hi and lo of B' (or R') for one K chunk
constexpr size_t kD2Smem = 2 * (size_t)kD2Stage + 2 * (size_t)kD2Half + 4 * 32 * 32 * 4 +
                           4 * (size_t)kDtSums * 128 * 4 + 1024;
static_assert(kD2Smem <= 227 * 1024, "shared memory of the f2 direction pass");

// The B operand images of B' (from Bn) and R' (from Rn): [K chunk][B' hi, B' lo, R' hi, R' lo] of
// kTcTile bytes each, element (n, k) = M[k][n] (zero below the diagonal for TriOFM).
__global__ void k_f2_bimage(const float* __restrict__ Rn, const float* __restrict__ Bn, int tri,
                            unsigned char* __restrict__ img, const Ctrl* ctrl, int ignore_done) {
  if (!ignore_done && ctrl->done) return;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 128 * 128; e += gridDim.x * blockDim.x) {
    const int n = e >> 7, k = e & 127;
    const bool keep = !tri || k <= n;
    const float b = keep ? Bn[k * 128 + n] : 0.0f;
    const float r = keep ? Rn[k * 128 + n] : 0.0f;
    const uint32_t bh = tf32_round(b), rh = tf32_round(r);
    unsigned char* t = img + (size_t)(k >> 5) * 4 * kTcTile;
    const uint32_t off = tile_off(n, k & 31);
    *(uint32_t*)(t + off) = bh;
    *(float*)(t + kTcTile + off) = b - __uint_as_float(bh);
    *(uint32_t*)(t + 2 * kTcTile + off) = rh;
    *(float*)(t + 3 * kTcTile + off) = r - __uint_as_float(rh);
  }
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

template <bool TRI>
__global__ void __launch_bounds__(kD2Threads, 1) k_direction_tc2(RowArgs a) {
  if (!a.ignore_done && a.ctrl->done) return;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t a_full[kDtStages], a_empty[kDtStages], d_full[2], d_empty[2];
  __shared__ uint64_t b_full[2], b_empty[2];  // [0] B' half, [1] R' half
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* ast = base;                               // [stage][X hi, X lo, AX hi, AX lo]
  unsigned char* bbuf = base + kDtStages * kD2Stage;       // [B' hi, B' lo][R' hi, R' lo]
  float* pst = (float*)(bbuf + 2 * kD2Half);               // [4 warps][32 rows][32 columns]
  float* csum = pst + 4 * 32 * 32;                         // [4 warps][6][128]
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int KP = 128;
  float* __restrict__ Xp = a.X;
  float* __restrict__ Yp = a.Y;
  const float* __restrict__ Vp = a.V;
  const float* __restrict__ Wp = a.W;
  float* __restrict__ Gp = a.G;
  const unsigned char* __restrict__ img = (const unsigned char*)a.bimg;
  const long long lim = spin_limit_of(a.ctrl);

  if (warp == 12) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < kDtStages; ++st) {
      mbar_init(&a_full[st], 8);
      mbar_init(&a_empty[st], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&d_full[b], 1);
      mbar_init(&d_empty[b], 4);
      mbar_init(&b_full[b], 1);
      mbar_init(&b_empty[b], 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;");
    if (a.update && blockIdx.x == 0) a.ctrl->it += 1;
  }
  for (int e = tid; e < 4 * kDtSums * KP; e += blockDim.x) csum[e] = 0.0f;
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_slot;

  const int64_t ntiles = (a.n + 127) / 128;
  const int64_t nt = ntiles > blockIdx.x ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;

  if (warp < 8) {  // converters: warps 0-3 X_new, warps 4-7 AX_new
    const bool isx = warp < 4;
    const int rw = warp & 3;  // the warp's 32 rows of the tile
    const int j = lane & 7;
    const float* __restrict__ src = isx ? Xp : Yp;
    const float* __restrict__ dir = isx ? Vp : Wp;
    bool ok = true;
    for (int64_t i = 0; i < nt && ok; ++i) {
      const int64_t row0 = (blockIdx.x + i * gridDim.x) * 128;
      for (int kc = 0; kc < 4; ++kc) {
        const int64_t u = i * 4 + kc;
        const int st = (int)(u % kDtStages);
        if (u >= kDtStages && !ws_wait(&a_empty[st], (uint32_t)((u / kDtStages - 1) & 1), &abort_flag, lim)) {
          ok = false;
          break;
        }
        const int f = kc * 32 + 4 * j;
        float4 al = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a.update) al = *(const float4*)(a.alpha + f);
        unsigned char* dh = ast + st * kD2Stage + (isx ? 0 : 2 * kTcTile);
        unsigned char* dl = dh + kTcTile;
        float4 xs[8], vs[8];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
          const int64_t row = row0 + rw * 32 + rr * 4 + (lane >> 3);
          const int64_t o = row * KP + f;
          xs[rr] = row < a.n ? *(const float4*)(src + o) : make_float4(0.f, 0.f, 0.f, 0.f);
          vs[rr] = (a.update && row < a.n) ? *(const float4*)(dir + o) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
          const int r = rw * 32 + rr * 4 + (lane >> 3);  // tile row
          const int64_t row = row0 + r;
          float4 x = xs[rr];
          if (a.update) {
            const float4 v = vs[rr];
            x = make_float4(fmaf(al.x, v.x, x.x), fmaf(al.y, v.y, x.y), fmaf(al.z, v.z, x.z), fmaf(al.w, v.w, x.w));
            if (isx && row < a.n) *(float4*)(Xp + row * KP + f) = x;
          }
          const uint32_t h0 = tf32_round(x.x), h1 = tf32_round(x.y), h2 = tf32_round(x.z), h3 = tf32_round(x.w);
          const uint32_t off = (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((j ^ (r & 7)) << 4));
          *(uint4*)(dh + off) = make_uint4(h0, h1, h2, h3);
          *(float4*)(dl + off) = make_float4(x.x - __uint_as_float(h0), x.y - __uint_as_float(h1),
                                             x.z - __uint_as_float(h2), x.w - __uint_as_float(h3));
        }
        asm volatile("fence.proxy.async.shared::cta;");  // generic-proxy stores -> tensor-core reads
        __syncwarp();
        if (lane == 0) mbar_arrive(&a_full[st]);
      }
    }
  } else if (warp < 12) {  // epilogue
    const int ew = warp - 8;
    const int j = lane & 7, rs = lane >> 3;
    float* ps = pst + ew * 32 * 32;
    float* cs = csum + ew * kDtSums * KP;
    for (int64_t i = 0; i < nt; ++i) {
      const int buf = (int)(i & 1);
      if (!ws_wait(&d_full[buf], (uint32_t)((i >> 1) & 1), &abort_flag, lim)) break;
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int64_t row0 = (blockIdx.x + i * gridDim.x) * 128 + ew * 32;
      for (int cc = 0; cc < 4; ++cc) {
        // P = (X_new B') + (AX_new R'): the two accumulators, added in FP32 through the staging tile
        for (int part = 0; part < 2; ++part) {
          uint32_t p[32];
          tmem_ld32(tmem + ((uint32_t)(ew * 32) << 16) + (uint32_t)(buf * 256 + part * 128 + cc * 32), p);
          asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
          for (int q = 0; q < 8; ++q) {
            float4* dst = (float4*)(ps + lane * 32 + ((q ^ (lane & 7)) << 2));
            float4 v = make_float4(__uint_as_float(p[4 * q]), __uint_as_float(p[4 * q + 1]),
                                   __uint_as_float(p[4 * q + 2]), __uint_as_float(p[4 * q + 3]));
            if (part) {
              const float4 o = *dst;
              v = make_float4(o.x + v.x, o.y + v.y, o.z + v.z, o.w + v.w);
            }
            *dst = v;
          }
        }
        __syncwarp();
        const int c = cc * 32 + 4 * j;
        float4 al = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a.update) al = *(const float4*)(a.alpha + c);
        float s[kDtSums][4];
#pragma unroll
        for (int w = 0; w < kDtSums; ++w) s[w][0] = s[w][1] = s[w][2] = s[w][3] = 0.0f;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          float4 ys[4], ws[4], vs[4], gs[4];
#pragma unroll
          for (int r4 = 0; r4 < 4; ++r4) {
            const int64_t row = row0 + (hh * 4 + r4) * 4 + rs;
            const int64_t o = row * KP + c;
            const bool in = row < a.n;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            ys[r4] = in ? *(const float4*)(Yp + o) : z;
            ws[r4] = (in && a.update) ? *(const float4*)(Wp + o) : z;
            vs[r4] = (in && (a.update || a.need_vy)) ? *(const float4*)(Vp + o) : z;
            gs[r4] = (in && !a.eval) ? *(const float4*)(Gp + o) : z;
          }
#pragma unroll
          for (int r4 = 0; r4 < 4; ++r4) {
            const int rl = (hh * 4 + r4) * 4 + rs;
            const int64_t row = row0 + rl;
            if (row >= a.n) continue;
            const float4 pv = *(const float4*)(ps + rl * 32 + ((j ^ (rl & 7)) << 2));
            const int64_t o = row * KP + c;
            float4 y = ys[r4];
            if (a.update) {
              const float4 w = ws[r4];
              y = make_float4(fmaf(al.x, w.x, y.x), fmaf(al.y, w.y, y.y), fmaf(al.z, w.z, y.z), fmaf(al.w, w.w, y.w));
              *(float4*)(Yp + o) = y;
            }
            const float4 v = vs[r4], gp = gs[r4];
            const float yv[4] = {y.x, y.y, y.z, y.w}, pp[4] = {pv.x, pv.y, pv.z, pv.w};
            const float vv[4] = {v.x, v.y, v.z, v.w}, gpv[4] = {gp.x, gp.y, gp.z, gp.w};
            float g[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
              g[q] = TRI ? 2.0f * yv[q] - pp[q] : 4.0f * yv[q] - 2.0f * pp[q];  // Eqs. (12), (10)
              s[0][q] = fmaf(g[q], g[q], s[0][q]);
              s[1][q] = fmaf(g[q] - gpv[q], g[q], s[1][q]);
              s[2][q] = fmaf(gpv[q], gpv[q], s[2][q]);
              s[3][q] = fmaf(g[q], yv[q], s[3][q]);
              s[4][q] = fmaf(vv[q], yv[q], s[4][q]);
              s[5][q] = fmaf(vv[q], g[q], s[5][q]);
            }
            *(float4*)(Gp + o) = make_float4(g[0], g[1], g[2], g[3]);
          }
        }
        __syncwarp();
#pragma unroll
        for (int w = 0; w < kDtSums; ++w)
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            s[w][q] += __shfl_xor_sync(0xffffffffu, s[w][q], 8);
            s[w][q] += __shfl_xor_sync(0xffffffffu, s[w][q], 16);
          }
        if (lane < 8) {
#pragma unroll
          for (int w = 0; w < kDtSums; ++w)
#pragma unroll
            for (int q = 0; q < 4; ++q) cs[w * KP + c + q] += s[w][q];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) mbar_arrive(&d_empty[buf]);
    }
  } else if (lane == 0) {  // warp 12: B chunk copies and the MMAs
    const uint32_t idesc = tf32_idesc(128);
    const int64_t nchunks = nt * 4;
    int64_t issued = 0;       // chunks whose MMAs were committed
    int64_t req[2] = {0, 0};  // chunks whose B' (R') half was requested; at most one in flight each
    bool ok = true;
    if (nchunks > 0)
      for (int h = 0; h < 2; ++h) {
        mbar_expect_tx(&b_full[h], kD2Half);
        bulk_g2s(bbuf + h * kD2Half, img + (size_t)h * kD2Half, kD2Half, &b_full[h]);
        req[h] = 1;
      }
    for (int64_t i = 0; i < nt && ok; ++i) {
      const int buf = (int)(i & 1);
      if (i >= 2 && !ws_wait(&d_empty[buf], (uint32_t)((i / 2 - 1) & 1), &abort_flag, lim)) break;
      for (int kc = 0; kc < 4; ++kc) {
        const int64_t u = i * 4 + kc;
        const int st = (int)(u % kDtStages);
        // every operand of the chunk before its first MMA, so an expired wait leaves none in flight
        ok = ws_wait(&a_full[st], (uint32_t)((u / kDtStages) & 1), &abort_flag, lim) &&
             ws_wait(&b_full[0], (uint32_t)(u & 1), &abort_flag, lim) &&
             ws_wait(&b_full[1], (uint32_t)(u & 1), &abort_flag, lim);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t as = smem_u32(ast + st * kD2Stage);
        for (int h = 0; h < 2; ++h) {  // h = 0: X_new with B'; h = 1: AX_new with R'
          // each product has its own accumulator, so neither chains more MMA updates than the f1 pass
          const uint32_t d = tmem + (uint32_t)(buf * 256 + h * 128);
          const uint32_t a_hi = as + h * 2 * kTcTile, a_lo = a_hi + kTcTile;
          const uint32_t b_hi = smem_u32(bbuf + h * kD2Half), b_lo = b_hi + kTcTile;
#pragma unroll
          for (int s = 0; s < 4; ++s) {  // K steps of 8 features (32 bytes)
            const uint64_t ah = sw128_desc(a_hi + s * 32), alo = sw128_desc(a_lo + s * 32);
            const uint64_t bh = sw128_desc(b_hi + s * 32), blo = sw128_desc(b_lo + s * 32);
            mma_tf32(d, ah, bh, idesc, (kc > 0 || s > 0) ? 1u : 0u);
            mma_tf32(d, ah, blo, idesc, 1u);
            mma_tf32(d, alo, bh, idesc, 1u);
          }
          mma_commit(&b_empty[h]);
        }
        mma_commit(&a_empty[st]);
        issued = u + 1;
        if (kc == 3) mma_commit(&d_full[buf]);
        // the next K chunk's halves, each once the MMAs reading its buffer have completed
        if (u + 1 < nchunks) {
          const int kn = (int)((u + 1) & 3);
          for (int h = 0; h < 2 && ok; ++h) {
            ok = ws_wait(&b_empty[h], (uint32_t)(u & 1), &abort_flag, lim);
            if (!ok) break;
            mbar_expect_tx(&b_full[h], kD2Half);
            bulk_g2s(bbuf + h * kD2Half, img + ((size_t)kn * 2 + h) * kD2Half, kD2Half, &b_full[h]);
            req[h] = u + 2;
          }
          if (!ok) break;
        }
      }
    }
    // the MMAs and copies already issued must finish before the tensor and shared memory go
    if (issued > 0) mbar_wait(&a_empty[(issued - 1) % kDtStages], (uint32_t)(((issued - 1) / kDtStages) & 1), lim);
    for (int h = 0; h < 2; ++h)
      if (req[h] > issued) mbar_wait(&b_full[h], (uint32_t)((req[h] - 1) & 1), lim);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  for (int t = tid; t < kDtSums * KP; t += blockDim.x) {
    double sum = 0.0;
    for (int ew = 0; ew < 4; ++ew) sum += (double)csum[ew * kDtSums * KP + t];
    a.colpart[(int64_t)blockIdx.x * kDtSums * KP + t] = sum;
  }
  if (abort_flag && tid == 0) {
    a.ctrl->status = OFSC_ERR_TIMEOUT;
    a.ctrl->done = 1;
  }
  if (warp == 12) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

template <bool TRI>
cudaError_t launch_dt2(const RowArgs& a, int grid, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_direction_tc2<TRI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kD2Smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_f2_bimage<<<16, 256, 0, s>>>(a.Rn, a.Bn, TRI ? 1 : 0, (unsigned char*)a.bimg, a.ctrl, a.ignore_done);
  k_direction_tc2<TRI><<<grid, kD2Threads, kD2Smem, s>>>(a);
  return cudaGetLastError();
}


template <bool TRI>
cudaError_t launch_dt(const RowArgs& a, int grid, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_direction_tc<TRI>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDtSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_direction_tc<TRI><<<grid, kDtThreads, kDtSmem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

bool direction_tc_supported(int method, int kp) { return kp == 128 && method >= OFSC_OFM_F1 && method <= OFSC_TRI_F2; }

cudaError_t direction_tc_launch(int method, const RowArgs& a, cudaStream_t s, int* nblk) {
  const int64_t ntiles = (a.n + 127) / 128;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, kNumSMs));
  *nblk = grid;
  switch (method) {
    case OFSC_OFM_F1: return launch_dt<false>(a, grid, s);
    case OFSC_TRI_F1: return launch_dt<true>(a, grid, s);
    case OFSC_OFM_F2: return launch_dt2<false>(a, grid, s);
    default: return launch_dt2<true>(a, grid, s);
  }
}

}  // namespace ofsc
