// Rayleigh-Ritz check of a feature block X (Sec. 5: the eigensolver view of the methods and its
// `relerr`): Ritz pairs of B = 2I - L = -A on span(X) and
//   relerr = ||B U - U Lam||_F / ||U Lam||_F,  U = X Z, Z^T (X^T X) Z = I.
// Everything is k x k FP64 algebra on the device from the Grams R = X^T X and XAX = X^T A X, plus
// one row pass for the residual:
//   R = L L^T (Cholesky),  T = L^-1,  R^-1 = T^T T,
//   C = T (-XAX) T^T, its eigenvalues (cyclic Jacobi) are the Ritz values Lam,
//   E = A X - X M with M = R^-1 XAX, so that B U - U Lam = -E Z and
//   relerr^2 = tr(E^T E R^-1) / ||C||_F^2   (Z Z^T = R^-1, sum Lam^2 = ||C||_F^2).
// E is formed row by row (no quantity cancels in E^T E), so relerr keeps its relative accuracy
// while it is well above the FP32 rounding of A X.
#include "common.cuh"

namespace ofsc {
namespace {

constexpr int kRitzThreads = 256;
constexpr int kJacobiSweeps = 40;

// Sum over the block of one value per thread, in a fixed order; every thread gets the result.
__device__ double block_total(double v, double* sh) {
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

// Cholesky, inverse factor, R^-1, M and C for the leading k x k blocks (row stride kp); C's
// eigenvalues by parallel cyclic Jacobi (the round-robin pair ordering of Golub and Van Loan,
// Sec. 8.5) in shared memory. work: [4][kp][kp] FP64 (L, T, Rinv, M). Writes Rn_out = -M as FP32
// (kp x kp, zero outside k x k), lam ascending, and sums[0] = ||C||_F^2. A pivot below 1e-6 of its
// diagonal entry (X numerically rank deficient) sets OFSC_ERR_INVALID_ARG in ctrl->status.
__global__ void __launch_bounds__(kRitzThreads, 1)
    k_ritz_prepare(const double* __restrict__ R, const double* __restrict__ XAX, int k, int kp,
                   double* __restrict__ work, float* __restrict__ Rn_out, double* __restrict__ lam,
                   double* __restrict__ sums, Ctrl* ctrl) {
  extern __shared__ double C[];  // [ke][ke], ke = k rounded up to even
  __shared__ int bad;
  __shared__ double red[kRitzThreads];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ke = (k + 1) & ~1;
  double* Lm = work;
  double* T = work + (size_t)kp * kp;
  double* Ri = T + (size_t)kp * kp;
  double* M = Ri + (size_t)kp * kp;
  if (tid == 0) bad = 0;
  for (int i = tid; i < kp * kp; i += nt) Lm[i] = T[i] = 0.0;
  __syncthreads();
  // Cholesky, column by column
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      double d = R[j * kp + j];
      for (int m = 0; m < j; ++m) d -= Lm[j * kp + m] * Lm[j * kp + m];
      // the Grams carry FP32-level rounding: a column whose part outside the span of the previous
      // ones has under 1e-6 of its squared norm cannot be told from a dependent one
      if (!(d > 1e-6 * R[j * kp + j])) bad = 1;
      Lm[j * kp + j] = d > 0.0 ? sqrt(d) : 1.0;
    }
    __syncthreads();
    const double ljj = Lm[j * kp + j];
    for (int i = j + 1 + tid; i < k; i += nt) {
      double v = R[i * kp + j];
      for (int m = 0; m < j; ++m) v -= Lm[i * kp + m] * Lm[j * kp + m];
      Lm[i * kp + j] = v / ljj;
    }
    __syncthreads();
  }
  // T = L^-1: column c by forward substitution, one thread per column
  for (int c = tid; c < k; c += nt) {
    for (int i = c; i < k; ++i) {
      double v = i == c ? 1.0 : 0.0;
      for (int m = c; m < i; ++m) v -= Lm[i * kp + m] * T[m * kp + c];
      T[i * kp + c] = v / Lm[i * kp + i];
    }
  }
  __syncthreads();
  // R^-1 = T^T T
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e % k;
    double v = 0.0;
    for (int m = (i > j ? i : j); m < k; ++m) v += T[m * kp + i] * T[m * kp + j];
    Ri[i * kp + j] = v;
  }
  __syncthreads();
  // M = R^-1 XAX (symmetrised XAX); Rn_out = -M
  for (int e = tid; e < kp * kp; e += nt) {
    const int i = e / kp, j = e % kp;
    double v = 0.0;
    if (i < k && j < k)
      for (int m = 0; m < k; ++m) v += Ri[i * kp + m] * 0.5 * (XAX[m * kp + j] + XAX[j * kp + m]);
    M[e] = v;
    Rn_out[e] = (float)(-v);
  }
  // C = T (-XAX) T^T = -(T XAX) T^T, two products in place in C
  for (int e = tid; e < ke * ke; e += nt) C[e] = 0.0;
  __syncthreads();
  for (int e = tid; e < k * k; e += nt) {  // C <- T XAX
    const int i = e / k, j = e % k;
    double v = 0.0;
    for (int m = 0; m <= i; ++m) v += T[i * kp + m] * 0.5 * (XAX[m * kp + j] + XAX[j * kp + m]);
    C[i * ke + j] = v;
  }
  __syncthreads();
  // C <- -(C T^T), one thread per row (the row copied to local storage first)
  for (int i = tid; i < k; i += nt) {
    double row[128];
    for (int m = 0; m < k; ++m) row[m] = C[i * ke + m];
    for (int j = 0; j < k; ++j) {
      double v = 0.0;
      for (int m = 0; m <= j; ++m) v += row[m] * T[j * kp + m];
      C[i * ke + j] = -v;
    }
  }
  __syncthreads();
  // symmetrise and ||C||_F^2
  for (int e = tid; e < k * k; e += nt) {
    const int i = e / k, j = e % k;
    if (i < j) {
      const double v = 0.5 * (C[i * ke + j] + C[j * ke + i]);
      C[i * ke + j] = v;
      C[j * ke + i] = v;
    }
  }
  __syncthreads();
  double fl = 0.0;
  for (int e = tid; e < k * k; e += nt) fl += C[(e / k) * ke + e % k] * C[(e / k) * ke + e % k];
  const double fro2 = block_total(fl, red);
  if (tid == 0) sums[0] = fro2;
  // cyclic Jacobi, round-robin ordering over ke indices (index ke-1 is a zero pad when k is odd)
  __shared__ double rc[64], rs[64];
  __shared__ int rp[64], rq[64];
  const int half = ke / 2;
  for (int sweep = 0; sweep < kJacobiSweeps; ++sweep) {
    for (int round = 0; round < ke - 1; ++round) {
      // pairs of this round: position 0 fixed, the others rotate
      for (int t = tid; t < half; t += nt) {
        auto pos = [&](int x) { return x == 0 ? 0 : 1 + (x - 1 + round) % (ke - 1); };
        int p = pos(t), q = pos(ke - 1 - t);
        if (p > q) { const int z = p; p = q; q = z; }
        rp[t] = p;
        rq[t] = q;
        const double apq = C[p * ke + q];
        double c = 1.0, s = 0.0;
        if (apq != 0.0) {
          const double tau = (C[q * ke + q] - C[p * ke + p]) / (2.0 * apq);
          const double tt = tau >= 0.0 ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : -1.0 / (-tau + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + tt * tt);
          s = tt * c;
        }
        rc[t] = c;
        rs[t] = s;
      }
      __syncthreads();
      // C <- C J (columns p, q of every row), then C <- J^T C (rows p, q of every column)
      for (int e = tid; e < ke * half; e += nt) {
        const int r = e / half, t = e % half;
        const int p = rp[t], q = rq[t];
        const double c = rc[t], s = rs[t];
        const double a = C[r * ke + p], b = C[r * ke + q];
        C[r * ke + p] = c * a - s * b;
        C[r * ke + q] = s * a + c * b;
      }
      __syncthreads();
      for (int e = tid; e < ke * half; e += nt) {
        const int r = e / half, t = e % half;
        const int p = rp[t], q = rq[t];
        const double c = rc[t], s = rs[t];
        const double a = C[p * ke + r], b = C[q * ke + r];
        C[p * ke + r] = c * a - s * b;
        C[q * ke + r] = s * a + c * b;
      }
      __syncthreads();
    }
    double ol = 0.0;
    for (int e = tid; e < k * k; e += nt)
      if (e / k != e % k) ol += C[(e / k) * ke + e % k] * C[(e / k) * ke + e % k];
    if (block_total(ol, red) <= 1e-30 * fro2) break;
  }
  // eigenvalues ascending (rank sort; ties by index)
  for (int i = tid; i < k; i += nt) {
    const double v = C[i * ke + i];
    int rank = 0;
    for (int j = 0; j < k; ++j) {
      const double w = C[j * ke + j];
      rank += (w < v) || (w == v && j < i);
    }
    lam[rank] = v;
  }
  if (tid == 0 && bad) {
    ctrl->status = OFSC_ERR_INVALID_ARG;
    ctrl->done = 1;
  }
}

// relerr = sqrt(tr(E^T E R^-1) / ||C||_F^2) with E^T E = G^T G / 16 (G = 4 E from the row pass).
__global__ void k_ritz_relerr(const double* __restrict__ GtG, const double* __restrict__ Ri, int k, int kp,
                              const double* __restrict__ sums, double* __restrict__ out) {
  __shared__ double sh[kRitzThreads];
  double v = 0.0;
  for (int e = threadIdx.x; e < k * k; e += blockDim.x) {
    const int i = e / k, j = e % k;
    v += GtG[i * kp + j] * Ri[j * kp + i];
  }
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double num = sh[0] / 16.0;
    out[0] = sums[0] > 0.0 ? sqrt((num > 0.0 ? num : 0.0) / sums[0]) : 0.0;
  }
}

}  // namespace

cudaError_t ritz_prepare_launch(const double* R64, const double* B64, int k, int kp, double* work, float* Rn,
                                double* lam, double* sums, Ctrl* ctrl, cudaStream_t s) {
  const int ke = (k + 1) & ~1;
  const size_t smem = (size_t)ke * ke * sizeof(double);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_ritz_prepare, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 128 * 8);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  k_ritz_prepare<<<1, kRitzThreads, smem, s>>>(R64, B64, k, kp, work, Rn, lam, sums, ctrl);
  return cudaGetLastError();
}

cudaError_t ritz_relerr_launch(const double* GtG, const double* work, int k, int kp, const double* sums, double* out,
                               cudaStream_t s) {
  k_ritz_relerr<<<1, kRitzThreads, 0, s>>>(GtG, work + 2 * (size_t)kp * kp, k, kp, sums, out);
  return cudaGetLastError();
}

}  // namespace ofsc
