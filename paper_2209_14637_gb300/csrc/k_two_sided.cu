// Two-sided sketching (Section 3.2): the small factors of the two-sided SCW
// step (Algorithm 3) and the panel of the second sketch.
//
// With the first sketch S (k x m) and the second W (l x n):
//
//   X = (S A)^T = Q R_X      (n x k)      Z = A W^T = P R_Z   (m x l)
//   Y = A X                  (m x k)
//
// the l x k core of Algorithm 3 is
//
//   C = P^T A Q = R_Z^{-T} (Z^T A X) R_X^{-1} = R_Z^{-T} (Z^T Y) R_X^{-1},
//
// so the one pass over A that gives X, Y (and, with W's panel in place of
// X, Z) leaves only k x l work per matrix: the product Z^T Y (reduced over
// the m rows), two triangular solves, a one-sided Jacobi SVD of C, and the
// error.  P and Q are orthonormal, so with B = P [C]_r Q^T
//
//   ||A - B||_F^2 = ||A||^2 - 2 <P^T A Q, [C]_r> + ||[C]_r||^2
//                 = ||A||^2 - sum_{i<=r} sigma_i(C)^2.
//
// The factored outputs are US = P U_r Sigma_r = Z (R_Z^{-1} U_r Sigma_r)
// (m x r) and Vt = (Q V_r)^T = (X R_X^{-1} V_r)^T (r x n), B = US Vt.
#include <cuda_bf16.h>

#include "tsk_internal.cuh"

namespace tsk {

namespace {

// W (l x n, row-major, leading dimension n; element Ts) -> the n x lp panel
// W^T (element Tp), columns l..lp-1 zero.
template <typename Ts, typename Tp>
__global__ void wt_panel_kernel(const Ts* __restrict__ W, int l, long long n, int lp,
                                Tp* __restrict__ out) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n * lp) return;
  const long long j = e / lp;
  const int c = (int)(e - j * lp);
  out[e] = c < l ? (Tp)W[(long long)c * n + j] : Tp(0);
}

constexpr int TS_T = 256;  // threads per CTA
constexpr int TS_RB = 32;  // rows of Z and Y per streamed chunk
constexpr int TS_MAXQ = 16;  // core entries per thread: l * k <= 64 * 64 = 16 * 256

struct TsLay {
  int L;  // leading dimension of the k / l sized arrays (max(kp, lp) + 1)
  size_t rx, rz, c, v, zs, ys, sig, order, bytes;
};

__host__ __device__ inline TsLay ts_layout(int kp, int lp) {
  TsLay t;
  t.L = (kp > lp ? kp : lp) + 1;
  size_t o = 0;
  t.rx = o;
  o += (size_t)kp * t.L;
  t.rz = o;
  o += (size_t)lp * t.L;
  t.c = o;
  o += (size_t)lp * t.L;
  t.v = o;
  o += (size_t)kp * t.L;
  t.zs = o;
  o += (size_t)TS_RB * lp;
  t.ys = o;
  o += (size_t)TS_RB * kp;
  t.sig = o;
  o += (size_t)kp;
  t.order = o;            // kp ints, stored in double slots
  o += (size_t)kp;
  t.bytes = o * sizeof(double) + 16;
  return t;
}

// Round-robin pairing of the one-sided Jacobi sweeps (the circle method).
__device__ __forceinline__ void ts_pair(int round, int i, int kk, int& p, int& q) {
  const int mm = kk - 1;
  if (i == 0) {
    p = round % mm;
    q = mm;
  } else {
    p = (round + i) % mm;
    q = (round - i + mm) % mm;
  }
}

// One-sided Jacobi on the ncol columns (length nrow) of M, rotations
// accumulated into V (ncol x ncol); M and V share the leading dimension ld.
__device__ void ts_jacobi(double* M, double* V, int nrow, int ncol, int ld, int* flag) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int kk = ncol + (ncol & 1);
  for (int sweep = 0; sweep < 60; ++sweep) {
    if (threadIdx.x == 0) *flag = 0;
    __syncthreads();
    for (int round = 0; round < kk - 1; ++round) {
      for (int pi = warp; pi < kk / 2; pi += nw) {
        int p, q;
        ts_pair(round, pi, kk, p, q);
        if (p >= ncol || q >= ncol) continue;
        double a = 0.0, b = 0.0, g = 0.0;
        for (int i = lane; i < nrow; i += 32) {
          const double x = M[i * ld + p], y = M[i * ld + q];
          a += x * x;
          b += y * y;
          g += x * y;
        }
        a = warp_sum(a);
        b = warp_sum(b);
        g = warp_sum(g);
        if (fabs(g) > 1e-15 * sqrt(a * b) && fabs(g) > 1e-280) {
          const double zeta = (b - a) / (2.0 * g);
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
          const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
          for (int i = lane; i < nrow; i += 32) {
            const double x = M[i * ld + p], y = M[i * ld + q];
            M[i * ld + p] = c * x - s * y;
            M[i * ld + q] = s * x + c * y;
          }
          for (int i = lane; i < ncol; i += 32) {
            const double x = V[i * ld + p], y = V[i * ld + q];
            V[i * ld + p] = c * x - s * y;
            V[i * ld + q] = s * x + c * y;
          }
          if (lane == 0) *flag = 1;
        }
      }
      __syncthreads();
    }
    if (*flag == 0) break;
    __syncthreads();
  }
}

// One CTA per matrix: the core C = R_Z^{-T} (Z^T Y) R_X^{-1}, its SVD, the
// error by the identity above, sigma (min(k, l) values, zeros after) and
// the output transforms WX = R_X^{-1} V_r (k x r, stride kp^2) and
// WZ = R_Z^{-1} U_r Sigma_r (l x r, stride lp^2).  Tp is the panel type;
// products of a chunk of rows are summed in Tp and chunks in double.
template <typename Tp>
__global__ void __launch_bounds__(TS_T)
two_sided_small_kernel(int kp, int lp, const MatDev* __restrict__ xm,
                       const MatDev* __restrict__ zm, const Tp* __restrict__ Y,
                       const Tp* __restrict__ Z, const double* __restrict__ RX,
                       const double* __restrict__ RZ, Tp* __restrict__ WX,
                       Tp* __restrict__ WZ, const double* __restrict__ normA2,
                       double* __restrict__ err, double rank_tol, int* __restrict__ status) {
  extern __shared__ __align__(16) double ts_sm[];
  __shared__ int flag;
  const TsLay Ly = ts_layout(kp, lp);
  const int L = Ly.L;
  double* Rx = ts_sm + Ly.rx;
  double* Rz = ts_sm + Ly.rz;
  double* Cm = ts_sm + Ly.c;
  double* V = ts_sm + Ly.v;
  Tp* Zs = reinterpret_cast<Tp*>(ts_sm + Ly.zs);
  Tp* Ys = reinterpret_cast<Tp*>(ts_sm + Ly.ys);
  double* sig = ts_sm + Ly.sig;
  int* order = reinterpret_cast<int*>(ts_sm + Ly.order);
  const int b = blockIdx.x, tid = threadIdx.x;
  const MatDev mx = xm[b], mz = zm[b];
  const int k = mx.k, l = mz.k, r = mx.r;
  const long long m = mx.m;
  const double* rx = RX + (long long)b * kp * kp;
  const double* rz = RZ + (long long)b * lp * lp;
  for (int e = tid; e < kp * kp; e += TS_T) {
    const int i = e / kp, c = e % kp;
    Rx[i * L + c] = rx[e];
    V[i * L + c] = (i == c) ? 1.0 : 0.0;
  }
  for (int e = tid; e < lp * lp; e += TS_T) {
    const int i = e / lp, c = e % lp;
    Rz[i * L + c] = rz[e];
  }
  __syncthreads();
  if (tid == 0) {
    double mx1 = 0.0, mz1 = 0.0;
    for (int c = 0; c < k; ++c) mx1 = fmax(mx1, fabs(Rx[c * L + c]));
    for (int c = 0; c < l; ++c) mz1 = fmax(mz1, fabs(Rz[c * L + c]));
    bool def = (mx1 == 0.0) || (mz1 == 0.0);
    for (int c = 0; c < k; ++c) def |= fabs(Rx[c * L + c]) <= rank_tol * mx1;
    for (int c = 0; c < l; ++c) def |= fabs(Rz[c * L + c]) <= rank_tol * mz1;
    if (def) atomicOr(status, kStatusRankDef);
  }
  // M = Z^T Y (l x k), thread t owns the entries e = t + 256 q
  const int nent = l * k;
  double acc[TS_MAXQ];
#pragma unroll
  for (int q = 0; q < TS_MAXQ; ++q) acc[q] = 0.0;
  const Tp* Zm = Z + mz.offY;
  const Tp* Ym = Y + mx.offY;
  for (long long r0 = 0; r0 < m; r0 += TS_RB) {
    const int nr = (int)((m - r0) < TS_RB ? (m - r0) : TS_RB);
    for (int e = tid; e < TS_RB * lp; e += TS_T) {
      const int rr = e / lp;
      Zs[e] = rr < nr ? Zm[(r0 + rr) * lp + (e - rr * lp)] : Tp(0);
    }
    for (int e = tid; e < TS_RB * kp; e += TS_T) {
      const int rr = e / kp;
      Ys[e] = rr < nr ? Ym[(r0 + rr) * kp + (e - rr * kp)] : Tp(0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < TS_MAXQ; ++q) {
      const int e = tid + q * TS_T;
      if (e < nent) {
        const int i = e / k, j = e - (e / k) * k;
        Tp s = Tp(0);
        for (int rr = 0; rr < nr; ++rr) s += Zs[rr * lp + i] * Ys[rr * kp + j];
        acc[q] += (double)s;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < TS_MAXQ; ++q) {
    const int e = tid + q * TS_T;
    if (e < nent) Cm[(e / k) * L + (e % k)] = acc[q];
  }
  __syncthreads();
  // C <- C R_X^{-1} (each row, forward substitution)
  for (int i = tid; i < l; i += TS_T) {
    double* row = Cm + i * L;
    for (int c = 0; c < k; ++c) {
      double t = row[c];
      for (int cc = 0; cc < c; ++cc) t -= row[cc] * Rx[cc * L + c];
      const double d = Rx[c * L + c];
      row[c] = d != 0.0 ? t / d : 0.0;
    }
  }
  __syncthreads();
  // C <- R_Z^{-T} C (each column, forward substitution with R_Z^T lower)
  for (int j = tid; j < k; j += TS_T) {
    for (int i = 0; i < l; ++i) {
      double t = Cm[i * L + j];
      for (int ii = 0; ii < i; ++ii) t -= Rz[ii * L + i] * Cm[ii * L + j];
      const double d = Rz[i * L + i];
      Cm[i * L + j] = d != 0.0 ? t / d : 0.0;
    }
  }
  __syncthreads();
  ts_jacobi(Cm, V, l, k, L, &flag);
  __syncthreads();
  for (int c = tid; c < k; c += TS_T) {
    double a = 0.0;
    for (int i = 0; i < l; ++i) a += Cm[i * L + c] * Cm[i * L + c];
    sig[c] = sqrt(a);
  }
  __syncthreads();
  for (int c = tid; c < k; c += TS_T) {
    int rank = 0;
    // NaN below everything: the ranking is a permutation whatever the values
    const double sc = sig[c] == sig[c] ? sig[c] : -INFINITY;
    for (int c2 = 0; c2 < k; ++c2) {
      const double s2 = sig[c2] == sig[c2] ? sig[c2] : -INFINITY;
      rank += (s2 > sc) || (s2 == sc && c2 < c);
    }
    order[rank] = c;
  }
  __syncthreads();
  if (mx.sigma != nullptr)
    for (int c = tid; c < k; c += TS_T) ((Tp*)mx.sigma)[c] = (Tp)sig[order[c]];
  if (tid == 0) {
    double cap = 0.0;
    for (int c = 0; c < r; ++c) cap += sig[order[c]] * sig[order[c]];
    const double e2 = normA2[b] - cap;
    err[b] = sqrt(e2 > 0.0 ? e2 : 0.0);
  }
  // WX = R_X^{-1} V_r, WZ = R_Z^{-1} (C V)_r (back substitution per column)
  Tp* wx = WX + (long long)b * kp * kp;
  Tp* wz = WZ + (long long)b * lp * lp;
  for (int e = tid; e < kp * kp; e += TS_T) wx[e] = Tp(0);
  for (int e = tid; e < lp * lp; e += TS_T) wz[e] = Tp(0);
  __syncthreads();
  for (int c = tid; c < 2 * r; c += TS_T) {
    const bool zside = c >= r;
    const int cc = zside ? c - r : c, col = order[cc];
    const double* R = zside ? Rz : Rx;
    const double* rhs = zside ? Cm : V;
    const int nn = zside ? l : k;
    double tmp[64];
    for (int i = nn - 1; i >= 0; --i) {
      double t = rhs[i * L + col];
      for (int i2 = i + 1; i2 < nn; ++i2) t -= R[i * L + i2] * tmp[i2];
      const double d = R[i * L + i];
      tmp[i] = d != 0.0 ? t / d : 0.0;
    }
    if (zside)
      for (int i = 0; i < nn; ++i) wz[i * lp + cc] = (Tp)tmp[i];
    else
      for (int i = 0; i < nn; ++i) wx[i * kp + cc] = (Tp)tmp[i];
  }
}

}  // namespace

cudaError_t launch_wt_panel(int prec, const void* W, int l, long long n, int lp, void* out,
                            cudaStream_t s) {
  const long long tot = n * lp;
  const unsigned blocks = (unsigned)((tot + 255) / 256);
  if (prec == 0)
    wt_panel_kernel<double, double><<<blocks, 256, 0, s>>>((const double*)W, l, n, lp,
                                                            (double*)out);
  else
    wt_panel_kernel<float, float><<<blocks, 256, 0, s>>>((const float*)W, l, n, lp,
                                                          (float*)out);
  return cudaGetLastError();
}

cudaError_t launch_two_sided_small(bool dbl, int kp, int lp, const MatDev* xm,
                                   const MatDev* zm, int count, const void* Y, const void* Z,
                                   const double* RX, const double* RZ, void* WX, void* WZ,
                                   const double* normA2, double* err, int* status,
                                   cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (kp > 64 || lp > 64) return cudaErrorInvalidValue;
  const size_t sm = ts_layout(kp, lp).bytes;
  cudaError_t e;
  if (dbl) {
    e = cudaFuncSetAttribute(two_sided_small_kernel<double>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    two_sided_small_kernel<double><<<count, TS_T, sm, s>>>(
        kp, lp, xm, zm, (const double*)Y, (const double*)Z, RX, RZ, (double*)WX, (double*)WZ,
        normA2, err, 1e-12, status);
  } else {
    e = cudaFuncSetAttribute(two_sided_small_kernel<float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    two_sided_small_kernel<float><<<count, TS_T, sm, s>>>(
        kp, lp, xm, zm, (const float*)Y, (const float*)Z, RX, RZ, (float*)WX, (float*)WZ,
        normA2, err, 1e-5, status);
  }
  return cudaGetLastError();
}

}  // namespace tsk
