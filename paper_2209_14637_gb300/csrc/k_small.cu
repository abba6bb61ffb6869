// Per-matrix small factorizations of the test pass and the eigensolver:
//
//  * tsqr_kernel: R factor of a tall skinny panel (n x k for X, m x k for Y)
//    by blockwise Householder QR ("TSQR"), optionally followed by one
//    refinement pass on Q1 = P R^{-1} (the same scheme run again; R <- R2 R).
//  * small_svd_kernel: with X = Q R_X and Y = A X = Q_Y R_Y,
//    A Q = Y R_X^{-1} = Q_Y (R_Y R_X^{-1}), so the singular values and right
//    singular vectors of A Q are those of the k x k matrix T = R_Y R_X^{-1}.
//    One-sided Jacobi (Hestenes) on T, then the error identity
//    ||A - [AQ]_r Q^T||^2 = ||A||^2 - sum_{i<=r} sigma_i^2 (proof of
//    Theorem 1, Eq. A.3) and W = R_X^{-1} V_r for the factored outputs.
//  * sym_eig_kernel: eigen-decomposition of the small symmetric PSD
//    Rayleigh-Ritz matrix of the subspace iteration (one-sided Jacobi).
#include <cuda_bf16.h>
#include <float.h>

#include <algorithm>

#include "tsk_internal.cuh"

namespace tsk {

namespace {

template <typename T>
struct Eps;
template <>
struct Eps<float> {
  // above the rounding noise of a k-term FP32 dot product (about
  // sqrt(k) * 6e-8), so that converged columns stop rotating
  static constexpr float jacobi = 4.0e-6f;
  static constexpr float tiny = 1.0e-30f;
};
template <>
struct Eps<double> {
  static constexpr double jacobi = 1.0e-14;
  static constexpr double tiny = 1.0e-280;
};

// Round-robin ("circle method") pairing: kk players (even), kk-1 rounds,
// kk/2 disjoint pairs per round; over a sweep every pair meets once.
__device__ __forceinline__ void rr_pair(int round, int i, int kk, int& p,
                                        int& q) {
  const int mm = kk - 1;
  if (i == 0) {
    p = round % mm;
    q = mm;
  } else {
    p = (round + i) % mm;
    q = (round - i + mm) % mm;
  }
}

// One-sided Jacobi on the columns of M (nrow x ncol, leading dimension ld)
// accumulating the rotations into V (ncol x ncol, ld).  On return the
// columns of M are mutually orthogonal: M_in V = M_out, and the column
// norms of M_out are the singular values.  Whole-block cooperative.
template <typename T>
__device__ void jacobi_columns(T* M, T* V, int nrow, int ncol, int ld,
                               int max_sweeps, int* rotated_flag) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  const int kk = ncol + (ncol & 1);
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (threadIdx.x == 0) *rotated_flag = 0;
    __syncthreads();
    for (int round = 0; round < kk - 1; ++round) {
      for (int pi = warp; pi < kk / 2; pi += nwarps) {
        int p, q;
        rr_pair(round, pi, kk, p, q);
        if (p >= ncol || q >= ncol) continue;
        T a = T(0), b = T(0), g = T(0);
        for (int i = lane; i < nrow; i += 32) {
          const T x = M[i * ld + p], y = M[i * ld + q];
          a += x * x;
          b += y * y;
          g += x * y;
        }
        a = warp_sum(a);
        b = warp_sum(b);
        g = warp_sum(g);
        if (fabs(g) > Eps<T>::jacobi * sqrt(a * b) && fabs(g) > Eps<T>::tiny) {
          const T zeta = (b - a) / (T(2) * g);
          const T t = (zeta >= T(0) ? T(1) : T(-1)) /
                      (fabs(zeta) + sqrt(T(1) + zeta * zeta));
          const T c = T(1) / sqrt(T(1) + t * t), s = c * t;
          for (int i = lane; i < nrow; i += 32) {
            const T x = M[i * ld + p], y = M[i * ld + q];
            M[i * ld + p] = c * x - s * y;
            M[i * ld + q] = s * x + c * y;
          }
          for (int i = lane; i < ncol; i += 32) {
            const T x = V[i * ld + p], y = V[i * ld + q];
            V[i * ld + p] = c * x - s * y;
            V[i * ld + q] = s * x + c * y;
          }
          if (lane == 0) *rotated_flag = 1;
        }
      }
      __syncthreads();
    }
    if (*rotated_flag == 0) break;
    __syncthreads();
  }
}

// NaN ordered below every number (-inf included: ties go by index), so a
// ranking by it is a permutation whatever the values.
template <typename T>
__device__ __forceinline__ T nan_low(T x) {
  return x == x ? x : -INFINITY;
}

// sig[c] = ||M[:, c]||, order[rank] = c with descending sig (stable; a
// permutation even when some norms are NaN).
template <typename T>
__device__ void column_norms_sorted(const T* M, int nrow, int ncol, int ld,
                                    T* sig, int* order) {
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    T a = T(0);
    for (int i = 0; i < nrow; ++i) a += M[i * ld + c] * M[i * ld + c];
    sig[c] = sqrt(a);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < ncol; c += blockDim.x) {
    int rank = 0;
    for (int c2 = 0; c2 < ncol; ++c2)
      rank += (nan_low(sig[c2]) > nan_low(sig[c])) ||
              (nan_low(sig[c2]) == nan_low(sig[c]) && c2 < c);
    order[rank] = c;
  }
  __syncthreads();
}

}  // namespace

// ---------------------------------------------------------------------------
// E2 / E4: R factor of a tall panel by blockwise Householder QR.
// The running R (k x k) is stacked on top of the next block of 64 rows and
// the stack is reduced column by column; only R's diagonal entry and the
// block's column take part in each reflector because R is already upper
// triangular.  With refine = 1 the panel is passed again as Q1 = P R0^{-1}
// (computed row by row on load), and the result is R = R2 R0.
// ---------------------------------------------------------------------------
template <typename T, typename Tin>
__global__ void __launch_bounds__(256)
tsqr_kernel(int kp, const PanelDev* __restrict__ panels, int refine) {
  constexpr int B = 64;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = kp + 1;
  T* Bs = (T*)smem_raw;
  T* Rs = Bs + B * ld;
  T* R0 = Rs + kp * ld;
  __shared__ T sh_tau;
  const PanelDev pd = panels[blockIdx.x];
  const int k = pd.k, pld = pd.ld;
  const long long rows = pd.rows;
  const Tin* __restrict__ P = (const Tin*)pd.P;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < kp * ld; e += blockDim.x) {
    Rs[e] = T(0);
    R0[e] = T(0);
  }
  __syncthreads();
  for (int pass = 0; pass <= refine; ++pass) {
    if (pass == 1) {
      for (int e = tid; e < kp * ld; e += blockDim.x) {
        R0[e] = Rs[e];
        Rs[e] = T(0);
      }
      __syncthreads();
    }
    for (long long r0 = 0; r0 < rows; r0 += B) {
      for (int e = tid; e < B * kp; e += blockDim.x) {
        const int ii = e / kp, c = e % kp;
        const long long gi = r0 + ii;
        Bs[ii * ld + c] = (gi < rows && c < k) ? (T)P[gi * pld + c] : T(0);
      }
      __syncthreads();
      if (pass == 1) {
        for (int ii = tid; ii < B; ii += blockDim.x) {
          T* row = Bs + ii * ld;
          for (int c = 0; c < k; ++c) {
            T t = row[c];
            for (int cc = 0; cc < c; ++cc) t -= row[cc] * R0[cc * ld + c];
            const T d = R0[c * ld + c];
            row[c] = (d != T(0)) ? t / d : T(0);
          }
        }
        __syncthreads();
      }
      for (int j = 0; j < k; ++j) {
        if (warp == 0) {
          T s2 = T(0);
          for (int ii = lane; ii < B; ii += 32) {
            const T v = Bs[ii * ld + j];
            s2 += v * v;
          }
          s2 = warp_sum(s2);
          const T alpha = Rs[j * ld + j];
          T tau = T(0);
          if (s2 > T(0)) {
            const T nrm = sqrt(alpha * alpha + s2);
            const T beta = (alpha >= T(0)) ? -nrm : nrm;
            const T scale = T(1) / (alpha - beta);
            tau = (beta - alpha) / beta;
            for (int ii = lane; ii < B; ii += 32) Bs[ii * ld + j] *= scale;
            if (lane == 0) Rs[j * ld + j] = beta;
          }
          if (lane == 0) sh_tau = tau;
        }
        __syncthreads();
        const T tau = sh_tau;
        if (tau != T(0)) {
          for (int c = j + 1 + warp; c < k; c += (blockDim.x >> 5)) {
            T w = T(0);
            for (int ii = lane; ii < B; ii += 32)
              w += Bs[ii * ld + j] * Bs[ii * ld + c];
            w = warp_sum(w) + Rs[j * ld + c];
            const T tw = tau * w;
            for (int ii = lane; ii < B; ii += 32)
              Bs[ii * ld + c] -= Bs[ii * ld + j] * tw;
            if (lane == 0) Rs[j * ld + c] -= tw;
          }
        }
        __syncthreads();
      }
    }
  }
  T* __restrict__ Rout = (T*)pd.R;
  for (int e = tid; e < kp * kp; e += blockDim.x) {
    const int a = e / kp, b = e % kp;
    T v = T(0);
    if (a < k && b < k && a <= b) {
      if (refine) {
        for (int c = a; c <= b; ++c) v += Rs[a * ld + c] * R0[c * ld + b];
      } else {
        v = Rs[a * ld + b];
      }
    }
    Rout[e] = v;
  }
}

static size_t tsqr_smem(int kp, size_t elt) {
  return (size_t)(64 + 2 * kp) * (kp + 1) * elt;
}

template <typename T, typename Tin>
static cudaError_t tsqr_t(int kp, const PanelDev* panels, int count, int refine,
                          cudaStream_t s) {
  const size_t sm = tsqr_smem(kp, sizeof(T));
  cudaError_t e = cudaFuncSetAttribute(tsqr_kernel<T, Tin>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  tsqr_kernel<T, Tin><<<count, 256, sm, s>>>(kp, panels, refine);
  return cudaGetLastError();
}

cudaError_t launch_tsqr(bool dbl, int kp, const PanelDev* panels, int count,
                        int refine, int* /*status*/, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  return dbl ? tsqr_t<double, double>(kp, panels, count, refine, s)
             : tsqr_t<float, float>(kp, panels, count, refine, s);
}

cudaError_t launch_tsqr_f32_in_f64(int kp, const PanelDev* panels, int count, int refine,
                                   cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  return tsqr_t<double, float>(kp, panels, count, refine, s);
}

// ---------------------------------------------------------------------------
// E4 + E5 per matrix: T = R_Y R_X^{-1}, one-sided Jacobi SVD of T, sort,
// error by the projection identity (double), W = R_X^{-1} V_r.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
small_svd_kernel(int kp, const MatDev* __restrict__ mats,
                 const T* __restrict__ RX, const T* __restrict__ RY,
                 T* __restrict__ Wm, const double* __restrict__ normA2,
                 double* __restrict__ err, int* __restrict__ flags, int err_mode,
                 double tau, int sigma_f32, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = kp + 1;
  T* Rx = (T*)smem_raw;
  T* Tm = Rx + kp * ld;
  T* V = Tm + kp * ld;
  T* sig = V + kp * ld;
  int* order = (int*)(sig + kp);
  __shared__ int rotated;
  const int b = blockIdx.x, tid = threadIdx.x;
  const MatDev md = mats[b];
  const int k = md.k, r = md.r;
  const T* rx = RX + (long long)b * kp * kp;
  const T* ry = RY + (long long)b * kp * kp;
  for (int e = tid; e < kp * kp; e += blockDim.x) {
    const int i = e / kp, c = e % kp;
    Rx[i * ld + c] = rx[e];
    Tm[i * ld + c] = ry[e];
    V[i * ld + c] = (i == c) ? T(1) : T(0);
  }
  __syncthreads();
  if (tid == 0) {
    T mx = T(0);
    for (int c = 0; c < k; ++c) mx = fmax(mx, fabs(Rx[c * ld + c]));
    const T tol = (sizeof(T) == 8) ? T(1e-12) : T(1e-5);
    bool def = (mx == T(0));
    for (int c = 0; c < k; ++c) def |= fabs(Rx[c * ld + c]) <= tol * mx;
    if (def) atomicOr(status, kStatusRankDef);
  }
  // T = R_Y R_X^{-1}, row by row, in place (row i of Tm starts as R_Y).
  for (int i = tid; i < k; i += blockDim.x) {
    T* row = Tm + i * ld;
    for (int c = 0; c < k; ++c) {
      T t = row[c];
      for (int cc = 0; cc < c; ++cc) t -= row[cc] * Rx[cc * ld + c];
      const T d = Rx[c * ld + c];
      row[c] = (d != T(0)) ? t / d : T(0);
    }
  }
  __syncthreads();
  jacobi_columns<T>(Tm, V, k, k, ld, 60, &rotated);
  __syncthreads();
  column_norms_sorted<T>(Tm, k, k, ld, sig, order);
  if (md.sigma != nullptr)
    for (int c = tid; c < k; c += blockDim.x) {
      if (sigma_f32)
        ((float*)md.sigma)[c] = (float)sig[order[c]];
      else
        ((T*)md.sigma)[c] = sig[order[c]];
    }
  if (tid == 0) {
    double cap = 0.0;
    for (int c = 0; c < r; ++c) {
      const double sv = (double)sig[order[c]];
      cap += sv * sv;
    }
    const double tot = normA2[b];
    const double e2 = tot - cap;
    err[b] = sqrt(e2 > 0.0 ? e2 : 0.0);
    // err_mode 0: identity, direct pass where it cancels; 2: direct always
    flags[b] = (err_mode == 2) || (err_mode == 0 && e2 < tau * tot);
  }
  // W = R_X^{-1} V_r (k x r): back substitution, one column per thread.
  T* Wout = Wm + (long long)b * kp * kp;
  for (int e = tid; e < kp * kp; e += blockDim.x) Wout[e] = T(0);
  __syncthreads();
  for (int c = tid; c < r; c += blockDim.x) {
    const int col = order[c];
    for (int i = k - 1; i >= 0; --i) {
      T t = V[i * ld + col];
      for (int i2 = i + 1; i2 < k; ++i2) t -= Rx[i * ld + i2] * Wout[i2 * kp + c];
      const T d = Rx[i * ld + i];
      Wout[i * kp + c] = (d != T(0)) ? t / d : T(0);
    }
  }
}

static size_t small_svd_smem(int kp, size_t elt) {
  return (size_t)3 * kp * (kp + 1) * elt + kp * elt + kp * sizeof(int) + 16;
}

cudaError_t launch_small_svd(bool dbl, int kp, const MatDev* mats, int count,
                             const void* RX, const void* RY, void* Wm,
                             double* normA2, double* err, int* flags, int err_mode,
                             double tau, int* status, cudaStream_t s, int sigma_f32) {
  if (count <= 0) return cudaSuccess;
  if (dbl) {
    const size_t sm = small_svd_smem(kp, sizeof(double));
    cudaError_t e = cudaFuncSetAttribute(small_svd_kernel<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    small_svd_kernel<double><<<count, 256, sm, s>>>(
        kp, mats, (const double*)RX, (const double*)RY, (double*)Wm, normA2,
        err, flags, err_mode, tau, sigma_f32, status);
  } else {
    const size_t sm = small_svd_smem(kp, sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(small_svd_kernel<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    small_svd_kernel<float><<<count, 256, sm, s>>>(
        kp, mats, (const float*)RX, (const float*)RY, (float*)Wm, normA2, err,
        flags, err_mode, tau, 0, status);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// T2: eigen-decomposition of the p x p symmetric PSD Rayleigh-Ritz matrix H
// (one CTA).  For a PSD matrix the right singular vectors are eigenvectors
// and the singular values the eigenvalues.  theta (p) descending; V (p x p)
// has the matching eigenvectors as columns.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
sym_eig_kernel(const T* __restrict__ H, int p, T* __restrict__ theta,
               T* __restrict__ Vout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = p + 1;
  T* M = (T*)smem_raw;
  T* V = M + p * ld;
  T* sig = V + p * ld;
  int* order = (int*)(sig + p);
  __shared__ int rotated;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, c = e % p;
    M[i * ld + c] = T(0.5) * (H[i * p + c] + H[c * p + i]);
    V[i * ld + c] = (i == c) ? T(1) : T(0);
  }
  __syncthreads();
  jacobi_columns<T>(M, V, p, p, ld, 60, &rotated);
  __syncthreads();
  column_norms_sorted<T>(M, p, p, ld, sig, order);
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int i = e / p, c = e % p;
    Vout[i * p + c] = V[i * ld + order[c]];
  }
  for (int c = threadIdx.x; c < p; c += blockDim.x) theta[c] = sig[order[c]];
}

// The same eigen-decomposition in FP32 with the columns in registers: thread
// (j, qt) = (tid / 4, tid % 4) holds rows [qt QMAX, qt QMAX + QMAX) of
// column j of M (H rotated) and of V.  Each round of the round-robin order
// the threads store their parts to one of two planes, read the partner
// column's parts after one barrier, sum the three dot products over the
// column's four threads, and both columns' threads derive the same rotation
// from the same sums (the rotation and the stopping rule are those of
// jacobi_columns).  p <= 4 QMAX <= 96.
__device__ __forceinline__ int rr_partner(int round, int j, int mm) {
  if (j == mm) return round;
  if (j == round) return mm;
  int x = 2 * round - j;
  if (x < 0) x += mm;
  if (x >= mm) x -= mm;
  return x;
}

template <int QMAX>
__global__ void __launch_bounds__(384)
sym_eig_reg_kernel(const float* __restrict__ H, int p, float* __restrict__ theta,
                   float* __restrict__ Vout) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int jl = 4 * QMAX + 4;  // column stride of a plane
  float* PL = (float*)smem_raw;     // [2 buffers][M, V][p][jl]
  float* lam = PL + 4 * p * jl;
  int* order = (int*)(lam + p);
  const int tid = threadIdx.x, lane = tid & 31;
  const int j = tid >> 2, qt = tid & 3, i0 = qt * QMAX;
  float m[QMAX], v[QMAX];
#pragma unroll
  for (int i = 0; i < QMAX; ++i) {
    const int row = i0 + i;
    const bool in = j < p && row < p;
    m[i] = in ? 0.5f * (H[row * p + j] + H[j * p + row]) : 0.f;
    v[i] = (in && row == j) ? 1.f : 0.f;
  }
  const unsigned gmask = 0xFu << (lane & 28);  // the column's four threads
  const int kk = p + (p & 1), mm = kk - 1;
  int t = 0;
  for (int sweep = 0; sweep < 60 && mm > 0; ++sweep) {
    int rot = 0;
    for (int round = 0; round < mm; ++round, ++t) {
      float* Bm = PL + (t & 1) * 2 * p * jl;
      float* Bv = Bm + p * jl;
      if (j < p) {
#pragma unroll
        for (int i = 0; i < QMAX; i += 4) {
          *reinterpret_cast<float4*>(Bm + j * jl + i0 + i) =
              make_float4(m[i], m[i + 1], m[i + 2], m[i + 3]);
          *reinterpret_cast<float4*>(Bv + j * jl + i0 + i) =
              make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
        }
      }
      __syncthreads();
      const int pj = j < p ? rr_partner(round, j, mm) : p;
      if (pj < p) {  // the column's four threads take this branch together
        float y[QMAX], w[QMAX];
#pragma unroll
        for (int i = 0; i < QMAX; i += 4) {
          const float4 a = *reinterpret_cast<const float4*>(Bm + pj * jl + i0 + i);
          const float4 b = *reinterpret_cast<const float4*>(Bv + pj * jl + i0 + i);
          y[i] = a.x;
          y[i + 1] = a.y;
          y[i + 2] = a.z;
          y[i + 3] = a.w;
          w[i] = b.x;
          w[i + 1] = b.y;
          w[i + 2] = b.z;
          w[i + 3] = b.w;
        }
        float aa = 0.f, pp = 0.f, ap = 0.f;
#pragma unroll
        for (int i = 0; i < QMAX; ++i) {
          aa = fmaf(m[i], m[i], aa);
          pp = fmaf(y[i], y[i], pp);
          ap = fmaf(m[i], y[i], ap);
        }
        aa += __shfl_xor_sync(gmask, aa, 1);
        pp += __shfl_xor_sync(gmask, pp, 1);
        ap += __shfl_xor_sync(gmask, ap, 1);
        aa += __shfl_xor_sync(gmask, aa, 2);
        pp += __shfl_xor_sync(gmask, pp, 2);
        ap += __shfl_xor_sync(gmask, ap, 2);
        const bool low = j < pj;  // the lower index is the first column of the pair
        const float alpha = low ? aa : pp, beta = low ? pp : aa, gamma = ap;
        if (fabsf(gamma) > Eps<float>::jacobi * sqrtf(alpha * beta) &&
            fabsf(gamma) > Eps<float>::tiny) {
          const float zeta = (beta - alpha) / (2.f * gamma);
          const float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float c = 1.f / sqrtf(1.f + tt * tt), sn = c * tt;
          // first column <- c first - s second; second <- s first + c second
          if (low) {
#pragma unroll
            for (int i = 0; i < QMAX; ++i) {
              m[i] = c * m[i] - sn * y[i];
              v[i] = c * v[i] - sn * w[i];
            }
          } else {
#pragma unroll
            for (int i = 0; i < QMAX; ++i) {
              m[i] = sn * y[i] + c * m[i];
              v[i] = sn * w[i] + c * v[i];
            }
          }
          rot = 1;
        }
      }
    }
    if (!__syncthreads_or(rot)) break;
  }
  // theta_j = ||M[:, j]||; V columns to plane 0
  float nn = 0.f;
#pragma unroll
  for (int i = 0; i < QMAX; ++i) nn = fmaf(m[i], m[i], nn);
  nn += __shfl_xor_sync(0xffffffffu, nn, 1);
  nn += __shfl_xor_sync(0xffffffffu, nn, 2);
  float* Vs = PL + p * jl;
  if (j < p) {
    if (qt == 0) lam[j] = sqrtf(nn);
#pragma unroll
    for (int i = 0; i < QMAX; i += 4)
      *reinterpret_cast<float4*>(Vs + j * jl + i0 + i) =
          make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
  }
  __syncthreads();
  for (int c = tid; c < p; c += blockDim.x) {  // descending; NaN ranks last
    const float lc = lam[c] == lam[c] ? lam[c] : -INFINITY;
    int rank = 0;
    for (int c2 = 0; c2 < p; ++c2) {
      const float l2 = lam[c2] == lam[c2] ? lam[c2] : -INFINITY;
      rank += (l2 > lc) || (l2 == lc && c2 < c);
    }
    order[rank] = c;
  }
  __syncthreads();
  for (int e = tid; e < p * p; e += blockDim.x) {
    const int i = e / p, c = e - i * p;
    Vout[e] = Vs[order[c] * jl + i];
  }
  for (int c = tid; c < p; c += blockDim.x) theta[c] = lam[order[c]];
}

template <int QMAX>
static cudaError_t launch_sym_eig_reg(const float* H, int p, float* theta, float* V,
                                      cudaStream_t s) {
  constexpr int jl = 4 * QMAX + 4;
  const size_t sm = (size_t)4 * p * jl * sizeof(float) + (size_t)p * (sizeof(float) + sizeof(int));
  cudaError_t e = cudaFuncSetAttribute(sym_eig_reg_kernel<QMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const unsigned nt = (unsigned)((4 * p + 31) / 32 * 32);
  sym_eig_reg_kernel<QMAX><<<1, nt, sm, s>>>(H, p, theta, V);
  return cudaGetLastError();
}

cudaError_t launch_sym_eig(bool dbl, const void* H, int p, void* theta,
                           void* V, cudaStream_t s) {
  if (!dbl && p >= 1 && p <= 96) {
    const int q = ((p + 3) / 4 + 3) / 4 * 4;  // rows per thread, a multiple of 4
    switch (q) {
      case 4: return launch_sym_eig_reg<4>((const float*)H, p, (float*)theta, (float*)V, s);
      case 8: return launch_sym_eig_reg<8>((const float*)H, p, (float*)theta, (float*)V, s);
      case 12: return launch_sym_eig_reg<12>((const float*)H, p, (float*)theta, (float*)V, s);
      case 16: return launch_sym_eig_reg<16>((const float*)H, p, (float*)theta, (float*)V, s);
      case 20: return launch_sym_eig_reg<20>((const float*)H, p, (float*)theta, (float*)V, s);
      default: return launch_sym_eig_reg<24>((const float*)H, p, (float*)theta, (float*)V, s);
    }
  }
  const size_t elt = dbl ? sizeof(double) : sizeof(float);
  const size_t sm = (size_t)2 * p * (p + 1) * elt + p * elt + p * sizeof(int) + 16;
  if (dbl) {
    cudaError_t e = cudaFuncSetAttribute(
        sym_eig_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    sym_eig_kernel<double><<<1, 256, sm, s>>>((const double*)H, p,
                                              (double*)theta, (double*)V);
  } else {
    cudaError_t e = cudaFuncSetAttribute(
        sym_eig_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    sym_eig_kernel<float><<<1, 256, sm, s>>>((const float*)H, p,
                                             (float*)theta, (float*)V);
  }
  return cudaGetLastError();
}



}  // namespace tsk
