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

// sig[c] = ||M[:, c]||, order[rank] = c with descending sig (stable).
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
      rank += (sig[c2] > sig[c]) || (sig[c2] == sig[c] && c2 < c);
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
template <typename T>
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
  const T* __restrict__ P = (const T*)pd.P;
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
        Bs[ii * ld + c] = (gi < rows && c < k) ? P[gi * pld + c] : T(0);
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

cudaError_t launch_tsqr(bool dbl, int kp, const PanelDev* panels, int count,
                        int refine, int* /*status*/, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (dbl) {
    const size_t sm = tsqr_smem(kp, sizeof(double));
    cudaError_t e = cudaFuncSetAttribute(
        tsqr_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    tsqr_kernel<double><<<count, 256, sm, s>>>(kp, panels, refine);
  } else {
    const size_t sm = tsqr_smem(kp, sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(
        tsqr_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    tsqr_kernel<float><<<count, 256, sm, s>>>(kp, panels, refine);
  }
  return cudaGetLastError();
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
                 double tau, int* __restrict__ status) {
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
    for (int c = tid; c < k; c += blockDim.x)
      ((T*)md.sigma)[c] = sig[order[c]];
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
                             double tau, int* status, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (dbl) {
    const size_t sm = small_svd_smem(kp, sizeof(double));
    cudaError_t e = cudaFuncSetAttribute(small_svd_kernel<double>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    small_svd_kernel<double><<<count, 256, sm, s>>>(
        kp, mats, (const double*)RX, (const double*)RY, (double*)Wm, normA2,
        err, flags, err_mode, tau, status);
  } else {
    const size_t sm = small_svd_smem(kp, sizeof(float));
    cudaError_t e = cudaFuncSetAttribute(small_svd_kernel<float>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sm);
    if (e != cudaSuccess) return e;
    small_svd_kernel<float><<<count, 256, sm, s>>>(
        kp, mats, (const float*)RX, (const float*)RY, (float*)Wm, normA2, err,
        flags, err_mode, tau, status);
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

cudaError_t launch_sym_eig(bool dbl, const void* H, int p, void* theta,
                           void* V, cudaStream_t s) {
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


// ---------------------------------------------------------------------------
// Gram route of the FP32 / BF16 paths (E2 + E4 without Householder).
//
//   R_X  = chol(X^T X)                       (X = Q R_X; kappa(X) is modest)
//   R_X <- chol(Q1^T Q1) R_X,  Q1 = X R_X^-1 (one refinement step on Q)
//   M    = Y R_X^-1 = A Q                    (m x k, well conditioned)
//   sigma_i(AQ)^2 = lambda_i(M^T M),  V = eigenvectors,  W = R_X^-1 V_r
//
// Y itself is not factored: its columns grow like sigma_i^2 and Y^T Y would
// lose everything in FP32.  Partial Gram matrices are summed in FP32 over
// chunks of 256 rows and in FP64 across chunks; the k x k Cholesky and
// inverse run in FP64; the captured energy sum_{i<=r} v_i^T (M^T M) v_i is
// formed in FP64 from the FP32 eigenvectors.
// ---------------------------------------------------------------------------
namespace {
constexpr int GCHUNK = 256;  // rows per partial Gram
constexpr int GSUB = 64;     // rows staged in shared memory at a time
}  // namespace

// One CTA per (panel, chunk): partial G = P_c^T P_c over the chunk's rows,
// where P_c = P or P R^{-1} (Rinv: kp x kp FP32, upper, per panel).  Only the
// upper triangle is formed: the 4x4 tiles with tile-row <= tile-column are
// spread over the threads, and when there are fewer tiles than threads,
// several row groups share the rows of each staged block and are summed at
// the end.  Entries below the diagonal of the partial are left unwritten.
__global__ void __launch_bounds__(256)
panel_gram_kernel(int kp, const PanelDev* __restrict__ panels, const int2* __restrict__ chunks,
                  const float* __restrict__ rinv, float* __restrict__ partial) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 ch = chunks[blockIdx.x];
  const PanelDev pd = panels[ch.x];
  const int k = pd.k, ld = pd.ld;
  const int ldp = kp + 4;              // 16-byte aligned rows
  float* Ps = (float*)smem_raw;        // GSUB x ldp
  float* Ts = Ps + GSUB * ldp;         // GSUB x ldp transformed rows
  float* Rs = Ts + GSUB * ldp;         // kp x kp
  float* Red = Rs + kp * kp;           // 256 x 16 partial tiles of the row groups
  const float* P = (const float*)pd.P;
  const bool tr = (rinv != nullptr);
  if (tr) {
    const float* R = rinv + (long long)ch.x * kp * kp;
    for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) Rs[e] = R[e];
  }
  const int nt = kp / 4;
  const int ntiles = nt * (nt + 1) / 2;
  const int groups = max(1, (int)blockDim.x / ntiles);
  const int tid = threadIdx.x;
  const bool active = tid < groups * ntiles;
  const int tile = tid % ntiles, grp = tid / ntiles;
  // tile -> (ty, tx) with ty <= tx
  int ty = 0, rem = tile;
  while (rem >= nt - ty) {
    rem -= nt - ty;
    ++ty;
  }
  const int tx = ty + rem;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  const long long r0 = (long long)ch.y * GCHUNK;
  const long long r1 = min(pd.rows, r0 + GCHUNK);
  const int q4 = kp / 4;  // float4 per row
  for (long long s0 = r0; s0 < r1; s0 += GSUB) {
    __syncthreads();
    for (int e = tid; e < GSUB * q4; e += blockDim.x) {
      const int ii = e / q4, c4 = (e % q4) * 4;
      const long long i = s0 + ii;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < r1) {
        v = *reinterpret_cast<const float4*>(P + i * ld + c4);
        if (c4 + 0 >= k) v.x = 0.f;
        if (c4 + 1 >= k) v.y = 0.f;
        if (c4 + 2 >= k) v.z = 0.f;
        if (c4 + 3 >= k) v.w = 0.f;
      }
      *reinterpret_cast<float4*>(Ps + ii * ldp + c4) = v;
    }
    __syncthreads();
    const float* src = Ps;
    if (tr) {
      // Ts = Ps Rinv (Rinv upper triangular), four columns per work item
      for (int e = tid; e < GSUB * q4; e += blockDim.x) {
        const int ii = e / q4, c4 = (e % q4) * 4;
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        const int top = min(k, c4 + 4);
        for (int cc = 0; cc < top; ++cc) {
          const float p = Ps[ii * ldp + cc];
          const float4 r = *reinterpret_cast<const float4*>(Rs + cc * kp + c4);
          t.x = fmaf(p, r.x, t.x);
          t.y = fmaf(p, r.y, t.y);
          t.z = fmaf(p, r.z, t.z);
          t.w = fmaf(p, r.w, t.w);
        }
        *reinterpret_cast<float4*>(Ts + ii * ldp + c4) = t;
      }
      __syncthreads();
      src = Ts;
    }
    if (active) {
#pragma unroll 4
      for (int ii = grp; ii < GSUB; ii += groups) {
        const float4 x4 = *reinterpret_cast<const float4*>(src + ii * ldp + ty * 4);
        const float4 y4 = *reinterpret_cast<const float4*>(src + ii * ldp + tx * 4);
        const float x[4] = {x4.x, x4.y, x4.z, x4.w};
        const float y[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(x[a], y[b], acc[a][b]);
      }
    }
  }
  // sum the row groups
  if (active && grp > 0) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) Red[tid * 16 + a * 4 + b] = acc[a][b];
  }
  __syncthreads();
  if (active && grp == 0) {
    for (int g2 = 1; g2 < groups; ++g2) {
      const int t2 = g2 * ntiles + tile;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += Red[t2 * 16 + a * 4 + b];
    }
    float* out = partial + (long long)blockIdx.x * kp * kp;
#pragma unroll
    for (int a = 0; a < 4; ++a)
      *reinterpret_cast<float4*>(out + (ty * 4 + a) * kp + tx * 4) =
          make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
  }
}

// Entry (i, c) of a symmetric matrix whose partials hold the upper triangle.
__device__ __forceinline__ double gram_entry(const float* partial, int c0, int c1, int kp,
                                             int i, int c) {
  const int a = min(i, c), b = max(i, c);
  double s = 0.0;
  for (int q = c0; q < c1; ++q) s += (double)partial[(long long)q * kp * kp + a * kp + b];
  return s;
}

// One CTA per matrix: G = sum of its partials (added in FP64), R = chol(G)
// (upper, FP32, right-looking: each step scales a row and updates the
// trailing triangle in parallel); with prev != NULL the result is R prev
// (the refinement step).  rinv receives (R prev)^{-1}.  A pivot that is not
// positive, or tiny next to the largest, raises the rank-deficiency status.
__global__ void __launch_bounds__(256)
chol_kernel(int kp, const MatDev* __restrict__ mats, const int* __restrict__ chunk_off,
            const float* __restrict__ partial, const float* __restrict__ prev,
            float* __restrict__ rfac, float* __restrict__ rinv, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = kp + 1;
  float* G = (float*)smem_raw;  // kp x ld, becomes R in place
  float* T = G + kp * ld;       // kp x ld scratch
  float* Ri = T + kp * ld;      // kp x ld
  __shared__ float inv_d;
  __shared__ int bad;
  const int b = blockIdx.x, tid = threadIdx.x;
  const int k = mats[b].k;
  const int c0 = chunk_off[b], c1 = chunk_off[b + 1];
  for (int e = tid; e < kp * kp; e += blockDim.x) {
    const int i = e / kp, c = e % kp;
    G[i * ld + c] = (i < k && c < k && i <= c) ? (float)gram_entry(partial, c0, c1, kp, i, c) : 0.f;
    Ri[i * ld + c] = 0.f;
  }
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    if (tid == 0) {
      const float d = G[j * ld + j];
      if (!(d > 0.f)) bad = 1;
      const float r = d > 0.f ? sqrtf(d) : 0.f;
      G[j * ld + j] = r;
      inv_d = r > 0.f ? 1.f / r : 0.f;
    }
    __syncthreads();
    for (int c = j + 1 + tid; c < k; c += blockDim.x) G[j * ld + c] *= inv_d;
    __syncthreads();
    const int w = k - j - 1;
    for (int e = tid; e < w * w; e += blockDim.x) {
      const int a = j + 1 + e / w, c = j + 1 + e % w;
      if (a <= c) G[a * ld + c] = fmaf(-G[j * ld + a], G[j * ld + c], G[a * ld + c]);
    }
    __syncthreads();
  }
  if (tid == 0) {
    float mx = 0.f;
    for (int c = 0; c < k; ++c) mx = fmaxf(mx, fabsf(G[c * ld + c]));
    for (int c = 0; c < k; ++c) bad |= !(fabsf(G[c * ld + c]) > 1e-6f * mx);
    if (bad) atomicOr(status, kStatusRankDef);
  }
  __syncthreads();
  if (prev != nullptr) {  // R <- R prev, both upper triangular
    const float* Pv = prev + (long long)b * kp * kp;
    for (int e = tid; e < kp * kp; e += blockDim.x) {
      const int a = e / kp, c = e % kp;
      float t = 0.f;
      if (a <= c && c < k)
        for (int q = a; q <= c; ++q) t = fmaf(G[a * ld + q], Pv[q * kp + c], t);
      T[a * ld + c] = t;
    }
    __syncthreads();
    for (int e = tid; e < kp * kp; e += blockDim.x) G[(e / kp) * ld + e % kp] = T[(e / kp) * ld + e % kp];
    __syncthreads();
  }
  // Ri = R^{-1}: column c by back substitution
  for (int c = tid; c < k; c += blockDim.x) {
    for (int i = c; i >= 0; --i) {
      float t = (i == c) ? 1.f : 0.f;
      for (int q = i + 1; q <= c; ++q) t = fmaf(-G[i * ld + q], Ri[q * ld + c], t);
      const float d = G[i * ld + i];
      Ri[i * ld + c] = (d != 0.f) ? t / d : 0.f;
    }
  }
  __syncthreads();
  float* ro = rfac + (long long)b * kp * kp;
  float* ri = rinv + (long long)b * kp * kp;
  for (int e = tid; e < kp * kp; e += blockDim.x) {
    const int i = e / kp, c = e % kp;
    ro[e] = (i <= c) ? G[i * ld + c] : 0.f;
    ri[e] = Ri[i * ld + c];
  }
}

// Two-sided cyclic Jacobi on the symmetric A (k x k, leading dimension ld) in
// the parallel round-robin order: each round computes the rotations of its
// disjoint pairs from (A_pp, A_qq, A_pq), then applies them to the columns
// of A and V, then to the rows of A.  Whole-block cooperative.  On return
// diag(A) holds the eigenvalues and the columns of V the eigenvectors.
template <typename T>
__device__ void jacobi_sym(T* A, T* V, int k, int ld, int max_sweeps, T tol, T* cs,
                           int* pq, int* rotated) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int kk = k + (k & 1), np = kk / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) *rotated = 0;
    __syncthreads();
    for (int round = 0; round < kk - 1; ++round) {
      for (int i = tid; i < np; i += nt) {
        int p, q;
        rr_pair(round, i, kk, p, q);
        T c = T(1), sn = T(0);
        if (p < k && q < k) {
          const T apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
          if (fabs(apq) > tol * sqrt(fabs(app * aqq)) && fabs(apq) > Eps<T>::tiny) {
            const T tau = (aqq - app) / (T(2) * apq);
            const T t = (tau >= T(0) ? T(1) : T(-1)) / (fabs(tau) + sqrt(T(1) + tau * tau));
            c = T(1) / sqrt(T(1) + t * t);
            sn = t * c;
            *rotated = 1;
          }
        } else {
          p = -1;
        }
        cs[2 * i] = c;
        cs[2 * i + 1] = sn;
        pq[2 * i] = p;
        pq[2 * i + 1] = q;
      }
      __syncthreads();
      for (int e = tid; e < np * k; e += nt) {  // columns of A and V
        const int i = e / k, r = e % k;
        const int p = pq[2 * i], q = pq[2 * i + 1];
        if (p < 0) continue;
        const T c = cs[2 * i], sn = cs[2 * i + 1];
        const T x = A[r * ld + p], y = A[r * ld + q];
        A[r * ld + p] = c * x - sn * y;
        A[r * ld + q] = sn * x + c * y;
        const T vx = V[r * ld + p], vy = V[r * ld + q];
        V[r * ld + p] = c * vx - sn * vy;
        V[r * ld + q] = sn * vx + c * vy;
      }
      __syncthreads();
      for (int e = tid; e < np * k; e += nt) {  // rows of A
        const int i = e / k, r = e % k;
        const int p = pq[2 * i], q = pq[2 * i + 1];
        if (p < 0) continue;
        const T c = cs[2 * i], sn = cs[2 * i + 1];
        const T x = A[p * ld + r], y = A[q * ld + r];
        A[p * ld + r] = c * x - sn * y;
        A[q * ld + r] = sn * x + c * y;
      }
      __syncthreads();
    }
    if (*rotated == 0) break;
  }
}

// One CTA per matrix: G_M (FP64) from its partials; eigenpairs of G_M by
// two-sided Jacobi in FP32; V_r brought back to orthonormal in FP64 with one
// step V <- V (I - (V^T V - I) / 2) (its error is quadratic in the FP32
// orthogonality error); captured energy tr(V_r^T G_M V_r) in FP64 (Ky Fan:
// equal to sum_{i<=r} lambda_i up to second-order terms); err, sigma and
// W = R_X^{-1} V_r.
__global__ void __launch_bounds__(256)
eig_finish_kernel(int kp, const MatDev* __restrict__ mats, const int* __restrict__ chunk_off,
                  const float* __restrict__ partial, const float* __restrict__ rinv,
                  float* __restrict__ Wm, const double* __restrict__ normA2,
                  double* __restrict__ err, int* __restrict__ flags, int err_mode, double tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = kp + 1;
  double* G = (double*)smem_raw;      // kp x kp
  double* Vd = G + kp * kp;           // kp x kp : V_r (FP64 copy of the FP32 result)
  double* Ed = Vd + kp * kp;          // kp x kp : V_r^T V_r - I
  double* Vc = Ed + kp * kp;          // kp x kp : corrected V_r
  float* Af = (float*)(Vc + kp * kp); // kp x ld
  float* V = Af + kp * ld;            // kp x ld
  float* cs = V + kp * ld;            // 2 * kp
  float* lam = cs + 2 * kp;           // kp
  int* pq = (int*)(lam + kp);         // 2 * kp
  int* order = pq + 2 * kp;           // kp
  __shared__ int rotated;
  __shared__ double red[8];
  const int b = blockIdx.x, tid = threadIdx.x;
  const MatDev md = mats[b];
  const int k = md.k, r = md.r;
  const int c0 = chunk_off[b], c1 = chunk_off[b + 1];
  for (int e = tid; e < kp * kp; e += blockDim.x) {
    const int i = e / kp, c = e % kp;
    const double g = (i < k && c < k) ? gram_entry(partial, c0, c1, kp, i, c) : 0.0;
    G[e] = g;
    Af[i * ld + c] = (float)g;
    V[i * ld + c] = (i == c) ? 1.f : 0.f;
  }
  __syncthreads();
  jacobi_sym<float>(Af, V, k, ld, 12, 4.0e-6f, cs, pq, &rotated);
  for (int c = tid; c < k; c += blockDim.x) lam[c] = Af[c * ld + c];
  __syncthreads();
  for (int c = tid; c < k; c += blockDim.x) {  // descending eigenvalues
    int rank = 0;
    for (int c2 = 0; c2 < k; ++c2) rank += (lam[c2] > lam[c]) || (lam[c2] == lam[c] && c2 < c);
    order[rank] = c;
  }
  __syncthreads();
  for (int e = tid; e < k * r; e += blockDim.x) {
    const int i = e / r, c = e % r;
    Vd[i * kp + c] = (double)V[i * ld + order[c]];
  }
  __syncthreads();
  for (int e = tid; e < r * r; e += blockDim.x) {  // E = V_r^T V_r - I
    const int a = e / r, c = e % r;
    double t = (a == c) ? -1.0 : 0.0;
    for (int i = 0; i < k; ++i) t += Vd[i * kp + a] * Vd[i * kp + c];
    Ed[a * kp + c] = t;
  }
  __syncthreads();
  for (int e = tid; e < k * r; e += blockDim.x) {  // V_r <- V_r - V_r E / 2
    const int i = e / r, c = e % r;
    double t = 0.0;
    for (int a = 0; a < r; ++a) t += Vd[i * kp + a] * Ed[a * kp + c];
    Vc[i * kp + c] = Vd[i * kp + c] - 0.5 * t;
  }
  __syncthreads();
  double part = 0.0;  // tr(V_r^T G V_r)
  for (int e = tid; e < k * r; e += blockDim.x) {
    const int i = e / r, c = e % r;
    double gv = 0.0;
    for (int j = 0; j < k; ++j) gv += G[i * kp + j] * Vc[j * kp + c];
    part += Vc[i * kp + c] * gv;
  }
  part = warp_sum(part);
  if ((tid & 31) == 0) red[tid >> 5] = part;
  __syncthreads();
  if (tid == 0) {
    double cap = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) cap += red[w];
    const double tot = normA2[b];
    const double e2 = tot - cap;
    err[b] = sqrt(e2 > 0.0 ? e2 : 0.0);
    flags[b] = (err_mode == 2) || (err_mode == 0 && e2 < tau * tot);
  }
  if (md.sigma != nullptr)
    for (int c = tid; c < k; c += blockDim.x)
      ((float*)md.sigma)[c] = sqrtf(fmaxf(lam[order[c]], 0.f));
  // W = R_X^{-1} V_r
  const float* Ri = rinv + (long long)b * kp * kp;
  float* Wout = Wm + (long long)b * kp * kp;
  for (int e = tid; e < kp * kp; e += blockDim.x) {
    const int i = e / kp, c = e % kp;
    float t = 0.f;
    if (i < k && c < r)
      for (int q = i; q < k; ++q) t = fmaf(Ri[i * kp + q], (float)Vc[q * kp + c], t);
    Wout[e] = t;
  }
}

cudaError_t launch_gram_route(int kp, const MatDev* mats, int count, const PanelDev* xpanels,
                              const PanelDev* ypanels, const int2* xchunks, int nxc,
                              const int* xoff, const int2* ychunks, int nyc, const int* yoff,
                              float* partial_x, float* partial_y, float* r1, float* r2,
                              float* rinv, float* Wm, double* normA2, double* err, int* flags,
                              int err_mode, double tau, int refine, int* status,
                              cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const size_t gsm = (size_t)(2 * GSUB * (kp + 4) + kp * kp + 256 * 16) * sizeof(float);
  const size_t csm = (size_t)3 * kp * (kp + 1) * sizeof(float);
  const size_t esm = (size_t)4 * kp * kp * sizeof(double) +
                     (size_t)2 * kp * (kp + 1) * sizeof(float) + 3 * kp * sizeof(float) +
                     3 * kp * sizeof(int) + 16;
  cudaError_t e = cudaFuncSetAttribute(eig_finish_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)esm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gsm);
  if (e != cudaSuccess) return e;
  // R1 = chol(X^T X)
  panel_gram_kernel<<<nxc, 256, gsm, s>>>(kp, xpanels, xchunks, nullptr, partial_x);
  chol_kernel<<<count, 256, csm, s>>>(kp, mats, xoff, partial_x, nullptr, r1, rinv, status);
  if (refine) {
    // R = chol(Q1^T Q1) R1 with Q1 = X R1^{-1}
    panel_gram_kernel<<<nxc, 256, gsm, s>>>(kp, xpanels, xchunks, rinv, partial_x);
    chol_kernel<<<count, 256, csm, s>>>(kp, mats, xoff, partial_x, r1, r2, rinv, status);
  }
  // G_M = (Y R^{-1})^T (Y R^{-1})
  panel_gram_kernel<<<nyc, 256, gsm, s>>>(kp, ypanels, ychunks, rinv, partial_y);
  eig_finish_kernel<<<count, 256, esm, s>>>(kp, mats, yoff, partial_y, rinv, Wm, normA2, err,
                                            flags, err_mode, tau);
  return cudaGetLastError();
}

int gram_route_chunks(long long rows) { return (int)((rows + GCHUNK - 1) / GCHUNK); }

}  // namespace tsk
