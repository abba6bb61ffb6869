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
// chunks of up to 512 rows, and across chunks in FP64 (Cholesky) or FP32
// (eigenpairs);
// the k x k Cholesky, its inverse and the eigenpairs run in FP32; the
// captured energy sum_{i<=r} v_i^T (M^T M) v_i is summed in FP64 from FP32
// products.
// ---------------------------------------------------------------------------
namespace {
constexpr int GCHUNK = 512;  // rows per partial Gram
constexpr int GSUB = 64;     // rows per block
constexpr int GSTAGES = 4;   // blocks in flight
constexpr int GTHREADS = 256;
constexpr long long GWAIT_NS = 4000000000ll;  // bound on one wait for a block

__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
}  // namespace

// Shared memory of panel_gram_kernel: GSTAGES blocks of GSUB rows (kp floats
// each, as stored: the panels have leading dimension kp), the transformed rows (GSUB x (kp + 4)), R^{-1} (kp x kp)
// and one mbarrier per stage; at the end the stages hold the row groups'
// tiles (at most GTHREADS x 16 floats).
size_t panel_gram_smem(int kp) {
  const size_t st = (size_t)GSTAGES * GSUB * kp, ts = (size_t)GSUB * (kp + 4);
  return (std::max(st, (size_t)GTHREADS * 16) + ts + (size_t)kp * kp) * sizeof(float) +
         GSTAGES * sizeof(uint64_t);
}

// One CTA per (panel, chunk of GCHUNK rows): partial G = P_c^T P_c over the
// chunk's rows, where P_c = P or P R^{-1} (Rinv: kp x kp FP32, upper, per
// panel).  A block of GSUB rows of a panel is one contiguous run of memory,
// so one thread brings each block in with a bulk copy (its bytes counted on
// the stage's mbarrier), GSTAGES blocks ahead.  The transform gives each
// thread a 4 x 4 tile of P R^{-1} (four rows of R^{-1} per step: eight
// 16-byte loads per 64 FMAs); the Gram gives each thread a 4 x 4 tile of the
// upper triangle, several row groups per tile when there are fewer tiles
// than threads.  Columns k .. kp-1 of the panels are zero (the plan clears
// them once).  Entries below the diagonal of the partial are left unwritten.
// A wait for a block is bounded; on expiry the kernel raises kStatusTimeout.
__global__ void __launch_bounds__(GTHREADS, 2)
panel_gram_kernel(int kp, const PanelDev* __restrict__ panels, const int2* __restrict__ chunks,
                  const float* __restrict__ rinv, float* __restrict__ partial,
                  int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int2 ch = chunks[blockIdx.x];
  const PanelDev pd = panels[ch.x];
  const int k = pd.k;
  const bool tr = (rinv != nullptr);
  const int ldp = kp + 4, blk = GSUB * kp;
  float* Ps = (float*)smem_raw;  // GSTAGES blocks, rows of kp floats
  float* Ts = Ps + max(GSTAGES * blk, GTHREADS * 16);
  float* Rs = Ts + GSUB * ldp;
  uint64_t* bars = (uint64_t*)(Rs + kp * kp);
  const float* P = (const float*)pd.P;
  const int tid = threadIdx.x;
  const long long r0 = (long long)ch.y * GCHUNK;
  const long long r1 = min(pd.rows, r0 + GCHUNK);
  const int nblk = (int)((r1 - r0 + GSUB - 1) / GSUB);
  auto bar = [&](int s) { return (uint32_t)__cvta_generic_to_shared(bars + s); };
  auto issue = [&](int b) {  // thread 0: block b into stage b % GSTAGES
    const int s = b % GSTAGES;
    const long long s0 = r0 + (long long)b * GSUB;
    const uint32_t bytes = (uint32_t)(min((long long)GSUB, r1 - s0) * kp * sizeof(float));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(s)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"((uint32_t)__cvta_generic_to_shared(Ps + s * blk)),
        "l"(P + s0 * pd.ld), "r"(bytes), "r"(bar(s))
        : "memory");
  };
  if (tid == 0) {
    for (int s = 0; s < GSTAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar(s)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0)
    for (int b = 0; b < min(GSTAGES - 1, nblk); ++b) issue(b);
  if (tr)
    for (int e = tid; e < kp * kp; e += GTHREADS) Rs[e] = rinv[(long long)ch.x * kp * kp + e];
  __syncthreads();  // R^{-1} in place before the first transform
  const int nt = kp / 4;
  const int ntiles = nt * (nt + 1) / 2;
  const int groups = max(1, GTHREADS / ntiles);
  const bool active = tid < groups * ntiles;
  const int tile = tid % ntiles, grp = tid / ntiles;
  int ty = 0, rem = tile;  // tile -> (ty, tx) with ty <= tx
  while (rem >= nt - ty) {
    rem -= nt - ty;
    ++ty;
  }
  const int tx = ty + rem;
  // transform tile of this thread: rows 4 rg .. 4 rg + 3, columns 4 cg .. 4 cg + 3
  const int rg = tid / nt, cg = tid % nt;
  const bool tact = tr && rg < GSUB / 4;
  const int top = min((k + 3) & ~3, 4 * cg + 4);  // R^{-1} is upper: rows < top
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2) acc[a][b2] = 0.f;
  bool ok = true;
  for (int b = 0; b < nblk; ++b) {
    const int s = b % GSTAGES;
    if (tid == 0 && ok && b + GSTAGES - 1 < nblk) issue(b + GSTAGES - 1);  // stage freed
    if (ok) {  // wait for block b (bounded)
      const uint32_t parity = (uint32_t)((b / GSTAGES) & 1);
      uint32_t done = 0;
      const uint64_t t0 = gtimer();
      for (;;) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar(s)), "r"(parity)
            : "memory");
        if (done) break;
        if ((long long)(gtimer() - t0) > GWAIT_NS) {
          atomicOr(status, kStatusTimeout);
          ok = false;
          break;
        }
      }
    }
    const float* Pb = Ps + s * blk;
    const int nrows = (int)min((long long)GSUB, r1 - r0 - (long long)b * GSUB);
    const float* src = Pb;
    int lds = kp;
    if (tr) {
      // Ts = Pb R^{-1}, four rows of R^{-1} per step
      if (tact) {
        float t[4][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b2 = 0; b2 < 4; ++b2) t[a][b2] = 0.f;
        for (int cc = 0; cc < top; cc += 4) {
          float pv[4][4], rv[4][4];
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const float4 p4 = *reinterpret_cast<const float4*>(Pb + (4 * rg + a) * kp + cc);
            pv[a][0] = p4.x;
            pv[a][1] = p4.y;
            pv[a][2] = p4.z;
            pv[a][3] = p4.w;
            const float4 r4 = *reinterpret_cast<const float4*>(Rs + (cc + a) * kp + 4 * cg);
            rv[a][0] = r4.x;
            rv[a][1] = r4.y;
            rv[a][2] = r4.z;
            rv[a][3] = r4.w;
          }
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
              for (int b2 = 0; b2 < 4; ++b2) t[a][b2] = fmaf(pv[a][q], rv[q][b2], t[a][b2]);
        }
#pragma unroll
        for (int a = 0; a < 4; ++a)
          *reinterpret_cast<float4*>(Ts + (4 * rg + a) * ldp + 4 * cg) =
              make_float4(t[a][0], t[a][1], t[a][2], t[a][3]);
      }
      __syncthreads();
      src = Ts;
      lds = ldp;
    }
    if (active) {
#pragma unroll 4
      for (int ii = grp; ii < nrows; ii += groups) {
        const float4 x4 = *reinterpret_cast<const float4*>(src + ii * lds + ty * 4);
        const float4 y4 = *reinterpret_cast<const float4*>(src + ii * lds + tx * 4);
        const float x[4] = {x4.x, x4.y, x4.z, x4.w};
        const float y[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b2 = 0; b2 < 4; ++b2) acc[a][b2] = fmaf(x[a], y[b2], acc[a][b2]);
      }
    }
    __syncthreads();  // stage s and Ts consumed: stage s may be refilled
  }
  // sum the row groups (the stages are free now; every issued copy landed)
  float* Red = Ps;
  if (active && grp > 0) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) Red[(tid - ntiles) * 16 + a * 4 + b2] = acc[a][b2];
  }
  __syncthreads();
  if (active && grp == 0) {
    for (int g2 = 1; g2 < groups; ++g2) {
      const int t2 = (g2 - 1) * ntiles + tile;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) acc[a][b2] += Red[t2 * 16 + a * 4 + b2];
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

// eig_finish_kernel: each matrix slot has 2 ks threads (ks = the largest k of
// the batch, <= EIG_KMAX), two per column; a CTA holds max(1, 128 / (2 ks))
// slots.
constexpr int EIG_KMAX = 48;
// Shared memory of one matrix slot: G and two buffers of B columns
// (ks x (ks + 1) floats each), eigenvalues, their order and the slot's
// energy parts.
__host__ __device__ constexpr size_t eig_slot_bytes(int ks) {
  return (size_t)3 * ks * (ks + 1) * sizeof(float) + (size_t)ks * (sizeof(float) + sizeof(int)) +
         (size_t)2 * ks * sizeof(double);
}
__host__ __device__ constexpr size_t eig_slot_stride(int ks) {  // 16-byte multiple
  return (eig_slot_bytes(ks) + 15) / 16 * 16;
}

// Partner of column j in round `round` of the round-robin order on kk = 2 m'
// columns (mm = kk - 1): the pairs of a round are (round, mm) and
// (round + i, round - i) mod mm, i = 1 .. kk/2 - 1, so two columns other than
// mm pair up when their indices sum to 2 round mod mm.
__device__ __forceinline__ int rr_partner(int round, int j, int mm) {
  const int r0 = round % mm;
  if (j == mm) return r0;
  if (j == r0) return mm;
  return ((2 * round - j) % mm + mm) % mm;
}

// G_M = sum of its FP32 partial Grams; eigenpairs of the symmetric positive
// semidefinite G_M by one-sided (Hestenes) Jacobi on B = G_M: rotations that
// make the columns of B mutually orthogonal leave B = G_M V = V Lambda, so
// the column norms are the eigenvalues and the normalised columns the
// eigenvectors (whose errors reach the captured energy, a Rayleigh quotient,
// only at second order).  Two adjacent threads keep the two halves of
// column j of B in registers (HMAX >= ceil(k / 2) rows each); each round of
// the parallel round-robin order they read their halves of the partner
// column from shared memory (double-buffered, one barrier per round), add
// their partial dot products with one shuffle, and all four threads of a
// pair of columns compute the same rotation from the same three sums.  Then
// V_r is brought back to orthonormal with one step V <- V (I - (V^T V - I) / 2);
// the captured energy tr(V_r^T G_M V_r) (Ky Fan: sum_{i<=r} lambda_i up to
// second-order terms) gives err^2 = ||A||^2 - energy; sigma = sqrt(lambda)
// and W = R_X^{-1} V_r.  Arithmetic is FP32 (the partial Grams are FP32
// sums already); the energy's per-thread parts are added in FP64.
template <int HMAX>
__global__ void __launch_bounds__(128, 4)
eig_finish_kernel(int kp, int ks, int count, const MatDev* __restrict__ mats,
                  const int* __restrict__ chunk_off, const float* __restrict__ partial,
                  const float* __restrict__ rinv, float* __restrict__ Wm,
                  const double* __restrict__ normA2, double* __restrict__ err,
                  int* __restrict__ flags, int err_mode, double tau) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const unsigned full = 0xffffffffu;
  const int tid = threadIdx.x, per = 2 * ks;
  const int mpc = max(1, 128 / per);
  const int slot = tid / per, q = tid % per;  // q: thread within the slot
  const int j = q >> 1, half = q & 1;         // column j, rows of this half
  const int b = blockIdx.x * mpc + slot;
  const bool live = slot < mpc && b < count;
  const int ld = ks + 1, plane = ks * ld;
  unsigned char* base = smem_raw + (size_t)min(slot, mpc - 1) * eig_slot_stride(ks);
  float* Gs = (float*)base;            // G_M, row-major
  float* Bs = Gs + plane;              // 2 planes: column j at Bs[buf * plane + j * ld]
  float* lam = Bs + 2 * plane;         // ks
  int* order = (int*)(lam + ks);       // ks
  double* acc = (double*)(base + ((size_t)3 * plane * sizeof(float) +
                                  (size_t)ks * (sizeof(float) + sizeof(int)) + 7) / 8 * 8);
  MatDev md;
  int k = 0, r = 0;
  if (live) {
    md = mats[b];
    k = md.k;
    r = md.r;
    const int c0 = chunk_off[b], c1 = chunk_off[b + 1];
    for (int e = q; e < k * k; e += per) {
      const int i = e / k, c = e - i * k;
      const int a = min(i, c), bb = max(i, c);  // partials hold the upper triangle
      float g = 0.f;
      for (int t = c0; t < c1; ++t) g += partial[(long long)t * kp * kp + a * kp + bb];
      Gs[i * ld + c] = g;
    }
  }
  __syncthreads();
  const int hr = (k + 1) >> 1;          // rows per half
  const int r0h = half * hr;            // first row of this half
  const int nh = max(0, min(hr, k - r0h));  // rows of this half
  float bc[HMAX];
#pragma unroll
  for (int i = 0; i < HMAX; ++i) bc[i] = (j < k && i < nh) ? Gs[(r0h + i) * ld + j] : 0.f;
  const int kk = k + (k & 1), mm = kk - 1;
  const int rounds = ks + (ks & 1) - 1;  // of the largest k in the CTA
  int t = 0;                             // rounds so far: selects the buffer
  for (int sweep = 0; sweep < 12; ++sweep) {
    int rot = 0;
    for (int round = 0; round < rounds; ++round, ++t) {
      float* Bb = Bs + (t & 1) * plane;
      if (j < k && round < mm) {
#pragma unroll
        for (int i = 0; i < HMAX; ++i)
          if (i < nh) Bb[j * ld + r0h + i] = bc[i];
      }
      __syncthreads();
      const int pj = (j < k && round < mm) ? rr_partner(round, j, mm) : k;
      if (pj < k) {  // both threads of the column take this branch together
        const float* pb = Bb + pj * ld + r0h;
        float y[HMAX];
        float aa = 0.f, pp = 0.f, ap = 0.f;
#pragma unroll
        for (int i = 0; i < HMAX; ++i) {
          y[i] = (i < nh) ? pb[i] : 0.f;
          aa = fmaf(bc[i], bc[i], aa);
          pp = fmaf(y[i], y[i], pp);
          ap = fmaf(bc[i], y[i], ap);
        }
        const unsigned m2 = 3u << (threadIdx.x & 30);  // this column's two lanes
        aa += __shfl_xor_sync(m2, aa, 1);
        pp += __shfl_xor_sync(m2, pp, 1);
        ap += __shfl_xor_sync(m2, ap, 1);
        const bool low = j < pj;  // the lower index is p of the pair (p, q)
        const float alpha = low ? aa : pp, beta = low ? pp : aa, gamma = ap;
        if (fabsf(gamma) > 4.0e-6f * sqrtf(alpha * beta) && fabsf(gamma) > 1.0e-30f) {
          const float zeta = (beta - alpha) / (2.f * gamma);
          const float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + sqrtf(1.f + zeta * zeta));
          const float c = 1.f / sqrtf(1.f + tt * tt), sn = tt * c;
          // [b_p b_q] <- [c b_p - s b_q, s b_p + c b_q]
          const float cp = low ? -sn : sn;
#pragma unroll
          for (int i = 0; i < HMAX; ++i) bc[i] = fmaf(c, bc[i], cp * y[i]);
          rot = 1;
        }
      }
    }
    if (!__syncthreads_or(rot)) break;
  }
  (void)full;
  // eigenvalues = column norms; normalised columns = eigenvectors (plane 0)
  float* Vs = Bs;           // column j at Vs[j * ld + i]
  float* Vc = Bs + plane;   // corrected V_r, column c at Vc[c * ld + i]
  {
    float nn = 0.f;
#pragma unroll
    for (int i = 0; i < HMAX; ++i) nn = fmaf(bc[i], bc[i], nn);
    nn += __shfl_xor_sync(0xffffffffu, nn, 1);
    if (j < k) {
      const float l = sqrtf(nn);
      if (half == 0) lam[j] = l;
      const float inv = l > 1.0e-30f ? 1.f / l : 0.f;
#pragma unroll
      for (int i = 0; i < HMAX; ++i)
        if (i < nh) Vs[j * ld + r0h + i] = (inv > 0.f) ? bc[i] * inv : (r0h + i == j ? 1.f : 0.f);
    }
  }
  __syncthreads();
  for (int c = q; c < k; c += per) {  // descending eigenvalues
    int rank = 0;
    for (int c2 = 0; c2 < k; ++c2) rank += (lam[c2] > lam[c]) || (lam[c2] == lam[c] && c2 < c);
    order[rank] = c;
  }
  __syncthreads();
  if (live && md.sigma != nullptr)
    for (int c = q; c < k; c += per) ((float*)md.sigma)[c] = sqrtf(lam[order[c]]);
  // column c < r of V_r (E = V_r^T V_r - I, then V_r <- V_r - V_r E / 2)
  for (int c = q; c < r; c += per) {
    const float* vc = Vs + order[c] * ld;
    float e[EIG_KMAX];
#pragma unroll
    for (int a = 0; a < EIG_KMAX; ++a) {
      float s2 = 0.f;
      if (a < r) {
        const float* va = Vs + order[a] * ld;
        s2 = (a == c) ? -1.f : 0.f;
        for (int i = 0; i < k; ++i) s2 = fmaf(va[i], vc[i], s2);
      }
      e[a] = s2;
    }
    for (int i = 0; i < k; ++i) {
      float s2 = 0.f;
#pragma unroll
      for (int a = 0; a < EIG_KMAX; ++a)
        if (a < r) s2 = fmaf(Vs[order[a] * ld + i], e[a], s2);
      Vc[c * ld + i] = fmaf(-0.5f, s2, vc[i]);
    }
  }
  __syncthreads();
  // row i of G V_r and of W = R_X^{-1} V_r; energy tr(V_r^T G V_r)
  double part = 0.0;
  if (live) {
    const float* Ri = rinv + (long long)b * kp * kp;
    float* Wout = Wm + (long long)b * kp * kp;
    for (int i = q; i < kp; i += per) {
      for (int c = 0; c < kp; ++c) {
        float w = 0.f;
        if (i < k && c < r) {
          const float* v = Vc + c * ld;
          float gv = 0.f;
          for (int qq = 0; qq < k; ++qq) gv = fmaf(Gs[i * ld + qq], v[qq], gv);
          part += (double)v[i] * (double)gv;
          for (int qq = i; qq < k; ++qq) w = fmaf(Ri[i * kp + qq], v[qq], w);  // R_X^{-1} upper
        }
        Wout[i * kp + c] = w;
      }
    }
  }
  if (slot < mpc) acc[q] = part;
  __syncthreads();
  if (live && q == 0) {
    double energy = 0.0;
    for (int qq = 0; qq < per; ++qq) energy += acc[qq];
    const double tot = normA2[b];
    const double e2 = tot - energy;
    err[b] = sqrt(e2 > 0.0 ? e2 : 0.0);
    flags[b] = (err_mode == 2) || (err_mode == 0 && e2 < tau * tot);
  }
}

// Launch shape of eig_finish_kernel for the largest k of a batch.
struct EigShape {
  int ks, mpc, threads;
  size_t smem;
};
EigShape eig_shape(int kmax) {
  EigShape e;
  e.ks = std::max(1, std::min(kmax, EIG_KMAX));
  const int per = 2 * e.ks;
  e.mpc = std::max(1, 128 / per);
  e.threads = (e.mpc * per + 31) / 32 * 32;
  e.smem = (size_t)e.mpc * eig_slot_stride(e.ks);
  return e;
}

template <int HMAX>
cudaError_t launch_eig_finish(const EigShape& es, int kp, int count, const MatDev* mats,
                              const int* yoff, const float* partial_y, const float* rinv,
                              float* Wm, double* normA2, double* err, int* flags, int err_mode,
                              double tau, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(eig_finish_kernel<HMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)es.smem);
  if (e != cudaSuccess) return e;
  eig_finish_kernel<HMAX><<<(count + es.mpc - 1) / es.mpc, es.threads, es.smem, s>>>(
      kp, es.ks, count, mats, yoff, partial_y, rinv, Wm, normA2, err, flags, err_mode, tau);
  return cudaGetLastError();
}

cudaError_t launch_gram_route(int kp, int kmax, const MatDev* mats, int count,
                              const PanelDev* xpanels,
                              const PanelDev* ypanels, const int2* xchunks, int nxc,
                              const int* xoff, const int2* ychunks, int nyc, const int* yoff,
                              float* partial_x, float* partial_y, float* r1, float* r2,
                              float* rinv, float* Wm, double* normA2, double* err, int* flags,
                              int err_mode, double tau, int refine, int* status,
                              cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const size_t gsm = panel_gram_smem(kp);
  const size_t csm = (size_t)3 * kp * (kp + 1) * sizeof(float);
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(chol_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(panel_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)gsm);
  if (e != cudaSuccess) return e;
  // R1 = chol(X^T X)
  panel_gram_kernel<<<nxc, GTHREADS, gsm, s>>>(kp, xpanels, xchunks, nullptr, partial_x,
                                                status);
  chol_kernel<<<count, 256, csm, s>>>(kp, mats, xoff, partial_x, nullptr, r1, rinv, status);
  if (refine) {
    // R = chol(Q1^T Q1) R1 with Q1 = X R1^{-1}
    panel_gram_kernel<<<nxc, GTHREADS, gsm, s>>>(kp, xpanels, xchunks, rinv, partial_x,
                                                  status);
    chol_kernel<<<count, 256, csm, s>>>(kp, mats, xoff, partial_x, r1, r2, rinv, status);
  }
  // G_M = (Y R^{-1})^T (Y R^{-1})
  panel_gram_kernel<<<nyc, GTHREADS, gsm, s>>>(kp, ypanels, ychunks, rinv, partial_y,
                                                status);
  const EigShape es = eig_shape(kmax);
  const int hm = (es.ks + 1) / 2;
  if (hm <= 4)
    return launch_eig_finish<4>(es, kp, count, mats, yoff, partial_y, rinv, Wm, normA2, err,
                                flags, err_mode, tau, s);
  if (hm <= 8)
    return launch_eig_finish<8>(es, kp, count, mats, yoff, partial_y, rinv, Wm, normA2, err,
                                flags, err_mode, tau, s);
  if (hm <= 12)
    return launch_eig_finish<12>(es, kp, count, mats, yoff, partial_y, rinv, Wm, normA2, err,
                                 flags, err_mode, tau, s);
  if (hm <= 16)
    return launch_eig_finish<16>(es, kp, count, mats, yoff, partial_y, rinv, Wm, normA2, err,
                                 flags, err_mode, tau, s);
  if (hm <= 20)
    return launch_eig_finish<20>(es, kp, count, mats, yoff, partial_y, rinv, Wm, normA2, err,
                                 flags, err_mode, tau, s);
  return launch_eig_finish<24>(es, kp, count, mats, yoff, partial_y, rinv, Wm, normA2, err, flags,
                               err_mode, tau, s);
}

int gram_route_chunks(long long rows) { return (int)((rows + GCHUNK - 1) / GCHUNK); }

}  // namespace tsk
