// Kernels of the learned sketch refiner S_theta = S_tensor + dS, trained on
// the IVY loss (Eq. 2.1) in its per-sample normalised form
//     L(S) = mean_A ||A - SCW(A, S, r)||_F^2 / ||A||_F^2.
//
// With X = (S A)^T = Q R, A Q = U Sigma V^T, Z = U_r Sigma_r = A Q V_r and
// W = R^{-1} V_r, the captured energy f = sum_{i<=r} sigma_i^2 has
//     df/dS = 2 W (A A^T Z - Z Sigma_r^2)^T            (k x m),
// so dL/dS = -(2 / ||A||^2) W (A A^T Z - Z Sigma_r^2)^T per sample.
// A A^T Z is one more pass over A with the sketch S' = Z^T (the same kernels
// as the forward sketch pass); the rest is small.
#include <cuda_bf16.h>

#include "tsk_internal.cuh"

namespace tsk {

// Zt (r x m, row-major) = (Y W)^T for every matrix of the batch; the
// backward pass uses it as its sketch.  blockIdx.x = matrix.
template <typename T>
__global__ void __launch_bounds__(256)
zt_kernel(int kp, const MatDev* __restrict__ mats, const T* __restrict__ Y,
          const T* __restrict__ Wm, T* __restrict__ Zt, long long zt_stride) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = (T*)smem_raw;
  const int b = blockIdx.x;
  const MatDev md = mats[b];
  const int k = md.k, r = md.r;
  const T* Wsrc = Wm + (long long)b * kp * kp;
  for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) Ws[e] = Wsrc[e];
  __syncthreads();
  T* out = Zt + (long long)b * zt_stride;
  for (long long i = (long long)blockIdx.y * blockDim.x + threadIdx.x; i < md.m;
       i += (long long)gridDim.y * blockDim.x) {
    const T* y = Y + md.offY + i * kp;
    for (int c = 0; c < r; ++c) {
      T a = T(0);
      for (int cc = 0; cc < k; ++cc) a += y[cc] * Ws[cc * kp + c];
      out[(long long)c * md.m + i] = a;
    }
  }
}

// grad[c'][i] = scale * sum_b coef_b * sum_{c<r} W_b[c'][c] *
//               (Y2_b[i][c] - Z_b[i][c] sigma_b[c]^2),   coef_b = -2/||A_b||^2
// (overwrites grad).  One thread per (c', i).
template <typename T>
__global__ void __launch_bounds__(256)
ivy_grad_kernel(int kp, int kp2, int count, const MatDev* __restrict__ mats,
                const MatDev* __restrict__ mats2, const T* __restrict__ Wm,
                const T* __restrict__ sig, const T* __restrict__ Zt,
                long long zt_stride, const T* __restrict__ Y2,
                const double* __restrict__ normA2, double scale, T* __restrict__ grad) {
  const MatDev m0 = mats[0];
  const long long m = m0.m;
  const int k = m0.k, r = m0.r;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)k * m) return;
  const int cp = (int)(e / m);
  const long long i = e % m;
  double acc = 0.0;
  for (int b = 0; b < count; ++b) {
    const T* W = Wm + (long long)b * kp * kp;
    const T* s = sig + (long long)b * kp;
    const T* z = Zt + (long long)b * zt_stride;
    const T* y2 = Y2 + mats2[b].offY + i * kp2;
    double t = 0.0;
    for (int c = 0; c < r; ++c) {
      const double sc = (double)s[c];
      t += (double)W[cp * kp + c] * ((double)y2[c] - (double)z[(long long)c * m + i] * sc * sc);
    }
    acc += (-2.0 / normA2[b]) * t;
  }
  grad[e] = (T)(scale * acc);
}

template <typename T>
__global__ void axpy_kernel(long long n, T alpha, const T* __restrict__ x, T* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += alpha * x[i];
}

template <typename T>
__global__ void add_kernel(long long n, const T* __restrict__ a, const T* __restrict__ b,
                           T* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] + b[i];
}

// loss = mean_b err_b^2 / ||A_b||^2  (one thread)
__global__ void batch_loss_kernel(int count, const double* __restrict__ err,
                                  const double* __restrict__ normA2, double* __restrict__ loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int b = 0; b < count; ++b) s += err[b] * err[b] / normA2[b];
  *loss = s / count;
}

cudaError_t launch_zt(bool dbl, int kp, const MatDev* mats, int count, const void* Y,
                      const void* Wm, void* Zt, long long zt_stride, cudaStream_t s) {
  const size_t sm = (size_t)kp * kp * (dbl ? 8 : 4);
  dim3 grid(count, 8);
  if (dbl)
    zt_kernel<double><<<grid, 256, sm, s>>>(kp, mats, (const double*)Y, (const double*)Wm,
                                            (double*)Zt, zt_stride);
  else
    zt_kernel<float><<<grid, 256, sm, s>>>(kp, mats, (const float*)Y, (const float*)Wm,
                                           (float*)Zt, zt_stride);
  return cudaGetLastError();
}

cudaError_t launch_ivy_grad(bool dbl, int kp, int kp2, int count, long long km,
                            const MatDev* mats, const MatDev* mats2, const void* Wm,
                            const void* sig, const void* Zt, long long zt_stride,
                            const void* Y2, const double* normA2, double scale, void* grad,
                            cudaStream_t s) {
  const unsigned blocks = (unsigned)((km + 255) / 256);
  if (dbl)
    ivy_grad_kernel<double><<<blocks, 256, 0, s>>>(
        kp, kp2, count, mats, mats2, (const double*)Wm, (const double*)sig,
        (const double*)Zt, zt_stride, (const double*)Y2, normA2, scale, (double*)grad);
  else
    ivy_grad_kernel<float><<<blocks, 256, 0, s>>>(
        kp, kp2, count, mats, mats2, (const float*)Wm, (const float*)sig,
        (const float*)Zt, zt_stride, (const float*)Y2, normA2, scale, (float*)grad);
  return cudaGetLastError();
}

cudaError_t launch_axpy(bool dbl, long long n, double alpha, const void* x, void* y,
                        cudaStream_t s) {
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (dbl)
    axpy_kernel<double><<<blocks, 256, 0, s>>>(n, alpha, (const double*)x, (double*)y);
  else
    axpy_kernel<float><<<blocks, 256, 0, s>>>(n, (float)alpha, (const float*)x, (float*)y);
  return cudaGetLastError();
}

cudaError_t launch_add(bool dbl, long long n, const void* a, const void* b, void* out,
                       cudaStream_t s) {
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (dbl)
    add_kernel<double><<<blocks, 256, 0, s>>>(n, (const double*)a, (const double*)b,
                                              (double*)out);
  else
    add_kernel<float><<<blocks, 256, 0, s>>>(n, (const float*)a, (const float*)b,
                                             (float*)out);
  return cudaGetLastError();
}

cudaError_t launch_batch_loss(int count, const double* err, const double* normA2,
                              double* loss, cudaStream_t s) {
  batch_loss_kernel<<<1, 32, 0, s>>>(count, err, normA2, loss);
  return cudaGetLastError();
}

}  // namespace tsk
