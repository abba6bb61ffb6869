// FP8 (E4M3) copies of training matrices for the tensor-core Gram (T1).
//
// E4M3 keeps 3 mantissa bits and a largest finite value of 448.  Each row of
// a group of eight consecutive training matrices (the matrices the Gram
// kernel sums in one TMEM accumulator before it flushes) gets one
// power-of-two scale s, the smallest with max |A_d[i, :]| / s <= 448 over
// the group; the stored byte is E4M3(A_d[i, j] / s), rounded to nearest.
// Since s is constant along a row and across the group,
//
//   sum_{d in group} A_d A_d^T  ~=  D_s (sum_{d in group} A8_d A8_d^T) D_s,
//
// D_s = diag(s), so the Gram kernel multiplies each flushed entry (i, j) by
// s_i s_j; powers of two make that product exact.
#include <cuda_fp8.h>

#include "tsk_internal.cuh"

namespace tsk {

namespace {

constexpr int QG = 8;  // matrices per scale group (the Gram kernel's flush group)

// One CTA per (row i, group g): the largest magnitude of row i over the
// group's matrices, and the scale it implies.
template <typename Tin>
__global__ void __launch_bounds__(256)
e4m3_scale_kernel(const void* const* __restrict__ dA, long long D, long long m, long long n,
                  long long lda, float* __restrict__ scales) {
  __shared__ float red[8];
  const long long i = blockIdx.x, g = blockIdx.y;
  float mx = 0.f;
  for (long long d = g * QG; d < D && d < (g + 1) * QG; ++d) {
    const Tin* row = (const Tin*)dA[d] + i * lda;
    for (long long j = threadIdx.x; j < n; j += blockDim.x) mx = fmaxf(mx, fabsf(to_float(row[j])));
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < 8; ++w) t = fmaxf(t, red[w]);
    float s = 1.f;
    if (t > 0.f && isfinite(t)) {
      int e = 0;
      frexpf(t / 448.f, &e);  // t / 448 < 2^e
      s = ldexpf(1.f, e);
    }
    scales[g * m + i] = s;
  }
}

// One CTA per (row i, matrix d): the row's E4M3 bytes.
template <typename Tin>
__global__ void __launch_bounds__(256)
e4m3_quant_kernel(const void* const* __restrict__ dA, long long m, long long n, long long lda,
                  unsigned char* const* __restrict__ dA8, long long ld8,
                  const float* __restrict__ scales) {
  const long long i = blockIdx.x, d = blockIdx.y;
  const float inv = 1.f / scales[(d / QG) * m + i];  // a power of two: exact
  const Tin* row = (const Tin*)dA[d] + i * lda;
  unsigned char* out = dA8[d] + i * ld8;
  for (long long j = threadIdx.x; j < n; j += blockDim.x)
    out[j] = (unsigned char)__nv_cvt_float_to_fp8(to_float(row[j]) * inv, __NV_SATFINITE,
                                                  __NV_E4M3);
}

}  // namespace

cudaError_t launch_quantize_e4m3(int in_type, const void* const* dA, long long D, long long m,
                                 long long n, long long lda, unsigned char* const* dA8,
                                 long long ld8, float* scales, cudaStream_t s) {
  if (D < 1 || m < 1 || n < 1) return cudaErrorInvalidValue;
  const long long groups = (D + QG - 1) / QG;
  if (m > 2147483647ll || groups > 65535 || D > 65535) return cudaErrorInvalidValue;
  const dim3 gs((unsigned)m, (unsigned)groups), gq((unsigned)m, (unsigned)D);
  if (in_type == 1) {
    e4m3_scale_kernel<float><<<gs, 256, 0, s>>>(dA, D, m, n, lda, scales);
    e4m3_quant_kernel<float><<<gq, 256, 0, s>>>(dA, m, n, lda, dA8, ld8, scales);
  } else if (in_type == 2) {
    e4m3_scale_kernel<__nv_bfloat16><<<gs, 256, 0, s>>>(dA, D, m, n, lda, scales);
    e4m3_quant_kernel<__nv_bfloat16><<<gq, 256, 0, s>>>(dA, m, n, lda, dA8, ld8, scales);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace tsk
