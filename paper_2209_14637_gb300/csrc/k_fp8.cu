// FP8 (E4M3) copies of training matrices for the tensor-core Gram (T1).
//
// E4M3 keeps 3 mantissa bits and a largest finite value of 448.  Each row of
// a group of eight consecutive training matrices (the matrices the Gram
// kernel sums in one accumulator before it goes to G) gets one power-of-two
// scale s: for t = max |A_d[i, :]| over the group, the smallest s >= 2^-149
// (FP32's smallest positive value) with t <= 448 s, and s = 1 where t = 0.
// The stored byte is E4M3(A_d[i, j] / s), rounded to nearest even; the
// quotient is exact (a power-of-two scaling that stays in FP32's range).
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

__device__ __forceinline__ float e4m3_in(float x) { return x; }
__device__ __forceinline__ float e4m3_in(__nv_bfloat16 x) { return __bfloat162float(x); }

// V consecutive inputs from one 16-byte load (V = 8 BF16 or 4 FP32) kept as
// raw words, or one scalar (V = 1, converted at once), and their FP32 values.
template <typename Tin, int V>
struct E4m3Raw {
  uint4 u;
};
template <typename Tin, int V>
__device__ __forceinline__ E4m3Raw<Tin, V> e4m3_load(const Tin* p) {
  E4m3Raw<Tin, V> r;
  if constexpr (V == 1)
    r.u.x = __float_as_uint(e4m3_in(p[0]));
  else
    r.u = *reinterpret_cast<const uint4*>(p);
  return r;
}
template <typename Tin, int V>
__device__ __forceinline__ void e4m3_unpack(const E4m3Raw<Tin, V>& r, float (&v)[V]) {
  if constexpr (V == 1) {
    v[0] = __uint_as_float(r.u.x);
  } else if constexpr (sizeof(Tin) == 4) {
    v[0] = __uint_as_float(r.u.x);
    v[1] = __uint_as_float(r.u.y);
    v[2] = __uint_as_float(r.u.z);
    v[3] = __uint_as_float(r.u.w);
  } else {  // BF16 -> FP32 is a 16-bit shift, exact
    const uint32_t w[4] = {r.u.x, r.u.y, r.u.z, r.u.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      v[2 * q] = __uint_as_float(w[q] << 16);
      v[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
    }
  }
}

__device__ __forceinline__ uint32_t e4m3_byte(float x) {
  return (uint32_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}

// x / s as x * inv.x * inv.y: 1 / s alone overflows FP32 for s < 2^-127,
// so there the reciprocal is split into two powers of two; every product is
// then exact (no intermediate leaves FP32's normal range).
__device__ __forceinline__ uint32_t e4m3_q(float x, float2 inv) {
  return e4m3_byte(x * inv.x * inv.y);
}

template <int V>
__device__ __forceinline__ void e4m3_store(unsigned char* out, const float (&x)[V], float2 inv) {
  if constexpr (V == 8) {
    uint2 b;
    b.x = e4m3_q(x[0], inv) | e4m3_q(x[1], inv) << 8 | e4m3_q(x[2], inv) << 16 |
          e4m3_q(x[3], inv) << 24;
    b.y = e4m3_q(x[4], inv) | e4m3_q(x[5], inv) << 8 | e4m3_q(x[6], inv) << 16 |
          e4m3_q(x[7], inv) << 24;
    *reinterpret_cast<uint2*>(out) = b;
  } else if constexpr (V == 4) {
    *reinterpret_cast<uint32_t*>(out) = e4m3_q(x[0], inv) | e4m3_q(x[1], inv) << 8 |
                                        e4m3_q(x[2], inv) << 16 | e4m3_q(x[3], inv) << 24;
  } else {
    out[0] = (unsigned char)e4m3_q(x[0], inv);
  }
}

// One CTA per (row i, group g): the largest magnitude of row i over the
// group's matrices gives the scale, and the rows are then written as E4M3
// bytes.  Each thread loads its vector of all QG matrices at once (QG loads
// in flight); where a row is at most one vector per thread the values stay
// in registers between the two steps, otherwise they are read again (from
// L2: the CTA read them a moment before).  V inputs per load and V bytes
// per store where every row start is aligned for it (the host checks),
// scalars otherwise and for the last n mod V.
template <typename Tin, int V>
__global__ void __launch_bounds__(256)
e4m3_quant_kernel(const void* const* __restrict__ dA, long long D, long long m, long long n,
                  long long lda, unsigned char* const* __restrict__ dA8, long long ld8,
                  float* __restrict__ scales) {
  __shared__ float red[8];
  const long long i = blockIdx.x, g = blockIdx.y;
  const long long d0 = g * QG;
  const int nd = (int)min((long long)QG, D - d0);
  const long long nv = n / V;
  const Tin* rows[QG];
#pragma unroll
  for (int q = 0; q < QG; ++q) rows[q] = q < nd ? (const Tin*)dA[d0 + q] + i * lda : nullptr;
  const bool one = nv <= (long long)blockDim.x;  // at most one vector per thread and matrix
  E4m3Raw<Tin, V> keep[QG];
  float mx = 0.f;
  for (long long v = threadIdx.x; v < nv; v += blockDim.x) {
#pragma unroll
    for (int q = 0; q < QG; ++q) {
      if (q < nd) keep[q] = e4m3_load<Tin, V>(rows[q] + v * V);
    }
#pragma unroll
    for (int q = 0; q < QG; ++q) {
      if (q < nd) {
        float x[V];
        e4m3_unpack(keep[q], x);
#pragma unroll
        for (int e = 0; e < V; ++e) mx = fmaxf(mx, fabsf(x[e]));
      }
    }
  }
#pragma unroll
  for (int q = 0; q < QG; ++q)
    for (long long jj = nv * V + threadIdx.x; q < nd && jj < n; jj += blockDim.x)
      mx = fmaxf(mx, fabsf(e4m3_in(rows[q][jj])));
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < 8; ++w) t = fmaxf(t, red[w]);
  // s = 2^es: with t = f 2^e, f in [0.5, 1) (exact), and 448 = 0.875 * 2^9,
  // t <= 448 * 2^(e - 9) exactly when f <= 0.875, else 2^(e - 8) is the
  // smallest; a zero (or non-finite) maximum keeps s = 1
  int es = 0;
  if (t > 0.f && isfinite(t)) {
    int e = 0;
    const float f = frexpf(t, &e);
    es = f <= 0.875f ? e - 9 : e - 8;
    if (es < -149) es = -149;
  }
  const float s = ldexpf(1.f, es);
  if (threadIdx.x == 0) scales[g * m + i] = s;
  const float2 inv = es >= -126 ? make_float2(ldexpf(1.f, -es), 1.f)
                                : make_float2(ldexpf(1.f, 64), ldexpf(1.f, -es - 64));
  unsigned char* outs[QG];
#pragma unroll
  for (int q = 0; q < QG; ++q) outs[q] = q < nd ? dA8[d0 + q] + i * ld8 : nullptr;
  for (long long v = threadIdx.x; v < nv; v += blockDim.x) {
    if (!one) {
#pragma unroll
      for (int q = 0; q < QG; ++q) {
        if (q < nd) keep[q] = e4m3_load<Tin, V>(rows[q] + v * V);
      }
    }
#pragma unroll
    for (int q = 0; q < QG; ++q) {
      if (q < nd) {
        float x[V];
        e4m3_unpack(keep[q], x);
        e4m3_store<V>(outs[q] + v * V, x, inv);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < QG; ++q)
    for (long long jj = nv * V + threadIdx.x; q < nd && jj < n; jj += blockDim.x)
      outs[q][jj] = (unsigned char)e4m3_q(e4m3_in(rows[q][jj]), inv);
}

}  // namespace

cudaError_t launch_quantize_e4m3(int in_type, const void* const* dA, long long D, long long m,
                                 long long n, long long lda, unsigned char* const* dA8,
                                 long long ld8, float* scales, bool vec, cudaStream_t s) {
  if (D < 1 || m < 1 || n < 1) return cudaErrorInvalidValue;
  const long long groups = (D + QG - 1) / QG;
  if (m > 2147483647ll || groups > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)m, (unsigned)groups);
  if (in_type == 1) {
    if (vec)
      e4m3_quant_kernel<float, 4><<<grid, 256, 0, s>>>(dA, D, m, n, lda, dA8, ld8, scales);
    else
      e4m3_quant_kernel<float, 1><<<grid, 256, 0, s>>>(dA, D, m, n, lda, dA8, ld8, scales);
  } else if (in_type == 2) {
    if (vec)
      e4m3_quant_kernel<__nv_bfloat16, 8><<<grid, 256, 0, s>>>(dA, D, m, n, lda, dA8, ld8,
                                                                scales);
    else
      e4m3_quant_kernel<__nv_bfloat16, 1><<<grid, 256, 0, s>>>(dA, D, m, n, lda, dA8, ld8,
                                                                scales);
  } else {
    return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace tsk
