// CUDA-core (SIMT) kernels of the sketch pass, the Gram matrices, the
// eigensolver's dense steps and the direct error.
//
// These are the plain FP64 / FP32 paths of the method and the building
// blocks of the training side.  The BF16 test pass has its own tcgen05
// kernel (k_tc.cu); the stages after the sketch pass (k_small.cu) are
// shared by every path.
#include <cuda_bf16.h>
#include <stdio.h>

#include <algorithm>

#include "tsk_internal.cuh"

namespace tsk {

// in_type: 0 = double, 1 = float, 2 = bfloat16 (mirrors tsk_prec)

// ---------------------------------------------------------------------------
// E1: X = (S A)^T = A^T S^T  (n x k), Algorithm 1 line 1 / Algorithm 3 line 1.
// One CTA owns 64 columns of one matrix and walks down all m rows in chunks
// of 32, so X needs no cross-CTA reduction.  The same pass accumulates
// ||A||_F^2 (every element of A is read exactly once here), which the error
// identity of the proof of Theorem 1 (Eq. A.3) needs.
// ---------------------------------------------------------------------------
template <typename Tin, typename Tc, int KP>
__global__ void __launch_bounds__(256)
sketch_x_kernel(const MatDev* __restrict__ mats, const int2* __restrict__ items,
                Tc* __restrict__ X, double* __restrict__ normA2) {
  constexpr int BJ = 64, BI = 32, CPT = KP / 16;
  __shared__ __align__(16) Tc As[BI][BJ];
  __shared__ Tc Ss[BI][KP + 1];
  __shared__ double red[8];
  const int2 it = items[blockIdx.x];
  const MatDev md = mats[it.x];
  const Tin* __restrict__ A = (const Tin*)md.A;
  const Tc* __restrict__ S = (const Tc*)md.S;
  const long long m = md.m, n = md.n, lda = md.lda;
  const int k = md.k;
  const int tid = threadIdx.x, jg = tid & 15, cg = tid >> 4;
  const long long j0 = (long long)it.y * BJ;
  Tc acc[4][CPT];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < CPT; ++p) acc[q][p] = Tc(0);
  double sq = 0.0;
  for (long long i0 = 0; i0 < m; i0 += BI) {
    Tc part = Tc(0);
    for (int e = tid; e < BI * BJ; e += 256) {
      const int ii = e / BJ, jj = e % BJ;
      const long long i = i0 + ii, j = j0 + jj;
      Tc v = Tc(0);
      if (i < m && j < n) v = convert_in<Tc>(A[i * lda + j]);
      As[ii][jj] = v;
      part += v * v;
    }
    sq += (double)part;
    for (int e = tid; e < BI * KP; e += 256) {
      const int c = e / BI, ii = e % BI;
      const long long i = i0 + ii;
      Ss[ii][c] = (c < k && i < m) ? S[(long long)c * m + i] : Tc(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int ii = 0; ii < BI; ++ii) {
      Tc a[4], s[CPT];
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = As[ii][jg * 4 + q];
#pragma unroll
      for (int p = 0; p < CPT; ++p) s[p] = Ss[ii][cg * CPT + p];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < CPT; ++p) acc[q][p] += a[q] * s[p];
    }
    __syncthreads();
  }
  Tc* __restrict__ Xm = X + md.offX;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const long long j = j0 + jg * 4 + q;
    if (j < n) {
#pragma unroll
      for (int p = 0; p < CPT; ++p) Xm[j * KP + cg * CPT + p] = acc[q][p];
    }
  }
  sq = warp_sum(sq);
  if ((tid & 31) == 0) red[tid >> 5] = sq;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    atomicAdd(normA2 + it.x, t);
  }
}

// ---------------------------------------------------------------------------
// E3: Y = A X (m x k).  With X = A^T S^T this is A Q R, so A Q = Y R^{-1}
// (Algorithm 1 line 2 with the QR of Section 3.2).  One CTA owns 64 rows of
// one matrix and walks across all n columns.
// ---------------------------------------------------------------------------
template <typename Tin, typename Tc, int KP>
__global__ void __launch_bounds__(256)
sketch_y_kernel(const MatDev* __restrict__ mats, const int2* __restrict__ items,
                const Tc* __restrict__ X, Tc* __restrict__ Y) {
  constexpr int BI = 64, BJ = 32, CPT = KP / 16;
  __shared__ Tc AsT[BJ][BI + 1];
  __shared__ __align__(16) Tc Xs[BJ][KP];
  const int2 it = items[blockIdx.x];
  const MatDev md = mats[it.x];
  const Tin* __restrict__ A = (const Tin*)md.A;
  const long long m = md.m, n = md.n, lda = md.lda;
  const Tc* __restrict__ Xm = X + md.offX;
  const int tid = threadIdx.x, ig = tid & 15, cg = tid >> 4;
  const long long i0 = (long long)it.y * BI;
  Tc acc[4][CPT];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < CPT; ++p) acc[q][p] = Tc(0);
  for (long long j0 = 0; j0 < n; j0 += BJ) {
    for (int e = tid; e < BI * BJ; e += 256) {
      const int ii = e / BJ, jj = e % BJ;
      const long long i = i0 + ii, j = j0 + jj;
      AsT[jj][ii] = (i < m && j < n) ? convert_in<Tc>(A[i * lda + j]) : Tc(0);
    }
    for (int e = tid; e < BJ * KP; e += 256) {
      const int jj = e / KP, c = e % KP;
      const long long j = j0 + jj;
      Xs[jj][c] = (j < n) ? Xm[j * KP + c] : Tc(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int jj = 0; jj < BJ; ++jj) {
      Tc a[4], x[CPT];
#pragma unroll
      for (int q = 0; q < 4; ++q) a[q] = AsT[jj][ig * 4 + q];
#pragma unroll
      for (int p = 0; p < CPT; ++p) x[p] = Xs[jj][cg * CPT + p];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < CPT; ++p) acc[q][p] += a[q] * x[p];
    }
    __syncthreads();
  }
  Tc* __restrict__ Ym = Y + md.offY;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const long long i = i0 + ig * 4 + q;
    if (i < m) {
#pragma unroll
      for (int p = 0; p < CPT; ++p) Ym[i * KP + cg * CPT + p] = acc[q][p];
    }
  }
}

// ---------------------------------------------------------------------------
// The same two kernels for float compute (FP32 and BF16 inputs): 128 threads
// per 64-wide item, each thread an 8 x KP/16 register tile fed by two float4
// shared loads and KP/16 broadcast loads per step (24 FMAs per 5 loads at
// KP = 48, against 12 per 7 above), and float4 / 8-byte global loads of A
// where its rows allow them.
// ---------------------------------------------------------------------------
template <typename Tin>
__device__ __forceinline__ bool rows_vec_ok(const Tin* A, long long lda) {
  // a 4-element vector at any multiple of 4 columns stays aligned
  return (((uintptr_t)A) % (4 * sizeof(Tin)) == 0) && (lda % 4 == 0);
}
__device__ __forceinline__ void load4(const float* p, float* v) {
  const float4 w = *reinterpret_cast<const float4*>(p);
  v[0] = w.x;
  v[1] = w.y;
  v[2] = w.z;
  v[3] = w.w;
}
__device__ __forceinline__ void load4(const __nv_bfloat16* p, float* v) {
  const uint2 w = *reinterpret_cast<const uint2*>(p);
  v[0] = __uint_as_float(w.x << 16);
  v[1] = __uint_as_float(w.x & 0xFFFF0000u);
  v[2] = __uint_as_float(w.y << 16);
  v[3] = __uint_as_float(w.y & 0xFFFF0000u);
}

template <typename Tin, int KP>
__global__ void __launch_bounds__(128)
sketch_x_f32_kernel(const MatDev* __restrict__ mats, const int2* __restrict__ items,
                    float* __restrict__ X, double* __restrict__ normA2) {
  constexpr int BJ = 64, BI = 32, CPT = KP / 16, SQ = BI * KP / 128;
  __shared__ __align__(16) float As[2][BI][BJ];
  __shared__ float Ss[2][BI][KP + 1];  // rows padded: the transposing stores hit 32 banks
  __shared__ double red[4];
  const int2 it = items[blockIdx.x];
  const MatDev md = mats[it.x];
  const Tin* __restrict__ A = (const Tin*)md.A;
  const float* __restrict__ S = (const float*)md.S;
  const long long m = md.m, n = md.n, lda = md.lda;
  const int k = md.k;
  const int tid = threadIdx.x, jg = tid & 7, cg = tid >> 3;
  const long long j0 = (long long)it.y * BJ;
  const bool vec = rows_vec_ok(A, lda);
  float acc[8][CPT];
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int p = 0; p < CPT; ++p) acc[q][p] = 0.f;
  // the next chunk is fetched into registers while the current one is used
  float va[4][4], vs[SQ];
  auto fetch = [&](long long i0) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {  // 512 quads of the 32 x 64 chunk
      const int e4 = tid + 128 * t, ii = e4 >> 4, c4 = (e4 & 15) * 4;
      const long long i = i0 + ii, j = j0 + c4;
#pragma unroll
      for (int u = 0; u < 4; ++u) va[t][u] = 0.f;
      if (i < m) {
        if (vec && j + 3 < n) {
          load4(A + i * lda + j, va[t]);
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (j + u < n) va[t][u] = to_float(A[i * lda + j + u]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < SQ; ++q) {
      const int e = tid + 128 * q, c = e / BI, ii = e % BI;
      const long long i = i0 + ii;
      vs[q] = (c < k && i < m) ? S[(long long)c * m + i] : 0.f;
    }
  };
  double sq = 0.0;
  auto park = [&](int buf) {  // registers -> shared buffer, squares summed
    float part = 0.f;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e4 = tid + 128 * t, ii = e4 >> 4, c4 = (e4 & 15) * 4;
#pragma unroll
      for (int u = 0; u < 4; ++u) part = fmaf(va[t][u], va[t][u], part);
      *reinterpret_cast<float4*>(&As[buf][ii][c4]) =
          make_float4(va[t][0], va[t][1], va[t][2], va[t][3]);
    }
    sq += (double)part;
#pragma unroll
    for (int q = 0; q < SQ; ++q) {
      const int e = tid + 128 * q;
      Ss[buf][e % BI][e / BI] = vs[q];
    }
  };
  const int nch = (int)((m + BI - 1) / BI);
  fetch(0);
  park(0);
  __syncthreads();
  for (int ch = 0; ch < nch; ++ch) {
    const int cur = ch & 1;
    if (ch + 1 < nch) fetch((long long)(ch + 1) * BI);
#pragma unroll 4
    for (int ii = 0; ii < BI; ++ii) {
      // columns jg*4 .. +3 and 32 + jg*4 .. +3: the eight threads of a
      // quarter-warp read 128 consecutive bytes, one per bank group
      float a[8], sv[CPT];
      const float4 a0 = *reinterpret_cast<const float4*>(&As[cur][ii][jg * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[cur][ii][32 + jg * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
#pragma unroll
      for (int p = 0; p < CPT; ++p) sv[p] = Ss[cur][ii][cg * CPT + p];
#pragma unroll
      for (int q = 0; q < 8; q += 2)
#pragma unroll
        for (int p = 0; p < CPT; ++p)
          ffma2(acc[q][p], acc[q + 1][p], a[q], a[q + 1], sv[p], sv[p]);
    }
    // the other buffer was last read in the previous chunk, before its barrier
    if (ch + 1 < nch) park(cur ^ 1);
    __syncthreads();
  }
  float* __restrict__ Xm = X + md.offX;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const long long j = j0 + (q < 4 ? jg * 4 + q : 32 + jg * 4 + q - 4);
    if (j < n) {
#pragma unroll
      for (int p = 0; p < CPT; ++p) Xm[j * KP + cg * CPT + p] = acc[q][p];
    }
  }
  sq = warp_sum(sq);
  if ((tid & 31) == 0) red[tid >> 5] = sq;
  __syncthreads();
  if (tid == 0) atomicAdd(normA2 + it.x, (red[0] + red[1]) + (red[2] + red[3]));
}

template <typename Tin, int KP>
__global__ void __launch_bounds__(128)
sketch_y_f32_kernel(const MatDev* __restrict__ mats, const int2* __restrict__ items,
                    const float* __restrict__ X, float* __restrict__ Y) {
  constexpr int BI = 64, BJ = 32, CPT = KP / 16, XQ = BJ * KP / 4 / 128;
  // A transposed: row jj holds the 64 rows ii of column jj as 16 float4
  // slots, slot ii / 4 stored at slot (ii / 4) ^ ((jj / 4) & 7), so that the
  // transposing stores and the float4 reads are both free of bank conflicts
  __shared__ __align__(16) float AsT[2][BJ][BI];
  __shared__ __align__(16) float Xs[2][BJ][KP];
  const int2 it = items[blockIdx.x];
  const MatDev md = mats[it.x];
  const Tin* __restrict__ A = (const Tin*)md.A;
  const long long m = md.m, n = md.n, lda = md.lda;
  const float* __restrict__ Xm = X + md.offX;
  const int tid = threadIdx.x, ig = tid & 7, cg = tid >> 3;
  const long long i0 = (long long)it.y * BI;
  const bool vec = rows_vec_ok(A, lda);
  float acc[8][CPT];
#pragma unroll
  for (int q = 0; q < 8; ++q)
#pragma unroll
    for (int p = 0; p < CPT; ++p) acc[q][p] = 0.f;
  float va[4][4];
  float4 vx[XQ];
  auto fetch = [&](long long j0) {
#pragma unroll
    for (int t = 0; t < 4; ++t) {  // 512 quads of the 64 x 32 chunk
      const int e4 = tid + 128 * t, ii = e4 >> 3, c4 = (e4 & 7) * 4;
      const long long i = i0 + ii, j = j0 + c4;
#pragma unroll
      for (int u = 0; u < 4; ++u) va[t][u] = 0.f;
      if (i < m) {
        if (vec && j + 3 < n) {
          load4(A + i * lda + j, va[t]);
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (j + u < n) va[t][u] = to_float(A[i * lda + j + u]);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < XQ; ++q) {  // X rows are KP floats, 16-byte aligned
      const int e = tid + 128 * q, jj = e / (KP / 4), c4 = (e % (KP / 4)) * 4;
      const long long j = j0 + jj;
      vx[q] = j < n ? *reinterpret_cast<const float4*>(Xm + j * KP + c4)
                    : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto park = [&](int buf) {  // registers -> shared buffer, A transposed
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int e4 = tid + 128 * t, ii = e4 >> 3, c4 = (e4 & 7) * 4;
      const int slot = ((ii >> 2) ^ (e4 & 7)) * 4 + (ii & 3);  // (c4 + u) / 4 = e4 & 7
#pragma unroll
      for (int u = 0; u < 4; ++u) AsT[buf][c4 + u][slot] = va[t][u];
    }
#pragma unroll
    for (int q = 0; q < XQ; ++q) {
      const int e = tid + 128 * q, jj = e / (KP / 4), c4 = (e % (KP / 4)) * 4;
      *reinterpret_cast<float4*>(&Xs[buf][jj][c4]) = vx[q];
    }
  };
  const int nch = (int)((n + BJ - 1) / BJ);
  fetch(0);
  park(0);
  __syncthreads();
  for (int ch = 0; ch < nch; ++ch) {
    const int cur = ch & 1;
    if (ch + 1 < nch) fetch((long long)(ch + 1) * BJ);
#pragma unroll 4
    for (int jj = 0; jj < BJ; ++jj) {
      // rows ig*4 .. +3 (slot ig) and 32 + ig*4 .. +3 (slot 8 + ig)
      const int h = (jj >> 2) & 7;
      float a[8], xv[CPT];
      const float4 a0 = *reinterpret_cast<const float4*>(&AsT[cur][jj][(ig ^ h) * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&AsT[cur][jj][(8 + (ig ^ h)) * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
#pragma unroll
      for (int p = 0; p < CPT; ++p) xv[p] = Xs[cur][jj][cg * CPT + p];
#pragma unroll
      for (int q = 0; q < 8; q += 2)
#pragma unroll
        for (int p = 0; p < CPT; ++p)
          ffma2(acc[q][p], acc[q + 1][p], a[q], a[q + 1], xv[p], xv[p]);
    }
    if (ch + 1 < nch) park(cur ^ 1);
    __syncthreads();
  }
  float* __restrict__ Ym = Y + md.offY;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const long long i = i0 + (q < 4 ? ig * 4 + q : 32 + ig * 4 + q - 4);
    if (i < m) {
#pragma unroll
      for (int p = 0; p < CPT; ++p) Ym[i * KP + cg * CPT + p] = acc[q][p];
    }
  }
}

template <typename Tin, typename Tc>
static cudaError_t sketch_dispatch_kp(int kp, const MatDev* mats,
                                      const int2* items, int nitems, void* X,
                                      double* normA2, const void* Xin, void* Y,
                                      bool is_x, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if constexpr (sizeof(Tc) == 4) {  // float compute: the 8 x KP/16 register-tile kernels
#define TSK_SK4(KPV)                                                                   \
  case KPV:                                                                            \
    if (is_x)                                                                          \
      sketch_x_f32_kernel<Tin, KPV><<<nitems, 128, 0, s>>>(mats, items, (float*)X,     \
                                                            normA2);                   \
    else                                                                               \
      sketch_y_f32_kernel<Tin, KPV><<<nitems, 128, 0, s>>>(mats, items,               \
                                                            (const float*)Xin,         \
                                                            (float*)Y);                \
    break;
    switch (kp) {
      TSK_SK4(16)
      TSK_SK4(32)
      TSK_SK4(48)
      TSK_SK4(64)
      default:
        return cudaErrorInvalidValue;
    }
#undef TSK_SK4
    return cudaGetLastError();
  }
#define TSK_SK(KPV)                                                        \
  case KPV:                                                                \
    if (is_x)                                                              \
      sketch_x_kernel<Tin, Tc, KPV>                                        \
          <<<nitems, 256, 0, s>>>(mats, items, (Tc*)X, normA2);            \
    else                                                                   \
      sketch_y_kernel<Tin, Tc, KPV>                                        \
          <<<nitems, 256, 0, s>>>(mats, items, (const Tc*)Xin, (Tc*)Y);    \
    break;
  switch (kp) {
    TSK_SK(16)
    TSK_SK(32)
    TSK_SK(48)
    TSK_SK(64)
    default:
      return cudaErrorInvalidValue;
  }
#undef TSK_SK
  return cudaGetLastError();
}

cudaError_t launch_sketch_x(int in_type, int kp, const MatDev* mats,
                            const int2* items, int nitems, void* X,
                            double* normA2, cudaStream_t s) {
  switch (in_type) {
    case 0:
      return sketch_dispatch_kp<double, double>(kp, mats, items, nitems, X,
                                                normA2, nullptr, nullptr, true,
                                                s);
    case 1:
      return sketch_dispatch_kp<float, float>(kp, mats, items, nitems, X,
                                              normA2, nullptr, nullptr, true, s);
    case 2:
      return sketch_dispatch_kp<__nv_bfloat16, float>(
          kp, mats, items, nitems, X, normA2, nullptr, nullptr, true, s);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_sketch_y(int in_type, int kp, const MatDev* mats,
                            const int2* items, int nitems, const void* X,
                            void* Y, cudaStream_t s) {
  switch (in_type) {
    case 0:
      return sketch_dispatch_kp<double, double>(kp, mats, items, nitems,
                                                nullptr, nullptr, X, Y, false,
                                                s);
    case 1:
      return sketch_dispatch_kp<float, float>(kp, mats, items, nitems, nullptr,
                                              nullptr, X, Y, false, s);
    case 2:
      return sketch_dispatch_kp<__nv_bfloat16, float>(
          kp, mats, items, nitems, nullptr, nullptr, X, Y, false, s);
  }
  return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// T1 / T1': Gram matrices of the training tensor.
//   mode 1: G[a][b] = sum_d sum_j A_d[a][j] A_d[b][j]   (Eq. 3.2)
//   mode 2: G[a][b] = sum_d sum_i A_d[i][a] A_d[i][b]   (mode-2 unfolding)
// 64 x 64 output tiles of the lower triangle; blockIdx.y splits the sum over
// d.  Tile sums are accumulated in the compute type and added into the
// double G with atomics (both (a,b) and (b,a) off the diagonal).
// ---------------------------------------------------------------------------
template <typename Tin, typename Tc>
__global__ void __launch_bounds__(256)
gram_kernel(const void* const* __restrict__ dA, long long D, long long m,
            long long n, long long lda, int mode, int ntile, long long dchunk,
            double* __restrict__ G) {
  constexpr int T = 64, KC = 32;
  __shared__ Tc P1[KC][T + 1];
  __shared__ Tc P2[KC][T + 1];
  // lower-triangle tile pair from the linear block index
  int t = blockIdx.x, ta = 0;
  while (t > ta) {
    t -= ta + 1;
    ++ta;
  }
  const int tb = t;
  const long long dim = (mode == 1) ? m : n;
  const long long K = (mode == 1) ? n : m;
  const long long a0 = (long long)ta * T, b0 = (long long)tb * T;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  Tc acc[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[q][p] = Tc(0);
  const long long d0 = (long long)blockIdx.y * dchunk;
  const long long d1 = (d0 + dchunk < D) ? d0 + dchunk : D;
  for (long long d = d0; d < d1; ++d) {
    const Tin* __restrict__ A = (const Tin*)dA[d];
    for (long long k0 = 0; k0 < K; k0 += KC) {
      for (int e = tid; e < KC * T; e += 256) {
        int kk, a;
        if (mode == 1) {
          a = e / KC;
          kk = e % KC;
        } else {
          kk = e / T;
          a = e % T;
        }
        const long long kg = k0 + kk;
        const long long ga = a0 + a, gb = b0 + a;
        Tc v1 = Tc(0), v2 = Tc(0);
        if (kg < K) {
          if (mode == 1) {
            if (ga < dim) v1 = convert_in<Tc>(A[ga * lda + kg]);
            if (gb < dim) v2 = convert_in<Tc>(A[gb * lda + kg]);
          } else {
            if (ga < dim) v1 = convert_in<Tc>(A[kg * lda + ga]);
            if (gb < dim) v2 = convert_in<Tc>(A[kg * lda + gb]);
          }
        }
        P1[kk][a] = v1;
        P2[kk][a] = v2;
      }
      __syncthreads();
#pragma unroll 8
      for (int kk = 0; kk < KC; ++kk) {
        Tc x[4], y[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) x[q] = P1[kk][ty * 4 + q];
#pragma unroll
        for (int p = 0; p < 4; ++p) y[p] = P2[kk][tx * 4 + p];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int p = 0; p < 4; ++p) acc[q][p] += x[q] * y[p];
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const long long a = a0 + ty * 4 + q;
    if (a >= dim) continue;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const long long b = b0 + tx * 4 + p;
      if (b >= dim) continue;
      atomicAdd(G + a * dim + b, (double)acc[q][p]);
      if (ta != tb) atomicAdd(G + b * dim + a, (double)acc[q][p]);
    }
  }
}

cudaError_t launch_gram(int in_type, const void* const* dA, long long D,
                        long long m, long long n, long long lda, int mode,
                        double* G, cudaStream_t s) {
  const long long dim = (mode == 1) ? m : n;
  const int ntile = (int)((dim + 63) / 64);
  const long long npairs = (long long)ntile * (ntile + 1) / 2;
  long long splits = (2 * 152 * 4 + npairs - 1) / npairs;
  if (splits > D) splits = D;
  if (splits < 1) splits = 1;
  if (splits > 65535) splits = 65535;
  const long long dchunk = (D + splits - 1) / splits;
  splits = (D + dchunk - 1) / dchunk;
  dim3 grid((unsigned)npairs, (unsigned)splits);
  switch (in_type) {
    case 0:
      gram_kernel<double, double>
          <<<grid, 256, 0, s>>>(dA, D, m, n, lda, mode, ntile, dchunk, G);
      break;
    case 1:
      gram_kernel<float, float>
          <<<grid, 256, 0, s>>>(dA, D, m, n, lda, mode, ntile, dchunk, G);
      break;
    case 2:
      gram_kernel<__nv_bfloat16, float>
          <<<grid, 256, 0, s>>>(dA, D, m, n, lda, mode, ntile, dchunk, G);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Small dense GEMM for the eigensolver: C = alpha op(A) op(B) + beta C,
// row-major, op = transpose when the flag is set.  64 x 64 tiles.  With a
// workspace the K range is split over blockIdx.z (each split writes its
// partial product to part[z]) and a second kernel sums the splits in order,
// so that the thin products (80 x 80 over 2048 rows, 2048 x 80 over 2048)
// fill the GPU; the result does not depend on timing.
// ---------------------------------------------------------------------------
template <typename T, bool PART>
__global__ void __launch_bounds__(256)
gemm_kernel(int transA, int transB, long long M, long long N, long long K, long long kchunk,
            T alpha, const T* __restrict__ A, long long lda,
            const T* __restrict__ B, long long ldb, T beta, T* __restrict__ C,
            long long ldc, T* __restrict__ part) {
  constexpr int TM = 64, TN = 64, KC = 16;
  __shared__ T As[KC][TM + 1];
  __shared__ T Bs[KC][TN + 1];
  const long long m0 = (long long)blockIdx.y * TM, n0 = (long long)blockIdx.x * TN;
  const long long kb = (long long)blockIdx.z * kchunk;
  const long long ke = min(K, kb + kchunk);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  T acc[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[q][p] = T(0);
  for (long long k0 = kb; k0 < ke; k0 += KC) {
    for (int e = tid; e < KC * TM; e += 256) {
      const int kk = e / TM, a = e % TM;
      const long long gm = m0 + a, gk = k0 + kk;
      T v = T(0);
      if (gm < M && gk < ke) v = transA ? A[gk * lda + gm] : A[gm * lda + gk];
      As[kk][a] = v;
      const long long gn = n0 + a;
      T w = T(0);
      if (gn < N && gk < ke) w = transB ? B[gn * ldb + gk] : B[gk * ldb + gn];
      Bs[kk][a] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      T x[4], y[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) x[q] = As[kk][ty * 4 + q];
#pragma unroll
      for (int p = 0; p < 4; ++p) y[p] = Bs[kk][tx * 4 + p];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[q][p] += x[q] * y[p];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const long long gm = m0 + ty * 4 + q;
    if (gm >= M) continue;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const long long gn = n0 + tx * 4 + p;
      if (gn >= N) continue;
      if (PART) {
        part[((long long)blockIdx.z * M + gm) * N + gn] = acc[q][p];
      } else {
        T* c = C + gm * ldc + gn;
        *c = alpha * acc[q][p] + (beta == T(0) ? T(0) : beta * *c);
      }
    }
  }
}

// C = alpha sum_z part[z] + beta C, the splits summed in index order.
template <typename T>
__global__ void __launch_bounds__(256)
splitk_reduce_kernel(const T* __restrict__ part, int S, long long M, long long N, T alpha,
                     T beta, T* __restrict__ C, long long ldc) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= M * N) return;
  const long long i = e / N, j = e - i * N;
  T acc = T(0);
  for (int z = 0; z < S; ++z) acc += part[(long long)z * M * N + e];
  T* c = C + i * ldc + j;
  *c = alpha * acc + (beta == T(0) ? T(0) : beta * *c);
}

template <typename T>
static cudaError_t gemm_t(int transA, int transB, long long M, long long N, long long K,
                          double alpha, const void* A, long long lda, const void* B,
                          long long ldb, double beta, void* C, long long ldc, void* work,
                          size_t work_bytes, cudaStream_t s) {
  const long long tiles = ((N + 63) / 64) * ((M + 63) / 64);
  long long S = 1;
  if (work && M * N > 0) {
    int dev = 0, nsm = 148;
    if (cudaGetDevice(&dev) == cudaSuccess)
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    S = std::max<long long>(1, (2LL * nsm + tiles - 1) / tiles);  // about two CTAs per SM
    S = std::min<long long>(S, (K + 63) / 64);                     // at least 64 of K each
    S = std::min<long long>(S, (long long)(work_bytes / (sizeof(T) * M * N)));
    S = std::min<long long>(S, 64);
  }
  if (S <= 1) {
    dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64), 1);
    gemm_kernel<T, false><<<grid, 256, 0, s>>>(transA, transB, M, N, K, K, (T)alpha,
                                               (const T*)A, lda, (const T*)B, ldb, (T)beta,
                                               (T*)C, ldc, nullptr);
    return cudaGetLastError();
  }
  const long long kchunk = ((K + S - 1) / S + 15) / 16 * 16;
  S = (K + kchunk - 1) / kchunk;
  dim3 grid((unsigned)((N + 63) / 64), (unsigned)((M + 63) / 64), (unsigned)S);
  gemm_kernel<T, true><<<grid, 256, 0, s>>>(transA, transB, M, N, K, kchunk, (T)alpha,
                                            (const T*)A, lda, (const T*)B, ldb, (T)beta,
                                            (T*)C, ldc, (T*)work);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  splitk_reduce_kernel<T><<<(unsigned)((M * N + 255) / 256), 256, 0, s>>>(
      (const T*)work, (int)S, M, N, (T)alpha, (T)beta, (T*)C, ldc);
  return cudaGetLastError();
}

cudaError_t launch_gemm(bool dbl, int transA, int transB, long long M,
                        long long N, long long K, double alpha, const void* A,
                        long long lda, const void* B, long long ldb,
                        double beta, void* C, long long ldc, cudaStream_t s, void* work,
                        size_t work_bytes) {
  if (dbl)
    return gemm_t<double>(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, work,
                          work_bytes, s);
  return gemm_t<float>(transA, transB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, work,
                       work_bytes, s);
}

// ---------------------------------------------------------------------------
// E5 outputs: US = Y W (m x r) = A Q V_r = U_r Sigma_r and
// Vt = (X W)^T (r x n) = (Q V_r)^T, where W = R^{-1} V_r (k x r) comes from
// the small-SVD kernel.  Item = (matrix, block of 256 rows or columns,
// which = 0 for US / 1 for Vt).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
project_out_kernel(int kp, const MatDev* __restrict__ mats,
                   const int4* __restrict__ items, const T* __restrict__ X,
                   const T* __restrict__ Y, const T* __restrict__ Wm) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = (T*)smem_raw;  // kp x kp
  const int4 it = items[blockIdx.x];
  const MatDev md = mats[it.x];
  const int k = md.k, r = md.r;
  const T* Wsrc = Wm + (long long)it.x * kp * kp;
  for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) Ws[e] = Wsrc[e];
  __syncthreads();
  const long long idx = (long long)it.y * 256 + threadIdx.x;
  if (it.z == 0) {
    if (md.US == nullptr || idx >= md.m) return;
    const T* y = Y + md.offY + idx * kp;
    T* out = (T*)md.US + idx * r;
    for (int c = 0; c < r; ++c) {
      T a = T(0);
      for (int cc = 0; cc < k; ++cc) a += y[cc] * Ws[cc * kp + c];
      out[c] = a;
    }
  } else {
    if (md.Vt == nullptr || idx >= md.n) return;
    const T* x = X + md.offX + idx * kp;
    T* out = (T*)md.Vt;
    for (int c = 0; c < r; ++c) {
      T a = T(0);
      for (int cc = 0; cc < k; ++cc) a += x[cc] * Ws[cc * kp + c];
      out[(long long)c * md.n + idx] = a;
    }
  }
}

cudaError_t launch_project_out(bool dbl, int kp, const MatDev* mats,
                               const int4* items, int nitems, const void* X,
                               const void* Y, const void* Wm, cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  if (dbl)
    project_out_kernel<double><<<nitems, 256, kp * kp * sizeof(double), s>>>(
        kp, mats, items, (const double*)X, (const double*)Y,
        (const double*)Wm);
  else
    project_out_kernel<float><<<nitems, 256, kp * kp * sizeof(float), s>>>(
        kp, mats, items, (const float*)X, (const float*)Y, (const float*)Wm);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Direct error ||A - US Vt||_F^2 (problem 1.1) in one more pass over A.
// Item = (matrix, block of 16 rows).  Squares are summed in double.
// ---------------------------------------------------------------------------
template <typename Tin, typename Tc>
__global__ void __launch_bounds__(256)
direct_error_kernel(const MatDev* __restrict__ mats,
                    const int2* __restrict__ items, double* __restrict__ err2) {
  constexpr int RB = 16;
  __shared__ Tc Us[RB][TSK_MAX_K + 1];
  __shared__ double red[8];
  const int2 it = items[blockIdx.x];
  const MatDev md = mats[it.x];
  const Tin* __restrict__ A = (const Tin*)md.A;
  const Tc* __restrict__ US = (const Tc*)md.US;
  const Tc* __restrict__ Vt = (const Tc*)md.Vt;
  const long long m = md.m, n = md.n, lda = md.lda;
  const int r = md.r;
  const long long i0 = (long long)it.y * RB;
  for (int e = threadIdx.x; e < RB * r; e += 256) {
    const int ii = e / r, c = e % r;
    Us[ii][c] = (i0 + ii < m) ? US[(i0 + ii) * r + c] : Tc(0);
  }
  __syncthreads();
  double acc = 0.0;
  for (long long j = threadIdx.x; j < n; j += 256) {
    Tc v[TSK_MAX_K];
    for (int c = 0; c < r; ++c) v[c] = Vt[(long long)c * n + j];
    for (int ii = 0; ii < RB; ++ii) {
      const long long i = i0 + ii;
      if (i >= m) break;
      Tc b = Tc(0);
      for (int c = 0; c < r; ++c) b += Us[ii][c] * v[c];
      const double dlt = (double)convert_in<Tc>(A[i * lda + j]) - (double)b;
      acc += dlt * dlt;
    }
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    atomicAdd(err2 + it.x, t);
  }
}

cudaError_t launch_direct_error(int in_type, const MatDev* mats,
                                const int2* items, int nitems, double* err2,
                                cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  switch (in_type) {
    case 0:
      direct_error_kernel<double, double><<<nitems, 256, 0, s>>>(mats, items, err2);
      break;
    case 1:
      direct_error_kernel<float, float><<<nitems, 256, 0, s>>>(mats, items, err2);
      break;
    case 2:
      direct_error_kernel<__nv_bfloat16, float>
          <<<nitems, 256, 0, s>>>(mats, items, err2);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Direct-residual fallback.  The projection identity loses accuracy when the
// error is tiny compared with ||A|| (its floor is about sqrt(eps) ||A||);
// for the matrices the small-SVD kernel flagged, the factors are formed in
// the workspace (U2 = Y W in Y's layout, V2 = X W in X's layout, so that
// B = U2 V2^T) and ||A - B||_F is summed directly.
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256)
factor_ws_kernel(int kp, const MatDev* __restrict__ mats, const int* __restrict__ flags,
                 const T* __restrict__ X, const T* __restrict__ Y,
                 const T* __restrict__ Wm, T* __restrict__ U2, T* __restrict__ V2) {
  const int b = blockIdx.x;
  if (!flags[b]) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Ws = (T*)smem_raw;
  const MatDev md = mats[b];
  const int k = md.k, r = md.r;
  const T* Wsrc = Wm + (long long)b * kp * kp;
  for (int e = threadIdx.x; e < kp * kp; e += blockDim.x) Ws[e] = Wsrc[e];
  __syncthreads();
  const long long total = md.m + md.n;
  for (long long idx = (long long)blockIdx.y * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.y * blockDim.x) {
    const bool isU = idx < md.m;
    const long long row = isU ? idx : idx - md.m;
    const T* src = isU ? Y + md.offY + row * kp : X + md.offX + row * kp;
    T* dst = isU ? U2 + md.offY + row * kp : V2 + md.offX + row * kp;
    for (int c = 0; c < r; ++c) {
      T a = T(0);
      for (int cc = 0; cc < k; ++cc) a += src[cc] * Ws[cc * kp + c];
      dst[c] = a;
    }
  }
}

template <typename Tin, typename Tc>
__global__ void __launch_bounds__(256)
direct_ws_kernel(int kp, const MatDev* __restrict__ mats, const int* __restrict__ flags,
                 const Tc* __restrict__ U2, const Tc* __restrict__ V2,
                 double* __restrict__ err2) {
  const int b = blockIdx.x;
  if (!flags[b]) return;
  constexpr int RB = 16;
  __shared__ Tc Us[RB][TSK_MAX_K + 1];
  __shared__ double red[8];
  const MatDev md = mats[b];
  const Tin* __restrict__ A = (const Tin*)md.A;
  const long long m = md.m, n = md.n, lda = md.lda;
  const int r = md.r;
  double acc = 0.0;
  const long long nrb = (m + RB - 1) / RB;
  for (long long rb = blockIdx.y; rb < nrb; rb += gridDim.y) {
    const long long i0 = rb * RB;
    __syncthreads();
    for (int e = threadIdx.x; e < RB * r; e += 256) {
      const int ii = e / r, c = e % r;
      Us[ii][c] = (i0 + ii < m) ? U2[md.offY + (i0 + ii) * kp + c] : Tc(0);
    }
    __syncthreads();
    for (long long j = threadIdx.x; j < n; j += 256) {
      Tc v[TSK_MAX_K];
      for (int c = 0; c < r; ++c) v[c] = V2[md.offX + j * kp + c];
      for (int ii = 0; ii < RB; ++ii) {
        const long long i = i0 + ii;
        if (i >= m) break;
        Tc bb = Tc(0);
        for (int c = 0; c < r; ++c) bb += Us[ii][c] * v[c];
        const double dlt = (double)convert_in<Tc>(A[i * lda + j]) - (double)bb;
        acc += dlt * dlt;
      }
    }
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    atomicAdd(err2 + b, t);
  }
}

__global__ void finalize_direct_kernel(const int* __restrict__ flags,
                                       const double* __restrict__ err2,
                                       double* __restrict__ err, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count && flags[i]) err[i] = sqrt(err2[i] > 0.0 ? err2[i] : 0.0);
}

cudaError_t launch_direct_fallback(int in_type, int kp, const MatDev* mats, int count,
                                   const int* flags, const void* X, const void* Y,
                                   const void* Wm, void* U2, void* V2, double* err2,
                                   double* err, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  const bool dbl = (in_type == 0);
  const size_t ws = (size_t)kp * kp * (dbl ? 8 : 4);
  dim3 g1(count, 8), g2(count, 16);
  if (dbl) {
    factor_ws_kernel<double><<<g1, 256, ws, s>>>(kp, mats, flags, (const double*)X,
                                                 (const double*)Y, (const double*)Wm,
                                                 (double*)U2, (double*)V2);
    direct_ws_kernel<double, double><<<g2, 256, 0, s>>>(kp, mats, flags, (const double*)U2,
                                                        (const double*)V2, err2);
  } else {
    factor_ws_kernel<float><<<g1, 256, ws, s>>>(kp, mats, flags, (const float*)X,
                                                (const float*)Y, (const float*)Wm,
                                                (float*)U2, (float*)V2);
    if (in_type == 1)
      direct_ws_kernel<float, float><<<g2, 256, 0, s>>>(kp, mats, flags, (const float*)U2,
                                                        (const float*)V2, err2);
    else
      direct_ws_kernel<__nv_bfloat16, float><<<g2, 256, 0, s>>>(
          kp, mats, flags, (const float*)U2, (const float*)V2, err2);
  }
  finalize_direct_kernel<<<(count + 255) / 256, 256, 0, s>>>(flags, err2, err, count);
  return cudaGetLastError();
}

__global__ void sqrt_inplace_kernel(double* v, int count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) v[i] = sqrt(v[i] > 0.0 ? v[i] : 0.0);
}

cudaError_t launch_sqrt_inplace(double* v, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  sqrt_inplace_kernel<<<(count + 255) / 256, 256, 0, s>>>(v, count);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Eigensolver helpers (training side, T2).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void convert_gram_kernel(const double* __restrict__ G,
                                    T* __restrict__ out, long long count) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) out[i] = (T)G[i];
}

cudaError_t launch_convert_gram(bool dbl, const double* G, void* out,
                                long long count, cudaStream_t s) {
  const unsigned blocks = (unsigned)((count + 255) / 256);
  if (dbl)
    convert_gram_kernel<double><<<blocks, 256, 0, s>>>(G, (double*)out, count);
  else
    convert_gram_kernel<float><<<blocks, 256, 0, s>>>(G, (float*)out, count);
  return cudaGetLastError();
}

// Deterministic start block for subspace iteration: a SplitMix64 hash of the
// element index mapped to [-1, 1).
template <typename T>
__global__ void random_fill_kernel(T* __restrict__ Z, long long count,
                                   unsigned long long seed) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  unsigned long long x = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(i + 1);
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  x = x ^ (x >> 31);
  const double u = (double)(x >> 11) * (1.0 / 9007199254740992.0);
  Z[i] = (T)(2.0 * u - 1.0);
}

cudaError_t launch_random_fill(bool dbl, void* Z, long long count,
                               unsigned long long seed, cudaStream_t s) {
  const unsigned blocks = (unsigned)((count + 255) / 256);
  if (dbl)
    random_fill_kernel<double><<<blocks, 256, 0, s>>>((double*)Z, count, seed);
  else
    random_fill_kernel<float><<<blocks, 256, 0, s>>>((float*)Z, count, seed);
  return cudaGetLastError();
}

// Q = P R^{-1} row by row (forward substitution with the upper R, ld p).
template <typename T>
__global__ void apply_rinv_kernel(const T* __restrict__ P,
                                  const T* __restrict__ R, T* __restrict__ Q,
                                  long long rows, int p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* Rs = (T*)smem_raw;
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) Rs[e] = R[e];
  __syncthreads();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= rows) return;
  const T* src = P + i * p;
  T* dst = Q + i * p;
  for (int c = 0; c < p; ++c) {
    T t = src[c];
    for (int cc = 0; cc < c; ++cc) t -= dst[cc] * Rs[cc * p + c];
    const T d = Rs[c * p + c];
    dst[c] = (d != T(0)) ? t / d : T(0);
  }
}

cudaError_t launch_apply_rinv(bool dbl, const void* P, const void* R, void* Q,
                              long long rows, int p, cudaStream_t s) {
  const unsigned blocks = (unsigned)((rows + 127) / 128);
  if (dbl)
    apply_rinv_kernel<double><<<blocks, 128, p * p * sizeof(double), s>>>(
        (const double*)P, (const double*)R, (double*)Q, rows, p);
  else
    apply_rinv_kernel<float><<<blocks, 128, p * p * sizeof(float), s>>>(
        (const float*)P, (const float*)R, (float*)Q, rows, p);
  return cudaGetLastError();
}

// Ri = R^{-1} where R (upper) has R^T R = Gm (p x p, row stride p, p <= 96),
// in one CTA of 1024 threads.  Cholesky right-looking in shared memory, the
// trailing updates of a step spread over a 32 x 32 grid of threads, one
// barrier per step; a pivot at or below 1e-12 of the largest diagonal entry
// makes that row of R the unit row e_j.  Then column c of R^{-1} by back
// substitution in the four threads 4c .. 4c + 3, each summing every fourth
// term.  Gm and Ri may be the same array.
template <typename T>
__global__ void __launch_bounds__(1024)
chol_inv_kernel(const T* Gm, int p, T* Ri) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ld = p + 1, tid = threadIdx.x;
  T* A = (T*)smem_raw;  // p x (p + 1): Gm, then R
  T* I = A + p * ld;    // p x (p + 1): R^{-1}
  T* dg = I + p * ld;   // p: the pivots
  for (int e = tid; e < p * p; e += blockDim.x) {
    const int a = e / p, c = e - a * p;
    A[a * ld + c] = Gm[e];
    I[a * ld + c] = T(0);
  }
  __syncthreads();
  T mx = T(0);
  for (int a = 0; a < p; ++a) mx = A[a * ld + a] > mx ? A[a * ld + a] : mx;
  const T thr = T(1e-12) * mx;
  const int ty = tid >> 5, tx = tid & 31;
  for (int j = 0; j < p; ++j) {
    const T d = A[j * ld + j];
    if (d > thr)
      for (int c = j + 1 + tx; c < p; c += 32) {
        const T f = A[j * ld + c] / d;
        for (int a = j + 1 + ty; a <= c; a += 32) A[a * ld + c] -= A[j * ld + a] * f;
      }
    __syncthreads();
  }
  for (int a = tid; a < p; a += blockDim.x) dg[a] = A[a * ld + a];
  __syncthreads();
  for (int e = tid; e < p * p; e += blockDim.x) {
    const int a = e / p, c = e - a * p;
    const T d = dg[a];
    T v = T(0);
    if (c >= a) v = (d > thr) ? A[a * ld + c] / sqrt(d) : (c == a ? T(1) : T(0));
    A[a * ld + c] = v;
  }
  __syncthreads();
  const int c = tid >> 2, q4 = tid & 3;
  const unsigned m4 = 0xFu << (tid & 28);
  if (c < p) {  // the column's four threads together
    const T dc = A[c * ld + c];
    if (q4 == 0) I[c * ld + c] = dc != T(0) ? T(1) / dc : T(0);
    __syncwarp(m4);
    for (int i = c - 1; i >= 0; --i) {
      T t = T(0);
      for (int q = i + 1 + q4; q <= c; q += 4) t += A[i * ld + q] * I[q * ld + c];
      t += __shfl_xor_sync(m4, t, 1);
      t += __shfl_xor_sync(m4, t, 2);
      const T d = A[i * ld + i];
      if (q4 == 0) I[i * ld + c] = d != T(0) ? -t / d : T(0);
      __syncwarp(m4);
    }
  }
  __syncthreads();
  for (int e = tid; e < p * p; e += blockDim.x) {
    const int a = e / p, cc = e - a * p;
    Ri[e] = I[a * ld + cc];
  }
}

cudaError_t launch_chol_inv(bool dbl, const void* Gm, int p, void* Ri, cudaStream_t s) {
  if (p < 1 || p > 96) return cudaErrorInvalidValue;
  const size_t es = dbl ? sizeof(double) : sizeof(float);
  const size_t sh = ((size_t)2 * p * (p + 1) + p) * es;
  cudaError_t e;
  if (dbl) {
    e = cudaFuncSetAttribute(chol_inv_kernel<double>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
    chol_inv_kernel<double><<<1, 1024, sh, s>>>((const double*)Gm, p, (double*)Ri);
  } else {
    e = cudaFuncSetAttribute(chol_inv_kernel<float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sh);
    if (e != cudaSuccess) return e;
    chol_inv_kernel<float><<<1, 1024, sh, s>>>((const float*)Gm, p, (float*)Ri);
  }
  return cudaGetLastError();
}


// P[:, c] /= |theta_c| (theta_c != 0): a subspace-iteration block G U whose
// columns are close to theta_c u_c becomes close to orthonormal.
template <typename T>
__global__ void scale_cols_kernel(T* __restrict__ P, long long rows, int p,
                                  const T* __restrict__ theta) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= rows * p) return;
  const T t = theta[e % p];
  const T a = t < T(0) ? -t : t;
  if (a > T(0)) P[e] /= a;
}

cudaError_t launch_scale_cols(bool dbl, void* P, long long rows, int p, const void* theta,
                              cudaStream_t s) {
  const unsigned blocks = (unsigned)((rows * p + 255) / 256);
  if (dbl)
    scale_cols_kernel<double><<<blocks, 256, 0, s>>>((double*)P, rows, p,
                                                     (const double*)theta);
  else
    scale_cols_kernel<float><<<blocks, 256, 0, s>>>((float*)P, rows, p, (const float*)theta);
  return cudaGetLastError();
}

// res[c] = ||GU[:, c] - theta_c U[:, c]||_2 for c < k (one CTA per column).
template <typename T>
__global__ void ritz_residual_kernel(const T* __restrict__ U,
                                     const T* __restrict__ GU,
                                     const T* __restrict__ theta,
                                     double* __restrict__ res, long long rows,
                                     int p) {
  __shared__ double red[8];
  const int c = blockIdx.x;
  const double th = (double)theta[c];
  double acc = 0.0;
  for (long long i = threadIdx.x; i < rows; i += blockDim.x) {
    const double d = (double)GU[i * p + c] - th * (double)U[i * p + c];
    acc += d * d;
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    res[c] = sqrt(t);
  }
}

cudaError_t launch_ritz_residual(bool dbl, const void* U, const void* GU,
                                 const void* theta, double* res,
                                 long long rows, int p, int k, cudaStream_t s) {
  if (dbl)
    ritz_residual_kernel<double><<<k, 256, 0, s>>>(
        (const double*)U, (const double*)GU, (const double*)theta, res, rows, p);
  else
    ritz_residual_kernel<float><<<k, 256, 0, s>>>(
        (const float*)U, (const float*)GU, (const float*)theta, res, rows, p);
  return cudaGetLastError();
}

// S[c][i] = sign_c * U[i][c] for c < k, the sign making the entry of largest
// magnitude (lowest index on a tie) positive.  One CTA per column.
template <typename T>
__global__ void emit_sketch_kernel(const T* __restrict__ U, long long rows,
                                   int p, T* __restrict__ S) {
  __shared__ double bv[256];
  __shared__ long long bi[256];
  const int c = blockIdx.x;
  double best = -1.0;
  long long besti = 0;
  for (long long i = threadIdx.x; i < rows; i += blockDim.x) {
    const double a = fabs((double)U[i * p + c]);
    if (a > best) {
      best = a;
      besti = i;
    }
  }
  bv[threadIdx.x] = best;
  bi[threadIdx.x] = besti;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double v2 = bv[threadIdx.x + o];
      const long long i2 = bi[threadIdx.x + o];
      if (v2 > bv[threadIdx.x] || (v2 == bv[threadIdx.x] && i2 < bi[threadIdx.x])) {
        bv[threadIdx.x] = v2;
        bi[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  const T sgn = (U[bi[0] * p + c] < T(0)) ? T(-1) : T(1);
  for (long long i = threadIdx.x; i < rows; i += blockDim.x)
    S[(long long)c * rows + i] = sgn * U[i * p + c];
}

cudaError_t launch_emit_sketch(bool dbl, const void* U, long long rows, int p,
                               int k, void* S, cudaStream_t s) {
  if (dbl)
    emit_sketch_kernel<double><<<k, 256, 0, s>>>((const double*)U, rows, p,
                                                 (double*)S);
  else
    emit_sketch_kernel<float><<<k, 256, 0, s>>>((const float*)U, rows, p,
                                                (float*)S);
  return cudaGetLastError();
}

// One CTA per 8 rows of one matrix.  A thread takes eight consecutive
// elements of a row: eight 2-byte loads in flight (the source rows have no
// alignment beyond 2 bytes) and one 16-byte store (the copy's rows start on
// 16-byte boundaries); past n it stores zeros, within the padding.
__global__ void __launch_bounds__(256) pack_rows_kernel(const PackDev* __restrict__ packs,
                                                        const int2* __restrict__ items) {
  const int2 it = items[blockIdx.x];
  const PackDev pk = packs[it.x];
  const unsigned short* src = (const unsigned short*)pk.src;
  unsigned short* dst = (unsigned short*)pk.dst;
  const long long r0 = (long long)it.y * 8;
  const long long r1 = min(pk.m, r0 + 8);
  const long long nch = (pk.n + 7) / 8;
  for (long long r = r0; r < r1; ++r) {
    const unsigned short* a = src + r * pk.lda;
    unsigned short* b = dst + r * pk.ldp;
    for (long long c = threadIdx.x; c < nch; c += blockDim.x) {
      const long long j0 = 8 * c;
      unsigned short v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) v[e] = (j0 + e < pk.n) ? a[j0 + e] : (unsigned short)0;
      uint4 w;
      w.x = (uint32_t)v[0] | ((uint32_t)v[1] << 16);
      w.y = (uint32_t)v[2] | ((uint32_t)v[3] << 16);
      w.z = (uint32_t)v[4] | ((uint32_t)v[5] << 16);
      w.w = (uint32_t)v[6] | ((uint32_t)v[7] << 16);
      *reinterpret_cast<uint4*>(b + j0) = w;
    }
  }
}

cudaError_t launch_pack_rows(const PackDev* packs, const int2* items, int nitems,
                             cudaStream_t s) {
  if (nitems <= 0) return cudaSuccess;
  pack_rows_kernel<<<nitems, 256, 0, s>>>(packs, items);
  return cudaGetLastError();
}

}  // namespace tsk
