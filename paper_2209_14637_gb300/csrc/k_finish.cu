// Small factors of the FP32 / BF16 test pass (E2 + E4 + E5 of the SCW step,
// Algorithm 1 in the QR form of Section 3.2), one CTA per matrix.
//
// From the panels X (n x k) and Y = A X (m x k) written by the sketch pass:
//
//   R1   = chol(X^T X)                        (X = Q R_X)
//   M1   = Y R1^{-1},  G_M = M1^T M1          (streamed)
//   sigma_i(AQ)^2 = lambda_i(G_M),  V = eigenvectors,  W = R1^{-1} V_r
//   err^2 = ||A||^2 - sum_{i<=r} v_i^T G_M v_i (Eq. A.3; Ky Fan)
//
// and, where the first-order bound on the energy's change from the FP32
// rounding of X^T X asks for it (or always, refine = 1), one CholeskyQR2
// step: Q1 = X R1^{-1} streamed, R2 = chol(Q1^T Q1), G_M <- R2^{-T} G_M
// R2^{-1}, R_X^{-1} = R1^{-1} R2^{-1}, and the eigenpairs again.
//
// Y itself is never factored: its columns scale like sigma_i^2 and Y^T Y
// would lose everything in FP32.  M1 = A Q1 is as well conditioned as A Q,
// and R2 is within rounding of the identity, so applying it in k x k space
// costs no accuracy.
//
// Streaming: each panel passes through shared memory in blocks of FSB rows
// (16-byte cp.async copies, NST - 1 blocks in flight) into padded rows of
// k_c + 4 floats, so eight consecutive rows fall in eight different 16-byte
// bank groups.  For the transform P R^{-1} (R^{-1} upper), warp w
// computes the output column tiles w and n4 - 1 - w of one row per lane, so
// every lane takes the same n4 + 1 steps and every R^{-1} load is a
// broadcast.  The Gram is accumulated in 8 x 4 register tiles by several
// row groups.
//
// Eigenpairs: G_M = R_M^T R_M (Cholesky), then one-sided (Hestenes) Jacobi on
// L = R_M^T.  Rotations that make the columns of L orthogonal give
// L V = U Sigma with G_M = U Sigma^2 U^T: the column norms are the sigma_i,
// the normalised columns the eigenvectors, and nothing is accumulated.
// Jacobi on L needs fewer sweeps than Jacobi on G_M (L^T L = R_M R_M^T is
// one step of the QR iteration further along).  Four threads hold a column
// in registers.
#include <stdint.h>

#include <algorithm>

#include "tsk_internal.cuh"

namespace tsk {

namespace {

constexpr int FT = 256;                       // threads per CTA
constexpr int FW = FT / 32;                   // warps
constexpr int FSB = 32;                       // rows per streamed block (one per lane)
constexpr int NST = 4;                        // stages: NST - 1 blocks in flight

// Rows per quarter of a Jacobi column (a multiple of 4) for compute width kc.
__host__ __device__ constexpr int fin_quarter(int kc) { return (((kc + 3) / 4) + 3) & ~3; }

// Shared-memory layout, offsets in floats; kcm = the batch's largest k
// rounded up to 8 (<= 64).  Sizes follow kcm, strides a matrix's own k_c.
struct FinLay {
  int kcm;
  int ri;     // R^{-1} of the transform, later R_X^{-1}: kcm x kcm
  int ga;     // Gram / Cholesky workspace kept across passes: kcm x (kcm + 1)
  int dv;     // 64 reciprocals of Cholesky diagonals
  int dx;     // 64 column norms of X
  int red;    // 2 FW + 2 doubles: block reductions and a broadcast slot
  int area;   // streaming stages and the block buffer; reused between passes
  int stage;  // floats per stage: FSB x (kcm + 4)
  size_t bytes;
};

FinLay fin_layout(int kcm) {
  FinLay L;
  L.kcm = kcm;
  const int gld = kcm + 1, jl = 4 * fin_quarter(kcm) + 4;
  const int g4 = (kcm * gld + 3) & ~3;
  int o = 0;
  L.ri = o;
  o += kcm * kcm;
  L.ga = o;
  o += g4;
  L.dv = o;
  o += 64;
  L.dx = o;
  o += 64;
  L.red = o;  // a multiple of 4 floats: doubles align
  o += 4 * FW + 4;
  L.area = o;
  L.stage = FSB * (kcm + 4);
  // what the area holds between the passes
  const int p5 = g4 + 2 * kcm * kcm;             // M1^T M1, R2^{-1}, product
  const int jac = g4 + 2 * kcm * jl + 2 * kcm;   // R_M, planes, lam, order
  o += std::max((NST + 1) * L.stage, std::max(p5, jac));
  L.bytes = (size_t)o * 4;
  return L;
}

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ float4 ld4(const float* p) {
  return *reinterpret_cast<const float4*>(p);
}

__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

__device__ __forceinline__ void cp16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(su32(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// One or two panels streamed back to back; the upper triangle (8 x 4 tiles,
// row stride kc + 1) of the Gram of each panel P, or of P R^{-1}, goes to
// the panel's target once its last block is in.
struct FinPass {
  const float *P0, *P1;
  long long rows0, rows1;
  float *out0, *out1;
  int nseg;
};

// The area is free on entry (a barrier precedes its reuse); a target in the
// area is written only after the last block.  The panel width KC (k rounded
// up to 8) is a compile-time constant, so that the block loops unroll.
template <int KC>
__device__ __forceinline__ void fin_stream_kc(const FinLay& L, float* sm, int kp, const FinPass& S,
                                           bool tr) {
  constexpr int kc = KC;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int srow = kc + 4, ldo = kc + 1, n4 = kc / 4;
  float* area = sm + L.area;
  float* Ts = area + NST * L.stage;
  const float* RI = sm + L.ri;
  const int nb0 = (int)((S.rows0 + FSB - 1) / FSB);
  const int nb = nb0 + (S.nseg > 1 ? (int)((S.rows1 + FSB - 1) / FSB) : 0);
  auto block_rows = [&](int bi, int& seg, long long& r0) {
    seg = bi < nb0 ? 0 : 1;
    r0 = (long long)(bi - (seg ? nb0 : 0)) * FSB;
    return (int)min((long long)FSB, (seg ? S.rows1 : S.rows0) - r0);
  };
  // Thread t copies the 16-byte pieces (row, quad) = (t / 16 + 16 i, t % 16),
  // i = 0, 1, of every block.
  static_assert(FSB * 16 == 2 * FT, "two pieces per thread and block");
  auto issue = [&](int bi) {  // every thread: its pieces of block bi
    const int crow = threadIdx.x >> 4, cq = threadIdx.x & 15;
    if (bi < nb && cq < n4) {
      int seg;
      long long r0;
      const int nrows = block_rows(bi, seg, r0);
      const float* P = (seg ? S.P1 : S.P0) + (r0 + crow) * kp + 4 * cq;
      float* dst = area + (bi % NST) * L.stage + crow * srow + 4 * cq;
      if (crow < nrows) cp16(dst, P);
      if (crow + 16 < nrows) cp16(dst + 16 * srow, P + 16 * kp);
    }
    cp_commit();  // one group per block, empty ones included
  };
  __syncthreads();
  for (int bi = 0; bi < NST - 1; ++bi) issue(bi);
  // Gram tiles (ty, tx) of 8 rows x 4 columns meeting the upper triangle
  // (tx >= 2 ty); `groups` row groups share each tile.
  constexpr int n8 = kc / 8;
  constexpr int ntiles = n8 * n4 - n8 * (n8 - 1);  // sum over ty of (n4 - 2 ty)
  constexpr int groups = FT / ntiles < 1 ? 1 : (FT / ntiles > 8 ? 8 : FT / ntiles);
  constexpr int per = (FSB + groups - 1) / groups;  // rows of a block per row group
  const bool active = tid < groups * ntiles;
  const int tile = tid % ntiles, grp = tid / ntiles;
  int ty = 0, rem = tile;
  while (rem >= n4 - 2 * ty) {
    rem -= n4 - 2 * ty;
    ++ty;
  }
  const int tx = 2 * ty + rem;
  constexpr int npairs = n4 / 2;
  float acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
  cp_wait<NST - 2>();  // this thread's pieces of block 0 have landed
  __syncthreads();
  for (int bi = 0; bi < nb; ++bi) {
    issue(bi + NST - 1);  // into the stage block bi - 1 used
    int seg;
    long long r0;
    const int nrows = block_rows(bi, seg, r0);
    const float* Pb = area + (bi % NST) * L.stage;
    const float* src = Pb;
    if (tr) {
      if (warp < npairs) {
        // row `lane` of Pb R^{-1}: column tile cg (R^{-1} rows < 4 cg + 4)
        // and column tile c2 = n4 - 1 - cg (rows < 4 c2 + 4); n4 + 1 steps
        // of four rows for every warp
        const int cg = warp, c2 = n4 - 1 - warp;
        const float* prow = Pb + lane * srow;
        float* trow = Ts + lane * srow;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          const int c = h ? c2 : cg;
          float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
#pragma unroll
          for (int q = 0; q < n4; ++q) {
            if (q > c) break;
            const float4 p = ld4(prow + 4 * q);
            const float* rr = RI + (4 * q) * kc + 4 * c;
            const float4 e0 = ld4(rr), e1 = ld4(rr + kc), e2 = ld4(rr + 2 * kc),
                         e3 = ld4(rr + 3 * kc);
            ffma2(t0, t1, p.x, p.x, e0.x, e0.y);
            ffma2(t2, t3, p.x, p.x, e0.z, e0.w);
            ffma2(t0, t1, p.y, p.y, e1.x, e1.y);
            ffma2(t2, t3, p.y, p.y, e1.z, e1.w);
            ffma2(t0, t1, p.z, p.z, e2.x, e2.y);
            ffma2(t2, t3, p.z, p.z, e2.z, e2.w);
            ffma2(t0, t1, p.w, p.w, e3.x, e3.y);
            ffma2(t2, t3, p.w, p.w, e3.z, e3.w);
          }
          st4(trow + 4 * c, t0, t1, t2, t3);
        }
      }
      __syncthreads();
      src = Ts;
    }
    if (active) {
#pragma unroll
      for (int t = 0; t < per; ++t) {
        const int ii = grp + t * groups;
        if (ii >= nrows) break;
        const float4 x0 = ld4(src + ii * srow + 8 * ty);
        const float4 x1 = ld4(src + ii * srow + 8 * ty + 4);
        const float4 y = ld4(src + ii * srow + 4 * tx);
        const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        const float yv[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int a = 0; a < 8; a += 2)
#pragma unroll
          for (int c = 0; c < 4; ++c)
            ffma2(acc[a][c], acc[a + 1][c], xv[a], xv[a + 1], yv[c], yv[c]);
      }
    }
    cp_wait<NST - 2>();  // this thread's pieces of block bi + 1 have landed
    __syncthreads();     // block bi (and Ts) consumed; block bi + 1 visible
    if (bi == nb0 - 1 || bi == nb - 1) {
      // the row groups' tiles summed in a fixed order into the target
      float* out = seg ? S.out1 : S.out0;
      for (int g = 0; g < groups; ++g) {
        if (active && grp == g) {
#pragma unroll
          for (int a = 0; a < 8; ++a)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              float* o = out + (8 * ty + a) * ldo + 4 * tx + c;
              *o = (g == 0) ? acc[a][c] : *o + acc[a][c];
            }
        }
        __syncthreads();
      }
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
    }
  }
  cp_wait<0>();
}


// Cholesky of the upper triangle of G (k x k, row stride ld) in place, right
// looking: at step j, thread (a0, c) = (t / 64, t % 64) updates entries
// (a, c), j < a <= c, a = a0 mod 4, from row j; one barrier per step.
// Afterwards row j of R = U_j / sqrt(U_jj), U_j the j-th row of the Schur
// complement at step j, and dinv[j] = 1 / R_jj.  A pivot
// U_jj <= 1e-12 max_i G_ii (|R_jj| <= 1e-6 max sqrt(G_ii)) is dropped (its
// row of R is zero, dinv 0) and, with `check`, raises kStatusRankDef.
__device__ void fin_chol(float* G, int ld, int k, float* dinv, bool check, int* status) {
  const int tid = threadIdx.x;
  const int a0 = tid >> 6, c = tid & 63;
  float mx = 0.f;
  for (int a = 0; a < k; ++a) mx = fmaxf(mx, G[a * ld + a]);
  const float thr = 1e-12f * mx;
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    const float d = G[j * ld + j];
    if (d > thr && c > j && c < k) {
      const float gc = G[j * ld + c] / d;
      for (int a = j + 1 + ((a0 - j - 1) & 3); a <= c; a += 4)
        G[a * ld + c] = fmaf(-G[j * ld + a], gc, G[a * ld + c]);
    }
    __syncthreads();
  }
  if (tid < 32) {
    bool bad = false;
    for (int a = tid; a < k; a += 32) {
      const float d = G[a * ld + a];
      const bool drop = !(d > thr);
      bad |= drop;
      dinv[a] = drop ? 0.f : rsqrtf(d);
    }
    if (check && __any_sync(0xffffffffu, bad) && tid == 0) atomicOr(status, kStatusRankDef);
  }
  __syncthreads();
  for (int e = tid; e < k * 64; e += FT) {
    const int a = e >> 6, cc = e & 63;
    if (cc >= a && cc < k) G[a * ld + cc] *= dinv[a];
  }
  __syncthreads();
}

// R^{-1} (upper, k x k, from fin_chol's R with row stride ld and dinv) into
// Ri (kc x kc, row stride kc, zero below the diagonal and past k): column c
// by back substitution in the four threads 4c .. 4c + 3, each summing every
// fourth term.
__device__ void fin_rinv(const float* __restrict__ R, int ld, const float* __restrict__ dinv,
                         int k, int kc, float* __restrict__ Ri) {
  const int tid = threadIdx.x;
  for (int e = tid; e < kc * kc; e += FT) Ri[e] = 0.f;
  __syncthreads();
  const int c = tid >> 2, qq = tid & 3;
  const unsigned m4 = 0xFu << (tid & 28);
  if (c < k) {  // the column's four lanes together
    if (qq == 0) Ri[c * kc + c] = dinv[c];
    __syncwarp(m4);
    for (int i = c - 1; i >= 0; --i) {
      float t = 0.f;
      for (int q = i + 1 + qq; q <= c; q += 4) t = fmaf(R[i * ld + q], Ri[q * kc + c], t);
      t += __shfl_xor_sync(m4, t, 1);
      t += __shfl_xor_sync(m4, t, 2);
      if (qq == 0) Ri[i * kc + c] = -t * dinv[i];
      __syncwarp(m4);
    }
  }
  __syncthreads();
}

// Partner of column j in round `round` (< mm) of the round-robin order on
// kk = mm + 1 columns: the pairs are (round, mm) and (round + i, round - i)
// mod mm, i = 1 .. kk/2 - 1.
__device__ __forceinline__ int fin_partner(int round, int j, int mm) {
  if (j == mm) return round;
  if (j == round) return mm;
  int x = 2 * round - j;
  if (x < 0) x += mm;
  if (x >= mm) x -= mm;
  return x;
}

// The CholeskyQR2 correction applied in k x k space: R2 = chol(GQ) (GQ =
// Q1^T Q1, upper, row stride gld, overwritten), G_M = R2^{-T} GM1 R2^{-1}
// (upper, into GA; GM1 = M1^T M1, upper, row stride gld, may be GA) and
// R_X^{-1} = R1^{-1} R2^{-1} (RI, in place).  Scratch: the area after GQ.
__device__ void fin_refine(float* GQ, const float* GM1, float* GA, float* RI, float* area,
                           float* DV, int k, int kc, int gld, int g4, int* status) {
  const int tid = threadIdx.x;
  float* RF = area + g4;     // R2^{-1}, row stride kc
  float* TT = RF + kc * kc;  // row stride kc
  float* RX = area;          // R1^{-1} R2^{-1}, row stride kc (GQ is dead by then)
  fin_chol(GQ, gld, k, DV, true, status);
  fin_rinv(GQ, gld, DV, k, kc, RF);
  // TT = GM1 R2^{-1}, four columns per thread
  for (int e = tid; e < k * 16; e += FT) {
    const int a = e >> 4, c4 = e & 15;
    if (4 * c4 < k) {
      float t0 = 0.f, t1 = 0.f, t2 = 0.f, t3 = 0.f;
      const int qm = min(k - 1, 4 * c4 + 3);
      for (int q = 0; q <= qm; ++q) {
        const float g = GM1[min(a, q) * gld + max(a, q)];
        const float4 f = ld4(RF + q * kc + 4 * c4);
        t0 = fmaf(g, f.x, t0);
        t1 = fmaf(g, f.y, t1);
        t2 = fmaf(g, f.z, t2);
        t3 = fmaf(g, f.w, t3);
      }
      st4(TT + a * kc + 4 * c4, t0, t1, t2, t3);
    }
  }
  __syncthreads();
  // GA = R2^{-T} TT (upper); RX = R1^{-1} R2^{-1}
  for (int e = tid; e < k * 16; e += FT) {
    const int a = e >> 4, c4 = e & 15;
    if (4 * c4 < k && 4 * c4 + 3 >= a) {
      float t[4] = {0.f, 0.f, 0.f, 0.f}, w[4] = {0.f, 0.f, 0.f, 0.f};
      for (int q = 0; q <= a; ++q) {
        const float f = RF[q * kc + a];
        const float4 v = ld4(TT + q * kc + 4 * c4);
        t[0] = fmaf(f, v.x, t[0]);
        t[1] = fmaf(f, v.y, t[1]);
        t[2] = fmaf(f, v.z, t[2]);
        t[3] = fmaf(f, v.w, t[3]);
      }
      const int qm = min(k - 1, 4 * c4 + 3);
      for (int q = a; q <= qm; ++q) {
        const float f = RI[a * kc + q];
        const float4 v = ld4(RF + q * kc + 4 * c4);
        w[0] = fmaf(f, v.x, w[0]);
        w[1] = fmaf(f, v.y, w[1]);
        w[2] = fmaf(f, v.z, w[2]);
        w[3] = fmaf(f, v.w, w[3]);
      }
#pragma unroll
      for (int z = 0; z < 4; ++z) {
        const int c = 4 * c4 + z;
        if (c >= a && c < k) GA[a * gld + c] = t[z];
      }
      st4(RX + a * kc + 4 * c4, w[0], w[1], w[2], w[3]);
    }
  }
  __syncthreads();
  for (int e = tid; e < kc * kc; e += FT) {
    const int a = e / kc, c = e - a * kc;
    RI[e] = (a < k && c < k && c >= a) ? RX[e] : 0.f;
  }
  __syncthreads();
}

// Eigenpairs of G_M (upper in GA, row stride gld) and what follows from
// them: sigma (md.sigma), V_r, W = R_X^{-1} V_r into WS (= the start of the
// area, row stride kc), and in red[0] / red[1] (after the final barrier) the
// captured energy tr(V_r^T G_M V_r) and the first-order bound
//   est = u sum_{c<r} lambda_c (sum_i DX_i |W_ic|)^2
// on its change from the rounding of X^T X (u = 2^-24): with
// R^T R = X^T X + E, |E_ij| <~ u DX_i DX_j, lambda_c moves by about
// lambda_c w_c^T E w_c, w_c = R^{-1} v_c, where ||X w_c|| = 1.
//
// G_M = R_M^T R_M (Cholesky), then one-sided Jacobi on L = R_M^T (column j
// of L = row j of R_M).  Thread (j, qt) = (tid / 4, tid % 4) keeps rows
// [qt QMAX, qt QMAX + QMAX) of column j in registers; each round of the
// parallel round-robin order it stores them to one of two planes, reads its
// part of the partner column after one barrier, sums the three partial dot
// products over the column's four lanes, and all eight threads of a pair
// compute the same rotation from the same sums.
template <int QMAX>
__device__ void fin_eigen(const MatDev& md, int k, int r, int kc, int gld, int g4,
                          const float* GA, const float* RI, const float* DX, float* DV,
                          float* area, double* red, int* status) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  constexpr int jl = 4 * QMAX + 4;  // column stride of the planes
  float* GC = area;                 // R_M, row stride gld; later E and WS
  float* PL = area + g4;            // two planes
  float* lam = PL + 2 * kc * jl;    // kc
  int* order = (int*)(lam + kc);    // kc
  for (int e = tid; e < k * 64; e += FT) {
    const int a = e >> 6, c = e & 63;
    if (c >= a && c < k) GC[a * gld + c] = GA[a * gld + c];
  }
  __syncthreads();
  fin_chol(GC, gld, k, DV, false, status);
  const int j = tid >> 2, qt = tid & 3;
  const int i0 = qt * QMAX;
  float bc[QMAX];
#pragma unroll
  for (int i = 0; i < QMAX; ++i) {
    const int row = i0 + i;  // L[row][j] = R_M[j][row], zero below the diagonal of R_M
    bc[i] = (j < k && row < k && row >= j) ? GC[j * gld + row] : 0.f;
  }
  const unsigned gmask = 0xFu << (lane & 28);  // the column's four lanes
  const int kk = k + (k & 1), mm = kk - 1;
  int t = 0;
  for (int sweep = 0; sweep < 15 && mm > 0; ++sweep) {
    int rot = 0;
    for (int round = 0; round < mm; ++round, ++t) {
      float* Bb = PL + (t & 1) * kc * jl;
      if (j < k) {
#pragma unroll
        for (int i = 0; i < QMAX; i += 4)
          st4(Bb + j * jl + i0 + i, bc[i], bc[i + 1], bc[i + 2], bc[i + 3]);
      }
      __syncthreads();
      const int pj = (j < k) ? fin_partner(round, j, mm) : k;
      if (pj < k) {  // the four threads of the column take this branch together
        const float* pb = Bb + pj * jl + i0;
        float y[QMAX];
        float aa = 0.f, pp = 0.f, ap = 0.f;
#pragma unroll
        for (int i = 0; i < QMAX; i += 4) {
          const float4 v = ld4(pb + i);
          y[i] = v.x;
          y[i + 1] = v.y;
          y[i + 2] = v.z;
          y[i + 3] = v.w;
        }
        float aa1 = 0.f, pp1 = 0.f, ap1 = 0.f;  // odd rows
#pragma unroll
        for (int i = 0; i < QMAX; i += 2) {
          ffma2(aa, aa1, bc[i], bc[i + 1], bc[i], bc[i + 1]);
          ffma2(pp, pp1, y[i], y[i + 1], y[i], y[i + 1]);
          ffma2(ap, ap1, bc[i], bc[i + 1], y[i], y[i + 1]);
        }
        aa += aa1;
        pp += pp1;
        ap += ap1;
        aa += __shfl_xor_sync(gmask, aa, 1);
        pp += __shfl_xor_sync(gmask, pp, 1);
        ap += __shfl_xor_sync(gmask, ap, 1);
        aa += __shfl_xor_sync(gmask, aa, 2);
        pp += __shfl_xor_sync(gmask, pp, 2);
        ap += __shfl_xor_sync(gmask, ap, 2);
        const bool low = j < pj;  // the lower index is p of the pair (p, q)
        const float alpha = low ? aa : pp, beta = low ? pp : aa, gamma = ap;
        // rotate unless |gamma| <= 4e-6 sqrt(alpha beta) (a zero column
        // gives rsqrt = inf: rotate if gamma != 0, skip if gamma == 0).  The
        // sweeps stop after one whose rotations all had |gamma| <=
        // 2e-3 sqrt(alpha beta): convergence is quadratic by then, so what
        // is left is of the order of the 4e-6 threshold.
        const float meas = fabsf(gamma) * rsqrtf(alpha) * rsqrtf(beta);
        if (meas > 4.0e-6f) {
          const float zeta = __fdividef(beta - alpha, 2.f * gamma);
          const float az = fabsf(zeta), z2 = fmaf(zeta, zeta, 1.f);
          const float hyp = az < 1.0e18f ? z2 * rsqrtf(z2) : az;  // sqrt(1 + zeta^2)
          const float tt = copysignf(__fdividef(1.f, az + hyp), zeta);
          const float cs = rsqrtf(fmaf(tt, tt, 1.f)), sn = tt * cs;
          // [b_p b_q] <- [c b_p - s b_q, s b_p + c b_q]
          const float cp = low ? -sn : sn;
#pragma unroll
          for (int i = 0; i < QMAX; i += 2) {
            float u0, u1;
            fmul2(u0, u1, cp, cp, y[i], y[i + 1]);
            ffma2(u0, u1, cs, cs, bc[i], bc[i + 1]);
            bc[i] = u0;
            bc[i + 1] = u1;
          }
          rot |= meas > 2.0e-3f;
        }
      }
    }
    if (!__syncthreads_or(rot)) break;
  }
  // sigma_j = column norm; the normalised column is an eigenvector (plane 0)
  float* Vs = PL;            // column j at Vs[j * jl + i]
  float* Vc = PL + kc * jl;  // corrected V_r, column c at Vc[c * jl + i]
  {
    float nn = 0.f;
#pragma unroll
    for (int i = 0; i < QMAX; ++i) nn = fmaf(bc[i], bc[i], nn);
    nn += __shfl_xor_sync(0xffffffffu, nn, 1);
    nn += __shfl_xor_sync(0xffffffffu, nn, 2);
    if (j < k) {
      if (qt == 0) lam[j] = nn;
      const float inv = nn > 1.0e-37f ? rsqrtf(nn) : 0.f;
#pragma unroll
      for (int i = 0; i < QMAX; i += 4) {
        float v[4];
#pragma unroll
        for (int z = 0; z < 4; ++z)
          v[z] = (inv > 0.f) ? bc[i + z] * inv : (i0 + i + z == j ? 1.f : 0.f);
        st4(Vs + j * jl + i0 + i, v[0], v[1], v[2], v[3]);
      }
    }
  }
  __syncthreads();
  for (int c = tid; c < k; c += FT) {  // descending eigenvalues
    // NaN ranks below everything (a total order), so `order` is a
    // permutation whatever the values: it indexes shared memory below
    int rank = 0;
    const float lc = lam[c] == lam[c] ? lam[c] : -INFINITY;
    for (int c2 = 0; c2 < k; ++c2) {
      const float l2 = lam[c2] == lam[c2] ? lam[c2] : -INFINITY;
      rank += (l2 > lc) || (l2 == lc && c2 < c);
    }
    order[rank] = c;
  }
  __syncthreads();
  if (md.sigma != nullptr)
    for (int c = tid; c < k; c += FT) ((float*)md.sigma)[c] = sqrtf(lam[order[c]]);
  // V_r <- V_r - V_r E / 2, E = V_r^T V_r - I (E in GC, row stride kc)
  float* E = GC;
  for (int e = tid; e < r * 64; e += FT) {
    const int a = e >> 6, c = e & 63;
    if (c < r) {
      const float* va = Vs + order[a] * jl;
      const float* vc = Vs + order[c] * jl;
      float s2 = (a == c) ? -1.f : 0.f;
      for (int i = 0; i < k; ++i) s2 = fmaf(va[i], vc[i], s2);
      E[a * kc + c] = s2;
    }
  }
  __syncthreads();
  for (int e = tid; e < r * 64; e += FT) {
    const int c = e >> 6, i = e & 63;
    if (i < k) {
      float s2 = 0.f;
      for (int a = 0; a < r; ++a) s2 = fmaf(Vs[order[a] * jl + i], E[a * kc + c], s2);
      Vc[c * jl + i] = fmaf(-0.5f, s2, Vs[order[c] * jl + i]);
    }
  }
  __syncthreads();
  // WS = R_X^{-1} V_r (row stride kc, E is dead); energy tr(V_r^T G_M V_r)
  float* WS = GC;
  double part = 0.0;
  for (int e = tid; e < k * 64; e += FT) {
    const int i = e >> 6, c = e & 63;
    if (c < r) {
      const float* v = Vc + c * jl;
      float gv = 0.f, w = 0.f;
      for (int q = 0; q < k; ++q) gv = fmaf(GA[min(i, q) * gld + max(i, q)], v[q], gv);
      part += (double)v[i] * (double)gv;
      for (int q = i; q < k; ++q) w = fmaf(RI[i * kc + q], v[q], w);  // R_X^{-1} upper
      WS[i * kc + c] = w;
    }
  }
  __syncthreads();
  double epart = 0.0;
  if (tid < r) {
    float sc = 0.f;
    for (int i = 0; i < k; ++i) sc = fmaf(DX[i], fabsf(WS[i * kc + tid]), sc);
    epart = 0x1p-24 * (double)lam[order[tid]] * (double)sc * (double)sc;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    part += __shfl_xor_sync(0xffffffffu, part, o);
    epart += __shfl_xor_sync(0xffffffffu, epart, o);
  }
  if (lane == 0) {
    red[2 + warp] = part;
    red[2 + FW + warp] = epart;
  }
  __syncthreads();
  if (tid == 0) {
    double energy = 0.0, est = 0.0;
    for (int w = 0; w < FW; ++w) {
      energy += red[2 + w];
      est += red[2 + FW + w];
    }
    red[0] = energy;
    red[1] = est;
  }
  __syncthreads();
}

// One CTA per matrix of a class (ids); KC = k rounded up to 8 for every
// matrix of the class, QMAX = fin_quarter(KC).  refine: 0 never, 1 always,
// 2 when est > 1e-3 (||A||^2 - energy) after the unrefined pass.
template <int KC>
__global__ void __launch_bounds__(FT, 4)
finish_kernel(FinLay L, int kp, const int* __restrict__ ids, const MatDev* __restrict__ mats,
              const PanelDev* __restrict__ xpanels, const PanelDev* __restrict__ ypanels,
              float* __restrict__ Wm, const double* __restrict__ normA2,
              double* __restrict__ err, int* __restrict__ flags, int err_mode, double tau,
              int refine, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = (float*)smem_raw;
  constexpr int QMAX = fin_quarter(KC);
  const int b = ids[blockIdx.x], tid = threadIdx.x;
  const MatDev md = mats[b];
  const int k = md.k, r = md.r;
  constexpr int kc = KC, gld = kc + 1, g4 = (kc * gld + 3) & ~3;
  const PanelDev px = xpanels[b], py = ypanels[b];
  float* RI = sm + L.ri;
  float* GA = sm + L.ga;
  float* DV = sm + L.dv;
  float* DX = sm + L.dx;
  double* red = (double*)(sm + L.red);
  float* area = sm + L.area;
  const double tot = normA2[b];
  // ---- R1 = chol(X^T X), R1^{-1} into RI
  FinPass ps;
  ps.P0 = (const float*)px.P;
  ps.rows0 = px.rows;
  ps.out0 = GA;
  ps.P1 = nullptr;
  ps.rows1 = 0;
  ps.out1 = nullptr;
  ps.nseg = 1;
  fin_stream_kc<KC>(L, sm, kp, ps, false);
  for (int i = tid; i < k; i += FT) DX[i] = sqrtf(fmaxf(GA[i * gld + i], 0.f));
  fin_chol(GA, gld, k, DV, true, status);
  fin_rinv(GA, gld, DV, k, kc, RI);
  // ---- G_M (upper) into GA, R_X^{-1} into RI
  float* GB = area;  // a Gram target in the area, row stride gld
  if (refine == 1) {
    ps.P1 = (const float*)py.P;
    ps.rows1 = py.rows;
    ps.out1 = GB;
    ps.nseg = 2;  // Q1 = X R1^{-1}: Gram into GA; M1 = Y R1^{-1}: Gram into GB
    fin_stream_kc<KC>(L, sm, kp, ps, true);
    fin_refine(GA, GB, GA, RI, area, DV, k, kc, gld, g4, status);
  } else {
    ps.P0 = (const float*)py.P;
    ps.rows0 = py.rows;
    ps.out0 = GA;  // M1 = Y R1^{-1}
    fin_stream_kc<KC>(L, sm, kp, ps, true);
  }
  // ---- eigenpairs, W, energy; one refinement afterwards if the bound asks
  for (int pass = 0;; ++pass) {
    fin_eigen<QMAX>(md, k, r, kc, gld, g4, GA, RI, DX, DV, area, red, status);
    const bool again = refine == 2 && pass == 0 && red[1] > 1e-3 * (tot - red[0]);
    if (!again) break;  // uniform: every thread reads the same red[]
    __syncthreads();    // red[] read before it is written again
    ps.P0 = (const float*)px.P;
    ps.rows0 = px.rows;
    ps.out0 = GB;  // Q1 = X R1^{-1}
    ps.nseg = 1;
    fin_stream_kc<KC>(L, sm, kp, ps, true);
    fin_refine(GB, GA, GA, RI, area, DV, k, kc, gld, g4, status);
  }
  // ---- outputs: W (kp x kp, zero outside k x r), err, flags
  const float* WS = area;
  float* Wout = Wm + (long long)b * kp * kp;
  for (int e = tid; e < kp * kp; e += FT) {
    const int i = e / kp, c = e - i * kp;
    Wout[e] = (i < k && c < r) ? WS[i * kc + c] : 0.f;
  }
  if (tid == 0) {
    const double e2 = tot - red[0];
    err[b] = sqrt(e2 > 0.0 ? e2 : 0.0);
    flags[b] = (err_mode == 2) || (err_mode == 0 && e2 < tau * tot);
  }
}

template <int KC>
cudaError_t launch_finish_t(int kp, const int* ids, int count, const MatDev* mats,
                            const PanelDev* xpanels, const PanelDev* ypanels, float* Wm,
                            double* normA2, double* err, int* flags, int err_mode, double tau,
                            int refine, int* status, cudaStream_t s) {
  const FinLay L = fin_layout(KC);
  cudaError_t e = cudaFuncSetAttribute(finish_kernel<KC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
  if (e != cudaSuccess) return e;
  finish_kernel<KC><<<count, FT, L.bytes, s>>>(L, kp, ids, mats, xpanels, ypanels, Wm, normA2,
                                               err, flags, err_mode, tau, refine, status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_finish(int kp, int kc, const int* ids, int count, const MatDev* mats,
                          const PanelDev* xpanels, const PanelDev* ypanels, float* Wm,
                          double* normA2, double* err, int* flags, int err_mode, double tau,
                          int refine, int* status, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (kp % 16 != 0 || kp > TSK_MAX_K || kc > kp || kc < 8 || kc % 8 != 0)
    return cudaErrorInvalidValue;
#define TSK_FIN_CASE(KCV)                                                                   \
  case KCV:                                                                                 \
    return launch_finish_t<KCV>(kp, ids, count, mats, xpanels, ypanels, Wm, normA2, err, flags, \
                                err_mode, tau, refine, status, s);
  switch (kc) {
    TSK_FIN_CASE(8)
    TSK_FIN_CASE(16)
    TSK_FIN_CASE(24)
    TSK_FIN_CASE(32)
    TSK_FIN_CASE(40)
    TSK_FIN_CASE(48)
    TSK_FIN_CASE(56)
    TSK_FIN_CASE(64)
    default:
      return cudaErrorInvalidValue;
  }
#undef TSK_FIN_CASE
}

}  // namespace tsk
