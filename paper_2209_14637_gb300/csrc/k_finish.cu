// Small factors of the FP32 / BF16 test pass (E2 + E4 + E5 of the SCW step,
// Algorithm 1 in the QR form of Section 3.2), one CTA per matrix.
//
// From the panels X (n x k) and Y = A X (m x k) written by the sketch pass:
//
//   R1   = chol(X^T X)                         (X = Q R_X; kappa(X) modest)
//   R2   = chol(Q1^T Q1),  Q1 = X R1^{-1}      (one CholeskyQR2 step)
//   R_X  = R2 R1,  R_X^{-1} = R1^{-1} R2^{-1}
//   G_M  = M^T M,  M = Y R_X^{-1} = A Q        (m x k, well conditioned)
//   sigma_i(AQ)^2 = lambda_i(G_M),  V = eigenvectors,  W = R_X^{-1} V_r
//   err^2 = ||A||^2 - sum_{i<=r} v_i^T G_M v_i (Eq. A.3; Ky Fan)
//
// Y itself is never factored: its columns scale like sigma_i^2 and Y^T Y
// would lose everything in FP32.  Each panel streams through shared memory
// in blocks of FSB rows (a block is one contiguous run: the panels have
// leading dimension kp), brought in by one thread with bulk copies FSTAGES-1
// blocks ahead; the Gram is accumulated in FP32 4 x 4 register tiles; the
// k x k steps run in FP32 in shared memory.  Eigenpairs come from one-sided
// (Hestenes) Jacobi on B = G_M with two threads per column (see the Jacobi
// section below).  Keeping a matrix's whole chain in one CTA removes the
// launches between the steps and the round trips of partial Grams through
// global memory; the SM interleaves the FMA-bound streaming of some CTAs
// with the latency-bound k x k steps of others.
#include <stdint.h>

#include <algorithm>

#include "tsk_internal.cuh"

namespace tsk {

namespace {

constexpr int FT = 128;       // threads per CTA
constexpr int FSB = 32;       // rows per streamed block
constexpr int FSTAGES = 3;    // blocks in flight
constexpr long long FWAIT_NS = 4000000000ll;  // bound on one wait for a block

// Shared-memory layout (offsets in floats, kp = k rounded up to 16 <= 64).
struct FinLay {
  int kp, ld;  // ld = kp + 1 for the k x k work arrays
  int ri;      // R^{-1} of the current transform, kp x kp (row stride kp)
  int stg;     // FSTAGES blocks of FSB x kp
  int ts;      // one transformed block, FSB x (kp + 4)
  int g;       // Gram / Cholesky workspace, kp x ld
  int rf;      // second k x k workspace, kp x ld
  int bars;    // byte offset of FSTAGES mbarriers
  size_t bytes;
};

__host__ __device__ inline FinLay fin_layout(int kp) {
  FinLay L;
  L.kp = kp;
  L.ld = kp + 1;
  int o = 0;
  L.ri = o;
  o += kp * kp;
  L.stg = o;
  o += FSTAGES * FSB * kp;
  L.ts = o;
  o += FSB * (kp + 4);
  L.g = o;
  o += kp * (kp + 1);
  L.rf = o;
  o += kp * (kp + 1);
  o = (o + 1) & ~1;
  L.bars = o * 4;
  L.bytes = (size_t)o * 4 + FSTAGES * sizeof(uint64_t);
  return L;
}

__device__ __forceinline__ uint64_t fin_timer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Upper triangle (4 x 4 tiles) of the Gram of a panel P (rows x kp, columns
// >= k zero) or of P R^{-1} (tr; R^{-1} upper in sm + L.ri) into sm + L.g
// (row stride L.ld).  gb counts the blocks streamed so far by this CTA, so
// the stage and the mbarrier parity of every block follow from it.
__device__ void fin_gram(const FinLay& L, float* sm, uint64_t* bars, const float* P,
                         long long rows, int k, bool tr, long long& gb, int* status,
                         bool& ok) {
  const int kp = L.kp, tid = threadIdx.x;
  float* stg = sm + L.stg;
  float* Ts = sm + L.ts;
  const float* Rs = sm + L.ri;
  const int blk = FSB * kp, ldp = kp + 4;
  const int nblk = (int)((rows + FSB - 1) / FSB);
  auto bar = [&](int s) { return (uint32_t)__cvta_generic_to_shared(bars + s); };
  auto issue = [&](int b) {  // thread 0: block b of this panel
    const int s = (int)((gb + b) % FSTAGES);
    const long long s0 = (long long)b * FSB;
    const uint32_t bytes = (uint32_t)(min((long long)FSB, rows - s0) * kp * sizeof(float));
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar(s)),
                 "r"(bytes)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"((uint32_t)__cvta_generic_to_shared(stg + s * blk)),
        "l"(P + s0 * kp), "r"(bytes), "r"(bar(s))
        : "memory");
  };
  // Earlier generic writes to the stages (scratch) are ordered before the
  // bulk copies that overwrite them.
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (tid == 0 && ok)
    for (int b = 0; b < min(FSTAGES - 1, nblk); ++b) issue(b);
  // Gram tiles: 8 x 4 blocks (8 rows, 4 columns) that meet the upper
  // triangle (column tile j >= 2 x row tile i); several row groups share each
  // tile when there are fewer tiles than threads and are summed at the end
  // (the groups' tiles must fit in the stages and Ts).
  const int nt = kp / 4;       // column tiles (and transform tiles per row)
  const int ntr = kp / 8;      // row tiles
  const int ntiles = ntr * nt - ntr * (ntr - 1);  // sum over i of (nt - 2 i)
  const int room = (FSTAGES * FSB * kp + FSB * (kp + 4)) / (ntiles * 32);
  const int groups = max(1, min(FT / ntiles, 1 + room));
  const bool active = tid < groups * ntiles;
  const int tile = tid % ntiles, grp = tid / ntiles;
  int ty = 0, rem = tile;  // tile -> (ty, tx): row tile ty, column tile tx >= 2 ty
  while (rem >= nt - 2 * ty) {
    rem -= nt - 2 * ty;
    ++ty;
  }
  const int tx = 2 * ty + rem;
  const int rg = tid / nt, cg = tid % nt;  // transform tile: rows 4 rg.., columns 4 cg..
  const bool tact = tr && rg < FSB / 4;
  const int top = min((k + 3) & ~3, 4 * cg + 4);  // R^{-1} is upper: rows < top
  float acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2) acc[a][b2] = 0.f;
  for (int b = 0; b < nblk; ++b) {
    const long long gi = gb + b;
    const int s = (int)(gi % FSTAGES);
    if (tid == 0 && ok && b + FSTAGES - 1 < nblk) issue(b + FSTAGES - 1);  // stage freed
    if (ok) {
      const uint32_t parity = (uint32_t)((gi / FSTAGES) & 1);
      const uint64_t t0 = fin_timer();
      for (;;) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar(s)), "r"(parity)
            : "memory");
        if (done) break;
        if ((long long)(fin_timer() - t0) > FWAIT_NS) {
          atomicOr(status, kStatusTimeout);
          ok = false;
          break;
        }
      }
    }
    const float* Pb = stg + s * blk;
    const int nrows = (int)min((long long)FSB, rows - (long long)b * FSB);
    const float* src = Pb;
    int lds = kp;
    if (tr) {
      if (tact) {  // 4 x 4 tile of Pb R^{-1}, four rows of R^{-1} per step
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
#pragma unroll 2
      for (int ii = grp; ii < nrows; ii += groups) {
        const float4 x0 = *reinterpret_cast<const float4*>(src + ii * lds + ty * 8);
        const float4 x1 = *reinterpret_cast<const float4*>(src + ii * lds + ty * 8 + 4);
        const float4 y4 = *reinterpret_cast<const float4*>(src + ii * lds + tx * 4);
        const float x[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
        const float y[4] = {y4.x, y4.y, y4.z, y4.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b2 = 0; b2 < 4; ++b2) acc[a][b2] = fmaf(x[a], y[b2], acc[a][b2]);
      }
    }
    __syncthreads();  // stage s (and Ts) consumed: stage s may be refilled
  }
  gb += nblk;
  float* Red = stg;  // the row groups' tiles (stages and Ts are free now)
  if (active && grp > 0) {
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) Red[(tid - ntiles) * 32 + a * 4 + b2] = acc[a][b2];
  }
  __syncthreads();
  if (active && grp == 0) {
    for (int g2 = 1; g2 < groups; ++g2) {
      const int t2 = (g2 - 1) * ntiles + tile;
#pragma unroll
      for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int b2 = 0; b2 < 4; ++b2) acc[a][b2] += Red[t2 * 32 + a * 4 + b2];
    }
    float* G = sm + L.g;
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) G[(ty * 8 + a) * L.ld + tx * 4 + b2] = acc[a][b2];
  }
  __syncthreads();
}

// Cholesky of the upper triangle of G (k x k, row stride ld) in place
// (right-looking, FP32) and R^{-1} (upper, zero below the diagonal) into Ri
// (row stride ldr).  A non-positive or tiny pivot raises kStatusRankDef.
__device__ void fin_chol(float* G, int ld, int k, float* Ri, int ldr, int nrows_ri,
                         int* status) {
  __shared__ float inv_d;
  __shared__ int bad;
  const int tid = threadIdx.x;
  for (int e = tid; e < nrows_ri * ldr; e += FT) Ri[e] = 0.f;
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
    for (int c = j + 1 + tid; c < k; c += FT) G[j * ld + c] *= inv_d;
    __syncthreads();
    const int w = k - j - 1;
    for (int e = tid; e < w * w; e += FT) {
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
  for (int c = tid; c < k; c += FT) {  // column c by back substitution
    for (int i = c; i >= 0; --i) {
      float t = (i == c) ? 1.f : 0.f;
      for (int q = i + 1; q <= c; ++q) t = fmaf(-G[i * ld + q], Ri[q * ldr + c], t);
      const float d = G[i * ld + i];
      Ri[i * ldr + c] = (d != 0.f) ? t / d : 0.f;
    }
  }
  __syncthreads();
}

// Partner of column j in round `round` of the round-robin order on kk = 2 m'
// columns (mm = kk - 1): the pairs of a round are (round, mm) and
// (round + i, round - i) mod mm, i = 1 .. kk/2 - 1, so two columns other than
// mm pair up when their indices sum to 2 round mod mm.
__device__ __forceinline__ int fin_partner(int round, int j, int mm) {
  const int r0 = round % mm;
  if (j == mm) return r0;
  if (j == r0) return mm;
  return ((2 * round - j) % mm + mm) % mm;
}

// One CTA per matrix; HMAX >= ceil(k / 2).
template <int HMAX>
__global__ void __launch_bounds__(FT, 4)
finish_kernel(int kp, const MatDev* __restrict__ mats, const PanelDev* __restrict__ xpanels,
              const PanelDev* __restrict__ ypanels, float* __restrict__ Wm,
              const double* __restrict__ normA2, double* __restrict__ err,
              int* __restrict__ flags, int err_mode, double tau, int refine,
              int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* sm = (float*)smem_raw;
  const FinLay L = fin_layout(kp);
  uint64_t* bars = (uint64_t*)(smem_raw + L.bars);
  const int b = blockIdx.x, tid = threadIdx.x;
  const MatDev md = mats[b];
  const int k = md.k, r = md.r;
  const PanelDev px = xpanels[b], py = ypanels[b];
  if (tid == 0) {
    for (int s = 0; s < FSTAGES; ++s)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(
          (uint32_t)__cvta_generic_to_shared(bars + s)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  long long gb = 0;
  bool ok = true;
  float* G = sm + L.g;
  float* RF = sm + L.rf;
  float* RI = sm + L.ri;
  // ---- R1 = chol(X^T X), R1^{-1} into RI
  fin_gram(L, sm, bars, (const float*)px.P, px.rows, k, false, gb, status, ok);
  fin_chol(G, L.ld, k, RI, kp, kp, status);
  if (refine) {
    // ---- R2 = chol(Q1^T Q1), Q1 = X R1^{-1}; R_X^{-1} = R1^{-1} R2^{-1}
    fin_gram(L, sm, bars, (const float*)px.P, px.rows, k, true, gb, status, ok);
    fin_chol(G, L.ld, k, RF, L.ld, kp, status);  // R2^{-1} into RF
    for (int e = tid; e < kp * kp; e += FT) {   // product (upper) into G
      const int i = e / kp, c = e % kp;
      float t = 0.f;
      if (i <= c && c < k)
        for (int q = i; q <= c; ++q) t = fmaf(RI[i * kp + q], RF[q * L.ld + c], t);
      G[i * L.ld + c] = t;
    }
    __syncthreads();
    for (int e = tid; e < kp * kp; e += FT) RI[e] = G[(e / kp) * L.ld + e % kp];
    __syncthreads();
  }
  // ---- G_M = (Y R_X^{-1})^T (Y R_X^{-1}) (upper, in G)
  fin_gram(L, sm, bars, (const float*)py.P, py.rows, k, true, gb, status, ok);

  // ---- eigenpairs of G_M: one-sided Jacobi on B = G_M.  Rotations that
  // make the columns of B mutually orthogonal leave B = G_M V = V Lambda, so
  // the column norms are the eigenvalues and the normalised columns the
  // eigenvectors (whose errors reach the captured energy, a Rayleigh
  // quotient, only at second order).  Two adjacent threads keep the two
  // halves of column j of B in registers; each round of the parallel
  // round-robin order they read their halves of the partner column from
  // shared memory (double-buffered, one barrier per round), add their
  // partial dot products with one shuffle, and all four threads of a pair of
  // columns compute the same rotation from the same three sums.
  const int jl = k + 1;  // row stride of the Jacobi planes
  float* Gs = sm + L.stg;            // G_M, full symmetric
  float* Bs = Gs + k * jl;           // 2 planes
  float* lam = Bs + 2 * k * jl;      // k
  int* order = (int*)(lam + k);      // k
  double* acc = (double*)(order + k);  // FT; float offset stg + 3k(k+1) + 2k is even
  for (int e = tid; e < k * k; e += FT) {
    const int i = e / k, c = e % k;
    Gs[i * jl + c] = G[min(i, c) * L.ld + max(i, c)];
  }
  __syncthreads();
  const int j = tid >> 1, half = tid & 1;
  const int hr = (k + 1) >> 1;
  const int r0h = half * hr;
  const int nh = max(0, min(hr, k - r0h));
  float bc[HMAX];
#pragma unroll
  for (int i = 0; i < HMAX; ++i) bc[i] = (j < k && i < nh) ? Gs[(r0h + i) * jl + j] : 0.f;
  const int kk = k + (k & 1), mm = kk - 1;
  int t = 0;
  for (int sweep = 0; sweep < 12 && mm > 0; ++sweep) {
    int rot = 0;
    for (int round = 0; round < mm; ++round, ++t) {
      float* Bb = Bs + (t & 1) * k * jl;
      if (j < k) {
#pragma unroll
        for (int i = 0; i < HMAX; ++i)
          if (i < nh) Bb[j * jl + r0h + i] = bc[i];
      }
      __syncthreads();
      const int pj = (j < k) ? fin_partner(round, j, mm) : k;
      if (pj < k) {  // both threads of the column take this branch together
        const float* pb = Bb + pj * jl + r0h;
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
  // eigenvalues = column norms; normalised columns = eigenvectors (plane 0)
  float* Vs = Bs;           // column j at Vs[j * jl + i]
  float* Vc = Bs + k * jl;  // corrected V_r, column c at Vc[c * jl + i]
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
        if (i < nh) Vs[j * jl + r0h + i] = (inv > 0.f) ? bc[i] * inv : (r0h + i == j ? 1.f : 0.f);
    }
  }
  __syncthreads();
  for (int c = tid; c < k; c += FT) {  // descending eigenvalues
    int rank = 0;
    for (int c2 = 0; c2 < k; ++c2) rank += (lam[c2] > lam[c]) || (lam[c2] == lam[c] && c2 < c);
    order[rank] = c;
  }
  __syncthreads();
  if (md.sigma != nullptr)
    for (int c = tid; c < k; c += FT) ((float*)md.sigma)[c] = sqrtf(lam[order[c]]);
  // column c < r of V_r (E = V_r^T V_r - I, then V_r <- V_r - V_r E / 2)
  for (int c = tid; c < r; c += FT) {
    const float* vc = Vs + order[c] * jl;
    float e[TSK_MAX_K];
#pragma unroll
    for (int a = 0; a < TSK_MAX_K; ++a) {
      float s2 = 0.f;
      if (a < r) {
        const float* va = Vs + order[a] * jl;
        s2 = (a == c) ? -1.f : 0.f;
        for (int i = 0; i < k; ++i) s2 = fmaf(va[i], vc[i], s2);
      }
      e[a] = s2;
    }
    for (int i = 0; i < k; ++i) {
      float s2 = 0.f;
#pragma unroll
      for (int a = 0; a < TSK_MAX_K; ++a)
        if (a < r) s2 = fmaf(Vs[order[a] * jl + i], e[a], s2);
      Vc[c * jl + i] = fmaf(-0.5f, s2, vc[i]);
    }
  }
  __syncthreads();
  // row i of G V_r and of W = R_X^{-1} V_r; energy tr(V_r^T G V_r)
  double part = 0.0;
  float* Wout = Wm + (long long)b * kp * kp;
  for (int e = tid; e < kp * kp; e += FT) {
    const int i = e / kp, c = e - i * kp;
    float w = 0.f;
    if (i < k && c < r) {
      const float* v = Vc + c * jl;
      float gv = 0.f;
      for (int q = 0; q < k; ++q) gv = fmaf(Gs[i * jl + q], v[q], gv);
      part += (double)v[i] * (double)gv;
      for (int q = i; q < k; ++q) w = fmaf(RI[i * kp + q], v[q], w);  // R_X^{-1} upper
    }
    Wout[e] = w;
  }
  acc[tid] = part;
  __syncthreads();
  if (tid == 0) {
    double energy = 0.0;
    for (int q = 0; q < FT; ++q) energy += acc[q];
    const double tot = normA2[b];
    const double e2 = tot - energy;
    err[b] = sqrt(e2 > 0.0 ? e2 : 0.0);
    flags[b] = (err_mode == 2) || (err_mode == 0 && e2 < tau * tot);
  }
}

template <int HMAX>
cudaError_t launch_finish_t(int kp, const MatDev* mats, int count, const PanelDev* xpanels,
                            const PanelDev* ypanels, float* Wm, double* normA2, double* err,
                            int* flags, int err_mode, double tau, int refine, int* status,
                            cudaStream_t s) {
  const FinLay L = fin_layout(kp);
  cudaError_t e = cudaFuncSetAttribute(finish_kernel<HMAX>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.bytes);
  if (e != cudaSuccess) return e;
  finish_kernel<HMAX><<<count, FT, L.bytes, s>>>(kp, mats, xpanels, ypanels, Wm, normA2, err,
                                                 flags, err_mode, tau, refine, status);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_finish(int kp, int kmax, const MatDev* mats, int count,
                          const PanelDev* xpanels, const PanelDev* ypanels, float* Wm,
                          double* normA2, double* err, int* flags, int err_mode, double tau,
                          int refine, int* status, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  if (kp % 16 != 0 || kp > TSK_MAX_K || kmax > kp) return cudaErrorInvalidValue;
  const int hm = (kmax + 1) / 2;
  if (hm <= 8)
    return launch_finish_t<8>(kp, mats, count, xpanels, ypanels, Wm, normA2, err, flags,
                              err_mode, tau, refine, status, s);
  if (hm <= 16)
    return launch_finish_t<16>(kp, mats, count, xpanels, ypanels, Wm, normA2, err, flags,
                               err_mode, tau, refine, status, s);
  if (hm <= 20)
    return launch_finish_t<20>(kp, mats, count, xpanels, ypanels, Wm, normA2, err, flags,
                               err_mode, tau, refine, status, s);
  if (hm <= 24)
    return launch_finish_t<24>(kp, mats, count, xpanels, ypanels, Wm, normA2, err, flags,
                               err_mode, tau, refine, status, s);
  return launch_finish_t<32>(kp, mats, count, xpanels, ypanels, Wm, normA2, err, flags,
                             err_mode, tau, refine, status, s);
}

}  // namespace tsk
