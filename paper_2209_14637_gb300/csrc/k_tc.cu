// BF16 test pass on the 5th-generation tensor cores (tcgen05 + TMEM + TMA).
//
// One pass over every stream matrix A (m x n, BF16, row-major) computes both
// contractions of the SCW step (Algorithm 1 in the QR form of Section 3.2):
//
//     X = (S A)^T = A^T S^T   (n x k)      and      Y = A X   (m x k),
//
// plus ||A||_F^2, so that A Q = Y R^{-1} once X = Q R is known.  Because
// Y = sum_j A[:, j] X[j, :] is local to a column block of A, each block is
// loaded from HBM once and used twice while it sits in shared memory.
//
// Work split.  A cluster of C CTAs owns one matrix at a time; CTA rank rho
// owns rows [rho*MC, (rho+1)*MC).  For every block of 64 columns:
//   1. TMA loads the CTA's MC x 64 tile (128-byte swizzle) into a stage.
//   2. MMA-X:  D_x(c, j) = sum_i S(c, i) A(i, j) over the CTA's rows
//      (A operand: the CTA's slice of S as BF16, K-major; B operand: the A
//      tile read MN-major), accumulated in TMEM (M = 128 lanes, N = 64).
//   3. The partial D_x of the C CTAs are reduce-scattered through
//      distributed shared memory; each CTA sums 64/C columns, rounds them
//      to BF16 (X~), writes them to X in HBM and into every peer's X~
//      buffer (st.shared::cluster).
//   4. MMA-Y:  D_y(i, c) += sum_j A(i, j) X~(j, c), the same A tile now read
//      K-major, accumulated in TMEM across all column blocks.
// After the last block D_y (the CTA's MC rows of Y) goes to HBM.  Two warps
// meanwhile sum the squares of every tile (Kahan-compensated, FP32 per
// block, FP64 across blocks) for ||A||_F^2.
//
// Y uses the BF16-rounded X~, so the R factor must be taken from X~ too;
// X holds exactly those values.
//
// Every wait on an mbarrier is bounded by %globaltimer; on expiry the
// kernel raises kStatusTimeout in the status word, stops issuing work,
// drains what it issued and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "tsk_internal.cuh"

namespace tsk {

namespace {

constexpr int NB = 64;         // columns of A per block (one 128-byte row)
constexpr int MC = 512;        // rows of A per CTA
constexpr int NST = 2;         // A stages
constexpr int KPAD_MAX = 48;   // largest padded k this kernel takes
constexpr int NTHREADS = 288;  // 9 warps
constexpr int BOX_ROWS = 256;  // TMA box height (hardware limit 256)

constexpr int STAGE_BYTES = MC * 128;
constexpr int OFF_A = 0;
constexpr int OFF_S = OFF_A + NST * STAGE_BYTES;
constexpr int S_BYTES = (MC / 64) * KPAD_MAX * 128;
constexpr int P_ROW = 272;  // 64 floats + 16 bytes of padding per row
constexpr int P_BYTES = KPAD_MAX * P_ROW;
constexpr int XB_BYTES = 2 * KPAD_MAX * 128;  // X_hi rows, then X_lo rows
constexpr int OFF_XB = OFF_S + S_BYTES;
constexpr int OFF_P = OFF_XB + 2 * XB_BYTES;
constexpr int OFF_BAR = OFF_P + 2 * P_BYTES;
constexpr int BAR_BYTES = 256;
// The kernel declares no static shared variables, so its dynamic shared
// memory starts on a 1024-byte boundary; the kernel checks this and reports
// misalignment instead of reserving slack.
constexpr int SMEM_BYTES = OFF_BAR + BAR_BYTES;
// MMA-X reads 128 rows of S per 64-row chunk although only kpad rows are
// real; the extra rows (whose results are never used) must stay inside the
// allocation: from the last chunk they reach at most 16 KB past its start.
static_assert(OFF_S + (MC / 64 - 1) * KPAD_MAX * 128 + 128 * 128 <= OFF_BAR,
              "S over-read leaves the shared-memory allocation");
static_assert(SMEM_BYTES <= 227 * 1024, "shared memory budget");
static_assert(OFF_S % 1024 == 0 && OFF_XB % 1024 == 0 && XB_BYTES % 1024 == 0 &&
                  STAGE_BYTES % 1024 == 0,
              "swizzled operands need 1024-byte aligned atoms");
static_assert(OFF_P % 16 == 0 && OFF_BAR % 8 == 0, "alignment");

// barrier slots
enum {
  B_AFULL = 0,
  B_AEMPTY = B_AFULL + NST,
  B_XFULL = B_AEMPTY + NST,
  B_XTEMPTY = B_XFULL + 2,
  B_PFULL = B_XTEMPTY + 2,
  B_PEMPTY = B_PFULL + 2,
  B_XBFULL = B_PEMPTY + 2,
  B_XBEMPTY = B_XBFULL + 2,
  B_YFULL = B_XBEMPTY + 2,
  B_YFREE = B_YFULL + 1,
  B_SFULL = B_YFREE + 1,
  B_SEMPTY = B_SFULL + 1,
  B_DRAIN = B_SEMPTY + 1,
  B_DRAIN2 = B_DRAIN + 1,
  B_COUNT = B_DRAIN2 + 1
};
static_assert(B_COUNT * 8 + 16 <= BAR_BYTES, "barrier area");

struct TcParams {
  const MatDev* mats;
  const CUtensorMap* tmaps;   // one per matrix of the plan
  const int* work;            // matrix ids, grouped by cluster
  const int* work_off;        // nclusters + 1 offsets into work
  const unsigned char* simg;  // pre-swizzled BF16 images of S
  const long long* simg_off;  // per matrix: byte offset of its rank-0 image
  float* X;
  float* Y;
  double* normA2;
  int* status;
  int kp;          // leading dimension of the X / Y panels
  int kpad;        // N of MMA-Y: padded k of this launch (16, 32 or 48)
  int img_rank_bytes;
  long long timeout_ns;
};

// ---- PTX wrappers ---------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint32_t cluster_id() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ uint64_t globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile(
      "mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr)
      : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
      "r"(bytes)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}
// Orders generic-proxy shared-memory writes before later async-proxy
// (tensor-core) reads of the same memory.
__device__ __forceinline__ void fence_proxy_async_cta() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void named_bar(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
               "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map,
                                            int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src,
                                          uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"((uint64_t)src), "r"(bytes), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void ld_cluster_v4(uint32_t addr, float& a, float& b,
                                              float& c, float& d) {
  asm volatile("ld.shared::cluster.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(a), "=f"(b), "=f"(c), "=f"(d)
               : "r"(addr)
               : "memory");
}
// tcgen05
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          bar)
      : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, "
      "%9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
        "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor, 128-byte swizzle (SM100 layout).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= 1ull << 46;  // descriptor version for tcgen05
  d |= 2ull << 61;  // SWIZZLE_128B
  return d;
}
// Instruction descriptor, kind::f16 with BF16 inputs and FP32 accumulation.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) |
         ((uint32_t)b_mn << 16) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

struct Ctl {
  int abort;
};

// Bounded wait.  Returns false on timeout (after raising the status bit and
// the CTA-wide abort flag) or when the CTA is already aborting.
__device__ __forceinline__ bool bwait(uint32_t bar, uint32_t parity, volatile Ctl* ctl,
                                      const TcParams& P) {
  if (ctl->abort) return false;
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = globaltimer();
  for (uint32_t i = 1;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 0) {
      if (ctl->abort) return false;
      if ((long long)(globaltimer() - t0) > P.timeout_ns) {
        atomicOr(P.status, kStatusTimeout);
        ctl->abort = 1;
        return false;
      }
    }
  }
}
// Warp-uniform bounded wait: lane 0 polls, the verdict is broadcast, and the
// warp leaves converged (the tcgen05.ld that follows is .sync.aligned).
__device__ __forceinline__ bool bwait_warp(uint32_t bar, uint32_t parity, volatile Ctl* ctl,
                                           const TcParams& P) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = bwait(bar, parity, ctl, P) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  return ok != 0;
}
// Bounded wait that ignores the abort flag (used to drain own copies).
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity,
                                           const TcParams& P) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if ((long long)(globaltimer() - t0) > P.timeout_ns) {
      atomicOr(P.status, kStatusTimeout);
      return;
    }
  }
}

// Sum of squares of one A stage (MC x 64 BF16), shared by 128 threads
// (t = 0..127).  Eight independent FP32 accumulators per thread, each summing
// 32 squares per stage, keep the dependent chains short; stages are summed
// in FP64.
__device__ __forceinline__ double stage_sumsq(const unsigned char* stage, int t) {
  const uint4* st = reinterpret_cast<const uint4*>(stage);
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = 0.f;
#pragma unroll 4
  for (int e = t; e < STAGE_BYTES / 16; e += 128) {
    const uint4 w = st[e];
    const uint32_t ww[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float lo = __uint_as_float(ww[i] << 16);
      const float hi = __uint_as_float(ww[i] & 0xFFFF0000u);
      a[2 * i] = fmaf(lo, lo, a[2 * i]);
      a[2 * i + 1] = fmaf(hi, hi, a[2 * i + 1]);
    }
  }
  return (double)((a[0] + a[1]) + (a[2] + a[3])) + (double)((a[4] + a[5]) + (a[6] + a[7]));
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<const uint32_t*>(&v);
}

template <int C>
__global__ void __launch_bounds__(NTHREADS, 1)
sketch_tc_kernel(const __grid_constant__ TcParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw;
  const uint32_t sb = smem_u32(sm);  // 1024-aligned shared address
  if (sb & 1023) {  // every CTA of the launch sees the same layout
    if (threadIdx.x == 0) atomicOr(P.status, kStatusTimeout);
    return;
  }
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = (C > 1) ? cluster_rank() : 0;
  const uint32_t cid = (C > 1) ? cluster_id() : blockIdx.x;
  const int kpad = P.kpad;
  auto bar = [&](int i) -> uint32_t { return sb + OFF_BAR + 8 * i; };
  volatile Ctl* ctl = (volatile Ctl*)(sm + OFF_BAR + 8 * B_COUNT);
  uint32_t* tmem_slot = (uint32_t*)(sm + OFF_BAR + 8 * B_COUNT + 8);

  const int w0 = P.work_off[cid], w1 = P.work_off[cid + 1];
  const uint32_t tmem_cols_needed = 2 * NB + (MC / 128) * 2 * kpad;
  const uint32_t tmem_cols = tmem_cols_needed <= 256 ? 256 : 512;

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(bar(B_AFULL + s), 1);
      mbar_init(bar(B_AEMPTY + s), 5);  // MMA-Y commit + four norm warps
    }
    for (int h = 0; h < 2; ++h) {
      mbar_init(bar(B_XFULL + h), 1);
      mbar_init(bar(B_XTEMPTY + h), 2);
      mbar_init(bar(B_PFULL + h), C);
      mbar_init(bar(B_PEMPTY + h), C);
      mbar_init(bar(B_XBFULL + h), 1);   // own epilogue built X~ locally
      mbar_init(bar(B_XBEMPTY + h), 1);  // own MMA-Y finished reading it
    }
    mbar_init(bar(B_YFULL), 1);
    mbar_init(bar(B_YFREE), 4);
    mbar_init(bar(B_SFULL), 1);
    mbar_init(bar(B_SEMPTY), 1);
    mbar_init(bar(B_DRAIN), 1);
    mbar_init(bar(B_DRAIN2), 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // X~ rows beyond k must read as zero in every MMA-Y.
  for (int e = tid; e < 2 * XB_BYTES / 16; e += NTHREADS)
    reinterpret_cast<uint4*>(sm + OFF_XB)[e] = make_uint4(0, 0, 0, 0);
  fence_proxy_async_cta();
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  if (C > 1) cluster_sync();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc_x = idesc_bf16(128, NB, 0, 1);
  const uint32_t idesc_y = idesc_bf16(128, 2 * kpad, 0, 0);

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      long long g = 0;
      int sloads = 0;
      const unsigned char* cur_img = nullptr;
      bool stop = false;
      for (int wi = w0; wi < w1 && !stop; ++wi) {
        const int d = P.work[wi];
        const MatDev& md = P.mats[d];
        const unsigned char* img = P.simg + P.simg_off[d] + (long long)rank * P.img_rank_bytes;
        if (img != cur_img) {
          if (sloads > 0 && !bwait(bar(B_SEMPTY), (sloads - 1) & 1, ctl, P)) {
            stop = true;
            break;
          }
          mbar_expect_tx(bar(B_SFULL), (uint32_t)P.img_rank_bytes);
          bulk_load(sb + OFF_S, img, (uint32_t)P.img_rank_bytes, bar(B_SFULL));
          ++sloads;
          cur_img = img;
        }
        const CUtensorMap* map = P.tmaps + d;
        const int nblk = (int)((md.n + NB - 1) / NB);
        for (int q = 0; q < nblk; ++q, ++g) {
          const int s = (int)(g % NST);
          const uint32_t u = (uint32_t)(g / NST);
          if (!bwait(bar(B_AEMPTY + s), (u & 1) ^ 1, ctl, P)) {
            stop = true;
            break;
          }
          mbar_expect_tx(bar(B_AFULL + s), STAGE_BYTES);
#pragma unroll
          for (int b = 0; b < MC / BOX_ROWS; ++b)
            tma_load_2d(sb + OFF_A + s * STAGE_BYTES + b * BOX_ROWS * 128, map, q * NB,
                        (int)(rank * MC + b * BOX_ROWS), bar(B_AFULL + s));
        }
      }
      // Drain: every load this thread issued must land before the CTA exits.
      for (int s = 0; s < NST; ++s) {
        if (g > s) {
          const long long last = ((g - 1 - s) / NST) * NST + s;
          drain_wait(bar(B_AFULL + s), (uint32_t)((last / NST) & 1), P);
        }
      }
      if (sloads > 0) drain_wait(bar(B_SFULL), (sloads - 1) & 1, P);
    }
  } else if (warp == 1 || warp == 8) {
    // ------------------------------- MMA issuers: warp 1 -> MMA-X, warp 8 -> MMA-Y
    // MMA-X of block g+1 must not wait for the exchange of block g, so the
    // two contractions are issued from different warps (a thread suspended in
    // an mbarrier wait would also hold up a sibling lane of its own warp);
    // each issuer commits and drains only its own tcgen05 operations.
    if (warp == 1 && lane == 0) {
      long long g = 0;
      int swaits = 0;
      const unsigned char* cur_img = nullptr;
      bool ok = true;
      for (int wi = w0; wi < w1 && ok; ++wi) {
        const int d = P.work[wi];
        const MatDev& md = P.mats[d];
        const unsigned char* img = P.simg + P.simg_off[d] + (long long)rank * P.img_rank_bytes;
        if (img != cur_img) {
          if (!bwait(bar(B_SFULL), swaits & 1, ctl, P)) {
            ok = false;
            break;
          }
          ++swaits;
          cur_img = img;
        }
        const unsigned char* next_img =
            (wi + 1 < w1) ? P.simg + P.simg_off[P.work[wi + 1]] +
                                (long long)rank * P.img_rank_bytes
                          : img;
        const int nblk = (int)((md.n + NB - 1) / NB);
        for (int q = 0; q < nblk && ok; ++q, ++g) {
          const int s = (int)(g % NST);
          const uint32_t u = (uint32_t)(g / NST);
          const int h = (int)(g & 1);
          const uint32_t v = (uint32_t)(g >> 1);
          if (!bwait(bar(B_AFULL + s), u & 1, ctl, P) ||
              !bwait(bar(B_XTEMPTY + h), (v & 1) ^ 1, ctl, P)) {
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll 4
          for (int kk = 0; kk < MC / 16; ++kk) {
            const uint64_t a =
                sdesc(sb + OFF_S + (kk >> 2) * kpad * 128 + (kk & 3) * 32, 16, 1024);
            const uint64_t b = sdesc(sb + OFF_A + s * STAGE_BYTES + kk * 16 * 128,
                                     BOX_ROWS * 128, 1024);
            tc_mma(tmem + h * NB, a, b, idesc_x, kk > 0 ? 1u : 0u);
          }
          tc_commit(bar(B_XFULL + h));
          if (q == nblk - 1 && next_img != img) tc_commit(bar(B_SEMPTY));
        }
      }
      tc_commit(bar(B_DRAIN));
      drain_wait(bar(B_DRAIN), 0, P);
    } else if (warp == 8 && lane == 0) {
      long long g = 0;
      int mi = 0;
      bool ok = true;
      for (int wi = w0; wi < w1 && ok; ++wi, ++mi) {
        const MatDev& md = P.mats[P.work[wi]];
        const int nblk = (int)((md.n + NB - 1) / NB);
        for (int q = 0; q < nblk && ok; ++q, ++g) {
          const int s = (int)(g % NST);
          const uint32_t u = (uint32_t)(g / NST);
          const int h = (int)(g & 1);
          const uint32_t v = (uint32_t)(g >> 1);
          if (!bwait(bar(B_AFULL + s), u & 1, ctl, P) ||
              !bwait(bar(B_XBFULL + h), v & 1, ctl, P) ||
              (q == 0 && mi > 0 && !bwait(bar(B_YFREE), (mi - 1) & 1, ctl, P))) {
            ok = false;
            break;
          }
          fence_proxy_async_cta();
          tc_fence_after();
#pragma unroll 1
          for (int t = 0; t < MC / 128; ++t) {
#pragma unroll
            for (int kk = 0; kk < NB / 16; ++kk) {
              const uint64_t a =
                  sdesc(sb + OFF_A + s * STAGE_BYTES + t * 128 * 128 + kk * 32, 16, 1024);
              const uint64_t b = sdesc(sb + OFF_XB + h * XB_BYTES + kk * 32, 16, 1024);
              tc_mma(tmem + 2 * NB + t * 2 * kpad, a, b, idesc_y, (q > 0 || kk > 0) ? 1u : 0u);
            }
          }
          tc_commit(bar(B_AEMPTY + s));
          tc_commit(bar(B_XBEMPTY + h));
          if (q == nblk - 1) tc_commit(bar(B_YFULL));
        }
      }
      tc_commit(bar(B_DRAIN2));
      drain_wait(bar(B_DRAIN2), 0, P);
    }
  } else if (warp >= 2 && warp <= 5) {
    // ------- X exchange (warps 4, 5) or ||A||^2 (warps 2, 3), then Y out (all four)
    const int lane_base = (warp & 3) * 32;
    const bool xwarp = (warp >= 4);
    double tot = 0.0;
    const int c = lane_base + lane;  // TMEM lane = row c of D_x / row of D_y tile
    long long g = 0;
    int mi = 0;
    constexpr int WC = NB / C;  // columns of X this CTA writes to HBM
    for (int wi = w0; wi < w1; ++wi, ++mi) {
      const int d = P.work[wi];
      const MatDev& md = P.mats[d];
      const int k = md.k;
      const long long n = md.n, m = md.m;
      const int nblk = (int)((n + NB - 1) / NB);
      for (int q = 0; q < nblk; ++q, ++g) {
        if (!xwarp) {
          const int s = (int)(g % NST);
          const uint32_t u = (uint32_t)(g / NST);
          if (bwait_warp(bar(B_AFULL + s), u & 1, ctl, P))
            tot += stage_sumsq(sm + OFF_A + s * STAGE_BYTES, tid - 64);
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(B_AEMPTY + s));
          continue;
        }
        const int h = (int)(g & 1);
        const uint32_t v = (uint32_t)(g >> 1);
        // publish this CTA's partial D_x rows, 16 columns at a time (peers
        // read them once they have all arrived on this CTA's PFULL)
        bwait(bar(B_PEMPTY + h), (v & 1) ^ 1, ctl, P);
        float* prow = (float*)(sm + OFF_P + h * P_BYTES + c * P_ROW);
        if (bwait_warp(bar(B_XFULL + h), v & 1, ctl, P)) {
          tc_fence_after();
#pragma unroll 1
          for (int j = 0; j < NB; j += 16) {
            float xr[16];
            tmem_ld16(tmem + ((uint32_t)lane_base << 16) + h * NB + j, xr);
            tmem_wait_ld();
            if (c < k) {
#pragma unroll
              for (int e = 0; e < 16; e += 4)
                *reinterpret_cast<float4*>(prow + j + e) =
                    make_float4(xr[e], xr[e + 1], xr[e + 2], xr[e + 3]);
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_XTEMPTY + h));
        // The CTA barrier orders both warps' writes before one thread's
        // cluster-scope release arrive, which publishes them to the peers.
        named_bar(1, 64);
        if (warp == 4 && lane == 0) {
          const uint32_t pf = bar(B_PFULL + h);
#pragma unroll
          for (int r = 0; r < C; ++r) mbar_arrive_cluster(mapa(pf, r));
        }
        bwait(bar(B_PFULL + h), v & 1, ctl, P);
        // X row c of this block = sum of the C partials (every CTA forms the
        // whole block itself: one round trip instead of reduce + gather).
        // Two-term BF16 split X = X_hi + X_lo (X_hi = BF16(X), X_lo =
        // BF16(X - X_hi)); MMA-Y multiplies A by both, so Y = A (X_hi + X_lo)
        // carries about 16 significant bits of X instead of 8.  X in HBM
        // holds X_hi + X_lo, the values Y is built from.  Done 16 columns at
        // a time to bound register use.
        bwait(bar(B_XBEMPTY + h), (v & 1) ^ 1, ctl, P);
        if (c < k) {
          const uint32_t src = smem_u32(prow);
          float* Xm = P.X + md.offX;
#pragma unroll 1
          for (int qb = 0; qb < 4; ++qb) {
            float acc[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) acc[j] = 0.f;
#pragma unroll
            for (int r = 0; r < C; ++r) {
              const uint32_t ra = mapa(src + qb * 64, r);
#pragma unroll
              for (int j = 0; j < 16; j += 4) {
                float a0, a1, a2, a3;
                ld_cluster_v4(ra + j * 4, a0, a1, a2, a3);
                acc[j] += a0;
                acc[j + 1] += a1;
                acc[j + 2] += a2;
                acc[j + 3] += a3;
              }
            }
            uint32_t phi[8], plo[8];
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
              const __nv_bfloat16 h0 = __float2bfloat16_rn(acc[j]);
              const __nv_bfloat16 h1 = __float2bfloat16_rn(acc[j + 1]);
              const float f0 = __bfloat162float(h0), f1 = __bfloat162float(h1);
              const __nv_bfloat16 l0 = __float2bfloat16_rn(acc[j] - f0);
              const __nv_bfloat16 l1 = __float2bfloat16_rn(acc[j + 1] - f1);
              acc[j] = f0 + __bfloat162float(l0);
              acc[j + 1] = f1 + __bfloat162float(l1);
              __nv_bfloat162 hh, ll;
              hh.x = h0;
              hh.y = h1;
              ll.x = l0;
              ll.y = l1;
              phi[j / 2] = *reinterpret_cast<const uint32_t*>(&hh);
              plo[j / 2] = *reinterpret_cast<const uint32_t*>(&ll);
            }
            const long long jb = (long long)q * NB + qb * 16;
#pragma unroll
            for (int j = 0; j < 16; ++j) {  // this CTA's 64/C columns go to HBM
              const long long jj = jb + j;
              if ((qb * 16 + j) / WC == (int)rank && jj < n) Xm[jj * P.kp + c] = acc[j];
            }
#pragma unroll
            for (int half = 0; half < 2; ++half) {
              const int row = c + half * kpad;
              const uint32_t* w = half ? plo : phi;
              unsigned char* xrow =
                  sm + OFF_XB + h * XB_BYTES + (row >> 3) * 1024 + (row & 7) * 128;
#pragma unroll
              for (int u = 0; u < 2; ++u) {
                const int unit = qb * 2 + u;
                *reinterpret_cast<uint4*>(xrow + (((unit ^ (row & 7)) & 7) << 4)) =
                    make_uint4(w[u * 4], w[u * 4 + 1], w[u * 4 + 2], w[u * 4 + 3]);
              }
            }
          }
        }
        fence_proxy_async_cta();
        named_bar(1, 64);
        if (warp == 4 && lane == 0) {
          // peers' partials are consumed: they may reuse their P buffers
          const uint32_t pe = bar(B_PEMPTY + h);
#pragma unroll
          for (int r = 0; r < C; ++r) mbar_arrive_cluster(mapa(pe, r));
        }
        if (warp == 4 && lane == 0) mbar_arrive(bar(B_XBFULL + h));
      }
      if (!xwarp) {
        tot = warp_sum(tot);
        if (lane == 0) atomicAdd(P.normA2 + d, tot);
        tot = 0.0;
      }
      // ---- Y epilogue for this matrix: the CTA's MC rows of Y = A X~
      if (bwait_warp(bar(B_YFULL), mi & 1, ctl, P)) {
        tc_fence_after();
        float* Ym = P.Y + md.offY;
#pragma unroll 1
        for (int t = 0; t < MC / 128; ++t) {
          const long long row = (long long)rank * MC + t * 128 + lane_base + lane;
#pragma unroll 1
          for (int j = 0; j < kpad; j += 16) {
            float yv[16], yl[16];
            const uint32_t col = tmem + ((uint32_t)lane_base << 16) + 2 * NB + t * 2 * kpad + j;
            tmem_ld16(col, yv);
            tmem_ld16(col + kpad, yl);
            tmem_wait_ld();
            if (row < m) {
              float4* dst = reinterpret_cast<float4*>(Ym + row * P.kp + j);
#pragma unroll
              for (int e = 0; e < 4; ++e)
                dst[e] = make_float4(yv[4 * e] + yl[4 * e], yv[4 * e + 1] + yl[4 * e + 1],
                                     yv[4 * e + 2] + yl[4 * e + 2], yv[4 * e + 3] + yl[4 * e + 3]);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_YFREE));
    }
    // Peers read this CTA's partials until they arrive on PEMPTY: wait for
    // the last phase of each buffer before leaving.
    if (xwarp && g > 0) {
      for (int h = 0; h < 2; ++h) {
        if (g > h) {
          const long long last = ((g - 1 - h) / 2) * 2 + h;
          drain_wait(bar(B_PEMPTY + h), (uint32_t)((last >> 1) & 1), P);
        }
      }
    }
  } else {
    // ------------------------------------------------ ||A||_F^2 (warps 6, 7)
    long long g = 0;
    for (int wi = w0; wi < w1; ++wi) {
      const int d = P.work[wi];
      const MatDev& md = P.mats[d];
      const int nblk = (int)((md.n + NB - 1) / NB);
      double tot = 0.0;
      for (int q = 0; q < nblk; ++q, ++g) {
        const int s = (int)(g % NST);
        const uint32_t u = (uint32_t)(g / NST);
        if (bwait_warp(bar(B_AFULL + s), u & 1, ctl, P))
          tot += stage_sumsq(sm + OFF_A + s * STAGE_BYTES, tid - 128);
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_AEMPTY + s));
      }
      tot = warp_sum(tot);
      if (lane == 0) atomicAdd(P.normA2 + d, tot);
    }
  }

  // ---- teardown: nobody leaves while a peer may still touch its memory
  tc_fence_before();
  __syncthreads();
  if (C > 1) cluster_sync();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
  }
}

// Pre-swizzled BF16 image of S for every (distinct sketch, cluster rank):
// the exact shared-memory layout the MMA-X A operand reads (K-major,
// 128-byte swizzle, one 64-column chunk of k_pad rows after another).
struct SImgDesc {
  const float* S;
  long long m;
  int k;
  int pad;
  long long off;
};

__global__ void simg_prep_kernel(const SImgDesc* __restrict__ descs, int kpad,
                                 int img_rank_bytes, unsigned char* __restrict__ simg) {
  const SImgDesc sd = descs[blockIdx.x];
  const int rank = blockIdx.y;
  unsigned char* img = simg + sd.off + (long long)rank * img_rank_bytes;
  const int nunits = (MC / 64) * kpad * 8;
  for (int e = threadIdx.x; e < nunits; e += blockDim.x) {
    const int qc = e / (kpad * 8);
    const int rem = e % (kpad * 8);
    const int c = rem / 8, u = rem % 8;
    uint32_t w[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float v2[2];
#pragma unroll
      for (int z = 0; z < 2; ++z) {
        const long long i = (long long)rank * MC + qc * 64 + u * 8 + 2 * t + z;
        v2[z] = (c < sd.k && i < sd.m) ? sd.S[(long long)c * sd.m + i] : 0.f;
      }
      w[t] = pack_bf16x2(v2[0], v2[1]);
    }
    uint4* dst = reinterpret_cast<uint4*>(img + qc * kpad * 128 + (c >> 3) * 1024 +
                                          (c & 7) * 128 + (((u ^ (c & 7)) & 7) << 4));
    *dst = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                         cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

template <int C>
cudaError_t set_attrs() {
  cudaError_t e = cudaFuncSetAttribute(sketch_tc_kernel<C>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       SMEM_BYTES);
  return e;
}

template <int C>
int max_clusters() {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(C * 256, 1, 1);
  cfg.blockDim = dim3(NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, sketch_tc_kernel<C>, &cfg) != cudaSuccess || n < 1) {
    cudaGetLastError();
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    n = std::max(1, sms / C);
  }
  return n;
}

template <int C>
cudaError_t launch_class(const TcParams& prm, int nclusters, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(C * nclusters, 1, 1);
  cfg.blockDim = dim3(NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = SMEM_BYTES;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sketch_tc_kernel<C>, prm);
}

}  // namespace

struct TcClass {
  int C;
  int nclusters;
  TcParams prm;
};

struct TcPlan {
  void* dev = nullptr;
  size_t bytes = 0;
  std::vector<TcClass> classes;
  const SImgDesc* d_sdesc = nullptr;
  int nsdesc = 0;
  int kpad = 16;
  int img_rank_bytes = 0;
  int cmax = 1;
  unsigned char* simg = nullptr;
};

bool tc_supported() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return false;
  return p.major == 10 && p.minor == 3 && get_encode() != nullptr;
}

cudaError_t tc_prepare(TcPlan** out, const MatDev* hm, const MatDev* d_mats, int count,
                       int kp, void* dev_X, void* dev_Y, double* dev_normA2,
                       int* status, long long spin_limit, char* msg, int msglen) {
  *out = nullptr;
  auto fail = [&](const char* why) {
    if (msg && msglen > 0) snprintf(msg, msglen, "%s", why);
    return cudaErrorNotSupported;
  };
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return fail("cuTensorMapEncodeTiled is unavailable");
  int kmax = 1;
  for (int i = 0; i < count; ++i) {
    if (hm[i].k > KPAD_MAX) return fail("k > 48 is not supported by the tensor-core kernel");
    if (hm[i].m > 8LL * MC) return fail("m > 4096 is not supported by the tensor-core kernel");
    kmax = std::max(kmax, hm[i].k);
  }
  TcPlan* p = new TcPlan();
  p->kpad = ((kmax + 15) / 16) * 16;
  p->img_rank_bytes = (MC / 64) * p->kpad * 128;
  // classes by cluster size
  std::map<int, std::vector<int>> byC;
  for (int i = 0; i < count; ++i) {
    const long long m = hm[i].m;
    const int C = m <= MC ? 1 : (m <= 2 * MC ? 2 : (m <= 4 * MC ? 4 : 8));
    byC[C].push_back(i);
    p->cmax = std::max(p->cmax, C);
  }
  // distinct sketch images
  std::map<std::tuple<const void*, long long, int>, long long> img_of;
  std::vector<SImgDesc> sdesc;
  std::vector<long long> simg_off(count);
  long long img_total = 0;
  for (int i = 0; i < count; ++i) {
    auto key = std::make_tuple(hm[i].S, hm[i].m, hm[i].k);
    auto it = img_of.find(key);
    if (it == img_of.end()) {
      const int C = hm[i].m <= MC ? 1 : (hm[i].m <= 2 * MC ? 2 : (hm[i].m <= 4 * MC ? 4 : 8));
      SImgDesc sd;
      sd.S = (const float*)hm[i].S;
      sd.m = hm[i].m;
      sd.k = hm[i].k;
      sd.pad = C;
      sd.off = img_total;
      img_total += (long long)p->cmax * p->img_rank_bytes;
      it = img_of.emplace(key, sd.off).first;
      sdesc.push_back(sd);
    }
    simg_off[i] = it->second;
  }
  // schedules: longest-processing-time-first over clusters of each class
  std::vector<int> work, work_off_all;
  struct ClassTmp {
    int C, ncl;
    size_t woff_start, work_start;
  };
  std::vector<ClassTmp> ctmp;
  for (auto& kv : byC) {
    const int C = kv.first;
    std::vector<int> ids = kv.second;
    int ncl = 1;
    cudaError_t ae = cudaSuccess;
    switch (C) {
      case 1: ae = set_attrs<1>(); if (ae == cudaSuccess) ncl = max_clusters<1>(); break;
      case 2: ae = set_attrs<2>(); if (ae == cudaSuccess) ncl = max_clusters<2>(); break;
      case 4: ae = set_attrs<4>(); if (ae == cudaSuccess) ncl = max_clusters<4>(); break;
      default: ae = set_attrs<8>(); if (ae == cudaSuccess) ncl = max_clusters<8>(); break;
    }
    if (ae != cudaSuccess) {
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (msg)
        snprintf(msg, msglen,
                 "cudaFuncSetAttribute(%d bytes of shared memory) failed: %s (device opt-in "
                 "limit %d bytes)",
                 SMEM_BYTES, cudaGetErrorString(ae), optin);
      cudaGetLastError();
      delete p;
      return ae;
    }
    ncl = std::min<int>(ncl, (int)ids.size());
    std::sort(ids.begin(), ids.end(), [&](int a, int b) {
      return hm[a].m * hm[a].n > hm[b].m * hm[b].n;
    });
    std::vector<std::vector<int>> lists(ncl);
    std::vector<long long> load(ncl, 0);
    for (int id : ids) {
      const int best = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      lists[best].push_back(id);
      load[best] += ((hm[id].n + NB - 1) / NB);
    }
    ClassTmp ct;
    ct.C = C;
    ct.ncl = ncl;
    ct.woff_start = work_off_all.size();
    ct.work_start = work.size();
    for (int c = 0; c < ncl; ++c) {
      work_off_all.push_back((int)(work.size() - ct.work_start));
      for (int id : lists[c]) work.push_back(id);
    }
    work_off_all.push_back((int)(work.size() - ct.work_start));
    ctmp.push_back(ct);
  }
  // one device allocation: tensor maps | simg offsets | work | offsets | sdesc | images
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  size_t o = 0;
  const size_t o_map = o;
  o = al(o + sizeof(CUtensorMap) * count);
  const size_t o_soff = o;
  o = al(o + sizeof(long long) * count);
  const size_t o_work = o;
  o = al(o + sizeof(int) * work.size());
  const size_t o_woff = o;
  o = al(o + sizeof(int) * work_off_all.size());
  const size_t o_sd = o;
  o = al(o + sizeof(SImgDesc) * sdesc.size());
  const size_t o_img = o;
  o = al(o + img_total);
  p->bytes = o;
  cudaError_t e = cudaMalloc(&p->dev, p->bytes);
  if (e != cudaSuccess) {
    delete p;
    if (msg) snprintf(msg, msglen, "workspace");
    return e;
  }
  std::vector<unsigned char> host(o_img, 0);
  for (int i = 0; i < count; ++i) {
    CUtensorMap* map = reinterpret_cast<CUtensorMap*>(host.data() + o_map) + i;
    cuuint64_t dims[2] = {(cuuint64_t)hm[i].n, (cuuint64_t)hm[i].m};
    cuuint64_t strides[1] = {(cuuint64_t)hm[i].lda * 2};
    cuuint32_t box[2] = {(cuuint32_t)NB, (cuuint32_t)BOX_ROWS};
    cuuint32_t es[2] = {1, 1};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(hm[i].A),
                     dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      cudaFree(p->dev);
      delete p;
      if (msg) snprintf(msg, msglen, "cuTensorMapEncodeTiled failed (%d) for matrix %d", (int)r, i);
      return cudaErrorInvalidValue;
    }
  }
  memcpy(host.data() + o_soff, simg_off.data(), sizeof(long long) * count);
  memcpy(host.data() + o_work, work.data(), sizeof(int) * work.size());
  memcpy(host.data() + o_woff, work_off_all.data(), sizeof(int) * work_off_all.size());
  memcpy(host.data() + o_sd, sdesc.data(), sizeof(SImgDesc) * sdesc.size());
  e = cudaMemcpy(p->dev, host.data(), o_img, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(p->dev);
    delete p;
    return e;
  }
  unsigned char* base = (unsigned char*)p->dev;
  p->d_sdesc = (const SImgDesc*)(base + o_sd);
  p->nsdesc = (int)sdesc.size();
  p->simg = base + o_img;
  const long long timeout_ns = std::max<long long>(spin_limit, 1) * 120;  // ~2 s default
  for (const ClassTmp& ct : ctmp) {
    TcClass cl;
    cl.C = ct.C;
    cl.nclusters = ct.ncl;
    TcParams& prm = cl.prm;
    prm.mats = d_mats;
    prm.tmaps = (const CUtensorMap*)(base + o_map);
    prm.work = (const int*)(base + o_work) + ct.work_start;
    prm.work_off = (const int*)(base + o_woff) + ct.woff_start;
    prm.simg = p->simg;
    prm.simg_off = (const long long*)(base + o_soff);
    prm.X = (float*)dev_X;
    prm.Y = (float*)dev_Y;
    prm.normA2 = dev_normA2;
    prm.status = status;
    prm.kp = kp;
    prm.kpad = p->kpad;
    prm.img_rank_bytes = p->img_rank_bytes;
    prm.timeout_ns = timeout_ns;
    p->classes.push_back(cl);
  }
  *out = p;
  return cudaSuccess;
}

cudaError_t tc_launch(TcPlan* p, cudaStream_t s) {
  if (!p) return cudaErrorInvalidValue;
  simg_prep_kernel<<<dim3(p->nsdesc, p->cmax), 256, 0, s>>>(p->d_sdesc, p->kpad,
                                                             p->img_rank_bytes, p->simg);
  cudaError_t e = cudaGetLastError();
  for (const TcClass& cl : p->classes) {
    if (e != cudaSuccess) break;
    switch (cl.C) {
      case 1: e = launch_class<1>(cl.prm, cl.nclusters, s); break;
      case 2: e = launch_class<2>(cl.prm, cl.nclusters, s); break;
      case 4: e = launch_class<4>(cl.prm, cl.nclusters, s); break;
      default: e = launch_class<8>(cl.prm, cl.nclusters, s); break;
    }
  }
  return e;
}

int tc_launches(const TcPlan* p) { return p ? 1 + (int)p->classes.size() : 0; }
long long tc_workspace_bytes(const TcPlan* p) { return p ? (long long)p->bytes : 0; }
void tc_destroy(TcPlan* p) {
  if (!p) return;
  if (p->dev) cudaFree(p->dev);
  delete p;
}

}  // namespace tsk
