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
// owns rows [rho*MC, (rho+1)*MC) of A and rows [rho*R, (rho+1)*R) of X
// (R = kq / C).  For every block of 64 columns:
//   1. TMA loads the CTA's MC x 64 tile (128-byte swizzle) into a stage.
//   2. MMA-X:  D_x(c, j) = sum_i S(c, i) A(i, j) over the CTA's rows
//      (A operand: the CTA's slice of S as BF16, K-major; B operand: the A
//      tile read MN-major), accumulated in TMEM with M = 64 (k <= 48 rows
//      are real; row c lands in lane 32 floor(c / 16) + c mod 16) and N = 64.
//   3. The partial D_x rows go to their owners by st.async (bytes counted
//      on the owner's barrier); each owner sums the C partials of its rows,
//      rounds them to X~ = X_hi + X_lo (two BF16 terms) and a signalling
//      warp bulk-copies those rows into every peer's X~ buffer; an X writer
//      warp stores the owner's rows of X~ to HBM.
//   4. MMA-Y:  D_y(i, c) += sum_j A(i, j) X~(j, c), the same A tile now read
//      K-major, accumulated in TMEM across all column blocks.
// After the last block D_y (the CTA's MC rows of Y) goes to HBM.  Four warps
// meanwhile sum the squares of every tile (FP32 per block, FP64 across
// blocks) for ||A||_F^2.
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
constexpr int KPAD_MAX = 48;   // largest padded k this kernel takes
constexpr int NTHREADS = 352;  // 11 warps
constexpr int BOX_ROWS = 256;  // TMA box height (hardware limit 256)
constexpr int NST_MAX = 4;     // barrier slots reserved for A stages

// Receive buffer of the X reduction: the owner of rows [rho*R, rho*R + R) of
// D_x gets them from every CTA of the cluster, slot by slot (C slots of R
// rows, C*R = kq <= KPAD_MAX rows in all).
constexpr int RECV_ROW = 272;  // 64 floats + 16 bytes of padding per row
constexpr int RECV_BYTES = KPAD_MAX * RECV_ROW;
constexpr int XB_BYTES = 2 * KPAD_MAX * 128;  // X_hi rows, then X_lo rows
constexpr int BAR_BYTES = 256;

// Shared-memory layout for MC rows of A per CTA.  With MC = 256 a stage is
// 32 KB and four of them are in flight; with MC = 512 two stages of 64 KB.  The kernel declares no static shared
// variables, so its dynamic shared memory starts on a 1024-byte boundary; the
// kernel checks this and reports misalignment instead of reserving slack.
template <int MC>
struct Lay {
  // stages of A in flight: four of 32 KB (256 rows), three of 48 KB (384
  // rows) or two of 64 KB (512 rows)
  static constexpr int NST = MC == 256 ? 4 : (MC == 384 ? 3 : 2);
  // TMA box height: 384 rows load as three boxes of 128
  static constexpr int BOX = MC == 384 ? 128 : BOX_ROWS;
  // rows of S image per 64-row chunk there is room for: 40 at 384 rows per
  // CTA (so k <= 40 there), 48 otherwise
  static constexpr int KPS = MC == 384 ? 40 : KPAD_MAX;
  static constexpr int STAGE_BYTES = MC * 128;
  static constexpr int OFF_A = 0;
  static constexpr int OFF_S = OFF_A + NST * STAGE_BYTES;
  static constexpr int S_BYTES = (MC / 64) * KPS * 128;
  static constexpr int OFF_XB = OFF_S + S_BYTES;
  static constexpr int OFF_RECV = OFF_XB + 2 * XB_BYTES;
  static constexpr int OFF_BAR = OFF_RECV + 2 * RECV_BYTES;
  static constexpr int SMEM_BYTES = OFF_BAR + BAR_BYTES;
  // MMA-X reads 64 rows of S per 64-row chunk although only kpad rows are
  // real; the extra rows (whose results are never used) must stay inside the
  // allocation: from the last chunk they reach at most 8 KB past its start.
  static_assert(OFF_S + (MC / 64 - 1) * KPS * 128 + 64 * 128 <= OFF_BAR,
                "S over-read leaves the shared-memory allocation");
  static_assert(MC % BOX == 0 && MC % 128 == 0, "whole boxes and MMA tiles");
  static_assert(SMEM_BYTES <= 227 * 1024, "shared memory budget");
  static_assert(NST <= NST_MAX, "barrier slots");
  static_assert(OFF_S % 1024 == 0 && OFF_XB % 1024 == 0 && XB_BYTES % 1024 == 0 &&
                    STAGE_BYTES % 1024 == 0,
                "swizzled operands need 1024-byte aligned atoms");
  static_assert(OFF_RECV % 16 == 0 && OFF_BAR % 8 == 0, "alignment");
};
template struct Lay<256>;
template struct Lay<384>;
template struct Lay<512>;

// barrier slots
enum {
  B_AFULL = 0,
  B_AEMPTY = B_AFULL + NST_MAX,
  B_XFULL = B_AEMPTY + NST_MAX,
  B_XTEMPTY = B_XFULL + 2,
  B_RFULL = B_XTEMPTY + 2,
  B_PEMPTY = B_RFULL + 2,
  B_XBFULL = B_PEMPTY + 2,
  B_XBEMPTY = B_XBFULL + 2,
  B_XREADY = B_XBEMPTY + 2,
  B_XWDONE = B_XREADY + 2,
  B_YFULL = B_XWDONE + 2,
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
  int kpad;        // rows of each 64-row chunk of the S image (k rounded up to 16,
                   // or to 8 at 384 rows per CTA)
  int kq;          // rows of X~_hi (and of X~_lo): k rounded up to a multiple of 8
                   // that the cluster size divides; N of MMA-Y = 2 kq
  int img_rank_bytes;  // bytes of S image per CTA: (MC / 64) chunks of kpad rows
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
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(bar),
      "r"(bytes)
      : "memory");
}
// CTA-scope acquire is enough for every barrier of the kernel: data from
// other CTAs arrives only by st.async and bulk copies, whose bytes complete
// on the waiting CTA's own barrier (as TMA loads do), and the remaining
// remote arrives only announce that a buffer has been read.
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
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
// Prefetch of one TMA box into L2 (no shared memory, no completion).
__device__ __forceinline__ void tma_prefetch_2d(const CUtensorMap* map, int x, int y) {
  asm volatile("cp.async.bulk.prefetch.tensor.2d.L2.global.tile [%0, {%1, %2}];" ::"l"(
                   (uint64_t)map),
               "r"(x), "r"(y)
               : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src,
                                          uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(dst), "l"((uint64_t)src), "r"(bytes), "r"(bar)
      : "memory");
}
// Asynchronous store of 16 bytes to the shared memory of a CTA of the
// cluster; on landing it counts its bytes on that CTA's mbarrier `bar`
// (addr, bar: mapa addresses).  No thread-side fence is involved.
__device__ __forceinline__ void st_async_v4(uint32_t addr, float a, float b, float c, float d,
                                            uint32_t bar) {
  asm volatile(
      "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, "
      "[%5];" ::"r"(addr),
      "f"(a), "f"(b), "f"(c), "f"(d), "r"(bar)
      : "memory");
}
// Arrive on a (possibly remote) mbarrier without release semantics: used
// only to say "I have finished reading that buffer", where the reads are
// complete (their values consumed) before the arrive is issued.
__device__ __forceinline__ void mbar_arrive_cluster_relaxed(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(
                   cluster_addr)
               : "memory");
}
// Bulk copy from this CTA's shared memory to a peer's (dst, bar: mapa
// addresses); completion is counted in bytes on the peer's mbarrier.
__device__ __forceinline__ void bulk_s2c(uint32_t dst, uint32_t src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.shared::cta.mbarrier::complete_tx::bytes [%0], [%1], "
      "%2, [%3];" ::"r"(dst),
      "r"(src), "r"(bytes), "r"(bar)
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
// Arrives, once the issuing thread's tcgen05 operations have completed, on
// the mbarrier at the same shared-memory offset in every CTA of `mask`.
__device__ __forceinline__ void tc_commit_mc(uint32_t bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster."
      "b64 [%0], %1;" ::"r"(bar),
      "h"(mask)
      : "memory");
}
// TMEM loads write their registers asynchronously: the values may be used
// only after tcgen05.wait::ld.  tmem_regs8 (an empty asm that claims to
// modify the registers), placed after the wait, keeps the compiler from
// touching them earlier.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, "
      "%9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
        "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
        "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_regs8(uint32_t* r) {
  asm volatile("" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                    "+r"(r[6]), "+r"(r[7])::"memory");
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

// try_wait whose suspension is capped at `hint_ns` nanoseconds (it returns
// at the phase change or when the cap runs out, whichever comes first).
__device__ __forceinline__ bool mbar_try_wait_hint(uint32_t bar, uint32_t parity,
                                                   uint32_t hint_ns) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(hint_ns)
      : "memory");
  return ok != 0;
}

// Bounded wait.  Returns false on timeout (after raising the status bit and
// the CTA-wide abort flag) or when the CTA is already aborting.  Each poll
// suspends for at most the time left (at most 100 us), and the clock is read
// after every poll, so the bound holds for any spin limit: a limit shorter
// than the work in flight makes the wait run out.
template <class PP>
__device__ __forceinline__ bool bwait(uint32_t bar, uint32_t parity, volatile Ctl* ctl,
                                      const PP& P) {
  if (ctl->abort) return false;
  const uint64_t t0 = globaltimer();
  const uint32_t hint = (uint32_t)(P.timeout_ns < 100000 ? P.timeout_ns : 100000);
  for (;;) {
    if (mbar_try_wait_hint(bar, parity, hint)) return true;
    if (ctl->abort) return false;
    if ((long long)(globaltimer() - t0) > P.timeout_ns) {
      atomicOr(P.status, kStatusTimeout);
      ctl->abort = 1;
      return false;
    }
  }
}
// Warp-uniform bounded wait: lane 0 polls, the verdict is broadcast, and the
// warp leaves converged (the tcgen05.ld that follows is .sync.aligned).
template <class PP>
__device__ __forceinline__ bool bwait_warp(uint32_t bar, uint32_t parity, volatile Ctl* ctl,
                                           const PP& P) {
  int ok = 0;
  if ((threadIdx.x & 31) == 0) ok = bwait(bar, parity, ctl, P) ? 1 : 0;
  ok = __shfl_sync(0xffffffffu, ok, 0);
  return ok != 0;
}
// Bounded wait that ignores the abort flag, used to drain the CTA's own TMA
// loads and tensor-core operations before it leaves.  Its bound is fixed
// (two seconds, far beyond any copy or MMA that was actually issued) and
// independent of the caller's spin limit: a short spin limit may cut the
// ordinary waits short, but never lets a CTA exit with its own operations
// still in flight.
constexpr long long kDrainTimeoutNs = 2000000000ll;
template <class PP>
__device__ __forceinline__ void drain_wait(uint32_t bar, uint32_t parity, const PP& P) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if ((long long)(globaltimer() - t0) > kDrainTimeoutNs) {
      atomicOr(P.status, kStatusTimeout);
      return;
    }
  }
}

// Bounded wait for arrives that peers of the cluster send (bounded by the
// spin limit like every wait on another CTA; a peer that aborted may never
// send them, and the teardown's cluster barrier covers what is in flight).
template <class PP>
__device__ __forceinline__ void peer_wait(uint32_t bar, uint32_t parity, const PP& P) {
  const uint64_t t0 = globaltimer();
  while (!mbar_try_wait(bar, parity)) {
    if ((long long)(globaltimer() - t0) > P.timeout_ns) {
      atomicOr(P.status, kStatusTimeout);
      return;
    }
  }
}

// Sum of squares of one A stage (MC x 64 BF16, SB bytes), shared by the 96
// threads of the three norm warps (t = 0..95).  Eight independent FP32
// accumulators per thread, each summing at most 43 squares per stage, keep
// the dependent chains short; stages are summed in FP64.
constexpr int NORM_THREADS = 96;
template <int SB>
__device__ __forceinline__ double stage_sumsq(const unsigned char* stage, int t) {
  const uint4* st = reinterpret_cast<const uint4*>(stage);
  float a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = 0.f;
#pragma unroll 4
  for (int e = t; e < SB / 16; e += NORM_THREADS) {
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

template <int C, int MC>
__global__ void __launch_bounds__(NTHREADS, 1)
sketch_tc_kernel(const __grid_constant__ TcParams P) {
  using L = Lay<MC>;
  constexpr int NST = L::NST, STAGE_BYTES = L::STAGE_BYTES;
  constexpr int OFF_A = L::OFF_A, OFF_S = L::OFF_S, OFF_XB = L::OFF_XB;
  constexpr int OFF_RECV = L::OFF_RECV, OFF_BAR = L::OFF_BAR;
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
  const int kpad = P.kpad, kq = P.kq;
  const int R = kq / C;  // rows of X this CTA reduces (C divides kq: kq % 8 == 0)
  auto bar = [&](int i) -> uint32_t { return sb + OFF_BAR + 8 * i; };
  volatile Ctl* ctl = (volatile Ctl*)(sm + OFF_BAR + 8 * B_COUNT);
  uint32_t* tmem_slot = (uint32_t*)(sm + OFF_BAR + 8 * B_COUNT + 8);

  const int w0 = P.work_off[cid], w1 = P.work_off[cid + 1];
  const uint32_t tmem_cols_needed = 2 * NB + (MC / 128) * 2 * kq;
  const uint32_t tmem_cols = tmem_cols_needed <= 256 ? 256 : 512;

  if (tid == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(bar(B_AFULL + s), 1);
      mbar_init(bar(B_AEMPTY + s), 4);  // MMA-Y commit + three norm warps
    }
    for (int h = 0; h < 2; ++h) {
      mbar_init(bar(B_XFULL + h), 1);
      mbar_init(bar(B_XTEMPTY + h), 3);  // the three sending warps
      mbar_init(bar(B_RFULL + h), 1);    // own expect-tx; senders' bytes by st.async
      mbar_init(bar(B_PEMPTY + h), C);   // every owner consumed this CTA's rows
      mbar_init(bar(B_XBFULL + h), 1);   // own rows written (+ bytes from peers)
      mbar_init(bar(B_XBEMPTY + h), C);  // every CTA's MMA-Y finished reading
      mbar_init(bar(B_XREADY + h), 64);  // own rows of X~ written by the 64 threads
      mbar_init(bar(B_XWDONE + h), 1);   // X writer has read those rows
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
  const uint32_t idesc_x = idesc_bf16(64, NB, 0, 1);  // M = 64 >= kpad
  const uint32_t idesc_y = idesc_bf16(128, 2 * kq, 0, 0);

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      long long g = 0;
      int sloads = 0;
      const unsigned char* cur_img = nullptr;
      bool stop = false;
      // L2 prefetch cursor, NST blocks ahead of the loads: a block is pulled
      // into L2 while the stage it will occupy is still busy, so its TMA
      // load later hits L2 instead of waiting on HBM.
      auto nblk_of = [&](int wi) { return (int)((P.mats[P.work[wi]].n + NB - 1) / NB); };
      int pwi = w0, pq = 0, pn = (w0 < w1) ? nblk_of(w0) : 0;
      auto padv = [&]() {
        if (++pq >= pn) {
          ++pwi;
          pq = 0;
          pn = (pwi < w1) ? nblk_of(pwi) : 0;
        }
      };
      for (int i = 0; i < NST && pwi < w1; ++i) padv();
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
          for (int b = 0; b < MC / L::BOX; ++b)
            tma_load_2d(sb + OFF_A + s * STAGE_BYTES + b * L::BOX * 128, map, q * NB,
                        (int)(rank * MC + b * L::BOX), bar(B_AFULL + s));
          if (pwi < w1) {
            const CUtensorMap* pmap = P.tmaps + P.work[pwi];
#pragma unroll
            for (int b = 0; b < MC / L::BOX; ++b)
              tma_prefetch_2d(pmap, pq * NB, (int)(rank * MC + b * L::BOX));
            padv();
          }
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
                                     L::BOX * 128, 1024);
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
              tc_mma(tmem + 2 * NB + t * 2 * kq, a, b, idesc_y, (q > 0 || kk > 0) ? 1u : 0u);
            }
          }
          tc_commit(bar(B_AEMPTY + s));
          // X~ buffer h is read: every owner may refill its rows here
          if (C > 1)
            tc_commit_mc(bar(B_XBEMPTY + h), (uint16_t)((1u << C) - 1));
          else
            tc_commit(bar(B_XBEMPTY + h));
          if (q == nblk - 1) tc_commit(bar(B_YFULL));
        }
      }
      tc_commit(bar(B_DRAIN2));
      drain_wait(bar(B_DRAIN2), 0, P);
    }
  } else if (warp >= 2 && warp <= 6) {
    // ------- X exchange (warps 4, 5; warp 6 sends only) or ||A||^2 (warps 2,
    // 3, with warp 7 below), then Y out (warps 2-5)
    const int lane_base = (warp & 3) * 32;  // this warp's TMEM lane quarter
    const bool xwarp = (warp == 4 || warp == 5);
    const bool sendonly = (warp == 6);
    double tot = 0.0;
    // row of D_x in this lane (M = 64: rows 16q .. 16q + 15 in lanes 0-15 of
    // quarter q); lanes 16-31 hold no row
    const int c = 16 * (warp & 3) + lane;
    long long g = 0;
    int mi = 0;
    for (int wi = w0; wi < w1; ++wi, ++mi) {
      const int d = P.work[wi];
      const MatDev& md = P.mats[d];
      const long long n = md.n, m = md.m;
      const int nblk = (int)((n + NB - 1) / NB);
      for (int q = 0; q < nblk; ++q, ++g) {
        if (!xwarp && !sendonly) {
          const int s = (int)(g % NST);
          const uint32_t u = (uint32_t)(g / NST);
          if (bwait_warp(bar(B_AFULL + s), u & 1, ctl, P))
            tot += stage_sumsq<STAGE_BYTES>(sm + OFF_A + s * STAGE_BYTES, tid - 64);
          __syncwarp();
          if (lane == 0) mbar_arrive(bar(B_AEMPTY + s));
          continue;
        }
        const int h = (int)(g & 1);
        const uint32_t v = (uint32_t)(g >> 1);
        const int xt = tid - 128;  // 0..63 over the two exchange warps
        // (a) Send.  Row c of this CTA's partial D_x goes to its owner
        // c / R, into slot rank of the owner's receive buffer h, straight
        // from the TMEM registers by asynchronous remote stores that count
        // their bytes on the owner's RFULL barrier.  After a timeout nothing
        // new goes to peers.
        bwait_warp(bar(B_PEMPTY + h), (v & 1) ^ 1, ctl, P);
        if (bwait_warp(bar(B_XFULL + h), v & 1, ctl, P)) {
          tc_fence_after();
          const int own = c / R;
          const uint32_t owner = (uint32_t)(own < C ? own : 0);
          const uint32_t dst0 = mapa(
              sb + OFF_RECV + h * RECV_BYTES + (rank * R + (c - own * R)) * RECV_ROW, owner);
          const uint32_t rfull = mapa(bar(B_RFULL + h), owner);
          uint32_t xr[NB];
#pragma unroll
          for (int j = 0; j < NB; j += 16)
            tmem_ld16(tmem + ((uint32_t)lane_base << 16) + h * NB + j, xr + j);
          tmem_wait_ld();
#pragma unroll
          for (int j = 0; j < NB; j += 8) tmem_regs8(xr + j);
          if (lane < 16 && c < kq && !ctl->abort) {
            // rows k <= c < kq are zero in X (the S image may be narrower
            // than kq, and then its rows there are another chunk's)
            const uint32_t keep = c < md.k ? 0xFFFFFFFFu : 0u;
#pragma unroll
            for (int e = 0; e < NB; e += 4)
              st_async_v4(dst0 + e * 4, __uint_as_float(xr[e] & keep),
                          __uint_as_float(xr[e + 1] & keep), __uint_as_float(xr[e + 2] & keep),
                          __uint_as_float(xr[e + 3] & keep), rfull);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_XTEMPTY + h));
        if (sendonly) continue;
        // The owner expects R rows of 256 bytes from each of the C CTAs.
        // After a timeout no bytes are sent, so the phase of RFULL can never
        // complete: a further arrive on it would take its pending count below
        // zero (undefined), so nothing arrives on it any more.
        if (xt == 63 && !ctl->abort) mbar_expect_tx(bar(B_RFULL + h), (uint32_t)(C * R * 256));
        // (b) Reduce.  X rows [rank*R, rank*R + R) of this block = sum of the
        // C slots, eight columns per work item.  Two-term BF16 split X =
        // X_hi + X_lo (X_hi = BF16(X), X_lo = BF16(X - X_hi)); MMA-Y
        // multiplies A by both, so Y = A (X_hi + X_lo) carries about 16
        // significant bits of X instead of 8.  The rows are written only
        // when every CTA's MMA-Y and this CTA's X writer are done with the
        // previous contents of buffer h.
        // (after a timeout the buffers hold nothing valid: skip the reduce,
        // but keep arriving so that no local wait is left hanging)
        const bool got = bwait_warp(bar(B_XBEMPTY + h), (v & 1) ^ 1, ctl, P) &&
                         bwait_warp(bar(B_XWDONE + h), (v & 1) ^ 1, ctl, P) &&
                         bwait_warp(bar(B_RFULL + h), v & 1, ctl, P);
        const unsigned char* rb = sm + OFF_RECV + h * RECV_BYTES;
        unsigned char* xb = sm + OFF_XB + h * XB_BYTES;
#pragma unroll 1
        for (int it = xt; got && it < R * 8; it += 64) {
          const int ri = it % R, ob = it / R;  // row, octet of columns
          const int cr = (int)rank * R + ri;
          float acc[8];
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[j] = 0.f;
#pragma unroll
          for (int sl = 0; sl < C; ++sl) {
            const float4* src =
                reinterpret_cast<const float4*>(rb + (sl * R + ri) * RECV_ROW + ob * 32);
            const float4 w0 = src[0], w1 = src[1];
            acc[0] += w0.x;
            acc[1] += w0.y;
            acc[2] += w0.z;
            acc[3] += w0.w;
            acc[4] += w1.x;
            acc[5] += w1.y;
            acc[6] += w1.z;
            acc[7] += w1.w;
          }
          uint32_t phi[4], plo[4];
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            const __nv_bfloat16 h0 = __float2bfloat16_rn(acc[j]);
            const __nv_bfloat16 h1 = __float2bfloat16_rn(acc[j + 1]);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(acc[j] - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(acc[j + 1] - __bfloat162float(h1));
            __nv_bfloat162 hh, ll;
            hh.x = h0;
            hh.y = h1;
            ll.x = l0;
            ll.y = l1;
            phi[j / 2] = *reinterpret_cast<const uint32_t*>(&hh);
            plo[j / 2] = *reinterpret_cast<const uint32_t*>(&ll);
          }
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            const int row = cr + half * kq;
            const uint32_t* w = half ? plo : phi;
            *reinterpret_cast<uint4*>(xb + (row >> 3) * 1024 + (row & 7) * 128 +
                                      (((ob ^ (row & 7)) & 7) << 4)) =
                make_uint4(w[0], w[1], w[2], w[3]);
          }
        }
        // (c) Hand the owned rows of X~ to the signalling warp, which copies
        // them to the peers.  The proxy fence makes these generic writes
        // visible to the bulk copies and to the tensor cores.  After a
        // timeout nothing is handed on: the signalling warp would otherwise
        // arm XBFULL again while its previous phase, waiting for bytes no
        // peer will send, is still open (an arrive below zero).  Every
        // waiter on XREADY is bounded and sees the abort flag.
        fence_proxy_async_cta();
        if (got) mbar_arrive(bar(B_XREADY + h));
      }
      if (sendonly) continue;  // the Y epilogue belongs to warps 2-5
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
          for (int j = 0; j < kq && j < P.kp; j += 8) {  // columns past the panel are zero
            uint32_t yv[8], yl[8];
            const uint32_t col = tmem + ((uint32_t)lane_base << 16) + 2 * NB + t * 2 * kq + j;
            tmem_ld8(col, yv);
            tmem_ld8(col + kq, yl);
            tmem_wait_ld();
            tmem_regs8(yv);
            tmem_regs8(yl);
            if (row < m) {
              float4* dst = reinterpret_cast<float4*>(Ym + row * P.kp + j);
              float y[8];
#pragma unroll
              for (int e = 0; e < 8; ++e) y[e] = __uint_as_float(yv[e]) + __uint_as_float(yl[e]);
              dst[0] = make_float4(y[0], y[1], y[2], y[3]);
              dst[1] = make_float4(y[4], y[5], y[6], y[7]);
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(B_YFREE));
    }
    // Owners arrive on PEMPTY and every CTA's MMA-Y on XBEMPTY after this
    // CTA's last use of a buffer: wait for those final phases, so that no
    // remote arrive is still in flight toward this CTA when it leaves.
    if (xwarp && lane == 0 && g > 0) {
      for (int h = 0; h < 2; ++h) {
        if (g > h) {
          const long long last = ((g - 1 - h) / 2) * 2 + h;
          peer_wait(bar(B_PEMPTY + h), (uint32_t)((last >> 1) & 1), P);
          peer_wait(bar(B_XBEMPTY + h), (uint32_t)((last >> 1) & 1), P);
        }
      }
    }
  } else if (warp == 10) {
    // ------------------------------------------------------ X writer
    // X in HBM holds X_hi + X_lo, the values Y is built from: once the owned
    // rows of X~ of a block are written (XREADY), this warp reads them back
    // and stores X rows [rank*R, rank*R + R) (rows < k) of the block's
    // columns, keeping global stores off the exchange warps.
    // Element e = lane + 32 t of a block is (column j, row ri) = (e / R,
    // e % R): consecutive lanes write consecutive rows of one column of X.
    // The pair advances by (32 / R, 32 % R) per step, so no division is
    // needed inside the loop.
    const int dj = 32 / R, dr = 32 % R;
    const int j0 = lane / R, r0 = lane % R;
    long long g = 0;
    for (int wi = w0; wi < w1; ++wi) {
      const MatDev& md = P.mats[P.work[wi]];
      const long long n = md.n;
      const int k = md.k;
      float* Xm = P.X + md.offX;
      const int nblk = (int)((n + NB - 1) / NB);
      for (int q = 0; q < nblk; ++q, ++g) {
        const int h = (int)(g & 1);
        const uint32_t v = (uint32_t)(g >> 1);
        // the abort flag is read again after the wait: rows written by an
        // exchange that ran out are not valid
        if (bwait_warp(bar(B_XREADY + h), v & 1, ctl, P) && !ctl->abort) {
          const unsigned char* xb = sm + OFF_XB + h * XB_BYTES;
          const long long jb = (long long)q * NB;
          const int jmax = (int)min((long long)NB, n - jb);
          int j = j0, ri = r0;
#pragma unroll 4
          for (int e = lane; e < R * NB; e += 32) {
            const int cr = (int)rank * R + ri;
            if (cr < k && j < jmax) {
              const int rl = cr + kq, un = j >> 3, w = (j & 7) * 2;
              const __nv_bfloat16 vh = *reinterpret_cast<const __nv_bfloat16*>(
                  xb + (cr >> 3) * 1024 + (cr & 7) * 128 + (((un ^ (cr & 7)) & 7) << 4) + w);
              const __nv_bfloat16 vl = *reinterpret_cast<const __nv_bfloat16*>(
                  xb + (rl >> 3) * 1024 + (rl & 7) * 128 + (((un ^ (rl & 7)) & 7) << 4) + w);
              Xm[(jb + j) * P.kp + cr] = __bfloat162float(vh) + __bfloat162float(vl);
            }
            j += dj;
            ri += dr;
            if (ri >= R) {
              ri -= R;
              ++j;
            }
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(bar(B_XWDONE + h));
      }
    }
  } else if (warp == 9) {
    // ---------------------------------------- signalling (lanes 0..C-1)
    // Once the owned rows of X~ are written (XREADY), lane r copies them
    // into peer r's X~ buffer (bulk copy; bytes complete on the peer's
    // XBFULL) or, for r == rank, announces the bytes the C - 1 peers will
    // send; then it tells CTA r that its slot of this CTA's receive buffer
    // is free again.  Remote operations can hold the issuing thread for a
    // microsecond or more, so they run here and not in the exchange warps.
    if (lane < C) {
      const uint32_t peer = (uint32_t)lane;
      long long g = 0;
      for (int wi = w0; wi < w1; ++wi) {
        const int nblk = (int)((P.mats[P.work[wi]].n + NB - 1) / NB);
        for (int q = 0; q < nblk; ++q, ++g) {
          const int h = (int)(g & 1);
          const uint32_t v = (uint32_t)(g >> 1);
          if (!bwait(bar(B_XREADY + h), v & 1, ctl, P)) continue;
          const uint32_t xs = sb + OFF_XB + h * XB_BYTES;
          const uint32_t xf = bar(B_XBFULL + h);
          if (peer != rank) {
            const uint32_t hi = xs + rank * R * 128, lo = xs + (kq + rank * R) * 128;
            bulk_s2c(mapa(hi, peer), hi, R * 128, mapa(xf, peer));
            bulk_s2c(mapa(lo, peer), lo, R * 128, mapa(xf, peer));
          } else {
            mbar_expect_tx(xf, (uint32_t)((C - 1) * 2 * R * 128));
          }
          mbar_arrive_cluster_relaxed(mapa(bar(B_PEMPTY + h), peer));
        }
      }
    }
  } else {
    // ------------------------------------------------ ||A||_F^2 (warp 7)
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
          tot += stage_sumsq<STAGE_BYTES>(sm + OFF_A + s * STAGE_BYTES, tid - 224 + 64);
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
  if (C > 1) {
    cluster_sync();
    // After a timeout the waits above were cut short, so stores, copies or
    // arrives that peers issued before the cluster barrier may still be
    // landing here: give them time (they take microseconds) before leaving.
    if (ctl->abort && tid == 0) {
      const uint64_t t0 = globaltimer();
      while (globaltimer() - t0 < 200000ull) {
      }
    }
    __syncthreads();
  }
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tmem_cols)
                 : "memory");
  }
}

// Pre-swizzled BF16 image of every distinct sketch S: the exact
// shared-memory layout the MMA-X A operand reads (K-major, 128-byte swizzle),
// one 64-row chunk of S^T (kpad rows of 128 bytes) after another.  The
// image of cluster rank rho is the contiguous run of chunks covering rows
// [rho*MC, rho*MC + MC), so one image serves every cluster size.
struct SImgDesc {
  const float* S;
  long long m;
  int k;
  int nchunks;  // 64-row chunks in this image (covers C * MC rows)
  int kpad;     // rows per chunk (the class's kpad)
  long long off;
};

__global__ void simg_prep_kernel(const SImgDesc* __restrict__ descs,
                                 unsigned char* __restrict__ simg) {
  const SImgDesc sd = descs[blockIdx.x];
  const int qc = blockIdx.y;  // chunk
  if (qc >= sd.nchunks) return;
  const int kpad = sd.kpad;
  unsigned char* img = simg + sd.off + (long long)qc * kpad * 128;
  for (int e = threadIdx.x; e < kpad * 8; e += blockDim.x) {
    const int c = e / 8, u = e % 8;
    uint32_t w[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      float v2[2];
#pragma unroll
      for (int z = 0; z < 2; ++z) {
        const long long i = (long long)qc * 64 + u * 8 + 2 * t + z;
        v2[z] = (c < sd.k && i < sd.m) ? sd.S[(long long)c * sd.m + i] : 0.f;
      }
      w[t] = pack_bf16x2(v2[0], v2[1]);
    }
    uint4* dst = reinterpret_cast<uint4*>(img + (c >> 3) * 1024 + (c & 7) * 128 +
                                          (((u ^ (c & 7)) & 7) << 4));
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

template <int C, int MC>
cudaError_t set_attrs() {
  cudaError_t e = cudaFuncSetAttribute(sketch_tc_kernel<C, MC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       Lay<MC>::SMEM_BYTES);
  return e;
}

template <int C, int MC>
int max_clusters() {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(C * 256, 1, 1);
  cfg.blockDim = dim3(NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = Lay<MC>::SMEM_BYTES;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, sketch_tc_kernel<C, MC>, &cfg) != cudaSuccess ||
      n < 1) {
    cudaGetLastError();
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    n = std::max(1, sms / C);
  }
  return n;
}

template <int C, int MC>
cudaError_t launch_class(const TcParams& prm, int nclusters, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute attr[1];
  cfg.gridDim = dim3(C * nclusters, 1, 1);
  cfg.blockDim = dim3(NTHREADS, 1, 1);
  cfg.dynamicSmemBytes = Lay<MC>::SMEM_BYTES;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, sketch_tc_kernel<C, MC>, prm);
}

// Cluster shape for an m-row matrix: MC rows per CTA and C CTAs, C the
// smallest power of two with C * MC >= m.  The X exchange costs about the
// same per column block whatever MC is, so 512 rows per CTA (two 64 KB
// stages) beat 256 rows (four 32 KB stages) once a cluster is needed; a
// matrix of at most 256 rows takes one CTA with four stages.
void cluster_shape(long long m, int* C, int* MC, int mc_pref = 0, int k = 0) {
  *MC = m <= 256 ? 256 : 512;
  if (mc_pref == 256 && m <= 8 * 256) *MC = 256;  // up to clusters of 8
  if (mc_pref == 512) *MC = 512;
  if (mc_pref == 384 && m <= 6 * 384 && (k + 7) / 8 * 8 <= 40) {
    // clusters of 1, 2, 3 or 6 CTAs of 384 rows
    *MC = 384;
    *C = m <= 384 ? 1 : (m <= 768 ? 2 : (m <= 1152 ? 3 : 6));
    return;
  }
  int c = 1;
  while ((long long)c * *MC < m) c *= 2;
  *C = c;
}

// Rows of X~ for a class: k rounded up to a multiple of 8 that the cluster
// size divides (each CTA reduces kq / C rows).
int class_kq(int kmax, int C) {
  const int unit = (C == 3 || C == 6) ? 24 : 8;
  return (kmax + unit - 1) / unit * unit;
}
// Rows per 64-row chunk of the S image: k rounded up to 16, or to 8 at 384
// rows per CTA (shared memory has room for 40 there).
int class_kpad(int kmax, int MC) {
  return MC == 384 ? (kmax + 7) / 8 * 8 : (kmax + 15) / 16 * 16;
}

// The instantiated (C, MC) pairs, in one place for attributes and launches.
cudaError_t class_attrs(int C, int MC, int* ncl) {
  cudaError_t e = cudaErrorInvalidValue;
#define TSK_TC_CASE(c_, mc_)                 \
  if (C == c_ && MC == mc_) {                \
    e = set_attrs<c_, mc_>();                \
    if (e == cudaSuccess) *ncl = max_clusters<c_, mc_>(); \
  }
  TSK_TC_CASE(1, 256)
  TSK_TC_CASE(2, 256)
  TSK_TC_CASE(4, 256)
  TSK_TC_CASE(8, 256)
  TSK_TC_CASE(1, 384)
  TSK_TC_CASE(2, 384)
  TSK_TC_CASE(3, 384)
  TSK_TC_CASE(6, 384)
  TSK_TC_CASE(1, 512)
  TSK_TC_CASE(2, 512)
  TSK_TC_CASE(4, 512)
  TSK_TC_CASE(8, 512)
#undef TSK_TC_CASE
  return e;
}

cudaError_t class_launch(int C, int MC, const TcParams& prm, int nclusters, cudaStream_t s) {
  if (C == 1 && MC == 256) return launch_class<1, 256>(prm, nclusters, s);
  if (C == 2 && MC == 256) return launch_class<2, 256>(prm, nclusters, s);
  if (C == 4 && MC == 256) return launch_class<4, 256>(prm, nclusters, s);
  if (C == 8 && MC == 256) return launch_class<8, 256>(prm, nclusters, s);
  if (C == 1 && MC == 384) return launch_class<1, 384>(prm, nclusters, s);
  if (C == 2 && MC == 384) return launch_class<2, 384>(prm, nclusters, s);
  if (C == 3 && MC == 384) return launch_class<3, 384>(prm, nclusters, s);
  if (C == 6 && MC == 384) return launch_class<6, 384>(prm, nclusters, s);
  if (C == 1 && MC == 512) return launch_class<1, 512>(prm, nclusters, s);
  if (C == 2 && MC == 512) return launch_class<2, 512>(prm, nclusters, s);
  if (C == 4 && MC == 512) return launch_class<4, 512>(prm, nclusters, s);
  if (C == 8 && MC == 512) return launch_class<8, 512>(prm, nclusters, s);
  return cudaErrorInvalidValue;
}


// ---------------------------------------------------------------------------
// T1 on the tensor cores: the mode-1 Gram matrix G = sum_d A_d A_d^T of BF16
// training matrices (Eq. 3.2; the Gram route of Section 3.1), FP32
// accumulation in TMEM, FP64 sums in G.
//
// One CTA per 128 x 128 tile (I, J), I <= J, of the upper block triangle
// (blockIdx.y splits the matrices when there are few tiles).  Both operands
// are K-major: rows I and rows J of A_d, 64 columns per stage, loaded by TMA
// with the 128-byte swizzle (a diagonal tile loads its rows once and uses
// them as both operands).  Warp 0 issues the loads into a ring of GSTG
// stages, warp 1 the MMAs (M = N = 128, K = 16, four per stage) into one of
// two TMEM accumulators of 128 columns; every GFL matrices the accumulator
// is handed to warps 2-5, which add it to G in FP64 while the MMAs go on in
// the other one.  The lower triangle is mirrored afterwards.
// ---------------------------------------------------------------------------
struct GramParams {
  const CUtensorMap* tmaps;  // one per matrix: box 64 columns x 128 rows (mode 1)
                             // or 64 columns x 64 rows (mode 2)
  long long D, m, n;
  double* G;                 // dim x dim, row-major (dim = m in mode 1, n in mode 2)
  int mode;                  // 1: G = sum A A^T; 2: G = sum A^T A
  int ntile;                 // ceil(dim / 128)
  int splits;                // CTAs per tile (contiguous ranges of matrices)
  int* status;
  long long timeout_ns;
};

constexpr int GNT = 192;              // 6 warps: TMA, MMA, four epilogue warps
constexpr int GSTG = 6;               // stages in flight
constexpr int GTILE = 128 * 128;      // 128 rows x 64 BF16 columns = 16 KB
constexpr int GSTAGE = 2 * GTILE;
constexpr int GFL = 8;                // matrices per TMEM flush
constexpr int G_OFF_BAR = GSTG * GSTAGE;
enum { GB_FULL = 0, GB_EMPTY = GSTG, GB_TFULL = 2 * GSTG, GB_TEMPTY = 2 * GSTG + 2,
       GB_DRAIN = 2 * GSTG + 4, GB_COUNT = 2 * GSTG + 5 };
constexpr int G_SMEM = G_OFF_BAR + 256;
static_assert(GB_COUNT * 8 + 16 <= 256, "gram barrier area");
static_assert(G_SMEM <= 227 * 1024, "gram shared memory");

__global__ void __launch_bounds__(GNT, 1) gram_tc_kernel(const __grid_constant__ GramParams P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw;
  const uint32_t sb = smem_u32(sm);
  if (sb & 1023) {
    if (threadIdx.x == 0) atomicOr(P.status, kStatusTimeout);
    return;
  }
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  auto bar = [&](int i) -> uint32_t { return sb + G_OFF_BAR + 8 * i; };
  volatile Ctl* ctl = (volatile Ctl*)(sm + G_OFF_BAR + 8 * GB_COUNT);
  uint32_t* tmem_slot = (uint32_t*)(sm + G_OFF_BAR + 8 * GB_COUNT + 8);
  int t = blockIdx.x, ti = 0;  // tile (ti, tj), ti <= tj, from the linear index
  while (t >= P.ntile - ti) {
    t -= P.ntile - ti;
    ++ti;
  }
  const int tj = ti + t;
  const bool diag = ti == tj;
  const long long d0 = P.D * (long long)blockIdx.y / P.splits;
  const long long d1 = P.D * (long long)(blockIdx.y + 1) / P.splits;
  // mode 1: rows of G are rows of A, the sum runs over the n columns;
  // mode 2: rows of G are columns of A, the sum runs over the m rows
  const bool m2 = P.mode == 2;
  const long long dim = m2 ? P.n : P.m;
  const int nkb = (int)(((m2 ? P.m : P.n) + 63) / 64);
  const int ngroups = (int)((d1 - d0 + GFL - 1) / GFL);
  if (tid == 0) {
    for (int s = 0; s < GSTG; ++s) {
      mbar_init(bar(GB_FULL + s), 1);
      mbar_init(bar(GB_EMPTY + s), 1);  // MMA commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(GB_TFULL + b), 1);   // MMA commit
      mbar_init(bar(GB_TEMPTY + b), 4);  // four epilogue warps
    }
    mbar_init(bar(GB_DRAIN), 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      long long q = 0;
      bool stop = false;
      for (long long d = d0; d < d1 && !stop; ++d) {
        const CUtensorMap* map = P.tmaps + d;
        for (int kb = 0; kb < nkb; ++kb, ++q) {
          const int s = (int)(q % GSTG);
          const uint32_t u = (uint32_t)(q / GSTG);
          if (!bwait(bar(GB_EMPTY + s), (u & 1) ^ 1, ctl, P)) {
            stop = true;
            break;
          }
          mbar_expect_tx(bar(GB_FULL + s), diag ? GTILE : GSTAGE);
          if (!m2) {
            // K-major: rows ti*128.. of A, 64 of its columns
            tma_load_2d(sb + s * GSTAGE, map, kb * 64, ti * 128, bar(GB_FULL + s));
            if (!diag)
              tma_load_2d(sb + s * GSTAGE + GTILE, map, kb * 64, tj * 128, bar(GB_FULL + s));
          } else {
            // MN-major: 64 rows of A (the K slice), its columns ti*128.. as
            // two boxes of 64 (the two 128-byte atoms along M)
            for (int hh = 0; hh < 2; ++hh) {
              tma_load_2d(sb + s * GSTAGE + hh * (GTILE / 2), map, ti * 128 + hh * 64, kb * 64,
                          bar(GB_FULL + s));
              if (!diag)
                tma_load_2d(sb + s * GSTAGE + GTILE + hh * (GTILE / 2), map, tj * 128 + hh * 64,
                            kb * 64, bar(GB_FULL + s));
            }
          }
        }
      }
      for (int s = 0; s < GSTG; ++s) {  // every load issued must land before exit
        if (q > s) {
          const long long last = ((q - 1 - s) / GSTG) * GSTG + s;
          drain_wait(bar(GB_FULL + s), (uint32_t)((last / GSTG) & 1), P);
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc = m2 ? idesc_bf16(128, 128, 1, 1) : idesc_bf16(128, 128, 0, 0);
      long long q = 0;
      bool ok = true;
      for (int grp = 0; grp < ngroups && ok; ++grp) {
        const int buf = grp & 1;
        const uint32_t v = (uint32_t)(grp >> 1);
        if (!bwait(bar(GB_TEMPTY + buf), (v & 1) ^ 1, ctl, P)) break;
        tc_fence_after();
        const long long dlo = d0 + (long long)grp * GFL;
        const long long dhi = dlo + GFL < d1 ? dlo + GFL : d1;
        bool first = true;
        for (long long d = dlo; d < dhi && ok; ++d) {
          for (int kb = 0; kb < nkb; ++kb, ++q) {
            const int s = (int)(q % GSTG);
            const uint32_t u = (uint32_t)(q / GSTG);
            if (!bwait(bar(GB_FULL + s), u & 1, ctl, P)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a0 = sb + s * GSTAGE, b0 = diag ? a0 : a0 + GTILE;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              // K-major: the K slice advances 32 bytes inside the 128-byte
              // rows; MN-major: it advances 16 rows (2 KB), the 8-row groups
              // are 1 KB apart and the two 64-wide atoms along M 8 KB apart
              const uint64_t da = m2 ? sdesc(a0 + kk * 2048, GTILE / 2, 1024)
                                     : sdesc(a0 + kk * 32, 16, 1024);
              const uint64_t db = m2 ? sdesc(b0 + kk * 2048, GTILE / 2, 1024)
                                     : sdesc(b0 + kk * 32, 16, 1024);
              tc_mma(tmem + buf * 128, da, db, idesc, (first && kk == 0) ? 0u : 1u);
            }
            first = false;
            tc_commit(bar(GB_EMPTY + s));
          }
        }
        if (ok) tc_commit(bar(GB_TFULL + buf));
      }
      tc_commit(bar(GB_DRAIN));
      drain_wait(bar(GB_DRAIN), 0, P);
    }
  } else {
    // ------------------------------------- epilogue (warps 2-5): TMEM -> G
    const int lane_base = (warp & 3) * 32;  // the TMEM lanes this warp may read
    const long long row = (long long)ti * 128 + lane_base + lane;
    const bool atomic = P.splits > 1;
    const long long ldg = dim;
    for (int grp = 0; grp < ngroups; ++grp) {
      const int buf = grp & 1;
      const uint32_t v = (uint32_t)(grp >> 1);
      if (!bwait_warp(bar(GB_TFULL + buf), v & 1, ctl, P)) break;
      tc_fence_after();
#pragma unroll 1
      for (int c0 = 0; c0 < 128; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)lane_base << 16) + buf * 128 + c0, r);
        tmem_wait_ld();
        tmem_regs8(r);
        tmem_regs8(r + 8);
        if (row < dim) {
          double* g = P.G + row * ldg + (long long)tj * 128 + c0;
          const long long cmax = dim - ((long long)tj * 128 + c0);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            if (i < cmax) {
              const double x = (double)__uint_as_float(r[i]);
              if (atomic)
                atomicAdd(g + i, x);
              else
                g[i] += x;
            }
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar(GB_TEMPTY + buf));
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// T1 on CTA pairs: the same Gram with 256 x 256 tiles of G, each computed by
// a cluster of two CTAs whose tensor cores work as one (tcgen05 .cta_group::2,
// M = N = 256, K = 16 per MMA).  CTA rank rho of the pair holds rows
// [rho * 128, rho * 128 + 128) of the tile's row block (the M half of the A
// operand) and the same rows of its column block (the N half of the B
// operand), and its TMEM receives those 128 rows of the 256 x 256 tile.
// Per 64-column stage a CTA loads 32 KB and its tensor core does half of a
// 256 x 256 x 64 product: twice the flops per loaded byte of the 128 x 128
// single-CTA tile, which is what bounds that kernel (its operand rows come
// from L2 faster than HBM, but not fast enough to keep the MMAs busy).
//
// Roles: in both CTAs warp 0 issues the TMA loads of its own halves, which
// count their bytes on the even CTA's FULL barrier (.cta_group::2 loads);
// warp 1 of the even CTA issues the MMAs and commits them to the EMPTY and
// TFULL barriers of both CTAs; warps 2-9 of each CTA read its 128 TMEM lanes
// into registers, arrive on the even CTA's TEMPTY barrier, and add their
// sums into G once per group of GFL matrices.
// ---------------------------------------------------------------------------
struct Gram2Params {
  const CUtensorMap* tmaps;  // one per matrix: box 128 bytes x 128 rows (mode 1) or
                             // 128 bytes x 64 rows (mode 2)
  long long D, m, n;         // m: rows of G; n: the summed length (n, or m in mode 2)
  int mode2;                 // G = sum A^T A: operands MN-major
  int fl;                    // matrices per TMEM flush (1, 2, 4 or 8; divides GFL)
  double* G;
  const float* scales;  // FP8 operands: per group of GFL matrices, m row scales
  int ntile;   // ceil(m / 256)
  int splits;  // pairs per tile (contiguous ranges of groups of GFL matrices)
  int* status;
  long long timeout_ns;
};

constexpr int G2STG = 6;
constexpr int G2HALF = 128 * 128;       // 128 rows x 64 BF16 columns = 16 KB
constexpr int G2STAGE = 2 * G2HALF;     // A half, B half
constexpr int G2_OFF_BAR = G2STG * G2STAGE;
enum { G2_FULL = 0, G2_EMPTY = G2STG, G2_TFULL = 2 * G2STG, G2_TEMPTY = 2 * G2STG + 2,
       G2_DRAIN = 2 * G2STG + 4, G2_COUNT = 2 * G2STG + 5 };
// 10 warps: TMA, MMA, and eight epilogue warps; epilogue warp w holds TMEM
// lanes 32 (w % 4) .. +31 and the tile's columns 128 ((w - 2) / 4) .. +127
constexpr int G2NT = 320;
// epilogue staging: each epilogue warp turns its 32 rows x 16 columns of a
// chunk around, so that its additions to G are coalesced
constexpr int G2_STG_LD = 17;
constexpr int G2_OFF_STG = G2_OFF_BAR + 256;
constexpr int G2_SMEM = G2_OFF_STG + 8 * 32 * G2_STG_LD * 4;
static_assert(G2_COUNT * 8 + 16 <= 256, "gram2 barrier area");
static_assert(G2_SMEM <= 227 * 1024, "gram2 shared memory");

__device__ __forceinline__ void tma_load_2d_pair(uint32_t dst, const CUtensorMap* map, int x,
                                                 int y, uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::"
      "bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"((uint64_t)map), "r"(x), "r"(y), "r"(bar_cluster)
      : "memory");
}
__device__ __forceinline__ void tc_mma_pair(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
// The same MMA on 8-bit operands (both E4M3), K = 32 per instruction.
__device__ __forceinline__ void tc_mma_pair_f8(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                               uint32_t idesc, uint32_t accum) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
      : "memory");
}
// Instruction descriptor, kind::f8f6f4 with E4M3 operands (format code 0)
// and FP32 accumulation, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_commit_pair_mc(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster."
      "b64 [%0], %1;" ::"r"(bar),
      "h"((uint16_t)3)
      : "memory");
}
__device__ __forceinline__ void tc_commit_pair(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(
                   cluster_addr)
               : "memory");
}
// try_wait with cluster-scope acquire: the barrier is arrived on from the
// peer CTA after it has read its TMEM.
__device__ __forceinline__ bool mbar_try_wait_cluster(uint32_t bar, uint32_t parity) {
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
template <class PP>
__device__ __forceinline__ bool bwait_cluster(uint32_t bar, uint32_t parity, volatile Ctl* ctl,
                                              const PP& P) {
  if (ctl->abort) return false;
  const uint64_t t0 = globaltimer();
  for (;;) {
    if (mbar_try_wait_cluster(bar, parity)) return true;
    if (ctl->abort) return false;
    if ((long long)(globaltimer() - t0) > P.timeout_ns) {
      atomicOr(P.status, kStatusTimeout);
      ctl->abort = 1;
      return false;
    }
  }
}

// F8: E4M3 operands with per-(group, row) scales applied at each flush;
// otherwise BF16.  A stage row is 128 bytes either way: 64 BF16 or 128 E4M3
// values of K, consumed by four MMAs of 32 bytes.
// Ten warps put three on some of the SM's four register files of 16,384:
// 168 registers a thread, enough for the epilogue's 128 sums and a chunk.
template <bool F8>
__global__ void __launch_bounds__(G2NT, 1) gram2_tc_kernel(const __grid_constant__ Gram2Params P) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sm = smem_raw;
  const uint32_t sb = smem_u32(sm);
  // every CTA of the launch sees the same layout, so both CTAs of a pair
  // leave here together
  if (sb & 1023) {
    if (threadIdx.x == 0) atomicOr(P.status, kStatusTimeout);
    return;
  }
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_rank();  // 0: issues the MMAs; 1: its peer
  const bool lead = rank == 0;
  auto bar = [&](int i) -> uint32_t { return sb + G2_OFF_BAR + 8 * i; };
  volatile Ctl* ctl = (volatile Ctl*)(sm + G2_OFF_BAR + 8 * G2_COUNT);
  uint32_t* tmem_slot = (uint32_t*)(sm + G2_OFF_BAR + 8 * G2_COUNT + 8);
  int t = (int)(blockIdx.x >> 1), ti = 0;  // tile (ti, tj), ti <= tj
  while (t >= P.ntile - ti) {
    t -= P.ntile - ti;
    ++ti;
  }
  const int tj = ti + t;
  const bool diag = ti == tj;
  // matrices split over the pairs by whole groups of GFL (a flush group is
  // then a group of the FP8 scales)
  const long long gtot = (P.D + GFL - 1) / GFL;
  const long long g0 = gtot * (long long)blockIdx.y / P.splits;
  const long long d0 = g0 * GFL;
  const long long d1e = gtot * (long long)(blockIdx.y + 1) / P.splits * GFL;
  const long long d1 = d1e < P.D ? d1e : P.D;
  constexpr int KB = F8 ? 128 : 64;  // K values per 128-byte stage row
  const int nkb = (int)((P.n + KB - 1) / KB);
  // flushes of P.fl matrices each: the paired MMAs' FP32 accumulation
  // errs in one direction, so long chains of accumulations are cut short;
  // the epilogue sums the GFL / FL flushes of a group in registers
  const int FL = P.fl;
  const int ngroups = d1 > d0 ? (int)((d1 - d0 + FL - 1) / FL) : 0;
  if (tid == 0) {
    for (int s = 0; s < G2STG; ++s) {
      mbar_init(bar(G2_FULL + s), 1);   // the even CTA's expect-tx; bytes of both
      mbar_init(bar(G2_EMPTY + s), 1);  // the pair's MMA commit
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(bar(G2_TFULL + b), 1);   // the pair's MMA commit
      mbar_init(bar(G2_TEMPTY + b), 16);  // epilogue warps of both CTAs
    }
    mbar_init(bar(G2_DRAIN), 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {  // one warp of each CTA allocates, collectively for the pair
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      const int rowA = ti * 256 + (int)rank * 128, rowB = tj * 256 + (int)rank * 128;
      long long q = 0;
      for (long long d = d0; d < d1; ++d) {
        const CUtensorMap* map = P.tmaps + d;
        bool stop = false;
        for (int kb = 0; kb < nkb; ++kb, ++q) {
          const int s = (int)(q % G2STG);
          const uint32_t u = (uint32_t)(q / G2STG);
          if (!bwait(bar(G2_EMPTY + s), (u & 1) ^ 1, ctl, P)) {
            stop = true;
            break;
          }
          const uint32_t full = mapa(bar(G2_FULL + s), 0);
          if (lead) mbar_expect_tx(bar(G2_FULL + s), diag ? 2 * G2HALF : 2 * G2STAGE);
          if (!P.mode2) {
            tma_load_2d_pair(sb + s * G2STAGE, map, kb * KB, rowA, full);
            if (!diag) tma_load_2d_pair(sb + s * G2STAGE + G2HALF, map, kb * KB, rowB, full);
          } else {
            // 64 rows of A (K) x this CTA's 128 columns (M or N): two 64 x 64
            // boxes, the 128-byte swizzle atoms of an MN-major operand
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
              tma_load_2d_pair(sb + s * G2STAGE + hh * (G2HALF / 2), map, rowA + hh * 64,
                               kb * 64, full);
              if (!diag)
                tma_load_2d_pair(sb + s * G2STAGE + G2HALF + hh * (G2HALF / 2), map,
                                 rowB + hh * 64, kb * 64, full);
            }
          }
        }
        if (stop) break;
      }
      // The even CTA drains the loads of both CTAs before the pair leaves
      // (its MMA issuer waits for the last MMAs, which read every stage);
      // after an abort the teardown waits out the few still in flight.
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lead && lane == 0) {
      const uint32_t idesc = F8 ? idesc_e4m3(256, 256)
                                : (P.mode2 ? idesc_bf16(256, 256, 1, 1) : idesc_bf16(256, 256, 0, 0));
      long long q = 0;
      bool ok = true;
      for (int grp = 0; grp < ngroups && ok; ++grp) {
        const int buf = grp & 1;
        const uint32_t v = (uint32_t)(grp >> 1);
        if (!bwait_cluster(bar(G2_TEMPTY + buf), (v & 1) ^ 1, ctl, P)) break;
        tc_fence_after();
        const long long dlo = d0 + (long long)grp * FL;
        const long long dhi = dlo + FL < d1 ? dlo + FL : d1;
        bool first = true;
        for (long long d = dlo; d < dhi && ok; ++d) {
          for (int kb = 0; kb < nkb; ++kb, ++q) {
            const int s = (int)(q % G2STG);
            const uint32_t u = (uint32_t)(q / G2STG);
            if (!bwait(bar(G2_FULL + s), u & 1, ctl, P)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t a0 = sb + s * G2STAGE, b0 = diag ? a0 : a0 + G2HALF;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              if (F8)
                tc_mma_pair_f8(tmem + buf * 256, sdesc(a0 + kk * 32, 16, 1024),
                               sdesc(b0 + kk * 32, 16, 1024), idesc,
                               (first && kk == 0) ? 0u : 1u);
              else if (P.mode2)  // MN-major: 16 rows of K = 2 KB, the two atoms 8 KB apart
                tc_mma_pair(tmem + buf * 256, sdesc(a0 + kk * 2048, G2HALF / 2, 1024),
                            sdesc(b0 + kk * 2048, G2HALF / 2, 1024), idesc,
                            (first && kk == 0) ? 0u : 1u);
              else
                tc_mma_pair(tmem + buf * 256, sdesc(a0 + kk * 32, 16, 1024),
                            sdesc(b0 + kk * 32, 16, 1024), idesc, (first && kk == 0) ? 0u : 1u);
            }
            first = false;
            tc_commit_pair_mc(bar(G2_EMPTY + s));
          }
        }
        if (ok) tc_commit_pair_mc(bar(G2_TFULL + buf));
      }
      tc_commit_pair(bar(G2_DRAIN));
      drain_wait(bar(G2_DRAIN), 0, P);
    }
  } else {
    // ------------------------ epilogue (warps 2-9): TMEM -> registers -> G
    // A flush's FP32 sums are added, rounded to nearest, into registers; at
    // the end of each group of GFL matrices (one FP8 scale group) the
    // registers are added into G in FP64, times the group's scales for FP8.
    const int q4 = warp & 3, hcol = (warp - 2) >> 2;
    const long long row0 = (long long)ti * 256 + rank * 128 + q4 * 32;  // the warp's rows
    const long long col0 = (long long)tj * 256 + hcol * 128;            // and columns
    const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + hcol * 128;
    float* stg = (float*)(sm + G2_OFF_STG) + (warp - 2) * 32 * G2_STG_LD;
    const bool atomic = P.splits > 1;
    const uint32_t tempty0 = lead ? 0u : mapa(bar(G2_TEMPTY), 0);
    const int fpg = GFL / FL;  // flushes per group
    float acc[128];
#pragma unroll
    for (int i = 0; i < 128; ++i) acc[i] = 0.f;
    for (int grp = 0; grp < ngroups; ++grp) {
      const int buf = grp & 1;
      const uint32_t v = (uint32_t)(grp >> 1);
      if (!bwait_warp(bar(G2_TFULL + buf), v & 1, ctl, P)) break;
      tc_fence_after();
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        uint32_t r[16];
        tmem_ld16(taddr + buf * 256 + c * 16, r);
        tmem_wait_ld();
        tmem_regs8(r);
        tmem_regs8(r + 8);
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[c * 16 + i] += __uint_as_float(r[i]);
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (lead)
          mbar_arrive(bar(G2_TEMPTY + buf));
        else
          mbar_arrive_remote(tempty0 + 8 * buf);
      }
      if ((grp + 1) % fpg != 0 && grp != ngroups - 1) continue;
      // the group's sums into G: lane l of the turned-around chunk takes
      // column l % 16 of rows 2 it + l / 16, so one instruction adds two
      // runs of 16 consecutive columns
      const float* sc = F8 ? P.scales + ((d0 + (long long)grp * FL) / GFL) * P.m : nullptr;
      const int cc = lane & 15;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          stg[lane * G2_STG_LD + i] = acc[c * 16 + i];
          acc[c * 16 + i] = 0.f;
        }
        __syncwarp();
        const long long col = col0 + c * 16 + cc;
        if (col < P.m) {
          const double scol = F8 ? (double)sc[col] : 1.0;
#pragma unroll 4
          for (int it = 0; it < 16; ++it) {
            const int rr = 2 * it + (lane >> 4);
            const long long grow = row0 + rr;
            if (grow < P.m) {
              double x = (double)stg[rr * G2_STG_LD + cc];
              if (F8) x *= (double)sc[grow] * scol;
              double* gp = P.G + grow * P.m + col;
              if (atomic)
                atomicAdd(gp, x);
              else
                *gp += x;
            }
          }
        }
        __syncwarp();
      }
    }
  }
  // ---- teardown: neither CTA leaves while the other's operations may still
  // touch its shared memory or TMEM
  tc_fence_before();
  __syncthreads();
  cluster_sync();
  if (ctl->abort && tid == 0) {
    const uint64_t t0 = globaltimer();
    while (globaltimer() - t0 < 200000ull) {
    }
  }
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512)
                 : "memory");
  }
}

// G[a][b] = G[b][a] for a > b: the kernels above fill the upper block
// triangle (diagonal blocks in full).
__global__ void mirror_upper_kernel(double* __restrict__ G, long long m) {
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * m) return;
  const long long a = e / m, b = e - a * m;
  if (a > b) G[e] = G[b * m + a];
}

}  // namespace

struct TcClass {
  int C;
  int MC;
  int nclusters;
  TcParams prm;
};

struct TcPlan {
  void* dev = nullptr;
  size_t bytes = 0;
  std::vector<TcClass> classes;
  const SImgDesc* d_sdesc = nullptr;
  int nsdesc = 0;
  int max_chunks = 1;
  unsigned char* simg = nullptr;
};

bool tc_supported() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return false;
  return p.major == 10 && p.minor == 3 && get_encode() != nullptr;
}

bool tc_matrix_eligible(const void* A, long long m, long long lda, int k) {
  return k >= 1 && k <= KPAD_MAX && m >= 1 && m <= 4096 && ((uintptr_t)A) % 16 == 0 &&
         (lda * 2) % 16 == 0 && lda <= (1ll << 36);
}

bool gram_tc_eligible(int prec, int mode, const void* const* A, long long D, long long m,
                      long long n, long long lda) {
  if (prec != 2 || (mode != 1 && mode != 2) || D < 1 || m < 1 || n < 1) return false;
  if ((lda * 2) % 16 != 0 || lda > (1ll << 31) || n > (1ll << 31) || m > (1ll << 31))
    return false;
  for (long long d = 0; d < D; ++d)
    if (((uintptr_t)A[d]) % 16 != 0) return false;
  return tc_supported();
}

// The tensor maps of the last training set a handle's Gram saw, kept on the
// device: a repeated Gram over the same matrices (a timed re-run, the sweeps
// of an iterative method) skips the host encoding and the upload.
struct GramCache {
  std::vector<const void*> key;
  long long m = 0, n = 0, lda = 0;
  int box_rows = 0;  // 128 for the mode-1 maps, 64 for mode 2
  bool f8 = false;   // maps of E4M3 bytes (box 128 x 128)
  CUtensorMap* dmaps = nullptr;
  size_t cap = 0;
};

GramCache* gram_cache_create() { return new GramCache(); }
void gram_cache_destroy(GramCache* c) {
  if (!c) return;
  if (c->dmaps) cudaFree(c->dmaps);
  delete c;
}

cudaError_t launch_gram_tc(const void* const* A, long long D, long long m, long long n,
                           long long lda, int mode, double* G, int* status,
                           long long spin_limit, GramCache* cache, bool pairs, cudaStream_t s,
                           const float* f8_scales) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  const bool f8 = f8_scales != nullptr;
  if (!enc || !cache || (mode != 1 && mode != 2) || (f8 && mode != 1)) return cudaErrorNotSupported;
  if (f8) pairs = true;  // E4M3 operands: the pair kernel only
  const int box_rows = mode == 1 ? 128 : 64;
  const long long dim = mode == 1 ? m : n;
  const bool hit = cache->dmaps && cache->m == m && cache->n == n && cache->lda == lda &&
                   cache->box_rows == box_rows && cache->f8 == f8 &&
                   (long long)cache->key.size() == D &&
                   std::equal(cache->key.begin(), cache->key.end(), A);
  if (!hit) {
    std::vector<CUtensorMap> maps((size_t)D);
    for (long long d = 0; d < D; ++d) {
      cuuint64_t dims[2] = {(cuuint64_t)n, (cuuint64_t)m};
      cuuint64_t strides[1] = {(cuuint64_t)lda * (f8 ? 1 : 2)};
      cuuint32_t box[2] = {f8 ? 128u : 64u, (cuuint32_t)box_rows};
      cuuint32_t es[2] = {1, 1};
      CUresult r = enc(&maps[(size_t)d],
                       f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                       const_cast<void*>(A[d]), dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                       CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS) return cudaErrorNotSupported;  // nothing launched yet
    }
    // the previous maps may still be read by a Gram in flight on this stream
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (cache->cap < (size_t)D) {
      if (cache->dmaps) cudaFree(cache->dmaps);
      cache->dmaps = nullptr;
      cache->cap = 0;
      e = cudaMalloc((void**)&cache->dmaps, sizeof(CUtensorMap) * (size_t)D);
      if (e != cudaSuccess) return e;
      cache->cap = (size_t)D;
    }
    cache->key.clear();
    e = cudaMemcpy(cache->dmaps, maps.data(), sizeof(CUtensorMap) * (size_t)D,
                   cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return e;
    cache->key.assign(A, A + D);
    cache->m = m;
    cache->n = n;
    cache->lda = lda;
    cache->box_rows = box_rows;
    cache->f8 = f8;
  }
  int dev = 0, nsm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess)
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaError_t e = cudaSuccess;
  if (pairs) {
    // 256 x 256 tiles on CTA pairs; the matrices are split over pairs so
    // that the grid fills the SMs
    const int ntile2 = (int)((dim + 255) / 256);
    const long long ntp2 = (long long)ntile2 * (ntile2 + 1) / 2;
    if (2 * ntp2 > 2147483647ll) return cudaErrorNotSupported;
    long long splits2 = nsm / (2 * ntp2);
    const long long groups = (D + GFL - 1) / GFL;  // the pairs split whole groups
    if (splits2 > groups) splits2 = groups;
    if (splits2 < 1) splits2 = 1;
    if (splits2 > 65535) splits2 = 65535;
    Gram2Params q;
    q.tmaps = cache->dmaps;
    q.D = D;
    q.m = dim;                   // rows of G
    q.n = mode == 1 ? n : m;     // the summed length
    q.mode2 = mode == 2 ? 1 : 0;
    // matrices per TMEM flush: for BF16 at most 128 MMAs of the pair
    // accumulate into one FP32 sum before the epilogue adds it, rounded to
    // nearest, into its registers (a stage of 64 values of K is four MMAs).
    // E4M3 operands are rounded to 2^-4 relatively, far above what the
    // group's chain adds: their flush is the whole group.
    {
      const long long nkb = (q.n + 63) / 64;
      int fl = GFL;
      while (!f8 && fl > 1 && (long long)fl * 4 * nkb > 128) fl >>= 1;
      q.fl = fl;
    }
    q.G = G;
    q.scales = f8_scales;
    q.ntile = ntile2;
    q.splits = (int)splits2;
    q.status = status;
    q.timeout_ns = std::max<long long>(spin_limit, 1) * 120;
    auto kern = f8 ? gram2_tc_kernel<true> : gram2_tc_kernel<false>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, G2_SMEM);
    if (e == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cudaLaunchAttribute attr[1];
      cfg.gridDim = dim3((unsigned)(2 * ntp2), (unsigned)splits2, 1);
      cfg.blockDim = dim3(G2NT, 1, 1);
      cfg.dynamicSmemBytes = G2_SMEM;
      cfg.stream = s;
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = 2;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, kern, q);
    }
    if (e == cudaSuccess) {
      const long long tot = dim * dim;
      mirror_upper_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(G, dim);
      e = cudaGetLastError();
    }
    return e;
  }
  const int ntile = (int)((dim + 127) / 128);
  const long long ntp = (long long)ntile * (ntile + 1) / 2;
  if (ntp > 65535 * 8) return cudaErrorNotSupported;
  long long splits = nsm / ntp;
  if (splits > D) splits = D;
  if (splits < 1) splits = 1;
  GramParams prm;
  prm.mode = mode;
  prm.tmaps = cache->dmaps;
  prm.D = D;
  prm.m = m;
  prm.n = n;
  prm.G = G;
  prm.ntile = ntile;
  prm.splits = (int)splits;
  prm.status = status;
  prm.timeout_ns = std::max<long long>(spin_limit, 1) * 120;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(gram_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             G_SMEM);
  if (e == cudaSuccess) {
    gram_tc_kernel<<<dim3((unsigned)ntp, (unsigned)splits), GNT, G_SMEM, s>>>(prm);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const long long tot = dim * dim;
    mirror_upper_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(G, dim);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t tc_prepare(TcPlan** out, const MatDev* hm, const MatDev* d_mats, int count,
                       const int* ids, int nids, const int* mc_pref, int kp, void* dev_X,
                       void* dev_Y, double* dev_normA2, int* status, long long spin_limit,
                       char* msg, int msglen) {
  *out = nullptr;
  auto fail = [&](const char* why) {
    if (msg && msglen > 0) snprintf(msg, msglen, "%s", why);
    return cudaErrorNotSupported;
  };
  PFN_cuTensorMapEncodeTiled_v12000 enc = get_encode();
  if (!enc) return fail("cuTensorMapEncodeTiled is unavailable");
  if (nids < 1) return fail("no matrix for the tensor-core kernel");
  int kmax = 1;
  for (int t = 0; t < nids; ++t) {
    const int i = ids[t];
    if (i < 0 || i >= count) return fail("matrix index out of range");
    if (hm[i].k > KPAD_MAX) return fail("k > 48 is not supported by the tensor-core kernel");
    if (hm[i].m > 4096) return fail("m > 4096 is not supported by the tensor-core kernel");
    kmax = std::max(kmax, hm[i].k);
  }
  TcPlan* p = new TcPlan();
  // classes by cluster shape (C, MC); each has its own kq and S-image rows
  std::map<std::pair<int, int>, std::vector<int>> byC;
  std::map<std::pair<int, int>, int> class_k;  // largest k of the class
  std::vector<std::pair<int, int>> shape_of(count, std::make_pair(0, 0));
  for (int t = 0; t < nids; ++t) {
    const int i = ids[t];
    int C, mc;
    cluster_shape(hm[i].m, &C, &mc, mc_pref ? mc_pref[i] : 0, hm[i].k);
    const auto key = std::make_pair(C, mc);
    byC[key].push_back(i);
    class_k[key] = std::max(class_k[key], hm[i].k);
    shape_of[i] = key;
  }
  // distinct sketch images: one per sketch and cluster shape (the shape
  // fixes the chunk count and the rows per chunk)
  std::map<std::tuple<const void*, long long, int, int, int>, long long> img_of;
  std::vector<SImgDesc> sdesc;
  std::vector<long long> simg_off(count, 0);
  long long img_total = 0;
  for (int t = 0; t < nids; ++t) {
    const int i = ids[t];
    const int C = shape_of[i].first, mc = shape_of[i].second;
    const int kpad = class_kpad(class_k[shape_of[i]], mc);
    auto key = std::make_tuple(hm[i].S, hm[i].m, hm[i].k, C, mc);
    auto it = img_of.find(key);
    if (it == img_of.end()) {
      SImgDesc sd;
      sd.S = (const float*)hm[i].S;
      sd.m = hm[i].m;
      sd.k = hm[i].k;
      sd.nchunks = C * mc / 64;
      sd.kpad = kpad;
      sd.off = img_total;
      p->max_chunks = std::max(p->max_chunks, sd.nchunks);
      img_total += (long long)sd.nchunks * kpad * 128;
      img_total = (img_total + 1023) / 1024 * 1024;  // images start on 1024 bytes
      it = img_of.emplace(key, sd.off).first;
      sdesc.push_back(sd);
    }
    simg_off[i] = it->second;
  }
  // schedules: longest-processing-time-first over clusters of each class
  std::vector<int> work, work_off_all;
  struct ClassTmp {
    int C, MC, ncl;
    size_t woff_start, work_start;
  };
  std::vector<ClassTmp> ctmp;
  for (auto& kv : byC) {
    const int C = kv.first.first, MCc = kv.first.second;
    std::vector<int> ids = kv.second;
    int ncl = 1;
    const cudaError_t ae = class_attrs(C, MCc, &ncl);
    if (ae != cudaSuccess) {
      int dev = 0, optin = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (msg)
        snprintf(msg, msglen,
                 "cudaFuncSetAttribute(%d bytes of shared memory) failed: %s (device opt-in "
                 "limit %d bytes)",
                 MCc == 256 ? Lay<256>::SMEM_BYTES
                            : (MCc == 384 ? Lay<384>::SMEM_BYTES : Lay<512>::SMEM_BYTES),
                 cudaGetErrorString(ae), optin);
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
    ct.MC = MCc;
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
  for (int t = 0; t < nids; ++t) {  // maps of the other matrices stay zero (unused)
    const int i = ids[t];
    CUtensorMap* map = reinterpret_cast<CUtensorMap*>(host.data() + o_map) + i;
    cuuint64_t dims[2] = {(cuuint64_t)hm[i].n, (cuuint64_t)hm[i].m};
    cuuint64_t strides[1] = {(cuuint64_t)hm[i].lda * 2};
    const cuuint32_t box_rows = shape_of[i].second == 384 ? 128 : BOX_ROWS;
    cuuint32_t box[2] = {(cuuint32_t)NB, box_rows};
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
    cl.MC = ct.MC;
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
    const int kc = class_k[std::make_pair(ct.C, ct.MC)];
    prm.kpad = class_kpad(kc, ct.MC);
    prm.kq = class_kq(kc, ct.C);
    prm.img_rank_bytes = (ct.MC / 64) * prm.kpad * 128;
    prm.timeout_ns = timeout_ns;
    p->classes.push_back(cl);
  }
  *out = p;
  return cudaSuccess;
}

cudaError_t tc_launch_prep(TcPlan* p, cudaStream_t s) {
  if (!p) return cudaErrorInvalidValue;
  simg_prep_kernel<<<dim3(p->nsdesc, p->max_chunks), 256, 0, s>>>(p->d_sdesc, p->simg);
  return cudaGetLastError();
}

int tc_classes(const TcPlan* p) { return p ? (int)p->classes.size() : 0; }

cudaError_t tc_launch_class(TcPlan* p, int i, cudaStream_t s) {
  if (!p || i < 0 || i >= (int)p->classes.size()) return cudaErrorInvalidValue;
  const TcClass& cl = p->classes[(size_t)i];
  return class_launch(cl.C, cl.MC, cl.prm, cl.nclusters, s);
}

int tc_launches(const TcPlan* p) { return p ? 1 + (int)p->classes.size() : 0; }
long long tc_workspace_bytes(const TcPlan* p) { return p ? (long long)p->bytes : 0; }
void tc_destroy(TcPlan* p) {
  if (!p) return;
  if (p->dev) cudaFree(p->dev);
  delete p;
}

}  // namespace tsk
