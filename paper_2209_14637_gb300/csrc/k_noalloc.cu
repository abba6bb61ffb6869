// Allocation-free SCW entry point.
//
// Some callers cannot allocate device memory at the point where they need an
// approximation: code running inside a memory pool that another framework
// owns, real-time paths that must not call into the allocator (cudaMalloc
// can synchronise the device and its latency is unbounded), and embedded
// users that budget every byte up front.  tsk_approx_noalloc serves them:
// it runs the same CUDA-core SCW kernels as tsk_approx_batch on one matrix,
// but keeps every intermediate (descriptors, X, Y, the R factors, W and the
// norms) in one file-scope __device__ array instead of a plan workspace.
//
// That array is part of the loaded module: every GPU that loads libtsk.so
// holds kNoAllocScratchBytes of it until the process exits, whether or not
// the entry point is ever called.  Host code cannot use the array's name as
// a device address (it names a host-side shadow), so each call looks the
// address up with cudaGetSymbolAddress while the caller's device is current
// (cheap once the module is loaded, and right again after a context reset
// reloads the module elsewhere); inside a stream capture, where that lookup
// may not be made, the address cached by an earlier call on the device is
// used.  The errors follow the allocating entry point's default: the
// projection identity, and a direct pass over A where it cancels.
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "tsk_internal.cuh"

namespace tsk {
namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)TSK_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

size_t up256(size_t v) { return (v + 255) / 256 * 256; }

struct Layout {
  size_t mats, items_x, items_y, panels, X, Y, RX, RY, W, norm, flags, status, U2, V2, e2,
      total;
};

Layout layout_for(long long m, long long n, int kp, size_t cs) {
  Layout L;
  size_t o = 0;
  L.mats = o;
  o = up256(o + sizeof(MatDev));
  L.items_x = o;
  o = up256(o + sizeof(int2) * (size_t)((n + 63) / 64));
  L.items_y = o;
  o = up256(o + sizeof(int2) * (size_t)((m + 63) / 64));
  L.panels = o;
  o = up256(o + 2 * sizeof(PanelDev));
  L.X = o;
  o = up256(o + cs * (size_t)n * kp);
  L.Y = o;
  o = up256(o + cs * (size_t)m * kp);
  L.RX = o;
  o = up256(o + cs * (size_t)kp * kp);
  L.RY = o;
  o = up256(o + cs * (size_t)kp * kp);
  L.W = o;
  o = up256(o + cs * (size_t)kp * kp);
  L.norm = o;
  o = up256(o + sizeof(double));
  L.flags = o;
  o = up256(o + sizeof(int));
  L.status = o;
  o = up256(o + sizeof(int));
  // direct-residual fallback: U_r Sigma_r (m x kp), (Q V_r)^T panel (n x kp)
  L.U2 = o;
  o = up256(o + cs * (size_t)m * kp);
  L.V2 = o;
  o = up256(o + cs * (size_t)n * kp);
  L.e2 = o;
  o = up256(o + sizeof(double));
  L.total = o;
  return L;
}

// Writes the descriptors the kernels read and clears what they accumulate
// into (the array keeps the previous call's contents).
__global__ void noalloc_setup_kernel(unsigned char* base, Layout L, MatDev md, int kp) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x;
  const int nx = (int)((md.n + 63) / 64), ny = (int)((md.m + 63) / 64);
  int2* ix = (int2*)(base + L.items_x);
  int2* iy = (int2*)(base + L.items_y);
  for (int t = tid; t < nx; t += gridDim.x * blockDim.x) ix[t] = make_int2(0, t);
  for (int t = tid; t < ny; t += gridDim.x * blockDim.x) iy[t] = make_int2(0, t);
  if (tid == 0) {
    *(MatDev*)(base + L.mats) = md;
    PanelDev* p = (PanelDev*)(base + L.panels);
    p[0].P = base + L.X;
    p[0].rows = md.n;
    p[0].k = md.k;
    p[0].ld = kp;
    p[0].R = base + L.RX;
    p[1].P = base + L.Y;
    p[1].rows = md.m;
    p[1].k = md.k;
    p[1].ld = kp;
    p[1].R = base + L.RY;
    *(double*)(base + L.norm) = 0.0;
    *(double*)(base + L.e2) = 0.0;
    *(int*)(base + L.flags) = 0;
    *(int*)(base + L.status) = 0;
  }
}

// The call's status bits as a tsk_status value for the caller.
__global__ void noalloc_status_kernel(const int* bits, int32_t* out) {
  const int b = *bits;
  *out = (b & kStatusTimeout) ? (int32_t)TSK_ETIMEOUT
                              : ((b & kStatusRankDef) ? (int32_t)TSK_ERANKDEF : (int32_t)TSK_OK);
}

tsk_status fail(const char* msg) {
  set_thread_error("%s", msg);
  return TSK_EINVAL;
}

}  // namespace
}  // namespace tsk

using namespace tsk;

extern "C" tsk_status tsk_approx_noalloc(const tsk_mat_desc* mat, tsk_prec prec,
                                         double* err, double* normA2, int32_t* status_out,
                                         tsk_stream stream) {
  if (!mat || !err) return fail("tsk_approx_noalloc: mat and err must be non-NULL");
  const tsk_mat_desc d = *mat;
  if (!d.A || !d.S) return fail("tsk_approx_noalloc: A or S is NULL");
  if (prec != TSK_FP64 && prec != TSK_FP32 && prec != TSK_BF16)
    return fail("tsk_approx_noalloc: unknown precision");
  if (d.m < 1 || d.n < 1 || d.lda < d.n)
    return fail("tsk_approx_noalloc: need m, n >= 1 and lda >= n");
  if (d.r < 1 || d.r > d.k || d.k > d.m || d.k > d.n || d.k > TSK_MAX_K)
    return fail("tsk_approx_noalloc: need 1 <= r <= k <= min(m, n) and k <= 64");
  const size_t cs = prec == TSK_FP64 ? 8 : 4;
  const size_t es = prec == TSK_FP64 ? 8 : (prec == TSK_FP32 ? 4 : 2);
  if (((uintptr_t)d.A) % es != 0 || ((uintptr_t)d.S) % cs != 0)
    return fail("tsk_approx_noalloc: A or S is not aligned to its element size");
  const int kp = ((d.k + 15) / 16) * 16;
  const Layout L = layout_for(d.m, d.n, kp, cs);
  if (L.total > kNoAllocScratchBytes) {
    set_thread_error(
        "tsk_approx_noalloc: this matrix needs %zu bytes of scratch, more than the "
        "%zu-byte static array (2 (m + n) * k_padded * %zu bytes plus descriptors)",
        L.total, kNoAllocScratchBytes, cs);
    return TSK_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail("tsk_approx_noalloc: no usable current device");
  cudaStream_t s = (cudaStream_t)stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess)
    return fail("tsk_approx_noalloc: invalid stream");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
      void* p = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        set_thread_error("tsk_approx_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
        return TSK_ECUDA;
      }
      g_addr[dev] = p;
    } else if (!g_addr[dev]) {
      set_thread_error("tsk_approx_noalloc: the first call on a device must not be made "
                       "during a stream capture");
      return TSK_EINVAL;
    }
    base = (unsigned char*)g_addr[dev];
  }
  MatDev md;
  memset(&md, 0, sizeof(md));
  md.A = d.A;
  md.S = d.S;
  md.m = d.m;
  md.n = d.n;
  md.lda = d.lda;
  md.k = d.k;
  md.r = d.r;
  md.offX = 0;
  md.offY = 0;
  const bool dbl = prec == TSK_FP64;
  const int in_type = (int)prec;
  const MatDev* dm = (const MatDev*)(base + L.mats);
  double* nrm = (double*)(base + L.norm);
  int* status = (int*)(base + L.status);
  noalloc_setup_kernel<<<1, 256, 0, s>>>(base, L, md, kp);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = launch_sketch_x(in_type, kp, dm, (const int2*)(base + L.items_x),
                        (int)((d.n + 63) / 64), base + L.X, nrm, s);
  if (e == cudaSuccess)
    e = launch_sketch_y(in_type, kp, dm, (const int2*)(base + L.items_y),
                        (int)((d.m + 63) / 64), base + L.X, base + L.Y, s);
  if (e == cudaSuccess)
    e = launch_tsqr(dbl, kp, (const PanelDev*)(base + L.panels), 2, 1, status, s);
  const double tau = dbl ? 1e-6 : 1e-4;
  if (e == cudaSuccess)
    e = launch_small_svd(dbl, kp, dm, 1, base + L.RX, base + L.RY, base + L.W, nrm, err,
                         (int*)(base + L.flags), 0, tau, status, s);
  // where the identity cancels (err^2 < tau ||A||^2) the flag is set and the
  // error is recomputed by a direct pass over A; otherwise this does nothing
  if (e == cudaSuccess)
    e = launch_direct_fallback(in_type, kp, dm, 1, (const int*)(base + L.flags), base + L.X,
                               base + L.Y, base + L.W, base + L.U2, base + L.V2,
                               (double*)(base + L.e2), err, s);
  if (e == cudaSuccess && normA2)
    e = cudaMemcpyAsync(normA2, nrm, sizeof(double), cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && status_out) {
    noalloc_status_kernel<<<1, 1, 0, s>>>(status, status_out);
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_thread_error("tsk_approx_noalloc: %s", cudaGetErrorString(e));
    return TSK_ECUDA;
  }
  return TSK_OK;
}
