// Internal declarations shared by the CUDA translation units of libtsk.
// Nothing here is part of the C ABI (include/tsk.h is).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/tsk.h"

namespace tsk {

// Bits of the device status word (most severe wins when reported).
enum : int {
  kStatusRankDef = 1,  // |R_jj| of a sketch panel fell below the threshold
  kStatusTimeout = 2,  // a bounded spin-wait ran out
};

// One test-side matrix as the kernels see it.  X (n x kp) and Y (m x kp) are
// per-matrix panels in the plan workspace; kp is the batch-wide padded k.
struct MatDev {
  const void* A;
  const void* S;
  long long m, n, lda;
  int k, r;
  long long offX, offY;  // element offsets of X and Y in the workspace
  void* US;
  void* Vt;
  void* sigma;
};

// A tall panel (rows x kp, leading dimension kp) whose R factor is wanted.
struct PanelDev {
  const void* P;  // rows x ld, row-major; columns [0, k) are used
  long long rows;
  int k;
  int ld;
  void* R;  // kp x kp row-major, upper triangle holds R
};

// Two FP32 operations in one instruction (fma / mul .rn.f32x2): lane 0 and
// lane 1 of each pair, each rounded as fmaf / __fmul_rn would round it.
__device__ __forceinline__ void ffma2(float& d0, float& d1, float a0, float a1, float b0,
                                      float b1) {
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mov.b64 rd, {%0, %1};\n\tfma.rn.f32x2 rd, ra, rb, rd;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "+f"(d0), "+f"(d1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}
__device__ __forceinline__ void fmul2(float& d0, float& d1, float a0, float a1, float b0,
                                      float b1) {
  asm("{\n\t.reg .b64 ra, rb, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "mul.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(d0), "=f"(d1)
      : "f"(a0), "f"(a1), "f"(b0), "f"(b1));
}

// Element conversions used by the loaders.
__device__ __forceinline__ float to_float(float x) { return x; }
__device__ __forceinline__ float to_float(double x) { return (float)x; }
__device__ __forceinline__ float to_float(__nv_bfloat16 x) {
  return __bfloat162float(x);
}
template <typename Tc, typename Tin>
__device__ __forceinline__ Tc convert_in(Tin x) {
  return (Tc)to_float(x);
}
template <>
__device__ __forceinline__ double convert_in<double, double>(double x) {
  return x;
}

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sets the calling thread's error text (what tsk_last_error(NULL) returns).
void set_thread_error(const char* fmt, ...);

// ---- launchers (host functions), defined in the .cu files ---------------

// k_simt.cu
// A BF16 matrix whose rows TMA cannot address (row starts off a 16-byte
// boundary) and its copy with a padded leading dimension ldp (n rounded up to
// 8 elements) in the plan's workspace, which the tensor-core kernel reads.
struct PackDev {
  const void* src;
  void* dst;
  long long m, n, lda, ldp;
};
// Copies rows [8 t, 8 t + 8) of pack items[i].x for t = items[i].y; the
// padding columns [n, ldp) are not written (the tensor maps stop at n).
cudaError_t launch_pack_rows(const PackDev* packs, const int2* items, int nitems,
                             cudaStream_t s);
cudaError_t launch_sketch_x(int in_type, int kp, const MatDev* mats,
                            const int2* items, int nitems, void* X,
                            double* normA2, cudaStream_t s);
cudaError_t launch_sketch_y(int in_type, int kp, const MatDev* mats,
                            const int2* items, int nitems, const void* X,
                            void* Y, cudaStream_t s);
cudaError_t launch_gram(int in_type, const void* const* dA, long long D,
                        long long m, long long n, long long lda, int mode,
                        double* G, cudaStream_t s);
// C = alpha op(A) op(B) + beta C (row-major); with a workspace of
// work_bytes the K range is split over CTAs and summed in a second kernel.
cudaError_t launch_gemm(bool dbl, int transA, int transB, long long M,
                        long long N, long long K, double alpha, const void* A,
                        long long lda, const void* B, long long ldb,
                        double beta, void* C, long long ldc, cudaStream_t s,
                        void* work = nullptr, size_t work_bytes = 0);
// Ri = R^{-1} with R the upper Cholesky factor of Gm (R^T R = Gm), p <= 96,
// one CTA; Gm and Ri may be the same array.
cudaError_t launch_chol_inv(bool dbl, const void* Gm, int p, void* Ri, cudaStream_t s);
cudaError_t launch_project_out(bool dbl, int kp, const MatDev* mats,
                               const int4* items, int nitems, const void* X,
                               const void* Y, const void* Wm, cudaStream_t s);
cudaError_t launch_direct_error(int in_type, const MatDev* mats,
                                const int2* items, int nitems, double* err2,
                                cudaStream_t s);
cudaError_t launch_sqrt_inplace(double* v, int count, cudaStream_t s);
cudaError_t launch_direct_fallback(int in_type, int kp, const MatDev* mats, int count,
                                   const int* flags, const void* X, const void* Y,
                                   const void* Wm, void* U2, void* V2, double* err2,
                                   double* err, cudaStream_t s);
cudaError_t launch_convert_gram(bool dbl, const double* G, void* out,
                                long long count, cudaStream_t s);
cudaError_t launch_random_fill(bool dbl, void* Z, long long count,
                               unsigned long long seed, cudaStream_t s);
cudaError_t launch_apply_rinv(bool dbl, const void* P, const void* R,
                              void* Q, long long rows, int p, cudaStream_t s);
// P[:, c] /= |theta_c| (theta_c != 0).
cudaError_t launch_scale_cols(bool dbl, void* P, long long rows, int p, const void* theta,
                              cudaStream_t s);
cudaError_t launch_ritz_residual(bool dbl, const void* U, const void* GU,
                                 const void* theta, double* res,
                                 long long rows, int p, int k, cudaStream_t s);
cudaError_t launch_emit_sketch(bool dbl, const void* U, long long rows, int p,
                               int k, void* S, cudaStream_t s);

// k_small.cu
cudaError_t launch_tsqr(bool dbl, int kp, const PanelDev* panels, int count,
                        int refine, int* status, cudaStream_t s);
// sigma_f32 != 0 writes the singular values as float (the FP32 / BF16
// outputs) from the double kernel.
cudaError_t launch_small_svd(bool dbl, int kp, const MatDev* mats, int count,
                             const void* RX, const void* RY, void* Wm,
                             double* normA2, double* err, int* flags,
                             int err_mode, double tau, int* status,
                             cudaStream_t s, int sigma_f32 = 0);
// R factors in double of float panels (the FP64 small-factor route of the
// FP32 / BF16 paths); the panel descriptors point at float data.
cudaError_t launch_tsqr_f32_in_f64(int kp, const PanelDev* panels, int count, int refine,
                                   cudaStream_t s);
cudaError_t launch_sym_eig(bool dbl, const void* H, int p, void* theta,
                           void* V, cudaStream_t s);
// Fused small factors of the FP32 / BF16 paths (k_finish.cu): one CTA per
// matrix takes the X and Y panels to W = R_X^{-1} V_r, sigma and err.
// The small factors of the FP32 / BF16 paths for the matrices ids[0 .. count)
// of mats, all with k rounded up to 8 equal to kc.
cudaError_t launch_finish(int kp, int kc, const int* ids, int count, const MatDev* mats,
                          const PanelDev* xpanels, const PanelDev* ypanels, float* Wm,
                          double* normA2, double* err, int* flags, int err_mode, double tau,
                          int refine, int* status, cudaStream_t s);

// k_refine.cu
cudaError_t launch_zt(bool dbl, int kp, const MatDev* mats, int count, const void* Y,
                      const void* Wm, void* Zt, long long zt_stride, cudaStream_t s);
cudaError_t launch_ivy_grad(bool dbl, int kp, int kp2, int count, long long km,
                            const MatDev* mats, const MatDev* mats2, const void* Wm,
                            const void* sig, const void* Zt, long long zt_stride,
                            const void* Y2, const double* normA2, double scale, void* grad,
                            cudaStream_t s);
cudaError_t launch_axpy(bool dbl, long long n, double alpha, const void* x, void* y,
                        cudaStream_t s);
cudaError_t launch_add(bool dbl, long long n, const void* a, const void* b, void* out,
                       cudaStream_t s);
cudaError_t launch_batch_loss(int count, const double* err, const double* normA2,
                              double* loss, cudaStream_t s);

// k_two_sided.cu
// W (l x n, double for prec 0, float otherwise) -> n x lp panel of W^T.
cudaError_t launch_wt_panel(int prec, const void* W, int l, long long n, int lp, void* out,
                            cudaStream_t s);
// Small factors of two-sided SCW: xm (k, r, offY of Y, sigma) and zm (k = l,
// offY of Z) per matrix; RX, RZ double R factors of the X and Z panels;
// writes err, sigma, WX (k x r, stride kp^2) and WZ (l x r, stride lp^2).
cudaError_t launch_two_sided_small(bool dbl, int kp, int lp, const MatDev* xm,
                                   const MatDev* zm, int count, const void* Y, const void* Z,
                                   const double* RX, const double* RZ, void* WX, void* WZ,
                                   const double* normA2, double* err, int* status,
                                   cudaStream_t s);

// k_tc.cu (tcgen05 / TMA kernels; BF16)
struct TcPlan;
bool tc_supported();
// Mode-1 Gram of BF16 matrices on the tensor cores (A: host array of D device
// pointers, 16-byte aligned, lda * 2 a multiple of 16); adds into G (m x m,
// double) and mirrors its upper triangle into the lower one.  Returns
// cudaErrorNotSupported, having launched nothing, when a tensor map cannot be
// encoded for these shapes.
bool gram_tc_eligible(int prec, int mode, const void* const* A, long long D, long long m,
                      long long n, long long lda);
struct GramCache;
GramCache* gram_cache_create();
void gram_cache_destroy(GramCache* c);
// pairs: 256 x 256 tiles on CTA pairs (tcgen05 .cta_group::2); otherwise
// 128 x 128 tiles on single CTAs.
// mode 1: G (m x m) += sum A A^T; mode 2: G (n x n) += sum A^T A (MN-major
// operands, 128 x 128 tiles on single CTAs).
// f8_scales != NULL: A holds E4M3 bytes (lda in bytes, a multiple of 16)
// with a power-of-two scale per row and group of eight matrices,
// f8_scales[(d / 8) * m + i]; mode 1 only, on CTA pairs.
cudaError_t launch_gram_tc(const void* const* A, long long D, long long m, long long n,
                           long long lda, int mode, double* G, int* status,
                           long long spin_limit, GramCache* cache, bool pairs, cudaStream_t s,
                           const float* f8_scales = nullptr);
// Quantizes D matrices (in_type 1 float, 2 bfloat16; host array of device
// pointers) to E4M3 in A8[d] (ld8 bytes per row) with the per-(group of 8,
// row) power-of-two scales that keep every |value| / scale <= 448.
cudaError_t launch_quantize_e4m3(int in_type, const void* const* dA, long long D, long long m,
                                 long long n, long long lda, unsigned char* const* dA8,
                                 long long ld8, float* scales, bool vec, cudaStream_t s);
// Builds the tensor-core part of a plan for the matrices ids[0..nids) of
// the plan's count matrices (tensor maps, S images, per-class schedules).
// mc_pref (count entries, nullable): per matrix 0 (default shape), 256 or
// 512 rows of A per CTA.
cudaError_t tc_prepare(TcPlan** out, const MatDev* host_mats,
                       const MatDev* dev_mats, int count, const int* ids, int nids,
                       const int* mc_pref, int kp, void* dev_X, void* dev_Y,
                       double* dev_normA2, int* status, long long spin_limit, char* msg,
                       int msglen);
// Whether one BF16 matrix can take the tensor-core sketch: k <= 48,
// m <= 4096, A 16-byte aligned, lda * 2 a multiple of 16.
bool tc_matrix_eligible(const void* A, long long m, long long lda, int k);
// The S images (one small kernel), then one launch per cluster-size class;
// the classes do not depend on each other and may run concurrently.
cudaError_t tc_launch_prep(TcPlan* p, cudaStream_t s);
int tc_classes(const TcPlan* p);
cudaError_t tc_launch_class(TcPlan* p, int i, cudaStream_t s);
int tc_launches(const TcPlan* p);
long long tc_workspace_bytes(const TcPlan* p);
void tc_destroy(TcPlan* p);

}  // namespace tsk
