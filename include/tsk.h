/*
 * tsk.h -- C ABI of the GB300 tensor-based sketching library.
 *
 * The library computes the data-parallel hot path of the tensor-based
 * sketching method for low-rank approximation of a data stream
 * {A_d in R^{m x n}} (arXiv 2209.14637):
 *
 *   training side  G = sum_d A_d A_d^T (mode-1 Gram of the training tensor,
 *                  Section 3.1, Eq. 3.2) and the sketch S (k x m) = its
 *                  leading eigenvectors, S* = (U^(1))_k^T (Eq. 3.3,
 *                  Algorithm 2, lines 1-2); optionally the mode-2 analogue
 *                  sum_d A_d^T A_d -> W (l x n) for the two-sided sketch
 *                  (Eq. 3.6);
 *   test side      for every stream matrix the SCW step (Algorithm 1 in the
 *                  QR form of Section 3.2): X = (S A)^T, X = Q R, A Q,
 *                  truncated rank-r SVD [A Q]_r, B = [A Q]_r Q^T and the
 *                  error ||A - B||_F (problem 1.1).
 *
 * Conventions shared by every call
 *   - Matrices are row-major.  A leading dimension (lda) counts elements.
 *   - Pointers named "device" must point to GPU memory (cudaMalloc, or a
 *     PyTorch CUDA tensor); the caller owns all of them.  The library owns
 *     only what it allocates inside a handle or a plan.
 *   - Element types follow the precision: TSK_FP64 -> double everywhere;
 *     TSK_FP32 -> float A, float S and float outputs; TSK_BF16 -> bfloat16 A
 *     (IEEE-754 binary32 truncated to its high 16 bits, round-to-nearest-even
 *     when produced), float S and float outputs.  Errors and norms are always
 *     double.
 *   - Every call is asynchronous on the given stream (a cudaStream_t; NULL is
 *     the legacy default stream) unless it says otherwise.  Argument errors
 *     are returned at once; errors found on the device (a wait that ran out,
 *     a rank-deficient sketch) are raised in a device status word that
 *     tsk_sync_status() reads after synchronising the stream.
 *   - No C++ exception crosses this boundary.  A handle must not be used by
 *     two host threads at the same time.
 *   - Requirements on sizes: 1 <= r <= k <= min(m, n) (thin QR of the n x k
 *     matrix (SA)^T needs k <= n; Theorem 1 needs k > r for its bound but
 *     r = k is accepted) and k <= TSK_MAX_K.  The tensor-core sketch of a
 *     BF16 matrix also needs k <= 48 and m <= 4096.  TMA moves rows that
 *     start on 16-byte boundaries: a matrix whose A is not 16-byte aligned
 *     or whose lda * 2 is not a multiple of 16 is copied, at every
 *     execution of its plan, to rows of ceil(n / 8) * 8 elements in the
 *     plan's workspace (2 m ceil(n / 8) * 8 bytes more workspace; one more
 *     read and write of A), and the tensor-core kernel reads the copy.
 *     With TSK_KERNEL_AUTO the BF16 matrices of a batch with k > 48 or
 *     m > 4096 go to the CUDA-core sketch kernels, in the same plan and
 *     concurrently with the rest; TSK_KERNEL_SIMT sends every matrix there
 *     and copies nothing.  The CUDA-core paths need only natural alignment.
 */
#ifndef TSK_H_
#define TSK_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TSK_MAX_K 64

typedef enum {
  TSK_OK = 0,
  TSK_EINVAL = 1,      /* an argument is out of range, null or misaligned   */
  TSK_ENOMEM = 2,      /* a device or host allocation failed                */
  TSK_ECUDA = 3,       /* a CUDA call failed; tsk_last_error() has the text */
  TSK_ENOCONV = 4,     /* the eigensolver hit its iteration cap             */
  TSK_ETIMEOUT = 5,    /* a bounded device wait ran out                     */
  TSK_ERANKDEF = 6,    /* warning: S A had rank < k for some matrix         */
  TSK_EUNSUPPORTED = 7 /* valid request this build/device cannot run        */
} tsk_status;

typedef enum { TSK_FP64 = 0, TSK_FP32 = 1, TSK_BF16 = 2 } tsk_prec;

/* Which kernels run the test-side sketch pass (X = A^T S^T and Y = A X). */
typedef enum {
  TSK_KERNEL_AUTO = 0, /* tensor cores for TSK_BF16 when k, m allow, else SIMT */
  TSK_KERNEL_SIMT = 1, /* CUDA-core kernels, two passes over A               */
  TSK_KERNEL_TC = 2    /* tcgen05/TMA kernel, one pass over A (TSK_BF16 only) */
} tsk_kernel;

typedef struct tsk_handle_s* tsk_handle;
typedef struct tsk_plan_s* tsk_plan;
typedef void* tsk_stream; /* cudaStream_t */

typedef struct {
  int32_t kernel;     /* tsk_kernel; default TSK_KERNEL_AUTO                  */
  int32_t refine_q;   /* one CholeskyQR2 / Householder refinement step on the
                         thin QR factor of the n x k panel X = (SA)^T:
                         0 never; 1 always; 2 (default) always on the FP64
                         path, and on the FP32 / BF16 paths only for matrices
                         where the first-order bound on the captured energy's
                         change from the FP32 rounding of X^T X,
                           u sum_{i<=r} lambda_i (sum_j ||x_j|| |W_ji|)^2,
                         u = 2^-24, W = R^{-1} V_r, exceeds 1e-3 of the
                         residual ||A||^2 - sum_{i<=r} lambda_i             */
  int32_t max_iter;   /* subspace-iteration cap of the eigensolver (300)      */
  int32_t err_mode;   /* how tsk_approx_batch gets ||A - B||_F:
                         0 (default): the projection identity
                           ||A||^2 - sum_{i<=r} sigma_i^2 (proof of Theorem 1,
                           Eq. A.3), followed by a direct pass over A for the
                           matrices where it cancels (err^2 < tau ||A||^2,
                           tau = 1e-6 for TSK_FP64, 1e-4 otherwise);
                         1: the identity only;
                         2: a direct pass over A for every matrix.          */
  double eig_tol;     /* eigensolver residual tolerance relative to lambda_1;
                         0 selects 1e-13 (FP64) or 2e-6 (FP32/BF16)           */
  int64_t spin_limit; /* iteration bound of every device spin-wait (1<<24)    */
  int32_t small_fp64; /* FP32 / BF16 paths only: 0 (default) takes the small
                         factors by the FP32 Gram route (Cholesky of X^T X,
                         one-sided Jacobi on the Cholesky factor of M^T M, M =
                         A Q; only the energy and the error in double); 1
                         takes them in double: blockwise Householder QR of the
                         X and Y panels (read from the FP32 panels, one
                         refinement pass) and one-sided Jacobi SVD of the k x k
                         R_Y R_X^{-1}, as on the TSK_FP64 path.  Slower (the
                         Householder steps are serial); it exists to run the
                         k x k steps in FP64 where a configuration asks.     */
  int32_t gram_tile;  /* tiles of the BF16 Grams (both modes) on the tensor
                         cores: 0 (default) 256 x 256 tiles, each on a pair
                         of CTAs whose tensor cores work as one (M = N = 256
                         MMAs); 1: 128 x 128 tiles on single CTAs          */
} tsk_options;

/* One test-side matrix.  A: device, m x n, leading dimension lda >= n.
   S: device, k x m row-major, leading dimension m (double for TSK_FP64,
   float otherwise).  r: target rank. */
typedef struct {
  const void* A;
  const void* S;
  int64_t m, n, lda;
  int32_t k, r;
} tsk_mat_desc;

/* Optional per-matrix outputs (each pointer may be NULL; all device).
   US    m x r   U_r Sigma_r = A Q V_r, row-major, leading dimension r
   Vt    r x n   (Q V_r)^T, row-major, leading dimension n; B = US * Vt
   sigma k       singular values of A Q, descending
   Output element type: double for TSK_FP64, float otherwise. */
typedef struct {
  void* US;
  void* Vt;
  void* sigma;
} tsk_mat_out;

/* ---- handles ----------------------------------------------------------- */

/* Creates a handle on the current CUDA device.  opts may be NULL for the
   defaults.  Returns TSK_ECUDA when no usable device is present. */
tsk_status tsk_create(tsk_handle* out, const tsk_options* opts);

/* Synchronises the device, frees every plan and workspace of the handle. */
tsk_status tsk_destroy(tsk_handle h);

/* Text of the last error on this handle (static storage; never NULL).
   With h == NULL, the last error of tsk_create on this thread. */
const char* tsk_last_error(tsk_handle h);

/* Fills *out with the defaults (the values noted in tsk_options).  Each
   environment variable TSK_KERNEL, TSK_REFINE_Q, TSK_MAX_ITER, TSK_ERR_MODE,
   TSK_EIG_TOL, TSK_SPIN_LIMIT, TSK_SMALL_FP64 and TSK_GRAM_TILE that is set
   to a value valid for its field (an integer in the field's range; a number
   in [0, 1] for TSK_EIG_TOL) replaces that default; others are ignored.  The
   environment is read at every call. */
void tsk_default_options(tsk_options* out);

/* Synchronises the stream, then returns and clears the device status word:
   TSK_OK, TSK_ETIMEOUT or TSK_ERANKDEF (the most severe one seen). */
tsk_status tsk_sync_status(tsk_handle h, tsk_stream stream);

/* ---- training side (Section 3.1, Algorithm 2 lines 1-2) ---------------- */

/* Mode-1 or mode-2 Gram matrix of the training tensor.
   A: host array of D device pointers, each an m x n matrix (lda >= n) of the
   precision's element type.  mode 1: G (device, m x m, double, row-major)
   receives sum_d A_d A_d^T (Eq. 3.2); mode 2: G (n x n) receives
   sum_d A_d^T A_d (the mode-2 unfolding of Eq. 3.6).  accumulate != 0 adds
   to G instead of overwriting it, so partial Gram matrices of disjoint
   training shards can be summed (the one exchange step of a multi-GPU
   training side).  Products are accumulated in the precision's compute type
   (double for TSK_FP64, float otherwise) and summed into G in double.
   TSK_BF16 with 16-byte aligned rows (lda * 2 a multiple of 16, 16-byte
   aligned A[d]) runs on the tensor cores and leaves G exactly symmetric:
   256 x 256 tiles on CTA pairs unless gram_tile = 1 (128 x 128 tiles on
   single CTAs); mode 2 reads A's columns as MN-major operands.  Products are
   summed in FP32 over eight matrices at a time, on the CTA pairs in chains
   of at most 128 MMAs (K = 16 each; whole matrices) whose FP32 results are
   added, rounded to nearest, over the eight; each eight then into G in
   double.  The tensor maps of the last training set are kept
   in the handle, so a repeated call on the same matrices skips encoding
   them. */
tsk_status tsk_gram(tsk_handle h, const void* const* A, int64_t D, int64_t m,
                    int64_t n, int64_t lda, tsk_prec prec, int32_t mode,
                    double* G, int32_t accumulate, tsk_stream stream);

/* FP8 training Gram (E4M3 with per-tile scaling).  tsk_quantize_e4m3 stores
   each training matrix A[d] (TSK_FP32 or TSK_BF16, m x n, lda >= n) as E4M3
   bytes in A8[d] (device, m x n, ld8 >= n bytes per row): with one
   power-of-two scale per row and per group of eight consecutive matrices,
   scales[(d / 8) * m + i] (device, ceil(D / 8) * m floats), the smallest
   power of two >= 2^-149 (FP32's smallest positive value) with
   max_{d in group, j} |A_d[i, j]| <= 448 scale (1 for a row of zeros), each
   byte is E4M3(A_d[i, j] / scale) of the exact quotient, rounded to nearest
   (ties to even).  E4M3 keeps 3
   mantissa bits: an element with |A| >= 2^-6 scale (the normal range) is
   stored within 2^-4 of itself, relatively; a smaller one within 2^-10 scale
   absolutely (subnormals, and zero below 2^-10 scale).  D <= 65535.
   tsk_gram_e4m3 then forms the mode-1 Gram of the stored values,
   G (device, m x m, double) = sum_d S_d A8_d A8_d^T S_d (S_d the diagonal of
   the group's scales), on the tensor cores (tcgen05 kind::f8f6f4, CTA pairs,
   FP32 accumulation over each group of eight, scaled and summed in double);
   ld8 must be a multiple of 16 and every A8[d] 16-byte aligned (the TMA rule),
   A8 is a host array of device pointers; accumulate != 0 adds to G.  Both
   block until done. */
tsk_status tsk_quantize_e4m3(tsk_handle h, const void* const* A, int64_t D, int64_t m,
                             int64_t n, int64_t lda, tsk_prec prec, void* const* A8,
                             int64_t ld8, float* scales, tsk_stream stream);
tsk_status tsk_gram_e4m3(tsk_handle h, const void* const* A8, const float* scales, int64_t D,
                         int64_t m, int64_t n, int64_t ld8, double* G, int32_t accumulate,
                         tsk_stream stream);

/* Leading k eigenvectors of the symmetric dim x dim G (device, double) as the
   rows of S (device, k x dim; double for TSK_FP64, float otherwise), in
   descending eigenvalue order, each row signed so that its entry of largest
   magnitude (lowest index on a tie) is positive.  eig (device, k doubles,
   nullable) receives the eigenvalues.  Subspace iteration with
   Rayleigh-Ritz; blocks the calling thread (it reads the residuals after
   every iteration).  Returns TSK_ENOCONV when max_iter is reached. */
tsk_status tsk_sketch_from_gram(tsk_handle h, const double* G, int64_t dim,
                                int32_t k, tsk_prec prec, void* S, double* eig,
                                tsk_stream stream);

/* Algorithm 2, lines 1-2: S (k x m) from the mode-1 Gram of the D training
   matrices A (host array of device pointers, m x n, lda >= n); with l > 0
   also W (l x n) from the mode-2 Gram.  eig (device, k + l doubles, nullable)
   receives the eigenvalues of both.  Blocks like tsk_sketch_from_gram. */
tsk_status tsk_train_sketch(tsk_handle h, const void* const* A, int64_t D,
                            int64_t m, int64_t n, int64_t lda, tsk_prec prec,
                            int32_t k, int32_t l, void* S, void* W,
                            double* eig, tsk_stream stream);

/* ---- test side (Algorithm 1 in QR form; Algorithm 2 line 3) ------------ */

/* SCW for a batch of count matrices (mats: host array).  err (device,
   count doubles, nullable) receives ||A_d - B_d||_F, computed from the
   projection identity ||A||^2 - ||[AQ]_r||^2 (proof of Theorem 1, Eq. A.3);
   normA2 (device, nullable) receives ||A_d||_F^2.  outs (host array of count
   entries, nullable) names the optional factor outputs.  The first call
   with a given argument set builds a plan (workspace, schedule, CUDA graph)
   and caches it in the handle; later calls with identical arguments replay
   it.  A and S are read when the work runs, not when the call returns. */
tsk_status tsk_approx_batch(tsk_handle h, int64_t count,
                            const tsk_mat_desc* mats, tsk_prec prec,
                            const tsk_mat_out* outs, double* err,
                            double* normA2, tsk_stream stream);

/* The same as an explicit plan: build once, execute many times.  The plan
   keeps pointers to the caller's buffers; they must stay valid. */
tsk_status tsk_plan_create(tsk_handle h, int64_t count,
                           const tsk_mat_desc* mats, tsk_prec prec,
                           const tsk_mat_out* outs, double* err,
                           double* normA2, tsk_plan* plan);
tsk_status tsk_plan_execute(tsk_plan plan, tsk_stream stream);
tsk_status tsk_plan_destroy(tsk_plan plan);

/* Timing probe for benchmarks.  The plan's graph is re-recorded with two
   event-record nodes around its sketch pass (the stage that streams every
   A_d from HBM: X = A^T S^T and Y = A X), so that cudaEventElapsedTime on the
   two caller-owned events (created with timing enabled) gives that stage's
   device time on every later execution.  Later calls only swap the events
   (no re-recording).  The events must stay alive while the plan can still
   execute with them; ev_begin = ev_end = NULL removes the probe (the graph is
   re-recorded without it).  Must not be called while the plan is executing. */
tsk_status tsk_plan_set_probe(tsk_plan plan, void* ev_begin, void* ev_end);

/* Bytes of device workspace a plan holds, and the number of kernel launches
   one execution makes (for reporting). */
tsk_status tsk_plan_info(tsk_plan plan, int64_t* workspace_bytes,
                         int32_t* launches_per_execute);

/* Autotuner of the tensor-core sketch pass (BF16).  For every size class of
   the batch where the kernel has more than one shape -- 256 < m <= 2304,
   where a matrix can be split over CTAs of 512 rows, of 256 rows (m <=
   2048) or of 384 rows (k <= 40; clusters of 1, 2, 3 or 6 CTAs, three
   stages of A in flight instead of two) -- it builds a plan of the class's
   matrices (up to 2048 of them: a shape's throughput depends on how many
   SMs the class fills) for each shape, times the sketch pass
   (CUDA events around it inside the plan's graph; best of reps executions
   after one warm-up) and keeps the faster shape in the handle.  A size
   class is (the cluster size at 512 rows per CTA, k rounded up to 8).  Plans
   built afterwards take the tuned shapes.  Runs the work on stream and
   synchronises it; the matrices are read, not changed. */
tsk_status tsk_autotune(tsk_handle h, int64_t count, const tsk_mat_desc* mats, tsk_prec prec,
                        int32_t reps, tsk_stream stream);
/* Writes the handle's tuned shapes to a JSON file (one object per size
   class with the times measured), or reads such a file back into the
   handle (replacing its table). */
tsk_status tsk_autotune_save(tsk_handle h, const char* path);
tsk_status tsk_autotune_load(tsk_handle h, const char* path);

/* Direct error ||A_d - US_d Vt_d||_F of factored approximations (problem
   1.1), one more pass over every A_d.  outs[i].US (m x r) and outs[i].Vt
   (r x n) must be non-NULL; err: device, count doubles. */
tsk_status tsk_error(tsk_handle h, int64_t count, const tsk_mat_desc* mats,
                     tsk_prec prec, const tsk_mat_out* outs, double* err,
                     tsk_stream stream);

/* ---- two-sided sketching (Section 3.2, Algorithms 3 and 5) ------------- */

/* One test-side matrix for two-sided SCW.  A: device, m x n (lda >= n).
   S: device, k x m row-major (leading dimension m); W: device, l x n
   row-major (leading dimension n); double for TSK_FP64, float otherwise.
   r: target rank. */
typedef struct {
  const void* A;
  const void* S;
  const void* W;
  int64_t m, n, lda;
  int32_t k, l, r, reserved;
} tsk_mat2_desc;

/* Algorithm 3 (two-sided SCW) for a batch: Q = qr((S A)^T) (n x k),
   P = qr(A W^T) (m x l), the l x k core P^T A Q, its rank-r truncation and
   B = P [P^T A Q]_r Q^T.  One pass over each A gives X = (S A)^T,
   Y = A X and Z = A W^T; the core is R_Z^{-T} (Z^T Y) R_X^{-1} with R_X, R_Z
   the R factors (blockwise Householder) of X and Z, its SVD is one-sided
   Jacobi in double, and err (device, count doubles, nullable) receives
   ||A - B||_F = sqrt(||A||^2 - sum_{i<=r} sigma_i(core)^2) (P and Q are
   orthonormal).  normA2 (device, nullable): ||A||_F^2.  outs (host array,
   nullable): US = P U_r Sigma_r (m x r), Vt = (Q V_r)^T (r x n), sigma
   (k values: the min(k, l) singular values of the core, then zeros).
   Needs 1 <= r <= min(k, l), k <= n, l <= m, k, l <= TSK_MAX_K.  Rank
   deficiency of S A or A W^T raises TSK_ERANKDEF in the status word.
   Blocks until the work is done (the descriptors are staged from the
   host). */
tsk_status tsk_approx_two_sided(tsk_handle h, int64_t count, const tsk_mat2_desc* mats,
                                tsk_prec prec, const tsk_mat_out* outs, double* err,
                                double* normA2, tsk_stream stream);

/* Training side of the two-sided sketch: the Tucker2 problem (Eq. 3.6) of
   the D training matrices A (host array of device pointers, m x n, lda >=
   n) by HOOI (Algorithm 5 with the mode-3 factor the identity), started
   from the HOSVD pair (leading eigenvectors of the mode-1 and mode-2 Gram
   matrices).  A sweep replaces S by the top k eigenvectors of
   sum_d (A_d W^T)(A_d W^T)^T and then W by the top l eigenvectors of
   sum_d (S A_d)^T (S A_d); it stops when the core energy
   sum_d ||S A_d W^T||_F^2 changed by less than tol * sum_d ||A_d||_F^2
   (tol <= 0 selects 1e-12 for TSK_FP64, 1e-7 otherwise) or after
   max_sweeps sweeps.  S (k x m) and W (l x n): device, double for TSK_FP64,
   float otherwise.  core_energy (host, nullable) receives the final core
   energy, sweeps (host, nullable) the number of sweeps made.  Blocks. */
tsk_status tsk_train_two_sided(tsk_handle h, const void* const* A, int64_t D, int64_t m,
                               int64_t n, int64_t lda, tsk_prec prec, int32_t k, int32_t l,
                               int32_t max_sweeps, double tol, void* S, void* W,
                               double* core_energy, int32_t* sweeps, tsk_stream stream);

/* ---- learned sketch refiner (IVY loss, Eq. 2.1) ------------------------ */

/* Batch IVY loss and its gradient with respect to the sketch.
   mats: host array of count matrices sharing m, n, k and r (their S fields
   are ignored); S: device, k x m (double for TSK_FP64, float for TSK_FP32;
   TSK_BF16 is not supported).  grad (device, k x m) receives
   dL/dS of L(S) = mean_A ||A - SCW(A, S, r)||_F^2 / ||A||_F^2, computed as
   -(2/||A||^2) W (A A^T Z - Z Sigma_r^2)^T averaged over the batch, with
   X = (SA)^T = QR, AQ = U Sigma V^T, Z = U_r Sigma_r, W = R^{-1} V_r (the
   derivation is the library's; the paper gives none).  loss (device double,
   nullable) receives L(S).  Needs sigma_r(AQ) > sigma_{r+1}(AQ).  Blocks
   until done. */
tsk_status tsk_ivy_grad(tsk_handle h, int64_t count, const tsk_mat_desc* mats,
                        tsk_prec prec, const void* S, void* grad, double* loss,
                        tsk_stream stream);

typedef struct {
  int32_t steps;          /* SGD steps (2000)                                 */
  int32_t batch;          /* matrices per step (16)                           */
  double lr;              /* learning rate (1e-3)                             */
  int32_t eval_every;     /* validation interval in steps (100)              */
  int32_t reserved;
  uint64_t seed;          /* seed of the batch order when order is NULL       */
  const int32_t* order;   /* host, steps*batch indices into the training set
                             (the random draws of SGD), or NULL               */
} tsk_refine_opts;

void tsk_default_refine_options(tsk_refine_opts* out);

/* Trains S_theta = S_tensor + dS by plain SGD on the IVY loss (Eq. 2.1, per-
   sample normalised) over the training matrices, validating on val every
   eval_every steps with the test-side SCW, and leaves in dS the value with
   the lowest validation loss seen -- the given dS (normally zero, i.e. the
   plain tensor sketch) included, so the result is never worse on val.
   train, val: host arrays of descriptors sharing m, n, k, r (S ignored);
   S_tensor (k x m) and dS (k x m, in/out): device, FP32 (FP64 for TSK_FP64).
   history (host, nullable): steps/eval_every + 1 validation losses, the
   first for the starting dS.  Blocks until done. */
tsk_status tsk_refine_sketch(tsk_handle h, const tsk_mat_desc* train,
                             int64_t ntrain, const tsk_mat_desc* val,
                             int64_t nval, tsk_prec prec,
                             const tsk_refine_opts* opts, const void* S_tensor,
                             void* dS, double* history, tsk_stream stream);

/* The same SGD run taken in pieces, so that it can stop and resume (with the
   checkpoint files below in between).  The run is the one opts describes:
   opts->steps steps in all, its batches drawn for all of them (from
   opts->order, or from opts->seed), so step t takes the same batch whether
   or not the run stopped before it.  This call takes steps state->step ..
   stop - 1 (0 <= state->step <= stop <= opts->steps).
   dS (device, k x m, in/out): the current SGD iterate, not the best one.
   state->best (device, k x m): the best validated dS so far; state->best_loss
   its validation loss.  With state->step == 0 the call first validates dS
   as given and sets both (the "never worse" reference).  After the call
   state->step is stop (or the step where an error stopped it).
   history (host, nullable): the whole run's steps/eval_every + 1 entries;
   the call writes only those of the validations it makes (entry t /
   eval_every after step t, entry 0 for the starting dS).
   tsk_refine_sketch is this call from step 0 to opts->steps followed by
   copying best into dS.  A resumed run equals the uninterrupted one up to
   the order of the FP64 atomic sums of ||A||^2 in the gradient (a relative
   difference near 1e-16 per step).  Blocks until done. */
typedef struct {
  int32_t step;      /* SGD steps taken so far                               */
  int32_t reserved;
  double best_loss;  /* validation loss of best                              */
  void* best;        /* device, k x m: the best validated dS so far          */
} tsk_refine_state;

tsk_status tsk_refine_sketch_steps(tsk_handle h, const tsk_mat_desc* train,
                                   int64_t ntrain, const tsk_mat_desc* val,
                                   int64_t nval, tsk_prec prec,
                                   const tsk_refine_opts* opts,
                                   const void* S_tensor, void* dS,
                                   tsk_refine_state* state, int32_t stop,
                                   double* history, tsk_stream stream);

/* ---- checkpoint files (no counterpart in the paper; host only) --------- */

/* Array file: the 8 bytes "TSKARR1\0", int32 precision (tsk_prec), int32 0,
   int64 rows, int64 cols, then rows x cols elements row-major; every number
   little-endian, whatever the host's byte order.  For S (k x m), W (l x n),
   a refiner's dS.  tsk_array_save writes host (rows x cols elements of the
   precision's type: double, float or BF16 bits) to path, through path.tmp
   renamed into place when complete.  tsk_array_load reads the header into
   *prec, *rows, *cols and, when host is non-NULL, the elements into host,
   which must hold capacity >= rows * cols * element size bytes.  Both return
   TSK_EINVAL (tsk_last_error(NULL) has the text) on bad arguments, a file
   that cannot be opened or written, a header not of this format, or a file
   shorter than its header says. */
tsk_status tsk_array_save(const char* path, const void* host, tsk_prec prec,
                          int64_t rows, int64_t cols);
tsk_status tsk_array_load(const char* path, void* host, int64_t capacity,
                          tsk_prec* prec, int64_t* rows, int64_t* cols);

/* Refiner checkpoint: "TSKREF1\0", int32 precision (TSK_FP64 or TSK_FP32),
   int32 state->step, int64 k, int64 m, double state->best_loss, double lr,
   uint64 seed, int32 steps, int32 batch, int32 eval_every, int32 1 if the
   run's batches came from an explicit order (else 0), then dS and best
   (k x m each, row-major), little-endian; written through path.tmp.
   dS_host, best_host: host copies of dS and state->best.  tsk_refine_load
   fills *prec, *k, *m, the run's options (opts->order NULL: a run with an
   explicit order, *order_given = 1, needs it passed again), state->step and
   state->best_loss (state->best is left as it is: the caller copies
   best_host to its device buffer), and, when dS_host and best_host are both
   non-NULL, the two arrays (capacity bytes each, at least k * m elements).
   Errors as for the array files. */
tsk_status tsk_refine_save(const char* path, tsk_prec prec, int64_t k, int64_t m,
                           const tsk_refine_opts* opts,
                           const tsk_refine_state* state, const void* dS_host,
                           const void* best_host);
tsk_status tsk_refine_load(const char* path, tsk_prec* prec, int64_t* k,
                           int64_t* m, tsk_refine_opts* opts,
                           int32_t* order_given, tsk_refine_state* state,
                           void* dS_host, void* best_host, int64_t capacity);

/* ---- allocation-free SCW (no counterpart in the paper) ------------------ */

/* Bytes of the static device array that tsk_approx_noalloc works in. */
#define TSK_NOALLOC_SCRATCH_BYTES (8u << 20)

/* SCW with errors (as tsk_approx_batch) for ONE matrix, for callers that must
   not allocate device memory at the point of the call: code that runs inside
   a memory pool owned by another framework, latency-critical paths where
   cudaMalloc (which may synchronise the device and has unbounded latency) is
   not allowed, and deployments that budget every byte of GPU memory in
   advance.  No handle is needed and nothing is allocated: every intermediate
   lives in a file-scope __device__ array of TSK_NOALLOC_SCRATCH_BYTES (8 MiB)
   that each GPU which loads the library holds until the process exits.
   Matrices needing more than that (2 (m + n) * k_pad * element size plus a
   few KB of descriptors, k_pad = k rounded up to 16, element size 8 for
   TSK_FP64 and 4 otherwise: the X and Y panels and the factors of the
   direct-error pass; for example m + n up to 21,800 at k = 48 in FP32) are
   rejected with TSK_EINVAL and a message in tsk_last_error(NULL).
   mat: host pointer to the descriptor (device A and S as for
   tsk_approx_batch; any of the three precisions, always the CUDA-core
   kernels).  err: device, one double; normA2: device, one double, nullable.
   status: device, one int32, nullable; when given it receives, once the
   work has run, the device status of this call: 0, or TSK_ERANKDEF when S A
   had rank < k (the error is then that of Householder's completion of the
   basis), or TSK_ETIMEOUT.  Errors follow the default err_mode of
   tsk_approx_batch: the projection identity, then a direct pass over A
   when the identity cancels (err^2 < tau ||A||^2, tau = 1e-6 for TSK_FP64,
   1e-4 otherwise).
   The first call on each device looks up the array's device address with
   cudaGetSymbolAddress while that device is current, so make that first call
   before any stream capture; later calls outside a capture look it up again
   (cheap once the module is loaded), so the address stays valid after the
   device's context has been reset and the module reloaded.  All calls share the one array and it keeps the
   previous call's contents (the call clears what it accumulates into): calls
   that overlap on the GPU -- on two streams, or from two host threads --
   race and corrupt each other's results.  Asynchronous on stream; other
   errors as in the rest of this header (tsk_last_error(NULL) has the text). */
tsk_status tsk_approx_noalloc(const tsk_mat_desc* mat, tsk_prec prec,
                              double* err, double* normA2, int32_t* status,
                              tsk_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* TSK_H_ */
