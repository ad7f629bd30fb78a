/*
 * sorsvd.h -- C ABI of the GB300 (sm_103a) SOR-SVD library.
 *
 * SOR-SVD (subspace-orbit randomized SVD) computes a rank-k approximation
 * A ~= U diag(S) V^T of a dense m x n matrix (Sec. III, Algorithm 3):
 *   T2 <- Omega (n x l Gaussian, l = k + p);
 *   repeat q+1 times: T1 <- A T2 ; T2 <- A^T T1;
 *   T1 = Q1 R1, T2 = Q2 R2 (QR);  M <- Q1^T A Q2 (l x l);
 *   M_k = U~_k S~_k V~_k^T (truncated SVD);  U = Q1 U~_k, S = S~_k, V = Q2 V~_k.
 *
 * Conventions shared by every entry point
 *   - Matrices are column-major (element (i, j) at base[i + j*ld]), ld >= rows.
 *   - Every data pointer is caller-owned DEVICE memory unless stated.  The
 *     library never allocates device memory on these paths: scratch space is
 *     the caller's workspace (sorsvd_workspace_size).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream; argument errors are
 *     returned synchronously, numerical trouble found on the device is
 *     recorded in a status word inside the workspace (sorsvd_get_status).
 *   - Return values are sorsvd_status codes.  Nothing traps or aborts.
 *   - Not thread-safe per workspace: two calls that overlap on the GPU must
 *     use different workspaces.
 */
#ifndef SORSVD_H
#define SORSVD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Storage / arithmetic type of the passes over A.
 *   F64  : A binary64; every stage in binary64 (CUDA cores).
 *   F32  : A binary32; the power passes that only steer the subspace run as
 *          TF32 tensor-core products, the last power pass and the core
 *          product as fp32-accurate split TF32 products (hi*hi + hi*lo +
 *          lo*hi); fp32 accumulation, Gram partials combined in binary64.
 *   TF32 : A binary32; every pass a TF32 tensor-core product.
 *   BF16 : A bfloat16; passes on tensor cores, fp32 accumulation.
 *   F16  : A binary16; as BF16.
 * Outputs U, S, V are binary64 for F64 and binary32 otherwise. */
typedef enum {
  SORSVD_F64 = 0, SORSVD_F32 = 1, SORSVD_TF32 = 2, SORSVD_BF16 = 3, SORSVD_F16 = 4
} sorsvd_dtype;

typedef enum {
  SORSVD_OK = 0,
  SORSVD_ERR_ARG = 1,            /* bad size, leading dimension, pointer or flag */
  SORSVD_ERR_DTYPE = 2,          /* unknown dtype */
  SORSVD_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  SORSVD_ERR_NOT_CONVERGED = 4,  /* (device) Jacobi SVD hit its sweep cap */
  SORSVD_ERR_BREAKDOWN = 5,      /* (device) Cholesky failed after shifted retries */
  SORSVD_ERR_TIMEOUT = 6,        /* (device) a bounded wait gave up */
  SORSVD_ERR_WORKSPACE = 7,      /* workspace NULL, misaligned or too small */
  SORSVD_ERR_UNSUPPORTED = 8     /* size beyond a documented limit */
} sorsvd_status;

/* Flags */
#define SORSVD_FLAG_LITERAL_POWER 0x1u /* power loop exactly as printed in
                                          Algorithm 3 (no re-orthonormalisation
                                          of T2 between passes) */
#define SORSVD_FLAG_REFINE        0x2u /* BF16/F16: Q2 enters the core pass as a
                                          hi+lo pair of 16-bit operands (two
                                          tensor-core passes over A, combined
                                          in binary64) */
#define SORSVD_FLAG_HOST_IO       0x4u /* sorsvd_workspace_size: size for
                                          sorsvd_run_host (adds the device
                                          copies of A, U, S and V); accepted
                                          and ignored by sorsvd_run_host */
#define SORSVD_FLAG_TWO_PASS      0x8u /* the two-pass core of Sec. III
                                          (second core option of Algorithm 3):
                                          M_approx = Q1^T T1 (Q2^T T2_prev)^+
                                          with T2_prev the operand of the last
                                          product T1 = A T2_prev; no core pass
                                          over A (2q + 2 passes instead of
                                          2q + 3).  REFINE is then ignored.
                                          Needs the same flag in
                                          sorsvd_workspace_size. */
#define SORSVD_FLAG_FIXED_TILES   0x10u /* batched plans: no autotuning, every
                                          grouped product on the 128 x 64
                                          tile shape */
#define SORSVD_FLAG_RSVD          0x20u /* sorsvd_run / sorsvd_run_host: the
                                          randomized SVD (R-SVD, Algorithm 1,
                                          Sec. II) on the same kernels:
                                          Y = (A A^T)^q A Omega, Y = Q R,
                                          B = Q^T A (the last A^T pass),
                                          rank-k truncation of B's SVD; B's SVD
                                          is that of M = (A^T Q)^T Q2 with Q2
                                          the QR factor of A^T Q (no core pass:
                                          2q + 2 passes over A).  Not with
                                          LITERAL_POWER, TWO_PASS or TSR. */
#define SORSVD_FLAG_TSR           0x40u /* sorsvd_run / sorsvd_run_host: the
                                          two-sided randomized SVD (TSR-SVD,
                                          Algorithm 2, Sec. II): Psi1 = Omega,
                                          Psi2 (m x l) the same Philox
                                          generator's stream 1, Y1 = A Psi1,
                                          Y2 = A^T Psi2, QR of both,
                                          B_approx = Q1^T Y1 (Q2^T Psi1)^+,
                                          rank-k truncation of its SVD.  Needs
                                          q = 0; not with LITERAL_POWER,
                                          TWO_PASS or RSVD.  Needs the same
                                          flag in sorsvd_workspace_size (as
                                          RSVD and TWO_PASS). */

/* Largest sketch width l = k + p supported (the small l x l factorisations
 * run in one thread block with the factor in shared memory). */
#define SORSVD_MAX_L      320
#define SORSVD_MAX_L_F64  224

/* Bytes of workspace sorsvd_run needs for this problem (0 on bad arguments).
 * The workspace must be 256-byte aligned device memory. */
size_t sorsvd_workspace_size(int64_t m, int64_t n, int k, int p, int dtype, unsigned flags);

/* Rank-k SOR-SVD of A (Algorithm 3; q = 0 is the basic algorithm of Sec. III).
 *   A      m x n, column-major, leading dimension lda >= m, type `dtype`.
 *   k, p   target rank and oversampling, l = k + p, 1 <= k, 0 <= p,
 *          l <= min(m, n), l <= SORSVD_MAX_L (SORSVD_MAX_L_F64 for F64).
 *   q      number of power passes (>= 0); A is read 2q + 3 times.
 *   seed   key of the Gaussian test matrix Omega (Philox4x64-10, stream 0;
 *          same values as sorsvd_gaussian).
 *   U      m x k (ldu >= m), S length k (descending), V n x k (ldv >= n):
 *          binary64 for F64, binary32 otherwise.
 * Returns SORSVD_OK when the work was queued; read the device status with
 * sorsvd_get_status after synchronising the stream. */
int sorsvd_run(const void* A, int64_t m, int64_t n, int64_t lda,
               int k, int p, int q, uint64_t seed, int dtype, unsigned flags,
               void* U, int64_t ldu, void* S, void* V, int64_t ldv,
               void* workspace, size_t ws_bytes, void* stream);

/* sorsvd_run with A, U, S and V in HOST memory.  The paper has no
 * counterpart: the entry point serves callers whose matrix lives on the host
 * (the end-to-end cost of the method then includes the copy of A).
 *   A, lda, U, ldu, S, V, ldv: as in sorsvd_run, but host pointers.  For the
 *          copies to run asynchronously and overlap the solve they must be
 *          page-locked (cudaHostAlloc / cudaHostRegister); pageable memory
 *          works, with copies that the CUDA runtime stages synchronously.
 *   workspace: device memory of at least
 *          sorsvd_workspace_size(m, n, k, p, dtype, flags | SORSVD_FLAG_HOST_IO)
 *          bytes, 256-byte aligned; it also holds the device copies of A,
 *          U, S and V.
 * A crosses in column blocks of about 64 MiB on a copy stream of the
 * library; Omega is drawn meanwhile, and for F32 / TF32 each block's part of
 * the transposed copy of A is made as soon as the block has landed.  The
 * solve and the copies of U, S, V back to the host are queued on `stream`
 * after every block (results identical to sorsvd_run on the same data).
 * Returns SORSVD_OK when the work was queued; the host outputs are valid
 * once `stream` has been synchronised; errors as sorsvd_run. */
int sorsvd_run_host(const void* A, int64_t m, int64_t n, int64_t lda,
                    int k, int p, int q, uint64_t seed, int dtype, unsigned flags,
                    void* U, int64_t ldu, void* S, void* V, int64_t ldv,
                    void* workspace, size_t ws_bytes, void* stream);

/* Maximum scratch of sorsvd_run_noalloc: 32 MiB of device memory, held by
 * every GPU that loads the library for the life of the process. */
#define SORSVD_NOALLOC_MAX_BYTES 33554432u

/* sorsvd_run without a caller workspace.  The paper has no counterpart: it
 * is an interface convenience for callers that cannot allocate device
 * memory when they call - for example code inside a host application that
 * owns all device memory through its own fixed pool, or latency-critical
 * loops that cannot afford cudaMalloc's possible device synchronisation.
 * The caller still provides A, U, S and V (same meaning, layout and errors
 * as sorsvd_run).  Scratch comes from one library-owned device array of
 * SORSVD_NOALLOC_MAX_BYTES: problems whose sorsvd_workspace_size exceeds it
 * return SORSVD_ERR_UNSUPPORTED.  The first call on each device looks the
 * array up (cudaGetSymbolAddress) with that device current; make it before
 * any stream capture.  Nothing is allocated or freed.  Every call shares the
 * array and leaves its contents behind: calls that may overlap on the GPU
 * (different streams or host threads) race and must be serialised by the
 * caller.  The cached address belongs to the primary context: do not call
 * it after a cudaDeviceReset or from another context.  Device-side status
 * (the workspace is internal): sorsvd_noalloc_get_status. */
int sorsvd_run_noalloc(const void* A, int64_t m, int64_t n, int64_t lda,
                       int k, int p, int q, uint64_t seed, int dtype, unsigned flags,
                       void* U, int64_t ldu, void* S, void* V, int64_t ldv, void* stream);

/* Device status word of the last sorsvd_run_noalloc call on the current
 * device, as sorsvd_get_status gives it for a caller workspace (synchronous
 * on `stream`; same meaning of *device_status and *info; either pointer may
 * be NULL).  The paper has no counterpart.  Returns SORSVD_ERR_CUDA when the
 * scratch array cannot be looked up. */
int sorsvd_noalloc_get_status(int* device_status, int* info, void* stream);

/* Copies the device status word of a workspace to the host (synchronous on
 * `stream`).  *device_status receives a sorsvd_status code (SORSVD_OK when
 * the last call finished cleanly); *info receives diagnostic bits
 * (bit 0: a Cholesky needed a shifted retry; bits 8..15: Jacobi sweeps of
 * the last call).  Either pointer may be NULL. */
int sorsvd_get_status(const void* workspace, int* device_status, int* info, void* stream);

/* Limits of the device-side failure paths, for tests of those paths (the
 * paper has no counterpart).  wait_cycles: how long (SM clock cycles) a
 * tensor-core pass waits for its pipeline to make progress before it
 * records SORSVD_ERR_TIMEOUT, stops, lets its copies and MMAs in flight
 * land, frees its tensor memory and returns; <= 0 restores the built-in
 * 4e9 cycles (about 2 s), larger values are clamped to it.  max_sweeps:
 * Jacobi sweeps before SORSVD_ERR_NOT_CONVERGED (1..30); <= 0 restores 30.
 * Applies to calls made afterwards by any thread of the process; the sweep
 * cap is set on the current device (synchronous copy: not during stream
 * capture).  Results of a call that hit either limit are not meaningful;
 * later calls with the defaults restored are unaffected.  Returns SORSVD_OK
 * or SORSVD_ERR_CUDA. */
int sorsvd_set_limits(long long wait_cycles, int max_sweeps);

/* Human-readable name of a status code (static string). */
const char* sorsvd_status_string(int status);

/* Gaussian test matrix Omega (Sec. III, "standard Gaussian matrix"):
 * out[i + j*ld] for i < rows, j < cols is the N(0,1) value of linear element
 * e = i + rows*j drawn from Philox4x64-10 with key (seed, 0) and counter
 * (e / 4, stream_id, 0, 0), Box-Muller on word pairs with the transform
 * in binary32 (series in correctly rounded operations); the binary32 value
 * is stored as is (F64: exactly; F32 / TF32) or rounded to the 16-bit type
 * (RNE).  Bit-identical to the CPU oracle. */
int sorsvd_gaussian(void* out, int64_t rows, int64_t cols, int64_t ld,
                    uint64_t seed, uint64_t stream_id, int dtype, void* stream);

/* One power pass of Algorithm 3 (the two products of its loop body):
 *   T1 = A X (m x l),  T2 = A^T T1 (n x l).
 * X is n x l (ldx >= n); X, T1, T2 are binary64 for F64 and binary32
 * otherwise; for BF16/F16 X and T1 are rounded to the 16-bit type before
 * they multiply A, exactly as inside sorsvd_run; F32 uses the fp32-accurate
 * products of the last power pass, TF32 plain TF32 products.  Uses the same
 * workspace as sorsvd_run for the same (m, n, k, p, dtype) with l = k + p. */
int sorsvd_power_pass(const void* A, int64_t m, int64_t n, int64_t lda, int dtype,
                      const void* X, int64_t ldx, int l,
                      void* T1, int64_t ldt1, void* T2, int64_t ldt2,
                      void* workspace, size_t ws_bytes, void* stream);

/* Core product of Algorithm 3 (eq. M):  M = Q1^T A Q2, l x l binary64
 * (ldm >= l).  Q1 is m x l, Q2 n x l, binary64 for F64 and binary32
 * otherwise.  `flags` may carry SORSVD_FLAG_REFINE. */
int sorsvd_core(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, unsigned flags,
                const void* Q1, int64_t ldq1, const void* Q2, int64_t ldq2, int l,
                double* M, int64_t ldm, void* workspace, size_t ws_bytes, void* stream);

/* R^{-1} of one CholeskyQR step (the QR of the sketches, Sec. III): with
 * D = diag(G) and G' = D^{-1/2} G D^{-1/2} + s I (s = shift_rel, relative to
 * the unit diagonal of G'), G' = L L^T and R^{-1} = D^{-1/2} L^{-T}, so that
 * T R^{-1} has orthonormal columns up to the conditioning of T when
 * G = T^T T.  A pivot that is not safely positive restarts with a 16x larger
 * shift (status info bit 0), at most 12 times, then SORSVD_ERR_BREAKDOWN
 * (R^{-1} = I).  G: l x l binary64, column-major, ld = l.  Rinv: l x l
 * upper triangular, ld = l, binary64 for dtype F64 and fp32 otherwise.
 * status: device memory of at least 64 bytes receiving the device status
 * word (read it with sorsvd_get_status; the call clears it first).
 * 1 <= l <= SORSVD_MAX_L (SORSVD_MAX_L_F64 for F64). */
int sorsvd_chol_inv(const double* G, int l, double shift_rel, int dtype, void* Rinv, void* status, void* stream);

/* Polar factor used by the second CholeskyQR3 pass of sorsvd_run (fp32
 * dtypes; Sec. III QR step): for a Gram G close to I, with D = diag(G) and
 * I + E = D^{-1/2} G D^{-1/2}, X = D^{-1/2} (I + E)^{-1/2} by the binomial
 * series to E^3, so that X^T G X = I and T X is an orthonormal basis of
 * range(T) when G = T^T T.  *ok (device int) = 1 when ||E||_F <= 0.02 (the
 * series then meets fp32 accuracy), else 0 and X must not be used (the
 * solve then factorises with Cholesky).
 * G: l x l binary64, column-major, ld = l.  X: l x l fp32, ld = l (full,
 * symmetric up to the left scaling).  scratch: device memory of at least
 * 8 l^2 + 8 (l + 31) / 32 * l + 4 l bytes.  1 <= l <= SORSVD_MAX_L. */
int sorsvd_polar_inv(const double* G, int l, float* X, int* ok, void* scratch, size_t scratch_bytes,
                     void* stream);

/* Out-of-core SOR-SVD (Algorithm 3 with the stabilised power loop, as
 * sorsvd_run without flags) for an A that stays in HOST memory, e.g. one
 * larger than the device's memory: the paper counts the method's cost in
 * passes over A (Sec. III, 2q + 3 passes), and every pass here streams A
 * to the device in blocks of block_rows rows, copying block b + 1 while the
 * tensor cores work on block b (two device block buffers).  T1 = A X and
 * W = A Q2 are formed block by block; T2 = A^T Q1 as the sum of the blocks'
 * products (so its rounding differs from sorsvd_run's).  A: column-major
 * m x n host array (lda >= m) of the dtype's element type; page-locked
 * memory (cudaHostAlloc / cudaHostRegister) lets the copies run
 * asynchronously, pageable memory works at lower speed.  U, S, V are device
 * outputs as in sorsvd_run; the workspace (device) holds the sketches, the
 * two blocks and the solve's scratch: sorsvd_streamed_workspace_size bytes,
 * 256-byte aligned.  A must stay valid and unchanged until the stream has
 * finished the call. */
size_t sorsvd_streamed_workspace_size(int64_t m, int64_t n, int k, int p, int dtype, int64_t block_rows);
int sorsvd_run_streamed(const void* A, int64_t m, int64_t n, int64_t lda, int k, int p, int q, uint64_t seed,
                        int dtype, int64_t block_rows, void* U, int64_t ldu, void* S, void* V, int64_t ldv,
                        void* workspace, size_t ws_bytes, void* stream);

/* Tall-skinny fp32 products of the QR step (CholeskyQR of a sketch T:
 * G = T^T T, then Q = T R^{-1}; Sec. III) and of the output assembly
 * (U = Q1 U~_k, V = Q2 V~_k; Algorithm 3), computed as sorsvd_run computes
 * them for the binary32 and 16-bit dtypes: for l <= 288 (Gram) or
 * K <= 288, N <= 320 (product) on the tensor cores, each operand split into
 * a TF32 hi and an fp32 lo part and each product formed as
 * hi*hi + hi*lo + lo*hi (fp32 accuracy; SORSVD_TSK=0 in the environment
 * selects the CUDA-core kernels instead), else on CUDA cores.
 *   sorsvd_gram:  G = X^T Y (Y = X when Y is NULL), l x l binary64
 *                 (ldg >= l), for X, Y rows x l (the CholeskyQR Gram, and
 *                 the core's Q1^T W); the per-CTA fp32 partials are summed
 *                 in binary64 in a fixed order (bitwise repeatable).
 *   sorsvd_apply: Y = X B, rows x N fp32 (ldy >= rows), for X rows x K and
 *                 B K x N (ldb >= K); upper_tri != 0 declares B upper
 *                 triangular (its entries below the diagonal must be zero).
 * X (and Y): fp32, 16-byte aligned, leading dimension >= rows and a
 * multiple of 4.  l, K, N in
 * [1, SORSVD_MAX_L].  workspace: at least
 * sorsvd_products_workspace_size(rows, l) bytes (l = max(K, N) for
 * sorsvd_apply), 256-byte aligned; it starts with the device status word
 * (sorsvd_get_status), where a bounded wait that gave up records
 * SORSVD_ERR_TIMEOUT. */
size_t sorsvd_products_workspace_size(int64_t rows, int l);
int sorsvd_gram(const float* X, int64_t ldx, const float* Y, int64_t ldy, int64_t rows, int l,
                double* G, int64_t ldg, void* workspace, size_t ws_bytes, void* stream);
int sorsvd_apply(const float* X, int64_t rows, int K, int64_t ldx, const float* B, int64_t ldb, int N,
                 int upper_tri, float* Y, int64_t ldy, void* workspace, size_t ws_bytes, void* stream);

/* Bounds of Sec. IV on the rank-k SOR-SVD approximation A_hat (l = k + p,
 * q power iterations) for a matrix with singular values sigma[0..r-1]
 * (descending, r >= k + 1; the tail beyond r is taken as zero), as an
 * a-posteriori quality check.  Host function: no GPU, no stream.
 *   ey_2, ey_fro:        the optimum (Theorem 1): sigma_{k+1} and
 *                        sqrt(sum_{j>k} sigma_j^2).
 *   thm7_upper_2 / _fro: Theorem 7, upper bound on E ||A - A_hat|| (2- and
 *                        F-norm) over the Gaussian test matrix.
 *   thm6_lower[j]:       Theorem 6, lower bound on E sigma_j(A_hat),
 *                        j = 1..k (k doubles; may be NULL).
 *   thm5_upper_2 / _fro: Theorem 5, deterministic upper bound on
 *                        ||A - A_hat|| for a given test matrix Omega, from
 *                        omega2_norm = ||V2^T Omega||_2 and
 *                        omega1_pinv_norm = ||(V1^T Omega)^+||_2 (V1 the
 *                        first k right singular vectors of A, V2 the rest);
 *                        NaN when either is negative (unknown).
 *   thm4_lower[j]:       Theorem 4, the deterministic lower bound for the
 *                        same Omega (k doubles; may be NULL; NaN when the
 *                        norms are unknown).  Its proof bounds
 *                        sigma_j(A Q2 Q2^T); Theorem 5's tau for q > 0 is
 *                        read as (sigma_k / sigma_{k+1}) beta.
 * The singular values an SOR-SVD returns are lower bounds on A's (Sec. IV),
 * so bounds evaluated on them are estimates, not guarantees.
 * SORSVD_ERR_ARG for a null pointer, k < 1, p < 0, q < 0, r < k + 1,
 * n < k + p, a negative or increasing sigma, or sigma_k = 0. */
typedef struct {
  double ey_2, ey_fro;
  double thm5_upper_2, thm5_upper_fro;
  double thm7_upper_2, thm7_upper_fro;
} sorsvd_bounds_out;
int sorsvd_bounds(const double* sigma, int r, int64_t n, int k, int p, int q,
                  double omega2_norm, double omega1_pinv_norm, sorsvd_bounds_out* out,
                  double* thm4_lower, double* thm6_lower);

/* ---- batched SOR-SVD -------------------------------------------------------
 * Many independent problems of uneven shape (m, n, k, p, q may all differ)
 * in one sequence of grouped launches: each launch runs one stage of
 * Algorithm 3 for every problem, from per-problem job descriptors that a
 * plan uploads into the workspace once; the plan can capture the launches
 * in a CUDA graph.  The paper has no batched form: this is the same
 * algorithm per problem (same Omega, same results up to rounding order as
 * sorsvd_run with the same arguments, except that every product runs on
 * CUDA cores in the accumulator precision and the passes over A are not
 * split into TF32 parts).  dtype: SORSVD_F64, SORSVD_F32 or SORSVD_TF32 (A
 * binary64 or fp32; U, S, V in the same type).  flags: 0 or
 * SORSVD_FLAG_LITERAL_POWER.  l = k + p <= min(m, n) and l <= 128 (F64) /
 * 160 (fp32), else SORSVD_ERR_UNSUPPORTED. */
typedef struct {
  const void* A; int64_t m, n, lda;   /* device, column-major */
  int k, p, q;
  uint64_t seed;                      /* Omega of this problem (stream 0) */
  void* U; int64_t ldu;               /* device outputs, as sorsvd_run */
  void* S;
  void* V; int64_t ldv;
} sorsvd_problem;

typedef struct sorsvd_batch_plan sorsvd_batch_plan;

/* Workspace bytes for a batch (host array of descriptors); 0 on bad
 * arguments.  256-byte aligned device memory. */
size_t sorsvd_batched_workspace_size(const sorsvd_problem* probs, int batch, int dtype, unsigned flags);

/* Builds a plan: checks every descriptor, lays out the workspace, uploads
 * the job descriptors (synchronous on `stream`) and, when use_graph != 0,
 * captures the launches in a CUDA graph (on a private stream).  The plan
 * keeps pointers to the problems' A, U, S, V and to the workspace: they
 * must stay valid while the plan is used.  *plan is NULL on error. */
int sorsvd_batched_plan_create(sorsvd_batch_plan** plan, const sorsvd_problem* probs, int batch, int dtype,
                               unsigned flags, int use_graph, void* workspace, size_t ws_bytes, void* stream);
/* Runs the batch on `stream` (graph replay or direct launches); async. */
int sorsvd_batched_plan_launch(sorsvd_batch_plan* plan, void* stream);
/* Device status of every problem of the last run (synchronous): codes has
 * `batch` entries. */
int sorsvd_batched_plan_status(const sorsvd_batch_plan* plan, int* codes, void* stream);
/* Kernel launches per run (for accounting). */
int sorsvd_batched_plan_launches(const sorsvd_batch_plan* plan);
/* The tile shape the plan's autotuner picked for each grouped product
 * stage, in stage order (0: 128 x 64, 1: 64 x 64, 2: 64 x 32 outputs per
 * block).  sorsvd_batched_plan_create times every shape of every stage on
 * the plan's own jobs (CUDA events, cached per stage shape for the process;
 * SORSVD_FLAG_FIXED_TILES keeps shape 0); the results do not depend on the
 * choice.  Writes up to max_tiles entries and returns the
 * number of product stages.  The paper has no counterpart (its method is
 * single-problem). */
int sorsvd_batched_plan_tiles(const sorsvd_batch_plan* plan, int* tiles, int max_tiles);
void sorsvd_batched_plan_destroy(sorsvd_batch_plan* plan);
/* One-shot: plan (no graph), launch, destroy.  Asynchronous except for the
 * descriptor upload. */
int sorsvd_run_batched(const sorsvd_problem* probs, int batch, int dtype, unsigned flags, void* workspace,
                       size_t ws_bytes, void* stream);

/* ---- robust PCA (Sec. V-C, Table 3) ---------------------------------------
 * Inexact augmented-Lagrange-multiplier RPCA with SOR-SVD as the low-rank
 * step ("ALM-SOR-SVD"): splits X = L + S, L of rank <= k and S sparse.  Per
 * iteration j (mu_j the penalty, lambda = 1 / sqrt(max(m, n))):
 *   (U, Z, V) = sorsvd_run(X - S_j + Y_j / mu_j; k, p, q, seed + j - 1)
 *   L = U shrink_{1/mu_j}(Z) V^T ;  S = shrink_{lambda/mu_j}(X - L + Y_j / mu_j)
 *   Y += mu_j (X - L - S) ;  mu_{j+1} = min(rho mu_j, 1e7 mu_0)
 * with shrink_e(x) = sgn(x) max(|x| - e, 0), stopping after the first
 * iteration with ||X - L - S||_F < tol ||X||_F, or after max_iter.  Start:
 * S = 0, Y = X / max(||X||_2, ||X||_inf / lambda), mu_0 = 1.25 / ||X||_2
 * (the paper defers these choices to the inexact-ALM literature; the table
 * prints the mu cap as a maximum, read here as the usual minimum). */
typedef struct {
  const float* X;  int64_t m, n, ldx;  /* input, m x n fp32, m, n >= 2 */
  float* L;        int64_t ldl;        /* output low-rank part, m x n */
  float* S;        int64_t lds;        /* output sparse part, m x n */
  double norm2;    /* ||X||_2 if > 0; otherwise estimated on the device by a
                      rank-1 SOR-SVD of X (p = 9, q = 2) */
  uint64_t seed;   /* Gaussian seed of the first inner SOR-SVD */
} sorsvd_rpca_problem;

/* Flag of sorsvd_rpca: run the inner SOR-SVD in `dtype` while the residual
 * is large and in binary64 once ||X - L - S||_F / ||X||_F < 30 tol.  An
 * fp32 SOR-SVD leaves about 1e-7 relative error in L, where the iteration
 * stalls (the ALM residual cannot fall below the error of the low-rank
 * step); the binary64 finish costs a few iterations. */
#define SORSVD_RPCA_FINISH_F64 0x100u

/* Workspace bytes for sorsvd_rpca on `batch` problems (host array); 0 on
 * bad arguments.  256-byte aligned device memory. */
size_t sorsvd_rpca_workspace_size(const sorsvd_rpca_problem* probs, int batch, int k, int p, int dtype,
                                  unsigned flags);

/* Runs RPCA on `batch` independent problems (host array of descriptors whose
 * X, L, S point to device memory).  dtype: the type of the inner SOR-SVD,
 * SORSVD_F32, SORSVD_TF32 or SORSVD_F64 (its input G = X - S + Y / mu is
 * then kept in that precision); the RPCA state S, Y is fp32 either way and
 * the elementwise updates use double-fp32 arithmetic.  flags: 0 or
 * SORSVD_RPCA_FINISH_F64.  k, p, q as in sorsvd_run (l = k + p <= min(m, n)).
 * tol > 0, max_iter >= 1, rho >= 1.  SYNCHRONOUS: the host drives the loop
 * and reads one residual per problem per iteration; returns when every
 * problem has stopped.  Host outputs: iters[b] iterations run, xi[b] the
 * last ||X - L - S||_F / ||X||_F, xi_history (optional, batch x max_iter,
 * row b = problem b) every iteration's value.  Returns SORSVD_OK, an
 * argument error, or the first device status an inner SOR-SVD raised. */
int sorsvd_rpca(const sorsvd_rpca_problem* probs, int batch, int k, int p, int q, int dtype, unsigned flags,
                double tol, int max_iter, double rho, int* iters, double* xi, double* xi_history,
                void* workspace, size_t ws_bytes, void* stream);

/* ---- launch accounting (host side, no device work) -----------------------
 * Kernel classes: 0 Gaussian, 1 pass over A in the power loop (T1 = A T2 or
 * T2 = A^T T1), 2 pass over A in the core product (A Q2), 3 small
 * tall-skinny products (Gram, T R^{-1}, Q1^T W, output assembly),
 * 4 split-K reductions and tile fix-ups, 5 Cholesky/inverse, 6 Jacobi SVD,
 * 7 conversions, copies and the transposed copy of A, 8 fp32-accurate
 * (split) power passes, 9 RPCA elementwise kernels. */
#define SORSVD_NUM_KCLASS 10

/* Number of kernel launches the library has issued in this process. */
uint64_t sorsvd_launch_count(void);

/* Start recording a CUDA event pair on the launching stream around every
 * kernel launch whose class bit is set in class_mask (bit c = class c),
 * discarding earlier records. */
int sorsvd_profile_begin(unsigned class_mask);

/* Stop recording; synchronise on the recorded events and return, per kernel
 * class c < nclass, the summed event time ms[c] (milliseconds) and the
 * number of launches launches[c].  Either array may be NULL. */
int sorsvd_profile_end(double* ms, int* launches, int nclass);

#ifdef __cplusplus
}
#endif

#endif /* SORSVD_H */
