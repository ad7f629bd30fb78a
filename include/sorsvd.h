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
                                          hi+lo pair of 16-bit operands */

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
 * caller.  Device-side status: sorsvd_get_status is not available for this
 * entry point (the workspace is internal); check the outputs. */
int sorsvd_run_noalloc(const void* A, int64_t m, int64_t n, int64_t lda,
                       int k, int p, int q, uint64_t seed, int dtype, unsigned flags,
                       void* U, int64_t ldu, void* S, void* V, int64_t ldv, void* stream);

/* Copies the device status word of a workspace to the host (synchronous on
 * `stream`).  *device_status receives a sorsvd_status code (SORSVD_OK when
 * the last call finished cleanly); *info receives diagnostic bits
 * (bit 0: a Cholesky needed a shifted retry; bits 8..15: Jacobi sweeps of
 * the last call).  Either pointer may be NULL. */
int sorsvd_get_status(const void* workspace, int* device_status, int* info, void* stream);

/* Human-readable name of a status code (static string). */
const char* sorsvd_status_string(int status);

/* Gaussian test matrix Omega (Sec. III, "standard Gaussian matrix"):
 * out[i + j*ld] for i < rows, j < cols is the N(0,1) value of linear element
 * e = i + rows*j drawn from Philox4x64-10 with key (seed, 0) and counter
 * (e / 4, stream_id, 0, 0), Box-Muller on word pairs, rounded to `dtype`
 * (binary64 -> fp32 RNE -> 16-bit RNE).  Bit-identical to the CPU oracle. */
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

/* ---- launch accounting (host side, no device work) -----------------------
 * Kernel classes: 0 Gaussian, 1 pass over A in the power loop (T1 = A T2 or
 * T2 = A^T T1), 2 pass over A in the core product (A Q2), 3 small
 * tall-skinny products (Gram, T R^{-1}, Q1^T W, output assembly),
 * 4 split-K reductions, 5 Cholesky/inverse, 6 Jacobi SVD, 7 conversions
 * and copies. */
#define SORSVD_NUM_KCLASS 8

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
