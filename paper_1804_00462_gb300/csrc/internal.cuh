// Internal declarations shared by the translation units of libsorsvd.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>
#include <stddef.h>

#include "../../include/sorsvd.h"

namespace sorsvd {

// ---------------------------------------------------------------------------
// device status word (lives at the start of every workspace)
// ---------------------------------------------------------------------------
struct DeviceStatus {
  int code;        // first non-OK sorsvd_status raised on the device
  int info;        // bit 0: shifted Cholesky retry; bits 8..15: Jacobi sweeps
  int pad[14];      // pad[0]: CholeskyQR3's second pass found Q orthonormal (the third is skipped);
                   // pad[1]: the second pass took the polar factor (its Cholesky kernel returned)
};

__device__ __forceinline__ void raise_status(DeviceStatus* st, int code) {
  atomicCAS(&st->code, 0, code);
}

// ---------------------------------------------------------------------------
// element types
// ---------------------------------------------------------------------------
typedef __nv_bfloat16 bf16;
typedef __half f16;

template <typename T> __device__ __forceinline__ float to_f32(T x);
template <> __device__ __forceinline__ float to_f32<float>(float x) { return x; }
template <> __device__ __forceinline__ float to_f32<bf16>(bf16 x) { return __bfloat162float(x); }
template <> __device__ __forceinline__ float to_f32<f16>(f16 x) { return __half2float(x); }

template <typename Acc, typename T> __device__ __forceinline__ Acc to_acc(T x) { return (Acc)to_f32<T>(x); }
template <> __device__ __forceinline__ double to_acc<double, double>(double x) { return x; }
template <> __device__ __forceinline__ float to_acc<float, double>(double x) { return (float)x; }

template <typename T> __device__ __forceinline__ T from_f64(double x);
template <> __device__ __forceinline__ double from_f64<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_f64<float>(double x) { return __double2float_rn(x); }
// two-step rounding binary64 -> fp32 -> 16-bit, both round-to-nearest-even
template <> __device__ __forceinline__ bf16 from_f64<bf16>(double x) { return __float2bfloat16_rn(__double2float_rn(x)); }
template <> __device__ __forceinline__ f16 from_f64<f16>(double x) { return __float2half_rn(__double2float_rn(x)); }

template <typename T> __device__ __forceinline__ T from_f32(float x);
template <> __device__ __forceinline__ float from_f32<float>(float x) { return x; }
template <> __device__ __forceinline__ double from_f32<double>(float x) { return (double)x; }
template <> __device__ __forceinline__ bf16 from_f32<bf16>(float x) { return __float2bfloat16_rn(x); }
template <> __device__ __forceinline__ f16 from_f32<f16>(float x) { return __float2half_rn(x); }

inline size_t dtype_size(int dt) {
  switch (dt) {
    case SORSVD_F64: return 8;
    case SORSVD_F32: case SORSVD_TF32: return 4;
    case SORSVD_BF16: case SORSVD_F16: return 2;
    default: return 0;
  }
}
inline bool dtype_is_16(int dt) { return dt == SORSVD_BF16 || dt == SORSVD_F16; }
inline size_t acc_size(int dt) { return dt == SORSVD_F64 ? 8 : 4; }

// ---------------------------------------------------------------------------
// host-side launchers (defined next to their kernels)
// ---------------------------------------------------------------------------
int num_sms();

// gaussian.cu
cudaError_t launch_gaussian(void* out, int64_t rows, int64_t cols, int64_t ld, uint64_t seed,
                            uint64_t stream_id, int dtype, cudaStream_t st);

// gemm_simt.cu
// C (M x N) = op(A) * B with A column-major.  trans_a = false: A is M x K;
// trans_a = true: A is K x M (used as A^T).  B is K x N column-major.  When
// `splits` > 1 the K range is cut in `splits` chunks and chunk s writes the
// partial product to C + s * split_stride; reduce_splits combines them.
// a_dt / b_dt: element types (sorsvd_dtype); c is fp32 for acc_f64 = false,
// binary64 otherwise.
// (skip: a device flag that, when an earlier kernel set it, makes the
// launch do nothing; for the products of a skipped CholeskyQR pass)
cudaError_t launch_gemm(bool trans_a, int64_t M, int64_t N, int64_t K,
                        const void* A, int64_t lda, int a_dt,
                        const void* B, int64_t ldb, int b_dt,
                        void* C, int64_t ldc, bool acc_f64,
                        int splits, int64_t split_stride, cudaStream_t st, const int* skip = nullptr);
// out = sum_s parts[s] (fixed order, binary64 sums); parts are fp32 or f64.
cudaError_t launch_reduce_splits(const void* parts, bool parts_f64, int splits, int64_t split_stride,
                                 int64_t rows, int64_t cols, int64_t ld_part,
                                 void* out, bool out_f64, int64_t ld_out, cudaStream_t st,
                                 const int* skip = nullptr);
// y (16-bit) = round(x) elementwise; x fp32 (rows x cols, ldx) -> y (ldy).
// When `lo` is non-null it also receives round(x - float(y)) (hi/lo split).
cudaError_t launch_convert_f32(const float* x, int64_t ldx, int64_t rows, int64_t cols,
                               void* y, int64_t ldy, int y_dt, void* lo, cudaStream_t st);
// At (cols x rows, ldt) = A^T of a column-major fp32 matrix
cudaError_t launch_transpose_f32(const float* A, int64_t lda, int64_t rows, int64_t cols, float* At, int64_t ldt,
                                 cudaStream_t st);
// y += x (binary64 / fp32, rows x cols, leading dimensions)
cudaError_t launch_add_f64(const double* x, int64_t ldx, double* y, int64_t ldy, int64_t rows, int64_t cols,
                           cudaStream_t st);
cudaError_t launch_add_f32(const float* x, int64_t ldx, float* y, int64_t ldy, int64_t rows, int64_t cols,
                           cudaStream_t st);
// copy with leading dimensions (same element size)
cudaError_t launch_copy2d(const void* x, int64_t ldx, void* y, int64_t ldy,
                          int64_t rows, int64_t cols, size_t elem, cudaStream_t st, const int* skip = nullptr);

// ---------------------------------------------------------------------------
// grouped ("batched") launches: one launch runs one stage of many problems,
// reading per-problem job descriptors from device memory
// ---------------------------------------------------------------------------
// C = op(A) B for job j, all operands of the accumulator type; K chunks of
// k_chunk, chunk s written to C + s * split_stride.
struct GemmJob {
  const void* A; const void* B; void* C;
  int64_t lda, ldb, ldc;
  int64_t M, N, K;
  int64_t k_chunk, split_stride;
};
// out = sum_{s < splits} parts[s * stride] (binary64 sums)
struct ReduceJob {
  const void* parts; void* out;
  int64_t rows, cols, ldp, ldo, stride;
  int splits, out_f64;
};
// Omega of one problem
struct GaussJob {
  void* out; int64_t rows, cols, ld; uint64_t seed;
};
// Cholesky inverse of one problem (chol.cu)
struct CholJob {
  const double* G; void* Rinv; DeviceStatus* status; int l; double shift;
};
// l x l SVD of one problem (jacobi.cu)
struct JacobiJob {
  const double* M; void* Ut; void* Vt; void* S; void* work; DeviceStatus* status; int l, k;
};
// units: int4 (job, m-tile, n-tile, k-split) in tiles of gemm_tile_shape()
// grouped tile shapes: 0 128 x 64, 1 64 x 64, 2 64 x 32 (kBatchedTiles)
constexpr int kBatchedTiles = 3;
cudaError_t launch_gemm_batched(bool trans_a, bool f64, int tile, const GemmJob* jobs, const int4* units, int nunits,
                                cudaStream_t st);
void gemm_tile_shape(int tile, int* bm, int* bn, int* bk);
cudaError_t launch_reduce_batched(bool parts_f64, const ReduceJob* jobs, int njobs, int64_t max_elems,
                                  cudaStream_t st);
cudaError_t launch_gaussian_batched(const GaussJob* jobs, int njobs, int64_t max_elems, int dtype,
                                    cudaStream_t st);
// largest l the one-block blocked Cholesky takes (shared-memory tiles)
int chol_batched_max_l(bool f64);
cudaError_t launch_chol_batched(const CholJob* jobs, int njobs, int max_l, bool f64, cudaStream_t st);
// largest l of the batched Jacobi (W in shared memory)
int jacobi_batched_max_l(bool f64);
size_t jacobi_batched_work_bytes(int l);
cudaError_t launch_jacobi_batched(const JacobiJob* jobs, int njobs, int max_l, bool f64, cudaStream_t st);

// chol.cu: R^{-1} (upper triangular, l x l, column-major, ld = l) of the
// Cholesky factor of G + s I, s = shift_rel * trace(G) / l.  G binary64.
// Output in binary64 (f64 = true) or fp32.
// Optional (blocked kernel only): skip_in non-null and *skip_in != 0 ->
// R^{-1} = I without factorising; conv_out non-null -> *conv_out = 1 when
// every off-diagonal entry of the equilibrated G is <= conv_tol (the columns
// are orthonormal to that level) and no shifted retry was needed, else 0.
cudaError_t launch_chol_inv(const double* G, int l, double shift_rel, void* Rinv, bool f64,
                            DeviceStatus* status, cudaStream_t st, const int* skip_in = nullptr,
                            int* conv_out = nullptr, float conv_tol = 0.f, const int* done_in = nullptr);

// polar.cu: X = D^{-1/2} (I + E)^{-1/2} (binomial series to E^3) for a Gram
// G close to I (I + E = D^{-1/2} G D^{-1/2}, D = diag G) into Rinv (fp32,
// l x l, ld l), so that X^T G X = I.  *ok = 1 when ||E||_F <= 0.02 (the
// series then reaches fp32 accuracy), else 0 (Rinv is not usable; the
// Cholesky kernel given done_in = ok then factorises).  *conv (optional) =
// *ok and max |E_ij| <= conv_tol.  scratch: polar_scratch_bytes(l), device.
size_t polar_scratch_bytes(int l);
cudaError_t launch_polar_inv(const double* G, int l, float* Rinv, float* scratch, int* ok, int* conv,
                             float conv_tol, cudaStream_t st);

// jacobi.cu: SVD of the l x l matrix M (binary64 input): one-sided Jacobi
// sweeps in binary64 (f64) or fp32, binary64 finish.  Writes sigma
// (descending) to S (k entries, S_f64 selects its type), U~ and V~ (l x l,
// ld = l, sweep precision) with the sign convention of the oracle.  Work
// buffer: jacobi_work_bytes(l).
cudaError_t launch_jacobi(const double* M, int l, int k, bool f64, void* Ut, void* Vt,
                          void* S, bool S_f64, void* work, DeviceStatus* status, cudaStream_t st);
size_t jacobi_work_bytes(int l);
// Sweep cap of the Jacobi kernels launched next on the current device
// (<= 0 or above the built-in cap of 30: 30).
cudaError_t set_jacobi_sweep_cap(int cap);
// Limit (SM cycles) of the tensor-core passes' waits for pipeline progress
// in the launches that follow (<= 0: the built-in ~2 s).
void set_tc_wait_cycles(long long cycles);

// rowblock.cu: fp32 row-block products (l <= SORSVD_MAX_L columns).
// launch_rb_gram: rb_gram_blocks(rows, lx, ly, sym) partials (lx x ly, ld lx,
// stride lx*ly) of X^T Y over the rows (sym: Y = X, both halves written);
// returns at once when *skip is set.  launch_rb_apply: Y = X B (X rows x K,
// B K x N, ld ldb; tri: B upper triangular), out of place, with an optional
// 16-bit rounding (kind16 1 bf16, 2 fp16); X 16-byte aligned, ldx % 4 == 0.
// launch_rb_copy: dst = src (rows x l, ld) plus the 16-bit rounding; with
// *skip set only the rounding of dst.
int64_t rb_gram_blocks(int64_t rows, int lx, int ly, bool sym);
size_t rb_gram_parts_bytes(int64_t rows, int lx, int ly, bool sym);
cudaError_t launch_rb_gram(const float* X, int64_t ldx, const float* Y, int64_t ldy, int64_t rows, int lx, int ly,
                           bool sym, float* parts, const int* skip, cudaStream_t st);
cudaError_t launch_rb_apply(const float* X, int64_t ldx, int64_t rows, int K, const float* B, int64_t ldb, int N,
                            bool tri, float* Y, int64_t ldy, void* Y16, int64_t ld16, int kind16, const int* skip,
                            cudaStream_t st);
cudaError_t launch_rb_copy(const float* src, float* dst, int64_t ld, int64_t rows, int l, void* Y16, int64_t ld16,
                           int kind16, const int* skip, cudaStream_t st);
// out (binary64, rows x cols, ldo) = fixed-order sum of nparts fp32
// partials (ld ldp, stride between partials), kRedLanes threads per
// element.  sym_split >= 0 (symmetric rows x rows result): the partials hold
// the lower triangle, except that entries (i, j) with i >= sym_split > j
// sit at (j, i); both halves of out are written.
cudaError_t launch_reduce_parts(const float* parts, int nparts, int64_t stride, int rows, int cols, int ldp,
                                double* out, int ldo, cudaStream_t st, int sym_split = -1);

// tsk_tc.cu: the tall-skinny fp32 products on the tensor cores (split TF32,
// fp32 accuracy), l <= kTskMaxL columns.  launch_tsk_gram: tsk_gram_parts()
// partials (l x l, ld l, stride l*l) of X^T X over the rows, to be summed by
// launch_reduce_parts(..., sym_split) with the split it returns.
// launch_tsk_apply: Y = X B (X rows x K, 16-byte aligned, ldx % 4 == 0;
// B K x N given as hi / lo parts by launch_split_tf32, ldb % 4 == 0; tri: B
// upper triangular), out of place, with an optional 16-bit rounding.  Both
// return at once when *skip is set, and are unavailable (false from the
// *_supported checks) with SORSVD_TSK=0.
constexpr int kTskMaxL = 288;
constexpr int kTskMaxN = 320;
bool tsk_enabled();
bool tsk_gram_supported(const float* X, int64_t ldx, int l);
int tsk_gram_parts(int64_t rows);
cudaError_t launch_tsk_gram(const float* X, int64_t ldx, int64_t rows, int l, float* parts, int* nparts,
                            int* sym_split, const int* skip, DeviceStatus* status, cudaStream_t st);
// launch_tsk_xty: tsk_xty_parts() partials (l x l, ld l, stride l*l) of
// X^T Y over the rows (plain reduction)
bool tsk_xty_supported(const float* X, int64_t ldx, const float* Y, int64_t ldy, int l);
int tsk_xty_parts(int64_t rows, int l);
cudaError_t launch_tsk_xty(const float* X, int64_t ldx, const float* Y, int64_t ldy, int64_t rows, int l,
                           float* parts, int* nparts, const int* skip, DeviceStatus* status, cudaStream_t st);
bool tsk_apply_supported(const float* X, int64_t ldx, int K, int N);
cudaError_t launch_tsk_apply(const float* X, int64_t ldx, int64_t rows, int K, const float* Bhi, const float* Blo,
                             int64_t ldb, int N, bool tri, float* Y, int64_t ldy, void* Y16, int64_t ld16,
                             int kind16, const int* skip, DeviceStatus* status, cudaStream_t st);

// twopass.cu: C (l x l) = op(A) op(B) in binary64 (op: transpose when the
// flag is set); exact widening of a column-major matrix: 16-bit (BF16/F16)
// to fp32, or fp32 to binary64 (y_f64).
cudaError_t launch_small_gemm64(const double* A, bool ta, const double* B, bool tb, double* C, int l,
                                cudaStream_t st);
cudaError_t launch_widen(const void* x, int in_dtype, int64_t ldx, int64_t rows, int64_t cols, void* y, bool y_f64,
                         int64_t ldy, cudaStream_t st);

// sorsvd.cu: the device status word of a sorsvd_run workspace
DeviceStatus* workspace_status(void* ws);

// gemm_tc.cu: tensor-core pass over A (tcgen05 + TMA), op(A) = A^T when
// trans_a.  elt: 0 bf16, 1 fp16, 2 tf32 (fp32 containers), 3 fp32-accurate
// split products (fp32 containers, trans_a only).  B is K x N column-major
// of the same element type; for elt 3, B and Blo are the hi / lo parts of
// the operand written by launch_split_tf32 (Blo unused otherwise).  Writes
// fp32 C (ldo) and, when out16 is non-null, its 16-bit rounding (out16_kind
// 1 bf16, 2 fp16).  Needs tc_supported() and tc_parts_bytes() of scratch in
// `parts`.
bool tc_supported(int elt, const void* A, int64_t lda, const void* B, int64_t ldb, int l);
size_t tc_parts_bytes(int elt, int64_t M, int64_t N, int64_t K);
cudaError_t launch_tc_gemm(bool trans_a, int elt, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                           const void* B, int64_t ldb, const void* Blo, float* out, int64_t ldo, void* out16,
                           int64_t ld16, int out16_kind, float* parts, int* tilecnt, int64_t ntilecnt,
                           DeviceStatus* status, int kcls, cudaStream_t st);
// hi = RN_tf32(X), lo = X - hi (exact in fp32) of a rows x cols fp32 matrix
// (column-major, ldx); hi and lo share the leading dimension ldh.
cudaError_t launch_split_tf32(const float* X, int64_t ldx, int64_t rows, int64_t cols, float* hi, float* lo,
                              int64_t ldh, cudaStream_t st);

}  // namespace sorsvd
