// The two-pass core of SOR-SVD (Sec. III, second core option of
// Algorithm 3): M_approx = Q1^T T1 (Q2^T T2_prev)^+, where T2_prev is the
// operand of the last product T1 = A T2_prev (the "non-updated" T2).  The
// core pass over A is replaced by two tall-skinny Grams and l x l work.
//
// With B = Q2^T T2_prev (l x l, full rank) the pseudo-inverse is
// B^+ = B^T (B B^T)^{-1}; the Cholesky-inverse kernel gives R^{-1} with
// R^{-T} (B B^T) R^{-1} = I, so (B B^T)^{-1} = R^{-1} R^{-T} and
//   M_approx = C B^T R^{-1} R^{-T},  C = Q1^T T1.
// The three l x l products run in binary64 (small_gemm64_kernel).
#include "internal.cuh"

#include <algorithm>

namespace sorsvd {
namespace {

// C (l x l, ld l) = op(A) op(B), binary64, op = transpose when the flag is
// set; one thread per output element, K = l in index order.
__global__ void small_gemm64_kernel(const double* __restrict__ A, bool ta, const double* __restrict__ B, bool tb,
                                    double* __restrict__ C, int l) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= l * l) return;
  const int i = e % l, j = e / l;
  double s = 0.0;
  for (int k = 0; k < l; ++k) {
    const double a = ta ? A[k + (size_t)i * l] : A[i + (size_t)k * l];
    const double b = tb ? B[j + (size_t)k * l] : B[k + (size_t)j * l];
    s = fma(a, b, s);
  }
  C[e] = s;
}

// y (binary64 or fp32, rows x cols, ldy) = x (16-bit or fp32, ldx), exact
template <typename In, typename Out>
__global__ void widen_kernel(const In* __restrict__ x, int64_t ldx, int64_t rows, int64_t cols, Out* __restrict__ y,
                             int64_t ldy) {
  const int64_t total = rows * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / rows, r = e - c * rows;
    y[r + c * ldy] = (Out)(float)x[r + c * ldx];
  }
}

template <typename In, typename Out>
cudaError_t widen(const In* x, int64_t ldx, int64_t rows, int64_t cols, Out* y, int64_t ldy, cudaStream_t st) {
  const int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 8);
  widen_kernel<In, Out><<<(unsigned)blocks, 256, 0, st>>>(x, ldx, rows, cols, y, ldy);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_small_gemm64(const double* A, bool ta, const double* B, bool tb, double* C, int l,
                                cudaStream_t st) {
  if (l <= 0) return cudaSuccess;
  const int threads = 128;
  small_gemm64_kernel<<<(l * l + threads - 1) / threads, threads, 0, st>>>(A, ta, B, tb, C, l);
  return cudaGetLastError();
}

cudaError_t launch_widen(const void* x, int in_dtype, int64_t ldx, int64_t rows, int64_t cols, void* y, bool y_f64,
                         int64_t ldy, cudaStream_t st) {
  if (y_f64) {
    if (in_dtype == SORSVD_F32 || in_dtype == SORSVD_TF32)
      return widen((const float*)x, ldx, rows, cols, (double*)y, ldy, st);
    return cudaErrorInvalidValue;
  }
  if (in_dtype == SORSVD_BF16) return widen((const bf16*)x, ldx, rows, cols, (float*)y, ldy, st);
  if (in_dtype == SORSVD_F16) return widen((const f16*)x, ldx, rows, cols, (float*)y, ldy, st);
  return cudaErrorInvalidValue;
}

}  // namespace sorsvd
