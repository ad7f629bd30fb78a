// CUDA-core GEMMs for the tall-skinny products of SOR-SVD, and the small
// elementwise helpers around them.
//
// The products of Algorithm 3 all have one long dimension (m or n, the rows
// of A) and one short one (l = k + p):
//   T1 = A T2, W = A Q2, Q = T R^{-1}, U = Q1 U~_k        (op(A) = A)
//   T2 = A^T T1, G = T^T T, M = Q1^T W                    (op(A) = A^T)
// The kernel below covers both with a 128 x 64 output tile, 16-deep K
// slices staged in shared memory and 8 x 4 register blocking per thread.
// Binary64 products with at most 32 columns use a 64 x 32 tile (4 x 2 per
// thread): GB300 runs binary64 FMAs at 1/64 of the fp32 rate, so padding a
// narrow product to 64 columns wastes most of a scarce unit.  K may be
// split across blockIdx.z; partial tiles are combined by reduce_splits in a
// fixed order (no atomics, deterministic results).
#include "internal.cuh"

#include <algorithm>

namespace sorsvd {

int num_sms() {
  static int cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (cache[dev] == 0) {
    int v = 0;
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    cache[dev] = v > 0 ? v : 1;
  }
  return cache[dev];
}

namespace {

template <int BM_, int BN_, int BK_, int TM_, int TN_>
struct TileCfg {
  static constexpr int BM = BM_, BN = BN_, BK = BK_, TM = TM_, TN = TN_;
  static constexpr int NT = (BM / TM) * (BN / TN);
};
using BigTile = TileCfg<128, 64, 16, 8, 4>;      // 256 threads
using MidTile = TileCfg<64, 64, 16, 4, 4>;       // 256 threads
using SkinnyTile = TileCfg<64, 32, 16, 4, 2>;    // 256 threads
constexpr int NT = 256;
static_assert(BigTile::NT == NT && MidTile::NT == NT && SkinnyTile::NT == NT,
              "tile configurations use 256 threads");

template <typename Acc, typename T> __device__ __forceinline__ Acc ld_as(const T* p) { return to_acc<Acc, T>(*p); }

// One BM x BN tile of C = op(A) B over the K range [kbeg, kend).
template <class Cfg, typename TA, typename TB, typename Acc, bool TRANS>
__device__ __forceinline__ void gemm_tile(int64_t M, int64_t N, const TA* __restrict__ A, int64_t lda,
                                          const TB* __restrict__ B, int64_t ldb, Acc* __restrict__ C,
                                          int64_t ldc, int64_t row0, int64_t col0, int64_t kbeg, int64_t kend) {
  constexpr int BM = Cfg::BM, BN = Cfg::BN, BK = Cfg::BK, TM = Cfg::TM, TN = Cfg::TN;
  __shared__ Acc As[BK][BM];
  __shared__ Acc Bs[BK][BN];
  const int t = threadIdx.x;
  const int tx = t % (BN / TN), ty = t / (BN / TN);

  Acc acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = Acc(0);

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / NT; ++r) {
      int idx = t + r * NT;
      int i, kk;
      if (TRANS) { kk = idx % BK; i = idx / BK; } else { i = idx % BM; kk = idx / BM; }
      int64_t gi = row0 + i, gk = k0 + kk;
      Acc v = Acc(0);
      if (gi < M && gk < kend) v = TRANS ? ld_as<Acc>(A + gk + gi * lda) : ld_as<Acc>(A + gi + gk * lda);
      As[kk][i] = v;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / NT; ++r) {
      int idx = t + r * NT;
      int kk = idx % BK, j = idx / BK;
      int64_t gj = col0 + j, gk = k0 + kk;
      Acc v = Acc(0);
      if (gj < N && gk < kend) v = ld_as<Acc>(B + gk + gj * ldb);
      Bs[kk][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      Acc a[TM], b[TN];
#pragma unroll
      for (int q = 0; q < TM; ++q) a[q] = As[kk][ty * TM + q];
#pragma unroll
      for (int q = 0; q < TN; ++q) b[q] = Bs[kk][tx * TN + q];
#pragma unroll
      for (int x = 0; x < TM; ++x)
#pragma unroll
        for (int y = 0; y < TN; ++y) acc[x][y] = fma(a[x], b[y], acc[x][y]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int y = 0; y < TN; ++y) {
    int64_t gj = col0 + tx * TN + y;
    if (gj >= N) continue;
#pragma unroll
    for (int x = 0; x < TM; ++x) {
      int64_t gi = row0 + ty * TM + x;
      if (gi < M) C[gi + gj * ldc] = acc[x][y];
    }
  }
}

template <class Cfg, typename TA, typename TB, typename Acc, bool TRANS>
__global__ void __launch_bounds__(NT)
gemm_kernel(int64_t M, int64_t N, int64_t K, const TA* __restrict__ A, int64_t lda,
            const TB* __restrict__ B, int64_t ldb, Acc* __restrict__ C, int64_t ldc,
            int64_t k_chunk, int64_t split_stride, const int* __restrict__ skip) {
  if (skip && *skip) return;                       // a device-side decision skipped this product
  const int64_t kbeg = (int64_t)blockIdx.z * k_chunk;
  gemm_tile<Cfg, TA, TB, Acc, TRANS>(M, N, A, lda, B, ldb, C + (int64_t)blockIdx.z * split_stride, ldc,
                                     (int64_t)blockIdx.x * Cfg::BM, (int64_t)blockIdx.y * Cfg::BN, kbeg,
                                     min(K, kbeg + k_chunk));
}

// Grouped form: block b computes unit units[b] = (job, m-tile, n-tile,
// k-split) of jobs[job]; one launch covers a stage of every problem.
template <class Cfg, typename Acc, bool TRANS>
__global__ void __launch_bounds__(NT)
gemm_batched_kernel(const GemmJob* __restrict__ jobs, const int4* __restrict__ units) {
  const int4 u = units[blockIdx.x];
  const GemmJob& j = jobs[u.x];
  const int64_t kbeg = (int64_t)u.w * j.k_chunk;
  gemm_tile<Cfg, Acc, Acc, Acc, TRANS>(j.M, j.N, (const Acc*)j.A, j.lda, (const Acc*)j.B, j.ldb,
                                       (Acc*)j.C + (int64_t)u.w * j.split_stride, j.ldc, (int64_t)u.y * Cfg::BM,
                                       (int64_t)u.z * Cfg::BN, kbeg, min(j.K, kbeg + j.k_chunk));
}

template <class Cfg, typename TA, typename TB, typename Acc>
cudaError_t gemm_dispatch_cfg(bool trans, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                              const void* B, int64_t ldb, void* C, int64_t ldc, int splits,
                              int64_t split_stride, cudaStream_t st, const int* skip) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  if (splits < 1) splits = 1;
  int64_t k_chunk = (K + splits - 1) / splits;
  k_chunk = ((k_chunk + Cfg::BK - 1) / Cfg::BK) * Cfg::BK;
  if (k_chunk < Cfg::BK) k_chunk = Cfg::BK;
  dim3 grid((unsigned)((M + Cfg::BM - 1) / Cfg::BM), (unsigned)((N + Cfg::BN - 1) / Cfg::BN), (unsigned)splits);
  if (trans)
    gemm_kernel<Cfg, TA, TB, Acc, true><<<grid, NT, 0, st>>>(M, N, K, (const TA*)A, lda, (const TB*)B, ldb,
                                                             (Acc*)C, ldc, k_chunk, split_stride, skip);
  else
    gemm_kernel<Cfg, TA, TB, Acc, false><<<grid, NT, 0, st>>>(M, N, K, (const TA*)A, lda, (const TB*)B, ldb,
                                                              (Acc*)C, ldc, k_chunk, split_stride, skip);
  return cudaGetLastError();
}

template <typename TA, typename TB, typename Acc>
cudaError_t gemm_dispatch(bool trans, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                          const void* B, int64_t ldb, void* C, int64_t ldc, int splits,
                          int64_t split_stride, cudaStream_t st, const int* skip = nullptr) {
  if (sizeof(Acc) == 8 && N <= SkinnyTile::BN)
    return gemm_dispatch_cfg<SkinnyTile, TA, TB, Acc>(trans, M, N, K, A, lda, B, ldb, C, ldc, splits, split_stride,
                                                      st, skip);
  return gemm_dispatch_cfg<BigTile, TA, TB, Acc>(trans, M, N, K, A, lda, B, ldb, C, ldc, splits, split_stride, st,
                                                 skip);
}

// Fixed-order sum of split partials.  fp32 partials are summed with
// Neumaier's compensated summation in fp32 (error about 2 eps of the sum of
// magnitudes, independent of the split count) and the pair is combined in
// binary64 once: binary64 adds run at a small fraction of the fp32 rate on
// this GPU.  Binary64 partials are summed in binary64.
__device__ __forceinline__ double sum_parts(const float* __restrict__ p, int splits, int64_t stride) {
  float s = 0.f, c = 0.f;
  for (int q = 0; q < splits; ++q) {
    const float x = p[q * stride];
    const float t = __fadd_rn(s, x);
    c = __fadd_rn(c, fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s));
    s = t;
  }
  return (double)s + (double)c;
}
__device__ __forceinline__ double sum_parts(const double* __restrict__ p, int splits, int64_t stride) {
  double s = 0.0;
  for (int q = 0; q < splits; ++q) s += p[q * stride];
  return s;
}

template <typename TP, typename TO>
__global__ void reduce_kernel(const TP* __restrict__ parts, int splits, int64_t stride, int64_t rows,
                              int64_t cols, int64_t ldp, TO* __restrict__ out, int64_t ldo,
                              const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = e / rows, i = e - j * rows;
    out[i + j * ldo] = (TO)sum_parts(parts + i + j * ldp, splits, stride);
  }
}

// Grouped reduce: blockIdx.y = job; parts fp32 or binary64 (Acc), out binary64
// or the accumulator type.
template <typename TP>
__global__ void reduce_batched_kernel(const ReduceJob* __restrict__ jobs) {
  const ReduceJob& j = jobs[blockIdx.y];
  const int64_t total = j.rows * j.cols;
  const TP* parts = (const TP*)j.parts;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = e / j.rows, i = e - c * j.rows;
    const double s = sum_parts(parts + i + c * j.ldp, j.splits, j.stride);
    if (j.out_f64) ((double*)j.out)[i + c * j.ldo] = s;
    else ((TP*)j.out)[i + c * j.ldo] = (TP)s;
  }
}

template <typename TY>
__global__ void convert_kernel(const float* __restrict__ x, int64_t ldx, int64_t rows, int64_t cols,
                               TY* __restrict__ y, int64_t ldy, TY* __restrict__ lo) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = e / rows, i = e - j * rows;
    float v = x[i + j * ldx];
    TY h = from_f32<TY>(v);
    y[i + j * ldy] = h;
    if (lo) lo[i + j * ldy] = from_f32<TY>(v - to_f32<TY>(h));
  }
}

template <typename T>
__global__ void copy2d_kernel(const T* __restrict__ x, int64_t ldx, T* __restrict__ y, int64_t ldy,
                              int64_t rows, int64_t cols, const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int64_t j = e / rows, i = e - j * rows;
    y[i + j * ldy] = x[i + j * ldx];
  }
}

// At (cols x rows, ldt) = A^T for column-major A (rows x cols, lda): 32 x 32
// tiles through shared memory (padded against bank conflicts), coalesced on
// both sides.
__global__ void __launch_bounds__(256)
transpose32_kernel(const float* __restrict__ A, int64_t lda, int64_t rows, int64_t cols, float* __restrict__ At,
                   int64_t ldt) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
#pragma unroll
  for (int k = 0; k < 32; k += 8) {
    const int64_t r = r0 + tx, c = c0 + ty + k;
    tile[ty + k][tx] = (r < rows && c < cols) ? A[r + c * lda] : 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 32; k += 8) {
    const int64_t c = c0 + tx, r = r0 + ty + k;
    if (c < cols && r < rows) At[c + r * ldt] = tile[tx][ty + k];
  }
}

// The same transpose in 64 x 64 tiles with 8-byte accesses: a lane moves
// two consecutive rows (loads) or columns (stores), so each thread keeps 8
// loads of 8 bytes in flight (the 32 x 32 kernel: 4 of 4 bytes), enough to
// cover HBM latency at full bandwidth.  Needs lda, ldt even and 8-byte
// aligned A, At; ragged edges fall back to scalar accesses.
__global__ void __launch_bounds__(256)
transpose64_kernel(const float* __restrict__ A, int64_t lda, int64_t rows, int64_t cols, float* __restrict__ At,
                   int64_t ldt) {
  __shared__ float tile[64][65];                  // tile[c][r]
  const int64_t r0 = (int64_t)blockIdx.x * 64, c0 = (int64_t)blockIdx.y * 64;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  const bool full = r0 + 64 <= rows && c0 + 64 <= cols;
  if (full) {
    float2 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k)
      v[k] = *reinterpret_cast<const float2*>(A + (r0 + 2 * tx) + (c0 + ty + 8 * k) * lda);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      tile[ty + 8 * k][2 * tx] = v[k].x;
      tile[ty + 8 * k][2 * tx + 1] = v[k].y;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t c = c0 + ty + 8 * k;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t r = r0 + 2 * tx + h;
        tile[ty + 8 * k][2 * tx + h] = (r < rows && c < cols) ? A[r + c * lda] : 0.f;
      }
    }
  }
  __syncthreads();
  if (full) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int rr = ty + 8 * k;
      float2 w;
      w.x = tile[2 * tx][rr];
      w.y = tile[2 * tx + 1][rr];
      *reinterpret_cast<float2*>(At + (c0 + 2 * tx) + (r0 + rr) * ldt) = w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t r = r0 + ty + 8 * k;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t c = c0 + 2 * tx + h;
        if (c < cols && r < rows) At[c + r * ldt] = tile[2 * tx + h][ty + 8 * k];
      }
    }
  }
}

inline int grid_for(int64_t total) {
  int64_t b = (total + 255) / 256;
  int64_t cap = (int64_t)num_sms() * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

cudaError_t launch_gemm(bool trans_a, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda, int a_dt,
                        const void* B, int64_t ldb, int b_dt, void* C, int64_t ldc, bool acc_f64,
                        int splits, int64_t split_stride, cudaStream_t st, const int* skip) {
  if (acc_f64) {
    if (a_dt == SORSVD_F64 && b_dt == SORSVD_F64)
      return gemm_dispatch<double, double, double>(trans_a, M, N, K, A, lda, B, ldb, C, ldc, splits, split_stride, st,
                                                   skip);
    return cudaErrorInvalidValue;
  }
  bool a32 = (a_dt == SORSVD_F32 || a_dt == SORSVD_TF32), b32 = (b_dt == SORSVD_F32 || b_dt == SORSVD_TF32);
  if (a32 && b32) return gemm_dispatch<float, float, float>(trans_a, M, N, K, A, lda, B, ldb, C, ldc, splits, split_stride, st);
  if (a_dt == SORSVD_BF16 && b_dt == SORSVD_BF16) return gemm_dispatch<bf16, bf16, float>(trans_a, M, N, K, A, lda, B, ldb, C, ldc, splits, split_stride, st);
  if (a_dt == SORSVD_BF16 && b32) return gemm_dispatch<bf16, float, float>(trans_a, M, N, K, A, lda, B, ldb, C, ldc, splits, split_stride, st);
  if (a_dt == SORSVD_F16 && b_dt == SORSVD_F16) return gemm_dispatch<f16, f16, float>(trans_a, M, N, K, A, lda, B, ldb, C, ldc, splits, split_stride, st);
  if (a_dt == SORSVD_F16 && b32) return gemm_dispatch<f16, float, float>(trans_a, M, N, K, A, lda, B, ldb, C, ldc, splits, split_stride, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_reduce_splits(const void* parts, bool parts_f64, int splits, int64_t split_stride,
                                 int64_t rows, int64_t cols, int64_t ld_part, void* out, bool out_f64,
                                 int64_t ld_out, cudaStream_t st, const int* skip) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  int g = grid_for(rows * cols);
  if (parts_f64 && out_f64)
    reduce_kernel<double, double><<<g, 256, 0, st>>>((const double*)parts, splits, split_stride, rows, cols, ld_part, (double*)out, ld_out, skip);
  else if (parts_f64)
    reduce_kernel<double, float><<<g, 256, 0, st>>>((const double*)parts, splits, split_stride, rows, cols, ld_part, (float*)out, ld_out, skip);
  else if (out_f64)
    reduce_kernel<float, double><<<g, 256, 0, st>>>((const float*)parts, splits, split_stride, rows, cols, ld_part, (double*)out, ld_out, skip);
  else
    reduce_kernel<float, float><<<g, 256, 0, st>>>((const float*)parts, splits, split_stride, rows, cols, ld_part, (float*)out, ld_out, skip);
  return cudaGetLastError();
}

cudaError_t launch_convert_f32(const float* x, int64_t ldx, int64_t rows, int64_t cols, void* y, int64_t ldy,
                               int y_dt, void* lo, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  int g = grid_for(rows * cols);
  if (y_dt == SORSVD_BF16)
    convert_kernel<bf16><<<g, 256, 0, st>>>(x, ldx, rows, cols, (bf16*)y, ldy, (bf16*)lo);
  else if (y_dt == SORSVD_F16)
    convert_kernel<f16><<<g, 256, 0, st>>>(x, ldx, rows, cols, (f16*)y, ldy, (f16*)lo);
  else
    return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_transpose_f32(const float* A, int64_t lda, int64_t rows, int64_t cols, float* At, int64_t ldt,
                                 cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const bool pairs = !(lda & 1) && !(ldt & 1) && !(reinterpret_cast<uintptr_t>(A) & 7) &&
                     !(reinterpret_cast<uintptr_t>(At) & 7);
  if (pairs && (cols + 63) / 64 <= 65535) {
    dim3 grid((unsigned)((rows + 63) / 64), (unsigned)((cols + 63) / 64));
    transpose64_kernel<<<grid, 256, 0, st>>>(A, lda, rows, cols, At, ldt);
    return cudaGetLastError();
  }
  dim3 grid((unsigned)((rows + 31) / 32), (unsigned)((cols + 31) / 32));
  if (grid.y > 65535) return cudaErrorInvalidValue;
  transpose32_kernel<<<grid, 256, 0, st>>>(A, lda, rows, cols, At, ldt);
  return cudaGetLastError();
}

cudaError_t launch_copy2d(const void* x, int64_t ldx, void* y, int64_t ldy, int64_t rows, int64_t cols,
                          size_t elem, cudaStream_t st, const int* skip) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  int g = grid_for(rows * cols);
  if (elem == 8) copy2d_kernel<double><<<g, 256, 0, st>>>((const double*)x, ldx, (double*)y, ldy, rows, cols, skip);
  else if (elem == 4) copy2d_kernel<float><<<g, 256, 0, st>>>((const float*)x, ldx, (float*)y, ldy, rows, cols, skip);
  else if (elem == 2) copy2d_kernel<uint16_t><<<g, 256, 0, st>>>((const uint16_t*)x, ldx, (uint16_t*)y, ldy, rows, cols, skip);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

template <class Cfg>
cudaError_t launch_gemm_batched_cfg(bool trans_a, bool f64, const GemmJob* jobs, const int4* units, int nunits,
                                    cudaStream_t st) {
  if (f64) {
    if (trans_a) gemm_batched_kernel<Cfg, double, true><<<nunits, NT, 0, st>>>(jobs, units);
    else gemm_batched_kernel<Cfg, double, false><<<nunits, NT, 0, st>>>(jobs, units);
  } else {
    if (trans_a) gemm_batched_kernel<Cfg, float, true><<<nunits, NT, 0, st>>>(jobs, units);
    else gemm_batched_kernel<Cfg, float, false><<<nunits, NT, 0, st>>>(jobs, units);
  }
  return cudaGetLastError();
}

cudaError_t launch_gemm_batched(bool trans_a, bool f64, int tile, const GemmJob* jobs, const int4* units, int nunits,
                                cudaStream_t st) {
  if (nunits <= 0) return cudaSuccess;
  switch (tile) {
    case 0: return launch_gemm_batched_cfg<BigTile>(trans_a, f64, jobs, units, nunits, st);
    case 1: return launch_gemm_batched_cfg<MidTile>(trans_a, f64, jobs, units, nunits, st);
    case 2: return launch_gemm_batched_cfg<SkinnyTile>(trans_a, f64, jobs, units, nunits, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_reduce_batched(bool parts_f64, const ReduceJob* jobs, int njobs, int64_t max_elems,
                                  cudaStream_t st) {
  if (njobs <= 0 || max_elems <= 0) return cudaSuccess;
  const int64_t bx = std::min<int64_t>((max_elems + 255) / 256, 64);
  dim3 grid((unsigned)bx, (unsigned)njobs);
  if (parts_f64) reduce_batched_kernel<double><<<grid, 256, 0, st>>>(jobs);
  else reduce_batched_kernel<float><<<grid, 256, 0, st>>>(jobs);
  return cudaGetLastError();
}

// the tile shapes of the grouped kernel (units are counted in these tiles;
// every shape takes 16-deep K slices, so a job's K chunks do not depend on
// the shape)
void gemm_tile_shape(int tile, int* bm, int* bn, int* bk) {
  switch (tile) {
    case 1: *bm = MidTile::BM; *bn = MidTile::BN; *bk = MidTile::BK; return;
    case 2: *bm = SkinnyTile::BM; *bn = SkinnyTile::BN; *bk = SkinnyTile::BK; return;
    default: *bm = BigTile::BM; *bn = BigTile::BN; *bk = BigTile::BK; return;
  }
}

namespace {
__global__ void add_f64_kernel(const double* __restrict__ x, int64_t ldx, double* __restrict__ y, int64_t ldy,
                               int64_t rows, int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / rows, i = e - j * rows;
    y[i + j * ldy] += x[i + j * ldx];
  }
}
__global__ void add_f32_kernel(const float* __restrict__ x, int64_t ldx, float* __restrict__ y, int64_t ldy,
                               int64_t rows, int64_t cols) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = e / rows, i = e - j * rows;
    y[i + j * ldy] += x[i + j * ldx];
  }
}
}  // namespace

cudaError_t launch_add_f32(const float* x, int64_t ldx, float* y, int64_t ldy, int64_t rows, int64_t cols,
                           cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  add_f32_kernel<<<grid_for(rows * cols), 256, 0, st>>>(x, ldx, y, ldy, rows, cols);
  return cudaGetLastError();
}

cudaError_t launch_add_f64(const double* x, int64_t ldx, double* y, int64_t ldy, int64_t rows, int64_t cols,
                           cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  add_f64_kernel<<<grid_for(rows * cols), 256, 0, st>>>(x, ldx, y, ldy, rows, cols);
  return cudaGetLastError();
}

}  // namespace sorsvd
