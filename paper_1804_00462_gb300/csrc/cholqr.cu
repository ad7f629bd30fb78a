// Row-block kernels of CholeskyQR for fp32 sketches with l <= kCqMaxL (the
// QR step of Algorithm 3 and the re-orthonormalisation of the power loop).
// A CholeskyQR pass is  G = T^T T,  R^{-1} = chol(G)^{-1} (chol.cu),
// T <- T R^{-1}.  Both tall-skinny products run here, a grid of CTAs
// striding over blocks of kCqRows rows of T, each block staged in shared
// memory:
//
//   cq_gram_kernel:   partial Gram of the CTA's blocks, sum_b T_b^T T_b
//                     (fp32, registers across blocks), to parts[cta]; the
//                     partials (one per SM) are summed in a fixed order by
//                     launch_reduce_parts_warp (compensated, binary64).
//   cq_apply_kernel:  T_b <- T_b R^{-1} in place (R^{-1} upper triangular:
//                     only k <= j terms), and, when a next pass follows, the
//                     partial Gram of the new blocks from the same shared
//                     copies - the next pass does not read T again.
//
// Shared layout: the block row-major, X[r][c] (r < kCqRows, c < lp = l
// rounded up to 4, row stride lp + 4), R^{-1} row-major [k][j] (stride lp).
// Each thread computes 4 x 4 output blocks from float4 loads: for the Gram
// all threads of a warp read the same row of X (broadcast / contiguous), for
// the product the same rows of X and contiguous pieces of R's rows.  Global
// loads and stores go through the shared copy, coalesced along the rows.
#include "internal.cuh"
#include "profile.cuh"

#include <algorithm>

namespace sorsvd {
namespace {

constexpr int kCqRows = 64;                 // rows of T per CTA
constexpr int kCqThreads = 256;

__host__ __device__ inline int cq_lp(int l) { return (l + 3) & ~3; }
__host__ __device__ inline int cq_xs(int lp) { return lp + 4; }
inline size_t cq_smem(int l, bool with_r) {
  const int lp = cq_lp(l);
  return (size_t)kCqRows * cq_xs(lp) * 4 + (with_r ? (size_t)lp * lp * 4 : 0);
}

// X[r][c] <- T[r0 + r + c ld] (rows past `rows`, columns past l: zero)
__device__ __forceinline__ void cq_load_block(const float* __restrict__ T, int64_t ld, int64_t rows, int l, int lp,
                                              int64_t r0, float* X) {
  const int xs = cq_xs(lp);
  for (int e = threadIdx.x; e < lp * kCqRows; e += blockDim.x) {
    const int c = e / kCqRows, r = e - c * kCqRows;
    const int64_t gr = r0 + r;
    X[r * xs + c] = (c < l && gr < rows) ? T[gr + (int64_t)c * ld] : 0.f;
  }
}

// Gram accumulation over the staged block: the thread's 4 x 4 blocks of the
// lower triangle (block q = threadIdx.x + i * blockDim.x, i < kGramPer) add
// sum_r X[r][i] X[r][j]; cq_gram_store writes them (both halves).
constexpr int kGramPer = ((kCqMaxL / 4) * (kCqMaxL / 4 + 1) / 2 + kCqThreads - 1) / kCqThreads;

__device__ __forceinline__ void cq_block_of(int q, int* i0, int* j0) {
  int bi = (int)((sqrtf(8.f * q + 1.f) - 1.f) * 0.5f);
  while ((bi + 1) * (bi + 2) / 2 <= q) ++bi;
  while (bi * (bi + 1) / 2 > q) --bi;
  *i0 = 4 * bi;
  *j0 = 4 * (q - bi * (bi + 1) / 2);
}

__device__ __forceinline__ void cq_gram_acc(const float* X, int lp, float (&acc)[kGramPer][4][4]) {
  const int xs = cq_xs(lp);
  const int nb = lp / 4;
  const int nblk = nb * (nb + 1) / 2;
#pragma unroll
  for (int p = 0; p < kGramPer; ++p) {
    const int q = threadIdx.x + p * kCqThreads;
    if (q >= nblk) break;
    int i0, j0;
    cq_block_of(q, &i0, &j0);
    for (int r = 0; r < kCqRows; ++r) {
      const float4 a = *reinterpret_cast<const float4*>(X + r * xs + i0);
      const float4 b = *reinterpret_cast<const float4*>(X + r * xs + j0);
      const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[p][u][v] = fmaf(av[u], bv[v], acc[p][u][v]);
    }
  }
}

__device__ __forceinline__ void cq_gram_store(int l, int lp, const float (&acc)[kGramPer][4][4], float* __restrict__ out) {
  const int nb = lp / 4;
  const int nblk = nb * (nb + 1) / 2;
#pragma unroll
  for (int p = 0; p < kGramPer; ++p) {
    const int q = threadIdx.x + p * kCqThreads;
    if (q >= nblk) break;
    int i0, j0;
    cq_block_of(q, &i0, &j0);
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const int i = i0 + u, j = j0 + v;
        if (i < l && j < l) {
          out[i + (size_t)j * l] = acc[p][u][v];
          out[j + (size_t)i * l] = acc[p][u][v];
        }
      }
  }
}

// grid-stride over the chunks of kCqRows rows: block b's partial Gram is
// the sum over its chunks (fixed chunk order: deterministic)
__global__ void __launch_bounds__(kCqThreads)
cq_gram_kernel(const float* __restrict__ T, int64_t ld, int64_t rows, int l, float* __restrict__ parts) {
  extern __shared__ __align__(16) float sm[];
  const int lp = cq_lp(l);
  float acc[kGramPer][4][4] = {};
  const int64_t nchunk = (rows + kCqRows - 1) / kCqRows;
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    __syncthreads();
    cq_load_block(T, ld, rows, l, lp, ch * kCqRows, sm);
    __syncthreads();
    cq_gram_acc(sm, lp, acc);
  }
  cq_gram_store(l, lp, acc, parts + (size_t)blockIdx.x * l * l);
}

__global__ void __launch_bounds__(kCqThreads)
cq_apply_kernel(float* __restrict__ T, int64_t ld, int64_t rows, int l, const float* __restrict__ Rinv,
                float* __restrict__ parts) {
  extern __shared__ __align__(16) float sm[];
  const int lp = cq_lp(l), xs = cq_xs(lp);
  float* X = sm;
  float* R = sm + (size_t)kCqRows * xs;        // R[k * lp + j] = R^{-1}(k, j)
  for (int e = threadIdx.x; e < lp * lp; e += blockDim.x) {
    const int j = e / lp, k = e - j * lp;       // coalesced read of column j of R^{-1}
    R[k * lp + j] = (k < l && j < l) ? Rinv[k + (size_t)j * l] : 0.f;
  }
  float gacc[kGramPer][4][4] = {};
  const int nrb = kCqRows / 4, njb = lp / 4;
  constexpr int kMaxPer = (kCqRows / 4) * (kCqMaxL / 4) / kCqThreads + 1;
  const int64_t nchunk = (rows + kCqRows - 1) / kCqRows;
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    const int64_t r0 = ch * kCqRows;
    __syncthreads();
    cq_load_block(T, ld, rows, l, lp, r0, X);
    __syncthreads();
    // Q[r][j] = sum_{k <= j} X[r][k] R[k][j]: 4 x 4 blocks, column block
    // fastest so a warp shares its rows of X
    float4 res[kMaxPer][4];                     // res[.][u]: row rr+u, columns j0..j0+3
#pragma unroll
    for (int p = 0; p < kMaxPer; ++p) {
      const int q = threadIdx.x + p * kCqThreads;
      if (q >= nrb * njb) break;
      const int jb = q % njb, rb = q / njb;
      const int rr = 4 * rb, j0 = 4 * jb;
      float acc[4][4] = {};
      const int kend = min(lp, j0 + 4);          // R^{-1} upper triangular
      for (int k = 0; k < kend; k += 4) {
        float xv[4][4], rv[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 x = *reinterpret_cast<const float4*>(X + (rr + u) * xs + k);
          xv[u][0] = x.x; xv[u][1] = x.y; xv[u][2] = x.z; xv[u][3] = x.w;
          const float4 rk = *reinterpret_cast<const float4*>(R + (k + u) * lp + j0);
          rv[u][0] = rk.x; rv[u][1] = rk.y; rv[u][2] = rk.z; rv[u][3] = rk.w;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(xv[u][kk], rv[kk][v], acc[u][v]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) res[p][u] = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
    }
    __syncthreads();
#pragma unroll
    for (int p = 0; p < kMaxPer; ++p) {
      const int q = threadIdx.x + p * kCqThreads;
      if (q >= nrb * njb) break;
      const int jb = q % njb, rb = q / njb;
      const int rr = 4 * rb, j0 = 4 * jb;
#pragma unroll
      for (int u = 0; u < 4; ++u) *reinterpret_cast<float4*>(X + (rr + u) * xs + j0) = res[p][u];
    }
    __syncthreads();
    // the new block back to T (in place), coalesced along the rows
    for (int e = threadIdx.x; e < l * kCqRows; e += blockDim.x) {
      const int c = e / kCqRows, r = e - c * kCqRows;
      const int64_t gr = r0 + r;
      if (gr < rows) T[gr + (int64_t)c * ld] = X[r * xs + c];
    }
    if (parts) cq_gram_acc(X, lp, gacc);
  }
  if (parts) cq_gram_store(l, lp, gacc, parts + (size_t)blockIdx.x * l * l);
}

// ---------------------------------------------------------------- wide
// kCqMaxL < l <= SORSVD_MAX_L: the Gram and the product no longer fit one
// CTA's registers / shared memory whole, so both are tiled.
//
//   cq_gram_wide_kernel:  grid (x: row chunks, y: groups of kCqThreads 8 x 8
//       blocks of the lower triangle); a thread accumulates one 8 x 8 block
//       over the CTA's chunks (the whole row chunk is staged, every column);
//       partial Grams per grid column x, both halves written.
//   cq_apply_wide_kernel: T_b <- T_b R^{-1} in place, panels of 128 output
//       columns from the last to the first (a panel only reads columns to
//       its left and its own, so it can overwrite itself in shared memory),
//       R^{-1} streamed through a 32 x 128 shared tile (zero below the
//       diagonal and past l).
constexpr int kWideKT = 32;                  // k rows per R^{-1} tile
constexpr int kWidePW = 128;                 // output columns per panel
constexpr int kWideRS = kWidePW + 4;         // R^{-1} tile row stride

__host__ __device__ inline int cq_lp8(int l) { return (l + 7) & ~7; }
inline int cq_wide_groups(int l) {
  const int nb = cq_lp8(l) / 8;
  return (nb * (nb + 1) / 2 + kCqThreads - 1) / kCqThreads;
}
inline size_t cq_wide_gram_smem(int l) { return (size_t)kCqRows * cq_xs(cq_lp8(l)) * 4; }
inline size_t cq_wide_apply_smem(int l) {
  return (size_t)kCqRows * cq_xs(cq_lp8(l)) * 4 + (size_t)kWideKT * kWideRS * 4;
}

__global__ void __launch_bounds__(kCqThreads, 2)
cq_gram_wide_kernel(const float* __restrict__ T, int64_t ld, int64_t rows, int l, float* __restrict__ parts,
                    const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) float sm[];
  const int lp = cq_lp8(l), xs = cq_xs(lp);
  const int nb = lp / 8, nblk = nb * (nb + 1) / 2;
  const int q = blockIdx.y * kCqThreads + threadIdx.x;
  const bool act = q < nblk;
  int i0 = 0, j0 = 0;
  if (act) {
    cq_block_of(q, &i0, &j0);                 // 4 x (block row, block column)
    i0 *= 2;
    j0 *= 2;
  }
  float acc[8][8] = {};
  const int64_t nchunk = (rows + kCqRows - 1) / kCqRows;
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    __syncthreads();
    cq_load_block(T, ld, rows, l, lp, ch * kCqRows, sm);
    __syncthreads();
    if (!act) continue;
    for (int r = 0; r < kCqRows; ++r) {
      const float* xr = sm + r * xs;
      const float4 a0 = *reinterpret_cast<const float4*>(xr + i0);
      const float4 a1 = *reinterpret_cast<const float4*>(xr + i0 + 4);
      const float4 b0 = *reinterpret_cast<const float4*>(xr + j0);
      const float4 b1 = *reinterpret_cast<const float4*>(xr + j0 + 4);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
  }
  if (!act) return;
  float* out = parts + (size_t)blockIdx.x * l * l;
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int i = i0 + u, j = j0 + v;
      if (i < l && j < l) {
        out[i + (size_t)j * l] = acc[u][v];
        out[j + (size_t)i * l] = acc[u][v];
      }
    }
}

__global__ void __launch_bounds__(kCqThreads, 2)
cq_apply_wide_kernel(float* __restrict__ T, int64_t ld, int64_t rows, int l, const float* __restrict__ Rinv,
                     const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) float sm[];
  const int lp = cq_lp8(l), xs = cq_xs(lp);
  float* X = sm;
  float* Rs = sm + (size_t)kCqRows * xs;      // Rs[kk * kWideRS + jj] = R^{-1}(k0 + kk, j0 + jj)
  // thread: rows 4 tr .. 4 tr + 3 of the chunk, panel columns 4 tc .. 4 tc + 3
  // and 64 + 4 tc .. 64 + 4 tc + 3 (a warp's R loads are two contiguous
  // 256-byte runs)
  const int tr = threadIdx.x / 16, tc = threadIdx.x % 16;
  const int npan = (lp + kWidePW - 1) / kWidePW;
  const int64_t nchunk = (rows + kCqRows - 1) / kCqRows;
  for (int64_t ch = blockIdx.x; ch < nchunk; ch += gridDim.x) {
    const int64_t r0 = ch * kCqRows;
    __syncthreads();
    cq_load_block(T, ld, rows, l, lp, r0, X);
    for (int J = npan - 1; J >= 0; --J) {
      const int j0 = J * kWidePW, pw = min(kWidePW, lp - j0), kend = j0 + pw;
      const bool act = 4 * tc < pw;
      float acc[4][8] = {};
      for (int k0 = 0; k0 < kend; k0 += kWideKT) {
        __syncthreads();                      // X staged / previous tile consumed
        for (int e = threadIdx.x; e < kWideKT * kWidePW; e += blockDim.x) {
          const int jj = e / kWideKT, kk = e - jj * kWideKT;
          const int k = k0 + kk, j = j0 + jj;
          Rs[kk * kWideRS + jj] = (j < l && k <= j) ? Rinv[k + (size_t)j * l] : 0.f;
        }
        __syncthreads();
        if (!act) continue;
        const int kn = min(kWideKT, kend - k0);   // a multiple of 8
        for (int kk = 0; kk < kn; kk += 4) {
          float xv[4][4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const float4 x = *reinterpret_cast<const float4*>(X + (4 * tr + u) * xs + k0 + kk);
            xv[u][0] = x.x; xv[u][1] = x.y; xv[u][2] = x.z; xv[u][3] = x.w;
          }
#pragma unroll
          for (int qq = 0; qq < 4; ++qq) {
            const float* rr = Rs + (kk + qq) * kWideRS;
            const float4 ra = *reinterpret_cast<const float4*>(rr + 4 * tc);
            const float4 rb = *reinterpret_cast<const float4*>(rr + 64 + 4 * tc);
            const float rv[8] = {ra.x, ra.y, ra.z, ra.w, rb.x, rb.y, rb.z, rb.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(xv[u][qq], rv[v], acc[u][v]);
          }
        }
      }
      __syncthreads();                        // every read of this panel's columns is done
      if (act) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          float* xr = X + (4 * tr + u) * xs + j0;
          *reinterpret_cast<float4*>(xr + 4 * tc) = make_float4(acc[u][0], acc[u][1], acc[u][2], acc[u][3]);
          if (64 + 4 * tc < pw)
            *reinterpret_cast<float4*>(xr + 64 + 4 * tc) = make_float4(acc[u][4], acc[u][5], acc[u][6], acc[u][7]);
        }
      }
    }
    __syncthreads();
    for (int e = threadIdx.x; e < l * kCqRows; e += blockDim.x) {
      const int c = e / kCqRows, r = e - c * kCqRows;
      const int64_t gr = r0 + r;
      if (gr < rows) T[gr + (int64_t)c * ld] = X[r * xs + c];
    }
  }
}

// out[i + j ldo] = sum_s parts[s * stride + i + j ldp] (binary64) for an
// rows x cols result: one warp per element, lane t takes the partials
// t, t + 32, ... (Neumaier compensated fp32 sums), then a fixed xor tree
// of the 32 (sum, compensation) pairs in binary64: deterministic.
__global__ void reduce_parts_warp_kernel(const float* __restrict__ parts, int nparts, int64_t stride, int rows,
                                         int cols, int ldp, double* __restrict__ out, int ldo) {
  const int lane = threadIdx.x & 31;
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (w >= (int64_t)rows * cols) return;
  const int j = (int)(w / rows), i = (int)(w - (int64_t)j * rows);
  const float* p = parts + i + (int64_t)j * ldp;
  float s = 0.f, c = 0.f;
  for (int q = lane; q < nparts; q += 32) {
    const float x = p[q * stride];
    const float t = __fadd_rn(s, x);
    c = __fadd_rn(c, fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s));
    s = t;
  }
  double v = (double)s + (double)c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if (lane == 0) out[i + (int64_t)j * ldo] = v;
}

}  // namespace

cudaError_t launch_reduce_parts_warp(const float* parts, int nparts, int64_t stride, int rows, int cols, int ldp,
                                     double* out, int ldo, cudaStream_t st) {
  const int64_t threads = (int64_t)rows * cols * 32;
  if (threads <= 0) return cudaSuccess;
  reduce_parts_warp_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(parts, nparts, stride, rows, cols, ldp,
                                                                           out, ldo);
  return cudaGetLastError();
}

// CTAs of the grid (= partial Grams): one per SM (the apply kernel's
// register footprint allows one resident CTA)
int64_t cq_blocks(int64_t rows) {
  const int64_t nchunk = (rows + kCqRows - 1) / kCqRows;
  return std::max<int64_t>(1, std::min<int64_t>(nchunk, (int64_t)num_sms()));
}

// wide Gram: grid columns (= partial Grams), about two CTAs per SM in all
int64_t cq_wide_blocks(int64_t rows, int l) {
  const int64_t nchunk = (rows + kCqRows - 1) / kCqRows;
  const int64_t gy = cq_wide_groups(l);
  const int64_t want = (2 * (int64_t)num_sms() + gy - 1) / gy;
  return std::max<int64_t>(1, std::min<int64_t>(nchunk, want));
}

cudaError_t launch_cq_gram_wide(const float* T, int64_t ld, int64_t rows, int l, float* parts, const int* skip,
                                cudaStream_t st) {
  if (l <= kCqMaxL || l > SORSVD_MAX_L || rows < 1) return cudaErrorInvalidValue;
  const size_t sm = cq_wide_gram_smem(l);
  cudaError_t e = cudaFuncSetAttribute(cq_gram_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)cq_wide_blocks(rows, l), (unsigned)cq_wide_groups(l));
  cq_gram_wide_kernel<<<grid, kCqThreads, sm, st>>>(T, ld, rows, l, parts, skip);
  return cudaGetLastError();
}

cudaError_t launch_cq_apply_wide(float* T, int64_t ld, int64_t rows, int l, const float* Rinv, const int* skip,
                                 cudaStream_t st) {
  if (l <= kCqMaxL || l > SORSVD_MAX_L || rows < 1) return cudaErrorInvalidValue;
  const size_t sm = cq_wide_apply_smem(l);
  cudaError_t e = cudaFuncSetAttribute(cq_apply_wide_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int64_t nchunk = (rows + kCqRows - 1) / kCqRows;
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(nchunk, 2 * (int64_t)num_sms()));
  cq_apply_wide_kernel<<<(unsigned)grid, kCqThreads, sm, st>>>(T, ld, rows, l, Rinv, skip);
  return cudaGetLastError();
}

cudaError_t launch_cq_gram(const float* T, int64_t ld, int64_t rows, int l, float* parts, cudaStream_t st) {
  if (l < 1 || l > kCqMaxL || rows < 1) return cudaErrorInvalidValue;
  const size_t sm = cq_smem(l, false);
  cudaError_t e = cudaFuncSetAttribute(cq_gram_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  cq_gram_kernel<<<(unsigned)cq_blocks(rows), kCqThreads, sm, st>>>(T, ld, rows, l, parts);
  return cudaGetLastError();
}

cudaError_t launch_cq_apply(float* T, int64_t ld, int64_t rows, int l, const float* Rinv, float* parts,
                            cudaStream_t st) {
  if (l < 1 || l > kCqMaxL || rows < 1) return cudaErrorInvalidValue;
  const size_t sm = cq_smem(l, true);
  cudaError_t e = cudaFuncSetAttribute(cq_apply_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  cq_apply_kernel<<<(unsigned)cq_blocks(rows), kCqThreads, sm, st>>>(T, ld, rows, l, Rinv, parts);
  return cudaGetLastError();
}

}  // namespace sorsvd
