// Second CholeskyQR pass of the QR step of Algorithm 3 (T1 = Q1 R1, T2 = Q2 R2) in polar form.
//
// After one CholeskyQR pass the Gram G = T^T T of the sketch is close to the
// identity.  Any l x l matrix X with X^T G X = I makes Q = T X an
// orthonormal basis of range(T), which is all the QR step is used for (R is
// not used afterwards; Lemma 1 makes the projector independent of the
// factor).  With D = diag(G) and I + E = D^{-1/2} G D^{-1/2} (unit
// diagonal, E symmetric) the symmetric choice is
//   X = D^{-1/2} (I + E)^{-1/2},
// and for ||E||_2 < 1 the binomial series converges:
//   (I + E)^{-1/2} = I - E/2 + (3/8) E^2 - (5/16) E^3 + (35/128) E^4 - ...
// Keeping the terms up to E^3 leaves a remainder below
// (35/128) ||E||^4 / (1 - ||E||); for ||E||_F <= kPolarMaxE = 0.02 that is
// < 5e-8, under the fp32 unit roundoff of the sketch.  The series is
// evaluated in Horner form with two l x l products,
//   Y = (3/8) E - (5/16) E^2,   X' = I - E/2 + E Y,
// on a grid of 32 x 32 output tiles in fp32 (the entries of E are small, so
// their fp32 rounding is far below the sketch's), where a one-block
// Cholesky factorisation is bound by its chain of barriers.  Larger ||E|| (the first pass left T far from
// orthonormal) sets *ok = 0 and the caller's Cholesky kernel, which returns
// at once when *ok is set, factorises instead.
//
// Three launches: E (and the scales), Y, X.  The decision and
// the largest off-diagonal |E_ij| (the column cosine that decides whether a
// third pass is needed) come from fixed-order reductions of per-tile row
// partials, so the result does not depend on scheduling.
#include "internal.cuh"

namespace sorsvd {
namespace {

constexpr int PT = 32;          // output tile
constexpr int PTHREADS = 256;   // 32 x 8: each thread 4 rows of one column
constexpr float kPolarMaxE = 0.02f;

// d_i = 1 / sqrt(G_ii) in binary64, rounded to fp32 (1 for a zero column,
// whose row and column of E are zero); E_ij = G_ij d_i d_j (i != j) in fp32,
// E_ii = 0 (the equilibrated diagonal is 1 by construction)
__global__ void __launch_bounds__(PTHREADS)
polar_e_kernel(const double* __restrict__ G, int l, float* __restrict__ E, float* __restrict__ d) {
  __shared__ float dr[PT], dc[PT];
  const int bi = blockIdx.x, bj = blockIdx.y;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (threadIdx.x < 2 * PT) {
    // v: the scale in E (0 for a zero column), d: the scale of X (1 there)
    const int k = threadIdx.x < PT ? bi * PT + threadIdx.x : bj * PT + threadIdx.x - PT;
    float v = 0.f;
    if (k < l) {
      const double g = G[k + (int64_t)k * l];
      v = g > 0.0 ? (float)(1.0 / sqrt(g)) : 0.f;
    }
    if (threadIdx.x < PT) dr[threadIdx.x] = v;
    else dc[threadIdx.x - PT] = v;
    if (threadIdx.x < PT && bj == 0 && k < l) d[k] = v > 0.f ? v : 1.f;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = bj * PT + ty + 8 * u, i = bi * PT + tx;       // lanes along i: coalesced
    if (i < l && j < l)
      E[i + (int64_t)j * l] = (i == j) ? 0.f : (float)G[i + (int64_t)j * l] * dr[tx] * dc[ty + 8 * u];
  }
}

// acc[u] = sum_k E[i, k] B[k, j] for the thread's outputs i = bi PT + tx,
// j = bj PT + ty + 8 u (lanes along the contiguous index i of the
// column-major results)
__device__ __forceinline__ void tile_product(const float* __restrict__ E, const float* __restrict__ B, int l,
                                             int bi, int bj, float (&acc)[4]) {
  __shared__ float sa[PT][PT + 1], sb[PT][PT + 1];   // sa[i][k], sb[k][j] (local indices)
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = 0.f;
  for (int k0 = 0; k0 < l; k0 += PT) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = ty + 8 * u;
      const int i = bi * PT + tx, k = k0 + c;                // E[i, k]: lanes along i
      sa[tx][c] = (i < l && k < l) ? E[i + (int64_t)k * l] : 0.f;
      const int kk = k0 + tx, jj = bj * PT + c;              // B[k, j]: lanes along k
      sb[tx][c] = (kk < l && jj < l) ? B[kk + (int64_t)jj * l] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < PT; ++kk) {
      const float a = sa[tx][kk];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fmaf(a, sb[kk][ty + 8 * u], acc[u]);
    }
    __syncthreads();
  }
}

// Y = (3/8) E - (5/16) E^2; per tile column bj and row i the sum of E_ij^2
// and the largest |E_ij| over the tile's columns
__global__ void __launch_bounds__(PTHREADS)
polar_y_kernel(const float* __restrict__ E, int l, float* __restrict__ Y, float* __restrict__ rsum,
               float* __restrict__ rmax) {
  const int bi = blockIdx.x, bj = blockIdx.y;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[4];
  tile_product(E, E, l, bi, bj, acc);
  __shared__ float ssum[PT][PT + 1], smax[PT][PT + 1];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = bi * PT + tx, j = bj * PT + ty + 8 * u;
    const float e = (i < l && j < l) ? E[i + (int64_t)j * l] : 0.f;
    if (i < l && j < l) Y[i + (int64_t)j * l] = 0.375f * e - 0.3125f * acc[u];
    ssum[tx][ty + 8 * u] = e * e;
    smax[tx][ty + 8 * u] = fabsf(e);
  }
  __syncthreads();
  // row partials over this tile's 32 columns, fixed order
  if (threadIdx.x < PT) {
    const int r = threadIdx.x, i = bi * PT + r;
    float s = 0.f, mx = 0.f;
    for (int c = 0; c < PT; ++c) {
      s += ssum[r][c];
      mx = fmaxf(mx, smax[r][c]);
    }
    if (i < l) {
      rsum[(int64_t)bj * l + i] = s;
      rmax[(int64_t)bj * l + i] = mx;
    }
  }
}

// X = D^{-1/2} (I - E/2 + E Y) into Rinv (l x l, ld l); block (0, 0) also
// decides: *ok = ||E||_F <= kPolarMaxE, *conv = *ok and max |E_ij| <= conv_tol
__global__ void __launch_bounds__(PTHREADS)
polar_x_kernel(const float* __restrict__ E, const float* __restrict__ Y, const float* __restrict__ d, int l,
               const float* __restrict__ rsum, const float* __restrict__ rmax, float* __restrict__ Rinv,
               int* __restrict__ ok, int* __restrict__ conv, float conv_tol) {
  const int bi = blockIdx.x, bj = blockIdx.y;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  float acc[4];
  tile_product(E, Y, l, bi, bj, acc);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = bi * PT + tx, j = bj * PT + ty + 8 * u;
    if (i < l && j < l) {
      const float x = (i == j ? 1.f : 0.f) + (-0.5f * E[i + (int64_t)j * l] + acc[u]);
      Rinv[i + (int64_t)j * l] = d[i] * x;
    }
  }
  if (bi != 0 || bj != 0) return;
  // fixed-order reduction of the row partials: thread t takes rows t, t + 256, ...
  __shared__ float ps[PTHREADS], pm[PTHREADS];
  const int nt = (l + PT - 1) / PT;
  float s = 0.f, mx = 0.f;
  for (int i = threadIdx.x; i < l; i += PTHREADS)
    for (int b = 0; b < nt; ++b) {
      s += rsum[(int64_t)b * l + i];
      mx = fmaxf(mx, rmax[(int64_t)b * l + i]);
    }
  ps[threadIdx.x] = s;
  pm[threadIdx.x] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.f, m = 0.f;
    for (int t = 0; t < PTHREADS; ++t) {
      tot += ps[t];
      m = fmaxf(m, pm[t]);
    }
    const int good = (tot <= kPolarMaxE * kPolarMaxE) ? 1 : 0;     // false for NaN
    *ok = good;
    if (conv) *conv = (good && m <= conv_tol) ? 1 : 0;
  }
}

}  // namespace

size_t polar_scratch_bytes(int l) {
  const size_t nt = (size_t)(l + PT - 1) / PT;
  return (2 * (size_t)l * l + (2 * nt + 1) * l) * sizeof(float);
}

cudaError_t launch_polar_inv(const double* G, int l, float* Rinv, float* scratch, int* ok, int* conv,
                             float conv_tol, cudaStream_t st) {
  if (l < 1) return cudaErrorInvalidValue;
  const int nt = (l + PT - 1) / PT;
  float* E = scratch;
  float* Y = E + (size_t)l * l;
  float* rsum = Y + (size_t)l * l;
  float* rmax = rsum + (size_t)nt * l;
  float* d = rmax + (size_t)nt * l;
  dim3 grid((unsigned)nt, (unsigned)nt);
  polar_e_kernel<<<grid, PTHREADS, 0, st>>>(G, l, E, d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  polar_y_kernel<<<grid, PTHREADS, 0, st>>>(E, l, Y, rsum, rmax);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  polar_x_kernel<<<grid, PTHREADS, 0, st>>>(E, Y, d, l, rsum, rmax, Rinv, ok, conv, conv_tol);
  return cudaGetLastError();
}

}  // namespace sorsvd
