// R^{-1} for the Cholesky QR of a tall-skinny sketch (the QR step of
// Algorithm 3: T = Q R).  With G = T^T T (binary64, l x l) this kernel forms
//   D = diag(G),  G' = D^{-1/2} G D^{-1/2} + s I,  G' = L L^T (Cholesky),
//   R^{-1} = D^{-1/2} L^{-T}
// so that Q = T R^{-1} has orthonormal columns up to the conditioning of T
// (the caller repeats the step: CholeskyQR2 / shifted CholeskyQR3).
// Equilibration by D makes the step invariant to column scaling of T; the
// shift s (relative to the unit diagonal of G') keeps a nearly rank-deficient
// Gram factorisable without changing range(Q) = range(T).  A pivot that is
// not safely positive restarts the factorisation with a larger shift
// (recorded in the status info bits); zero columns of T stay zero.
//
// One thread block; L is kept packed (row-major lower triangle) in shared
// memory in the factor precision F (binary64 or fp32):
// l <= SORSVD_MAX_L_F64 / SORSVD_MAX_L.
#include "internal.cuh"

namespace sorsvd {
namespace {

constexpr int CT = 1024;

__device__ __forceinline__ int pidx(int i, int c) { return i * (i + 1) / 2 + c; }

template <typename F>
__global__ void __launch_bounds__(CT)
chol_inv_kernel(const double* __restrict__ G, int l, double shift_rel, F* __restrict__ Rinv,
                DeviceStatus* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  F* L = reinterpret_cast<F*>(smem_raw);
  F* tmp = L + (l * (l + 1) / 2);
  const size_t dofs = (sizeof(F) * ((size_t)l * (l + 1) / 2 + l + 2) + 7) & ~(size_t)7;
  double* dscale = reinterpret_cast<double*>(smem_raw + dofs);  // D^{-1/2}
  __shared__ int s_fail;
  __shared__ int s_retry;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = CT / 32;
  const double eps = sizeof(F) == 8 ? 2.220446049250313e-16 : 1.1920928955078125e-07;

  for (int i = t; i < l; i += CT) {
    double d = G[i + (int64_t)i * l];
    dscale[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
  }
  if (t == 0) s_retry = 0;
  __syncthreads();

  double shift = shift_rel;
  const int max_try = 12;
  int attempt = 0;
  for (; attempt < max_try; ++attempt) {
    for (int e = t; e < l * (l + 1) / 2; e += CT) {
      // packed (i, c), c <= i
      int i = (int)((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
      while (i * (i + 1) / 2 > e) --i;
      while ((i + 1) * (i + 2) / 2 <= e) ++i;
      int c = e - i * (i + 1) / 2;
      double v;
      if (dscale[i] == 0.0 || dscale[c] == 0.0) v = (i == c) ? 1.0 : 0.0;   // zero column
      else v = G[i + (int64_t)c * l] * dscale[i] * dscale[c] + (i == c ? shift : 0.0);
      L[e] = (F)v;
    }
    if (t == 0) s_fail = 0;
    __syncthreads();
    for (int j = 0; j < l; ++j) {
      if (t == 0) {
        F d = L[pidx(j, j)];
        if (!(d > (F)(4.0 * eps))) s_fail = 1;
        else L[pidx(j, j)] = sqrt(d);
      }
      __syncthreads();
      if (s_fail) break;
      F piv = L[pidx(j, j)];
      for (int i = j + 1 + t; i < l; i += CT) {
        F v = L[pidx(i, j)] / piv;
        L[pidx(i, j)] = v;
        tmp[i] = v;
      }
      __syncthreads();
      // trailing update: L[i][c] -= L[i][j] L[c][j], j < c <= i
      for (int i = j + 1 + warp; i < l; i += nwarps) {
        F lij = tmp[i];
        F* row = L + pidx(i, 0);
        for (int c = j + 1 + lane; c <= i; c += 32) row[c] -= lij * tmp[c];
      }
      __syncthreads();
    }
    if (!s_fail) break;
    shift = fmax(shift * 16.0, 64.0 * eps);
    if (t == 0) s_retry = 1;
    __syncthreads();
  }
  if (attempt == max_try) {
    if (t == 0) raise_status(status, SORSVD_ERR_BREAKDOWN);
    for (int e = t; e < l * l; e += CT) Rinv[e] = (e % l == e / l) ? (F)1 : (F)0;
    return;
  }
  if (t == 0 && s_retry) atomicOr(&status->info, 1);

  // in-place inverse of the lower factor, last column first:
  // Linv[j][j] = 1/L[j][j];  Linv[i][j] = -(sum_{k=j+1}^{i} Linv[i][k] L[k][j]) / L[j][j]
  for (int j = l - 1; j >= 0; --j) {
    for (int k = j + 1 + t; k < l; k += CT) tmp[k] = L[pidx(k, j)];
    F dinv = (F)1 / L[pidx(j, j)];
    __syncthreads();
    for (int i = j + 1 + warp; i < l; i += nwarps) {
      const F* row = L + pidx(i, 0);
      F s = 0;
      for (int k = j + 1 + lane; k <= i; k += 32) s += row[k] * tmp[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) L[pidx(i, j)] = -s * dinv;
    }
    if (t == 0) L[pidx(j, j)] = dinv;
    __syncthreads();
  }
  // R^{-1} = D^{-1/2} Linv^T : upper triangular, column-major
  for (int e = t; e < l * l; e += CT) {
    int r = e % l, c = e / l;
    F v = 0;
    if (r <= c) {
      double sc = dscale[r] == 0.0 ? 1.0 : dscale[r];
      v = (F)((double)L[pidx(c, r)] * sc);
    }
    Rinv[e] = v;
  }
}

template <typename F>
size_t chol_smem(int l) {
  size_t b = sizeof(F) * ((size_t)l * (l + 1) / 2 + l + 2);
  b = (b + 7) & ~(size_t)7;
  return b + sizeof(double) * l;
}

}  // namespace

cudaError_t launch_chol_inv(const double* G, int l, double shift_rel, void* Rinv, bool f64,
                            DeviceStatus* status, cudaStream_t st) {
  if (f64) {
    size_t sm = chol_smem<double>(l);
    cudaError_t e = cudaFuncSetAttribute(chol_inv_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    chol_inv_kernel<double><<<1, CT, sm, st>>>(G, l, shift_rel, (double*)Rinv, status);
  } else {
    size_t sm = chol_smem<float>(l);
    cudaError_t e = cudaFuncSetAttribute(chol_inv_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    chol_inv_kernel<float><<<1, CT, sm, st>>>(G, l, shift_rel, (float*)Rinv, status);
  }
  return cudaGetLastError();
}

}  // namespace sorsvd
