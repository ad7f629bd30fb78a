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
// One thread block, the factor packed (row-major lower triangle) in shared
// memory in the factor precision F (binary64 or fp32);
// l <= SORSVD_MAX_L_F64 / SORSVD_MAX_L.  Both phases need one block-wide
// barrier per column:
//   factorisation, right-looking without the square roots:
//     a_ic -= a_ij a_cj / a_jj  (j < c <= i),  then l_ij = a_ij / sqrt(a_jj);
//   inverse, in place, row-oriented: with X = L^{-1} diag(L) kept unscaled
//   (unit diagonal), after row i of X is final every later row r takes
//     x_rj -= (l_ri / l_ii) x_ij  (j <= i),
//   and finally Linv_ij = x_ij / l_ii.
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
  F* P = reinterpret_cast<F*>(smem_raw);
  F* dg = P + (l * (l + 1) / 2);                                  // diagonal of L
  const size_t dofs = (sizeof(F) * ((size_t)l * (l + 1) / 2 + l + 2) + 7) & ~(size_t)7;
  double* dscale = reinterpret_cast<double*>(smem_raw + dofs);     // D^{-1/2}
  __shared__ int s_retry;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = blockDim.x >> 5;
  const int NT = blockDim.x;
  const F eps = sizeof(F) == 8 ? (F)2.220446049250313e-16 : (F)1.1920928955078125e-07;
  const F thr = (F)4 * eps;

  for (int i = t; i < l; i += NT) {
    double d = G[i + (int64_t)i * l];
    dscale[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
  }
  if (t == 0) s_retry = 0;
  __syncthreads();

  double shift = shift_rel;
  const int max_try = 12;
  int attempt = 0;
  for (; attempt < max_try; ++attempt) {
    for (int i = warp; i < l; i += nwarps) {
      const double si = dscale[i];
      F* row = P + pidx(i, 0);
      for (int c = lane; c <= i; c += 32) {
        const double sc = dscale[c];
        double v;
        if (si == 0.0 || sc == 0.0) v = (i == c) ? 1.0 : 0.0;       // zero column of T
        else v = G[i + (int64_t)c * l] * si * sc + (i == c ? shift : 0.0);
        row[c] = (F)v;
      }
    }
    __syncthreads();
    bool fail = false;
    for (int j = 0; j < l; ++j) {
      const F d = P[pidx(j, j)];          // final since the previous barrier
      if (!(d > thr)) { fail = true; break; }   // same decision in every thread
      const F rinv = (F)1 / d;
      for (int i = j + 1 + warp; i < l; i += nwarps) {
        F* row = P + pidx(i, 0);
        const F aij = row[j] * rinv;
        for (int c = j + 1 + lane; c <= i; c += 32) row[c] -= aij * P[pidx(c, j)];
      }
      __syncthreads();
    }
    if (!fail) break;
    __syncthreads();
    shift = fmax(shift * 16.0, 64.0 * (double)eps);
    if (t == 0) s_retry = 1;
  }
  if (attempt == max_try) {
    if (t == 0) raise_status(status, SORSVD_ERR_BREAKDOWN);
    for (int e = t; e < l * l; e += NT) Rinv[e] = (e % l == e / l) ? (F)1 : (F)0;
    return;
  }
  if (t == 0 && s_retry) atomicOr(&status->info, 1);

  // scale the columns: l_ij = a_ij / sqrt(a_jj); keep diag(L) aside and put
  // the unit diagonal of X in its place
  for (int j = t; j < l; j += NT) dg[j] = sqrt(P[pidx(j, j)]);
  __syncthreads();
  for (int i = warp; i < l; i += nwarps) {
    F* row = P + pidx(i, 0);
    for (int c = lane; c < i; c += 32) row[c] = row[c] / dg[c];
    if (lane == 0) row[i] = (F)1;
  }
  __syncthreads();
  // in-place inverse, row i of X final at step i
  for (int i = 0; i + 1 < l; ++i) {
    const F dinv = (F)1 / dg[i];
    const F* xi = P + pidx(i, 0);
    for (int r = i + 1 + warp; r < l; r += nwarps) {
      F* row = P + pidx(r, 0);
      const F f = row[i] * dinv;         // l_ri / l_ii, read before the row changes
      __syncwarp();
      for (int j = lane; j <= i; j += 32) row[j] = (j == i ? (F)0 : row[j]) - f * xi[j];
    }
    __syncthreads();
  }
  // R^{-1} = D^{-1/2} Linv^T : upper triangular, column-major;
  // Linv_cr = x_cr / l_cc
  for (int e = t; e < l * l; e += NT) {
    const int r = e % l, c = e / l;
    F v = 0;
    if (r <= c) {
      const double sc = dscale[r] == 0.0 ? 1.0 : dscale[r];
      v = (F)((double)(P[pidx(c, r)] / dg[c]) * sc);
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
