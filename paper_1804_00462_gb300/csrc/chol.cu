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
// Two kernels, both one thread block with the factor in shared memory in the
// factor precision F (binary64 or fp32):
//
// chol_inv_blocked_kernel (when its tiles fit in shared memory): the matrix
// is padded to nb x 32 with an identity block and kept as the nb(nb+1)/2
// lower 32 x 32 tiles (row stride 33: conflict-free row and column access).
//   factorisation, right-looking by tile column K, the column itself in
//   8-wide sub-panels (short dependency chains, every warp busy):
//     chol of the 8 x 8 diagonal block        (one warp, shuffles)
//     the panel rows below it times its L^{-T} (one thread per row, registers)
//     rank-8 update of the sub-panel's remaining columns (one thread per element)
//   then A_IJ -= L_IK L_JK^T, K < J <= I      (one thread per element)
//   inverse X = L^{-1}, in place:
//     X_II = L_II^{-1} for every I at once     (every warp, columns
//                                              interleaved, shuffles)
//     for I = 1..: X_IJ = -X_II sum_{K=J}^{I-1} L_IK X_KJ for all J < I
//   (the sums for block row I are all formed before any X_IJ replaces the
//   L_IJ they read.)
//
// chol_inv_kernel (largest l), the factor packed (row-major lower triangle);
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
                DeviceStatus* status, const int* done_in) {
  // an earlier kernel has already written R^{-1}
  if (done_in && *done_in) return;
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

// ---------------------------------------------------------------- blocked
constexpr int TB = 32;            // tile size
constexpr int TLD = TB + 1;       // tile row stride
constexpr int TS = TB * TLD;      // elements per tile

__device__ __forceinline__ int tid_of(int I, int J) { return I * (I + 1) / 2 + J; }
// q -> (i, j), j <= i, for q = i (i + 1) / 2 + j
__device__ __forceinline__ void tri_index(int q, int* i, int* j) {
  int b = (int)((sqrtf(8.f * q + 1.f) - 1.f) * 0.5f);
  while ((b + 1) * (b + 2) / 2 <= q) ++b;
  while (b * (b + 1) / 2 > q) --b;
  *i = b;
  *j = q - b * (b + 1) / 2;
}

constexpr int BT = 512;           // threads of the blocked kernel

constexpr int SB = 8;             // sub-panel width inside a tile column

// correctly rounded 1/sqrt (fp32 intrinsic; binary64 through sqrt and a
// division, only used by the binary64 factor)
__device__ __forceinline__ float rsqrt_rn(float x) { return __frsqrt_rn(x); }
__device__ __forceinline__ double rsqrt_rn(double x) { return 1.0 / sqrt(x); }

// L = chol of the SB x SB diagonal sub-block at (c0, c0) of tile D, lanes
// 0..SB-1 own its rows; 1 / L_jj goes to rdiag[c0 + j].  Returns false when
// a pivot is not safely positive (same answer in every lane).
template <typename F>
__device__ __forceinline__ bool chol_sub_warp(F* D, int c0, F thr, int lane, F* rdiag) {
  F* row = D + (c0 + (lane & (SB - 1))) * TLD + c0;
  for (int j = 0; j < SB; ++j) {
    const F d = D[(c0 + j) * TLD + c0 + j];
    if (!(d > thr)) return false;
    const F rs = rsqrt_rn(d);
    F lcol = 0;
    if (lane < SB && lane > j) { lcol = row[j] * rs; row[j] = lcol; }
    __syncwarp();
    if (lane == j) { row[j] = d * rs; rdiag[c0 + j] = rs; }
#pragma unroll
    for (int c = j + 1; c < SB; ++c) {
      const F lcj = __shfl_sync(0xffffffffu, lcol, c);
      if (lane < SB && lane >= c) row[c] -= lcol * lcj;
    }
    __syncwarp();
  }
  return true;
}

// x <- x L^{-T} for the SB entries of one row at x (L the SB x SB lower
// block at Lb, row stride TLD, reciprocal diagonal rd): forward substitution
// in registers
template <typename F>
__device__ __forceinline__ void trsm_sub(F* x, const F* Lb, const F* rd) {
  F v[SB];
#pragma unroll
  for (int j = 0; j < SB; ++j) v[j] = x[j];
#pragma unroll
  for (int j = 0; j < SB; ++j) {
    F s = v[j];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= v[k] * Lb[j * TLD + k];
    v[j] = s * rd[j];
  }
#pragma unroll
  for (int j = 0; j < SB; ++j) x[j] = v[j];
}

// column c of X = L^{-1} for a lower-triangular tile, one warp, lane = row:
// forward substitution with the solved entry broadcast by shuffle; the
// column is written back after the whole warp has read the tile's column
// entries it needed (the column below the diagonal is L's until then)
template <typename F>
__device__ __forceinline__ F inv_col_warp(const F* D, int c, int lane, const F* rdiag) {
  F b = (lane == c) ? (F)1 : (F)0;
  for (int i = c; i < TB; ++i) {
    const F xi = __shfl_sync(0xffffffffu, b, i) * rdiag[i];
    if (lane == i) b = xi;
    else if (lane > i) b -= D[lane * TLD + i] * xi;
  }
  return lane >= c ? b : (F)0;
}

template <typename F>
__device__ __forceinline__ void chol_inv_blocked_body(const double* __restrict__ G, int l, double shift_rel,
                                                      F* __restrict__ Rinv, DeviceStatus* status,
                                                      const int* skip_in, int* conv_out, float conv_tol,
                                                      const int* done_in) {
  // an earlier kernel has already written R^{-1} (and the convergence flag)
  if (done_in && *done_in) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nb = (l + TB - 1) / TB;
  const int ntile = nb * (nb + 1) / 2;
  F* T = reinterpret_cast<F*>(smem_raw);
  const size_t dofs = (sizeof(F) * (size_t)ntile * TS + 7) & ~(size_t)7;
  double* dscale = reinterpret_cast<double*>(smem_raw + dofs);     // D^{-1/2}, nb * 32
  F* dsf = reinterpret_cast<F*>(dscale + nb * TB);                   // the same in F
  F* rdiag = dsf + nb * TB;                                          // 1 / L_jj
  __shared__ int s_fail, s_retry;
  __shared__ unsigned s_offmax;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const F eps = sizeof(F) == 8 ? (F)2.220446049250313e-16 : (F)1.1920928955078125e-07;
  const F thr = (F)4 * eps;
  auto tile = [&](int I, int J) { return T + (size_t)tid_of(I, J) * TS; };
  // an earlier pass found the columns orthonormal: R^{-1} = I
  if (skip_in && *skip_in) {
    for (int e = t; e < l * l; e += BT) Rinv[e] = (e % l == e / l) ? (F)1 : (F)0;
    return;
  }
  if (t == 0) s_offmax = 0u;

  for (int i = t; i < nb * TB; i += BT) {
    double d = i < l ? G[i + (int64_t)i * l] : 0.0;
    dscale[i] = d > 0.0 ? 1.0 / sqrt(d) : 0.0;
    dsf[i] = (F)dscale[i];
  }
  if (t == 0) s_retry = 0;
  __syncthreads();

  double shift = shift_rel;
  const int max_try = 12;
  int attempt = 0;
  for (; attempt < max_try; ++attempt) {
    // equilibrated, shifted Gram in the lower tiles (factor precision);
    // padding and zero columns of T become identity rows / columns; the
    // largest off-diagonal entry (a column cosine) is recorded for conv_out
    const F fshift = (F)shift;
    float offmax = 0.f;
    for (int I = 0; I < nb; ++I)
      for (int J = 0; J <= I; ++J) {
        F* D = tile(I, J);
        for (int e = t; e < TB * TB; e += BT) {
          const int r = e >> 5, c = e & 31;
          const int gi = I * TB + r, gc = J * TB + c;
          const F si = dsf[gi], sc = dsf[gc];
          F v;
          if (si == (F)0 || sc == (F)0) v = (gi == gc) ? (F)1 : (F)0;
          else {
            v = (F)G[gc + (int64_t)gi * l] * si * sc;   // G symmetric: coalesced
            if (gi > gc) offmax = fmaxf(offmax, fabsf((float)v));
            if (gi == gc) v += fshift;
          }
          D[r * TLD + c] = v;
        }
      }
    if (conv_out && attempt == 0) atomicMax(&s_offmax, __float_as_uint(offmax));
    if (t == 0) s_fail = 0;
    __syncthreads();
    for (int K = 0; K < nb && !s_fail; ++K) {
      F* DK = tile(K, K);
      // tile column K in SB-wide sub-panels: factor the SB x SB diagonal
      // block, solve the rows below it (rest of tile K and tiles I > K),
      // rank-SB update of the sub-panel's remaining columns
      for (int c0 = 0; c0 < TB; c0 += SB) {
        if (warp == 0) {
          const bool ok = chol_sub_warp(DK, c0, thr, lane, rdiag + K * TB);
          if (!ok && lane == 0) s_fail = 1;
        }
        __syncthreads();
        if (s_fail) break;
        const int below = TB - c0 - SB;                 // rows of tile K under the block
        const int rows = below + TB * (nb - K - 1);
        for (int rr = t; rr < rows; rr += BT) {
          F* x = rr < below ? DK + (c0 + SB + rr) * TLD + c0
                            : tile(K + 1 + (rr - below) / TB, K) + ((rr - below) % TB) * TLD + c0;
          trsm_sub(x, DK + c0 * TLD + c0, rdiag + K * TB + c0);
        }
        __syncthreads();
        if (below > 0) {
          // columns c in [c0+SB, TB) of every panel row r (tile K: r >= c)
          const int ncol = below;
          const int total = rows * ncol;
          for (int e = t; e < total; e += BT) {
            const int rr = e / ncol, cc = e - rr * ncol;
            const int c = c0 + SB + cc;
            F* xr;
            if (rr < below) {
              const int r = c0 + SB + rr;
              if (c > r) continue;
              xr = DK + r * TLD;
            } else {
              xr = tile(K + 1 + (rr - below) / TB, K) + ((rr - below) % TB) * TLD;
            }
            const F* lc = DK + c * TLD + c0;
            F s = 0;
#pragma unroll
            for (int k = 0; k < SB; ++k) s += xr[c0 + k] * lc[k];
            xr[c] -= s;
          }
          __syncthreads();
        }
      }
      if (s_fail) break;
      // A_IJ -= L_IK L_JK^T for K < J <= I: 64 threads per tile, a 4 x 4
      // block of it each (8 row and column values per k for 16 FMAs)
      {
        const int nrem = nb - K - 1, ntr = nrem * (nrem + 1) / 2;
        const int sub = t & 63, r0 = 4 * (sub >> 3), c0 = 4 * (sub & 7);
        for (int q = t >> 6; q < ntr; q += BT / 64) {
          int bi, bj;
          tri_index(q, &bi, &bj);
          const F* a = tile(K + 1 + bi, K) + r0 * TLD;
          const F* b = tile(K + 1 + bj, K) + c0 * TLD;
          F acc[4][4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = (F)0;
#pragma unroll 4
          for (int k = 0; k < TB; ++k) {
            F av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) { av[u] = a[u * TLD + k]; bv[u] = b[u * TLD + k]; }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
          }
          F* out = tile(K + 1 + bi, K + 1 + bj) + r0 * TLD + c0;
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) out[u * TLD + v] -= acc[u][v];
        }
      }
      __syncthreads();
    }
    if (!s_fail) break;
    __syncthreads();
    shift = fmax(shift * 16.0, 64.0 * (double)eps);
    if (t == 0) s_retry = 1;
  }
  if (attempt == max_try) {
    if (t == 0) raise_status(status, SORSVD_ERR_BREAKDOWN);
    for (int e = t; e < l * l; e += BT) Rinv[e] = (e % l == e / l) ? (F)1 : (F)0;
    return;
  }
  if (t == 0 && s_retry) atomicOr(&status->info, 1);
  if (conv_out && t == 0) *conv_out = (__uint_as_float(s_offmax) <= conv_tol && !s_retry) ? 1 : 0;

  // X_II = L_II^{-1}: warp w solves L x = e_c for the columns c = w, w + NW,
  // ... of every diagonal tile, all its columns' chains interleaved (lane =
  // row, the solved entry broadcast by shuffle); a column c starts from e_c,
  // so the steps i < c leave it zero.  Every column is read before any is
  // written back.
  {
    constexpr int NW = BT / 32;
    constexpr int CPW = (SORSVD_MAX_L + TB - 1) / TB * TB / NW;   // columns per warp, at most
    F b[CPW];
    const int ncol = nb * TB / NW;                  // this warp's columns (nb * TB is a multiple of NW)
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      const int col = warp + q * NW;
      b[q] = (q < ncol && lane == col % TB) ? (F)1 : (F)0;
    }
    for (int i = 0; i < TB; ++i) {
#pragma unroll
      for (int q = 0; q < CPW; ++q) {
        if (q < ncol) {
          const int col = warp + q * NW, I = col / TB;
          const F xi = __shfl_sync(0xffffffffu, b[q], i) * rdiag[I * TB + i];
          if (lane == i) b[q] = xi;
          else if (lane > i) b[q] -= tile(I, I)[lane * TLD + i] * xi;
        }
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < CPW; ++q) {
      if (q < ncol) {
        const int col = warp + q * NW, c = col % TB;
        tile(col / TB, col / TB)[lane * TLD + c] = lane >= c ? b[q] : (F)0;
      }
    }
  }
  __syncthreads();
  // Off-diagonal blocks one block row I at a time: X_IJ = -X_II S_IJ with
  // S_IJ = sum_{K=J}^{I-1} L_IK X_KJ for every J < I at once (block rows
  // above I are final); all S_IJ are formed before any X_IJ overwrites the
  // L_IJ they read.  64 threads per tile, a 4 x 4 block each; the I tiles
  // of a block row take ceil(I / 8) waves of the 512 threads.
  {
    constexpr int NWAVE = ((SORSVD_MAX_L + TB - 1) / TB + 7) / 8;
    const int sub = t & 63, r0 = 4 * (sub >> 3), c0 = 4 * (sub & 7), slot = t >> 6;
    for (int I = 1; I < nb; ++I) {
      F acc[NWAVE][4][4];
#pragma unroll
      for (int w = 0; w < NWAVE; ++w) {
        const int J = slot + 8 * w;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[w][u][v] = (F)0;
        if (J < I) {
          for (int K = J; K < I; ++K) {
            const F* a = tile(I, K) + r0 * TLD;          // L_IK (rows r0..)
            const F* bb = tile(K, J) + c0;               // X_KJ (X_JJ, lower, when K == J)
#pragma unroll 4
            for (int k = 0; k < TB; ++k) {
              F av[4], bv[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) { av[u] = a[u * TLD + k]; bv[u] = bb[k * TLD + u]; }
#pragma unroll
              for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[w][u][v] += av[u] * bv[v];
            }
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int w = 0; w < NWAVE; ++w) {
        const int J = slot + 8 * w;
        if (J < I) {
          F* o = tile(I, J) + r0 * TLD + c0;
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) o[u * TLD + v] = acc[w][u][v];
        }
      }
      __syncthreads();
      // X_IJ = -X_II S_IJ, X_II lower triangular (k <= row)
      const F* xi0 = tile(I, I);
#pragma unroll
      for (int w = 0; w < NWAVE; ++w) {
        const int J = slot + 8 * w;
        if (J < I) {
          const F* sm = tile(I, J) + c0;
          F x[4][4];
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) x[u][v] = (F)0;
          for (int k = 0; k < r0 + 4; ++k) {
            F av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              av[u] = k <= r0 + u ? xi0[(r0 + u) * TLD + k] : (F)0;
              bv[u] = sm[k * TLD + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) x[u][v] += av[u] * bv[v];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[w][u][v] = -x[u][v];
        }
      }
      __syncthreads();
#pragma unroll
      for (int w = 0; w < NWAVE; ++w) {
        const int J = slot + 8 * w;
        if (J < I) {
          F* o = tile(I, J) + r0 * TLD + c0;
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) o[u * TLD + v] = acc[w][u][v];
        }
      }
      __syncthreads();
    }
  }
  // R^{-1} = D^{-1/2} X^T: upper triangular, column-major
  for (int c = warp; c < l; c += BT / 32)
    for (int r = lane; r < l; r += 32) {
      F v = 0;
      if (r <= c) {
        const F sc = dsf[r] == (F)0 ? (F)1 : dsf[r];
        v = tile(c / TB, r / TB)[(c % TB) * TLD + (r % TB)] * sc;
      }
      Rinv[r + (size_t)c * l] = v;
    }
}

template <typename F>
__global__ void __launch_bounds__(BT)
chol_inv_blocked_kernel(const double* __restrict__ G, int l, double shift_rel, F* __restrict__ Rinv,
                        DeviceStatus* status, const int* skip_in, int* conv_out, float conv_tol,
                        const int* done_in) {
  chol_inv_blocked_body<F>(G, l, shift_rel, Rinv, status, skip_in, conv_out, conv_tol, done_in);
}

// one problem per block
template <typename F>
__global__ void __launch_bounds__(BT) chol_batched_kernel(const CholJob* __restrict__ jobs) {
  const CholJob& j = jobs[blockIdx.x];
  chol_inv_blocked_body<F>(j.G, j.l, j.shift, (F*)j.Rinv, j.status, nullptr, nullptr, 0.f, nullptr);
}

template <typename F>
size_t chol_blocked_smem(int l) {
  const int nb = (l + TB - 1) / TB;
  size_t b = (sizeof(F) * (size_t)(nb * (nb + 1) / 2) * TS + 7) & ~(size_t)7;
  return b + sizeof(double) * nb * TB + 2 * sizeof(F) * nb * TB;
}

constexpr size_t kCholSmemMax = 220 * 1024;

template <typename F>
size_t chol_smem(int l) {
  size_t b = sizeof(F) * ((size_t)l * (l + 1) / 2 + l + 2);
  b = (b + 7) & ~(size_t)7;
  return b + sizeof(double) * l;
}

}  // namespace

cudaError_t launch_chol_inv(const double* G, int l, double shift_rel, void* Rinv, bool f64,
                            DeviceStatus* status, cudaStream_t st, const int* skip_in, int* conv_out,
                            float conv_tol, const int* done_in) {
  if (f64) {
    size_t sb = chol_blocked_smem<double>(l);
    if (sb <= kCholSmemMax) {
      cudaError_t e = cudaFuncSetAttribute(chol_inv_blocked_kernel<double>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
      if (e != cudaSuccess) return e;
      chol_inv_blocked_kernel<double><<<1, BT, sb, st>>>(G, l, shift_rel, (double*)Rinv, status, skip_in, conv_out,
                                                         conv_tol, done_in);
      return cudaGetLastError();
    }
    // the packed kernel always factorises and reports no convergence (the
    // caller's next pass then runs)
    if (conv_out && cudaMemsetAsync(conv_out, 0, sizeof(int), st) != cudaSuccess) return cudaErrorUnknown;
    size_t sm = chol_smem<double>(l);
    cudaError_t e = cudaFuncSetAttribute(chol_inv_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    chol_inv_kernel<double><<<1, CT, sm, st>>>(G, l, shift_rel, (double*)Rinv, status, done_in);
  } else {
    size_t sb = chol_blocked_smem<float>(l);
    if (sb <= kCholSmemMax) {
      cudaError_t e = cudaFuncSetAttribute(chol_inv_blocked_kernel<float>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sb);
      if (e != cudaSuccess) return e;
      chol_inv_blocked_kernel<float><<<1, BT, sb, st>>>(G, l, shift_rel, (float*)Rinv, status, skip_in, conv_out,
                                                        conv_tol, done_in);
      return cudaGetLastError();
    }
    if (conv_out && cudaMemsetAsync(conv_out, 0, sizeof(int), st) != cudaSuccess) return cudaErrorUnknown;
    size_t sm = chol_smem<float>(l);
    cudaError_t e = cudaFuncSetAttribute(chol_inv_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    chol_inv_kernel<float><<<1, CT, sm, st>>>(G, l, shift_rel, (float*)Rinv, status, done_in);
  }
  return cudaGetLastError();
}

int chol_batched_max_l(bool f64) {
  int l = TB;
  while ((f64 ? chol_blocked_smem<double>(l + TB) : chol_blocked_smem<float>(l + TB)) <= kCholSmemMax) l += TB;
  return l;
}

cudaError_t launch_chol_batched(const CholJob* jobs, int njobs, int max_l, bool f64, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  if (max_l > chol_batched_max_l(f64)) return cudaErrorInvalidValue;
  if (f64) {
    const size_t sb = chol_blocked_smem<double>(max_l);
    cudaError_t e = cudaFuncSetAttribute(chol_batched_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sb);
    if (e != cudaSuccess) return e;
    chol_batched_kernel<double><<<njobs, BT, sb, st>>>(jobs);
  } else {
    const size_t sb = chol_blocked_smem<float>(max_l);
    cudaError_t e = cudaFuncSetAttribute(chol_batched_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sb);
    if (e != cudaSuccess) return e;
    chol_batched_kernel<float><<<njobs, BT, sb, st>>>(jobs);
  }
  return cudaGetLastError();
}

}  // namespace sorsvd
