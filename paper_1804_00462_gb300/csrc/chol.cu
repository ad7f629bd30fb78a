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
//   factorisation, right-looking by tile column K:
//     L_KK: factored in one warp's registers (ahead of time, see below)
//     L_IK = A_IK L_KK^{-T} for I > K         (one thread per row, registers),
//       while warp 0 inverts L_KK into the diagonal tile
//     A_IJ -= L_IK L_JK^T, K < J <= I          (one warp per tile); warp 0
//       updates A_{K+1,K+1} first and factors it (look-ahead)
//   inverse Z = L^{-1}, in place, right-looking by K:
//     Z_KJ = X_KK Z_KJ (J < K), then Z_IJ -= L_IK Z_KJ and
//     Z_IK = -L_IK X_KK for I > K              (one warp per tile)
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

// 1/sqrt of a pivot: fp32, the correctly rounded intrinsic; binary64, the
// fp32 estimate refined by two Newton steps y <- y (3 - x y^2) / 2 (each
// squares the relative error: 2^-23 -> ~2^-46 -> below binary64 rounding),
// a few FMAs where a binary64 square root and division cost tens of FP64
// operations each on this GPU's FP64 rate
__device__ __forceinline__ float rsqrt_rn(float x) { return __frsqrt_rn(x); }
__device__ __forceinline__ double rsqrt_rn(double x) {
  if (!(x > 1e-36 && x < 1e36)) return 1.0 / sqrt(x);     // outside fp32's range (and NaN, <= 0)
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x, y * y, 1.5);
  y = y * fma(-0.5 * x, y * y, 1.5);
  return y;
}

// 16-byte vector of shared memory (4 fp32 or 2 binary64 values)
__device__ __forceinline__ void load_vec16(const float* p, float (&x)[4]) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  x[0] = t.x; x[1] = t.y; x[2] = t.z; x[3] = t.w;
}
__device__ __forceinline__ void load_vec16(const double* p, double (&x)[2]) {
  const double2 t = *reinterpret_cast<const double2*>(p);
  x[0] = t.x; x[1] = t.y;
}

// Cholesky factor of the 32 x 32 diagonal tile DK in one warp's registers
// (lane = row), right-looking.  Column j goes through shared memory: every
// lane stores its a_ij, and each lane then reads the pivot a_jj and the
// column below it as 16-byte broadcast vectors (a few loads per column
// where shuffles took one per entry), and updates its row by
//   a_ic -= (a_ij / a_jj) a_cj   (c > j),   then l_ij = a_ij / sqrt(a_jj).
// The scratch is the first two columns' worth of Ld (alternating, so one
// __syncwarp per column orders the stores and loads); Ld then receives L_KK
// densely (row-major, stride 32, zeros above the diagonal) and rd 1 / L_jj.
// Entries above the diagonal are updated too (selects, no divergence) and
// never read.  Returns false (in every lane) when a pivot is not safely
// positive; Ld must be 16-byte aligned.
template <typename F>
__device__ __noinline__ bool chol_tile_warp(const F* DK, F* Ld, F* rd, F thr, int lane) {
  constexpr int V = 16 / (int)sizeof(F);
  F a[TB];
#pragma unroll
  for (int c = 0; c < TB; ++c) a[c] = DK[lane * TLD + c];
  bool ok = true;
  F my_rs = (F)0;
#pragma unroll
  for (int j = 0; j < TB; ++j) {
    F* cb = Ld + (j & 1) * TB;
    cb[lane] = a[j];
    __syncwarp();
    const F d = cb[j];
    ok = ok && (d > thr);
    const F rs = rsqrt_rn(d);
    const F f = a[j] * (rs * rs);
#pragma unroll
    for (int v0 = (j + 1) / V * V; v0 < TB; v0 += V) {
      F x[V];
      load_vec16(cb + v0, x);
#pragma unroll
      for (int u = 0; u < V; ++u)
        if (v0 + u > j) a[v0 + u] -= f * x[u];
    }
    a[j] = lane == j ? d * rs : a[j] * rs;
    my_rs = lane == j ? rs : my_rs;
  }
  __syncwarp();                      // every read of the scratch is done
  rd[lane] = my_rs;
#pragma unroll
  for (int c = 0; c < TB; ++c) Ld[lane * TB + c] = c <= lane ? a[c] : (F)0;
  return ok;
}

// v <- v L^{-T} for one row v of 32 values (forward substitution with the
// dense L of stride 32 and its reciprocal diagonal rd; L read as broadcast
// vectors)
template <typename F>
__device__ __forceinline__ void trsm_row(F (&v)[TB], const F* Ld, const F* rd) {
#pragma unroll
  for (int j = 0; j < TB; ++j) {
    F s = v[j];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= v[k] * Ld[j * TB + k];
    v[j] = s * rd[j];
  }
}

// 8 x 4 block (rows r0.., columns c0..) of A B (BT: A B^T) for 32 x 32
// tiles: one warp per output tile, lane -> (r0, c0) = (8 (lane / 8),
// 4 (lane % 8)); per k the warp reads 4 distinct rows of A and 8 distinct
// columns of B, each load one conflict-free wavefront, for 32 FMAs
template <typename F, bool BT>
__device__ __forceinline__ void tile_mm84(const F* A, const F* B, int r0, int c0, F (&acc)[8][4]) {
#pragma unroll 4
  for (int k = 0; k < TB; ++k) {
    F av[8], bv[4];
#pragma unroll
    for (int u = 0; u < 8; ++u) av[u] = A[(r0 + u) * TLD + k];
#pragma unroll
    for (int v = 0; v < 4; ++v) bv[v] = BT ? B[(c0 + v) * TLD + k] : B[k * TLD + c0 + v];
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) acc[u][v] += av[u] * bv[v];
  }
}

template <typename F>
__device__ __forceinline__ void zero84(F (&acc)[8][4]) {
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = (F)0;
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
  const size_t dofs = (sizeof(F) * (size_t)ntile * TS + 15) & ~(size_t)15;
  F* Ld = reinterpret_cast<F*>(smem_raw + dofs);                     // dense L_KK, 32 x 32
  double* dscale = reinterpret_cast<double*>(Ld + TB * TB);          // D^{-1/2}, nb * 32
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
  // one warp per 32 x 32 output tile, an 8 x 4 block per lane
  const int r0 = 8 * (lane >> 3), c0 = 4 * (lane & 7);
  constexpr int NW = BT / 32;
  for (; attempt < max_try; ++attempt) {
    // equilibrated, shifted Gram in the lower tiles (factor precision);
    // padding and zero columns of T become identity rows / columns; the
    // largest off-diagonal entry (a column cosine) is recorded for conv_out.
    // Tiles in groups of GQ, their loads (2 GQ per thread) issued before any
    // is used: the Gram comes from L2, and the load is latency-bound.
    constexpr int GQ = 8;
    const F fshift = (F)shift;
    float offmax = 0.f;
    {
      int I0 = 0, J0 = 0;                          // (I, J) of tile q0
      for (int q0 = 0; q0 < ntile; q0 += GQ) {
        double gv[GQ][2];
        int Iq[GQ], Jq[GQ];
        int I = I0, J = J0;
#pragma unroll
        for (int u = 0; u < GQ; ++u) {
          Iq[u] = I;
          Jq[u] = J;
          if (++J > I) { ++I; J = 0; }
        }
        I0 = I;
        J0 = J;
#pragma unroll
        for (int u = 0; u < GQ; ++u)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int e = t + h * BT, r = e >> 5, c = e & 31;
            const int gi = Iq[u] * TB + r, gc = Jq[u] * TB + c;
            gv[u][h] = (q0 + u < ntile && gi < l && gc < l) ? G[gc + (int64_t)gi * l] : 0.0;   // symmetric: coalesced
          }
#pragma unroll
        for (int u = 0; u < GQ; ++u) {
          if (q0 + u >= ntile) break;
          F* D = T + (size_t)(q0 + u) * TS;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int e = t + h * BT, r = e >> 5, c = e & 31;
            const int gi = Iq[u] * TB + r, gc = Jq[u] * TB + c;
            const F si = dsf[gi], sc = dsf[gc];
            F v;
            if (si == (F)0 || sc == (F)0) v = (gi == gc) ? (F)1 : (F)0;
            else {
              v = (F)gv[u][h] * si * sc;
              if (gi > gc) offmax = fmaxf(offmax, fabsf((float)v));
              if (gi == gc) v += fshift;
            }
            D[r * TLD + c] = v;
          }
        }
      }
    }
    if (conv_out && attempt == 0) atomicMax(&s_offmax, __float_as_uint(offmax));
    if (t == 0) s_fail = 0;
    __syncthreads();
    // (a) for tile column 0: L_00 in one warp's registers (later diagonal
    // tiles are factored ahead, inside the previous column's update)
    if (warp == 0 && !chol_tile_warp(tile(0, 0), Ld, rdiag, thr, lane) && lane == 0) s_fail = 1;
    __syncthreads();
    // The factorisation and the in-place inverse Z = L^{-1} run together,
    // the inverse one tile column behind: its step K - 1 shares the two
    // phases of factorisation step K (see the inverse's description below).
    // Z_{I,K-1} = -L_{I,K-1} X_{K-1,K-1} replaces L_{I,K-1}, which the phase
    // that forms it still reads, so its warp holds it in registers (pend)
    // and writes it at the start of the next phase.  Pass K = nb is the
    // inverse's last step alone.
    // binary64 factors form the inverse afterwards (the held tile would not
    // fit in the registers)
    constexpr bool IL = sizeof(F) == 4;
    F pend[8][4];
    bool has_pend = false;
    int pend_i = 0, pend_j = 0;
    for (int K = 0; K <= nb && !s_fail; ++K) {
      // ---- phase (b): warp 0 inverts L_KK into the diagonal tile (lane =
      // column: X_ic = (delta_ic - sum_k L_ik X_kc) / L_ii); the last warps
      // solve the panel rows L_IK = A_IK L_KK^{-T} (a warp per tile, a row
      // per lane); the first warps write the held tiles Z_{I,K-2} and form
      // row K - 1 of Z: Z_{K-1,J} = X_{K-1,K-1} Z_{K-1,J}, J < K - 1
      if (warp == 0) {
        if (K < nb) {
          F* DK = tile(K, K);
          const F* rd = rdiag + K * TB;
          F x[TB];
#pragma unroll
          for (int i = 0; i < TB; ++i) {
            F s = (i == lane) ? (F)1 : (F)0;
#pragma unroll
            for (int k = 0; k < i; ++k) s -= Ld[i * TB + k] * x[k];
            x[i] = s * rd[i];
          }
#pragma unroll
          for (int i = 0; i < TB; ++i) DK[i * TLD + lane] = x[i];
        }
      } else {
        if (IL && has_pend) {
          F* o = tile(pend_i, pend_j) + r0 * TLD + c0;
#pragma unroll
          for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) o[u * TLD + v] = -pend[u][v];
          has_pend = false;
          __syncwarp();
        }
        // row K - 1: J = K - 2 on warp 1 (which held that tile), J < K - 2
        // on warps nb - K + 2 + J (after the holders, before the panel)
        int jj = -1;
        if (IL && K >= 2 && warp == 1) jj = K - 2;
        if (IL && K >= 3 && warp >= nb - K + 2 && warp - (nb - K + 2) < K - 2) jj = warp - (nb - K + 2);
        if (jj >= 0) {
          F acc[8][4];
          zero84(acc);
          tile_mm84<F, false>(tile(K - 1, K - 1), tile(K - 1, jj), r0, c0, acc);
          __syncwarp();                        // the warp has read the whole tile
          F* o = tile(K - 1, jj) + r0 * TLD + c0;
#pragma unroll
          for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) o[u * TLD + v] = acc[u][v];
        }
        const int pi = K + 1 + (NW - 1 - warp);   // panel tile of this warp
        if (K < nb && pi < nb) {
          const F* rd = rdiag + K * TB;
          F* xr = tile(pi, K) + lane * TLD;
          F v[TB];
#pragma unroll
          for (int c = 0; c < TB; ++c) v[c] = xr[c];
          trsm_row(v, Ld, rd);
#pragma unroll
          for (int c = 0; c < TB; ++c) xr[c] = v[c];
        }
      }
      __syncthreads();
      if (K == nb) break;
      // ---- phase (c): A_IJ -= L_IK L_JK^T for K < J <= I, a warp per tile.
      // Warp 0 takes the next diagonal tile (K+1, K+1) alone and then factors
      // it (look-ahead).  Inverse step K - 1 (K >= 1): warps 1..nb-K form
      // Z_{I,K-1} = -L_{I,K-1} X_{K-1,K-1} (I >= K, held), and the remaining
      // warps share the trailing tiles with Z_IJ -= L_{I,K-1} Z_{K-1,J}
      // (I >= K, J < K - 1).
      {
        const int nrem = nb - K - 1, ntr = nrem * (nrem + 1) / 2;
        if (warp == 0) {
          if (nrem > 0) {
            F acc[8][4];
            zero84(acc);
            const F* lk = tile(K + 1, K);
            tile_mm84<F, true>(lk, lk, r0, c0, acc);
            F* out = tile(K + 1, K + 1) + r0 * TLD + c0;
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) out[u * TLD + v] -= acc[u][v];
            __syncwarp();
            if (!chol_tile_warp(tile(K + 1, K + 1), Ld, rdiag + (K + 1) * TB, thr, lane) && lane == 0) s_fail = 1;
          }
        } else if (IL && K >= 1 && warp <= nb - K) {
          const int I = K + warp - 1;
          zero84(pend);
          tile_mm84<F, false>(tile(I, K - 1), tile(K - 1, K - 1), r0, c0, pend);
          has_pend = true;
          pend_i = I;
          pend_j = K - 1;
        } else {
          const int w0 = (IL && K >= 1) ? nb - K + 1 : 1;   // first free warp
          const int nfw = NW - w0;
          const int ntrail = ntr > 0 ? ntr - 1 : 0;
          const int nupd = (IL && K >= 2) ? (nb - K) * (K - 1) : 0;
          for (int f = warp - w0; f < ntrail + nupd; f += nfw) {
            F acc[8][4];
            zero84(acc);
            F* out;
            if (f < ntrail) {
              int bi, bj;
              tri_index(f + 1, &bi, &bj);
              tile_mm84<F, true>(tile(K + 1 + bi, K), tile(K + 1 + bj, K), r0, c0, acc);
              out = tile(K + 1 + bi, K + 1 + bj) + r0 * TLD + c0;
            } else {
              const int g = f - ntrail, I = K + g / (K - 1), J = g % (K - 1);
              tile_mm84<F, false>(tile(I, K - 1), tile(K - 1, J), r0, c0, acc);
              out = tile(I, J) + r0 * TLD + c0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) out[u * TLD + v] -= acc[u][v];
          }
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

  // Z = L^{-1} (formed in place above, right-looking: L^{-1} =
  // E_{nb-1}^{-1} ... E_0^{-1}, E_K the identity with L's block column K).
  // The diagonal tiles hold X_KK = L_KK^{-1}; step K finalises block row K,
  // Z_KJ = X_KK Z_KJ (J < K), then updates the rows below, Z_IJ -= L_IK Z_KJ
  // (J < K) and Z_IK = -L_IK X_KK, which replaces L_IK.  Step K's first part
  // runs in phase (b) of factorisation step K + 1, its second part in phase
  // (c) of step K + 1, when column K of L has served its trailing update;
  // the tiles each phase writes are read by no other warp in that phase.
  if constexpr (sizeof(F) == 8) {
    for (int K = 0; K < nb; ++K) {
      if (K > 0) {
        F acc[8][4];
        zero84(acc);
        const bool act = warp < K;
        if (act) tile_mm84<F, false>(tile(K, K), tile(K, warp), r0, c0, acc);
        __syncthreads();
        if (act) {
          F* o = tile(K, warp) + r0 * TLD + c0;
#pragma unroll
          for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) o[u * TLD + v] = acc[u][v];
        }
        __syncthreads();
      }
      const int nbelow = nb - K - 1;
      if (nbelow > 0) {
        // J < K: these tiles are read by no one in this phase
        for (int q = warp; q < nbelow * K; q += NW) {
          const int I = K + 1 + q / K, J = q % K;
          F acc[8][4];
          zero84(acc);
          tile_mm84<F, false>(tile(I, K), tile(K, J), r0, c0, acc);
          F* o = tile(I, J) + r0 * TLD + c0;
#pragma unroll
          for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) o[u * TLD + v] -= acc[u][v];
        }
        F acc[8][4];
        zero84(acc);
        // J = K: the last warps, so that the J < K tiles start on the first
        const int w2 = NW - 1 - warp;
        const bool act = w2 < nbelow;
        if (act) tile_mm84<F, false>(tile(K + 1 + w2, K), tile(K, K), r0, c0, acc);
        __syncthreads();
        if (act) {
          F* o = tile(K + 1 + w2, K) + r0 * TLD + c0;
#pragma unroll
          for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) o[u * TLD + v] = -acc[u][v];
        }
        __syncthreads();
      }
    }
  }
  // R^{-1} = D^{-1/2} Z^T: upper triangular, column-major
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

// shared memory of the blocked kernel (the lower tiles, the dense diagonal
// factor and the scale vectors); beyond 9 tile rows the in-place inverse
// would need a second round of thread slots, and the packed kernel is used
template <typename F>
size_t chol_blocked_smem(int l) {
  const int nb = (l + TB - 1) / TB;
  if (nb > BT / 64 + 1) return ~(size_t)0 >> 1;
  size_t b = (sizeof(F) * (size_t)(nb * (nb + 1) / 2) * TS + 15) & ~(size_t)15;
  return b + sizeof(F) * TB * TB + sizeof(double) * nb * TB + 2 * sizeof(F) * nb * TB;
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
