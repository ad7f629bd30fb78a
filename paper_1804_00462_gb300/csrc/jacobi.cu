// Truncated SVD of the small core matrix M (l x l) of Algorithm 3
// ("compute the rank-k truncated SVD of M").  One-sided (Hestenes) Jacobi:
// columns w_p, w_q of W = M V are rotated until every pair is orthogonal to
// a relative tolerance, the same rotations accumulating V; then
// sigma_j = ||M v_j|| and u_j = M v_j / sigma_j.
//
// Three kernels:
//  1. sweeps (one block): W and V in shared memory when 2 l^2 words fit,
//     else in the caller's work buffer; round-robin pair schedule (see the
//     kernel).  Rotations are applied while a pair's cosine exceeds l * eps
//     of the sweep precision.  The sweep count is capped; hitting the cap
//     with a cosine above 32 l eps raises SORSVD_ERR_NOT_CONVERGED.
//     fp32 sweeps of l >= 48 run block-cyclic on a 16-CTA cluster; binary64
//     sweeps are preceded by fp32 sweeps and polish their result
//     (jacobi_f64_mixed).
//  2. finish (one block per column), binary64: v_j normalised (fp32
//     rotations keep its norm only to a few ulps each), z = M v_j,
//     sigma_j = ||z||, u_j = z / sigma_j.  V stays orthonormal to the sweep precision whatever
//     the grading of M, so the rank-k result M V_k V_k^T is as accurate as
//     the subspace of V_k; sigma_j is a Rayleigh quotient of M^T M (error
//     quadratic in the error of v_j).  (Recovering v_j = M^T u_j / sigma_j
//     from the rotated W instead multiplies the sweep's rounding in u_j by
//     sigma_1 / sigma_j: with fp32 sweeps on a matrix graded like i^-2 the
//     factors lost orthogonality at the 1e-2 level.)
//  3. order (one block): sigma descending (ties by column index); sign: the
//     largest-magnitude entry of each column of U~ is made positive and the
//     matching column of V~ follows.
#include "internal.cuh"

#include <cooperative_groups.h>

#include <algorithm>
#include <cstdlib>

namespace sorsvd {
namespace {

constexpr int kMaxSweeps = 30;
// sweep cap of the next launches on this device (1..kMaxSweeps; a test
// lowers it to make SORSVD_ERR_NOT_CONVERGED happen)
__device__ int g_sweep_cap = kMaxSweeps;
__device__ __forceinline__ int sweep_cap() { return min(max(g_sweep_cap, 1), kMaxSweeps); }

__device__ __forceinline__ int rr_player(int pos, int round, int N) {
  // position 0 is fixed; positions 1..N-1 rotate by one place per round
  if (pos == 0) return 0;
  int x = (pos - 1 - round) % (N - 1);
  if (x < 0) x += N - 1;
  return 1 + x;
}

// Jacobi rotation (c, s) that orthogonalises two columns with squared norms
// al, be and inner product ga: t = sign(z) / (|z| + sqrt(1 + z^2)),
// z = (be - al) / (2 ga), c = 1 / sqrt(1 + t^2), s = c t.  For |z| beyond
// 1e18 (fp32) 1 + z^2 overflows, t becomes 0 and the pair is left as is.
__device__ __forceinline__ void rotation(float al, float be, float ga, float* c, float* s) {
  const float z = __fdividef(be - al, 2.f * ga);
  const float az = fabsf(z);
  const float t = copysignf(__fdividef(1.f, az + sqrtf(fmaf(az, az, 1.f))), z);
  const float cs = rsqrtf(fmaf(t, t, 1.f));
  *c = cs;
  *s = cs * t;
}
// Binary64 rotation: the tangent t to binary32 accuracy (enough for the
// angle: a relative error e in t leaves e times the original off-diagonal
// term, and the sweeps repeat until every term is below tolerance), the
// rotation itself orthogonal to binary64 accuracy: c = (1 + t^2)^{-1/2} by
// two Newton steps x <- x (3 - w x^2) / 2 from the binary32 estimate (each
// step squares the relative error), s = c t.  One binary64 division instead
// of three divisions and three square roots, all slow at the FP64 rate.
// For |z| > 1e8, t = 1 / (2 z) in binary64 (relative error below 1e-16
// there): a binary32 t would underflow for the columns of a null space,
// whose rotations against columns 1e30 larger still matter to them.
__device__ __forceinline__ void rotation(double al, double be, double ga, double* c, double* s) {
  const double z = (be - al) / (2.0 * ga);
  double t;
  if (fabs(z) > 1e8) {
    t = 0.5 / z;
  } else {
    const float az = (float)fabs(z);
    t = (double)copysignf(1.f / (az + sqrtf(fmaf(az, az, 1.f))), (float)z);
  }
  const double w = fma(t, t, 1.0);
  double x = (double)rsqrtf((float)w);
  x = x * fma(-0.5 * w, x * x, 1.5);
  x = x * fma(-0.5 * w, x * x, 1.5);
  *c = x;
  *s = x * t;
}

template <typename J>
__device__ __forceinline__ J group8_sum(J v, unsigned mask) {
  v += __shfl_xor_sync(mask, v, 4);
  v += __shfl_xor_sync(mask, v, 2);
  v += __shfl_xor_sync(mask, v, 1);
  return v;
}

// Sweep kernel.  Pairs follow the round-robin tournament (circle method):
// in each of the N - 1 rounds of a sweep (N = l rounded up to even) the N/2
// disjoint pairs are rotated concurrently, one 8-lane group per pair, which
// keeps the pair's two W columns in registers between the inner products and
// the update; the same rotation is applied to the two V columns.  One
// barrier separates rounds.  EPL: elements per lane (>= l/8).  W (l x l) and
// V (l x l) sit in shared memory (IN_SMEM) or in gwork; V is written to Vout.
template <typename J, bool IN_SMEM, int EPL>
__device__ __forceinline__ void jacobi_sweep_body(const double* __restrict__ Min, int l, J* __restrict__ Vout,
                                                  J* __restrict__ gwork, DeviceStatus* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_rot, s_big;
  J* W = IN_SMEM ? reinterpret_cast<J*>(smem_raw) : gwork;
  J* V = W + (size_t)l * l;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int grp = lane >> 3, gl = lane & 7;
  const int ngroups = (blockDim.x >> 5) * 4;
  const unsigned gmask = 0xFFu << (grp * 8);
  const J eps = sizeof(J) == 8 ? (J)2.220446049250313e-16 : (J)1.1920928955078125e-07;
  const J tol = (J)l * eps, tol2 = tol * tol;
  const J big = (J)32 * tol, big2 = big * big;

  for (int e = t; e < l * l; e += blockDim.x) {
    W[e] = (J)Min[e];
    V[e] = (e % l == e / l) ? (J)1 : (J)0;
  }
  __syncthreads();

  const int N = (l + 1) & ~1;
  int sweep;
  const int cap = sweep_cap();
  for (sweep = 1; sweep <= cap; ++sweep) {
    if (t == 0) { s_rot = 0; s_big = 0; }
    __syncthreads();
    int rot_local = 0, big_local = 0;
    for (int r = 0; r < N - 1; ++r) {
      for (int pr = warp * 4 + grp; pr < N / 2; pr += ngroups) {
        const int a = rr_player(pr, r, N), b = rr_player(N - 1 - pr, r, N);
        if (a >= l || b >= l) continue;                // bye (whole group)
        const size_t oa = (size_t)min(a, b) * l, ob = (size_t)max(a, b) * l;
        J* wp = W + oa;
        J* wq = W + ob;
        J x[EPL], y[EPL];
        J al = 0, be = 0, ga = 0;
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int i = gl + 8 * e;
          x[e] = (i < l) ? wp[i] : (J)0;
          y[e] = (i < l) ? wq[i] : (J)0;
          al += x[e] * x[e]; be += y[e] * y[e]; ga += x[e] * y[e];
        }
        // xor butterflies leave bitwise-identical sums in all 8 lanes, so the
        // group takes one decision and one rotation
        al = group8_sum(al, gmask); be = group8_sum(be, gmask); ga = group8_sum(ga, gmask);
        if (!(ga * ga > tol2 * al * be)) continue;
        if (ga * ga > big2 * al * be) big_local = 1;
        J cs, sn;
        rotation(al, be, ga, &cs, &sn);
        J* vp = V + oa;
        J* vq = V + ob;
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
          const int i = gl + 8 * e;
          if (i < l) {
            wp[i] = cs * x[e] - sn * y[e];
            wq[i] = sn * x[e] + cs * y[e];
            const J u = vp[i], v = vq[i];
            vp[i] = cs * u - sn * v;
            vq[i] = sn * u + cs * v;
          }
        }
        rot_local = 1;
      }
      __syncthreads();
    }
    if (rot_local) s_rot = 1;
    if (big_local) s_big = 1;
    __syncthreads();
    const int rot = s_rot, bg = s_big;
    __syncthreads();
    if (!rot) break;
    if (sweep == cap) {
      if (bg && t == 0) raise_status(status, SORSVD_ERR_NOT_CONVERGED);
      break;
    }
  }
  if (t == 0) atomicOr(&status->info, (min(sweep, cap)) << 8);
  for (int e = t; e < l * l; e += blockDim.x) Vout[e] = V[e];
}

// fp32 sweeps with packed pairs: W and V columns are zero-padded to
// ldw = 16 EP rows, lane gl of a pair's 8-lane group holds the element
// pairs (2 (gl + 8 e), +1), e < EP, so the loops need no bounds tests, and
// the inner products and the rotation run as paired fp32 operations
// (__ffma2_rn / __fmul2_rn: two lanes of fp32 FMA per instruction, same
// rounding as two fma calls).  Same pair schedule, tolerance and cap as the
// generic body.
template <int EP>
__device__ __forceinline__ void jacobi_sweep_body_f2(const double* __restrict__ Min, int l, float* __restrict__ Vout,
                                                     DeviceStatus* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_rot, s_big;
  const int ldw = 16 * EP;
  float* W = reinterpret_cast<float*>(smem_raw);
  float* V = W + (size_t)ldw * l;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int grp = lane >> 3, gl = lane & 7;
  const int ngroups = (blockDim.x >> 5) * 4;
  const unsigned gmask = 0xFFu << (grp * 8);
  const float eps = 1.1920928955078125e-07f;
  const float tol = (float)l * eps, tol2 = tol * tol;
  const float big = 32.f * tol, big2 = big * big;

  for (int e = t; e < ldw * l; e += blockDim.x) {
    const int c = e / ldw, i = e - c * ldw;
    W[e] = i < l ? (float)Min[i + (size_t)c * l] : 0.f;
    V[e] = (i == c) ? 1.f : 0.f;
  }
  __syncthreads();

  const int N = (l + 1) & ~1;
  int sweep;
  const int cap = sweep_cap();
  for (sweep = 1; sweep <= cap; ++sweep) {
    if (t == 0) { s_rot = 0; s_big = 0; }
    __syncthreads();
    int rot_local = 0, big_local = 0;
    for (int r = 0; r < N - 1; ++r) {
      for (int pr = warp * 4 + grp; pr < N / 2; pr += ngroups) {
        const int a = rr_player(pr, r, N), b = rr_player(N - 1 - pr, r, N);
        if (a >= l || b >= l) continue;                // bye (whole group)
        const size_t oa = (size_t)min(a, b) * ldw, ob = (size_t)max(a, b) * ldw;
        float2* wp = reinterpret_cast<float2*>(W + oa);
        float2* wq = reinterpret_cast<float2*>(W + ob);
        float2 x[EP], y[EP];
        float2 al2 = make_float2(0.f, 0.f), be2 = al2, ga2 = al2;
#pragma unroll
        for (int e = 0; e < EP; ++e) {
          x[e] = wp[gl + 8 * e];
          y[e] = wq[gl + 8 * e];
          al2 = __ffma2_rn(x[e], x[e], al2);
          be2 = __ffma2_rn(y[e], y[e], be2);
          ga2 = __ffma2_rn(x[e], y[e], ga2);
        }
        float al = al2.x + al2.y, be = be2.x + be2.y, ga = ga2.x + ga2.y;
        al = group8_sum(al, gmask); be = group8_sum(be, gmask); ga = group8_sum(ga, gmask);
        if (!(ga * ga > tol2 * al * be)) continue;
        if (ga * ga > big2 * al * be) big_local = 1;
        float cs, sn;
        rotation(al, be, ga, &cs, &sn);
        const float2 c2 = make_float2(cs, cs), s2 = make_float2(sn, sn), ns2 = make_float2(-sn, -sn);
        float2* vp = reinterpret_cast<float2*>(V + oa);
        float2* vq = reinterpret_cast<float2*>(V + ob);
#pragma unroll
        for (int e = 0; e < EP; ++e) {
          const int i = gl + 8 * e;
          wp[i] = __ffma2_rn(c2, x[e], __fmul2_rn(ns2, y[e]));
          wq[i] = __ffma2_rn(s2, x[e], __fmul2_rn(c2, y[e]));
          const float2 u = vp[i], v = vq[i];
          vp[i] = __ffma2_rn(c2, u, __fmul2_rn(ns2, v));
          vq[i] = __ffma2_rn(s2, u, __fmul2_rn(c2, v));
        }
        rot_local = 1;
      }
      __syncthreads();
    }
    if (rot_local) s_rot = 1;
    if (big_local) s_big = 1;
    __syncthreads();
    const int rot = s_rot, bg = s_big;
    __syncthreads();
    if (!rot) break;
    if (sweep == cap) {
      if (bg && t == 0) raise_status(status, SORSVD_ERR_NOT_CONVERGED);
      break;
    }
  }
  if (t == 0) atomicOr(&status->info, (min(sweep, cap)) << 8);
  for (int e = t; e < l * l; e += blockDim.x) {
    const int c = e / l, i = e - c * l;
    Vout[e] = V[i + (size_t)c * ldw];
  }
}

// The same sweep with G-lane groups (G = 16; measured 13 % faster per sweep
// than 8 lanes at l = 110, 4 lanes was 30 % slower): lane gl of a pair's group
// holds the element pairs (2 (gl + G e), +1), e < EP (ldw = 2 G EP rows);
// the round-robin pairs come from a table built once in shared memory
// (pairs[r * N/2 + pr] = a | b << 16, a < b).
template <int G, int EP>
__device__ __forceinline__ void jacobi_sweep_body_g(const double* __restrict__ Min, int l, float* __restrict__ Vout,
                                                    DeviceStatus* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_rot, s_big;
  const int ldw = 2 * G * EP;
  float* W = reinterpret_cast<float*>(smem_raw);
  float* V = W + (size_t)ldw * l;
  const int N = (l + 1) & ~1;
  uint32_t* pairs = reinterpret_cast<uint32_t*>(V + (size_t)ldw * l);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int GPW = 32 / G;                   // groups per warp
  const int grp = lane / G, gl = lane % G;
  const int ngroups = (blockDim.x >> 5) * GPW;
  const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (grp * G));
  const float eps = 1.1920928955078125e-07f;
  const float tol = (float)l * eps, tol2 = tol * tol;
  const float big = 32.f * tol, big2 = big * big;

  for (int e = t; e < ldw * l; e += blockDim.x) {
    const int c = e / ldw, i = e - c * ldw;
    W[e] = i < l ? (float)Min[i + (size_t)c * l] : 0.f;
    V[e] = (i == c) ? 1.f : 0.f;
  }
  for (int e = t; e < (N - 1) * (N / 2); e += blockDim.x) {
    const int r = e / (N / 2), pr = e - r * (N / 2);
    const int a = rr_player(pr, r, N), b = rr_player(N - 1 - pr, r, N);
    pairs[e] = (uint32_t)min(a, b) | ((uint32_t)max(a, b) << 16);
  }
  __syncthreads();

  int sweep;
  const int cap = sweep_cap();
  for (sweep = 1; sweep <= cap; ++sweep) {
    if (t == 0) { s_rot = 0; s_big = 0; }
    __syncthreads();
    int rot_local = 0, big_local = 0;
    for (int r = 0; r < N - 1; ++r) {
      for (int pr = warp * GPW + grp; pr < N / 2; pr += ngroups) {
        const uint32_t ab = pairs[r * (N / 2) + pr];
        const int a = (int)(ab & 0xFFFFu), b = (int)(ab >> 16);
        if (b >= l) continue;                          // bye (whole group)
        float2* wp = reinterpret_cast<float2*>(W + (size_t)a * ldw);
        float2* wq = reinterpret_cast<float2*>(W + (size_t)b * ldw);
        float2 x[EP], y[EP];
        float2 al2 = make_float2(0.f, 0.f), be2 = al2, ga2 = al2;
#pragma unroll
        for (int e = 0; e < EP; ++e) {
          x[e] = wp[gl + G * e];
          y[e] = wq[gl + G * e];
          al2 = __ffma2_rn(x[e], x[e], al2);
          be2 = __ffma2_rn(y[e], y[e], be2);
          ga2 = __ffma2_rn(x[e], y[e], ga2);
        }
        float al = al2.x + al2.y, be = be2.x + be2.y, ga = ga2.x + ga2.y;
        // xor butterflies: bitwise-identical sums in every lane of the group
#pragma unroll
        for (int o = G / 2; o > 0; o >>= 1) {
          al += __shfl_xor_sync(gmask, al, o);
          be += __shfl_xor_sync(gmask, be, o);
          ga += __shfl_xor_sync(gmask, ga, o);
        }
        if (!(ga * ga > tol2 * al * be)) continue;
        if (ga * ga > big2 * al * be) big_local = 1;
        float cs, sn;
        rotation(al, be, ga, &cs, &sn);
        const float2 c2 = make_float2(cs, cs), s2 = make_float2(sn, sn), ns2 = make_float2(-sn, -sn);
        float2* vp = reinterpret_cast<float2*>(V + (size_t)a * ldw);
        float2* vq = reinterpret_cast<float2*>(V + (size_t)b * ldw);
#pragma unroll
        for (int e = 0; e < EP; ++e) {
          const int i = gl + G * e;
          wp[i] = __ffma2_rn(c2, x[e], __fmul2_rn(ns2, y[e]));
          wq[i] = __ffma2_rn(s2, x[e], __fmul2_rn(c2, y[e]));
          const float2 u = vp[i], v = vq[i];
          vp[i] = __ffma2_rn(c2, u, __fmul2_rn(ns2, v));
          vq[i] = __ffma2_rn(s2, u, __fmul2_rn(c2, v));
        }
        rot_local = 1;
      }
      __syncthreads();
    }
    if (rot_local) s_rot = 1;
    if (big_local) s_big = 1;
    __syncthreads();
    const int rot = s_rot, bg = s_big;
    __syncthreads();
    if (!rot) break;
    if (sweep == cap) {
      if (bg && t == 0) raise_status(status, SORSVD_ERR_NOT_CONVERGED);
      break;
    }
  }
  if (t == 0) atomicOr(&status->info, (min(sweep, cap)) << 8);
  for (int e = t; e < l * l; e += blockDim.x) {
    const int c = e / l, i = e - c * l;
    Vout[e] = V[i + (size_t)c * ldw];
  }
}

template <int G, int EP>
__global__ void __launch_bounds__(1024)
jacobi_sweep_g_kernel(const double* __restrict__ Min, int l, float* __restrict__ Vout, DeviceStatus* status) {
  jacobi_sweep_body_g<G, EP>(Min, l, Vout, status);
}

// Large l (W and V do not fit one SM's shared memory): the same sweep as
// one cooperative grid, W and V in global memory (they stay in L2), 16-lane
// groups, kCoopPairsPerCta pairs per CTA, one grid-wide barrier per round.
// The "any rotation" / "large cosine" flags of sweep s live in
// flags[2 s], flags[2 s + 1] (zeroed by the launcher), so no flag is
// reused within the kernel.
constexpr int kCoopPairsPerCta = 8;
constexpr int kCoopThreads = kCoopPairsPerCta * 16;

template <int EP>
__global__ void __launch_bounds__(kCoopThreads)
jacobi_sweep_coop_kernel(const double* __restrict__ Min, int l, int ldw, float* __restrict__ W, float* __restrict__ V,
                         float* __restrict__ Vout, int* __restrict__ flags, DeviceStatus* status) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  const int t = threadIdx.x, lane = t & 31;
  const int grp = t >> 4, gl = lane & 15;
  const unsigned gmask = 0xFFFFu << ((lane >> 4) * 16);
  const float eps = 1.1920928955078125e-07f;
  const float tol = (float)l * eps, tol2 = tol * tol;
  const float big = 32.f * tol, big2 = big * big;
  const int64_t gt = (int64_t)blockIdx.x * blockDim.x + t, gn = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = gt; e < (int64_t)ldw * l; e += gn) {
    const int c = (int)(e / ldw), i = (int)(e - (int64_t)c * ldw);
    W[e] = i < l ? (float)Min[i + (size_t)c * l] : 0.f;
    V[e] = (i == c) ? 1.f : 0.f;
  }
  grid.sync();
  const int N = (l + 1) & ~1;
  const int pr_base = blockIdx.x * kCoopPairsPerCta + grp;
  int sweep;
  const int cap = sweep_cap();
  for (sweep = 1; sweep <= cap; ++sweep) {
    int rot_local = 0, big_local = 0;
    for (int r = 0; r < N - 1; ++r) {
      for (int pr = pr_base; pr < N / 2; pr += gridDim.x * kCoopPairsPerCta) {
        const int a0 = rr_player(pr, r, N), b0 = rr_player(N - 1 - pr, r, N);
        const int a = min(a0, b0), b = max(a0, b0);
        if (b >= l) continue;                          // bye (whole group)
        float2* wp = reinterpret_cast<float2*>(W + (size_t)a * ldw);
        float2* wq = reinterpret_cast<float2*>(W + (size_t)b * ldw);
        float2 x[EP], y[EP];
        float2 al2 = make_float2(0.f, 0.f), be2 = al2, ga2 = al2;
#pragma unroll
        for (int e = 0; e < EP; ++e) {
          x[e] = wp[gl + 16 * e];
          y[e] = wq[gl + 16 * e];
          al2 = __ffma2_rn(x[e], x[e], al2);
          be2 = __ffma2_rn(y[e], y[e], be2);
          ga2 = __ffma2_rn(x[e], y[e], ga2);
        }
        float al = al2.x + al2.y, be = be2.x + be2.y, ga = ga2.x + ga2.y;
#pragma unroll
        for (int o = 8; o > 0; o >>= 1) {
          al += __shfl_xor_sync(gmask, al, o);
          be += __shfl_xor_sync(gmask, be, o);
          ga += __shfl_xor_sync(gmask, ga, o);
        }
        if (!(ga * ga > tol2 * al * be)) continue;
        if (ga * ga > big2 * al * be) big_local = 1;
        float cs, sn;
        rotation(al, be, ga, &cs, &sn);
        const float2 c2 = make_float2(cs, cs), s2 = make_float2(sn, sn), ns2 = make_float2(-sn, -sn);
        float2* vp = reinterpret_cast<float2*>(V + (size_t)a * ldw);
        float2* vq = reinterpret_cast<float2*>(V + (size_t)b * ldw);
#pragma unroll
        for (int e = 0; e < EP; ++e) {
          const int i = gl + 16 * e;
          wp[i] = __ffma2_rn(c2, x[e], __fmul2_rn(ns2, y[e]));
          wq[i] = __ffma2_rn(s2, x[e], __fmul2_rn(c2, y[e]));
          const float2 u = vp[i], v = vq[i];
          vp[i] = __ffma2_rn(c2, u, __fmul2_rn(ns2, v));
          vq[i] = __ffma2_rn(s2, u, __fmul2_rn(c2, v));
        }
        rot_local = 1;
      }
      grid.sync();                                     // the round's columns are final
    }
    if (rot_local) atomicOr(&flags[2 * sweep], 1);
    if (big_local) atomicOr(&flags[2 * sweep + 1], 1);
    grid.sync();
    const int rot = *((volatile int*)&flags[2 * sweep]), bg = *((volatile int*)&flags[2 * sweep + 1]);
    if (!rot) break;
    if (sweep == cap) {
      if (bg && gt == 0) raise_status(status, SORSVD_ERR_NOT_CONVERGED);
      break;
    }
  }
  if (gt == 0) atomicOr(&status->info, (min(sweep, cap)) << 8);
  for (int64_t e = gt; e < (int64_t)l * l; e += gn) {
    const int c = (int)(e / l), i = (int)(e - (int64_t)c * l);
    Vout[e] = V[i + (size_t)c * ldw];
  }
}

template <int EP>
__global__ void __launch_bounds__(512)
jacobi_sweep_f2_kernel(const double* __restrict__ Min, int l, float* __restrict__ Vout, DeviceStatus* status) {
  jacobi_sweep_body_f2<EP>(Min, l, Vout, status);
}

template <typename J, bool IN_SMEM, int EPL, int NT>
__global__ void __launch_bounds__(NT)
jacobi_sweep_kernel(const double* __restrict__ Min, int l, J* __restrict__ Vout, J* __restrict__ gwork,
                    DeviceStatus* status) {
  jacobi_sweep_body<J, IN_SMEM, EPL>(Min, l, Vout, gwork, status);
}

template <typename J>
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0;
  for (int w = 0; w < nw; ++w) s += red[w];
  return s;
}

// ---------------------------------------------------------------- cluster
// Sweeps on a thread-block cluster of kClusterCtas CTAs (one per SM): the
// columns move between the CTAs' shared memory by asynchronous stores that
// the receiving CTA's mbarrier counts, with no cluster-wide barrier per
// exchange.  A CTA can run at most one exchange ahead of a neighbour (it
// needs that neighbour's columns), so with two buffers no column is
// overwritten before it has been read.  The convergence flags of a sweep
// are OR-ed into CTA 0 and read back by all CTAs before any of them
// decides, so every CTA runs the same barriers.  The ordering (blocks of
// columns, local rounds between exchanges) is described at the kernel.
constexpr int kClusterCtas = 16;
constexpr int kClusterMinL = 48;                 // below: the one-block sweeps

__device__ __forceinline__ int next_pos(int p, int N) { return p == 0 ? 0 : (p == N - 1 ? 1 : p + 1); }
__device__ __forceinline__ int prev_pos(int q, int N) { return q == 0 ? 0 : (q == 1 ? N - 1 : q - 1); }

__device__ __forceinline__ uint32_t cl_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// shared::cluster address of the same variable in CTA `rank`
__device__ __forceinline__ uint32_t cl_mapa(uint32_t a, int rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
// 8-byte store into another CTA's shared memory that reports its bytes to
// that CTA's mbarrier when they land
__device__ __forceinline__ void cl_st_async(uint32_t addr, float2 v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];" ::"r"(addr),
               "f"(v.x), "f"(v.y), "r"(mbar)
               : "memory");
}
__device__ __forceinline__ void cl_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(cl_smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void cl_mbar_arm(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cl_smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool cl_mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
      " selp.b32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(cl_smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
constexpr long long kClusterWaitCycles = 4000000000ll;   // about 2 s

// Block-cyclic sweeps on the 16-CTA cluster.  The l columns (padded with
// zero columns) form NB = 32 blocks of b = ceil(l / 32); CTA c holds the
// blocks at positions c (slot 0) and NB - 1 - c (slot 1).  A sweep is
// NB - 1 block rounds of the round-robin over blocks (position 0 fixed,
// the others move one place per round).  In a block round a CTA rotates
// every pair (x of slot 0, y of slot 1) in b local rounds of b disjoint pairs
// (x_i, y_{(i + s) mod b}), and in the first block round of a sweep also the
// pairs inside each of its two blocks (round-robin, b' - 1 local rounds of
// b' / 2 pairs per block, b' = b rounded up to even): every pair of columns
// once per sweep.  Local rounds touch only this CTA's shared memory (one
// __syncthreads each); the blocks then move to their next positions,
// neighbouring CTAs by st.async counted by the receiver's mbarrier - one
// exchange per b^2 pairs, where the column-cyclic kernel exchanges after
// every pair.  Convergence flags per sweep as in that kernel.
constexpr int kBlockNb = 2 * kClusterCtas;

__device__ __forceinline__ void cl_st_async4(uint32_t addr, float4 v, uint32_t mbar) {
  asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.f32 [%0], {%1, %2, %3, %4}, [%5];" ::"r"(addr),
               "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "r"(mbar)
               : "memory");
}

// One Jacobi rotation of columns (x, y) of W and (u, v) of V (V at column +
// LDW), 16 lanes, in place.  Returns the lanes' flags: bit 0 rotated, bit 1
// a large rotation (cosine above 32 tol).
template <int EP>
__device__ __forceinline__ int rotate_pair16(float* cx, float* cy, int gl, unsigned gmask, float tol2, float big2) {
  constexpr int LDW = 32 * EP;
  float2* wx = reinterpret_cast<float2*>(cx);
  float2* wy = reinterpret_cast<float2*>(cy);
  float2* vx = reinterpret_cast<float2*>(cx + LDW);
  float2* vy = reinterpret_cast<float2*>(cy + LDW);
  float2 x[EP], y[EP], u[EP], v[EP];
  float2 al2 = make_float2(0.f, 0.f), be2 = al2, ga2 = al2;
#pragma unroll
  for (int e = 0; e < EP; ++e) {
    x[e] = wx[gl + 16 * e];
    y[e] = wy[gl + 16 * e];
    al2 = __ffma2_rn(x[e], x[e], al2);
    be2 = __ffma2_rn(y[e], y[e], be2);
    ga2 = __ffma2_rn(x[e], y[e], ga2);
  }
  float al = al2.x + al2.y, be = be2.x + be2.y, ga = ga2.x + ga2.y;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    al += __shfl_xor_sync(gmask, al, o);
    be += __shfl_xor_sync(gmask, be, o);
    ga += __shfl_xor_sync(gmask, ga, o);
  }
  if (!(ga * ga > tol2 * al * be)) return 0;
  const int flags = (ga * ga > big2 * al * be) ? 3 : 1;
  float cs, sn;
  rotation(al, be, ga, &cs, &sn);
  const float2 c2 = make_float2(cs, cs), s2 = make_float2(sn, sn), ns2 = make_float2(-sn, -sn);
#pragma unroll
  for (int e = 0; e < EP; ++e) {
    u[e] = vx[gl + 16 * e];
    v[e] = vy[gl + 16 * e];
  }
#pragma unroll
  for (int e = 0; e < EP; ++e) {
    wx[gl + 16 * e] = __ffma2_rn(c2, x[e], __fmul2_rn(ns2, y[e]));
    wy[gl + 16 * e] = __ffma2_rn(s2, x[e], __fmul2_rn(c2, y[e]));
    vx[gl + 16 * e] = __ffma2_rn(c2, u[e], __fmul2_rn(ns2, v[e]));
    vy[gl + 16 * e] = __ffma2_rn(s2, u[e], __fmul2_rn(c2, v[e]));
  }
  return flags;
}

// The same rotation with column x (W) and its V column u held in the
// lanes' registers (the group keeps them through every cross round of a
// block round); column y and its V column come from shared memory.
template <int EP>
__device__ __forceinline__ int rotate_xreg16(float2 (&x)[EP], float2 (&u)[EP], float* cy, int gl, unsigned gmask,
                                             float tol2, float big2) {
  constexpr int LDW = 32 * EP;
  float2* wy = reinterpret_cast<float2*>(cy);
  float2* vy = reinterpret_cast<float2*>(cy + LDW);
  float2 y[EP], v[EP];
  float2 al2 = make_float2(0.f, 0.f), be2 = al2, ga2 = al2;
#pragma unroll
  for (int e = 0; e < EP; ++e) {
    y[e] = wy[gl + 16 * e];
    al2 = __ffma2_rn(x[e], x[e], al2);
    be2 = __ffma2_rn(y[e], y[e], be2);
    ga2 = __ffma2_rn(x[e], y[e], ga2);
  }
  float al = al2.x + al2.y, be = be2.x + be2.y, ga = ga2.x + ga2.y;
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) {
    al += __shfl_xor_sync(gmask, al, o);
    be += __shfl_xor_sync(gmask, be, o);
    ga += __shfl_xor_sync(gmask, ga, o);
  }
  if (!(ga * ga > tol2 * al * be)) return 0;
  const int flags = (ga * ga > big2 * al * be) ? 3 : 1;
  float cs, sn;
  rotation(al, be, ga, &cs, &sn);
  const float2 c2 = make_float2(cs, cs), s2 = make_float2(sn, sn), ns2 = make_float2(-sn, -sn);
#pragma unroll
  for (int e = 0; e < EP; ++e) v[e] = vy[gl + 16 * e];
#pragma unroll
  for (int e = 0; e < EP; ++e) {
    const float2 xn = __ffma2_rn(c2, x[e], __fmul2_rn(ns2, y[e]));
    wy[gl + 16 * e] = __ffma2_rn(s2, x[e], __fmul2_rn(c2, y[e]));
    x[e] = xn;
    const float2 un = __ffma2_rn(c2, u[e], __fmul2_rn(ns2, v[e]));
    vy[gl + 16 * e] = __ffma2_rn(s2, u[e], __fmul2_rn(c2, v[e]));
    u[e] = un;
  }
  return flags;
}

template <int EP, int C>
__global__ void __launch_bounds__(352)
jacobi_block_cluster_kernel(const double* __restrict__ Min, int l, int b, float* __restrict__ Vout,
                            DeviceStatus* status) {
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  constexpr int LDW = 32 * EP;                       // floats per column (W or V)
  constexpr int NB = 2 * C;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* S = reinterpret_cast<float*>(smem_raw);     // [buffer 2][slot 2][column b][W, V][LDW]
  __shared__ int s_flag[2], s_big[2];                // used in CTA 0, by sweep parity
  __shared__ __align__(8) uint64_t s_mbar[2];        // incoming remote blocks, by buffer
  const int t = threadIdx.x, lane = t & 31;
  const int grp = t >> 4, gl = t & 15;
  const unsigned gmask = 0xFFFFu << ((lane >> 4) * 16);
  const int bp = b + (b & 1);
  const float eps = 1.1920928955078125e-07f;
  const float tol = (float)l * eps, tol2 = tol * tol;
  const float big = 32.f * tol, big2 = big * big;
  const int colf = 2 * LDW;                          // floats per column slot (W and V)
  auto col = [&](int bf, int sl, int j) { return S + ((size_t)(bf * 2 + sl) * b + j) * colf; };
  const int pos[2] = {rank, NB - 1 - rank};          // the positions of this CTA's two slots

  // sweep start: position p holds block p; zero columns past l
  for (int e = t; e < 2 * b * LDW; e += blockDim.x) {
    const int sj = e / LDW, i = e - sj * LDW;
    const int sl = sj / b, j = sj - sl * b;
    const int g = pos[sl] * b + j;
    float* w = col(0, sl, j);
    w[i] = (i < l && g < l) ? (float)Min[i + (size_t)g * l] : 0.f;
    w[LDW + i] = (i == g && g < l) ? 1.f : 0.f;
  }
  if (rank == 0 && t == 0) { s_flag[0] = s_flag[1] = 0; s_big[0] = s_big[1] = 0; }
  if (t == 0) {
    cl_mbar_init(&s_mbar[0], 1);
    cl_mbar_init(&s_mbar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // where each slot's block goes (next position), and the bytes this CTA
  // receives from other CTAs per block round
  int dcta[2], dslot[2], rem_blocks = 0;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int q = next_pos(pos[h], NB);
    dcta[h] = q < C ? q : NB - 1 - q;
    dslot[h] = q < C ? 0 : 1;
    const int pp = prev_pos(pos[h], NB);
    if ((pp < C ? pp : NB - 1 - pp) != rank) ++rem_blocks;
  }
  uint32_t rem_bytes = (uint32_t)rem_blocks * (uint32_t)b * (uint32_t)colf * 4u;
  uint32_t mpar0 = 0u, mpar1 = 0u;
  cluster.sync();

  int buf = 0, sweep;
  const int cap = sweep_cap();
  for (sweep = 1; sweep <= cap; ++sweep) {
    const int par = sweep & 1;
    int fl = 0;                                      // bit 0 rotated, bit 1 large rotation
    for (int r = 0; r < NB - 1; ++r) {
      if (t == 0 && rem_bytes) cl_mbar_arm(&s_mbar[buf ^ 1], rem_bytes);
      if (r == 0) {
        // the pairs inside each block: round-robin on bp players
        for (int s = 0; s < bp - 1; ++s) {
          if (grp < bp) {
            const int sl = grp / (bp / 2), pr = grp - sl * (bp / 2);
            const int i = rr_player(pr, s, bp), j = rr_player(bp - 1 - pr, s, bp);
            if (i < b && j < b)
              fl |= rotate_pair16<EP>(col(buf, sl, min(i, j)), col(buf, sl, max(i, j)), gl, gmask, tol2, big2);
          }
          __syncthreads();
        }
      }
      // the pairs across the two blocks: group grp keeps column grp of
      // slot 0 (W and V) in registers through the b cross rounds
      {
        float2 xr[EP], ur[EP];
        if (grp < b) {
          const float2* wx = reinterpret_cast<const float2*>(col(buf, 0, grp));
#pragma unroll
          for (int e = 0; e < EP; ++e) {
            xr[e] = wx[gl + 16 * e];
            ur[e] = wx[LDW / 2 + gl + 16 * e];
          }
        }
        for (int s = 0; s < b; ++s) {
          if (grp < b) {
            int j = grp + s;
            if (j >= b) j -= b;
            fl |= rotate_xreg16<EP>(xr, ur, col(buf, 1, j), gl, gmask, tol2, big2);
          }
          __syncthreads();
        }
        if (grp < b) {
          float2* wx = reinterpret_cast<float2*>(col(buf, 0, grp));
#pragma unroll
          for (int e = 0; e < EP; ++e) {
            wx[gl + 16 * e] = xr[e];
            wx[LDW / 2 + gl + 16 * e] = ur[e];
          }
        }
        __syncthreads();
      }
      // every block to its next position (buffer buf ^ 1): 16-byte pieces
      const int per = b * colf / 4;                  // float4 per block
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float4* src = reinterpret_cast<const float4*>(col(buf, h, 0));
        float* dst = col(buf ^ 1, dslot[h], 0);
        if (dcta[h] == rank) {
          float4* d4 = reinterpret_cast<float4*>(dst);
          for (int e = t; e < per; e += blockDim.x) d4[e] = src[e];
        } else {
          const uint32_t rd = cl_mapa(cl_smem_u32(dst), dcta[h]);
          const uint32_t rb = cl_mapa(cl_smem_u32(&s_mbar[buf ^ 1]), dcta[h]);
          for (int e = t; e < per; e += blockDim.x) cl_st_async4(rd + 16u * (uint32_t)e, src[e], rb);
        }
      }
      __syncthreads();                               // this CTA's own block moves
      if (rem_bytes) {
        // the neighbours' blocks (bounded wait: on a timeout the status
        // records it and the sweeps run on without waiting, so every CTA
        // still meets every cluster barrier)
        const uint32_t ph = (buf ^ 1) ? mpar1 : mpar0;
        if (!cl_mbar_try_wait(&s_mbar[buf ^ 1], ph)) {
          const long long t0 = clock64();
          while (!cl_mbar_try_wait(&s_mbar[buf ^ 1], ph)) {
            if (clock64() - t0 > kClusterWaitCycles) {
              if (t == 0) raise_status(status, SORSVD_ERR_TIMEOUT);
              rem_bytes = 0;
              break;
            }
          }
        }
        if (buf ^ 1) mpar1 ^= 1u;
        else mpar0 ^= 1u;
      }
      buf ^= 1;
    }
    const int rot_local = __syncthreads_or(fl & 1);
    const int big_local = __syncthreads_or(fl & 2);
    if (t == 0) {
      if (rot_local) atomicOr(cluster.map_shared_rank(&s_flag[par], 0), 1);
      if (big_local) atomicOr(cluster.map_shared_rank(&s_big[par], 0), 1);
    }
    cluster.sync();
    const int rot = *cluster.map_shared_rank(&s_flag[par], 0);
    const int bg = *cluster.map_shared_rank(&s_big[par], 0);
    cluster.sync();                                  // every CTA has read CTA 0's flags
    // this parity's flags are next used two sweeps on, after two more barriers
    if (rank == 0 && t == 0) { s_flag[par] = 0; s_big[par] = 0; }
    if (!rot) break;
    if (sweep == cap) {
      if (bg && rank == 0 && t == 0) raise_status(status, SORSVD_ERR_NOT_CONVERGED);
      break;
    }
  }
  if (rank == 0 && t == 0) atomicOr(&status->info, (min(sweep, cap)) << 8);
  // a sweep ends where it began: slot h holds block pos[h]
  for (int e = t; e < 2 * b * LDW; e += blockDim.x) {
    const int sj = e / LDW, i = e - sj * LDW;
    const int sl = sj / b, j = sj - sl * b;
    const int g = pos[sl] * b + j;
    if (g < l && i < l) Vout[i + (size_t)g * l] = col(buf, sl, j)[LDW + i];
  }
}

// From the accumulated right vector v_j (sweep precision): z = M v_j,
// sigma_j = ||z||, u_j = z / sigma_j, all in binary64.
template <typename J>
__device__ __forceinline__ void jacobi_finish_body(const double* __restrict__ M, int l, const J* __restrict__ Vin,
                                                   double* __restrict__ U64, double* __restrict__ V64,
                                                   double* __restrict__ sig, int j) {
  __shared__ double v[SORSVD_MAX_L];
  __shared__ double red[32];
  // the rotations keep ||v_j|| = 1 only to a few ulps each: normalise first
  double nv = 0;
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    const double x = (double)Vin[i + (size_t)j * l];
    v[i] = x;
    nv += x * x;
  }
  nv = block_sum<J>(nv, red);
  const double inv_nv = nv > 0 ? 1.0 / sqrt(nv) : 0.0;
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    const double x = v[i] * inv_nv;
    v[i] = x;
    V64[i + (size_t)j * l] = x;
  }
  __syncthreads();
  double nz = 0;
  double zloc[(SORSVD_MAX_L + 255) / 256];
  int q = 0;
  for (int i = threadIdx.x; i < l; i += blockDim.x, ++q) {     // z_i = sum_c M_ic v_c
    double s = 0;
    for (int c = 0; c < l; ++c) s += M[i + (size_t)c * l] * v[c];
    zloc[q] = s;
    nz += s * s;
  }
  nz = block_sum<J>(nz, red);
  const double sg = sqrt(nz);
  const double inv_sg = sg > 0 ? 1.0 / sg : 0.0;
  q = 0;
  for (int i = threadIdx.x; i < l; i += blockDim.x, ++q) U64[i + (size_t)j * l] = zloc[q] * inv_sg;
  if (threadIdx.x == 0) sig[j] = sg;
}

template <typename J>
__global__ void __launch_bounds__(256)
jacobi_finish_kernel(const double* __restrict__ M, int l, const J* __restrict__ Vin, double* __restrict__ U64,
                     double* __restrict__ V64, double* __restrict__ sig) {
  jacobi_finish_body<J>(M, l, Vin, U64, V64, sig, blockIdx.x);
}

template <typename J, typename TS>
__device__ __forceinline__ void jacobi_order_body(int l, int k, const double* __restrict__ U64,
                                                  const double* __restrict__ V64, const double* __restrict__ sig,
                                                  J* __restrict__ Ut, J* __restrict__ Vt, TS* __restrict__ S) {
  __shared__ int s_order[SORSVD_MAX_L];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = blockDim.x / 32;
  const int NTH = blockDim.x;
  for (int c = t; c < l; c += NTH) {
    const double sc = sig[c];
    int rank = 0;
    for (int d = 0; d < l; ++d) {
      const double sd = sig[d];
      rank += (sd > sc) || (sd == sc && d < c);
    }
    s_order[rank] = c;
  }
  __syncthreads();
  for (int j = warp; j < l; j += nwarps) {
    const int c = s_order[j];
    const double* uc = U64 + (size_t)c * l;
    const double* vc = V64 + (size_t)c * l;
    double best = -1;
    int bi = l;
    for (int i = lane; i < l; i += 32) {
      const double a = fabs(uc[i]);
      if (a > best) { best = a; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    const double sgn = (bi < l && uc[bi] < 0.0) ? -1.0 : 1.0;
    for (int i = lane; i < l; i += 32) {
      Ut[(size_t)j * l + i] = (J)(sgn * uc[i]);
      Vt[(size_t)j * l + i] = (J)(sgn * vc[i]);
    }
    if (lane == 0 && j < k) S[j] = (TS)sig[c];
  }
}


// The same ordering and sign convention with one block per column c of the
// finish (the rank of sigma_c and the sign are block reductions, then the
// block writes its column to position rank): the binary64 compares and
// conversions spread over l blocks instead of one.
template <typename J, typename TS>
__global__ void __launch_bounds__(256)
jacobi_order_col_kernel(int l, int k, const double* __restrict__ U64, const double* __restrict__ V64,
                        const double* __restrict__ sig, J* __restrict__ Ut, J* __restrict__ Vt, TS* __restrict__ S) {
  __shared__ int s_rank[8], s_bi[8];
  __shared__ double s_best[8];
  const int c = blockIdx.x, t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
  const double sc = sig[c];
  int rank = 0;
  for (int d = t; d < l; d += blockDim.x) {
    const double sd = sig[d];
    rank += (sd > sc) || (sd == sc && d < c);
  }
  const double* uc = U64 + (size_t)c * l;
  double best = -1;
  int bi = l;
  for (int i = t; i < l; i += blockDim.x) {
    const double a = fabs(uc[i]);
    if (a > best) { best = a; bi = i; }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rank += __shfl_xor_sync(0xffffffffu, rank, o);
    const double ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if (lane == 0) { s_rank[warp] = rank; s_best[warp] = best; s_bi[warp] = bi; }
  __syncthreads();
  rank = 0;
  best = -1;
  bi = l;
  for (int w = 0; w < nw; ++w) {
    rank += s_rank[w];
    if (s_best[w] > best || (s_best[w] == best && s_bi[w] < bi)) { best = s_best[w]; bi = s_bi[w]; }
  }
  const double sgn = (bi < l && uc[bi] < 0.0) ? -1.0 : 1.0;
  const double* vc = V64 + (size_t)c * l;
  for (int i = t; i < l; i += blockDim.x) {
    Ut[(size_t)rank * l + i] = (J)(sgn * uc[i]);
    Vt[(size_t)rank * l + i] = (J)(sgn * vc[i]);
  }
  if (t == 0 && rank < k) S[rank] = (TS)sc;
}

// ---------------------------------------------------------------- batched
// work of one problem: [V out: l^2 J][U64, V64: 2 l^2 f64][sig: l f64]
template <typename J>
struct BatchedWork {
  J* vout; double* u64; double* v64; double* sig;
  __host__ __device__ BatchedWork(void* w, int l) {
    char* c = static_cast<char*>(w);
    vout = reinterpret_cast<J*>(c);
    u64 = reinterpret_cast<double*>(c + (((size_t)l * l * sizeof(J) + 15) & ~(size_t)15));
    v64 = u64 + (size_t)l * l;
    sig = v64 + (size_t)l * l;
  }
};

template <typename J, int EPL, int NT>
__global__ void __launch_bounds__(NT) jacobi_sweep_batched_kernel(const JacobiJob* __restrict__ jobs) {
  const JacobiJob& jb = jobs[blockIdx.x];
  BatchedWork<J> w(jb.work, jb.l);
  jacobi_sweep_body<J, true, EPL>(jb.M, jb.l, w.vout, nullptr, jb.status);
}

template <typename J>
__global__ void __launch_bounds__(256) jacobi_finish_batched_kernel(const JacobiJob* __restrict__ jobs) {
  const JacobiJob& jb = jobs[blockIdx.y];
  if ((int)blockIdx.x >= jb.l) return;
  BatchedWork<J> w(jb.work, jb.l);
  jacobi_finish_body<J>(jb.M, jb.l, w.vout, w.u64, w.v64, w.sig, blockIdx.x);
}

template <typename J>
__global__ void __launch_bounds__(256) jacobi_order_batched_kernel(const JacobiJob* __restrict__ jobs) {
  const JacobiJob& jb = jobs[blockIdx.x];
  BatchedWork<J> w(jb.work, jb.l);
  jacobi_order_body<J, J>(jb.l, jb.k, w.u64, w.v64, w.sig, (J*)jb.Ut, (J*)jb.Vt, (J*)jb.S);
}

template <typename J, bool IN_SMEM>
cudaError_t launch_sweep(const double* M, int l, J* vout, J* gwork, size_t smem, DeviceStatus* status,
                         cudaStream_t st) {
  const int epl = (l + 7) / 8;
  // block size from the per-lane register footprint (2 EPL words per lane)
#define SWEEP(E)                                                                                      \
  {                                                                                                   \
    constexpr int NT = (E * sizeof(J) <= 64) ? 1024 : ((E * sizeof(J) <= 160) ? 512 : 256);          \
    if (IN_SMEM) {                                                                                    \
      cudaError_t e = cudaFuncSetAttribute(jacobi_sweep_kernel<J, IN_SMEM, E, NT>,                   \
                                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
      if (e != cudaSuccess) return e;                                                                 \
    }                                                                                                 \
    jacobi_sweep_kernel<J, IN_SMEM, E, NT><<<1, NT, smem, st>>>(M, l, vout, gwork, status);          \
    return cudaGetLastError();                                                                        \
  }
  if (epl <= 4) SWEEP(4)
  if (epl <= 8) SWEEP(8)
  if (epl <= 16) SWEEP(16)
  if (epl <= 24) SWEEP(24)
  if (epl <= 32) SWEEP(32)
  SWEEP(40)
#undef SWEEP
}

constexpr size_t kSweepSmemMax = 200 * 1024;

// [W, V fallback: 2 l^2 J][V out: l^2 J][U64, V64: 2 l^2 f64][sig: l f64], sized for J = double;
// the cooperative sweep's own W, V and flags follow (256-aligned)
inline size_t jacobi_base_bytes(int l) {
  return ((3 * (size_t)l * l * sizeof(double) + 15) & ~(size_t)15) + 2 * (size_t)l * l * 8 + (size_t)l * 8;
}

// template EP of the paired sweep for l (the kernel's row stride is 16 EP)
inline int sweep_f2_ep(int l) {
  const int need = (l + 15) / 16;
  const int eps[] = {2, 4, 6, 7, 8, 10};
  for (int e : eps)
    if (need <= e) return e;
  return 0;                                        // l > 160: not handled
}
inline size_t sweep_f2_smem(int l) {
  const int ep = sweep_f2_ep(l);
  return ep ? 2 * (size_t)16 * ep * l * sizeof(float) : (size_t)-1;
}

// template EP of the 16-lane sweep for l (row stride 32 EP)
inline int sweep_g_ep(int l) {
  const int need = (l + 31) / 32;
  return need <= 5 ? need : 0;
}
inline size_t sweep_g_smem(int l) {
  const int ep = sweep_g_ep(l);
  const int N = (l + 1) & ~1;
  return ep ? 2 * (size_t)32 * ep * l * sizeof(float) + (size_t)(N - 1) * (N / 2) * 4 : (size_t)-1;
}

// cooperative sweep: ldw = 32 EP rows; work = [W ldw*l][V ldw*l][flags 2*(kMaxSweeps+1) ints]
inline int sweep_coop_ep(int l) {
  const int need = (l + 31) / 32;
  return need <= 10 ? need : 0;
}
size_t sweep_coop_work_bytes(int l) {
  const int ep = std::max(1, sweep_coop_ep(l));
  return 2 * (size_t)32 * ep * l * sizeof(float) + 2 * (kMaxSweeps + 1) * sizeof(int) + 256;
}

cudaError_t launch_sweep_coop(const double* M, int l, float* vout, void* work, DeviceStatus* status, cudaStream_t st) {
  const int ep = sweep_coop_ep(l);
  if (!ep) return cudaErrorInvalidValue;
  int ldw = 32 * ep;
  float* W = reinterpret_cast<float*>(work);
  float* V = W + (size_t)ldw * l;
  int* flags = reinterpret_cast<int*>(V + (size_t)ldw * l);
  cudaError_t e = cudaMemsetAsync(flags, 0, 2 * (kMaxSweeps + 1) * sizeof(int), st);
  if (e != cudaSuccess) return e;
  const int npairs = (l + 1) / 2;
  int grid = (npairs + kCoopPairsPerCta - 1) / kCoopPairsPerCta;
  grid = std::min(grid, num_sms());
  void* args[] = {(void*)&M, (void*)&l, (void*)&ldw, (void*)&W, (void*)&V, (void*)&vout, (void*)&flags, (void*)&status};
#define COOP(E)                                                                                                    \
  return cudaLaunchCooperativeKernel((const void*)jacobi_sweep_coop_kernel<E>, dim3(grid), dim3(kCoopThreads), args, \
                                     0, st);
  switch (ep) {
    case 1: COOP(1)
    case 2: COOP(2)
    case 3: COOP(3)
    case 4: COOP(4)
    case 5: COOP(5)
    case 6: COOP(6)
    case 7: COOP(7)
    case 8: COOP(8)
    case 9: COOP(9)
    case 10: COOP(10)
    default: return cudaErrorInvalidValue;
  }
#undef COOP
}

// cluster sweep: 16 lanes per pair, columns of 32 EP floats
inline int sweep_cluster_ep(int l) {
  const int need = (l + 31) / 32;
  return need <= 10 ? need : 0;
}

// block-cyclic cluster sweep on C CTAs: b = ceil(l / 2C) columns per block,
// 16 lanes per pair, (b rounded up to even) pairs per CTA at once.  The
// cluster has 16 CTAs, or 8 (SORSVD_JACOBI_CLUSTER=8: half the block
// rounds and exchanges per sweep, twice the columns per local round) when
// its blocks fit in shared memory.
inline int block_cluster_b(int l, int C = kClusterCtas) { return (l + 2 * C - 1) / (2 * C); }
inline size_t block_cluster_smem(int l, int C = kClusterCtas) {
  return (size_t)2 * 2 * block_cluster_b(l, C) * 2 * 32 * std::max(1, sweep_cluster_ep(l)) * sizeof(float);
}
inline int block_cluster_ctas(int l) {
  static const int env = [] { const char* v = std::getenv("SORSVD_JACOBI_CLUSTER"); return v ? std::atoi(v) : 16; }();
  if (env == 8 && block_cluster_smem(l, 8) <= kSweepSmemMax && 16 * (block_cluster_b(l, 8) + 1) <= 352) return 8;
  return 16;
}

cudaError_t launch_block_cluster(const double* M, int l, float* vout, DeviceStatus* status, cudaStream_t st) {
  const int C = block_cluster_ctas(l);
  const int ep = sweep_cluster_ep(l), b = block_cluster_b(l, C);
  const size_t smem = block_cluster_smem(l, C);
  const int nt = 16 * (b + (b & 1));
  if (!ep || nt > 352 || smem > kSweepSmemMax) return cudaErrorInvalidValue;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(C, 1, 1);
  cfg.blockDim = dim3(nt, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
#define BLSWEEP(E)                                                                                  \
  {                                                                                                 \
    auto kern = C == 8 ? jacobi_block_cluster_kernel<E, 8> : jacobi_block_cluster_kernel<E, 16>;    \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);  \
    if (e == cudaSuccess)                                                                           \
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);       \
    if (e != cudaSuccess) return e;                                                                 \
    return cudaLaunchKernelEx(&cfg, kern, M, l, b, vout, status);                                   \
  }
  switch (ep) {
    case 1: BLSWEEP(1)
    case 2: BLSWEEP(2)
    case 3: BLSWEEP(3)
    case 4: BLSWEEP(4)
    case 5: BLSWEEP(5)
    case 6: BLSWEEP(6)
    case 7: BLSWEEP(7)
    case 8: BLSWEEP(8)
    case 9: BLSWEEP(9)
    case 10: BLSWEEP(10)
    default: return cudaErrorInvalidValue;
  }
#undef BLSWEEP
}

cudaError_t launch_sweep_g(const double* M, int l, float* vout, DeviceStatus* status, cudaStream_t st) {
  const int ep = sweep_g_ep(l);
  const size_t smem = sweep_g_smem(l);
  if (!ep || smem > kSweepSmemMax) return cudaErrorInvalidValue;
  // one 16-lane group per pair, whole warps, <= 1024
  const int nt = std::min(1024, (((l + 1) / 2 * 16 + 31) / 32) * 32);
#define GSWEEP(E)                                                                                   \
  {                                                                                                 \
    cudaError_t e = cudaFuncSetAttribute(jacobi_sweep_g_kernel<16, E>,                             \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
    if (e != cudaSuccess) return e;                                                                 \
    jacobi_sweep_g_kernel<16, E><<<1, nt, smem, st>>>(M, l, vout, status);                         \
    return cudaGetLastError();                                                                      \
  }
  switch (ep) {
    case 1: GSWEEP(1)
    case 2: GSWEEP(2)
    case 3: GSWEEP(3)
    case 4: GSWEEP(4)
    case 5: GSWEEP(5)
    default: return cudaErrorInvalidValue;
  }
#undef GSWEEP
}

cudaError_t launch_sweep_f2(const double* M, int l, float* vout, DeviceStatus* status, cudaStream_t st) {
  const int ep = sweep_f2_ep(l);
  const size_t smem = sweep_f2_smem(l);            // sized with the same EP the kernel indexes with
  if (!ep || smem > kSweepSmemMax) return cudaErrorInvalidValue;
  // one 8-lane group per pair: (l/2 pairs) x 8 lanes, whole warps, <= 512
  const int nt = std::min(512, (((l + 1) / 2 * 8 + 31) / 32) * 32);
#define F2SWEEP(E)                                                                                  \
  {                                                                                                 \
    cudaError_t e = cudaFuncSetAttribute(jacobi_sweep_f2_kernel<E>,                                \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);  \
    if (e != cudaSuccess) return e;                                                                 \
    jacobi_sweep_f2_kernel<E><<<1, nt, smem, st>>>(M, l, vout, status);                            \
    return cudaGetLastError();                                                                      \
  }
  switch (ep) {
    case 2: F2SWEEP(2)
    case 4: F2SWEEP(4)
    case 6: F2SWEEP(6)
    case 7: F2SWEEP(7)
    case 8: F2SWEEP(8)
    case 10: F2SWEEP(10)
    default: return cudaErrorInvalidValue;
  }
#undef F2SWEEP
}

// binary64 Jacobi work beyond the common areas: the fp32 rotations (l^2
// fp32), six l x l binary64 matrices and a scratch status word
inline size_t jacobi_mixed_bytes(int l) {
  return (((size_t)l * l * 4 + 255) & ~(size_t)255) + 6 * (size_t)l * l * 8 + 256;
}

// fp32 sweeps of M (one block, or the cluster for l >= kClusterMinL); false
// when neither form takes l
bool launch_sweep32(const double* M, int l, float* vout, DeviceStatus* status, cudaStream_t st, cudaError_t* e) {
  if (l >= kClusterMinL && sweep_cluster_ep(l) && block_cluster_smem(l) <= kSweepSmemMax) {
    *e = launch_block_cluster(M, l, vout, status, st);
    return true;
  }
  if (sweep_g_smem(l) <= kSweepSmemMax) {
    *e = launch_sweep_g(M, l, vout, status, st);
    return true;
  }
  return false;
}

// The binary64 SVD of M by fp32 sweeps polished in binary64: fp32 sweeps
// give rotations V32 (orthogonal to fp32 level); V = V32 R^{-1} with
// R^T R = V32^T V32 (binary64 Cholesky) is orthonormal to binary64 level;
// binary64 sweeps of W = M V (columns already orthogonal to fp32 level, so
// one or two sweeps reach the binary64 tolerance: Jacobi converges
// quadratically) give V'; the right vectors are V V'.  The binary64 sweeps
// are the expensive part on this GPU (binary64 runs at 1/64 of the fp32
// rate, one block), so most of the rotation work moves to fp32.  The fp32
// sweeps only precondition: they report into a scratch status word, since
// on a core with an exact null space (columns at 1e-17 of sigma_1, below
// fp32 rounding) they cannot meet their own tolerance - the binary64 sweeps
// decide convergence.
// Returns false (nothing launched) when the fp32 sweeps do not take l.
bool jacobi_f64_mixed(const double* M, int l, double* vout, char* mixed, double* gwork, DeviceStatus* status,
                      cudaStream_t st, cudaError_t* e) {
  if (l < 2 || l > SORSVD_MAX_L_F64) return false;
  float* v32 = reinterpret_cast<float*>(mixed);
  double* d = reinterpret_cast<double*>(mixed + (((size_t)l * l * 4 + 255) & ~(size_t)255));
  const size_t ll = (size_t)l * l;
  double *V64 = d, *G = d + ll, *R = d + 2 * ll, *V = d + 3 * ll, *W = d + 4 * ll, *Vp = d + 5 * ll;
  DeviceStatus* scratch = reinterpret_cast<DeviceStatus*>(d + 6 * ll);
  if (!launch_sweep32(M, l, v32, scratch, st, e)) return false;
  if (*e != cudaSuccess) return true;
  if ((*e = launch_widen(v32, SORSVD_F32, l, l, l, V64, true, l, st)) != cudaSuccess) return true;
  if ((*e = launch_small_gemm64(V64, true, V64, false, G, l, st)) != cudaSuccess) return true;      // V32^T V32
  if ((*e = launch_chol_inv(G, l, 0.0, R, true, status, st)) != cudaSuccess) return true;
  if ((*e = launch_small_gemm64(V64, false, R, false, V, l, st)) != cudaSuccess) return true;      // V32 R^{-1}
  if ((*e = launch_small_gemm64(M, false, V, false, W, l, st)) != cudaSuccess) return true;        // W = M V
  const size_t need = 2 * ll * sizeof(double);
  *e = (need <= kSweepSmemMax) ? launch_sweep<double, true>(W, l, Vp, gwork, need, status, st)
                               : launch_sweep<double, false>(W, l, Vp, gwork, 0, status, st);
  if (*e != cudaSuccess) return true;
  *e = launch_small_gemm64(V, false, Vp, false, vout, l, st);                                      // V V'
  return true;
}

template <typename J, typename TS>
cudaError_t run_all(const double* M, int l, int k, void* Ut, void* Vt, void* S, void* work, DeviceStatus* status,
                    cudaStream_t st) {
  // work: [W, V fallback: 2 l^2 J][V out: l^2 J][U64, V64: 2 l^2 f64][sig: l f64]
  char* w = static_cast<char*>(work);
  J* gwork = reinterpret_cast<J*>(w);
  J* vout = gwork + 2 * (size_t)l * l;
  double* u64 = reinterpret_cast<double*>(w + ((3 * (size_t)l * l * sizeof(J) + 15) & ~(size_t)15));
  double* v64 = u64 + (size_t)l * l;
  double* sig = v64 + (size_t)l * l;
  const size_t need = 2 * (size_t)l * l * sizeof(J);
  cudaError_t e;
  static const int lanes = [] { const char* v = std::getenv("SORSVD_JACOBI_LANES"); return v ? std::atoi(v) : 16; }();
  char* mixed = w + ((jacobi_base_bytes(l) + 255) & ~(size_t)255) + sweep_coop_work_bytes(l);
  if (sizeof(J) == 8 && jacobi_f64_mixed(M, l, reinterpret_cast<double*>(vout), mixed,
                                          reinterpret_cast<double*>(gwork), status, st, &e)) {
    // binary64: fp32 sweeps polished in binary64
  } else if (sizeof(J) == 4 && lanes == 16 && l >= kClusterMinL && sweep_cluster_ep(l) &&
      block_cluster_smem(l) <= kSweepSmemMax)
    e = launch_block_cluster(M, l, reinterpret_cast<float*>(vout), status, st);
  else if (sizeof(J) == 4 && lanes == 16 && sweep_g_smem(l) <= kSweepSmemMax)
    e = launch_sweep_g(M, l, reinterpret_cast<float*>(vout), status, st);
  else if (sizeof(J) == 4 && sweep_coop_ep(l) && sweep_f2_smem(l) > kSweepSmemMax)
    e = launch_sweep_coop(M, l, reinterpret_cast<float*>(vout), w + ((jacobi_base_bytes(l) + 255) & ~(size_t)255),
                          status, st);
  else if (sizeof(J) == 4 && sweep_f2_smem(l) <= kSweepSmemMax)
    e = launch_sweep_f2(M, l, reinterpret_cast<float*>(vout), status, st);
  else
    e = (need <= kSweepSmemMax) ? launch_sweep<J, true>(M, l, vout, gwork, need, status, st)
                                : launch_sweep<J, false>(M, l, vout, gwork, 0, status, st);
  if (e != cudaSuccess) return e;
  jacobi_finish_kernel<J><<<l, 256, 0, st>>>(M, l, vout, u64, v64, sig);
  jacobi_order_col_kernel<J, TS><<<l, 256, 0, st>>>(l, k, u64, v64, sig, (J*)Ut, (J*)Vt, (TS*)S);
  return cudaGetLastError();
}

}  // namespace

cudaError_t set_jacobi_sweep_cap(int cap) {
  const int v = (cap > 0 && cap < kMaxSweeps) ? cap : kMaxSweeps;
  return cudaMemcpyToSymbol(g_sweep_cap, &v, sizeof(int));
}

size_t jacobi_work_bytes(int l) {
  return ((jacobi_base_bytes(l) + 255) & ~(size_t)255) + sweep_coop_work_bytes(l) + jacobi_mixed_bytes(l);
}

cudaError_t launch_jacobi(const double* M, int l, int k, bool f64, void* Ut, void* Vt, void* S, bool S_f64,
                          void* work, DeviceStatus* status, cudaStream_t st) {
  if (f64) return run_all<double, double>(M, l, k, Ut, Vt, S, work, status, st);
  if (S_f64) return cudaErrorInvalidValue;
  return run_all<float, float>(M, l, k, Ut, Vt, S, work, status, st);
}

int jacobi_batched_max_l(bool f64) { return f64 ? 112 : 160; }

size_t jacobi_batched_work_bytes(int l) {
  return (((size_t)l * l * sizeof(double) + 15) & ~(size_t)15) + 2 * (size_t)l * l * 8 + (size_t)l * 8;
}

cudaError_t launch_jacobi_batched(const JacobiJob* jobs, int njobs, int max_l, bool f64, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  if (max_l < 1 || max_l > jacobi_batched_max_l(f64)) return cudaErrorInvalidValue;
  const size_t smem = 2 * (size_t)max_l * max_l * (f64 ? 8 : 4);
  const int epl = (max_l + 7) / 8;
  // one problem per block: (l/2 pairs) x 8 lanes, rounded up to whole warps
  const int pairs = (max_l + 1) / 2;
  int nt = ((pairs * 8 + 31) / 32) * 32;
#define BSWEEP(J, E)                                                                                        \
  {                                                                                                         \
    cudaError_t e = cudaFuncSetAttribute(jacobi_sweep_batched_kernel<J, E, 512>,                            \
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);           \
    if (e != cudaSuccess) return e;                                                                         \
    jacobi_sweep_batched_kernel<J, E, 512><<<njobs, std::min(nt, 512), smem, st>>>(jobs);                   \
  }
  if (f64) {
    if (epl <= 4) BSWEEP(double, 4)
    else if (epl <= 8) BSWEEP(double, 8)
    else BSWEEP(double, 16)
  } else {
    if (epl <= 4) BSWEEP(float, 4)
    else if (epl <= 8) BSWEEP(float, 8)
    else if (epl <= 16) BSWEEP(float, 16)
    else BSWEEP(float, 20)
  }
#undef BSWEEP
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (f64) {
    jacobi_finish_batched_kernel<double><<<dim3(max_l, njobs), 256, 0, st>>>(jobs);
    jacobi_order_batched_kernel<double><<<njobs, 256, 0, st>>>(jobs);
  } else {
    jacobi_finish_batched_kernel<float><<<dim3(max_l, njobs), 256, 0, st>>>(jobs);
    jacobi_order_batched_kernel<float><<<njobs, 256, 0, st>>>(jobs);
  }
  return cudaGetLastError();
}

}  // namespace sorsvd
