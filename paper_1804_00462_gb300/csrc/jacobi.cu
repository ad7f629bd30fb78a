// Truncated SVD of the small core matrix M (l x l) of Algorithm 3
// ("compute the rank-k truncated SVD of M").  One-sided (Hestenes) Jacobi:
// columns w_p, w_q of W = M V are rotated until every pair is orthogonal to
// a relative tolerance; then sigma_j = ||M v_j|| / ||v_j||, U~ = M V diag(sigma)^{-1}.
//
// Three kernels:
//  1. sweeps (one block): W and V in shared memory when 2 l^2 words fit, else
//     in the caller's work buffer.  Pair schedule: round-robin tournament
//     (circle method); in each of the N - 1 rounds (N = l rounded up to even)
//     the N/2 disjoint pairs are independent, one 8-lane group of a warp
//     rotates each pair, one barrier separates rounds.  Rotations are applied
//     while a pair's cosine exceeds l * eps of the sweep precision.  The
//     sweep count is capped; hitting the cap with a cosine above 32 l eps
//     raises SORSVD_ERR_NOT_CONVERGED.
//  2. finish (one block per column), binary64: w_j = M v_j, sigma_j =
//     ||w_j|| / ||v_j||.  sigma_j is a Rayleigh quotient of M^T M, so its error
//     is quadratic in the departure of v_j from a singular vector: fp32 sweeps
//     followed by this step give singular values to about 1e-8 of sigma_1,
//     while fp32 rotations alone leak about 1e-5 of sigma_1 into the small
//     columns.
//  3. order (one block): sigma descending (ties by column index), U~ =
//     w / ||w||, V~ = v / ||v||; sign: the largest-magnitude entry of each
//     column of U~ is made positive and the matching column of V~ follows.
#include "internal.cuh"

namespace sorsvd {
namespace {

constexpr int JT = 1024;
constexpr int kMaxSweeps = 30;

__device__ __forceinline__ int rr_player(int pos, int round, int N) {
  // position 0 is fixed; positions 1..N-1 rotate by one place per round
  if (pos == 0) return 0;
  int x = (pos - 1 - round) % (N - 1);
  if (x < 0) x += N - 1;
  return 1 + x;
}

template <typename J>
__device__ __forceinline__ J group8_sum(J v, unsigned mask) {
  v += __shfl_xor_sync(mask, v, 4);
  v += __shfl_xor_sync(mask, v, 2);
  v += __shfl_xor_sync(mask, v, 1);
  return v;
}

template <typename J>
__global__ void __launch_bounds__(JT)
jacobi_sweep_kernel(const double* __restrict__ Min, int l, J* __restrict__ Vout, J* __restrict__ gwork,
                    int in_smem, DeviceStatus* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_rot, s_big;
  J* W;
  J* V;
  if (in_smem) { W = reinterpret_cast<J*>(smem_raw); V = W + (size_t)l * l; }
  else { W = gwork; V = gwork + (size_t)l * l; }
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int grp = lane >> 3, gl = lane & 7;
  const unsigned gmask = 0xFFu << (grp * 8);
  const int ngroups = (JT / 32) * 4;
  const J eps = sizeof(J) == 8 ? (J)2.220446049250313e-16 : (J)1.1920928955078125e-07;
  const J tol = (J)l * eps, tol2 = tol * tol;
  const J big = (J)32 * tol, big2 = big * big;

  for (int e = t; e < l * l; e += JT) {
    W[e] = (J)Min[e];
    V[e] = (e % l == e / l) ? (J)1 : (J)0;
  }
  __syncthreads();

  const int N = (l + 1) & ~1;
  int sweep;
  for (sweep = 1; sweep <= kMaxSweeps; ++sweep) {
    if (t == 0) { s_rot = 0; s_big = 0; }
    __syncthreads();
    for (int r = 0; r < N - 1; ++r) {
      for (int pr = warp * 4 + grp; pr < N / 2; pr += ngroups) {
        const int a = rr_player(pr, r, N), b = rr_player(N - 1 - pr, r, N);
        if (a >= l || b >= l) continue;                // bye (whole group)
        const int p = min(a, b), q = max(a, b);
        J* wp = W + (size_t)p * l;
        J* wq = W + (size_t)q * l;
        J al = 0, be = 0, ga = 0;
        for (int i = gl; i < l; i += 8) {
          const J x = wp[i], y = wq[i];
          al += x * x; be += y * y; ga += x * y;
        }
        // xor butterflies leave bitwise-identical sums in all 8 lanes, so
        // the group takes one decision and one rotation
        al = group8_sum(al, gmask); be = group8_sum(be, gmask); ga = group8_sum(ga, gmask);
        if (!(ga * ga > tol2 * al * be)) continue;
        if (gl == 0 && ga * ga > big2 * al * be) s_big = 1;
        const J zeta = (be - al) / ((J)2 * ga);
        const J az = fabs(zeta);
        const J root = az > (J)1 ? az * sqrt((J)1 + ((J)1 / az) * ((J)1 / az)) : sqrt((J)1 + az * az);
        const J tt = (zeta >= (J)0 ? (J)1 : (J)-1) / (az + root);
        const J cs = (J)1 / sqrt((J)1 + tt * tt);
        const J sn = cs * tt;
        for (int i = gl; i < l; i += 8) {
          const J x = wp[i], y = wq[i];
          wp[i] = cs * x - sn * y;
          wq[i] = sn * x + cs * y;
        }
        J* vp = V + (size_t)p * l;
        J* vq = V + (size_t)q * l;
        for (int i = gl; i < l; i += 8) {
          const J x = vp[i], y = vq[i];
          vp[i] = cs * x - sn * y;
          vq[i] = sn * x + cs * y;
        }
        if (gl == 0) s_rot = 1;
      }
      __syncthreads();
    }
    const int rot = s_rot, bg = s_big;
    __syncthreads();
    if (!rot) break;
    if (sweep == kMaxSweeps) {
      if (bg && t == 0) raise_status(status, SORSVD_ERR_NOT_CONVERGED);
      break;
    }
  }
  if (t == 0) atomicOr(&status->info, (min(sweep, kMaxSweeps)) << 8);
  for (int e = t; e < l * l; e += JT) Vout[e] = V[e];
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

// w_j = M v_j (binary64), sigma_j = ||w_j|| / ||v_j||
template <typename J>
__global__ void __launch_bounds__(256)
jacobi_finish_kernel(const double* __restrict__ M, int l, const J* __restrict__ Vin, double* __restrict__ W64,
                     double* __restrict__ sig, double* __restrict__ vnorm) {
  __shared__ double v[SORSVD_MAX_L];
  __shared__ double red[32];
  const int j = blockIdx.x;
  double nv = 0;
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    const double x = (double)Vin[i + (size_t)j * l];
    v[i] = x;
    nv += x * x;
  }
  nv = block_sum<J>(nv, red);
  double nw = 0;
  for (int i = threadIdx.x; i < l; i += blockDim.x) {
    double s = 0;
    for (int c = 0; c < l; ++c) s += M[i + (size_t)c * l] * v[c];
    W64[i + (size_t)j * l] = s;
    nw += s * s;
  }
  nw = block_sum<J>(nw, red);
  if (threadIdx.x == 0) {
    const double n_v = sqrt(nv);
    sig[j] = n_v > 0 ? sqrt(nw) / n_v : 0.0;
    vnorm[j] = n_v;
  }
}

template <typename J, typename TS>
__global__ void __launch_bounds__(JT)
jacobi_order_kernel(int l, int k, const double* __restrict__ W64, const J* __restrict__ Vin,
                    const double* __restrict__ sig, const double* __restrict__ vnorm, J* __restrict__ Ut,
                    J* __restrict__ Vt, TS* __restrict__ S) {
  __shared__ int s_order[SORSVD_MAX_L];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = JT / 32;
  for (int c = t; c < l; c += JT) {
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
    const double sg = sig[c], nv = vnorm[c];
    const double uinv = (sg > 0.0 && nv > 0.0) ? 1.0 / (sg * nv) : 0.0;
    const double vinv = nv > 0.0 ? 1.0 / nv : 0.0;
    const double* wc = W64 + (size_t)c * l;
    double best = -1;
    int bi = l;
    for (int i = lane; i < l; i += 32) {
      const double a = fabs(wc[i]);
      if (a > best) { best = a; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    const double sgn = (bi < l && wc[bi] < 0.0) ? -1.0 : 1.0;
    for (int i = lane; i < l; i += 32) {
      Ut[(size_t)j * l + i] = (J)(sgn * wc[i] * uinv);
      Vt[(size_t)j * l + i] = (J)(sgn * (double)Vin[(size_t)c * l + i] * vinv);
    }
    if (lane == 0 && j < k) S[j] = (TS)sg;
  }
}

template <typename J, typename TS>
cudaError_t run_all(const double* M, int l, int k, void* Ut, void* Vt, void* S, void* work, DeviceStatus* status,
                    cudaStream_t st) {
  // work: [sweep W,V fallback: 2 l^2 J][V out: l^2 J][W64: l^2 f64][sig, vnorm: 2 l f64]
  char* w = static_cast<char*>(work);
  J* gwork = reinterpret_cast<J*>(w);
  J* vout = gwork + 2 * (size_t)l * l;
  double* w64 = reinterpret_cast<double*>(w + ((3 * (size_t)l * l * sizeof(J) + 15) & ~(size_t)15));
  double* sig = w64 + (size_t)l * l;
  double* vn = sig + l;
  const size_t need = 2 * (size_t)l * l * sizeof(J);
  const int in_smem = need <= 200 * 1024 ? 1 : 0;
  cudaError_t e = cudaFuncSetAttribute(jacobi_sweep_kernel<J>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       200 * 1024);
  if (e != cudaSuccess) return e;
  jacobi_sweep_kernel<J><<<1, JT, in_smem ? need : 0, st>>>(M, l, vout, gwork, in_smem, status);
  jacobi_finish_kernel<J><<<l, 256, 0, st>>>(M, l, vout, w64, sig, vn);
  jacobi_order_kernel<J, TS><<<1, JT, 0, st>>>(l, k, w64, vout, sig, vn, (J*)Ut, (J*)Vt, (TS*)S);
  return cudaGetLastError();
}

}  // namespace

size_t jacobi_work_bytes(int l) {
  return ((3 * (size_t)l * l * sizeof(double) + 15) & ~(size_t)15) + (size_t)l * l * 8 + 2 * (size_t)l * 8;
}

cudaError_t launch_jacobi(const double* M, int l, int k, bool f64, void* Ut, void* Vt, void* S, bool S_f64,
                          void* work, DeviceStatus* status, cudaStream_t st) {
  if (f64) return run_all<double, double>(M, l, k, Ut, Vt, S, work, status, st);
  if (S_f64) return cudaErrorInvalidValue;
  return run_all<float, float>(M, l, k, Ut, Vt, S, work, status, st);
}

}  // namespace sorsvd
