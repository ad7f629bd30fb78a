// Truncated SVD of the small core matrix M (l x l) of Algorithm 3
// ("compute the rank-k truncated SVD of M").  One-sided (Hestenes) Jacobi:
// columns w_p, w_q of W = M V are rotated until every pair is orthogonal to
// a relative tolerance; then sigma_j = ||w_j||, U~ = W diag(sigma)^{-1}.
//
// Pair schedule: round-robin tournament (circle method) - in each of the
// N - 1 rounds (N = l rounded up to even) the N/2 disjoint pairs are
// independent, so each warp of the block rotates its pairs concurrently and
// one __syncthreads separates rounds.  Ordering of the results: sigma
// descending (ties by column index); sign: the largest-magnitude entry of
// each column of U~ is made positive and the matching column of V~ follows.
//
// W and V live in shared memory when 2 l^2 words fit, else in the caller's
// global work buffer (same code through generic pointers).  The sweep count
// is capped; hitting the cap raises SORSVD_ERR_NOT_CONVERGED.
#include "internal.cuh"

namespace sorsvd {
namespace {

constexpr int JT = 1024;
constexpr int kMaxSweeps = 40;

__device__ __forceinline__ int rr_player(int pos, int round, int N) {
  // position 0 is fixed; positions 1..N-1 rotate by one place per round
  if (pos == 0) return 0;
  int x = (pos - 1 - round) % (N - 1);
  if (x < 0) x += N - 1;
  return 1 + x;
}

template <typename J>
__device__ __forceinline__ J warp_sum(J v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename J, typename TS>
__global__ void __launch_bounds__(JT)
jacobi_kernel(const double* __restrict__ Min, int l, int k, J* __restrict__ Ut, J* __restrict__ Vt,
              TS* __restrict__ S, J* __restrict__ gwork, int in_smem, DeviceStatus* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int s_rot;
  J* W;
  J* V;
  if (in_smem) { W = reinterpret_cast<J*>(smem_raw); V = W + (size_t)l * l; }
  else { W = gwork; V = gwork + (size_t)l * l; }
  // small per-column arrays always in shared memory (l <= SORSVD_MAX_L)
  __shared__ double s_sig[SORSVD_MAX_L];
  __shared__ int s_order[SORSVD_MAX_L];

  const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nwarps = JT / 32;
  const J eps = sizeof(J) == 8 ? (J)2.220446049250313e-16 : (J)1.1920928955078125e-07;
  const J tol = (J)(l > 32 ? l : 32) * eps;

  for (int e = t; e < l * l; e += JT) {
    W[e] = (J)Min[e];
    V[e] = (e % l == e / l) ? (J)1 : (J)0;
  }
  __syncthreads();

  const int N = (l + 1) & ~1;
  int sweep = 0;
  for (sweep = 1; sweep <= kMaxSweeps; ++sweep) {
    if (t == 0) s_rot = 0;
    __syncthreads();
    for (int r = 0; r < N - 1; ++r) {
      for (int pr = warp; pr < N / 2; pr += nwarps) {
        int a = rr_player(pr, r, N), b = rr_player(N - 1 - pr, r, N);
        if (a >= l || b >= l) continue;            // bye
        int p = min(a, b), q = max(a, b);
        J* wp = W + (size_t)p * l;
        J* wq = W + (size_t)q * l;
        J al = 0, be = 0, ga = 0;
        for (int i = lane; i < l; i += 32) {
          J x = wp[i], y = wq[i];
          al += x * x; be += y * y; ga += x * y;
        }
        al = warp_sum(al); be = warp_sum(be); ga = warp_sum(ga);
        if (!(ga != (J)0) || !(fabs(ga) > tol * sqrt(al * be))) continue;
        J zeta = (be - al) / ((J)2 * ga);
        J az = fabs(zeta);
        J root = az > (J)1 ? az * sqrt((J)1 + ((J)1 / az) * ((J)1 / az)) : sqrt((J)1 + az * az);
        J tt = (zeta >= (J)0 ? (J)1 : (J)-1) / (az + root);
        J cs = (J)1 / sqrt((J)1 + tt * tt);
        J sn = cs * tt;
        for (int i = lane; i < l; i += 32) {
          J x = wp[i], y = wq[i];
          wp[i] = cs * x - sn * y;
          wq[i] = sn * x + cs * y;
        }
        J* vp = V + (size_t)p * l;
        J* vq = V + (size_t)q * l;
        for (int i = lane; i < l; i += 32) {
          J x = vp[i], y = vq[i];
          vp[i] = cs * x - sn * y;
          vq[i] = sn * x + cs * y;
        }
        if (lane == 0) s_rot = 1;
      }
      __syncthreads();
    }
    int rot = s_rot;
    __syncthreads();
    if (!rot) break;
  }
  if (sweep > kMaxSweeps) {
    if (t == 0) raise_status(status, SORSVD_ERR_NOT_CONVERGED);
    sweep = kMaxSweeps;
  }
  if (t == 0) atomicOr(&status->info, (min(sweep, 255)) << 8);

  for (int c = warp; c < l; c += nwarps) {
    J s = 0;
    for (int i = lane; i < l; i += 32) { J x = W[(size_t)c * l + i]; s += x * x; }
    s = warp_sum(s);
    if (lane == 0) s_sig[c] = sqrt((double)s);
  }
  __syncthreads();
  for (int c = t; c < l; c += JT) {
    double sc = s_sig[c];
    int rank = 0;
    for (int d = 0; d < l; ++d) {
      double sd = s_sig[d];
      rank += (sd > sc) || (sd == sc && d < c);
    }
    s_order[rank] = c;
  }
  __syncthreads();
  for (int j = warp; j < l; j += nwarps) {
    int c = s_order[j];
    double sg = s_sig[c];
    J inv = sg > 0.0 ? (J)(1.0 / sg) : (J)0;
    const J* wc = W + (size_t)c * l;
    // sign: largest |U~(i, j)| positive (first index on ties)
    J best = -1;
    int bi = l;
    for (int i = lane; i < l; i += 32) {
      J v = fabs(wc[i]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      J ob = __shfl_xor_sync(0xffffffffu, best, o);
      int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    J sgn = (bi < l && wc[bi] < (J)0) ? (J)-1 : (J)1;
    for (int i = lane; i < l; i += 32) {
      Ut[(size_t)j * l + i] = sgn * wc[i] * inv;
      Vt[(size_t)j * l + i] = sgn * V[(size_t)c * l + i];
    }
    if (lane == 0 && j < k) S[j] = (TS)sg;
  }
}

}  // namespace

cudaError_t launch_jacobi(const double* M, int l, int k, bool f64, void* Ut, void* Vt, void* S, bool S_f64,
                          void* work, DeviceStatus* status, cudaStream_t st) {
  size_t word = f64 ? 8 : 4;
  size_t need = 2 * (size_t)l * l * word;
  int in_smem = need <= 200 * 1024 ? 1 : 0;
  size_t sm = in_smem ? need : 0;
  cudaError_t e;
  if (f64) {
    e = cudaFuncSetAttribute(jacobi_kernel<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(200 * 1024));
    if (e != cudaSuccess) return e;
    jacobi_kernel<double, double><<<1, JT, sm, st>>>(M, l, k, (double*)Ut, (double*)Vt, (double*)S, (double*)work, in_smem, status);
  } else if (S_f64) {
    return cudaErrorInvalidValue;
  } else {
    e = cudaFuncSetAttribute(jacobi_kernel<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(200 * 1024));
    if (e != cudaSuccess) return e;
    jacobi_kernel<float, float><<<1, JT, sm, st>>>(M, l, k, (float*)Ut, (float*)Vt, (float*)S, (float*)work, in_smem, status);
  }
  return cudaGetLastError();
}

}  // namespace sorsvd
