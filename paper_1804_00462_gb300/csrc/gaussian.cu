// Gaussian test matrix Omega (Sec. III: "a standard Gaussian matrix", first
// step of Algorithms 1 and 3), generated on the GPU from a counter-based RNG.
//
// Generator (published definitions, implemented here from scratch):
//   Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): key (seed, 0),
//   counter (e / 4, stream_id, 0, 0) for column-major element e of Omega.
//   Each word x -> u = ((x >> 12) + 1/2) 2^-52 in (0, 1).
//   Box-Muller on (w0, w1) -> elements 4g, 4g+1 and (w2, w3) -> 4g+2, 4g+3:
//   z = sqrt(-2 ln u_a) * {cos, sin}(2 pi u_b).
// ln and sin/cos are series evaluated with one explicitly rounded IEEE
// operation per step (__dadd_rn / __dmul_rn / __ddiv_rn / __dsqrt_rn, which
// the compiler may not fuse), so the result depends only on IEEE-754 and is
// identical on any conforming implementation:
//   ln u : u = f 2^e, f in [sqrt(1/2), sqrt(2)); s = (f-1)/(f+1);
//          ln f = 2 s sum_{i=0}^{12} s^{2i}/(2i+1)  (atanh series, Horner in s^2)
//   2 pi u: t = 4u, q = rint(t), r = t - q, theta = r * pi/2;
//          sin, cos by Taylor series to theta^19 / theta^18 (Horner in theta^2),
//          then rotated by the quadrant q mod 4.
#include "internal.cuh"

#include <algorithm>

namespace sorsvd {
namespace {

__device__ __forceinline__ void philox4x64_10(uint64_t c[4], uint64_t k0, uint64_t k1) {
  const uint64_t M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
  const uint64_t W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k0 += W0; k1 += W1; }
    uint64_t hi0 = __umul64hi(M0, c[0]), lo0 = M0 * c[0];
    uint64_t hi1 = __umul64hi(M1, c[2]), lo1 = M1 * c[2];
    uint64_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
  }
}

__device__ __forceinline__ double unit_open(uint64_t x) {
  double v = __ull2double_rn(x >> 12);           // exact: < 2^52
  return __dmul_rn(__dadd_rn(v, 0.5), 0x1p-52);   // both exact
}

// 1/(2i+1), i = 0..12 (each a correctly rounded quotient of exact integers)
__constant__ double kLogC[13] = {1.0 / 1.0, 1.0 / 3.0, 1.0 / 5.0, 1.0 / 7.0, 1.0 / 9.0,
                                 1.0 / 11.0, 1.0 / 13.0, 1.0 / 15.0, 1.0 / 17.0, 1.0 / 19.0,
                                 1.0 / 21.0, 1.0 / 23.0, 1.0 / 25.0};
// (-1)^i / (2i+1)!, i = 1..9
__constant__ double kSinC[9] = {-(1.0 / 6.0), 1.0 / 120.0, -(1.0 / 5040.0), 1.0 / 362880.0,
                                -(1.0 / 39916800.0), 1.0 / 6227020800.0, -(1.0 / 1307674368000.0),
                                1.0 / 355687428096000.0, -(1.0 / 121645100408832000.0)};
// (-1)^i / (2i)!, i = 1..9
__constant__ double kCosC[9] = {-(1.0 / 2.0), 1.0 / 24.0, -(1.0 / 720.0), 1.0 / 40320.0,
                                -(1.0 / 3628800.0), 1.0 / 479001600.0, -(1.0 / 87178291200.0),
                                1.0 / 20922789888000.0, -(1.0 / 6402373705728000.0)};

__device__ __forceinline__ double ln_series(double u) {
  const double LN2 = 0.6931471805599453, SQRT_HALF = 0.7071067811865476;
  long long b = __double_as_longlong(u);
  int ex = (int)((b >> 52) & 0x7FF) - 1022;                       // u normal
  double fr = __longlong_as_double((b & 0x800FFFFFFFFFFFFFll) | (1022ll << 52));  // [0.5, 1)
  double f = fr;
  int e = ex;
  if (fr < SQRT_HALF) { f = __dmul_rn(fr, 2.0); e = ex - 1; }
  double s = __ddiv_rn(__dsub_rn(f, 1.0), __dadd_rn(f, 1.0));
  double s2 = __dmul_rn(s, s);
  double p = kLogC[12];
#pragma unroll
  for (int i = 11; i >= 0; --i) p = __dadd_rn(__dmul_rn(p, s2), kLogC[i]);
  double lnf = __dmul_rn(__dmul_rn(2.0, s), p);
  return __dadd_rn(__dmul_rn((double)e, LN2), lnf);
}

__device__ __forceinline__ void sincos_2pi(double u, double* sn, double* cs) {
  const double HALF_PI = 1.5707963267948966;
  double t = __dmul_rn(4.0, u);
  double q = rint(t);
  double r = __dsub_rn(t, q);
  double th = __dmul_rn(r, HALF_PI);
  double x2 = __dmul_rn(th, th);
  double ps = kSinC[8];
#pragma unroll
  for (int i = 7; i >= 0; --i) ps = __dadd_rn(__dmul_rn(ps, x2), kSinC[i]);
  double s = __dadd_rn(th, __dmul_rn(__dmul_rn(th, x2), ps));
  double pc = kCosC[8];
#pragma unroll
  for (int i = 7; i >= 0; --i) pc = __dadd_rn(__dmul_rn(pc, x2), kCosC[i]);
  double c = __dadd_rn(1.0, __dmul_rn(x2, pc));
  int quad = ((int)q) & 3;
  double sv, cv;
  if (quad == 0) { sv = s; cv = c; }
  else if (quad == 1) { sv = c; cv = -s; }
  else if (quad == 2) { sv = -s; cv = -c; }
  else { sv = -c; cv = s; }
  *sn = sv;
  *cs = cv;
}

template <typename T>
__device__ __forceinline__ void gaussian_body(T* __restrict__ out, int64_t rows, int64_t cols, int64_t ld,
                                              uint64_t seed, uint64_t stream_id) {
  const int64_t total = rows * cols;
  const int64_t groups = (total + 3) / 4;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < groups;
       g += (int64_t)gridDim.x * blockDim.x) {
    uint64_t c[4] = {(uint64_t)g, stream_id, 0ull, 0ull};
    philox4x64_10(c, seed, 0ull);
    double z[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double ua = unit_open(c[2 * h]), ub = unit_open(c[2 * h + 1]);
      double r = __dsqrt_rn(__dmul_rn(-2.0, ln_series(ua)));
      double sn, cs;
      sincos_2pi(ub, &sn, &cs);
      z[2 * h] = __dmul_rn(r, cs);
      z[2 * h + 1] = __dmul_rn(r, sn);
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      int64_t e = 4 * g + h;
      if (e < total) {
        int64_t j = e / rows, i = e - j * rows;
        out[i + j * ld] = from_f64<T>(z[h]);
      }
    }
  }
}

template <typename T>
__global__ void gaussian_kernel(T* __restrict__ out, int64_t rows, int64_t cols, int64_t ld,
                                uint64_t seed, uint64_t stream_id) {
  gaussian_body<T>(out, rows, cols, ld, seed, stream_id);
}

// blockIdx.y = job; Omega of each problem from stream 0
template <typename T>
__global__ void gaussian_batched_kernel(const GaussJob* __restrict__ jobs) {
  const GaussJob& j = jobs[blockIdx.y];
  gaussian_body<T>((T*)j.out, j.rows, j.cols, j.ld, j.seed, 0ull);
}

}  // namespace

cudaError_t launch_gaussian(void* out, int64_t rows, int64_t cols, int64_t ld, uint64_t seed,
                            uint64_t stream_id, int dtype, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  int64_t groups = (rows * cols + 3) / 4;
  int threads = 256;
  int64_t blocks = (groups + threads - 1) / threads;
  // binary64-ALU bound: two blocks per SM keep the FP64 pipes busy and
  // leave the SMs' other thread slots to a memory-bound kernel beside it
  int cap = num_sms() * 2;
  if (blocks > cap) blocks = cap;
  switch (dtype) {
    case SORSVD_F64: gaussian_kernel<double><<<(int)blocks, threads, 0, st>>>((double*)out, rows, cols, ld, seed, stream_id); break;
    case SORSVD_F32: case SORSVD_TF32: gaussian_kernel<float><<<(int)blocks, threads, 0, st>>>((float*)out, rows, cols, ld, seed, stream_id); break;
    case SORSVD_BF16: gaussian_kernel<bf16><<<(int)blocks, threads, 0, st>>>((bf16*)out, rows, cols, ld, seed, stream_id); break;
    case SORSVD_F16: gaussian_kernel<f16><<<(int)blocks, threads, 0, st>>>((f16*)out, rows, cols, ld, seed, stream_id); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_gaussian_batched(const GaussJob* jobs, int njobs, int64_t max_elems, int dtype,
                                    cudaStream_t st) {
  if (njobs <= 0 || max_elems <= 0) return cudaSuccess;
  const int64_t groups = (max_elems + 3) / 4;
  const int64_t bx = std::min<int64_t>((groups + 255) / 256, 64);
  dim3 grid((unsigned)bx, (unsigned)njobs);
  switch (dtype) {
    case SORSVD_F64: gaussian_batched_kernel<double><<<grid, 256, 0, st>>>(jobs); break;
    case SORSVD_F32: case SORSVD_TF32: gaussian_batched_kernel<float><<<grid, 256, 0, st>>>(jobs); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace sorsvd
