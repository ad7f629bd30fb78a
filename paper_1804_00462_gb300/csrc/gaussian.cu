// Gaussian test matrix Omega (Sec. III: "a standard Gaussian matrix", first
// step of Algorithms 1 and 3), generated on the GPU from a counter-based RNG.
//
// Generator (published definitions, implemented here from scratch):
//   Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11): key (seed, 0),
//   counter (e / 4, stream_id, 0, 0) for column-major element e of Omega.
//   Each word x -> u = ((x >> 41) + 1/2) 2^-23, a binary32 value in (0, 1).
//   Box-Muller on (w0, w1) -> elements 4g, 4g+1 and (w2, w3) -> 4g+2, 4g+3:
//   z = sqrt(-2 ln u_a) * {cos, sin}(2 pi u_b).
// The transform runs in binary32 (GB300's binary64 rate is 1/64 of its
// binary32 rate): ln and sin/cos are series evaluated with one explicitly
// rounded IEEE operation per step (__fadd_rn / __fmul_rn / __fdiv_rn /
// __fsqrt_rn, which the compiler may not fuse), so the result depends only
// on IEEE-754 and is identical on any conforming implementation:
//   ln u : u = f 2^e, f in [sqrt(1/2), sqrt(2)); s = (f-1)/(f+1);
//          ln f = 2 s sum_{i=0}^{5} s^{2i}/(2i+1)  (atanh series, Horner in s^2)
//   2 pi u: t = 4u, q = rint(t), r = t - q, theta = r * pi/2;
//          sin, cos by Taylor series to theta^11 / theta^12 (Horner in theta^2),
//          then rotated by the quadrant q mod 4.
// Constants: the nearest binary32 values of ln 2, pi/2, sqrt(1/2) and of the
// series coefficients.
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

// ((x >> 41) + 1/2) 2^-23: both steps exact in binary32
__device__ __forceinline__ float unit_open(uint64_t x) {
  const float k = (float)(uint32_t)(x >> 41);       // < 2^23: exact
  return __fmul_rn(__fadd_rn(k, 0.5f), 0x1p-23f);
}

// 1/(2i+1), i = 0..5
__constant__ float kLogC[6] = {0x1p+0f, 0x1.555556p-2f, 0x1.99999ap-3f, 0x1.24924ap-3f, 0x1.c71c72p-4f,
                               0x1.745d18p-4f};
// (-1)^i / (2i+1)!, i = 1..5
__constant__ float kSinC[5] = {-0x1.555556p-3f, 0x1.111112p-7f, -0x1.a01a02p-13f, 0x1.71de3ap-19f,
                               -0x1.ae6456p-26f};
// (-1)^i / (2i)!, i = 1..6
__constant__ float kCosC[6] = {-0x1p-1f, 0x1.555556p-5f, -0x1.6c16c2p-10f, 0x1.a01a02p-16f, -0x1.27e4fcp-22f,
                               0x1.1eed8ep-29f};

__device__ __forceinline__ float ln_series(float u) {
  const float LN2 = 0x1.62e430p-1f, SQRT_HALF = 0x1.6a09e6p-1f;
  const uint32_t b = __float_as_uint(u);
  const int ex = (int)((b >> 23) & 0xFF) - 126;                     // u normal: u = fr 2^ex
  const float fr = __uint_as_float((b & 0x807FFFFFu) | (126u << 23));   // [0.5, 1)
  float f = fr;
  int e = ex;
  if (fr < SQRT_HALF) { f = __fmul_rn(fr, 2.0f); e = ex - 1; }
  const float s = __fdiv_rn(__fsub_rn(f, 1.0f), __fadd_rn(f, 1.0f));
  const float s2 = __fmul_rn(s, s);
  float p = kLogC[5];
#pragma unroll
  for (int i = 4; i >= 0; --i) p = __fadd_rn(__fmul_rn(p, s2), kLogC[i]);
  const float lnf = __fmul_rn(__fmul_rn(2.0f, s), p);
  return __fadd_rn(__fmul_rn((float)e, LN2), lnf);
}

__device__ __forceinline__ void sincos_2pi(float u, float* sn, float* cs) {
  const float HALF_PI = 0x1.921fb6p+0f;
  const float t = __fmul_rn(4.0f, u);
  const float q = rintf(t);
  const float r = __fsub_rn(t, q);
  const float th = __fmul_rn(r, HALF_PI);
  const float x2 = __fmul_rn(th, th);
  float ps = kSinC[4];
#pragma unroll
  for (int i = 3; i >= 0; --i) ps = __fadd_rn(__fmul_rn(ps, x2), kSinC[i]);
  const float s = __fadd_rn(th, __fmul_rn(__fmul_rn(th, x2), ps));
  float pc = kCosC[5];
#pragma unroll
  for (int i = 4; i >= 0; --i) pc = __fadd_rn(__fmul_rn(pc, x2), kCosC[i]);
  const float c = __fadd_rn(1.0f, __fmul_rn(x2, pc));
  const int quad = ((int)q) & 3;
  float sv, cv;
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
    float z[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float ua = unit_open(c[2 * h]), ub = unit_open(c[2 * h + 1]);
      const float r = __fsqrt_rn(__fmul_rn(-2.0f, ln_series(ua)));
      float sn, cs;
      sincos_2pi(ub, &sn, &cs);
      z[2 * h] = __fmul_rn(r, cs);
      z[2 * h + 1] = __fmul_rn(r, sn);
    }
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      int64_t e = 4 * g + h;
      if (e < total) {
        int64_t j = e / rows, i = e - j * rows;
        out[i + j * ld] = from_f32<T>(z[h]);
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
  // ALU bound (Philox's 64-bit products, the binary32 series): two blocks
  // per SM leave the SMs' other thread slots to a memory-bound kernel that
  // may run beside it (the transposed copy of A)
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
