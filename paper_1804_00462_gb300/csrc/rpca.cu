// Robust PCA by the inexact augmented Lagrange multiplier method with
// SOR-SVD as the low-rank step (Sec. V-C, Table 3): X = L + S with L of low
// rank and S sparse.  Per iteration, with mu_j the penalty and
// lambda = 1 / sqrt(max(m, n)):
//   (U, Z, V) = SOR-SVD_k(G_j),   G_j = X - S_j + Y_j / mu_j
//   L_{j+1}   = U shrink_{1/mu_j}(Z) V^T
//   S_{j+1}   = shrink_{lambda/mu_j}(X - L_{j+1} + Y_j / mu_j)
//   Y_{j+1}   = Y_j + mu_j (X - L_{j+1} - S_{j+1})
//   mu_{j+1}  = min(rho mu_j, 1e7 mu_0)
// until ||X - L - S||_F < tol ||X||_F.  Readings where the paper is silent:
// the cap of mu is a minimum (the table prints a maximum), and the initial
// values follow the usual inexact-ALM choice Y_0 = X / max(||X||_2,
// ||X||_inf / lambda), mu_0 = 1.25 / ||X||_2, S_0 = 0; the SOR-SVD of
// iteration j (1-based) draws its Gaussian matrix from seed + j - 1.
//
// GPU design.  The state lives in HBM in fp32: S (the caller's output), Y
// and G (workspace).  L is never stored during the loop: one fused
// elementwise kernel per iteration recomputes L_{j+1}(i, c) from the rank-k
// factors (U, shrunk Z, V, a few hundred KB that stay in L2), forms S, the
// residual R, Y and the next SOR-SVD input G in one read of X, Y and one
// write of S, Y, G (5 fp32 arrays per iteration), and leaves per-block
// partial sums of ||R||_F^2 for a fixed-order reduction (deterministic).
// The elementwise arithmetic is double-float (pairs of fp32 with Knuth's
// TwoSum and the fma-based exact product): X - L - S stored in fp32 loses
// about one fp32 ulp of |X| per element, which plain fp32 arithmetic would
// put at ~1e-7 relative - the stopping tolerance; error-free pairs keep the
// residual's own error at the rounding of the stored S.  The loop is driven
// from the host: mu_j is data-independent, and the only value read back per
// iteration is ||R||_F^2 (and the SOR-SVD status word).
#include "internal.cuh"
#include "profile.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace sorsvd {
namespace {

constexpr int kEwThreads = 256;
constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }
inline int64_t pad16(int64_t x) { return (x + 15) / 16 * 16; }

// ------------------------------------------------------------ double-float
struct df { float hi, lo; };

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ df fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ df df_add(df x, df y) {
  df s = two_sum(x.hi, y.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_add_f(df x, float b) {
  df s = two_sum(x.hi, b);
  s.lo = __fadd_rn(s.lo, x.lo);
  return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ df df_mul_f(df x, float b) {
  df p = two_prod(x.hi, b);
  p.lo = __fmaf_rn(x.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ df df_neg(df x) { return {-x.hi, -x.lo}; }

struct DfScalar { float hi, lo; };
DfScalar to_df(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}

// ------------------------------------------------------------ kernels
// Per-block partials of sum(X^2) (binary64) and max |X|.
__global__ void rpca_stats_kernel(const float* __restrict__ X, int64_t m, int64_t n, int64_t ldx,
                                  double* __restrict__ part) {
  __shared__ double ssum[kEwThreads];
  __shared__ float smax[kEwThreads];
  double s = 0.0;
  float mx = 0.f;
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / m, r = e - c * m;
    const float x = X[r + c * ldx];
    s += (double)x * (double)x;
    mx = fmaxf(mx, fabsf(x));
  }
  ssum[threadIdx.x] = s;
  smax[threadIdx.x] = mx;
  __syncthreads();
  for (int w = kEwThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      ssum[threadIdx.x] += ssum[threadIdx.x + w];
      smax[threadIdx.x] = fmaxf(smax[threadIdx.x], smax[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = ssum[0];
    part[2 * blockIdx.x + 1] = (double)smax[0];
  }
}

// Fixed-order reduction of `nblk` partials (stride `stride`): out[0] = sum of
// field 0, out[1] = max of field 1 (when stride == 2).
__global__ void rpca_reduce_kernel(const double* __restrict__ part, int nblk, int stride, double* __restrict__ out) {
  __shared__ double ssum[kEwThreads], smax[kEwThreads];
  double s = 0.0, mx = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    s += part[(size_t)b * stride];
    if (stride > 1) mx = fmax(mx, part[(size_t)b * stride + 1]);
  }
  ssum[threadIdx.x] = s;
  smax[threadIdx.x] = mx;
  __syncthreads();
  for (int w = kEwThreads / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      ssum[threadIdx.x] += ssum[threadIdx.x + w];
      smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + w]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = ssum[0];
    if (stride > 1) out[1] = smax[0];
  }
}

// Y_0 = c X, S_0 = 0, G_1 = X + Y_0 / mu_0 (fp32 into G, or binary64 into G64)
__global__ void rpca_init_kernel(const float* __restrict__ X, int64_t m, int64_t n, int64_t ldx, float c,
                                 DfScalar inv_mu, float* __restrict__ Y, float* __restrict__ S, int64_t lds,
                                 float* __restrict__ G, double* __restrict__ G64, int64_t ldg) {
  const int64_t total = m * n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / m, r = e - col * m;
    const float x = X[r + col * ldx];
    const float y = __fmul_rn(c, x);
    const df g = df_add_f(df_mul_f(df{inv_mu.hi, inv_mu.lo}, y), x);
    Y[r + col * ldg] = y;
    S[r + col * lds] = 0.f;
    if (G) G[r + col * ldg] = g.hi;
    if (G64) G64[r + col * ldg] = (double)g.hi + (double)g.lo;
  }
}

// shrink_{1/mu}(Z), in double-float, for the k singular values
__device__ __forceinline__ df shrink_sv(float z, DfScalar inv_mu) {
  // z >= 0: max(z - 1/mu, 0)
  const df d = df_add_f(df_neg(df{inv_mu.hi, inv_mu.lo}), z);
  return (d.hi > 0.f) ? d : df{0.f, 0.f};
}

constexpr int kMaxRank = SORSVD_MAX_L;

struct UpdParams {
  const float* X; int64_t ldx;
  float* Y; int64_t ldg;
  float* G;              // next SOR-SVD input, fp32 (or null)
  double* G64;           // the same in binary64 (or null)
  float* S; int64_t lds;
  const void* U; int64_t ldu;   // factors: fp32, or binary64 when f64
  const void* V; int64_t ldv;
  const void* Z;
  int f64;
  int64_t m, n;
  int k;
  DfScalar inv_mu, thr, mu, inv_mu_next;
  double inv_mu_d;
  double* part;
  const int* status_in;  // device status code of the inner SOR-SVD
  double* res;           // res[1] <- that code (res[0]: ||R||_F^2, reduced later)
};

// shrunk singular values in shared memory, for both factor precisions
struct ShrunkZ {
  df f[kMaxRank];
  double d[kMaxRank];
};
__device__ __forceinline__ void load_shrunk(const UpdParams& P, ShrunkZ& z) {
  for (int t = threadIdx.x; t < P.k; t += blockDim.x) {
    if (P.f64) z.d[t] = fmax(((const double*)P.Z)[t] - P.inv_mu_d, 0.0);
    else z.f[t] = shrink_sv(((const float*)P.Z)[t], P.inv_mu);
  }
}

// L(r, c) = sum_t U(r, t) w_t with w_t = shrink(Z_t) V(c, t): double-float
// for fp32 factors, binary64 for binary64 factors
__device__ __forceinline__ df lowrank_at(const UpdParams& P, const ShrunkZ& z, int64_t r, int64_t col) {
  if (P.f64) {
    const double* U = (const double*)P.U;
    const double* V = (const double*)P.V;
    double l = 0.0;
    for (int t = 0; t < P.k; ++t) l = fma(U[r + (int64_t)t * P.ldu], z.d[t] * V[col + (int64_t)t * P.ldv], l);
    const float h = __double2float_rn(l);
    return df{h, __double2float_rn(l - (double)h)};
  }
  const float* U = (const float*)P.U;
  const float* V = (const float*)P.V;
  df l{0.f, 0.f};
  for (int t = 0; t < P.k; ++t) {
    const float v = V[col + (int64_t)t * P.ldv];
    const df p = two_prod(z.f[t].hi, v);
    const df wt{p.hi, __fmaf_rn(z.f[t].lo, v, p.lo)};
    const float u = U[r + (int64_t)t * P.ldu];
    const df q = two_prod(wt.hi, u);
    l = df_add(l, df{q.hi, __fmaf_rn(wt.lo, u, q.lo)});
  }
  return l;
}

// One ALM iteration after the SOR-SVD (see the file comment); one thread
// per element, grid-stride over the column-major index.
__global__ void __launch_bounds__(kEwThreads) rpca_update_kernel(const UpdParams P) {
  __shared__ ShrunkZ zs;
  __shared__ double ssum[kEwThreads];
  load_shrunk(P, zs);
  __syncthreads();
  const df inv_mu{P.inv_mu.hi, P.inv_mu.lo}, thr{P.thr.hi, P.thr.lo}, mu{P.mu.hi, P.mu.lo};
  const df inv_mu_next{P.inv_mu_next.hi, P.inv_mu_next.lo};
  double acc = 0.0;
  const int64_t total = P.m * P.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / P.m, r = e - col * P.m;
    const df l = lowrank_at(P, zs, r, col);
    const float x = P.X[r + col * P.ldx];
    const float y = P.Y[r + col * P.ldg];
    // a = X - L + Y / mu
    const df xl = df_add_f(df_neg(l), x);
    const df yq = df_mul_f(inv_mu, y);
    const df a = df_add(xl, yq);
    // S = shrink_{lambda/mu}(a), stored in fp32
    float s = 0.f;
    if (a.hi > thr.hi || (a.hi == thr.hi && a.lo > thr.lo)) s = df_add(a, df_neg(thr)).hi;
    else if (-a.hi > thr.hi || (-a.hi == thr.hi && -a.lo > thr.lo)) s = df_add(a, thr).hi;
    // R = X - L - S (with the stored S)
    const df rr = df_add_f(xl, -s);
    // Y += mu R
    const df mr = df_add(df_mul_f(mu, rr.hi), df_mul_f(mu, rr.lo));
    const float ynew = df_add_f(mr, y).hi;
    // G = X - S + Y / mu_next
    const df g = df_add(two_sum(x, -s), df_mul_f(inv_mu_next, ynew));
    P.S[r + col * P.lds] = s;
    P.Y[r + col * P.ldg] = ynew;
    if (P.G) P.G[r + col * P.ldg] = g.hi;
    if (P.G64) P.G64[r + col * P.ldg] = (double)g.hi + (double)g.lo;
    const double rd = (double)rr.hi + (double)rr.lo;
    acc = fma(rd, rd, acc);
  }
  ssum[threadIdx.x] = acc;
  __syncthreads();
  for (int wdt = kEwThreads / 2; wdt > 0; wdt >>= 1) {
    if ((int)threadIdx.x < wdt) ssum[threadIdx.x] += ssum[threadIdx.x + wdt];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.part[blockIdx.x] = ssum[0];
    if (blockIdx.x == 0) P.res[1] = (double)*P.status_in;
  }
}

// L = U shrink_{1/mu}(Z) V^T, rounded once to fp32
__global__ void __launch_bounds__(kEwThreads) rpca_lowrank_kernel(const UpdParams P, float* __restrict__ L,
                                                                  int64_t ldl) {
  __shared__ ShrunkZ zs;
  load_shrunk(P, zs);
  __syncthreads();
  const int64_t total = P.m * P.n;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / P.m, r = e - col * P.m;
    L[r + col * ldl] = lowrank_at(P, zs, r, col).hi;
  }
}

// ------------------------------------------------------------ host side
struct RpcaLayout {
  int64_t ldg, ldu, ldv;
  size_t ws, G, G64, Y, U, V, Z, part, total;
  size_t ws_bytes;
};

int ew_blocks(int64_t total) {
  int64_t b = (total + kEwThreads - 1) / kEwThreads;
  const int64_t cap = (int64_t)num_sms() * 8;
  return (int)std::max<int64_t>(1, std::min(b, cap));
}
int max_ew_blocks() { return num_sms() * 8; }

// parameters of the ||X||_2 estimate when the caller does not supply it
constexpr int kNormK = 1, kNormQ = 2;
inline int norm_p(int64_t m, int64_t n) {
  return (int)std::max<int64_t>(0, std::min<int64_t>(9, std::min(m, n) - 1 - kNormK));
}
// FINISH_F64: binary64 SOR-SVD once ||R||_F / ||X||_F < kSwitch * tol
constexpr double kSwitch = 30.0;

inline bool uses_f64(int dt, unsigned flags) { return dt == SORSVD_F64 || (flags & SORSVD_RPCA_FINISH_F64); }
inline bool uses_f32(int dt) { return dt != SORSVD_F64; }

bool rpca_layout(const sorsvd_rpca_problem& P, int k, int p, int dt, unsigned flags, RpcaLayout* out) {
  RpcaLayout L{};
  L.ldg = pad16(P.m);
  L.ldu = pad16(P.m);
  L.ldv = pad16(P.n);
  if (k < 1 || k > kMaxRank) return false;
  size_t w = 0;
  if (uses_f32(dt)) {
    const size_t w1 = sorsvd_workspace_size(P.m, P.n, k, p, dt, 0);
    if (w1 == 0) return false;
    w = std::max(w, w1);
  }
  if (uses_f64(dt, flags)) {
    const size_t w1 = sorsvd_workspace_size(P.m, P.n, k, p, SORSVD_F64, 0);
    if (w1 == 0) return false;
    w = std::max(w, w1);
  }
  if (!(P.norm2 > 0.0)) {
    const size_t w2 = sorsvd_workspace_size(P.m, P.n, kNormK, norm_p(P.m, P.n), SORSVD_F32, 0);
    if (w2 == 0) return false;
    w = std::max(w, w2);
  }
  const size_t fsz = uses_f64(dt, flags) ? 8 : 4;     // factor buffers hold either precision
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  L.ws_bytes = w;
  L.ws = take(L.ws_bytes);
  L.G = uses_f32(dt) ? take((size_t)L.ldg * P.n * 4) : 0;
  L.G64 = uses_f64(dt, flags) ? take((size_t)L.ldg * P.n * 8) : 0;
  L.Y = take((size_t)L.ldg * P.n * 4);
  L.U = take((size_t)L.ldu * k * fsz);
  L.V = take((size_t)L.ldv * k * fsz);
  L.Z = take((size_t)k * fsz);
  L.part = take((size_t)max_ew_blocks() * 2 * sizeof(double));
  L.total = off;
  *out = L;
  return true;
}

// bytes of the batch header: 2 doubles per problem, read back every iteration
inline size_t header_bytes(int batch) { return align_up((size_t)batch * 2 * sizeof(double)); }

int check_problem(const sorsvd_rpca_problem& P) {
  if (!P.X || !P.L || !P.S) return SORSVD_ERR_ARG;
  if (P.m < 2 || P.n < 2) return SORSVD_ERR_ARG;
  if (P.ldx < P.m || P.ldl < P.m || P.lds < P.m) return SORSVD_ERR_ARG;
  if (P.norm2 != P.norm2) return SORSVD_ERR_ARG;   // NaN
  return SORSVD_OK;
}

inline bool dtype_ok(int dt) { return dt == SORSVD_F32 || dt == SORSVD_TF32 || dt == SORSVD_F64; }

#define CKR(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return SORSVD_ERR_CUDA; } while (0)

}  // namespace
}  // namespace sorsvd

using namespace sorsvd;

extern "C" size_t sorsvd_rpca_workspace_size(const sorsvd_rpca_problem* probs, int batch, int k, int p, int dtype,
                                             unsigned flags) {
  if (!probs || batch < 1 || !dtype_ok(dtype) || (flags & ~SORSVD_RPCA_FINISH_F64)) return 0;
  size_t total = header_bytes(batch);
  for (int b = 0; b < batch; ++b) {
    if (check_problem(probs[b]) != SORSVD_OK) return 0;
    RpcaLayout L;
    if (!rpca_layout(probs[b], k, p, dtype, flags, &L)) return 0;
    total += align_up(L.total);
  }
  return total;
}

extern "C" int sorsvd_rpca(const sorsvd_rpca_problem* probs, int batch, int k, int p, int q, int dtype,
                           unsigned flags, double tol, int max_iter, double rho, int* iters, double* xi,
                           double* xi_history, void* workspace, size_t ws_bytes, void* stream) {
  if (!dtype_ok(dtype)) return SORSVD_ERR_DTYPE;
  if (!probs || batch < 1 || !iters || !xi) return SORSVD_ERR_ARG;
  if (flags & ~SORSVD_RPCA_FINISH_F64) return SORSVD_ERR_ARG;
  if (!(tol > 0.0) || max_iter < 1 || !(rho >= 1.0) || q < 0) return SORSVD_ERR_ARG;
  for (int b = 0; b < batch; ++b)
    if (int r = check_problem(probs[b])) return r;
  const size_t need = sorsvd_rpca_workspace_size(probs, batch, k, p, dtype, flags);
  if (need == 0) return SORSVD_ERR_ARG;
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < need) return SORSVD_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  char* base = (char*)workspace;
  double* res = (double*)base;       // res[2b]: ||R||_F^2 (or ||X||_F^2), res[2b+1]: status (or ||X||_inf)

  struct State {
    RpcaLayout L;
    char* w;
    double mu, mu_bar, lam, nx, mu_used, xi_prev;
    bool active, g64, svd64;
  };
  std::vector<State> S(batch);
  size_t off = header_bytes(batch);
  for (int b = 0; b < batch; ++b) {
    rpca_layout(probs[b], k, p, dtype, flags, &S[b].L);
    S[b].w = base + off;
    off += align_up(S[b].L.total);
  }
  auto at = [&](int b, size_t o) { return (void*)(S[b].w + o); };

  // ||X||_F^2 and ||X||_inf of every problem, then (when not supplied) ||X||_2
  std::vector<double> host(2 * (size_t)batch, 0.0), nrm2(batch, 0.0);
  for (int b = 0; b < batch; ++b) {
    const sorsvd_rpca_problem& P = probs[b];
    const int nb = ew_blocks(P.m * P.n);
    double* part = (double*)at(b, S[b].L.part);
    {
      ProfScope ps(K_RPCA, st);
      rpca_stats_kernel<<<nb, kEwThreads, 0, st>>>(P.X, P.m, P.n, P.ldx, part);
      CKR(cudaGetLastError());
    }
    ProfScope ps(K_REDUCE, st);
    rpca_reduce_kernel<<<1, kEwThreads, 0, st>>>(part, nb, 2, res + 2 * b);
    CKR(cudaGetLastError());
  }
  CKR(cudaMemcpyAsync(host.data(), res, host.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
  CKR(cudaStreamSynchronize(st));
  for (int b = 0; b < batch; ++b) {
    const sorsvd_rpca_problem& P = probs[b];
    nrm2[b] = P.norm2;
    if (P.norm2 > 0.0 || !(host[2 * b] > 0.0)) continue;
    int r = sorsvd_run(P.X, P.m, P.n, P.ldx, kNormK, norm_p(P.m, P.n), kNormQ, P.seed ^ 0x9E3779B97F4A7C15ull,
                       SORSVD_F32, 0, at(b, S[b].L.U), S[b].L.ldu, at(b, S[b].L.Z), at(b, S[b].L.V), S[b].L.ldv,
                       at(b, S[b].L.ws), S[b].L.ws_bytes, st);
    if (r) return r;
    float s1 = 0.f;
    CKR(cudaMemcpyAsync(&s1, at(b, S[b].L.Z), sizeof(float), cudaMemcpyDeviceToHost, st));
    int dst = 0;
    CKR(cudaMemcpyAsync(&dst, workspace_status(at(b, S[b].L.ws)), sizeof(int), cudaMemcpyDeviceToHost, st));
    CKR(cudaStreamSynchronize(st));
    if (dst) return dst;
    nrm2[b] = (double)s1;
  }

  int n_active = 0;
  for (int b = 0; b < batch; ++b) {
    const sorsvd_rpca_problem& P = probs[b];
    State& s = S[b];
    s.nx = std::sqrt(host[2 * b]);
    const double ninf = host[2 * b + 1];
    s.lam = 1.0 / std::sqrt((double)std::max(P.m, P.n));
    iters[b] = 0;
    xi[b] = 0.0;
    s.active = false;
    s.xi_prev = 1.0;
    if (!(s.nx > 0.0) || !(nrm2[b] > 0.0)) {
      // X = 0: L = S = 0 is exact
      CKR(cudaMemset2DAsync(P.L, P.ldl * 4, 0, P.m * 4, P.n, st));
      CKR(cudaMemset2DAsync(P.S, P.lds * 4, 0, P.m * 4, P.n, st));
      continue;
    }
    const double c = 1.0 / std::max(nrm2[b], ninf / s.lam);
    s.mu = 1.25 / nrm2[b];
    s.mu_bar = s.mu * 1e7;
    s.active = true;
    s.g64 = (dtype == SORSVD_F64);
    ++n_active;
    ProfScope ps(K_RPCA, st);
    rpca_init_kernel<<<ew_blocks(P.m * P.n), kEwThreads, 0, st>>>(
        P.X, P.m, P.n, P.ldx, (float)c, to_df(1.0 / s.mu), (float*)at(b, s.L.Y), P.S,
        P.lds, s.g64 ? nullptr : (float*)at(b, s.L.G), s.g64 ? (double*)at(b, s.L.G64) : nullptr, s.L.ldg);
    CKR(cudaGetLastError());
  }

  auto factors = [&](int b, UpdParams& U) {
    const sorsvd_rpca_problem& P = probs[b];
    const State& s = S[b];
    U.U = at(b, s.L.U); U.ldu = s.L.ldu;
    U.V = at(b, s.L.V); U.ldv = s.L.ldv;
    U.Z = at(b, s.L.Z);
    U.f64 = s.svd64 ? 1 : 0;
    U.m = P.m; U.n = P.n; U.k = k;
  };

  for (int it = 1; it <= max_iter && n_active > 0; ++it) {
    for (int b = 0; b < batch; ++b) {
      State& s = S[b];
      if (!s.active) continue;
      const sorsvd_rpca_problem& P = probs[b];
      // the SOR-SVD takes G in the precision it was written in
      s.svd64 = s.g64;
      int r = s.svd64
          ? sorsvd_run(at(b, s.L.G64), P.m, P.n, s.L.ldg, k, p, q, P.seed + (uint64_t)(it - 1), SORSVD_F64, 0,
                       at(b, s.L.U), s.L.ldu, at(b, s.L.Z), at(b, s.L.V), s.L.ldv, at(b, s.L.ws), s.L.ws_bytes, st)
          : sorsvd_run(at(b, s.L.G), P.m, P.n, s.L.ldg, k, p, q, P.seed + (uint64_t)(it - 1), dtype, 0,
                       at(b, s.L.U), s.L.ldu, at(b, s.L.Z), at(b, s.L.V), s.L.ldv, at(b, s.L.ws), s.L.ws_bytes, st);
      if (r) return r;
      // the next G in binary64 from here on once the residual is near tol
      if (dtype != SORSVD_F64 && (flags & SORSVD_RPCA_FINISH_F64) && s.xi_prev < kSwitch * tol) s.g64 = true;
      const double mu_next = std::min(rho * s.mu, s.mu_bar);
      UpdParams U{};
      factors(b, U);
      U.X = P.X; U.ldx = P.ldx;
      U.Y = (float*)at(b, s.L.Y); U.ldg = s.L.ldg;
      U.G = s.g64 ? nullptr : (float*)at(b, s.L.G);
      U.G64 = s.g64 ? (double*)at(b, s.L.G64) : nullptr;
      U.S = P.S; U.lds = P.lds;
      U.inv_mu = to_df(1.0 / s.mu);
      U.inv_mu_d = 1.0 / s.mu;
      U.thr = to_df(s.lam / s.mu);
      U.mu = to_df(s.mu);
      U.inv_mu_next = to_df(1.0 / mu_next);
      U.part = (double*)at(b, s.L.part);
      U.status_in = &workspace_status(at(b, s.L.ws))->code;
      U.res = res + 2 * b;
      const int nb = ew_blocks(P.m * P.n);
      {
        ProfScope ps(K_RPCA, st);
        rpca_update_kernel<<<nb, kEwThreads, 0, st>>>(U);
        CKR(cudaGetLastError());
      }
      {
        ProfScope ps(K_REDUCE, st);
        rpca_reduce_kernel<<<1, kEwThreads, 0, st>>>(U.part, nb, 1, res + 2 * b);
        CKR(cudaGetLastError());
      }
      s.mu_used = s.mu;
      s.mu = mu_next;
    }
    CKR(cudaMemcpyAsync(host.data(), res, host.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CKR(cudaStreamSynchronize(st));
    for (int b = 0; b < batch; ++b) {
      State& s = S[b];
      if (!s.active) continue;
      if (host[2 * b + 1] != 0.0) return (int)host[2 * b + 1];
      const double x = std::sqrt(host[2 * b]) / s.nx;
      iters[b] = it;
      xi[b] = x;
      s.xi_prev = x;
      if (xi_history) xi_history[(size_t)b * max_iter + (it - 1)] = x;
      if (x < tol || it == max_iter) {
        s.active = false;
        --n_active;
        // L of the last iteration, from its factors
        const sorsvd_rpca_problem& P = probs[b];
        UpdParams U{};
        factors(b, U);
        U.inv_mu = to_df(1.0 / s.mu_used);
        U.inv_mu_d = 1.0 / s.mu_used;
        ProfScope ps(K_RPCA, st);
        rpca_lowrank_kernel<<<ew_blocks(P.m * P.n), kEwThreads, 0, st>>>(U, P.L, P.ldl);
        CKR(cudaGetLastError());
      }
    }
  }
  CKR(cudaStreamSynchronize(st));
  return SORSVD_OK;
}
