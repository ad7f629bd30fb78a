// Row-block products of fp32 tall-skinny matrices (the QR step of
// Algorithm 3 by CholeskyQR, the core product M = Q1^T W and the assembly
// U = Q1 U~_k, V = Q2 V~_k).  One dimension is long (m or n rows), the
// others are at most SORSVD_MAX_L columns.
//
//   rb_gram_kernel<SYM>:  partial products X^T Y over row chunks.  Output
//       tiles of 32 x 32, one per warp; a lane owns a 4 x 8 block (lanes
//       8 x 4), so per staged row a warp reads 32 + 32 distinct floats in
//       three conflict-free 128-bit loads and issues 32 FMAs per lane.  Rows
//       are staged 32 at a time in shared memory, the next chunk prefetched
//       into registers during the current one.  SYM (Y = X): lower tiles
//       only, written to both halves.  CTA x of the grid sums its chunks
//       (x, x + G, ...) into partial x, in order; the partials are summed
//       by launch_reduce_parts in a fixed order.
//   rb_apply_kernel<TRI>: Y = X B, B small (K x N).  A CTA computes 256
//       rows x 32 columns (8 warps, lane 4 x 8 again); its column tile of B
//       is staged once, X streams through a 2-stage cp.async ring of 32-deep
//       K slices stored K-major (a column of X is contiguous rows, so the
//       copies are plain 16-byte chunks).  TRI: B upper triangular, the K
//       loop stops at the tile's last column.  Out of place; an optional
//       16-bit rounding of Y is written next to it.
#include "internal.cuh"
#include "profile.cuh"

#include <algorithm>

namespace sorsvd {
namespace {

constexpr int kT = 32;               // output tile edge
constexpr int kGramRows = 32;        // rows per staged chunk (Gram)
constexpr int kGramMaxWarps = 16;
constexpr int kApRows = 256;         // rows per CTA (apply), 32 per warp
constexpr int kApThreads = kApRows;  // 8 warps
constexpr int kApKT = 32;            // K slice depth (apply)
constexpr int kApStages = 2;
constexpr int kBs = kT + 4;          // row stride of B's staged tile (4-way conflicts on the one-time fill)

__host__ __device__ inline int ntile(int l) { return (l + kT - 1) / kT; }

// lower-triangle tile q -> (ti, tj), tj <= ti, row-major over ti
__device__ __forceinline__ void tri_tile(int q, int* ti, int* tj) {
  int b = (int)((sqrtf(8.f * q + 1.f) - 1.f) * 0.5f);
  while ((b + 1) * (b + 2) / 2 <= q) ++b;
  while (b * (b + 1) / 2 > q) --b;
  *ti = b;
  *tj = q - b * (b + 1) / 2;
}

// cp.async of one 16-byte chunk, zero-filled past `bytes`
__device__ __forceinline__ void cp_async16(float* dst, const float* src, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// Staged chunk of kGramRows rows of a column-major matrix: column c is 32
// consecutive floats (rows), its 16-byte row quads permuted by
// quad ^ ((c >> 2) & 7).  With that swizzle the quads a warp reads in the
// Gram (8 lane groups x one column each, or 4 groups x 8 columns) fall in
// distinct banks.
__device__ __forceinline__ int swz(int c, int q) { return 4 * (q ^ ((c >> 2) & 7)); }

struct GramGeom {
  int ntiles, warps, gy, stages;
  size_t smem;
};

GramGeom gram_geom(int lx, int ly, bool sym) {
  GramGeom g{};
  g.ntiles = sym ? ntile(lx) * (ntile(lx) + 1) / 2 : ntile(lx) * ntile(ly);
  g.gy = (g.ntiles + kGramMaxWarps - 1) / kGramMaxWarps;
  g.warps = (g.ntiles + g.gy - 1) / g.gy;
  g.warps = std::max(4, (g.warps + 1) & ~1);            // even, so every thread keeps one row quad
  const size_t per = (size_t)kGramRows * kT * (ntile(lx) + (sym ? 0 : ntile(ly))) * sizeof(float);
  g.stages = (3 * per <= 200u * 1024u) ? 3 : 2;
  g.smem = g.stages * per;
  return g;
}

// issue the copies of chunk r0 of M (rows x l, ld) into S (ncol = 32 ntile
// columns): chunk e = t + i * nthreads -> column e / 8, quad e % 8; the
// thread count is a multiple of 64, so the quad is fixed per thread and
// the column steps by nthreads / 8
__device__ __forceinline__ void chunk_issue(const float* __restrict__ M, int64_t ldm, int64_t rows, int l, int ncol,
                                            int64_t r0, float* S) {
  const int nt = blockDim.x, q = threadIdx.x & 7;
  const int64_t r = r0 + 4 * q;
  const int rbytes = r < rows ? (int)(4 * std::min<int64_t>(4, rows - r)) : 0;
  const int cstep = nt >> 3;
  int c = threadIdx.x >> 3;
  const float* src = M + r + (int64_t)c * ldm;
  const int64_t sstep = (int64_t)cstep * ldm;
  for (; c < ncol; c += cstep, src += sstep) {
    const int bytes = c < l ? rbytes : 0;
    cp_async16(S + c * kGramRows + swz(c, q), bytes ? src : M, bytes);
  }
}

template <bool SYM, int NSTAGE>
__global__ void __launch_bounds__(kGramMaxWarps * 32)
rb_gram_kernel(const float* __restrict__ X, int64_t ldx, const float* __restrict__ Y, int64_t ldy, int64_t rows,
               int lx, int ly, float* __restrict__ parts, int64_t pstride, const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) float sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int ntx = ntile(lx), nty = ntile(ly);
  const int ncx = kT * ntx, ncy = kT * nty;
  const int per = kGramRows * (ncx + (SYM ? 0 : ncy));
  const int ntiles = SYM ? ntx * (ntx + 1) / 2 : ntx * nty;
  const int q = blockIdx.y * nw + warp;
  const bool act = q < ntiles;
  int ti = 0, tj = 0;
  if (act) {
    if (SYM) tri_tile(q, &ti, &tj);
    else { ti = q / nty; tj = q - ti * nty; }
  }
  const int gi = lane >> 2, gj = lane & 3;
  const int ca = kT * ti + 4 * gi;                   // columns ca .. ca + 3 of X
  const int cb = kT * tj + 8 * gj;                   // columns cb .. cb + 7 of Y
  float acc[4][8] = {};

  const int64_t nchunk = (rows + kGramRows - 1) / kGramRows;
  const int64_t first = blockIdx.x, stride = gridDim.x;
#pragma unroll
  for (int s = 0; s < NSTAGE - 1; ++s) {
    const int64_t ch = first + s * stride;
    if (ch < nchunk) {
      float* S = sm + s * per;
      chunk_issue(X, ldx, rows, lx, ncx, ch * kGramRows, S);
      if (!SYM) chunk_issue(Y, ldy, rows, ly, ncy, ch * kGramRows, S + kGramRows * ncx);
    }
    cp_async_commit();
  }
  int it = 0;
  for (int64_t ch = first; ch < nchunk; ch += stride, ++it) {
    cp_async_wait<NSTAGE - 2>();
    __syncthreads();                                 // chunk ch landed; the buffer refilled below was consumed
    const int64_t cn = ch + (NSTAGE - 1) * stride;
    if (cn < nchunk) {
      float* S = sm + ((it + NSTAGE - 1) % NSTAGE) * per;
      chunk_issue(X, ldx, rows, lx, ncx, cn * kGramRows, S);
      if (!SYM) chunk_issue(Y, ldy, rows, ly, ncy, cn * kGramRows, S + kGramRows * ncx);
    }
    cp_async_commit();
    if (!act) continue;
    const float* Sx = sm + (it % NSTAGE) * per;
    const float* Sy = SYM ? Sx : Sx + kGramRows * ncx;
#pragma unroll 2
    for (int qd = 0; qd < kGramRows / 4; ++qd) {
      float4 xa[4], yb[8];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        xa[u] = *reinterpret_cast<const float4*>(Sx + (ca + u) * kGramRows + swz(ca + u, qd));
#pragma unroll
      for (int v = 0; v < 8; ++v)
        yb[v] = *reinterpret_cast<const float4*>(Sy + (cb + v) * kGramRows + swz(cb + v, qd));
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) {
          acc[u][v] = fmaf(xa[u].x, yb[v].x, acc[u][v]);
          acc[u][v] = fmaf(xa[u].y, yb[v].y, acc[u][v]);
          acc[u][v] = fmaf(xa[u].z, yb[v].z, acc[u][v]);
          acc[u][v] = fmaf(xa[u].w, yb[v].w, acc[u][v]);
        }
    }
  }
  cp_async_wait<0>();
  if (!act) return;
  float* out = parts + (int64_t)blockIdx.x * pstride;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int i = ca + u, j = cb + v;
      if (i < lx && j < ly) {
        out[i + (int64_t)j * lx] = acc[u][v];
        if (SYM && ti != tj) out[j + (int64_t)i * lx] = acc[u][v];
      }
    }
}

// ---------------------------------------------------------------- apply

// K slice (rows r0 .. r0 + 255 of columns k0 .. k0 + 31 of X) into
// Xt[kk * kApRows + r]: thread t copies the 16-byte row quad t % 64 of
// columns k0 + t / 64 + 4 i, i < 8 (zero-filled past rows / K)
__device__ __forceinline__ void slice_issue(const float* __restrict__ X, int64_t ldx, int K, int rbytes, int k0,
                                            const float* xq, float* Xt) {
  const int q4 = threadIdx.x & 63, kk0 = threadIdx.x >> 6;
#pragma unroll
  for (int i = 0; i < kApKT / 4; ++i) {
    const int kk = kk0 + 4 * i;
    const int bytes = (k0 + kk < K) ? rbytes : 0;
    cp_async16(Xt + kk * kApRows + 4 * q4, bytes ? xq + (int64_t)(k0 + kk) * ldx : X, bytes);
  }
}

template <bool TRI>
__global__ void __launch_bounds__(kApThreads)
rb_apply_kernel(const float* __restrict__ X, int64_t ldx, int64_t rows, int K, const float* __restrict__ B,
                int64_t ldb, int N, float* __restrict__ Yo, int64_t ldy, void* __restrict__ Y16, int64_t ld16,
                int kind16, const int* __restrict__ skip) {
  if (skip && *skip) return;
  extern __shared__ __align__(16) float sm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int jt = blockIdx.y;
  const int64_t r0 = (int64_t)blockIdx.x * kApRows;
  const int kend = TRI ? std::min(K, kT * (jt + 1)) : K;
  const int nslice = (kend + kApKT - 1) / kApKT;
  float* Bs = sm;                                          // [nslice * 32][kBs]
  float* Xt = sm + (size_t)nslice * kApKT * kBs;           // kApStages x [32][128]
  // this thread's row quad of X (the same in every slice)
  const int64_t rq = r0 + 4 * (threadIdx.x & 63);
  const int rbytes = rq < rows ? (int)(4 * std::min<int64_t>(4, rows - rq)) : 0;
  const float* xq = X + rq;
  // prologue: the first kApStages - 1 slices in flight
#pragma unroll
  for (int s = 0; s < kApStages - 1; ++s) {
    if (s < nslice) slice_issue(X, ldx, K, rbytes, s * kApKT, xq, Xt + s * (kApKT * kApRows));
    cp_async_commit();
  }
  // B's column tile, zero below the diagonal (TRI) and past K / N; a warp
  // reads one column of B (contiguous k) at a time
  const int nk = nslice * kApKT;
  for (int jj = warp; jj < kT; jj += kApThreads / 32) {
    const int j = kT * jt + jj;
    const float* bc = B + (int64_t)j * ldb;
    for (int k = lane; k < nk; k += 32) {
      float v = 0.f;
      if (k < kend && j < N && (!TRI || k <= j)) v = bc[k];
      Bs[k * kBs + jj] = v;
    }
  }
  const int a_off = kT * warp + 4 * (lane >> 2);
  const int b_off = 8 * (lane & 3);
  float acc[4][8] = {};
  for (int s = 0; s < nslice; ++s) {
    cp_async_wait<kApStages - 2>();
    __syncthreads();                                       // slice s landed; slice s - 1 consumed
    const int sn = s + kApStages - 1;
    if (sn < nslice) slice_issue(X, ldx, K, rbytes, sn * kApKT, xq, Xt + (sn % kApStages) * (kApKT * kApRows));
    cp_async_commit();
    const float* xs = Xt + (s % kApStages) * (kApKT * kApRows);
    const float* bs = Bs + s * kApKT * kBs;
#pragma unroll 8
    for (int kk = 0; kk < kApKT; ++kk) {
      const float4 a = *reinterpret_cast<const float4*>(xs + kk * kApRows + a_off);
      const float4 b0 = *reinterpret_cast<const float4*>(bs + kk * kBs + b_off);
      const float4 b1 = *reinterpret_cast<const float4*>(bs + kk * kBs + b_off + 4);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
  }
  cp_async_wait<0>();
  const int64_t rb = r0 + a_off;
  const bool vec = ((reinterpret_cast<uintptr_t>(Yo) & 15) == 0) && ((ldy & 3) == 0) && rb + 3 < rows;
#pragma unroll
  for (int v = 0; v < 8; ++v) {
    const int j = kT * jt + b_off + v;
    if (j >= N) continue;
    if (!Yo) {
      // only the 16-bit copy is wanted
    } else if (vec) {
      *reinterpret_cast<float4*>(Yo + rb + (int64_t)j * ldy) = make_float4(acc[0][v], acc[1][v], acc[2][v], acc[3][v]);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (rb + u < rows) Yo[rb + u + (int64_t)j * ldy] = acc[u][v];
    }
    if (kind16) {
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int64_t r = rb + u;
        if (r >= rows) continue;
        if (kind16 == 1) reinterpret_cast<bf16*>(Y16)[r + (int64_t)j * ld16] = __float2bfloat16_rn(acc[u][v]);
        else reinterpret_cast<f16*>(Y16)[r + (int64_t)j * ld16] = __float2half_rn(acc[u][v]);
      }
    }
  }
}

size_t apply_smem(int K, int N, bool tri, int jt_max) {
  (void)N;
  const int kend = tri ? std::min(K, kT * (jt_max + 1)) : K;
  const int nslice = (kend + kApKT - 1) / kApKT;
  return ((size_t)nslice * kApKT * kBs + (size_t)kApStages * kApKT * kApRows) * sizeof(float);
}

// dst (rows x l) = src, plus the 16-bit rounding; with *skip set src is
// already in dst (only the 16-bit copy is written)
__global__ void rb_copy_kernel(const float* __restrict__ src, float* __restrict__ dst, int64_t ld, int64_t rows,
                               int l, void* __restrict__ Y16, int64_t ld16, int kind16, const int* __restrict__ skip) {
  const bool skipped = skip && *skip;
  if (skipped && !kind16) return;
  const float* from = skipped ? dst : src;
  const int64_t total = rows * l;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / rows, r = e - c * rows;
    const float x = from[r + c * ld];
    if (!skipped) dst[r + c * ld] = x;
    if (kind16 == 1) reinterpret_cast<bf16*>(Y16)[r + c * ld16] = __float2bfloat16_rn(x);
    else if (kind16 == 2) reinterpret_cast<f16*>(Y16)[r + c * ld16] = __float2half_rn(x);
  }
}

// out[i + j ldo] = sum_s parts[s * stride + i + j ldp] (binary64) for an
// rows x cols result.  A block takes 32 consecutive elements (column-major
// index); warp w of its kRedWarps sums the partials w, w + kRedWarps, ... in
// index order with Neumaier's compensation in fp32 (error ~ 2 eps |sum| plus
// second-order terms), a lane per element, so every load of a warp is one
// run of 32 neighbouring floats.  The warps' (sum + compensation) values are
// then added in binary64 in warp order: deterministic.  The sum is
// latency-bound (a few MB from L2); kRedWarps independent chains per
// element keep the loads in flight.
constexpr int kRedWarps = 8;
__global__ void __launch_bounds__(32 * kRedWarps)
reduce_parts_kernel(const float* __restrict__ parts, int nparts, int64_t stride, int rows, int cols, int ldp,
                    double* __restrict__ out, int ldo, int sym_split) {
  __shared__ double part[kRedWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  bool ok = e < (int64_t)rows * cols;
  int oi = 0, oj = 0;
  if (ok) {
    oj = (int)(e / rows);
    oi = (int)(e - (int64_t)oj * rows);
    // symmetric: the lower-triangle element writes both halves
    if (sym_split >= 0 && oi < oj) ok = false;
  }
  float s = 0.f, c = 0.f;
  if (ok) {
    int i = oi, j = oj;
    if (sym_split >= 0 && i >= sym_split && j < sym_split) { i = oj; j = oi; }
    const float* p = parts + i + (int64_t)j * ldp;
#pragma unroll 4
    for (int q = w; q < nparts; q += kRedWarps) {
      const float x = p[(int64_t)q * stride];
      const float t = __fadd_rn(s, x);
      c = __fadd_rn(c, fabsf(s) >= fabsf(x) ? __fadd_rn(__fsub_rn(s, t), x) : __fadd_rn(__fsub_rn(x, t), s));
      s = t;
    }
  }
  part[w][lane] = (double)s + (double)c;
  __syncthreads();
  if (w == 0 && ok) {
    double v = part[0][lane];
#pragma unroll
    for (int u = 1; u < kRedWarps; ++u) v += part[u][lane];
    out[oi + (int64_t)oj * ldo] = v;
    if (sym_split >= 0 && oi != oj) out[oj + (int64_t)oi * ldo] = v;
  }
}

template <bool SYM, int NSTAGE>
cudaError_t gram_launch(const float* X, int64_t ldx, const float* Y, int64_t ldy, int64_t rows, int lx, int ly,
                        float* parts, const int* skip, cudaStream_t st) {
  const GramGeom g = gram_geom(lx, ly, SYM);
  auto kern = rb_gram_kernel<SYM, NSTAGE>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)rb_gram_blocks(rows, lx, ly, SYM), (unsigned)g.gy);
  kern<<<grid, g.warps * 32, g.smem, st>>>(X, ldx, Y, ldy, rows, lx, ly, parts, (int64_t)lx * ly, skip);
  return cudaGetLastError();
}

}  // namespace

// Partial count of the Gram: the CTAs resident at once (from the kernel's
// occupancy), split over the tile groups, at most one per row chunk.
int64_t rb_gram_blocks(int64_t rows, int lx, int ly, bool sym) {
  const GramGeom g = gram_geom(lx, ly, sym);
  const int threads = g.warps * 32;
  // resident CTAs per SM, bounded by threads, shared memory and registers
  // (about 128 registers per thread)
  int per_sm = std::max(1, std::min<int>(2048 / threads, (int)(227u * 1024u / std::max<size_t>(g.smem, 1))));
  per_sm = std::max(1, std::min(per_sm, 65536 / (threads * 128)));
  const int64_t nchunk = (rows + kGramRows - 1) / kGramRows;
  const int64_t want = std::max<int64_t>(1, (int64_t)num_sms() * per_sm / g.gy);
  return std::max<int64_t>(1, std::min(nchunk, want));
}

size_t rb_gram_parts_bytes(int64_t rows, int lx, int ly, bool sym) {
  return (size_t)rb_gram_blocks(rows, lx, ly, sym) * lx * ly * sizeof(float);
}

cudaError_t launch_rb_gram(const float* X, int64_t ldx, const float* Y, int64_t ldy, int64_t rows, int lx, int ly,
                           bool sym, float* parts, const int* skip, cudaStream_t st) {
  if (rows < 1 || lx < 1 || ly < 1 || lx > SORSVD_MAX_L || ly > SORSVD_MAX_L) return cudaErrorInvalidValue;
  if (sym && (X != Y || lx != ly || ldx != ldy)) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (reinterpret_cast<uintptr_t>(Y) & 15) || (ldx & 3) || (ldy & 3))
    return cudaErrorInvalidValue;                  // cp.async copies 16-byte row quads
  const GramGeom g = gram_geom(lx, ly, sym);
  if (sym) return g.stages == 3 ? gram_launch<true, 3>(X, ldx, Y, ldy, rows, lx, ly, parts, skip, st)
                                : gram_launch<true, 2>(X, ldx, Y, ldy, rows, lx, ly, parts, skip, st);
  return g.stages == 3 ? gram_launch<false, 3>(X, ldx, Y, ldy, rows, lx, ly, parts, skip, st)
                       : gram_launch<false, 2>(X, ldx, Y, ldy, rows, lx, ly, parts, skip, st);
}

cudaError_t launch_rb_apply(const float* X, int64_t ldx, int64_t rows, int K, const float* B, int64_t ldb, int N,
                            bool tri, float* Y, int64_t ldy, void* Y16, int64_t ld16, int kind16, const int* skip,
                            cudaStream_t st) {
  if (rows < 1 || K < 1 || N < 1) return cudaSuccess;
  if (K > SORSVD_MAX_L || N > SORSVD_MAX_L) return cudaErrorInvalidValue;
  // cp.async copies 16-byte chunks of X's columns
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (ldx & 3)) return cudaErrorInvalidValue;
  const int ntj = ntile(N);
  const size_t smem = apply_smem(K, N, tri, ntj - 1);
  cudaError_t e;
  const dim3 grid((unsigned)((rows + kApRows - 1) / kApRows), (unsigned)ntj);
  if (tri) {
    e = cudaFuncSetAttribute(rb_apply_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    rb_apply_kernel<true><<<grid, kApThreads, smem, st>>>(X, ldx, rows, K, B, ldb, N, Y, ldy, Y16, ld16, kind16, skip);
  } else {
    e = cudaFuncSetAttribute(rb_apply_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    rb_apply_kernel<false><<<grid, kApThreads, smem, st>>>(X, ldx, rows, K, B, ldb, N, Y, ldy, Y16, ld16, kind16, skip);
  }
  return cudaGetLastError();
}

cudaError_t launch_rb_copy(const float* src, float* dst, int64_t ld, int64_t rows, int l, void* Y16, int64_t ld16,
                           int kind16, const int* skip, cudaStream_t st) {
  const int64_t total = rows * l;
  if (total <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((total + 255) / 256, (int64_t)num_sms() * 8);
  rb_copy_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, dst, ld, rows, l, Y16, ld16, kind16, skip);
  return cudaGetLastError();
}

cudaError_t launch_reduce_parts(const float* parts, int nparts, int64_t stride, int rows, int cols, int ldp,
                                double* out, int ldo, cudaStream_t st, int sym_split) {
  const int64_t elems = (int64_t)rows * cols;
  if (elems <= 0) return cudaSuccess;
  if (sym_split >= 0 && rows != cols) return cudaErrorInvalidValue;
  reduce_parts_kernel<<<(unsigned)((elems + 31) / 32), 32 * kRedWarps, 0, st>>>(parts, nparts, stride, rows, cols,
                                                                             ldp, out, ldo, sym_split);
  return cudaGetLastError();
}

}  // namespace sorsvd
