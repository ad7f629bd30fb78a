// Tall-skinny products of the QR step of Algorithm 3 (CholeskyQR:
// G = T^T T, Q = T R^{-1}), of the polar pass (Q = T X) and of the output
// assembly (U = Q1 U~_k, V = Q2 V~_k) on the tensor cores, at fp32 accuracy.
// T is rows x l, column-major (rows = m or n, up to the matrix size),
// l <= kTskMaxL.
//
// fp32 accuracy from TF32 MMAs (kind::tf32 reads the top 19 bits of an fp32
// container): every operand x is taken as hi + lo with hi = x truncated to
// TF32 (what the MMA reads from the container itself) and lo = x - hi
// (exact in fp32), and each product as hi*hi + hi*lo + lo*hi; the dropped
// lo*lo term and the TF32 truncation of lo are below 2^-20 relative.
//
// tsk_gram_kernel: partial sums of G = T^T T over row ranges.  Both MMA
// operands are K-major straight from T's column-major storage (a column of
// T is a run of rows = K), so a staged K atom is 32 rows of every column of
// T, 128 bytes per column, 128-byte swizzled by TMA.  A CTA keeps the lower
// triangle of G in TMEM as blocks of 128 MMA rows:
//   L16 <= 128:         rows 0..127 x columns 0..L16
//   L16 <= 256:         + rows 128..255 x columns 0..L16
//   L16 in {272, 288}:  rows 0..127 x 0..127, rows 128..255 x 0..255, and
//                       columns 256..L16 of every row (three 16- or 32-wide
//                       blocks; the third takes MMA rows L16-128.. and keeps
//                       rows >= 256), which fit in 512 TMEM columns where a
//                       third 128-row block of full width would not.
// A converter warpgroup writes lo of each staged atom next to it in shared
// memory; the MMA thread issues the three products per block and K step.
// Partials are written column-major (l x l, the entries each block owns)
// and summed in a fixed order by the reduction kernel, which mirrors the
// lower triangle (deterministic).
//
// tsk_xty_kernel: partial sums of C = X^T Y (two rows x l operands, the
// core product Q1^T W and the cross products of the two-pass core).  The
// full l x l result does not fit in TMEM next to its operands, so CTAs come
// in ceil(L16 / 128) types (blockIdx.y): type t holds MMA rows = columns
// a0_t .. a0_t + 127 of X (a0_t = min(128 t, L16 - 128), keeping rows
// >= 128 t) against all L16 columns of Y, and each row range is one
// partial shared by the types.
//
// tsk_apply_kernel: Y = T B with B small (K x N, K = l).  Here T's
// contiguous dimension (rows) is an M dimension of the product, and a TF32
// operand must be K-major, so the 128-row tile of T goes to TMEM as the A
// operand: a converter thread per row (= TMEM lane) reads its row's 32
// values of a staged K atom (stored column by column, conflict-free) and
// writes hi and lo to a TMEM slot.  B comes split into hi (rounded to TF32)
// and lo by the caller, K-major (B is column-major: a column is a run of K),
// streamed from L2 per K atom.  T and B come in separate rings: the atoms
// of T (16 KB each, from HBM) in a deep ring that the converter releases as
// soon as it has read an atom, those of B (hi and lo, up to 74 KB per atom,
// from L2) in a two-stage ring that the MMAs release; each ring has its own
// TMA warp.  One accumulator of N <= 320 columns per row tile (two MMA
// column chunks when N > 256); an epilogue warpgroup drains it while the
// converter prepares the next tile.  For an upper-triangular B the K atoms
// below a chunk's last column are skipped.
//
// Every mbarrier wait is bounded (the library's tensor-core wait limit); a
// timeout records SORSVD_ERR_TIMEOUT, stops every role, waits for the
// copies and MMAs already issued, frees TMEM and returns.
#include "internal.cuh"
#include "profile.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cstdlib>

namespace sorsvd {
namespace {

constexpr int kAtomK = 32;                 // fp32 elements per 128-byte swizzle row
constexpr int kMaxGramBlocks = 5;
constexpr int kGramThreads = 192;          // warp 0 TMA, warp 1 MMA, warps 2-5 low parts + epilogue
// warp 0 TMA of T, warp 1 MMA, warps 2-5 convert, warps 6-9 epilogue, warp 10 TMA of B
constexpr int kApplyThreads = 352;
constexpr uint32_t kTmemCols = 512;
constexpr uint32_t kApplySlotCol = 320;    // first TMEM column of the apply's A slots (hi 32 + lo 32 each)
constexpr int kApplySlots = 3;
constexpr int kApplyBStages = 2;           // B (hi and lo) from L2
constexpr int kApplyMaxTStages = 8;        // K atoms of T from HBM
constexpr uint32_t kSmemBudget = 220u * 1024u;

struct GramBlock {
  int a0, b0, n, tcol, row_lo;   // MMA rows = T columns a0.., MMA columns = T columns b0..b0+n; kept rows >= row_lo
};

struct GramParams {
  int64_t rows, natoms;
  int l, L16, nbox, boxc, nblk, stages;
  uint32_t tile_bytes;           // TR x 128 bytes: one K atom of the TR >= L16 columns the MMAs read
  GramBlock blk[kMaxGramBlocks];
  float* parts;
  int64_t pstride;
  const int* skip;
  DeviceStatus* status;
  long long wait_cycles;
};

struct XtyParams {
  int64_t rows, natoms;
  int l, L16, ntypes, nch, ch0, nboxy, boxy, stages;
  uint32_t x_bytes, y_bytes, stage_bytes;   // X: 128 columns, Y: nboxy boxes of boxy columns (x 128 bytes)
  float* parts;
  int64_t pstride;
  const int* skip;
  DeviceStatus* status;
  long long wait_cycles;
};

struct ApplyParams {
  int64_t rows, ntiles;
  int K, N, NP, nch, ch0, katoms, tri;
  uint32_t x_bytes, b_bytes, stage_bytes;   // b_bytes: one of B_hi / B_lo (2 ch0 rows x 128 bytes)
  int tstages;                               // depth of the ring of T atoms
  float* Y;
  int64_t ldy;
  void* Y16;
  int64_t ld16;
  int kind16;
  const int* skip;
  DeviceStatus* status;
  long long wait_cycles;
};

// x - trunc_tf32(x): the part of x a TF32 MMA ignores (exact in fp32)
__device__ __forceinline__ float tf32_rest(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint8_t* align1024(uint8_t* p) {
  return reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(p) + 1023) & ~(uintptr_t)1023);
}

// bounded wait for the copies a producer armed and never saw consumed
__device__ __forceinline__ void drain_armed(uint64_t* full, int stages, uint32_t armed, uint32_t armed_par) {
  for (int s = 0; s < stages; ++s)
    if (armed & (1u << s)) {
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(&full[s], (armed_par >> s) & 1u) && clock64() - t0 < tc::kWaitCycles) {}
    }
}

template <int NBLK>
__global__ void __launch_bounds__(kGramThreads, 1)
tsk_gram_kernel(const __grid_constant__ CUtensorMap tmX, const GramParams P) {
  if (P.skip && *P.skip) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)P.stages * 2 * P.tile_bytes);
  uint64_t* lofull = full + P.stages;
  uint64_t* empty = lofull + P.stages;
  uint64_t* dfull = empty + P.stages;
  uint64_t* done = dfull + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abortp = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&lofull[s], 4);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(dfull, 1);
    tc::mbar_init(done, 1);
    *abortp = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tslot, kTmemCols);
    tc::tmem_relinquish();
  }
  if (warp == 0 && lane == 0) tc::prefetch_tmap(&tmX);
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int64_t a0 = (int64_t)blockIdx.x * P.natoms / gridDim.x;
  const int64_t a1 = (int64_t)(blockIdx.x + 1) * P.natoms / gridDim.x;
  const long long wc = P.wait_cycles;

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer
    if (lane == 0) {
      uint32_t armed = 0, armed_par = 0;
      int stage = 0;
      uint32_t phase = 0;
      for (int64_t a = a0; a < a1; ++a) {
        if (!tc::mbar_wait(&empty[stage], phase ^ 1u, abortp, wc)) break;
        tc::mbar_arrive_expect_tx(&full[stage], P.tile_bytes);
        armed |= 1u << stage;
        armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
        uint8_t* dst = smem + (size_t)stage * 2 * P.tile_bytes;
        for (int b = 0; b < P.nbox; ++b)
          tc::tma_load_2d(dst + (size_t)b * P.boxc * 128, &tmX, &full[stage], (int)(a * kAtomK), b * P.boxc);
        if (++stage == P.stages) { stage = 0; phase ^= 1u; }
      }
      if (*abortp) drain_armed(full, P.stages, armed, armed_par);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t idesc[NBLK];
#pragma unroll
      for (int b = 0; b < NBLK; ++b) idesc[b] = tc::idesc_make(2u, false, false, 128, P.blk[b].n);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t a = a0; a < a1 && ok; ++a) {
        if (!tc::mbar_wait(&lofull[stage], phase, abortp, wc) || !tc::mbar_wait(&full[stage], phase, abortp, wc)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t sraw = tc::smem_u32(smem + (size_t)stage * 2 * P.tile_bytes);
        const uint32_t slo = sraw + P.tile_bytes;
#pragma unroll
        for (int ks = 0; ks < kAtomK / 8; ++ks) {
          const uint32_t acc0 = (a > a0 || ks > 0) ? 1u : 0u;
#pragma unroll
          for (int b = 0; b < NBLK; ++b) {
            const GramBlock& g = P.blk[b];
            const uint32_t d = tbase + (uint32_t)g.tcol;
            const uint64_t ahi = tc::desc_sw128(sraw + (uint32_t)g.a0 * 128u + ks * 32, 16, 1024);
            const uint64_t bhi = tc::desc_sw128(sraw + (uint32_t)g.b0 * 128u + ks * 32, 16, 1024);
            const uint64_t alo = tc::desc_sw128(slo + (uint32_t)g.a0 * 128u + ks * 32, 16, 1024);
            const uint64_t blo = tc::desc_sw128(slo + (uint32_t)g.b0 * 128u + ks * 32, 16, 1024);
            tc::mma_tf32(d, ahi, bhi, idesc[b], acc0);
            tc::mma_tf32(d, ahi, blo, idesc[b], 1u);
            tc::mma_tf32(d, alo, bhi, idesc[b], 1u);
          }
        }
        tc::mma_commit(&empty[stage]);
        if (++stage == P.stages) { stage = 0; phase ^= 1u; }
      }
      if (ok) tc::mma_commit(dfull);
      // every MMA issued by this thread has completed once `done` flips
      tc::mma_commit(done);
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(done, 0) && clock64() - t0 < tc::kWaitCycles) {}
    }
  } else {
    // ------------------------------------------------------------ low parts, then the epilogue
    const int ct = threadIdx.x - 64;            // 0..127
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    const int n4 = (int)(P.tile_bytes / 16);
    for (int64_t a = a0; a < a1; ++a) {
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&full[stage], phase, abortp, wc))) { ok = false; break; }
      const float4* src = reinterpret_cast<const float4*>(smem + (size_t)stage * 2 * P.tile_bytes);
      float4* dst = reinterpret_cast<float4*>(smem + (size_t)stage * 2 * P.tile_bytes + P.tile_bytes);
      for (int e = ct; e < n4; e += 128) {
        const float4 x = src[e];
        dst[e] = make_float4(tf32_rest(x.x), tf32_rest(x.y), tf32_rest(x.z), tf32_rest(x.w));
      }
      fence_proxy_async();                      // the MMAs read the low parts through the async proxy
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&lofull[stage]);
      if (++stage == P.stages) { stage = 0; phase ^= 1u; }
    }
    // drain: thread = TMEM lane q*32 + lane = MMA row of each block
    if (ok && __all_sync(0xffffffffu, tc::mbar_wait(dfull, 0, abortp, wc))) {
      tc::fence_after_sync();
      const int q = warp & 3;
      const int r = q * 32 + lane;
      float* out = P.parts + (size_t)blockIdx.x * P.pstride;
#pragma unroll
      for (int b = 0; b < NBLK; ++b) {
        const GramBlock& g = P.blk[b];
        const int i = g.a0 + r;
        const bool keep = i >= g.row_lo && i < P.l;
        for (int c = 0; c < g.n; c += 16) {
          float v[16];
          tc::tmem_ld16(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(g.tcol + c), v);
          tc::tmem_ld_wait();
          if (keep) {
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              const int j = g.b0 + c + u;
              if (j < P.l) out[i + (size_t)j * P.l] = v[u];
            }
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x == 0 && *abortp) raise_status(P.status, SORSVD_ERR_TIMEOUT);
  if (warp == 1) tc::tmem_dealloc(tbase, kTmemCols);
}


template <int NCH>
__global__ void __launch_bounds__(kGramThreads, 1)
tsk_xty_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmY, const XtyParams P) {
  if (P.skip && *P.skip) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  // stage s: [X hi | Y hi | X lo | Y lo]; X and Y lo sit x_bytes + y_bytes after their hi
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)P.stages * P.stage_bytes);
  uint64_t* lofull = full + P.stages;
  uint64_t* empty = lofull + P.stages;
  uint64_t* dfull = empty + P.stages;
  uint64_t* done = dfull + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abortp = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int type = blockIdx.y;
  const int a0 = min(128 * type, P.L16 - 128 > 0 ? P.L16 - 128 : 0);
  const int row_lo = 128 * type;
  const uint32_t hbytes = P.x_bytes + P.y_bytes;
  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) {
      tc::mbar_init(&full[s], 1);
      tc::mbar_init(&lofull[s], 4);
      tc::mbar_init(&empty[s], 1);
    }
    tc::mbar_init(dfull, 1);
    tc::mbar_init(done, 1);
    *abortp = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tslot, kTmemCols);
    tc::tmem_relinquish();
  }
  if (warp == 0 && lane == 0) {
    tc::prefetch_tmap(&tmX);
    tc::prefetch_tmap(&tmY);
  }
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const int64_t at0 = (int64_t)blockIdx.x * P.natoms / gridDim.x;
  const int64_t at1 = (int64_t)(blockIdx.x + 1) * P.natoms / gridDim.x;
  const long long wc = P.wait_cycles;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t armed = 0, armed_par = 0;
      int stage = 0;
      uint32_t phase = 0;
      for (int64_t a = at0; a < at1; ++a) {
        if (!tc::mbar_wait(&empty[stage], phase ^ 1u, abortp, wc)) break;
        tc::mbar_arrive_expect_tx(&full[stage], hbytes);
        armed |= 1u << stage;
        armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
        uint8_t* dst = smem + (size_t)stage * P.stage_bytes;
        tc::tma_load_2d(dst, &tmX, &full[stage], (int)(a * kAtomK), a0);
        for (int b = 0; b < P.nboxy; ++b)
          tc::tma_load_2d(dst + P.x_bytes + (size_t)b * P.boxy * 128, &tmY, &full[stage], (int)(a * kAtomK),
                          b * P.boxy);
        if (++stage == P.stages) { stage = 0; phase ^= 1u; }
      }
      if (*abortp) drain_armed(full, P.stages, armed, armed_par);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t id0 = tc::idesc_make(2u, false, false, 128, P.ch0);
      const uint32_t id1 = tc::idesc_make(2u, false, false, 128, NCH > 1 ? P.L16 - P.ch0 : 16);
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t a = at0; a < at1 && ok; ++a) {
        if (!tc::mbar_wait(&lofull[stage], phase, abortp, wc) || !tc::mbar_wait(&full[stage], phase, abortp, wc)) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        const uint32_t sx = tc::smem_u32(smem + (size_t)stage * P.stage_bytes);
        const uint32_t sy = sx + P.x_bytes;
#pragma unroll
        for (int ks = 0; ks < kAtomK / 8; ++ks) {
          const uint32_t acc0 = (a > at0 || ks > 0) ? 1u : 0u;
          const uint64_t ahi = tc::desc_sw128(sx + ks * 32, 16, 1024);
          const uint64_t alo = tc::desc_sw128(sx + hbytes + ks * 32, 16, 1024);
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch) {
            const uint32_t boff = (uint32_t)(ch * P.ch0 * 128 + ks * 32);
            const uint64_t bhi = tc::desc_sw128(sy + boff, 16, 1024);
            const uint64_t blo = tc::desc_sw128(sy + hbytes + boff, 16, 1024);
            const uint32_t d = tbase + (uint32_t)(ch * P.ch0);
            const uint32_t id = ch ? id1 : id0;
            tc::mma_tf32(d, ahi, bhi, id, acc0);
            tc::mma_tf32(d, ahi, blo, id, 1u);
            tc::mma_tf32(d, alo, bhi, id, 1u);
          }
        }
        tc::mma_commit(&empty[stage]);
        if (++stage == P.stages) { stage = 0; phase ^= 1u; }
      }
      if (ok) tc::mma_commit(dfull);
      tc::mma_commit(done);
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(done, 0) && clock64() - t0 < tc::kWaitCycles) {}
    }
  } else {
    const int ct = threadIdx.x - 64;
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    const int n4 = (int)(hbytes / 16);
    for (int64_t a = at0; a < at1; ++a) {
      if (!__all_sync(0xffffffffu, tc::mbar_wait(&full[stage], phase, abortp, wc))) { ok = false; break; }
      const float4* src = reinterpret_cast<const float4*>(smem + (size_t)stage * P.stage_bytes);
      float4* dst = reinterpret_cast<float4*>(smem + (size_t)stage * P.stage_bytes + hbytes);
      for (int e = ct; e < n4; e += 128) {
        const float4 x = src[e];
        dst[e] = make_float4(tf32_rest(x.x), tf32_rest(x.y), tf32_rest(x.z), tf32_rest(x.w));
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&lofull[stage]);
      if (++stage == P.stages) { stage = 0; phase ^= 1u; }
    }
    if (ok && __all_sync(0xffffffffu, tc::mbar_wait(dfull, 0, abortp, wc))) {
      tc::fence_after_sync();
      const int q = warp & 3;
      const int i = a0 + q * 32 + lane;
      const bool keep = i >= row_lo && i < P.l;
      float* out = P.parts + (size_t)blockIdx.x * P.pstride;
      for (int c = 0; c < P.L16; c += 16) {
        float v[16];
        tc::tmem_ld16(tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)c, v);
        tc::tmem_ld_wait();
        if (keep) {
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int j = c + u;
            if (j < P.l) out[i + (size_t)j * P.l] = v[u];
          }
        }
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x == 0 && *abortp) raise_status(P.status, SORSVD_ERR_TIMEOUT);
  if (warp == 1) tc::tmem_dealloc(tbase, kTmemCols);
}

template <int NCH>
__global__ void __launch_bounds__(kApplyThreads, 1)
tsk_apply_kernel(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmBhi,
                 const __grid_constant__ CUtensorMap tmBlo, const ApplyParams P) {
  if (P.skip && *P.skip) return;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = align1024(smem_raw);
  // B stage s: B_hi (2 ch0 rows x 128 B), B_lo (same); then the T ring (a K
  // atom of T, 32 columns x 128 rows, per stage)
  uint8_t* tring = smem + (size_t)kApplyBStages * 2 * P.b_bytes;
  uint64_t* bfull = reinterpret_cast<uint64_t*>(tring + (size_t)P.tstages * P.x_bytes);
  uint64_t* bempty = bfull + kApplyBStages;
  uint64_t* tfull = bempty + kApplyBStages;    // a T atom landed
  uint64_t* tempty = tfull + kApplyMaxTStages; // a T atom read by the converter (4 warps)
  uint64_t* afull = tempty + kApplyMaxTStages; // a TMEM slot written (4 converter warps)
  uint64_t* aempty = afull + kApplySlots;      // a slot read by its MMAs
  uint64_t* dfull = aempty + kApplySlots;      // the tile's accumulator complete
  uint64_t* dempty = dfull + 1;                // the accumulator drained (4 epilogue warps)
  uint64_t* done = dempty + 1;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abortp = reinterpret_cast<volatile int*>(tslot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kApplyBStages; ++s) { tc::mbar_init(&bfull[s], 1); tc::mbar_init(&bempty[s], 1); }
    for (int s = 0; s < P.tstages; ++s) { tc::mbar_init(&tfull[s], 1); tc::mbar_init(&tempty[s], 4); }
    for (int s = 0; s < kApplySlots; ++s) { tc::mbar_init(&afull[s], 4); tc::mbar_init(&aempty[s], 1); }
    tc::mbar_init(dfull, 1);
    tc::mbar_init(dempty, 4);
    tc::mbar_init(done, 1);
    *abortp = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tslot, kTmemCols);
    tc::tmem_relinquish();
  }
  if (warp == 0 && lane == 0) tc::prefetch_tmap(&tmX);
  if (warp == 10 && lane == 0) {
    tc::prefetch_tmap(&tmBhi);
    tc::prefetch_tmap(&tmBlo);
  }
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const long long wc = P.wait_cycles;
  const int ch1 = P.NP - P.ch0;
  // K atoms a chunk needs: all, or (upper-triangular B) those starting at or
  // before the chunk's last column
  auto atoms_of = [&](int ch) {
    if (!P.tri) return P.katoms;
    const int c1 = ch == 0 ? min(P.ch0, P.N) : P.N;
    return min(P.katoms, (c1 + kAtomK - 1) / kAtomK);
  };

  if (warp == 0) {
    // ------------------------------------------------------------ TMA producer of T
    if (lane == 0) {
      uint32_t armed = 0, armed_par = 0;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x) {
        for (int a = 0; a < P.katoms; ++a) {
          if (!tc::mbar_wait(&tempty[stage], phase ^ 1u, abortp, wc)) { ok = false; break; }
          tc::mbar_arrive_expect_tx(&tfull[stage], P.x_bytes);
          armed |= 1u << stage;
          armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
          tc::tma_load_2d(tring + (size_t)stage * P.x_bytes, &tmX, &tfull[stage], (int)(t * 128), a * kAtomK);
          if (++stage == P.tstages) { stage = 0; phase ^= 1u; }
        }
      }
      if (*abortp) drain_armed(tfull, P.tstages, armed, armed_par);
    }
  } else if (warp == 10) {
    // ------------------------------------------------------------ TMA producer of B
    if (lane == 0) {
      uint32_t armed = 0, armed_par = 0;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x) {
        for (int a = 0; a < P.katoms; ++a) {
          if (!tc::mbar_wait(&bempty[stage], phase ^ 1u, abortp, wc)) { ok = false; break; }
          tc::mbar_arrive_expect_tx(&bfull[stage], 2 * P.b_bytes);
          armed |= 1u << stage;
          armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
          uint8_t* sb = smem + (size_t)stage * 2 * P.b_bytes;
#pragma unroll
          for (int ch = 0; ch < NCH; ++ch) {
            tc::tma_load_2d(sb + (size_t)ch * P.ch0 * 128, &tmBhi, &bfull[stage], a * kAtomK, ch * P.ch0);
            tc::tma_load_2d(sb + P.b_bytes + (size_t)ch * P.ch0 * 128, &tmBlo, &bfull[stage], a * kAtomK,
                            ch * P.ch0);
          }
          if (++stage == kApplyBStages) { stage = 0; phase ^= 1u; }
        }
      }
      if (*abortp) drain_armed(bfull, kApplyBStages, armed, armed_par);
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t id0 = tc::idesc_make(2u, false, false, 128, P.ch0);
      const uint32_t id1 = tc::idesc_make(2u, false, false, 128, NCH > 1 ? ch1 : 16);
      int na[NCH];
#pragma unroll
      for (int ch = 0; ch < NCH; ++ch) na[ch] = atoms_of(ch);
      int stage = 0, slot = 0;
      uint32_t phase = 0, sphase = 0;
      bool ok = true;
      int tcount = 0;
      for (int64_t t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x, ++tcount) {
        // the previous tile's accumulator has been drained
        if (tcount > 0 && !tc::mbar_wait(dempty, (uint32_t)(tcount - 1) & 1u, abortp, wc)) { ok = false; break; }
        tc::fence_after_sync();
        for (int a = 0; a < P.katoms; ++a) {
          if (!tc::mbar_wait(&afull[slot], sphase, abortp, wc) || !tc::mbar_wait(&bfull[stage], phase, abortp, wc)) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sb = tc::smem_u32(smem + (size_t)stage * 2 * P.b_bytes);
          const uint32_t ahi = tbase + kApplySlotCol + (uint32_t)slot * 64u;
          const uint32_t alo = ahi + 32u;
#pragma unroll
          for (int ks = 0; ks < kAtomK / 8; ++ks) {
            const uint32_t acc0 = (a > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) {
              if (a >= na[ch]) continue;
              const uint32_t d = tbase + (uint32_t)(ch * P.ch0);
              const uint32_t id = ch ? id1 : id0;
              const uint32_t boff = (uint32_t)(ch * P.ch0 * 128 + ks * 32);
              const uint64_t bhi = tc::desc_sw128(sb + boff, 16, 1024);
              const uint64_t blo = tc::desc_sw128(sb + P.b_bytes + boff, 16, 1024);
              tc::mma_tf32_ts(d, ahi + (uint32_t)(ks * 8), bhi, id, acc0);
              tc::mma_tf32_ts(d, ahi + (uint32_t)(ks * 8), blo, id, 1u);
              tc::mma_tf32_ts(d, alo + (uint32_t)(ks * 8), bhi, id, 1u);
            }
          }
          tc::mma_commit(&bempty[stage]);
          tc::mma_commit(&aempty[slot]);
          if (++stage == kApplyBStages) { stage = 0; phase ^= 1u; }
          if (++slot == kApplySlots) { slot = 0; sphase ^= 1u; }
        }
        if (!ok) break;
        tc::mma_commit(dfull);
      }
      tc::mma_commit(done);
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(done, 0) && clock64() - t0 < tc::kWaitCycles) {}
    }
  } else if (warp < 6) {
    // ------------------------------------------------------------ converter
    // thread = row r of the tile = TMEM lane r: the row's 32 values of the
    // staged atom (column c at c * 128 + r: a warp reads 32 consecutive
    // floats per column) go to the slot as hi (the container) and lo; the
    // T stage is released once read
    const int q = warp & 3;
    const int r = q * 32 + lane;
    const uint32_t tl = tbase + ((uint32_t)(q * 32) << 16) + kApplySlotCol;
    int stage = 0, slot = 0;
    uint32_t phase = 0, sphase = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < P.ntiles && ok; t += gridDim.x) {
      for (int a = 0; a < P.katoms; ++a) {
        if (!__all_sync(0xffffffffu, tc::mbar_wait(&tfull[stage], phase, abortp, wc))) { ok = false; break; }
        const float* xs = reinterpret_cast<const float*>(tring + (size_t)stage * P.x_bytes);
        float hi[2][16], lo[2][16];
#pragma unroll
        for (int c = 0; c < kAtomK; ++c) {
          const float x = xs[c * 128 + r];
          hi[c >> 4][c & 15] = x;
          lo[c >> 4][c & 15] = tf32_rest(x);
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&tempty[stage]);
        if (!__all_sync(0xffffffffu, tc::mbar_wait(&aempty[slot], sphase ^ 1u, abortp, wc))) { ok = false; break; }
        tc::fence_after_sync();
        const uint32_t ts = tl + (uint32_t)slot * 64u;
        tc::tmem_st16(ts, hi[0]);
        tc::tmem_st16(ts + 16u, hi[1]);
        tc::tmem_st16(ts + 32u, lo[0]);
        tc::tmem_st16(ts + 48u, lo[1]);
        tc::tmem_st_wait();
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&afull[slot]);
        if (++stage == P.tstages) { stage = 0; phase ^= 1u; }
        if (++slot == kApplySlots) { slot = 0; sphase ^= 1u; }
      }
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;
    const int r = q * 32 + lane;
    const uint32_t tl = tbase + ((uint32_t)(q * 32) << 16);
    int tcount = 0;
    for (int64_t t = blockIdx.x; t < P.ntiles; t += gridDim.x, ++tcount) {
      if (!__all_sync(0xffffffffu, tc::mbar_wait(dfull, (uint32_t)tcount & 1u, abortp, wc))) break;
      tc::fence_after_sync();
      const int64_t grow = t * 128 + r;
      const bool rok = grow < P.rows;
      // the 16-bit copy as pairs of rows (one 4-byte store per lane and
      // column pair) when the tile's rows are all in range and aligned
      const bool pack = P.kind16 && t * 128 + 128 <= P.rows && (P.ld16 & 1) == 0 &&
                        (reinterpret_cast<uintptr_t>(P.Y16) & 3) == 0;
      for (int c = 0; c < P.NP; c += 16) {
        float v[16];
        tc::tmem_ld16(tl + (uint32_t)c, v);
        tc::tmem_ld_wait();
        if (rok && P.Y) {
#pragma unroll
          for (int u = 0; u < 16; ++u)
            if (c + u < P.N) P.Y[grow + (int64_t)(c + u) * P.ldy] = v[u];
        }
        if (pack) {
          // even lanes: rows (r, r + 1) of column j; odd lanes: rows
          // (r - 1, r) of column j + 1
          const int odd = lane & 1;
#pragma unroll
          for (int u = 0; u < 16; u += 2) {
            const int j = c + u;
            const float got = __shfl_xor_sync(0xffffffffu, odd ? v[u] : v[u + 1], 1);
            const float a = odd ? got : v[u], b = odd ? v[u + 1] : got;
            const int64_t off = (grow - odd) + (int64_t)(j + odd) * P.ld16;
            if (j + odd < P.N) {
              if (P.kind16 == 1) reinterpret_cast<__nv_bfloat162*>(reinterpret_cast<bf16*>(P.Y16) + off)[0] =
                  __floats2bfloat162_rn(a, b);
              else reinterpret_cast<__half2*>(reinterpret_cast<f16*>(P.Y16) + off)[0] = __floats2half2_rn(a, b);
            }
          }
        } else if (rok && P.kind16) {
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const int j = c + u;
            if (j < P.N) {
              if (P.kind16 == 1)
                reinterpret_cast<bf16*>(P.Y16)[grow + (int64_t)j * P.ld16] = __float2bfloat16_rn(v[u]);
              else
                reinterpret_cast<f16*>(P.Y16)[grow + (int64_t)j * P.ld16] = __float2half_rn(v[u]);
            }
          }
        }
      }
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(dempty);
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (threadIdx.x == 0 && *abortp) raise_status(P.status, SORSVD_ERR_TIMEOUT);
  if (warp == 1) tc::tmem_dealloc(tbase, kTmemCols);
}

int env_tsk() {
  static const int v = [] {
    const char* s = std::getenv("SORSVD_TSK");
    return s ? std::atoi(s) : 1;
  }();
  return v;
}

int round16(int x) { return (x + 15) / 16 * 16; }

// the TMEM blocks of the lower triangle of an l x l Gram (see the header)
int gram_blocks(int l, GramBlock* blk, int* sym_split) {
  const int L16 = round16(l);
  int n = 0;
  if (L16 <= 128) {
    blk[n++] = {0, 0, L16, 0, 0};
    *sym_split = L16;
  } else if (L16 <= 256) {
    blk[n++] = {0, 0, 128, 0, 0};
    blk[n++] = {128, 0, L16, 128, 0};
    *sym_split = L16;
  } else {
    const int w = L16 - 256;
    blk[n++] = {0, 0, 128, 0, 0};
    blk[n++] = {128, 0, 256, 128, 0};
    blk[n++] = {0, 256, w, 384, 0};
    blk[n++] = {128, 256, w, 384 + w, 0};
    blk[n++] = {L16 - 128, 256, w, 384 + 2 * w, 256};
    *sym_split = 256;
  }
  return n;
}

}  // namespace

bool tsk_enabled() { return env_tsk() != 0; }

bool tsk_gram_supported(const float* X, int64_t ldx, int l) {
  if (!tsk_enabled() || l < 1 || l > kTskMaxL) return false;
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (ldx & 3)) return false;
  return true;
}

int tsk_gram_parts(int64_t rows) {
  const int64_t natoms = (rows + kAtomK - 1) / kAtomK;
  return (int)std::max<int64_t>(1, std::min<int64_t>(natoms, num_sms()));
}

cudaError_t launch_tsk_gram(const float* X, int64_t ldx, int64_t rows, int l, float* parts, int* nparts,
                            int* sym_split, const int* skip, DeviceStatus* status, cudaStream_t st) {
  if (rows < 1 || !tsk_gram_supported(X, ldx, l)) return cudaErrorInvalidValue;
  GramParams P{};
  P.rows = rows;
  P.natoms = (rows + kAtomK - 1) / kAtomK;
  P.l = l;
  P.L16 = round16(l);
  P.nblk = gram_blocks(l, P.blk, sym_split);
  // staged columns: every MMA row block reads 128 columns of the tile
  int TR = P.L16;
  for (int b = 0; b < P.nblk; ++b) TR = std::max(TR, P.blk[b].a0 + 128);
  P.nbox = TR > 256 ? 2 : 1;
  P.boxc = TR / P.nbox;                            // a multiple of 8: boxes start on 1024-byte boundaries
  P.tile_bytes = (uint32_t)TR * 128u;
  const uint32_t bar_bytes = 256;
  P.stages = (int)std::min<uint32_t>(4u, (kSmemBudget - bar_bytes) / (2u * P.tile_bytes));
  if (P.stages < 2) return cudaErrorInvalidValue;
  P.parts = parts;
  P.pstride = (int64_t)l * l;
  P.skip = skip;
  P.status = status;
  P.wait_cycles = tc_wait_cycles();
  CUtensorMap m;
  if (!tc_map_2d(&m, X, 2, rows, l, ldx, (uint32_t)kAtomK, (uint32_t)P.boxc, true)) return cudaErrorInvalidValue;
  const int G = tsk_gram_parts(rows);
  *nparts = G;
  const size_t smem = (size_t)P.stages * 2 * P.tile_bytes + bar_bytes + 1024;
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<G, kGramThreads, smem, st>>>(m, P);
    return cudaGetLastError();
  };
  switch (P.nblk) {
    case 1: return go(tsk_gram_kernel<1>);
    case 2: return go(tsk_gram_kernel<2>);
    case 5: return go(tsk_gram_kernel<5>);
    default: return cudaErrorInvalidValue;
  }
}

bool tsk_xty_supported(const float* X, int64_t ldx, const float* Y, int64_t ldy, int l) {
  return tsk_gram_supported(X, ldx, l) && tsk_gram_supported(Y, ldy, l);
}

int tsk_xty_parts(int64_t rows, int l) {
  const int64_t natoms = (rows + kAtomK - 1) / kAtomK;
  const int ntypes = std::max(1, (round16(l) + 127) / 128);
  return (int)std::max<int64_t>(1, std::min<int64_t>(natoms, std::max(1, num_sms() / ntypes)));
}

cudaError_t launch_tsk_xty(const float* X, int64_t ldx, const float* Y, int64_t ldy, int64_t rows, int l,
                           float* parts, int* nparts, const int* skip, DeviceStatus* status, cudaStream_t st) {
  if (rows < 1 || !tsk_xty_supported(X, ldx, Y, ldy, l)) return cudaErrorInvalidValue;
  XtyParams P{};
  P.rows = rows;
  P.natoms = (rows + kAtomK - 1) / kAtomK;
  P.l = l;
  P.L16 = std::max(round16(l), 16);
  P.ntypes = (P.L16 + 127) / 128;
  P.nch = P.L16 > 256 ? 2 : 1;
  P.ch0 = P.nch == 2 ? 256 : P.L16;
  // Y: all L16 columns (two boxes past 256, each starting on a 1024-byte boundary)
  P.nboxy = P.L16 > 256 ? 2 : 1;
  P.boxy = P.L16 / P.nboxy;
  P.x_bytes = 128u * 128u;
  P.y_bytes = (uint32_t)P.L16 * 128u;
  P.stage_bytes = 2u * (P.x_bytes + P.y_bytes);
  const uint32_t bar_bytes = 256;
  P.stages = (int)std::min<uint32_t>(4u, (kSmemBudget - bar_bytes) / P.stage_bytes);
  if (P.stages < 2) return cudaErrorInvalidValue;
  P.parts = parts;
  P.pstride = (int64_t)l * l;
  P.skip = skip;
  P.status = status;
  P.wait_cycles = tc_wait_cycles();
  CUtensorMap mx, my;
  if (!tc_map_2d(&mx, X, 2, rows, l, ldx, (uint32_t)kAtomK, 128u, true)) return cudaErrorInvalidValue;
  if (!tc_map_2d(&my, Y, 2, rows, l, ldy, (uint32_t)kAtomK, (uint32_t)P.boxy, true)) return cudaErrorInvalidValue;
  const int G = tsk_xty_parts(rows, l);
  *nparts = G;
  const size_t smem = (size_t)P.stages * P.stage_bytes + bar_bytes + 1024;
  const dim3 grid((unsigned)G, (unsigned)P.ntypes);
  auto go = [&](auto kern) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, kGramThreads, smem, st>>>(mx, my, P);
    return cudaGetLastError();
  };
  return P.nch == 2 ? go(tsk_xty_kernel<2>) : go(tsk_xty_kernel<1>);
}

bool tsk_apply_supported(const float* X, int64_t ldx, int K, int N) {
  if (!tsk_enabled() || K < 1 || N < 1 || K > kTskMaxL || N > kTskMaxN) return false;
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (ldx & 3)) return false;
  return true;
}

cudaError_t launch_tsk_apply(const float* X, int64_t ldx, int64_t rows, int K, const float* Bhi, const float* Blo,
                             int64_t ldb, int N, bool tri, float* Y, int64_t ldy, void* Y16, int64_t ld16,
                             int kind16, const int* skip, DeviceStatus* status, cudaStream_t st) {
  if (rows < 1) return cudaSuccess;
  if (!tsk_apply_supported(X, ldx, K, N)) return cudaErrorInvalidValue;
  if ((reinterpret_cast<uintptr_t>(Bhi) & 15) || (reinterpret_cast<uintptr_t>(Blo) & 15) || (ldb & 3))
    return cudaErrorInvalidValue;
  ApplyParams P{};
  P.rows = rows;
  P.ntiles = (rows + 127) / 128;
  P.K = K;
  P.N = N;
  P.NP = round16(N);
  P.nch = P.NP > 256 ? 2 : 1;
  P.ch0 = P.nch == 2 ? round16((P.NP + 1) / 2) : P.NP;
  P.katoms = (K + kAtomK - 1) / kAtomK;
  P.tri = tri ? 1 : 0;
  P.b_bytes = (uint32_t)(P.nch * P.ch0) * 128u;
  P.x_bytes = 128u * 128u;
  P.stage_bytes = 2 * P.b_bytes;
  P.Y = Y;
  P.ldy = ldy;
  P.Y16 = Y16;
  P.ld16 = ld16;
  P.kind16 = Y16 ? kind16 : 0;
  P.skip = skip;
  P.status = status;
  P.wait_cycles = tc_wait_cycles();
  const size_t bar_bytes = 512;
  const size_t bring = (size_t)kApplyBStages * P.stage_bytes;
  if (bring + 2 * (size_t)P.x_bytes > kSmemBudget) return cudaErrorInvalidValue;
  P.tstages = (int)std::min<size_t>(kApplyMaxTStages, (kSmemBudget - bring) / P.x_bytes);
  const size_t smem = bring + (size_t)P.tstages * P.x_bytes + bar_bytes + 1024;
  if (smem > 227u * 1024u) return cudaErrorInvalidValue;
  CUtensorMap mx, mh, ml;
  // T: 128 rows x 32 columns per box, unswizzled (column c of the box at c x 512 bytes)
  if (!tc_map_2d(&mx, X, 2, rows, K, ldx, 128u, (uint32_t)kAtomK, false)) return cudaErrorInvalidValue;
  // B: K-major, 32 K x ch0 columns per box, 128-byte swizzle
  if (!tc_map_2d(&mh, Bhi, 2, K, N, ldb, (uint32_t)kAtomK, (uint32_t)P.ch0, true)) return cudaErrorInvalidValue;
  if (!tc_map_2d(&ml, Blo, 2, K, N, ldb, (uint32_t)kAtomK, (uint32_t)P.ch0, true)) return cudaErrorInvalidValue;
  const int G = (int)std::max<int64_t>(1, std::min<int64_t>(P.ntiles, num_sms()));
  cudaError_t e;
  if (P.nch == 2) {
    e = cudaFuncSetAttribute(tsk_apply_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tsk_apply_kernel<2><<<G, kApplyThreads, smem, st>>>(mx, mh, ml, P);
  } else {
    e = cudaFuncSetAttribute(tsk_apply_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    tsk_apply_kernel<1><<<G, kApplyThreads, smem, st>>>(mx, mh, ml, P);
  }
  return cudaGetLastError();
}

}  // namespace sorsvd
