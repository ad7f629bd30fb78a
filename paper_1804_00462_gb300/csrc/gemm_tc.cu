// Tensor-core passes over A (the dense contractions of Algorithm 3):
//   T1 = A T2 and W = A Q2   (op(A) = A:   A is MN-major for the MMA)
//   T2 = A^T T1              (op(A) = A^T: A is K-major for the MMA)
// Output tiles of MT x 128 rows x Npad columns accumulate in tensor memory
// (TMEM) through tcgen05.mma (kind::f16 for bf16/fp16 operands, kind::tf32
// for fp32 containers), fed by TMA loads into 128-byte-swizzled
// shared-memory stages.  A stage holds KA "atoms" along K (one atom = one
// 128-byte swizzle row per matrix row: 64 bf16 / 32 fp32 elements) for each
// of the MT row blocks, and the matching KA atoms of the skinny operand B,
// which all MT row blocks share.  KA sets the contiguous run read from each
// column of a column-major A per stage (KA x 128 bytes); MT = 2 halves the
// re-reads of B from L2.
//
// Work decomposition: a persistent grid of G <= #SM units splits the
// tiles x K-stages iteration space into G contiguous ranges ("stream-K"),
// so every SM streams the same share of A whatever the tile count.  A unit
// is one CTA; it walks its range as segments (one per output tile it
// touches).  A segment that covers a whole tile is
// written straight to the output; the at most two partial segments of a CTA
// (head and tail of its range) go to a per-CTA partial buffer, and the CTA
// that finishes a split tile last (a per-tile counter) sums its shares in
// CTA order and writes the tile: deterministic, no atomics on the data.
// Without counters a separate fix-up kernel does the same sum.
//
// Split mode (ELT 3, fp32 containers, K-major only, MT = 1, KA = 1): the
// MMAs read the staged fp32 tile x of A as hi = trunc_tf32(x) (kind::tf32
// ignores the low 13 mantissa bits of a container), and a fourth warpgroup
// reads x (one row per thread) and puts lo = x - hi (exact in fp32) into a
// TMEM slot (or, for N > 112, next to the tile in shared memory).  B comes split
// the same way from two tensors prepared by the caller and sits in the stage
// as one 2 N-row operand [B_hi | B_lo].  Every K step issues two MMAs:
// hi x [B_hi | B_lo] (N = 2 Npad) into [D1 | D2] of the current fill buffer
// and lo x B_hi into D2 of the other buffer.  Back-to-back MMAs on one
// accumulator serialise (~115 cycles each for N <= 224, measured), so one
// wide MMA plus one on an independent accumulator keeps the tensor pipe
// busy where three N = Npad MMAs on one accumulator left it half idle.  The
// neglected lo*lo term and the TF32 truncation of lo are below 2^-20
// relative and of random sign, so the products carry fp32-level error.
// The hi*hi columns D1 drain every kDrainAtoms atoms; the correction
// columns D2 (2^-11 of the result) drain once per tile segment.
//
// Warp roles (224 threads): warp 0 issues the TMA loads of A into a deep
// ring (HBM latency), warp 6 those of B into a short ring (B is re-read
// from L2), warp 1 owns the TMEM allocation and issues MMAs (one lane),
// warps 2-5 drain accumulators (tcgen05.ld, 32 TMEM lanes per warp) into
// fp32 output and, optionally, a 16-bit copy used as the next pass's
// operand; in split mode warps 7-10 convert.  Accumulators are
// double-buffered in TMEM when 2 MT Npad <= 512 columns, so the epilogue of
// one segment overlaps the MMAs of the next.  Every mbarrier wait is
// bounded (tc::kWaitCycles); a timeout records SORSVD_ERR_TIMEOUT, stops all
// roles, waits for the copies and MMAs already issued, frees TMEM and exits.
#include "internal.cuh"
#include "profile.cuh"
#include "tc_ptx.cuh"

#include <algorithm>
#include <cstdlib>

namespace sorsvd {

struct TcParams {
  int64_t M, K;          // output rows, reduction length
  int N, Npad, nch, ch0; // output columns, padded, N-chunks of ch0 rows
  int KA, MT;            // K atoms per stage, 128-row blocks per tile
  int64_t tiles, ipt, total;
  int G;                 // stream-K units (CTAs)
  int nbuf;
  int pair;              // CTA pairs (cta_group::2): G pairs of CTAs, 256-row tiles
  int hb;                // pair mode: rows of B per CTA in one N-chunk box
  uint32_t tmem_cols;
  int lo_tmem;           // split mode: A's low parts in TMEM slots (else next to A in shared memory)
  int aslots;            // split mode: converted stages in flight (TMEM slots / handshakes)
  uint32_t aslot_col;    // split mode: first TMEM column of the low-part slots
  int stages, bstages;   // ring depths: A (from HBM), B (from L2)
  uint32_t stage_bytes, a_bytes, b_atom, b_bytes, bstage_bytes;
  float* out;
  int64_t ldo;
  void* out16;           // optional 16-bit copy of the output (bf16 / fp16)
  int64_t ld16;
  int out16_kind;        // 0 none, 1 bf16, 2 fp16
  float* parts;          // G x 2 x (128 MT) x Npad fp32
  int* tilecnt;          // per tile: shares written so far (zero between launches), or null
  DeviceStatus* status;
  long long wait_cycles; // limit of the waits for pipeline progress (the waits for
                         // copies and MMAs in flight after an abort keep tc::kWaitCycles)
};

namespace {

constexpr int kThreads = 224;
constexpr int kThreadsSplit = 352;
// Split mode drains each accumulator fill of kDrainAtoms K atoms into a
// running sum held in the epilogue threads' registers (round-to-nearest fp32
// adds): tensor-core accumulation truncates, which over thousands of MMA
// steps biases long fp32 sums by ~1e-5; short fills bound that bias (the
// correction block D2, 2^-11 of the result, drains once per segment).  The
// two fill buffers [D1 | D2] take 4 Npad <= 512 TMEM columns (l <= kAccCols).
constexpr int kDrainAtoms = 4;
constexpr int kAccCols = 128;
// split mode: the two fill buffers [D1 | D2] take 4 Npad TMEM columns; the
// low parts of A take 32 columns per stage above them when they fit (up to
// kASlots stages in flight)
constexpr uint32_t kASlotCols = 32u;
constexpr uint32_t kASlots = 4u;
constexpr int kLoTmemMaxNpad = 112;
constexpr uint32_t kAtomBytes = 128u * 128u;   // 128 rows x 128 bytes
constexpr int kMaxKA = 2;                      // K atoms per stage, at most

// round-to-nearest-even of an fp32 value to TF32 (10 explicit mantissa bits);
// finite inputs
__device__ __forceinline__ float rn_tf32(float x) {
  uint32_t u = __float_as_uint(x);
  u = (u + 0xFFFu + ((u >> 13) & 1u)) & 0xFFFFE000u;
  return __uint_as_float(u);
}
// x - trunc_tf32(x): the part of x a TF32 MMA ignores (exact in fp32)
__device__ __forceinline__ float tf32_rest(float x) {
  return x - __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__host__ __device__ __forceinline__ int64_t cta_of(int64_t x, int64_t total, int64_t G) {
  // the CTA whose iteration range [c*total/G, (c+1)*total/G) holds x
  return ((x + 1) * G + total - 1) / total - 1;
}

__device__ __forceinline__ void store_out(const TcParams& P, int64_t grow, int col, float v) {
  P.out[grow + (int64_t)col * P.ldo] = v;
  if (P.out16_kind == 1) reinterpret_cast<bf16*>(P.out16)[grow + (int64_t)col * P.ld16] = __float2bfloat16_rn(v);
  else if (P.out16_kind == 2) reinterpret_cast<f16*>(P.out16)[grow + (int64_t)col * P.ld16] = __float2half_rn(v);
}

// Sum of the shares of split tile t (rows row0.., mrows x N), CTA c0's share
// from slot slot0 and the others' from slot 0, in CTA order (fp32); 4
// consecutive rows per float4, 4 float4 per thread in flight.
// The shares of unit cc live in the partial slots of CTA cc * cs + cr (CTA
// pairs: cs = 2 and cr the CTA's rank in its pair).
__device__ void sum_split_tile(const TcParams& P, int64_t row0, int mrows, int64_t c0, int64_t c1, int slot0,
                               int cs = 1, int cr = 0) {
  const int per = mrows * P.N;
  const size_t seg = (size_t)mrows * P.Npad;
  auto share = [&](int64_t cc, int slot) {
    return reinterpret_cast<const float4*>(P.parts + ((size_t)(cc * cs + cr) * 2 + slot) * seg);
  };
  const int q4 = mrows / 4, nv = per / 4;
  const float4* first = share(c0, slot0);
  for (int f0 = threadIdx.x; f0 < nv; f0 += 4 * blockDim.x) {
    float acc[4][4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int f = f0 + b * blockDim.x;
      if (f < nv) {
        const int col = f / q4, r4 = f - col * q4;
        const float4 x = first[(size_t)r4 + (size_t)col * q4];
        acc[b][0] = x.x; acc[b][1] = x.y; acc[b][2] = x.z; acc[b][3] = x.w;
      }
    }
    for (int64_t cc = c0 + 1; cc <= c1; ++cc) {
      const float4* pc = share(cc, 0);
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int f = f0 + b * blockDim.x;
        if (f < nv) {
          const int col = f / q4, r4 = f - col * q4;
          const float4 x = pc[(size_t)r4 + (size_t)col * q4];
          acc[b][0] += x.x; acc[b][1] += x.y; acc[b][2] += x.z; acc[b][3] += x.w;
        }
      }
    }
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      const int f = f0 + b * blockDim.x;
      if (f >= nv) continue;
      const int col = f / q4, r4 = f - col * q4;
      const int64_t grow = row0 + 4 * r4;
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (grow + u < P.M) store_out(P, grow + u, col, acc[b][u]);
    }
  }
}

// ELT: 0 bf16, 1 fp16, 2 tf32, 3 tf32 split (3 MMAs).  A_MN: A operand
// MN-major (op(A) = A).  MT, NCH, KA: the launch's row blocks per tile,
// N-chunks and K atoms per stage, fixed at compile time so that the MMA
// issue loop is straight-line code (issued from a rolled loop, the same
// tcgen05.mma sequence ran 2-4x slower, measured).
template <int ELT, bool A_MN, int MT, int NCH, int KA>
__global__ void __launch_bounds__((ELT == 3 ? kThreadsSplit : kThreads), 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const __grid_constant__ CUtensorMap tmBlo, const TcParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* bring = smem + (size_t)P.stages * P.stage_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(bring + (size_t)P.bstages * P.bstage_bytes);
  uint64_t* empty = full + P.stages;
  uint64_t* bfull = empty + P.stages;
  uint64_t* bempty = bfull + P.bstages;
  uint64_t* tfull = bempty + P.bstages;
  uint64_t* tempty = tfull + 2;
  uint64_t* done = tempty + 2;
  uint64_t* afull = done + 1;         // split mode: stage converted (4 converter warps)
  uint64_t* aempty = afull + kASlots; // split mode: its low-part slot consumed by the MMAs
  uint32_t* tslot = reinterpret_cast<uint32_t*>(aempty + kASlots);
  volatile int* abortp = reinterpret_cast<volatile int*>(tslot + 1);
  volatile int* lastp = abortp + 1;   // split tiles this CTA finishes: bit 0 head, bit 1 tail

  constexpr bool SPLIT = (ELT == 3);
  constexpr int AK = (ELT >= 2) ? 32 : 64;              // K elements per atom
  constexpr int KMMA = (ELT >= 2) ? 8 : 16;             // K per MMA
  constexpr int AMN = (ELT >= 2) ? 32 : 64;             // MN width of an MN-major box
  constexpr uint32_t AMN_BOX = (uint32_t)AK * 128u;     // bytes of one MN-major A box
  constexpr uint32_t FMT = (ELT == 0) ? 1u : (ELT == 1 ? 0u : 2u);
  // accumulator fill length in stages (split mode drains every kDrainAtoms atoms)
  const int64_t CHUNK = SPLIT ? (int64_t)((kDrainAtoms + KA - 1) / KA) : ((int64_t)1 << 40);
  const int mrows = 128 * MT;
  const int64_t urows = mrows;                           // rows of a unit tile

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
    for (int s = 0; s < P.bstages; ++s) { tc::mbar_init(&bfull[s], 1); tc::mbar_init(&bempty[s], 1); }
    for (int b = 0; b < 2; ++b) { tc::mbar_init(&tfull[b], 1); tc::mbar_init(&tempty[b], 128); }
    tc::mbar_init(done, 1);
    if (SPLIT)
      for (uint32_t b = 0; b < kASlots; ++b) { tc::mbar_init(&afull[b], 4); tc::mbar_init(&aempty[b], 1); }
    *abortp = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tslot, P.tmem_cols);
    tc::tmem_relinquish();
  }
  if (warp == 0 && lane == 0) tc::prefetch_tmap(&tmA);
  if (warp == 6 && lane == 0) { tc::prefetch_tmap(&tmB); if (SPLIT) tc::prefetch_tmap(&tmBlo); }
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  if constexpr (SPLIT) {
    // the MMAs always accumulate: the fill buffers start at zero, and the
    // epilogue zeroes what it drains
    if (warp >= 2 && warp <= 5) {
      const uint32_t tz = tbase + ((uint32_t)((warp & 3) * 32) << 16);
      float z[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) z[i] = 0.f;
      for (int c = 0; c < 4 * P.Npad; c += 16) tc::tmem_st16(tz + (uint32_t)c, z);
      tc::tmem_st_wait();
      tc::fence_before_sync();
    }
    __syncthreads();
    tc::fence_after_sync();
  }

  // the stream-K unit of this CTA
  const int rank = 0;
  const int64_t cta = (int64_t)blockIdx.x;
  const int64_t it0 = cta * P.total / P.G, it1 = (cta + 1) * P.total / P.G;

  if (warp == 0) {
    // ------------------------------------------------------------ producer of A
    if (lane == 0) {
      const uint64_t polA = tc::policy_evict_first();
      uint32_t stage = 0, phase = 0;
      uint32_t armed = 0;          // bit s: stage s armed and not yet seen consumed
      uint32_t armed_par = 0;      // parity of that armed phase
      bool ok = true;
      for (int64_t g = it0; g < it1 && ok;) {
        const int64_t t = g / P.ipt;
        const int64_t gend = min(it1, (t + 1) * P.ipt);
        for (int64_t kb = g - t * P.ipt; kb < gend - t * P.ipt; ++kb) {
          if (!tc::mbar_wait(&empty[stage], phase ^ 1, abortp, P.wait_cycles)) { ok = false; break; }
          tc::mbar_arrive_expect_tx(&full[stage], P.a_bytes);
          armed |= 1u << stage;
          armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
          uint8_t* sa = smem + (size_t)stage * P.stage_bytes;
          for (int j = 0; j < KA; ++j) {
            const int k = (int)((kb * KA + j) * AK);
            for (int mt = 0; mt < MT; ++mt) {
              uint8_t* dst = sa + (size_t)(mt * KA + j) * kAtomBytes;
              const int row0 = (int)(t * urows) + rank * mrows + mt * 128;
              if (A_MN) {
#pragma unroll
                for (int h = 0; h < 128 / AMN; ++h)
                  tc::tma_load_2d_hint(dst + h * AMN_BOX, &tmA, &full[stage], row0 + h * AMN, k, polA);
              } else {
                tc::tma_load_2d_hint(dst, &tmA, &full[stage], k, row0, polA);
              }
            }
          }
          if (++stage == (uint32_t)P.stages) { stage = 0; phase ^= 1; }
        }
        g = gend;
      }
      if (!ok) {
        // let the copies already issued land before the CTA exits
        for (int s = 0; s < P.stages; ++s)
          if (armed & (1u << s)) {
            const long long t0 = clock64();
            while (!tc::mbar_try_wait(&full[s], (armed_par >> s) & 1u) && clock64() - t0 < tc::kWaitCycles) {}
          }
      }
    }
  } else if (warp == 6) {
    // ------------------------------------------------------------ producer of B
    // the skinny operand comes from L2: a short ring suffices
    if (lane == 0) {
      const uint64_t polB = tc::policy_evict_last();
      uint32_t stage = 0, phase = 0;
      uint32_t armed = 0, armed_par = 0;
      bool ok = true;
      for (int64_t g = it0; g < it1 && ok;) {
        const int64_t t = g / P.ipt;
        const int64_t gend = min(it1, (t + 1) * P.ipt);
        for (int64_t kb = g - t * P.ipt; kb < gend - t * P.ipt; ++kb) {
          if (!tc::mbar_wait(&bempty[stage], phase ^ 1, abortp, P.wait_cycles)) { ok = false; break; }
          tc::mbar_arrive_expect_tx(&bfull[stage], (SPLIT ? 2u : 1u) * P.b_bytes);
          armed |= 1u << stage;
          armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
          uint8_t* sb = bring + (size_t)stage * P.bstage_bytes;
          for (int j = 0; j < KA; ++j) {
            const int k = (int)((kb * KA + j) * AK);
            for (int ch = 0; ch < NCH; ++ch) {
              const size_t off = (size_t)j * P.b_atom + (size_t)ch * P.ch0 * 128;
              tc::tma_load_2d_hint(sb + off, &tmB, &bfull[stage], k, ch * P.ch0, polB);
              if (SPLIT) tc::tma_load_2d_hint(sb + P.b_bytes + off, &tmBlo, &bfull[stage], k, ch * P.ch0, polB);
            }
          }
          if (++stage == (uint32_t)P.bstages) { stage = 0; phase ^= 1; }
        }
        g = gend;
      }
      if (!ok) {
        for (int s2 = 0; s2 < P.bstages; ++s2)
          if (armed & (1u << s2)) {
            const long long t0 = clock64();
            while (!tc::mbar_try_wait(&bfull[s2], (armed_par >> s2) & 1u) && clock64() - t0 < tc::kWaitCycles) {}
          }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      const uint32_t idesc0 = tc::idesc_make(FMT, A_MN, false, 128, P.ch0);
      // the last N-chunk takes what the equal chunks before it leave
      const uint32_t idesc1 = tc::idesc_make(FMT, A_MN, false, 128, NCH > 1 ? P.Npad - (NCH - 1) * P.ch0 : 16);
      // split mode: hi x [B_hi | B_lo], N = 2 Npad
      const uint32_t idescW = tc::idesc_make(FMT, false, false, 128, SPLIT ? 2 * P.Npad : 16);
      uint32_t stage = 0, phase = 0, bstage = 0, bphase = 0;
      uint32_t aslot = 0, aphase = 0;  // split mode: converted-stage ring
      int chunk = 0;                 // accumulator fills (TMEM buffer alternation)
      bool ok = true;
      for (int64_t g = it0; g < it1 && ok;) {
        const int64_t t = g / P.ipt;
        const int64_t gend = min(it1, (t + 1) * P.ipt);
        const int64_t kb0 = g - t * P.ipt, kb1 = gend - t * P.ipt;
        for (int64_t c0 = kb0; c0 < kb1 && ok; c0 += CHUNK) {
          const int64_t c1 = min(kb1, c0 + CHUNK);
          const int b = (P.nbuf == 2) ? (chunk & 1) : 0;
          const uint32_t use = (P.nbuf == 2) ? (uint32_t)(chunk >> 1) : (uint32_t)chunk;
          if (!tc::mbar_wait(&tempty[b], (use & 1u) ^ 1u, abortp, P.wait_cycles)) { ok = false; break; }
          if (SPLIT && c0 == kb0 && chunk > 0) {
            // a new segment: the previous fill (the last of the previous
            // segment) has had both correction blocks D2 read and zeroed
            const int pc = chunk - 1;
            if (!tc::mbar_wait(&tempty[pc & 1], (uint32_t)(pc >> 1) & 1u, abortp, P.wait_cycles)) { ok = false; break; }
          }
          tc::fence_after_sync();
          const uint32_t dcol = tbase + (uint32_t)(b * MT * P.Npad);
          for (int64_t kb = c0; kb < c1; ++kb) {
            if constexpr (SPLIT) {
              if (!tc::mbar_wait(&afull[aslot], aphase, abortp, P.wait_cycles)) { ok = false; break; }
            } else {
              if (!tc::mbar_wait(&full[stage], phase, abortp, P.wait_cycles)) { ok = false; break; }
            }
            if (!tc::mbar_wait(&bfull[bstage], bphase, abortp, P.wait_cycles)) { ok = false; break; }
            tc::fence_after_sync();
            const uint32_t sb = tc::smem_u32(bring + (size_t)bstage * P.bstage_bytes);
            if constexpr (SPLIT) {
              // hi x [B_hi | B_lo] into [D1 | D2] of buffer b (A_hi: the fp32
              // stage itself), lo x B_hi into D2 of buffer 1 - b (A_lo from
              // its TMEM slot, or from the stage after the tile)
              const uint32_t sa = tc::smem_u32(smem + (size_t)stage * P.stage_bytes);
              const uint32_t dw = tbase + (uint32_t)(b * 2 * P.Npad);
              const uint32_t dc = tbase + (uint32_t)((1 - b) * 2 * P.Npad + P.Npad);
              const uint32_t alo = tbase + P.aslot_col + aslot * kASlotCols;
#pragma unroll
              for (int ks = 0; ks < AK / KMMA; ++ks) {
                const uint64_t ad = tc::desc_sw128(sa + ks * 32, 16, 1024);
                const uint64_t bd = tc::desc_sw128(sb + ks * 32, 16, 1024);
                tc::mma_tf32(dw, ad, bd, idescW, 1u);
                if (P.lo_tmem) tc::mma_tf32_ts(dc, alo + (uint32_t)(ks * KMMA), bd, idesc0, 1u);
                else tc::mma_tf32(dc, tc::desc_sw128(sa + P.a_bytes + ks * 32, 16, 1024), bd, idesc0, 1u);
              }
              tc::mma_commit(&empty[stage]);
              tc::mma_commit(&aempty[aslot]);
              tc::mma_commit(&bempty[bstage]);
              if (++stage == (uint32_t)P.stages) { stage = 0; phase ^= 1; }
              if (++aslot == (uint32_t)P.aslots) { aslot = 0; aphase ^= 1u; }
            } else {
            const uint32_t sa = tc::smem_u32(smem + (size_t)stage * P.stage_bytes);
#pragma unroll
            for (int j = 0; j < KA; ++j) {
#pragma unroll
              for (int ks = 0; ks < AK / KMMA; ++ks) {
                const uint32_t acc = (kb > c0 || j > 0 || ks > 0) ? 1u : 0u;
#pragma unroll
                for (int mt = 0; mt < MT; ++mt) {
                  const uint32_t aat = sa + (uint32_t)(mt * KA + j) * kAtomBytes;
                  const uint64_t ad = A_MN ? tc::desc_sw128(aat + ks * KMMA * 128, AMN_BOX, 1024)
                                           : tc::desc_sw128(aat + ks * 32, 16, 1024);
                  const uint32_t dm = dcol + (uint32_t)(mt * P.Npad);
#pragma unroll
                  for (int ch = 0; ch < NCH; ++ch) {
                    const uint32_t id = (ch == NCH - 1 && NCH > 1) ? idesc1 : idesc0;
                    const uint32_t dch = dm + (uint32_t)(ch * P.ch0);
                    const uint32_t bat = sb + (uint32_t)j * P.b_atom + (uint32_t)(ch * P.ch0 * 128);
                    const uint64_t bd = tc::desc_sw128(bat + ks * 32, 16, 1024);
                    if (ELT == 2) tc::mma_tf32(dch, ad, bd, id, acc);
                    else tc::mma_f16(dch, ad, bd, id, acc);
                  }
                }
              }
            }
            tc::mma_commit(&empty[stage]);
            tc::mma_commit(&bempty[bstage]);
            if (++stage == (uint32_t)P.stages) { stage = 0; phase ^= 1; }
            }
            if (++bstage == (uint32_t)P.bstages) { bstage = 0; bphase ^= 1; }
          }
          if (!ok) break;
          tc::mma_commit(&tfull[b]);
          ++chunk;
        }
        g = gend;
      }
      // every MMA issued by this thread has completed once `done` flips
      tc::mma_commit(done);
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(done, 0) && clock64() - t0 < tc::kWaitCycles) {}
    }
  } else if (SPLIT && warp >= 7) {
    // ------------------------------------------------------------ converter
    // thread = row r of the 128-row block = TMEM lane r (warp 7 + i covers
    // lanes 32 ((7 + i) mod 4) ..): the row's 32 fp32 values come from the
    // 128-byte-swizzled stage (16-byte chunk c of row r sits at chunk
    // c ^ (r mod 8), conflict-free across 8 rows); lo goes to the row's TMEM
    // lane in the slot (tcgen05.st) or to the same place one tile on.  B
    // arrives already split (hi and lo tensors).
    const int q = warp & 3;
    const int r = q * 32 + lane;
    const uint32_t tlane = tbase + ((uint32_t)(q * 32) << 16) + P.aslot_col;
    uint32_t stage = 0, phase = 0, aslot = 0, aphase = 0;
    bool ok = true;
    for (int64_t g = it0; g < it1 && ok;) {
      const int64_t t = g / P.ipt;
      const int64_t gend = min(it1, (t + 1) * P.ipt);
      for (int64_t kb = g - t * P.ipt; kb < gend - t * P.ipt; ++kb) {
        // warp-uniform: the tcgen05.st below is a warp-collective
        if (!__all_sync(0xffffffffu, tc::mbar_wait(&full[stage], phase, abortp, P.wait_cycles))) { ok = false; break; }
        uint8_t* row = smem + (size_t)stage * P.stage_bytes + (size_t)r * 128;
        float lo[2][16];
#pragma unroll
        for (int c = 0; c < 8; ++c) {
          const float4* px = reinterpret_cast<const float4*>(row + ((c ^ (r & 7)) << 4));
          const float4 x = *px;
          const float4 l = make_float4(tf32_rest(x.x), tf32_rest(x.y), tf32_rest(x.z), tf32_rest(x.w));
          if (P.lo_tmem) {
            lo[c >> 2][(4 * c) & 15] = l.x;
            lo[c >> 2][(4 * c + 1) & 15] = l.y;
            lo[c >> 2][(4 * c + 2) & 15] = l.z;
            lo[c >> 2][(4 * c + 3) & 15] = l.w;
          } else {
            *reinterpret_cast<float4*>(reinterpret_cast<uint8_t*>(const_cast<float4*>(px)) + P.a_bytes) = l;
          }
        }
        if (!P.lo_tmem) fence_proxy_async();   // generic writes -> tensor-core reads
        // at most aslots converted stages ahead of the MMAs
        if (!__all_sync(0xffffffffu, tc::mbar_wait(&aempty[aslot], aphase ^ 1u, abortp, P.wait_cycles))) {
          ok = false;
          break;
        }
        if (P.lo_tmem) {
          tc::fence_after_sync();
          const uint32_t ta = tlane + aslot * kASlotCols;
          tc::tmem_st16(ta, lo[0]);
          tc::tmem_st16(ta + 16, lo[1]);
          tc::tmem_st_wait();
          tc::fence_before_sync();
        }
        __syncwarp();
        if (lane == 0) tc::mbar_arrive(&afull[aslot]);
        if (++stage == (uint32_t)P.stages) { stage = 0; phase ^= 1; }
        if (++aslot == (uint32_t)P.aslots) { aslot = 0; aphase ^= 1u; }
      }
      g = gend;
    }
  } else if (warp >= 2 && warp <= 5) {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                    // TMEM lane quarter of this warp
    int chunk = 0;
    bool ok = true;
    for (int64_t g = it0; g < it1 && ok;) {
      const int64_t t = g / P.ipt;
      const int64_t gend = min(it1, (t + 1) * P.ipt);
      const int64_t kb0 = g - t * P.ipt, kb1 = gend - t * P.ipt;
      const bool whole = (g == t * P.ipt) && (gend == (t + 1) * P.ipt);
      float* pdst = nullptr;
      if (!whole) {
        const int slot = (t == it0 / P.ipt) ? 0 : 1;
        pdst = P.parts + ((size_t)blockIdx.x * 2 + slot) * mrows * P.Npad;
      }
      if constexpr (SPLIT) {
        // MT = 1: one row per thread; the running sum of the fills lives in
        // registers (columns past Npad stay unused)
        const int row = q * 32 + lane;
        const int64_t grow = t * urows + rank * mrows + row;
        float sum[kAccCols];
#pragma unroll
        for (int i = 0; i < kAccCols; ++i) sum[i] = 0.f;
        const uint32_t tq = tbase + ((uint32_t)(q * 32) << 16);
        float z[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) z[i] = 0.f;
        // add TMEM columns [col, col + Npad) of this row into the running
        // sum (round-to-nearest fp32 adds) and zero them for the next fill
        auto drain = [&](uint32_t col) {
#pragma unroll
          for (int cc = 0; cc < kAccCols; cc += 16) {
            if (cc < P.Npad) {
              float v[16];
              tc::tmem_ld16(tq + col + cc, v);
              tc::tmem_ld_wait();
#pragma unroll
              for (int i = 0; i < 16; ++i) sum[cc + i] += v[i];
              tc::tmem_st16(tq + col + cc, z);
            }
          }
        };
        for (int64_t c0 = kb0; c0 < kb1; c0 += CHUNK) {
          const int b = chunk & 1;
          const uint32_t use = (uint32_t)(chunk >> 1);
          // warp-uniform: tcgen05.ld / st are warp-collectives
          if (!__all_sync(0xffffffffu, tc::mbar_wait(&tfull[b], use & 1u, abortp, P.wait_cycles))) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          drain((uint32_t)(b * 2 * P.Npad));               // D1 of this fill
          if (c0 + CHUNK >= kb1) {
            // the segment's last fill: every MMA of the segment is complete,
            // so both correction blocks D2 are final
            drain((uint32_t)P.Npad);
            drain((uint32_t)(3 * P.Npad));
          }
          tc::tmem_st_wait();
          tc::fence_before_sync();
          tc::mbar_arrive(&tempty[b]);
          ++chunk;
        }
        if (ok) {
#pragma unroll
          for (int cb = 0; cb < kAccCols; cb += 16) {
            if (cb < P.N) {
#pragma unroll
              for (int i = 0; i < 16; ++i) {
                if (cb + i < P.N) {
                  if (whole) { if (grow < P.M) store_out(P, grow, cb + i, sum[cb + i]); }
                  else pdst[row + (size_t)(cb + i) * mrows] = sum[cb + i];
                }
              }
            }
          }
        }
      } else {
      for (int64_t c0 = kb0; c0 < kb1; c0 += CHUNK) {
        const int b = (P.nbuf == 2) ? (chunk & 1) : 0;
        const uint32_t use = (P.nbuf == 2) ? (uint32_t)(chunk >> 1) : (uint32_t)chunk;
        if (!__all_sync(0xffffffffu, tc::mbar_wait(&tfull[b], use & 1u, abortp, P.wait_cycles))) {
          ok = false;
          break;
        }
        tc::fence_after_sync();
        for (int mt = 0; mt < MT; ++mt) {
          const uint32_t taddr =
              tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * MT * P.Npad + mt * P.Npad);
          const int row = mt * 128 + q * 32 + lane;
          const int64_t grow = t * urows + rank * mrows + row;
          for (int cb = 0; cb < P.N; cb += 16) {
            float v[16];
            tc::tmem_ld16(taddr + cb, v);
            tc::tmem_ld_wait();
            if (whole) {
              if (grow < P.M) {
#pragma unroll
                for (int i = 0; i < 16; ++i)
                  if (cb + i < P.N) store_out(P, grow, cb + i, v[i]);
              }
            } else {
#pragma unroll
              for (int i = 0; i < 16; ++i)
                if (cb + i < P.N) pdst[row + (size_t)(cb + i) * mrows] = v[i];
            }
          }
        }
        tc::fence_before_sync();
        tc::mbar_arrive(&tempty[b]);
        ++chunk;
      }
      }
      g = gend;
    }
  }
  // every share of a split tile is in memory before its counter moves
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0 && *abortp) raise_status(P.status, SORSVD_ERR_TIMEOUT);
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, P.tmem_cols);
  }
  // Split tiles: the CTA that writes the last share of a tile sums the
  // shares in CTA order (as the separate fix-up kernel does) and writes the
  // tile; no CTA waits for another.
  if (P.tilecnt && !*abortp) {
    const int64_t th = it0 / P.ipt, tt = (it1 - 1) / P.ipt;
    const bool head_split = (it0 % P.ipt != 0) || (it1 < (th + 1) * P.ipt);
    const bool tail_split = tt != th && (it1 % P.ipt != 0);
    if (threadIdx.x == 0) {
      int bits = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool split = h ? tail_split : head_split;
        if (!split) continue;
        const int64_t t = h ? tt : th;
        const int64_t c0 = cta_of(t * P.ipt, P.total, P.G), c1 = cta_of(t * P.ipt + P.ipt - 1, P.total, P.G);
        if (atomicAdd(&P.tilecnt[t], 1) == (int)(c1 - c0)) bits |= 1 << h;
      }
      *lastp = bits;
    }
    __syncthreads();
    const int bits = *lastp;
    if (bits) {
      __threadfence();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!((bits >> h) & 1)) continue;
        const int64_t t = h ? tt : th;
        const int64_t c0 = cta_of(t * P.ipt, P.total, P.G), c1 = cta_of(t * P.ipt + P.ipt - 1, P.total, P.G);
        const int slot0 = (c0 * P.total / P.G < t * P.ipt) ? 1 : 0;
        sum_split_tile(P, t * urows + rank * mrows, mrows, c0, c1, slot0);
        if (threadIdx.x == 0) P.tilecnt[t] = 0;     // ready for the next launch
      }
    }
  }
}

// Pair mode (16-bit operands, N > 128): the 152 SMs run as 76 CTA pairs, a
// pair per 256-row tile.  Each CTA stages its own 128 rows of A and half of
// the columns of each N-chunk of B; the even CTA issues cta_group::2 MMAs
// (M = 256) that read both CTAs' stages and accumulate each CTA's 128 rows
// in its own tensor memory.  Per SM this halves the bytes of B staged from
// L2 and the shared memory B needs, which leaves room for a deeper ring of
// A (HBM latency): at l = 266 a K atom of B is 2.3 times the matching atom
// of A in a single CTA.
//   barriers: the stage barriers (full, bfull) and the accumulator-drained
//   barrier (tempty, 2 x 128 epilogue threads) of the even CTA count both
//   CTAs' copies and drains; each CTA has its own empty, bempty and tfull,
//   which the even CTA's MMA thread signals by one commit per barrier,
//   addressed to that CTA.  Both CTAs walk the same stream-K range; the
//   odd CTA writes rows 128..255 of every tile.  Every wait is bounded;
//   both CTAs meet at a cluster barrier before the tensor memory is freed.
template <int ELT, bool A_MN, int NCH, int KA>
__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(kThreads, 1)
tc_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const TcParams P) {
  static_assert(ELT == 0 || ELT == 1, "pair mode: 16-bit operands");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint8_t* bring = smem + (size_t)P.stages * P.stage_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(bring + (size_t)P.bstages * P.bstage_bytes);
  uint64_t* empty = full + P.stages;
  uint64_t* bfull = empty + P.stages;
  uint64_t* bempty = bfull + P.bstages;
  uint64_t* tfull = bempty + P.bstages;
  uint64_t* tempty = tfull + 2;
  uint64_t* done = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abortp = reinterpret_cast<volatile int*>(tslot + 1);
  volatile int* lastp = abortp + 1;

  constexpr int AK = 64, KMMA = 16, AMN = 64;
  constexpr uint32_t AMN_BOX = (uint32_t)AK * 128u;
  constexpr uint32_t FMT = (ELT == 0) ? 1u : 0u;
  const uint32_t rank = tc::cluster_rank();
  const bool leader = rank == 0;
  const uint32_t peer = rank ^ 1u;
  constexpr int mrows = 128;
  constexpr int64_t urows = 256;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
    for (int s = 0; s < P.bstages; ++s) { tc::mbar_init(&bfull[s], 1); tc::mbar_init(&bempty[s], 1); }
    for (int b = 0; b < 2; ++b) { tc::mbar_init(&tfull[b], 1); tc::mbar_init(&tempty[b], 2 * 128); }
    tc::mbar_init(done, 1);
    *abortp = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc_pair(tslot, P.tmem_cols);
    tc::tmem_relinquish_pair();
    tc::fence_before_sync();
  }
  if (warp == 0 && lane == 0) tc::prefetch_tmap(&tmA);
  if (warp == 6 && lane == 0) tc::prefetch_tmap(&tmB);
  // the barriers of both CTAs are initialised before either CTA signals one
  tc::cluster_sync();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;

  // the stream-K unit of this pair
  const int64_t unit = (int64_t)(blockIdx.x >> 1);
  const int64_t it0 = unit * P.total / P.G, it1 = (unit + 1) * P.total / P.G;
  auto lead_cl = [&](uint64_t* b) { return tc::mapa(tc::smem_u32(b), 0u); };
  // the last use of each ring slot is released (by a commit of the even
  // CTA) before this CTA may exit: n fills of a ring of depth d
  auto drain_ring = [&](uint64_t* rel, int d, int64_t n) {
    for (int s = 0; s < d && s < n; ++s) {
      const uint32_t par = (uint32_t)(((n - 1 - s) / d) & 1);
      const long long t0 = clock64();
      while (!tc::mbar_try_wait_cl(&rel[s], par) && clock64() - t0 < tc::kWaitCycles) {}
    }
  };

  if (warp == 0) {
    // ------------------------------------------------------------ producer of A
    if (lane == 0) {
      const uint64_t polA = tc::policy_evict_first();
      uint32_t stage = 0, phase = 0;
      uint32_t armed = 0, armed_par = 0;
      int64_t fills = 0;
      bool ok = true;
      for (int64_t g = it0; g < it1 && ok;) {
        const int64_t t = g / P.ipt;
        const int64_t gend = min(it1, (t + 1) * P.ipt);
        for (int64_t kb = g - t * P.ipt; kb < gend - t * P.ipt; ++kb) {
          if (!tc::mbar_wait_cl(&empty[stage], phase ^ 1, abortp, P.wait_cycles)) { ok = false; break; }
          if (leader) {
            tc::mbar_arrive_expect_tx(&full[stage], 2u * P.a_bytes);
            armed |= 1u << stage;
            armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
          }
          const uint32_t fb = lead_cl(&full[stage]);
          uint8_t* sa = smem + (size_t)stage * P.stage_bytes;
          const int row0 = (int)(t * urows) + (int)rank * mrows;
#pragma unroll
          for (int j = 0; j < KA; ++j) {
            const int k = (int)((kb * KA + j) * AK);
            uint8_t* dst = sa + (size_t)j * kAtomBytes;
            if (A_MN) {
#pragma unroll
              for (int h = 0; h < 128 / AMN; ++h) tc::tma_load_2d_pair(dst + h * AMN_BOX, &tmA, fb, row0 + h * AMN, k, polA);
            } else {
              tc::tma_load_2d_pair(dst, &tmA, fb, k, row0, polA);
            }
          }
          ++fills;
          if (++stage == (uint32_t)P.stages) { stage = 0; phase ^= 1; }
        }
        g = gend;
      }
      if (ok) {
        drain_ring(empty, P.stages, fills);
      } else if (leader) {
        for (int s = 0; s < P.stages; ++s)
          if (armed & (1u << s)) {
            const long long t0 = clock64();
            while (!tc::mbar_try_wait_cl(&full[s], (armed_par >> s) & 1u) && clock64() - t0 < tc::kWaitCycles) {}
          }
      }
    }
  } else if (warp == 6) {
    // ------------------------------------------------------------ producer of B
    if (lane == 0) {
      const uint64_t polB = tc::policy_evict_last();
      uint32_t stage = 0, phase = 0;
      uint32_t armed = 0, armed_par = 0;
      int64_t fills = 0;
      bool ok = true;
      for (int64_t g = it0; g < it1 && ok;) {
        const int64_t t = g / P.ipt;
        const int64_t gend = min(it1, (t + 1) * P.ipt);
        for (int64_t kb = g - t * P.ipt; kb < gend - t * P.ipt; ++kb) {
          if (!tc::mbar_wait_cl(&bempty[stage], phase ^ 1, abortp, P.wait_cycles)) { ok = false; break; }
          if (leader) {
            tc::mbar_arrive_expect_tx(&bfull[stage], 2u * P.b_bytes);
            armed |= 1u << stage;
            armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
          }
          const uint32_t fb = lead_cl(&bfull[stage]);
          uint8_t* sb = bring + (size_t)stage * P.bstage_bytes;
#pragma unroll
          for (int j = 0; j < KA; ++j) {
            const int k = (int)((kb * KA + j) * AK);
#pragma unroll
            for (int ch = 0; ch < NCH; ++ch) {
              // this CTA's half of N-chunk ch (chunk widths: ch0, the last
              // what the others leave)
              const int w = (ch == NCH - 1) ? P.Npad - (NCH - 1) * P.ch0 : P.ch0;
              const int y = ch * P.ch0 + (int)rank * (w / 2);
              const size_t off = (size_t)j * P.b_atom + (size_t)ch * P.hb * 128;
              tc::tma_load_2d_pair(sb + off, &tmB, fb, k, y, polB);
            }
          }
          ++fills;
          if (++stage == (uint32_t)P.bstages) { stage = 0; phase ^= 1; }
        }
        g = gend;
      }
      if (ok) {
        drain_ring(bempty, P.bstages, fills);
      } else if (leader) {
        for (int s2 = 0; s2 < P.bstages; ++s2)
          if (armed & (1u << s2)) {
            const long long t0 = clock64();
            while (!tc::mbar_try_wait_cl(&bfull[s2], (armed_par >> s2) & 1u) && clock64() - t0 < tc::kWaitCycles) {}
          }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer (even CTA)
    if (lane == 0 && leader) {
      const uint32_t idesc0 = tc::idesc_make(FMT, A_MN, false, 256, P.ch0);
      const uint32_t idesc1 = tc::idesc_make(FMT, A_MN, false, 256, NCH > 1 ? P.Npad - (NCH - 1) * P.ch0 : 16);
      uint32_t stage = 0, phase = 0, bstage = 0, bphase = 0;
      int chunk = 0;
      bool ok = true;
      for (int64_t g = it0; g < it1 && ok;) {
        const int64_t t = g / P.ipt;
        const int64_t gend = min(it1, (t + 1) * P.ipt);
        const int64_t kb0 = g - t * P.ipt, kb1 = gend - t * P.ipt;
        const int b = (P.nbuf == 2) ? (chunk & 1) : 0;
        const uint32_t use = (P.nbuf == 2) ? (uint32_t)(chunk >> 1) : (uint32_t)chunk;
        // both CTAs have drained this accumulator buffer
        if (!tc::mbar_wait_cl(&tempty[b], (use & 1u) ^ 1u, abortp, P.wait_cycles)) { ok = false; break; }
        tc::fence_after_sync();
        const uint32_t dcol = tbase + (uint32_t)(b * P.Npad);
        for (int64_t kb = kb0; kb < kb1; ++kb) {
          if (!tc::mbar_wait_cl(&full[stage], phase, abortp, P.wait_cycles)) { ok = false; break; }
          if (!tc::mbar_wait_cl(&bfull[bstage], bphase, abortp, P.wait_cycles)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + (size_t)stage * P.stage_bytes);
          const uint32_t sb = tc::smem_u32(bring + (size_t)bstage * P.bstage_bytes);
#pragma unroll
          for (int j = 0; j < KA; ++j) {
#pragma unroll
            for (int ks = 0; ks < AK / KMMA; ++ks) {
              const uint32_t acc = (kb > kb0 || j > 0 || ks > 0) ? 1u : 0u;
              const uint32_t aat = sa + (uint32_t)j * kAtomBytes;
              const uint64_t ad = A_MN ? tc::desc_sw128(aat + ks * KMMA * 128, AMN_BOX, 1024)
                                       : tc::desc_sw128(aat + ks * 32, 16, 1024);
#pragma unroll
              for (int ch = 0; ch < NCH; ++ch) {
                const uint32_t id = (ch == NCH - 1 && NCH > 1) ? idesc1 : idesc0;
                const uint32_t bat = sb + (uint32_t)j * P.b_atom + (uint32_t)(ch * P.hb * 128);
                tc::mma_f16_pair(dcol + (uint32_t)(ch * P.ch0), ad, tc::desc_sw128(bat + ks * 32, 16, 1024), id, acc);
              }
            }
          }
          // release the stage in both CTAs
          tc::mma_commit_pair(tc::mapa(tc::smem_u32(&empty[stage]), rank));
          tc::mma_commit_pair(tc::mapa(tc::smem_u32(&empty[stage]), peer));
          tc::mma_commit_pair(tc::mapa(tc::smem_u32(&bempty[bstage]), rank));
          tc::mma_commit_pair(tc::mapa(tc::smem_u32(&bempty[bstage]), peer));
          if (++stage == (uint32_t)P.stages) { stage = 0; phase ^= 1; }
          if (++bstage == (uint32_t)P.bstages) { bstage = 0; bphase ^= 1; }
        }
        if (!ok) break;
        tc::mma_commit_pair(tc::mapa(tc::smem_u32(&tfull[b]), rank));
        tc::mma_commit_pair(tc::mapa(tc::smem_u32(&tfull[b]), peer));
        ++chunk;
        g = gend;
      }
      tc::mma_commit_pair(tc::mapa(tc::smem_u32(done), rank));
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(done, 0) && clock64() - t0 < tc::kWaitCycles) {}
    }
  } else if (warp >= 2 && warp <= 5) {
    // ------------------------------------------------------------ epilogue (both CTAs)
    const int q = warp & 3;
    const uint32_t temp_cl[2] = {tc::mapa(tc::smem_u32(&tempty[0]), 0u), tc::mapa(tc::smem_u32(&tempty[1]), 0u)};
    int chunk = 0;
    bool ok = true;
    for (int64_t g = it0; g < it1 && ok;) {
      const int64_t t = g / P.ipt;
      const int64_t gend = min(it1, (t + 1) * P.ipt);
      const bool whole = (g == t * P.ipt) && (gend == (t + 1) * P.ipt);
      float* pdst = nullptr;
      if (!whole) {
        const int slot = (t == it0 / P.ipt) ? 0 : 1;
        pdst = P.parts + ((size_t)blockIdx.x * 2 + slot) * mrows * P.Npad;
      }
      const int b = (P.nbuf == 2) ? (chunk & 1) : 0;
      const uint32_t use = (P.nbuf == 2) ? (uint32_t)(chunk >> 1) : (uint32_t)chunk;
      if (!__all_sync(0xffffffffu, tc::mbar_wait_cl(&tfull[b], use & 1u, abortp, P.wait_cycles))) {
        ok = false;
        break;
      }
      tc::fence_after_sync();
      const uint32_t taddr = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * P.Npad);
      const int row = q * 32 + lane;
      const int64_t grow = t * urows + (int64_t)rank * mrows + row;
      for (int cb = 0; cb < P.N; cb += 16) {
        float v[16];
        tc::tmem_ld16(taddr + cb, v);
        tc::tmem_ld_wait();
        if (whole) {
          if (grow < P.M) {
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (cb + i < P.N) store_out(P, grow, cb + i, v[i]);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (cb + i < P.N) pdst[row + (size_t)(cb + i) * mrows] = v[i];
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive_cluster(temp_cl[b]);
      ++chunk;
      g = gend;
    }
  }
  __syncwarp();
  // every share of a split tile is in memory before its counter moves
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0 && *abortp) raise_status(P.status, SORSVD_ERR_TIMEOUT);
  // no MMA of the pair, copy or arrival aimed at either CTA is in flight
  // past this point
  tc::cluster_sync();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc_pair(tbase, P.tmem_cols);
  }
  if (P.tilecnt && !*abortp) {
    const int64_t th = it0 / P.ipt, tt = (it1 - 1) / P.ipt;
    const bool head_split = (it0 % P.ipt != 0) || (it1 < (th + 1) * P.ipt);
    const bool tail_split = tt != th && (it1 % P.ipt != 0);
    if (threadIdx.x == 0) {
      int bits = 0;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool split = h ? tail_split : head_split;
        if (!split) continue;
        const int64_t t = h ? tt : th;
        const int64_t c0 = cta_of(t * P.ipt, P.total, P.G), c1 = cta_of(t * P.ipt + P.ipt - 1, P.total, P.G);
        if (atomicAdd(&P.tilecnt[2 * t + rank], 1) == (int)(c1 - c0)) bits |= 1 << h;
      }
      *lastp = bits;
    }
    __syncthreads();
    const int bits = *lastp;
    if (bits) {
      __threadfence();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (!((bits >> h) & 1)) continue;
        const int64_t t = h ? tt : th;
        const int64_t c0 = cta_of(t * P.ipt, P.total, P.G), c1 = cta_of(t * P.ipt + P.ipt - 1, P.total, P.G);
        const int slot0 = (c0 * P.total / P.G < t * P.ipt) ? 1 : 0;
        sum_split_tile(P, t * urows + (int64_t)rank * mrows, mrows, c0, c1, slot0, 2, (int)rank);
        if (threadIdx.x == 0) P.tilecnt[2 * t + rank] = 0;
      }
    }
  }
}

// Sum the partial segments of every tile touched by more than one CTA, in
// CTA order (deterministic), and write the tile to the output.  Only split
// tiles need work, and each holds at least one CTA boundary: block x takes
// the boundary of CTA b = x + 1 and handles the tile that boundary falls
// in when b is the first CTA boundary inside it; blockIdx.y splits the
// tile's elements.  The CTAs that cover tile t are c0..c1 (consecutive);
// tile t is the head segment (slot 0) of each of them except c0 when c0's
// range starts inside an earlier tile (then it is c0's tail, slot 1).
// sum of the shares c0..c1 of one tile element (fp32; four independent
// chains for loads in flight, combined in a fixed order)
__device__ __forceinline__ float sum_shares(const TcParams& P, int64_t c0, int64_t c1, int slot0, size_t off,
                                            size_t seg) {
  float a0 = P.parts[((size_t)c0 * 2 + slot0) * seg + off], a1 = 0.f, a2 = 0.f, a3 = 0.f;
  int64_t c = c0 + 1;
  for (; c + 3 <= c1; c += 4) {
    a0 += P.parts[(size_t)c * 2 * seg + off];
    a1 += P.parts[(size_t)(c + 1) * 2 * seg + off];
    a2 += P.parts[(size_t)(c + 2) * 2 * seg + off];
    a3 += P.parts[(size_t)(c + 3) * 2 * seg + off];
  }
  for (; c <= c1; ++c) a0 += P.parts[(size_t)c * 2 * seg + off];
  return (a0 + a1) + (a2 + a3);
}

__global__ void tc_fixup_kernel(const TcParams P) {
  const int mrows = 128 * P.MT;
  const int per = mrows * P.N;
  const int64_t b = (int64_t)blockIdx.x + 1;
  const int64_t x = b * P.total / P.G;           // first iteration of CTA b
  const int64_t t = x / P.ipt;
  if (x == t * P.ipt || t >= P.tiles) return;     // the boundary is a tile start
  const int64_t c0 = cta_of(t * P.ipt, P.total, P.G);
  if (c0 != b - 1) return;                        // an earlier boundary handles tile t
  {
    const int64_t c1 = cta_of(t * P.ipt + P.ipt - 1, P.total, P.G);
    const int slot0 = (c0 * P.total / P.G < t * P.ipt) ? 1 : 0;
    for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < per; e += gridDim.y * blockDim.x) {
      const int col = e / mrows, row = e - col * mrows;
      const int64_t grow = t * mrows + row;
      if (grow >= P.M) continue;
      const size_t off = (size_t)row + (size_t)col * mrows;
      const size_t seg = (size_t)mrows * P.Npad;
      store_out(P, grow, col, sum_shares(P, c0, c1, slot0, off, seg));
    }
  }
}

__global__ void split_tf32_kernel(const float* __restrict__ X, int64_t ldx, int64_t rows, int64_t cols,
                                  float* __restrict__ hi, float* __restrict__ lo, int64_t ldh) {
  const int64_t total = rows * cols;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c = e / rows, r = e - c * rows;
    const float x = X[r + c * ldx];
    const float h = rn_tf32(x);
    hi[r + c * ldh] = h;
    lo[r + c * ldh] = x - h;
  }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 2-D map of a column-major matrix (inner = rows, outer = cols, ld in elements)
bool make_map(CUtensorMap* map, const void* ptr, int elt, int64_t rows, int64_t cols, int64_t ld,
              uint32_t box_inner, uint32_t box_outer, bool swizzle = true) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const CUtensorMapDataType dt = elt == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                 : elt == 1 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                            : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const uint64_t esz = elt == 2 ? 4 : 2;
  cuuint64_t dims[2] = {(cuuint64_t)rows, (cuuint64_t)cols};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * esz)};
  cuuint32_t box[2] = {box_inner, box_outer};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, dt, 2, const_cast<void*>(ptr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int ELT, bool A_MN, int MT, int NCH, int KA>
cudaError_t launch_shape(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mblo, const TcParams& P,
                         size_t smem, cudaStream_t st) {
  auto kern = tc_gemm_kernel<ELT, A_MN, MT, NCH, KA>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<P.G, ELT == 3 ? kThreadsSplit : kThreads, smem, st>>>(ma, mb, mblo, P);
  return cudaGetLastError();
}

// the instantiation for the plan's (MT, nch, KA); split mode has MT = 1 and
// one N-chunk (l <= 128)
template <int ELT, bool A_MN>
cudaError_t launch_typed(const CUtensorMap& ma, const CUtensorMap& mb, const CUtensorMap& mblo, const TcParams& P,
                         size_t smem, cudaStream_t st) {
  if constexpr (ELT == 3) {
    if (P.MT != 1 || P.nch != 1 || P.KA != 1) return cudaErrorInvalidValue;
    return launch_shape<ELT, A_MN, 1, 1, 1>(ma, mb, mblo, P, smem, st);
  } else {
  // more N-chunks (independent accumulators in flight) for one row block
  if (P.nch == 3 && P.MT == 1 && P.KA == 1) return launch_shape<ELT, A_MN, 1, 3, 1>(ma, mb, mblo, P, smem, st);
  if (P.nch == 4 && P.MT == 1 && P.KA == 1) return launch_shape<ELT, A_MN, 1, 4, 1>(ma, mb, mblo, P, smem, st);
  if (P.nch > 2) return cudaErrorInvalidValue;
  const int code = (P.MT - 1) * 4 + (P.nch - 1) * 2 + (P.KA - 1);
  switch (code) {
    case 0: return launch_shape<ELT, A_MN, 1, 1, 1>(ma, mb, mblo, P, smem, st);
    case 1: return launch_shape<ELT, A_MN, 1, 1, 2>(ma, mb, mblo, P, smem, st);
    case 2: return launch_shape<ELT, A_MN, 1, 2, 1>(ma, mb, mblo, P, smem, st);
    case 3: return launch_shape<ELT, A_MN, 1, 2, 2>(ma, mb, mblo, P, smem, st);
    case 4: return launch_shape<ELT, A_MN, 2, 1, 1>(ma, mb, mblo, P, smem, st);
    case 5: return launch_shape<ELT, A_MN, 2, 1, 2>(ma, mb, mblo, P, smem, st);
    case 6: return launch_shape<ELT, A_MN, 2, 2, 1>(ma, mb, mblo, P, smem, st);
    case 7: return launch_shape<ELT, A_MN, 2, 2, 2>(ma, mb, mblo, P, smem, st);
    default: return cudaErrorInvalidValue;
  }
  }
}

template <int ELT, bool A_MN, int NCH, int KA>
cudaError_t launch_pair_shape(const CUtensorMap& ma, const CUtensorMap& mb, const TcParams& P, size_t smem,
                              cudaStream_t st) {
  auto kern = tc_pair_kernel<ELT, A_MN, NCH, KA>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<2 * P.G, kThreads, smem, st>>>(ma, mb, P);
  return cudaGetLastError();
}

template <int ELT, bool A_MN>
cudaError_t launch_pair(const CUtensorMap& ma, const CUtensorMap& mb, const TcParams& P, size_t smem,
                        cudaStream_t st) {
  switch ((P.nch - 1) * 2 + (P.KA - 1)) {
    case 0: return launch_pair_shape<ELT, A_MN, 1, 1>(ma, mb, P, smem, st);
    case 1: return launch_pair_shape<ELT, A_MN, 1, 2>(ma, mb, P, smem, st);
    case 2: return launch_pair_shape<ELT, A_MN, 2, 1>(ma, mb, P, smem, st);
    case 3: return launch_pair_shape<ELT, A_MN, 2, 2>(ma, mb, P, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

// limit of the progress waits of the next launches (0: tc::kWaitCycles)
long long g_wait_cycles = 0;

int env_int(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v ? std::atoi(v) : dflt;
}

constexpr uint32_t kSmemBudget = 220u * 1024u;

// Shape of a launch for a given (KA, MT); stages = 0 when it does not fit.
TcParams shape(int elt, int64_t M, int64_t N, int64_t K, int KA, int MT, int bst = 0) {
  TcParams P{};
  P.M = M; P.K = K; P.N = (int)N;
  P.Npad = (int)((N + 15) / 16 * 16);
  // N-chunks: independent accumulators whose MMAs overlap in the tensor
  // pipe (SORSVD_TC_NCH 1..4 overrides; 3 and 4 only with one row block
  // and one K atom per stage)
  const int envN = env_int("SORSVD_TC_NCH", 0);
  P.nch = (envN >= 1 && envN <= 4 && (envN <= 2 || (MT == 1 && KA == 1)) && elt != 3) ? envN
          : (P.Npad <= 256 ? 1 : 2);
  P.ch0 = (int)((P.Npad + P.nch - 1) / P.nch + 15) / 16 * 16;
  if (P.nch > 1 && P.Npad - (P.nch - 1) * P.ch0 < 16) { P.nch = P.Npad <= 256 ? 1 : 2; P.ch0 = (P.Npad / P.nch + 15) / 16 * 16; }
  P.KA = KA; P.MT = MT;
  const int AK = elt >= 2 ? 32 : 64;
  const int64_t urows = 128 * MT;
  P.tiles = (M + urows - 1) / urows;
  P.ipt = (K + (int64_t)AK * KA - 1) / ((int64_t)AK * KA);
  P.total = P.tiles * P.ipt;
  P.G = (int)std::min<int64_t>(num_sms(), P.total);
  if (P.G < 1) P.G = 1;
  P.nbuf = (2 * MT * P.Npad <= 512) ? 2 : 1;
  uint32_t cols = 32;
  // split mode: two fill buffers [D1 | D2] (4 Npad columns), then the
  // low-part slots of A when they fit (Npad <= kLoTmemMaxNpad)
  if (elt == 3) {
    P.lo_tmem = P.Npad <= kLoTmemMaxNpad ? 1 : 0;
    P.aslot_col = (uint32_t)(4 * P.Npad);
    P.aslots = P.lo_tmem ? (int)std::min<uint32_t>(kASlots, (512u - P.aslot_col) / kASlotCols) : (int)kASlots;
  }
  const uint32_t need_cols = elt == 3 ? 512u : (uint32_t)(P.nbuf * MT * P.Npad);
  while (cols < need_cols) cols <<= 1;
  P.tmem_cols = cols;
  P.a_bytes = (uint32_t)(MT * KA) * kAtomBytes;
  P.b_atom = (uint32_t)P.nch * (uint32_t)P.ch0 * 128u;
  P.b_bytes = (uint32_t)KA * P.b_atom;
  // split mode: a B stage holds the hi and lo tensors; A's parts live in TMEM
  P.stage_bytes = (elt == 3 && !P.lo_tmem ? 2u : 1u) * P.a_bytes;
  P.bstage_bytes = (elt == 3 ? 2u : 1u) * P.b_bytes;
  // B ring depth (SORSVD_TC_BSTAGES overrides, 2..4)
  const int envB = env_int("SORSVD_TC_BSTAGES", 0);
  // a B stage larger than the A stage (16-bit operands, N > 128): one more
  // (split mode: a B stage holds hi and lo, twice the A stage)
  P.bstages = (envB >= 2 && envB <= 4) ? envB
              : bst ? bst : ((elt < 2 && P.b_bytes > P.a_bytes) || (elt == 3 && P.lo_tmem) ? 3 : 2);
  const uint32_t left = kSmemBudget > P.bstages * P.bstage_bytes ? kSmemBudget - P.bstages * P.bstage_bytes : 0;
  P.stages = (int)std::min<uint32_t>(12u, left / P.stage_bytes);
  if (MT * P.Npad > 512 || cols > 512) P.stages = 0;
  if (elt == 3 && (MT != 1 || KA != 1 || P.nbuf != 2 || 4 * P.Npad > 512 || P.aslots < 2)) P.stages = 0;
  return P;
}

// Pair mode (16-bit operands, 128 < Npad <= 512): G pairs of CTAs over
// 256-row tiles; each CTA stages its 128 rows of A and half of each
// N-chunk of B (hb rows per chunk box; a last chunk narrower than ch0 reads
// a few rows past its half, which its MMA does not use).
TcParams shape_pair(int elt, int64_t M, int64_t N, int64_t K, int KA, int bst) {
  TcParams P{};
  P.pair = 1;
  P.M = M; P.K = K; P.N = (int)N;
  P.Npad = (int)((N + 15) / 16 * 16);
  P.nch = P.Npad <= 256 ? 1 : 2;
  P.ch0 = P.nch == 1 ? P.Npad : (P.Npad / 2 + 15) / 16 * 16;
  P.hb = P.ch0 / 2;
  P.KA = KA; P.MT = 1;
  P.tiles = (M + 255) / 256;
  P.ipt = (K + (int64_t)64 * KA - 1) / ((int64_t)64 * KA);
  P.total = P.tiles * P.ipt;
  P.G = (int)std::min<int64_t>(num_sms() / 2, P.total);
  if (P.G < 1) P.G = 1;
  P.nbuf = (2 * P.Npad <= 512) ? 2 : 1;
  uint32_t cols = 32;
  while (cols < (uint32_t)(P.nbuf * P.Npad)) cols <<= 1;
  P.tmem_cols = cols;
  P.a_bytes = (uint32_t)KA * kAtomBytes;
  P.b_atom = (uint32_t)P.nch * (uint32_t)P.hb * 128u;
  P.b_bytes = (uint32_t)KA * P.b_atom;
  P.stage_bytes = P.a_bytes;
  P.bstage_bytes = P.b_bytes;
  const int envB = env_int("SORSVD_TC_BSTAGES", 0);
  P.bstages = (envB >= 2 && envB <= 4) ? envB : bst ? bst : (KA >= 2 ? 2 : 3);
  const uint32_t left = kSmemBudget > P.bstages * P.bstage_bytes ? kSmemBudget - P.bstages * P.bstage_bytes : 0;
  P.stages = (int)std::min<uint32_t>(12u, left / P.stage_bytes);
  if (elt > 1 || P.Npad <= 128 || P.Npad > 512 || cols > 512 || (num_sms() & 1) ||
      P.Npad - (P.nch - 1) * P.ch0 < 16)
    P.stages = 0;
  return P;
}

// pair mode for 16-bit passes with 128 < Npad <= 512 (SORSVD_TC_PAIR=0 turns
// it off); not with a shortened wait limit, whose tests exercise the
// single-CTA kernel's abort path
bool pair_wanted(int elt, int64_t N) {
  const int64_t Npad = (N + 15) / 16 * 16;
  return elt <= 1 && Npad > 128 && Npad <= 512 && env_int("SORSVD_TC_PAIR", 1) != 0 && (num_sms() % 2) == 0;
}

TcParams tc_plan_pair(int elt, int64_t M, int64_t N, int64_t K) {
  const int envKA = env_int("SORSVD_TC_KATOMS", 0);
  TcParams P = shape_pair(elt, M, N, K, (envKA >= 1 && envKA <= kMaxKA) ? envKA : 2, 0);
  if (P.stages < 3 && envKA == 0) {
    TcParams Q = shape_pair(elt, M, N, K, 1, 0);
    if (Q.stages >= 3) P = Q;
  }
  return P;
}

}  // namespace

// Planned shape of a launch (shared by the launcher and the workspace size).
// Default tiling: two 128-row blocks per tile when they fit in TMEM
// double-buffered (not in split mode), then the most K atoms per stage (the
// longest contiguous run per column of A, up to 4) that still leaves >= 3
// stages.  SORSVD_TC_KATOMS and SORSVD_TC_MTILES override the choice.
TcParams tc_plan_single(int elt, int64_t M, int64_t N, int64_t K) {
  const int envKA = env_int("SORSVD_TC_KATOMS", 0), envMT = env_int("SORSVD_TC_MTILES", 0);
  const int64_t Npad = (N + 15) / 16 * 16;
  int MT = envMT > 0 ? envMT : ((elt != 3 && 4 * Npad <= 512) ? 2 : 1);
  if (elt == 3 || MT * Npad > 512 || MT < 1 || MT > 2) MT = 1;
  TcParams best = shape(elt, M, N, K, 1, MT);
  if (envKA > kMaxKA || elt >= 2) return best;     // fp32 containers: one K atom per stage
  if (envKA > 0) {
    TcParams P = shape(elt, M, N, K, envKA, MT);
    return P.stages >= 2 ? P : best;
  }
  for (int KA = 2; KA <= kMaxKA; ++KA) {
    TcParams P = shape(elt, M, N, K, KA, MT);
    if (P.stages >= 4) best = P;
  }
  // 16-bit operands with N > 256 (two N-chunks, 36 KB of B per K atom): two
  // K atoms per stage in a two-stage B ring (two stages of A), which halves
  // the stage hand-offs; measured on the 65536 x 16384 workload
  // (l = 266): 3.09 -> 2.92 ms for the six passes
  if (best.KA == 1 && best.nch == 2 && envKA == 0 && env_int("SORSVD_TC_BSTAGES", 0) == 0) {
    TcParams P = shape(elt, M, N, K, 2, MT, 2);
    if (P.stages >= 2) best = P;
  }
  return best;
}

bool tc_supported(int elt, const void* A, int64_t lda, const void* B, int64_t ldb, int l) {
  const int64_t esz = elt >= 2 ? 4 : 2;
  if (l < 1 || l > 512) return false;
  if (elt == 3 && l > kAccCols) return false;       // split mode: 4 Npad TMEM columns
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15)) return false;
  if ((lda * esz) % 16 || (ldb * esz) % 16) return false;
  return encode_fn() != nullptr;
}

TcParams tc_plan(int elt, int64_t M, int64_t N, int64_t K) {
  if (pair_wanted(elt, N)) {
    TcParams P = tc_plan_pair(elt, M, N, K);
    if (P.stages >= 2) return P;
  }
  return tc_plan_single(elt, M, N, K);
}

size_t tc_parts_bytes(int elt, int64_t M, int64_t N, int64_t K) {
  // the launcher may fall back from pair mode to single CTAs: room for both
  const TcParams P = tc_plan(elt, M, N, K), S = tc_plan_single(elt, M, N, K);
  const size_t bp = (size_t)P.G * (P.pair ? 2 : 1) * 2 * 128 * P.MT * P.Npad * sizeof(float);
  const size_t bs = (size_t)S.G * 2 * 128 * S.MT * S.Npad * sizeof(float);
  return std::max(bp, bs);
}

namespace {

cudaError_t launch_tc_gemm_impl(bool trans_a, int elt, int64_t M, int64_t N, int64_t K, const void* A,
                                int64_t lda, const void* B, int64_t ldb, const void* Blo, float* out, int64_t ldo,
                                void* out16, int64_t ld16, int out16_kind, float* parts, int* tilecnt,
                                int64_t ntilecnt, DeviceStatus* status, int kcls, cudaStream_t st, bool allow_pair) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  if (elt == 3 && (!Blo || (reinterpret_cast<uintptr_t>(Blo) & 15))) return cudaErrorInvalidValue;
  // an MN-major TF32 operand gave all-zero products on GB300: fp32 products
  // of the form A X go through a transposed copy of A instead
  if (elt >= 2 && !trans_a) return cudaErrorInvalidValue;
  TcParams P = tc_plan(elt, M, N, K);
  // pair mode needs the per-tile counters (two per 256-row tile) and the
  // default wait limit
  if (P.pair && (!allow_pair || !tilecnt || 2 * P.tiles > ntilecnt ||
                 (g_wait_cycles > 0 && g_wait_cycles < tc::kWaitCycles)))
    P = tc_plan_single(elt, M, N, K);
  if (P.stages < 2) return cudaErrorInvalidValue;
  P.out = out; P.ldo = ldo; P.out16 = out16; P.ld16 = ld16; P.out16_kind = out16 ? out16_kind : 0;
  P.parts = parts; P.status = status;
  P.wait_cycles = (g_wait_cycles > 0 && g_wait_cycles < tc::kWaitCycles) ? g_wait_cycles : tc::kWaitCycles;

  P.tilecnt = (tilecnt && (P.pair ? 2 : 1) * P.tiles <= ntilecnt) ? tilecnt : nullptr;
  const int AK = elt >= 2 ? 32 : 64, AMN = elt >= 2 ? 32 : 64;
  const int map_elt = elt == 3 ? 2 : elt;
  CUtensorMap ma, mb;
  // A is stored column-major (inner = rows of A).  op(A) = A^T: MMA rows are
  // columns of A, K runs along A's rows.  op(A) = A: MMA rows are A's rows.
  const int64_t a_rows = trans_a ? K : M, a_cols = trans_a ? M : K;
  const bool okA = trans_a ? make_map(&ma, A, map_elt, a_rows, a_cols, lda, (uint32_t)AK, 128u)
                           : make_map(&ma, A, map_elt, a_rows, a_cols, lda, (uint32_t)AMN, (uint32_t)AK);
  const bool okB = make_map(&mb, B, map_elt, K, N, ldb, (uint32_t)AK, (uint32_t)(P.pair ? P.hb : P.ch0));
  CUtensorMap mblo = mb;
  const bool okBlo = elt != 3 || make_map(&mblo, Blo, map_elt, K, N, ldb, (uint32_t)AK, (uint32_t)P.ch0);
  if (!okA || !okB || !okBlo) return cudaErrorInvalidValue;
  const size_t smem = (size_t)P.stages * P.stage_bytes + (size_t)P.bstages * P.bstage_bytes + 1024 + 512;
  cudaError_t e;
  if (P.pair) {
    ProfScope ps(kcls, st);
    if (elt == 0) e = trans_a ? launch_pair<0, false>(ma, mb, P, smem, st) : launch_pair<0, true>(ma, mb, P, smem, st);
    else e = trans_a ? launch_pair<1, false>(ma, mb, P, smem, st) : launch_pair<1, true>(ma, mb, P, smem, st);
    return e;
  }
  {
    ProfScope ps(kcls, st);
    if (elt == 0) e = trans_a ? launch_typed<0, false>(ma, mb, mblo, P, smem, st) : launch_typed<0, true>(ma, mb, mblo, P, smem, st);
    else if (elt == 1) e = trans_a ? launch_typed<1, false>(ma, mb, mblo, P, smem, st) : launch_typed<1, true>(ma, mb, mblo, P, smem, st);
    else if (elt == 2) e = launch_typed<2, false>(ma, mb, mblo, P, smem, st);
    else e = launch_typed<3, false>(ma, mb, mblo, P, smem, st);
  }
  if (e != cudaSuccess) return e;
  // fix-up of the tiles split across CTAs (when no counters were given):
  // one block row per CTA boundary, about 4 elements of the tile per thread
  if (P.G < 2 || P.tilecnt) return cudaSuccess;
  const int64_t per = (int64_t)128 * P.MT * P.N;
  const int64_t gy = std::max<int64_t>(1, std::min<int64_t>((per + 255) / 256, 65535));
  ProfScope ps2(K_REDUCE, st);
  tc_fixup_kernel<<<dim3((unsigned)(P.G - 1), (unsigned)gy), 256, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace

// A pass on CTA pairs whose launch is refused (no room for a two-CTA
// cluster, for instance) runs on single CTAs instead.
cudaError_t launch_tc_gemm(bool trans_a, int elt, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                           const void* B, int64_t ldb, const void* Blo, float* out, int64_t ldo, void* out16,
                           int64_t ld16, int out16_kind, float* parts, int* tilecnt, int64_t ntilecnt,
                           DeviceStatus* status, int kcls, cudaStream_t st) {
  const cudaError_t e = launch_tc_gemm_impl(trans_a, elt, M, N, K, A, lda, B, ldb, Blo, out, ldo, out16, ld16,
                                            out16_kind, parts, tilecnt, ntilecnt, status, kcls, st, true);
  if (e == cudaSuccess || !pair_wanted(elt, N)) return e;
  cudaGetLastError();                        // clear the launch error (not a sticky one)
  return launch_tc_gemm_impl(trans_a, elt, M, N, K, A, lda, B, ldb, Blo, out, ldo, out16, ld16, out16_kind, parts,
                             tilecnt, ntilecnt, status, kcls, st, false);
}

void set_tc_wait_cycles(long long cycles) { g_wait_cycles = cycles > 0 ? cycles : 0; }

long long tc_wait_cycles() {
  return (g_wait_cycles > 0 && g_wait_cycles < tc::kWaitCycles) ? g_wait_cycles : tc::kWaitCycles;
}

bool tc_map_2d(CUtensorMap* map, const void* ptr, int elt, int64_t rows, int64_t cols, int64_t ld, uint32_t box_inner,
               uint32_t box_outer, bool swizzle128) {
  return make_map(map, ptr, elt, rows, cols, ld, box_inner, box_outer, swizzle128);
}

cudaError_t launch_split_tf32(const float* X, int64_t ldx, int64_t rows, int64_t cols, float* hi, float* lo,
                              int64_t ldh, cudaStream_t st) {
  const int64_t total = rows * cols;
  if (total <= 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
  split_tf32_kernel<<<(unsigned)blocks, 256, 0, st>>>(X, ldx, rows, cols, hi, lo, ldh);
  return cudaGetLastError();
}

}  // namespace sorsvd
