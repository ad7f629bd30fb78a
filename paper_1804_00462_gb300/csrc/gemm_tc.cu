// Tensor-core passes over A (the dense contractions of Algorithm 3):
//   T1 = A T2 and W = A Q2   (op(A) = A:   A is MN-major for the MMA)
//   T2 = A^T T1              (op(A) = A^T: A is K-major for the MMA)
// D[128 x Npad] tiles accumulate in tensor memory (TMEM) through
// tcgen05.mma (kind::f16 for bf16/fp16 operands, kind::tf32 for fp32
// containers), fed by TMA loads into 128-byte-swizzled shared-memory stages.
//
// Work decomposition: a persistent grid of G <= #SM CTAs splits the
// tiles x K-blocks iteration space into G contiguous ranges ("stream-K"),
// so every SM streams the same share of A whatever the tile count.  A CTA
// walks its range as segments (one per output tile it touches).  A segment
// that covers a whole tile is written straight to the output; the at most
// two partial segments of a CTA (head and tail of its range) go to a
// per-CTA partial buffer and a fix-up kernel sums them per tile in CTA
// order: the result is deterministic and uses no atomics.
//
// Warp roles (192 threads): warp 0 issues TMA (one lane), warp 1 owns the
// TMEM allocation and issues MMAs (one lane), warps 2-5 drain accumulators
// (tcgen05.ld, 32 TMEM lanes per warp) into fp32 output and, optionally, a
// 16-bit copy used as the next pass's operand.  Accumulators are
// double-buffered in TMEM when 2 Npad <= 512 columns, so the epilogue of
// one segment overlaps the MMAs of the next.  Every mbarrier wait is
// bounded (tc::kWaitCycles); a timeout records SORSVD_ERR_TIMEOUT, stops all
// roles, waits for the copies and MMAs already issued, frees TMEM and exits.
#include "internal.cuh"
#include "profile.cuh"
#include "tc_ptx.cuh"

#include <algorithm>

namespace sorsvd {

struct TcParams {
  int64_t M, K;          // output rows, reduction length
  int N, Npad, nch, ch0; // output columns, padded, N-chunks of ch0 rows
  int64_t tiles, ipt, total;
  int G;
  int nbuf;
  uint32_t tmem_cols;
  int stages;
  uint32_t stage_bytes, a_bytes, tx_bytes;
  float* out;
  int64_t ldo;
  void* out16;           // optional 16-bit copy of the output (bf16 / fp16)
  int64_t ld16;
  int out16_kind;        // 0 none, 1 bf16, 2 fp16
  float* parts;          // G x 2 x 128 x Npad fp32
  DeviceStatus* status;
};

namespace {

constexpr int kThreads = 192;

__host__ __device__ __forceinline__ int64_t cta_of(int64_t x, int64_t total, int64_t G) {
  // the CTA whose iteration range [c*total/G, (c+1)*total/G) holds x
  return ((x + 1) * G + total - 1) / total - 1;
}

__device__ __forceinline__ void store_out(const TcParams& P, int64_t grow, int col, float v) {
  P.out[grow + (int64_t)col * P.ldo] = v;
  if (P.out16_kind == 1) reinterpret_cast<bf16*>(P.out16)[grow + (int64_t)col * P.ld16] = __float2bfloat16_rn(v);
  else if (P.out16_kind == 2) reinterpret_cast<f16*>(P.out16)[grow + (int64_t)col * P.ld16] = __float2half_rn(v);
}

// ELT: 0 bf16, 1 fp16, 2 tf32.  A_MN: A operand MN-major (op(A) = A).
template <int ELT, bool A_MN>
__global__ void __launch_bounds__(kThreads, 1)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const TcParams P) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + (size_t)P.stages * P.stage_bytes);
  uint64_t* empty = full + P.stages;
  uint64_t* tfull = empty + P.stages;
  uint64_t* tempty = tfull + 2;
  uint64_t* done = tempty + 2;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  volatile int* abortp = reinterpret_cast<volatile int*>(tslot + 1);

  // K elements per stage (one 128-byte swizzle row), K per MMA, MN width of
  // one swizzle row for the MN-major A boxes
  constexpr int BK = (ELT == 2) ? 32 : 64;
  constexpr int KMMA = (ELT == 2) ? 8 : 16;
  constexpr int AMN = (ELT == 2) ? 32 : 64;
  constexpr uint32_t AMN_BOX = (uint32_t)BK * 128u;     // bytes of one MN-major A box
  constexpr uint32_t FMT = (ELT == 0) ? 1u : (ELT == 1 ? 0u : 2u);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < P.stages; ++s) { tc::mbar_init(&full[s], 1); tc::mbar_init(&empty[s], 1); }
    for (int b = 0; b < 2; ++b) { tc::mbar_init(&tfull[b], 1); tc::mbar_init(&tempty[b], 128); }
    tc::mbar_init(done, 1);
    *abortp = 0;
    tc::fence_barrier_init();
  }
  if (warp == 1) {
    tc::tmem_alloc(tslot, P.tmem_cols);
    tc::tmem_relinquish();
  }
  if (warp == 0 && lane == 0) { tc::prefetch_tmap(&tmA); tc::prefetch_tmap(&tmB); }
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;

  const int64_t cta = blockIdx.x;
  const int64_t it0 = cta * P.total / P.G, it1 = (cta + 1) * P.total / P.G;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      const uint64_t polA = tc::policy_evict_first(), polB = tc::policy_evict_last();
      uint32_t stage = 0, phase = 0;
      uint32_t armed = 0;          // bit s: stage s armed and not yet seen consumed
      uint32_t armed_par = 0;      // parity of that armed phase
      bool ok = true;
      for (int64_t g = it0; g < it1 && ok;) {
        const int64_t t = g / P.ipt;
        const int64_t gend = min(it1, (t + 1) * P.ipt);
        for (int64_t kb = g - t * P.ipt; kb < gend - t * P.ipt; ++kb) {
          if (!tc::mbar_wait(&empty[stage], phase ^ 1, abortp)) { ok = false; break; }
          armed &= ~(1u << stage);
          tc::mbar_arrive_expect_tx(&full[stage], P.tx_bytes);
          armed |= 1u << stage;
          armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
          uint8_t* sa = smem + (size_t)stage * P.stage_bytes;
          uint8_t* sb = sa + P.a_bytes;
          const int k0 = (int)(kb * BK);
          if (A_MN) {
#pragma unroll
            for (int j = 0; j < 128 / AMN; ++j)
              tc::tma_load_2d_hint(sa + j * AMN_BOX, &tmA, &full[stage], (int)(t * 128) + j * AMN, k0, polA);
          } else {
            tc::tma_load_2d_hint(sa, &tmA, &full[stage], k0, (int)(t * 128), polA);
          }
          for (int ch = 0; ch < P.nch; ++ch)
            tc::tma_load_2d_hint(sb + (size_t)ch * P.ch0 * 128, &tmB, &full[stage], k0, ch * P.ch0, polB);
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
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      uint32_t idesc[2];
      idesc[0] = tc::idesc_make(FMT, A_MN, false, 128, P.ch0);
      idesc[1] = tc::idesc_make(FMT, A_MN, false, 128, P.Npad - P.ch0);
      uint32_t stage = 0, phase = 0;
      int seg = 0;
      bool ok = true;
      for (int64_t g = it0; g < it1 && ok;) {
        const int64_t t = g / P.ipt;
        const int64_t gend = min(it1, (t + 1) * P.ipt);
        const int b = (P.nbuf == 2) ? (seg & 1) : 0;
        const uint32_t use = (P.nbuf == 2) ? (uint32_t)(seg >> 1) : (uint32_t)seg;
        if (!tc::mbar_wait(&tempty[b], (use & 1u) ^ 1u, abortp)) { ok = false; break; }
        tc::fence_after_sync();
        const uint32_t dcol = tbase + (uint32_t)(b * P.Npad);
        const int64_t kb0 = g - t * P.ipt, kb1 = gend - t * P.ipt;
        for (int64_t kb = kb0; kb < kb1; ++kb) {
          if (!tc::mbar_wait(&full[stage], phase, abortp)) { ok = false; break; }
          tc::fence_after_sync();
          const uint32_t sa = tc::smem_u32(smem + (size_t)stage * P.stage_bytes);
          const uint32_t sb = sa + P.a_bytes;
#pragma unroll
          for (int ks = 0; ks < BK / KMMA; ++ks) {
            const uint64_t ad = A_MN ? tc::desc_sw128(sa + ks * KMMA * 128, AMN_BOX, 1024)
                                     : tc::desc_sw128(sa + ks * 32, 16, 1024);
            const uint32_t acc = (kb > kb0 || ks > 0) ? 1u : 0u;
            for (int ch = 0; ch < P.nch; ++ch) {
              const uint64_t bd = tc::desc_sw128(sb + ch * P.ch0 * 128 + ks * 32, 16, 1024);
              if (ELT == 2) tc::mma_tf32(dcol + ch * P.ch0, ad, bd, idesc[ch], acc);
              else tc::mma_f16(dcol + ch * P.ch0, ad, bd, idesc[ch], acc);
            }
          }
          tc::mma_commit(&empty[stage]);
          if (++stage == (uint32_t)P.stages) { stage = 0; phase ^= 1; }
        }
        if (!ok) break;
        tc::mma_commit(&tfull[b]);
        ++seg;
        g = gend;
      }
      // every MMA issued by this thread has completed once `done` flips
      tc::mma_commit(done);
      const long long t0 = clock64();
      while (!tc::mbar_try_wait(done, 0) && clock64() - t0 < tc::kWaitCycles) {}
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp & 3;                    // TMEM lane quarter of this warp
    const int row = q * 32 + lane;
    int seg = 0;
    for (int64_t g = it0; g < it1;) {
      const int64_t t = g / P.ipt;
      const int64_t gend = min(it1, (t + 1) * P.ipt);
      const int b = (P.nbuf == 2) ? (seg & 1) : 0;
      const uint32_t use = (P.nbuf == 2) ? (uint32_t)(seg >> 1) : (uint32_t)seg;
      if (!tc::mbar_wait(&tfull[b], use & 1u, abortp)) break;
      tc::fence_after_sync();
      const bool whole = (g == t * P.ipt) && (gend == (t + 1) * P.ipt);
      const int64_t grow = t * 128 + row;
      const uint32_t taddr = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(b * P.Npad);
      float* pdst = nullptr;
      if (!whole) {
        const int slot = (t == it0 / P.ipt) ? 0 : 1;
        pdst = P.parts + ((size_t)cta * 2 + slot) * 128 * P.Npad;
      }
      for (int c0 = 0; c0 < P.N; c0 += 16) {
        float v[16];
        tc::tmem_ld16(taddr + c0, v);
        tc::tmem_ld_wait();
        if (whole) {
          if (grow < P.M) {
#pragma unroll
            for (int i = 0; i < 16; ++i)
              if (c0 + i < P.N) store_out(P, grow, c0 + i, v[i]);
          }
        } else {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c0 + i < P.N) pdst[row + (size_t)(c0 + i) * 128] = v[i];
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(&tempty[b]);
      ++seg;
      g = gend;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && *abortp) raise_status(P.status, SORSVD_ERR_TIMEOUT);
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tbase, P.tmem_cols);
  }
}

// Sum the partial segments of every tile touched by more than one CTA, in
// CTA order, and write the tile to the output.
__global__ void tc_fixup_kernel(const TcParams P) {
  const int64_t per_tile = 128 * (int64_t)P.N;
  const int64_t total = P.tiles * per_tile;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t t = e / per_tile;
    const int64_t r = e - t * per_tile;
    const int col = (int)(r / 128), row = (int)(r - (int64_t)col * 128);
    const int64_t grow = t * 128 + row;
    if (grow >= P.M) continue;
    const int64_t c_first = cta_of(t * P.ipt, P.total, P.G);
    const int64_t c_last = cta_of(t * P.ipt + P.ipt - 1, P.total, P.G);
    if (c_first == c_last) continue;
    double s = 0.0;
    for (int64_t c = c_first; c <= c_last; ++c) {
      const int64_t head_tile = (c * P.total / P.G) / P.ipt;
      const int slot = (t == head_tile) ? 0 : 1;
      s += (double)P.parts[((size_t)c * 2 + slot) * 128 * P.Npad + row + (size_t)col * 128];
    }
    store_out(P, grow, col, (float)s);
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
              uint32_t box_inner, uint32_t box_outer) {
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
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int ELT, bool A_MN>
cudaError_t launch_typed(const CUtensorMap& ma, const CUtensorMap& mb, const TcParams& P, size_t smem,
                         cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(tc_gemm_kernel<ELT, A_MN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  tc_gemm_kernel<ELT, A_MN><<<P.G, kThreads, smem, st>>>(ma, mb, P);
  return cudaGetLastError();
}

}  // namespace

bool tc_supported(int elt, const void* A, int64_t lda, const void* B, int64_t ldb, int l) {
  const int64_t esz = elt == 2 ? 4 : 2;
  if (l < 1 || l > 512) return false;
  if ((reinterpret_cast<uintptr_t>(A) & 15) || (reinterpret_cast<uintptr_t>(B) & 15)) return false;
  if ((lda * esz) % 16 || (ldb * esz) % 16) return false;
  return encode_fn() != nullptr;
}

// Planned shape of a launch (shared by the launcher and the workspace size).
TcParams tc_plan(int elt, int64_t M, int64_t N, int64_t K) {
  TcParams P{};
  P.M = M; P.K = K; P.N = (int)N;
  P.Npad = (int)((N + 15) / 16 * 16);
  if (P.Npad <= 256) { P.nch = 1; P.ch0 = P.Npad; }
  else { P.nch = 2; P.ch0 = (P.Npad / 2 + 15) / 16 * 16; }
  const int BK = elt == 2 ? 32 : 64;
  P.tiles = (M + 127) / 128;
  P.ipt = (K + BK - 1) / BK;
  P.total = P.tiles * P.ipt;
  P.G = (int)std::min<int64_t>(num_sms(), P.total);
  if (P.G < 1) P.G = 1;
  P.nbuf = (2 * P.Npad <= 512) ? 2 : 1;
  uint32_t cols = 32;
  while (cols < (uint32_t)(P.nbuf * P.Npad)) cols <<= 1;
  P.tmem_cols = cols;
  P.a_bytes = 128u * 128u;                                   // 128 rows x 128 bytes
  P.stage_bytes = P.a_bytes + (uint32_t)P.nch * (uint32_t)P.ch0 * 128u;
  P.tx_bytes = P.stage_bytes;
  const uint32_t budget = 220u * 1024u;
  P.stages = (int)std::min<uint32_t>(8u, budget / P.stage_bytes);
  return P;
}

size_t tc_parts_bytes(int elt, int64_t M, int64_t N, int64_t K) {
  TcParams P = tc_plan(elt, M, N, K);
  return (size_t)P.G * 2 * 128 * P.Npad * sizeof(float);
}

cudaError_t launch_tc_gemm(bool trans_a, int elt, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
                           const void* B, int64_t ldb, float* out, int64_t ldo, void* out16, int64_t ld16,
                           int out16_kind, float* parts, DeviceStatus* status, int kcls, cudaStream_t st) {
  if (M <= 0 || N <= 0 || K <= 0) return cudaSuccess;
  // an MN-major TF32 operand gave all-zero products on GB300: fp32 products
  // of the form A X go through a transposed copy of A instead
  if (elt == 2 && !trans_a) return cudaErrorInvalidValue;
  TcParams P = tc_plan(elt, M, N, K);
  if (P.stages < 2) return cudaErrorInvalidValue;
  P.out = out; P.ldo = ldo; P.out16 = out16; P.ld16 = ld16; P.out16_kind = out16 ? out16_kind : 0;
  P.parts = parts; P.status = status;
  const int BK = elt == 2 ? 32 : 64, AMN = elt == 2 ? 32 : 64;
  CUtensorMap ma, mb;
  // A is stored column-major (inner = rows of A).  op(A) = A^T: MMA rows are
  // columns of A, K runs along A's rows.  op(A) = A: MMA rows are A's rows.
  const int64_t a_rows = trans_a ? K : M, a_cols = trans_a ? M : K;
  const bool okA = trans_a ? make_map(&ma, A, elt, a_rows, a_cols, lda, (uint32_t)BK, 128u)
                           : make_map(&ma, A, elt, a_rows, a_cols, lda, (uint32_t)AMN, (uint32_t)BK);
  const bool okB = make_map(&mb, B, elt, K, N, ldb, (uint32_t)BK, (uint32_t)P.ch0);
  if (!okA || !okB) return cudaErrorInvalidValue;
  const size_t smem = (size_t)P.stages * P.stage_bytes + 1024 + 256;
  cudaError_t e;
  {
    ProfScope ps(kcls, st);
    if (elt == 0) e = trans_a ? launch_typed<0, false>(ma, mb, P, smem, st) : launch_typed<0, true>(ma, mb, P, smem, st);
    else if (elt == 1) e = trans_a ? launch_typed<1, false>(ma, mb, P, smem, st) : launch_typed<1, true>(ma, mb, P, smem, st);
    else e = launch_typed<2, false>(ma, mb, P, smem, st);
  }
  if (e != cudaSuccess) return e;
  // fix-up of tiles split across CTAs (a no-op grid when every tile is whole)
  const int64_t work = P.tiles * 128 * P.N;
  int64_t blocks = (work + 255) / 256;
  if (blocks > (int64_t)num_sms() * 8) blocks = (int64_t)num_sms() * 8;
  ProfScope ps2(K_REDUCE, st);
  tc_fixup_kernel<<<(unsigned)blocks, 256, 0, st>>>(P);
  return cudaGetLastError();
}

}  // namespace sorsvd
