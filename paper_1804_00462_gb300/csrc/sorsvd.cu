// Host driver of the C ABI: argument checks, workspace layout, and the
// sequence of kernels that realises Algorithm 3 (SOR-SVD with power method):
//
//   Omega -> T2op                                 (sorsvd_gaussian)
//   for i = 1 .. q+1:                             (power loop)
//     [i > 1] T2 <- orth(T2)   shifted CholeskyQR, one pass: keeps range(T2)
//                              (Lemma 1: QR projectors are invariant under
//                              right multiplication by a nonsingular matrix)
//     T1 = A T2op ; T2 = A^T T1op                 (eqs. T1, AT1)
//   Q1 = orth3(T1), Q2 = orth3(T2)                (QR step: shifted CholeskyQR3)
//   M = Q1^T (A Q2)                               (eq. M)
//   M = U~ S~ V~^T (one-sided Jacobi), keep k     (truncated SVD)
//   U = Q1 U~_k, V = Q2 V~_k                      (output assembly)
//
// "op" buffers hold the operand that multiplies A: the 16-bit rounding of the
// fp32 sketch for BF16/F16, the sketch itself otherwise.
#include "internal.cuh"
#include "profile.cuh"

#include <algorithm>
#include <cstdlib>
#include <vector>

namespace sorsvd {
namespace {

// Dispatch knob read once from the environment: SORSVD_TC=0 sends every pass
// to the CUDA-core kernels.
int env_flag(const char* name, int dflt) {
  const char* v = std::getenv(name);
  return v ? std::atoi(v) : dflt;
}
bool tc_enabled() { static const int v = env_flag("SORSVD_TC", 1); return v != 0; }
// SORSVD_POLAR=0: the second CholeskyQR3 pass factorises (Cholesky) instead
// of taking the polar factor of its near-identity Gram
bool polar_enabled() { static const int v = env_flag("SORSVD_POLAR", 1); return v != 0; }


constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// relative shift of the first CholeskyQR pass (unit-diagonal Gram)
inline double first_shift(int dt) { return dt == SORSVD_F64 ? 1e-13 : 1e-5; }
// largest column cosine of the second pass's input for which the third
// CholeskyQR pass is skipped: the second pass then leaves Q orthonormal to
// working precision (its error grows with cond(Q)^2 <= (1 + l tol) / (1 - l tol))
constexpr float kOrthTol = 1e-4f;

// K splits of a product with an M x N output and reduction length K, for
// the CUDA-core tiles: 128 x 64 with at least 256 K per split, or for
// binary64 products of <= 32 columns 64 x 32 with at least 16 K per split
// (binary64 FMAs are scarce: the product is spread over every SM)
int splits_for(int64_t M, int64_t N, int64_t K, int cap, bool f64 = false) {
  const bool skinny = f64 && N <= 32;
  int64_t tiles = skinny ? ((M + 63) / 64) * ((N + 31) / 32) : ((M + 127) / 128) * ((N + 63) / 64);
  int64_t want = 2 * (int64_t)num_sms();
  int64_t s = (want + tiles - 1) / tiles;
  int64_t by_k = skinny ? (K + 15) / 16 : (K + 255) / 256;
  s = std::min<int64_t>(s, by_k);
  s = std::min<int64_t>(s, cap);
  return (int)std::max<int64_t>(s, 1);
}
constexpr int kCapBig = 16, kCapSmall = 256;
// split tensor-core products: widest skinny operand of one launch (the
// low parts of A then fit in TMEM beside the two accumulator fills)
constexpr int64_t kSplitMaxCols = 128, kSplitChunkCols = 112;

inline int64_t pad16(int64_t x) { return (x + 15) / 16 * 16; }

// Tensor-core element kind of the passes over A for a dtype: 0 bf16, 1 fp16,
// 2 tf32 (F32 and TF32 both keep fp32 containers), -1 none (binary64).
inline int elt_of(int dt) {
  switch (dt) {
    case SORSVD_BF16: return 0;
    case SORSVD_F16: return 1;
    case SORSVD_TF32: case SORSVD_F32: return 2;
    default: return -1;
  }
}

struct Layout {
  int64_t ldm, ldn;      // leading dimensions of the m x l / n x l sketches
  size_t status, tilecnt, at, t2op, t2, t1, t1op, q2op, tmp, bhi, blo, parts, G, Rinv, M, Ut, Vt, jwork, total;
  size_t t1s, t2s, tp;   // two-pass core: T1 before its QR, T2_prev, five l x l binary64 matrices
  size_t bsplit;         // hi / lo parts of the small factor of a tall-skinny tensor-core product
  int64_t ntilecnt;      // counters of the split tiles of a tensor-core pass
  int64_t ldb;           // leading dimension of bhi / blo
  int64_t ldk;           // leading dimension of the parts in bsplit (l rounded up to 32)
  bool has_at;           // fp32 containers: A^T kept for the products A X
};

// at_rows: the rows of A the transposed copy holds (m; a block of rows for
// the streamed entry point)
Layout make_layout(int64_t m, int64_t n, int l, int dt, unsigned flags = 0, int64_t at_rows = -1) {
  Layout L{};
  const size_t acc = acc_size(dt), op = dtype_size(dt);
  const bool h16 = dtype_is_16(dt);
  L.ldm = pad16(m);
  L.ldn = pad16(n);
  const int64_t ldx = std::max(L.ldm, L.ldn);
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  L.status = take(sizeof(DeviceStatus));
  L.ntilecnt = (std::max(m, n) + 127) / 128 + 1;
  L.tilecnt = take((size_t)L.ntilecnt * sizeof(int));
  // TF32 tensor cores read A only K-major (an MN-major TF32 operand gave
  // all-zero products on GB300), so the fp32-container dtypes keep a
  // transposed copy A^T (n x m, ld ldn) for T1 = A T2 and W = A Q2.
  L.has_at = (dt == SORSVD_F32 || dt == SORSVD_TF32);
  L.at = L.has_at ? take((size_t)L.ldn * (at_rows >= 0 ? at_rows : m) * 4) : 0;
  L.t2op = h16 ? take((size_t)L.ldn * l * op) : 0;
  L.t2 = take((size_t)L.ldn * l * acc);
  if (!h16) L.t2op = L.t2;
  L.t1 = take((size_t)L.ldm * l * acc);
  L.t1op = h16 ? take((size_t)L.ldm * l * op) : L.t1;
  L.q2op = h16 ? take((size_t)2 * L.ldn * l * op) : 0;
  L.tmp = take((size_t)ldx * l * acc);
  // F32: hi / lo TF32 parts of the skinny operand of the split products
  L.ldb = ldx;
  if (dt == SORSVD_F32) {
    L.bhi = take((size_t)ldx * l * 4);
    L.blo = take((size_t)ldx * l * 4);
  }
  // split-K partials of the CUDA-core products and the stream-K partials of
  // the tensor-core passes share one buffer (never live at the same time);
  // an l x l product always goes through it because its binary64 result is
  // a reduction.
  size_t pb = 0;
  auto need = [&](int64_t M, int64_t N, int64_t K, int cap, bool always) {
    int s = splits_for(M, N, K, cap, dt == SORSVD_F64);
    if (s > 1 || always) pb = std::max(pb, (size_t)s * M * N * acc);
  };
  need(m, l, n, kCapBig, false);     // T1 = A T2, W = A Q2
  need(n, l, m, kCapBig, false);     // T2 = A^T T1
  need(l, l, m, kCapSmall, true);    // Gram of T1, M = Q1^T W
  need(l, l, n, kCapSmall, true);    // Gram of T2
  need(m, l, l, kCapBig, false);     // T1 R^{-1}
  need(n, l, l, kCapBig, false);     // T2 R^{-1}
  for (int k = 1; k <= l; ++k) {     // U = Q1 U~_k, V = Q2 V~_k (k unknown here)
    need(m, k, l, kCapBig, false);
    need(n, k, l, kCapBig, false);
  }
  const int elt = elt_of(dt);
  if (elt >= 0) {
    pb = std::max(pb, tc_parts_bytes(elt, m, l, n));
    pb = std::max(pb, tc_parts_bytes(elt, n, l, m));
  }
  if (dt == SORSVD_F32) {                           // fp32-accurate split passes
    pb = std::max(pb, tc_parts_bytes(3, m, l, n));
    pb = std::max(pb, tc_parts_bytes(3, n, l, m));
  }
  if (dt != SORSVD_F64) {                           // row-block Gram partials
    pb = std::max(pb, rb_gram_parts_bytes(m, l, l, true));
    pb = std::max(pb, rb_gram_parts_bytes(n, l, l, true));
    pb = std::max(pb, rb_gram_parts_bytes(m, l, l, false));
    if (l <= kTskMaxL) {                            // tensor-core Gram partials
      pb = std::max(pb, (size_t)tsk_gram_parts(m) * l * l * sizeof(float));
      pb = std::max(pb, (size_t)tsk_gram_parts(n) * l * l * sizeof(float));
      pb = std::max(pb, (size_t)tsk_xty_parts(m, l) * l * l * sizeof(float));
      pb = std::max(pb, (size_t)tsk_xty_parts(n, l) * l * l * sizeof(float));
    }
  }
  L.parts = take(pb);
  L.G = take((size_t)l * l * 8);
  L.Rinv = take((size_t)l * l * acc);
  L.M = take((size_t)l * l * 8);
  L.Ut = take((size_t)l * l * acc);
  L.Vt = take((size_t)l * l * acc);
  // the Jacobi work area doubles as the scratch of the polar second
  // CholeskyQR pass (the two are never live at the same time)
  L.jwork = take(std::max(jacobi_work_bytes(l), polar_scratch_bytes(l)));
  L.ldk = (l + 31) / 32 * 32;
  L.bsplit = dt != SORSVD_F64 ? take((size_t)2 * L.ldk * L.ldk * sizeof(float)) : 0;
  if (flags & (SORSVD_FLAG_TWO_PASS | SORSVD_FLAG_RSVD | SORSVD_FLAG_TSR)) {
    L.t1s = take((size_t)L.ldm * l * acc);
    L.t2s = take((size_t)L.ldn * l * acc);
    L.tp = take((size_t)5 * l * l * 8);
  }
  L.total = off;
  return L;
}

struct Ctx {
  char* ws;
  Layout L;
  int dt;
  bool f64;
  cudaStream_t st;
  DeviceStatus* status() const { return reinterpret_cast<DeviceStatus*>(ws + L.status); }
  void* at(size_t o) const { return ws + o; }
};

// clear the status word and the split-tile counters of the passes (the
// counters return to zero after every complete pass)
cudaError_t begin_call(const Ctx& c) {
  cudaError_t e = cudaMemsetAsync(c.status(), 0, sizeof(DeviceStatus), c.st);
  if (e != cudaSuccess) return e;
  return cudaMemsetAsync(c.at(c.L.tilecnt), 0, (size_t)c.L.ntilecnt * sizeof(int), c.st);
}

#define CK(x) do { cudaError_t e_ = (x); if (e_ != cudaSuccess) return SORSVD_ERR_CUDA; } while (0)

// C (M x N, ldc) = op(A) B on CUDA cores, with split-K through the partial
// buffer when useful.
int gemm(const Ctx& c, int kcls, bool trans, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
         int adt, const void* B, int64_t ldb, int bdt, void* C, int64_t ldc, bool c_f64, int cap,
         const int* skip = nullptr) {
  const bool accf = c.f64;
  int s = splits_for(M, N, K, cap, accf);
  if (s == 1 && (c_f64 == accf)) {
    ProfScope ps(kcls, c.st);
    CK(launch_gemm(trans, M, N, K, A, lda, adt, B, ldb, bdt, C, ldc, accf, 1, 0, c.st, skip));
    return SORSVD_OK;
  }
  int64_t stride = M * N;
  {
    ProfScope ps(kcls, c.st);
    CK(launch_gemm(trans, M, N, K, A, lda, adt, B, ldb, bdt, c.at(c.L.parts), M, accf, s, stride, c.st, skip));
  }
  ProfScope ps(K_REDUCE, c.st);
  CK(launch_reduce_splits(c.at(c.L.parts), accf, s, stride, M, N, M, C, c_f64, ldc, c.st, skip));
  return SORSVD_OK;
}

// a single launch of class `kcls`
#define LAUNCH(kcls, expr) do { ProfScope ps_(kcls, c.st); CK(expr); } while (0)

// One pass over A: C (fp32, M x N) = op(A) B with B in the pass element type,
// plus an optional 16-bit copy of C.  Tensor cores when the operands allow
// TMA (16-byte aligned bases and strides), CUDA cores otherwise.
// `precise` asks fp32 containers (F32) for fp32-accurate products: the split
// tensor-core mode (hi*hi + hi*lo + lo*hi TF32 MMAs).
int pass(const Ctx& c, int kcls, bool trans, int64_t M, int64_t N, int64_t K, const void* A, int64_t lda,
         const void* B, int64_t ldb, int bdt, void* C, int64_t ldc, void* C16, int64_t ld16, bool precise) {
  const int dt = c.dt;
  const int elt = (precise && dt == SORSVD_F32) ? 3 : elt_of(dt);
  const bool b_ok = (elt >= 2) ? (bdt == SORSVD_F32 || bdt == SORSVD_TF32) : (bdt == dt);
  if (elt >= 0 && b_ok && tc_enabled()) {
    // fp32 containers: A X = (A^T)^T X through the transposed copy
    const bool use_at = (elt >= 2 && !trans);
    const void* Aop = use_at ? c.at(c.L.at) : A;
    const int64_t ldop = use_at ? c.L.ldn : lda;
    // split mode keeps two [D1 | D2] accumulator fills of <= kSplitMaxCols
    // columns in TMEM: wider skinny operands run as column chunks, one
    // launch each (every chunk re-reads A; at these widths the split
    // products are bound by their MMAs, not by the reads of A)
    const int nchunk = (elt == 3 && N > kSplitMaxCols) ? (int)((N + kSplitChunkCols - 1) / kSplitChunkCols) : 1;
    const int64_t wchunk = nchunk > 1 ? (N + nchunk - 1) / nchunk : N;
    const int64_t wpad = nchunk > 1 ? (wchunk + 15) / 16 * 16 : N;
    if ((!use_at || c.L.has_at) && tc_supported(elt, Aop, ldop, B, ldb, (int)wpad)) {
      const void* Bop = B;
      int64_t ldbop = ldb;
      if (elt == 3) {
        // the skinny operand is split once per pass, the A tiles in the kernel
        LAUNCH(K_MISC, launch_split_tf32((const float*)B, ldb, K, N, (float*)c.at(c.L.bhi),
                                         (float*)c.at(c.L.blo), c.L.ldb, c.st));
        Bop = c.at(c.L.bhi);
        ldbop = c.L.ldb;
      }
      for (int64_t c0 = 0; c0 < N; c0 += wpad) {
        const int64_t w = std::min<int64_t>(wpad, N - c0);
        const size_t eb = elt >= 2 ? 4 : 2;
        const void* Bc = (const char*)Bop + (size_t)c0 * ldbop * eb;
        const void* Blo = (const char*)c.at(c.L.blo) + (size_t)c0 * c.L.ldb * 4;
        void* C16c = C16 ? (void*)((char*)C16 + (size_t)c0 * ld16 * 2) : nullptr;
        CK(launch_tc_gemm(trans || use_at, elt, M, w, K, Aop, ldop, Bc, ldbop, Blo, (float*)C + c0 * ldc, ldc,
                          C16c, ld16, dt == SORSVD_BF16 ? 1 : 2, (float*)c.at(c.L.parts), (int*)c.at(c.L.tilecnt),
                          c.L.ntilecnt, c.status(), kcls, c.st));
      }
      return SORSVD_OK;
    }
  }
  int r = gemm(c, kcls, trans, M, N, K, A, lda, dt, B, ldb, bdt, C, ldc, c.f64, kCapBig);
  if (r) return r;
  if (C16) LAUNCH(K_MISC, launch_convert_f32((const float*)C, ldc, M, N, C16, ld16, dt, nullptr, c.st));
  return SORSVD_OK;
}

// Non-blocking streams of this device for work that runs beside the
// caller's stream (created once per device; nullptr when that fails).
// which = 0: Omega, highest priority (its blocks are placed before the
// caller's queued ones); which = 1: host <-> device copies.
cudaStream_t side_stream(int which = 0) {
  static cudaStream_t streams[2][64] = {{nullptr}};
  static bool tried[2][64] = {{false}};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64 || which < 0 || which > 1) return nullptr;
  if (!tried[which][dev]) {
    tried[which][dev] = true;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (cudaStreamCreateWithPriority(&streams[which][dev], cudaStreamNonBlocking, which == 0 ? hi : lo) != cudaSuccess)
      streams[which][dev] = nullptr;
  }
  return streams[which][dev];
}

// Omega on the side stream while `work` runs on the caller's stream; the
// caller's stream then waits for Omega (fork and join by events, which
// stream capture also follows)
template <typename Work>
int gaussian_beside(const Ctx& c, void* out, int64_t rows, int cols, int64_t ld, uint64_t seed, int dtype, Work work) {
  cudaStream_t side = side_stream();
  cudaEvent_t fork = nullptr, join = nullptr;
  if (!side || cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
    if (fork) cudaEventDestroy(fork);
    int r = work();
    if (r) return r;
    LAUNCH(K_GAUSSIAN, launch_gaussian(out, rows, cols, ld, seed, 0, dtype, c.st));
    return SORSVD_OK;
  }
  int r = SORSVD_OK;
  if (cudaEventRecord(fork, c.st) != cudaSuccess || cudaStreamWaitEvent(side, fork, 0) != cudaSuccess) {
    r = SORSVD_ERR_CUDA;
  } else {
    {
      ProfScope ps(K_GAUSSIAN, side);
      if (launch_gaussian(out, rows, cols, ld, seed, 0, dtype, side) != cudaSuccess) r = SORSVD_ERR_CUDA;
    }
    if (cudaEventRecord(join, side) != cudaSuccess) r = SORSVD_ERR_CUDA;
    const int rw = work();
    if (!r) r = rw;
    if (cudaStreamWaitEvent(c.st, join, 0) != cudaSuccess && !r) r = SORSVD_ERR_CUDA;
  }
  cudaEventDestroy(fork);
  cudaEventDestroy(join);
  return r;
}

// A^T into the workspace (fp32 containers), once per call that passes over A
int prepare_at(const Ctx& c, const void* A, int64_t m, int64_t n, int64_t lda) {
  if (!c.L.has_at || !tc_enabled()) return SORSVD_OK;
  LAUNCH(K_MISC, launch_transpose_f32((const float*)A, lda, m, n, (float*)c.at(c.L.at), c.L.ldn, c.st));
  return SORSVD_OK;
}

// T (rows x l, ld, accumulator type) <- T R^{-1}, repeated `passes` times
// (CholeskyQR); the first pass is shifted by shift0.  fp32 sketches use the
// row-block kernels: the products ping-pong between T and the tmp buffer
// (same ld) and the result is copied back to T after an odd number of
// passes; the third pass of CholeskyQR3 only runs when the second pass's
// Gram was not already within kOrthTol of the identity (decided on the
// device; a skipped pass leaves the result in T).  out16, when non-null,
// receives the 16-bit rounding of the result (the operand of the next
// BF16 / F16 pass).  With `result` non-null and a single pass the
// product stays in the tmp buffer (ld unchanged) and *result points to it:
// no copy back.  binary64 sketches use the CUDA-core GEMMs.
// G (binary64, l x l) = T^T T of an fp32 rows x l matrix: tensor cores
// (split TF32) when they apply, else the row-block kernel; the partials are
// summed in a fixed order
int gram_sym(const Ctx& c, const float* T, int64_t ld, int64_t rows, int l, const int* skip, double* G = nullptr,
             int64_t ldg = 0) {
  float* parts = (float*)c.at(c.L.parts);
  if (!G) { G = (double*)c.at(c.L.G); ldg = l; }
  if (tsk_gram_supported(T, ld, l)) {
    int np = 0, split = -1;
    LAUNCH(K_SMALL_GEMM, launch_tsk_gram(T, ld, rows, l, parts, &np, &split, skip, c.status(), c.st));
    LAUNCH(K_REDUCE, launch_reduce_parts(parts, np, (int64_t)l * l, l, l, l, G, (int)ldg, c.st, split));
    return SORSVD_OK;
  }
  LAUNCH(K_SMALL_GEMM, launch_rb_gram(T, ld, T, ld, rows, l, l, true, parts, skip, c.st));
  LAUNCH(K_REDUCE, launch_reduce_parts(parts, (int)rb_gram_blocks(rows, l, l, true), (int64_t)l * l, l, l, l, G,
                                       (int)ldg, c.st));
  return SORSVD_OK;
}

// Y (rows x N, ldy) = T B for fp32 T (rows x K) and B (K x N, ldb), out of
// place, with an optional 16-bit rounding: tensor cores (B split into TF32
// hi / lo first) when they apply, else the row-block kernel
int apply(const Ctx& c, const float* T, int64_t ld, int64_t rows, int K, const float* B, int64_t ldb, int N,
          bool tri, float* Y, int64_t ldy, void* Y16, int64_t ld16, int kind16, const int* skip) {
  // bsplit holds 2 ldk x ldk floats' worth: K <= ldk rows, N <= ldk columns each
  if (c.L.bsplit && K <= c.L.ldk && N <= c.L.ldk && tsk_apply_supported(T, ld, K, N)) {
    float* hi = (float*)c.at(c.L.bsplit);
    float* lo = hi + (size_t)c.L.ldk * N;
    LAUNCH(K_SMALL_GEMM, launch_split_tf32(B, ldb, K, N, hi, lo, c.L.ldk, c.st));
    LAUNCH(K_SMALL_GEMM, launch_tsk_apply(T, ld, rows, K, hi, lo, c.L.ldk, N, tri, Y, ldy, Y16, ld16, kind16, skip,
                                          c.status(), c.st));
    return SORSVD_OK;
  }
  LAUNCH(K_SMALL_GEMM, launch_rb_apply(T, ld, rows, K, B, ldb, N, tri, Y, ldy, Y16, ld16, kind16, skip, c.st));
  return SORSVD_OK;
}

int orth(const Ctx& c, void* T, int64_t rows, int64_t ld, int l, int passes, double shift0, void* out16 = nullptr,
         int64_t ld16 = 0, void** result = nullptr) {
  const int kind16 = out16 ? (c.dt == SORSVD_BF16 ? 1 : 2) : 0;
  if (result) *result = T;
  if (!c.f64 && result && passes == 1) {
    // with a 16-bit copy requested, that copy is the only result the
    // caller reads (the next product's operand): the fp32 Q is not written
    // and *result is null
    float* Y = out16 ? nullptr : (float*)c.at(c.L.tmp);
    int r = gram_sym(c, (const float*)T, ld, rows, l, nullptr);
    if (r) return r;
    LAUNCH(K_CHOL, launch_chol_inv((const double*)c.at(c.L.G), l, shift0, c.at(c.L.Rinv), false, c.status(), c.st));
    r = apply(c, (const float*)T, ld, rows, l, (const float*)c.at(c.L.Rinv), l, l, true, Y, ld, out16, ld16, kind16,
              nullptr);
    if (r) return r;
    *result = Y;
    return SORSVD_OK;
  }
  if (!c.f64) {
    int* conv = c.status()->pad;
    int* pol_ok = c.status()->pad + 1;
    float* X = (float*)T;
    float* Y = (float*)c.at(c.L.tmp);
    for (int p = 0; p < passes; ++p) {
      const int* skip = p == 2 ? conv : nullptr;
      // second pass: the Gram is close to I; its polar factor (series) when
      // it converges, the Cholesky factorisation otherwise (decided on the
      // device); the polar factor is a full matrix
      const bool polar = p == 1 && polar_enabled();
      int r = gram_sym(c, X, ld, rows, l, skip);
      if (r) return r;
      if (polar)
        LAUNCH(K_CHOL, launch_polar_inv((const double*)c.at(c.L.G), l, (float*)c.at(c.L.Rinv),
                                        (float*)c.at(c.L.jwork), pol_ok, conv, kOrthTol, c.st));
      LAUNCH(K_CHOL, launch_chol_inv((const double*)c.at(c.L.G), l, p == 0 ? shift0 : 0.0, c.at(c.L.Rinv), false,
                                     c.status(), c.st, skip, p == 1 ? conv : nullptr, kOrthTol,
                                     polar ? pol_ok : nullptr));
      // the 16-bit copy comes from the last pass that runs: the last pass,
      // and the second of three (the third may be skipped on the device)
      void* o16 = (p == passes - 1 || (passes == 3 && p == 1)) ? out16 : nullptr;
      r = apply(c, X, ld, rows, l, (const float*)c.at(c.L.Rinv), l, l, !polar, Y, ld, o16, ld16, o16 ? kind16 : 0,
                skip);
      if (r) return r;
      std::swap(X, Y);
    }
    // the fp32 result back into T (not when a skipped third pass left it there)
    if (X != (float*)T)
      LAUNCH(K_MISC, launch_rb_copy(X, (float*)T, ld, rows, l, nullptr, 0, 0, passes == 3 ? conv : nullptr, c.st));
    return SORSVD_OK;
  }
  // binary64: the same device-side skip of the third pass as above (the
  // second pass's input within kOrthTol of orthonormal leaves T
  // orthonormal to working precision)
  const int adt = SORSVD_F64;
  int* conv = c.status()->pad;
  for (int p = 0; p < passes; ++p) {
    const int* skip = p == 2 ? conv : nullptr;
    int r = gemm(c, K_SMALL_GEMM, true, l, l, rows, T, ld, adt, T, ld, adt, c.at(c.L.G), l, true, kCapSmall, skip);
    if (r) return r;
    LAUNCH(K_CHOL, launch_chol_inv((const double*)c.at(c.L.G), l, p == 0 ? shift0 : 0.0, c.at(c.L.Rinv), c.f64,
                                   c.status(), c.st, skip, p == 1 ? conv : nullptr, kOrthTol));
    r = gemm(c, K_SMALL_GEMM, false, rows, l, l, T, ld, adt, c.at(c.L.Rinv), l, adt, c.at(c.L.tmp), ld, c.f64,
             kCapBig, skip);
    if (r) return r;
    LAUNCH(K_MISC, launch_copy2d(c.at(c.L.tmp), ld, T, ld, rows, l, acc_size(c.dt), c.st, skip));
  }
  return SORSVD_OK;
}

// M (l x l, binary64, ldm) = X^T Y for X, Y rows x l in the accumulator type
int cross_gram(const Ctx& c, const void* X, int64_t ldx, const void* Y, int64_t ldy, int64_t rows, int l, double* M,
               int64_t ldm) {
  const bool aligned = !((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) & 15) && !((ldx | ldy) & 3);
  if (c.f64 || !aligned) {
    const int adt = c.f64 ? SORSVD_F64 : SORSVD_F32;
    return gemm(c, K_SMALL_GEMM, true, l, l, rows, X, ldx, adt, Y, ldy, adt, M, ldm, true, kCapSmall);
  }
  float* parts = (float*)c.at(c.L.parts);
  if (tsk_xty_supported((const float*)X, ldx, (const float*)Y, ldy, l)) {
    int np = 0;
    LAUNCH(K_SMALL_GEMM, launch_tsk_xty((const float*)X, ldx, (const float*)Y, ldy, rows, l, parts, &np, nullptr,
                                        c.status(), c.st));
    LAUNCH(K_REDUCE, launch_reduce_parts(parts, np, (int64_t)l * l, l, l, l, M, (int)ldm, c.st));
    return SORSVD_OK;
  }
  LAUNCH(K_SMALL_GEMM, launch_rb_gram((const float*)X, ldx, (const float*)Y, ldy, rows, l, l, false, parts, nullptr,
                                      c.st));
  LAUNCH(K_REDUCE, launch_reduce_parts(parts, (int)rb_gram_blocks(rows, l, l, false), (int64_t)l * l, l, l, l, M,
                                       (int)ldm, c.st));
  return SORSVD_OK;
}

// C (rows x k, ldc) = Q (rows x l) B (l x k, ld l), accumulator type
int assemble(const Ctx& c, const void* Q, int64_t ldq, int64_t rows, int l, const void* B, int k, void* C,
             int64_t ldc) {
  if (c.f64 || (reinterpret_cast<uintptr_t>(Q) & 15) || (ldq & 3))
    return gemm(c, K_SMALL_GEMM, false, rows, k, l, Q, ldq, c.f64 ? SORSVD_F64 : SORSVD_F32, B, l,
                c.f64 ? SORSVD_F64 : SORSVD_F32, C, ldc, c.f64, kCapBig);
  return apply(c, (const float*)Q, ldq, rows, l, (const float*)B, l, k, false, (float*)C, ldc, nullptr, 0, 0, nullptr);
}

// T1 = A X (X: the operand buffer of the pass type), then T2 = A^T T1 (the
// 16-bit rounding of T1 for BF16/F16, kept in t1op).
int power_pass_impl(const Ctx& c, const void* A, int64_t m, int64_t n, int64_t lda, const void* xop,
                    int64_t ldx, int l, void* T1, int64_t ldt1, void* T2, int64_t ldt2, bool precise) {
  const int dt = c.dt;
  const bool h16 = dtype_is_16(dt);
  const int opdt = c.f64 ? SORSVD_F64 : (h16 ? dt : SORSVD_F32);
  void* t1op = h16 ? c.at(c.L.t1op) : nullptr;
  const int kc = (precise && c.dt == SORSVD_F32) ? K_PASS_SPLIT : K_PASS;
  int r = pass(c, kc, false, m, l, n, A, lda, xop, ldx, opdt, T1, ldt1, t1op, c.L.ldm, precise);
  if (r) return r;
  const void* y = h16 ? t1op : T1;
  const int64_t ldy = h16 ? c.L.ldm : ldt1;
  return pass(c, kc, true, n, l, m, A, lda, y, ldy, opdt, T2, ldt2, nullptr, 0, precise);
}

// M (l x l, f64, ldm) = Q1^T (A Q2)
int core_impl(const Ctx& c, const void* A, int64_t m, int64_t n, int64_t lda, unsigned flags,
              const void* Q1, int64_t ldq1, const void* Q2, int64_t ldq2, int l, double* M, int64_t ldm) {
  const int dt = c.dt, adt = c.f64 ? SORSVD_F64 : SORSVD_F32;
  const int64_t ldw = c.L.ldm;
  int r;
  if (dtype_is_16(dt) && !(flags & SORSVD_FLAG_REFINE)) {
    LAUNCH(K_MISC, launch_convert_f32((const float*)Q2, ldq2, n, l, c.at(c.L.q2op), c.L.ldn, dt, nullptr, c.st));
    r = pass(c, K_CORE, false, m, l, n, A, lda, c.at(c.L.q2op), c.L.ldn, dt, c.at(c.L.tmp), ldw, nullptr, 0, false);
  } else if (dtype_is_16(dt) && tc_enabled()) {
    // REFINE: Q2 = hi + lo as a pair of 16-bit operands (lo = round(Q2 - hi)
    // carries the next 8-11 bits), two tensor-core passes over A, and
    // M = Q1^T (A hi) + Q1^T (A lo) combined in binary64
    char* hi = (char*)c.at(c.L.q2op);
    char* lo = hi + (size_t)c.L.ldn * l * dtype_size(dt);
    LAUNCH(K_MISC, launch_convert_f32((const float*)Q2, ldq2, n, l, hi, c.L.ldn, dt, lo, c.st));
    r = pass(c, K_CORE, false, m, l, n, A, lda, hi, c.L.ldn, dt, c.at(c.L.tmp), ldw, nullptr, 0, false);
    if (r) return r;
    r = cross_gram(c, Q1, ldq1, c.at(c.L.tmp), ldw, m, l, M, ldm);
    if (r) return r;
    r = pass(c, K_CORE, false, m, l, n, A, lda, lo, c.L.ldn, dt, c.at(c.L.tmp), ldw, nullptr, 0, false);
    if (r) return r;
    r = cross_gram(c, Q1, ldq1, c.at(c.L.tmp), ldw, m, l, (double*)c.at(c.L.G), l);
    if (r) return r;
    LAUNCH(K_MISC, launch_add_f64((const double*)c.at(c.L.G), l, M, ldm, l, l, c.st));
    return SORSVD_OK;
  } else if (dt == SORSVD_TF32 || dt == SORSVD_F32) {
    // TF32: one TF32 product; F32: the split (fp32-accurate) product
    r = pass(c, K_CORE, false, m, l, n, A, lda, Q2, ldq2, SORSVD_F32, c.at(c.L.tmp), ldw, nullptr, 0, true);
  } else {
    // binary64, and BF16/F16 with REFINE when tensor cores are switched
    // off: the fp32 Q2 multiplies the stored A exactly on CUDA cores
    r = gemm(c, K_CORE, false, m, l, n, A, lda, dt, Q2, ldq2, adt, c.at(c.L.tmp), ldw, c.f64, kCapBig);
  }
  if (r) return r;
  return cross_gram(c, Q1, ldq1, c.at(c.L.tmp), ldw, m, l, M, ldm);
}

int check_dtype(int dt) { return (dt >= SORSVD_F64 && dt <= SORSVD_F16) ? SORSVD_OK : SORSVD_ERR_DTYPE; }

// the method flags of sorsvd_run / sorsvd_run_host: at most one of
// TWO_PASS, RSVD and TSR; RSVD and TSR need the stabilised loop; TSR is a
// single round (q = 0)
bool method_flags_ok(unsigned flags, int q) {
  const int methods = !!(flags & SORSVD_FLAG_TWO_PASS) + !!(flags & SORSVD_FLAG_RSVD) + !!(flags & SORSVD_FLAG_TSR);
  if (methods > 1) return false;
  if ((flags & (SORSVD_FLAG_RSVD | SORSVD_FLAG_TSR)) && (flags & SORSVD_FLAG_LITERAL_POWER)) return false;
  if ((flags & SORSVD_FLAG_TSR) && q != 0) return false;
  return true;
}

int check_ws(void* ws, size_t ws_bytes, const Layout& L) {
  if (!ws) return SORSVD_ERR_WORKSPACE;
  if (((uintptr_t)ws) % kAlign) return SORSVD_ERR_WORKSPACE;
  if (ws_bytes < L.total) return SORSVD_ERR_WORKSPACE;
  return SORSVD_OK;
}

int max_l(int dt) { return dt == SORSVD_F64 ? SORSVD_MAX_L_F64 : SORSVD_MAX_L; }

// Device copies of A, U, S, V for sorsvd_run_host, after the solve's own
// workspace (256-byte aligned regions; leading dimensions padded so that
// the tensor-core passes can map A).
struct HostIo {
  size_t a, u, s, v, total;
  int64_t lda, ldu, ldv;
};

HostIo host_io_layout(size_t base, int64_t m, int64_t n, int k, int dt) {
  HostIo H{};
  const size_t op = dtype_size(dt), acc = acc_size(dt);
  size_t off = align_up(base);
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  H.lda = pad16(m);
  H.ldu = pad16(m);
  H.ldv = pad16(n);
  H.a = take((size_t)H.lda * n * op);
  H.u = take((size_t)H.ldu * k * acc);
  H.s = take((size_t)k * acc);
  H.v = take((size_t)H.ldv * k * acc);
  H.total = off;
  return H;
}

// A (host, column-major, lda) -> its device copy Ad (ld ldd) in column
// blocks of about 64 MiB on the copy stream.  For the fp32 containers each
// block's part of the transposed copy A^T is made on c.st as soon as the
// block has landed, so the transpose runs under the remaining copies; c.st
// waits for every block before it goes on.
int upload_a(const Ctx& c, const void* Ah, int64_t lda, int64_t m, int64_t n, void* Ad, int64_t ldd) {
  const size_t esz = dtype_size(c.dt);
  const bool at = c.L.has_at && tc_enabled();
  const size_t col_bytes = std::max<size_t>(1, (size_t)m * esz);
  int64_t cols = std::max<int64_t>(1, (int64_t)((size_t)(64u << 20) / col_bytes));
  const int nblk = (int)std::min<int64_t>(32, (n + cols - 1) / cols);
  cols = ((n + nblk - 1) / nblk + 63) / 64 * 64;   // whole 64-column tiles of the transpose
  auto copy_cols = [&](int64_t j0, int64_t j1, cudaStream_t st) {
    return cudaMemcpy2DAsync((char*)Ad + (size_t)j0 * ldd * esz, (size_t)ldd * esz,
                             (const char*)Ah + (size_t)j0 * lda * esz, (size_t)lda * esz, (size_t)m * esz,
                             (size_t)(j1 - j0), cudaMemcpyHostToDevice, st);
  };
  float* At = at ? (float*)c.at(c.L.at) : nullptr;
  cudaStream_t cs = side_stream(1);
  std::vector<cudaEvent_t> ev(nblk + 1, nullptr);
  bool events = cs != nullptr;
  for (int b = 0; b <= nblk && events; ++b)
    events = cudaEventCreateWithFlags(&ev[b], cudaEventDisableTiming) == cudaSuccess;
  int r = SORSVD_OK;
  if (!events) {
    // no copy stream: one copy, then the transposed copy, both on c.st
    if (copy_cols(0, n, c.st) != cudaSuccess) r = SORSVD_ERR_CUDA;
    else if (at) r = prepare_at(c, Ad, m, n, ldd);
  } else if (cudaEventRecord(ev[nblk], c.st) != cudaSuccess || cudaStreamWaitEvent(cs, ev[nblk], 0) != cudaSuccess) {
    r = SORSVD_ERR_CUDA;
  } else {
    for (int b = 0; b < nblk && !r; ++b) {
      const int64_t j0 = b * cols, j1 = std::min<int64_t>(n, j0 + cols);
      if (j0 >= j1) break;
      if (copy_cols(j0, j1, cs) != cudaSuccess || cudaEventRecord(ev[b], cs) != cudaSuccess) { r = SORSVD_ERR_CUDA; break; }
      if (at || j1 == n) {
        if (cudaStreamWaitEvent(c.st, ev[b], 0) != cudaSuccess) { r = SORSVD_ERR_CUDA; break; }
      }
      if (at) {
        ProfScope ps(K_MISC, c.st);
        if (launch_transpose_f32((const float*)((char*)Ad + (size_t)j0 * ldd * esz), ldd, m, j1 - j0, At + j0,
                                 c.L.ldn, c.st) != cudaSuccess)
          r = SORSVD_ERR_CUDA;
      }
    }
  }
  for (cudaEvent_t e : ev)
    if (e) cudaEventDestroy(e);
  return r;
}

// Keep the operand X (n x l, ldx; the pass element type) of the last
// product T1 = A X as T2_prev for the two-pass core: fp32 (binary64 for
// F64), the 16-bit operand widened exactly.
int save_t2prev(const Ctx& c, const void* X, int64_t ldx, int64_t n, int l) {
  if (dtype_is_16(c.dt)) {
    LAUNCH(K_MISC, launch_widen(X, c.dt, ldx, n, l, c.at(c.L.t2s), false, c.L.ldn, c.st));
  } else {
    LAUNCH(K_MISC, launch_copy2d(X, ldx, c.at(c.L.t2s), c.L.ldn, n, l, acc_size(c.dt), c.st));
  }
  return SORSVD_OK;
}

// The two-pass core (Sec. III): M (l x l, binary64) = C B^+ with
// C = Q1^T T1 and B = Q2^T T2_prev, B^+ = B^T (B B^T)^{-1} and
// (B B^T)^{-1} = R^{-1} R^{-T} from the Cholesky-inverse kernel (binary64
// factor for l <= SORSVD_MAX_L_F64, fp32 above: then the error grows with
// cond(B)^2, which stays near 1 once the power loop has converged).
int core_two_pass(const Ctx& c, int64_t m, int64_t n, int l, double* M) {
  const Layout& L = c.L;
  double* tp = (double*)c.at(L.tp);
  const size_t ll = (size_t)l * l;
  double *Cm = tp, *Bm = tp + ll, *R = tp + 2 * ll, *W = tp + 3 * ll, *V = tp + 4 * ll;
  double* G = (double*)c.at(L.G);
  int r = cross_gram(c, c.at(L.t1), L.ldm, c.at(L.t1s), L.ldm, m, l, Cm, l);
  if (r) return r;
  r = cross_gram(c, c.at(L.t2), L.ldn, c.at(L.t2s), L.ldn, n, l, Bm, l);
  if (r) return r;
  LAUNCH(K_SMALL_GEMM, launch_small_gemm64(Bm, false, Bm, true, G, l, c.st));         // B B^T
  const bool r64 = l <= SORSVD_MAX_L_F64;
  LAUNCH(K_CHOL, launch_chol_inv(G, l, 0.0, r64 ? (void*)R : c.at(L.Rinv), r64, c.status(), c.st));
  if (!r64) LAUNCH(K_MISC, launch_widen(c.at(L.Rinv), SORSVD_F32, l, l, l, R, true, l, c.st));
  LAUNCH(K_SMALL_GEMM, launch_small_gemm64(Cm, false, Bm, true, W, l, c.st));          // C B^T
  LAUNCH(K_SMALL_GEMM, launch_small_gemm64(W, false, R, false, V, l, c.st));           // . R^{-1}
  LAUNCH(K_SMALL_GEMM, launch_small_gemm64(V, false, R, true, M, l, c.st));            // . R^{-T}
  return SORSVD_OK;
}

// Algorithm 3 after Omega (in t2op) and, for the fp32 containers, the
// transposed copy of A are in place: the power loop, the QR step, the core,
// its truncated SVD and the output assembly, all queued on c.st.
int solve(const Ctx& c, const void* A, int64_t m, int64_t n, int64_t lda, int k, int l, int q, unsigned flags,
          uint64_t seed, void* U, int64_t ldu, void* S, void* V, int64_t ldv) {
  const Layout& L = c.L;
  const int dtype = c.dt;
  const int adt = c.f64 ? SORSVD_F64 : SORSVD_F32;
  const bool h16 = dtype_is_16(dtype);
  const bool two = (flags & SORSVD_FLAG_TWO_PASS) != 0;
  const bool rsvd = (flags & SORSVD_FLAG_RSVD) != 0;
  const bool tsr = (flags & SORSVD_FLAG_TSR) != 0;
  auto orth1 = [&](int np, void* o16, void** res) {
    return orth(c, c.at(L.t1), m, L.ldm, l, np, first_shift(dtype), o16, L.ldm, res);
  };
  auto orth2 = [&](int np, void* o16, void** res) {
    return orth(c, c.at(L.t2), n, L.ldn, l, np, first_shift(dtype), o16, L.ldn, res);
  };
  int r;
  if (tsr) {
    // Algorithm 2 (TSR-SVD): Y1 = A Psi1 with Psi1 = Omega (in t2op) and
    // Y2 = A^T Psi2 with Psi2 (m x l) from Philox stream 1, one round; QR of
    // both; B_approx = Q1^T Y1 (Q2^T Psi1)^+ by the two-pass core, with Y1
    // and Psi1 kept before the QR
    // (for the fp32 and binary64 containers Omega shares its buffer with T2,
    // so Psi1 is read from its saved copy and Psi2 waits in the T1 copy)
    const int kc = dtype == SORSVD_F32 ? K_PASS_SPLIT : K_PASS;
    r = save_t2prev(c, c.at(L.t2op), L.ldn, n, l);
    if (r) return r;
    void* psi2 = h16 ? c.at(L.t1op) : c.at(L.t1s);
    const void* psi1 = h16 ? c.at(L.t2op) : c.at(L.t2s);
    LAUNCH(K_GAUSSIAN, launch_gaussian(psi2, m, l, L.ldm, seed, 1, dtype, c.st));
    r = pass(c, kc, true, n, l, m, A, lda, psi2, L.ldm, h16 ? dtype : adt, c.at(L.t2), L.ldn, nullptr, 0, true);
    if (r) return r;
    r = pass(c, kc, false, m, l, n, A, lda, psi1, L.ldn, h16 ? dtype : adt, c.at(L.t1), L.ldm, nullptr, 0, true);
    if (r) return r;
    LAUNCH(K_MISC, launch_copy2d(c.at(L.t1), L.ldm, c.at(L.t1s), L.ldm, m, l, acc_size(dtype), c.st));
    r = orth1(3, nullptr, nullptr);
    if (r) return r;
    r = orth2(3, nullptr, nullptr);
    if (r) return r;
  } else if (flags & SORSVD_FLAG_LITERAL_POWER) {
    // Algorithm 3 as printed: the sketches are orthonormalised only at the end
    for (int i = 1; i <= q + 1; ++i) {
      if (i > 1 && h16)
        LAUNCH(K_MISC, launch_convert_f32((const float*)c.at(L.t2), L.ldn, n, l, c.at(L.t2op), L.ldn, dtype, nullptr,
                                          c.st));
      if (i == q + 1 && two) {
        r = save_t2prev(c, c.at(L.t2op), L.ldn, n, l);
        if (r) return r;
      }
      r = power_pass_impl(c, A, m, n, lda, c.at(L.t2op), L.ldn, l, c.at(L.t1), L.ldm, c.at(L.t2), L.ldn,
                          i == q + 1);
      if (r) return r;
    }
    if (two) LAUNCH(K_MISC, launch_copy2d(c.at(L.t1), L.ldm, c.at(L.t1s), L.ldm, m, l, acc_size(dtype), c.st));
    r = orth1(3, nullptr, nullptr);
    if (r) return r;
    r = orth2(3, nullptr, nullptr);
    if (r) return r;
  } else {
    // Each sketch is orthonormalised as soon as it is formed: T1 before the
    // product A^T T1 and T2 before the next A T2.  By Lemma 1 this leaves
    // range(T1) and range(T2) - hence Q1, Q2 and the result - unchanged,
    // while every product sees the conditioning of A instead of its square
    // (the trailing directions of a fast-decaying spectrum survive fp32).
    // One CholeskyQR pass while the loop only steers the subspace, three
    // (CholeskyQR3) in the last iteration, which fixes Q1 and Q2.
    const int kc = dtype == SORSVD_F32 ? K_PASS_SPLIT : K_PASS;
    void* t1op = h16 ? c.at(L.t1op) : c.at(L.t1);
    const void* x2 = c.at(L.t2op);           // operand of the next product A X (Omega first)
    for (int i = 1; i <= q + 1; ++i) {
      const bool last = (i == q + 1);
      const int np = last ? 3 : 1;
      // F32: TF32 products while the loop only steers the subspace, the
      // fp32-accurate split products in the last iteration.  Inside the
      // loop the orthonormalised sketch may stay in the tmp buffer: it is
      // only the operand of the next product.
      if (last && two) {
        r = save_t2prev(c, x2, L.ldn, n, l);
        if (r) return r;
      }
      r = pass(c, last ? kc : K_PASS, false, m, l, n, A, lda, x2, L.ldn, h16 ? dtype : adt, c.at(L.t1), L.ldm,
               nullptr, 0, last);
      if (r) return r;
      if (last && two)
        LAUNCH(K_MISC, launch_copy2d(c.at(L.t1), L.ldm, c.at(L.t1s), L.ldm, m, l, acc_size(dtype), c.st));
      void* q1 = nullptr;
      r = orth1(np, h16 ? t1op : nullptr, last ? nullptr : &q1);
      if (r) return r;
      const void* y1 = h16 ? t1op : (q1 ? q1 : c.at(L.t1));
      r = pass(c, last ? kc : K_PASS, true, n, l, m, A, lda, y1, L.ldm, h16 ? dtype : adt, c.at(L.t2), L.ldn,
               nullptr, 0, last);
      if (r) return r;
      // R-SVD keeps B^T = A^T Q1 (the last T2) before its QR
      if (last && rsvd)
        LAUNCH(K_MISC, launch_copy2d(c.at(L.t2), L.ldn, c.at(L.t2s), L.ldn, n, l, acc_size(dtype), c.st));
      void* q2 = nullptr;
      r = orth2(np, (!last && h16) ? c.at(L.t2op) : nullptr, last ? nullptr : &q2);
      if (r) return r;
      x2 = h16 ? c.at(L.t2op) : (q2 ? q2 : c.at(L.t2));
    }
  }
  if (two || tsr) {
    r = core_two_pass(c, m, n, l, (double*)c.at(L.M));
  } else if (rsvd) {
    // Algorithm 1 (R-SVD): B = Q1^T A = (A^T Q1)^T, whose rows lie in
    // range(Q2) = range(A^T Q1): B = M Q2^T with M = (A^T Q1)^T Q2 (l x l),
    // so the SVD of B is that of M with its right factor multiplied by Q2 -
    // no pass over A beyond the sketch's (2q + 2 in all)
    r = cross_gram(c, c.at(L.t2s), L.ldn, c.at(L.t2), L.ldn, n, l, (double*)c.at(L.M), l);
  } else {
    r = core_impl(c, A, m, n, lda, flags, c.at(L.t1), L.ldm, c.at(L.t2), L.ldn, l, (double*)c.at(L.M), l);
  }
  if (r) return r;
  LAUNCH(K_JACOBI, launch_jacobi((const double*)c.at(L.M), l, k, c.f64, c.at(L.Ut), c.at(L.Vt), S, c.f64,
                                  c.at(L.jwork), c.status(), c.st));
  r = assemble(c, c.at(L.t1), L.ldm, m, l, c.at(L.Ut), k, U, ldu);
  if (r) return r;
  r = assemble(c, c.at(L.t2), L.ldn, n, l, c.at(L.Vt), k, V, ldv);
  if (r) return r;
  return SORSVD_OK;
}

// ---- out-of-core A: host memory, streamed to the device once per pass -----
// The passes over A (Sec. III counts them: 2q + 3 for Algorithm 3) read A
// from host memory in blocks of rows, two device block buffers in
// alternation: the copy of block b + 1 (copy stream) overlaps the products of
// block b (caller's stream).  T1 = A X and W = A Q2 are row-blockwise;
// T2 = A^T Q1 is the sum of the blocks' A_b^T Q1_b.  The sketches, the QR
// step, the core and the small SVD stay on the device as in sorsvd_run.
struct StreamLayout {
  Layout L;              // the solve's regions; the transposed copy holds one block
  size_t blk[2], t2p, total;
  int64_t rows, ldb;     // rows per block, leading dimension of the device blocks
};

StreamLayout stream_layout(int64_t m, int64_t n, int l, int dt, int64_t block_rows) {
  StreamLayout S{};
  S.rows = std::max<int64_t>(1, std::min(block_rows, m));
  S.L = make_layout(m, n, l, dt, 0, S.rows);
  S.ldb = pad16(S.rows);
  size_t off = S.L.total;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  const size_t blk_bytes = (size_t)S.ldb * n * dtype_size(dt);
  S.blk[0] = take(blk_bytes);
  S.blk[1] = take(blk_bytes);
  S.t2p = take((size_t)S.L.ldn * l * acc_size(dt));
  S.total = off;
  return S;
}

// One pass over A: `work(r0, rows, block, ldb)` queues the products of block
// [r0, r0 + rows) on c.st once its copy has landed.
template <typename Work>
int stream_blocks(const Ctx& c, const StreamLayout& SL, const void* Ah, int64_t lda, int64_t m, int64_t n, Work work) {
  const size_t esz = dtype_size(c.dt);
  cudaStream_t cs = side_stream(1);
  if (!cs) cs = c.st;
  cudaEvent_t ev[5] = {};                        // ready[2], freed[2], start
  for (cudaEvent_t& e : ev)
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      for (cudaEvent_t& f : ev)
        if (f) cudaEventDestroy(f);
      return SORSVD_ERR_CUDA;
    }
  int r = SORSVD_OK;
  // the copies start after what is already queued on c.st (earlier readers of the buffers)
  if (cudaEventRecord(ev[4], c.st) != cudaSuccess || cudaStreamWaitEvent(cs, ev[4], 0) != cudaSuccess)
    r = SORSVD_ERR_CUDA;
  const int64_t nb = (m + SL.rows - 1) / SL.rows;
  for (int64_t b = 0; b < nb && !r; ++b) {
    const int i = (int)(b & 1);
    const int64_t r0 = b * SL.rows, rows = std::min<int64_t>(SL.rows, m - r0);
    void* blk = c.at(SL.blk[i]);
    if (b >= 2 && cudaStreamWaitEvent(cs, ev[2 + i], 0) != cudaSuccess) { r = SORSVD_ERR_CUDA; break; }
    if (cudaMemcpy2DAsync(blk, (size_t)SL.ldb * esz, (const char*)Ah + (size_t)r0 * esz, (size_t)lda * esz,
                          (size_t)rows * esz, (size_t)n, cudaMemcpyHostToDevice, cs) != cudaSuccess ||
        cudaEventRecord(ev[i], cs) != cudaSuccess || cudaStreamWaitEvent(c.st, ev[i], 0) != cudaSuccess) {
      r = SORSVD_ERR_CUDA;
      break;
    }
    r = work(r0, rows, blk, SL.ldb);
    if (!r && cudaEventRecord(ev[2 + i], c.st) != cudaSuccess) r = SORSVD_ERR_CUDA;
  }
  for (cudaEvent_t e : ev) cudaEventDestroy(e);
  return r;
}

// Algorithm 3 with the stabilised power loop (as solve() without method
// flags), every pass over A streamed from host memory.
int solve_streamed(const Ctx& c, const StreamLayout& SL, const void* Ah, int64_t m, int64_t n, int64_t lda, int k,
                   int l, int q, void* U, int64_t ldu, void* S, void* V, int64_t ldv) {
  const Layout& L = c.L;
  const int dtype = c.dt;
  const int adt = c.f64 ? SORSVD_F64 : SORSVD_F32;
  const bool h16 = dtype_is_16(dtype);
  const size_t acc = acc_size(dtype);
  const int kc = dtype == SORSVD_F32 ? K_PASS_SPLIT : K_PASS;
  void* t1op = h16 ? c.at(L.t1op) : c.at(L.t1);
  const void* x2 = c.at(L.t2op);
  int r;
  for (int i = 1; i <= q + 1; ++i) {
    const bool last = (i == q + 1);
    const int np = last ? 3 : 1;
    const int kind = last ? kc : K_PASS;
    // T1 = A X, a block of rows of T1 per block of A
    r = stream_blocks(c, SL, Ah, lda, m, n, [&](int64_t r0, int64_t rows, void* blk, int64_t ldb) -> int {
      int e = prepare_at(c, blk, rows, n, ldb);
      if (e) return e;
      return pass(c, kind, false, rows, l, n, blk, ldb, x2, L.ldn, h16 ? dtype : adt,
                  (char*)c.at(L.t1) + (size_t)r0 * acc, L.ldm, nullptr, 0, last);
    });
    if (r) return r;
    void* q1 = nullptr;
    r = orth(c, c.at(L.t1), m, L.ldm, l, np, first_shift(dtype), h16 ? t1op : nullptr, L.ldm, last ? nullptr : &q1);
    if (r) return r;
    const char* y1 = (const char*)(h16 ? t1op : (q1 ? q1 : c.at(L.t1)));
    const size_t ysz = h16 ? dtype_size(dtype) : acc;
    // T2 = A^T Q1 = sum over the blocks of A_b^T Q1_b
    r = stream_blocks(c, SL, Ah, lda, m, n, [&](int64_t r0, int64_t rows, void* blk, int64_t ldb) -> int {
      void* out = r0 == 0 ? c.at(L.t2) : c.at(SL.t2p);
      int e = pass(c, kind, true, n, l, rows, blk, ldb, y1 + (size_t)r0 * ysz, L.ldm, h16 ? dtype : adt, out, L.ldn,
                   nullptr, 0, last);
      if (e || r0 == 0) return e;
      if (c.f64) LAUNCH(K_MISC, launch_add_f64((const double*)out, L.ldn, (double*)c.at(L.t2), L.ldn, n, l, c.st));
      else LAUNCH(K_MISC, launch_add_f32((const float*)out, L.ldn, (float*)c.at(L.t2), L.ldn, n, l, c.st));
      return SORSVD_OK;
    });
    if (r) return r;
    void* q2 = nullptr;
    r = orth(c, c.at(L.t2), n, L.ldn, l, np, first_shift(dtype), (!last && h16) ? c.at(L.t2op) : nullptr, L.ldn,
             last ? nullptr : &q2);
    if (r) return r;
    x2 = h16 ? c.at(L.t2op) : (q2 ? q2 : c.at(L.t2));
  }
  // core: W = A Q2 a block of rows at a time (in tmp), then M = Q1^T W
  const void* q2op = c.at(L.t2);
  int q2dt = adt;
  if (h16) {
    LAUNCH(K_MISC, launch_convert_f32((const float*)c.at(L.t2), L.ldn, n, l, c.at(L.q2op), L.ldn, dtype, nullptr,
                                      c.st));
    q2op = c.at(L.q2op);
    q2dt = dtype;
  }
  r = stream_blocks(c, SL, Ah, lda, m, n, [&](int64_t r0, int64_t rows, void* blk, int64_t ldb) -> int {
    int e = prepare_at(c, blk, rows, n, ldb);
    if (e) return e;
    return pass(c, K_CORE, false, rows, l, n, blk, ldb, q2op, L.ldn, q2dt, (char*)c.at(L.tmp) + (size_t)r0 * acc,
                L.ldm, nullptr, 0, !h16);
  });
  if (r) return r;
  r = cross_gram(c, c.at(L.t1), L.ldm, c.at(L.tmp), L.ldm, m, l, (double*)c.at(L.M), l);
  if (r) return r;
  LAUNCH(K_JACOBI, launch_jacobi((const double*)c.at(L.M), l, k, c.f64, c.at(L.Ut), c.at(L.Vt), S, c.f64,
                                  c.at(L.jwork), c.status(), c.st));
  r = assemble(c, c.at(L.t1), L.ldm, m, l, c.at(L.Ut), k, U, ldu);
  if (r) return r;
  return assemble(c, c.at(L.t2), L.ldn, n, l, c.at(L.Vt), k, V, ldv);
}

}  // namespace

// the status word is the first region of every workspace layout
DeviceStatus* workspace_status(void* ws) { return reinterpret_cast<DeviceStatus*>(ws); }

}  // namespace sorsvd

using namespace sorsvd;

extern "C" {

size_t sorsvd_workspace_size(int64_t m, int64_t n, int k, int p, int dtype, unsigned flags) {
  if (check_dtype(dtype) || m < 1 || n < 1 || k < 1 || p < 0) return 0;
  int l = k + p;
  if (l > std::min(m, n) || l > max_l(dtype)) return 0;
  const size_t base = make_layout(m, n, l, dtype, flags).total;
  return (flags & SORSVD_FLAG_HOST_IO) ? host_io_layout(base, m, n, k, dtype).total : base;
}

const char* sorsvd_status_string(int s) {
  switch (s) {
    case SORSVD_OK: return "ok";
    case SORSVD_ERR_ARG: return "invalid argument";
    case SORSVD_ERR_DTYPE: return "unknown dtype";
    case SORSVD_ERR_CUDA: return "CUDA runtime error";
    case SORSVD_ERR_NOT_CONVERGED: return "Jacobi SVD did not converge";
    case SORSVD_ERR_BREAKDOWN: return "Cholesky breakdown after shifted retries";
    case SORSVD_ERR_TIMEOUT: return "bounded wait timed out";
    case SORSVD_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case SORSVD_ERR_UNSUPPORTED: return "size beyond a documented limit";
    default: return "unknown status";
  }
}

int sorsvd_set_limits(long long wait_cycles, int max_sweeps) {
  set_tc_wait_cycles(wait_cycles);
  return set_jacobi_sweep_cap(max_sweeps) == cudaSuccess ? SORSVD_OK : SORSVD_ERR_CUDA;
}

int sorsvd_get_status(const void* workspace, int* device_status, int* info, void* stream) {
  if (!workspace) return SORSVD_ERR_WORKSPACE;
  DeviceStatus h{};
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&h, workspace, sizeof(h), cudaMemcpyDeviceToHost, st) != cudaSuccess) return SORSVD_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return SORSVD_ERR_CUDA;
  if (device_status) *device_status = h.code;
  if (info) *info = h.info;
  return SORSVD_OK;
}

int sorsvd_gaussian(void* out, int64_t rows, int64_t cols, int64_t ld, uint64_t seed, uint64_t stream_id,
                    int dtype, void* stream) {
  if (check_dtype(dtype)) return SORSVD_ERR_DTYPE;
  if (!out || rows < 0 || cols < 0 || ld < rows || ld < 1) return SORSVD_ERR_ARG;
  ProfScope ps(K_GAUSSIAN, (cudaStream_t)stream);
  if (launch_gaussian(out, rows, cols, ld, seed, stream_id, dtype, (cudaStream_t)stream) != cudaSuccess)
    return SORSVD_ERR_CUDA;
  return SORSVD_OK;
}

int sorsvd_chol_inv(const double* G, int l, double shift_rel, int dtype, void* Rinv, void* status, void* stream) {
  if (check_dtype(dtype)) return SORSVD_ERR_DTYPE;
  if (!G || !Rinv || !status || l < 1 || !(shift_rel >= 0.0)) return SORSVD_ERR_ARG;
  if (l > max_l(dtype)) return SORSVD_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(status, 0, sizeof(DeviceStatus), st));
  ProfScope ps(K_CHOL, st);
  CK(launch_chol_inv(G, l, shift_rel, Rinv, dtype == SORSVD_F64, (DeviceStatus*)status, st));
  return SORSVD_OK;
}

int sorsvd_polar_inv(const double* G, int l, float* X, int* ok, void* scratch, size_t scratch_bytes,
                     void* stream) {
  if (!G || !X || !ok || !scratch || l < 1) return SORSVD_ERR_ARG;
  if (l > SORSVD_MAX_L) return SORSVD_ERR_UNSUPPORTED;
  if (scratch_bytes < polar_scratch_bytes(l) || ((uintptr_t)scratch) % 16) return SORSVD_ERR_WORKSPACE;
  cudaStream_t st = (cudaStream_t)stream;
  ProfScope ps(K_CHOL, st);
  CK(launch_polar_inv(G, l, X, (float*)scratch, ok, nullptr, 0.f, st));
  return SORSVD_OK;
}

// workspace of sorsvd_gram / sorsvd_apply: the status word, the Gram
// partials (tensor-core or row-block form, whichever is larger) and the
// TF32 hi / lo parts of the small factor
static Layout products_layout(int64_t rows, int l) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  L.status = take(sizeof(DeviceStatus));
  size_t pb = std::max(rb_gram_parts_bytes(rows, l, l, true), rb_gram_parts_bytes(rows, l, l, false));
  if (l <= kTskMaxL)
    pb = std::max({pb, (size_t)tsk_gram_parts(rows) * l * l * sizeof(float),
                   (size_t)tsk_xty_parts(rows, l) * l * l * sizeof(float)});
  L.parts = take(pb);
  L.ldk = (l + 31) / 32 * 32;
  L.bsplit = take((size_t)2 * L.ldk * L.ldk * sizeof(float));
  L.total = off;
  return L;
}

size_t sorsvd_streamed_workspace_size(int64_t m, int64_t n, int k, int p, int dtype, int64_t block_rows) {
  if (check_dtype(dtype) || m < 1 || n < 1 || k < 1 || p < 0 || block_rows < 1) return 0;
  const int l = k + p;
  if (l > std::min(m, n) || l > max_l(dtype)) return 0;
  return stream_layout(m, n, l, dtype, block_rows).total;
}

int sorsvd_run_streamed(const void* A, int64_t m, int64_t n, int64_t lda, int k, int p, int q, uint64_t seed,
                        int dtype, int64_t block_rows, void* U, int64_t ldu, void* S, void* V, int64_t ldv,
                        void* workspace, size_t ws_bytes, void* stream) {
  if (check_dtype(dtype)) return SORSVD_ERR_DTYPE;
  if (!A || !U || !S || !V) return SORSVD_ERR_ARG;
  if (m < 1 || n < 1 || k < 1 || p < 0 || q < 0 || q > 1000 || lda < m || ldu < m || ldv < n || block_rows < 1)
    return SORSVD_ERR_ARG;
  const int l = k + p;
  if (l > std::min(m, n)) return SORSVD_ERR_ARG;
  if (l > max_l(dtype)) return SORSVD_ERR_UNSUPPORTED;
  const StreamLayout SL = stream_layout(m, n, l, dtype, block_rows);
  if (!workspace || ((uintptr_t)workspace) % kAlign || ws_bytes < SL.total) return SORSVD_ERR_WORKSPACE;
  Ctx c{(char*)workspace, SL.L, dtype, dtype == SORSVD_F64, (cudaStream_t)stream};
  CK(begin_call(c));
  LAUNCH(K_GAUSSIAN, launch_gaussian(c.at(SL.L.t2op), n, l, SL.L.ldn, seed, 0, dtype, c.st));
  return solve_streamed(c, SL, A, m, n, lda, k, l, q, U, ldu, S, V, ldv);
}

size_t sorsvd_products_workspace_size(int64_t rows, int l) {
  if (rows < 1 || l < 1 || l > SORSVD_MAX_L) return 0;
  return products_layout(rows, l).total;
}

int sorsvd_gram(const float* X, int64_t ldx, const float* Y, int64_t ldy, int64_t rows, int l, double* G,
                int64_t ldg, void* workspace, size_t ws_bytes, void* stream) {
  if (!X || !G || rows < 1 || l < 1 || ldx < rows || ldg < l || ldg > INT32_MAX) return SORSVD_ERR_ARG;
  if (Y && ldy < rows) return SORSVD_ERR_ARG;
  if (l > SORSVD_MAX_L) return SORSVD_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (ldx & 3)) return SORSVD_ERR_ARG;
  if (Y && ((reinterpret_cast<uintptr_t>(Y) & 15) || (ldy & 3))) return SORSVD_ERR_ARG;
  const Layout L = products_layout(rows, l);
  if (int r = check_ws(workspace, ws_bytes, L)) return r;
  Ctx c{(char*)workspace, L, SORSVD_F32, false, (cudaStream_t)stream};
  CK(cudaMemsetAsync(c.status(), 0, sizeof(DeviceStatus), c.st));
  if (Y) return cross_gram(c, X, ldx, Y, ldy, rows, l, G, ldg);
  return gram_sym(c, X, ldx, rows, l, nullptr, G, ldg);
}

int sorsvd_apply(const float* X, int64_t rows, int K, int64_t ldx, const float* B, int64_t ldb, int N, int upper_tri,
                 float* Y, int64_t ldy, void* workspace, size_t ws_bytes, void* stream) {
  if (!X || !B || !Y || rows < 1 || K < 1 || N < 1 || ldx < rows || ldb < K || ldy < rows) return SORSVD_ERR_ARG;
  if (K > SORSVD_MAX_L || N > SORSVD_MAX_L) return SORSVD_ERR_UNSUPPORTED;
  if ((reinterpret_cast<uintptr_t>(X) & 15) || (ldx & 3)) return SORSVD_ERR_ARG;
  const Layout L = products_layout(rows, std::max(K, N));
  if (int r = check_ws(workspace, ws_bytes, L)) return r;
  Ctx c{(char*)workspace, L, SORSVD_F32, false, (cudaStream_t)stream};
  CK(cudaMemsetAsync(c.status(), 0, sizeof(DeviceStatus), c.st));
  return apply(c, X, ldx, rows, K, B, ldb, N, upper_tri != 0, Y, ldy, nullptr, 0, 0, nullptr);
}

int sorsvd_power_pass(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, const void* X, int64_t ldx,
                      int l, void* T1, int64_t ldt1, void* T2, int64_t ldt2, void* workspace, size_t ws_bytes,
                      void* stream) {
  if (check_dtype(dtype)) return SORSVD_ERR_DTYPE;
  if (!A || !X || !T1 || !T2 || m < 1 || n < 1 || l < 1 || lda < m || ldx < n || ldt1 < m || ldt2 < n)
    return SORSVD_ERR_ARG;
  if (l > std::min(m, n) || l > max_l(dtype)) return SORSVD_ERR_UNSUPPORTED;
  Layout L = make_layout(m, n, l, dtype);
  if (int r = check_ws(workspace, ws_bytes, L)) return r;
  Ctx c{(char*)workspace, L, dtype, dtype == SORSVD_F64, (cudaStream_t)stream};
  CK(begin_call(c));
  if (int r = prepare_at(c, A, m, n, lda)) return r;
  const void* xop = X;
  int64_t ldop = ldx;
  if (dtype_is_16(dtype)) {
    LAUNCH(K_MISC, launch_convert_f32((const float*)X, ldx, n, l, c.at(L.t2op), L.ldn, dtype, nullptr, c.st));
    xop = c.at(L.t2op);
    ldop = L.ldn;
  }
  return power_pass_impl(c, A, m, n, lda, xop, ldop, l, T1, ldt1, T2, ldt2, true);
}

int sorsvd_core(const void* A, int64_t m, int64_t n, int64_t lda, int dtype, unsigned flags, const void* Q1,
                int64_t ldq1, const void* Q2, int64_t ldq2, int l, double* M, int64_t ldm, void* workspace,
                size_t ws_bytes, void* stream) {
  if (check_dtype(dtype)) return SORSVD_ERR_DTYPE;
  if (!A || !Q1 || !Q2 || !M || m < 1 || n < 1 || l < 1 || lda < m || ldq1 < m || ldq2 < n || ldm < l)
    return SORSVD_ERR_ARG;
  if (flags & ~(SORSVD_FLAG_LITERAL_POWER | SORSVD_FLAG_REFINE)) return SORSVD_ERR_ARG;
  if (l > std::min(m, n) || l > max_l(dtype)) return SORSVD_ERR_UNSUPPORTED;
  Layout L = make_layout(m, n, l, dtype);
  if (int r = check_ws(workspace, ws_bytes, L)) return r;
  Ctx c{(char*)workspace, L, dtype, dtype == SORSVD_F64, (cudaStream_t)stream};
  CK(begin_call(c));
  if (int r = prepare_at(c, A, m, n, lda)) return r;
  return core_impl(c, A, m, n, lda, flags, Q1, ldq1, Q2, ldq2, l, M, ldm);
}

int sorsvd_run(const void* A, int64_t m, int64_t n, int64_t lda, int k, int p, int q, uint64_t seed, int dtype,
               unsigned flags, void* U, int64_t ldu, void* S, void* V, int64_t ldv, void* workspace,
               size_t ws_bytes, void* stream) {
  if (check_dtype(dtype)) return SORSVD_ERR_DTYPE;
  if (!A || !U || !S || !V) return SORSVD_ERR_ARG;
  if (m < 1 || n < 1 || k < 1 || p < 0 || q < 0 || q > 1000 || lda < m || ldu < m || ldv < n)
    return SORSVD_ERR_ARG;
  if (flags & ~(SORSVD_FLAG_LITERAL_POWER | SORSVD_FLAG_REFINE | SORSVD_FLAG_TWO_PASS | SORSVD_FLAG_RSVD |
                SORSVD_FLAG_TSR))
    return SORSVD_ERR_ARG;
  if (!method_flags_ok(flags, q)) return SORSVD_ERR_ARG;
  const int l = k + p;
  if (l > std::min(m, n)) return SORSVD_ERR_ARG;
  if (l > max_l(dtype)) return SORSVD_ERR_UNSUPPORTED;
  Layout L = make_layout(m, n, l, dtype, flags);
  if (int r = check_ws(workspace, ws_bytes, L)) return r;
  Ctx c{(char*)workspace, L, dtype, dtype == SORSVD_F64, (cudaStream_t)stream};
  int r;

  CK(begin_call(c));
  if (L.has_at && tc_enabled()) {
    // the transposed copy of A (memory-bound) and Omega (binary64 ALU-bound)
    // are independent: Omega is drawn on a side stream meanwhile
    r = gaussian_beside(c, c.at(L.t2op), n, l, L.ldn, seed, dtype, [&] { return prepare_at(c, A, m, n, lda); });
    if (r) return r;
  } else {
    r = prepare_at(c, A, m, n, lda);
    if (r) return r;
    LAUNCH(K_GAUSSIAN, launch_gaussian(c.at(L.t2op), n, l, L.ldn, seed, 0, dtype, c.st));
  }
  return solve(c, A, m, n, lda, k, l, q, flags, seed, U, ldu, S, V, ldv);
}

int sorsvd_run_host(const void* A, int64_t m, int64_t n, int64_t lda, int k, int p, int q, uint64_t seed, int dtype,
                    unsigned flags, void* U, int64_t ldu, void* S, void* V, int64_t ldv, void* workspace,
                    size_t ws_bytes, void* stream) {
  if (check_dtype(dtype)) return SORSVD_ERR_DTYPE;
  if (!A || !U || !S || !V) return SORSVD_ERR_ARG;
  if (m < 1 || n < 1 || k < 1 || p < 0 || q < 0 || q > 1000 || lda < m || ldu < m || ldv < n)
    return SORSVD_ERR_ARG;
  if (flags & ~(SORSVD_FLAG_LITERAL_POWER | SORSVD_FLAG_REFINE | SORSVD_FLAG_HOST_IO | SORSVD_FLAG_TWO_PASS |
                SORSVD_FLAG_RSVD | SORSVD_FLAG_TSR))
    return SORSVD_ERR_ARG;
  if (!method_flags_ok(flags, q)) return SORSVD_ERR_ARG;
  const int l = k + p;
  if (l > std::min(m, n)) return SORSVD_ERR_ARG;
  if (l > max_l(dtype)) return SORSVD_ERR_UNSUPPORTED;
  Layout L = make_layout(m, n, l, dtype, flags & ~SORSVD_FLAG_HOST_IO);
  const HostIo H = host_io_layout(L.total, m, n, k, dtype);
  if (!workspace || ((uintptr_t)workspace) % kAlign || ws_bytes < H.total) return SORSVD_ERR_WORKSPACE;
  Ctx c{(char*)workspace, L, dtype, dtype == SORSVD_F64, (cudaStream_t)stream};
  void* Ad = c.at(H.a);
  void* Ud = c.at(H.u);
  void* Sd = c.at(H.s);
  void* Vd = c.at(H.v);
  int r;

  CK(begin_call(c));
  // Omega (no dependence on A) on the side stream while A crosses
  r = gaussian_beside(c, c.at(L.t2op), n, l, L.ldn, seed, dtype,
                      [&] { return upload_a(c, A, lda, m, n, Ad, H.lda); });
  if (r) return r;
  r = solve(c, Ad, m, n, H.lda, k, l, q, flags & ~SORSVD_FLAG_HOST_IO, seed, Ud, H.ldu, Sd, Vd, H.ldv);
  if (r) return r;
  const size_t acc = acc_size(dtype);
  CK(cudaMemcpy2DAsync(U, (size_t)ldu * acc, Ud, (size_t)H.ldu * acc, (size_t)m * acc, (size_t)k,
                       cudaMemcpyDeviceToHost, c.st));
  CK(cudaMemcpyAsync(S, Sd, (size_t)k * acc, cudaMemcpyDeviceToHost, c.st));
  CK(cudaMemcpy2DAsync(V, (size_t)ldv * acc, Vd, (size_t)H.ldv * acc, (size_t)n * acc, (size_t)k,
                       cudaMemcpyDeviceToHost, c.st));
  return SORSVD_OK;
}

}  // extern "C"
