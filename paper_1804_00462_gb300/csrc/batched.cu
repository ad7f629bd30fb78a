// Batched SOR-SVD: many independent problems of uneven m, n, k (and q) run
// as one sequence of grouped launches.  Each launch performs one stage of
// Algorithm 3 for every problem that has that stage, reading per-problem job
// descriptors from device memory (grouped GEMM units, one-block-per-problem
// Cholesky and Jacobi), so the whole batch takes a few dozen launches
// regardless of the batch size.  A plan uploads the descriptors once and
// captures the launches in a CUDA graph; replaying the graph runs the batch.
//
// Stages (problem b: l_b = k_b + p_b, q_b power passes):
//   Omega_b -> T2_b
//   i = 1 .. max q_b + 1 (problems with i <= q_b + 1):
//     T1_b = A_b T2_b ;  T1_b <- orth(T1_b)
//     T2_b = A_b^T T1_b ;  T2_b <- orth(T2_b)
//   with one shifted CholeskyQR pass inside the loop and CholeskyQR3 in the
//   problem's last iteration (giving Q1_b, Q2_b); with
//   SORSVD_FLAG_LITERAL_POWER the loop runs without orth and both sketches
//   get CholeskyQR3 (in the same launches) at the end
//   W_b = A_b Q2_b ;  M_b = Q1_b^T W_b
//   M_b = U~ S~ V~^T (one-sided Jacobi), keep k_b
//   U_b = Q1_b U~_k, V_b = Q2_b V~_k
// CholeskyQR: G = T^T T (split-K partials summed in binary64), R^{-1} from
// the blocked Cholesky, T <- T R^{-1} into the other half of a ping-pong
// pair (no copies).
#include "internal.cuh"
#include "profile.cuh"

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <utility>
#include <vector>

enum StageKind { ST_GAUSS, ST_GEMM_N, ST_GEMM_T, ST_REDUCE, ST_CHOL, ST_JACOBI };

struct BatchStage {
  StageKind kind;
  size_t jobs_off;       // byte offset of the job array in the header's job area
  int njobs;
  // gemm: one int4 unit list per tile shape (byte offset, count), and the
  // shape the autotuner picked
  size_t units_off[sorsvd::kBatchedTiles];
  int nunits[sorsvd::kBatchedTiles];
  int tile;
  double work;           // gemm: sum of 2 M N K over the jobs (the autotuner's key)
  int max_n;
  int64_t max_elems;     // gauss / reduce: largest element count of a job
  int max_l;             // chol / jacobi
};

struct sorsvd_batch_plan {
  int batch = 0;
  int dtype = 0;
  char* ws = nullptr;
  size_t hdr_bytes = 0;
  sorsvd::DeviceStatus* status = nullptr;      // batch entries, contiguous
  std::vector<BatchStage> stages;
  int launches = 0;                            // kernels per run
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace sorsvd {
namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }
inline int64_t pad16(int64_t x) { return (x + 15) / 16 * 16; }
// relative shift of the first CholeskyQR pass (the same values as the
// single-problem driver)
inline double first_shift(int dt) { return dt == SORSVD_F64 ? 1e-13 : 1e-5; }
// K splits of the l x l products (Gram, Q1^T W): about 256 rows per split
inline int splits_of(int64_t K) { return (int)std::max<int64_t>(1, std::min<int64_t>((K + 255) / 256, 64)); }

int max_l_batched(bool f64) { return std::min(chol_batched_max_l(f64), jacobi_batched_max_l(f64)); }

// per-problem workspace layout
struct PLayout {
  int64_t ldm, ldn;
  int l, s;
  size_t t1a, t1b, t2a, t2b, w, M, Ut, Vt, jwork, total;
  size_t parts[2], G[2], Rinv[2];   // one CholeskyQR set per sketch (T1, T2)
};

PLayout playout(const sorsvd_problem& P, size_t acc) {
  PLayout L{};
  L.l = P.k + P.p;
  L.ldm = pad16(P.m);
  L.ldn = pad16(P.n);
  L.s = splits_of(std::max(P.m, P.n));
  size_t off = 0;
  auto take = [&](size_t bytes) { size_t o = off; off = align_up(off + bytes); return o; };
  L.t1a = take((size_t)L.ldm * L.l * acc);
  L.t1b = take((size_t)L.ldm * L.l * acc);
  L.t2a = take((size_t)L.ldn * L.l * acc);
  L.t2b = take((size_t)L.ldn * L.l * acc);
  L.w = take((size_t)L.ldm * L.l * acc);
  for (int i = 0; i < 2; ++i) {
    L.parts[i] = take((size_t)L.s * L.l * L.l * acc);
    L.G[i] = take((size_t)L.l * L.l * 8);
    L.Rinv[i] = take((size_t)L.l * L.l * acc);
  }
  L.M = take((size_t)L.l * L.l * 8);
  L.Ut = take((size_t)L.l * L.l * acc);
  L.Vt = take((size_t)L.l * L.l * acc);
  L.jwork = take(jacobi_batched_work_bytes(L.l));
  L.total = off;
  return L;
}

int check_problem(const sorsvd_problem& P, int dt) {
  if (!P.A || !P.U || !P.S || !P.V) return SORSVD_ERR_ARG;
  if (P.m < 1 || P.n < 1 || P.k < 1 || P.p < 0 || P.q < 0 || P.q > 1000) return SORSVD_ERR_ARG;
  if (P.lda < P.m || P.ldu < P.m || P.ldv < P.n) return SORSVD_ERR_ARG;
  const int l = P.k + P.p;
  if (l > std::min(P.m, P.n)) return SORSVD_ERR_ARG;
  if (l > max_l_batched(dt == SORSVD_F64)) return SORSVD_ERR_UNSUPPORTED;
  return SORSVD_OK;
}

inline bool batched_dtype(int dt) { return dt == SORSVD_F64 || dt == SORSVD_F32 || dt == SORSVD_TF32; }

// Host-side assembly of job / unit arrays: everything goes into one byte
// buffer that is copied to the workspace header once.
struct Builder {
  std::vector<char> buf;
  std::vector<BatchStage> stages;
  template <typename T>
  size_t put(const std::vector<T>& v) {
    size_t off = align_up(buf.size());
    buf.resize(off + v.size() * sizeof(T));
    if (!v.empty()) std::memcpy(buf.data() + off, v.data(), v.size() * sizeof(T));
    return off;
  }
  void gemm(bool trans, const std::vector<GemmJob>& jobs) {
    if (jobs.empty()) return;
    BatchStage s{};
    s.kind = trans ? ST_GEMM_T : ST_GEMM_N;
    s.jobs_off = put(jobs);
    s.njobs = (int)jobs.size();
    for (const GemmJob& g : jobs) {
      s.work += 2.0 * (double)g.M * (double)g.N * (double)g.K;
      s.max_n = std::max(s.max_n, (int)g.N);
    }
    for (int tile = 0; tile < kBatchedTiles; ++tile) {
      int bm, bn, bk;
      gemm_tile_shape(tile, &bm, &bn, &bk);
      std::vector<int4> units;
      for (size_t j = 0; j < jobs.size(); ++j) {
        const GemmJob& g = jobs[j];
        const int mt = (int)((g.M + bm - 1) / bm), nt = (int)((g.N + bn - 1) / bn);
        const int ks = (int)((g.K + g.k_chunk - 1) / g.k_chunk);
        for (int z = 0; z < ks; ++z)
          for (int y = 0; y < nt; ++y)
            for (int x = 0; x < mt; ++x) units.push_back(make_int4((int)j, x, y, z));
      }
      s.units_off[tile] = put(units);
      s.nunits[tile] = (int)units.size();
    }
    s.tile = 0;
    stages.push_back(s);
  }
  void reduce(const std::vector<ReduceJob>& jobs) {
    if (jobs.empty()) return;
    BatchStage s{};
    s.kind = ST_REDUCE;
    s.jobs_off = put(jobs);
    s.njobs = (int)jobs.size();
    for (const ReduceJob& r : jobs) s.max_elems = std::max(s.max_elems, r.rows * r.cols);
    stages.push_back(s);
  }
  template <typename J>
  void simple(StageKind kind, const std::vector<J>& jobs, int64_t max_elems, int max_l) {
    if (jobs.empty()) return;
    BatchStage s{};
    s.kind = kind;
    s.jobs_off = put(jobs);
    s.njobs = (int)jobs.size();
    s.max_elems = max_elems;
    s.max_l = max_l;
    stages.push_back(s);
  }
};

// one GEMM job with full K (no split)
GemmJob gjob(const void* A, int64_t lda, const void* B, int64_t ldb, void* C, int64_t ldc, int64_t M, int64_t N,
             int64_t K) {
  GemmJob g{};
  g.A = A; g.B = B; g.C = C;
  g.lda = lda; g.ldb = ldb; g.ldc = ldc;
  g.M = M; g.N = N; g.K = K;
  int bm, bn, bk;
  gemm_tile_shape(0, &bm, &bn, &bk);
  g.k_chunk = std::max<int64_t>(bk, (K + bk - 1) / bk * bk);
  g.split_stride = 0;
  return g;
}

struct ProbState {
  PLayout L;
  char* base;
  bool t1_in_a, t2_in_a;      // which half of each ping-pong pair holds the sketch
  char* t1() const { return base + (t1_in_a ? L.t1a : L.t1b); }
  char* t1o() const { return base + (t1_in_a ? L.t1b : L.t1a); }
  char* t2() const { return base + (t2_in_a ? L.t2a : L.t2b); }
  char* t2o() const { return base + (t2_in_a ? L.t2b : L.t2a); }
};

// One CholeskyQR pass over a list of sketches (problem, which: 1 = T1,
// 2 = T2), all in the same four launches: Gram -> reduce -> Cholesky
// inverse -> T R^{-1} (into the other half of the sketch's pair)
void orth_pass(Builder& B, std::vector<ProbState>& ps, const std::vector<std::pair<int, int>>& items, double shift,
               DeviceStatus* status, const sorsvd_problem* probs) {
  std::vector<GemmJob> gram;
  std::vector<ReduceJob> red;
  std::vector<CholJob> ch;
  std::vector<GemmJob> apply;
  int max_l = 1;
  int bm, bn, bk;
  gemm_tile_shape(0, &bm, &bn, &bk);
  for (const auto& it : items) {
    const int b = it.first, which = it.second, set = which - 1;
    ProbState& s = ps[b];
    const int64_t rows = which == 1 ? probs[b].m : probs[b].n;
    const int64_t ld = which == 1 ? s.L.ldm : s.L.ldn;
    char* T = which == 1 ? s.t1() : s.t2();
    char* To = which == 1 ? s.t1o() : s.t2o();
    const int l = s.L.l;
    const int sp = splits_of(rows);
    GemmJob g = gjob(T, ld, T, ld, s.base + s.L.parts[set], l, l, l, rows);
    g.k_chunk = std::max<int64_t>(bk, ((rows + sp - 1) / sp + bk - 1) / bk * bk);
    g.split_stride = (int64_t)l * l;
    gram.push_back(g);
    ReduceJob r{};
    r.parts = s.base + s.L.parts[set];
    r.out = s.base + s.L.G[set];
    r.rows = l; r.cols = l; r.ldp = l; r.ldo = l;
    r.stride = (int64_t)l * l;
    r.splits = (int)((rows + g.k_chunk - 1) / g.k_chunk);
    r.out_f64 = 1;
    red.push_back(r);
    CholJob c{};
    c.G = (const double*)(s.base + s.L.G[set]);
    c.Rinv = s.base + s.L.Rinv[set];
    c.status = status + b;
    c.l = l;
    c.shift = shift;
    ch.push_back(c);
    apply.push_back(gjob(T, ld, s.base + s.L.Rinv[set], l, To, ld, rows, l, l));
    max_l = std::max(max_l, l);
    if (which == 1) s.t1_in_a = !s.t1_in_a;
    else s.t2_in_a = !s.t2_in_a;
  }
  B.gemm(true, gram);
  B.reduce(red);
  B.simple(ST_CHOL, ch, 0, max_l);
  B.gemm(false, apply);
}

int build_plan(sorsvd_batch_plan* plan, const sorsvd_problem* probs, int batch, int dt, unsigned flags,
               Builder& B, std::vector<ProbState>& ps, size_t hdr_reserve) {
  const bool f64 = dt == SORSVD_F64;
  const size_t acc = f64 ? 8 : 4;
  char* ws = plan->ws;
  DeviceStatus* status = plan->status;
  // per-problem regions after the header
  size_t off = hdr_reserve;
  ps.resize(batch);
  int qmax = 0, max_l = 1;
  for (int b = 0; b < batch; ++b) {
    ps[b].L = playout(probs[b], acc);
    ps[b].base = ws + off;
    ps[b].t1_in_a = true;
    ps[b].t2_in_a = true;
    off += align_up(ps[b].L.total);
    qmax = std::max(qmax, probs[b].q);
    max_l = std::max(max_l, ps[b].L.l);
  }
  // Omega
  {
    std::vector<GaussJob> g;
    int64_t mx = 0;
    for (int b = 0; b < batch; ++b) {
      GaussJob j{};
      j.out = ps[b].t2();
      j.rows = probs[b].n; j.cols = ps[b].L.l; j.ld = ps[b].L.ldn; j.seed = probs[b].seed;
      g.push_back(j);
      mx = std::max(mx, j.rows * j.cols);
    }
    B.simple(ST_GAUSS, g, mx, 0);
  }
  // CholeskyQR passes (pass index < passes[b]) over sketch `which` of `sel`
  auto orth_n = [&](const std::vector<int>& sel, int which, const std::vector<int>& passes) {
    int mx = 0;
    for (int b : sel) mx = std::max(mx, passes[b]);
    for (int pass = 0; pass < mx; ++pass) {
      std::vector<std::pair<int, int>> items;
      for (int b : sel)
        if (pass < passes[b]) items.push_back({b, which});
      orth_pass(B, ps, items, pass == 0 ? first_shift(dt) : 0.0, status, probs);
    }
  };
  auto products = [&](const std::vector<int>& sel, bool trans) {
    std::vector<GemmJob> jobs;
    for (int b : sel) {
      ProbState& s = ps[b];
      const sorsvd_problem& P = probs[b];
      if (!trans) jobs.push_back(gjob(P.A, P.lda, s.t2(), s.L.ldn, s.t1(), s.L.ldm, P.m, s.L.l, P.n));
      else jobs.push_back(gjob(P.A, P.lda, s.t1(), s.L.ldm, s.t2(), s.L.ldn, P.n, s.L.l, P.m));
    }
    B.gemm(trans, jobs);
  };
  if (flags & SORSVD_FLAG_LITERAL_POWER) {
    // Algorithm 3 as printed, then CholeskyQR3 of both sketches
    for (int i = 1; i <= qmax + 1; ++i) {
      std::vector<int> sel;
      for (int b = 0; b < batch; ++b)
        if (i <= probs[b].q + 1) sel.push_back(b);
      products(sel, false);
      products(sel, true);
    }
    for (int pass = 0; pass < 3; ++pass) {
      std::vector<std::pair<int, int>> both;
      for (int b = 0; b < batch; ++b) {
        both.push_back({b, 1});
        both.push_back({b, 2});
      }
      orth_pass(B, ps, both, pass == 0 ? first_shift(dt) : 0.0, status, probs);
    }
  } else {
    // each sketch orthonormalised as soon as it is formed (Lemma 1: ranges
    // unchanged), one pass inside the loop, CholeskyQR3 in a problem's last
    // iteration
    for (int i = 1; i <= qmax + 1; ++i) {
      std::vector<int> sel;
      std::vector<int> passes(batch, 0);
      for (int b = 0; b < batch; ++b)
        if (i <= probs[b].q + 1) {
          sel.push_back(b);
          passes[b] = (i == probs[b].q + 1) ? 3 : 1;
        }
      products(sel, false);
      orth_n(sel, 1, passes);
      products(sel, true);
      orth_n(sel, 2, passes);
    }
  }
  // core: W = A Q2, M = Q1^T W
  {
    std::vector<GemmJob> w, mm;
    std::vector<ReduceJob> red;
    int bm, bn, bk;
    gemm_tile_shape(0, &bm, &bn, &bk);
    for (int b = 0; b < batch; ++b) {
      ProbState& s = ps[b];
      const sorsvd_problem& P = probs[b];
      const int l = s.L.l;
      w.push_back(gjob(P.A, P.lda, s.t2(), s.L.ldn, s.base + s.L.w, s.L.ldm, P.m, l, P.n));
      const int sp = splits_of(P.m);
      GemmJob g = gjob(s.t1(), s.L.ldm, s.base + s.L.w, s.L.ldm, s.base + s.L.parts[0], l, l, l, P.m);
      g.k_chunk = std::max<int64_t>(bk, ((P.m + sp - 1) / sp + bk - 1) / bk * bk);
      g.split_stride = (int64_t)l * l;
      mm.push_back(g);
      ReduceJob r{};
      r.parts = s.base + s.L.parts[0];
      r.out = s.base + s.L.M;
      r.rows = l; r.cols = l; r.ldp = l; r.ldo = l;
      r.stride = (int64_t)l * l;
      r.splits = (int)((P.m + g.k_chunk - 1) / g.k_chunk);
      r.out_f64 = 1;
      red.push_back(r);
    }
    B.gemm(false, w);
    B.gemm(true, mm);
    B.reduce(red);
  }
  // l x l SVD
  {
    std::vector<JacobiJob> jj;
    for (int b = 0; b < batch; ++b) {
      ProbState& s = ps[b];
      JacobiJob j{};
      j.M = (const double*)(s.base + s.L.M);
      j.Ut = s.base + s.L.Ut;
      j.Vt = s.base + s.L.Vt;
      j.S = probs[b].S;
      j.work = s.base + s.L.jwork;
      j.status = status + b;
      j.l = s.L.l;
      j.k = probs[b].k;
      jj.push_back(j);
    }
    B.simple(ST_JACOBI, jj, 0, max_l);
  }
  // U = Q1 U~_k, V = Q2 V~_k
  {
    std::vector<GemmJob> out;
    for (int b = 0; b < batch; ++b) {
      ProbState& s = ps[b];
      const sorsvd_problem& P = probs[b];
      const int l = s.L.l;
      out.push_back(gjob(s.t1(), s.L.ldm, s.base + s.L.Ut, l, P.U, P.ldu, P.m, P.k, l));
      out.push_back(gjob(s.t2(), s.L.ldn, s.base + s.L.Vt, l, P.V, P.ldv, P.n, P.k, l));
    }
    B.gemm(false, out);
  }
  return SORSVD_OK;
}

// the header holds the status words and the job / unit arrays; its size is
// known only after the build, so the build runs twice (size, then place)
size_t header_size(size_t jobs_bytes, int batch) {
  return align_up(sizeof(DeviceStatus) * (size_t)batch) + align_up(jobs_bytes);
}

int enqueue(const sorsvd_batch_plan* plan, cudaStream_t st, bool count) {
  const bool f64 = plan->dtype == SORSVD_F64;
  char* hdr = plan->ws + align_up(sizeof(DeviceStatus) * (size_t)plan->batch);
  if (cudaMemsetAsync(plan->status, 0, sizeof(DeviceStatus) * (size_t)plan->batch, st) != cudaSuccess)
    return SORSVD_ERR_CUDA;
  for (const BatchStage& s : plan->stages) {
    cudaError_t e = cudaSuccess;
    switch (s.kind) {
      case ST_GAUSS:
        e = launch_gaussian_batched((const GaussJob*)(hdr + s.jobs_off), s.njobs, s.max_elems, plan->dtype, st);
        break;
      case ST_GEMM_N:
      case ST_GEMM_T:
        e = launch_gemm_batched(s.kind == ST_GEMM_T, f64, s.tile, (const GemmJob*)(hdr + s.jobs_off),
                                (const int4*)(hdr + s.units_off[s.tile]), s.nunits[s.tile], st);
        break;
      case ST_REDUCE:
        e = launch_reduce_batched(f64, (const ReduceJob*)(hdr + s.jobs_off), s.njobs, s.max_elems, st);
        break;
      case ST_CHOL:
        e = launch_chol_batched((const CholJob*)(hdr + s.jobs_off), s.njobs, s.max_l, f64, st);
        break;
      case ST_JACOBI:
        e = launch_jacobi_batched((const JacobiJob*)(hdr + s.jobs_off), s.njobs, s.max_l, f64, st);
        break;
    }
    if (e != cudaSuccess) return SORSVD_ERR_CUDA;
  }
  if (count) count_launches(plan->launches);
  return SORSVD_OK;
}

// ------------------------------------------------------------ autotuner
// The tile shape of every grouped GEMM stage is picked by timing: each
// shape's launch of the stage, on the plan's own jobs and workspace (the
// plan's first run overwrites whatever the trials wrote), is timed with
// CUDA events (one untimed launch, then kTuneReps) and the fastest is kept.
// The choice is cached per (kind, precision, job count, work to a quarter
// octave, widest output), so plans of the same shape reuse it.  The per-
// element K order of the grouped kernel does not depend on the shape, so
// the results are the same bit for bit whatever the choice.
// SORSVD_FLAG_FIXED_TILES keeps the 128 x 64 shape.
constexpr int kTuneReps = 3;

struct TuneKey {
  int kind, f64, njobs, work_q, max_n;
  bool operator<(const TuneKey& o) const {
    return std::tie(kind, f64, njobs, work_q, max_n) < std::tie(o.kind, o.f64, o.njobs, o.work_q, o.max_n);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, int> g_tune_cache;

int autotune(sorsvd_batch_plan* plan, cudaStream_t st) {
  const bool f64 = plan->dtype == SORSVD_F64;
  char* hdr = plan->ws + align_up(sizeof(DeviceStatus) * (size_t)plan->batch);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return SORSVD_ERR_CUDA;
  }
  int r = SORSVD_OK;
  for (BatchStage& s : plan->stages) {
    if (s.kind != ST_GEMM_N && s.kind != ST_GEMM_T) continue;
    const TuneKey key{(int)s.kind, f64 ? 1 : 0, s.njobs, (int)std::lround(4.0 * std::log2(std::max(1.0, s.work))),
                      s.max_n};
    {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      auto it = g_tune_cache.find(key);
      if (it != g_tune_cache.end()) { s.tile = it->second; continue; }
    }
    float best_ms = 0.f;
    int best = 0;
    for (int tile = 0; tile < kBatchedTiles && !r; ++tile) {
      auto launch = [&] {
        return launch_gemm_batched(s.kind == ST_GEMM_T, f64, tile, (const GemmJob*)(hdr + s.jobs_off),
                                   (const int4*)(hdr + s.units_off[tile]), s.nunits[tile], st);
      };
      if (launch() != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess) { r = SORSVD_ERR_CUDA; break; }
      for (int i = 0; i < kTuneReps; ++i)
        if (launch() != cudaSuccess) r = SORSVD_ERR_CUDA;
      float ms = 0.f;
      if (r || cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
          cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        r = SORSVD_ERR_CUDA;
        break;
      }
      if (tile == 0 || ms < best_ms) { best_ms = ms; best = tile; }
    }
    if (r) break;
    s.tile = best;
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return r;
}

int launches_of(const std::vector<BatchStage>& st) {
  int n = 0;
  for (const BatchStage& s : st) n += (s.kind == ST_JACOBI) ? 3 : 1;
  return n;
}

int validate(const sorsvd_problem* probs, int batch, int dtype, unsigned flags) {
  if (!batched_dtype(dtype)) return SORSVD_ERR_DTYPE;
  if (!probs || batch < 1) return SORSVD_ERR_ARG;
  if (flags & ~(SORSVD_FLAG_LITERAL_POWER | SORSVD_FLAG_FIXED_TILES)) return SORSVD_ERR_ARG;
  for (int b = 0; b < batch; ++b)
    if (int r = check_problem(probs[b], dtype)) return r;
  return SORSVD_OK;
}

// total workspace: header + per-problem regions
size_t total_size(const sorsvd_problem* probs, int batch, int dtype, unsigned flags, size_t* hdr_out) {
  sorsvd_batch_plan tmp;
  tmp.ws = nullptr;
  tmp.batch = batch;
  tmp.dtype = dtype;
  Builder B;
  std::vector<ProbState> ps;
  build_plan(&tmp, probs, batch, dtype, flags, B, ps, 0);
  const size_t hdr = header_size(B.buf.size(), batch);
  size_t per = 0;
  for (const ProbState& s : ps) per += align_up(s.L.total);
  if (hdr_out) *hdr_out = hdr;
  return hdr + per;
}

}  // namespace
}  // namespace sorsvd

using namespace sorsvd;

extern "C" size_t sorsvd_batched_workspace_size(const sorsvd_problem* probs, int batch, int dtype, unsigned flags) {
  if (validate(probs, batch, dtype, flags)) return 0;
  return total_size(probs, batch, dtype, flags, nullptr);
}

extern "C" int sorsvd_batched_plan_create(sorsvd_batch_plan** out, const sorsvd_problem* probs, int batch,
                                          int dtype, unsigned flags, int use_graph, void* workspace,
                                          size_t ws_bytes, void* stream) {
  if (!out) return SORSVD_ERR_ARG;
  *out = nullptr;
  if (int r = validate(probs, batch, dtype, flags)) return r;
  size_t hdr = 0;
  const size_t need = total_size(probs, batch, dtype, flags, &hdr);
  if (!workspace || ((uintptr_t)workspace % kAlign) || ws_bytes < need) return SORSVD_ERR_WORKSPACE;
  sorsvd_batch_plan* plan = new sorsvd_batch_plan();
  plan->batch = batch;
  plan->dtype = dtype;
  plan->ws = (char*)workspace;
  plan->hdr_bytes = hdr;
  plan->status = (DeviceStatus*)workspace;
  Builder B;
  std::vector<ProbState> ps;
  build_plan(plan, probs, batch, dtype, flags, B, ps, hdr);
  plan->stages = B.stages;
  plan->launches = launches_of(plan->stages);
  cudaStream_t st = (cudaStream_t)stream;
  char* dst = plan->ws + align_up(sizeof(DeviceStatus) * (size_t)batch);
  if (!B.buf.empty() && (cudaMemcpyAsync(dst, B.buf.data(), B.buf.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
                         cudaStreamSynchronize(st) != cudaSuccess)) {
    sorsvd_batched_plan_destroy(plan);
    return SORSVD_ERR_CUDA;
  }
  if (int r = (flags & SORSVD_FLAG_FIXED_TILES) ? SORSVD_OK : autotune(plan, st)) {
    sorsvd_batched_plan_destroy(plan);
    return r;
  }
  if (use_graph) {
    // capture on a private stream (the caller's may be the legacy stream)
    cudaStream_t cs;
    if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
      sorsvd_batched_plan_destroy(plan);
      return SORSVD_ERR_CUDA;
    }
    int r = SORSVD_OK;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess) r = SORSVD_ERR_CUDA;
    if (!r) {
      // the launches recorded in the graph run (and are counted) at replay
      r = enqueue(plan, cs, false);
      if (cudaStreamEndCapture(cs, &plan->graph) != cudaSuccess) r = SORSVD_ERR_CUDA;
    }
    if (!r && cudaGraphInstantiate(&plan->exec, plan->graph, 0) != cudaSuccess) r = SORSVD_ERR_CUDA;
    cudaStreamDestroy(cs);
    if (r) {
      sorsvd_batched_plan_destroy(plan);
      return r;
    }
  }
  *out = plan;
  return SORSVD_OK;
}

extern "C" int sorsvd_batched_plan_launch(sorsvd_batch_plan* plan, void* stream) {
  if (!plan) return SORSVD_ERR_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  if (plan->exec) {
    if (cudaGraphLaunch(plan->exec, st) != cudaSuccess) return SORSVD_ERR_CUDA;
    count_launches(plan->launches);
    return SORSVD_OK;
  }
  return enqueue(plan, st, true);
}

extern "C" int sorsvd_batched_plan_status(const sorsvd_batch_plan* plan, int* codes, void* stream) {
  if (!plan || !codes) return SORSVD_ERR_ARG;
  std::vector<DeviceStatus> h(plan->batch);
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(h.data(), plan->status, sizeof(DeviceStatus) * h.size(), cudaMemcpyDeviceToHost, st) !=
          cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return SORSVD_ERR_CUDA;
  for (int b = 0; b < plan->batch; ++b) codes[b] = h[b].code;
  return SORSVD_OK;
}

extern "C" int sorsvd_batched_plan_launches(const sorsvd_batch_plan* plan) { return plan ? plan->launches : 0; }

extern "C" int sorsvd_batched_plan_tiles(const sorsvd_batch_plan* plan, int* tiles, int max_tiles) {
  if (!plan) return 0;
  int n = 0;
  for (const BatchStage& s : plan->stages) {
    if (s.kind != ST_GEMM_N && s.kind != ST_GEMM_T) continue;
    if (tiles && n < max_tiles) tiles[n] = s.tile;
    ++n;
  }
  return n;
}

extern "C" void sorsvd_batched_plan_destroy(sorsvd_batch_plan* plan) {
  if (!plan) return;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  delete plan;
}

extern "C" int sorsvd_run_batched(const sorsvd_problem* probs, int batch, int dtype, unsigned flags, void* workspace,
                                  size_t ws_bytes, void* stream) {
  sorsvd_batch_plan* plan = nullptr;
  if (int r = sorsvd_batched_plan_create(&plan, probs, batch, dtype, flags, 0, workspace, ws_bytes, stream)) return r;
  int r = sorsvd_batched_plan_launch(plan, stream);
  sorsvd_batched_plan_destroy(plan);
  return r;
}
