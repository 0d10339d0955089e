// Batched Rand-QLP: many independent problems, each with its own sizes,
// k, p and buffers (one q for the batch), factored by the same chain as
// rqlp_factor (Algorithm 1 steps 3-5 with q power passes, truncated to
// d = k + p columns, CholeskyQR orthonormalisations) in plain FP32.
//
// Every step of the chain is one grouped launch over all problems: the
// products are persistent grouped GEMMs over a flattened tile list, the
// Choleskys one CTA per problem, the small steps one CTA per problem. Stage
// boundaries are kernel boundaries, so no kernel waits on another. The
// launch sequence is fixed at plan creation (gates are device flags), so it
// is captured once into a CUDA graph and replayed as one launch.
//
// Problems are grouped into two width buckets (d <= 32, d > 32); each GEMM
// stage runs one launch per non-empty bucket with the tile shape and grid
// mode (persistent or one CTA per tile) that the autotuner picked for its
// (product shape, bucket).
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <queue>
#include <new>
#include <vector>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace rqlp {
namespace {

// Product shapes the tuner distinguishes.
enum Shape { kTallT = 0, kTallN = 1, kGram = 2, kTrmm = 3, kSmall = 4, kShapes = 5 };
constexpr int kBuckets = 2;
constexpr int kGates = 4;       // [0..2] final orthonormalisations, [3] intermediate ones
constexpr int kInterGate = 3;

int bucket_of(int d) { return d <= 32 ? 0 : 1; }

// A tall Gram X^T X (X: K x d) runs as K slices of at most kGramSliceRows
// rows (four at most), each into its own partial d x d slot, summed by
// gram_reduce_batched_kernel: one CTA per tile over the whole K left the
// problems with K near 4096 running long after the others.
constexpr int64_t kGramSliceRows = 1024;
constexpr int kGramSlicesMax = 4;
int gram_slices(int64_t K) {
  return (int)std::min<int64_t>(kGramSlicesMax, std::max<int64_t>(1, cdiv(K, kGramSliceRows)));
}

// Sum of a problem's Gram slices into G (lower triangle, slice order,
// Kahan-compensated FP32); nothing when slices <= 1 (the product wrote G)
// or when the gate is down (the Gram was skipped, and so is its Cholesky).
struct GramRedJob {
  float* G;
  const float* part;   // slices x d x ld
  int64_t ld;
  int d, slices;
  const int* gate;
};

// Untuned choice per (shape, bucket): what the tuner picked for the mixed
// 512-problem workload (tile shape 0..5, + kGroupCfgs = one CTA per tile).
int default_cfg(int shape, int bucket) {
  constexpr int kOne = kGroupCfgs;
  switch (shape) {
    case kTallT:
    case kTallN: return bucket == 0 ? kOne + 3 : kOne + 0;
    case kTrmm: return bucket == 0 ? 2 : kOne + 2;
    case kGram: return bucket == 0 ? 5 : kOne + 3;
    default: return bucket == 0 ? kOne + 4 : 5;
  }
}

// Per-problem device buffers (in the workspace). The BF16x3 form adds A's
// halves in 64-column panels, the pass operand's halves (X^T, d x ldk) and
// eight tensor maps (see tc_grouped.cu).
struct Bufs {
  float *Y, *Z, *Pt, *T1, *G, *R[3], *Ri[3], *Ra, *Rb, *Rh, *Ts, *Ts2, *Ph;
  float* Gp = nullptr;   // Gram slices (gslices x d x ld) when a tall Gram is split
  int gslices = 1;
  double* scal;
  int* gates;
  int64_t ld;
  uint16_t *Ahi = nullptr, *Alo = nullptr, *XTh = nullptr, *XTl = nullptr;
  uint16_t *Alo2 = nullptr, *XTl2 = nullptr;   // three-part form only
  int64_t ldk = 0;
  char* maps = nullptr;     // 8 x kTcMapBytes
  int* flag = nullptr;      // X low part nonzero (per pass)
};
// Tensor maps of one problem, in this order.
enum TcMap {
  kMapAhiT, kMapAloT, kMapAhiN, kMapAloN, kMapXhiM, kMapXloM, kMapXhiN, kMapXloN,
  kMapAlo2T, kMapAlo2N, kMapXlo2M, kMapXlo2N,   // three-part form only
  kTcMaps
};
constexpr int kMaxTcCtas = 1024;

struct GemmStage {
  bool transA;
  int shape;
  size_t jobs_off;                           // GroupGemm[count] (bucket order)
  size_t tiles_off[kBuckets][kGroupCfgs];    // int[njobs_b + 1] per bucket and cfg
  int total[kBuckets][kGroupCfgs];
  int njobs[kBuckets];                       // jobs per bucket (the problems', or their slices)
  bool gated;
};

// A grouped tensor-core pass (BF16x3 form): prep of X, then the pass.
struct TcStage {
  bool transA;
  size_t jobs_off;        // TcGJob[count]
  size_t prep_off;        // PrepJob[count]
  size_t prep_start_off;  // int[count + 1]
  int prep_total;
  size_t units_off;       // int2[units]
  size_t cta_off;         // int[kMaxTcCtas + 1]
  int G;
  int npad_max;
  int stall;              // test hook: CTA 0 withholds its first stage (first pass only)
  bool exact;             // A and X in three BF16 parts, six products
};

struct Stage {
  enum Kind { kInit, kGemm, kChol, kTranspose, kWriteL, kFinish, kSplit, kTc, kGateClear, kCopyGated, kGramReduce } kind;
  int gemm = -1;         // index into gemms / tcs
  size_t jobs_off = 0;   // CholJob[], SmallJob[] or SplitJob[]
  size_t start_off = 0;  // kSplit: int[count + 1] block prefix
  int total = 0;         // kSplit: blocks
};

}  // namespace
}  // namespace rqlp

struct rqlp_batch_s {
  int count = 0, q = 0, dmax = 0;
  long long sums[rqlp::kBuckets][3] = {};    // per bucket: sum of m, n, d (tuning key)
  int cnt[rqlp::kBuckets] = {0, 0};          // problems per bucket (bucket 0 first)
  rqlp_opts opts{};
  bool exact = false;                        // BF16x3 passes in three parts
  char* dev = nullptr;                       // plan area in the workspace
  std::vector<rqlp::Stage> stages;
  std::vector<rqlp::GemmStage> gemms;
  std::vector<rqlp::TcStage> tcs;
  int* flags = nullptr;                      // TC form: one int per problem (bucket order)
  int* info0 = nullptr;                      // status row that a timed-out grouped pass reports to
  std::vector<char> maps_h;                  // TC form: host copy of the tensor maps
  char* maps_d = nullptr;
  int cfg[rqlp::kShapes][rqlp::kBuckets];
  cudaStream_t cap = nullptr;                // capture stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long graph_kernels = 0;
};

namespace rqlp {
namespace {

std::mutex g_tune_mu;
std::map<std::vector<long long>, std::vector<int>> g_tuned;   // plan signature -> cfg table

std::vector<long long> signature(const rqlp_batch_s* b) {
  // Per bucket: count and the sums of m, n, d (the tuner's choice depends on
  // the size mix, not on the exact problems).
  std::vector<long long> s = {b->q, b->opts.small_fp64};
  for (int bk = 0; bk < kBuckets; ++bk) {
    s.push_back(b->cnt[bk]);
    for (int t = 0; t < 3; ++t) s.push_back(b->sums[bk][t]);
  }
  return s;
}

// Host staging of the plan area; offsets are 256-byte aligned.
struct Stager {
  std::vector<char> h;
  template <typename T>
  size_t put(const T* p, size_t n) {
    size_t off = (size_t)round_up((int64_t)h.size(), 256);
    h.resize(off + n * sizeof(T));
    if (n) std::memcpy(h.data() + off, p, n * sizeof(T));
    return off;
  }
};

struct Builder {
  rqlp_batch_s* b;
  const std::vector<rqlp_problem>& pr;   // bucket order
  const std::vector<Bufs>& bf;
  const std::vector<int>& orig;          // caller's index of each position
  int* info;                             // caller order, 2 ints per problem
  double* diag;                          // caller order, 4 doubles (optional)
  Stager& sg;

  bool tc;                               // BF16x3: passes over A on the tensor cores

  int* info_of(int i) const { return info + 2 * (int64_t)orig[i]; }

  int n() const { return (int)pr.size(); }
  int d(int i) const { return pr[i].k + pr[i].p; }

  // jobs in bucket order; per_bucket: jobs per bucket (default one per problem)
  void gemm(bool transA, int shape, const std::vector<GroupGemm>& jobs, bool gated, const int* per_bucket = nullptr) {
    GemmStage g{};
    g.transA = transA;
    g.shape = shape;
    g.gated = gated;
    g.jobs_off = sg.put(jobs.data(), jobs.size());
    int lo = 0;
    for (int bk = 0; bk < kBuckets; ++bk) {
      const int c = per_bucket != nullptr ? per_bucket[bk] : b->cnt[bk];
      g.njobs[bk] = c;
      for (int cfg = 0; cfg < kGroupCfgs; ++cfg) {
        int bm, bn;
        grouped_tile(cfg, &bm, &bn);
        std::vector<int> ts(c + 1, 0);
        for (int i = 0; i < c; ++i) {
          const GroupGemm& j = jobs[lo + i];
          const int64_t t = (j.M > 0 && j.N > 0) ? cdiv(j.M, bm) * cdiv(j.N, bn) : 0;
          ts[i + 1] = ts[i] + (int)t;
        }
        g.tiles_off[bk][cfg] = sg.put(ts.data(), ts.size());
        g.total[bk][cfg] = ts[c];
      }
      lo += c;
    }
    Stage s;
    s.kind = Stage::kGemm;
    s.gemm = (int)b->gemms.size();
    b->gemms.push_back(g);
    b->stages.push_back(s);
  }
  void chol(const std::vector<CholJob>& jobs) {
    Stage s;
    s.kind = Stage::kChol;
    s.jobs_off = sg.put(jobs.data(), jobs.size());
    b->stages.push_back(s);
  }
  void small(Stage::Kind kind, const std::vector<SmallJob>& jobs) {
    Stage s;
    s.kind = kind;
    s.jobs_off = sg.put(jobs.data(), jobs.size());
    b->stages.push_back(s);
  }

  // BF16 halves of every A (and ||A||_F^2), once per factorisation.
  void split_stage() {
    std::vector<SplitJob> js;
    std::vector<int> st(n() + 1, 0);
    for (int i = 0; i < n(); ++i) {
      SplitJob j{};
      j.A = pr[i].A;
      j.lda = pr[i].lda;
      j.m = pr[i].m;
      j.n = pr[i].n;
      j.npan = cdiv(pr[i].n, 64);
      j.hi = bf[i].Ahi;
      j.lo = bf[i].Alo;
      j.lo2 = b->exact ? bf[i].Alo2 : nullptr;
      j.sumsq = &bf[i].scal[0];
      j.vec = (reinterpret_cast<uintptr_t>(pr[i].A) % 16 == 0 && pr[i].lda % 4 == 0) ? 1 : 0;
      js.push_back(j);
      st[i + 1] = st[i] + tc_split_blocks(pr[i].m, pr[i].n);
    }
    Stage s;
    s.kind = Stage::kSplit;
    s.jobs_off = sg.put(js.data(), js.size());
    s.start_off = sg.put(st.data(), st.size());
    s.total = st[n()];
    b->stages.push_back(s);
  }
  // One grouped tensor-core pass: out(i) = op(A_i) X(i). The (problem, tile)
  // units go longest first onto the least loaded CTA.
  template <typename XF, typename LF, typename OF>
  void tc_pass(bool transA, XF X, LF ldx, OF out) {
    TcStage ts{};
    ts.transA = transA;
    std::vector<TcGJob> js;
    std::vector<PrepJob> ps;
    std::vector<int> pst(n() + 1, 0);
    std::vector<std::pair<long long, int2>> units;
    ts.npad_max = 16;
    for (int i = 0; i < n(); ++i) {
      const int di = d(i), np = tc_npad(di);
      const int64_t M = transA ? pr[i].n : pr[i].m, K = transA ? pr[i].m : pr[i].n;
      ts.npad_max = std::max(ts.npad_max, np);
      TcGJob j{};
      const char* mp = bf[i].maps;
      j.mAhi = mp + (transA ? kMapAhiT : kMapAhiN) * kTcMapBytes;
      j.mAlo = mp + (transA ? kMapAloT : kMapAloN) * kTcMapBytes;
      j.mXhi = mp + (transA ? kMapXhiM : kMapXhiN) * kTcMapBytes;
      j.mXlo = mp + (transA ? kMapXloM : kMapXloN) * kTcMapBytes;
      j.mAlo2 = mp + (transA ? kMapAlo2T : kMapAlo2N) * kTcMapBytes;
      j.mXlo2 = mp + (transA ? kMapXlo2M : kMapXlo2N) * kTcMapBytes;
      j.out = out(i);
      j.ldo = bf[i].ld;
      j.M = (int)M;
      j.d = di;
      j.npad = np;
      j.kblocks = (int)cdiv(K, 32);
      j.vec_out = (reinterpret_cast<uintptr_t>(j.out) % 16 == 0 && j.ldo % 4 == 0) ? 1 : 0;
      j.idesc = tc_idesc(np, transA);
      j.xlo_nonzero = bf[i].flag;
      js.push_back(j);
      PrepJob p{};
      p.X = X(i);
      p.ldx = ldx(i);
      p.K = K;
      p.d = di;
      p.th = bf[i].XTh;
      p.tl = bf[i].XTl;
      p.tl2 = b->exact ? bf[i].XTl2 : nullptr;
      p.ldk = bf[i].ldk;
      p.flag = bf[i].flag;
      ps.push_back(p);
      pst[i + 1] = pst[i] + tc_prep_blocks(K, di);
      for (int t = 0; t < (int)cdiv(M, 128); ++t) units.push_back({(long long)j.kblocks * (np + 64), int2{i, t}});
    }
    std::stable_sort(units.begin(), units.end(), [](const auto& a, const auto& c) { return a.first > c.first; });
    const int G = (int)std::max<size_t>(1, std::min<size_t>(units.size(), std::min(kMaxTcCtas, sm_count())));
    std::vector<std::vector<int2>> per(G);
    std::priority_queue<std::pair<long long, int>, std::vector<std::pair<long long, int>>, std::greater<>> load;
    for (int c = 0; c < G; ++c) load.push({0, c});
    for (const auto& u : units) {
      auto top = load.top();
      load.pop();
      per[top.second].push_back(u.second);
      load.push({top.first + u.first, top.second});
    }
    std::vector<int2> flat;
    std::vector<int> cs(kMaxTcCtas + 1, 0);
    for (int c = 0; c < G; ++c) {
      cs[c] = (int)flat.size();
      flat.insert(flat.end(), per[c].begin(), per[c].end());
    }
    for (int c = G; c <= kMaxTcCtas; ++c) cs[c] = (int)flat.size();
    ts.jobs_off = sg.put(js.data(), js.size());
    ts.prep_off = sg.put(ps.data(), ps.size());
    ts.prep_start_off = sg.put(pst.data(), pst.size());
    ts.prep_total = pst[n()];
    ts.units_off = sg.put(flat.data(), flat.size());
    ts.cta_off = sg.put(cs.data(), cs.size());
    ts.G = G;
    ts.stall = (b->opts.test_stall != 0 && b->tcs.empty()) ? 1 : 0;
    ts.exact = b->exact;
    Stage s;
    s.kind = Stage::kTc;
    s.gemm = (int)b->tcs.size();
    b->tcs.push_back(ts);
    b->stages.push_back(s);
  }

  GroupGemm job(const float* A, int64_t lda, const float* B, int64_t ldb, float* C, int64_t ldc, int64_t M,
                int64_t N, int64_t K) {
    GroupGemm j{};
    j.A = A; j.lda = lda; j.B = B; j.ldb = ldb; j.C = C; j.ldc = ldc;
    j.M = M; j.N = N; j.K = K;
    return j;
  }

  // G = X^T X over `rows(i)` rows; a tall Gram (shape kGram) in K slices of
  // at most kGramSliceRows rows, summed by a reduction stage.
  template <typename XF, typename RF>
  void gram(XF X, RF rows, int shape, int gate_slot) {
    std::vector<GroupGemm> js;
    std::vector<GramRedJob> rj;
    int per_bucket[kBuckets] = {0, 0};
    bool split = false;
    for (int i = 0; i < n(); ++i) {
      const int bk = i < b->cnt[0] ? 0 : 1;   // problems are in bucket order
      const int64_t K = rows(i);
      const int s = shape == kGram ? std::min(bf[i].gslices, gram_slices(K)) : 1;
      const int64_t kc = s > 1 ? round_up(cdiv(K, s), 16) : K;
      int used = 0;
      for (int64_t k0 = 0; k0 < K; k0 += kc, ++used) {
        const int64_t kl = std::min(kc, K - k0);
        float* C = s > 1 ? bf[i].Gp + (int64_t)used * d(i) * bf[i].ld : bf[i].G;
        const float* Xk = X(i) + k0 * bf[i].ld;
        GroupGemm j = job(Xk, bf[i].ld, Xk, bf[i].ld, C, bf[i].ld, d(i), d(i), kl);
        j.lower_only = 1;   // the Cholesky reads G(i, j) for j <= i
        if (gate_slot >= 0) {
          j.gate = &bf[i].gates[gate_slot];
          j.gate_mode = kGateSkip;
        }
        js.push_back(j);
        ++per_bucket[bk];
      }
      GramRedJob r{};
      r.G = bf[i].G;
      r.part = bf[i].Gp;
      r.ld = bf[i].ld;
      r.d = d(i);
      r.slices = s > 1 ? used : 1;
      r.gate = gate_slot >= 0 ? &bf[i].gates[gate_slot] : nullptr;
      rj.push_back(r);
      split = split || s > 1;
    }
    gemm(true, shape, js, gate_slot >= 0, per_bucket);
    if (split) {
      Stage st;
      st.kind = Stage::kGramReduce;
      st.jobs_off = sg.put(rj.data(), rj.size());
      b->stages.push_back(st);
    }
  }
  void cholesky(int slot, int gate_out, int gate_in) {
    std::vector<CholJob> js;
    for (int i = 0; i < n(); ++i) {
      CholJob j{};
      j.d = d(i);
      j.G = bf[i].G; j.ldg = bf[i].ld;
      j.R = bf[i].R[slot]; j.Rinv = bf[i].Ri[slot]; j.ldr = bf[i].ld;
      j.info = info_of(i);
      j.shift_count = &bf[i].scal[2];
      j.gate_out = gate_out >= 0 ? &bf[i].gates[gate_out] : nullptr;
      j.gate_in = gate_in >= 0 ? &bf[i].gates[gate_in] : nullptr;
      js.push_back(j);
    }
    chol(js);
  }
  // out = X R_slot^{-1}; gate_slot >= 0: when that gate is 0, out = X
  // (kGateCopy) or no work (kGateSkip).
  template <typename XF, typename OF, typename LF, typename RF>
  void trmm(XF X, OF out, LF ldout, RF rows, int slot, int shape, int gate_slot, int gate_mode = kGateCopy) {
    std::vector<GroupGemm> js;
    for (int i = 0; i < n(); ++i) {
      GroupGemm j = job(X(i), bf[i].ld, bf[i].Ri[slot], bf[i].ld, out(i), ldout(i), rows(i), d(i), d(i));
      j.b_upper = 1;
      if (gate_slot >= 0) {
        j.gate = &bf[i].gates[gate_slot];
        j.gate_mode = gate_mode;
      }
      js.push_back(j);
    }
    gemm(false, shape, js, gate_slot >= 0);
  }
  // Gate word `slot` of every problem back to 0.
  void gate_clear(int slot) {
    std::vector<SmallJob> js(n());
    for (int i = 0; i < n(); ++i) {
      js[i].gates = bf[i].gates;
      js[i].ngates = slot;
    }
    small(Stage::kGateClear, js);
  }
  // out = X for the problems whose gate `slot` is raised.
  template <typename XF, typename OF, typename RF>
  void copy_gated(XF X, OF out, RF rows, int slot) {
    std::vector<SmallJob> js(n());
    for (int i = 0; i < n(); ++i) {
      js[i].d = d(i);
      js[i].X = X(i); js[i].ldx = bf[i].ld;
      js[i].Y = out(i); js[i].ldy = bf[i].ld;
      js[i].rows = rows(i);
      js[i].gates = bf[i].gates;
      js[i].ngates = slot;
    }
    small(Stage::kCopyGated, js);
  }
  // One CholeskyQR pass, out = X R^{-1} (slot 0), and a second one for the
  // problems whose first Cholesky had to shift (gate kInterGate): a shifted
  // factor keeps the span but leaves out far from orthonormal, which the
  // next pass over A would carry into its small directions. X is dead after.
  template <typename XF, typename OF, typename RF>
  void orth_inter(XF X, OF out, RF rows, bool tall) {
    const int gs = tall ? kGram : kSmall, ts = tall ? kTrmm : kSmall;
    auto ld = [&](int i) { return bf[i].ld; };
    gate_clear(kInterGate);
    gram(X, rows, gs, -1);
    cholesky(0, kInterGate, -1);
    trmm(X, out, ld, rows, 0, ts, -1);
    gram(out, rows, gs, kInterGate);
    cholesky(1, -1, kInterGate);
    trmm(out, X, ld, rows, 1, ts, kInterGate, kGateSkip);
    copy_gated(X, out, rows, kInterGate);
  }
  // CholeskyQR2 plus a third pass gated on a shifted Cholesky; X is
  // overwritten; Racc (optional) receives R3 R2 R1.
  template <typename XF, typename OF, typename LF, typename TF, typename RF, typename AF>
  void orth_final(XF X, OF out, LF ldout, TF tmp, RF rows, bool tall, int g, AF Racc, bool with_r) {
    const int gs = tall ? kGram : kSmall, ts = tall ? kTrmm : kSmall;
    auto ld = [&](int i) { return bf[i].ld; };
    gram(X, rows, gs, -1);
    cholesky(0, g, -1);
    trmm(X, tmp, ld, rows, 0, ts, -1);
    gram(tmp, rows, gs, -1);
    cholesky(1, g, -1);
    trmm(tmp, X, ld, rows, 1, ts, -1);
    gram(X, rows, gs, g);
    cholesky(2, -1, g);
    trmm(X, out, ldout, rows, 2, ts, g);
    if (with_r) {
      std::vector<GroupGemm> a, c;
      for (int i = 0; i < n(); ++i) {
        GroupGemm j = job(bf[i].R[1], bf[i].ld, bf[i].R[0], bf[i].ld, bf[i].Ra, bf[i].ld, d(i), d(i), d(i));
        j.b_upper = 1;
        a.push_back(j);
        GroupGemm k2 = job(bf[i].R[2], bf[i].ld, bf[i].Ra, bf[i].ld, Racc(i), bf[i].ld, d(i), d(i), d(i));
        k2.b_upper = 1;
        c.push_back(k2);
      }
      gemm(false, kSmall, a, false);
      gemm(false, kSmall, c, false);
    }
  }

  void build() {
    const int q = b->q;
    auto ld = [&](int i) { return bf[i].ld; };
    auto rows_n = [&](int i) { return (int64_t)pr[i].n; };
    auto rows_m = [&](int i) { return (int64_t)pr[i].m; };
    auto rows_d = [&](int i) { return (int64_t)d(i); };
    auto Y = [&](int i) { return bf[i].Y; };
    auto Z = [&](int i) { return bf[i].Z; };
    auto Pt = [&](int i) { return bf[i].Pt; };
    auto T1 = [&](int i) { return bf[i].T1; };
    auto none = [&](int) { return (float*)nullptr; };

    std::vector<SmallJob> sj;
    for (int i = 0; i < n(); ++i) {
      SmallJob j{};
      j.d = d(i);
      j.scal = bf[i].scal;
      j.info = info_of(i);
      j.diag = diag != nullptr ? diag + 4 * (int64_t)orig[i] : nullptr;
      j.gates = bf[i].gates;
      j.ngates = kGates;
      sj.push_back(j);
    }
    small(Stage::kInit, sj);

    // A pass over every problem: grouped tensor-core passes in the BF16x3
    // form, grouped FP32 products otherwise (sumsq: ||A||_F^2 rides along).
    auto pass = [&](bool transA, auto X, auto ldx, auto out, bool sumsq) {
      if (tc) {
        tc_pass(transA, X, ldx, out);
        return;
      }
      std::vector<GroupGemm> js;
      for (int i = 0; i < n(); ++i) {
        const int64_t M = transA ? pr[i].n : pr[i].m, K = transA ? pr[i].m : pr[i].n;
        GroupGemm j = job(pr[i].A, pr[i].lda, X(i), ldx(i), out(i), bf[i].ld, M, d(i), K);
        if (sumsq) j.sumsq = &bf[i].scal[0];
        js.push_back(j);
      }
      gemm(transA, transA ? kTallT : kTallN, js, false);
    };
    // Y = A^T Omega (Algorithm 1 step 3); ||A||_F^2 comes with it (or with
    // the split in the BF16x3 form).
    if (tc) split_stage();
    pass(true, [&](int i) { return pr[i].Omega; }, [&](int i) { return pr[i].ldo; }, Y, true);
    auto passN = [&](auto X, auto out) { pass(false, X, ld, out, false); };   // out (m x d) = A X
    auto passT = [&](auto X, auto out) { pass(true, X, ld, out, false); };    // out (n x d) = A^T X

    if (q == 0) orth_final(Y, Pt, ld, T1, rows_n, true, 0, none, false);
    else orth_inter(Y, Pt, rows_n, true);
    for (int it = 1; it <= q; ++it) {
      passN(Pt, Z);                          // Z = A P~
      orth_inter(Z, T1, rows_m, true);       // Z = qf(Z), one pass
      passT(T1, Y);                          // Y = A^T Z
      if (it == q) orth_final(Y, Pt, ld, T1, rows_n, true, 0, none, false);
      else orth_inter(Y, Pt, rows_n, true);
    }
    // (Q, R) = qr(A P~)  (Algorithm 1 step 4)
    passN(Pt, Z);
    orth_final(Z, [&](int i) { return pr[i].Q; }, [&](int i) { return pr[i].ldq; }, T1, rows_m, true, 1,
               [&](int i) { return bf[i].Rb; }, true);
    // (P^, R^) = qr(R^T), L = R^^T  (step 5 applied to the d x d factor)
    std::vector<SmallJob> tj = sj;
    for (int i = 0; i < n(); ++i) {
      tj[i].X = bf[i].Rb; tj[i].ldx = bf[i].ld;
      tj[i].Y = bf[i].Ts; tj[i].ldy = bf[i].ld;
    }
    small(Stage::kTranspose, tj);
    orth_final([&](int i) { return bf[i].Ts; }, [&](int i) { return bf[i].Ph; }, ld,
               [&](int i) { return bf[i].Ts2; }, rows_d, false, 2, [&](int i) { return bf[i].Rh; }, true);
    std::vector<SmallJob> lj = sj;
    for (int i = 0; i < n(); ++i) {
      lj[i].X = bf[i].Rh; lj[i].ldx = bf[i].ld;
      lj[i].Y = pr[i].L; lj[i].ldy = pr[i].ldl;
    }
    small(Stage::kWriteL, lj);
    // P = P~ P^
    {
      std::vector<GroupGemm> js;
      for (int i = 0; i < n(); ++i)
        js.push_back(job(bf[i].Pt, bf[i].ld, bf[i].Ph, bf[i].ld, pr[i].P, pr[i].ldp, pr[i].n, d(i), d(i)));
      gemm(false, kTrmm, js, false);
    }
    small(Stage::kFinish, sj);
  }
};

Bufs take_bufs(Arena& ar, const rqlp_problem& p, bool tc, bool exact) {
  Bufs f{};
  const int d = p.k + p.p;
  f.ld = round_up(d, 4);
  const int64_t dd = (int64_t)d * f.ld, tall = std::max(p.m, p.n);
  f.Y = ar.take<float>(p.n * f.ld);
  f.Z = ar.take<float>(p.m * f.ld);
  f.Pt = ar.take<float>(p.n * f.ld);
  f.T1 = ar.take<float>(tall * f.ld);
  f.G = ar.take<float>(dd);
  f.gslices = gram_slices(tall);
  if (f.gslices > 1) f.Gp = ar.take<float>((size_t)f.gslices * dd);
  for (int s = 0; s < 3; ++s) {
    f.R[s] = ar.take<float>(dd);
    f.Ri[s] = ar.take<float>(dd);
  }
  f.Ra = ar.take<float>(dd);
  f.Rb = ar.take<float>(dd);
  f.Rh = ar.take<float>(dd);
  f.Ts = ar.take<float>(dd);
  f.Ts2 = ar.take<float>(dd);
  f.Ph = ar.take<float>(dd);
  f.scal = ar.take<double>(4);
  f.gates = ar.take<int>(kGates);
  if (tc) {
    const int64_t cols = round_up(p.n, 64);
    f.Ahi = ar.take<uint16_t>(p.m * cols);
    f.Alo = ar.take<uint16_t>(p.m * cols);
    f.ldk = round_up(tall, 8);
    f.XTh = ar.take<uint16_t>(d * f.ldk);
    f.XTl = ar.take<uint16_t>(d * f.ldk);
    if (exact) {
      f.Alo2 = ar.take<uint16_t>(p.m * cols);
      f.XTl2 = ar.take<uint16_t>(d * f.ldk);
    }
  }
  return f;
}

// The tensor maps of one problem (host encoding; false on failure): eight,
// and four more for the third parts in the three-part form.
bool encode_maps(const Bufs& f, const rqlp_problem& p, char* out, bool exact) {
  const int d = p.k + p.p, np = tc_npad(d);
  const long long npan = cdiv(p.n, 64);
  auto at_map = [&](int k) { return out + k * kTcMapBytes; };
  return tc_panel_map(at_map(kMapAhiT), f.Ahi, p.m, npan, 64, 32, 2, true) &&
         tc_panel_map(at_map(kMapAloT), f.Alo, p.m, npan, 64, 32, 2, true) &&
         tc_panel_map(at_map(kMapAhiN), f.Ahi, p.m, npan, 32, 128, 1, false) &&
         tc_panel_map(at_map(kMapAloN), f.Alo, p.m, npan, 32, 128, 1, false) &&
         tc_map2d(at_map(kMapXhiM), f.XTh, p.m, d, f.ldk, 32, np, false) &&
         tc_map2d(at_map(kMapXloM), f.XTl, p.m, d, f.ldk, 32, np, false) &&
         tc_map2d(at_map(kMapXhiN), f.XTh, p.n, d, f.ldk, 32, np, false) &&
         tc_map2d(at_map(kMapXloN), f.XTl, p.n, d, f.ldk, 32, np, false) &&
         (!exact || (tc_panel_map(at_map(kMapAlo2T), f.Alo2, p.m, npan, 64, 32, 2, true) &&
                     tc_panel_map(at_map(kMapAlo2N), f.Alo2, p.m, npan, 32, 128, 1, false) &&
                     tc_map2d(at_map(kMapXlo2M), f.XTl2, p.m, d, f.ldk, 32, np, false) &&
                     tc_map2d(at_map(kMapXlo2N), f.XTl2, p.n, d, f.ldk, 32, np, false)));
}

bool valid_problem(const rqlp_problem& p) {
  if (p.A == nullptr || p.Omega == nullptr || p.Q == nullptr || p.L == nullptr || p.P == nullptr) return false;
  if (p.m <= 0 || p.n <= 0 || p.k < 1 || p.p < 0) return false;
  const int64_t d = (int64_t)p.k + p.p;
  if (d > std::min(p.m, p.n) || d > RQLP_BATCH_MAX_D) return false;
  return p.lda >= p.n && p.ldo >= d && p.ldq >= d && p.ldl >= d && p.ldp >= d;
}

// Bucket order: the permutation that puts the d <= 32 problems first.
std::vector<int> bucket_order(int count, const rqlp_problem* probs, int* cnt) {
  std::vector<int> ord;
  cnt[0] = cnt[1] = 0;
  for (int bk = 0; bk < kBuckets; ++bk)
    for (int i = 0; i < count; ++i)
      if (bucket_of(probs[i].k + probs[i].p) == bk) {
        ord.push_back(i);
        ++cnt[bk];
      }
  return ord;
}

// Lays out the workspace (per-problem buffers first, plan area last) and
// builds the stage list into `sg`; a dry arena only measures.
size_t layout(rqlp_batch_s* b, int count, const rqlp_problem* probs, Arena& ar, int* d_info, double* d_diag,
              Stager& sg) {
  std::vector<int> ord = bucket_order(count, probs, b->cnt);
  std::vector<rqlp_problem> pr;
  std::vector<Bufs> bf;
  const bool tc = b->opts.precision == RQLP_PREC_BF16X3;
  // Three BF16 parts unless the caller asked for two: the batch's problems are
  // the small and medium sizes where the two-part rounding, amplified by an
  // ill-conditioned leading block, reaches the 1e-4 |L_ii| bound.
  b->exact = tc && b->opts.bf16_parts != 2;
  int* flags = nullptr;
  char* maps = nullptr;
  if (tc) {
    flags = ar.take<int>(count);
    maps = ar.take<char>((size_t)count * kTcMaps * kTcMapBytes);
  }
  b->flags = flags;
  b->maps_d = maps;
  b->info0 = d_info;
  b->maps_h.clear();
  b->dmax = 0;
  for (int bk = 0; bk < kBuckets; ++bk)
    for (int t = 0; t < 3; ++t) b->sums[bk][t] = 0;
  for (int i : ord) {
    const int d = probs[i].k + probs[i].p, bk = bucket_of(d);
    pr.push_back(probs[i]);
    bf.push_back(take_bufs(ar, probs[i], tc, b->exact));
    if (tc) {
      const size_t pos = bf.size() - 1;
      bf.back().flag = ar.dry ? nullptr : flags + pos;
      bf.back().maps = ar.dry ? nullptr : maps + pos * kTcMaps * kTcMapBytes;
    }
    b->dmax = std::max(b->dmax, d);
    b->sums[bk][0] += probs[i].m;
    b->sums[bk][1] += probs[i].n;
    b->sums[bk][2] += d;
  }
  if (tc && !ar.dry) {
    b->maps_h.assign((size_t)count * kTcMaps * kTcMapBytes, 0);
    for (size_t i = 0; i < bf.size(); ++i)
      if (!encode_maps(bf[i], pr[i], b->maps_h.data() + i * kTcMaps * kTcMapBytes, b->exact)) b->maps_h.clear();
  }
  b->stages.clear();
  b->gemms.clear();
  b->tcs.clear();
  Builder bd{b, pr, bf, ord, d_info, d_diag, sg, tc};
  bd.build();
  char* plan = ar.take<char>(sg.h.size() + 256);
  b->dev = ar.dry ? nullptr : plan;
  return ar.off;
}

template <typename T>
const T* at(const rqlp_batch_s* b, size_t off) {
  return reinterpret_cast<const T*>(b->dev + off);
}

// One CTA per problem (see GramRedJob).
__global__ void __launch_bounds__(256) gram_reduce_batched_kernel(const GramRedJob* __restrict__ jobs, int count) {
  if ((int)blockIdx.x >= count) return;
  const GramRedJob j = jobs[blockIdx.x];
  if (j.slices <= 1 || (j.gate != nullptr && *j.gate == 0)) return;
  const int64_t slot = (int64_t)j.d * j.ld;
  for (int e = threadIdx.x; e < j.d * j.d; e += blockDim.x) {
    const int r = e / j.d, c = e % j.d;
    if (c > r) continue;
    const float* p = j.part + (int64_t)r * j.ld + c;
    float s = 0.f, comp = 0.f;
    for (int z = 0; z < j.slices; ++z) {
      const float y = p[z * slot] - comp, t = s + y;
      comp = (t - s) - y;
      s = t;
    }
    j.G[(int64_t)r * j.ld + c] = s;
  }
}

cudaError_t run_gemm(const rqlp_batch_s* b, const GemmStage& g, cudaStream_t st, int only_bucket = -1,
                     int force_cfg = -1) {
  const GroupGemm* jobs = at<GroupGemm>(b, g.jobs_off);
  int lo = 0;
  for (int bk = 0; bk < kBuckets; ++bk) {
    const int c = g.njobs[bk];
    if (c > 0 && (only_bucket < 0 || only_bucket == bk)) {
      const int choice = force_cfg >= 0 ? force_cfg : b->cfg[g.shape][bk];
      const int cfg = choice % kGroupCfgs;   // tile shape; the choice also fixes the grid mode
      CK(gemm_grouped(g.transA, choice, jobs + lo, at<int>(b, g.tiles_off[bk][cfg]), c, g.total[bk][cfg], st));
    }
    lo += c;
  }
  return cudaSuccess;
}

cudaError_t run_stages(const rqlp_batch_s* b, cudaStream_t st) {
  Range r("rqlp: batch stages");
  const bool fp64 = b->opts.small_fp64 != 0;
  for (const Stage& s : b->stages) {
    switch (s.kind) {
      case Stage::kInit: CK(init_batched(at<SmallJob>(b, s.jobs_off), b->count, st)); break;
      case Stage::kGemm: CK(run_gemm(b, b->gemms[s.gemm], st)); break;
      case Stage::kChol: CK(chol_inv_batched(at<CholJob>(b, s.jobs_off), b->count, b->dmax, fp64, st)); break;
      case Stage::kTranspose: CK(transpose_batched(at<SmallJob>(b, s.jobs_off), b->count, st)); break;
      case Stage::kWriteL: CK(write_L_batched(at<SmallJob>(b, s.jobs_off), b->count, st)); break;
      case Stage::kFinish: CK(finish_diag_batched(at<SmallJob>(b, s.jobs_off), b->count, st)); break;
      case Stage::kSplit:
        CK(split_grouped(at<SplitJob>(b, s.jobs_off), at<int>(b, s.start_off), b->count, s.total, st));
        break;
      case Stage::kGateClear: CK(gate_clear_batched(at<SmallJob>(b, s.jobs_off), b->count, st)); break;
      case Stage::kCopyGated: CK(copy_gated_batched(at<SmallJob>(b, s.jobs_off), b->count, st)); break;
      case Stage::kGramReduce:
        gram_reduce_batched_kernel<<<b->count, 256, 0, st>>>(at<GramRedJob>(b, s.jobs_off), b->count);
        note_launch();
        CK(cudaGetLastError());
        break;
      case Stage::kTc: {
        const TcStage& t = b->tcs[s.gemm];
        CK(cudaMemsetAsync(b->flags, 0, sizeof(int) * b->count, st));
        CK(prep_grouped(at<PrepJob>(b, t.prep_off), at<int>(b, t.prep_start_off), b->count, t.prep_total, st));
        CK(tc_grouped_pass(t.transA, at<TcGJob>(b, t.jobs_off), at<int2>(b, t.units_off), at<int>(b, t.cta_off),
                           t.G, t.npad_max, b->info0, t.stall, t.exact, st));
        break;
      }
    }
  }
  return cudaSuccess;
}

void drop_graph(rqlp_batch_s* b) {
  if (b->exec != nullptr) cudaGraphExecDestroy(b->exec);
  if (b->graph != nullptr) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

rqlp_opts resolve_opts(const rqlp_opts* o) {
  rqlp_opts r;
  rqlp_default_opts(&r);
  if (o != nullptr) r = *o;
  return r;
}

bool valid_batch(int count, const rqlp_problem* probs, int q, const rqlp_opts& o) {
  if (count <= 0 || probs == nullptr || q < 0 || q > 64) return false;
  if ((o.precision != RQLP_PREC_FP32 && o.precision != RQLP_PREC_BF16X3) || (o.small_fp64 != 0 && o.small_fp64 != 1))
    return false;
  if (o.test_stall != 0 && (o.test_stall != 1 || o.precision != RQLP_PREC_BF16X3)) return false;
  if (o.bf16_parts != 0 && (o.precision != RQLP_PREC_BF16X3 || (o.bf16_parts != 2 && o.bf16_parts != 3)))
    return false;
  if (o.literal_step5 != 0 || o.fused_power != 0) return false;
  for (int i = 0; i < 2; ++i)
    if (o.reserved[i] != 0) return false;
  for (int i = 0; i < count; ++i)
    if (!valid_problem(probs[i])) return false;
  return true;
}

}  // namespace
}  // namespace rqlp

using namespace rqlp;

extern "C" {

size_t rqlp_batch_workspace_bytes(int count, const rqlp_problem* probs, int q, const rqlp_opts* opts) {
  const rqlp_opts o = resolve_opts(opts);
  if (!valid_batch(count, probs, q, o)) return 0;
  rqlp_batch_s b;
  b.count = count;
  b.q = q;
  b.opts = o;
  Arena ar;
  ar.dry = true;
  Stager sg;
  return layout(&b, count, probs, ar, nullptr, nullptr, sg);
}

rqlp_status rqlp_batch_create(int count, const rqlp_problem* probs, int q, void* workspace, size_t ws_bytes,
                              int* d_info, double* d_diag, const rqlp_opts* opts, void* stream, rqlp_batch* out) {
  if (out == nullptr) return RQLP_ERR_ARG;
  *out = nullptr;
  const rqlp_opts o = resolve_opts(opts);
  if (o.precision == RQLP_PREC_BF16X3 && !tc_supported(nullptr, 0, nullptr, 0)) return RQLP_ERR_UNSUPPORTED;
  if (!valid_batch(count, probs, q, o) || d_info == nullptr) return RQLP_ERR_ARG;
  if (!chol_batched_fits(RQLP_BATCH_MAX_D, o.small_fp64 != 0)) return RQLP_ERR_UNSUPPORTED;
  const size_t need = rqlp_batch_workspace_bytes(count, probs, q, &o);
  if (workspace == nullptr || ws_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 255) != 0)
    return RQLP_ERR_WORKSPACE;
  rqlp_batch_s* b = new (std::nothrow) rqlp_batch_s();
  if (b == nullptr) return RQLP_ERR_CUDA;
  b->count = count;
  b->q = q;
  b->opts = o;
  Arena ar;
  ar.base = static_cast<char*>(workspace);
  ar.cap = ws_bytes;
  Stager sg;
  layout(b, count, probs, ar, d_info, d_diag, sg);
  for (int s = 0; s < kShapes; ++s)
    for (int bk = 0; bk < kBuckets; ++bk) b->cfg[s][bk] = default_cfg(s, bk);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(signature(b));
    if (it != g_tuned.end())
      for (int s = 0; s < kShapes; ++s)
        for (int bk = 0; bk < kBuckets; ++bk) b->cfg[s][bk] = it->second[s * kBuckets + bk];
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const bool tc = o.precision == RQLP_PREC_BF16X3;
  if (tc && b->maps_h.empty()) {   // a tensor map was rejected
    delete b;
    return RQLP_ERR_UNSUPPORTED;
  }
  if (gemm_grouped_prepare() != cudaSuccess ||
      chol_inv_batched(nullptr, 0, 0, o.small_fp64 != 0, st) != cudaSuccess ||
      (tc && (tc_grouped_pass(true, nullptr, nullptr, nullptr, 0, 16, nullptr, 0, false, st) != cudaSuccess ||
              tc_grouped_pass(false, nullptr, nullptr, nullptr, 0, 16, nullptr, 0, false, st) != cudaSuccess ||
              cudaMemcpyAsync(b->maps_d, b->maps_h.data(), b->maps_h.size(), cudaMemcpyHostToDevice, st) !=
                  cudaSuccess)) ||
      cudaMemcpyAsync(b->dev, sg.h.data(), sg.h.size(), cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess ||
      cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return RQLP_ERR_CUDA;
  }
  *out = b;
  return RQLP_OK;
}

rqlp_status rqlp_batch_run(rqlp_batch b, void* stream) {
  if (b == nullptr) return RQLP_ERR_ARG;
  return run_stages(b, static_cast<cudaStream_t>(stream)) == cudaSuccess ? RQLP_OK : RQLP_ERR_CUDA;
}

rqlp_status rqlp_batch_launch(rqlp_batch b, void* stream) {
  if (b == nullptr) return RQLP_ERR_ARG;
  if (b->exec == nullptr) {
    const unsigned long long before = rqlp_kernel_launches();
    if (cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return RQLP_ERR_CUDA;
    const cudaError_t e = run_stages(b, b->cap);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(b->cap, &g);
    const long long captured = (long long)(rqlp_kernel_launches() - before);
    note_launch((int)-captured);   // counted when the graph runs
    if (e != cudaSuccess || e2 != cudaSuccess || g == nullptr) {
      if (g != nullptr) cudaGraphDestroy(g);
      return RQLP_ERR_CUDA;
    }
    if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
      cudaGraphDestroy(g);
      b->exec = nullptr;
      return RQLP_ERR_CUDA;
    }
    b->graph = g;
    b->graph_kernels = captured;
  }
  if (cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) return RQLP_ERR_CUDA;
  note_launch((int)b->graph_kernels);
  return RQLP_OK;
}

rqlp_status rqlp_batch_autotune(rqlp_batch b, int reps, void* stream) {
  if (b == nullptr || reps < 1) return RQLP_ERR_ARG;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return RQLP_ERR_CUDA;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return RQLP_ERR_CUDA;
  }
  rqlp_status rc = RQLP_OK;
  // Representative stage per (shape, bucket): the first ungated one. Timing
  // is data-independent for these FP32 products, so the workspace contents
  // do not matter.
  for (int shape = 0; shape < kShapes && rc == RQLP_OK; ++shape) {
    const GemmStage* rep = nullptr;
    for (const GemmStage& g : b->gemms)
      if (g.shape == shape && !g.gated) {
        rep = &g;
        break;
      }
    if (rep == nullptr) continue;
    for (int bk = 0; bk < kBuckets && rc == RQLP_OK; ++bk) {
      if (b->cnt[bk] == 0) continue;
      float best = 1e30f;
      for (int cfg = 0; cfg < kGroupChoices; ++cfg) {
        float ms = 0.f;
        if (run_gemm(b, *rep, st, bk, cfg) != cudaSuccess ||      // warm-up
            cudaEventRecord(e0, st) != cudaSuccess) {
          rc = RQLP_ERR_CUDA;
          break;
        }
        for (int r = 0; r < reps; ++r)
          if (run_gemm(b, *rep, st, bk, cfg) != cudaSuccess) rc = RQLP_ERR_CUDA;
        if (rc != RQLP_OK || cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
          rc = RQLP_ERR_CUDA;
          break;
        }
        if (ms < best) {
          best = ms;
          b->cfg[shape][bk] = cfg;
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != RQLP_OK) return rc;
  drop_graph(b);   // recaptured with the new tiles on the next launch
  std::vector<int> t(kShapes * kBuckets);
  for (int s = 0; s < kShapes; ++s)
    for (int bk = 0; bk < kBuckets; ++bk) t[s * kBuckets + bk] = b->cfg[s][bk];
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tuned[signature(b)] = t;
  return RQLP_OK;
}

int rqlp_batch_tuning(rqlp_batch b, int* cfg, int cap) {
  if (b == nullptr) return 0;
  int n = 0;
  for (int s = 0; s < kShapes; ++s)
    for (int bk = 0; bk < kBuckets; ++bk) {
      if (cfg != nullptr && n < cap) cfg[n] = b->cfg[s][bk];
      ++n;
    }
  return n;
}

rqlp_status rqlp_batch_destroy(rqlp_batch b) {
  if (b == nullptr) return RQLP_OK;
  drop_graph(b);
  if (b->cap != nullptr) cudaStreamDestroy(b->cap);
  delete b;
  return RQLP_OK;
}

rqlp_status rqlp_factor_batched(int count, const rqlp_problem* probs, int q, void* workspace, size_t ws_bytes,
                                int* d_info, double* d_diag, const rqlp_opts* opts, void* stream) {
  rqlp_batch b = nullptr;
  rqlp_status s = rqlp_batch_create(count, probs, q, workspace, ws_bytes, d_info, d_diag, opts, stream, &b);
  if (s != RQLP_OK) return s;
  s = rqlp_batch_launch(b, stream);
  if (s == RQLP_OK && cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess) s = RQLP_ERR_CUDA;
  rqlp_batch_destroy(b);
  return s;
}

}  // extern "C"
