// Host-side runtime services of the library: the kernel-launch counter, the
// optional per-pass event timing used by the benchmark and NVTX ranges over
// the steps of the chain.
#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace rqlp {

Range::Range(const char* name) { nvtxRangePushA(name); }
Range::~Range() { nvtxRangePop(); }

namespace {

std::atomic<unsigned long long> g_launches{0};

struct Rec {
  cudaEvent_t b, e;
  int tag;
};

struct Prof {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> pool;
  std::vector<Rec> recs;
  cudaEvent_t pending = nullptr;
};

Prof& prof() {
  static Prof p;
  return p;
}

cudaEvent_t take_event(Prof& p) {
  if (!p.pool.empty()) {
    cudaEvent_t ev = p.pool.back();
    p.pool.pop_back();
    return ev;
  }
  cudaEvent_t ev = nullptr;
  if (cudaEventCreate(&ev) != cudaSuccess) return nullptr;
  return ev;
}

}  // namespace

void note_launch(int n) { g_launches.fetch_add((unsigned long long)n, std::memory_order_relaxed); }

bool profiling_on() { return prof().on; }

void profile_mark_begin(cudaStream_t st) {
  Prof& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (!p.on) return;
  p.pending = take_event(p);
  if (p.pending != nullptr) cudaEventRecord(p.pending, st);
}

void profile_mark_end(cudaStream_t st, int tag) {
  Prof& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (!p.on || p.pending == nullptr) return;
  cudaEvent_t e = take_event(p);
  if (e == nullptr) return;
  cudaEventRecord(e, st);
  p.recs.push_back({p.pending, e, tag});
  p.pending = nullptr;
}

}  // namespace rqlp

using namespace rqlp;

extern "C" {

unsigned long long rqlp_kernel_launches(void) { return g_launches.load(); }

int rqlp_profile_enable(int on) {
  Prof& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  int prev = p.on ? 1 : 0;
  p.on = on != 0;
  return prev;
}

int rqlp_profile_read(float* ms, int* tags, int cap) {
  Prof& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  int n = 0;
  for (const Rec& r : p.recs) {
    if (n < cap) {
      float t = -1.f;
      if (cudaEventSynchronize(r.e) == cudaSuccess) cudaEventElapsedTime(&t, r.b, r.e);
      if (ms != nullptr) ms[n] = t;
      if (tags != nullptr) tags[n] = r.tag;
    }
    ++n;
    p.pool.push_back(r.b);
    p.pool.push_back(r.e);
  }
  p.recs.clear();
  return n < cap ? n : cap;
}

}  // extern "C"
