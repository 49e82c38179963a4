// Opt-in per-kernel timing: while profiling is on, every kernel launch made by
// the library is bracketed by two CUDA events on its stream; sc_profile_end()
// waits for them and sums the elapsed time per kernel kind.  Off by default
// (then the only cost is one atomic increment of the launch counter).
#include <atomic>
#include <mutex>
#include <vector>

#include "sc_common.cuh"

namespace sc {

namespace {
struct Rec {
  int kind;
  cudaEvent_t a, b;
};
std::mutex g_mu;
bool g_on = false;
std::vector<cudaEvent_t> g_pool;
size_t g_used = 0;
std::vector<Rec> g_recs;
std::vector<Rec> g_open;  // one open record per kind (launches of one kind do not nest)
double g_ms[PK_COUNT];
long g_n[PK_COUNT];
std::atomic<unsigned long long> g_launches{0};

cudaEvent_t take_event() {
  if (g_used == g_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    g_pool.push_back(e);
  }
  return g_pool[g_used++];
}
}  // namespace

void prof_start(int kind, cudaStream_t st) {
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  cudaEvent_t a = take_event();
  if (!a) return;
  cudaEventRecord(a, st);
  g_open.push_back(Rec{kind, a, nullptr});
}

void prof_stop(int kind, cudaStream_t st) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_on) return;
  std::lock_guard<std::mutex> lk(g_mu);
  for (size_t i = g_open.size(); i-- > 0;) {
    if (g_open[i].kind == kind) {
      cudaEvent_t b = take_event();
      if (!b) return;
      cudaEventRecord(b, st);
      g_recs.push_back(Rec{kind, g_open[i].a, b});
      g_open.erase(g_open.begin() + i);
      return;
    }
  }
}

unsigned long long launch_count() { return g_launches.load(); }

void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

bool prof_active() {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_on;
}

int prof_begin() {
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.clear();
  g_open.clear();
  g_used = 0;
  for (int k = 0; k < PK_COUNT; ++k) {
    g_ms[k] = 0.0;
    g_n[k] = 0;
  }
  g_on = true;
  return 0;
}

int prof_end() {
  std::lock_guard<std::mutex> lk(g_mu);
  g_on = false;
  for (const Rec& r : g_recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) return -1;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return -1;
    g_ms[r.kind] += ms;
    g_n[r.kind] += 1;
  }
  g_recs.clear();
  g_open.clear();
  g_used = 0;
  return 0;
}

void prof_read(int kind, long* n, double* ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  *n = g_n[kind];
  *ms = g_ms[kind];
}

}  // namespace sc
