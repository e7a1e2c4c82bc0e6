// Optional per-kernel timing: when enabled, every kernel the library enqueues is
// bracketed by a pair of CUDA events on its stream, together with the algorithmic
// bytes and floating-point operations of that launch.  The event pairs are read
// at the synchronisation points the calls already have (the end of a call, and
// each GMRES panel), and accumulated per kernel kind.
#include <mutex>
#include <vector>

#include "rbo_internal.cuh"

namespace rbo {

namespace {
struct Rec {
  cudaEvent_t a, b;
  int kind, tag;
  double bytes, flops;
};
std::mutex mu;
bool enabled = false;
std::vector<Rec> pending;
std::vector<cudaEvent_t> pool;
long long cnt[PROF_KINDS] = {0};
double ms[PROF_KINDS] = {0}, bytes[PROF_KINDS] = {0}, flops[PROF_KINDS] = {0};

cudaEvent_t get_event() {
  if (!pool.empty()) {
    cudaEvent_t e = pool.back();
    pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

bool prof_on() { return enabled; }

ProfToken prof_start(cudaStream_t st) {
  ProfToken t;
  if (!enabled) return t;
  std::lock_guard<std::mutex> lk(mu);
  t.ev = get_event();
  cudaEventRecord((cudaEvent_t)t.ev, st);
  return t;
}

void prof_stop(const ProfToken& t, cudaStream_t st, int kind, double b, double f, int tag) {
  if (!enabled || t.ev == nullptr) return;
  std::lock_guard<std::mutex> lk(mu);
  cudaEvent_t e2 = get_event();
  cudaEventRecord(e2, st);
  pending.push_back(Rec{(cudaEvent_t)t.ev, e2, kind, tag, b, f});
}

void prof_drain() {
  std::lock_guard<std::mutex> lk(mu);
  for (auto& r : pending) {
    float t = 0.f;
    if (cudaEventSynchronize(r.b) == cudaSuccess && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
      for (int k : {r.kind, r.tag >= 0 ? 8 + r.tag : -1}) {
        if (k < 0 || k >= PROF_KINDS) continue;
        cnt[k] += 1;
        ms[k] += t;
        bytes[k] += r.bytes;
        flops[k] += r.flops;
      }
    }
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  pending.clear();
  cudaGetLastError();
}

}  // namespace rbo

extern "C" {

int rbo_profile_enable(int on) {
  rbo::prof_drain();
  rbo::enabled = on != 0;
  return RBO_OK;
}

int rbo_profile_reset(void) {
  rbo::prof_drain();
  std::lock_guard<std::mutex> lk(rbo::mu);
  for (int k = 0; k < rbo::PROF_KINDS; ++k) {
    rbo::cnt[k] = 0;
    rbo::ms[k] = rbo::bytes[k] = rbo::flops[k] = 0.0;
  }
  return RBO_OK;
}

int rbo_profile_read(int32_t kind, int64_t* launches, double* ms, double* bytes, double* flops) {
  if (kind < 0 || kind >= rbo::PROF_KINDS) return RBO_ERR_ARG;
  rbo::prof_drain();
  std::lock_guard<std::mutex> lk(rbo::mu);
  if (launches) *launches = rbo::cnt[kind];
  if (ms) *ms = rbo::ms[kind];
  if (bytes) *bytes = rbo::bytes[kind];
  if (flops) *flops = rbo::flops[kind];
  return RBO_OK;
}

}  // extern "C"
