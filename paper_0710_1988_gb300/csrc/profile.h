// Optional per-handle kernel timing (CUDA events on the launching stream).
//
// An API entry point installs the handle's profiler as the thread's current
// one (ProfScope); every launch wrapper brackets its launch with a ProfLaunch,
// which records an event pair when profiling is on for that kernel category
// and costs one branch otherwise.  Event pairs are resolved when the handle's
// counters are read, or when the pending list grows past a bound.
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/wd.h"

namespace wd {

enum ProfCat {
  PC_DSLASH = 0, PC_STREAM = 1, PC_TS = 2, PC_DENSE = 3, PC_DSLASH_LOW = 4, PC_STREAM_LOW = 5,
  PC_COUNT = 6
};

struct Profiler {
  unsigned mask = 0;              // categories being recorded
  struct Rec {
    int cat;
    cudaEvent_t a, b;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> spare;
  long long launches[PC_COUNT] = {0, 0, 0, 0, 0, 0};
  double ms[PC_COUNT] = {0, 0, 0, 0, 0, 0};
  // device counters of sites x systems processed: [0] FP64 dslash,
  // [1] FP32/FP16 dslash
  unsigned long long *d_sites = nullptr;
  cudaEvent_t take();
  void flush();                   // synchronises the pending events and accumulates
  void reset();
  void destroy();
};

Profiler *current_profiler();
void set_current_profiler(Profiler *p);

struct ProfScope {
  Profiler *prev;
  explicit ProfScope(Profiler *p) : prev(current_profiler()) { set_current_profiler(p); }
  ~ProfScope() { set_current_profiler(prev); }
};

struct ProfLaunch {
  Profiler *p = nullptr;
  int cat;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfLaunch(int c, cudaStream_t st) : cat(c), s(st) {
    Profiler *q = current_profiler();
    if (q != nullptr && ((q->mask >> c) & 1u)) {
      p = q;
      a = p->take();
      cudaEventRecord(a, s);
    }
  }
  ~ProfLaunch() {
    if (p == nullptr) return;
    cudaEvent_t b = p->take();
    cudaEventRecord(b, s);
    p->pending.push_back({cat, a, b});
    if (p->pending.size() >= 16384) p->flush();
  }
};

// Device counters of dslash work (nullptr unless that category is profiled).
inline unsigned long long *prof_site_counter() {
  Profiler *q = current_profiler();
  return (q != nullptr && ((q->mask >> PC_DSLASH) & 1u)) ? q->d_sites : nullptr;
}
inline unsigned long long *prof_site_counter_low() {
  Profiler *q = current_profiler();
  return (q != nullptr && ((q->mask >> PC_DSLASH_LOW) & 1u)) ? q->d_sites + 1 : nullptr;
}

}  // namespace wd
