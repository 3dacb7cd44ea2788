// Optional per-kernel timing with CUDA events recorded on the launching
// stream (enabled by helm_set_profiling).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

namespace helm {

struct Profiler {
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Mark {
    int name;
    cudaEvent_t a, b;
  };
  std::vector<Mark> marks;
  std::vector<std::string> names;
  int open_name = -1;
  cudaEvent_t open_ev = nullptr;

  cudaEvent_t next() {
    if (used == pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      pool.push_back(e);
    }
    return pool[used++];
  }
  void begin(const char* name, cudaStream_t st) {
    if (!on) return;
    int id = -1;
    for (size_t i = 0; i < names.size(); ++i)
      if (names[i] == name) id = (int)i;
    if (id < 0) {
      names.emplace_back(name);
      id = (int)names.size() - 1;
    }
    open_name = id;
    open_ev = next();
    if (open_ev) cudaEventRecord(open_ev, st);
  }
  void end(cudaStream_t st) {
    if (!on || open_name < 0) return;
    cudaEvent_t b = next();
    if (b && open_ev) {
      cudaEventRecord(b, st);
      marks.push_back({open_name, open_ev, b});
    }
    open_name = -1;
  }
  void reset() {
    marks.clear();
    used = 0;
  }
  void destroy() {
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
    marks.clear();
    used = 0;
  }
};

// RAII helper: times one launch when profiling is on.
struct ProfScope {
  Profiler* p;
  cudaStream_t st;
  ProfScope(Profiler* prof, const char* name, cudaStream_t s) : p(prof), st(s) {
    if (p) p->begin(name, st);
  }
  ~ProfScope() {
    if (p) p->end(st);
  }
};

}  // namespace helm
