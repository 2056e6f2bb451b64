// prof.h -- launch counting and CUDA-event timing per kernel family.
#pragma once
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>

#include <map>
#include <string>
#include <vector>

namespace sdpg {

struct ProfPending {
  int fam;
  cudaEvent_t a, b;
  double flops, bytes;
  const char* name;
};

// counters of one named kernel (or launch group)
struct ProfNamed {
  long long launches = 0, timed = 0;
  double ms = 0.0, flops = 0.0, bytes = 0.0;
};

struct Prof {
  bool on = false;
  long long launches[10] = {};
  long long timed[10] = {};
  double ms[10] = {};
  double flops[10] = {};
  double bytes[10] = {};
  std::vector<ProfPending> pending;
  std::vector<cudaEvent_t> pool;
  std::map<std::string, ProfNamed> named;
  cudaEvent_t get() {
    cudaEvent_t e;
    if (!pool.empty()) {
      e = pool.back();
      pool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    return e;
  }
  void flush() {
    for (auto& p : pending) {
      float t = 0.f;
      if (cudaEventSynchronize(p.b) == cudaSuccess && cudaEventElapsedTime(&t, p.a, p.b) == cudaSuccess) {
        ms[p.fam] += t;
        timed[p.fam]++;
        if (p.name && *p.name) {
          ProfNamed& q = named[p.name];
          q.ms += t;
          q.timed++;
          q.flops += p.flops;
          q.bytes += p.bytes;
        }
      }
      pool.push_back(p.a);
      pool.push_back(p.b);
    }
    pending.clear();
  }
};

Prof& prof();

// Bracket one launch of family `fam` on stream `s`.
struct ProfScope {
  int fam;
  cudaStream_t s;
  double fl, by;
  const char* name;
  cudaEvent_t a = nullptr;
  ProfScope(int f, cudaStream_t st, double flops = 0, double bytes = 0, const char* nm = "")
      : fam(f), s(st), fl(flops), by(bytes), name(nm) {
    Prof& P = prof();
    P.launches[fam]++;
    P.flops[fam] += fl;
    P.bytes[fam] += by;
    if (name && *name) P.named[name].launches++;
    if (P.on) {
      a = P.get();
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    Prof& P = prof();
    static const int dbg = getenv("SDP_DEBUG") ? atoi(getenv("SDP_DEBUG")) : 0;
    if (dbg) {  // debugging aid: name the kernel family of the first failing launch
      cudaError_t e = cudaStreamSynchronize(s);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) fprintf(stderr, "[sdpgpu] CUDA error after a launch of family %d (%s): %s\n", fam,
                                    name, cudaGetErrorString(e));
    }
    if (a) {
      cudaEvent_t b = P.get();
      cudaEventRecord(b, s);
      P.pending.push_back({fam, a, b, fl, by, name});
      if (P.pending.size() > 8192) P.flush();
    }
  }
};

}  // namespace sdpg
