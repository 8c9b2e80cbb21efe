// profile.cpp - launch counting and optional per-kernel CUDA-event timing.
//
// Every kernel launch of the library goes through prof_begin / prof_end. The
// launch counter is always on (one atomic add). When timing is enabled, each
// launch is bracketed by two events recorded on the launch stream; he_profile_read
// synchronises and accumulates the elapsed times per kernel name.
#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/he_gb300.h"
#include "he_internal.h"

namespace he {

static std::atomic<uint64_t> g_launches{0};
static std::atomic<bool> g_timing{false};
static std::mutex g_mu;

struct Rec {
  const char* name;
  double bytes, products;
  cudaEvent_t a, b;
};
static std::vector<Rec> g_recs;
static std::vector<cudaEvent_t> g_free;

static cudaEvent_t take_event() {
  if (!g_free.empty()) {
    cudaEvent_t e = g_free.back();
    g_free.pop_back();
    return e;
  }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void* prof_begin(const char* name, cudaStream_t st, double bytes, double products) {
  g_launches.fetch_add(1, std::memory_order_relaxed);
  if (!g_timing.load(std::memory_order_relaxed)) return nullptr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  Rec r{name, bytes, products, take_event(), take_event()};
  cudaEventRecord(r.a, st);
  g_recs.push_back(r);
  return (void*)(g_recs.size());
}

void prof_add_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void prof_end(void* tok, cudaStream_t st) {
  if (!tok) return;
  std::lock_guard<std::mutex> lk(g_mu);
  const size_t i = (size_t)tok - 1;
  if (i < g_recs.size()) cudaEventRecord(g_recs[i].b, st);
}

}  // namespace he

using namespace he;

extern "C" {

uint64_t he_kernel_launches(void) { return g_launches.load(); }

int he_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_timing.store(on != 0);
  return HE_OK;
}

int he_profile_read(char* names, size_t names_len, double* ms, uint64_t* counts, double* bytes, double* products,
                    int max_kernels, int* n_kernels) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!n_kernels) return HE_E_ARG;
  std::vector<std::string> nm;
  std::vector<double> t, by, pr;
  std::vector<uint64_t> c;
  for (const Rec& r : g_recs) {
    float e = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&e, r.a, r.b) != cudaSuccess) {
      cudaGetLastError();
      e = 0.f;
    }
    size_t k = 0;
    for (; k < nm.size(); k++)
      if (nm[k] == r.name) break;
    if (k == nm.size()) {
      nm.push_back(r.name);
      t.push_back(0);
      c.push_back(0);
      by.push_back(0);
      pr.push_back(0);
    }
    t[k] += e;
    c[k] += 1;
    by[k] += r.bytes;
    pr[k] += r.products;
    g_free.push_back(r.a);
    g_free.push_back(r.b);
  }
  g_recs.clear();
  *n_kernels = (int)nm.size();
  std::string joined;
  for (size_t k = 0; k < nm.size(); k++) {
    if ((int)k < max_kernels) {
      if (ms) ms[k] = t[k];
      if (counts) counts[k] = c[k];
      if (bytes) bytes[k] = by[k];
      if (products) products[k] = pr[k];
    }
    joined += nm[k];
    joined += '\n';
  }
  if (names && names_len) {
    const size_t n = joined.size() < names_len - 1 ? joined.size() : names_len - 1;
    joined.copy(names, n);
    names[n] = 0;
  }
  return HE_OK;
}

}  // extern "C"
