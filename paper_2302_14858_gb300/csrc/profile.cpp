// Launch counting and optional per-launch CUDA-event timing (diagnostics).
#include <mutex>
#include <vector>

#include "cfd_internal.h"

namespace cfd {
namespace {

struct Rec {
  int family;
  cudaEvent_t a, b;
};

std::mutex g_mu;
unsigned long long g_launches = 0;
bool g_on = false;
std::vector<Rec> g_open;      // started, not yet ended (per family, last)
std::vector<Rec> g_done;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t get_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

void launch_begin(int family, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  ++g_launches;
  if (!g_on) return;
  Rec r{family, get_event(), nullptr};
  cudaEventRecord(r.a, st);
  g_open.push_back(r);
}

void launch_end(int family, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_on) return;
  for (size_t i = g_open.size(); i-- > 0;) {
    if (g_open[i].family == family) {
      Rec r = g_open[i];
      g_open.erase(g_open.begin() + i);
      r.b = get_event();
      cudaEventRecord(r.b, st);
      g_done.push_back(r);
      return;
    }
  }
}

}  // namespace cfd

using namespace cfd;

extern "C" unsigned long long cfd_kernel_launches(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  return g_launches;
}

extern "C" cfd_status cfd_profile_enable(int on) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (Rec &r : g_done) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_done.clear();
  for (Rec &r : g_open) g_pool.push_back(r.a);
  g_open.clear();
  g_on = on != 0;
  return CFD_OK;
}

extern "C" cfd_status cfd_profile_read(int family, unsigned long long *launches, double *ms) {
  if (family < 0 || family >= KF_COUNT || !launches || !ms) {
    set_error("cfd_profile_read: bad argument");
    return CFD_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  unsigned long long n = 0;
  double t = 0;
  for (Rec &r : g_done) {
    if (r.family != family) continue;
    float e = 0;
    cudaError_t err = cudaEventSynchronize(r.b);
    if (err == cudaSuccess) err = cudaEventElapsedTime(&e, r.a, r.b);
    if (err != cudaSuccess) return cuda_fail(err, "cfd_profile_read");
    ++n;
    t += e;
  }
  *launches = n;
  *ms = t;
  return CFD_OK;
}
