// api.cu -- status reporting and parameter defaults of libkb_b300.so.
#include <atomic>
#include <cmath>
#include <cstring>

#include "kb_internal.cuh"

namespace kb {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

void clear_error() { g_last_error.clear(); }

int fail(int code, const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

static std::atomic<unsigned long long> g_launches{0};
static thread_local cudaEvent_t g_prof_start = nullptr, g_prof_stop = nullptr;

void count_launch(unsigned int n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void profile_events(cudaEvent_t* start, cudaEvent_t* stop) {
  *start = g_prof_start;
  *stop = g_prof_stop;
}

}  // namespace kb

extern "C" unsigned long long kb_launch_count(void) { return kb::g_launches.load(); }

extern "C" void kb_profile_events(void* start, void* stop) {
  kb::g_prof_start = static_cast<cudaEvent_t>(start);
  kb::g_prof_stop = static_cast<cudaEvent_t>(stop);
}

extern "C" int kb_version(void) { return 120; }  // 0.1.2

extern "C" const char* kb_last_error(void) { return kb::g_last_error.c_str(); }

extern "C" void kb_search_params_default(kb_search_params* p, int H, int W) {
  if (!p) return;
  p->k_per_pixel = 8;
  p->lh_min = 10.0f;
  p->min_obs = 15;
  p->clip = 1;
  p->q_lo = 0.25f;
  p->q_mid = 0.5f;
  p->q_hi = 0.75f;
  p->n_sigma = 2.0f;
  p->clip_on = 0;
  p->x_lo = 0;
  p->x_hi = W;
  p->y_lo = 0;
  p->y_hi = H;
}
