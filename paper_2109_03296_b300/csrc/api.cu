// api.cu -- status reporting and parameter defaults of libkb_b300.so.
#include <atomic>
#include <cmath>
#include <cstdlib>
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

bool fault_injected(const char* site) {
  const char* v = std::getenv("KB_FAULT_INJECT");
  if (!v || !*v) return false;
  const size_t n = std::strlen(site);
  for (const char* p = v;;) {
    const char* e = std::strchr(p, ',');
    const size_t len = e ? (size_t)(e - p) : std::strlen(p);
    if ((len == 1 && *p == '*') || (len == n && std::strncmp(p, site, n) == 0)) return true;
    if (!e) return false;
    p = e + 1;
  }
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

extern "C" int kb_version(void) { return 158; }  // 0.1.58

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
  p->bound_rows = 0;
}

// ------------------------------------------------------------------------------------------------
// L2 read probe (measurement utility): reads an L2-resident buffer `reps` times with 16-byte
// loads from a persistent grid; the caller times it (bytes * reps / time = L2 read bandwidth).
// ------------------------------------------------------------------------------------------------
namespace kb {
__global__ void l2_probe_kernel(const float4* __restrict__ buf, size_t n_vec, int reps,
                                float* __restrict__ out) {
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const size_t stride = (size_t)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r)
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_vec; i += stride) {
      const float4 v = __ldcg(buf + i);  // cached in L2 only
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
  const float s = acc.x + acc.y + acc.z + acc.w;
  if (s == 1.2345678e-30f) out[blockIdx.x] = s;  // keeps the loads; never true for the probe data
}
}  // namespace kb

// ------------------------------------------------------------------------------------------------
// Shared-memory read probe (measurement utility): every warp streams conflict-free 32-bit
// shared loads (lane-contiguous words, one 128-byte wavefront per instruction), the access the
// search kernel's bound pass makes; the caller times it.
// ------------------------------------------------------------------------------------------------
namespace kb {
constexpr int kSmemProbeThreads = 1024;
__global__ void __launch_bounds__(kSmemProbeThreads) smem_probe_kernel(int iters,
                                                                       unsigned int* out) {
  __shared__ __align__(16) unsigned int buf[8192];  // 32 KB
  for (int i = threadIdx.x; i < 8192; i += blockDim.x) buf[i] = (unsigned int)i * 2654435761u;
  __syncthreads();
  const unsigned int base =
      static_cast<unsigned int>(__cvta_generic_to_shared(buf)) + (threadIdx.x & 31) * 4u;
  unsigned int acc[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  for (int it = 0; it < iters; ++it) {
    const unsigned int b = base + (unsigned int)(it & 7) * 4096u;
#pragma unroll
    for (int u = 0; u < 32; ++u) {
      unsigned int v;
      asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(b + (unsigned int)u * 128u));
      acc[u & 7] += v;
    }
  }
  unsigned int s = 0u;
#pragma unroll
  for (int k = 0; k < 8; ++k) s ^= acc[k];
  if (s == 0x9e3779b9u && threadIdx.x == 0) out[blockIdx.x] = s;  // keeps the loads
}
}  // namespace kb

extern "C" int kb_smem_probe(int blocks, int iters, unsigned int* scratch, void* stream) {
  using namespace kb;
  if (!scratch || blocks < 1 || iters < 1)
    return fail(KB_ERR_INVALID_ARG, "kb_smem_probe: bad arguments");
  smem_probe_kernel<<<blocks, kSmemProbeThreads, 0, static_cast<cudaStream_t>(stream)>>>(iters,
                                                                                        scratch);
  KB_LAUNCH_CHECK("smem_probe_kernel");
  return KB_OK;
}

extern "C" int kb_l2_probe(const void* buf, size_t bytes, int reps, float* scratch, int blocks,
                           void* stream) {
  using namespace kb;
  if (!buf || !scratch || bytes < 16 || reps < 1 || blocks < 1)
    return fail(KB_ERR_INVALID_ARG, "kb_l2_probe: bad arguments");
  if (reinterpret_cast<uintptr_t>(buf) % 16)
    return fail(KB_ERR_INVALID_ARG, "kb_l2_probe: buffer not 16-byte aligned");
  l2_probe_kernel<<<blocks, 512, 0, static_cast<cudaStream_t>(stream)>>>(
      static_cast<const float4*>(buf), bytes / 16, reps, scratch);
  KB_LAUNCH_CHECK("l2_probe_kernel");
  return KB_OK;
}
