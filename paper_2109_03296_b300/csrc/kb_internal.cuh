// kb_internal.cuh -- helpers shared by the kernels of libkb_b300.so (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "../../include/kb.h"

namespace kb {

// ---------------------------------------------------------------------------------------------
// Host-side status handling: every entry point returns a kb_status and records a message.
// ---------------------------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();
int fail(int code, const char* fmt, ...);

#define KB_CUDA_TRY(expr)                                                              \
  do {                                                                                 \
    cudaError_t _e = (expr);                                                           \
    if (_e != cudaSuccess)                                                             \
      return ::kb::fail(KB_ERR_CUDA, "%s failed: %s", #expr, cudaGetErrorString(_e));  \
  } while (0)

void count_launch(unsigned int n = 1);
void profile_events(cudaEvent_t* start, cudaEvent_t* stop);

#define KB_LAUNCH_CHECK(what)                                                          \
  do {                                                                                 \
    ::kb::count_launch();                                                              \
    cudaError_t _e = cudaGetLastError();                                               \
    if (_e != cudaSuccess)                                                             \
      return ::kb::fail(KB_ERR_CUDA, "launch of %s failed: %s", what,                  \
                        cudaGetErrorString(_e));                                       \
  } while (0)

// Host-side fault injection for tests of the callers' failure handling: an entry point named in
// the environment variable KB_FAULT_INJECT (a comma-separated list of entry-point names, or "*"
// for all) fails with KB_ERR_CUDA after validating its arguments and before any device work.
bool fault_injected(const char* site);

#define KB_FAULT_POINT(site)                                                           \
  do {                                                                                 \
    if (::kb::fault_injected(site))                                                    \
      return ::kb::fail(KB_ERR_CUDA, "%s: injected fault (KB_FAULT_INJECT)", site);    \
  } while (0)

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Device error flag bits (kb_search_stats()[3]).
constexpr unsigned int kErrTimeout = 0x1u;
constexpr unsigned int kErrBounds = 0x2u;  // a device-side check of the checked build failed

// The checked build (nvcc -DKB_BOUNDS_CHECK=1: libkb_b300_checked.so) tests, before each access,
// that a staged-box read lies inside the box, that a TMA x coordinate is 16-byte aligned and
// that a result slot lies inside the output window; a failed check sets kErrBounds and skips
// the access.  The regular build compiles the checks away.
#ifndef KB_BOUNDS_CHECK
#define KB_BOUNDS_CHECK 0
#endif

// Every device-side wait is bounded in time: after this many nanoseconds of %globaltimer the
// waiter gives up, records an error flag and stops using the buffer it waited for.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;

// ---------------------------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile(
      "mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
      "r"(bytes)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity, uint32_t hint_ns) {
  uint32_t done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity), "r"(hint_ns)
      : "memory");
  return done != 0u;
}

// Returns true once the phase with the given parity has completed, false after limit_ns
// (the caller records the timeout and stops using the buffer).  Each attempt may suspend the
// thread for up to 20 us, so a waiting warp issues few instructions.
__device__ __forceinline__ bool mbar_wait_parity(uint64_t* bar, uint32_t parity,
                                                 unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity, 20000u)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity, 20000u)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

// 3-D tiled TMA load (global -> shared), completion signalled on an mbarrier as tx bytes.
__device__ __forceinline__ void tma_load_3d(void* smem_dst, const void* tmap, uint64_t* bar,
                                            int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(smem_u32(bar)), "r"(x), "r"(y), "r"(z)
      : "memory");
}

// 1-D bulk copy global -> shared (16-byte aligned addresses, size a multiple of 16), completion
// signalled on an mbarrier as tx bytes.
__device__ __forceinline__ void bulk_copy_g2s(void* smem_dst, const void* gsrc, uint32_t bytes,
                                              uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(gsrc)), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const void* tmap) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(tmap)) : "memory");
}

}  // namespace kb
