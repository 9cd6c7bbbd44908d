// collect.cu -- device-side handoff of the search survivors (Section 3.1 reworked GPU -> Python
// handoff; Section 3.2 results returned per start pixel): every filled slot of the per-pixel
// lists is keyed by (LH' descending, slot position ascending) as one 64-bit integer, the n_max
// smallest keys are found by an exact 8-pass radix select (8 bits per pass), gathered, and
// sorted with a bitonic network.  No host synchronisation: the survivor count stays on the
// device until the caller reads it.
#include <algorithm>

#include "kb_internal.cuh"

namespace kb {

struct SelState {
  unsigned long long prefix;  // key bits fixed so far
  unsigned long long mask;    // which bits are fixed
  unsigned int remaining;     // how many keys still to take among those matching prefix
  unsigned int count;         // filled slots
  unsigned int take_all;      // count <= n_max
  unsigned int ngathered;
};

__device__ __forceinline__ unsigned long long slot_key(float L, uint32_t pos) {
  uint32_t u = __float_as_uint(L);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);  // order-preserving map to unsigned
  return ((unsigned long long)(~u) << 32) | pos;   // LH' descending, then position
}

struct CollectLayout {
  size_t state, hist, keys, total;
  int P;
};

static CollectLayout collect_layout(int n_max) {
  CollectLayout L{};
  int P = 1;
  while (P < n_max) P <<= 1;
  L.P = P;
  size_t o = 0;
  L.state = o;
  o = align_up(o + sizeof(SelState), KB_WORKSPACE_ALIGN);
  L.hist = o;
  o = align_up(o + 256 * sizeof(unsigned int), KB_WORKSPACE_ALIGN);
  L.keys = o;
  o = align_up(o + (size_t)P * sizeof(unsigned long long), KB_WORKSPACE_ALIGN);
  L.total = o;
  return L;
}

__global__ void sel_init_kernel(SelState* s, unsigned int* hist, unsigned long long* keys, int P) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 256) hist[i] = 0u;
  if (i == 0) {
    s->prefix = 0ull;
    s->mask = 0ull;
    s->remaining = 0u;
    s->count = 0u;
    s->take_all = 0u;
    s->ngathered = 0u;
  }
  for (int k = i; k < P; k += gridDim.x * blockDim.x) keys[k] = ~0ull;
}

__global__ void sel_hist_kernel(const float* __restrict__ lh, const int32_t* __restrict__ idx,
                                size_t nslots, int pass, SelState* s, unsigned int* hist) {
  __shared__ unsigned int h[256];
  __shared__ unsigned int cnt;
  if (pass > 0 && s->take_all) return;
  for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0u;
  if (threadIdx.x == 0) cnt = 0u;
  __syncthreads();
  const unsigned long long prefix = s->prefix, mask = s->mask;
  const int shift = 56 - 8 * pass;
  unsigned int mycnt = 0u;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslots;
       i += (size_t)gridDim.x * blockDim.x) {
    if (idx[i] < 0) continue;
    ++mycnt;
    const unsigned long long key = slot_key(lh[i], (uint32_t)i);
    if ((key & mask) == prefix) atomicAdd(&h[(key >> shift) & 0xffu], 1u);
  }
  if (pass == 0 && mycnt) atomicAdd(&cnt, mycnt);
  __syncthreads();
  for (int i = threadIdx.x; i < 256; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
  if (pass == 0 && threadIdx.x == 0 && cnt) atomicAdd(&s->count, cnt);
}

// One warp: fix the next 8 bits of the n_max-th smallest key.
__global__ void sel_pick_kernel(int pass, int n_max, SelState* s, unsigned int* hist) {
  const int lane = threadIdx.x;
  if (pass == 0) {
    if (lane == 0) {
      s->take_all = s->count <= (unsigned int)n_max ? 1u : 0u;
      s->remaining = (unsigned int)n_max;
    }
    __syncwarp();
  }
  if (s->take_all) {
    for (int i = lane; i < 256; i += 32) hist[i] = 0u;
    return;
  }
  if (lane == 0) {
    const int shift = 56 - 8 * pass;
    unsigned int rem = s->remaining, cum = 0u;
    int d = 0;
    for (; d < 256; ++d) {
      if (cum + hist[d] >= rem) break;
      cum += hist[d];
    }
    if (d > 255) d = 255;
    s->remaining = rem - cum;
    s->prefix |= (unsigned long long)d << shift;
    s->mask |= 0xffull << shift;
  }
  __syncwarp();
  for (int i = lane; i < 256; i += 32) hist[i] = 0u;
}

__global__ void sel_gather_kernel(const float* __restrict__ lh, const int32_t* __restrict__ idx,
                                  size_t nslots, int P, SelState* s, unsigned long long* keys) {
  const bool all = s->take_all != 0u;
  const unsigned long long thr = s->prefix;  // after 8 passes: the n_max-th smallest key
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < nslots;
       i += (size_t)gridDim.x * blockDim.x) {
    if (idx[i] < 0) continue;
    const unsigned long long key = slot_key(lh[i], (uint32_t)i);
    if (all || key <= thr) {
      const unsigned int at = atomicAdd(&s->ngathered, 1u);
      if (at < (unsigned int)P) keys[at] = key;
    }
  }
}

__global__ void bitonic_pass_kernel(unsigned long long* keys, int P, int k, int j) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const int p = i ^ j;
  if (p <= i) return;
  const unsigned long long a = keys[i], b = keys[p];
  const bool up = (i & k) == 0;
  if ((a > b) == up) {
    keys[i] = b;
    keys[p] = a;
  }
}

__global__ void sel_write_kernel(const unsigned long long* __restrict__ keys, int n_max, int K,
                                 const SelState* s, int32_t* cand_pix, int32_t* cand_slot,
                                 int32_t* count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *count = (int32_t)s->count;
  if (i >= n_max) return;
  const unsigned long long key = keys[i];
  if (key == ~0ull) {
    cand_pix[i] = -1;
    cand_slot[i] = -1;
  } else {
    const uint32_t pos = (uint32_t)(key & 0xffffffffull);
    cand_pix[i] = (int32_t)(pos / (uint32_t)K);
    cand_slot[i] = (int32_t)(pos % (uint32_t)K);
  }
}

__global__ void candidate_tracks_kernel(const int32_t* __restrict__ cand_pix,
                                        const int32_t* __restrict__ cand_slot, int n,
                                        const int32_t* __restrict__ idx, int K,
                                        const float* __restrict__ vx, const float* __restrict__ vy,
                                        int x_lo, int y_lo, int wx, int32_t* x0, int32_t* y0,
                                        float* ovx, float* ovy, int32_t* traj) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int p = cand_pix[i];
  if (p < 0) {
    x0[i] = -(1 << 28);
    y0[i] = -(1 << 28);
    ovx[i] = 0.0f;
    ovy[i] = 0.0f;
    traj[i] = -1;
    return;
  }
  const int j = idx[(size_t)p * K + cand_slot[i]];
  x0[i] = x_lo + p % wx;
  y0[i] = y_lo + p / wx;
  traj[i] = j;
  ovx[i] = j >= 0 ? vx[j] : 0.0f;
  ovy[i] = j >= 0 ? vy[j] : 0.0f;
}

}  // namespace kb

extern "C" int kb_candidate_tracks(const int32_t* cand_pix, const int32_t* cand_slot, int n,
                                   const int32_t* idx, int K, const float* vx, const float* vy,
                                   int x_lo, int y_lo, int wx, int32_t* x0, int32_t* y0,
                                   float* out_vx, float* out_vy, int32_t* traj, void* stream) {
  using namespace kb;
  if (n < 0 || K < 1 || K > KB_MAX_K || wx < 1)
    return fail(KB_ERR_INVALID_ARG, "kb_candidate_tracks: bad sizes");
  if (n == 0) return KB_OK;
  if (!cand_pix || !cand_slot || !idx || !vx || !vy || !x0 || !y0 || !out_vx || !out_vy || !traj)
    return fail(KB_ERR_INVALID_ARG, "kb_candidate_tracks: null pointer argument");
  KB_FAULT_POINT("kb_candidate_tracks");
  candidate_tracks_kernel<<<(n + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(
      cand_pix, cand_slot, n, idx, K, vx, vy, x_lo, y_lo, wx, x0, y0, out_vx, out_vy, traj);
  KB_LAUNCH_CHECK("candidate_tracks_kernel");
  return KB_OK;
}

extern "C" int kb_collect_workspace_size(int n_max, size_t* bytes) {
  using namespace kb;
  if (!bytes) return fail(KB_ERR_INVALID_ARG, "kb_collect_workspace_size: null pointer");
  if (n_max < 1) return fail(KB_ERR_INVALID_ARG, "kb_collect_workspace_size: n_max < 1");
  if (n_max > (1 << 24)) return fail(KB_ERR_UNSUPPORTED, "kb_collect_workspace_size: n_max > 2^24");
  *bytes = collect_layout(n_max).total;
  return KB_OK;
}

extern "C" int kb_collect(const float* lh, const int32_t* idx, int npix, int K, int n_max,
                          int32_t* cand_pix, int32_t* cand_slot, int32_t* count, void* workspace,
                          size_t ws_bytes, void* stream) {
  using namespace kb;
  if (!lh || !idx || !cand_pix || !cand_slot || !count)
    return fail(KB_ERR_INVALID_ARG, "kb_collect: null pointer argument");
  if (npix < 1 || K < 1 || K > KB_MAX_K || n_max < 1)
    return fail(KB_ERR_INVALID_ARG, "kb_collect: bad sizes");
  if ((unsigned long long)npix * K >= (1ull << 32))
    return fail(KB_ERR_UNSUPPORTED, "kb_collect: more than 2^32 slots");
  if (n_max > (1 << 24)) return fail(KB_ERR_UNSUPPORTED, "kb_collect: n_max > 2^24");
  const CollectLayout L = collect_layout(n_max);
  if (!workspace || ws_bytes < L.total)
    return fail(KB_ERR_WORKSPACE, "kb_collect: workspace of %zu bytes, %zu needed", ws_bytes, L.total);
  if (reinterpret_cast<uintptr_t>(workspace) % KB_WORKSPACE_ALIGN)
    return fail(KB_ERR_WORKSPACE, "kb_collect: workspace not aligned");
  KB_FAULT_POINT("kb_collect");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  SelState* s = reinterpret_cast<SelState*>(ws + L.state);
  unsigned int* hist = reinterpret_cast<unsigned int*>(ws + L.hist);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(ws + L.keys);
  const size_t nslots = (size_t)npix * K;
  int sms = 0, dev = 0;
  KB_CUDA_TRY(cudaGetDevice(&dev));
  KB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)std::min<size_t>((nslots + 255) / 256, (size_t)sms * 8);
  sel_init_kernel<<<std::max(1, std::min((L.P + 255) / 256, sms * 8)), 256, 0, st>>>(s, hist, keys, L.P);
  KB_LAUNCH_CHECK("sel_init_kernel");
  for (int pass = 0; pass < 8; ++pass) {
    sel_hist_kernel<<<grid, 256, 0, st>>>(lh, idx, nslots, pass, s, hist);
    KB_LAUNCH_CHECK("sel_hist_kernel");
    sel_pick_kernel<<<1, 32, 0, st>>>(pass, n_max, s, hist);
    KB_LAUNCH_CHECK("sel_pick_kernel");
  }
  sel_gather_kernel<<<grid, 256, 0, st>>>(lh, idx, nslots, L.P, s, keys);
  KB_LAUNCH_CHECK("sel_gather_kernel");
  for (int k = 2; k <= L.P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      bitonic_pass_kernel<<<(L.P + 255) / 256, 256, 0, st>>>(keys, L.P, k, j);
      KB_LAUNCH_CHECK("bitonic_pass_kernel");
    }
  sel_write_kernel<<<(n_max + 255) / 256, 256, 0, st>>>(keys, n_max, K, s, cand_pix, cand_slot, count);
  KB_LAUNCH_CHECK("sel_write_kernel");
  return KB_OK;
}
