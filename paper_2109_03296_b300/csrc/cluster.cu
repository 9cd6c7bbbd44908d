// cluster.cu -- de-duplication of candidates (the clustering step of the paper's Fig. 3 pipeline;
// the paper names the step without its algorithm).  In priority order (index 0 first, e.g.
// kb_collect's LH' order) a candidate is kept unless its track agrees within r pixels, at the
// first epoch and at the last, with an already kept candidate.
//
// The greedy order is resolved in parallel rounds.  Candidates are bucketed by their start
// position on a grid of r-sized cells (a duplicate starts within r, so in the same or an adjacent
// cell) and the (cell, index) keys are sorted.  Each round suppresses every candidate with an
// earlier duplicate already kept, and keeps every candidate whose earlier duplicates are all
// decided and none kept; decisions are final, so this is exactly the greedy result (by induction
// over the priority order).  A group of mutual duplicates is settled in two rounds; only chains of
// duplicates that are not duplicates of each other take longer.  A last pass names each
// suppressed candidate's representative, the first kept duplicate.  Distances are compared in float64 with separately rounded operations, the same
// decisions as a plain double-precision loop.
#include <algorithm>

#include "kb_internal.cuh"

namespace kb {

__global__ void bitonic_pass_kernel(unsigned long long* keys, int P, int k, int j);  // collect.cu

constexpr uint8_t CL_UNDECIDED = 0, CL_KEPT = 1, CL_SUPPRESSED = 2, CL_IGNORED = 3;
constexpr int CL_ROUNDS_PER_CHECK = 4;

struct ClusterLayout {
  size_t keys, state0, state1, undecided, total;
  int P;
};

static ClusterLayout cluster_layout(int n) {
  ClusterLayout L{};
  L.P = 2;
  while (L.P < n) L.P <<= 1;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes, KB_WORKSPACE_ALIGN);
    return at;
  };
  L.keys = take(sizeof(unsigned long long) * (size_t)L.P);
  L.state0 = take((size_t)n);
  L.state1 = take((size_t)n);
  L.undecided = take(sizeof(unsigned int) * CL_ROUNDS_PER_CHECK);
  L.total = o;
  return L;
}

// key = cell row (20 bits) | cell column (20 bits) | index (24 bits); padding and ignored
// candidates sort last
__global__ void cluster_keys_kernel(const int32_t* __restrict__ x0, const int32_t* __restrict__ y0,
                                    const uint8_t* __restrict__ valid, int n, double r, int P,
                                    unsigned long long* __restrict__ keys,
                                    uint8_t* __restrict__ state) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  unsigned long long key = ~0ull;
  if (i < n) {
    // candidates outside the 2^20 x 2^20 start-pixel range take no part, like valid[i] == 0
    const bool ok = (!valid || valid[i]) && x0[i] >= 0 && x0[i] < (1 << 20) && y0[i] >= 0 &&
                    y0[i] < (1 << 20);
    state[i] = ok ? CL_UNDECIDED : CL_IGNORED;
    if (ok) {
      const unsigned long long cx = (unsigned long long)floor((double)x0[i] / r);
      const unsigned long long cy = (unsigned long long)floor((double)y0[i] / r);
      key = (cy << 44) | (cx << 24) | (unsigned long long)i;
    }
  }
  keys[i] = key;
}

__device__ __forceinline__ int lower_bound_key(const unsigned long long* keys, int P,
                                               unsigned long long v) {
  int lo = 0, hi = P;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (keys[mid] < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ double sq_dist(double ax, double ay, double bx, double by) {
  const double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by);
  return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
}

// Scans candidate i's earlier duplicates in states st: returns the first kept one (INT_MAX if
// none) and whether any is still undecided.
__device__ __forceinline__ int scan_earlier(const int32_t* __restrict__ x0,
                                            const int32_t* __restrict__ y0,
                                            const float* __restrict__ vx,
                                            const float* __restrict__ vy, int i, double dt,
                                            double r, const unsigned long long* keys, int P,
                                            const uint8_t* __restrict__ st, bool& pending) {
  const double r2 = __dmul_rn(r, r);
  const double xi = (double)x0[i], yi = (double)y0[i];
  const double xi1 = __dadd_rn(xi, __dmul_rn((double)vx[i], dt));
  const double yi1 = __dadd_rn(yi, __dmul_rn((double)vy[i], dt));
  const long long cx = (long long)floor(xi / r), cy = (long long)floor(yi / r);
  int first_kept = INT_MAX;
  for (long long yy = cy - 1; yy <= cy + 1; ++yy) {
    if (yy < 0 || yy >= (1LL << 20)) continue;
    for (long long xx = cx - 1; xx <= cx + 1; ++xx) {
      if (xx < 0 || xx >= (1LL << 20)) continue;
      const unsigned long long base =
          ((unsigned long long)yy << 44) | ((unsigned long long)xx << 24);
      // the cell's candidates in index order; only those before i matter
      for (int e = lower_bound_key(keys, P, base); e < P; ++e) {
        const unsigned long long k = keys[e];
        if ((k >> 24) != (base >> 24)) break;
        const int j = (int)(k & 0xffffffull);
        if (j >= i) break;
        const double xj = (double)x0[j], yj = (double)y0[j];
        if (sq_dist(xi, yi, xj, yj) > r2) continue;
        const double xj1 = __dadd_rn(xj, __dmul_rn((double)vx[j], dt));
        const double yj1 = __dadd_rn(yj, __dmul_rn((double)vy[j], dt));
        if (sq_dist(xi1, yi1, xj1, yj1) > r2) continue;
        const uint8_t sj = st[j];
        if (sj == CL_KEPT) first_kept = min(first_kept, j);
        else if (sj == CL_UNDECIDED) pending = true;
      }
    }
  }
  return first_kept;
}

__global__ void cluster_round_kernel(const int32_t* __restrict__ x0,
                                     const int32_t* __restrict__ y0,
                                     const float* __restrict__ vx, const float* __restrict__ vy,
                                     int n, double dt, double r, const unsigned long long* keys,
                                     int P, const uint8_t* __restrict__ st_in,
                                     uint8_t* __restrict__ st_out, unsigned int* undecided) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint8_t s = st_in[i];
  if (s != CL_UNDECIDED) {
    st_out[i] = s;
    return;
  }
  bool pending = false;
  const int first_kept = scan_earlier(x0, y0, vx, vy, i, dt, r, keys, P, st_in, pending);
  if (first_kept != INT_MAX) {
    st_out[i] = CL_SUPPRESSED;       // an earlier duplicate is kept: final
  } else if (pending) {
    st_out[i] = CL_UNDECIDED;
    atomicAdd(undecided, 1u);
  } else {
    st_out[i] = CL_KEPT;
  }
}

__global__ void cluster_out_kernel(const int32_t* __restrict__ x0, const int32_t* __restrict__ y0,
                                   const float* __restrict__ vx, const float* __restrict__ vy,
                                   int n, double dt, double r, const unsigned long long* keys,
                                   int P, const uint8_t* __restrict__ st,
                                   uint8_t* __restrict__ keep, int32_t* __restrict__ rep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint8_t s = st[i];
  keep[i] = s == CL_KEPT ? 1 : 0;
  if (s == CL_IGNORED) {
    rep[i] = -1;
  } else if (s == CL_KEPT) {
    rep[i] = i;
  } else {
    bool pending = false;
    rep[i] = scan_earlier(x0, y0, vx, vy, i, dt, r, keys, P, st, pending);
  }
}

}  // namespace kb

extern "C" int kb_cluster_workspace_size(int n, size_t* bytes) {
  using namespace kb;
  if (!bytes || n < 0) return fail(KB_ERR_INVALID_ARG, "kb_cluster_workspace_size: bad arguments");
  if (n > (1 << 24)) return fail(KB_ERR_UNSUPPORTED, "kb_cluster_workspace_size: n > 2^24");
  *bytes = cluster_layout(std::max(n, 1)).total;
  return KB_OK;
}

extern "C" int kb_cluster(const int32_t* x0, const int32_t* y0, const float* vx, const float* vy,
                          const uint8_t* valid, int n, double dt, double radius,
                          uint8_t* out_keep, int32_t* out_rep, void* workspace, size_t ws_bytes,
                          int* rounds, void* stream) {
  using namespace kb;
  if (n < 0) return fail(KB_ERR_INVALID_ARG, "kb_cluster: n < 0");
  if (n > (1 << 24)) return fail(KB_ERR_UNSUPPORTED, "kb_cluster: n > 2^24");
  if (!(radius >= 1.0) || !std::isfinite(radius))
    return fail(KB_ERR_INVALID_ARG, "kb_cluster: radius must be finite and >= 1 pixel");
  if (!std::isfinite(dt)) return fail(KB_ERR_INVALID_ARG, "kb_cluster: dt not finite");
  if (rounds) *rounds = 0;
  if (n == 0) return KB_OK;
  if (!x0 || !y0 || !vx || !vy || !out_keep || !out_rep)
    return fail(KB_ERR_INVALID_ARG, "kb_cluster: null pointer argument");
  const ClusterLayout L = cluster_layout(n);
  if (!workspace || ws_bytes < L.total)
    return fail(KB_ERR_WORKSPACE, "kb_cluster: workspace of %zu bytes, %zu needed", ws_bytes, L.total);
  if (reinterpret_cast<uintptr_t>(workspace) % KB_WORKSPACE_ALIGN)
    return fail(KB_ERR_WORKSPACE, "kb_cluster: workspace not %d-byte aligned", KB_WORKSPACE_ALIGN);
  KB_FAULT_POINT("kb_cluster");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  unsigned long long* keys = reinterpret_cast<unsigned long long*>(ws + L.keys);
  uint8_t* s0 = reinterpret_cast<uint8_t*>(ws + L.state0);
  uint8_t* s1 = reinterpret_cast<uint8_t*>(ws + L.state1);
  unsigned int* und = reinterpret_cast<unsigned int*>(ws + L.undecided);
  const int P = L.P;
  cluster_keys_kernel<<<(P + 255) / 256, 256, 0, st>>>(x0, y0, valid, n, radius, P, keys, s0);
  KB_LAUNCH_CHECK("cluster_keys_kernel");
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      bitonic_pass_kernel<<<(P + 255) / 256, 256, 0, st>>>(keys, P, k, j);
      KB_LAUNCH_CHECK("bitonic_pass_kernel");
    }
  // rounds in groups of CL_ROUNDS_PER_CHECK, with one host read of the undecided counts per
  // group; every round decides at least the first undecided candidate, so n rounds suffice
  // (in practice a few: rounds grow only with chains of duplicates that are not mutual)
  int done_rounds = 0;
  for (;;) {
    KB_CUDA_TRY(cudaMemsetAsync(und, 0, sizeof(unsigned int) * CL_ROUNDS_PER_CHECK, st));
    for (int q = 0; q < CL_ROUNDS_PER_CHECK; ++q) {
      cluster_round_kernel<<<(n + 255) / 256, 256, 0, st>>>(x0, y0, vx, vy, n, dt, radius, keys,
                                                            P, s0, s1, und + q);
      KB_LAUNCH_CHECK("cluster_round_kernel");
      std::swap(s0, s1);
    }
    done_rounds += CL_ROUNDS_PER_CHECK;
    unsigned int left[CL_ROUNDS_PER_CHECK];
    KB_CUDA_TRY(cudaMemcpyAsync(left, und, sizeof(left), cudaMemcpyDeviceToHost, st));
    KB_CUDA_TRY(cudaStreamSynchronize(st));
    if (left[CL_ROUNDS_PER_CHECK - 1] == 0u) break;
    if (done_rounds > n + CL_ROUNDS_PER_CHECK)
      return fail(KB_ERR_CUDA, "kb_cluster: no progress after %d rounds", done_rounds);
  }
  if (rounds) *rounds = done_rounds;
  cluster_out_kernel<<<(n + 255) / 256, 256, 0, st>>>(x0, y0, vx, vy, n, dt, radius, keys, P, s0,
                                                      out_keep, out_rep);
  KB_LAUNCH_CHECK("cluster_out_kernel");
  return KB_OK;
}
