// search.cu -- integer-pixel shift-and-stack search with the in-line sigma-G clip and the
// per-start-pixel top-K (Section 3 pointer arithmetic, Section 3.1 clip and LH', Section 3.2
// in-line filtering before the per-pixel selection).
//
// Design (B300, sm_103a):
//
//  * Exact pruning bound.  For any subset S of a trajectory's valid epochs (in particular the
//    epochs the sigma-G clip keeps), Cauchy-Schwarz gives
//        LH'(S) = sum_S psi / sqrt(sum_S phi) <= sqrt( sum_{valid, psi>0} psi^2 / phi ).
//    So a (start pixel, trajectory) pair can only enter a top-K list if that bound reaches the
//    list's current admission threshold (lh_min, or the K-th LH' once the list is full).  The
//    search therefore runs in two levels:
//      1. bound pass: B(p, j) = sum_t nu2[t, p + d_t(j)] with nu2 = psi^2/phi (psi > 0, valid),
//         one float load + one add per trajectory-epoch;
//      2. full evaluation of the few pairs whose bound reaches the threshold: gather psi/phi,
//         sigma-G clip, LH', alpha, then insertion into the pixel's list.
//    Pairs are dropped only when B < thr^2 (1 - 1e-4); the FP32 rounding of B is far below that
//    margin, so the output equals evaluating every pair.
//
//  * Bound pass layout.  nu2 is written once per call into the workspace as [T][H][Wp] float32
//    (Wp = W rounded up to 32, zero padded) so that a 3-D TMA tensor map can address it.  A
//    block owns a tile of 32 x 64 start pixels (lane = x, 8 rows per thread) and sweeps the
//    velocity list in chunks of 16 trajectories that are close in velocity space (the list is
//    reordered by a Morton key of (vx, vy) in the plan kernels).  For each (chunk, epoch) the
//    union of the tile's 16 shifted footprints is one small rectangle; it is fetched with TMA
//    into a double-buffered shared-memory stage (zero fill outside the image) while the
//    previous epoch is being summed.  Each thread then does 8 x 16 shared loads + adds per
//    epoch with immediate row offsets.  A (chunk, epoch) rectangle too large for a stage falls
//    back to direct global loads.
//
//  * Full evaluation.  After each chunk, the block queues the pairs whose bound passes; one
//    warp evaluates one pair with lanes over epochs (up to 4 epochs per lane): gather, validity
//    ballot, warp bitonic sort of the lightcurve for the three percentiles, clip, butterfly sums
//    (same order for identical inputs, so identical tracks give bit-identical LH').  The owner
//    thread of the start pixel then inserts the result into the pixel's list in the output
//    arrays (LH' descending, trajectory index ascending).
#include <cuda.h>
#include <cudaTypedefs.h>

#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "kb_internal.cuh"

namespace kb {

// ---------------------------------------------------------------------------------------------
// Compile-time configuration of the search kernel
// ---------------------------------------------------------------------------------------------
constexpr int S_TX = 32;                 // tile width (lane = x)
constexpr int S_ROWS = 8;                // rows per thread
constexpr int S_WARPS = 8;
constexpr int S_THREADS = S_WARPS * 32;  // 256
constexpr int S_TY = S_WARPS * S_ROWS;   // 64
constexpr int S_C = 16;                  // trajectories per chunk
constexpr int S_PITCH = 128;             // staged row pitch in floats (= TMA box width)
constexpr int S_BOX_Y = 8;               // TMA box height
constexpr int S_CAP_ROWS = 128;          // staged rows per stage
constexpr int S_STAGE_FLOATS = S_CAP_ROWS * S_PITCH;
constexpr int S_QCAP = 1024;             // queued full evaluations per round
constexpr int S_REC_WORDS = 8;           // L', alpha, nvalid|nkept<<16, mask[4], pad
constexpr float S_PRUNE_MARGIN = 1.0f - 1e-4f;

constexpr int MORTON_BITS = 8;           // per axis: 256 x 256 velocity cells
constexpr int N_CELLS = 1 << (2 * MORTON_BITS);

struct SearchConsts {
  float dt[KB_MAX_T];   // (float)(t_t - t_0)
};

struct EvalParams {
  int T, H, W, min_obs, clip, clip_on, K, mw;
  float q_lo, q_mid, q_hi, n_sigma, c_sigma, lh_min;
};

// Workspace layout (offsets in bytes from the workspace base).
struct WsLayout {
  size_t ctrl, vbox, keys, counts, cursor, sorted, orig, offs, box, rel, bound, total;
  int n_pad, nchunk, Wp;
};

static WsLayout ws_layout(int T, int H, int W, int n_traj) {
  WsLayout L{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes, KB_WORKSPACE_ALIGN);
    return at;
  };
  L.n_pad = (n_traj + S_C - 1) / S_C * S_C;
  L.nchunk = L.n_pad / S_C;
  L.Wp = (W + 31) / 32 * 32;
  L.ctrl = take(256);
  L.vbox = take(16);
  L.keys = take(sizeof(uint32_t) * (size_t)n_traj);
  L.counts = take(sizeof(uint32_t) * N_CELLS);
  L.cursor = take(sizeof(uint32_t) * N_CELLS);
  L.sorted = take(sizeof(int32_t) * (size_t)n_traj);
  L.orig = take(sizeof(int32_t) * (size_t)L.n_pad);
  L.offs = take(sizeof(int2) * (size_t)L.n_pad * T);
  L.box = take(sizeof(int4) * (size_t)L.nchunk * T);
  L.rel = take(sizeof(int32_t) * (size_t)L.nchunk * T * S_C);
  L.bound = take(sizeof(float) * (size_t)T * H * L.Wp);
  L.total = o;
  return L;
}

// ctrl block: [0] error flags (u32), [8] stats: te, evals, inserts (u64 each)
struct Ctrl {
  unsigned int err;
  unsigned int pad;
  unsigned long long te, evals, inserts;
};

// ---------------------------------------------------------------------------------------------
// Plan kernels: velocity ordering, track offsets, per-(chunk, epoch) staging rectangles
// ---------------------------------------------------------------------------------------------
__global__ void plan_reset_kernel(Ctrl* ctrl, uint32_t* counts, unsigned long long te) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N_CELLS) counts[i] = 0u;
  if (i == 0) {
    ctrl->err = 0u;
    ctrl->te = te;
    ctrl->evals = 0ull;
    ctrl->inserts = 0ull;
  }
}

__global__ void __launch_bounds__(1024) plan_minmax_kernel(const float* __restrict__ vx, const float* __restrict__ vy,
                                   int n, float4* vbox) {
  __shared__ float s[4][32];
  float a = INFINITY, b = -INFINITY, c = INFINITY, d = -INFINITY;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float x = vx[i], y = vy[i];
    a = fminf(a, x); b = fmaxf(b, x); c = fminf(c, y); d = fmaxf(d, y);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = fminf(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = fmaxf(b, __shfl_xor_sync(0xffffffffu, b, o));
    c = fminf(c, __shfl_xor_sync(0xffffffffu, c, o));
    d = fmaxf(d, __shfl_xor_sync(0xffffffffu, d, o));
  }
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { s[0][w] = a; s[1][w] = b; s[2][w] = c; s[3][w] = d; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nw = blockDim.x >> 5;
    for (int i = 1; i < nw; ++i) {
      a = fminf(a, s[0][i]); b = fmaxf(b, s[1][i]); c = fminf(c, s[2][i]); d = fmaxf(d, s[3][i]);
    }
    *vbox = make_float4(a, b, c, d);
  }
}

__device__ __forceinline__ uint32_t spread_bits8(uint32_t v) {
  v &= 0xffu;
  v = (v | (v << 4)) & 0x0f0fu;
  v = (v | (v << 2)) & 0x3333u;
  v = (v | (v << 1)) & 0x5555u;
  return v;
}

__global__ void plan_hist_kernel(const float* __restrict__ vx, const float* __restrict__ vy,
                                 int n, const float4* vbox, uint32_t* keys, uint32_t* counts) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 b = *vbox;
  const float cells = (float)(1 << MORTON_BITS);
  float sx = (b.y > b.x) ? cells / (b.y - b.x) : 0.0f;
  float sy = (b.w > b.z) ? cells / (b.w - b.z) : 0.0f;
  int qx = min((int)((vx[i] - b.x) * sx), (1 << MORTON_BITS) - 1);
  int qy = min((int)((vy[i] - b.z) * sy), (1 << MORTON_BITS) - 1);
  qx = max(qx, 0);
  qy = max(qy, 0);
  uint32_t key = spread_bits8((uint32_t)qx) | (spread_bits8((uint32_t)qy) << 1);
  keys[i] = key;
  atomicAdd(&counts[key], 1u);
}

// Exclusive scan of N_CELLS counts by one block of 1024 threads (64 consecutive cells each).
__global__ void __launch_bounds__(1024) plan_scan_kernel(const uint32_t* __restrict__ counts,
                                                         uint32_t* cursor) {
  __shared__ uint32_t part[1024];
  constexpr int PER = N_CELLS / 1024;
  int t = threadIdx.x;
  uint32_t s = 0;
  for (int i = 0; i < PER; ++i) s += counts[t * PER + i];
  part[t] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    uint32_t v = t >= o ? part[t - o] : 0u;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  uint32_t base = part[t] - s;
  for (int i = 0; i < PER; ++i) {
    cursor[t * PER + i] = base;
    base += counts[t * PER + i];
  }
}

__global__ void plan_scatter_kernel(const uint32_t* __restrict__ keys, int n, uint32_t* cursor,
                                    int32_t* sorted) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t pos = atomicAdd(&cursor[keys[i]], 1u);
  sorted[pos] = i;
}

// After the scatter, cursor[c] is the end of cell c's segment and counts[c] its length; sort each
// segment by trajectory index so that the order is deterministic.
__global__ void plan_cellsort_kernel(const uint32_t* __restrict__ counts,
                                     const uint32_t* __restrict__ cursor, int32_t* sorted) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= N_CELLS) return;
  uint32_t len = counts[c];
  if (len < 2) return;
  uint32_t end = cursor[c], beg = end - len;
  for (uint32_t i = beg + 1; i < end; ++i) {
    int32_t v = sorted[i];
    uint32_t j = i;
    while (j > beg && sorted[j - 1] > v) {
      sorted[j] = sorted[j - 1];
      --j;
    }
    sorted[j] = v;
  }
}

// Offsets are clamped to +-2^24: images are at most 2^20 pixels on a side, so a clamped position
// is outside the image exactly when the unclamped one is, and no later sum can overflow int32.
constexpr float kMaxOffset = 16777216.0f;

__device__ __forceinline__ int track_offset(float v, float dt) {
  // one IEEE float32 multiply, one IEEE float32 add, floor: round half up
  const float d = floorf(__fadd_rn(__fmul_rn(v, dt), 0.5f));
  return (int)fminf(fmaxf(d, -kMaxOffset), kMaxOffset);  // NaN -> -2^24 (off the image)
}

__global__ void plan_offsets_kernel(const float* __restrict__ vx, const float* __restrict__ vy,
                                    const int32_t* __restrict__ sorted, int n, int n_pad, int T,
                                    SearchConsts cs, int32_t* orig, int2* offs) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_pad) return;
  int j = sorted[s < n ? s : n - 1];
  orig[s] = s < n ? j : -1;
  float x = vx[j], y = vy[j];
  for (int t = 0; t < T; ++t)
    offs[(size_t)s * T + t] = make_int2(track_offset(x, cs.dt[t]), track_offset(y, cs.dt[t]));
}

// One thread per (chunk, epoch): staging rectangle and per-trajectory byte offsets into it.
// box = {x offset of the rectangle from the tile origin (x_lo + dxmin - xshift is a multiple
// of 4 so that the TMA x coordinate is 16-byte aligned), y offset, number of 8-row boxes,
// fits-in-a-stage flag}.
__global__ void plan_boxes_kernel(const int2* __restrict__ offs, int nchunk, int T, int x_lo,
                                  int4* box, int32_t* rel) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nchunk * T) return;
  int c = i / T, t = i - c * T;
  int dxmin = INT_MAX, dxmax = INT_MIN, dymin = INT_MAX, dymax = INT_MIN;
  for (int v = 0; v < S_C; ++v) {
    int2 o = offs[(size_t)(c * S_C + v) * T + t];
    dxmin = min(dxmin, o.x); dxmax = max(dxmax, o.x);
    dymin = min(dymin, o.y); dymax = max(dymax, o.y);
  }
  int xshift = ((x_lo + dxmin) % 4 + 4) % 4;
  int rw = S_TX + (dxmax - dxmin) + xshift;
  int rh = S_TY + (dymax - dymin);
  int nb = (rh + S_BOX_Y - 1) / S_BOX_Y;
  // overflow-safe check: spans are compared before being added
  bool fits = (dxmax - dxmin) <= S_PITCH && (dymax - dymin) <= S_CAP_ROWS && rw <= S_PITCH &&
              nb * S_BOX_Y <= S_CAP_ROWS;
  box[i] = make_int4(dxmin - xshift, dymin, nb, fits ? 1 : 0);
  for (int v = 0; v < S_C; ++v) {
    int2 o = offs[(size_t)(c * S_C + v) * T + t];
    rel[(size_t)i * S_C + v] =
        fits ? ((o.y - dymin) * S_PITCH + (o.x - dxmin + xshift)) * (int)sizeof(float) : 0;
  }
}

// nu2 = psi^2/phi for valid epochs with psi > 0, else 0; [T][H][Wp] with zero padding.
__global__ void bound_prep_kernel(const float* __restrict__ psi, const float* __restrict__ phi,
                                  int T, int H, int W, int Wp, float* __restrict__ bound) {
  size_t total = (size_t)T * H * Wp;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    int x = (int)(i % Wp);
    size_t row = i / Wp;  // t*H + y
    float v = 0.0f;
    if (x < W) {
      size_t s = row * W + x;
      float p = __ldg(psi + s), f = __ldg(phi + s);
      if (f > 0.0f && p > 0.0f && isfinite(p) && isfinite(f)) v = __fdiv_rn(__fmul_rn(p, p), f);
    }
    bound[i] = v;
  }
}

// ---------------------------------------------------------------------------------------------
// Warp-level full evaluation of one (start pixel, trajectory) pair
// ---------------------------------------------------------------------------------------------
template <int J>
__device__ __forceinline__ void warp_bitonic_sort(float (&v)[J], int lane) {
#pragma unroll
  for (int k = 2; k <= 32 * J; k <<= 1) {
#pragma unroll
    for (int d = k >> 1; d > 0; d >>= 1) {
      if (d >= 32) {
        const int dj = d >> 5;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int jp = j ^ dj;
          if (jp > j) {
            const bool up = (((j << 5) | lane) & k) == 0;
            const float a = v[j], b = v[jp];
            const float lo = fminf(a, b), hi = fmaxf(a, b);
            v[j] = up ? lo : hi;
            v[jp] = up ? hi : lo;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const float other = __shfl_xor_sync(0xffffffffu, v[j], d);
          const bool up = (((j << 5) | lane) & k) == 0;
          const bool lower = (lane & d) == 0;
          v[j] = (lower == up) ? fminf(v[j], other) : fmaxf(v[j], other);
        }
      }
    }
  }
}

template <int J>
__device__ __forceinline__ float warp_get_sorted(const float (&v)[J], int r) {
  float x = v[0];
#pragma unroll
  for (int j = 1; j < J; ++j)
    if ((r >> 5) == j) x = v[j];
  return __shfl_sync(0xffffffffu, x, r & 31);
}

template <int J>
__device__ __forceinline__ float warp_percentile(const float (&s)[J], int n, float q) {
  const float h = (float)(n - 1) * q;
  int lo = (int)floorf(h);
  lo = max(0, min(lo, n - 1));
  const int hi = min(lo + 1, n - 1);
  const float f = h - (float)lo;
  const float a = warp_get_sorted<J>(s, lo), b = warp_get_sorted<J>(s, hi);
  return a + f * (b - a);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Writes rec[0..7]: L' (NaN when the pair is not eligible), alpha, nvalid | nkept << 16,
// mask words.  All lanes take part; lane 0 writes.
template <int J>
__device__ void eval_pair_warp(const float* __restrict__ psi, const float* __restrict__ phi,
                               const EvalParams& ep, int x0, int y0,
                               const int2* __restrict__ off, uint32_t* rec, int lane) {
  float ps[J], ph[J], a[J];
  bool valid[J];
  const size_t plane = (size_t)ep.H * ep.W;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int t = (j << 5) | lane;
    ps[j] = 0.0f;
    ph[j] = 0.0f;
    valid[j] = false;
    if (t < ep.T) {
      const int2 o = __ldg(off + t);
      const int x = x0 + o.x, y = y0 + o.y;
      if (x >= 0 && x < ep.W && y >= 0 && y < ep.H) {
        const size_t i = (size_t)t * plane + (size_t)y * ep.W + x;
        const float p = __ldg(psi + i), f = __ldg(phi + i);
        if (f > 0.0f && isfinite(p) && isfinite(f)) {
          ps[j] = p;
          ph[j] = f;
          valid[j] = true;
        }
      }
    }
  }
  int nvalid = 0;
#pragma unroll
  for (int j = 0; j < J; ++j) nvalid += __popc(__ballot_sync(0xffffffffu, valid[j]));
  if (nvalid < ep.min_obs || nvalid == 0) {
    if (lane == 0) {
      rec[0] = __float_as_uint(NAN);
      rec[2] = (uint32_t)nvalid;
    }
    return;
  }
  bool keep[J];
  if (ep.clip) {
    float s[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      a[j] = valid[j] ? (ep.clip_on ? __fdiv_rn(ps[j], __fsqrt_rn(ph[j])) : __fdiv_rn(ps[j], ph[j]))
                      : INFINITY;
      s[j] = a[j];
    }
    warp_bitonic_sort<J>(s, lane);
    const float x_lo = warp_percentile<J>(s, nvalid, ep.q_lo);
    const float x_mid = warp_percentile<J>(s, nvalid, ep.q_mid);
    const float x_hi = warp_percentile<J>(s, nvalid, ep.q_hi);
    const float sg = ep.c_sigma * (x_hi - x_lo);
    const float lo_b = x_mid - ep.n_sigma * sg, hi_b = x_mid + ep.n_sigma * sg;
#pragma unroll
    for (int j = 0; j < J; ++j) keep[j] = valid[j] && a[j] >= lo_b && a[j] <= hi_b;
  } else {
#pragma unroll
    for (int j = 0; j < J; ++j) keep[j] = valid[j];
  }
  float sp = 0.0f, sf = 0.0f;
  int nkept = 0;
  uint32_t mw[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int j = 0; j < J; ++j) {
    sp += keep[j] ? ps[j] : 0.0f;
    sf += keep[j] ? ph[j] : 0.0f;
    const uint32_t b = __ballot_sync(0xffffffffu, keep[j]);
    mw[j] = b;
    nkept += __popc(b);
  }
  sp = warp_sum(sp);
  sf = warp_sum(sf);
  if (lane == 0) {
    float L = NAN, alpha = 0.0f;
    if (nkept > 0 && sf > 0.0f) {
      L = __fdiv_rn(sp, __fsqrt_rn(sf));
      alpha = __fdiv_rn(sp, sf);
    }
    rec[0] = __float_as_uint(L);
    rec[1] = __float_as_uint(alpha);
    rec[2] = (uint32_t)nvalid | ((uint32_t)nkept << 16);
#pragma unroll
    for (int j = 0; j < 4; ++j) rec[3 + j] = mw[j];
  }
}

// ---------------------------------------------------------------------------------------------
// The search kernel
// ---------------------------------------------------------------------------------------------
struct SearchArgs {
  const float* psi;
  const float* phi;
  const float* bound;
  const int32_t* orig;
  const int2* offs;
  const int4* box;
  const int32_t* rel;
  float* out_lh;
  float* out_flux;
  int32_t* out_idx;
  uint16_t* out_nvalid;
  uint16_t* out_nkept;
  uint32_t* out_mask;
  Ctrl* ctrl;
  EvalParams ep;
  int n_traj, nchunk, Wp;
  int x_lo, x_hi, y_lo, y_hi, ntx, nty, ntiles;
};

struct SmemLayout {
  static constexpr size_t stage = 0;  // 2 stages
  static constexpr size_t rec = stage + 2 * S_STAGE_FLOATS * sizeof(float);
  static constexpr size_t queue = rec + S_QCAP * S_REC_WORDS * sizeof(uint32_t);
  static constexpr size_t filled = queue + S_QCAP * sizeof(uint16_t);
  static constexpr size_t misc = filled + S_TX * S_TY;
  static constexpr size_t total = misc + 64;
};

__device__ __forceinline__ void issue_stage(const CUtensorMap* tmap, const SearchArgs& A,
                                            float* stage, uint64_t* bar, long long it) {
  const int T = A.ep.T;
  const long long per_tile = (long long)A.nchunk * T;
  const int k = (int)(it / per_tile);
  const int rem = (int)(it - (long long)k * per_tile);
  const int c = rem / T, t = rem - c * T;
  const int tile = blockIdx.x + k * gridDim.x;
  const int tx0 = A.x_lo + (tile % A.ntx) * S_TX;
  const int ty0 = A.y_lo + (tile / A.ntx) * S_TY;
  const int4 b = __ldg(A.box + (size_t)c * T + t);
  if (b.w) {
    mbar_arrive_expect_tx(bar, (uint32_t)(b.z * S_BOX_Y * S_PITCH * sizeof(float)));
    for (int i = 0; i < b.z; ++i)
      tma_load_3d(stage + i * S_BOX_Y * S_PITCH, tmap, bar, tx0 + b.x, ty0 + b.y + i * S_BOX_Y, t);
  } else {
    mbar_arrive(bar);
  }
}

// Inserts (L, j, record) into the ordered list of window pixel wp that holds nf entries
// (LH' descending, trajectory index ascending).  Returns true if it entered the list.
__device__ __noinline__ bool insert_sorted(const SearchArgs& A, size_t wp, int K, int mw, int nf,
                                           float L, int j, const uint32_t* rc) {
  float* lh = A.out_lh + wp * K;
  int32_t* ix = A.out_idx + wp * K;
  int s = 0;
  while (s < nf && (lh[s] > L || (lh[s] == L && ix[s] < j))) ++s;
  if (s >= K) return false;
  const int last = min(nf, K - 1);
  for (int m = last; m > s; --m) {
    lh[m] = lh[m - 1];
    ix[m] = ix[m - 1];
    A.out_flux[wp * K + m] = A.out_flux[wp * K + m - 1];
    A.out_nvalid[wp * K + m] = A.out_nvalid[wp * K + m - 1];
    A.out_nkept[wp * K + m] = A.out_nkept[wp * K + m - 1];
    for (int w = 0; w < mw; ++w)
      A.out_mask[(wp * K + m) * mw + w] = A.out_mask[(wp * K + m - 1) * mw + w];
  }
  lh[s] = L;
  ix[s] = j;
  A.out_flux[wp * K + s] = __uint_as_float(rc[1]);
  A.out_nvalid[wp * K + s] = (uint16_t)(rc[2] & 0xffffu);
  A.out_nkept[wp * K + s] = (uint16_t)(rc[2] >> 16);
  for (int w = 0; w < mw; ++w) A.out_mask[(wp * K + s) * mw + w] = rc[3 + w];
  return true;
}

template <int J>
__global__ void __launch_bounds__(S_THREADS, 1)
search_kernel(const __grid_constant__ CUtensorMap tmap, const SearchArgs A) {
  extern __shared__ __align__(1024) unsigned char smem[];
  float* stages = reinterpret_cast<float*>(smem + SmemLayout::stage);
  uint32_t* recs = reinterpret_cast<uint32_t*>(smem + SmemLayout::rec);
  uint16_t* queue = reinterpret_cast<uint16_t*>(smem + SmemLayout::queue);
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + SmemLayout::misc);
  unsigned int* s_qcount = reinterpret_cast<unsigned int*>(smem + SmemLayout::misc + 16);
  unsigned int* s_evals = s_qcount + 1;
  unsigned int* s_ins = s_qcount + 2;
  uint8_t* s_filled = reinterpret_cast<uint8_t*>(smem + SmemLayout::filled);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int T = A.ep.T, K = A.ep.K, mw = A.ep.mw;
  const int my_tiles = (A.ntiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const long long per_tile = (long long)A.nchunk * T;
  const long long total_it = (long long)my_tiles * per_tile;

  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    *s_evals = 0u;
    *s_ins = 0u;
    fence_mbar_init();
    prefetch_tmap(&tmap);
  }
  __syncthreads();
  if (tid == 0) {
    if (total_it > 0) issue_stage(&tmap, A, stages, &bars[0], 0);
    if (total_it > 1) issue_stage(&tmap, A, stages + S_STAGE_FLOATS, &bars[1], 1);
  }

  const float lh_min = A.ep.lh_min;
  const size_t wx = (size_t)(A.x_hi - A.x_lo);
  long long it = 0;
  bool aborted = false;

  for (int k = 0; k < my_tiles && !aborted; ++k) {
    const int tile = blockIdx.x + k * gridDim.x;
    const int tx0 = A.x_lo + (tile % A.ntx) * S_TX;
    const int ty0 = A.y_lo + (tile / A.ntx) * S_TY;
    const int px = tx0 + lane;
    // per-pixel state of the 8 owned pixels: admission threshold for the bound, list fill
    float thr2[S_ROWS];
    uint32_t active = 0u;
#pragma unroll
    for (int i = 0; i < S_ROWS; ++i) {
      const int py = ty0 + warp * S_ROWS + i;
      const bool act = px < A.x_hi && py < A.y_hi;
      active |= (act ? 1u : 0u) << i;
      s_filled[((warp * S_ROWS + i) << 5) | lane] = 0;
      thr2[i] = lh_min > 0.0f ? lh_min * lh_min * S_PRUNE_MARGIN : -1.0f;
      if (act) {
        const size_t wp = (size_t)(py - A.y_lo) * wx + (size_t)(px - A.x_lo);
        for (int s = 0; s < K; ++s) {
          A.out_lh[wp * K + s] = -INFINITY;
          A.out_flux[wp * K + s] = 0.0f;
          A.out_idx[wp * K + s] = -1;
          A.out_nvalid[wp * K + s] = 0;
          A.out_nkept[wp * K + s] = 0;
          for (int m = 0; m < mw; ++m) A.out_mask[(wp * K + s) * mw + m] = 0u;
        }
      }
    }

    for (int c = 0; c < A.nchunk && !aborted; ++c) {
      float acc[S_ROWS][S_C];
#pragma unroll
      for (int i = 0; i < S_ROWS; ++i)
#pragma unroll
        for (int v = 0; v < S_C; ++v) acc[i][v] = 0.0f;

      for (int t = 0; t < T; ++t, ++it) {
        const int st = (int)(it & 1);
        const bool ok = mbar_wait_parity(&bars[st], (uint32_t)((it >> 1) & 1));
        const int4 b = __ldg(A.box + (size_t)c * T + t);
        if (ok) {
          if (b.w) {
            const int4* relv = reinterpret_cast<const int4*>(A.rel + ((size_t)c * T + t) * S_C);
            const char* base = reinterpret_cast<const char*>(stages + st * S_STAGE_FLOATS) +
                               (size_t)(warp * S_ROWS * S_PITCH + lane) * sizeof(float);
#pragma unroll
            for (int vq = 0; vq < S_C / 4; ++vq) {
              const int4 r4 = __ldg(relv + vq);
              const int rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const float* p = reinterpret_cast<const float*>(base + rr[u]);
#pragma unroll
                for (int i = 0; i < S_ROWS; ++i) acc[i][vq * 4 + u] += p[i * S_PITCH];
              }
            }
          } else {
            const float* bp = A.bound + (size_t)t * A.ep.H * A.Wp;
#pragma unroll
            for (int v = 0; v < S_C; ++v) {
              const int2 o = __ldg(A.offs + (size_t)(c * S_C + v) * T + t);
              const int x = px + o.x;
#pragma unroll
              for (int i = 0; i < S_ROWS; ++i) {
                const int y = ty0 + warp * S_ROWS + i + o.y;
                if (x >= 0 && x < A.Wp && y >= 0 && y < A.ep.H)
                  acc[i][v] += __ldg(bp + (size_t)y * A.Wp + x);
              }
            }
          }
        }
        const int bad = __syncthreads_or(ok ? 0 : 1);
        if (bad) {
          aborted = true;
          break;
        }
        if (tid == 0 && it + 2 < total_it) {
          fence_proxy_async_smem();
          issue_stage(&tmap, A, stages + st * S_STAGE_FLOATS, &bars[st], it + 2);
        }
      }
      if (aborted) break;

      // ---- candidates of this chunk: pairs whose bound reaches the admission threshold ----
      const int nv = min(S_C, A.n_traj - c * S_C);
      uint32_t cb0 = 0u, cb1 = 0u, cb2 = 0u, cb3 = 0u;  // 16 bits per owned pixel
      int ncand = 0;
#pragma unroll
      for (int i = 0; i < S_ROWS; ++i) {
        uint32_t bits = 0u;
#pragma unroll
        for (int v = 0; v < S_C; ++v)
          if (((active >> i) & 1u) && v < nv && acc[i][v] >= thr2[i]) bits |= 1u << v;
        ncand += __popc(bits);
        const uint32_t sh = bits << ((i & 1) * 16);
        if ((i >> 1) == 0) cb0 |= sh;
        else if ((i >> 1) == 1) cb1 |= sh;
        else if ((i >> 1) == 2) cb2 |= sh;
        else cb3 |= sh;
      }
      // block-wide exclusive rank of this thread's candidates
      int incl = ncand;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (tid == 0) *s_qcount = 0u;
      __syncthreads();
      unsigned int wbase = 0;
      if (lane == 31 && incl > 0) wbase = atomicAdd(s_qcount, (unsigned int)incl);
      wbase = __shfl_sync(0xffffffffu, wbase, 31);
      const int my_base = (int)wbase + incl - ncand;
      __syncthreads();
      const int total = (int)*s_qcount;

      for (int r0 = 0; r0 < total; r0 += S_QCAP) {
        // enqueue this round's candidates (bit order: owned pixel, then trajectory)
        if (ncand > 0) {
          int rank = my_base;
#pragma unroll 1
          for (int w4 = 0; w4 < 4; ++w4) {
            uint32_t bits = w4 == 0 ? cb0 : w4 == 1 ? cb1 : w4 == 2 ? cb2 : cb3;
            while (bits) {
              const int b = __ffs(bits) - 1;
              bits &= bits - 1u;
              if (rank >= r0 && rank < r0 + S_QCAP) {
                const int i = 2 * w4 + (b >> 4), v = b & 15;
                queue[rank - r0] = (uint16_t)((((warp * S_ROWS + i) << 5) | lane) << 4 | v);
              }
              ++rank;
            }
          }
        }
        __syncthreads();
        const int nq = min(S_QCAP, total - r0);
        for (int q = warp; q < nq; q += S_WARPS) {
          const uint32_t e = queue[q];
          const int v = (int)(e & 15u), pl = (int)(e >> 4);
          const int x0 = tx0 + (pl & 31), y0 = ty0 + (pl >> 5);
          eval_pair_warp<J>(A.psi, A.phi, A.ep, x0, y0, A.offs + (size_t)(c * S_C + v) * T,
                            recs + q * S_REC_WORDS, lane);
        }
        __syncthreads();
        // owners insert their results into the output lists
        if (ncand > 0) {
          int rank = my_base;
#pragma unroll 1
          for (int w4 = 0; w4 < 4; ++w4) {
            uint32_t bits = w4 == 0 ? cb0 : w4 == 1 ? cb1 : w4 == 2 ? cb2 : cb3;
            while (bits) {
              const int b = __ffs(bits) - 1;
              bits &= bits - 1u;
              if (rank >= r0 && rank < r0 + S_QCAP) {
                const int i = 2 * w4 + (b >> 4), v = b & 15;
                const uint32_t* rc = recs + (rank - r0) * S_REC_WORDS;
                const float L = __uint_as_float(rc[0]);
                if (L >= lh_min) {  // false for NaN (pair not eligible)
                  const int row = warp * S_ROWS + i;
                  const int j = A.orig[c * S_C + v];
                  const size_t wp = (size_t)(ty0 + row - A.y_lo) * wx + (size_t)(px - A.x_lo);
                  const int nf = s_filled[(row << 5) | lane];
                  if (insert_sorted(A, wp, K, mw, nf, L, j, rc)) {
                    s_filled[(row << 5) | lane] = (uint8_t)min(nf + 1, K);
                    atomicAdd(s_ins, 1u);
                  }
                }
              }
              ++rank;
            }
          }
        }
        __syncthreads();
      }
      if (tid == 0 && total > 0) atomicAdd(s_evals, (unsigned int)total);
      // new admission thresholds: once a list is full, its K-th LH' (with the same margin)
#pragma unroll
      for (int i = 0; i < S_ROWS; ++i) {
        const int row = warp * S_ROWS + i;
        if (((active >> i) & 1u) && s_filled[(row << 5) | lane] == K) {
          const size_t wp = (size_t)(ty0 + row - A.y_lo) * wx + (size_t)(px - A.x_lo);
          const float thr = fmaxf(A.out_lh[wp * K + K - 1], lh_min);
          thr2[i] = thr > 0.0f ? thr * thr * S_PRUNE_MARGIN : -1.0f;
        }
      }
    }
  }

  if (aborted) {
    if (tid == 0) {
      atomicOr(&A.ctrl->err, kErrTimeout);
      // wait (bounded) for copies still in flight into either stage before leaving
      mbar_wait_parity(&bars[it & 1], (uint32_t)((it >> 1) & 1));
      mbar_wait_parity(&bars[(it + 1) & 1], (uint32_t)(((it + 1) >> 1) & 1));
    }
    return;
  }
  __syncthreads();
  if (tid == 0) {
    atomicAdd(&A.ctrl->evals, (unsigned long long)*s_evals);
    atomicAdd(&A.ctrl->inserts, (unsigned long long)*s_ins);
  }
}

// ---------------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 get_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// erf^{-1} by Newton's method on std::erf, started from 0 (erf is increasing and convex for
// negative and concave for positive arguments, so the iteration converges monotonically).
static double erfinv_newton(double y) {
  double x = 0.0;
  for (int i = 0; i < 100; ++i) {
    double e = std::erf(x) - y;
    double d = 2.0 / std::sqrt(M_PI) * std::exp(-x * x);
    double nx = x - e / d;
    if (nx == x) break;
    x = nx;
  }
  return x;
}

static int validate(const float* psi, const float* phi, const double* times, int T, int H,
                    int W, const float* vx, const float* vy, int n_traj,
                    const kb_search_params* p) {
  if (!psi || !phi || !times || !vx || !vy || !p)
    return fail(KB_ERR_INVALID_ARG, "kb_search: null pointer argument");
  if (T < 1 || H < 1 || W < 1 || n_traj < 1)
    return fail(KB_ERR_INVALID_ARG, "kb_search: T, H, W and n_traj must be positive");
  if (T > KB_MAX_T) return fail(KB_ERR_UNSUPPORTED, "kb_search: T = %d > KB_MAX_T = %d", T, KB_MAX_T);
  if (n_traj > (1 << 24)) return fail(KB_ERR_UNSUPPORTED, "kb_search: n_traj > 2^24");
  if (H > (1 << 20) || W > (1 << 20))
    return fail(KB_ERR_UNSUPPORTED, "kb_search: image sides are limited to 2^20 pixels");
  if ((long long)H * ((W + 31) / 32 * 32) >= (1LL << 31))
    return fail(KB_ERR_UNSUPPORTED, "kb_search: image plane beyond 2^31 pixels");
  if (p->k_per_pixel < 1 || p->k_per_pixel > KB_MAX_K)
    return fail(KB_ERR_INVALID_ARG, "kb_search: k_per_pixel must be in 1..%d", KB_MAX_K);
  if (!std::isfinite(p->lh_min) || !std::isfinite(p->n_sigma) || p->n_sigma < 0.0f)
    return fail(KB_ERR_INVALID_ARG, "kb_search: lh_min / n_sigma must be finite, n_sigma >= 0");
  if (p->clip != 0 && p->clip != 1) return fail(KB_ERR_INVALID_ARG, "kb_search: clip must be 0 or 1");
  if (p->clip_on != 0 && p->clip_on != 1)
    return fail(KB_ERR_INVALID_ARG, "kb_search: clip_on must be 0 or 1");
  if (p->clip) {
    if (!(p->q_lo >= 0.0f && p->q_lo < p->q_hi && p->q_hi <= 1.0f && p->q_mid >= 0.0f &&
          p->q_mid <= 1.0f))
      return fail(KB_ERR_INVALID_ARG, "kb_search: need 0 <= q_lo < q_hi <= 1, 0 <= q_mid <= 1");
    if (p->q_lo <= 0.0f || p->q_hi >= 1.0f)
      return fail(KB_ERR_INVALID_ARG, "kb_search: sigma_G quantiles must lie strictly in (0,1)");
  }
  if (p->min_obs < 0) return fail(KB_ERR_INVALID_ARG, "kb_search: min_obs < 0");
  if (p->x_lo < 0 || p->x_hi > W || p->y_lo < 0 || p->y_hi > H || p->x_lo >= p->x_hi ||
      p->y_lo >= p->y_hi)
    return fail(KB_ERR_INVALID_ARG, "kb_search: start-pixel window outside the image or empty");
  for (int t = 0; t < T; ++t)
    if (!std::isfinite(times[t])) return fail(KB_ERR_INVALID_ARG, "kb_search: times[%d] not finite", t);
  return KB_OK;
}

static int g_num_sms = 0;

}  // namespace kb

extern "C" int kb_search_workspace_size(int T, int H, int W, int n_traj,
                                        const kb_search_params* p, size_t* bytes) {
  using namespace kb;
  if (!bytes || !p) return fail(KB_ERR_INVALID_ARG, "kb_search_workspace_size: null pointer");
  if (T < 1 || H < 1 || W < 1 || n_traj < 1)
    return fail(KB_ERR_INVALID_ARG, "kb_search_workspace_size: bad sizes");
  if (T > KB_MAX_T) return fail(KB_ERR_UNSUPPORTED, "kb_search_workspace_size: T > KB_MAX_T");
  if (n_traj > (1 << 24)) return fail(KB_ERR_UNSUPPORTED, "kb_search_workspace_size: n_traj > 2^24");
  *bytes = ws_layout(T, H, W, n_traj).total;
  return KB_OK;
}

extern "C" int kb_search(const float* psi, const float* phi, const double* times, int T, int H,
                         int W, const float* vx, const float* vy, int n_traj,
                         const kb_search_params* p, float* out_lh, float* out_flux,
                         int32_t* out_idx, uint16_t* out_nvalid, uint16_t* out_nkept,
                         uint32_t* out_mask, void* workspace, size_t ws_bytes, void* stream) {
  using namespace kb;
  int rc = validate(psi, phi, times, T, H, W, vx, vy, n_traj, p);
  if (rc != KB_OK) return rc;
  if (!out_lh || !out_flux || !out_idx || !out_nvalid || !out_nkept || !out_mask)
    return fail(KB_ERR_INVALID_ARG, "kb_search: null output pointer");
  const WsLayout L = ws_layout(T, H, W, n_traj);
  if (!workspace || ws_bytes < L.total)
    return fail(KB_ERR_WORKSPACE, "kb_search: workspace of %zu bytes, %zu needed", ws_bytes, L.total);
  if (reinterpret_cast<uintptr_t>(workspace) % KB_WORKSPACE_ALIGN)
    return fail(KB_ERR_WORKSPACE, "kb_search: workspace not %d-byte aligned", KB_WORKSPACE_ALIGN);
  auto enc = get_encode_fn();
  if (!enc) return fail(KB_ERR_CUDA, "kb_search: cuTensorMapEncodeTiled unavailable");
  if (g_num_sms == 0) {
    int dev = 0;
    KB_CUDA_TRY(cudaGetDevice(&dev));
    KB_CUDA_TRY(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* ws = static_cast<char*>(workspace);
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
  float4* vbox = reinterpret_cast<float4*>(ws + L.vbox);
  uint32_t* keys = reinterpret_cast<uint32_t*>(ws + L.keys);
  uint32_t* counts = reinterpret_cast<uint32_t*>(ws + L.counts);
  uint32_t* cursor = reinterpret_cast<uint32_t*>(ws + L.cursor);
  int32_t* sorted = reinterpret_cast<int32_t*>(ws + L.sorted);
  int32_t* orig = reinterpret_cast<int32_t*>(ws + L.orig);
  int2* offs = reinterpret_cast<int2*>(ws + L.offs);
  int4* box = reinterpret_cast<int4*>(ws + L.box);
  int32_t* rel = reinterpret_cast<int32_t*>(ws + L.rel);
  float* bound = reinterpret_cast<float*>(ws + L.bound);

  SearchConsts cs{};
  for (int t = 0; t < T; ++t) cs.dt[t] = (float)(times[t] - times[0]);

  const int npix_w = (p->x_hi - p->x_lo) * (p->y_hi - p->y_lo);
  const unsigned long long te = (unsigned long long)npix_w * n_traj * T;

  plan_reset_kernel<<<N_CELLS / 256, 256, 0, st>>>(ctrl, counts, te);
  KB_LAUNCH_CHECK("plan_reset_kernel");
  plan_minmax_kernel<<<1, 1024, 0, st>>>(vx, vy, n_traj, vbox);
  KB_LAUNCH_CHECK("plan_minmax_kernel");
  plan_hist_kernel<<<(n_traj + 255) / 256, 256, 0, st>>>(vx, vy, n_traj, vbox, keys, counts);
  KB_LAUNCH_CHECK("plan_hist_kernel");
  plan_scan_kernel<<<1, 1024, 0, st>>>(counts, cursor);
  KB_LAUNCH_CHECK("plan_scan_kernel");
  plan_scatter_kernel<<<(n_traj + 255) / 256, 256, 0, st>>>(keys, n_traj, cursor, sorted);
  KB_LAUNCH_CHECK("plan_scatter_kernel");
  plan_cellsort_kernel<<<N_CELLS / 256, 256, 0, st>>>(counts, cursor, sorted);
  KB_LAUNCH_CHECK("plan_cellsort_kernel");
  plan_offsets_kernel<<<(L.n_pad + 255) / 256, 256, 0, st>>>(vx, vy, sorted, n_traj, L.n_pad, T,
                                                               cs, orig, offs);
  KB_LAUNCH_CHECK("plan_offsets_kernel");
  plan_boxes_kernel<<<(L.nchunk * T + 255) / 256, 256, 0, st>>>(offs, L.nchunk, T, p->x_lo, box, rel);
  KB_LAUNCH_CHECK("plan_boxes_kernel");
  {
    size_t total = (size_t)T * H * L.Wp;
    int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)g_num_sms * 16);
    bound_prep_kernel<<<blocks, 256, 0, st>>>(psi, phi, T, H, W, L.Wp, bound);
    KB_LAUNCH_CHECK("bound_prep_kernel");
  }

  CUtensorMap tmap;
  {
    cuuint64_t dims[3] = {(cuuint64_t)L.Wp, (cuuint64_t)H, (cuuint64_t)T};
    cuuint64_t strides[2] = {(cuuint64_t)L.Wp * sizeof(float), (cuuint64_t)L.Wp * H * sizeof(float)};
    cuuint32_t boxd[3] = {(cuuint32_t)S_PITCH, (cuuint32_t)S_BOX_Y, 1u};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, bound, dims, strides, boxd, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(KB_ERR_CUDA, "kb_search: cuTensorMapEncodeTiled failed (%d)", (int)r);
  }

  SearchArgs A{};
  A.psi = psi;
  A.phi = phi;
  A.bound = bound;
  A.orig = orig;
  A.offs = offs;
  A.box = box;
  A.rel = rel;
  A.out_lh = out_lh;
  A.out_flux = out_flux;
  A.out_idx = out_idx;
  A.out_nvalid = out_nvalid;
  A.out_nkept = out_nkept;
  A.out_mask = out_mask;
  A.ctrl = ctrl;
  A.ep.T = T;
  A.ep.H = H;
  A.ep.W = W;
  A.ep.min_obs = p->min_obs;
  A.ep.clip = p->clip;
  A.ep.clip_on = p->clip_on;
  A.ep.K = p->k_per_pixel;
  A.ep.mw = (T + 31) / 32;
  A.ep.q_lo = p->q_lo;
  A.ep.q_mid = p->q_mid;
  A.ep.q_hi = p->q_hi;
  A.ep.n_sigma = p->n_sigma;
  A.ep.c_sigma = p->clip ? (float)(1.0 / (std::sqrt(2.0) * (erfinv_newton(2.0 * p->q_hi - 1.0) -
                                                             erfinv_newton(2.0 * p->q_lo - 1.0))))
                         : 0.0f;
  A.ep.lh_min = p->lh_min;
  A.n_traj = n_traj;
  A.nchunk = L.nchunk;
  A.Wp = L.Wp;
  A.x_lo = p->x_lo;
  A.x_hi = p->x_hi;
  A.y_lo = p->y_lo;
  A.y_hi = p->y_hi;
  A.ntx = (p->x_hi - p->x_lo + S_TX - 1) / S_TX;
  A.nty = (p->y_hi - p->y_lo + S_TY - 1) / S_TY;
  A.ntiles = A.ntx * A.nty;
  const int grid = std::min(A.ntiles, g_num_sms);
  const size_t smem = SmemLayout::total;
  const int J = (T + 31) / 32;
#define KB_SEARCH_LAUNCH(JJ)                                                                   \
  do {                                                                                         \
    KB_CUDA_TRY(cudaFuncSetAttribute(search_kernel<JJ>,                                        \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)); \
    search_kernel<JJ><<<grid, S_THREADS, smem, st>>>(tmap, A);                                 \
  } while (0)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  profile_events(&ev0, &ev1);
  if (ev0 && ev1) KB_CUDA_TRY(cudaEventRecord(ev0, st));
  if (J == 1) KB_SEARCH_LAUNCH(1);
  else if (J == 2) KB_SEARCH_LAUNCH(2);
  else KB_SEARCH_LAUNCH(4);
#undef KB_SEARCH_LAUNCH
  KB_LAUNCH_CHECK("search_kernel");
  if (ev0 && ev1) KB_CUDA_TRY(cudaEventRecord(ev1, st));
  return KB_OK;
}

extern "C" int kb_search_stats(const void* workspace, unsigned long long* stats, void* stream) {
  using namespace kb;
  if (!workspace || !stats) return fail(KB_ERR_INVALID_ARG, "kb_search_stats: null pointer");
  Ctrl c{};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KB_CUDA_TRY(cudaMemcpyAsync(&c, workspace, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  KB_CUDA_TRY(cudaStreamSynchronize(st));
  stats[0] = c.te;
  stats[1] = c.evals;
  stats[2] = c.inserts;
  stats[3] = c.err;
  return KB_OK;
}
