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
//      1. bound pass, B(p, j) = sum_t nu2[t, p + d_t(j)] with nu2 = psi^2/phi (psi > 0, valid),
//         taken either per start pixel or, when that pays (pool_blocks: 1.5 T <= lh_min^2),
//         over blocks of two vertically adjacent start pixels, B2 = sum_t of the larger nu2 of
//         the two shifted pixels, which bounds the sum of either;
//      2. full evaluation of the few pairs (of both pixels of a passing block) whose bound
//         reaches the admission threshold (a block: the smaller of its pixels' thresholds):
//         gather psi/phi, sigma-G clip, LH', alpha, then insertion into the pixel's list.
//    Pairs are dropped only when the sum is below thr^2 (1 - 1e-4) (with the fp16 rounding of
//    the sums accounted for, see admission_threshold), so the output equals evaluating every
//    pair.
//
//  * Bound pass layout.  The terms are written once per call into the workspace as fp16 pairs,
//    rounded up: word (t, r, x) of a [T][H+3][Wp] uint32 array (Wp = W rounded up to 32) holds
//    rows r-3 and r-2 (single rows) or the maxima of rows (r-3, r-2) and (r-1, r) (blocks) at
//    column x.  A block owns a tile of 32 x 56 start pixels (lane = x, 4 rows per consumer
//    thread), or 64 x 56 with blocks on large windows (columns x and x + 32 per thread), and
//    sweeps the velocity list in chunks of 32 trajectories that are close in velocity space
//    (Hilbert order of (vx, vy) from the plan kernels), the epochs of a chunk in the order
//    0, T-1, 1, T-2, ...  For each (chunk, epoch)
//    the union of the tile's 32 shifted footprints is one small rectangle, fetched with one TMA
//    box into a shared-memory ring by producer warps while the consumer warps sum earlier ones.
//    A consumer thread then does, per trajectory, one address add, one 32-bit shared load and
//    one fp16x2 add (blocks), or two loads two rows apart and two adds (single rows).  A
//    (chunk, epoch) rectangle too large for a stage falls back to direct global loads.
//
//  * Full evaluation.  After each chunk, the pairs whose bound passes are appended to a queue
//    in shared memory; once it holds S_FLUSH_MIN pairs the largest whole number of rounds (one
//    pair per consumer thread, half-warp or warp) is evaluated and the rest stays queued, and at
//    the end of a tile everything, so no round leaves threads idle and no warp waits at a
//    barrier for a lone candidate.  For T <= 32 one thread evaluates one pair: gather into
//    registers, an exact filter that drops pairs which cannot reach lh_min once the epochs the
//    clip must reject are left out, then for the rest a bitonic sorting network on the
//    lightcurve, percentiles, clip, sums in epoch order (identical tracks give bit-identical
//    LH').  For 32 < T <= 64 a half-warp evaluates one pair with lanes over epochs (two pairs per
//    warp), for T > 64 a warp, each with an exact filter of the same kind before its sort.
//    Results that reach lh_min (a small fraction) are pushed onto a per-pixel list; the owner
//    thread of each start pixel then walks its list and inserts them into the pixel's output
//    list (LH' descending, trajectory index ascending).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <climits>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <mutex>
#include <type_traits>
#include <vector>

#include "kb_internal.cuh"

namespace kb {

// ---------------------------------------------------------------------------------------------
// Compile-time configuration of the search kernel
// ---------------------------------------------------------------------------------------------
constexpr int S_TX = 32;                 // columns of one warp (lane = x)
constexpr int S_ROWS = 4;                // rows per consumer thread (two row pairs)
constexpr int S_CWARPS = 14;             // consumer warps
constexpr int S_PWARPS = 2;              // producer warps: iteration `it` belongs to it % S_PWARPS
constexpr int S_CTHREADS = S_CWARPS * 32;
constexpr int S_THREADS = (S_CWARPS + S_PWARPS) * 32;
constexpr int S_TY = S_CWARPS * S_ROWS;  // 56
// Two-row-block kernels can give each thread two columns (x and x + 32): tiles 64 wide, so a
// staged box serves twice the start pixels for the same halo and one offset load serves two data
// loads; with one column the tiles are 32 wide.  Single-row kernels (which keep twice the sums
// per column) are always 32 wide.  The width is automatic by default (kb_schedule.tile_cols = 0):
// 64-wide only when the window holds at least S_WIDE_MIN_WAVES tiles of that width per SM, since
// with fewer the last wave of tiles leaves SMs idle (decam recipe, one stack: 1024 x 2048
// 148.5 ms with 32-wide tiles against 163.7 ms with 64-wide; 2046 x 2048 300.0 against 242.3).
constexpr int S_TILE_COLS_DEFAULT = 0;
constexpr int S_WIDE_MIN_WAVES = 8;
constexpr int S_C = 32;                  // trajectories per chunk
constexpr int S_D = 8;                   // pipeline slots (iterations in flight), S_D % S_PWARPS == 0
constexpr int S_REGION_MAX = 64 * 1024;  // larger rectangles use direct loads
constexpr int S_QCAP = 2048;             // block queue of full evaluations
constexpr int S_FLUSH_MIN = 2 * S_CTHREADS;  // evaluate once the queue holds two pairs per thread
constexpr int S_REC_WORDS = 8;           // L', alpha, nvalid|nkept<<16, mask[4], pad
constexpr int S_REC_BLOCKS = 256;        // most blocks of a launch (records in the workspace)
constexpr float S_PRUNE_MARGIN = 1.0f - 1e-4f;
static_assert(S_D % S_PWARPS == 0, "pipeline configuration");
static_assert((S_D & (S_D - 1)) == 0, "slot indices from a 32-bit iteration count");
// A staged rectangle is one TMA box: width class w = 1..S_NW (rows of 32, 40, ..., 128 words)
// and height class h = 0..S_NH-1 (S_TY, S_TY + 8, ..., 128 word rows); mode 0 = direct global
// loads.  Classes 8 words apart keep the padding of a box small, so more boxes fit in the ring
// and fewer bytes are staged.
constexpr int S_NW = 13, S_NH = (128 - S_TY) / 8 + 1;
__host__ __device__ constexpr int stage_width(int mode) { return 32 + 8 * (mode - 1); }
__host__ __device__ constexpr int stage_height(int h) { return S_TY + 8 * h; }
static_assert(stage_width(S_NW) == 128 && stage_height(S_NH - 1) == 128 && S_TY % 8 == 0,
              "box classes");
constexpr int S_MODE_MASK = 15, S_UNIFORM_BIT = 16;  // PlanRec box.w: mode | uniform

constexpr int S_ORDER_MAX = 16384;       // tiles ordered by predicted cost (one-block sort)
constexpr int HILBERT_BITS = 8;          // 256 x 256 velocity cells
constexpr int N_CELLS = 1 << (2 * HILBERT_BITS);
static_assert(N_CELLS >= 3 * (KB_MAX_T + 1), "plan_reset_kernel writes the rank table");

// Staging plan of one (chunk, epoch): the rectangle and the 32 per-trajectory byte offsets
// into it.  Copied into shared memory with the rectangle it describes.
struct __align__(16) PlanRec {
  int4 box;           // x offset, y offset, height class, mode (0 direct loads, 1..4 row width)
  int32_t rel[32];    // byte offset of each trajectory's footprint in the staged rectangle
};
static_assert(sizeof(PlanRec) == 144, "plan record layout");

struct SearchConsts {
  float dt[KB_MAX_T];   // (float)(t_t - t_0)
};

struct EvalParams {
  int T, H, W, min_obs, clip, clip_on, K, mw;
  float q_lo, q_mid, q_hi, n_sigma, c_sigma, lh_min;
  float prune_scale, prune_slack;  // fp16 bound sums: see admission_threshold()
  // a pair whose fp32 sum of psi^2/phi over its valid epochs with psi > 0 (less the epochs the
  // clip must reject) is below this cannot reach lh_min (Cauchy-Schwarz; lh_min^2 (1 - 1e-3),
  // -inf when lh_min <= 0): the evaluations drop it before the sort
  float nu2_floor;
};

// Interpolation ranks of the sigma-G percentiles (linear interpolation between order statistics,
// h = (n - 1) q).  h is formed in float64 from the float32 quantile, as the definition states it,
// and rounded once: entry (k, n) = {floor(h) clamped to [0, n-1], float32 of h - floor(h)} for
// quantile k (0 = q_lo, 1 = q_mid, 2 = q_hi) of n valid epochs.  The table follows the epoch
// offsets dt[KB_MAX_T] in the workspace, so an evaluation reaches it from the dt pointer it has.
__host__ __device__ constexpr int rank_entry(int k, int n) { return k * (KB_MAX_T + 1) + n; }
__device__ __forceinline__ const int2* rank_table(const float* dtf) {
  return reinterpret_cast<const int2*>(dtf + KB_MAX_T);
}

// Workspace layout (offsets in bytes from the workspace base).
struct WsLayout {
  size_t ctrl, vbox, keys, counts, cursor, sorted, orig, offs, vsort, dtf, plan, bound, pairs, recs,
      tkeys, torder, total;
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
  L.vsort = take(sizeof(float2) * (size_t)L.n_pad);
  L.dtf = take(sizeof(float) * KB_MAX_T + sizeof(int2) * 3 * (KB_MAX_T + 1));
  L.plan = take(sizeof(PlanRec) * (size_t)L.nchunk * T);
  L.bound = take(sizeof(uint32_t) * (size_t)T * (H + 3) * L.Wp);
  L.pairs = take(sizeof(float2) * (size_t)T * H * W);
  L.recs = take(sizeof(uint32_t) * S_REC_WORDS * S_QCAP * S_REC_BLOCKS);
  L.tkeys = take(sizeof(unsigned long long) * S_ORDER_MAX);
  L.torder = take(sizeof(int32_t) * S_ORDER_MAX);
  L.total = o;
  return L;
}

// ctrl block: error flags, the tile counter, and the statistics kb_search_stats reports
struct Ctrl {
  unsigned int err;
  unsigned int tile_counter;  // dynamic tile scheduling of the search kernel
  unsigned long long te, evals, inserts;
  // stage counts of the pairs evaluated in full: n_valid >= min_obs; LH' >= lh_min after the
  // clip; and, over the latter, the sums of n_kept and n_valid (the mean kept fraction)
  unsigned long long stage_valid, stage_pass, stage_kept, stage_nvalid;
  // bound-pass iterations (tile, chunk, epoch) by kind: staged box with per-trajectory offsets,
  // staged box with one offset for the chunk, direct global loads; and the bytes staged by TMA
  unsigned long long it_staged, it_uniform, it_direct, tma_bytes;
  // 4-byte shared loads per trajectory of each bound-pass thread in the kernel that ran (1 or 2)
  unsigned int loads_per_traj;
};
static_assert(sizeof(Ctrl) <= 256, "control block");

// ---------------------------------------------------------------------------------------------
// Plan kernels: velocity ordering, track offsets, per-(chunk, epoch) staging rectangles
// ---------------------------------------------------------------------------------------------
__global__ void plan_reset_kernel(Ctrl* ctrl, uint32_t* counts, unsigned long long te, float q_lo,
                                  float q_mid, float q_hi, int2* rank) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N_CELLS) counts[i] = 0u;
  if (i < 3 * (KB_MAX_T + 1)) {
    const int k = i / (KB_MAX_T + 1), n = i - k * (KB_MAX_T + 1);
    const double q = (double)(k == 0 ? q_lo : k == 1 ? q_mid : q_hi);
    const double h = __dmul_rn((double)(n > 0 ? n - 1 : 0), q);
    const double fl = floor(h);
    int lo = (int)fl;
    lo = max(0, min(lo, max(n - 1, 0)));
    rank[i] = make_int2(lo, __float_as_int(__double2float_rn(__dsub_rn(h, (double)lo))));
  }
  if (i == 0) {
    *ctrl = Ctrl{};
    ctrl->te = te;
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

// Hilbert index of cell (x, y) on a 2^HILBERT_BITS square: consecutive indices are adjacent
// cells, so consecutive trajectories of the sorted list are close in velocity space.
__device__ __forceinline__ uint32_t hilbert_index(uint32_t x, uint32_t y) {
  const uint32_t n1 = (1u << HILBERT_BITS) - 1u;
  uint32_t d = 0;
  for (uint32_t sq = 1u << (HILBERT_BITS - 1); sq > 0; sq >>= 1) {
    const uint32_t rx = (x & sq) ? 1u : 0u, ry = (y & sq) ? 1u : 0u;
    d += sq * sq * ((3u * rx) ^ ry);
    if (ry == 0u) {  // rotate the quadrant (only the lower bits matter from here on)
      if (rx == 1u) {
        x ^= n1;
        y ^= n1;
      }
      const uint32_t tmp = x;
      x = y;
      y = tmp;
    }
  }
  return d;
}

// Velocities quantised on square cells (the same cell size along vx and vy).
__global__ void plan_hist_kernel(const float* __restrict__ vx, const float* __restrict__ vy,
                                 int n, const float4* vbox, uint32_t* keys, uint32_t* counts) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 b = *vbox;
  const int nc = 1 << HILBERT_BITS;
  const float ext = fmaxf(b.y - b.x, b.w - b.z);
  const float sc = ext > 0.0f ? (float)nc / ext : 0.0f;
  int qx = min(max((int)((vx[i] - b.x) * sc), 0), nc - 1);
  int qy = min(max((int)((vy[i] - b.z) * sc), 0), nc - 1);
  uint32_t key = hilbert_index((uint32_t)qx, (uint32_t)qy);
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
                                    SearchConsts cs, int32_t* orig, int2* offs, float2* vsort,
                                    float* dtf) {
  int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s == 0)
    for (int t = 0; t < T; ++t) dtf[t] = cs.dt[t];
  if (s >= n_pad) return;
  int j = sorted[s < n ? s : n - 1];
  orig[s] = s < n ? j : -1;
  float x = vx[j], y = vy[j];
  vsort[s] = make_float2(x, y);
  for (int t = 0; t < T; ++t)
    offs[(size_t)s * T + t] = make_int2(track_offset(x, cs.dt[t]), track_offset(y, cs.dt[t]));
}

// Epoch of the k-th (chunk, epoch) iteration of a chunk: 0, T-1, 1, T-2, ...  The footprint of
// a chunk's 32 trajectories grows with the time since the first epoch, so early epochs stage
// small boxes and late ones large boxes; alternating them keeps the staging rings from filling
// with the largest boxes at the end of every chunk.  The bound pass may sum the epochs in any
// order: the admission threshold's rounding allowance holds for every order.
__host__ __device__ __forceinline__ int epoch_of(int k, int T) {
  return (k & 1) ? T - 1 - (k >> 1) : (k >> 1);
}

// One thread per (chunk, epoch): staging rectangle and per-trajectory byte offsets into it.
// box = {x offset of the rectangle from the tile origin (x_lo + dxmin - xshift is a multiple
// of 4 so that the TMA x coordinate is 16-byte aligned), y offset, height class, mode} with
// mode 1..S_NW = the width class and height class of the smallest TMA box that holds the
// rectangle; mode 0 = no box within S_REGION_MAX (direct loads); S_UNIFORM_BIT of the last field
// set when all of the chunk's offsets are equal in this epoch.
__global__ void plan_boxes_kernel(const int2* __restrict__ offs, int nchunk, int T, int x_lo,
                                  int tx, PlanRec* plan) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nchunk * T) return;
  const int c = i / T, t = epoch_of(i - c * T, T);
  int dxmin = INT_MAX, dxmax = INT_MIN, dymin = INT_MAX, dymax = INT_MIN;
  for (int v = 0; v < S_C; ++v) {
    int2 o = offs[(size_t)(c * S_C + v) * T + t];
    dxmin = min(dxmin, o.x); dxmax = max(dxmax, o.x);
    dymin = min(dymin, o.y); dymax = max(dymax, o.y);
  }
  // offsets are clamped to +-2^24, so these spans cannot overflow
  const int xshift = ((x_lo + dxmin) % 4 + 4) % 4;
  const int rw = tx + (dxmax - dxmin) + xshift;
  const int rh = S_TY + (dymax - dymin);
  // the smallest width and height classes that hold the rectangle
  const int m = 1 + max(0, (rw - stage_width(1) + 7) / 8);
  const int h = max(0, (rh - stage_height(0) + 7) / 8);
  int mode = 0, pitch = 0, hcls = 0;
  if (m <= S_NW && h < S_NH && stage_width(m) * stage_height(h) * 4 <= S_REGION_MAX) {
    mode = m;
    pitch = stage_width(m);
    hcls = h;
  }
  PlanRec& pr = plan[i];
  // S_UNIFORM_BIT of box.w: every trajectory of the chunk has the same offset in this epoch
  // (always at t = 0, often in the first hours), so one load (per row pair) serves all of them
  const int uniform = (dxmin == dxmax && dymin == dymax) ? S_UNIFORM_BIT : 0;
  pr.box = make_int4(dxmin - xshift, dymin, hcls, mode | uniform);
  for (int v = 0; v < S_C; ++v) {
    int2 o = offs[(size_t)(c * S_C + v) * T + t];
    pr.rel[v] = mode ? ((o.y - dymin) * pitch + (o.x - dxmin + xshift)) * 4 : 0;
  }
}

// nu2 = psi^2/phi at a valid pixel with psi > 0, else 0 (also outside the image).
__device__ __forceinline__ float nu2_at(const float* __restrict__ psi,
                                        const float* __restrict__ phi, int H, int W, size_t plane,
                                        int y, int x) {
  if (y < 0 || y >= H || x >= W) return 0.0f;
  const size_t s = plane + (size_t)y * W + x;
  const float p = __ldg(psi + s), f = __ldg(phi + s);
  if (f > 0.0f && p > 0.0f && isfinite(p) && isfinite(f)) return __fdiv_rn(__fmul_rn(p, p), f);
  return 0.0f;
}

// The smallest fp16 value >= v (v >= 0); values above the fp16 range become +inf.
__device__ __forceinline__ unsigned short half_round_up(float v) {
  __half h = __float2half_rn(v);
  unsigned short u = __half_as_ushort(h);
  if (__half2float(h) < v) ++u;  // v >= 0: the next encoding is the next larger value (or inf)
  return u;
}

// Bound planes, [T][H+3][Wp] 32-bit words of two fp16 values, each rounded up, zero in the
// padding (nu2 = 0 outside the image):
//  * pool = 1 (two-row blocks): with M2(y) = max(nu2(y), nu2(y+1)) at column x, word (t, r, x)
//    holds M2(r-3) (low half) and M2(r-1) (high half).  A thread summing the blocks (y, y+1)
//    and (y+2, y+3) at row offset dy reads the single word at r = y + dy + 3.
//  * pool = 0 (single rows): word (t, r, x) holds nu2(r-3) and nu2(r-2).  A thread summing rows
//    y .. y+3 reads the words at r = y + dy + 3 and r + 2.
// With three leading word rows, a word row outside 0 .. H+2 (which TMA fills with zeros) holds
// no image row.
__global__ void bound_prep_kernel(const float* __restrict__ psi, const float* __restrict__ phi,
                                  int T, int H, int W, int Wp, int pool,
                                  uint32_t* __restrict__ bound) {
  const size_t total = (size_t)T * (H + 3) * Wp;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % Wp);
    const size_t row = i / Wp;
    const int t = (int)(row / (H + 3)), r = (int)(row % (H + 3));
    const size_t plane = (size_t)t * H * W;
    auto m2 = [&](int y) {
      return fmaxf(nu2_at(psi, phi, H, W, plane, y, x), nu2_at(psi, phi, H, W, plane, y + 1, x));
    };
    const unsigned short lo =
        half_round_up(pool ? m2(r - 3) : nu2_at(psi, phi, H, W, plane, r - 3, x));
    const unsigned short hi =
        half_round_up(pool ? m2(r - 1) : nu2_at(psi, phi, H, W, plane, r - 2, x));
    bound[i] = (uint32_t)lo | ((uint32_t)hi << 16);
  }
}

// (psi, phi) interleaved, [T][H][W] float2: a full evaluation gathers both with one 8-byte load
// per epoch (one sector per lane instead of two).
__global__ void pair_planes_kernel(const float* __restrict__ psi, const float* __restrict__ phi,
                                   size_t n, float2* __restrict__ pairs) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (size_t)gridDim.x * blockDim.x)
    pairs[i] = make_float2(__ldg(psi + i), __ldg(phi + i));
}

// ---------------------------------------------------------------------------------------------
// Tile order.  A start pixel near a bright source in an epoch whose offsets are all small (the
// first night) gets a candidate pair from nearly every trajectory, so the few tiles around such
// sources carry most of the full evaluations; handed out last, they leave most SMs idle at the
// end.  The score of a tile is the number of pixels with nu2 >= tau in its footprint at each
// epoch whose offsets span at most `span` pixels; tiles are handed out in decreasing score
// (ties and unscored tiles in row-major order).  The order only schedules work: the results do
// not depend on it.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) tile_score_kernel(
    const uint32_t* __restrict__ bound, int T, int H, int W, int Wp, const float4* vbox,
    SearchConsts cs, int x_lo, int y_lo, int x_hi, int y_hi, int ntx, int tx, int ntiles,
    float tau, int span, unsigned long long* __restrict__ keys) {
  const int tile = blockIdx.x;
  if (tile >= ntiles) return;
  __shared__ unsigned int s_count;
  if (threadIdx.x == 0) s_count = 0u;
  __syncthreads();
  const float4 b = *vbox;  // vx min, vx max, vy min, vy max
  const int tx0 = x_lo + (tile % ntx) * tx, ty0 = y_lo + (tile / ntx) * S_TY;
  const int tx1 = min(tx0 + tx, x_hi), ty1 = min(ty0 + S_TY, y_hi);
  unsigned int cnt = 0u;
  for (int t = 0; t < T; ++t) {
    const int oxa = track_offset(b.x, cs.dt[t]), oxb = track_offset(b.y, cs.dt[t]);
    const int oya = track_offset(b.z, cs.dt[t]), oyb = track_offset(b.w, cs.dt[t]);
    if (oxb - oxa > span || oyb - oya > span) continue;
    const int xa = max(tx0 + oxa, 0), xb = min(tx1 - 1 + oxb, W - 1);
    const int ya = max(ty0 + oya, 0), yb = min(ty1 - 1 + oyb, H - 1);
    if (xa > xb || ya > yb) continue;
    const int w = xb - xa + 1, n = w * (yb - ya + 1);
    const uint32_t* plane = bound + (size_t)t * (H + 3) * Wp;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      const int y = ya + i / w, x = xa + i % w;
      // image row y (pool = 0) or the block of rows (y, y+1) (pool = 1): low half of word row y+3
      const float v = __half2float(__ushort_as_half((unsigned short)(__ldg(plane + (size_t)(y + 3) * Wp + x) & 0xffffu)));
      cnt += v >= tau ? 1u : 0u;
    }
  }
  atomicAdd(&s_count, cnt);
  __syncthreads();
  if (threadIdx.x == 0)
    keys[tile] = ((unsigned long long)(0xffffffffu - s_count) << 32) | (unsigned int)tile;
}

// One block sorts the ntiles keys (ntiles <= S_ORDER_MAX) in shared memory with a bitonic
// network and writes the tile order.
__global__ void __launch_bounds__(1024) tile_order_kernel(const unsigned long long* __restrict__ keys,
                                                          int ntiles, int32_t* __restrict__ order) {
  extern __shared__ unsigned long long sk[];
  int n = 1;
  while (n < ntiles) n <<= 1;
  for (int i = threadIdx.x; i < n; i += blockDim.x) sk[i] = i < ntiles ? keys[i] : ~0ull;
  __syncthreads();
  for (int k = 2; k <= n; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const unsigned long long a = sk[i], c = sk[l];
          const bool up = (i & k) == 0;
          if ((a > c) == up) {
            sk[i] = c;
            sk[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < ntiles; i += blockDim.x) order[i] = (int32_t)(sk[i] & 0xffffffffu);
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

// Percentile of the n smallest sorted values from its rank entry r = {lo, frac} (rank_table).
template <int J>
__device__ __forceinline__ float warp_percentile(const float (&s)[J], int n, int2 r) {
  const int lo = r.x, hi = min(lo + 1, n - 1);
  const float f = __int_as_float(r.y);
  const float a = warp_get_sorted<J>(s, lo), b = warp_get_sorted<J>(s, hi);
  return a + f * (b - a);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Writes rec[0..7]: L' (NaN when the pair is not eligible), alpha, nvalid | nkept << 16,
// mask words.  All lanes take part; lane 0 writes and gets L' back (the other lanes get NaN).
template <int J>
__device__ float eval_pair_warp(const float2* __restrict__ pairs, const EvalParams& ep, int x0,
                               int y0, const int2* __restrict__ off,
                               const float* __restrict__ dtf, uint32_t* rec, int lane) {
  float ps[J], ph[J], a[J];
  bool valid[J];
  const size_t plane = (size_t)ep.H * ep.W;
  // all of the lane's offset loads, then all of its (psi, phi) loads, then the tests (an epoch
  // off the image or beyond T reads element 0 of a plane and is masked off)
  int2 o[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int t = (j << 5) | lane;
    o[j] = t < ep.T ? __ldg(off + t) : make_int2(0, 0);
  }
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int t = (j << 5) | lane;
    const int x = x0 + o[j].x, y = y0 + o[j].y;
    valid[j] = t < ep.T && x >= 0 && x < ep.W && y >= 0 && y < ep.H;
    const size_t at = t < ep.T ? (size_t)t * plane + (valid[j] ? (size_t)y * ep.W + x : 0) : 0;
    const float2 pf = __ldg(pairs + at);
    ps[j] = pf.x;
    ph[j] = pf.y;
  }
#pragma unroll
  for (int j = 0; j < J; ++j) {
    valid[j] = valid[j] && ph[j] > 0.0f && isfinite(ps[j]) && isfinite(ph[j]);
    if (!valid[j]) {
      ps[j] = 0.0f;
      ph[j] = 0.0f;
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
    return NAN;
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
    if (ep.nu2_floor > 0.0f) {
      // Exact filter before the sort.  A percentile interpolates between the order statistics
      // of ranks lo and lo + 1 (rank table), so q_mid and q_hi are at most any value V with at
      // least min(lo + 2, n) valid values <= V, and q_lo is at least any value V with at most lo
      // valid values < V.  Candidates for the three V come from the sorted lightcurve values of
      // the first 32 epochs (a sample, 15 shuffle stages), taken a few ranks outward; counting
      // over all epochs (one warp reduction each) checks them.  When all three hold, the upper
      // clip bound is at most ub = V_mid + n_sigma C (V_hi - V_lo) (the same float32 operations
      // on larger operands, plus a margin for the rounding of the interpolation), every epoch
      // above ub is clipped, and by Cauchy-Schwarz LH' of any kept set is at most the square
      // root of the sum of nu2 = psi^2/phi (psi a for the flux curve, a^2 for the likelihood
      // curve) over the other valid epochs with psi > 0.  A pair whose sum is below
      // lh_min^2 (1 - 1e-3) cannot reach lh_min and skips the sort.  This drops the pairs whose
      // pruning bound passed only through a few bright epochs (a mover crossed once, spikes).
      // Without the checks (or the sample) ub is +inf: the sum over every valid epoch.
      float ub = INFINITY;
      float x = a[0];  // +inf where epoch `lane` is not valid
      const int m = __popc(__ballot_sync(0xffffffffu, valid[0]));
      if (m >= 16) {
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
          for (int d = k >> 1; d > 0; d >>= 1) {
            const float o = __shfl_xor_sync(0xffffffffu, x, d);
            const bool up = (lane & k) == 0;
            x = (((lane & d) == 0) == up) ? fminf(x, o) : fmaxf(x, o);
          }
        // sample ranks a few places outward of the quantiles (the sample's order statistics
        // scatter by about sqrt(m q (1 - q)) ranks)
        const int i_lo = max(0, (int)(ep.q_lo * (float)(m - 1)) - 3);
        const int i_mid = min(m - 1, (int)(ep.q_mid * (float)(m - 1)) + 4);
        const int i_hi = min(m - 1, (int)(ep.q_hi * (float)(m - 1)) + 4);
        const float v_lo = __shfl_sync(0xffffffffu, x, i_lo);
        const float v_mid = __shfl_sync(0xffffffffu, x, i_mid);
        const float v_hi = __shfl_sync(0xffffffffu, x, i_hi);
        unsigned int c_lo = 0u, c_mid = 0u, c_hi = 0u;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          c_lo += (valid[j] && a[j] < v_lo) ? 1u : 0u;
          c_mid += (valid[j] && a[j] <= v_mid) ? 1u : 0u;
          c_hi += (valid[j] && a[j] <= v_hi) ? 1u : 0u;
        }
        c_lo = __reduce_add_sync(0xffffffffu, c_lo);
        c_mid = __reduce_add_sync(0xffffffffu, c_mid);
        c_hi = __reduce_add_sync(0xffffffffu, c_hi);
        const int2* rk = rank_table(dtf);
        const int r_lo = __ldg(rk + rank_entry(0, nvalid)).x;
        const int r_mid = __ldg(rk + rank_entry(1, nvalid)).x;
        const int r_hi = __ldg(rk + rank_entry(2, nvalid)).x;
        if ((int)c_lo <= r_lo && (int)c_mid >= min(r_mid + 2, nvalid) &&
            (int)c_hi >= min(r_hi + 2, nvalid)) {
          const float spread = ep.n_sigma * (ep.c_sigma * (v_hi - v_lo));
          ub = v_mid + spread +
               1e-5f * (fabsf(v_mid) + fabsf(v_hi) + fabsf(v_lo) + spread) + 1e-30f;
          if (!(ub == ub)) ub = INFINITY;  // NaN (infinite values): no epoch is excluded
        }
      }
      float s_keep = 0.0f;
#pragma unroll
      for (int j = 0; j < J; ++j)
        if (valid[j] && ps[j] > 0.0f && !(a[j] > ub))
          s_keep += ep.clip_on ? a[j] * a[j] : ps[j] * a[j];
      // lane 0's total decides for the whole warp (lanes may differ in the last bit)
      if (__shfl_sync(0xffffffffu, warp_sum(s_keep), 0) < ep.nu2_floor) {
        if (lane == 0) {
          rec[0] = __float_as_uint(NAN);
          rec[2] = (uint32_t)nvalid;
        }
        return NAN;
      }
    }
    warp_bitonic_sort<J>(s, lane);
    const int2* rk = rank_table(dtf);
    const float x_lo = warp_percentile<J>(s, nvalid, __ldg(rk + rank_entry(0, nvalid)));
    const float x_mid = warp_percentile<J>(s, nvalid, __ldg(rk + rank_entry(1, nvalid)));
    const float x_hi = warp_percentile<J>(s, nvalid, __ldg(rk + rank_entry(2, nvalid)));
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
  float L = NAN;
  if (lane == 0) {
    float alpha = 0.0f;
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
  return L;
}

// ---------------------------------------------------------------------------------------------
// Half-warp full evaluation (32 < T <= 64): lanes 0-15 evaluate one (start pixel, trajectory)
// pair and lanes 16-31 another, with the same instruction stream.  Epoch t = 16 j + h (h = lane & 15) is
// slot j of lane h of the pair's half; J slots hold up to 16 J epochs.
// ---------------------------------------------------------------------------------------------
constexpr unsigned int kAll = 0xffffffffu;

// Sum over the 16 lanes of each half (every lane of a half gets its half's sum, in an order that
// depends on the lane: callers take one lane's value).
__device__ __forceinline__ float half_sum(float v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(kAll, v, o);
  return v;
}

// Ascending bitonic sort of each half's 16 J values (index (j << 4) | h): exchanges between
// lanes (distance < 16) stay inside the half; longer ones are between slots of a lane.
template <int J>
__device__ __forceinline__ void half_bitonic_sort(float (&v)[J], int h) {
#pragma unroll
  for (int k = 2; k <= 16 * J; k <<= 1) {
#pragma unroll
    for (int d = k >> 1; d > 0; d >>= 1) {
      if (d >= 16) {
        const int dj = d >> 4;
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const int jp = j ^ dj;
          if (jp > j) {
            const bool up = (((j << 4) | h) & k) == 0;
            const float x = v[j], y = v[jp];
            const float lo = fminf(x, y), hi = fmaxf(x, y);
            v[j] = up ? lo : hi;
            v[jp] = up ? hi : lo;
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const float other = __shfl_xor_sync(kAll, v[j], d);
          const bool up = (((j << 4) | h) & k) == 0;
          const bool lower = (h & d) == 0;
          v[j] = (lower == up) ? fminf(v[j], other) : fmaxf(v[j], other);
        }
      }
    }
  }
}

// Element r of each half's sorted values (r may differ between the halves; hb = lane & 16).
template <int J>
__device__ __forceinline__ float half_get_sorted(const float (&v)[J], int r, int hb) {
  float x = v[0];
#pragma unroll
  for (int j = 1; j < J; ++j)
    if ((r >> 4) == j) x = v[j];
  return __shfl_sync(kAll, x, hb | (r & 15));
}

// Percentile of the n smallest sorted values from its rank entry r = {lo, frac} (rank_table).
template <int J>
__device__ __forceinline__ float half_percentile(const float (&s)[J], int n, int2 r, int hb) {
  const int lo = r.x, hi = min(lo + 1, n - 1);
  const float f = __int_as_float(r.y);
  const float a = half_get_sorted<J>(s, lo, hb), b = half_get_sorted<J>(s, hi, hb);
  return a + f * (b - a);
}

// The gathered (psi, phi) of one pair for a half-warp.
template <int J>
struct HalfPair {
  float ps[J], ph[J];
  uint32_t inb;  // bit j: epoch 16 j + h lies on the image
};

// Issues the loads of one pair (none for a half without a pair).  The track offsets are
// recomputed from the pair's velocity with the plan's own arithmetic (track_offset on the same
// float dt), bit-identical to the stored ones, so no offset load precedes the gathers; an epoch
// off the image or beyond T reads element 0 of a plane and is masked off later.
template <int J>
__device__ __forceinline__ void half_gather(const float2* __restrict__ pairs, const EvalParams& ep,
                                            int x0, int y0, float2 v,
                                            const float* __restrict__ dtf, int h, bool active,
                                            HalfPair<J>& g) {
  const size_t plane = (size_t)ep.H * ep.W;
  g.inb = 0u;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int t = (j << 4) | h;
    float2 pf = make_float2(0.0f, 0.0f);
    if (active) {
      size_t at = 0;
      if (t < ep.T) {
        const float dt = __ldg(dtf + t);
        const int x = x0 + track_offset(v.x, dt), y = y0 + track_offset(v.y, dt);
        const bool in = x >= 0 && x < ep.W && y >= 0 && y < ep.H;
        g.inb |= (in ? 1u : 0u) << j;
        at = (size_t)t * plane + (in ? (size_t)y * ep.W + x : 0);
      }
      pf = __ldg(pairs + at);
    }
    g.ps[j] = pf.x;
    g.ph[j] = pf.y;
  }
}

// Evaluates each half's pair.  The lane of h = 0 of a half writes its rec[0..7]: L' (NaN when
// the pair is not eligible or cannot reach lh_min), alpha, nvalid | nkept << 16, mask words, and
// gets L' back (the other lanes get NaN).  All 32 lanes take part; steps that no half needs are
// skipped by the whole warp.
template <int J>
__device__ float eval_pair_half(HalfPair<J>& g, const EvalParams& ep,
                                const float* __restrict__ dtf, uint32_t* rec, int lane) {
  const int h = lane & 15, hb = lane & 16;
  const bool lead = h == 0;
  float* const ps = g.ps;
  float* const ph = g.ph;
  bool valid[J];
  int nvalid = 0;
#pragma unroll
  for (int j = 0; j < J; ++j) {
    valid[j] = ((g.inb >> j) & 1u) && ph[j] > 0.0f && isfinite(ps[j]) && isfinite(ph[j]);
    if (!valid[j]) {
      ps[j] = 0.0f;
      ph[j] = 0.0f;
    }
    nvalid += __popc((__ballot_sync(kAll, valid[j]) >> hb) & 0xffffu);
  }
  bool live = nvalid >= ep.min_obs && nvalid > 0;  // the same in every lane of a half
  auto dead = [&]() {
    if (lead) {
      rec[0] = __float_as_uint(NAN);
      rec[2] = (uint32_t)nvalid;
    }
    return NAN;
  };
  if (!__any_sync(kAll, live)) return dead();
  float a[J];
  bool keep[J];
  if (ep.clip) {
    float s[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      a[j] = valid[j] ? (ep.clip_on ? __fdiv_rn(ps[j], __fsqrt_rn(ph[j])) : __fdiv_rn(ps[j], ph[j]))
                      : INFINITY;
      s[j] = a[j];
    }
    if (ep.nu2_floor > 0.0f) {
      // Exact filter before the sort.  A percentile interpolates between the order statistics
      // of ranks lo and lo + 1 (rank table), so q_mid and q_hi are at most any value V with at
      // least min(lo + 2, n) valid values <= V, and q_lo is at least any value V with at most lo
      // valid values < V.  Candidates for the three V come from the sorted lightcurve values of
      // the half's first 32 epochs (a sample), taken a few ranks outward; counts over all
      // epochs check them.  When all three hold, the upper clip bound is at most
      // ub = V_mid + n_sigma C (V_hi - V_lo) (the same float32 operations on larger operands,
      // plus a margin for the rounding of the interpolation), every epoch above ub is clipped,
      // and by Cauchy-Schwarz LH' of any kept set is at most the square root of the sum of
      // nu2 = psi^2/phi (psi a for the flux curve, a^2 for the likelihood curve) over the other
      // valid epochs with psi > 0.  A pair whose sum is below lh_min^2 (1 - 1e-3) cannot reach
      // lh_min.  Without the checks (or the sample) ub is +inf: the sum over every valid epoch.
      float ub = INFINITY;
      float x0 = a[0], x1 = a[1];  // +inf where the epoch is not valid
      const int m = __popc((__ballot_sync(kAll, valid[0]) >> hb) & 0xffffu) +
                    __popc((__ballot_sync(kAll, valid[1]) >> hb) & 0xffffu);
      // ascending sort of the half's 32 samples (index (j << 4) | h, j = 0, 1)
#pragma unroll
      for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
        for (int d = k >> 1; d > 0; d >>= 1) {
          if (d == 16) {
            const float lo = fminf(x0, x1), hi = fmaxf(x0, x1);
            x0 = lo;  // k = 32: ascending
            x1 = hi;
          } else {
            const float o0 = __shfl_xor_sync(kAll, x0, d), o1 = __shfl_xor_sync(kAll, x1, d);
            const bool lower = (h & d) == 0;
            const bool up0 = (h & k) == 0, up1 = ((16 | h) & k) == 0;
            x0 = (lower == up0) ? fminf(x0, o0) : fmaxf(x0, o0);
            x1 = (lower == up1) ? fminf(x1, o1) : fmaxf(x1, o1);
          }
        }
      const float xs[2] = {x0, x1};
      // sample ranks a few places outward of the quantiles (the sample's order statistics
      // scatter by about sqrt(m q (1 - q)) ranks)
      const int i_lo = max(0, (int)(ep.q_lo * (float)(m - 1)) - 3);
      const int i_mid = min(m - 1, (int)(ep.q_mid * (float)(m - 1)) + 4);
      const int i_hi = min(m - 1, (int)(ep.q_hi * (float)(m - 1)) + 4);
      const float v_lo = half_get_sorted<2>(xs, i_lo, hb);
      const float v_mid = half_get_sorted<2>(xs, max(i_mid, 0), hb);
      const float v_hi = half_get_sorted<2>(xs, max(i_hi, 0), hb);
      // the three counts in one word (each at most 16 J <= 128 < 2^10)
      unsigned int c = 0u;
#pragma unroll
      for (int j = 0; j < J; ++j) {
        c += (valid[j] && a[j] < v_lo) ? 1u : 0u;
        c += (valid[j] && a[j] <= v_mid) ? (1u << 10) : 0u;
        c += (valid[j] && a[j] <= v_hi) ? (1u << 20) : 0u;
      }
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) c += __shfl_xor_sync(kAll, c, o);
      const int c_lo = (int)(c & 1023u), c_mid = (int)((c >> 10) & 1023u), c_hi = (int)(c >> 20);
      const int2* rk = rank_table(dtf);
      const int n_r = live ? nvalid : 0;
      const int r_lo = __ldg(rk + rank_entry(0, n_r)).x;
      const int r_mid = __ldg(rk + rank_entry(1, n_r)).x;
      const int r_hi = __ldg(rk + rank_entry(2, n_r)).x;
      if (m >= 16 && c_lo <= r_lo && c_mid >= min(r_mid + 2, nvalid) &&
          c_hi >= min(r_hi + 2, nvalid)) {
        const float spread = ep.n_sigma * (ep.c_sigma * (v_hi - v_lo));
        ub = v_mid + spread + 1e-5f * (fabsf(v_mid) + fabsf(v_hi) + fabsf(v_lo) + spread) + 1e-30f;
        if (!(ub == ub)) ub = INFINITY;  // NaN (infinite values): no epoch is excluded
      }
      float s_keep = 0.0f;
#pragma unroll
      for (int j = 0; j < J; ++j)
        if (valid[j] && ps[j] > 0.0f && !(a[j] > ub))
          s_keep += ep.clip_on ? a[j] * a[j] : ps[j] * a[j];
      // the half's lead lane's total decides for the half (lanes may differ in the last bit);
      // every lane takes part in the shuffles, live or not
      const float s_tot = __shfl_sync(kAll, half_sum(s_keep), hb);
      live = live && !(s_tot < ep.nu2_floor);
      if (!__any_sync(kAll, live)) return dead();
    }
    half_bitonic_sort<J>(s, h);
    const int2* rk = rank_table(dtf);
    const int n_r = live ? nvalid : 0;
    const float x_lo = half_percentile<J>(s, nvalid, __ldg(rk + rank_entry(0, n_r)), hb);
    const float x_mid = half_percentile<J>(s, nvalid, __ldg(rk + rank_entry(1, n_r)), hb);
    const float x_hi = half_percentile<J>(s, nvalid, __ldg(rk + rank_entry(2, n_r)), hb);
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
    const uint32_t b = (__ballot_sync(kAll, keep[j]) >> hb) & 0xffffu;
    mw[j >> 1] |= b << ((j & 1) * 16);
    nkept += __popc(b);
  }
  sp = half_sum(sp);
  sf = half_sum(sf);
  if (!lead) return NAN;
  if (!live) return dead();
  float L = NAN, alpha = 0.0f;
  if (nkept > 0 && sf > 0.0f) {
    L = __fdiv_rn(sp, __fsqrt_rn(sf));
    alpha = __fdiv_rn(sp, sf);
  }
  rec[0] = __float_as_uint(L);
  rec[1] = __float_as_uint(alpha);
  rec[2] = (uint32_t)nvalid | ((uint32_t)nkept << 16);
#pragma unroll
  for (int w = 0; w < 4; ++w) rec[3 + w] = mw[w];
  return L;
}

// ---------------------------------------------------------------------------------------------
// Thread-level full evaluation (T <= NT <= 32): one thread, one (start pixel, trajectory) pair
// ---------------------------------------------------------------------------------------------
template <int NT>
__device__ __forceinline__ void thread_bitonic_sort(float (&v)[NT]) {
#pragma unroll
  for (int k = 2; k <= NT; k <<= 1)
#pragma unroll
    for (int d = k >> 1; d > 0; d >>= 1)
#pragma unroll
      for (int i = 0; i < NT; ++i) {
        const int p = i ^ d;
        if (p > i) {
          const bool up = (i & k) == 0;
          const float a = v[i], b = v[p];
          v[i] = up ? fminf(a, b) : fmaxf(a, b);
          v[p] = up ? fmaxf(a, b) : fminf(a, b);
        }
      }
}

// Element idx of a register array (selects, no dynamically indexed local memory).
template <int NT>
__device__ __forceinline__ float sel_sorted(const float (&v)[NT], int idx) {
  float r = v[0];
#pragma unroll
  for (int k = 1; k < NT; ++k) r = (k == idx) ? v[k] : r;
  return r;
}

template <int NT>
__device__ __forceinline__ float sorted_percentile(const float (&loc)[NT], int n, int2 r) {
  const int lo = r.x, hi = min(lo + 1, n - 1);
  const float f = __int_as_float(r.y);
  const float a = sel_sorted<NT>(loc, lo), b = sel_sorted<NT>(loc, hi);
  return a + f * (b - a);
}

// One pair, one thread.  psi_t and phi_t stay in registers from the single gather; the
// lightcurve value of an epoch (flux psi/phi, or psi/sqrt(phi) when clip_on) is recomputed with
// the same IEEE operations where it is needed (sort input, clip test), so no epoch is read twice.
//
// The track offsets are recomputed from the pair's velocity with the plan's own arithmetic
// (track_offset on the same float dt), so they equal the stored ones bit for bit; this replaces
// T scattered offset loads per pair (one per lane and epoch) by one velocity load and broadcast
// loads of dt.  Returns L' (NaN when the pair is not eligible).  FILTER: only the gather and the
// exact filter below (no sort); returns NaN for a pair that cannot reach lh_min, +inf otherwise.
template <int NT, bool FILTER>
__device__ float eval_pair_thread(const float2* __restrict__ pairs,
                                  const EvalParams& ep, int x0, int y0, float2 v,
                                  const float* __restrict__ dtf, uint32_t* rec) {
  float pv[NT], fv[NT];
  uint32_t vm = 0u, inb = 0u;
  const size_t plane = (size_t)ep.H * ep.W;
  // every epoch's load is issued before any is used: an epoch off the image (or beyond T) reads
  // element 0 of its plane instead and is masked off afterwards, so the gathers overlap instead
  // of waiting one after another behind the bounds and validity tests
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    size_t at = 0;
    if (t < ep.T) {
      const float dt = __ldg(dtf + t);
      const int x = x0 + track_offset(v.x, dt), y = y0 + track_offset(v.y, dt);
      const bool in = x >= 0 && x < ep.W && y >= 0 && y < ep.H;
      inb |= (in ? 1u : 0u) << t;
      at = (size_t)t * plane + (in ? (size_t)y * ep.W + x : 0);
    }
    const float2 pf = __ldg(pairs + at);
    pv[t] = pf.x;
    fv[t] = pf.y;
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    const float p = pv[t], f = fv[t];
    if (((inb >> t) & 1u) && f > 0.0f && isfinite(p) && isfinite(f)) {
      vm |= 1u << t;
    } else {
      pv[t] = 0.0f;
      fv[t] = 0.0f;
    }
  }
  const int nvalid = __popc(vm);
  if (nvalid < ep.min_obs || nvalid == 0) {
    rec[0] = __float_as_uint(NAN);
    rec[2] = (uint32_t)nvalid;
    return NAN;
  }
  const bool on_lh = ep.clip_on != 0;
  auto curve = [&](int t) {
    return on_lh ? __fdiv_rn(pv[t], __fsqrt_rn(fv[t])) : __fdiv_rn(pv[t], fv[t]);
  };
  uint32_t km = vm;
  if (FILTER) {
    // Exact filter before the sort.  A percentile interpolates between the order statistics of
    // ranks lo and lo + 1 (rank table), so with the M largest and M smallest lightcurve values
    // kept in registers: q_mid and q_hi are at most the value of rank n - k (k = min(n - (lo + 1),
    // M) largest, which is at or above rank lo + 1), and q_lo is at least the value of rank
    // min(lo, M - 1) (at or below rank lo).  The upper clip bound is then at most
    // ub = V_mid + n_sigma C (V_hi - V_lo) (the same float32 operations on larger operands, plus
    // a margin for the rounding of the interpolation).  Every epoch above ub is clipped whatever
    // the quantiles are, and by Cauchy-Schwarz LH' of any kept set is at most the square root of
    // the sum of nu2 = psi^2/phi over the other valid epochs with psi > 0; a pair whose sum is
    // below lh_min^2 (1 - 1e-3) cannot reach lh_min.  Without the clip the sum runs over every
    // valid epoch.  This drops most pairs whose pruning bound passed only through a few bright
    // epochs (a +20 sigma spike, a mover crossed once) or through the other pixel of a two-row
    // block.  Returns NaN for a dropped pair, +inf for one that needs the full evaluation.
    if (!(ep.nu2_floor > 0.0f)) {
      rec[2] = (uint32_t)nvalid;
      return INFINITY;
    }
    // the M largest (descending) and the M smallest (ascending) lightcurve values
    constexpr int M = 8;
    float top[M], bot[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      top[i] = -INFINITY;
      bot[i] = INFINITY;
    }
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      if ((vm >> t) & 1u) {
        const float a = curve(t);
        float ch = a, cl = a;
#pragma unroll
        for (int i = 0; i < M; ++i) {
          const float hi = fmaxf(top[i], ch), lo = fminf(bot[i], cl);
          ch = fminf(top[i], ch);
          cl = fmaxf(bot[i], cl);
          top[i] = hi;
          bot[i] = lo;
        }
      }
    }
    float ub = INFINITY;
    if (ep.clip) {
      const int2* rk = rank_table(dtf);
      const int u_mid = min(__ldg(rk + rank_entry(1, nvalid)).x + 1, nvalid - 1);
      const int u_hi = min(__ldg(rk + rank_entry(2, nvalid)).x + 1, nvalid - 1);
      const int l_lo = __ldg(rk + rank_entry(0, nvalid)).x;
      // sorted[u] <= top[k - 1] for k = min(n - u, M); sorted[l] >= bot[min(l, M - 1)]
      const int k_mid = min(nvalid - u_mid, M) - 1, k_hi = min(nvalid - u_hi, M) - 1;
      const int k_lo = min(l_lo, M - 1);
      float v_mid = top[0], v_hi = top[0], v_lo = bot[0];
#pragma unroll
      for (int i = 1; i < M; ++i) {
        v_mid = i == k_mid ? top[i] : v_mid;
        v_hi = i == k_hi ? top[i] : v_hi;
        v_lo = i == k_lo ? bot[i] : v_lo;
      }
      const float spread = ep.n_sigma * (ep.c_sigma * (v_hi - v_lo));
      ub = v_mid + spread + 1e-5f * (fabsf(v_mid) + fabsf(v_hi) + fabsf(v_lo) + spread) + 1e-30f;
      if (!(ub == ub)) ub = INFINITY;  // NaN (infinite values): no epoch is excluded
    }
    float s_keep = 0.0f;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      if (((vm >> t) & 1u) && pv[t] > 0.0f) {
        const float a = curve(t);
        if (!(a > ub)) s_keep += on_lh ? a * a : pv[t] * a;
      }
    }
    rec[2] = (uint32_t)nvalid;
    return s_keep < ep.nu2_floor ? NAN : INFINITY;
  }
  if (ep.clip) {
    float loc[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) loc[t] = ((vm >> t) & 1u) ? curve(t) : INFINITY;
    thread_bitonic_sort<NT>(loc);
    const int2* rk = rank_table(dtf);
    const float x_lo = sorted_percentile<NT>(loc, nvalid, __ldg(rk + rank_entry(0, nvalid)));
    const float x_mid = sorted_percentile<NT>(loc, nvalid, __ldg(rk + rank_entry(1, nvalid)));
    const float x_hi = sorted_percentile<NT>(loc, nvalid, __ldg(rk + rank_entry(2, nvalid)));
    const float sg = ep.c_sigma * (x_hi - x_lo);
    const float lo_b = x_mid - ep.n_sigma * sg, hi_b = x_mid + ep.n_sigma * sg;
    km = 0u;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      if ((vm >> t) & 1u) {
        const float a = curve(t);
        if (a >= lo_b && a <= hi_b) km |= 1u << t;
      }
    }
  }
  // sums over the kept epochs, in epoch order
  float sp = 0.0f, sf = 0.0f;
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    if ((km >> t) & 1u) {
      sp += pv[t];
      sf += fv[t];
    }
  }
  const int nkept = __popc(km);
  float L = NAN, alpha = 0.0f;
  if (nkept > 0 && sf > 0.0f) {
    L = __fdiv_rn(sp, __fsqrt_rn(sf));
    alpha = __fdiv_rn(sp, sf);
  }
  rec[0] = __float_as_uint(L);
  rec[1] = __float_as_uint(alpha);
  rec[2] = (uint32_t)nvalid | ((uint32_t)nkept << 16);
  rec[3] = km;
  rec[4] = rec[5] = rec[6] = 0u;
  return L;
}

// ---------------------------------------------------------------------------------------------
// The search kernel
// ---------------------------------------------------------------------------------------------
struct SearchArgs {
  const float* psi;
  const float* phi;
  const float2* pairs;  // (psi, phi) interleaved, [T][H][W]
  uint32_t* recs;       // [S_REC_BLOCKS][S_QCAP][S_REC_WORDS] evaluation records, one set per block
  const uint32_t* bound;
  const int32_t* orig;
  const int2* offs;
  const float2* vsort;  // velocities in list order (thread evaluation recomputes the offsets)
  const float* dtf;     // [T] epoch offsets t_t - t_0 as float, as used for the track offsets
  const PlanRec* plan;
  float* out_lh;
  float* out_flux;
  int32_t* out_idx;
  uint16_t* out_nvalid;
  uint16_t* out_nkept;
  uint32_t* out_mask;
  Ctrl* ctrl;
  const int32_t* order;  // tile order (nullptr: row-major)
  EvalParams ep;
  int n_traj, nchunk, Wp;
  int x_lo, x_hi, y_lo, y_hi, ntx, nty, ntiles;
  int tx;  // tile width in pixels: 32 x columns per bound-pass thread
};

struct TmapSet {
  CUtensorMap m[S_NW * S_NH];  // box (width class w, height class h) at m[(w-1)*S_NH + h]
};

// A batch of stacks searched by one launch: the tiles of stack s (in schedule order) are the
// global tiles tile_base[s] .. tile_base[s+1]-1; the tile counter and statistics are shared.
struct BatchArgs {
  const SearchArgs* stacks;     // [nstacks], device memory
  const TmapSet* maps;          // [nstacks], device memory (64-byte aligned)
  const int* tile_base;         // [nstacks + 1]
  int nstacks, total_tiles;
  Ctrl* ctrl;
  unsigned int* done_tiles;     // [nstacks] tiles finished
  unsigned long long* done_ns;  // [nstacks] %globaltimer when the stack's last tile finished
};

// Stack of global tile g (binary search of the tile prefix).
__device__ __forceinline__ int batch_stack_of(const BatchArgs& B, int g) {
  int lo = 0, hi = B.nstacks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(B.tile_base + mid) <= g) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void tmap_acquire(const void* tmap) {
  asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                   reinterpret_cast<uint64_t>(tmap))
               : "memory");
}

// Shared memory of one kernel instance: the staging arena (one ring of staged rectangles per
// producer) and the tables, the pixel tables sized for the instance's tile width and the
// survivor list only where a thread-per-pair evaluation uses it.  The unified L1/shared memory
// of an SM is split in fixed steps (228, 196, 164, ... KB of shared memory); the driver takes the
// smallest step that holds the block and the rest is L1, which caches the evaluations' gathers.
// So the arena is sized per instance (arena_kb) to land below a step: 152 KB keeps every block
// under 196 KB (about 60 KB of L1; decam_half 226.8 ms with a 184 KB arena and 28 KB of L1,
// 224.6 ms with this), and the T > 32 kernels, whose evaluations dominate, keep 136 KB under
// 164 KB (about 92 KB of L1).
__host__ __device__ constexpr int arena_kb(int nt, bool batch, bool pool, int ncol) {
  return (nt <= 0 && !batch) ? 136 : 152;
}

template <int NT, bool BATCH, bool POOL, int NCOL>
struct SmemLayout {
  static constexpr int arena_bytes = arena_kb(NT, BATCH, POOL, NCOL) * 1024;
  static constexpr int ring_bytes = arena_bytes / S_PWARPS;
  static constexpr int npix = S_TX * NCOL * S_TY;  // start pixels of a tile
  static constexpr bool has_surv = NT > 0 || BATCH;
  static constexpr size_t arena = 0;
  static constexpr size_t qtraj = arena + arena_bytes;
  static constexpr size_t qpix = qtraj + S_QCAP * sizeof(int32_t);
  static constexpr size_t qnext = qpix + S_QCAP * sizeof(uint16_t);
  static constexpr size_t surv = qnext + S_QCAP * sizeof(int16_t);  // pairs past the filter
  static constexpr size_t head =
      (surv + (has_surv ? S_QCAP * sizeof(int16_t) : 0) + 15) / 16 * 16;  // [pixel]
  static constexpr size_t filled = head + npix * sizeof(int32_t);
  static constexpr size_t slots = (filled + npix + 15) / 16 * 16;          // S_D plan records
  static constexpr size_t sinfo = slots + S_D * sizeof(PlanRec);  // S_D x {offset, tile, bytes}
  static constexpr size_t full = sinfo + S_D * sizeof(int4);       // S_D mbarriers: data landed
  static constexpr size_t empty = full + S_D * sizeof(uint64_t);   // S_D mbarriers: slot released
  static constexpr size_t misc = empty + S_D * sizeof(uint64_t);
  static constexpr size_t sargs = misc + 128;  // consumers' copy of the tile's stack arguments
  static constexpr size_t total = sargs + (sizeof(SearchArgs) + 15) / 16 * 16;
  static_assert(total <= 232448, "shared memory budget");
  static_assert(slots % 16 == 0 && full % 8 == 0, "alignment");
  static_assert(S_REGION_MAX <= ring_bytes, "a ring holds the largest staged rectangle");
};

// Admission threshold of a pixel for the fp16 bound sums.  With every stored term rounded up,
// an RN fp16 sum of T non-negative terms satisfies  exact <= sum (1 + 2^-11)^T + T 2^-25  (the
// second term covers subnormal rounding), and the fp32 nu2 itself is within (1 + 2^-23) of the
// exact value.  A pair is dropped only if  sum < (thr^2 (1 - 1e-4) - slack) * scale, which
// implies  sqrt(exact bound) < thr.
__device__ __forceinline__ float admission_threshold(float thr, const EvalParams& ep) {
  if (!(thr > 0.0f)) return -1.0f;
  return (thr * thr * S_PRUNE_MARGIN - ep.prune_slack) * ep.prune_scale;
}

// The largest fp16 value <= x (admission thresholds are compared in fp16; rounding them down
// keeps every pair the fp32 test would keep).
__device__ __forceinline__ __half half_round_down(float x) {
  __half h = __float2half_rn(x);
  if (__half2float(h) > x) {
    unsigned short u = __half_as_ushort(h);
    u = (u & 0x8000u) ? (unsigned short)(u + 1u) : (unsigned short)(u - 1u);
    h = __ushort_as_half(u);
  }
  return h;
}

// mbar_wait_parity for the consumers: the flag set by a warp that gave up is checked only while
// waiting (the fast path is one try_wait), so the other warps stop promptly after a timeout.
__device__ __forceinline__ bool consumer_wait(uint64_t* bar, uint32_t parity,
                                              const unsigned int* abort_flag,
                                              unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_try_wait(bar, parity, 20000u)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (;;) {
    if (*(volatile const unsigned int*)abort_flag != 0u) return false;
    if (mbar_try_wait(bar, parity, 20000u)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}

__device__ __forceinline__ void consumer_sync() {
  asm volatile("bar.sync 1, %0;" ::"r"(S_CTHREADS) : "memory");
}

// Barrier of the consumer threads that returns whether any of them passed pred != 0.
__device__ __forceinline__ bool consumer_sync_or(int pred) {
  int r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\t"
      "bar.red.or.pred q, 1, %2, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"(pred), "r"(S_CTHREADS)
      : "memory");
  return r != 0;
}

// Shared tile sequence of the producers: producer 0 takes tiles from the global counter and
// publishes them; the others read them in the same order.
struct TileRing {
  int tile[4];
  unsigned int published;
};

// Producer warp p (all lanes run the same control flow; lane 0 issues) handles the iterations
// it with it % S_PWARPS == p: for each, it retires its own released iterations (in order,
// waiting on their 'empty' barriers) until its slot and room in its own arena ring are free,
// writes the plan record and copies the staged rectangle (one TMA box).  Each producer issuing
// its own TMA operations keeps the per-thread issue cost of TMA off the critical path.  The plan
// records of the next 32 iterations are loaded by the 32 lanes at once.  The slot after the last
// tile carries tile -1.
template <bool BATCH>
__device__ void producer_loop(const TmapSet& pmaps, const SearchArgs& A0, const BatchArgs& B,
                              unsigned char* ring, int ring_base, PlanRec* slots, int4* sinfo,
                              uint64_t* full, uint64_t* empty, unsigned int* s_abort,
                              TileRing* tr, long long* issued_out, int pw, int lane,
                              unsigned int loads_per_traj, int ring_bytes) {
  Ctrl* const ctrl = BATCH ? B.ctrl : A0.ctrl;
  const int total_tiles = BATCH ? B.total_tiles : A0.ntiles;
  int cur_stack = -1;
  long long it_base = 0;        // global iteration number of the current tile's first iteration
  long long oldest = pw;        // oldest unretired iteration of this producer
  long long last_issued = -1;
  int head = 0, tail = 0, live = 0;  // ring: [tail, head) cyclically, `live` regions
  unsigned long long n_staged = 0, n_uniform = 0, n_direct = 0, n_bytes = 0;  // lane 0
  for (int k = 0;; ++k) {
    int tile = 0;  // the global tile (counter value) first; resolved below
    if (pw == 0) {
      if (lane == 0) {
        tile = (int)atomicAdd(&ctrl->tile_counter, 1u);
        tr->tile[k & 3] = tile;
        __threadfence_block();
        *(volatile unsigned int*)&tr->published = (unsigned int)(k + 1);
      }
    } else if (lane == 0) {
      const unsigned long long t0 = globaltimer_ns();
      while (*(volatile unsigned int*)&tr->published <= (unsigned int)k) {
        if (*(volatile unsigned int*)s_abort != 0u || globaltimer_ns() - t0 > kWaitLimitNs) {
          tile = -2;
          break;
        }
        __nanosleep(32);
      }
      if (tile != -2) {
        __threadfence_block();
        tile = *(volatile int*)&tr->tile[k & 3];
      }
    }
    tile = __shfl_sync(0xffffffffu, tile, 0);
    if (tile == -2) {
      if (lane == 0 && atomicExch(s_abort, 1u) == 0u) atomicOr(&ctrl->err, kErrTimeout);
      break;
    }
    const bool last = tile >= total_tiles;
    // the tile's stack, its arguments and its tile within the stack (in the stack's tile order)
    int stack = 0;
    const SearchArgs* Sp = &A0;
    const TmapSet* maps = &pmaps;
    if (BATCH && !last) {
      stack = batch_stack_of(B, tile);
      Sp = B.stacks + stack;
      maps = B.maps + stack;
      tile -= __ldg(B.tile_base + stack);
      if (stack != cur_stack) {  // the stack's tensor maps were written before the launch
        for (int i = lane; i < S_NW * S_NH; i += 32) {
          tmap_acquire(&maps->m[i]);
          prefetch_tmap(&maps->m[i]);
        }
        __syncwarp();
        cur_stack = stack;
      }
    }
    const PlanRec* const plan = Sp->plan;
    const int T = last ? 1 : Sp->ep.T;
    if (!last && Sp->order) tile = __ldg(Sp->order + tile);
    const int n_it = last ? 1 : Sp->nchunk * T;
    const int tx0 = last ? 0 : Sp->x_lo + (tile % Sp->ntx) * Sp->tx;
    const int ty0 = last ? 0 : Sp->y_lo + (tile / Sp->ntx) * S_TY;
    // this producer's iterations of the tile: q = first_q, first_q + S_PWARPS, ...
    const int first_q = (int)(((pw - it_base) % S_PWARPS + S_PWARPS) % S_PWARPS);
    for (int qb = first_q; qb < n_it; qb += 32 * S_PWARPS) {
      int4 rec[sizeof(PlanRec) / 16];
#pragma unroll
      for (int i = 0; i < (int)(sizeof(PlanRec) / 16); ++i) rec[i] = make_int4(0, 0, 0, 0);
      const int my_q = qb + lane * S_PWARPS;
      if (!last && my_q < n_it) {
        const int4* src = reinterpret_cast<const int4*>(plan + my_q);
#pragma unroll
        for (int i = 0; i < (int)(sizeof(PlanRec) / 16); ++i) rec[i] = __ldg(src + i);
      }
      const int4 mine = rec[0];
      for (int kk = 0; kk < 32; ++kk) {
        const int q = qb + kk * S_PWARPS;
        if (q >= n_it) break;
        const long long it = it_base + q;
        const int t = last ? 0 : epoch_of(q % T, T);
        const int slot = (int)(it % S_D);
        int4 b;
        b.x = __shfl_sync(0xffffffffu, mine.x, kk);
        b.y = __shfl_sync(0xffffffffu, mine.y, kk);
        b.z = __shfl_sync(0xffffffffu, mine.z, kk);
        b.w = __shfl_sync(0xffffffffu, mine.w, kk);
        const int mode = b.w & S_MODE_MASK;
        const int sz = (!last && mode) ? stage_width(mode) * stage_height(b.z) * 4 : 0;
        int pos = 0;
        for (;;) {
          bool room = it - oldest < S_D;
          if (room && sz > 0) {
            if (live == 0) {
              head = tail = 0;
              pos = 0;
            } else if (head > tail) {
              if (head + sz <= ring_bytes) pos = head;
              else if (sz <= tail) pos = 0;
              else room = false;
            } else if (head + sz <= tail) {
              pos = head;
            } else {
              room = false;
            }
          }
          if (room) break;
          // retire this producer's oldest iteration once every consumer warp has released it
          const bool ok = *(volatile unsigned int*)s_abort == 0u &&
                          mbar_wait_parity(&empty[oldest % S_D], (uint32_t)((oldest / S_D) & 1));
          if (!__all_sync(0xffffffffu, ok)) {
            if (lane == 0 && atomicExch(s_abort, 1u) == 0u) atomicOr(&ctrl->err, kErrTimeout);
            *issued_out = last_issued;
            return;
          }
          const int4 so = sinfo[oldest % S_D];
          if (so.z > 0) {
            --live;
            for (long long j = oldest + S_PWARPS; j < it; j += S_PWARPS) {
              const int4 sj = sinfo[j % S_D];
              if (sj.z > 0) {
                tail = sj.x - ring_base;
                break;
              }
            }
          }
          oldest += S_PWARPS;
        }
        if (sz > 0) {
          if (live == 0) tail = pos;
          head = pos + sz;
          ++live;
        }
        __syncwarp();  // every lane has read sinfo before this slot is rewritten
        if (!last && lane == kk) {  // the plan record, from the registers of the lane holding it
          int4* dst = reinterpret_cast<int4*>(&slots[slot]);
#pragma unroll
          for (int i = 0; i < (int)(sizeof(PlanRec) / 16); ++i) dst[i] = rec[i];
        }
        __syncwarp();
        if (lane == 0) {
          sinfo[slot] = make_int4(ring_base + pos, last ? -1 : tile, sz, stack);
          if (sz == 0) {
            mbar_arrive(&full[slot]);
          } else if (KB_BOUNDS_CHECK && ((tx0 + b.x) & 3) != 0) {
            // checked build: a TMA x coordinate off the 16-byte grid is reported, not issued
            atomicOr(&ctrl->err, kErrBounds);
            mbar_arrive(&full[slot]);
          } else {  // word row = first image row + 3 (the planes carry three leading rows)
            mbar_arrive_expect_tx(&full[slot], (uint32_t)sz);
            tma_load_3d(ring + pos, &maps->m[(mode - 1) * S_NH + b.z], &full[slot], tx0 + b.x,
                        ty0 + b.y + 3, t);
          }
        }
        if (!last && lane == 0) {
          if (mode == 0) ++n_direct;
          else if (b.w & S_UNIFORM_BIT) ++n_uniform;
          else ++n_staged;
          n_bytes += (unsigned long long)sz;
        }
        last_issued = it;
        __syncwarp();
      }
    }
    it_base += n_it;
    if (last) break;
  }
  if (lane == 0) {
    if (pw == 0 && blockIdx.x == 0) ctrl->loads_per_traj = loads_per_traj;
    atomicAdd(&ctrl->it_staged, n_staged);
    atomicAdd(&ctrl->it_uniform, n_uniform);
    atomicAdd(&ctrl->it_direct, n_direct);
    atomicAdd(&ctrl->tma_bytes, n_bytes);
  }
  *issued_out = last_issued;
}

// Shared-memory loads with 32-bit shared-window addresses (the staged regions are addressed
// through offsets read from shared memory; explicit forms keep the loop on 32-bit arithmetic).
__device__ __forceinline__ uint32_t lds_u32(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
  return v;
}
template <int OFF>
__device__ __forceinline__ uint32_t lds_u32_off(uint32_t addr) {
  uint32_t v;
  asm volatile("ld.shared.u32 %0, [%1+%2];" : "=r"(v) : "r"(addr), "n"(OFF));
  return v;
}
__device__ __forceinline__ int4 lds_v4(uint32_t addr) {
  int4 v;
  asm volatile("ld.shared.v4.s32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "r"(addr));
  return v;
}

// Sums one staged (chunk, epoch), a rectangle of `pitch`-word rows, into the fp16 accumulators.
// POOL, NCOL = 2: the thread's two columns x and x + 32; per trajectory one address add, two
// shared loads (the second at an immediate offset, 32 words on) and two fp16x2 adds; each word
// holds the thread's two blocks of a column (acc[c]).  POOL, NCOL = 1: one column, one load and
// one add (acc[0]).  Otherwise one column, its two row pairs two rows apart (acc[0] rows 0-1,
// acc[1] rows 2-3).  One code path for every box width (the pitch only
// moves the row bases).  uniform: all trajectories share rel[0] (the same values in the same
// order as the general path).
template <bool POOL, int NCOL>
__device__ __forceinline__ void accumulate_stage(__half2 (&acc)[2][S_C], const unsigned char* st,
                                                 int pitch, bool uniform, const PlanRec* slot,
                                                 int warp, int lane, int box_bytes,
                                                 unsigned int* err) {
  // words per trajectory: two (two columns, or two row pairs), or one (two-row blocks of one
  // column: both blocks of the thread in one word)
  constexpr bool TWO = !(POOL && NCOL == 1);
  const uint32_t base = smem_u32(st) + (uint32_t)(warp * S_ROWS * pitch + lane) * 4u;
  const uint32_t base1 = base + 8u * (uint32_t)pitch;  // two rows further (single rows only)
  // checked build: the last byte this thread reads for a trajectory at offset rel lies in the box
  const uint32_t first = (uint32_t)(warp * S_ROWS * pitch + lane) * 4u;
  const uint32_t span = (TWO ? (POOL ? 4u * S_TX : 8u * (uint32_t)pitch) : 0u) + 4u;
  auto outside = [&](uint32_t rel) {
    if (!KB_BOUNDS_CHECK) return false;
    const bool bad = (int)rel < 0 || first + rel + span > (uint32_t)box_bytes;
    if (bad) atomicOr(err, kErrBounds);
    return bad;
  };
  if (uniform) {
    const uint32_t r0 = (uint32_t)slot->rel[0];
    if (outside(r0)) return;
    const uint32_t w0 = lds_u32(base + r0);
    uint32_t w1 = 0u;
    if (TWO) w1 = POOL ? lds_u32_off<4 * S_TX>(base + r0) : lds_u32(base1 + r0);
#pragma unroll
    for (int v = 0; v < S_C; ++v) {
      acc[0][v] = __hadd2(acc[0][v], *reinterpret_cast<const __half2*>(&w0));
      if (TWO) acc[1][v] = __hadd2(acc[1][v], *reinterpret_cast<const __half2*>(&w1));
    }
    return;
  }
  const uint32_t relv = smem_u32(slot->rel);
#pragma unroll
  for (int vq = 0; vq < S_C / 4; ++vq) {
    const int4 r4 = lds_v4(relv + 16u * vq);
    const int rr[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (outside((uint32_t)rr[u])) continue;
      const uint32_t q = base + (uint32_t)rr[u];
      const uint32_t w0 = lds_u32(q);
      acc[0][vq * 4 + u] = __hadd2(acc[0][vq * 4 + u], *reinterpret_cast<const __half2*>(&w0));
      if (TWO) {
        const uint32_t w1 = POOL ? lds_u32_off<4 * S_TX>(q) : lds_u32(base1 + (uint32_t)rr[u]);
        acc[1][vq * 4 + u] = __hadd2(acc[1][vq * 4 + u], *reinterpret_cast<const __half2*>(&w1));
      }
    }
  }
}

// Inserts (L, j, record) into the ordered list of window pixel wp that holds nf entries
// (LH' descending, trajectory index ascending).  Returns true if it entered the list.
__device__ __noinline__ bool insert_sorted(const SearchArgs& A, size_t wp, int K, int mw, int nf,
                                           float L, int j, const uint32_t* rc) {
  if (KB_BOUNDS_CHECK &&
      wp >= (size_t)(A.x_hi - A.x_lo) * (size_t)(A.y_hi - A.y_lo)) {  // outside the window
    atomicOr(&A.ctrl->err, kErrBounds);
    return false;
  }
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

// NT > 0: thread-per-pair evaluation with an NT-wide sorting network (T <= NT <= 32);
// NT == -1: two pairs per warp, one per half-warp, with J slots per lane (32 < T <= 16 J);
// NT == 0: warp-per-pair evaluation with J epochs per lane (32 < T <= 32 J).
//
// BATCH: the tiles of several stacks (BatchArgs), each with its own T; the evaluation path is
// chosen per tile from the stack's T (the template arguments are unused).
//
// POOL: the bound planes hold two-row block maxima (see bound_prep_kernel); a passing block
// queues both of its pixels.  Otherwise the planes hold single rows and each pixel is tested on
// its own sum.
template <int NT, int J, bool BATCH, bool POOL, int NCOL>
__global__ void __launch_bounds__(S_THREADS, 1)
search_kernel(const __grid_constant__ TmapSet maps, const SearchArgs A0, const BatchArgs B) {
  extern __shared__ __align__(1024) unsigned char smem[];
  using SL = SmemLayout<NT, BATCH, POOL, NCOL>;
  unsigned char* arena = smem + SL::arena;
  int32_t* q_traj = reinterpret_cast<int32_t*>(smem + SL::qtraj);
  uint16_t* q_pix = reinterpret_cast<uint16_t*>(smem + SL::qpix);
  int16_t* q_next = reinterpret_cast<int16_t*>(smem + SL::qnext);
  int16_t* q_surv = reinterpret_cast<int16_t*>(smem + SL::surv);
  PlanRec* slots = reinterpret_cast<PlanRec*>(smem + SL::slots);
  int4* sinfo = reinterpret_cast<int4*>(smem + SL::sinfo);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + SL::full);
  uint64_t* empty = reinterpret_cast<uint64_t*>(smem + SL::empty);
  int* head = reinterpret_cast<int*>(smem + SL::head);
  uint8_t* s_filled = reinterpret_cast<uint8_t*>(smem + SL::filled);
  unsigned int* s_qcount = reinterpret_cast<unsigned int*>(smem + SL::misc);
  unsigned int* s_evals = s_qcount + 1;
  unsigned int* s_ins = s_qcount + 2;
  unsigned int* s_abort = s_qcount + 3;
  int* s_tile = reinterpret_cast<int*>(s_qcount + 4);
  TileRing* tr = reinterpret_cast<TileRing*>(s_qcount + 5);       // 20 bytes
  int* s_stack = reinterpret_cast<int*>(s_qcount + 10);
  long long* s_issued = reinterpret_cast<long long*>(smem + SL::misc + 48);  // [2]
  // stage counters: pairs with n_valid >= min_obs, pairs reaching lh_min, and the sums of
  // n_kept and n_valid over the latter
  unsigned int* s_stage = reinterpret_cast<unsigned int*>(smem + SL::misc + 64);     // [2]
  unsigned long long* s_stage64 =
      reinterpret_cast<unsigned long long*>(smem + SL::misc + 80);                   // [2]
  // s_stage[2] (misc + 72): pairs of the current flush that need the full evaluation
  SearchArgs* s_args = reinterpret_cast<SearchArgs*>(smem + SL::sargs);
  Ctrl* const ctrl = BATCH ? B.ctrl : A0.ctrl;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // tile geometry: NCOL columns per bound-pass thread, TXW = 2^TXS pixels wide; NACC fp16x2 sums
  // per trajectory (two columns, or two row pairs, or one word of two blocks)
  constexpr int TXW = S_TX * NCOL, TXS = NCOL == 2 ? 6 : 5;
  constexpr int NACC = (POOL && NCOL == 1) ? 1 : 2;
  static_assert((NCOL == 1 || (NCOL == 2 && POOL)) && (1 << TXS) == TXW && TXW * S_TY == SL::npix,
                "tile geometry");

  for (int i = tid; i < SL::npix; i += S_THREADS) head[i] = -1;
  if (tid == 0) {
    for (int i = 0; i < S_D; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], S_CWARPS);
    }
    *s_qcount = 0u;
    *s_evals = 0u;
    *s_ins = 0u;
    s_stage[0] = s_stage[1] = s_stage[2] = 0u;
    s_stage64[0] = s_stage64[1] = 0ull;
    *s_abort = 0u;
    *s_tile = -1;
    tr->published = 0u;
    s_issued[0] = s_issued[1] = -1;
    fence_mbar_init();
  }
  __syncthreads();

  if (warp >= S_CWARPS) {
    // ------------------------------- producer warps --------------------------------------
    const int pw = warp - S_CWARPS;
    if (!BATCH && pw == 0)
      for (int i = lane; i < S_NW * S_NH; i += 32) prefetch_tmap(&maps.m[i]);
    long long issued = -1;
    producer_loop<BATCH>(maps, A0, B, arena + pw * SL::ring_bytes, pw * SL::ring_bytes, slots,
                         sinfo, full, empty, s_abort, tr, &issued, pw, lane, (unsigned int)NACC,
                         SL::ring_bytes);
    if (lane == 0) s_issued[pw] = issued;
  } else {
    // ------------------------------- consumer warps --------------------------------------
    // consumer iteration counter: only its low bits (slot, phase parity) are used, and they
    // agree with the producers' 64-bit count modulo 2^32 (S_D divides 2^32)
    uint32_t it = 0u;
    for (;;) {
      // the first slot of the next tile names it (-1: none left) and its stack; decided by one
      // thread
      consumer_sync();
      if (tid == 0) {
        const int slot0 = (int)(it % S_D);
        const bool ok = consumer_wait(&full[slot0], (it / S_D) & 1u, s_abort);
        if (!ok && atomicExch(s_abort, 1u) == 0u) atomicOr(&ctrl->err, kErrTimeout);
        *s_tile = ok ? sinfo[slot0].y : -1;
        *s_stack = ok ? sinfo[slot0].w : 0;
      }
      consumer_sync();
      const int tile = *s_tile;
      if (tile < 0) break;
      const int stack = *s_stack;
      if (BATCH) {  // the stack's arguments, copied once per tile
        if (warp == 0) {
          const uint32_t* src = reinterpret_cast<const uint32_t*>(B.stacks + stack);
          uint32_t* dst = reinterpret_cast<uint32_t*>(s_args);
          for (int i = lane; i < (int)(sizeof(SearchArgs) / 4); i += 32) dst[i] = __ldg(src + i);
        }
        consumer_sync();
      }
      const SearchArgs& A = BATCH ? *s_args : A0;
      // evaluation records of this block (global memory, L2-resident: a few MB per launch)
      uint32_t* const recs = A.recs + (size_t)blockIdx.x * S_QCAP * S_REC_WORDS;
      const int T = A.ep.T, K = A.ep.K, mw = A.ep.mw;
      const float lh_min = A.ep.lh_min;
      const size_t wx = (size_t)(A.x_hi - A.x_lo);
      const int tx0 = A.x_lo + (tile % A.ntx) * TXW;
      const int ty0 = A.y_lo + (tile / A.ntx) * S_TY;
      const int px = tx0 + lane;  // column c of the thread: px + 32 c
      // per (column c, row i): bit c * S_ROWS + i of active, thr2[c * S_ROWS + i]
      float thr2[NCOL * S_ROWS];
      uint32_t active = 0u;
#pragma unroll
      for (int c = 0; c < NCOL; ++c)
#pragma unroll
        for (int i = 0; i < S_ROWS; ++i) {
          const int row = warp * S_ROWS + i;
          const int py = ty0 + row, pxc = px + S_TX * c;
          const bool act = pxc < A.x_hi && py < A.y_hi;
          active |= (act ? 1u : 0u) << (c * S_ROWS + i);
          s_filled[(row << TXS) | (lane + S_TX * c)] = 0;
          thr2[c * S_ROWS + i] = admission_threshold(lh_min, A.ep);
          if (act) {
            const size_t wp = (size_t)(py - A.y_lo) * wx + (size_t)(pxc - A.x_lo);
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

      // Evaluate every queued pair (all consumer threads), insert the results (owner threads
      // walk their pixels' lists), empty the queue.  Called by all consumer threads after a
      // consumer barrier.
      // all = false: evaluate only whole rounds (a multiple of the evaluating threads or warps)
      // and keep the remainder queued for the next flush, so no round leaves most threads idle.
      auto flush = [&](bool all) {
        const int nq_all = min((int)*s_qcount, S_QCAP);
        const int round = (NT > 0 || (BATCH && T <= 32)) ? S_CTHREADS
                          : (NT < 0 || (BATCH && T <= 64)) ? 2 * S_CWARPS
                                                           : S_CWARPS;
        const int nq = all ? nq_all : nq_all - nq_all % round;
        // a batch's arguments live in shared memory: the evaluations read theirs from registers
        EvalParams ep_copy;
        if (BATCH) ep_copy = A.ep;
        const EvalParams& EP = BATCH ? ep_copy : A.ep;
        const float2* const e_pairs = A.pairs;
        const int2* const e_offs = A.offs;
        const float2* const e_vs = A.vsort;
        const float* const e_dt = A.dtf;
        // a result that reaches lh_min is written to the block's records and joins its pixel's
        // list (pushed with one shared atomic); the others (almost all of them) are dropped
        auto keep = [&](int e, int pl, const uint32_t (&r)[S_REC_WORDS]) {
          uint4* dst = reinterpret_cast<uint4*>(recs + e * S_REC_WORDS);
          dst[0] = make_uint4(r[0], r[1], r[2], r[3]);
          dst[1] = make_uint4(r[4], r[5], r[6], 0u);
          q_next[e] = (int16_t)atomicExch(&head[pl], e);
          atomicAdd(&s_stage[1], 1u);
          atomicAdd(&s_stage64[0], (unsigned long long)(r[2] >> 16));
          atomicAdd(&s_stage64[1], (unsigned long long)(r[2] & 0xffffu));
        };
        // pairs eligible for the clip (n_valid >= max(min_obs, 1)), counted per warp
        auto count_valid = [&](bool evaluated, uint32_t nvk) {
          const uint32_t nv = nvk & 0xffffu;
          const bool v = evaluated && nv > 0u && (int)nv >= EP.min_obs;
          const unsigned int n = __popc(__ballot_sync(0xffffffffu, v));
          if (lane == 0 && n) atomicAdd(&s_stage[0], n);
        };
        // A pair per thread, in two phases: every queued pair is gathered and passed through
        // the exact filter (no sort); the pairs it cannot drop are collected and evaluated in
        // full, so that the sorting networks run in warps of pairs that all need them.
        auto by_thread = [&](auto nt) {
          constexpr int NTv = decltype(nt)::value;
          unsigned int* s_nsurv = s_stage + 2;
          for (int eb = 0; eb < nq; eb += S_CTHREADS) {
            const int e = eb + tid;
            uint32_t r[S_REC_WORDS];
            r[2] = 0u;
            bool more = false;
            if (e < nq) {
              const int pl = q_pix[e], j = q_traj[e];
              const float F = eval_pair_thread<NTv, true>(
                  e_pairs, EP, tx0 + (pl & (TXW - 1)), ty0 + (pl >> TXS), __ldg(e_vs + j), e_dt,
                  r);
              more = F > 0.0f;  // +inf: needs the full evaluation (NaN: dropped)
            }
            // the dropped pairs are counted here, the others after their full evaluation
            count_valid(e < nq && !more, r[2]);
            const unsigned int mb = __ballot_sync(0xffffffffu, more);
            unsigned int wpos = 0u;
            if (lane == 0 && mb) wpos = atomicAdd(s_nsurv, (unsigned int)__popc(mb));
            wpos = __shfl_sync(0xffffffffu, wpos, 0);
            if (more) q_surv[wpos + __popc(mb & ((1u << lane) - 1u))] = (int16_t)e;
          }
          consumer_sync();
          const int ns = (int)*s_nsurv;
          for (int kb = 0; kb < ns; kb += S_CTHREADS) {
            const int k = kb + tid;
            uint32_t r[S_REC_WORDS];
            r[2] = 0u;
            if (k < ns) {
              const int e = q_surv[k];
              const int pl = q_pix[e], j = q_traj[e];
              const float L = eval_pair_thread<NTv, false>(
                  e_pairs, EP, tx0 + (pl & (TXW - 1)), ty0 + (pl >> TXS), __ldg(e_vs + j), e_dt,
                  r);
              if (L >= lh_min) keep(e, pl, r);
            }
            count_valid(k < ns, r[2]);
          }
          consumer_sync();
          if (tid == 0) *s_nsurv = 0u;
        };
        // Two pairs per warp, one per half (32 < T <= 64)
        auto by_half = [&](auto jj) {
          constexpr int JH = decltype(jj)::value;
          const int half = lane >> 4;
          for (int eb = 2 * warp; eb < nq; eb += 2 * S_CWARPS) {
            const int e = eb + half;
            const bool active = e < nq;
            const int pl = active ? q_pix[e] : 0;
            const float2 v = active ? __ldg(e_vs + q_traj[e]) : make_float2(0.0f, 0.0f);
            HalfPair<JH> g;
            half_gather<JH>(e_pairs, EP, tx0 + (pl & (TXW - 1)), ty0 + (pl >> TXS), v, e_dt,
                            lane & 15, active, g);
            uint32_t r[S_REC_WORDS];
            r[2] = 0u;
            const float L = eval_pair_half<JH>(g, EP, e_dt, r, lane);
            if ((lane & 15) == 0 && active && L >= lh_min) keep(e, pl, r);
            // pairs eligible for the clip, counted by the halves' lead lanes
            const bool ev = (lane & 15) == 0 && active && (r[2] & 0xffffu) > 0u &&
                            (int)(r[2] & 0xffffu) >= EP.min_obs;
            const unsigned int n = __popc(__ballot_sync(0xffffffffu, ev));
            if (lane == 0 && n) atomicAdd(&s_stage[0], n);
          }
        };
        auto by_warp = [&](auto jj) {
          for (int e = warp; e < nq; e += S_CWARPS) {
            const int pl = q_pix[e];
            uint32_t r[S_REC_WORDS];
            const float L = eval_pair_warp<decltype(jj)::value>(
                e_pairs, EP, tx0 + (pl & (TXW - 1)), ty0 + (pl >> TXS),
                e_offs + (size_t)q_traj[e] * T, e_dt, r, lane);
            if (lane == 0 && L >= lh_min) keep(e, pl, r);
            const uint32_t nvk = __shfl_sync(0xffffffffu, r[2], 0);
            if (lane == 0 && (nvk & 0xffffu) > 0u && (int)(nvk & 0xffffu) >= EP.min_obs)
              atomicAdd(&s_stage[0], 1u);
          }
        };
        if (BATCH) {
          // three evaluation paths serve every stack (fewer registers than one per epoch
          // class): the 32-wide network sorts a T <= 16 lightcurve into the same order as the
          // 16-wide one (the extra entries sort last), so the results are bit-identical to
          // kb_search's, which takes the same half-warp and warp paths for T > 32
          if (T <= 32) by_thread(std::integral_constant<int, 32>{});
          else if (T <= 64) by_half(std::integral_constant<int, 4>{});
          else by_warp(std::integral_constant<int, 4>{});
        } else if (NT > 0) {
          by_thread(std::integral_constant<int, (NT > 0 ? NT : 1)>{});
        } else if (NT < 0) {
          by_half(std::integral_constant<int, J>{});
        } else {
          by_warp(std::integral_constant<int, J>{});
        }
        consumer_sync();
        if (tid == 0) atomicAdd(s_evals, (unsigned int)nq);
#pragma unroll 1
        for (int ci = 0; ci < NCOL * S_ROWS; ++ci) {
          const int c = ci / S_ROWS, i = ci % S_ROWS;
          const int row = warp * S_ROWS + i;
          const int pl = (row << TXS) | (lane + S_TX * c);
          int e = head[pl];
          if (e < 0) continue;
          const size_t wp =
              (size_t)(ty0 + row - A.y_lo) * wx + (size_t)(px + S_TX * c - A.x_lo);
          int nf = s_filled[pl];
          while (e >= 0) {
            const uint32_t* rc = recs + e * S_REC_WORDS;
            const float L = __uint_as_float(rc[0]);
            if (L >= lh_min) {  // false for NaN (pair not eligible)
              if (insert_sorted(A, wp, K, mw, nf, L, A.orig[q_traj[e]], rc)) {
                nf = min(nf + 1, K);
                atomicAdd(s_ins, 1u);
              }
            }
            e = q_next[e];
          }
          head[pl] = -1;
          s_filled[pl] = (uint8_t)nf;
          if (nf == K) {
            const float t2 = admission_threshold(fmaxf(A.out_lh[wp * K + K - 1], lh_min), A.ep);
#pragma unroll
            for (int ii = 0; ii < NCOL * S_ROWS; ++ii)
              if (ii == ci) thr2[ii] = t2;
          }
        }
        consumer_sync();
        // the remainder moves to the front (it lies above nq > remainder: no overlap)
        const int rem = nq_all - nq;
        for (int i = tid; i < rem; i += S_CTHREADS) {
          q_traj[i] = q_traj[nq + i];
          q_pix[i] = q_pix[nq + i];
        }
        if (tid == 0) *s_qcount = (unsigned int)rem;
        consumer_sync();
      };

      for (int c = 0; c < A.nchunk; ++c) {
        // per trajectory: POOL: column cc's (block of rows 0-1, block of rows 2-3) in acc[cc];
        // otherwise (row 0, row 1) in acc[0] and (row 2, row 3) in acc[1]
        __half2 acc[2][S_C];
#pragma unroll
        for (int pp = 0; pp < NACC; ++pp)
#pragma unroll
          for (int v = 0; v < S_C; ++v) acc[pp][v] = __float2half2_rn(0.0f);

        for (int k = 0; k < T; ++k, ++it) {
          const int t = epoch_of(k, T);  // the plan's epoch order
          const int slot = (int)(it % S_D);
          const bool ok = consumer_wait(&full[slot], (it / S_D) & 1u, s_abort);
          if (ok) {
            const PlanRec* rec = &slots[slot];
            const int mode = rec->box.w & S_MODE_MASK;
            const unsigned char* st = arena + sinfo[slot].x;
            if (mode != 0) {
              const bool uni = (rec->box.w & S_UNIFORM_BIT) != 0;
              accumulate_stage<POOL, NCOL>(acc, st, stage_width(mode), uni, rec, warp, lane,
                                           sinfo[slot].z, &ctrl->err);
            } else {
              // direct loads from the block planes (word row = first image row + 3)
              const uint32_t* bp = A.bound + (size_t)t * (A.ep.H + 3) * A.Wp;
#pragma unroll
              for (int v = 0; v < S_C; ++v) {
                const int2 o = __ldg(A.offs + (size_t)(c * S_C + v) * T + t);
#pragma unroll
                for (int pp = 0; pp < NACC; ++pp) {
                  // POOL: column pp of the thread; otherwise its row pair pp
                  const int x = px + o.x + (POOL ? S_TX * pp : 0);
                  const int r = ty0 + warp * S_ROWS + (POOL ? 0 : 2 * pp) + o.y + 3;
                  if (x >= 0 && x < A.Wp && r >= 0 && r < A.ep.H + 3) {
                    const uint32_t w = __ldg(bp + (size_t)r * A.Wp + x);
                    acc[pp][v] = __hadd2(acc[pp][v], *reinterpret_cast<const __half2*>(&w));
                  }
                }
              }
            }
          } else if (lane == 0 && atomicExch(s_abort, 1u) == 0u) {
            atomicOr(&ctrl->err, kErrTimeout);
          }
          __syncwarp();  // every lane's reads of the slot come before the warp's release
          if (lane == 0) mbar_arrive(&empty[slot]);
        }

        // ---- pairs whose bound reaches the admission threshold join the block queue ----
        const int nv = min(S_C, A.n_traj - c * S_C);
        const uint32_t vmask = nv >= 32 ? 0xffffffffu : ((1u << nv) - 1u);
        // POOL: a block passes against the smaller threshold of its two pixels; both are then
        // queued.  Otherwise each row against its own threshold.  cb[cc * S_ROWS + i]: the
        // passing trajectories of the pixel in column cc, row i.
        uint32_t cb[NCOL * S_ROWS];
#pragma unroll
        for (int pp = 0; pp < NACC; ++pp) {
          const int o = POOL ? pp * S_ROWS : 0;  // thresholds of column pp (POOL)
          const __half2 th =
              POOL ? __halves2half2(half_round_down(fminf(thr2[o], thr2[o + 1])),
                                    half_round_down(fminf(thr2[o + 2], thr2[o + 3])))
                   : __halves2half2(half_round_down(thr2[2 * pp]), half_round_down(thr2[2 * pp + 1]));
          uint32_t b0 = 0u, b1 = 0u;
          // most chunks have no candidate in the whole warp: test the maxima first
          __half2 mx = acc[pp][0];
#pragma unroll
          for (int v = 1; v < S_C; ++v) mx = __hmax2(mx, acc[pp][v]);
          if (__any_sync(0xffffffffu, __hge2_mask(mx, th) != 0u))
#pragma unroll
            for (int v = 0; v < S_C; ++v) {
              const uint32_t m = __hge2_mask(acc[pp][v], th);
              b0 |= (m & 1u) << v;
              b1 |= ((m >> 16) & 1u) << v;
            }
          if (POOL) {
            cb[o] = ((active >> o) & 1u) ? (b0 & vmask) : 0u;
            cb[o + 1] = ((active >> (o + 1)) & 1u) ? (b0 & vmask) : 0u;
            cb[o + 2] = ((active >> (o + 2)) & 1u) ? (b1 & vmask) : 0u;
            cb[o + 3] = ((active >> (o + 3)) & 1u) ? (b1 & vmask) : 0u;
          } else {
            cb[2 * pp] = ((active >> (2 * pp)) & 1u) ? (b0 & vmask) : 0u;
            cb[2 * pp + 1] = ((active >> (2 * pp + 1)) & 1u) ? (b1 & vmask) : 0u;
          }
        }
        // Append without a barrier: each warp reserves queue positions with one atomic; pairs
        // beyond the capacity stay in cb and are appended after a flush.
        for (;;) {
          int ncand = 0;
#pragma unroll
          for (int i = 0; i < NCOL * S_ROWS; ++i) ncand += __popc(cb[i]);
          int incl = ncand;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
          }
          const int wtotal = __shfl_sync(0xffffffffu, incl, 31);
          unsigned int wbase = 0;
          if (lane == 31 && wtotal > 0) wbase = atomicAdd(s_qcount, (unsigned int)wtotal);
          wbase = __shfl_sync(0xffffffffu, wbase, 31);
          int pos = (int)wbase + incl - ncand;
          bool deferred = false;
          if (ncand > 0) {
#pragma unroll
            for (int ci = 0; ci < NCOL * S_ROWS; ++ci) {
              uint32_t bits = cb[ci];
              uint32_t left = 0u;
              const uint16_t pl =
                  (uint16_t)(((warp * S_ROWS + ci % S_ROWS) << TXS) | (lane + S_TX * (ci / S_ROWS)));
              while (bits) {
                const int v = __ffs(bits) - 1;
                bits &= bits - 1u;
                if (pos < S_QCAP) {
                  q_traj[pos] = c * S_C + v;
                  q_pix[pos] = pl;
                } else {
                  left |= 1u << v;
                  deferred = true;
                }
                ++pos;
              }
              cb[ci] = left;
            }
          }
          // one barrier per chunk decides, for all consumer threads alike, whether to flush
          const bool full_q = consumer_sync_or(deferred);
          if (full_q || *(volatile unsigned int*)s_qcount >= (unsigned int)S_FLUSH_MIN) {
            flush(false);
            if (full_q) continue;  // append the pairs that did not fit
          }
          break;
        }
      }
      consumer_sync();
      if (*(volatile unsigned int*)s_qcount > 0u) flush(true);
      if (BATCH && tid == 0) {  // completion time of the stack whose last tile this was
        __threadfence();
        if (atomicAdd(B.done_tiles + stack, 1u) + 1u == (unsigned int)A.ntiles)
          B.done_ns[stack] = globaltimer_ns();
      }
    }
  }

  __syncthreads();
  if (tid == 0) {
    atomicAdd(&ctrl->evals, (unsigned long long)*s_evals);
    atomicAdd(&ctrl->inserts, (unsigned long long)*s_ins);
    atomicAdd(&ctrl->stage_valid, (unsigned long long)s_stage[0]);
    atomicAdd(&ctrl->stage_pass, (unsigned long long)s_stage[1]);
    atomicAdd(&ctrl->stage_kept, s_stage64[0]);
    atomicAdd(&ctrl->stage_nvalid, s_stage64[1]);
  }
  if (warp >= S_CWARPS && lane == 0 && *(volatile unsigned int*)s_abort != 0u) {
    // a wait gave up: wait (bounded) for this producer's last copies
    const long long n = s_issued[warp - S_CWARPS];
    for (long long j = n; j >= 0 && j > n - S_D; j -= S_PWARPS)
      mbar_wait_parity(&full[j % S_D], (uint32_t)((j / S_D) & 1));
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
  if (p->bound_rows < 0 || p->bound_rows > 2)
    return fail(KB_ERR_INVALID_ARG, "kb_search: bound_rows must be 0, 1 or 2");
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

namespace kb {

// Everything kb_search needs to know about one stack: its arguments for the search kernel, its
// tensor maps, and the inputs of its preparation kernels.
struct StackPrep {
  SearchArgs A;
  TmapSet maps;
  SearchConsts cs;
  WsLayout L;
  const float *psi, *phi, *vx, *vy;
  int T, H, W, n_traj;
  int x_lo, x_hi, y_lo, y_hi;
  char* ws;
  unsigned long long te;
  bool pool;  // sum two-row blocks (see pool_blocks)
};

// Whether the bound pass sums two-row blocks.  A block's sum bounds both of its pixels, at the
// price of looser sums: for an epoch of pure noise, psi/sqrt(phi) ~ N(0, 1), a pixel adds
// nu2 = z^2 (z > 0) with mean 1/2 and a block the maximum of two (correlated) such terms, about
// 3/4.  Blocks pay while their expected noise sum stays well below the admission threshold,
// taken as 1.5 T <= lh_min^2 (the decam workload: 39 <= 100); at T = 100 (75 against 100) they
// evaluate 38x more pairs and the search runs 10x slower, so single rows are summed there.
static bool pool_blocks(int T, float lh_min) {
  return !(lh_min > 0.0f) || 1.5 * T <= (double)lh_min * lh_min;
}

// Validates one stack, lays out its workspace, encodes its tensor maps and fills its kernel
// arguments (no launch).  ctrl: the control block the search kernel will use.
// SMs of the current device (148 if it cannot be queried: the tile width is then still valid).
static int sm_count() {
  if (g_num_sms == 0) {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && n > 0)
      g_num_sms = n;
    else
      (void)cudaGetLastError();  // clear the failed query's error
  }
  return g_num_sms > 0 ? g_num_sms : 148;
}

// Tiles of `cols` columns per bound-pass thread (32 * cols pixels wide; single-row bounds always
// take one column) over the stack's window; cols = 0: automatic (S_WIDE_MIN_WAVES).
static void set_tile_geometry(SearchArgs& A, bool pool, int cols) {
  if (cols == 0) {
    const long long wide = (long long)((A.x_hi - A.x_lo + 2 * S_TX - 1) / (2 * S_TX)) *
                           ((A.y_hi - A.y_lo + S_TY - 1) / S_TY);
    cols = wide >= (long long)S_WIDE_MIN_WAVES * sm_count() ? 2 : 1;
  }
  A.tx = S_TX * (pool ? cols : 1);
  A.ntx = (A.x_hi - A.x_lo + A.tx - 1) / A.tx;
  A.nty = (A.y_hi - A.y_lo + S_TY - 1) / S_TY;
  A.ntiles = A.ntx * A.nty;
}

static int prepare_stack(const char* who, const float* psi, const float* phi, const double* times,
                         int T, int H, int W, const float* vx, const float* vy, int n_traj,
                         const kb_search_params* p, float* out_lh, float* out_flux,
                         int32_t* out_idx, uint16_t* out_nvalid, uint16_t* out_nkept,
                         uint32_t* out_mask, char* ws, size_t ws_bytes, StackPrep& sp) {
  int rc = validate(psi, phi, times, T, H, W, vx, vy, n_traj, p);
  if (rc != KB_OK) return rc;
  if (!out_lh || !out_flux || !out_idx || !out_nvalid || !out_nkept || !out_mask)
    return fail(KB_ERR_INVALID_ARG, "%s: null output pointer", who);
  const WsLayout L = ws_layout(T, H, W, n_traj);
  if (!ws || ws_bytes < L.total)
    return fail(KB_ERR_WORKSPACE, "%s: workspace of %zu bytes, %zu needed", who, ws_bytes, L.total);
  if (reinterpret_cast<uintptr_t>(ws) % KB_WORKSPACE_ALIGN)
    return fail(KB_ERR_WORKSPACE, "%s: workspace not %d-byte aligned", who, KB_WORKSPACE_ALIGN);
  auto enc = get_encode_fn();
  if (!enc) return fail(KB_ERR_CUDA, "%s: cuTensorMapEncodeTiled unavailable", who);
  sp.L = L;
  sp.ws = ws;
  sp.psi = psi;
  sp.phi = phi;
  sp.vx = vx;
  sp.vy = vy;
  sp.T = T;
  sp.H = H;
  sp.W = W;
  sp.n_traj = n_traj;
  sp.x_lo = p->x_lo;
  sp.x_hi = p->x_hi;
  sp.y_lo = p->y_lo;
  sp.y_hi = p->y_hi;
  sp.cs = SearchConsts{};
  for (int t = 0; t < T; ++t) sp.cs.dt[t] = (float)(times[t] - times[0]);
  sp.pool = p->bound_rows == 2 || (p->bound_rows == 0 && pool_blocks(T, p->lh_min));
  sp.te = (unsigned long long)(p->x_hi - p->x_lo) * (p->y_hi - p->y_lo) * n_traj * T;
  uint32_t* bound = reinterpret_cast<uint32_t*>(ws + L.bound);
  for (int w = 1; w <= S_NW; ++w)
    for (int h = 0; h < S_NH; ++h) {
      cuuint64_t dims[3] = {(cuuint64_t)L.Wp, (cuuint64_t)H + 3, (cuuint64_t)T};
      cuuint64_t strides[2] = {(cuuint64_t)L.Wp * 4, (cuuint64_t)L.Wp * (H + 3) * 4};
      cuuint32_t boxd[3] = {(cuuint32_t)stage_width(w), (cuuint32_t)stage_height(h), 1u};
      cuuint32_t estr[3] = {1u, 1u, 1u};
      CUresult r = enc(&sp.maps.m[(w - 1) * S_NH + h], CU_TENSOR_MAP_DATA_TYPE_UINT32, 3, bound,
                       dims, strides, boxd, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                       CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
      if (r != CUDA_SUCCESS)
        return fail(KB_ERR_CUDA, "%s: cuTensorMapEncodeTiled failed (%d)", who, (int)r);
    }
  SearchArgs& A = sp.A;
  A = SearchArgs{};
  A.psi = psi;
  A.phi = phi;
  A.pairs = reinterpret_cast<float2*>(ws + L.pairs);
  A.recs = reinterpret_cast<uint32_t*>(ws + L.recs);
  A.bound = bound;
  A.orig = reinterpret_cast<int32_t*>(ws + L.orig);
  A.offs = reinterpret_cast<int2*>(ws + L.offs);
  A.vsort = reinterpret_cast<float2*>(ws + L.vsort);
  A.dtf = reinterpret_cast<float*>(ws + L.dtf);
  A.plan = reinterpret_cast<PlanRec*>(ws + L.plan);
  A.out_lh = out_lh;
  A.out_flux = out_flux;
  A.out_idx = out_idx;
  A.out_nvalid = out_nvalid;
  A.out_nkept = out_nkept;
  A.out_mask = out_mask;
  A.ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
  A.order = nullptr;
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
  A.ep.prune_scale = (float)(1.0 / (std::pow(1.0 + std::ldexp(1.0, -11), T) * (1.0 + 3e-7)));
  A.ep.prune_slack = (float)(T * std::ldexp(1.0, -25) * 2.0);
  A.ep.nu2_floor = p->lh_min > 0.0f ? (float)((double)p->lh_min * p->lh_min * (1.0 - 1e-3))
                                    : -INFINITY;
  A.n_traj = n_traj;
  A.nchunk = L.nchunk;
  A.Wp = L.Wp;
  A.x_lo = p->x_lo;
  A.x_hi = p->x_hi;
  A.y_lo = p->y_lo;
  A.y_hi = p->y_hi;
  set_tile_geometry(A, sp.pool, S_TILE_COLS_DEFAULT);
  return KB_OK;
}

// Enqueues a stack's preparation: velocity ordering, track offsets, staging plan, bound planes
// and (when sch.tile_order and the stack has at most S_ORDER_MAX tiles) its tile order.  Sets
// sp.A.order accordingly.
static int launch_prep(StackPrep& sp, const kb_schedule& sch, bool pool, cudaStream_t st) {
  const WsLayout& L = sp.L;
  char* ws = sp.ws;
  const int T = sp.T, H = sp.H, W = sp.W, n_traj = sp.n_traj;
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(ws + L.ctrl);
  float4* vbox = reinterpret_cast<float4*>(ws + L.vbox);
  uint32_t* keys = reinterpret_cast<uint32_t*>(ws + L.keys);
  uint32_t* counts = reinterpret_cast<uint32_t*>(ws + L.counts);
  uint32_t* cursor = reinterpret_cast<uint32_t*>(ws + L.cursor);
  int32_t* sorted = reinterpret_cast<int32_t*>(ws + L.sorted);
  int32_t* orig = reinterpret_cast<int32_t*>(ws + L.orig);
  int2* offs = reinterpret_cast<int2*>(ws + L.offs);
  float2* vsort = reinterpret_cast<float2*>(ws + L.vsort);
  float* dtf = reinterpret_cast<float*>(ws + L.dtf);
  PlanRec* plan = reinterpret_cast<PlanRec*>(ws + L.plan);
  uint32_t* bound = reinterpret_cast<uint32_t*>(ws + L.bound);
  if (g_num_sms == 0) {
    int dev = 0;
    KB_CUDA_TRY(cudaGetDevice(&dev));
    KB_CUDA_TRY(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  plan_reset_kernel<<<N_CELLS / 256, 256, 0, st>>>(ctrl, counts, sp.te, sp.A.ep.q_lo,
                                                    sp.A.ep.q_mid, sp.A.ep.q_hi,
                                                    reinterpret_cast<int2*>(dtf + KB_MAX_T));
  KB_LAUNCH_CHECK("plan_reset_kernel");
  plan_minmax_kernel<<<1, 1024, 0, st>>>(sp.vx, sp.vy, n_traj, vbox);
  KB_LAUNCH_CHECK("plan_minmax_kernel");
  plan_hist_kernel<<<(n_traj + 255) / 256, 256, 0, st>>>(sp.vx, sp.vy, n_traj, vbox, keys, counts);
  KB_LAUNCH_CHECK("plan_hist_kernel");
  plan_scan_kernel<<<1, 1024, 0, st>>>(counts, cursor);
  KB_LAUNCH_CHECK("plan_scan_kernel");
  plan_scatter_kernel<<<(n_traj + 255) / 256, 256, 0, st>>>(keys, n_traj, cursor, sorted);
  KB_LAUNCH_CHECK("plan_scatter_kernel");
  plan_cellsort_kernel<<<N_CELLS / 256, 256, 0, st>>>(counts, cursor, sorted);
  KB_LAUNCH_CHECK("plan_cellsort_kernel");
  plan_offsets_kernel<<<(L.n_pad + 255) / 256, 256, 0, st>>>(sp.vx, sp.vy, sorted, n_traj, L.n_pad,
                                                               T, sp.cs, orig, offs, vsort, dtf);
  KB_LAUNCH_CHECK("plan_offsets_kernel");
  plan_boxes_kernel<<<(L.nchunk * T + 255) / 256, 256, 0, st>>>(offs, L.nchunk, T, sp.x_lo,
                                                               sp.A.tx, plan);
  KB_LAUNCH_CHECK("plan_boxes_kernel");
  {
    size_t total = (size_t)T * (H + 3) * L.Wp;
    int blocks = (int)std::min<size_t>((total + 255) / 256, (size_t)g_num_sms * 16);
    bound_prep_kernel<<<blocks, 256, 0, st>>>(sp.psi, sp.phi, T, H, W, L.Wp, pool ? 1 : 0,
                                              bound);
    KB_LAUNCH_CHECK("bound_prep_kernel");
    const size_t npx = (size_t)T * H * W;
    pair_planes_kernel<<<(int)std::min<size_t>((npx + 255) / 256, (size_t)g_num_sms * 16), 256, 0,
                         st>>>(sp.psi, sp.phi, npx, reinterpret_cast<float2*>(ws + L.pairs));
    KB_LAUNCH_CHECK("bound_prep_kernel");
  }
  const int ntiles = sp.A.ntiles;
  sp.A.order = nullptr;
  if (sch.tile_order && ntiles > 1 && ntiles <= S_ORDER_MAX) {
    unsigned long long* tkeys = reinterpret_cast<unsigned long long*>(ws + L.tkeys);
    int32_t* torder = reinterpret_cast<int32_t*>(ws + L.torder);
    tile_score_kernel<<<ntiles, 256, 0, st>>>(bound, T, H, W, L.Wp, vbox, sp.cs, sp.x_lo, sp.y_lo,
                                              sp.x_hi, sp.y_hi, sp.A.ntx, sp.A.tx, ntiles,
                                              sch.hot_nu2, sch.score_span, tkeys);
    KB_LAUNCH_CHECK("tile_score_kernel");
    int n2 = 1;
    while (n2 < ntiles) n2 <<= 1;
    const size_t osm = sizeof(unsigned long long) * (size_t)n2;
    KB_CUDA_TRY(cudaFuncSetAttribute(tile_order_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)osm));
    tile_order_kernel<<<1, 1024, osm, st>>>(tkeys, ntiles, torder);
    KB_LAUNCH_CHECK("tile_order_kernel");
    sp.A.order = torder;
  }
  return KB_OK;
}

// The search kernel of one stack (its arguments and tensor maps in parameter space).
static int launch_search_single(const StackPrep& sp, cudaStream_t st) {
  const SearchArgs& A = sp.A;
  const int T = sp.T;
  const int grid = std::min(A.ntiles, g_num_sms);
  if (grid > S_REC_BLOCKS)
    return fail(KB_ERR_UNSUPPORTED, "kb_search: %d SMs, at most %d supported", g_num_sms,
                S_REC_BLOCKS);
#define KB_SEARCH_LAUNCH(NT, JJ, PL, NC)                                                          \
  do {                                                                                           \
    const size_t smem = SmemLayout<NT, false, PL, NC>::total;                                    \
    KB_CUDA_TRY(cudaFuncSetAttribute(search_kernel<NT, JJ, false, PL, NC>,                       \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));   \
    search_kernel<NT, JJ, false, PL, NC><<<grid, S_THREADS, smem, st>>>(sp.maps, A, BatchArgs{}); \
  } while (0)
#define KB_SEARCH_LAUNCH_T(PL, NC)                     \
  do {                                                 \
    if (T <= 16) KB_SEARCH_LAUNCH(16, 1, PL, NC);      \
    else if (T <= 32) KB_SEARCH_LAUNCH(32, 1, PL, NC); \
    else if (T <= 64) KB_SEARCH_LAUNCH(-1, 4, PL, NC); \
    else KB_SEARCH_LAUNCH(0, 4, PL, NC);               \
  } while (0)
  if (!sp.pool) KB_SEARCH_LAUNCH_T(false, 1);
  else if (A.tx == 2 * S_TX) KB_SEARCH_LAUNCH_T(true, 2);
  else KB_SEARCH_LAUNCH_T(true, 1);
#undef KB_SEARCH_LAUNCH_T
#undef KB_SEARCH_LAUNCH
  KB_LAUNCH_CHECK("search_kernel");
  return KB_OK;
}

// hot_nu2 64: with block maxima in the planes a lower threshold counts noise; on decam_half
// 16 -> 64 took the search from 276.5 to 272.7 ms (25..100 all within 0.5%)
static const kb_schedule kDefaultSchedule = {1, 64.0f, 64, 1, 1, S_TILE_COLS_DEFAULT};

static int check_schedule(const kb_schedule* s) {
  if (!s) return fail(KB_ERR_INVALID_ARG, "schedule: null pointer");
  if (s->tile_order != 0 && s->tile_order != 1)
    return fail(KB_ERR_INVALID_ARG, "schedule: tile_order must be 0 or 1");
  if (s->stack_order != 0 && s->stack_order != 1)
    return fail(KB_ERR_INVALID_ARG, "schedule: stack_order must be 0 or 1");
  if (!(s->hot_nu2 > 0.0f) || !std::isfinite(s->hot_nu2))
    return fail(KB_ERR_INVALID_ARG, "schedule: hot_nu2 must be finite and > 0");
  if (s->score_span < 0 || s->score_span > (1 << 20))
    return fail(KB_ERR_INVALID_ARG, "schedule: score_span outside 0..2^20");
  if (s->mode != 0 && s->mode != 1) return fail(KB_ERR_INVALID_ARG, "schedule: mode must be 0 or 1");
  if (s->tile_cols < 0 || s->tile_cols > 2)
    return fail(KB_ERR_INVALID_ARG, "schedule: tile_cols must be 0 (automatic), 1 or 2");
  return KB_OK;
}

}  // namespace kb

extern "C" void kb_schedule_default(kb_schedule* s) {
  if (s) *s = kb::kDefaultSchedule;
}

extern "C" int kb_search(const float* psi, const float* phi, const double* times, int T, int H,
                         int W, const float* vx, const float* vy, int n_traj,
                         const kb_search_params* p, float* out_lh, float* out_flux,
                         int32_t* out_idx, uint16_t* out_nvalid, uint16_t* out_nkept,
                         uint32_t* out_mask, void* workspace, size_t ws_bytes, void* stream) {
  using namespace kb;
  StackPrep sp;
  int rc = prepare_stack("kb_search", psi, phi, times, T, H, W, vx, vy, n_traj, p, out_lh,
                         out_flux, out_idx, out_nvalid, out_nkept, out_mask,
                         static_cast<char*>(workspace), ws_bytes, sp);
  if (rc != KB_OK) return rc;
  KB_FAULT_POINT("kb_search");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  rc = launch_prep(sp, kDefaultSchedule, sp.pool, st);
  if (rc != KB_OK) return rc;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  profile_events(&ev0, &ev1);
  if (ev0 && ev1) KB_CUDA_TRY(cudaEventRecord(ev0, st));
  rc = launch_search_single(sp, st);
  if (rc != KB_OK) return rc;
  if (ev0 && ev1) KB_CUDA_TRY(cudaEventRecord(ev1, st));
  return KB_OK;
}

// ---------------------------------------------------------------------------------------------
// Batched search: many stacks, one persistent launch
// ---------------------------------------------------------------------------------------------
namespace kb {

__global__ void batch_reset_kernel(Ctrl* ctrl, unsigned int* done_tiles,
                                   unsigned long long* done_ns, unsigned long long* start_ns,
                                   int n, unsigned long long te) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    done_tiles[i] = 0u;
    done_ns[i] = 0ull;
  }
  if (i == 0) {
    *ctrl = Ctrl{};
    ctrl->te = te;
    *start_ns = globaltimer_ns();
  }
}

__global__ void stack_done_kernel(unsigned long long* done_ns) { *done_ns = globaltimer_ns(); }

// Totals of the concurrent mode: each stack's search counted into its own control block.
__global__ void batch_sum_kernel(Ctrl* const* __restrict__ ctrls, int n, Ctrl* total) {
  unsigned long long ev = 0, ins = 0, sv = 0, sp = 0, sk = 0, sn = 0;
  unsigned int err = 0;
  for (int k = 0; k < n; ++k) {
    ev += ctrls[k]->evals;
    ins += ctrls[k]->inserts;
    sv += ctrls[k]->stage_valid;
    sp += ctrls[k]->stage_pass;
    sk += ctrls[k]->stage_kept;
    sn += ctrls[k]->stage_nvalid;
    err |= ctrls[k]->err;
    total->it_staged += ctrls[k]->it_staged;
    total->it_uniform += ctrls[k]->it_uniform;
    total->it_direct += ctrls[k]->it_direct;
    total->tma_bytes += ctrls[k]->tma_bytes;
    total->loads_per_traj = max(total->loads_per_traj, ctrls[k]->loads_per_traj);
  }
  total->evals = ev;
  total->inserts = ins;
  total->stage_valid = sv;
  total->stage_pass = sp;
  total->stage_kept = sk;
  total->stage_nvalid = sn;
  total->err = err;
}

struct BatchTables {
  size_t args, maps, tile_base, done_tiles, done_ns, start_ns, ctrl, ctrls, total;
};

static BatchTables batch_tables(int n) {
  BatchTables b{};
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + bytes, KB_WORKSPACE_ALIGN);
    return at;
  };
  b.args = take(sizeof(SearchArgs) * (size_t)n);
  b.maps = take(sizeof(TmapSet) * (size_t)n);
  b.tile_base = take(sizeof(int) * (size_t)(n + 1));
  b.done_tiles = take(sizeof(unsigned int) * (size_t)n);
  b.done_ns = take(sizeof(unsigned long long) * (size_t)n);
  b.start_ns = take(sizeof(unsigned long long));
  b.ctrl = take(256);
  b.ctrls = take(sizeof(Ctrl*) * (size_t)n);
  b.total = o;
  return b;
}

}  // namespace kb

struct kb_batch {
  int n = 0;
  std::vector<kb::StackPrep> sp;   // in the caller's order
  std::vector<int> order;          // schedule position -> caller's index
  kb_schedule sch{};
  char* ws = nullptr;
  kb::BatchTables tb{};
  int total_tiles = 0;
  unsigned long long te_total = 0;
  int device = 0;
  cudaStream_t gstream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  unsigned int graph_kernels = 0;
  static constexpr int NS = 4;     // streams of the concurrent mode
  cudaStream_t cs[NS] = {};
  cudaEvent_t fork = nullptr, join[NS] = {};
};

namespace kb {

static size_t stack_ws_bytes(const kb_stack& s) {
  return ws_layout(s.T, s.H, s.W, s.n_traj).total;
}

static void drop_graph(kb_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

// Writes the schedule-ordered tables (stack arguments, tensor maps, tile prefix) to the device.
// The tile orders themselves are computed on the device by each run.
static int write_tables(kb_batch* b) {
  const int n = b->n;
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  if (b->sch.stack_order == 1)  // predicted cost (trajectory-epochs), largest first
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int a, int c) { return b->sp[a].te > b->sp[c].te; });
  b->order = idx;
  std::vector<SearchArgs> args(n);
  std::vector<TmapSet> maps(n);
  std::vector<int> base(n + 1, 0);
  std::vector<Ctrl*> ctrls(n);
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(b->ws + b->tb.ctrl);
  for (int k = 0; k < n; ++k) {
    StackPrep& sp = b->sp[idx[k]];
    args[k] = sp.A;
    args[k].ctrl = ctrl;
    // the tile order lives in the stack's own workspace; used when it was computed
    const bool ordered = b->sch.tile_order && sp.A.ntiles > 1 && sp.A.ntiles <= S_ORDER_MAX;
    args[k].order = ordered ? reinterpret_cast<int32_t*>(sp.ws + sp.L.torder) : nullptr;
    maps[k] = sp.maps;
    ctrls[k] = sp.A.ctrl;
    base[k + 1] = base[k] + sp.A.ntiles;
  }
  b->total_tiles = base[n];
  KB_CUDA_TRY(cudaMemcpy(b->ws + b->tb.args, args.data(), sizeof(SearchArgs) * n,
                         cudaMemcpyHostToDevice));
  KB_CUDA_TRY(cudaMemcpy(b->ws + b->tb.maps, maps.data(), sizeof(TmapSet) * n,
                         cudaMemcpyHostToDevice));
  KB_CUDA_TRY(cudaMemcpy(b->ws + b->tb.tile_base, base.data(), sizeof(int) * (n + 1),
                         cudaMemcpyHostToDevice));
  KB_CUDA_TRY(cudaMemcpy(b->ws + b->tb.ctrls, ctrls.data(), sizeof(Ctrl*) * n,
                         cudaMemcpyHostToDevice));
  return KB_OK;
}

static int batch_enqueue(kb_batch* b, cudaStream_t st) {
  const int n = b->n;
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(b->ws + b->tb.ctrl);
  unsigned int* done_tiles = reinterpret_cast<unsigned int*>(b->ws + b->tb.done_tiles);
  unsigned long long* done_ns = reinterpret_cast<unsigned long long*>(b->ws + b->tb.done_ns);
  unsigned long long* start_ns = reinterpret_cast<unsigned long long*>(b->ws + b->tb.start_ns);
  batch_reset_kernel<<<(n + 255) / 256, 256, 0, st>>>(ctrl, done_tiles, done_ns, start_ns, n,
                                                      b->te_total);
  KB_LAUNCH_CHECK("batch_reset_kernel");
  if (b->sch.mode == 1) {
    // concurrent per-stack launches on the batch's streams: a stack's kernel starts on the SMs
    // that the previous one's last tiles leave idle
    KB_CUDA_TRY(cudaEventRecord(b->fork, st));
    for (int q = 0; q < kb_batch::NS; ++q) KB_CUDA_TRY(cudaStreamWaitEvent(b->cs[q], b->fork, 0));
    for (int k = 0; k < n; ++k) {
      cudaStream_t q = b->cs[k % kb_batch::NS];
      StackPrep& sp = b->sp[b->order[k]];
      int rc = launch_prep(sp, b->sch, sp.pool, q);
      if (rc == KB_OK) rc = launch_search_single(sp, q);
      if (rc != KB_OK) return rc;
      stack_done_kernel<<<1, 1, 0, q>>>(done_ns + k);
      KB_LAUNCH_CHECK("stack_done_kernel");
    }
    for (int q = 0; q < kb_batch::NS; ++q) {
      KB_CUDA_TRY(cudaEventRecord(b->join[q], b->cs[q]));
      KB_CUDA_TRY(cudaStreamWaitEvent(st, b->join[q], 0));
    }
    batch_sum_kernel<<<1, 1, 0, st>>>(reinterpret_cast<Ctrl* const*>(b->ws + b->tb.ctrls), n, ctrl);
    KB_LAUNCH_CHECK("batch_sum_kernel");
    return KB_OK;
  }
  // one persistent launch: one kind of bound planes for all stacks (blocks only if every stack
  // takes them)
  bool pool = true;
  for (int k = 0; k < n; ++k) pool = pool && b->sp[k].pool;
  for (int k = 0; k < n; ++k) {
    int rc = launch_prep(b->sp[b->order[k]], b->sch, pool, st);
    if (rc != KB_OK) return rc;
  }
  BatchArgs B{};
  B.stacks = reinterpret_cast<const SearchArgs*>(b->ws + b->tb.args);
  B.maps = reinterpret_cast<const TmapSet*>(b->ws + b->tb.maps);
  B.tile_base = reinterpret_cast<const int*>(b->ws + b->tb.tile_base);
  B.nstacks = n;
  B.total_tiles = b->total_tiles;
  B.ctrl = ctrl;
  B.done_tiles = done_tiles;
  B.done_ns = done_ns;
  // every stack of the batch has the batch's bound kind and tile width
  const bool wide = b->sp[0].A.tx == 2 * S_TX;
  auto kern = !pool ? search_kernel<0, 1, true, false, 1>
                    : (wide ? search_kernel<0, 1, true, true, 2> : search_kernel<0, 1, true, true, 1>);
  const size_t smem = !pool ? SmemLayout<0, true, false, 1>::total
                            : (wide ? SmemLayout<0, true, true, 2>::total
                                    : SmemLayout<0, true, true, 1>::total);
  KB_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int grid = std::min(b->total_tiles, g_num_sms);
  if (grid > S_REC_BLOCKS)
    return fail(KB_ERR_UNSUPPORTED, "kb_batch_run: %d SMs, at most %d supported", g_num_sms,
                S_REC_BLOCKS);
  static const TmapSet kNoMaps{};
  kern<<<grid, S_THREADS, smem, st>>>(kNoMaps, SearchArgs{}, B);
  KB_LAUNCH_CHECK("search_kernel (batch)");
  return KB_OK;
}

}  // namespace kb

extern "C" int kb_batch_workspace_size(const kb_stack* stacks, int n, size_t* bytes) {
  using namespace kb;
  if (!stacks || !bytes || n < 1) return fail(KB_ERR_INVALID_ARG, "kb_batch_workspace_size: bad arguments");
  size_t total = batch_tables(n).total;
  for (int i = 0; i < n; ++i) {
    const kb_stack& s = stacks[i];
    if (s.T < 1 || s.H < 1 || s.W < 1 || s.n_traj < 1)
      return fail(KB_ERR_INVALID_ARG, "kb_batch_workspace_size: stack %d has bad sizes", i);
    if (s.T > KB_MAX_T) return fail(KB_ERR_UNSUPPORTED, "kb_batch_workspace_size: stack %d: T > KB_MAX_T", i);
    if (s.n_traj > (1 << 24))
      return fail(KB_ERR_UNSUPPORTED, "kb_batch_workspace_size: stack %d: n_traj > 2^24", i);
    total = align_up(total + stack_ws_bytes(s), KB_WORKSPACE_ALIGN);
  }
  *bytes = total;
  return KB_OK;
}

extern "C" int kb_batch_create(const kb_stack* stacks, int n, void* workspace, size_t ws_bytes,
                               kb_batch** out) {
  using namespace kb;
  if (!out) return fail(KB_ERR_INVALID_ARG, "kb_batch_create: null output handle");
  *out = nullptr;
  size_t need = 0;
  int rc = kb_batch_workspace_size(stacks, n, &need);
  if (rc != KB_OK) return rc;
  if (!workspace || ws_bytes < need)
    return fail(KB_ERR_WORKSPACE, "kb_batch_create: workspace of %zu bytes, %zu needed", ws_bytes, need);
  if (reinterpret_cast<uintptr_t>(workspace) % KB_WORKSPACE_ALIGN)
    return fail(KB_ERR_WORKSPACE, "kb_batch_create: workspace not %d-byte aligned", KB_WORKSPACE_ALIGN);
  kb_batch* b = new kb_batch();
  b->n = n;
  b->sp.resize(n);
  b->sch = kDefaultSchedule;
  b->ws = static_cast<char*>(workspace);
  b->tb = batch_tables(n);
  size_t off = b->tb.total;
  // one kind of bound for the whole batch (one persistent launch runs one kernel): two-row
  // blocks only if every stack takes them; the stacks' tile geometry follows it
  bool batch_pool = true;
  for (int i = 0; i < n; ++i) {
    const kb_search_params& q = stacks[i].params;
    batch_pool = batch_pool &&
                 (q.bound_rows == 2 || (q.bound_rows == 0 && pool_blocks(stacks[i].T, q.lh_min)));
  }
  for (int i = 0; i < n; ++i) {
    const kb_stack& s = stacks[i];
    const size_t sz = stack_ws_bytes(s);
    char who[48];
    snprintf(who, sizeof(who), "kb_batch_create (stack %d)", i);
    kb_search_params prm = s.params;
    if (prm.bound_rows >= 0 && prm.bound_rows <= 2) prm.bound_rows = batch_pool ? 2 : 1;
    rc = prepare_stack(who, s.psi, s.phi, s.times, s.T, s.H, s.W, s.vx, s.vy, s.n_traj,
                       &prm, s.out_lh, s.out_flux, s.out_idx, s.out_nvalid, s.out_nkept,
                       s.out_mask, b->ws + off, sz, b->sp[i]);
    if (rc != KB_OK) {
      delete b;
      char msg[256];
      snprintf(msg, sizeof(msg), "%s", kb_last_error());
      return fail(rc, "kb_batch_create: stack %d: %s", i, msg);
    }
    b->te_total += b->sp[i].te;
    off = align_up(off + sz, KB_WORKSPACE_ALIGN);
  }
  if (fault_injected("kb_batch_create")) {
    delete b;
    return fail(KB_ERR_CUDA, "kb_batch_create: injected fault (KB_FAULT_INJECT)");
  }
  cudaError_t e = cudaGetDevice(&b->device);
  if (e == cudaSuccess && g_num_sms == 0)
    e = cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, b->device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
  for (int q = 0; q < kb_batch::NS && e == cudaSuccess; ++q) {
    e = cudaStreamCreateWithFlags(&b->cs[q], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[q], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    kb_batch_destroy(b);
    return fail(KB_ERR_CUDA, "kb_batch_create: %s", cudaGetErrorString(e));
  }
  rc = write_tables(b);
  if (rc != KB_OK) {
    kb_batch_destroy(b);
    return rc;
  }
  *out = b;
  return KB_OK;
}

extern "C" int kb_batch_run(kb_batch* b, void* stream) {
  using namespace kb;
  if (!b) return fail(KB_ERR_INVALID_ARG, "kb_batch_run: null batch");
  KB_FAULT_POINT("kb_batch_run");
  return batch_enqueue(b, static_cast<cudaStream_t>(stream));
}

extern "C" int kb_batch_run_graph(kb_batch* b, void* stream) {
  using namespace kb;
  if (!b) return fail(KB_ERR_INVALID_ARG, "kb_batch_run_graph: null batch");
  KB_FAULT_POINT("kb_batch_run_graph");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!b->exec) {
    const unsigned long long before = kb_launch_count();
    KB_CUDA_TRY(cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal));
    int rc = batch_enqueue(b, b->gstream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->gstream, &g);
    if (rc != KB_OK) {
      if (g) cudaGraphDestroy(g);
      return rc;
    }
    if (e != cudaSuccess) return fail(KB_ERR_CUDA, "kb_batch_run_graph: capture failed: %s", cudaGetErrorString(e));
    b->graph = g;
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) {
      drop_graph(b);
      return fail(KB_ERR_CUDA, "kb_batch_run_graph: instantiation failed: %s", cudaGetErrorString(e));
    }
    // the capture counted the graph's kernels once; each replay launches them again
    b->graph_kernels = (unsigned int)(kb_launch_count() - before);
  }
  KB_CUDA_TRY(cudaEventRecord(b->ev_in, st));
  KB_CUDA_TRY(cudaStreamWaitEvent(b->gstream, b->ev_in, 0));
  KB_CUDA_TRY(cudaGraphLaunch(b->exec, b->gstream));
  KB_CUDA_TRY(cudaEventRecord(b->ev_out, b->gstream));
  KB_CUDA_TRY(cudaStreamWaitEvent(st, b->ev_out, 0));
  count_launch(b->graph_kernels);
  return KB_OK;
}

extern "C" int kb_batch_get_schedule(const kb_batch* b, kb_schedule* s) {
  using namespace kb;
  if (!b || !s) return fail(KB_ERR_INVALID_ARG, "kb_batch_get_schedule: null pointer");
  *s = b->sch;
  return KB_OK;
}

extern "C" int kb_batch_set_schedule(kb_batch* b, const kb_schedule* s) {
  using namespace kb;
  if (!b) return fail(KB_ERR_INVALID_ARG, "kb_batch_set_schedule: null batch");
  int rc = check_schedule(s);
  if (rc != KB_OK) return rc;
  // the tables may be in use by work already enqueued
  KB_CUDA_TRY(cudaDeviceSynchronize());
  b->sch = *s;
  drop_graph(b);
  // one persistent launch runs one kernel: every stack takes the same width (automatic: 64-wide;
  // the batch has one tail, at its end)
  const int cols = (s->mode == 0 && s->tile_cols == 0) ? 2 : s->tile_cols;
  for (kb::StackPrep& sp : b->sp) set_tile_geometry(sp.A, sp.pool, cols);
  return write_tables(b);
}

extern "C" int kb_batch_autotune(kb_batch* b, void* stream, int reps, kb_schedule* best) {
  using namespace kb;
  if (!b) return fail(KB_ERR_INVALID_ARG, "kb_batch_autotune: null batch");
  if (reps < 1 || reps > 100) return fail(KB_ERR_INVALID_ARG, "kb_batch_autotune: reps outside 1..100");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  KB_CUDA_TRY(cudaEventCreate(&e0));
  KB_CUDA_TRY(cudaEventCreate(&e1));
  auto time_of = [&](const kb_schedule& s, float* ms) -> int {
    int rc = kb_batch_set_schedule(b, &s);
    if (rc != KB_OK) return rc;
    float bestt = 1e30f;
    for (int r = 0; r < reps; ++r) {
      KB_CUDA_TRY(cudaEventRecord(e0, st));
      rc = batch_enqueue(b, st);
      if (rc != KB_OK) return rc;
      KB_CUDA_TRY(cudaEventRecord(e1, st));
      KB_CUDA_TRY(cudaEventSynchronize(e1));
      float t = 0.0f;
      KB_CUDA_TRY(cudaEventElapsedTime(&t, e0, e1));
      bestt = std::min(bestt, t);
    }
    *ms = bestt;
    return KB_OK;
  };
  // coordinate descent over the scheduling knobs, starting from the defaults
  kb_schedule cur = kDefaultSchedule;
  float cur_ms = 0.0f;
  int rc = time_of(cur, &cur_ms);
  const float hot[] = {64.0f, 16.0f, 144.0f};
  const int span[] = {64, 32, 128};
  for (int pass = 0; rc == KB_OK && pass < 4; ++pass) {
    std::vector<kb_schedule> cand;
    if (pass == 0) {
      kb_schedule c = cur;
      c.mode = 1 - cur.mode;
      cand.push_back(c);
      c = cur;
      c.stack_order = 1 - cur.stack_order;
      cand.push_back(c);
    } else if (pass == 1) {
      kb_schedule c = cur;
      c.tile_order = 1 - cur.tile_order;
      cand.push_back(c);
      if (b->sp[0].pool)  // the tile width (two-row blocks only): automatic, 32 or 64
        for (int w = 0; w <= 2; ++w)
          if (w != cur.tile_cols) {
            c = cur;
            c.tile_cols = w;
            cand.push_back(c);
          }
    } else if (pass == 2 && cur.tile_order) {
      for (float h : hot)
        if (h != cur.hot_nu2) {
          kb_schedule c = cur;
          c.hot_nu2 = h;
          cand.push_back(c);
        }
    } else if (pass == 3 && cur.tile_order) {
      for (int sp : span)
        if (sp != cur.score_span) {
          kb_schedule c = cur;
          c.score_span = sp;
          cand.push_back(c);
        }
    }
    for (const kb_schedule& c : cand) {
      float ms = 0.0f;
      rc = time_of(c, &ms);
      if (rc != KB_OK) break;
      if (ms < cur_ms) {
        cur = c;
        cur_ms = ms;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != KB_OK) return rc;
  rc = kb_batch_set_schedule(b, &cur);
  if (rc != KB_OK) return rc;
  if (best) *best = cur;
  return KB_OK;
}

extern "C" int kb_batch_stats(kb_batch* b, unsigned long long* done_ns, unsigned long long* totals,
                              void* stream) {
  using namespace kb;
  if (!b || !done_ns || !totals) return fail(KB_ERR_INVALID_ARG, "kb_batch_stats: null pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<unsigned long long> dn(b->n);
  unsigned long long start = 0;
  Ctrl c{};
  KB_CUDA_TRY(cudaMemcpyAsync(dn.data(), b->ws + b->tb.done_ns, sizeof(unsigned long long) * b->n,
                              cudaMemcpyDeviceToHost, st));
  KB_CUDA_TRY(cudaMemcpyAsync(&start, b->ws + b->tb.start_ns, sizeof(start), cudaMemcpyDeviceToHost, st));
  KB_CUDA_TRY(cudaMemcpyAsync(&c, b->ws + b->tb.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  KB_CUDA_TRY(cudaStreamSynchronize(st));
  for (int k = 0; k < b->n; ++k) done_ns[b->order[k]] = dn[k] >= start ? dn[k] - start : 0ull;
  totals[0] = c.te;
  totals[1] = c.evals;
  totals[2] = c.inserts;
  totals[3] = c.err;
  return KB_OK;
}

extern "C" void kb_batch_destroy(kb_batch* b) {
  if (!b) return;
  kb::drop_graph(b);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  if (b->gstream) cudaStreamDestroy(b->gstream);
  if (b->fork) cudaEventDestroy(b->fork);
  for (int q = 0; q < kb_batch::NS; ++q) {
    if (b->cs[q]) cudaStreamDestroy(b->cs[q]);
    if (b->join[q]) cudaEventDestroy(b->join[q]);
  }
  delete b;
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

extern "C" int kb_search_stage_counts(const void* workspace, unsigned long long* out,
                                      void* stream) {
  using namespace kb;
  if (!workspace || !out) return fail(KB_ERR_INVALID_ARG, "kb_search_stage_counts: null pointer");
  Ctrl c{};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KB_CUDA_TRY(cudaMemcpyAsync(&c, workspace, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  KB_CUDA_TRY(cudaStreamSynchronize(st));
  out[0] = c.stage_valid;
  out[1] = c.stage_pass;
  out[2] = c.stage_kept;
  out[3] = c.stage_nvalid;
  return KB_OK;
}

namespace kb {

// Shared-memory traffic of the bound pass from a control block's counters.
static void pass_counts_of(const Ctrl& c, unsigned long long* out) {
  // per (tile, chunk, epoch): each bound-pass thread makes one or two 4-byte shared loads per
  // trajectory (two: its two columns, or its two row pairs; one: two-row blocks of one column),
  // and as many in all when the chunk shares one offset; and one 16-byte offset load per four
  // trajectories (a warp-wide broadcast)
  const unsigned long long words = (unsigned long long)c.loads_per_traj * S_CTHREADS;
  out[0] = (c.it_staged * S_C + c.it_uniform) * words * 4ull;
  out[1] = c.it_staged * (unsigned long long)(S_C / 4) * S_CWARPS * 16ull;
  out[2] = c.tma_bytes;
  out[3] = c.it_direct;
}

static int read_pass_counts(const char* who, const void* ctrl, unsigned long long* out,
                            void* stream) {
  if (!ctrl || !out) return fail(KB_ERR_INVALID_ARG, "%s: null pointer", who);
  Ctrl c{};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  KB_CUDA_TRY(cudaMemcpyAsync(&c, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st));
  KB_CUDA_TRY(cudaStreamSynchronize(st));
  pass_counts_of(c, out);
  return KB_OK;
}

}  // namespace kb

extern "C" int kb_search_pass_counts(const void* workspace, unsigned long long* out,
                                     void* stream) {
  return kb::read_pass_counts("kb_search_pass_counts", workspace, out, stream);
}

extern "C" int kb_batch_pass_counts(kb_batch* b, unsigned long long* out, void* stream) {
  using namespace kb;
  if (!b) return fail(KB_ERR_INVALID_ARG, "kb_batch_pass_counts: null batch");
  return read_pass_counts("kb_batch_pass_counts", b->ws + b->tb.ctrl, out, stream);
}

// ---------------------------------------------------------------------------------------------
// kb_search_no_alloc: kb_search with scratch memory built into the library
// ---------------------------------------------------------------------------------------------
namespace kb {

// The built-in scratch: file-scope device memory, present on every device that loads the
// library.  Host code must not take its address directly (that is a host-side stand-in); the
// device address is looked up per device with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_no_alloc_scratch[KB_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
static std::mutex g_no_alloc_mu;
static void* g_no_alloc_ptr[kMaxDevices] = {};

}  // namespace kb

extern "C" int kb_search_no_alloc(const float* psi, const float* phi, const double* times, int T,
                                  int H, int W, const float* vx, const float* vy, int n_traj,
                                  const kb_search_params* p, float* out_lh, float* out_flux,
                                  int32_t* out_idx, uint16_t* out_nvalid, uint16_t* out_nkept,
                                  uint32_t* out_mask, void* stream) {
  using namespace kb;
  int rc = validate(psi, phi, times, T, H, W, vx, vy, n_traj, p);
  if (rc != KB_OK) return rc;
  const size_t need = ws_layout(T, H, W, n_traj).total;
  if (need > (size_t)KB_STATIC_SCRATCH_BYTES)
    return fail(KB_ERR_UNSUPPORTED,
                "kb_search_no_alloc: this search needs %zu bytes of scratch, more than the %u "
                "built into the library; use kb_search with a workspace",
                need, (unsigned)KB_STATIC_SCRATCH_BYTES);
  KB_FAULT_POINT("kb_search_no_alloc");
  int dev = 0;
  KB_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices)
    return fail(KB_ERR_UNSUPPORTED, "kb_search_no_alloc: device ordinal %d beyond %d", dev,
                kMaxDevices);
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_no_alloc_mu);
    if (!g_no_alloc_ptr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_no_alloc_scratch);
      if (e != cudaSuccess || !ptr)
        return fail(KB_ERR_CUDA, "kb_search_no_alloc: cudaGetSymbolAddress failed: %s",
                    cudaGetErrorString(e));
      g_no_alloc_ptr[dev] = ptr;
    }
    scratch = g_no_alloc_ptr[dev];
  }
  return kb_search(psi, phi, times, T, H, W, vx, vy, n_traj, p, out_lh, out_flux, out_idx,
                   out_nvalid, out_nkept, out_mask, scratch, (size_t)KB_STATIC_SCRATCH_BYTES,
                   stream);
}

extern "C" int kb_search_no_alloc_stats(unsigned long long* stats, void* stream) {
  using namespace kb;
  if (!stats) return fail(KB_ERR_INVALID_ARG, "kb_search_no_alloc_stats: null pointer");
  int dev = 0;
  KB_CUDA_TRY(cudaGetDevice(&dev));
  void* scratch = nullptr;
  if (dev >= 0 && dev < kMaxDevices) {
    std::lock_guard<std::mutex> lock(g_no_alloc_mu);
    scratch = g_no_alloc_ptr[dev];
  }
  if (!scratch)
    return fail(KB_ERR_INVALID_ARG,
                "kb_search_no_alloc_stats: no kb_search_no_alloc call on device %d yet", dev);
  return kb_search_stats(scratch, stats, stream);
}

// ---------------------------------------------------------------------------------------------
// kb_wait_check: the search kernel's bounded waits, on waits that cannot complete
// ---------------------------------------------------------------------------------------------
namespace kb {

// [0] status bits, [1..3] duration of each wait in ns (kernel-written, read back by the host)
static __device__ unsigned long long g_wait_status[4];

// One thread waits on phase 0 of an mbarrier that expects one arrival and never gets it: first
// as a producer retiring a slot (mbar_wait_parity), then as a consumer waiting for a staged box
// (consumer_wait), both with the given limit; then, with the block's abort flag raised, once
// more as a consumer, which must return at the flag rather than at the limit.  Every wait is
// bounded by limit_ns of %globaltimer, so the kernel ends after about twice the limit.
__global__ void wait_check_kernel(unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  __shared__ unsigned int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1u);
    abort_flag = 0u;
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  unsigned long long st = 0ull;
  const unsigned long long t0 = globaltimer_ns();
  if (!mbar_wait_parity(&bar, 0u, limit_ns)) st |= 0x1ull;
  const unsigned long long t1 = globaltimer_ns();
  if (!consumer_wait(&bar, 0u, &abort_flag, limit_ns)) st |= 0x2ull;
  const unsigned long long t2 = globaltimer_ns();
  *(volatile unsigned int*)&abort_flag = 1u;
  if (!consumer_wait(&bar, 0u, &abort_flag, limit_ns)) st |= 0x4ull;
  const unsigned long long t3 = globaltimer_ns();
  g_wait_status[0] = st;
  g_wait_status[1] = t1 - t0;
  g_wait_status[2] = t2 - t1;
  g_wait_status[3] = t3 - t2;
}

}  // namespace kb

extern "C" int kb_wait_check(unsigned long long limit_ns, unsigned long long* out, void* stream) {
  using namespace kb;
  if (limit_ns < 1000ull || limit_ns > 10000000000ull)
    return fail(KB_ERR_INVALID_ARG, "kb_wait_check: limit_ns outside 1e3 .. 1e10");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  wait_check_kernel<<<1, 32, 0, st>>>(limit_ns);
  KB_LAUNCH_CHECK("wait_check_kernel");
  unsigned long long h[4] = {0ull, 0ull, 0ull, 0ull};
  KB_CUDA_TRY(cudaMemcpyFromSymbolAsync(h, g_wait_status, sizeof(h), 0, cudaMemcpyDeviceToHost, st));
  KB_CUDA_TRY(cudaStreamSynchronize(st));
  if (out)
    for (int i = 0; i < 4; ++i) out[i] = h[i];
  if (h[0] != 0x7ull)
    return fail(KB_ERR_CUDA, "kb_wait_check: status bits %llu, expected 7 (a wait that cannot "
                "complete reported success)", h[0]);
  if (h[3] >= limit_ns)
    return fail(KB_ERR_CUDA, "kb_wait_check: the raised abort flag did not end the wait (%llu ns)",
                h[3]);
  return fail(KB_ERR_TIMEOUT, "kb_wait_check: device-side waits gave up after %llu and %llu ns "
              "(limit %llu ns); the abort flag ended the third after %llu ns", h[1], h[2],
              limit_ns, h[3]);
}
