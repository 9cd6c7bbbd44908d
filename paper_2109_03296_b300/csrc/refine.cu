// refine.cu -- sub-pixel evaluation of single trajectories, its backward pass, and gradient
// ascent of the likelihood off the velocity grid (Section 4.1: the grid spacing bounds how
// closely a found trajectory follows the object; single given trajectories are evaluated along
// their own tracks).
//
// For a candidate with real start (x0, y0) and velocity (vx, vy), epoch t is read at
// (x0 + vx dt_t, y0 + vy dt_t) by bilinear interpolation of psi_t and phi_t (pixel centres at
// integer coordinates; taps outside the image read zero), and over the kept epochs
//   Psi = sum psi_t(.),  Phi = sum phi_t(.),  L = Psi / sqrt(Phi),  alpha = Psi / Phi.
// The kept set is an input and stays fixed, so L is differentiable almost everywhere in
// (x0, y0, vx, vy) (piecewise bilinear) and linear / rational in the psi / phi pixels.
//
// A group of G lanes per candidate (a warp for T > 16; 16 or 8 lanes, several candidates per warp,
// for smaller T) with E epochs per lane (epoch sub + G j for sub-lane `sub`, j < E).  Each lane forms its positions in
// float-float arithmetic (an unevaluated sum hi + lo of two float32 values, about 48 significant
// bits, built from exact two-sum and FMA two-product steps; float64 runs at a small fraction of
// the float32 rate on this part), splits them into cell and fraction, reads the four taps of
// psi_t and phi_t through the read-only path, and adds to ten float32 partial sums: Psi, Phi and
// the derivatives of both in the four parameters.  A butterfly reduction within the group leaves
// the same sums, bit for bit, in every lane of the group, so the Adam update of the refine loop
// runs redundantly in all of them with no further communication.
#include <cmath>
#include <type_traits>

#include "kb_internal.cuh"

namespace kb {

constexpr int RF_THREADS = 256;

struct EpochDt {
  float hi[KB_MAX_T];  // dt_t = times[t] - times[0] as hi + lo (float-float)
  float lo[KB_MAX_T];
};

// Float-float values: hi + lo with |lo| <= ulp(hi)/2.  The _rn intrinsics keep every step a
// separately rounded IEEE operation (no contraction into FMAs), which the error-free
// transformations below rely on.
struct FF {
  float hi, lo;
};

// a + b = s + e exactly (Knuth's two-sum)
__device__ __forceinline__ FF two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return FF{s, e};
}

// a + b = s + e exactly when |a| >= |b| (Dekker's fast two-sum)
__device__ __forceinline__ FF fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  FF s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ FF ff_add_f(FF a, float b) {
  FF s = two_sum(a.hi, b);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

// product with the exact error of hi*hi from an FMA; lo*lo is below the format's precision
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  return fast_two_sum(p, e);
}

// The four bilinear taps of one epoch: flat index of the lower-left tap (may point before the
// image when a tap row or column is outside), fractions, and a validity bit per tap
// (bit 0: (ix, iy), 1: (ix+1, iy), 2: (ix, iy+1), 3: (ix+1, iy+1)).
struct Taps {
  long long base;
  float ax, ay;
  unsigned valid;
};

// cell floor(v) and fraction v - floor(v) of a float-float value, the cell decided by the sign of
// lo where hi is an integer
__device__ __forceinline__ void ff_floor_frac(FF v, float& cell, float& frac) {
  cell = floorf(v.hi);
  frac = __fadd_rn(__fsub_rn(v.hi, cell), v.lo);   // hi - floor(hi) is exact
  if (frac < 0.f) {
    cell -= 1.f;
    frac = __fadd_rn(frac, 1.f);
  } else if (frac >= 1.f) {
    cell += 1.f;
    frac = __fsub_rn(frac, 1.f);
  }
}

__device__ __forceinline__ Taps make_taps(FF x, FF y, int H, int W) {
  Taps tp;
  tp.base = 0;
  tp.ax = 0.f;
  tp.ay = 0.f;
  tp.valid = 0u;
  float fx, fy, ax, ay;
  ff_floor_frac(x, fx, ax);
  ff_floor_frac(y, fy, ay);
  // also false for NaN: such a position has no tap inside the image
  if (!(fx >= -1.f && fx <= (float)(W - 1) && fy >= -1.f && fy <= (float)(H - 1))) return tp;
  int ix = (int)fx, iy = (int)fy;
  tp.ax = ax;
  tp.ay = ay;
  bool c0 = ix >= 0, c1 = ix + 1 < W, r0 = iy >= 0, r1 = iy + 1 < H;
  tp.valid = (unsigned)(c0 && r0) | (unsigned)(c1 && r0) << 1 | (unsigned)(c0 && r1) << 2 |
             (unsigned)(c1 && r1) << 3;
  tp.base = (long long)iy * W + ix;
  return tp;
}

struct Quad {
  float v00, v01, v10, v11;
};

__device__ __forceinline__ Quad load_quad(const float* __restrict__ plane, const Taps& tp, int W) {
  Quad q;
  q.v00 = (tp.valid & 1u) ? __ldg(plane + tp.base) : 0.f;
  q.v01 = (tp.valid & 2u) ? __ldg(plane + tp.base + 1) : 0.f;
  q.v10 = (tp.valid & 4u) ? __ldg(plane + tp.base + W) : 0.f;
  q.v11 = (tp.valid & 8u) ? __ldg(plane + tp.base + W + 1) : 0.f;
  return q;
}

// value and d/dx, d/dy of the bilinear sample
__device__ __forceinline__ void bilerp(const Quad& q, float ax, float ay, float& v, float& gx,
                                       float& gy) {
  float top = fmaf(ax, q.v01 - q.v00, q.v00);
  float bot = fmaf(ax, q.v11 - q.v10, q.v10);
  v = fmaf(ay, bot - top, top);
  gx = fmaf(ay, (q.v11 - q.v10) - (q.v01 - q.v00), q.v01 - q.v00);
  gy = bot - top;
}

// s[0] = Psi, s[1] = Phi, s[2..5] = dPsi/d(x0, y0, vx, vy), s[6..9] = dPhi/d(...)
constexpr int NSUM = 10;

// Track parameters in float-float: the inputs are float32, but the refine loop accumulates its
// steps in float-float so that the side of a bilinear cell edge on which an epoch falls is
// decided as in exact arithmetic (float32 parameters near x ~ 4000 px carry 2.4e-4 px of
// rounding, times dt for the velocities).
struct Track {
  FF x0, y0, vx, vy;
};

__device__ __forceinline__ Track to_track(float4 p) {
  return Track{FF{p.x, 0.f}, FF{p.y, 0.f}, FF{p.z, 0.f}, FF{p.w, 0.f}};
}

__device__ __forceinline__ float4 round_track(const Track& p) {
  return make_float4(__fadd_rn(p.x0.hi, p.x0.lo), __fadd_rn(p.y0.hi, p.y0.lo),
                     __fadd_rn(p.vx.hi, p.vx.lo), __fadd_rn(p.vy.hi, p.vy.lo));
}

__device__ __forceinline__ FF track_pos(FF p0, FF v, FF dt) { return ff_add(p0, ff_mul(v, dt)); }

// Lane layout of a candidate group: G lanes (a power of two dividing 32), E epochs per lane.
template <int G>
struct Group {
  static constexpr int PER_BLOCK = RF_THREADS / G;
  __device__ static int sub() { return threadIdx.x & (G - 1); }
  __device__ static long long cand() {
    return (long long)blockIdx.x * PER_BLOCK + (threadIdx.x / G);
  }
  __device__ static unsigned mask() {
    return G == 32 ? 0xffffffffu : ((1u << G) - 1u) << (threadIdx.x & 31 & ~(G - 1));
  }
  // butterfly sum over the group: every lane of the group ends with the same value, bit for bit
  __device__ static float sum(float v) {
    const unsigned m = mask();
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(m, v, o);
    return v;
  }
};

// The lane's partial sums over its own epochs: s[0] = psi, s[1] = phi, s[2..5] = d psi /
// d(x0, y0, vx, vy), s[6..9] = d phi / d(...).
template <int G, int E>
__device__ __forceinline__ void lane_partials(const float* __restrict__ psi,
                                              const float* __restrict__ phi, int T, int H, int W,
                                              const FF (&dt)[E], unsigned kbits, const Track& p,
                                              float (&s)[NSUM]) {
  const int sub = Group<G>::sub();
#pragma unroll
  for (int i = 0; i < NSUM; ++i) s[i] = 0.f;
  const size_t hw = (size_t)H * W;
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int t = sub + G * j;
    if (t >= T || !((kbits >> j) & 1u)) continue;
    Taps tp = make_taps(track_pos(p.x0, p.vx, dt[j]), track_pos(p.y0, p.vy, dt[j]), H, W);
    if (!tp.valid) continue;
    Quad qp = load_quad(psi + (size_t)t * hw, tp, W);
    Quad qf = load_quad(phi + (size_t)t * hw, tp, W);
    float vp, gpx, gpy, vf, gfx, gfy;
    bilerp(qp, tp.ax, tp.ay, vp, gpx, gpy);
    bilerp(qf, tp.ax, tp.ay, vf, gfx, gfy);
    float d = dt[j].hi;
    s[0] += vp;
    s[1] += vf;
    s[2] += gpx;
    s[3] += gpy;
    s[4] = fmaf(gpx, d, s[4]);
    s[5] = fmaf(gpy, d, s[5]);
    s[6] += gfx;
    s[7] += gfy;
    s[8] = fmaf(gfx, d, s[8]);
    s[9] = fmaf(gfy, d, s[9]);
  }
}

template <int G>
__device__ __forceinline__ void group_sums(float (&s)[NSUM]) {
  const unsigned m = Group<G>::mask();
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1)
#pragma unroll
    for (int i = 0; i < NSUM; ++i) s[i] += __shfl_xor_sync(m, s[i], o);
}

// a dPsi/dparams + b dPhi/dparams from the group sums
__device__ __forceinline__ float4 param_grad(const float (&s)[NSUM], float a, float b) {
  return make_float4(fmaf(b, s[6], a * s[2]), fmaf(b, s[7], a * s[3]), fmaf(b, s[8], a * s[4]),
                     fmaf(b, s[9], a * s[5]));
}

// Per-lane state loaded once per candidate: the lane's dt values and its kept bits (bit j for
// epoch sub + G j).
template <int G, int E>
__device__ __forceinline__ unsigned lane_setup(const EpochDt& e, const uint32_t* __restrict__ keep,
                                               int MW, long long c, int T, FF (&dt)[E]) {
  const int sub = Group<G>::sub();
  unsigned kbits = 0u;
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int t = sub + G * j;
    dt[j] = t < T ? FF{e.hi[t], e.lo[t]} : FF{0.f, 0.f};
    unsigned b = 0u;
    if (t < T) b = keep ? ((__ldg(keep + c * MW + (t >> 5)) >> (t & 31)) & 1u) : 1u;
    kbits |= b << j;
  }
  return kbits;
}

template <int G, int E>
__global__ void __launch_bounds__(RF_THREADS) traj_fwd_kernel(
    const float* __restrict__ psi, const float* __restrict__ phi, int T, int H, int W,
    const float4* __restrict__ params, const uint32_t* __restrict__ keep, int MW, int n,
    EpochDt e, float* __restrict__ out_lh, float* __restrict__ out_flux,
    float4* __restrict__ out_grad) {
  const long long c = Group<G>::cand();
  if (c >= n) return;
  const bool leader = Group<G>::sub() == 0;
  FF dt[E];
  unsigned kbits = lane_setup<G, E>(e, keep, MW, c, T, dt);
  const Track p = to_track(__ldg(params + c));
  float s[NSUM];
  lane_partials<G, E>(psi, phi, T, H, W, dt, kbits, p, s);
  group_sums<G>(s);
  if (!leader) return;
  if (!(s[1] > 0.f)) {
    out_lh[c] = __int_as_float(0x7fc00000);
    out_flux[c] = __int_as_float(0x7fc00000);
    if (out_grad) out_grad[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const float rs = sqrtf(s[1]);
  out_lh[c] = s[0] / rs;
  out_flux[c] = s[0] / s[1];
  if (out_grad) out_grad[c] = param_grad(s, 1.f / rs, -0.5f * s[0] / (s[1] * rs));
}

template <int G, int E>
__global__ void __launch_bounds__(RF_THREADS) traj_bwd_kernel(
    const float* __restrict__ psi, const float* __restrict__ phi, int T, int H, int W,
    const float4* __restrict__ params, const uint32_t* __restrict__ keep, int MW, int n,
    EpochDt e, const float* __restrict__ grad_lh, const float* __restrict__ grad_flux,
    float4* __restrict__ out_grad, float* __restrict__ grad_psi, float* __restrict__ grad_phi) {
  const long long c = Group<G>::cand();
  if (c >= n) return;
  const int sub = Group<G>::sub();
  FF dt[E];
  unsigned kbits = lane_setup<G, E>(e, keep, MW, c, T, dt);
  const Track p = to_track(__ldg(params + c));
  float s[NSUM];
  lane_partials<G, E>(psi, phi, T, H, W, dt, kbits, p, s);
  group_sums<G>(s);
  const float Ps = s[0], Ph = s[1];
  if (!(Ph > 0.f)) {
    if (sub == 0 && out_grad) out_grad[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    return;
  }
  const float gL = grad_lh ? __ldg(grad_lh + c) : 0.f;
  const float gA = grad_flux ? __ldg(grad_flux + c) : 0.f;
  const float rs = sqrtf(Ph);
  // dL/dPsi = 1/sqrt(Phi), dL/dPhi = -Psi/(2 Phi^1.5); dalpha/dPsi = 1/Phi, dalpha/dPhi = -Psi/Phi^2
  const float cps = gL / rs + gA / Ph;
  const float cph = -0.5f * gL * Ps / (Ph * rs) - gA * Ps / (Ph * Ph);
  if (sub == 0 && out_grad) out_grad[c] = param_grad(s, cps, cph);
  if (!grad_psi && !grad_phi) return;
  const size_t hw = (size_t)H * W;
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int t = sub + G * j;
    if (t >= T || !((kbits >> j) & 1u)) continue;
    Taps tp = make_taps(track_pos(p.x0, p.vx, dt[j]), track_pos(p.y0, p.vy, dt[j]), H, W);
    const float w[4] = {(1.f - tp.ax) * (1.f - tp.ay), tp.ax * (1.f - tp.ay),
                        (1.f - tp.ax) * tp.ay, tp.ax * tp.ay};
    const long long off[4] = {0, 1, W, (long long)W + 1};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (!((tp.valid >> k) & 1u)) continue;
      size_t i = (size_t)t * hw + (size_t)(tp.base + off[k]);
      if (grad_psi) atomicAdd(grad_psi + i, cps * w[k]);
      if (grad_phi) atomicAdd(grad_phi + i, cph * w[k]);
    }
  }
}

struct AdamConsts {
  int n_steps;
  float lr_pos, lr_vel, b1, b2, eps;
};

// Adam runs redundantly in every lane of the group on the group sums, so all lanes hold the same
// parameters; the bias corrections are applied as products with correctly rounded reciprocals.
// A minimum of one block per SM leaves the register budget to the compiler: at T = 26 it takes 69
// registers (4 blocks of 256 per SM) and runs 1.5x faster than when held to 48 for 5 blocks.
template <int G, int E>
__global__ void __launch_bounds__(RF_THREADS, 1) refine_kernel(
    const float* __restrict__ psi, const float* __restrict__ phi, int T, int H, int W,
    float4* __restrict__ params, const uint32_t* __restrict__ keep, int MW, int n, EpochDt e,
    AdamConsts ac, float* __restrict__ out_lh, float* __restrict__ out_flux,
    float* __restrict__ out_lh_start) {
  const long long c = Group<G>::cand();
  if (c >= n) return;
  const bool leader = Group<G>::sub() == 0;
  FF dt[E];
  unsigned kbits = lane_setup<G, E>(e, keep, MW, c, T, dt);
  Track p = to_track(params[c]);
  float m[4] = {0.f, 0.f, 0.f, 0.f}, v[4] = {0.f, 0.f, 0.f, 0.f};
  float b1k = 1.f, b2k = 1.f;
  float s[NSUM];
  bool ok = true;
  for (int k = 0; k <= ac.n_steps; ++k) {
    // the returned params are float32: evaluate the final L and alpha at exactly those
    if (k == ac.n_steps && k > 0) p = to_track(round_track(p));
    lane_partials<G, E>(psi, phi, T, H, W, dt, kbits, p, s);
    group_sums<G>(s);
    if (!(s[1] > 0.f)) {
      if (k == 0 && out_lh_start && leader) out_lh_start[c] = __int_as_float(0x7fc00000);
      ok = false;
      break;
    }
    const float rs = sqrtf(s[1]);
    if (k == 0 && out_lh_start && leader) out_lh_start[c] = s[0] / rs;
    if (k == ac.n_steps) break;
    const float4 g4 = param_grad(s, 1.f / rs, -0.5f * s[0] / (s[1] * rs));
    const float g[4] = {g4.x, g4.y, g4.z, g4.w};
    b1k *= ac.b1;
    b2k *= ac.b2;
    const float c1 = __frcp_rn(1.f - b1k), c2 = __frcp_rn(1.f - b2k);
    float step[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      m[i] = fmaf(ac.b1, m[i], (1.f - ac.b1) * g[i]);
      v[i] = fmaf(ac.b2, v[i], (1.f - ac.b2) * g[i] * g[i]);
      step[i] = (i < 2 ? ac.lr_pos : ac.lr_vel) * (m[i] * c1) / (sqrtf(v[i] * c2) + ac.eps);
    }
    p.x0 = ff_add_f(p.x0, step[0]);
    p.y0 = ff_add_f(p.y0, step[1]);
    p.vx = ff_add_f(p.vx, step[2]);
    p.vy = ff_add_f(p.vy, step[3]);
  }
  if (!leader) return;
  params[c] = round_track(p);
  if (ok) {
    out_lh[c] = s[0] / sqrtf(s[1]);
    out_flux[c] = s[0] / s[1];
  } else {
    out_lh[c] = __int_as_float(0x7fc00000);
    out_flux[c] = __int_as_float(0x7fc00000);
  }
}

__global__ void candidate_params_kernel(const int32_t* __restrict__ cand_pix,
                                        const int32_t* __restrict__ cand_slot, int n,
                                        const int32_t* __restrict__ idx,
                                        const uint32_t* __restrict__ mask, int K, int MW,
                                        const float* __restrict__ vx, const float* __restrict__ vy,
                                        int x_lo, int y_lo, int wx, float4* __restrict__ out_params,
                                        uint32_t* __restrict__ out_keep) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int pix = cand_pix[i];
  int traj = -1;
  long long slot = -1;
  if (pix >= 0) {
    slot = (long long)pix * K + cand_slot[i];
    traj = idx[slot];
  }
  if (traj < 0) {
    float q = __int_as_float(0x7fc00000);
    out_params[i] = make_float4(q, q, q, q);
    if (out_keep)
      for (int w = 0; w < MW; ++w) out_keep[i * MW + w] = 0u;
    return;
  }
  out_params[i] = make_float4((float)(x_lo + pix % wx), (float)(y_lo + pix / wx), vx[traj],
                              vy[traj]);
  if (out_keep)
    for (int w = 0; w < MW; ++w) out_keep[i * MW + w] = mask[slot * MW + w];
}

// params, gradients and out_params are read and written as float4: a row of 4 floats must start on
// a 16-byte boundary (NULL passes; the callers test it separately).
static inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

static int check_common(const char* who, const float* psi, const float* phi, const double* times,
                        int T, int H, int W, const void* params, int n, EpochDt& e) {
  if (!psi || !phi || !times) return fail(KB_ERR_INVALID_ARG, "%s: null pointer argument", who);
  if (n < 0 || T < 1 || H < 1 || W < 1) return fail(KB_ERR_INVALID_ARG, "%s: bad sizes", who);
  if (n > 0 && !params) return fail(KB_ERR_INVALID_ARG, "%s: null params", who);
  if (n > 0 && !aligned16(params))
    return fail(KB_ERR_INVALID_ARG, "%s: params not 16-byte aligned", who);
  if (T > KB_MAX_T) return fail(KB_ERR_UNSUPPORTED, "%s: T > KB_MAX_T", who);
  if (H > (1 << 20) || W > (1 << 20))
    return fail(KB_ERR_UNSUPPORTED, "%s: image sides are limited to 2^20 pixels", who);
  for (int t = 0; t < T; ++t) {
    if (!std::isfinite(times[t])) return fail(KB_ERR_INVALID_ARG, "%s: times not finite", who);
    double dt = times[t] - times[0];
    e.hi[t] = (float)dt;
    e.lo[t] = (float)(dt - (double)e.hi[t]);
  }
  return KB_OK;
}

// Group shape by T: G lanes per candidate, E = ceil(T / G) epochs per lane.  A whole warp per
// candidate wherever T fills most of it: packing two candidates into a warp (16 lanes x 2 epochs)
// issues fewer instructions but doubles the candidates resident per SM, and their taps then no
// longer fit the L1 (measured at T = 26: hit rate 84% -> 62%, 0.75 -> 1.0 ms).
template <typename F>
static void with_shape(int T, F&& f) {
  if (T <= 8)
    f(std::integral_constant<int, 8>{}, std::integral_constant<int, 1>{});
  else if (T <= 16)
    f(std::integral_constant<int, 16>{}, std::integral_constant<int, 1>{});
  else if (T <= 32)
    f(std::integral_constant<int, 32>{}, std::integral_constant<int, 1>{});
  else if (T <= 64)
    f(std::integral_constant<int, 32>{}, std::integral_constant<int, 2>{});
  else
    f(std::integral_constant<int, 32>{}, std::integral_constant<int, 4>{});
}

template <int G>
static inline unsigned rf_blocks(int n) {
  return (unsigned)(((long long)n + Group<G>::PER_BLOCK - 1) / Group<G>::PER_BLOCK);
}

}  // namespace kb

extern "C" int kb_traj_eval_fwd(const float* psi, const float* phi, const double* times, int T,
                                int H, int W, const float* params, const uint32_t* keep, int n,
                                float* out_lh, float* out_flux, float* out_grad, void* stream) {
  using namespace kb;
  EpochDt e{};
  if (int rc = check_common("kb_traj_eval_fwd", psi, phi, times, T, H, W, params, n, e)) return rc;
  if (n > 0 && (!out_lh || !out_flux))
    return fail(KB_ERR_INVALID_ARG, "kb_traj_eval_fwd: null output");
  if (n > 0 && !aligned16(out_grad))
    return fail(KB_ERR_INVALID_ARG, "kb_traj_eval_fwd: out_grad not 16-byte aligned");
  if (n == 0) return KB_OK;
  KB_FAULT_POINT("kb_traj_eval_fwd");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int MW = (T + 31) / 32;
  const float4* p4 = reinterpret_cast<const float4*>(params);
  float4* g4 = reinterpret_cast<float4*>(out_grad);
  with_shape(T, [&](auto G, auto E) {
    traj_fwd_kernel<G(), E()><<<rf_blocks<G()>(n), RF_THREADS, 0, st>>>(
        psi, phi, T, H, W, p4, keep, MW, n, e, out_lh, out_flux, g4);
  });
  KB_LAUNCH_CHECK("traj_fwd_kernel");
  return KB_OK;
}

extern "C" int kb_traj_eval_bwd(const float* psi, const float* phi, const double* times, int T,
                                int H, int W, const float* params, const uint32_t* keep, int n,
                                const float* grad_lh, const float* grad_flux,
                                float* out_grad_params, float* grad_psi, float* grad_phi,
                                void* stream) {
  using namespace kb;
  EpochDt e{};
  if (int rc = check_common("kb_traj_eval_bwd", psi, phi, times, T, H, W, params, n, e)) return rc;
  if (n > 0 && !aligned16(out_grad_params))
    return fail(KB_ERR_INVALID_ARG, "kb_traj_eval_bwd: out_grad_params not 16-byte aligned");
  if (n == 0) return KB_OK;
  if (!out_grad_params && !grad_psi && !grad_phi) return KB_OK;
  KB_FAULT_POINT("kb_traj_eval_bwd");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int MW = (T + 31) / 32;
  const float4* p4 = reinterpret_cast<const float4*>(params);
  float4* g4 = reinterpret_cast<float4*>(out_grad_params);
  with_shape(T, [&](auto G, auto E) {
    traj_bwd_kernel<G(), E()><<<rf_blocks<G()>(n), RF_THREADS, 0, st>>>(
        psi, phi, T, H, W, p4, keep, MW, n, e, grad_lh, grad_flux, g4, grad_psi, grad_phi);
  });
  KB_LAUNCH_CHECK("traj_bwd_kernel");
  return KB_OK;
}

extern "C" void kb_refine_params_default(kb_refine_params* rp) {
  if (!rp) return;
  rp->n_steps = 20;
  rp->lr_pos = 0.1f;
  rp->lr_vel = 0.2f;
  rp->beta1 = 0.9f;
  rp->beta2 = 0.999f;
  rp->eps = 1e-8f;
}

extern "C" int kb_refine(const float* psi, const float* phi, const double* times, int T, int H,
                         int W, float* params, const uint32_t* keep, int n,
                         const kb_refine_params* rp, float* out_lh, float* out_flux,
                         float* out_lh_start, void* stream) {
  using namespace kb;
  EpochDt e{};
  if (int rc = check_common("kb_refine", psi, phi, times, T, H, W, params, n, e)) return rc;
  if (!rp) return fail(KB_ERR_INVALID_ARG, "kb_refine: null refine parameters");
  if (rp->n_steps < 0 || rp->n_steps > 100000)
    return fail(KB_ERR_INVALID_ARG, "kb_refine: n_steps outside 0..100000");
  if (!(std::isfinite(rp->lr_pos) && rp->lr_pos >= 0.f && std::isfinite(rp->lr_vel) &&
        rp->lr_vel >= 0.f))
    return fail(KB_ERR_INVALID_ARG, "kb_refine: learning rates must be finite and >= 0");
  if (!(rp->beta1 >= 0.f && rp->beta1 < 1.f && rp->beta2 >= 0.f && rp->beta2 < 1.f))
    return fail(KB_ERR_INVALID_ARG, "kb_refine: beta1, beta2 must lie in [0, 1)");
  if (!(rp->eps > 0.f && std::isfinite(rp->eps)))
    return fail(KB_ERR_INVALID_ARG, "kb_refine: eps must be finite and > 0");
  if (n > 0 && (!out_lh || !out_flux)) return fail(KB_ERR_INVALID_ARG, "kb_refine: null output");
  if (n == 0) return KB_OK;
  KB_FAULT_POINT("kb_refine");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  AdamConsts ac{rp->n_steps, rp->lr_pos, rp->lr_vel, rp->beta1, rp->beta2, rp->eps};
  const int MW = (T + 31) / 32;
  float4* p4 = reinterpret_cast<float4*>(params);
  with_shape(T, [&](auto G, auto E) {
    refine_kernel<G(), E()><<<rf_blocks<G()>(n), RF_THREADS, 0, st>>>(
        psi, phi, T, H, W, p4, keep, MW, n, e, ac, out_lh, out_flux, out_lh_start);
  });
  KB_LAUNCH_CHECK("refine_kernel");
  return KB_OK;
}

extern "C" int kb_candidate_params(const int32_t* cand_pix, const int32_t* cand_slot, int n,
                                   const int32_t* idx, const uint32_t* mask, int K, int T,
                                   const float* vx, const float* vy, int x_lo, int y_lo, int wx,
                                   float* out_params, uint32_t* out_keep, void* stream) {
  using namespace kb;
  if (n < 0 || K < 1 || K > KB_MAX_K || T < 1 || wx < 1)
    return fail(KB_ERR_INVALID_ARG, "kb_candidate_params: bad sizes");
  if (T > KB_MAX_T) return fail(KB_ERR_UNSUPPORTED, "kb_candidate_params: T > KB_MAX_T");
  if (n == 0) return KB_OK;
  if (!cand_pix || !cand_slot || !idx || !vx || !vy || !out_params || (out_keep && !mask))
    return fail(KB_ERR_INVALID_ARG, "kb_candidate_params: null pointer argument");
  if (!aligned16(out_params))
    return fail(KB_ERR_INVALID_ARG, "kb_candidate_params: out_params not 16-byte aligned");
  KB_FAULT_POINT("kb_candidate_params");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  candidate_params_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
      cand_pix, cand_slot, n, idx, mask, K, (T + 31) / 32, vx, vy, x_lo, y_lo, wx,
      reinterpret_cast<float4*>(out_params), out_keep);
  KB_LAUNCH_CHECK("candidate_params_kernel");
  return KB_OK;
}
