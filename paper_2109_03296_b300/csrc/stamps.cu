// stamps.cu -- coadded postage stamps along trajectories (Section 3.3: per-pixel median of the
// stamps along the trajectory, which suppresses differencing artifacts; also the mean).
//
// One block per candidate, one warp per stamp pixel at a time with lanes over epochs (up to 4
// epochs per lane): each lane gathers its epoch's pixel, a ballot counts the contributing epochs,
// the mean is a butterfly sum, and the median comes from a warp bitonic sort of the values
// (non-contributing epochs sort last as +inf).
#include <cmath>

#include "kb_internal.cuh"

namespace kb {

constexpr int ST_WARPS = 8;

struct StampConsts {
  float dt[KB_MAX_T];
};

template <int J>
__device__ __forceinline__ void st_bitonic(float (&v)[J], int lane) {
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
            v[j] = up ? fminf(a, b) : fmaxf(a, b);
            v[jp] = up ? fmaxf(a, b) : fminf(a, b);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < J; ++j) {
          const float o = __shfl_xor_sync(0xffffffffu, v[j], d);
          const bool up = (((j << 5) | lane) & k) == 0;
          v[j] = (((lane & d) == 0) == up) ? fminf(v[j], o) : fmaxf(v[j], o);
        }
      }
    }
  }
}

template <int J>
__device__ __forceinline__ float st_get(const float (&v)[J], int r) {
  float x = v[0];
#pragma unroll
  for (int j = 1; j < J; ++j)
    if ((r >> 5) == j) x = v[j];
  return __shfl_sync(0xffffffffu, x, r & 31);
}

template <int J>
__global__ void __launch_bounds__(ST_WARPS * 32)
stamps_kernel(const float* __restrict__ img, const float* __restrict__ var,
              const uint8_t* __restrict__ mask, int T, int H, int W,
              const int32_t* __restrict__ x0, const int32_t* __restrict__ y0,
              const float* __restrict__ vx, const float* __restrict__ vy,
              const uint32_t* __restrict__ keep_mask, int radius, StampConsts cs,
              float* __restrict__ out_mean, float* __restrict__ out_median) {
  const int c = blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int side = 2 * radius + 1;
  const int mw = (T + 31) / 32;
  const size_t plane = (size_t)H * W;
  const int cx = x0[c], cy = y0[c];
  const float cvx = vx[c], cvy = vy[c];
  int xt[J], yt[J];
  bool use[J];
#pragma unroll
  for (int j = 0; j < J; ++j) {
    const int t = (j << 5) | lane;
    use[j] = t < T;
    xt[j] = yt[j] = 0;
    if (use[j]) {
      const float dt = cs.dt[t];
      // offsets clamped to +-2^24 (sides are at most 2^20): out-of-image stays out of image
      xt[j] = cx + (int)fminf(fmaxf(floorf(__fadd_rn(__fmul_rn(cvx, dt), 0.5f)), -16777216.0f),
                              16777216.0f);
      yt[j] = cy + (int)fminf(fmaxf(floorf(__fadd_rn(__fmul_rn(cvy, dt), 0.5f)), -16777216.0f),
                              16777216.0f);
      if (keep_mask) use[j] = (keep_mask[(size_t)c * mw + (t >> 5)] >> (t & 31)) & 1u;
    }
  }
  for (int s = warp; s < side * side; s += ST_WARPS) {
    const int sy = s / side - radius, sx = s % side - radius;
    float v[J];
    bool ok[J];
#pragma unroll
    for (int j = 0; j < J; ++j) {
      ok[j] = false;
      v[j] = INFINITY;
      const int x = xt[j] + sx, y = yt[j] + sy;
      if (use[j] && x >= 0 && x < W && y >= 0 && y < H) {
        const int t = (j << 5) | lane;
        const size_t i = (size_t)t * plane + (size_t)y * W + x;
        const float a = __ldg(img + i), w = __ldg(var + i);
        if (!(mask && mask[i]) && w > 0.0f && isfinite(w) && isfinite(a)) {
          ok[j] = true;
          v[j] = a;
        }
      }
    }
    int n = 0;
    float sum = 0.0f;
#pragma unroll
    for (int j = 0; j < J; ++j) {
      n += __popc(__ballot_sync(0xffffffffu, ok[j]));
      sum += ok[j] ? v[j] : 0.0f;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    float med = NAN, mean = NAN;
    if (n > 0) {
      mean = __fdiv_rn(sum, (float)n);
      st_bitonic<J>(v, lane);
      const float hi = st_get<J>(v, n >> 1);
      med = (n & 1) ? hi : 0.5f * (st_get<J>(v, (n >> 1) - 1) + hi);
    }
    if (lane == 0) {
      const size_t o = (size_t)c * side * side + (size_t)s;
      out_mean[o] = mean;
      out_median[o] = med;
    }
  }
}

}  // namespace kb

extern "C" int kb_stamps(const float* img, const float* var, const uint8_t* mask,
                         const double* times, int T, int H, int W, const int32_t* x0,
                         const int32_t* y0, const float* vx, const float* vy,
                         const uint32_t* keep_mask, int n, int radius, float* out_mean,
                         float* out_median, void* stream) {
  using namespace kb;
  if (!img || !var || !times || !out_mean || !out_median)
    return fail(KB_ERR_INVALID_ARG, "kb_stamps: null pointer argument");
  if (n < 0 || T < 1 || H < 1 || W < 1) return fail(KB_ERR_INVALID_ARG, "kb_stamps: bad sizes");
  if (H > (1 << 20) || W > (1 << 20))
    return fail(KB_ERR_UNSUPPORTED, "kb_stamps: image sides are limited to 2^20 pixels");
  if (n > 0 && (!x0 || !y0 || !vx || !vy))
    return fail(KB_ERR_INVALID_ARG, "kb_stamps: null candidate array");
  if (T > KB_MAX_T) return fail(KB_ERR_UNSUPPORTED, "kb_stamps: T > KB_MAX_T");
  if (radius < 0 || radius > 15) return fail(KB_ERR_INVALID_ARG, "kb_stamps: radius outside 0..15");
  if (n > 2147483647 / ((2 * radius + 1) * (2 * radius + 1)))
    return fail(KB_ERR_UNSUPPORTED, "kb_stamps: too many candidates");
  StampConsts cs{};
  for (int t = 0; t < T; ++t) {
    if (!std::isfinite(times[t])) return fail(KB_ERR_INVALID_ARG, "kb_stamps: times not finite");
    cs.dt[t] = (float)(times[t] - times[0]);
  }
  if (n == 0) return KB_OK;
  KB_FAULT_POINT("kb_stamps");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int J = (T + 31) / 32;
  if (J == 1)
    stamps_kernel<1><<<n, ST_WARPS * 32, 0, st>>>(img, var, mask, T, H, W, x0, y0, vx, vy,
                                                  keep_mask, radius, cs, out_mean, out_median);
  else if (J == 2)
    stamps_kernel<2><<<n, ST_WARPS * 32, 0, st>>>(img, var, mask, T, H, W, x0, y0, vx, vy,
                                                  keep_mask, radius, cs, out_mean, out_median);
  else
    stamps_kernel<4><<<n, ST_WARPS * 32, 0, st>>>(img, var, mask, T, H, W, x0, y0, vx, vy,
                                                  keep_mask, radius, cs, out_mean, out_median);
  KB_LAUNCH_CHECK("stamps_kernel");
  return KB_OK;
}

// ------------------------------------------------------------------------------------------------
// Central-moment filter of coadded stamps (Section 3.3): moments about the stamp centre of the
// weights w = S - min S (NaN pixels left out), normalised by their sum; a stamp passes when they
// are those of a compact source at the centre.  One warp per stamp, lanes striding over the
// pixels: a warp minimum, then the six weighted sums in float64 (a few hundred terms per stamp,
// so the cost is negligible), so that a decision differs from the exact one only for moments
// within ~1e-15 relative of a limit.
// ------------------------------------------------------------------------------------------------
namespace kb {

struct MomentLimits {
  double x, y, xy, xx, yy;
};

__global__ void stamp_moments_kernel(const float* __restrict__ stamps, int n, int radius,
                                     MomentLimits lim, float* __restrict__ out_moments,
                                     uint8_t* __restrict__ out_pass) {
  const long long c = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= n) return;
  const int lane = threadIdx.x & 31;
  const int side = 2 * radius + 1, npx = side * side;
  const float* S = stamps + c * npx;
  float lo = INFINITY;
  for (int i = lane; i < npx; i += 32) {
    float v = __ldg(S + i);
    if (!isnan(v)) lo = fminf(lo, v);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
  double m[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (int i = lane; i < npx; i += 32) {
    float v = __ldg(S + i);
    if (isnan(v)) continue;
    double dv = (double)v - (double)lo;
    double dx = (double)(i % side - radius), dy = (double)(i / side - radius);
    m[0] += dv;
    m[1] += dx * dv;
    m[2] += dy * dv;
    m[3] += dx * dy * dv;
    m[4] += dx * dx * dv;
    m[5] += dy * dy * dv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1)
#pragma unroll
    for (int k = 0; k < 6; ++k) m[k] += __shfl_xor_sync(0xffffffffu, m[k], o);
  if (lane != 0) return;
  const double x = m[1] / m[0], y = m[2] / m[0], xy = m[3] / m[0], xx = m[4] / m[0],
               yy = m[5] / m[0];
  if (out_moments) {
    float* o = out_moments + c * 6;
    o[0] = (float)m[0];
    o[1] = (float)x;
    o[2] = (float)y;
    o[3] = (float)xy;
    o[4] = (float)xx;
    o[5] = (float)yy;
  }
  const bool pass = m[0] > 0.0 && fabs(x) < lim.x && fabs(y) < lim.y && fabs(xy) < lim.xy &&
                    xx < lim.xx && yy < lim.yy;
  out_pass[c] = pass ? 1 : 0;
}

}  // namespace kb

extern "C" int kb_stamp_filter(const float* stamps, int n, int radius, const float* limits,
                               float* out_moments, uint8_t* out_pass, void* stream) {
  using namespace kb;
  if (n < 0) return fail(KB_ERR_INVALID_ARG, "kb_stamp_filter: n < 0");
  if (radius < 0 || radius > 15)
    return fail(KB_ERR_INVALID_ARG, "kb_stamp_filter: radius outside 0..15");
  if (n == 0) return KB_OK;
  if (!stamps || !out_pass) return fail(KB_ERR_INVALID_ARG, "kb_stamp_filter: null pointer");
  MomentLimits lim{0.5, 0.5, 1.5, 36.5, 36.5};
  if (limits) {
    lim = MomentLimits{limits[0], limits[1], limits[2], limits[3], limits[4]};
    for (int k = 0; k < 5; ++k)
      if (std::isnan(limits[k])) return fail(KB_ERR_INVALID_ARG, "kb_stamp_filter: NaN limit");
  }
  KB_FAULT_POINT("kb_stamp_filter");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int warps = 8;
  stamp_moments_kernel<<<(unsigned)((n + warps - 1) / warps), warps * 32, 0, st>>>(
      stamps, n, radius, lim, out_moments, out_pass);
  KB_LAUNCH_CHECK("stamp_moments_kernel");
  return KB_OK;
}
