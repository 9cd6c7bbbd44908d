// psi_phi.cu -- PSF-matched likelihood images psi_t, phi_t (Section 3, first paragraph).
//
// psi = (w I) correlated with P, phi = w correlated with P^2, w = 1/var (0 outside the image and
// at masked pixels); psi = phi = 0 at a masked pixel.  One block computes a 32 x 32 output tile
// of one epoch.  The weighted image w*I and the weight w of the tile plus its halo are staged in
// shared memory once; each thread then produces 8 vertically adjacent outputs, so every staged
// value it loads feeds up to 8 multiply-adds per output plane (register blocking along y).
// At k = 15 this is ~2 x 225 FMAs per output pixel for 16 bytes of HBM traffic: the kernel is
// bound by FP32 issue, not by HBM.
#include "kb_internal.cuh"

namespace kb {

constexpr int PP_TX = 32;         // output tile width (one warp of x)
constexpr int PP_ROWS = 8;        // outputs per thread along y
constexpr int PP_TY = 32;         // output tile height
constexpr int PP_THREADS = PP_TX * (PP_TY / PP_ROWS);  // 128

__device__ __forceinline__ bool masked_px(float img, float var, const uint8_t* mask, size_t i) {
  if (mask && mask[i]) return true;
  if (!(var > 0.0f) || !isfinite(var)) return true;
  if (!isfinite(img)) return true;
  return false;
}

template <int KS>
__global__ void __launch_bounds__(PP_THREADS)
psi_phi_kernel(const float* __restrict__ img, const float* __restrict__ var,
               const uint8_t* __restrict__ mask, const float* __restrict__ psf, int H, int W,
               float* __restrict__ psi, float* __restrict__ phi) {
  constexpr int R = KS / 2;
  constexpr int SW = PP_TX + 2 * R;   // staged width
  constexpr int SH = PP_TY + 2 * R;   // staged height
  __shared__ float sA[SH][SW];        // w * I
  __shared__ float sW[SH][SW];        // w
  __shared__ float sP[KS * KS];
  __shared__ float sP2[KS * KS];

  const int t = blockIdx.z;
  const int x0 = blockIdx.x * PP_TX, y0 = blockIdx.y * PP_TY;
  const size_t plane = (size_t)H * W;
  const float* I = img + (size_t)t * plane;
  const float* V = var + (size_t)t * plane;
  const uint8_t* M = mask ? mask + (size_t)t * plane : nullptr;
  const int tid = threadIdx.y * PP_TX + threadIdx.x;

  for (int i = tid; i < KS * KS; i += PP_THREADS) {
    float p = psf[(size_t)t * KS * KS + i];
    sP[i] = p;
    sP2[i] = p * p;
  }
  for (int i = tid; i < SH * SW; i += PP_THREADS) {
    int sy = i / SW, sx = i - sy * SW;
    int y = y0 - R + sy, x = x0 - R + sx;
    float a = 0.0f, w = 0.0f;
    if (y >= 0 && y < H && x >= 0 && x < W) {
      size_t o = (size_t)y * W + x;
      float iv = __ldg(I + o), vv = __ldg(V + o);
      if (!masked_px(iv, vv, M, o)) {
        w = __frcp_rn(vv);
        a = w * iv;
      }
    }
    sA[sy][sx] = a;
    sW[sy][sx] = w;
  }
  __syncthreads();

  const int lx = threadIdx.x, ly = threadIdx.y * PP_ROWS;
  float s1[PP_ROWS], s2[PP_ROWS];
#pragma unroll
  for (int i = 0; i < PP_ROWS; ++i) s1[i] = s2[i] = 0.0f;

#pragma unroll 1
  for (int ux = 0; ux < KS; ++ux) {
    float pc[KS], p2c[KS];
#pragma unroll
    for (int uy = 0; uy < KS; ++uy) {
      pc[uy] = sP[uy * KS + ux];
      p2c[uy] = sP2[uy * KS + ux];
    }
#pragma unroll
    for (int j = 0; j < PP_ROWS + KS - 1; ++j) {
      const float a = sA[ly + j][lx + ux];
      const float w = sW[ly + j][lx + ux];
#pragma unroll
      for (int i = 0; i < PP_ROWS; ++i) {
        const int uy = j - i;
        if (uy >= 0 && uy < KS) {
          s1[i] = fmaf(a, pc[uy], s1[i]);
          s2[i] = fmaf(w, p2c[uy], s2[i]);
        }
      }
    }
  }

  const int x = x0 + lx;
  if (x >= W) return;
#pragma unroll
  for (int i = 0; i < PP_ROWS; ++i) {
    const int y = y0 + ly + i;
    if (y >= H) break;
    const size_t o = (size_t)y * W + x;
    // centre pixel masked <=> its staged weight is zero
    const bool m = sW[ly + i + R][lx + R] == 0.0f;
    psi[(size_t)t * plane + o] = m ? 0.0f : s1[i];
    phi[(size_t)t * plane + o] = m ? 0.0f : s2[i];
  }
}

template <int KS>
static void launch_pp(const float* img, const float* var, const uint8_t* mask, const float* psf,
                      int T, int H, int W, float* psi, float* phi, cudaStream_t st) {
  dim3 grid((W + PP_TX - 1) / PP_TX, (H + PP_TY - 1) / PP_TY, T);
  dim3 block(PP_TX, PP_TY / PP_ROWS);
  psi_phi_kernel<KS><<<grid, block, 0, st>>>(img, var, mask, psf, H, W, psi, phi);
}

}  // namespace kb

extern "C" int kb_make_psi_phi(const float* img, const float* var, const uint8_t* mask,
                               const float* psf, int T, int H, int W, int k, float* psi,
                               float* phi, void* stream) {
  using namespace kb;
  if (!img || !var || !psf || !psi || !phi)
    return fail(KB_ERR_INVALID_ARG, "kb_make_psi_phi: null pointer argument");
  if (T < 1 || H < 1 || W < 1) return fail(KB_ERR_INVALID_ARG, "kb_make_psi_phi: bad T/H/W");
  if (T > 65535) return fail(KB_ERR_UNSUPPORTED, "kb_make_psi_phi: T > 65535");
  if (k < 1 || k > 31 || (k & 1) == 0)
    return fail(KB_ERR_INVALID_ARG, "kb_make_psi_phi: k must be odd and in 1..31 (got %d)", k);
  if (psi == img || phi == img || psi == phi)
    return fail(KB_ERR_INVALID_ARG, "kb_make_psi_phi: outputs alias inputs");
  KB_FAULT_POINT("kb_make_psi_phi");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  switch (k) {
#define KB_PP_CASE(K) \
  case K: launch_pp<K>(img, var, mask, psf, T, H, W, psi, phi, st); break;
    KB_PP_CASE(1) KB_PP_CASE(3) KB_PP_CASE(5) KB_PP_CASE(7) KB_PP_CASE(9) KB_PP_CASE(11)
    KB_PP_CASE(13) KB_PP_CASE(15) KB_PP_CASE(17) KB_PP_CASE(19) KB_PP_CASE(21) KB_PP_CASE(23)
    KB_PP_CASE(25) KB_PP_CASE(27) KB_PP_CASE(29) KB_PP_CASE(31)
#undef KB_PP_CASE
  }
  KB_LAUNCH_CHECK("psi_phi_kernel");
  return KB_OK;
}
