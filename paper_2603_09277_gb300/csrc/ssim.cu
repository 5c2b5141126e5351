// ssim.cu -- the D-SSIM term of L_base (Sec. 3 Eq. base): D-SSIM = 1 - SSIM
// with an 11x11 Gaussian window (sigma 1.5, normalised), zero padding outside
// the image, C1 = 0.01^2, C2 = 0.03^2, SSIM = mean over the view's pixels and
// channels (the 3DGS reading; the paper does not define the term).
//
// Forward, one CTA per 16x16 block of output pixels of one view: the block and
// its 5-pixel halo of image and target (all three channels) are staged in
// shared memory; each thread forms the window moments of its pixel from the
// 121 samples centred on the pixel's own value c (d = s - c; padding samples
// are s = 0): mu = c + E[d], sigma^2 = E[d^2] - E[d]^2, so smooth regions do
// not cancel two large FP32 sums.  Per pixel and channel it writes
// (mu_x, mu_y, dS/dmu_x, dS/dsigma_x^2, dS/dsigma_xy) for the backward and adds
// lambda (1 - S) / (3 M_v V) to the loss partials.
//
// Backward, same blocking over the saved maps:
//   dL/dx(p) -= lambda / (3 M_v V) sum_q G(q - p) [dS/dmu_x(q)
//               + 2 (x(p) - mu_x(q)) dS/dsigma_x^2(q) + (y(p) - mu_y(q)) dS/dsigma_xy(q)]
// over the window centres q inside the image (dsigma_x^2(q)/dx(p) =
// 2 G(q-p)(x(p) - mu_x(q)) because the window weights sum to 1).
#include <cmath>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kSsimR = 5;                   // window radius
constexpr int kSsimB = 16;                  // output block side
constexpr int kSsimS = kSsimB + 2 * kSsimR; // staged side (26)
constexpr int kSsimThreads = kSsimB * kSsimB;
constexpr float kC1 = 0.01f * 0.01f;
constexpr float kC2 = 0.03f * 0.03f;

struct SsimViews {
  int V;
  long long pix_off[GS_MAX_VIEWS];
  int W[GS_MAX_VIEWS], H[GS_MAX_VIEWS], BX[GS_MAX_VIEWS];
  int block_off[GS_MAX_VIEWS + 1];
  float scale[GS_MAX_VIEWS];  // lambda / (3 M_v V)
  float win[2 * kSsimR + 1];  // normalised 1D Gaussian, sigma 1.5
};

__device__ __forceinline__ int view_of_block(const SsimViews& sv, int b) {
  int v = 0;
  while (v + 1 < sv.V && b >= sv.block_off[v + 1]) ++v;
  return v;
}

__global__ void __launch_bounds__(kSsimThreads) ssim_fwd_kernel(
    const float* __restrict__ image, const float* __restrict__ target, const SsimViews sv,
    float* __restrict__ maps /* [P][3][5] */, double* __restrict__ partials) {
  __shared__ float sx[3][kSsimS][kSsimS];
  __shared__ float sy[3][kSsimS][kSsimS];
  const int b = blockIdx.x;
  const int v = view_of_block(sv, b);
  const int lb = b - sv.block_off[v];
  const int W = sv.W[v], H = sv.H[v];
  const int bx = (lb % sv.BX[v]) * kSsimB, by = (lb / sv.BX[v]) * kSsimB;
  const long long base = sv.pix_off[v];
  for (int i = threadIdx.x; i < kSsimS * kSsimS; i += kSsimThreads) {
    const int yy = by - kSsimR + i / kSsimS, xx = bx - kSsimR + i % kSsimS;
    const bool in = xx >= 0 && xx < W && yy >= 0 && yy < H;
    const long long p = base + (long long)yy * W + xx;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      sx[ch][i / kSsimS][i % kSsimS] = in ? image[3 * p + ch] : 0.f;
      sy[ch][i / kSsimS][i % kSsimS] = in ? target[3 * p + ch] : 0.f;
    }
  }
  __syncthreads();
  const int lx = threadIdx.x % kSsimB, ly = threadIdx.x / kSsimB;
  const int px = bx + lx, py = by + ly;
  double acc = 0.0;
  if (px < W && py < H) {
    const long long p = base + (long long)py * W + px;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float cx = sx[ch][ly + kSsimR][lx + kSsimR], cy = sy[ch][ly + kSsimR][lx + kSsimR];
      float m1 = 0.f, n1 = 0.f, dxx = 0.f, dyy = 0.f, dxy = 0.f;
      for (int j = 0; j < 2 * kSsimR + 1; ++j) {
        const float wj = sv.win[j];
#pragma unroll
        for (int i = 0; i < 2 * kSsimR + 1; ++i) {
          const float w = wj * sv.win[i];
          const float d = sx[ch][ly + j][lx + i] - cx, e = sy[ch][ly + j][lx + i] - cy;
          const float wd = w * d, we = w * e;
          m1 += wd;
          n1 += we;
          dxx = __fmaf_rn(wd, d, dxx);
          dyy = __fmaf_rn(we, e, dyy);
          dxy = __fmaf_rn(wd, e, dxy);
        }
      }
      const float mx = cx + m1, my = cy + n1;
      const float sxx = __fmaf_rn(-m1, m1, dxx), syy = __fmaf_rn(-n1, n1, dyy);
      const float sxy = __fmaf_rn(-m1, n1, dxy);
      const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
      const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
      const float D = B1 * B2;
      const float S = A1 * A2 / D;
      acc += (double)(1.f - S);
      float* m = maps + 15 * p + 5 * ch;
      m[0] = mx;
      m[1] = my;
      m[2] = (2.f * my * A2 - S * 2.f * mx * B2) / D;  // dS/dmu_x, sigmas fixed
      m[3] = -S / B2;                                  // dS/dsigma_x^2
      m[4] = 2.f * A1 / D;                             // dS/dsigma_xy
    }
  }
  acc *= (double)sv.scale[v];
  __shared__ double s_red[kSsimThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kSsimThreads / 32; ++k) t += s_red[k];
    partials[b] = t;
  }
}

__global__ void __launch_bounds__(kSsimThreads) ssim_bwd_kernel(
    const float* __restrict__ image, const float* __restrict__ target, const SsimViews sv,
    const float* __restrict__ maps, float* __restrict__ dimg) {
  __shared__ float sm[5][kSsimS][kSsimS];  // one channel at a time
  const int b = blockIdx.x;
  const int v = view_of_block(sv, b);
  const int lb = b - sv.block_off[v];
  const int W = sv.W[v], H = sv.H[v];
  const int bx = (lb % sv.BX[v]) * kSsimB, by = (lb / sv.BX[v]) * kSsimB;
  const long long base = sv.pix_off[v];
  const int lx = threadIdx.x % kSsimB, ly = threadIdx.x / kSsimB;
  const int px = bx + lx, py = by + ly;
  const bool mine = px < W && py < H;
  const long long p = base + (long long)py * W + px;
  for (int ch = 0; ch < 3; ++ch) {
    __syncthreads();  // the previous channel's readers are done
    for (int i = threadIdx.x; i < kSsimS * kSsimS; i += kSsimThreads) {
      const int yy = by - kSsimR + i / kSsimS, xx = bx - kSsimR + i % kSsimS;
      const bool in = xx >= 0 && xx < W && yy >= 0 && yy < H;  // window centres in the image
      const long long q = base + (long long)yy * W + xx;
#pragma unroll
      for (int k = 0; k < 5; ++k) sm[k][i / kSsimS][i % kSsimS] = in ? maps[15 * q + 5 * ch + k] : 0.f;
    }
    __syncthreads();
    if (mine) {
      const float xp = image[3 * p + ch], yp = target[3 * p + ch];
      float acc = 0.f;
      for (int j = 0; j < 2 * kSsimR + 1; ++j) {
        const float wj = sv.win[j];
#pragma unroll
        for (int i = 0; i < 2 * kSsimR + 1; ++i) {
          const float w = wj * sv.win[i];
          const int r = ly + j, c = lx + i;
          const float t = __fmaf_rn(2.f * (xp - sm[0][r][c]), sm[3][r][c],
                                    __fmaf_rn(yp - sm[1][r][c], sm[4][r][c], sm[2][r][c]));
          acc = __fmaf_rn(w, t, acc);
        }
      }
      dimg[3 * p + ch] -= sv.scale[v] * acc;
    }
  }
}

}  // namespace

size_t ssim_workspace_bytes(long long total_pixels) {
  return sizeof(float) * 15 * (size_t)total_pixels;
}

int ssim_blocks(const CamTable& ct) {
  long long n = 0;
  for (int v = 0; v < ct.V; ++v)
    n += (long long)((ct.c[v].W + kSsimB - 1) / kSsimB) * ((ct.c[v].H + kSsimB - 1) / kSsimB);
  return (int)n;
}

// Adds lambda (1 - SSIM_v) / V per view to the partials (one per block) and
// the term's gradient to dimg; maps is ssim_workspace_bytes(P) of scratch.
int launch_ssim(const float* image, const float* target, const CamTable& ct, float lambda,
                float* maps, double* partials, float* dimg, cudaStream_t st) {
  SsimViews sv;
  {
    double g[2 * kSsimR + 1], sum = 0.0;
    for (int k = -kSsimR; k <= kSsimR; ++k) {
      g[k + kSsimR] = exp(-(double)(k * k) / (2.0 * 1.5 * 1.5));
      sum += g[k + kSsimR];
    }
    for (int k = 0; k < 2 * kSsimR + 1; ++k) sv.win[k] = (float)(g[k] / sum);
  }
  sv.V = ct.V;
  sv.block_off[0] = 0;
  for (int v = 0; v < ct.V; ++v) {
    const CamInfo& c = ct.c[v];
    sv.pix_off[v] = c.pix_off;
    sv.W[v] = c.W;
    sv.H[v] = c.H;
    sv.BX[v] = (c.W + kSsimB - 1) / kSsimB;
    sv.block_off[v + 1] = sv.block_off[v] + sv.BX[v] * ((c.H + kSsimB - 1) / kSsimB);
    sv.scale[v] = (float)((double)lambda / (3.0 * (double)c.W * c.H * ct.V));
  }
  const int nb = sv.block_off[ct.V];
  if (nb == 0) return GS_OK;
  ssim_fwd_kernel<<<nb, kSsimThreads, 0, st>>>(image, target, sv, maps, partials);
  ssim_bwd_kernel<<<nb, kSsimThreads, 0, st>>>(image, target, sv, maps, dimg);
  count_launches(2);
  return check_launch();
}

}  // namespace gs
