// ssim.cu -- the D-SSIM term of L_base (Sec. 3 Eq. base): D-SSIM = 1 - SSIM
// with an 11x11 Gaussian window (sigma 1.5, normalised), zero padding outside
// the image, C1 = 0.01^2, C2 = 0.03^2, SSIM = mean over the view's pixels and
// channels (the 3DGS reading; the paper does not define the term).
//
// Forward, one CTA per 16x16 block of output pixels of one view: the block and
// its 5-pixel halo of image and target (all three channels) are staged in
// shared memory.  The window moments are taken about a constant per block and
// channel (the staged value at the block centre, c): with d = s - c (padding
// samples s = 0), mu = c + E[d] and sigma^2 = E[d^2] - E[d]^2 hold exactly
// for any constant, and around a value of the block two large FP32 sums do
// not cancel in smooth regions.  Because c is constant over the block, the
// 11x11 window sums are separable: a horizontal pass over the 26 staged rows
// and a vertical pass per output pixel.  Per pixel and channel the forward
// saves (mu_x, mu_y, dS/dmu_x, dS/dsigma_x^2, dS/dsigma_xy) (planar, one plane
// per quantity) and adds lambda (1 - S) / (3 M_v V) to the loss partials.
//
// Backward, same blocking:
//   dL/dx(p) -= lambda / (3 M_v V) sum_q G(q - p) [dS/dmu_x(q)
//               + 2 (x(p) - mu_x(q)) dS/dsigma_x^2(q) + (y(p) - mu_y(q)) dS/dsigma_xy(q)]
// over the window centres q inside the image (dsigma_x^2(q)/dx(p) =
// 2 G(q-p)(x(p) - mu_x(q)) because the window weights sum to 1); with the
// block constant c the bracket splits into five separable correlations:
// G*a + 2 (x(p) - c) G*b - 2 G*((mu_x - c) b) + (y(p) - c') G*e - G*((mu_y - c') e).
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

// Horizontal pass of the separable window: h[k][r][x] = sum_i w_i f_k(r, x + i)
// for the 26 staged rows and 16 output columns.
constexpr int kHN = kSsimS * kSsimB;  // 416 horizontal outputs per quantity

__global__ void __launch_bounds__(kSsimThreads) ssim_fwd_kernel(
    const float* __restrict__ image, const float* __restrict__ target, const SsimViews sv,
    float* __restrict__ maps /* 15 planes of P */, long long P, double* __restrict__ partials) {
  __shared__ float sx[3][kSsimS][kSsimS];
  __shared__ float sy[3][kSsimS][kSsimS];
  __shared__ float sh[5][kHN];
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
  const bool mine = px < W && py < H;
  const long long p = base + (long long)py * W + px;
  float acc = 0.f;  // 1 - S >= 0: FP32 within the thread and the warp, FP64 beyond
  for (int ch = 0; ch < 3; ++ch) {
    const float cx = sx[ch][kSsimR + kSsimB / 2][kSsimR + kSsimB / 2];
    const float cy = sy[ch][kSsimR + kSsimB / 2][kSsimR + kSsimB / 2];
    for (int t = threadIdx.x; t < kHN; t += kSsimThreads) {
      const int r = t / kSsimB, x = t % kSsimB;
      float m = 0.f, n = 0.f, dd = 0.f, ee = 0.f, de = 0.f;
#pragma unroll
      for (int i = 0; i < 2 * kSsimR + 1; ++i) {
        const float w = sv.win[i];
        const float d = sx[ch][r][x + i] - cx, e = sy[ch][r][x + i] - cy;
        const float wd = w * d, we = w * e;
        m += wd;
        n += we;
        dd = __fmaf_rn(wd, d, dd);
        ee = __fmaf_rn(we, e, ee);
        de = __fmaf_rn(wd, e, de);
      }
      sh[0][t] = m;
      sh[1][t] = n;
      sh[2][t] = dd;
      sh[3][t] = ee;
      sh[4][t] = de;
    }
    __syncthreads();
    if (mine) {
      float m1 = 0.f, n1 = 0.f, dxx = 0.f, dyy = 0.f, dxy = 0.f;
#pragma unroll
      for (int j = 0; j < 2 * kSsimR + 1; ++j) {
        const float w = sv.win[j];
        const int t = (ly + j) * kSsimB + lx;
        m1 = __fmaf_rn(w, sh[0][t], m1);
        n1 = __fmaf_rn(w, sh[1][t], n1);
        dxx = __fmaf_rn(w, sh[2][t], dxx);
        dyy = __fmaf_rn(w, sh[3][t], dyy);
        dxy = __fmaf_rn(w, sh[4][t], dxy);
      }
      const float mx = cx + m1, my = cy + n1;
      const float sxx = __fmaf_rn(-m1, m1, dxx), syy = __fmaf_rn(-n1, n1, dyy);
      const float sxy = __fmaf_rn(-m1, n1, dxy);
      const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
      const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
      const float D = B1 * B2;
      const float S = A1 * A2 / D;
      acc += 1.f - S;
      float* m = maps + (long long)(5 * ch) * P + p;
      m[0] = mx;
      m[P] = my;
      m[2 * P] = (2.f * my * A2 - S * 2.f * mx * B2) / D;  // dS/dmu_x, sigmas fixed
      m[3 * P] = -S / B2;                                  // dS/dsigma_x^2
      m[4 * P] = 2.f * A1 / D;                             // dS/dsigma_xy
    }
    __syncthreads();  // sh is rewritten for the next channel
  }
  __shared__ double s_red[kSsimThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = (double)acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kSsimThreads / 32; ++k) t += s_red[k];
    partials[b] = t * (double)sv.scale[v];
  }
}

__global__ void __launch_bounds__(kSsimThreads) ssim_bwd_kernel(
    const float* __restrict__ image, const float* __restrict__ target, const SsimViews sv,
    const float* __restrict__ maps, long long P, float* __restrict__ dimg) {
  __shared__ float sm[5][kSsimS][kSsimS];  // one channel at a time
  __shared__ float sh[5][kHN];
  __shared__ float s_c[2];
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
  // block constants: the image and target at the block's first pixel
  const long long p0 = base + (long long)by * W + bx;
  for (int ch = 0; ch < 3; ++ch) {
    if (threadIdx.x == 0) {
      s_c[0] = image[3 * p0 + ch];
      s_c[1] = target[3 * p0 + ch];
    }
    __syncthreads();  // (also: the previous channel's readers are done)
    const float cx = s_c[0], cy = s_c[1];
    const float* mp = maps + (long long)(5 * ch) * P;
    for (int i = threadIdx.x; i < kSsimS * kSsimS; i += kSsimThreads) {
      const int yy = by - kSsimR + i / kSsimS, xx = bx - kSsimR + i % kSsimS;
      const bool in = xx >= 0 && xx < W && yy >= 0 && yy < H;  // window centres in the image
      const long long q = base + (long long)yy * W + xx;
      float a = 0.f, bb = 0.f, e = 0.f, pm = 0.f, qm = 0.f;
      if (in) {
        const float mx = mp[q], my = mp[P + q];
        a = mp[2 * P + q];
        bb = mp[3 * P + q];
        e = mp[4 * P + q];
        pm = (mx - cx) * bb;
        qm = (my - cy) * e;
      }
      sm[0][i / kSsimS][i % kSsimS] = a;
      sm[1][i / kSsimS][i % kSsimS] = bb;
      sm[2][i / kSsimS][i % kSsimS] = e;
      sm[3][i / kSsimS][i % kSsimS] = pm;
      sm[4][i / kSsimS][i % kSsimS] = qm;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kHN; t += kSsimThreads) {
      const int r = t / kSsimB, x = t % kSsimB;
      float h[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < 2 * kSsimR + 1; ++i) {
        const float w = sv.win[i];
#pragma unroll
        for (int k = 0; k < 5; ++k) h[k] = __fmaf_rn(w, sm[k][r][x + i], h[k]);
      }
#pragma unroll
      for (int k = 0; k < 5; ++k) sh[k][t] = h[k];
    }
    __syncthreads();
    if (mine) {
      float g[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int j = 0; j < 2 * kSsimR + 1; ++j) {
        const float w = sv.win[j];
        const int t = (ly + j) * kSsimB + lx;
#pragma unroll
        for (int k = 0; k < 5; ++k) g[k] = __fmaf_rn(w, sh[k][t], g[k]);
      }
      const float xp = image[3 * p + ch], yp = target[3 * p + ch];
      const float grad = g[0] + 2.f * ((xp - cx) * g[1] - g[3]) + (yp - cy) * g[2] - g[4];
      dimg[3 * p + ch] -= sv.scale[v] * grad;
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
  const long long P = ct.c[ct.V - 1].pix_off + (long long)ct.c[ct.V - 1].W * ct.c[ct.V - 1].H;
  ssim_fwd_kernel<<<nb, kSsimThreads, 0, st>>>(image, target, sv, maps, P, partials);
  ssim_bwd_kernel<<<nb, kSsimThreads, 0, st>>>(image, target, sv, maps, P, dimg);
  count_launches(2);
  return check_launch();
}

}  // namespace gs
