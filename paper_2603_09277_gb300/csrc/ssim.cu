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

// Both passes of the separable window are register-blocked: a thread takes
// kRun consecutive outputs along the pass direction, loads the kRun + 10
// samples they share from shared memory once, and sums each output's 11 taps
// in tap order (the same arithmetic per output as a tap-by-tap loop).  All
// three channels are passed together.
constexpr int kRun = 4;                          // outputs per thread and pass
constexpr int kSpan = kRun + 2 * kSsimR;         // samples per run (14)
constexpr int kHItems = 3 * kSsimS * (kSsimB / kRun);  // horizontal runs (312)
constexpr int kVItems = 3 * kSsimB * (kSsimB / kRun);  // vertical runs (192)
static_assert(kSsimB % kRun == 0, "runs tile the block");
static_assert(kVItems <= kSsimThreads, "one vertical run per thread");

// Exclusive per-block partial of sum (1 - S) (FP32 within the thread and the
// warp: every term is >= 0; FP64 across the warps).
__device__ __forceinline__ void block_partial(float acc, double scale, double* out) {
  __shared__ double s_red[kSsimThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = (double)acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kSsimThreads / 32; ++k) t += s_red[k];
    *out = t * scale;
  }
}

__global__ void __launch_bounds__(kSsimThreads) ssim_fwd_kernel(
    const float* __restrict__ image, const float* __restrict__ target, const SsimViews sv,
    float* __restrict__ maps /* 15 planes of P */, long long P, double* __restrict__ partials) {
  __shared__ float sx[3][kSsimS][kSsimS];
  __shared__ float sy[3][kSsimS][kSsimS];
  __shared__ __align__(16) float sh[3][5][kSsimS][kSsimB];  // horizontal sums
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
  // horizontal: run (ch, staged row r, columns x0 .. x0 + kRun - 1)
  for (int it = threadIdx.x; it < kHItems; it += kSsimThreads) {
    const int g = it % (kSsimB / kRun), r = (it / (kSsimB / kRun)) % kSsimS;
    const int ch = it / (kSsimS * (kSsimB / kRun));
    const int x0 = g * kRun;
    const float cx = sx[ch][kSsimR + kSsimB / 2][kSsimR + kSsimB / 2];
    const float cy = sy[ch][kSsimR + kSsimB / 2][kSsimR + kSsimB / 2];
    float d[kSpan], e[kSpan];
#pragma unroll
    for (int j = 0; j < kSpan; ++j) {
      d[j] = sx[ch][r][x0 + j] - cx;
      e[j] = sy[ch][r][x0 + j] - cy;
    }
    float m[kRun], n[kRun], dd[kRun], ee[kRun], de[kRun];
#pragma unroll
    for (int o = 0; o < kRun; ++o) m[o] = n[o] = dd[o] = ee[o] = de[o] = 0.f;
#pragma unroll
    for (int i = 0; i < 2 * kSsimR + 1; ++i) {
      const float w = sv.win[i];
#pragma unroll
      for (int o = 0; o < kRun; ++o) {
        const float wd = w * d[o + i], we = w * e[o + i];
        m[o] += wd;
        n[o] += we;
        dd[o] = __fmaf_rn(wd, d[o + i], dd[o]);
        ee[o] = __fmaf_rn(we, e[o + i], ee[o]);
        de[o] = __fmaf_rn(wd, e[o + i], de[o]);
      }
    }
    *reinterpret_cast<float4*>(&sh[ch][0][r][x0]) = make_float4(m[0], m[1], m[2], m[3]);
    *reinterpret_cast<float4*>(&sh[ch][1][r][x0]) = make_float4(n[0], n[1], n[2], n[3]);
    *reinterpret_cast<float4*>(&sh[ch][2][r][x0]) = make_float4(dd[0], dd[1], dd[2], dd[3]);
    *reinterpret_cast<float4*>(&sh[ch][3][r][x0]) = make_float4(ee[0], ee[1], ee[2], ee[3]);
    *reinterpret_cast<float4*>(&sh[ch][4][r][x0]) = make_float4(de[0], de[1], de[2], de[3]);
  }
  __syncthreads();
  // vertical: run (ch, column c, output rows y0 .. y0 + kRun - 1)
  float acc = 0.f;
  if (threadIdx.x < kVItems) {
    const int c = threadIdx.x % kSsimB, q = (threadIdx.x / kSsimB) % (kSsimB / kRun);
    const int ch = threadIdx.x / (kSsimB * (kSsimB / kRun));
    const int y0 = q * kRun;
    const float cx = sx[ch][kSsimR + kSsimB / 2][kSsimR + kSsimB / 2];
    const float cy = sy[ch][kSsimR + kSsimB / 2][kSsimR + kSsimB / 2];
    float mom[5][kRun];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      float col[kSpan];
#pragma unroll
      for (int j = 0; j < kSpan; ++j) col[j] = sh[ch][k][y0 + j][c];
#pragma unroll
      for (int o = 0; o < kRun; ++o) {
        float t = 0.f;
#pragma unroll
        for (int j = 0; j < 2 * kSsimR + 1; ++j) t = __fmaf_rn(sv.win[j], col[o + j], t);
        mom[k][o] = t;
      }
    }
    const int px = bx + c;
#pragma unroll
    for (int o = 0; o < kRun; ++o) {
      const int py = by + y0 + o;
      if (px < W && py < H) {
        const long long p = base + (long long)py * W + px;
        const float m1 = mom[0][o], n1 = mom[1][o];
        const float mx = cx + m1, my = cy + n1;
        const float sxx = __fmaf_rn(-m1, m1, mom[2][o]), syy = __fmaf_rn(-n1, n1, mom[3][o]);
        const float sxy = __fmaf_rn(-m1, n1, mom[4][o]);
        const float A1 = 2.f * mx * my + kC1, A2 = 2.f * sxy + kC2;
        const float B1 = mx * mx + my * my + kC1, B2 = sxx + syy + kC2;
        const float D = B1 * B2;
        const float S = A1 * A2 / D;
        acc += 1.f - S;
        float* mp = maps + (long long)(5 * ch) * P + p;
        mp[0] = mx;
        mp[P] = my;
        mp[2 * P] = (2.f * my * A2 - S * 2.f * mx * B2) / D;  // dS/dmu_x, sigmas fixed
        mp[3 * P] = -S / B2;                                   // dS/dsigma_x^2
        mp[4 * P] = 2.f * A1 / D;                              // dS/dsigma_xy
      }
    }
  }
  block_partial(acc, (double)sv.scale[v], partials + b);
}

__global__ void __launch_bounds__(kSsimThreads) ssim_bwd_kernel(
    const float* __restrict__ image, const float* __restrict__ target, const SsimViews sv,
    const float* __restrict__ maps, long long P, float* __restrict__ dimg) {
  __shared__ float sm[3][5][kSsimS][kSsimS + 1];             // staged map terms
  __shared__ __align__(16) float sh[3][5][kSsimS][kSsimB];  // horizontal sums
  __shared__ float s_c[3][2];
  const int b = blockIdx.x;
  const int v = view_of_block(sv, b);
  const int lb = b - sv.block_off[v];
  const int W = sv.W[v], H = sv.H[v];
  const int bx = (lb % sv.BX[v]) * kSsimB, by = (lb / sv.BX[v]) * kSsimB;
  const long long base = sv.pix_off[v];
  // block constants: the image and target at the block's first pixel
  const long long p0 = base + (long long)by * W + bx;
  if (threadIdx.x < 3) {
    s_c[threadIdx.x][0] = image[3 * p0 + threadIdx.x];
    s_c[threadIdx.x][1] = target[3 * p0 + threadIdx.x];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kSsimS * kSsimS; i += kSsimThreads) {
    const int yy = by - kSsimR + i / kSsimS, xx = bx - kSsimR + i % kSsimS;
    const bool in = xx >= 0 && xx < W && yy >= 0 && yy < H;  // window centres in the image
    const long long q = base + (long long)yy * W + xx;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
      const float* mp = maps + (long long)(5 * ch) * P;
      float a = 0.f, bb = 0.f, e = 0.f, pm = 0.f, qm = 0.f;
      if (in) {
        const float mx = mp[q], my = mp[P + q];
        a = mp[2 * P + q];
        bb = mp[3 * P + q];
        e = mp[4 * P + q];
        pm = (mx - s_c[ch][0]) * bb;
        qm = (my - s_c[ch][1]) * e;
      }
      sm[ch][0][i / kSsimS][i % kSsimS] = a;
      sm[ch][1][i / kSsimS][i % kSsimS] = bb;
      sm[ch][2][i / kSsimS][i % kSsimS] = e;
      sm[ch][3][i / kSsimS][i % kSsimS] = pm;
      sm[ch][4][i / kSsimS][i % kSsimS] = qm;
    }
  }
  __syncthreads();
  for (int it = threadIdx.x; it < kHItems; it += kSsimThreads) {
    const int g = it % (kSsimB / kRun), r = (it / (kSsimB / kRun)) % kSsimS;
    const int ch = it / (kSsimS * (kSsimB / kRun));
    const int x0 = g * kRun;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      float row[kSpan];
#pragma unroll
      for (int j = 0; j < kSpan; ++j) row[j] = sm[ch][k][r][x0 + j];
      float h[kRun];
#pragma unroll
      for (int o = 0; o < kRun; ++o) {
        float t = 0.f;
#pragma unroll
        for (int i = 0; i < 2 * kSsimR + 1; ++i) t = __fmaf_rn(sv.win[i], row[o + i], t);
        h[o] = t;
      }
      *reinterpret_cast<float4*>(&sh[ch][k][r][x0]) = make_float4(h[0], h[1], h[2], h[3]);
    }
  }
  __syncthreads();
  if (threadIdx.x < kVItems) {
    const int c = threadIdx.x % kSsimB, q = (threadIdx.x / kSsimB) % (kSsimB / kRun);
    const int ch = threadIdx.x / (kSsimB * (kSsimB / kRun));
    const int y0 = q * kRun;
    float gsum[5][kRun];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      float col[kSpan];
#pragma unroll
      for (int j = 0; j < kSpan; ++j) col[j] = sh[ch][k][y0 + j][c];
#pragma unroll
      for (int o = 0; o < kRun; ++o) {
        float t = 0.f;
#pragma unroll
        for (int j = 0; j < 2 * kSsimR + 1; ++j) t = __fmaf_rn(sv.win[j], col[o + j], t);
        gsum[k][o] = t;
      }
    }
    const float cx = s_c[ch][0], cy = s_c[ch][1];
    const int px = bx + c;
#pragma unroll
    for (int o = 0; o < kRun; ++o) {
      const int py = by + y0 + o;
      if (px < W && py < H) {
        const long long p = base + (long long)py * W + px;
        const float xp = image[3 * p + ch], yp = target[3 * p + ch];
        const float grad = gsum[0][o] + 2.f * ((xp - cx) * gsum[1][o] - gsum[3][o]) +
                           (yp - cy) * gsum[2][o] - gsum[4][o];
        dimg[3 * p + ch] -= sv.scale[v] * grad;
      }
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
