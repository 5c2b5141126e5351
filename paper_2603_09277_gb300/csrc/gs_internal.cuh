// gs_internal.cuh -- types and device helpers shared by the libgs CUDA
// translation units (preprocess, binning, render, loss/api).  Not part of the
// public ABI (include/gs.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "gs.h"

namespace gs {

constexpr int kTile = GS_TILE;               // 16x16 pixel tiles
constexpr int kTilePix = kTile * kTile;      // 256 pixels per tile
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// Per-view constants, passed by value in kernel parameters (<= 64 views).
struct CamInfo {
  float R[9];        // world -> camera rotation, row-major
  float t[3];        // world -> camera translation
  float fx, fy, cx, cy;
  float cp[3];       // camera centre in world space
  float limx, limy;  // clamp of x/z, y/z in the EWA Jacobian
  int W, H, TX, TY;
  int tile_off;      // first global tile id of this view
  long long pix_off; // first pixel of this view in per-pixel arrays
};

struct CamTable {
  int V;
  int total_tiles;
  CamInfo c[GS_MAX_VIEWS];
};

// Threshold constants in the forms the kernels test them.
struct RenderConsts {
  float alpha_max;
  float alpha_min;
  float log2_alpha_min;  // entries with exponent (base 2) below this are skipped
  float t_min;
};

// ---------------------------------------------------------------------------
// Render record: what the blending loop needs of one (view, Gaussian) row.
// The exponent is kept in base 2 with the opacity folded in:
//   e = A2 dx^2 + B2 dx dy + C2 dy^2 + L2S,   alpha = 2^e,
//   A2 = -a/2 log2(e), B2 = -b log2(e), C2 = -c/2 log2(e), L2S = log2(sigma),
// where (a, b, c) is the conic and dx, dy = pixel - mean2d.
// ---------------------------------------------------------------------------
struct __align__(16) RecF32 {  // 48 bytes
  float4 r0;  // mx, my, A2, B2
  float4 r1;  // C2, L2S, R, G
  float4 r2;  // B, sigma, 0, 0
};
struct __align__(16) RecH16 {  // 32 bytes: mean in FP32, the rest in 16-bit
  float2 m;           // mx, my
  uint32_t ab;        // A2, B2
  uint32_t cl;        // C2, L2S
  uint32_t rg;        // R, G
  uint32_t bs;        // B, sigma
  uint32_t pad0, pad1;
};

// The unpacked record staged in shared memory (FP32 in every variant).
struct Splat {
  float mx, my, A2, B2;
  float C2, L2S, R, G;
  float B, sigma;
};

template <int DT>
struct Half2Of;
template <>
struct Half2Of<GS_ATTR_F16> {
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ float2 unpack(uint32_t u) {
    __half2 h = *reinterpret_cast<__half2*>(&u);
    return __half22float2(h);
  }
};
template <>
struct Half2Of<GS_ATTR_BF16> {
  static __device__ __forceinline__ uint32_t pack(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ float2 unpack(uint32_t u) {
    __nv_bfloat162 h = *reinterpret_cast<__nv_bfloat162*>(&u);
    return __bfloat1622float2(h);
  }
};

template <int DT>
__device__ __forceinline__ void store_record(void* recs, long long row, const Splat& s) {
  if constexpr (DT == GS_ATTR_F32) {
    RecF32* r = reinterpret_cast<RecF32*>(recs) + row;
    r->r0 = make_float4(s.mx, s.my, s.A2, s.B2);
    r->r1 = make_float4(s.C2, s.L2S, s.R, s.G);
    r->r2 = make_float4(s.B, s.sigma, 0.f, 0.f);
  } else {
    RecH16 h;
    h.m = make_float2(s.mx, s.my);
    h.ab = Half2Of<DT>::pack(s.A2, s.B2);
    h.cl = Half2Of<DT>::pack(s.C2, s.L2S);
    h.rg = Half2Of<DT>::pack(s.R, s.G);
    h.bs = Half2Of<DT>::pack(s.B, s.sigma);
    h.pad0 = h.pad1 = 0u;
    uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<RecH16*>(recs) + row);
    const uint4* src = reinterpret_cast<const uint4*>(&h);
    dst[0] = src[0];
    dst[1] = src[1];
  }
}

template <int DT>
__device__ __forceinline__ Splat load_record(const void* recs, unsigned row) {
  Splat s;
  if constexpr (DT == GS_ATTR_F32) {
    const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const RecF32*>(recs) + row);
    float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    s.mx = a.x; s.my = a.y; s.A2 = a.z; s.B2 = a.w;
    s.C2 = b.x; s.L2S = b.y; s.R = b.z; s.G = b.w;
    s.B = c.x; s.sigma = c.y;
  } else {
    const uint4* p = reinterpret_cast<const uint4*>(reinterpret_cast<const RecH16*>(recs) + row);
    uint4 a = __ldg(p), b = __ldg(p + 1);
    s.mx = __uint_as_float(a.x); s.my = __uint_as_float(a.y);
    float2 ab = Half2Of<DT>::unpack(a.z), cl = Half2Of<DT>::unpack(a.w);
    float2 rg = Half2Of<DT>::unpack(b.x), bs = Half2Of<DT>::unpack(b.y);
    s.A2 = ab.x; s.B2 = ab.y; s.C2 = cl.x; s.L2S = cl.y;
    s.R = rg.x; s.G = rg.y; s.B = bs.x; s.sigma = bs.y;
  }
  return s;
}

// Base-2 exponent of alpha at pixel offset (dx, dy).  The forward and the
// backward kernels both call this, with explicit roundings, so that they take
// identical skip/stop decisions.
__device__ __forceinline__ float splat_exponent(float A2, float B2, float C2, float L2S, float dx,
                                                float dy) {
  float t = __fmaf_rn(B2, dy, __fmul_rn(A2, dx));   // A2 dx + B2 dy
  float e = __fmaf_rn(__fmul_rn(C2, dy), dy, L2S);   // C2 dy^2 + L2S
  return __fmaf_rn(dx, t, e);
}

__device__ __forceinline__ float fast_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float fast_log2(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ int find_view_of_tile(const CamTable& ct, int tile) {
  int v = 0;
  while (v + 1 < ct.V && tile >= ct.c[v + 1].tile_off) ++v;
  return v;
}

__device__ __forceinline__ int find_view_of_pixel(const CamTable& ct, long long pix) {
  int v = 0;
  while (v + 1 < ct.V && pix >= ct.c[v + 1].pix_off) ++v;
  return v;
}

}  // namespace gs

// ---------------------------------------------------------------------------
// Host-side helpers shared by the translation units (defined in api.cu).
// ---------------------------------------------------------------------------
namespace gs {
int set_cuda_error(cudaError_t e);
void count_launches(int n);
int check_launch();
bool build_cam_table(const gs_camera* cams, int V, const gs_params* prm, CamTable* ct);
RenderConsts render_consts(const gs_params* prm);
}  // namespace gs

#define GS_TRY_CUDA(expr)                               \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) return gs::set_cuda_error(_e); \
  } while (0)
