// gs_internal.cuh -- types and device helpers shared by the libgs CUDA
// translation units (preprocess, binning, render, loss/api).  Not part of the
// public ABI (include/gs.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <stdio.h>

#include "gs.h"

namespace gs {

// ---------------------------------------------------------------------------
// Bounds-checked debug build (compiled with -DGS_DEBUG_BOUNDS): a checked
// access tests its index against the extent of its buffer; a failing test
// records the check's id in the translation unit's device status word (the
// first failure wins) and the access is skipped.  No assert and no trap, so
// the context stays usable; gs_debug_bounds_status reads and clears the
// words.  In the normal build GS_IN_BOUNDS is `true` and costs nothing.
// ---------------------------------------------------------------------------
#ifdef GS_DEBUG_BOUNDS
static __device__ unsigned g_bounds_status;
__device__ __forceinline__ bool gs_in_bounds(unsigned long long i, unsigned long long n,
                                             unsigned id) {
  if (i < n) return true;
  atomicCAS(&g_bounds_status, 0u, id);
  return false;
}
#define GS_IN_BOUNDS(i, n, id) \
  ::gs::gs_in_bounds((unsigned long long)(i), (unsigned long long)(n), (unsigned)(id))
#define GS_BOUNDS_READER(name)                                                      \
  int name(unsigned* out, bool clear) {                                             \
    cudaError_t e = cudaMemcpyFromSymbol(out, g_bounds_status, sizeof(unsigned));   \
    if (e == cudaSuccess && clear) {                                                \
      const unsigned z = 0u;                                                        \
      e = cudaMemcpyToSymbol(g_bounds_status, &z, sizeof(unsigned));                \
    }                                                                               \
    return e == cudaSuccess ? GS_OK : set_cuda_error(e);                            \
  }
#else
#define GS_IN_BOUNDS(i, n, id) true
#define GS_BOUNDS_READER(name) \
  int name(unsigned* out, bool) {  \
    *out = 0u;                     \
    return GS_ERR_UNSUPPORTED;     \
  }
#endif

constexpr int kTile = GS_TILE;               // default tile side (16 px; 8 also supported)
constexpr int kSuperTile = 8;                // binning groups 8x8 tiles into a super-tile
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
  int STX, STY;      // super-tiles (kSuperTile x kSuperTile tiles) per row / column
  int st_off;        // first global super-tile id of this view
  int tile_off;      // first global tile id of this view
  long long pix_off; // first pixel of this view in per-pixel arrays
};

struct CamTable {
  int V;
  int tile;  // tile side in pixels (16 or 8)
  int total_tiles;
  int total_st;  // super-tiles over all views
  CamInfo c[GS_MAX_VIEWS];
};

// gs_proj.rect8 carries the rects when every view is at most 255 tiles per
// side (the projection writes it and the list construction reads it under
// this same rule).
inline bool rect8_fits(const CamTable& ct) {
  for (int v = 0; v < ct.V; ++v)
    if (ct.c[v].TX > 255 || ct.c[v].TY > 255) return false;
  return true;
}

// Threshold constants in the forms the kernels test them.
struct RenderConsts {
  float alpha_max;
  float alpha_min;
  float log2_alpha_min;  // entries with exponent (base 2) below this are skipped
  float t_min;
};

// ---------------------------------------------------------------------------
// Render record: what the blending loop needs of one (view, Gaussian) row.
// The exponent is kept in base 2 with the opacity folded in and the inverse
// covariance in square-root form:
//   p = f11 dx,  q = f21 dx + f22 dy,   e = L2S - p^2 - q^2,   alpha = 2^e,
// with F = [[f11, 0], [f21, f22]] = sqrt(log2(e)/2) L^-1, L the Cholesky
// factor of the 2D covariance (so F^T F = log2(e)/2 conic), L2S = log2(sigma)
// and (dx, dy) = pixel - mean2d.  The 2D mean is stored as an integer part
// (hx, hy) and a fraction (lx, ly); blending kernels rebase it on the tile.
// ---------------------------------------------------------------------------
struct __align__(16) RecF32 {  // 48 bytes
  float4 r0;  // hx, hy, lx, ly
  float4 r1;  // f11, f21, f22, L2S
  float4 r2;  // R, G, B, sigma
};
struct __align__(16) RecH16 {  // 32 bytes: mean in FP32, the rest in 16-bit
  float4 m;           // hx, hy, lx, ly
  uint32_t f1;        // f11, f21
  uint32_t f2;        // f22, L2S
  uint32_t rg;        // R, G
  uint32_t bs;        // B, sigma
};

// The unpacked record.
struct Splat {
  float hx, hy, lx, ly;
  float f11, f21, f22, L2S;
  float R, G, B, sigma;
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
    r->r0 = make_float4(s.hx, s.hy, s.lx, s.ly);
    r->r1 = make_float4(s.f11, s.f21, s.f22, s.L2S);
    r->r2 = make_float4(s.R, s.G, s.B, s.sigma);
  } else {
    RecH16* r = reinterpret_cast<RecH16*>(recs) + row;
    r->m = make_float4(s.hx, s.hy, s.lx, s.ly);
    uint4 q;
    q.x = Half2Of<DT>::pack(s.f11, s.f21);
    q.y = Half2Of<DT>::pack(s.f22, s.L2S);
    q.z = Half2Of<DT>::pack(s.R, s.G);
    q.w = Half2Of<DT>::pack(s.B, s.sigma);
    *reinterpret_cast<uint4*>(&r->f1) = q;
  }
}

template <int DT>
__device__ __forceinline__ Splat load_record(const void* recs, unsigned row) {
  Splat s;
  if constexpr (DT == GS_ATTR_F32) {
    const float4* p = reinterpret_cast<const float4*>(reinterpret_cast<const RecF32*>(recs) + row);
    float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    s.hx = a.x; s.hy = a.y; s.lx = a.z; s.ly = a.w;
    s.f11 = b.x; s.f21 = b.y; s.f22 = b.z; s.L2S = b.w;
    s.R = c.x; s.G = c.y; s.B = c.z; s.sigma = c.w;
  } else {
    const uint4* p = reinterpret_cast<const uint4*>(reinterpret_cast<const RecH16*>(recs) + row);
    uint4 a = __ldg(p), b = __ldg(p + 1);
    s.hx = __uint_as_float(a.x); s.hy = __uint_as_float(a.y);
    s.lx = __uint_as_float(a.z); s.ly = __uint_as_float(a.w);
    float2 f1 = Half2Of<DT>::unpack(b.x), f2 = Half2Of<DT>::unpack(b.y);
    float2 rg = Half2Of<DT>::unpack(b.z), bs = Half2Of<DT>::unpack(b.w);
    s.f11 = f1.x; s.f21 = f1.y; s.f22 = f2.x; s.L2S = f2.y;
    s.R = rg.x; s.G = rg.y; s.B = bs.x; s.sigma = bs.y;
  }
  return s;
}

// Mean relative to a tile origin (ox, oy): the integer parts subtract
// exactly, so the result is accurate to the rounding of a small number.
__device__ __forceinline__ float2 tile_relative_mean(const Splat& s, float ox, float oy) {
  return make_float2(__fadd_rn(__fsub_rn(s.hx, ox), s.lx), __fadd_rn(__fsub_rn(s.hy, oy), s.ly));
}

// Base-2 exponent of alpha at the tile-relative pixel offset (dx, dy):
//   p = f11 dx, q = f22 dy + f21 dx, e = (L2S - p^2) - q^2.
// The column part (p, f21 dx, L2S - p^2) is shared by the pixels of one
// column.  The forward and the backward kernels both evaluate it with these
// explicit roundings, so that they take identical skip/stop decisions.
struct SplatColumn {
  float p, qx, base;
};

__device__ __forceinline__ SplatColumn splat_column(float f11, float f21, float L2S, float dx) {
  SplatColumn c;
  c.p = __fmul_rn(f11, dx);
  c.qx = __fmul_rn(f21, dx);
  c.base = __fmaf_rn(-c.p, c.p, L2S);
  return c;
}

__device__ __forceinline__ float splat_row(const SplatColumn& c, float f22, float dy, float& q) {
  q = __fmaf_rn(f22, dy, c.qx);
  return __fmaf_rn(-q, q, c.base);
}

__device__ __forceinline__ float fast_exp2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ float fast_rcp(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
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
int set_error_text_and_status(const char* msg, int status);
void count_launches(int n);
int check_launch();
// tile: the tile side (0 means 16); fov_clamp comes from prm (1.3 if NULL).
bool build_cam_table(const gs_camera* cams, int V, const gs_params* prm, int tile, CamTable* ct);
RenderConsts render_consts(const gs_params* prm);
// The calling thread's events of a stage (gs_stage_events), recorded on
// `st` before / after the stage's kernel when set.
int stage_event(int stage, bool end, cudaStream_t st);
}  // namespace gs

#define GS_TRY_CUDA(expr)                               \
  do {                                                  \
    cudaError_t _e = (expr);                            \
    if (_e != cudaSuccess) return gs::set_cuda_error(_e); \
  } while (0)
