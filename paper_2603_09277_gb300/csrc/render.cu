// render.cu -- per-tile front-to-back blending with the weight entropy
// (forward) and its reverse-order adjoint with Algorithm 1 fused in.
//
// One CTA of 256 threads owns one 16x16 tile, one thread per pixel.  The
// tile's list is streamed through shared memory in batches of 256 records
// (one gathered 16-byte-vector record per thread), and every thread walks the
// batch from shared memory (warp-broadcast reads).  The forward stops a CTA
// as soon as every pixel is done (__syncthreads_count over the batch).
//
// Forward, per pixel (Sec. 3 and Sec. 4.3):
//   e = log2(sigma g) = L2S - |F (x - mean)|^2 (base 2, opacity folded in,
//   F the square-root factor of the conic; the mean is rebased on the tile)
//   skip if e < log2(alpha_min); alpha = min(alpha_max, 2^e)
//   stop before blending if T (1 - alpha) < t_min
//   w = alpha T; C += w c; sum_wl += w log2 w; T *= 1 - alpha
//   H = -ln 2 (sum_wl + T log2 T)
// Backward, per pixel, from its last blended entry down (Sec. 4.4, Suppl. B-C):
//   T_i = T_{i+1} / (1 - alpha_i), w_i = alpha_i T_i
//   dL/dalpha_i = sum_ch g_ch (T_i c_i - S / (1 - alpha_i))
//               + gH ((-ln w_i - 1) T_i + R / (1 - alpha_i))
//   S += w_i c_i; R += (ln w_i + 1) w_i    (R starts at (ln T_N+1 + 1) T_N+1)
//   then dsigma = dalpha g, dd = dalpha alpha (unless clamped),
//   dconic = dd (-dx^2/2, -dx dy, -dy^2/2), dmean = dd conic (dx, dy).
// The 9 per-Gaussian values are summed over the warp with shuffles and added
// to grad2d with vector atomics by one lane.
//
// Launch forms: one CTA per tile (optionally in a given tile order), or a
// persistent grid whose CTAs claim tiles from a queue with one atomicAdd per
// tile (no CTA ever waits for another).
#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kThreads = kTilePix;  // 256
constexpr int kBatch = kThreads;

struct TileCoord {
  int view, px, py;
  bool inside;
  long long pix;   // global pixel index (valid when inside)
  float ox, oy;    // tile origin in pixels
  float rx, ry;    // pixel centre relative to the tile origin
};

__device__ __forceinline__ TileCoord tile_coord(const CamTable& ct, int tile) {
  TileCoord t;
  t.view = find_view_of_tile(ct, tile);
  const CamInfo& c = ct.c[t.view];
  int local = tile - c.tile_off;
  int tx = local % c.TX, ty = local / c.TX;
  t.px = tx * kTile + (threadIdx.x & (kTile - 1));
  t.py = ty * kTile + (threadIdx.x >> 4);
  t.inside = t.px < c.W && t.py < c.H;
  t.pix = c.pix_off + (long long)t.py * c.W + t.px;
  t.ox = (float)(tx * kTile);
  t.oy = (float)(ty * kTile);
  t.rx = (float)(threadIdx.x & (kTile - 1)) + 0.5f;
  t.ry = (float)(threadIdx.x >> 4) + 0.5f;
  return t;
}

struct FwdArgs {
  const void* recs;
  const unsigned* vals;
  const uint2* ranges;
  float* image;
  float* final_T;
  unsigned* last_idx;
  float* entropy;
  const unsigned* order;
  unsigned* counter;
  unsigned long long* stats;
};

template <int DT>
__device__ __forceinline__ void fwd_tile(const CamTable& ct, const RenderConsts& rc,
                                         const FwdArgs& a, int tile, unsigned long long& n_bl,
                                         unsigned long long& n_ev) {
  __shared__ float4 s0[kBatch];
  __shared__ float4 s1[kBatch];
  __shared__ float s2[kBatch];
  const int tid = threadIdx.x;
  TileCoord tc = tile_coord(ct, tile);
  const float pxf = tc.rx, pyf = tc.ry;
  const uint2 r = a.ranges[tile];
  float T = 1.f, cr = 0.f, cg = 0.f, cb = 0.f, swl = 0.f;
  unsigned last = 0;
  bool done = !tc.inside;
  unsigned nb = 0, ne = 0;
  for (unsigned base = r.x; base < r.y; base += kBatch) {
    if (__syncthreads_count(done) == kThreads) break;
    unsigned idx = base + tid;
    if (idx < r.y) {
      Splat s = load_record<DT>(a.recs, a.vals[idx]);
      const float2 m = tile_relative_mean(s, tc.ox, tc.oy);
      s0[tid] = make_float4(m.x, m.y, s.f11, s.f21);
      s1[tid] = make_float4(s.f22, s.L2S, s.R, s.G);
      s2[tid] = s.B;
    }
    __syncthreads();
    const int cnt = min((unsigned)kBatch, r.y - base);
    if (!done) {
      for (int k = 0; k < cnt; ++k) {
        const float4 g0 = s0[k];
        const float4 g1 = s1[k];
        const float dx = pxf - g0.x, dy = pyf - g0.y;
        float pp, qq;
        const float e = splat_exponent(g0.z, g0.w, g1.x, g1.y, dx, dy, pp, qq);
        ++ne;
        if (e < rc.log2_alpha_min) continue;
        const float alpha = fminf(rc.alpha_max, fast_exp2(e));
        const float test_T = T * (1.f - alpha);
        if (test_T < rc.t_min) {
          done = true;
          break;
        }
        const float w = alpha * T;
        cr = __fmaf_rn(w, g1.z, cr);
        cg = __fmaf_rn(w, g1.w, cg);
        cb = __fmaf_rn(w, s2[k], cb);
        swl = __fmaf_rn(w, fast_log2(w), swl);
        T = test_T;
        last = base - r.x + k + 1;
        ++nb;
      }
    }
  }
  if (tc.inside) {
    const long long p = tc.pix;
    a.image[3 * p] = cr;
    a.image[3 * p + 1] = cg;
    a.image[3 * p + 2] = cb;
    a.final_T[p] = T;
    a.last_idx[p] = last;
    if (a.entropy) a.entropy[p] = -kLn2 * (swl + T * fast_log2(T));
  }
  n_bl += nb;
  n_ev += ne;
  __syncthreads();  // shared staging is reused by the next tile
}

__device__ __forceinline__ void flush_stats(unsigned long long* stats, unsigned long long nb,
                                            unsigned long long ne) {
  if (!stats) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nb += __shfl_xor_sync(0xffffffffu, nb, o);
    ne += __shfl_xor_sync(0xffffffffu, ne, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(stats, nb);
    atomicAdd(stats + 1, ne);
  }
}

template <int DT>
__global__ void __launch_bounds__(kThreads) render_fwd_kernel(const CamTable ct,
                                                              const RenderConsts rc,
                                                              const FwdArgs a, int persistent) {
  unsigned long long nb = 0, ne = 0;
  if (persistent) {
    __shared__ unsigned s_t;
    for (;;) {
      if (threadIdx.x == 0) s_t = atomicAdd(a.counter, 1u);
      __syncthreads();
      const unsigned t = s_t;
      __syncthreads();
      if (t >= (unsigned)ct.total_tiles) break;
      fwd_tile<DT>(ct, rc, a, a.order ? (int)a.order[t] : (int)t, nb, ne);
    }
  } else {
    const int t = blockIdx.x;
    fwd_tile<DT>(ct, rc, a, a.order ? (int)a.order[t] : t, nb, ne);
  }
  flush_stats(a.stats, nb, ne);
}

// ---------------------------------------------------------------------------
// Backward
// ---------------------------------------------------------------------------
struct BwdArgs {
  const void* recs;
  const unsigned* vals;
  const uint2* ranges;
  const float* final_T;
  const unsigned* last_idx;
  const float* dL_dimage;
  const float* dL_dentropy;
  float* grad2d;  // [rows][12]
  const unsigned* order;
  unsigned* counter;
};

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

template <int DT>
__device__ __forceinline__ void bwd_tile(const CamTable& ct, const RenderConsts& rc,
                                         const BwdArgs& a, int tile) {
  __shared__ float4 s0[kBatch];
  __shared__ float4 s1[kBatch];
  __shared__ float2 s2[kBatch];
  __shared__ unsigned s_row[kBatch];
  __shared__ unsigned s_max;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  TileCoord tc = tile_coord(ct, tile);
  const float pxf = tc.rx, pyf = tc.ry;
  const uint2 r = a.ranges[tile];
  float T = 1.f, gr = 0.f, gg = 0.f, gb = 0.f, gH = 0.f;
  unsigned last = 0;
  if (tc.inside) {
    const long long p = tc.pix;
    T = a.final_T[p];
    last = a.last_idx[p];
    gr = a.dL_dimage[3 * p];
    gg = a.dL_dimage[3 * p + 1];
    gb = a.dL_dimage[3 * p + 2];
    if (a.dL_dentropy) gH = a.dL_dentropy[p];
  }
  if (tid == 0) s_max = 0u;
  __syncthreads();
  if (last) atomicMax(&s_max, last);
  __syncthreads();
  const unsigned maxlast = s_max;
  // colour accumulator S = sum_{k > i} w_k c_k and entropy accumulator R
  float Sr = 0.f, Sg = 0.f, Sb = 0.f;
  float Rent = (fast_log2(T) * kLn2 + 1.f) * T;
  for (unsigned end = maxlast; end > 0;) {
    const unsigned start = end > (unsigned)kBatch ? end - kBatch : 0u;
    const int cnt = (int)(end - start);
    __syncthreads();
    if (tid < cnt) {
      const unsigned row = a.vals[r.x + start + tid];
      Splat s = load_record<DT>(a.recs, row);
      const float2 m = tile_relative_mean(s, tc.ox, tc.oy);
      s0[tid] = make_float4(m.x, m.y, s.f11, s.f21);
      s1[tid] = make_float4(s.f22, s.L2S, s.R, s.G);
      s2[tid] = make_float2(s.B, s.sigma);
      s_row[tid] = row;
    }
    __syncthreads();
    for (int k = cnt - 1; k >= 0; --k) {
      const unsigned pos = start + (unsigned)k;  // 0-based list position
      float d_mx = 0.f, d_my = 0.f, d_a = 0.f, d_b = 0.f, d_c = 0.f, d_s = 0.f;
      float d_r = 0.f, d_g = 0.f, d_bl = 0.f;
      bool contrib = false;
      const float4 g0 = s0[k];
      const float4 g1 = s1[k];
      if (pos < last) {
        const float dx = pxf - g0.x, dy = pyf - g0.y;
        float pp, qq;
        const float e = splat_exponent(g0.z, g0.w, g1.x, g1.y, dx, dy, pp, qq);
        if (e >= rc.log2_alpha_min) {
          contrib = true;
          const float2 g2 = s2[k];
          const float araw = fast_exp2(e);
          const float alpha = fminf(rc.alpha_max, araw);
          const float om = 1.f - alpha;
          const float iom = 1.f / om;
          const float Ti = T * iom;
          const float w = alpha * Ti;
          const float lnw = fast_log2(w) * kLn2;
          float dA = gr * (Ti * g1.z - Sr * iom) + gg * (Ti * g1.w - Sg * iom) +
                     gb * (Ti * g2.x - Sb * iom);
          dA += gH * ((-lnw - 1.f) * Ti + Rent * iom);
          d_r = w * gr;
          d_g = w * gg;
          d_bl = w * gb;
          Sr = __fmaf_rn(w, g1.z, Sr);
          Sg = __fmaf_rn(w, g1.w, Sg);
          Sb = __fmaf_rn(w, g2.x, Sb);
          Rent = __fmaf_rn(lnw + 1.f, w, Rent);
          T = Ti;
          if (araw <= rc.alpha_max) {
            const float dd = dA * araw;
            d_s = dd / g2.y;  // dA * g with g = araw / sigma
            d_a = -0.5f * dd * dx * dx;
            d_b = -dd * dx * dy;
            d_c = -0.5f * dd * dy * dy;
            // d d / d mean = conic (dx, dy) = F^T (p, q) / (log2(e) / 2)
            const float k2 = 2.f * kLn2 * dd;
            d_mx = k2 * (g0.z * pp + g0.w * qq);
            d_my = k2 * (g1.x * qq);
          }
        }
      }
      if (__any_sync(0xffffffffu, contrib)) {
        d_mx = warp_sum(d_mx);
        d_my = warp_sum(d_my);
        d_a = warp_sum(d_a);
        d_b = warp_sum(d_b);
        d_c = warp_sum(d_c);
        d_s = warp_sum(d_s);
        d_r = warp_sum(d_r);
        d_g = warp_sum(d_g);
        d_bl = warp_sum(d_bl);
        if (lane == 0) {
          float4* G = reinterpret_cast<float4*>(a.grad2d + 12ll * s_row[k]);
          atomicAdd(G, make_float4(d_mx, d_my, d_a, d_b));
          atomicAdd(G + 1, make_float4(d_c, d_s, d_r, d_g));
          atomicAdd(reinterpret_cast<float*>(G + 2), d_bl);
        }
      }
    }
    end = start;
  }
  __syncthreads();
}

template <int DT>
__global__ void __launch_bounds__(kThreads) render_bwd_kernel(const CamTable ct,
                                                              const RenderConsts rc,
                                                              const BwdArgs a, int persistent) {
  if (persistent) {
    __shared__ unsigned s_t;
    for (;;) {
      if (threadIdx.x == 0) s_t = atomicAdd(a.counter, 1u);
      __syncthreads();
      const unsigned t = s_t;
      __syncthreads();
      if (t >= (unsigned)ct.total_tiles) break;
      bwd_tile<DT>(ct, rc, a, a.order ? (int)a.order[t] : (int)t);
    }
  } else {
    const int t = blockIdx.x;
    bwd_tile<DT>(ct, rc, a, a.order ? (int)a.order[t] : t);
  }
}

int record_event(void* ev, cudaStream_t st) {
  if (!ev) return GS_OK;
  GS_TRY_CUDA(cudaEventRecord(reinterpret_cast<cudaEvent_t>(ev), st));
  return GS_OK;
}

template <int DT>
int launch_fwd_t(const CamTable& ct, const RenderConsts& rc, const FwdArgs& a, int ctas,
                 const gs_launch* opt, cudaStream_t st) {
  int e = record_event(opt ? opt->ev_begin : nullptr, st);
  if (e != GS_OK) return e;
  if (ct.total_tiles > 0) {
    if (ctas > 0) {
      render_fwd_kernel<DT><<<ctas, kThreads, 0, st>>>(ct, rc, a, 1);
    } else {
      render_fwd_kernel<DT><<<ct.total_tiles, kThreads, 0, st>>>(ct, rc, a, 0);
    }
    count_launches(1);
  }
  e = record_event(opt ? opt->ev_end : nullptr, st);
  if (e != GS_OK) return e;
  return check_launch();
}

template <int DT>
int launch_bwd_t(const CamTable& ct, const RenderConsts& rc, const BwdArgs& a, int ctas,
                 const gs_launch* opt, cudaStream_t st) {
  int e = record_event(opt ? opt->ev_begin : nullptr, st);
  if (e != GS_OK) return e;
  if (ct.total_tiles > 0) {
    if (ctas > 0) {
      render_bwd_kernel<DT><<<ctas, kThreads, 0, st>>>(ct, rc, a, 1);
    } else {
      render_bwd_kernel<DT><<<ct.total_tiles, kThreads, 0, st>>>(ct, rc, a, 0);
    }
    count_launches(1);
  }
  e = record_event(opt ? opt->ev_end : nullptr, st);
  if (e != GS_OK) return e;
  return check_launch();
}

}  // namespace

int launch_render_fwd(const gs_proj* proj, const CamTable& ct, const gs_params* prm,
                      const unsigned* vals, const unsigned* ranges, float* image, float* final_T,
                      unsigned* last_idx, float* entropy, const gs_launch* opt, cudaStream_t st) {
  FwdArgs a;
  a.recs = proj->records;
  a.vals = vals;
  a.ranges = reinterpret_cast<const uint2*>(ranges);
  a.image = image;
  a.final_T = final_T;
  a.last_idx = last_idx;
  a.entropy = entropy;
  a.order = opt ? opt->tile_order : nullptr;
  a.counter = opt ? opt->work_counter : nullptr;
  a.stats = opt ? opt->stats : nullptr;
  int ctas = opt ? opt->ctas : 0;
  if (ctas > 0) GS_TRY_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(unsigned), st));
  RenderConsts rc = render_consts(prm);
  switch (prm->attr_dtype) {
    case GS_ATTR_F32: return launch_fwd_t<GS_ATTR_F32>(ct, rc, a, ctas, opt, st);
    case GS_ATTR_F16: return launch_fwd_t<GS_ATTR_F16>(ct, rc, a, ctas, opt, st);
    case GS_ATTR_BF16: return launch_fwd_t<GS_ATTR_BF16>(ct, rc, a, ctas, opt, st);
  }
  return GS_ERR_INVALID_ARG;
}

int launch_render_bwd(const gs_proj* proj, const CamTable& ct, const gs_params* prm,
                      const unsigned* vals, const unsigned* ranges, const float* final_T,
                      const unsigned* last_idx, const float* dL_dimage, const float* dL_dentropy,
                      float* grad2d, const gs_launch* opt, cudaStream_t st) {
  BwdArgs a;
  a.recs = proj->records;
  a.vals = vals;
  a.ranges = reinterpret_cast<const uint2*>(ranges);
  a.final_T = final_T;
  a.last_idx = last_idx;
  a.dL_dimage = dL_dimage;
  a.dL_dentropy = dL_dentropy;
  a.grad2d = grad2d;
  a.order = opt ? opt->tile_order : nullptr;
  a.counter = opt ? opt->work_counter : nullptr;
  int ctas = opt ? opt->ctas : 0;
  if (ctas > 0) GS_TRY_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(unsigned), st));
  RenderConsts rc = render_consts(prm);
  switch (prm->attr_dtype) {
    case GS_ATTR_F32: return launch_bwd_t<GS_ATTR_F32>(ct, rc, a, ctas, opt, st);
    case GS_ATTR_F16: return launch_bwd_t<GS_ATTR_F16>(ct, rc, a, ctas, opt, st);
    case GS_ATTR_BF16: return launch_bwd_t<GS_ATTR_BF16>(ct, rc, a, ctas, opt, st);
  }
  return GS_ERR_INVALID_ARG;
}

}  // namespace gs
