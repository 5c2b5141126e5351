// render.cu -- per-tile front-to-back blending with the weight entropy
// (forward) and its reverse-order adjoint with Algorithm 1 fused in.
//
// One CTA owns one tile of TS x TS pixels (TS = 16, or 8 as in the paper's
// runs).  A thread owns PPT (1, 2 or 4; 1 or 2 for 8x8 tiles) vertically
// adjacent pixels of one column, so a warp covers a TS x (32 / TS) PPT block
// and the column-dependent part of every exponent is shared by the thread's
// pixels.
// The tile's list is streamed through shared memory in batches of 256
// records (gathered with 16-byte vector loads) and every thread walks the
// batch from shared memory (warp-broadcast reads).  The forward stops a CTA
// as soon as every pixel is done (__syncthreads_count per batch).
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
//   (only g . S is needed, so it is carried instead of S: g . S += w_i g . c_i;
//   R and gH are carried in base-2 units, R / ln 2 and gH ln 2)
//   then with dd = dalpha alpha (where alpha is not clamped) and (dx, dy)
//   the pixel centre minus the 2D mean: dsigma = dd / sigma,
//   dconic = dd (-dx^2/2, -dx dy, -dy^2/2), dmean = dd conic (dx, dy).
//   Every one of these is linear in the moments dd (1, dx, dy, dx^2, dx dy,
//   dy^2), so the kernel sums the moments and the projection's adjoint
//   applies 1 / sigma, the conic and the signs once per Gaussian.
// The thread sums the 9 per-Gaussian values (6 moments, 3 colour weights)
// over its pixels.  When at most kDirectLanes lanes of the warp contribute,
// each of them adds its values to grad2d with three vector atomics;
// otherwise the warp sums them with a split-transpose shuffle reduction (12
// shuffles leave one of the 9 totals in each of 9 lane pairs) and 9 lanes
// add them with one atomic instruction.  (All 32 lanes adding to one address
// in one instruction serialise in L2: the threshold stays below 32.)
// With two pixels per thread both pixels go through packed FP32 (f32x2)
// arithmetic, in the forward as well.
//
// Launch forms: one CTA per tile (optionally in a given tile order), or a
// persistent grid whose CTAs claim tiles from a queue with one atomicAdd per
// tile (no CTA ever waits for another); 1, 2 or 4 pixels per thread; 256 or
// (F32 records, 16-pixel tiles) 128 list entries staged per batch.  The
// batch size changes only how the list is staged, never which entries a
// pixel meets or their order: the forward outputs do not depend on it.
#include "gs_internal.cuh"

namespace gs {
namespace {

// Records per shared-memory staging batch: a template argument B of the
// kernels, 256 or (F32 records, 16-pixel tiles) 128; at most 256 (a batch
// position is one byte in the per-warp entry lists).
constexpr int kMaxBatch = 256;
constexpr int kDirectLanes = 24;  // up to this many contributing lanes add directly
constexpr unsigned kFull = 0xffffffffu;
// A row coordinate this far from every mean makes the exponent -inf (f22 > 0),
// so a finished or outside pixel never passes the alpha_min test again.
constexpr float kFar = 1e30f;

template <int TS, int PPT>
struct TileGeom {
  static constexpr int kThreads = TS * TS / PPT;
  int view;
  long long pix0;   // global index of the thread's first pixel
  int W;            // view width (pixel stride of a row)
  float ox, oy;     // tile origin
  float rx;         // pixel-centre x relative to the tile origin
  float ry0;        // first pixel-centre y relative to the tile origin
  unsigned inside;  // bit k: pixel k lies in the image
  float xmax;       // largest pixel-centre x of the tile inside the image (relative)
  unsigned rows;    // bit r: tile row r lies in the image
};

template <int TS, int PPT>
__device__ __forceinline__ TileGeom<TS, PPT> tile_geom(const CamTable& ct, int tile) {
  TileGeom<TS, PPT> g;
  g.view = find_view_of_tile(ct, tile);
  const CamInfo& c = ct.c[g.view];
  const int local = tile - c.tile_off;
  const int tx = local % c.TX, ty = local / c.TX;
  const int lx = threadIdx.x & (TS - 1);
  const int ly0 = (threadIdx.x / TS) * PPT;
  const int px = tx * TS + lx, py0 = ty * TS + ly0;
  g.W = c.W;
  g.pix0 = c.pix_off + (long long)py0 * c.W + px;
  g.ox = (float)(tx * TS);
  g.oy = (float)(ty * TS);
  g.rx = (float)lx + 0.5f;
  g.ry0 = (float)ly0 + 0.5f;
  g.inside = 0u;
#pragma unroll
  for (int k = 0; k < PPT; ++k)
    if (px < c.W && py0 + k < c.H) g.inside |= 1u << k;
  g.xmax = (float)(min(TS, c.W - tx * TS) - 1) + 0.5f;
  const int nrow = min(TS, c.H - ty * TS);
  g.rows = (1u << nrow) - 1u;
  return g;
}

// Rows of the tile (bit r: pixel centres at tile-relative y = r + 0.5) in
// which some pixel centre with x in [0.5, xmax] may pass the alpha_min test.
// A pixel passes when e = L2S - p^2 - q^2 >= log2(alpha_min), that is when
// p^2 + q^2 <= rho2 = L2S - log2(alpha_min).  Along one row p^2 + q^2 is a
// convex quadratic in x; its least value over the segment is taken at the
// stationary point clamped to the segment.  The limit is widened by a bound
// on the FP32 rounding of this test and of the per-pixel exponent (32 times
// the first-order estimate), so a row left out holds no pixel the per-pixel
// test would blend, and skipping it leaves every output unchanged.
template <int TS>
__device__ __forceinline__ unsigned splat_rows(float mx, float my, float f11, float f21, float f22,
                                               float L2S, float log2_amin, float xmax,
                                               unsigned rows) {
  const float rho2 = L2S - log2_amin;
  if (!(rho2 >= 0.f)) return 0u;  // e <= L2S < log2(alpha_min) everywhere
  const float rho = sqrtf(rho2);
  const float x0 = 0.5f - mx, x1 = xmax - mx;
  const float X =
      (fabsf(f11) + fabsf(f21)) * ((float)TS + fabsf(mx)) + fabsf(f22) * ((float)TS + fabsf(my)) +
      rho;
  const float lim = rho2 + 0x1p-18f * (rho * X + rho2 + 8.f);
  const float a = __fmaf_rn(f11, f11, f21 * f21);
  const float k = -f21 * f22 / a;  // stationary x of row dy is k dy
  unsigned m = 0u;
#pragma unroll 4
  for (int r = 0; r < TS; ++r) {
    const float dy = ((float)r + 0.5f) - my;
    const float dx = fminf(fmaxf(k * dy, x0), x1);
    const float pv = f11 * dx;
    const float qv = __fmaf_rn(f21, dx, f22 * dy);
    if (__fmaf_rn(pv, pv, qv * qv) <= lim) m |= 1u << r;
  }
  return m & rows;
}

// Builds the warp's list of staged entries (ascending) whose rows mask meets
// the warp's rows; returns its length.
template <int TS, int PPT>
__device__ __forceinline__ int warp_entries(const unsigned short* s_rows, unsigned char* list,
                                            int cnt, int lane, int warp) {
  constexpr int kRows = (32 / TS) * PPT;  // tile rows of one warp
  constexpr unsigned kBand = (1u << kRows) - 1u;
  const unsigned band = kBand << (warp * kRows);
  const unsigned below = (1u << lane) - 1u;
  int n = 0;
  for (int c = 0; c < cnt; c += 32) {
    const int j = c + lane;
    const bool hit = j < cnt && (s_rows[j] & band);
    const unsigned b = __ballot_sync(kFull, hit);
    if (hit) list[n + __popc(b & below)] = (unsigned char)j;
    n += __popc(b);
  }
  __syncwarp();
  return n;
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
  unsigned long long rows, pixels;  // extents of the record and per-pixel arrays
  uint4* zero;                      // zeroed by the kernel's CTAs (optional)
  unsigned long long zero_n16;      // its size in 16-byte units
};

// A CTA's stripe of FwdArgs::zero, stored at the start of the forward with
// evict-first stores: the blending is bound by instruction issue and leaves
// the memory bandwidth mostly idle, so this costs a few issue slots where a
// separate zeroing kernel (even on a second stream: the forward's CTAs fill
// the register file, nothing runs beside them) added its whole duration.
__device__ __forceinline__ void zero_stripe(uint4* __restrict__ z, unsigned long long n16) {
  const unsigned long long per = (n16 + gridDim.x - 1) / gridDim.x;
  const unsigned long long b = (unsigned long long)blockIdx.x * per;
  const unsigned long long e = min(n16, b + per);
  for (unsigned long long i = b + threadIdx.x; i < e; i += blockDim.x)
    __stcs(z + i, make_uint4(0u, 0u, 0u, 0u));
}

// One list entry against a thread's two pixels (rows ry and ry + 1 of one
// column) in the forward, both through the same steps with packed FP32
// (f32x2); the exponent is the scalar path's value exactly (RN(q^2 - base)
// is -RN(base - q^2)).  A pixel that is not reached gets w = 0 (every sum
// unchanged, its T kept by a select); a pixel whose T (1 - alpha) would drop
// below t_min finishes: its live bit clears and its row moves to kFar.
// Returns the number of pixels blended.
__device__ __forceinline__ int fwd_pair(const RenderConsts& rc, const float4 g0, const float4 g1,
                                        const float cB, float rx, float2& ry2, float2& T2,
                                        float2& cr2, float2& cg2, float2& cb2, float2& swl2,
                                        unsigned& last0, unsigned& last1, unsigned& live,
                                        unsigned pos1, unsigned& stop0, unsigned& stop1) {
  const SplatColumn col = splat_column(g0.z, g0.w, g1.y, rx - g0.x);
  const float2 dy = __fadd2_rn(ry2, make_float2(-g0.y, -g0.y));
  const float2 qv = __ffma2_rn(make_float2(g1.x, g1.x), dy, make_float2(col.qx, col.qx));
  const float2 en = __ffma2_rn(qv, qv, make_float2(-col.base, -col.base));  // -e
  const bool p0 = !(-en.x < rc.log2_alpha_min), p1 = !(-en.y < rc.log2_alpha_min);
  if (!(p0 || p1)) return 0;
  const float2 al = make_float2(p0 ? fminf(rc.alpha_max, fast_exp2(-en.x)) : 0.f,
                                p1 ? fminf(rc.alpha_max, fast_exp2(-en.y)) : 0.f);
  const float2 tT = __fmul2_rn(T2, __fadd2_rn(make_float2(1.f, 1.f), make_float2(-al.x, -al.y)));
  const bool f0 = p0 && tT.x < rc.t_min, f1 = p1 && tT.y < rc.t_min;
  if (f0) {
    live &= ~1u;
    ry2.x = kFar;
    stop0 = pos1;
  }
  if (f1) {
    live &= ~2u;
    ry2.y = kFar;
    stop1 = pos1;
  }
  const bool b0 = p0 && !f0, b1 = p1 && !f1;
  const float2 w = __fmul2_rn(make_float2(b0 ? al.x : 0.f, b1 ? al.y : 0.f), T2);
  cr2 = __ffma2_rn(w, make_float2(g1.z, g1.z), cr2);
  cg2 = __ffma2_rn(w, make_float2(g1.w, g1.w), cg2);
  cb2 = __ffma2_rn(w, make_float2(cB, cB), cb2);
  swl2 = __ffma2_rn(
      w, make_float2(fast_log2(fmaxf(w.x, 1e-30f)), fast_log2(fmaxf(w.y, 1e-30f))), swl2);
  T2 = make_float2(b0 ? tT.x : T2.x, b1 ? tT.y : T2.y);
  if (b0) last0 = pos1;
  if (b1) last1 = pos1;
  return (int)b0 + (int)b1;
}

template <int DT, int TS, int PPT, int B, bool STATS>
__device__ __forceinline__ void fwd_tile(const CamTable& ct, const RenderConsts& rc,
                                         const FwdArgs& a, int tile, unsigned long long& n_bl,
                                         unsigned long long& n_ev) {
  constexpr int NT = TileGeom<TS, PPT>::kThreads;
  constexpr int NW = NT / 32;
  static_assert(NW >= 1, "a tile needs at least one full warp");
  static_assert(B % 32 == 0 && B <= kMaxBatch, "batch: a multiple of 32, at most 256");
  __shared__ float4 s0[B];
  __shared__ float4 s1[B];
  __shared__ float s2[B];
  __shared__ unsigned short s_rows[B];
  __shared__ unsigned char s_list[NW][B];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const TileGeom<TS, PPT> tg = tile_geom<TS, PPT>(ct, tile);
  const uint2 r = a.ranges[tile];
  float T[PPT], cr[PPT], cg[PPT], cb[PPT], swl[PPT];
  unsigned last[PPT];
  unsigned stop[PPT];         // entries the definition tests (statistics only)
  unsigned live = tg.inside;  // bit k: pixel k still walking
  float ry[PPT];              // pixel-centre y relative to the tile; kFar once finished
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    T[k] = 1.f;
    cr[k] = cg[k] = cb[k] = swl[k] = 0.f;
    last[k] = 0u;
    stop[k] = r.y - r.x;
    ry[k] = (live & (1u << k)) ? tg.ry0 + (float)k : kFar;
  }
  // two pixels per thread: the state as FP32 pairs (packed f32x2 arithmetic)
  float2 T2, cr2, cg2, cb2, swl2, ry2;
  if constexpr (PPT == 2) {
    T2 = make_float2(T[0], T[1]);
    cr2 = cg2 = cb2 = swl2 = make_float2(0.f, 0.f);
    ry2 = make_float2(ry[0], ry[1]);
  }
  unsigned nb = 0, ne = 0;
  for (unsigned base = r.x; base < r.y; base += B) {
    if (__syncthreads_count(live == 0u) == NT) break;
    for (int j = tid; j < B; j += NT) {
      const unsigned idx = base + j;
      if (idx < r.y) {
        unsigned row = a.vals[idx];
        if (!GS_IN_BOUNDS(row, a.rows, 101)) row = 0u;
        const Splat s = load_record<DT>(a.recs, row);
        const float2 m = tile_relative_mean(s, tg.ox, tg.oy);
        s0[j] = make_float4(m.x, m.y, s.f11, s.f21);
        s1[j] = make_float4(s.f22, s.L2S, s.R, s.G);
        s2[j] = s.B;
        s_rows[j] = (unsigned short)splat_rows<TS>(m.x, m.y, s.f11, s.f21, s.f22, s.L2S,
                                                   rc.log2_alpha_min, tg.xmax, tg.rows);
      }
    }
    __syncthreads();
    const int cnt = (int)min((unsigned)B, r.y - base);
    // only the entries that may reach a pixel of this warp's rows
    const int n = __any_sync(kFull, live != 0u)
                      ? warp_entries<TS, PPT>(s_rows, s_list[warp], cnt, lane, warp)
                      : 0;
    for (int i = 0; i < n && live; ++i) {
      const int k = s_list[warp][i];
      if constexpr (PPT == 2) {
        const int nbl = fwd_pair(rc, s0[k], s1[k], s2[k], tg.rx, ry2, T2, cr2, cg2, cb2, swl2,
                                 last[0], last[1], live, base - r.x + k + 1, stop[0], stop[1]);
        if (STATS) nb += nbl;
        continue;
      }
      const float4 g0 = s0[k];
      const float4 g1 = s1[k];
      const SplatColumn col = splat_column(g0.z, g0.w, g1.y, tg.rx - g0.x);
      float e[PPT];
      float emax = -INFINITY;
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        float qq;
        e[q] = splat_row(col, g1.x, ry[q] - g0.y, qq);
        emax = fmaxf(emax, e[q]);
      }
      if (emax < rc.log2_alpha_min) continue;  // no pixel of this thread is reached
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        if (e[q] < rc.log2_alpha_min) continue;
        const float alpha = fminf(rc.alpha_max, fast_exp2(e[q]));
        const float test_T = T[q] * (1.f - alpha);
        if (test_T < rc.t_min) {
          live &= ~(1u << q);
          ry[q] = kFar;  // finished pixels evaluate to e = -inf from here on
          if (STATS) stop[q] = base - r.x + k + 1;
          continue;
        }
        const float w = alpha * T[q];
        cr[q] = __fmaf_rn(w, g1.z, cr[q]);
        cg[q] = __fmaf_rn(w, g1.w, cg[q]);
        cb[q] = __fmaf_rn(w, s2[k], cb[q]);
        swl[q] = __fmaf_rn(w, fast_log2(w), swl[q]);
        T[q] = test_T;
        last[q] = base - r.x + k + 1;
        if (STATS) ++nb;
      }
    }
  }
  if constexpr (PPT == 2) {
    T[0] = T2.x;
    T[1] = T2.y;
    cr[0] = cr2.x;
    cr[1] = cr2.y;
    cg[0] = cg2.x;
    cg[1] = cg2.y;
    cb[0] = cb2.x;
    cb[1] = cb2.y;
    swl[0] = swl2.x;
    swl[1] = swl2.y;
  }
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    if (!(tg.inside & (1u << q))) continue;
    const long long p = tg.pix0 + (long long)q * tg.W;
    if (!GS_IN_BOUNDS(p, a.pixels, 102)) continue;
    a.image[3 * p] = cr[q];
    a.image[3 * p + 1] = cg[q];
    a.image[3 * p + 2] = cb[q];
    a.final_T[p] = T[q];
    a.last_idx[p] = last[q];
    if (a.entropy) a.entropy[p] = -kLn2 * (swl[q] + T[q] * fast_log2(T[q]));
    if (STATS) ne += stop[q];
  }
  if (STATS) {
    n_bl += nb;
    n_ev += ne;
  }
  __syncthreads();  // shared staging is reused by the next tile
}

__device__ __forceinline__ void flush_stats(unsigned long long* stats, unsigned long long nb,
                                            unsigned long long ne) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nb += __shfl_xor_sync(kFull, nb, o);
    ne += __shfl_xor_sync(kFull, ne, o);
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(stats, nb);
    atomicAdd(stats + 1, ne);
  }
}

template <int DT, int TS, int PPT, int B, bool STATS>
__global__ void __launch_bounds__(TS * TS / PPT) render_fwd_kernel(const CamTable ct,
                                                                    const RenderConsts rc,
                                                                    const FwdArgs a,
                                                                    int persistent) {
  unsigned long long nb = 0, ne = 0;
  if (a.zero) zero_stripe(a.zero, a.zero_n16);
  if (persistent) {
    __shared__ unsigned s_t;
    for (;;) {
      if (threadIdx.x == 0) s_t = atomicAdd(a.counter, 1u);
      __syncthreads();
      const unsigned t = s_t;
      __syncthreads();
      if (t >= (unsigned)ct.total_tiles) break;
      fwd_tile<DT, TS, PPT, B, STATS>(ct, rc, a, a.order ? (int)a.order[t] : (int)t, nb, ne);
    }
  } else {
    const int t = blockIdx.x;
    fwd_tile<DT, TS, PPT, B, STATS>(ct, rc, a, a.order ? (int)a.order[t] : t, nb, ne);
  }
  if (STATS) flush_stats(a.stats, nb, ne);
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
  float* grad2d;  // [rows][12]: sums dd (dx, dy, dx^2, dx dy, dy^2, 1), w (r, g, b), pad
  const unsigned* order;
  unsigned* counter;
  unsigned long long rows, pixels;  // extents of the record and per-pixel arrays
};

// Split-transpose warp sum of v[0..8]: at each butterfly level a lane keeps
// one part of its values and sends the other, so 5 + 3 + 2 + 1 + 1 shuffles
// leave the warp total of value slot(lane) in the lane; returns the slot
// (0..8) or -1 for lanes left without a distinct total.  Lane pairs (l, l^1)
// hold the same total.
__device__ __forceinline__ float warp_sum9(const float v[9], int lane, int& slot) {
  const bool b = lane & 16, c = lane & 8, d = lane & 4, e = lane & 2;
  float u[5];
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    const float hi = i < 4 ? v[5 + i] : 0.f;
    const float keep = b ? hi : v[i];
    const float send = b ? v[i] : hi;
    u[i] = keep + __shfl_xor_sync(kFull, send, 16);
  }
  float w[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float hi = i < 2 ? u[3 + i] : 0.f;
    const float keep = c ? hi : u[i];
    const float send = c ? u[i] : hi;
    w[i] = keep + __shfl_xor_sync(kFull, send, 8);
  }
  float x[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const float hi = i < 1 ? w[2] : 0.f;
    const float keep = d ? hi : w[i];
    const float send = d ? w[i] : hi;
    x[i] = keep + __shfl_xor_sync(kFull, send, 4);
  }
  float y = (e ? x[1] : x[0]) + __shfl_xor_sync(kFull, e ? x[0] : x[1], 2);
  y += __shfl_xor_sync(kFull, y, 1);
  // slot held by the lane group (b, c, d, e) = index 8b + 4c + 2d + e, as
  // 4-bit fields (0xF: no distinct total)
  constexpr unsigned long long kSlots = 0xFFF8F765FF43F210ull;
  const unsigned sel = (unsigned)((kSlots >> (4 * ((lane >> 1) & 15))) & 0xF);
  slot = (sel == 0xF || (lane & 1)) ? -1 : (int)sel;
  return y;
}

// One list entry against a thread's two pixels (rows ry and ry + 1 of one
// column), both through the same steps with packed FP32 (f32x2: one
// instruction for the pair).  A pixel that does not take part (the entry
// lies after its last blended one, or its alpha is below alpha_min) gets
// alpha = 0: its transmittance is kept by a select and every contribution
// is zero, and its L stays finite (w is floored at 1e-30 inside the log).
// The exponent is the scalar path's value exactly: RN(q^2 - base) is
// -RN(base - q^2).  Sets gsum to the pixel sums of the 6 moments and 3
// colour weights, which are exact zeros where neither pixel takes part
// (alpha = 0 makes w and dd zero; every other factor is finite), so a lane
// past its last blended entry needs no branch of its own.  Returns the
// warp's lanes where either pixel took part (gsum is left unset when there
// are none).
__device__ __forceinline__ unsigned bwd_pair(const RenderConsts& rc, const float4 g0, const float4 g1,
                                         const float cB, float rx, float2 ry2, unsigned pos,
                                         unsigned last0, unsigned last1, float2& T2,
                                         const float2 gr2, const float2 gg2, const float2 gb2,
                                         const float2 gH2, float2& gS2, float2& R2,
                                         float gsum[9]) {
  const float dx = rx - g0.x;
  const SplatColumn col = splat_column(g0.z, g0.w, g1.y, dx);
  const float2 dy = __fadd2_rn(ry2, make_float2(-g0.y, -g0.y));
  const float2 qv = __ffma2_rn(make_float2(g1.x, g1.x), dy, make_float2(col.qx, col.qx));
  const float2 en = __ffma2_rn(qv, qv, make_float2(-col.base, -col.base));  // -e
  const bool a0 = pos < last0 && !(-en.x < rc.log2_alpha_min);
  const bool a1 = pos < last1 && !(-en.y < rc.log2_alpha_min);
  const unsigned who = __ballot_sync(kFull, a0 || a1);
  if (!who) return 0u;  // (warp-uniform) no pixel of the warp takes part
  const float ar0 = a0 ? fast_exp2(-en.x) : 0.f;
  const float ar1 = a1 ? fast_exp2(-en.y) : 0.f;
  const float2 al = make_float2(fminf(rc.alpha_max, ar0), fminf(rc.alpha_max, ar1));
  const float2 om = __fadd2_rn(make_float2(1.f, 1.f), make_float2(-al.x, -al.y));
  const float2 iom = make_float2(fast_rcp(om.x), fast_rcp(om.y));
  const float2 Ti = __fmul2_rn(T2, iom);
  const float2 w = __fmul2_rn(al, Ti);
  const float2 L = __fadd2_rn(
      make_float2(fast_log2(fmaxf(w.x, 1e-30f)), fast_log2(fmaxf(w.y, 1e-30f))),
      make_float2(kLog2e, kLog2e));
  // colour part T_i gc - gS / (1 - alpha_i), entropy part gH (-L T_i + R / (1 - alpha_i))
  const float2 gc = __ffma2_rn(gb2, make_float2(cB, cB),
                               __ffma2_rn(gg2, make_float2(g1.w, g1.w),
                                          __fmul2_rn(gr2, make_float2(g1.z, g1.z))));
  const float2 sq = __fmul2_rn(gS2, iom);
  float2 dA = __ffma2_rn(Ti, gc, make_float2(-sq.x, -sq.y));
  const float2 ent = __ffma2_rn(make_float2(-L.x, -L.y), Ti, __fmul2_rn(R2, iom));
  dA = __ffma2_rn(gH2, ent, dA);
  const float2 c6 = __fmul2_rn(w, gr2), c7 = __fmul2_rn(w, gg2), c8 = __fmul2_rn(w, gb2);
  gS2 = __ffma2_rn(w, gc, gS2);
  R2 = __ffma2_rn(L, w, R2);
  T2 = make_float2(a0 ? Ti.x : T2.x, a1 ? Ti.y : T2.y);
  // dd = dalpha alpha where alpha is below its clamp, then the moments
  const float2 dd = __fmul2_rn(dA, make_float2(ar0 <= rc.alpha_max ? ar0 : 0.f,
                                               ar1 <= rc.alpha_max ? ar1 : 0.f));
  // the two pixels share the column offset dx: the dx-moments are dx times
  // the pixel sums of dd and dd dy
  const float2 ddy = __fmul2_rn(dd, dy);
  gsum[5] = dd.x + dd.y;
  gsum[1] = ddy.x + ddy.y;
  gsum[0] = dx * gsum[5];
  gsum[2] = dx * gsum[0];
  gsum[3] = dx * gsum[1];
  gsum[4] = __fmaf_rn(ddy.x, dy.x, ddy.y * dy.y);
  gsum[6] = c6.x + c6.y;
  gsum[7] = c7.x + c7.y;
  gsum[8] = c8.x + c8.y;
  return who;
}

template <int DT, int TS, int PPT, int B>
__device__ __forceinline__ void bwd_tile(const CamTable& ct, const RenderConsts& rc,
                                         const BwdArgs& a, int tile) {
  static_assert(B % 32 == 0 && B <= kMaxBatch, "batch: a multiple of 32, at most 256");
  __shared__ float4 s0[B];
  __shared__ float4 s1[B];
  __shared__ float s2[B];  // blue
  __shared__ unsigned s_row[B];
  __shared__ unsigned short s_rows[B];
  constexpr int NT = TileGeom<TS, PPT>::kThreads;
  constexpr int NW = NT / 32;
  static_assert(NW >= 1, "a tile needs at least one full warp");
  __shared__ unsigned char s_list[NW][B];
  __shared__ unsigned s_max;
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const TileGeom<TS, PPT> tg = tile_geom<TS, PPT>(ct, tile);
  const uint2 r = a.ranges[tile];
  // per pixel: T, dL/dC, dL/dH, gS = dL/dC . S (S = sum_{k>i} w_k c_k) and R
  float T[PPT], gr[PPT], gg[PPT], gb[PPT], gH[PPT], gS[PPT], Rent[PPT];
  unsigned last[PPT];
  unsigned mylast = 0;
#pragma unroll
  for (int q = 0; q < PPT; ++q) {
    T[q] = 1.f;
    gr[q] = gg[q] = gb[q] = gH[q] = 0.f;
    last[q] = 0u;
    if ((tg.inside & (1u << q)) && GS_IN_BOUNDS(tg.pix0 + (long long)q * tg.W, a.pixels, 112)) {
      const long long p = tg.pix0 + (long long)q * tg.W;
      T[q] = a.final_T[p];
      last[q] = a.last_idx[p];
      gr[q] = a.dL_dimage[3 * p];
      gg[q] = a.dL_dimage[3 * p + 1];
      gb[q] = a.dL_dimage[3 * p + 2];
      if (a.dL_dentropy) gH[q] = a.dL_dentropy[p];
    }
    gS[q] = 0.f;
    Rent[q] = (fast_log2(T[q]) + kLog2e) * T[q];
    gH[q] *= kLn2;
    mylast = max(mylast, last[q]);
  }
  // two pixels per thread: the state as FP32 pairs (packed f32x2 arithmetic)
  float2 T2, gr2, gg2, gb2, gH2, gS2, R2;
  if constexpr (PPT == 2) {
    T2 = make_float2(T[0], T[1]);
    gr2 = make_float2(gr[0], gr[1]);
    gg2 = make_float2(gg[0], gg[1]);
    gb2 = make_float2(gb[0], gb[1]);
    gH2 = make_float2(gH[0], gH[1]);
    gS2 = make_float2(0.f, 0.f);
    R2 = make_float2(Rent[0], Rent[1]);
  }
  const float2 ry2 = make_float2(tg.ry0, tg.ry0 + 1.f);
  if (tid == 0) s_max = 0u;
  __syncthreads();
  if (mylast) atomicMax(&s_max, mylast);
  __syncthreads();
  const unsigned maxlast = s_max;
  for (unsigned end = maxlast; end > 0;) {
    const unsigned start = end > (unsigned)B ? end - B : 0u;
    const int cnt = (int)(end - start);
    __syncthreads();
    for (int j = tid; j < cnt; j += NT) {
      unsigned row = a.vals[r.x + start + j];
      if (!GS_IN_BOUNDS(row, a.rows, 111)) row = 0u;
      const Splat s = load_record<DT>(a.recs, row);
      const float2 m = tile_relative_mean(s, tg.ox, tg.oy);
      s0[j] = make_float4(m.x, m.y, s.f11, s.f21);
      s1[j] = make_float4(s.f22, s.L2S, s.R, s.G);
      s2[j] = s.B;
      s_row[j] = row;
      s_rows[j] = (unsigned short)splat_rows<TS>(m.x, m.y, s.f11, s.f21, s.f22, s.L2S,
                                                 rc.log2_alpha_min, tg.xmax, tg.rows);
    }
    __syncthreads();
    // only the entries that may reach a pixel of this warp's rows, last first
    const int n = __any_sync(kFull, mylast > start)
                      ? warp_entries<TS, PPT>(s_rows, s_list[warp], cnt, lane, warp)
                      : 0;
    for (int i = n - 1; i >= 0; --i) {
      const int k = s_list[warp][i];
      const unsigned pos = start + (unsigned)k;  // 0-based list position
      const bool any_here = pos < mylast;
      if (!__any_sync(kFull, any_here)) continue;
      float gsum[9];
      bool contrib = false;
      unsigned who = 0u;
      if constexpr (PPT == 2) {
        // every lane (one past its last blended entry takes no part and adds zeros)
        who = bwd_pair(rc, s0[k], s1[k], s2[k], tg.rx, ry2, pos, last[0], last[1], T2, gr2, gg2,
                       gb2, gH2, gS2, R2, gsum);
        contrib = (who >> lane) & 1u;
      } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) gsum[i] = 0.f;
      }
      if (PPT != 2 && any_here) {
        const float4 g0 = s0[k];
        const float4 g1 = s1[k];
        const float cB = s2[k];
        const float dx = tg.rx - g0.x;
        const SplatColumn col = splat_column(g0.z, g0.w, g1.y, dx);
#pragma unroll
        for (int q = 0; q < PPT; ++q) {
          if (pos >= last[q]) continue;
          const float dy = tg.ry0 + (float)q - g0.y;
          float qq;
          const float e = splat_row(col, g1.x, dy, qq);
          if (e < rc.log2_alpha_min) continue;
          contrib = true;
          const float araw = fast_exp2(e);
          const float alpha = fminf(rc.alpha_max, araw);
          const float iom = fast_rcp(1.f - alpha);
          const float Ti = T[q] * iom;
          const float w = alpha * Ti;
          const float L = fast_log2(w) + kLog2e;
          // colour part: dL/dC . (T_i c_i - S / (1 - alpha_i)) = T_i gc - gS / (1 - alpha_i)
          const float gc = __fmaf_rn(gb[q], cB, __fmaf_rn(gg[q], g1.w, gr[q] * g1.z));
          float dA = __fmaf_rn(Ti, gc, -gS[q] * iom);
          dA = __fmaf_rn(gH[q], __fmaf_rn(-L, Ti, Rent[q] * iom), dA);
          gsum[6] += w * gr[q];
          gsum[7] += w * gg[q];
          gsum[8] += w * gb[q];
          gS[q] = __fmaf_rn(w, gc, gS[q]);  // S += w c  =>  dL/dC . S += w gc
          Rent[q] = __fmaf_rn(L, w, Rent[q]);
          T[q] = Ti;
          if (araw <= rc.alpha_max) {
            const float dd = dA * araw;
            const float ddx = dd * dx, ddy = dd * dy;
            gsum[0] += ddx;
            gsum[1] += ddy;
            gsum[2] = __fmaf_rn(ddx, dx, gsum[2]);
            gsum[3] = __fmaf_rn(ddx, dy, gsum[3]);
            gsum[4] = __fmaf_rn(ddy, dy, gsum[4]);
            gsum[5] += dd;
          }
        }
      }
      if constexpr (PPT != 2) who = __ballot_sync(kFull, contrib);
      if (who) {
        float* G = a.grad2d + 12ll * s_row[k];
        if (__popc(who) <= kDirectLanes) {
          // few contributing lanes: each adds its own values (three vector
          // atomics) instead of the 12-shuffle warp reduction
          if (contrib) {
            atomicAdd(reinterpret_cast<float4*>(G), make_float4(gsum[0], gsum[1], gsum[2], gsum[3]));
            atomicAdd(reinterpret_cast<float4*>(G) + 1,
                      make_float4(gsum[4], gsum[5], gsum[6], gsum[7]));
            atomicAdd(G + 8, gsum[8]);
          }
        } else {
          int slot;
          const float tot = warp_sum9(gsum, lane, slot);
          if (slot >= 0) atomicAdd(G + slot, tot);
        }
      }
    }
    end = start;
  }
  __syncthreads();
}

template <int DT, int TS, int PPT, int B>
__global__ void __launch_bounds__(TS * TS / PPT, (TS == 16 && PPT != 4) ? 4 * PPT : 1)
    render_bwd_kernel(const CamTable ct,
                                                                    const RenderConsts rc,
                                                                    const BwdArgs a,
                                                                    int persistent) {
  if (persistent) {
    __shared__ unsigned s_t;
    for (;;) {
      if (threadIdx.x == 0) s_t = atomicAdd(a.counter, 1u);
      __syncthreads();
      const unsigned t = s_t;
      __syncthreads();
      if (t >= (unsigned)ct.total_tiles) break;
      bwd_tile<DT, TS, PPT, B>(ct, rc, a, a.order ? (int)a.order[t] : (int)t);
    }
  } else {
    const int t = blockIdx.x;
    bwd_tile<DT, TS, PPT, B>(ct, rc, a, a.order ? (int)a.order[t] : t);
  }
}

int record_event(void* ev, cudaStream_t st) {
  if (!ev) return GS_OK;
  GS_TRY_CUDA(cudaEventRecord(reinterpret_cast<cudaEvent_t>(ev), st));
  return GS_OK;
}

template <int DT, int TS, int PPT, int B>
void launch_fwd_b(const CamTable& ct, const RenderConsts& rc, const FwdArgs& a, int ctas,
                  cudaStream_t st) {
  const int grid = ctas > 0 ? ctas : ct.total_tiles;
  const int pers = ctas > 0 ? 1 : 0;
  if (a.stats)
    render_fwd_kernel<DT, TS, PPT, B, true><<<grid, TS * TS / PPT, 0, st>>>(ct, rc, a, pers);
  else
    render_fwd_kernel<DT, TS, PPT, B, false><<<grid, TS * TS / PPT, 0, st>>>(ct, rc, a, pers);
}

template <int DT, int TS, int PPT, int B>
void launch_bwd_b(const CamTable& ct, const RenderConsts& rc, const BwdArgs& a, int ctas,
                  cudaStream_t st) {
  const int grid = ctas > 0 ? ctas : ct.total_tiles;
  render_bwd_kernel<DT, TS, PPT, B><<<grid, TS * TS / PPT, 0, st>>>(ct, rc, a, ctas > 0 ? 1 : 0);
}

// The 128-record batch exists for F32 records on 16-pixel tiles only (the
// host rejects it elsewhere); every other form stages 256 records.
template <int DT, int TS, int PPT>
void launch_fwd_ppt(const CamTable& ct, const RenderConsts& rc, const FwdArgs& a, int ctas,
                    int batch, cudaStream_t st) {
  if constexpr (DT == GS_ATTR_F32 && TS == 16) {
    if (batch == 128) return launch_fwd_b<DT, TS, PPT, 128>(ct, rc, a, ctas, st);
  }
  launch_fwd_b<DT, TS, PPT, kMaxBatch>(ct, rc, a, ctas, st);
}

template <int DT, int TS, int PPT>
void launch_bwd_ppt(const CamTable& ct, const RenderConsts& rc, const BwdArgs& a, int ctas,
                    int batch, cudaStream_t st) {
  if constexpr (DT == GS_ATTR_F32 && TS == 16) {
    if (batch == 128) return launch_bwd_b<DT, TS, PPT, 128>(ct, rc, a, ctas, st);
  }
  launch_bwd_b<DT, TS, PPT, kMaxBatch>(ct, rc, a, ctas, st);
}

template <int DT>
int launch_fwd_t(const CamTable& ct, const RenderConsts& rc, const FwdArgs& a, int ctas,
                 const gs_launch* opt, cudaStream_t st) {
  int e = record_event(opt ? opt->ev_begin : nullptr, st);
  if (e != GS_OK) return e;
  const int ppt = (opt && opt->pixels_per_thread) ? opt->pixels_per_thread : 2;
  const int batch = (opt && opt->batch) ? opt->batch : kMaxBatch;
  if (ct.total_tiles > 0) {
    if (ct.tile == 8) {  // 8x8 tiles: 1 or 2 px per thread (a CTA is at least one warp)
      if (ppt == 1) launch_fwd_ppt<DT, 8, 1>(ct, rc, a, ctas, batch, st);
      else launch_fwd_ppt<DT, 8, 2>(ct, rc, a, ctas, batch, st);
    } else {
      if (ppt == 1) launch_fwd_ppt<DT, 16, 1>(ct, rc, a, ctas, batch, st);
      else if (ppt == 4) launch_fwd_ppt<DT, 16, 4>(ct, rc, a, ctas, batch, st);
      else launch_fwd_ppt<DT, 16, 2>(ct, rc, a, ctas, batch, st);
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
  const int ppt = (opt && opt->pixels_per_thread) ? opt->pixels_per_thread : 2;
  const int batch = (opt && opt->batch) ? opt->batch : kMaxBatch;
  if (ct.total_tiles > 0) {
    if (ct.tile == 8) {
      if (ppt == 1) launch_bwd_ppt<DT, 8, 1>(ct, rc, a, ctas, batch, st);
      else launch_bwd_ppt<DT, 8, 2>(ct, rc, a, ctas, batch, st);
    } else {
      if (ppt == 1) launch_bwd_ppt<DT, 16, 1>(ct, rc, a, ctas, batch, st);
      else if (ppt == 4) launch_bwd_ppt<DT, 16, 4>(ct, rc, a, ctas, batch, st);
      else launch_bwd_ppt<DT, 16, 2>(ct, rc, a, ctas, batch, st);
    }
    count_launches(1);
  }
  e = record_event(opt ? opt->ev_end : nullptr, st);
  if (e != GS_OK) return e;
  return check_launch();
}

}  // namespace

GS_BOUNDS_READER(bounds_status_render)

int launch_render_fwd(const gs_proj* proj, long long rows, const CamTable& ct,
                      const gs_params* prm, const unsigned* vals, const unsigned* ranges,
                      float* image, float* final_T, unsigned* last_idx, float* entropy,
                      const gs_launch* opt, cudaStream_t st) {
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
  a.rows = (unsigned long long)rows;
  a.pixels = (unsigned long long)(ct.c[ct.V - 1].pix_off + (long long)ct.c[ct.V - 1].W * ct.c[ct.V - 1].H);
  // memory to zero beside the blending: the kernel's CTAs take the 16-byte
  // aligned whole units, a memset the ragged ends
  a.zero = nullptr;
  a.zero_n16 = 0;
  if (opt && opt->zero_beside && opt->zero_bytes > 0) {
    const uintptr_t z0 = reinterpret_cast<uintptr_t>(opt->zero_beside);
    const uintptr_t z1 = z0 + (uintptr_t)opt->zero_bytes;
    const uintptr_t a0 = (z0 + 15) & ~uintptr_t(15), a1 = z1 & ~uintptr_t(15);
    if (a1 > a0) {
      a.zero = reinterpret_cast<uint4*>(a0);
      a.zero_n16 = (unsigned long long)((a1 - a0) / 16);
      if (a0 > z0) GS_TRY_CUDA(cudaMemsetAsync(opt->zero_beside, 0, a0 - z0, st));
      if (z1 > a1) GS_TRY_CUDA(cudaMemsetAsync(reinterpret_cast<void*>(a1), 0, z1 - a1, st));
    } else {
      GS_TRY_CUDA(cudaMemsetAsync(opt->zero_beside, 0, (size_t)opt->zero_bytes, st));
    }
  }
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

int launch_render_bwd(const gs_proj* proj, long long rows, const CamTable& ct,
                      const gs_params* prm, const unsigned* vals, const unsigned* ranges,
                      const float* final_T, const unsigned* last_idx, const float* dL_dimage,
                      const float* dL_dentropy, float* grad2d, const gs_launch* opt,
                      cudaStream_t st) {
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
  a.rows = (unsigned long long)rows;
  a.pixels = (unsigned long long)(ct.c[ct.V - 1].pix_off + (long long)ct.c[ct.V - 1].W * ct.c[ct.V - 1].H);
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
