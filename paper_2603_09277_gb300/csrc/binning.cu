// binning.cu -- per-tile Gaussian lists (Sec. 3: each pixel's list of the
// Gaussians that cover it, sorted by depth).
//
// The lists are the (tile, depth, id)-ordered pairs of every visible
// (view, Gaussian) row with every tile of its rect.  Instead of sorting all
// P pairs, the sort works on rows and on row x super-tile items (a
// super-tile is 8x8 tiles), and the pairs are only ever written once, into
// their final slots:
//   1. compact the visible rows (scan of a visibility flag);
//   2. stable LSD radix sort of the visible rows by FP32 depth bits, on the
//      bits that vary over the visible rows (up to 9-bit digits: 3 passes
//      for a range of up to 27 bits; ties keep row order = Gaussian id order);
//   3. gather every row's rect in depth order (16-bit packed); block scans
//      give the pair count P and each block's first super-tile item (count
//      Q <= P);
//   4. duplicate: each block of rows scans its rows' item offsets and writes
//      (super-tile, row) for the super-tiles each rect meets, in depth order
//      (4 consecutive items per thread, owners by binary search);
//   5. stable radix sort of the items by super-tile id (one pass for up to
//      512 super-tiles), so every super-tile holds its rows in depth order;
//   6. per segment of 1024 rows of a super-tile: each row's rect within the
//      super-tile and per-tile counts; scans over segments and over all
//      tiles give every tile's list start (the ranges);
//   7. expansion: each segment writes its rows into the lists of the tiles
//      they cover, ranked by warp ballots, which keeps the depth order.
// The result is exactly the order of a 64-bit (tile << 32 | depth) key sort
// with ties by Gaussian id.
//
// All kernels read their element counts from device memory and use grids
// sized from host-known upper bounds (blocks beyond the actual counts leave
// at once), so the whole sequence can be captured in a CUDA graph (no host
// synchronisation needed).  None of them waits on another block: where a
// single-block scan follows a kernel, the kernel's last block to finish runs
// it (each block counts its arrival after a __threadfence).
#include <cuda.h>

#include <algorithm>
#include <mutex>

#include <atomic>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kScanThreads = 256;
// Scan blocks: ITEMS rows per thread (4 or 16, chosen from the row count at
// launch); the workspace is sized for the smaller blocks (the most blocks).
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;  // 1024 rows per block

// ----------------------------------------------------------------------------
// Block-wide exclusive scan helpers (256 threads).
// ----------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long warp_incl_scan(unsigned long long x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

// Returns the exclusive prefix of x over the block; *total receives the block
// total in every thread.
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long x,
                                                              unsigned long long* total) {
  __shared__ unsigned long long s_w[kScanThreads / 32 + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long inc = warp_incl_scan(x);
  if (lane == 31) s_w[w] = inc;
  __syncthreads();
  if (w == 0) {
    unsigned long long t = lane < kScanThreads / 32 ? s_w[lane] : 0ull;
    unsigned long long ti = warp_incl_scan(t);
    if (lane < kScanThreads / 32) s_w[lane] = ti - t;
    if (lane == 31) s_w[kScanThreads / 32] = ti;
  }
  __syncthreads();
  unsigned long long r = s_w[w] + inc - x;
  *total = s_w[kScanThreads / 32];
  __syncthreads();
  return r;
}

// The block's total of x (256 threads), in every thread.
__device__ __forceinline__ unsigned long long block_sum(unsigned long long x) {
  __shared__ unsigned long long s_ws[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if (lane == 0) s_ws[w] = x;
  __syncthreads();
  unsigned long long t = 0ull;
#pragma unroll
  for (int k = 0; k < kScanThreads / 32; ++k) t += s_ws[k];
  __syncthreads();  // s_ws is read by every thread before a later call reuses it
  return t;
}

// A CTA's arrival at the end of a kernel whose last CTA goes on to a step
// over every CTA's results (a scan of the block sums, say), in place of a
// separate single-CTA launch.  Each CTA makes its results visible
// (__threadfence) before it counts itself, so the CTA that counts last sees
// all of them; it reads them through L2 (__ldcg).  No CTA waits for another.
// The counter is zeroed with the pipeline's counters before the launch.
// Returns true in every thread of the last CTA.
__device__ __forceinline__ bool last_block_arrives(unsigned long long* counter,
                                                   unsigned long long expected) {
  __shared__ int s_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(counter, 1ull) == expected - 1ull ? 1 : 0;
  __syncthreads();
  const bool last = s_last != 0;
  if (last) __threadfence();
  return last;
}

__device__ __forceinline__ long long scan_blocks_dev(unsigned long long* block_sums, int nblocks);

// Exclusive scan of the block sums in one block (in place); returns
// the grand total.  Each warp takes a contiguous chunk of the sums: its total
// (a lane's loads in flight together), one scan of the warp totals, then the
// chunk again with the warp's running offset -- no block-wide barrier per
// round of 256 sums (cfg3-sized inputs have ~6,000 blocks).
__device__ __forceinline__ long long scan_blocks_dev(unsigned long long* block_sums, int nblocks) {
  constexpr int NW = kScanThreads / 32;
  __shared__ unsigned long long s_wt[NW + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int per = (nblocks + NW - 1) / NW;
  const int b0 = min(nblocks, w * per), b1 = min(nblocks, b0 + per);
  unsigned long long tot = 0ull;
#pragma unroll 4
  for (int i = b0 + lane; i < b1; i += 32) tot += __ldcg(block_sums + i);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  if (lane == 0) s_wt[w] = tot;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long run = 0ull;
    for (int k = 0; k < NW; ++k) {
      const unsigned long long x = s_wt[k];
      s_wt[k] = run;
      run += x;
    }
    s_wt[NW] = run;
  }
  __syncthreads();
  unsigned long long carry = s_wt[w];
  const long long total = (long long)s_wt[NW];
#pragma unroll 4
  for (int b = b0; b < b1; b += 32) {  // (warp-uniform)
    const int i = b + lane;
    const unsigned long long x = i < b1 ? __ldcg(block_sums + i) : 0ull;
    const unsigned long long incl = warp_incl_scan(x);
    if (i < b1) block_sums[i] = carry + incl - x;
    carry += __shfl_sync(0xffffffffu, incl, 31);
  }
  __syncthreads();  // s_wt is read by every thread before a later call reuses it
  return total;
}


// Exclusive scans of the super-tile counts (sums_q) and the pair counts
// (sums_p) over the blocks, then the capacity check: P, Q, the reported
// count, the status and the counts later stages use (0 on overflow).
struct CountsOut {
  unsigned long long* sums_q;
  unsigned long long* sums_p;
  long long capacity;
  long long *Q, *P, *q_eff, *p_eff, *num_pairs_dev;
  int* status;
};

__device__ __forceinline__ void scan_counts_check_dev(const CountsOut& o, int nblocks);

__global__ void __launch_bounds__(kScanThreads) scan_counts_check_kernel(const CountsOut o,
                                                                         int nblocks) {
  scan_counts_check_dev(o, nblocks);
}

__device__ __forceinline__ void scan_counts_check_dev(const CountsOut& o, int nblocks) {
  unsigned long long* sums_q = o.sums_q;
  unsigned long long* sums_p = o.sums_p;
  const long long capacity = o.capacity;
  long long *Q = o.Q, *P = o.P, *q_eff = o.q_eff, *p_eff = o.p_eff;
  long long* num_pairs_dev = o.num_pairs_dev;
  int* status = o.status;
  const long long q = scan_blocks_dev(sums_q, nblocks);
  const long long pp = scan_blocks_dev(sums_p, nblocks);
  if (threadIdx.x == 0) {
    const bool over = pp > capacity;
    *Q = q;
    *P = pp;
    *num_pairs_dev = pp;
    *status = over ? GS_ERR_CAPACITY : GS_OK;
    *p_eff = over ? 0 : pp;  // on overflow every later stage sees zero pairs
    *q_eff = over ? 0 : q;   // (Q <= P: a super-pair holds at least one pair)
  }
}


// ----------------------------------------------------------------------------
// Per visible row (depth order): its tile rect clamped to the view, the
// number of pairs it makes (rect area) and the number of super-tiles its
// rect meets.  Every later stage derives counts from this same clamped rect,
// so the pair and super-tile counts agree everywhere.
// ----------------------------------------------------------------------------
static_assert(kSuperTile == 8, "super-tile masks hold 8x8 tiles");

__device__ __forceinline__ int4 view_rect(const int* __restrict__ rect, unsigned row, int N,
                                          const CamTable& ct) {
  int4 r = reinterpret_cast<const int4*>(rect)[row];
  const CamInfo& c = ct.c[row / (unsigned)N];
  r.x = max(r.x, 0);
  r.y = max(r.y, 0);
  r.z = min(r.z, c.TX);
  r.w = min(r.w, c.TY);
  if (r.z <= r.x || r.w <= r.y) r = make_int4(0, 0, 0, 0);
  return r;
}

// Super-tile span [x0, x1) x [y0, y1) of a non-empty tile rect.
__device__ __forceinline__ int4 st_span(const int4 r) {
  return make_int4(r.x >> 3, r.y >> 3, ((r.z - 1) >> 3) + 1, ((r.w - 1) >> 3) + 1);
}

__device__ __forceinline__ unsigned st_count(const int4 r) {
  if (r.z <= r.x) return 0u;
  const int4 q = st_span(r);
  return (unsigned)((q.z - q.x) * (q.w - q.y));
}

// A clamped tile rect packed in 16-bit fields (x0 | y0 << 16, x1 | y1 << 16);
// views are at most 65535 tiles wide and high.
__device__ __forceinline__ uint2 pack_rect(const int4 r) {
  return make_uint2((unsigned)r.x | ((unsigned)r.y << 16), (unsigned)r.z | ((unsigned)r.w << 16));
}
__device__ __forceinline__ int4 unpack_rect(const uint2 p) {
  return make_int4((int)(p.x & 0xffffu), (int)(p.x >> 16), (int)(p.y & 0xffffu), (int)(p.y >> 16));
}

// The projection's 8-bit packed rect (gs_proj.rect8: x0 | y0 << 8 | x1 << 16 |
// y1 << 24, views of at most 255 tiles per side): the depth-ordered gather
// reads 4 bytes from an array a quarter the size of the int4 rects, most of
// which stays in L2 (a random 16-byte gather from the int4 rects fetches
// several times its size from DRAM).
__device__ __forceinline__ int4 unpack_rect8(unsigned p) {
  return make_int4((int)(p & 0xffu), (int)((p >> 8) & 0xffu), (int)((p >> 16) & 0xffu),
                   (int)(p >> 24));
}

__device__ __forceinline__ int radix_result(const unsigned* range, int bits);

// The depth-sorted rows: the buffer the sort left them in follows from the
// device-side key range (the number of passes it ran).
struct SortedRows {
  const unsigned* buf0;
  const unsigned* buf1;
  const unsigned* range;
  __device__ __forceinline__ const unsigned* get() const {
    return radix_result(range, 32) ? buf1 : buf0;
  }
};

// Gathers the clamped rect of every depth-ordered row (so later stages read
// them in order) and forms per-block sums of the super-tile counts and of
// the pair counts.
// The last CTA to finish scans both sums over the blocks and runs the
// capacity check (scan_counts_check_dev).
template <int ITEMS>
__global__ void __launch_bounds__(kScanThreads) rows_gather_kernel(
    const SortedRows sorted, const long long* __restrict__ n_dev,
    const int* __restrict__ rect, const unsigned* __restrict__ rect8, int N, const CamTable ct,
    uint2* __restrict__ rect_sorted, unsigned long long* __restrict__ arrive,
    const CountsOut co) {
  unsigned long long* sums_q = co.sums_q;
  unsigned long long* sums_p = co.sums_p;
  const unsigned* __restrict__ rows = sorted.get();
  const long long n = *n_dev;
  const long long base = (long long)blockIdx.x * (kScanThreads * ITEMS);
  if (base >= n) {  // (the whole CTA) no rows: zero sums
    if (threadIdx.x == 0) {
      sums_q[blockIdx.x] = 0ull;
      sums_p[blockIdx.x] = 0ull;
    }
    if (last_block_arrives(arrive, gridDim.x)) scan_counts_check_dev(co, (int)gridDim.x);
    return;
  }
  unsigned long long q = 0, pp = 0;
  // groups of kGather rows: their ids, then their rect gathers in flight
  // before any use (more per group would cost occupancy on large inputs)
  constexpr int kGather = 4;
  static_assert(ITEMS % kGather == 0, "whole groups");
#pragma unroll 1
  for (int k0 = 0; k0 < ITEMS; k0 += kGather) {
    unsigned row[kGather];
#pragma unroll
    for (int k = 0; k < kGather; ++k) {
      const long long i = base + (long long)(k0 + k) * kScanThreads + threadIdx.x;
      row[k] = i < n ? __ldcs(rows + i) : 0xffffffffu;  // streamed: evict first
    }
    int4 rr[kGather];
    if (rect8) {  // (uniform)
      unsigned p8[kGather];
#pragma unroll
      for (int k = 0; k < kGather; ++k)
        p8[k] = row[k] != 0xffffffffu && GS_IN_BOUNDS(row[k], (long long)N * ct.V, 205)
                    ? rect8[row[k]] : 0u;
#pragma unroll
      for (int k = 0; k < kGather; ++k) rr[k] = unpack_rect8(p8[k]);
    } else {
#pragma unroll
      for (int k = 0; k < kGather; ++k)
        rr[k] = row[k] != 0xffffffffu && GS_IN_BOUNDS(row[k], (long long)N * ct.V, 204)
                    ? view_rect(rect, row[k], N, ct) : make_int4(0, 0, 0, 0);
    }
#pragma unroll
    for (int k = 0; k < kGather; ++k) {
      const long long i = base + (long long)(k0 + k) * kScanThreads + threadIdx.x;
      if (i < n) {
        const int4 r = rr[k];
        __stcs(rect_sorted + i, pack_rect(r));  // streamed: keeps rect8 in L2
        q += st_count(r);
        pp += (unsigned long long)((r.z - r.x) * (r.w - r.y));
      }
    }
  }
  const unsigned long long tq = block_sum(q), tp = block_sum(pp);
  if (threadIdx.x == 0) {
    sums_q[blockIdx.x] = tq;
    sums_p[blockIdx.x] = tp;
  }
  if (last_block_arrives(arrive, gridDim.x)) scan_counts_check_dev(co, (int)gridDim.x);
}

// ----------------------------------------------------------------------------
// Stable LSD radix sort of (u32 key, u32 value) pairs, up to 8-bit digits,
// reduce-then-scan with a fixed grid.  Each block owns a contiguous chunk of
// whole 2048-item tiles; n is read from device memory.
//
// The depth sort reads the rows themselves in its first pass (RadixRows):
// the visible rows' depth bits with their row ids, the culled rows dropped,
// so no separate compaction runs.  That pass's upsweep folds in the visible
// rows' key range (smallest and largest depth bits); the later passes sort
// digits of (key - min) on the range's significant bits, their number and
// width following from the range on the device (radix_plan).  The kernels of
// passes beyond the plan return at once, so the launch sequence, and a graph
// of it, is fixed.  The result is in buffer (passes mod 2).
// ----------------------------------------------------------------------------
constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixIpt = 8;                                // items per thread per tile
constexpr int kRadixTile = kRadixThreads * kRadixIpt;       // 2048
constexpr int kRadixMaxBits = 8;
constexpr int kRadixBins = 1 << kRadixMaxBits;              // 256
constexpr int kRadixMaxPasses = (32 + kRadixMaxBits - 1) / kRadixMaxBits;  // 4
static_assert(kRadixThreads == kRadixBins, "the scatter's threads own one digit each");

struct RadixPlan {
  unsigned kmin;  // subtracted from every key
  int passes;
  int d0;         // digit width of the first pass
  int dbits;      // digit width of the later passes
};

// bits: significant bits of (key - kmin), in digits of equal width.
__host__ __device__ __forceinline__ RadixPlan radix_plan_bits(unsigned kmin, int bits) {
  RadixPlan p;
  p.kmin = kmin;
  p.passes = (bits + kRadixMaxBits - 1) / kRadixMaxBits;
  p.dbits = p.passes ? (bits + p.passes - 1) / p.passes : 0;
  p.d0 = p.dbits;
  return p;
}

// range (device, nullable): [0] = ~(smallest key), [1] = largest key, both
// folded in with atomicMax from zero (no key: range[0] = range[1] = 0, an
// empty range).  Without a range every one of `bits` bits is sorted.
//
// With a range the first pass reads the rows themselves and runs before the
// range is known (its upsweep folds the range in): its digit is the low byte
// of the key.  The smallest key is therefore rounded down to a multiple of
// 256, which leaves the low byte of (key - kmin) equal to that of the key;
// the later passes take the remaining significant bits of (key - kmin) in
// digits of equal width.  There is always at least the first pass.
__device__ __forceinline__ RadixPlan radix_plan(const unsigned* __restrict__ range, int bits) {
  if (!range) return radix_plan_bits(0u, bits);
  RadixPlan p;
  p.kmin = 0u;
  p.passes = 1;
  p.d0 = kRadixMaxBits;
  p.dbits = kRadixMaxBits;
  const unsigned kmin = ~__ldcg(range), kmax = __ldcg(range + 1);
  if (kmax > kmin) {
    p.kmin = kmin & ~(unsigned)(kRadixBins - 1);
    const int b = 32 - __clz(kmax - p.kmin);
    if (b > p.d0) {
      const int rest = (b - p.d0 + kRadixMaxBits - 1) / kRadixMaxBits;
      p.passes = 1 + rest;
      p.dbits = (b - p.d0 + rest - 1) / rest;
    }
  }
  return p;
}

// Bit offset of a pass's digit in (key - kmin), and its mask.
__device__ __forceinline__ int radix_shift(const RadixPlan& p, int pass) {
  return pass == 0 ? 0 : p.d0 + (pass - 1) * p.dbits;
}
__device__ __forceinline__ unsigned radix_mask(const RadixPlan& p, int pass) {
  return (1u << (pass == 0 ? p.d0 : p.dbits)) - 1u;
}
__device__ __forceinline__ unsigned radix_digit(unsigned key, const RadixPlan& p, int shift,
                                                unsigned mask) {
  return ((key - p.kmin) >> shift) & mask;
}

// Rows as the first pass's input (the depth sort): the key of row j is the
// bits of depth[j], its value j, and only the rows with tiles_touched[j] > 0
// take part (the visible rows: depth > near_z > 0, so the bits order like
// the values).  The pass writes the visible rows' count to *n_vis.
struct RadixRows {
  const float* depth;
  const unsigned* tiles_touched;
  long long n;     // rows
  long long* n_vis;
};

// Arguments of one pass.
struct RadixPass {
  const unsigned* keys_in;
  const unsigned* vals_in;
  unsigned* keys_out;
  unsigned* vals_out;
  const long long* n_dev;  // item count (the later passes with rows)
  const unsigned* range;   // device key range or nullptr
  int bits;                // significant bits without a range
  int pass;                // pass index
  unsigned* hist;          // [256][grid] per-CTA digit counts, then their scan
  unsigned* digit_tot;     // [256] items per digit
  int keys_last;           // write the keys in the last pass too
  RadixRows rows;          // rows.depth set: the first pass reads the rows
  __device__ __forceinline__ bool from_rows() const { return pass == 0 && rows.depth; }
  __device__ __forceinline__ long long count() const { return from_rows() ? rows.n : *n_dev; }
};

__device__ __forceinline__ long long radix_chunk(long long n, int nblocks) {
  long long per = (n + nblocks - 1) / nblocks;
  return (per + kRadixTile - 1) / kRadixTile * kRadixTile;
}

// CTAs of a pass that own items: the grid is sized for the bound on the
// item count, so with few items (a small visible set) most CTAs own none;
// they leave at once and the histogram scan covers only the active ones.
__device__ __forceinline__ int radix_active(long long n, int nblocks) {
  const long long chunk = radix_chunk(n, nblocks);
  return chunk > 0 ? (int)min((long long)nblocks, (n + chunk - 1) / chunk) : 0;
}

// Item j of a pass: key, value and whether it takes part.
__device__ __forceinline__ void radix_load(const RadixPass& a, long long j, long long end,
                                           unsigned& k, unsigned& v, bool& in) {
  if (a.from_rows()) {
    const unsigned t = j < end ? a.rows.tiles_touched[j] : 0u;
    k = j < end ? __float_as_uint(a.rows.depth[j]) : 0u;
    in = t > 0u;
    v = (unsigned)j;
  } else {
    in = j < end;
    k = in ? a.keys_in[j] : 0u;
    v = in ? a.vals_in[j] : 0u;
  }
}

__global__ void __launch_bounds__(kRadixThreads) radix_upsweep_kernel(const RadixPass a) {
  // the first pass over rows folds the key range in, so it cannot read the
  // plan: its digit is the low byte of the key
  const bool rows = a.from_rows();
  RadixPlan pl;
  if (rows) {
    pl.kmin = 0u;
    pl.passes = 1;
    pl.d0 = pl.dbits = kRadixMaxBits;
  } else {
    pl = radix_plan(a.range, a.bits);
    if (a.pass >= pl.passes) return;  // (the whole grid)
  }
  const int shift = radix_shift(pl, a.pass);
  const unsigned mask = radix_mask(pl, a.pass);
  unsigned* __restrict__ hist = a.hist;  // [256][nblocks]
  __shared__ unsigned s_h[kRadixWarps][kRadixBins];
  __shared__ unsigned s_kmin[kRadixWarps], s_kmax[kRadixWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long n = a.count();
  if ((int)blockIdx.x >= radix_active(n, gridDim.x)) return;  // (the whole CTA)
  const long long chunk = radix_chunk(n, gridDim.x);
  const long long b0 = (long long)blockIdx.x * chunk;
  const long long b1 = min(n, b0 + chunk);
  // kRadixIpt loads in flight per thread; the first tile's are requested
  // before the histogram is cleared
  unsigned kk[kRadixIpt], unused;
  bool in[kRadixIpt];
#pragma unroll
  for (int i = 0; i < kRadixIpt; ++i)
    radix_load(a, b0 + i * kRadixThreads + threadIdx.x, b1, kk[i], unused, in[i]);
  for (int i = threadIdx.x; i < kRadixWarps * kRadixBins; i += kRadixThreads)
    (&s_h[0][0])[i] = 0u;
  __syncthreads();
  unsigned kmin = 0xffffffffu, kmax = 0u;  // (rows) range of the keys taking part
  for (long long t0 = b0; t0 < b1; t0 += kRadixTile) {
    if (t0 != b0) {
#pragma unroll
      for (int i = 0; i < kRadixIpt; ++i)
        radix_load(a, t0 + i * kRadixThreads + threadIdx.x, b1, kk[i], unused, in[i]);
    }
#pragma unroll
    for (int i = 0; i < kRadixIpt; ++i) {
      if (in[i]) {
        atomicAdd(&s_h[w][radix_digit(kk[i], pl, shift, mask)], 1u);
        if (rows) {
          kmin = min(kmin, kk[i]);
          kmax = max(kmax, kk[i]);
        }
      }
    }
  }
  if (rows) {
    kmin = __reduce_min_sync(0xffffffffu, kmin);
    kmax = __reduce_max_sync(0xffffffffu, kmax);
    if (lane == 0) {
      s_kmin[w] = kmin;
      s_kmax[w] = kmax;
    }
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadixBins; d += kRadixThreads) {
    unsigned s = 0;
    for (int k = 0; k < kRadixWarps; ++k) s += s_h[k][d];
    hist[(long long)d * gridDim.x + blockIdx.x] = s;
  }
  if (rows && threadIdx.x == 0) {
    for (int q = 1; q < kRadixWarps; ++q) {
      kmin = min(kmin, s_kmin[q]);
      kmax = max(kmax, s_kmax[q]);
    }
    if (kmin <= kmax) {  // (folded in from zero: range[0] holds the complement)
      atomicMax(const_cast<unsigned*>(a.range), ~kmin);
      atomicMax(const_cast<unsigned*>(a.range) + 1, kmax);
    }
  }
}

// Per-digit exclusive scan over the blocks: block d scans hist[d][0..Ga) in
// place (Ga = the pass's active CTAs) and writes the digit total to
// totals[d].  G <= 1024.
__global__ void __launch_bounds__(kScanThreads) radix_scan_kernel(const RadixPass a, int G) {
  const RadixPlan pl = radix_plan(a.range, a.bits);
  if (a.pass >= pl.passes) return;
  unsigned* totals = a.digit_tot;
  unsigned* h = a.hist + (long long)blockIdx.x * G;
  const int Ga = radix_active(a.count(), G);
  constexpr int kPer = 4;  // 256 threads x 4 >= 1024 blocks
  unsigned loc[kPer];
  unsigned long long s = 0;
  const int first = threadIdx.x * kPer;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    loc[k] = first + k < Ga ? h[first + k] : 0u;
    s += loc[k];
  }
  unsigned long long tot;
  unsigned long long off = block_excl_scan(s, &tot);
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    if (first + k < Ga) h[first + k] = (unsigned)off;
    off += loc[k];
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = (unsigned)tot;
}

// Scatter of one radix pass (digit = (key >> shift) & dmask, at most 8
// bits).  Per 2048-item tile: digits ranked within each warp from bit
// ballots (stable within the tile), the tile is reordered by digit in shared
// memory, then written out so that consecutive threads store consecutive
// addresses of one digit's run (coalesced), and each digit's running global
// offset advances by the tile's count.  The next tile's keys and values are
// loaded into registers while the current one is ranked and written.
#ifndef GS_RADIX_CTAS
#define GS_RADIX_CTAS 3  // resident scatter CTAs per SM the register budget targets
#endif
__global__ void __launch_bounds__(kRadixThreads, GS_RADIX_CTAS) radix_downsweep_kernel(
    const RadixPass a) {
  const RadixPlan pl = radix_plan(a.range, a.bits);
  if (a.pass >= pl.passes) return;
  unsigned* __restrict__ keys_out = a.keys_out;
  unsigned* __restrict__ vals_out = a.vals_out;
  const unsigned* __restrict__ offsets = a.hist;
  const unsigned* __restrict__ totals = a.digit_tot;
  const int shift = radix_shift(pl, a.pass);
  const unsigned mask = radix_mask(pl, a.pass);
  const bool wkeys = a.keys_last || a.pass + 1 < pl.passes;
  __shared__ unsigned s_wc[kRadixWarps][kRadixBins + 1];  // per-warp digit counters (+ dummy)
  __shared__ unsigned s_pre[kRadixWarps][kRadixBins];     // per-warp start within the digit's run
  __shared__ unsigned s_off[kRadixBins];                  // tile-local start per digit
  __shared__ unsigned s_gl[kRadixBins];                   // global minus tile-local start per digit
  __shared__ unsigned s_ws[kRadixWarps];                  // warp totals of the digit scan
  __shared__ unsigned s_nt;                               // items of the tile taking part
  __shared__ unsigned s_key[kRadixTile];
  __shared__ unsigned s_val[kRadixTile];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  const long long n = a.count();
  if ((int)blockIdx.x >= radix_active(n, gridDim.x)) return;  // (the whole CTA)
  const long long chunk = radix_chunk(n, gridDim.x);
  const long long b0 = (long long)blockIdx.x * chunk;
  const long long b1 = min(n, b0 + chunk);
  // the first tile's keys and values are requested before the digit bases
  // (independent loads, their latency overlaps the scan)
  unsigned nk[kRadixIpt], nv[kRadixIpt];
  unsigned nin = 0u;  // bit i: item i takes part
  const int lbase = w * (32 * kRadixIpt) + lane;
#pragma unroll
  for (int i = 0; i < kRadixIpt; ++i) {
    bool in;
    radix_load(a, b0 + lbase + i * 32, b1, nk[i], nv[i], in);
    nin |= (in ? 1u : 0u) << i;
  }
  // thread d owns digit d (kRadixThreads == kRadixBins): its running global
  // offset = exclusive scan of the digit totals + this CTA's offset
  const int dd = threadIdx.x;
  unsigned gbase;
  {
    const unsigned off = offsets[(long long)dd * gridDim.x + blockIdx.x];
    unsigned long long tot;
    gbase = (unsigned)block_excl_scan(totals[dd], &tot) + off;
    // the first pass over rows reports the count of the rows taking part
    if (a.from_rows() && blockIdx.x == 0 && threadIdx.x == 0) *a.rows.n_vis = (long long)tot;
  }
  for (int i = threadIdx.x; i < kRadixWarps * (kRadixBins + 1); i += kRadixThreads)
    (&s_wc[0][0])[i] = 0u;
  __syncthreads();
  // Four barriers per tile.  The counters s_wc are read and cleared between
  // the first two, so the next tile's ranking may start while this tile is
  // still being written out; the next tile's first barrier orders that
  // write-out before the shared tile and the offsets are overwritten.
  for (long long t0 = b0; t0 < b1; t0 += kRadixTile) {
    unsigned k[kRadixIpt], v[kRadixIpt], dg[kRadixIpt], loc[kRadixIpt];
#pragma unroll
    for (int i = 0; i < kRadixIpt; ++i) {
      k[i] = nk[i];
      v[i] = nv[i];
      dg[i] = (nin >> i) & 1u ? radix_digit(k[i], pl, shift, mask) : (unsigned)kRadixBins;
    }
    const long long t1 = t0 + kRadixTile;
    if (t1 < b1) {
      nin = 0u;
#pragma unroll
      for (int i = 0; i < kRadixIpt; ++i) {
        bool in;
        radix_load(a, t1 + lbase + i * 32, b1, nk[i], nv[i], in);
        nin |= (in ? 1u : 0u) << i;
      }
    }
#pragma unroll
    for (int i = 0; i < kRadixIpt; ++i) {
      // lanes holding the same digit: one ballot per digit bit plus validity
      const bool valid = dg[i] < (unsigned)kRadixBins;
      const unsigned vm = __ballot_sync(0xffffffffu, valid);
      unsigned peers = valid ? vm : ~vm;
      // (digit bits at or above the pass's width are zero in every lane:
      // their ballots leave peers unchanged)
#pragma unroll
      for (int b = 0; b < kRadixMaxBits; ++b) {
        const bool bit = (dg[i] >> b) & 1u;
        const unsigned m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
      }
      const unsigned rank = __popc(peers & lt_mask);
      const unsigned base = s_wc[w][dg[i]];
      __syncwarp();
      if (rank == 0) s_wc[w][dg[i]] = base + __popc(peers);
      __syncwarp();
      loc[i] = base + rank;
    }
    __syncthreads();
    unsigned run = 0, inc;
    {
      // digit dd: prefix over the warps (counters cleared for the next
      // tile), then a 32-bit scan of the tile counts over the digits
#pragma unroll
      for (int ww = 0; ww < kRadixWarps; ++ww) {
        const unsigned c = s_wc[ww][dd];
        s_pre[ww][dd] = run;
        s_wc[ww][dd] = 0u;
        run += c;
      }
      inc = run;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
      }
      if (lane == 31) s_ws[w] = inc;
    }
    __syncthreads();
    {
      unsigned wo = 0;
#pragma unroll
      for (int ww = 0; ww < kRadixWarps - 1; ++ww) wo += ww < w ? s_ws[ww] : 0u;
      const unsigned off = wo + inc - run;
      s_off[dd] = off;
      s_gl[dd] = gbase - off;
      gbase += run;
      if (dd == kRadixBins - 1) s_nt = off + run;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRadixIpt; ++i) {
      if (dg[i] < (unsigned)kRadixBins) {
        const unsigned lp = s_off[dg[i]] + s_pre[w][dg[i]] + loc[i];
        s_key[lp] = k[i];
        s_val[lp] = v[i];
      }
    }
    __syncthreads();
    const int nt = (int)s_nt;
    for (int i = threadIdx.x; i < nt; i += kRadixThreads) {
      const unsigned kk = s_key[i];
      const unsigned pos = s_gl[radix_digit(kk, pl, shift, mask)] + (unsigned)i;
      if (!GS_IN_BOUNDS(pos, n, 202)) continue;
      if (wkeys) keys_out[pos] = kk;
      vals_out[pos] = s_val[i];
    }
  }
}

// Buffer index (0 or 1) holding the sorted result.
__device__ __forceinline__ int radix_result(const unsigned* range, int bits) {
  return radix_plan(range, bits).passes & 1;
}

// ----------------------------------------------------------------------------
// Super-pair generation, per-tile expansion.
// ----------------------------------------------------------------------------
// Super-pair duplication.  Each CTA takes one scan block of the depth-sorted
// visible rows (the blocks of rows_gather_kernel, whose item counts are
// already scanned into the blocks' item bases), scans its rows' super-tile
// counts in shared memory, and expands its items: every thread takes 4
// consecutive items, finds the row owning the first by a binary search over
// the rows' item offsets, walks through the owner's super-tile span (and on
// to the next rows) and stores the 4 (super-tile, row) items with one
// 16-byte store per array where aligned.  Items keep the rows' depth order.
// floor(a / d) for a < 2^32 from m = floor(2^32 / d) (d >= 2) or m = 2^32 - 1
// (d = 1): the product's high word is the quotient or one less.
__device__ __forceinline__ unsigned div_magic(unsigned a, unsigned d, unsigned m) {
  unsigned q = __umulhi(a, m);
  if (a - q * d >= d) ++q;
  return q;
}
unsigned div_magic_host(unsigned d) {
  return d <= 1u ? 0xffffffffu : (unsigned)((1ull << 32) / d);
}

// floor(a / d) for 0 <= a < 2^27, d >= 1 from a float reciprocal, corrected
// to the exact quotient.
__device__ __forceinline__ int div_small(int a, int d) {
  int q = __float2int_rz(__int2float_rn(a) * __frcp_rn(__int2float_rn(d)));
  while (q * d > a) --q;
  while ((q + 1) * d <= a) ++q;
  return q;
}

template <int ITEMS>
__global__ void __launch_bounds__(kScanThreads) rows_expand_kernel(
    const SortedRows sorted, const uint2* __restrict__ rect_sorted,
    const long long* __restrict__ n_dev, const unsigned long long* __restrict__ block_items,
    const long long* __restrict__ q_eff, int N, unsigned n_magic, const CamTable ct,
    unsigned* __restrict__ skeys, unsigned* __restrict__ svals, int vec16, int packed,
    unsigned* __restrict__ hist, int hgrid, unsigned hmask) {
  constexpr int RB = kScanThreads * ITEMS;
  __shared__ unsigned s_off[RB + 1];  // item offset of each row in the block (+ the total)
  // the super-tile sort's first-pass histogram (hist: [256][hgrid], zeroed):
  // the block's items are one contiguous range of positions, which meets
  // one or two of the sort's chunks; their digit counts are summed here
  __shared__ unsigned s_h[2][kRadixBins];
  const long long n = *n_dev, Q = *q_eff;
  const long long base = (long long)blockIdx.x * RB;
  if (base >= n || Q == 0) return;  // (the whole CTA)
  if (hist)
    for (int i = threadIdx.x; i < 2 * kRadixBins; i += kScanThreads) (&s_h[0][0])[i] = 0u;
  const int nr = (int)min((long long)RB, n - base);
  const int first = threadIdx.x * ITEMS;
  unsigned loc[ITEMS];
  unsigned long long sum = 0;
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    const int i = first + k;
    loc[k] = i < nr ? st_count(unpack_rect(rect_sorted[base + i])) : 0u;
    sum += loc[k];
  }
  unsigned long long tot;
  unsigned off = (unsigned)block_excl_scan(sum, &tot);
#pragma unroll
  for (int k = 0; k < ITEMS; ++k) {
    s_off[first + k] = off;
    off += loc[k];
  }
  if (threadIdx.x == 0) s_off[RB] = (unsigned)tot;
  __syncthreads();
  const unsigned total = (unsigned)tot;
  const long long gbase = (long long)block_items[blockIdx.x];
  const unsigned* __restrict__ rows = sorted.get();
  // the sort's chunk of a position: div_magic by the chunk (Q < 2^32)
  const unsigned hchunk = hist ? (unsigned)radix_chunk(Q, hgrid) : 1u;
  const unsigned hmagic = hist ? (unsigned)(0x100000000ull / hchunk) : 0u;
  const unsigned hc0 = hist ? div_magic((unsigned)gbase, hchunk, hmagic) : 0u;
  for (unsigned c0 = 0; c0 < total; c0 += 4 * kScanThreads) {
    const unsigned e0 = c0 + 4u * threadIdx.x;
    if (e0 >= total) continue;
    // the owner of e0: the last row whose items start at or before it (rows
    // without items share their start with the next row)
    int lo = 0, hi = nr - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_off[mid] <= e0) lo = mid;
      else hi = mid - 1;
    }
    int j = lo;
    unsigned kk[4], vv[4];
    unsigned row = 0u;
    int4 r = make_int4(0, 0, 0, 0), q = r;
    int id0 = 0, wdt = 1, stx = 1, x = 0, y = 0;
    int cur = -1;
    int cnt = 0;
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const unsigned e = e0 + (unsigned)t;
      if (e >= total) break;
      while (s_off[j + 1] <= e) ++j;  // (s_off[nr .. RB] = total > e)
      if (j != cur) {
        row = rows[base + j];
        if (!GS_IN_BOUNDS(row, (long long)N * ct.V, 205)) row = 0u;
        r = unpack_rect(rect_sorted[base + j]);
        q = st_span(r);
        const CamInfo& c = ct.c[div_magic(row, (unsigned)N, n_magic)];
        id0 = c.st_off + q.y * c.STX + q.x;
        wdt = max(q.z - q.x, 1);
        stx = c.STX;
        const int k = (int)(e - s_off[j]);
        y = div_small(k, wdt);
        x = k - y * wdt;
        cur = j;
      } else if (++x == wdt) {  // next span row
        x = 0;
        ++y;
      }
      unsigned key = (unsigned)(id0 + y * stx + x);
      if (packed) {
        // the row's rect inside this super-tile: x0 | x1 << 4 | y0 << 8 | y1 << 12
        const int ox = 8 * (q.x + x), oy = 8 * (q.y + y);
        const unsigned dx0 = (unsigned)max(r.x - ox, 0), dx1 = (unsigned)min(r.z - ox, 8);
        const unsigned dy0 = (unsigned)max(r.y - oy, 0), dy1 = (unsigned)min(r.w - oy, 8);
        key |= (dx0 | (dx1 << 4) | (dy0 << 8) | (dy1 << 12)) << 16;
      }
      kk[t] = key;
      vv[t] = row;
      cnt = t + 1;
    }
    const long long g0 = gbase + e0;
    if (hist) {
      // the 4 positions cross at most one chunk boundary (chunks hold whole
      // 2048-item tiles)
      const unsigned c = div_magic((unsigned)g0, hchunk, hmagic);
      const unsigned long long next = (unsigned long long)(c + 1u) * hchunk;
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        if (t < cnt && g0 + t < Q) {
          const unsigned ct_ = (unsigned long long)(g0 + t) >= next ? c + 1u : c;
          const unsigned d = kk[t] & hmask;
          if (ct_ - hc0 < 2u) atomicAdd(&s_h[ct_ - hc0][d], 1u);
          else atomicAdd(hist + (long long)d * hgrid + ct_, 1u);
        }
      }
    }
    if (vec16 && cnt == 4 && (g0 & 3) == 0 && g0 + 3 < Q) {  // skeys, svals 16-byte aligned
      reinterpret_cast<uint4*>(skeys + g0)[0] = make_uint4(kk[0], kk[1], kk[2], kk[3]);
      reinterpret_cast<uint4*>(svals + g0)[0] = make_uint4(vv[0], vv[1], vv[2], vv[3]);
    } else {
#pragma unroll
      for (int t = 0; t < 4; ++t)
        if (t < cnt && g0 + t < Q) {
          skeys[g0 + t] = kk[t];
          svals[g0 + t] = vv[t];
        }
    }
  }
  if (hist) {
    __syncthreads();
    for (int i = threadIdx.x; i < 2 * kRadixBins; i += kScanThreads) {
      const unsigned v = (&s_h[0][0])[i];
      if (v) atomicAdd(hist + (long long)(i % kRadixBins) * hgrid + hc0 + i / kRadixBins, v);
    }
  }
}

// Per-key [start, end) from sorted u32 keys: each thread reads 4
// consecutive keys with one 16-byte load (the array is 256-byte aligned) plus
// its neighbours, and marks where the key changes.
__global__ void __launch_bounds__(256) ranges_kernel(const unsigned* __restrict__ tkeys,
                                                     const long long* __restrict__ p_eff,
                                                     unsigned kmask,
                                                     unsigned* __restrict__ ranges) {
  const long long P = *p_eff;
  const long long groups = (P + 3) / 4;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < groups;
       g += (long long)gridDim.x * blockDim.x) {
    const long long i0 = 4 * g;
    unsigned k[6];
    if (i0 + 3 < P) {
      const uint4 v = reinterpret_cast<const uint4*>(tkeys)[g];
      k[1] = v.x & kmask; k[2] = v.y & kmask; k[3] = v.z & kmask; k[4] = v.w & kmask;
    } else {
      for (int q = 0; q < 4; ++q) k[1 + q] = i0 + q < P ? tkeys[i0 + q] & kmask : 0u;
    }
    k[0] = i0 > 0 ? tkeys[i0 - 1] & kmask : 0xffffffffu;
    k[5] = i0 + 4 < P ? tkeys[i0 + 4] & kmask : 0xffffffffu;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long i = i0 + q;
      if (i >= P) break;
      const unsigned t = k[1 + q];
      if (i == 0 || k[q] != t) ranges[2ll * t] = (unsigned)i;
      const unsigned nxt = (i == P - 1) ? 0xffffffffu : (q < 3 ? k[2 + q] : k[5]);
      if (i == P - 1 || nxt != t) ranges[2ll * t + 1] = (unsigned)(i + 1);
    }
  }
}

// ----------------------------------------------------------------------------
// Expansion of the super-tile-sorted rows into per-tile lists.  A super-tile's
// rows (depth order) are cut into segments of kSeg; per segment and per tile
// of the super-tile (64), the count of rows covering the tile; per tile, the
// exclusive scan of those counts over the super-tile's segments; per tile,
// the list start (scan over all tiles); then every segment writes each of
// its rows into the lists of the tiles it covers, ranks from warp ballots,
// so each list keeps the depth order of the rows.
// ----------------------------------------------------------------------------
constexpr int kSeg = 1024;
static_assert(kSeg % 256 == 0, "st_count_kernel loads a segment in groups of 256");

__device__ __forceinline__ int view_of_st(const CamTable& ct, int s) {
  int v = 0;
  while (v + 1 < ct.V && ct.c[v + 1].st_off <= s) ++v;
  return v;
}

// Segments of every super-tile: seg_first[s] (exclusive scan of
// ceil(len_s / kSeg)), seg_first[S] = total, seg_st[g] = super-tile of g.
// One CTA of 1024 threads.
__global__ void __launch_bounds__(1024) st_segments_kernel(uint2* __restrict__ st_ranges,
                                                           int S, const unsigned* __restrict__ totals,
                                                           const long long* __restrict__ q_eff,
                                                           unsigned* __restrict__ seg_first,
                                                           unsigned* __restrict__ seg_st,
                                                           long long* __restrict__ n_seg) {
  __shared__ unsigned s_w[32];
  __shared__ unsigned s_carry;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (totals) {
    // one radix pass sorted the items by super-tile (S <= 512): the per-digit
    // totals are the per-super-tile counts, and their exclusive scan the starts
    // (S <= 256: the first 8 warps, one block-level scan)
    const unsigned tot = tid < S ? totals[tid] : 0u;
    unsigned incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
      const unsigned x = s_w[lane];
      unsigned xi = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, xi, o);
        if (lane >= o) xi += y;
      }
      s_w[lane] = xi - x;
    }
    __syncthreads();
    if (tid < S) {
      const unsigned run = s_w[w] + incl - tot;
      st_ranges[tid] = make_uint2(tot ? run : 0u, tot ? run + tot : 0u);
    }
  } else if (S == 1 && tid == 0) {  // no sort: one super-tile holds every item
    const unsigned q = (unsigned)*q_eff;
    st_ranges[0] = make_uint2(0u, q);
  }
  if (tid == 0) s_carry = 0u;
  __syncthreads();
  for (int base = 0; base < S; base += 1024) {
    const int s = base + tid;
    unsigned cnt = 0u;
    if (s < S) {
      const uint2 r = st_ranges[s];
      cnt = (r.y - r.x + kSeg - 1) / kSeg;
    }
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
      const unsigned t = s_w[lane];
      unsigned ti = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += y;
      }
      s_w[lane] = ti - t;
    }
    __syncthreads();
    if (s < S) seg_first[s] = s_carry + s_w[w] + incl - cnt;
    __syncthreads();
    if (tid == 1023) s_carry += s_w[31] + incl;
    __syncthreads();
  }
  if (tid == 0) {
    seg_first[S] = s_carry;
    *n_seg = (long long)s_carry;
  }
  __syncthreads();
  // the super-tile of every segment: a warp per super-tile
  for (int s = w; s < S; s += 32) {
    const unsigned g0 = seg_first[s], g1 = seg_first[s + 1];
    for (unsigned g = g0 + lane; g < g1; g += 32) seg_st[g] = (unsigned)s;
  }
}

// Rows [b, e) of segment g of super-tile s, its view and tile origin.
struct SegInfo {
  unsigned b, e;
  int view, ox, oy;
};

__device__ __forceinline__ SegInfo seg_info(long long g, const uint2* __restrict__ st_ranges,
                                            const unsigned* __restrict__ seg_first,
                                            const unsigned* __restrict__ seg_st,
                                            const CamTable& ct) {
  SegInfo si;
  const int s = (int)seg_st[g];
  const uint2 rg = st_ranges[s];
  si.b = rg.x + (unsigned)(g - seg_first[s]) * (unsigned)kSeg;
  si.e = min(rg.y, si.b + (unsigned)kSeg);
  si.view = view_of_st(ct, s);
  const CamInfo& c = ct.c[si.view];
  const int sl = s - c.st_off;
  si.ox = (sl % c.STX) * kSuperTile;
  si.oy = (sl / c.STX) * kSuperTile;
  return si;
}

// Ballots of a warp's 32 rows (one per lane) over the rows and the columns of
// an 8x8 super-tile: B[r] = lanes whose rect covers tile row r, X[c] = lanes
// whose rect covers tile column c; the lanes covering tile (r, c) are
// B[r] & X[c].  d = x0 | x1 << 4 | y0 << 8 | y1 << 12 (0: no tile).
// The descriptor's rows and columns as 8-bit masks (bit k: k in [lo, hi)).
__device__ __forceinline__ unsigned desc_rows(unsigned d) {
  return ((1u << ((d >> 12) & 15u)) - 1u) & ~((1u << ((d >> 8) & 15u)) - 1u);
}
__device__ __forceinline__ unsigned desc_cols(unsigned d) {
  return ((1u << ((d >> 4) & 15u)) - 1u) & ~((1u << (d & 15u)) - 1u);
}

// MASKS: each ballot tests one bit of the rect's 8-bit row or column mask
// (st_emit_kernel: 1117 -> 1079 us on cfg3); otherwise two comparisons
// (st_count_kernel: 245 us, against 291 us with the masks, measured
// back to back in one session).
template <bool MASKS>
__device__ __forceinline__ void rect_ballots(unsigned d, unsigned B[8], unsigned X[8]) {
  if (MASKS) {
    const unsigned rm = desc_rows(d), cm = desc_cols(d);
#pragma unroll
    for (unsigned r = 0; r < 8; ++r) {
      B[r] = __ballot_sync(0xffffffffu, (rm >> r) & 1u);
      X[r] = __ballot_sync(0xffffffffu, (cm >> r) & 1u);
    }
  } else {
    const unsigned x0 = d & 15u, x1 = (d >> 4) & 15u, y0 = (d >> 8) & 15u, y1 = (d >> 12) & 15u;
#pragma unroll
    for (unsigned r = 0; r < 8; ++r) {
      B[r] = __ballot_sync(0xffffffffu, y0 <= r && r < y1);
      X[r] = __ballot_sync(0xffffffffu, x0 <= r && r < x1);
    }
  }
}

// Counts of the warp's rows covering tiles `lane` and `lane + 32` of the
// super-tile (tile b = 8 row + column).
// The lanes of the warp's rows covering tiles `lane` and `lane + 32`.
__device__ __forceinline__ void lane_tile_masks(const unsigned B[8], const unsigned X[8],
                                                int lane, unsigned& m0, unsigned& m1) {
  const int r = lane >> 3, c = lane & 7;
  unsigned b0 = B[0], b1 = B[4], x = X[0];
#pragma unroll
  for (int k = 1; k < 4; ++k) {
    b0 = r == k ? B[k] : b0;
    b1 = r == k ? B[k + 4] : b1;
  }
#pragma unroll
  for (int k = 1; k < 8; ++k) x = c == k ? X[k] : x;
  m0 = b0 & x;
  m1 = b1 & x;
}

__device__ __forceinline__ void lane_tile_counts(const unsigned B[8], const unsigned X[8],
                                                 int lane, unsigned& c0, unsigned& c1) {
  unsigned m0, m1;
  lane_tile_masks(B, X, lane, m0, m1);
  c0 = __popc(m0);
  c1 = __popc(m1);
}

// Rect of row `row` inside the super-tile with tile origin (ox, oy), as a
// descriptor (0 when it covers no tile of it).
__device__ __forceinline__ unsigned st_desc(const int* __restrict__ rect, unsigned row, int N,
                                            const CamTable& ct, int ox, int oy) {
  const int4 r = view_rect(rect, row, N, ct);
  const int x0 = max(r.x - ox, 0), x1 = min(r.z - ox, kSuperTile);
  const int y0 = max(r.y - oy, 0), y1 = min(r.w - oy, kSuperTile);
  if (x1 <= x0 || y1 <= y0) return 0u;  // (not produced by consistent inputs)
  return (unsigned)(x0 | (x1 << 4) | (y0 << 8) | (y1 << 12));
}

// Per segment: the count of rows covering each of the 64 tiles (warp ballots,
// summed over the CTA's warps).  The rect descriptors travel in the items'
// keys (bits 16-31) when `packed`; otherwise they are formed here from the
// rects and stored in desc for the expansion.
__global__ void __launch_bounds__(256) st_count_kernel(
    const unsigned* __restrict__ sp_keys, const unsigned* __restrict__ sp_rows,
    const uint2* __restrict__ st_ranges, const unsigned* __restrict__ seg_first,
    const unsigned* __restrict__ seg_st, const long long* __restrict__ n_seg, int packed,
    const int* __restrict__ rect, int N, const CamTable ct, unsigned* __restrict__ desc,
    unsigned* __restrict__ hist) {
  __shared__ unsigned s_cnt[8][64];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long long G = *n_seg;
  for (long long g = blockIdx.x; g < G; g += gridDim.x) {
    const SegInfo si = seg_info(g, st_ranges, seg_first, seg_st, ct);
    unsigned a0 = 0u, a1 = 0u;
    // a segment holds at most kSeg = 4 x 256 items: each warp's (up to) four
    // groups of 32 are loaded before any is counted
    constexpr int kGroups = kSeg / 256;
    unsigned dd[kGroups];
#pragma unroll
    for (int k = 0; k < kGroups; ++k) {
      const unsigned i = si.b + 32u * w + 256u * k + lane;
      dd[k] = 0u;
      if (i < si.e) {
        if (packed) {
          dd[k] = sp_keys[i] >> 16;
        } else {
          dd[k] = st_desc(rect, sp_rows[i], N, ct, si.ox, si.oy);
          desc[i] = dd[k];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kGroups; ++k) {
      if (si.b + 32u * w + 256u * k >= si.e) break;  // warp-uniform
      unsigned B[8], X[8], n0, n1;
      rect_ballots<false>(dd[k], B, X);
      lane_tile_counts(B, X, lane, n0, n1);
      a0 += n0;
      a1 += n1;
    }
    s_cnt[w][lane] = a0;
    s_cnt[w][lane + 32] = a1;
    __syncthreads();
    if (tid < 64) {
      unsigned sum = 0u;
#pragma unroll
      for (int ww = 0; ww < 8; ++ww) sum += s_cnt[ww][tid];
      hist[g * 64 + tid] = sum;
    }
    __syncthreads();
  }
}

// One CTA per super-tile, 16 groups x 64 tiles: exclusive scan of every
// tile's counts over the super-tile's segments (in place), and the tile's
// total list length.
__device__ __forceinline__ void tile_scan_dev(const unsigned* __restrict__ tile_cnt, int T,
                                              unsigned* __restrict__ tile_start,
                                              unsigned* __restrict__ ranges);

__global__ void __launch_bounds__(1024) st_scan_kernel(const unsigned* __restrict__ seg_first,
                                                       const CamTable ct,
                                                       unsigned* __restrict__ hist,
                                                       unsigned* __restrict__ tile_cnt,
                                                       unsigned long long* __restrict__ arrive,
                                                       unsigned* __restrict__ tile_start,
                                                       unsigned* __restrict__ ranges) {
  __shared__ unsigned s_part[16][64];
  const int s = blockIdx.x;
  const int k = threadIdx.x >> 6, bt = threadIdx.x & 63;
  const unsigned g0 = seg_first[s], L = seg_first[s + 1] - g0;
  const unsigned per = (L + 15u) / 16u;
  const unsigned a = min(L, (unsigned)k * per), e = min(L, a + per);
  unsigned sum = 0u;
  for (unsigned g = a; g < e; ++g) sum += hist[(long long)(g0 + g) * 64 + bt];
  s_part[k][bt] = sum;
  __syncthreads();
  if (k == 0) {
    unsigned run = 0u;
    for (int kk = 0; kk < 16; ++kk) {
      const unsigned x = s_part[kk][bt];
      s_part[kk][bt] = run;
      run += x;
    }
    const CamInfo& c = ct.c[view_of_st(ct, s)];
    const int sl = s - c.st_off;
    const int tx = (sl % c.STX) * kSuperTile + (bt & 7);
    const int ty = (sl / c.STX) * kSuperTile + (bt >> 3);
    if (tx < c.TX && ty < c.TY) tile_cnt[c.tile_off + ty * c.TX + tx] = run;
  }
  __syncthreads();
  unsigned run = s_part[k][bt];
  for (unsigned g = a; g < e; ++g) {
    unsigned* h = hist + (long long)(g0 + g) * 64 + bt;
    const unsigned x = *h;
    *h = run;
    run += x;
  }
  if (last_block_arrives(arrive, gridDim.x)) tile_scan_dev(tile_cnt, ct.total_tiles, tile_start, ranges);
}

// Exclusive scan of the list lengths over all T tiles (one CTA of 1024
// threads): list starts, and ranges [start, end) ((0, 0) for an empty list).
// Run by the last CTA of st_scan_kernel (tile_cnt read through L2).
__device__ __forceinline__ void tile_scan_dev(const unsigned* __restrict__ tile_cnt, int T,
                                              unsigned* __restrict__ tile_start,
                                              unsigned* __restrict__ ranges) {
  __shared__ unsigned s_w[32];
  __shared__ unsigned s_carry;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) s_carry = 0u;
  __syncthreads();
  for (int base = 0; base < T; base += 1024) {
    const int t = base + tid;
    const unsigned cnt = t < T ? __ldcg(tile_cnt + t) : 0u;
    unsigned incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) s_w[w] = incl;
    __syncthreads();
    if (w == 0) {
      const unsigned x = s_w[lane];
      unsigned xi = x;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xffffffffu, xi, o);
        if (lane >= o) xi += y;
      }
      s_w[lane] = xi - x;
    }
    __syncthreads();
    const unsigned start = s_carry + s_w[w] + incl - cnt;
    if (t < T) {
      tile_start[t] = start;
      ranges[2ll * t] = cnt ? start : 0u;
      ranges[2ll * t + 1] = cnt ? start + cnt : 0u;
    }
    __syncthreads();
    if (tid == 1023) s_carry = start + cnt;
    __syncthreads();
  }
}

// Expansion: per segment, rows in chunks of 256 (one per thread, 8 warps of
// 32 consecutive rows).  Each warp takes its row and column ballots over the
// super-tile, counts its rows per tile, a prefix over the warps and the
// running list positions give every warp its first slot per tile, and the
// lanes covering tile (r, c) (B[r] & X[c]) write their rows at consecutive
// slots, so every list receives its rows in the segment's (depth) order with
// coalesced stores.
template <bool KEYS>
__global__ void __launch_bounds__(256) st_emit_kernel(
    const unsigned* __restrict__ sp_keys, const unsigned* __restrict__ sp_rows,
    const unsigned* __restrict__ desc, int packed, const uint2* __restrict__ st_ranges,
    const unsigned* __restrict__ seg_first, const unsigned* __restrict__ seg_st,
    const long long* __restrict__ n_seg, const unsigned* __restrict__ hist,
    const unsigned* __restrict__ tile_start, const CamTable ct, const float* __restrict__ depth,
    unsigned* __restrict__ out_vals, unsigned long long* __restrict__ out_keys, long long cap) {
  __shared__ unsigned s_run[64];                   // next list slot per tile of the super-tile
  __shared__ unsigned s_cnt[8][64];                // per-warp counts per tile
  __shared__ __align__(16) unsigned s_pos[8][64];  // per-warp first slot per tile
  __shared__ int s_tile[64];                       // global tile id (-1 outside the view)
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const unsigned lt = (1u << lane) - 1u;
  const long long G = *n_seg;
  for (long long g = blockIdx.x; g < G; g += gridDim.x) {
    const SegInfo si = seg_info(g, st_ranges, seg_first, seg_st, ct);
    __syncthreads();  // the previous segment's readers of s_run / s_tile are done
    if (tid < 64) {
      const CamInfo& c = ct.c[si.view];
      const int tx = si.ox + (tid & 7), ty = si.oy + (tid >> 3);
      const bool in = tx < c.TX && ty < c.TY;
      const int t = in ? c.tile_off + ty * c.TX + tx : -1;
      s_tile[tid] = t;
      s_run[tid] = in ? tile_start[t] + hist[g * 64 + tid] : 0u;
    }
    for (unsigned c0 = si.b; c0 < si.e; c0 += 256) {
      const unsigned i = c0 + tid;
      unsigned d = 0u, row = 0u;
      if (i < si.e) {
        d = packed ? (sp_keys[i] >> 16) : desc[i];
        row = sp_rows[i];
      }
      unsigned B[8], X[8], n0, n1;
      rect_ballots<true>(d, B, X);
      lane_tile_counts(B, X, lane, n0, n1);
      s_cnt[w][lane] = n0;
      s_cnt[w][lane + 32] = n1;
      __syncthreads();
      if (tid < 64) {
        unsigned run = s_run[tid];
#pragma unroll
        for (int ww = 0; ww < 8; ++ww) {
          s_pos[ww][tid] = run;
          run += s_cnt[ww][tid];
        }
        s_run[tid] = run;
      }
      __syncthreads();
      // this lane's rect in the super-tile, and the column ballots restricted
      // to the lanes before it (ranks by population counts, no branches per
      // tile: in the dense case nearly every tile has a covering row)
      const unsigned rows = desc_rows(d), cols = desc_cols(d);
      unsigned Xl[8];
#pragma unroll
      for (int c = 0; c < 8; ++c) Xl[c] = X[c] & lt;
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        if (B[r] == 0u) continue;  // warp-uniform
        const uint4 pa = *reinterpret_cast<const uint4*>(&s_pos[w][8 * r]);
        const uint4 pb = *reinterpret_cast<const uint4*>(&s_pos[w][8 * r + 4]);
        const unsigned sp[8] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
        const unsigned cov = ((rows >> r) & 1u) ? cols : 0u;
#pragma unroll
        for (unsigned c = 0; c < 8; ++c) {
          // this lane covers tile (r, c): its rank among the covering lanes
          const unsigned pos = sp[c] + __popc(B[r] & Xl[c]);
          if ((cov & (1u << c)) && GS_IN_BOUNDS(pos, cap, 201)) {
            out_vals[pos] = row;
            if (KEYS)
              out_keys[pos] = ((unsigned long long)(unsigned)s_tile[8 * r + c] << 32) |
                              __float_as_uint(depth[row]);
          }
        }
      }
    }
  }
}


__global__ void set_value_kernel(long long* __restrict__ dst, long long v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = v;
}

// ----------------------------------------------------------------------------
// Workspace layout.
// ----------------------------------------------------------------------------
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Workspace {
  unsigned long long* block_sums;  // scan block sums
  unsigned long long* block_sums2; // second scan's block sums
  long long* counters;             // [0] n_vis, [1] P, [2] P eff., [3] Q, [4] Q eff., [5] segments
  unsigned* rk[2];                 // row keys (depth bits), double buffer
  unsigned* rv[2];                 // row values, double buffer
  uint2* rect_sorted;              // clamped rect per visible row, depth order (16-bit packed)
  unsigned* pk[2];                 // super-pair keys (super-tile), double buffer; later descriptors
  unsigned* pv;                    // super-pair values (rows)
  unsigned* hist;                  // radix histograms
  unsigned* st_ranges;             // [2 * super-tiles] rows of each super-tile
  unsigned* seg_first;             // [super-tiles + 1] first segment of each super-tile
  unsigned* seg_st;                // super-tile of every segment
  unsigned* seg_hist;              // [segments][64] per-tile counts, then bases
  unsigned* tile_cnt;              // [tiles] list lengths
  unsigned* tile_start;            // [tiles] list starts
  size_t bytes;
};

constexpr int kRadixGrid = 4 * 152;  // largest radix grid (4 CTAs per SM of a GB300)

// Radix histograms: [256][grid] per-CTA digit counts and their scan, then the
// 256 digit totals.
constexpr size_t radix_hist_bytes() { return 4ull * kRadixBins * (kRadixGrid + 1); }

// CTAs of radix_downsweep_kernel resident on the current device at once
// (cached per device).
int radix_resident_ctas() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return kRadixGrid;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  int per_sm = 0, sms = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, radix_downsweep_kernel,
                                                    kRadixThreads, 0) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      per_sm < 1 || sms < 1) {
    cudaGetLastError();
    return kRadixGrid;
  }
  v = per_sm * sms;
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

inline long long scan_blocks(long long n) { return (n + kScanTile - 1) / kScanTile; }

// Upper bound of the expansion segments: sum over super-tiles of
// ceil(len / kSeg) <= Q / kSeg + super-tiles, and Q <= P <= cap.
inline long long max_segments(long long cap, long long tiles) { return cap / kSeg + tiles + 2; }

constexpr int kCounters = 14;  // 8 counts, 3 arrival counters, spare, the depth-key range

Workspace carve(void* base, long long n_rows, long long cap, long long tiles) {
  Workspace w;
  char* p = reinterpret_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* r = p ? p + off : nullptr;
    off += align256(bytes);
    return r;
  };
  const long long nb = scan_blocks(n_rows > cap ? n_rows : cap) + 1;
  const long long ms = max_segments(cap, tiles);
  w.block_sums = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * nb));
  w.block_sums2 = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * nb));
  w.counters = reinterpret_cast<long long*>(take(sizeof(long long) * kCounters));
  for (int i = 0; i < 2; ++i) w.rk[i] = reinterpret_cast<unsigned*>(take(4 * (n_rows + 1)));
  for (int i = 0; i < 2; ++i) w.rv[i] = reinterpret_cast<unsigned*>(take(4 * (n_rows + 1)));
  w.rect_sorted = reinterpret_cast<uint2*>(take(8 * (n_rows + 1)));
  for (int i = 0; i < 2; ++i) w.pk[i] = reinterpret_cast<unsigned*>(take(4 * (cap + 1)));
  w.pv = reinterpret_cast<unsigned*>(take(4 * (cap + 1)));
  w.hist = reinterpret_cast<unsigned*>(take(radix_hist_bytes()));
  w.st_ranges = reinterpret_cast<unsigned*>(take(8ull * (tiles + 1)));
  w.seg_first = reinterpret_cast<unsigned*>(take(4ull * (tiles + 2)));
  w.seg_st = reinterpret_cast<unsigned*>(take(4ull * ms));
  w.seg_hist = reinterpret_cast<unsigned*>(take(4ull * 64 * ms));
  w.tile_cnt = reinterpret_cast<unsigned*>(take(4ull * (tiles + 1)));
  w.tile_start = reinterpret_cast<unsigned*>(take(4ull * (tiles + 1)));
  w.bytes = off;
  return w;
}

// Radix sort of the pairs in (k[0], v[0]) (n_dev items, at most n_bound):
// with `range` on the significant bits of (key - smallest key), else on
// `bits` bits.  The result is in buffer (passes mod 2): radix_result on the
// device, or the host's plan when there is no range.  keys_last: the last
// pass writes the keys as well (only the values are needed otherwise).
// The radix grid for at most n_bound items.
int radix_grid(long long n_bound) {
  return (int)std::max<long long>(
      1, std::min<long long>(std::min(kRadixGrid, radix_resident_ctas()),
                             (n_bound + kRadixTile - 1) / kRadixTile));
}

void radix_sort(unsigned* k[2], unsigned* v[2], const long long* n_dev, long long n_bound,
                const unsigned* range, int bits, unsigned* hist, bool keys_last,
                cudaStream_t st, const RadixRows* rows = nullptr, bool hist0_ready = false) {
  if (n_bound == 0) return;
  const int passes = range ? kRadixMaxPasses : radix_plan_bits(0u, bits).passes;
  // one wave: at most the CTAs of the scatter kernel resident on the device
  const int grid = radix_grid(n_bound);
  RadixPass a;
  a.n_dev = n_dev;
  a.range = range;
  a.bits = bits;
  a.hist = hist;
  a.digit_tot = hist + kRadixBins * grid;
  a.keys_last = keys_last ? 1 : 0;
  a.rows = rows ? *rows : RadixRows{nullptr, nullptr, 0, nullptr};
  for (int p = 0; p < passes; ++p) {
    a.keys_in = k[p & 1];
    a.vals_in = v[p & 1];
    a.keys_out = k[(p + 1) & 1];
    a.vals_out = v[(p + 1) & 1];
    a.pass = p;
    // (hist0_ready: the first pass's per-CTA digit counts are already in
    // hist, summed by the kernel that wrote the items)
    if (p > 0 || !hist0_ready) radix_upsweep_kernel<<<grid, kRadixThreads, 0, st>>>(a);
    radix_scan_kernel<<<kRadixBins, kScanThreads, 0, st>>>(a, grid);
    radix_downsweep_kernel<<<grid, kRadixThreads, 0, st>>>(a);
    count_launches(p > 0 || !hist0_ready ? 3 : 2);
  }
}

int bits_for(long long count) {
  int b = 0;
  while (b < 32 && (1ll << b) < count) ++b;
  return b;
}

}  // namespace

GS_BOUNDS_READER(bounds_status_binning)

size_t bin_sort_workspace_size(long long n_rows, long long cap, long long total_tiles) {
  return carve(nullptr, n_rows, cap, total_tiles).bytes;
}

int launch_bin_sort(const gs_proj* proj, int N, const CamTable& ct, void* workspace,
                    size_t ws_bytes, long long cap, unsigned* sorted_vals,
                    unsigned long long* sorted_keys, unsigned* ranges, long long* num_pairs_dev,
                    long long* num_pairs_host, int* status_dev, cudaStream_t st) {
  const long long n_rows = (long long)N * ct.V;
  const long long T = ct.total_tiles;
  const int S = ct.total_st;
  Workspace w = carve(workspace, n_rows, cap, T);
  if (ws_bytes < w.bytes) return GS_ERR_INVALID_ARG;
  long long* n_vis = w.counters;
  long long* P = w.counters + 1;
  long long* p_eff = w.counters + 2;
  long long* Q = w.counters + 3;
  long long* q_eff = w.counters + 4;
  long long* n_seg = w.counters + 5;
  // arrival counters of the kernels whose last CTA runs the following scan
  unsigned long long* arrive = reinterpret_cast<unsigned long long*>(w.counters + 8);
  GS_TRY_CUDA(cudaMemsetAsync(w.counters, 0, kCounters * sizeof(long long), st));
  const CountsOut co{w.block_sums, w.block_sums2, cap, Q, P, q_eff, p_eff, num_pairs_dev,
                     status_dev};
  // the visible rows' depth-bit range (complement of the smallest, largest)
  unsigned* range = reinterpret_cast<unsigned*>(w.counters + 12);
  const SortedRows rows_sorted{w.rv[0], w.rv[1], range};
  // scan blocks of 1,024 rows (4 per thread) keep many CTAs in flight when
  // few rows are visible; on large row counts 4,096-row blocks (16 per
  // thread) are faster
  // the projection's 8-bit packed rects (views of at most 255 tiles per side)
  const unsigned* rect8 = rect8_fits(ct) ? proj->rect8 : nullptr;
  const bool small = n_rows <= (4ll << 20);
  const int items = small ? 4 : 16;
  const long long nb = (n_rows + kScanThreads * items - 1) / (kScanThreads * items);
  if (n_rows > 0) {
    // 1-2. stable depth sort of the visible rows (ties keep row order = id
    //    order) on the significant bits of their depth range; the first pass
    //    reads the rows (depth bits, visible when tiles_touched > 0), drops
    //    the culled ones, folds the range in and counts the visible rows
    const RadixRows rr{proj->depth, proj->tiles_touched, n_rows, n_vis};
    radix_sort(w.rk, w.rv, n_vis, n_rows, range, 32, w.hist, false, st, &rr);
    // 3. per row in depth order: super-tile offsets, the super-pair count Q
    //    and the pair count P
    //    (its last CTA: the scans of Q and P over the blocks, the capacity
    //    check and the reported count)
    if (small)
      rows_gather_kernel<4><<<(unsigned)nb, kScanThreads, 0, st>>>(
          rows_sorted, n_vis, proj->rect, rect8, N, ct, w.rect_sorted, arrive + 1, co);
    else
      rows_gather_kernel<16><<<(unsigned)nb, kScanThreads, 0, st>>>(
          rows_sorted, n_vis, proj->rect, rect8, N, ct, w.rect_sorted, arrive + 1, co);
    count_launches(1);
  } else {
    scan_counts_check_kernel<<<1, kScanThreads, 0, st>>>(co, 0);
    count_launches(1);
  }
  GS_TRY_CUDA(cudaGetLastError());
  long long p_bound = cap;
  if (num_pairs_host) {
    long long p_host = 0;
    GS_TRY_CUDA(cudaMemcpyAsync(&p_host, P, sizeof(long long), cudaMemcpyDeviceToHost, st));
    GS_TRY_CUDA(cudaStreamSynchronize(st));
    *num_pairs_host = p_host;
    if (p_host > cap) {
      GS_TRY_CUDA(cudaMemsetAsync(ranges, 0, 2 * sizeof(unsigned) * (size_t)T, st));
      return GS_ERR_CAPACITY;
    }
    p_bound = p_host;
  }
  if (n_rows == 0 || p_bound == 0 || S == 0) {
    GS_TRY_CUDA(cudaMemsetAsync(ranges, 0, 2 * sizeof(unsigned) * (size_t)T, st));
    return check_launch();
  }
  // 4. super-pairs (super-tile, row) in depth order of the rows, into the
  //    buffers that the super-tile sort leaves in (pk[res], pv)
  const int sbits = bits_for(S);
  const int spasses = radix_plan_bits(0u, sbits).passes;
  unsigned* sk[2] = {w.pk[0], w.pk[1]};
  unsigned* sv[2];
  if (spasses % 2 == 0) {
    sv[0] = w.pv;
    sv[1] = sorted_vals;
  } else {
    sv[0] = sorted_vals;
    sv[1] = w.pv;
  }
  const long long q_bound = p_bound;  // Q <= P
  // the rect descriptors ride in the keys' upper 16 bits when the super-tile
  // ids fit the lower 16 and every rect end fits the packed field
  int packed = S <= 65536 ? 1 : 0;
  for (int v = 0; v < ct.V; ++v)
    if (ct.c[v].TX > 8000 || ct.c[v].TY > 8000) packed = 0;
  // the expansion sums the super-tile sort's first-pass histogram as it
  // writes the items (positions below 2^31)
  const bool hist0 = q_bound < (1ll << 31);
  const int sgrid = radix_grid(q_bound);
  if (hist0)
    GS_TRY_CUDA(cudaMemsetAsync(w.hist, 0, sizeof(unsigned) * kRadixBins * (size_t)sgrid, st));
  {
    // (the scan blocks of rows_gather_kernel: their item bases are scanned)
    const int vec16 = (reinterpret_cast<uintptr_t>(sv[0]) % 16 == 0 &&
                       reinterpret_cast<uintptr_t>(sk[0]) % 16 == 0) ? 1 : 0;
    unsigned* h = hist0 ? w.hist : nullptr;
    const unsigned hmask = (1u << radix_plan_bits(0u, sbits).d0) - 1u;
    if (small)
      rows_expand_kernel<4><<<(unsigned)nb, kScanThreads, 0, st>>>(
          rows_sorted, w.rect_sorted, n_vis, w.block_sums, q_eff, N, div_magic_host((unsigned)N),
          ct, sk[0], sv[0], vec16, packed, h, sgrid, hmask);
    else
      rows_expand_kernel<16><<<(unsigned)nb, kScanThreads, 0, st>>>(
          rows_sorted, w.rect_sorted, n_vis, w.block_sums, q_eff, N, div_magic_host((unsigned)N),
          ct, sk[0], sv[0], vec16, packed, h, sgrid, hmask);
    count_launches(1);
  }
  // 5. stable sort of the super-pairs by super-tile id
  radix_sort(sk, sv, q_eff, q_bound, nullptr, sbits, w.hist, true, st, nullptr, hist0);
  const int sres = spasses & 1;
  const unsigned* sp_keys = sk[sres];
  const unsigned* sp_rows = sv[sres];  // == w.pv
  unsigned* desc = sk[1 - sres];
  // 6. rows of every super-tile (from the one-pass sort's digit totals, or
  //    marked on the sorted keys), segments, per-tile counts and list starts
  const unsigned* st_totals = nullptr;
  if (spasses == 1) {  // the digit totals are the per-super-tile item counts
    st_totals = w.hist + kRadixBins * radix_grid(q_bound);
  } else if (spasses > 1) {
    GS_TRY_CUDA(cudaMemsetAsync(w.st_ranges, 0, 2 * sizeof(unsigned) * (size_t)S, st));
    const unsigned gq = (unsigned)std::min<long long>((q_bound + 1023) / 1024, 152ll * 16);
    ranges_kernel<<<gq, 256, 0, st>>>(sp_keys, q_eff, packed ? 0xffffu : 0xffffffffu,
                                      w.st_ranges);
    count_launches(1);
  }
  st_segments_kernel<<<1, 1024, 0, st>>>(reinterpret_cast<uint2*>(w.st_ranges), S, st_totals,
                                         q_eff, w.seg_first, w.seg_st, n_seg);
  const unsigned gs = (unsigned)std::min<long long>(max_segments(q_bound, S), 152ll * 8);
  st_count_kernel<<<gs, 256, 0, st>>>(sp_keys, sp_rows,
                                      reinterpret_cast<const uint2*>(w.st_ranges), w.seg_first,
                                      w.seg_st, n_seg, packed, proj->rect, N, ct, desc,
                                      w.seg_hist);
  st_scan_kernel<<<(unsigned)S, 1024, 0, st>>>(w.seg_first, ct, w.seg_hist, w.tile_cnt,
                                                arrive + 2, w.tile_start, ranges);
  // 7. every row into the lists of the tiles it covers, in depth order
  {
    const int e = stage_event(GS_STAGE_EXPANSION, false, st);
    if (e != GS_OK) return e;
  }
  if (sorted_keys)
    st_emit_kernel<true><<<gs, 256, 0, st>>>(
        sp_keys, sp_rows, desc, packed, reinterpret_cast<const uint2*>(w.st_ranges), w.seg_first,
        w.seg_st, n_seg, w.seg_hist, w.tile_start, ct, proj->depth, sorted_vals, sorted_keys,
        cap);
  else
    st_emit_kernel<false><<<gs, 256, 0, st>>>(
        sp_keys, sp_rows, desc, packed, reinterpret_cast<const uint2*>(w.st_ranges), w.seg_first,
        w.seg_st, n_seg, w.seg_hist, w.tile_start, ct, proj->depth, sorted_vals, nullptr, cap);
  {
    const int e = stage_event(GS_STAGE_EXPANSION, true, st);
    if (e != GS_OK) return e;
  }
  count_launches(4);
  return check_launch();
}

// ----------------------------------------------------------------------------
// Tile queue: global tile ids ordered by list length, longest first.
// ----------------------------------------------------------------------------
namespace {
__global__ void queue_keys_kernel(const unsigned* __restrict__ ranges, long long T,
                                  unsigned* __restrict__ keys, unsigned* __restrict__ vals) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < T;
       t += (long long)gridDim.x * blockDim.x) {
    unsigned len = ranges[2 * t + 1] - ranges[2 * t];
    keys[t] = 0xffffffffu - len;
    vals[t] = (unsigned)t;
  }
}
}  // namespace

size_t tile_queue_workspace_size(long long T) {
  return align256(4 * (T + 1)) * 3 + align256(sizeof(long long) * 2) +
         align256(radix_hist_bytes());
}

int launch_tile_queue(const unsigned* ranges, long long T, unsigned* order, void* ws,
                      size_t ws_bytes, cudaStream_t st) {
  if (ws_bytes < tile_queue_workspace_size(T)) return GS_ERR_INVALID_ARG;
  if (T == 0) return GS_OK;
  char* p = reinterpret_cast<char*>(ws);
  unsigned* k0 = reinterpret_cast<unsigned*>(p);
  p += align256(4 * (T + 1));
  unsigned* k1 = reinterpret_cast<unsigned*>(p);
  p += align256(4 * (T + 1));
  unsigned* v1 = reinterpret_cast<unsigned*>(p);
  p += align256(4 * (T + 1));
  long long* n_dev = reinterpret_cast<long long*>(p);
  p += align256(sizeof(long long) * 2);
  unsigned* hist = reinterpret_cast<unsigned*>(p);
  set_value_kernel<<<1, 32, 0, st>>>(n_dev, T);
  count_launches(1);
  unsigned grid = (unsigned)std::min<long long>((T + 255) / 256, 1024);
  // 4 passes (even): the result ends in the first buffer, i.e. `order`
  queue_keys_kernel<<<grid, 256, 0, st>>>(ranges, T, k0, order);
  count_launches(1);
  unsigned* k[2] = {k0, k1};
  unsigned* v[2] = {order, v1};
  radix_sort(k, v, n_dev, T, nullptr, 32, hist, false, st);
  return check_launch();
}

}  // namespace gs

// ----------------------------------------------------------------------------
// Tile queue without allocation: the same sort, run in a fixed scratch array
// in device global memory that the library owns (see gs_tile_queue_static in
// include/gs.h).
// ----------------------------------------------------------------------------

// Scratch of the no-allocation tile queue, sized for
// GS_TILE_QUEUE_STATIC_MAX_TILES tiles with the layout of launch_tile_queue:
// three key/value arrays, the count, and the radix histograms.  Every GPU that
// loads the library holds these bytes until the process exits.
static __device__ __align__(256) unsigned char g_queue_scratch[
    ((4ull * (GS_TILE_QUEUE_STATIC_MAX_TILES + 1) + 255) / 256 * 256) * 3 + 256 +
    (gs::radix_hist_bytes() + 255) / 256 * 256];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_queue_scratch_mutex;
struct ScratchAddr {
  unsigned long long ctx_id;  // context the address belongs to (0: none yet)
  void* ptr;
};
ScratchAddr g_queue_scratch_addr[kMaxDevices] = {};

// Unique id of the calling thread's current CUDA context (ids are never
// reused within a process), through the driver entry points the runtime
// exposes; 0 when there is no current context or the query is unavailable.
unsigned long long current_context_id() {
  typedef CUresult (*GetCurrent)(CUcontext*);
  typedef CUresult (*GetId)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<GetCurrent>(f);
    f = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
            cudaSuccess && q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<GetId>(f);
    cudaGetLastError();
  });
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx ||
      get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of g_queue_scratch in the current device's context (in host
// code the array's name is only a stand-in, not a device address).  Looked
// up once per device and context: a device reset or a new primary context
// (the module is then loaded again, at another address) brings a new lookup.
int queue_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gs::set_cuda_error(e);
  if (dev < 0 || dev >= kMaxDevices)
    return gs::set_error_text_and_status("unsupported device index", GS_ERR_UNSUPPORTED);
  std::lock_guard<std::mutex> lock(g_queue_scratch_mutex);
  ScratchAddr& a = g_queue_scratch_addr[dev];
  unsigned long long ctx = current_context_id();
  if (!a.ptr || ctx == 0 || ctx != a.ctx_id) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_queue_scratch);  // makes the primary context current if needed
    if (e != cudaSuccess) return gs::set_cuda_error(e);
    if (ctx == 0) ctx = current_context_id();
    a.ptr = p;
    a.ctx_id = ctx;
  }
  *out = a.ptr;
  return GS_OK;
}

}  // namespace

extern "C" int gs_tile_queue_static(const unsigned* tile_ranges, long long total_tiles,
                                    unsigned* tile_order, gs_stream stream) {
  if (total_tiles < 0 || total_tiles > GS_TILE_QUEUE_STATIC_MAX_TILES) {
    char buf[160];
    snprintf(buf, sizeof buf,
             "invalid argument: gs_tile_queue_static supports at most %d tiles (got %lld)",
             GS_TILE_QUEUE_STATIC_MAX_TILES, total_tiles);
    return gs::set_error_text_and_status(buf, GS_ERR_INVALID_ARG);
  }
  if (total_tiles > 0 && (!tile_ranges || !tile_order))
    return gs::set_error_text_and_status("invalid argument: pointers", GS_ERR_INVALID_ARG);
  void* scratch = nullptr;
  const int rc = queue_scratch_address(&scratch);
  if (rc != GS_OK) return rc;
  // Nothing in the scratch needs to start at zero: each call writes every word
  // it reads (keys, values, histograms, the count) before reading it.
  return gs::launch_tile_queue(tile_ranges, total_tiles, tile_order, scratch,
                               sizeof(g_queue_scratch), (cudaStream_t)stream);
}
