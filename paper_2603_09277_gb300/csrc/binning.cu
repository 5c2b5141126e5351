// binning.cu -- per-tile Gaussian lists (Sec. 3: each pixel's list of the
// Gaussians that cover it, sorted by depth).
//
// The lists are the (tile, depth, id)-ordered pairs of every visible
// (view, Gaussian) row with every tile of its rect.  Instead of one sort
// of 64-bit (tile << 32 | depth) keys over all P pairs, the work is split
// so that the P-sized sort only carries the tile bits:
//   1. compact the visible rows (scan of a visibility flag);
//   2. stable LSD radix sort of the visible rows by FP32 depth bits
//      (N-sized: 4 passes of 8 bits over 8-byte items);
//   3. exclusive scan of tiles_touched in depth order -> pair offsets, P;
//   4. duplicate: each row writes (global tile, row) for its rect, in depth
//      order (so equal tiles appear in (depth, id) order);
//   5. stable LSD radix sort of the pairs by tile id, ceil(log2 tiles) bits;
//   6. per-tile [start, end) ranges from the sorted tile ids.
// The stable tile sort of depth-ordered pairs yields exactly the order of
// the 64-bit key sort with ties by Gaussian id.
//
// All kernels read their element counts from device memory and use grids
// sized from host-known upper bounds, so the whole sequence can be captured
// in a CUDA graph (no host synchronisation needed).  None of them waits on
// another block.
#include <algorithm>
#include <mutex>

#include "gs_internal.cuh"

namespace gs {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;                       // per thread
constexpr int kScanTile = kScanThreads * kScanItems; // 4096 items per block

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

// Value source for the scans: either tiles_touched[i] (or its gather through
// an index array) or a visibility flag.
struct ScanSrc {
  const unsigned* vals;   // values
  const unsigned* index;  // optional gather index (vals[index[i]])
  int flag;               // 1: use (value > 0) instead of the value
  __device__ __forceinline__ unsigned get(long long i) const {
    unsigned v = index ? vals[index[i]] : vals[i];
    return flag ? (v > 0u ? 1u : 0u) : v;
  }
};

// Phase 1: per-block sums.
__global__ void __launch_bounds__(kScanThreads) scan_reduce_kernel(ScanSrc src, const long long* n_dev,
                                                                   long long n_host,
                                                                   unsigned long long* block_sums) {
  long long n = n_dev ? *n_dev : n_host;
  long long base = (long long)blockIdx.x * kScanTile;
  unsigned long long s = 0;
  for (int k = 0; k < kScanItems; ++k) {
    long long i = base + (long long)k * kScanThreads + threadIdx.x;
    if (i < n) s += src.get(i);
  }
  unsigned long long tot;
  block_excl_scan(s, &tot);
  if (threadIdx.x == 0) block_sums[blockIdx.x] = tot;
}

// Phase 2: exclusive scan of the block sums in one block; writes the grand
// total to *total.
__global__ void __launch_bounds__(kScanThreads) scan_blocks_kernel(unsigned long long* block_sums,
                                                                   int nblocks,
                                                                   long long* total) {
  __shared__ unsigned long long s_carry;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < nblocks; base += kScanThreads) {
    int i = base + threadIdx.x;
    unsigned long long x = i < nblocks ? block_sums[i] : 0ull;
    unsigned long long tot;
    unsigned long long ex = block_excl_scan(x, &tot);
    if (i < nblocks) block_sums[i] = s_carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) s_carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = (long long)s_carry;
}

// Phase 3 (compaction form): rows with tiles_touched > 0 are written, in
// order, as (depth bits, row) to keys/vals.
__global__ void __launch_bounds__(kScanThreads) compact_visible_kernel(
    const unsigned* __restrict__ tiles_touched, const float* __restrict__ depth, long long n,
    const unsigned long long* __restrict__ block_offsets, unsigned* __restrict__ keys,
    unsigned* __restrict__ vals) {
  long long base = (long long)blockIdx.x * kScanTile;
  // each thread owns kScanItems consecutive items for an ordered compaction
  long long first = base + (long long)threadIdx.x * kScanItems;
  unsigned cnt = 0;
  for (int k = 0; k < kScanItems; ++k) {
    long long i = first + k;
    if (i < n && tiles_touched[i] > 0u) ++cnt;
  }
  unsigned long long tot;
  unsigned long long off = block_excl_scan(cnt, &tot) + block_offsets[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k) {
    long long i = first + k;
    if (i < n && tiles_touched[i] > 0u) {
      keys[off] = __float_as_uint(depth[i]);
      vals[off] = (unsigned)i;
      ++off;
    }
  }
}

// Phase 3 (offsets form): out[i] = exclusive prefix of tiles_touched in
// depth order (rows given by `rows`), for i < n_dev.
__global__ void __launch_bounds__(kScanThreads) scan_offsets_kernel(
    const unsigned* __restrict__ tiles_touched, const unsigned* __restrict__ rows,
    const long long* __restrict__ n_dev, const unsigned long long* __restrict__ block_offsets,
    unsigned long long* __restrict__ out) {
  long long n = *n_dev;
  long long base = (long long)blockIdx.x * kScanTile;
  long long first = base + (long long)threadIdx.x * kScanItems;
  if (base >= n) return;
  unsigned long long s = 0;
  unsigned loc[kScanItems];
  for (int k = 0; k < kScanItems; ++k) {
    long long i = first + k;
    loc[k] = i < n ? tiles_touched[rows[i]] : 0u;
    s += loc[k];
  }
  unsigned long long tot;
  unsigned long long off = block_excl_scan(s, &tot) + block_offsets[blockIdx.x];
  for (int k = 0; k < kScanItems; ++k) {
    long long i = first + k;
    if (i < n) out[i] = off;
    off += loc[k];
  }
}

// ----------------------------------------------------------------------------
// Stable LSD radix sort of (u32 key, u32 value) pairs, 8-bit digits,
// reduce-then-scan with a fixed grid.  Each block owns a contiguous chunk of
// whole 2048-item tiles; n is read from device memory.
// ----------------------------------------------------------------------------
constexpr int kRadixThreads = 256;
constexpr int kRadixWarps = kRadixThreads / 32;
constexpr int kRadixIpt = 8;                                // items per thread per tile
constexpr int kRadixTile = kRadixThreads * kRadixIpt;       // 2048
constexpr int kRadixBins = 256;

__device__ __forceinline__ long long radix_chunk(long long n, int nblocks) {
  long long per = (n + nblocks - 1) / nblocks;
  return (per + kRadixTile - 1) / kRadixTile * kRadixTile;
}

__global__ void __launch_bounds__(kRadixThreads) radix_upsweep_kernel(
    const unsigned* __restrict__ keys, const long long* __restrict__ n_dev, int shift,
    unsigned* __restrict__ hist /* [256][nblocks] */) {
  __shared__ unsigned s_h[kRadixWarps][kRadixBins];
  const int w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kRadixWarps * kRadixBins; i += kRadixThreads)
    (&s_h[0][0])[i] = 0u;
  __syncthreads();
  long long n = *n_dev;
  long long chunk = radix_chunk(n, gridDim.x);
  long long b0 = (long long)blockIdx.x * chunk;
  long long b1 = min(n, b0 + chunk);
  for (long long i = b0 + threadIdx.x; i < b1; i += kRadixThreads) {
    unsigned d = (keys[i] >> shift) & 0xffu;
    atomicAdd(&s_h[w][d], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadixBins; d += kRadixThreads) {
    unsigned s = 0;
    for (int k = 0; k < kRadixWarps; ++k) s += s_h[k][d];
    hist[(long long)d * gridDim.x + blockIdx.x] = s;
  }
}

// Per-digit exclusive scan over the blocks: block d scans hist[d][0..G) in
// place and writes the digit total to totals[d].  G <= 1024.
__global__ void __launch_bounds__(kScanThreads) radix_scan_kernel(unsigned* __restrict__ hist,
                                                                  int G,
                                                                  unsigned* __restrict__ totals) {
  unsigned* h = hist + (long long)blockIdx.x * G;
  constexpr int kPer = 4;  // 256 threads x 4 >= 1024 blocks
  unsigned loc[kPer];
  unsigned long long s = 0;
  const int first = threadIdx.x * kPer;
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    loc[k] = first + k < G ? h[first + k] : 0u;
    s += loc[k];
  }
  unsigned long long tot;
  unsigned long long off = block_excl_scan(s, &tot);
#pragma unroll
  for (int k = 0; k < kPer; ++k) {
    if (first + k < G) h[first + k] = (unsigned)off;
    off += loc[k];
  }
  if (threadIdx.x == 0) totals[blockIdx.x] = (unsigned)tot;
}

// Scatter of one radix pass.  Per 2048-item tile: digits ranked within each
// warp from bit ballots (stable within the tile), the tile is reordered by digit in shared
// memory, then written out so that consecutive threads store consecutive
// addresses of one digit's run (coalesced), and each digit's running global
// offset advances by the tile's count.
__global__ void __launch_bounds__(kRadixThreads) radix_downsweep_kernel(
    const unsigned* __restrict__ keys_in, const unsigned* __restrict__ vals_in,
    unsigned* __restrict__ keys_out, unsigned* __restrict__ vals_out,
    const long long* __restrict__ n_dev, int shift, const unsigned* __restrict__ offsets,
    const unsigned* __restrict__ totals) {
  __shared__ unsigned s_wc[kRadixWarps][kRadixBins + 1];  // per-warp digit counters (+ dummy)
  __shared__ unsigned s_base[kRadixBins];                 // running global offset per digit
  __shared__ unsigned s_tot[kRadixBins];                  // tile count per digit
  __shared__ unsigned s_off[kRadixBins];                  // tile-local start per digit
  __shared__ unsigned s_key[kRadixTile];
  __shared__ unsigned s_val[kRadixTile];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt_mask = (1u << lane) - 1u;
  long long n = *n_dev;
  long long chunk = radix_chunk(n, gridDim.x);
  long long b0 = (long long)blockIdx.x * chunk;
  long long b1 = min(n, b0 + chunk);
  {
    // digit base = exclusive scan of the digit totals (256 threads, one digit each)
    unsigned long long tot;
    unsigned long long db = block_excl_scan(totals[threadIdx.x], &tot);
    s_base[threadIdx.x] = (unsigned)db + offsets[(long long)threadIdx.x * gridDim.x + blockIdx.x];
  }
  for (int i = threadIdx.x; i < kRadixWarps * (kRadixBins + 1); i += kRadixThreads)
    (&s_wc[0][0])[i] = 0u;
  __syncthreads();
  for (long long t0 = b0; t0 < b1; t0 += kRadixTile) {
    const int cnt = (int)min((long long)kRadixTile, b1 - t0);
    unsigned k[kRadixIpt], v[kRadixIpt], dg[kRadixIpt], loc[kRadixIpt];
#pragma unroll
    for (int i = 0; i < kRadixIpt; ++i) {
      const int li = w * (32 * kRadixIpt) + i * 32 + lane;
      const bool ok = li < cnt;
      k[i] = ok ? keys_in[t0 + li] : 0u;
      v[i] = ok ? vals_in[t0 + li] : 0u;
      dg[i] = ok ? ((k[i] >> shift) & 0xffu) : (unsigned)kRadixBins;
    }
#pragma unroll
    for (int i = 0; i < kRadixIpt; ++i) {
      // lanes holding the same digit: one ballot per digit bit plus validity
      const bool valid = dg[i] < (unsigned)kRadixBins;
      const unsigned vm = __ballot_sync(0xffffffffu, valid);
      unsigned peers = valid ? vm : ~vm;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const bool bit = (dg[i] >> b) & 1u;
        const unsigned m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
      }
      unsigned rank = __popc(peers & lt_mask);
      unsigned base = s_wc[w][dg[i]];
      __syncwarp();
      if (rank == 0) s_wc[w][dg[i]] = base + __popc(peers);
      __syncwarp();
      loc[i] = base + rank;
    }
    __syncthreads();
    {
      // per digit (one per thread): prefix over warps, tile count, tile-local start
      const int d = threadIdx.x;
      unsigned run = 0;
      for (int ww = 0; ww < kRadixWarps; ++ww) {
        unsigned c = s_wc[ww][d];
        s_wc[ww][d] = run;
        run += c;
      }
      s_tot[d] = run;
      unsigned long long tt;
      s_off[d] = (unsigned)block_excl_scan(run, &tt);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kRadixIpt; ++i) {
      if (dg[i] < (unsigned)kRadixBins) {
        const unsigned lp = s_off[dg[i]] + s_wc[w][dg[i]] + loc[i];
        s_key[lp] = k[i];
        s_val[lp] = v[i];
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < cnt; i += kRadixThreads) {
      const unsigned kk = s_key[i];
      const unsigned d = (kk >> shift) & 0xffu;
      const unsigned pos = s_base[d] + (unsigned)i - s_off[d];
      keys_out[pos] = kk;
      vals_out[pos] = s_val[i];
    }
    __syncthreads();
    {
      const int d = threadIdx.x;
      s_base[d] += s_tot[d];
      for (int ww = 0; ww < kRadixWarps; ++ww) s_wc[ww][d] = 0u;
      if (d < kRadixWarps) s_wc[d][kRadixBins] = 0u;
    }
    __syncthreads();
  }
}

// ----------------------------------------------------------------------------
// Pair generation, ranges, capacity check.
// ----------------------------------------------------------------------------
__global__ void capacity_check_kernel(const long long* __restrict__ P, long long capacity,
                                      int* __restrict__ status, long long* __restrict__ p_eff) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    bool over = *P > capacity;
    *status = over ? GS_ERR_CAPACITY : GS_OK;
    *p_eff = over ? 0 : *P;  // on overflow every later stage sees zero pairs
  }
}

// Pair duplication, load-balanced over pairs.  The depth-sorted visible rows
// own contiguous pair ranges [offset_j, offset_j + tiles_j).  Pairs are cut
// into blocks of kDupPairs; mark_block_starts records, for every block, the row
// that owns its first pair (each block boundary lies in exactly one row), and
// duplicate_kernel then has each CTA load the descriptors of the rows that
// overlap its pairs into shared memory and find the row of each of its pairs
// by binary search there.  Every CTA writes kDupPairs consecutive pairs with
// coalesced stores, however the tile counts are distributed over the rows.
constexpr int kDupThreads = 256;
constexpr int kDupPairs = 1024;

__global__ void __launch_bounds__(256) mark_block_starts_kernel(
    const unsigned* __restrict__ rows, const long long* __restrict__ n_vis,
    const unsigned long long* __restrict__ offsets, const unsigned* __restrict__ tiles_touched,
    const long long* __restrict__ p_eff, unsigned* __restrict__ block_row) {
  const long long n = *n_vis;
  if (*p_eff == 0) return;
  for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const unsigned long long o = offsets[j];
    const unsigned long long c = tiles_touched[rows[j]];
    for (unsigned long long b = (o + kDupPairs - 1) / kDupPairs; b * kDupPairs < o + c; ++b)
      block_row[b] = (unsigned)j;
  }
}

__global__ void __launch_bounds__(kDupThreads) duplicate_kernel(
    const unsigned* __restrict__ rows, const long long* __restrict__ n_vis,
    const unsigned long long* __restrict__ offsets, const int* __restrict__ rect, int N,
    const CamTable ct, const long long* __restrict__ p_eff,
    const unsigned* __restrict__ block_row, unsigned* __restrict__ tkeys,
    unsigned* __restrict__ tvals) {
  __shared__ long long s_off[kDupPairs];  // row pair offset relative to the block start
  __shared__ int4 s_rect[kDupPairs];
  __shared__ unsigned s_row[kDupPairs];
  __shared__ int s_nrows;
  const long long P = *p_eff;
  const long long start = (long long)blockIdx.x * kDupPairs;
  if (start >= P) return;
  const long long end = min(P, start + kDupPairs);
  const long long n = *n_vis;
  const long long j0 = block_row[blockIdx.x];
  // rows j0 .. j1 overlap [start, end): j1 is the row holding the next block's
  // first pair (it belongs here only if it starts before `end`), or the last row
  const long long j1 = (end < P) ? (long long)block_row[blockIdx.x + 1] : n - 1;
  const int cand = (int)min((long long)kDupPairs, j1 - j0 + 1);
  for (int i = threadIdx.x; i < cand; i += kDupThreads) {
    const long long j = j0 + i;
    const unsigned long long o = offsets[j];
    if ((long long)o < end) {
      const unsigned row = rows[j];
      s_off[i] = (long long)o - start;  // negative for a row that began before the block
      s_rect[i] = reinterpret_cast<const int4*>(rect)[row];
      s_row[i] = row;
    }
  }
  if (threadIdx.x == 0)
    s_nrows = (j1 - j0 + 1 <= kDupPairs && (long long)offsets[j1] < end) ? (int)(j1 - j0 + 1)
                                                                         : (int)(j1 - j0);
  __syncthreads();
  const int nr = s_nrows;
  for (int t = threadIdx.x; t < (int)(end - start); t += kDupThreads) {
    int lo = 0, hi = nr - 1;  // last row with s_off <= t
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (s_off[mid] <= (long long)t) lo = mid; else hi = mid - 1;
    }
    const int4 r = s_rect[lo];
    const unsigned rw = s_row[lo];
    const int k = (int)((long long)t - s_off[lo]);
    const int w = r.z - r.x;
    const CamInfo& c = ct.c[(int)(rw / (unsigned)N)];
    const int ty = r.y + k / w, tx = r.x + k % w;
    tkeys[start + t] = (unsigned)(c.tile_off + ty * c.TX + tx);
    tvals[start + t] = rw;
  }
}

// Per-tile [start, end) from the sorted tile ids: each thread reads 4
// consecutive ids with one 16-byte load (the array is 256-byte aligned) plus
// its neighbours, and marks where the id changes.
__global__ void __launch_bounds__(256) ranges_kernel(const unsigned* __restrict__ tkeys,
                                                     const long long* __restrict__ p_eff,
                                                     unsigned* __restrict__ ranges) {
  const long long P = *p_eff;
  const long long groups = (P + 3) / 4;
  for (long long g = (long long)blockIdx.x * blockDim.x + threadIdx.x; g < groups;
       g += (long long)gridDim.x * blockDim.x) {
    const long long i0 = 4 * g;
    unsigned k[6];
    if (i0 + 3 < P) {
      const uint4 v = reinterpret_cast<const uint4*>(tkeys)[g];
      k[1] = v.x; k[2] = v.y; k[3] = v.z; k[4] = v.w;
    } else {
      for (int q = 0; q < 4; ++q) k[1 + q] = i0 + q < P ? tkeys[i0 + q] : 0u;
    }
    k[0] = i0 > 0 ? tkeys[i0 - 1] : 0xffffffffu;
    k[5] = i0 + 4 < P ? tkeys[i0 + 4] : 0xffffffffu;
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

__global__ void __launch_bounds__(256) keys64_kernel(const unsigned* __restrict__ tkeys,
                                                     const unsigned* __restrict__ tvals,
                                                     const float* __restrict__ depth,
                                                     const long long* __restrict__ p_eff,
                                                     unsigned long long* __restrict__ out) {
  long long P = *p_eff;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < P;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = ((unsigned long long)tkeys[i] << 32) | __float_as_uint(depth[tvals[i]]);
}

__global__ void set_count_kernel(long long* __restrict__ dst, const long long* __restrict__ src) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *dst = *src;
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
  long long* counters;             // [0] n_vis, [1] P, [2] P effective
  unsigned* rk[2];                 // row keys (depth bits), double buffer
  unsigned* rv[2];                 // row values, double buffer
  unsigned long long* offsets;     // pair offsets per visible row
  unsigned* pk[2];                 // pair keys (tile), double buffer; pk[1] may alias output
  unsigned* pv;                    // pair values scratch
  unsigned* hist;                  // radix histograms
  unsigned* block_row;             // first row of every duplication block
  size_t bytes;
};

constexpr int kRadixGrid = 4 * 152;  // fixed radix grid (4 CTAs per SM)

inline long long scan_blocks(long long n) { return (n + kScanTile - 1) / kScanTile; }

Workspace carve(void* base, long long n_rows, long long cap) {
  Workspace w;
  char* p = reinterpret_cast<char*>(base);
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* r = p ? p + off : nullptr;
    off += align256(bytes);
    return r;
  };
  long long nb = scan_blocks(n_rows > cap ? n_rows : cap) + 1;
  w.block_sums = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * nb));
  w.counters = reinterpret_cast<long long*>(take(sizeof(long long) * 4));
  for (int i = 0; i < 2; ++i) w.rk[i] = reinterpret_cast<unsigned*>(take(4 * (n_rows + 1)));
  for (int i = 0; i < 2; ++i) w.rv[i] = reinterpret_cast<unsigned*>(take(4 * (n_rows + 1)));
  w.offsets = reinterpret_cast<unsigned long long*>(take(8 * (n_rows + 1)));
  for (int i = 0; i < 2; ++i) w.pk[i] = reinterpret_cast<unsigned*>(take(4 * (cap + 1)));
  w.pv = reinterpret_cast<unsigned*>(take(4 * (cap + 1)));
  w.hist = reinterpret_cast<unsigned*>(take(4ull * kRadixBins * (kRadixGrid + 1)));
  w.block_row = reinterpret_cast<unsigned*>(take(4ull * ((cap + kDupPairs - 1) / kDupPairs + 1)));
  w.bytes = off;
  return w;
}

// Runs the radix passes over bits [0, bits) of keys; data starts in
// (k[0], v[0]) and ends in (k[res], v[res]); returns res.
int radix_sort(unsigned* k[2], unsigned* v[2], const long long* n_dev, long long n_bound, int bits,
               unsigned* hist, cudaStream_t st) {
  int cur = 0;
  if (n_bound == 0) return cur;
  int grid = (int)std::min<long long>(kRadixGrid, (n_bound + kRadixTile - 1) / kRadixTile);
  if (grid < 1) grid = 1;
  for (int shift = 0; shift < bits; shift += 8) {
    radix_upsweep_kernel<<<grid, kRadixThreads, 0, st>>>(k[cur], n_dev, shift, hist);
    radix_scan_kernel<<<kRadixBins, kScanThreads, 0, st>>>(hist, grid, hist + kRadixBins * grid);
    radix_downsweep_kernel<<<grid, kRadixThreads, 0, st>>>(k[cur], v[cur], k[1 - cur], v[1 - cur],
                                                           n_dev, shift, hist,
                                                           hist + kRadixBins * grid);
    count_launches(3);
    cur = 1 - cur;
  }
  return cur;
}

int bits_for(long long count) {
  int b = 0;
  while (b < 32 && (1ll << b) < count) ++b;
  return b;
}

}  // namespace

size_t bin_sort_workspace_size(long long n_rows, long long cap, long long total_tiles) {
  (void)total_tiles;
  return carve(nullptr, n_rows, cap).bytes;
}

int launch_bin_sort(const gs_proj* proj, int N, const CamTable& ct, void* workspace,
                    size_t ws_bytes, long long cap, unsigned* sorted_vals,
                    unsigned long long* sorted_keys, unsigned* ranges, long long* num_pairs_dev,
                    long long* num_pairs_host, int* status_dev, cudaStream_t st) {
  const long long n_rows = (long long)N * ct.V;
  Workspace w = carve(workspace, n_rows, cap);
  if (ws_bytes < w.bytes) return GS_ERR_INVALID_ARG;
  long long* n_vis = w.counters;
  long long* P = w.counters + 1;
  long long* p_eff = w.counters + 2;
  GS_TRY_CUDA(cudaMemsetAsync(w.counters, 0, 4 * sizeof(long long), st));
  GS_TRY_CUDA(cudaMemsetAsync(ranges, 0, 2 * sizeof(unsigned) * (size_t)ct.total_tiles, st));
  unsigned* rows_sorted = w.rv[0];
  const long long nb = scan_blocks(n_rows);
  if (n_rows > 0) {
    // 1. compaction of the visible rows, keyed by FP32 depth bits
    ScanSrc vis{proj->tiles_touched, nullptr, 1};
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(vis, nullptr, n_rows, w.block_sums);
    scan_blocks_kernel<<<1, kScanThreads, 0, st>>>(w.block_sums, (int)nb, n_vis);
    compact_visible_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(
        proj->tiles_touched, proj->depth, n_rows, w.block_sums, w.rk[0], w.rv[0]);
    // 2. stable depth sort of the visible rows (ties keep row order = id order)
    int res = radix_sort(w.rk, w.rv, n_vis, n_rows, 32, w.hist, st);
    rows_sorted = w.rv[res];
    // 3. pair offsets in depth order and the pair count P
    ScanSrc tt{proj->tiles_touched, rows_sorted, 0};
    scan_reduce_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(tt, n_vis, 0, w.block_sums);
    scan_blocks_kernel<<<1, kScanThreads, 0, st>>>(w.block_sums, (int)nb, P);
    scan_offsets_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(proj->tiles_touched, rows_sorted,
                                                               n_vis, w.block_sums, w.offsets);
    count_launches(6);
  }
  capacity_check_kernel<<<1, 32, 0, st>>>(P, cap, status_dev, p_eff);
  set_count_kernel<<<1, 32, 0, st>>>(num_pairs_dev, P);
  count_launches(2);
  GS_TRY_CUDA(cudaGetLastError());
  long long p_bound = cap;
  if (num_pairs_host) {
    long long p_host = 0;
    GS_TRY_CUDA(cudaMemcpyAsync(&p_host, P, sizeof(long long), cudaMemcpyDeviceToHost, st));
    GS_TRY_CUDA(cudaStreamSynchronize(st));
    *num_pairs_host = p_host;
    if (p_host > cap) return GS_ERR_CAPACITY;
    p_bound = p_host;
  }
  if (n_rows == 0 || p_bound == 0) return check_launch();
  // 4. duplicate in depth order, into the buffer pair the last tile pass
  //    reads from so that the sorted values end in sorted_vals
  const int tbits = bits_for(ct.total_tiles);
  const int passes = (tbits + 7) / 8;
  unsigned* pk[2] = {w.pk[0], w.pk[1]};
  unsigned* pv[2];
  if (passes % 2 == 0) {
    pv[0] = sorted_vals;
    pv[1] = w.pv;
  } else {
    pv[0] = w.pv;
    pv[1] = sorted_vals;
  }
  {
    const unsigned g1 = (unsigned)std::min<long long>((n_rows + 255) / 256, 152ll * 32);
    mark_block_starts_kernel<<<g1, 256, 0, st>>>(rows_sorted, n_vis, w.offsets,
                                                proj->tiles_touched, p_eff, w.block_row);
    const unsigned g2 = (unsigned)((p_bound + kDupPairs - 1) / kDupPairs);
    duplicate_kernel<<<g2, kDupThreads, 0, st>>>(rows_sorted, n_vis, w.offsets, proj->rect, N, ct,
                                                p_eff, w.block_row, pk[0], pv[0]);
    count_launches(2);
  }
  // 5. stable sort of the pairs by global tile id
  int res2 = radix_sort(pk, pv, p_eff, p_bound, tbits, w.hist, st);
  // 6. per-tile ranges (and the optional 64-bit keys)
  unsigned grid = (unsigned)std::min<long long>((p_bound + 255) / 256, 152ll * 16);
  ranges_kernel<<<grid, 256, 0, st>>>(pk[res2], p_eff, ranges);
  count_launches(1);
  if (sorted_keys) {
    keys64_kernel<<<grid, 256, 0, st>>>(pk[res2], pv[res2], proj->depth, p_eff, sorted_keys);
    count_launches(1);
  }
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
         align256(4ull * kRadixBins * (kRadixGrid + 1));
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
  radix_sort(k, v, n_dev, T, 32, hist, st);
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
    (4ull * gs::kRadixBins * (gs::kRadixGrid + 1) + 255) / 256 * 256];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_queue_scratch_mutex;
void* g_queue_scratch_ptr[kMaxDevices] = {};

// Device address of g_queue_scratch on the current device, looked up once per
// device (in host code the array's name is only a stand-in, not a device
// address).
int queue_scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return gs::set_cuda_error(e);
  if (dev < 0 || dev >= kMaxDevices)
    return gs::set_error_text_and_status("unsupported device index", GS_ERR_UNSUPPORTED);
  std::lock_guard<std::mutex> lock(g_queue_scratch_mutex);
  if (!g_queue_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_queue_scratch);
    if (e != cudaSuccess) return gs::set_cuda_error(e);
    g_queue_scratch_ptr[dev] = p;
  }
  *out = g_queue_scratch_ptr[dev];
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
