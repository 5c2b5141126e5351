// api.cu -- the extern "C" entry points of include/gs.h: argument checks,
// per-call camera tables, and the small kernels that do not belong to a
// larger stage (loss, scale reset).
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <mutex>

#include "gs_internal.cuh"

namespace gs {

// Stage launchers defined in the other translation units.
int launch_preprocess(const float* means, const float* log_scales, const float* quats,
                      const float* opacity_logits, const float* sh, int N, const CamTable& ct,
                      const gs_params* prm, const gs_proj* out, cudaStream_t st);
int launch_preprocess_bwd(const float* means, const float* log_scales, const float* quats,
                          const float* opacity_logits, const float* sh, int N, const CamTable& ct,
                          const gs_params* prm, const unsigned* tiles_touched, const float* grad2d,
                          float* g_means, float* g_ls, float* g_quats, float* g_opac, float* g_sh,
                          cudaStream_t st);
int launch_adjoint_list(const unsigned* tiles_touched, int N, int V, float* grad2d,
                        cudaStream_t st);
int launch_grad2d_attributes(const gs_proj* proj, long long rows, const gs_params* prm,
                             const float* grad2d, float* out, cudaStream_t st);
size_t bin_sort_workspace_size(long long n_rows, long long cap, long long total_tiles);
size_t ssim_workspace_bytes(long long total_pixels);
int ssim_blocks(const CamTable& ct);
int launch_ssim(const float* image, const float* target, const CamTable& ct, float lambda,
                float* maps, double* partials, float* dimg, cudaStream_t st);
int launch_bin_sort(const gs_proj* proj, int N, const CamTable& ct, void* workspace,
                    size_t ws_bytes, long long cap, unsigned* sorted_vals,
                    unsigned long long* sorted_keys, unsigned* ranges, long long* num_pairs_dev,
                    long long* num_pairs_host, int* status_dev, cudaStream_t st);
size_t tile_queue_workspace_size(long long T);
int launch_tile_queue(const unsigned* ranges, long long T, unsigned* order, void* ws,
                      size_t ws_bytes, cudaStream_t st);
int launch_render_fwd(const gs_proj* proj, long long rows, const CamTable& ct,
                      const gs_params* prm, const unsigned* vals, const unsigned* ranges,
                      float* image, float* final_T, unsigned* last_idx, float* entropy,
                      const gs_launch* opt, cudaStream_t st);
int launch_render_bwd(const gs_proj* proj, long long rows, const CamTable& ct,
                      const gs_params* prm, const unsigned* vals, const unsigned* ranges,
                      const float* final_T, const unsigned* last_idx, const float* dL_dimage,
                      const float* dL_dentropy, float* grad2d, const gs_launch* opt,
                      cudaStream_t st);
int bounds_status_render(unsigned* out, bool clear);
int bounds_status_binning(unsigned* out, bool clear);
int bounds_status_preprocess(unsigned* out, bool clear);

namespace {
thread_local char g_err[512] = "";
unsigned long long g_launches = 0;

void set_error_text(const char* msg) {
  strncpy(g_err, msg, sizeof(g_err) - 1);
  g_err[sizeof(g_err) - 1] = 0;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

int invalid(const char* what) {
  char buf[512];
  snprintf(buf, sizeof buf, "invalid argument: %s", what);
  set_error_text(buf);
  return GS_ERR_INVALID_ARG;
}

// A second stream per device for work a call can run beside its own kernels.
// The call forks it from the caller's stream with an event and joins it back
// before the dependent kernel, so the ordering on the caller's stream is
// unchanged and a stream capture records the side work as a parallel branch.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  bool tried = false, ok = false;
};
constexpr int kMaxDevices = 64;
SideStream g_side[kMaxDevices];
std::mutex g_side_mu;  // guards g_side and every fork..join sequence

// The current device's side stream, or nullptr (then the call stays on one
// stream).  It is created on first use outside a stream capture.
SideStream* side_stream_locked(cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  SideStream& ss = g_side[dev];
  if (!ss.tried) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone)
      return nullptr;
    ss.tried = true;
    ss.ok = cudaStreamCreateWithFlags(&ss.s, cudaStreamNonBlocking) == cudaSuccess &&
            cudaEventCreateWithFlags(&ss.fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaEventCreateWithFlags(&ss.join, cudaEventDisableTiming) == cudaSuccess;
  }
  return ss.ok ? &ss : nullptr;
}
}  // namespace

namespace {
thread_local void* g_stage_ev[4][2] = {};
}  // namespace

int stage_event(int stage, bool end, cudaStream_t st) {
  if (stage < 1 || stage > 3) return GS_OK;
  void* ev = g_stage_ev[stage][end ? 1 : 0];
  if (!ev) return GS_OK;
  GS_TRY_CUDA(cudaEventRecord(reinterpret_cast<cudaEvent_t>(ev), st));
  return GS_OK;
}

int set_error_text_and_status(const char* msg, int status) {
  set_error_text(msg);
  return status;
}

int set_cuda_error(cudaError_t e) {
  char buf[512];
  snprintf(buf, sizeof buf, "CUDA error %d: %s", (int)e, cudaGetErrorString(e));
  set_error_text(buf);
  return GS_ERR_CUDA;
}

void count_launches(int n) { __atomic_fetch_add(&g_launches, (unsigned long long)n, __ATOMIC_RELAXED); }

int check_launch() {
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GS_OK : set_cuda_error(e);
}

bool build_cam_table(const gs_camera* cams, int V, const gs_params* prm, int tile, CamTable* ct) {
  if (!cams || V < 1 || V > GS_MAX_VIEWS) return false;
  if (tile == 0) tile = kTile;
  if (tile != 16 && tile != 8) return false;
  memset(ct, 0, sizeof(*ct));
  ct->V = V;
  ct->tile = tile;
  long long tiles = 0, pix = 0, sts = 0;
  const float fovc = prm ? prm->fov_clamp : 1.3f;
  for (int v = 0; v < V; ++v) {
    const gs_camera& c = cams[v];
    if (c.width <= 0 || c.height <= 0 || !(c.fx > 0.f) || !(c.fy > 0.f)) return false;
    CamInfo& d = ct->c[v];
    for (int r = 0; r < 3; ++r) {
      for (int j = 0; j < 3; ++j) d.R[r * 3 + j] = c.world_to_cam[r * 4 + j];
      d.t[r] = c.world_to_cam[r * 4 + 3];
      d.cp[r] = c.cam_pos[r];
    }
    d.fx = c.fx; d.fy = c.fy; d.cx = c.cx; d.cy = c.cy;
    d.limx = fovc * (0.5f * (float)c.width / c.fx);
    d.limy = fovc * (0.5f * (float)c.height / c.fy);
    d.W = c.width; d.H = c.height;
    d.TX = (c.width + tile - 1) / tile;
    d.TY = (c.height + tile - 1) / tile;
    if (d.TX > 65535 || d.TY > 65535) return false;  // tile rects travel in 16-bit fields
    d.STX = (d.TX + kSuperTile - 1) / kSuperTile;
    d.STY = (d.TY + kSuperTile - 1) / kSuperTile;
    d.st_off = (int)sts;
    d.tile_off = (int)tiles;
    d.pix_off = pix;
    sts += (long long)d.STX * d.STY;
    tiles += (long long)d.TX * d.TY;
    pix += (long long)c.width * c.height;
    if (tiles >= (1ll << 31)) return false;
  }
  ct->total_tiles = (int)tiles;
  ct->total_st = (int)sts;
  return true;
}

RenderConsts render_consts(const gs_params* prm) {
  RenderConsts rc;
  rc.alpha_max = prm->alpha_max;
  rc.alpha_min = prm->alpha_min;
  rc.log2_alpha_min = log2f(prm->alpha_min);
  rc.t_min = prm->t_min;
  return rc;
}

namespace {

bool params_ok(const gs_params* p) {
  if (!p) return false;
  if (p->sh_degree < 0 || p->sh_degree > 3) return false;
  int K = (p->sh_degree + 1) * (p->sh_degree + 1);
  if (p->sh_stride < K || p->sh_stride > GS_SH_COEFFS_MAX) return false;
  if (p->sh_layout != 0 && p->sh_layout != 1) return false;
  if (p->attr_dtype < GS_ATTR_F32 || p->attr_dtype > GS_ATTR_BF16) return false;
  if (!(p->alpha_max > 0.f && p->alpha_max < 1.f)) return false;
  if (!(p->alpha_min > 0.f && p->alpha_min < p->alpha_max)) return false;
  if (!(p->t_min > 0.f && p->t_min < 1.f)) return false;
  if (!(p->dilation >= 0.f) || !(p->near_z > 0.f) || !(p->fov_clamp > 0.f)) return false;
  if (p->tile_size != 0 && p->tile_size != 8 && p->tile_size != 16) return false;
  return true;
}

bool proj_ok(const gs_proj* p, bool need_records) {
  if (!p || !p->depth || !p->tiles_touched) return false;
  if (!p->rect && !p->rect8) return false;
  if (need_records && (!p->records || !aligned(p->records, 16))) return false;
  if (p->rect && !aligned(p->rect, 16)) return false;
  if (p->mean2d && !aligned(p->mean2d, 8)) return false;
  if (p->conic_opacity && !aligned(p->conic_opacity, 16)) return false;
  return true;
}

// ---------------------------------------------------------------------------
// Loss kernels: per-pixel L1 + gamma H contributions with their gradients,
// block partial sums in double, then one block sums the partials in a fixed
// order (deterministic).
// ---------------------------------------------------------------------------
constexpr int kLossThreads = 256;
constexpr int kLossMaxBlocks = 1024;

struct LossViews {
  int V;
  long long pix_off[GS_MAX_VIEWS];
  float g_img[GS_MAX_VIEWS];  // 1 / (3 M_v V): |dL/dC| per channel
  float g_ent[GS_MAX_VIEWS];  // gamma / (M_v V)
  float w[GS_MAX_VIEWS];      // 1 / (M_v V)
};

// One pixel of the L1 + entropy loss: writes dL/dC (3 floats) and dL/dH,
// returns the pixel's term (1/(M_v V)) ((1 - lambda) |r|_1 / 3 + gamma H).
__device__ __forceinline__ float loss_pixel(const LossViews& lv, int v, float gamma,
                                            float l1_weight, const float c[3], const float t[3],
                                            float h, float g[3], float& gh) {
  float l1 = 0.f;
#pragma unroll
  for (int ch = 0; ch < 3; ++ch) {
    const float r = c[ch] - t[ch];
    l1 += fabsf(r);
    g[ch] = r > 0.f ? lv.g_img[v] : (r < 0.f ? -lv.g_img[v] : 0.f);
  }
  gh = lv.g_ent[v];
  return lv.w[v] * __fmaf_rn(l1_weight * (1.f / 3.f), l1, gamma * h);
}

__device__ __forceinline__ int view_of_pixel(const LossViews& lv, long long i) {
  int v = 0;
  while (v + 1 < lv.V && i >= lv.pix_off[v + 1]) ++v;
  return v;
}

// Every term is >= 0: a thread's few terms and the warp's 32 partials are
// summed in FP32 (relative error below 1e-6), the warps and blocks in FP64.
// (FP64 arithmetic runs at a small fraction of the FP32 rate here.)  With
// vec (every array 16-byte aligned) a thread takes 4 pixels at a time with
// 16-byte loads and stores; the last P mod 4 pixels go through block 0.
__global__ void __launch_bounds__(kLossThreads) loss_kernel(
    const float* __restrict__ image, const float* __restrict__ target,
    const float* __restrict__ entropy, const LossViews lv, long long P, float gamma,
    float l1_weight, float* __restrict__ dimg, float* __restrict__ dent,
    double* __restrict__ partials, int vec) {
  float acc = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long done = 0;
  if (vec) {
    const long long Q4 = P / 4;
    for (long long k = t0; k < Q4; k += stride) {
      const float4* ci = reinterpret_cast<const float4*>(image) + 3 * k;
      const float4* ti = reinterpret_cast<const float4*>(target) + 3 * k;
      const float4 c0 = ci[0], c1 = ci[1], c2 = ci[2];
      const float4 u0 = ti[0], u1 = ti[1], u2 = ti[2];
      const float4 hh = entropy ? reinterpret_cast<const float4*>(entropy)[k]
                                : make_float4(0.f, 0.f, 0.f, 0.f);
      const float cc[12] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w, c2.x, c2.y, c2.z, c2.w};
      const float tt[12] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w, u2.x, u2.y, u2.z, u2.w};
      const float hv[4] = {hh.x, hh.y, hh.z, hh.w};
      float gg[12], gh[4];
      const int v0 = view_of_pixel(lv, 4 * k);
      const bool one_view = v0 + 1 >= lv.V || 4 * k + 3 < lv.pix_off[v0 + 1];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int v = one_view ? v0 : view_of_pixel(lv, 4 * k + j);
        acc += loss_pixel(lv, v, gamma, l1_weight, cc + 3 * j, tt + 3 * j, hv[j], gg + 3 * j, gh[j]);
      }
      float4* gi = reinterpret_cast<float4*>(dimg) + 3 * k;
      gi[0] = make_float4(gg[0], gg[1], gg[2], gg[3]);
      gi[1] = make_float4(gg[4], gg[5], gg[6], gg[7]);
      gi[2] = make_float4(gg[8], gg[9], gg[10], gg[11]);
      if (dent) reinterpret_cast<float4*>(dent)[k] = make_float4(gh[0], gh[1], gh[2], gh[3]);
    }
    done = 4 * Q4;
  }
  // scalar pixels: all of them without vec, else the last P mod 4 (block 0)
  const long long s0 = vec ? (blockIdx.x == 0 ? done + threadIdx.x : P) : t0;
  const long long sstep = vec ? (long long)blockDim.x : stride;
  for (long long i = s0; i < P; i += sstep) {
    const int v = view_of_pixel(lv, i);
    const float c[3] = {image[3 * i], image[3 * i + 1], image[3 * i + 2]};
    const float t[3] = {target[3 * i], target[3 * i + 1], target[3 * i + 2]};
    float g[3], gh;
    acc += loss_pixel(lv, v, gamma, l1_weight, c, t, entropy ? entropy[i] : 0.f, g, gh);
    dimg[3 * i] = g[0];
    dimg[3 * i + 1] = g[1];
    dimg[3 * i + 2] = g[2];
    if (dent) dent[i] = gh;
  }
  __shared__ double s[kLossThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = (double)acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < kLossThreads / 32; ++k) t += s[k];
    partials[blockIdx.x] = t;
  }
}

// Sums the block partials in a fixed order: thread t adds partials t, t+256,
// ..., then a fixed shuffle tree and a fixed sum over the 8 warps.
__global__ void __launch_bounds__(kLossThreads) loss_finalize_kernel(
    const double* __restrict__ partials, int n, double* __restrict__ out) {
  double t = 0.0;
  for (int i = threadIdx.x; i < n; i += kLossThreads) t += partials[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  __shared__ double s[kLossThreads / 32];
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int k = 0; k < kLossThreads / 32; ++k) r += s[k];
    *out = r;
  }
}

// log s += ln(zeta), 16-byte accesses for the aligned body.
__global__ void scale_reset_kernel(float* __restrict__ ls, long long n, float delta) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long head = (long long)((16 - (reinterpret_cast<uintptr_t>(ls) & 15)) & 15) / 4;
  if ((reinterpret_cast<uintptr_t>(ls) & 3) != 0) head = n;
  head = head < n ? head : n;
  for (long long i = t0; i < head; i += stride) ls[i] += delta;
  float4* q = reinterpret_cast<float4*>(ls + head);
  const long long n4 = (n - head) / 4;
  for (long long i = t0; i < n4; i += stride) {
    float4 v = q[i];
    v.x += delta;
    v.y += delta;
    v.z += delta;
    v.w += delta;
    q[i] = v;
  }
  for (long long i = head + 4 * n4 + t0; i < n; i += stride) ls[i] += delta;
}

int loss_blocks(long long P) {
  return (int)std::max<long long>(1, std::min<long long>(kLossMaxBlocks, (P + kLossThreads - 1) / kLossThreads));
}

}  // namespace
}  // namespace gs

using namespace gs;

extern "C" {

int gs_stage_events(int stage, void* ev_begin, void* ev_end) {
  if (stage < GS_STAGE_EXPANSION || stage > GS_STAGE_ADJOINT) return invalid("stage");
  g_stage_ev[stage][0] = ev_begin;
  g_stage_ev[stage][1] = ev_end;
  return GS_OK;
}

int gs_debug_bounds_status(unsigned* status, int clear) {
  if (!status) return invalid("status");
  unsigned s[3] = {0u, 0u, 0u};
  int rc = bounds_status_render(&s[0], clear != 0);
  if (rc == GS_OK) rc = bounds_status_binning(&s[1], clear != 0);
  if (rc == GS_OK) rc = bounds_status_preprocess(&s[2], clear != 0);
  *status = s[0] ? s[0] : (s[1] ? s[1] : s[2]);
  return rc;
}

int gs_record_bytes(int attr_dtype) {
  switch (attr_dtype) {
    case GS_ATTR_F32: return (int)sizeof(RecF32);
    case GS_ATTR_F16:
    case GS_ATTR_BF16: return (int)sizeof(RecH16);
  }
  return -1;
}

long long gs_total_tiles(const gs_camera* cams, int V, int tile_size) {
  CamTable ct;
  if (!build_cam_table(cams, V, nullptr, tile_size, &ct)) return -1;
  return ct.total_tiles;
}

long long gs_total_pixels(const gs_camera* cams, int V) {
  CamTable ct;
  if (!build_cam_table(cams, V, nullptr, 0, &ct)) return -1;
  return ct.c[V - 1].pix_off + (long long)ct.c[V - 1].W * ct.c[V - 1].H;
}

size_t gs_bin_sort_workspace_size(long long n_rows, long long cap, long long total_tiles) {
  if (n_rows < 0 || cap < 0 || total_tiles < 0) return 0;
  return bin_sort_workspace_size(n_rows, cap, total_tiles);
}

size_t gs_loss_workspace_size(long long total_pixels) {
  return sizeof(double) * (size_t)loss_blocks(total_pixels);
}

size_t gs_tile_queue_workspace_size(long long total_tiles) {
  return tile_queue_workspace_size(total_tiles);
}

const char* gs_status_string(int s) {
  switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_INVALID_ARG: return "invalid argument";
    case GS_ERR_CUDA: return "CUDA error";
    case GS_ERR_CAPACITY: return "pair capacity exceeded";
    case GS_ERR_TIMEOUT: return "timeout";
    case GS_ERR_UNSUPPORTED: return "unsupported";
  }
  return "unknown status";
}

const char* gs_last_error_string(void) { return g_err; }

const char* gs_version(void) { return "libgs 0.1 sm_103a tile16"; }

unsigned long long gs_kernel_launches(void) { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }

int gs_preprocess(const float* means, const float* log_scales, const float* quats,
                  const float* opacity_logits, const float* sh, int N, const gs_camera* cams,
                  int V, const gs_params* prm, const gs_proj* out, gs_stream stream) {
  if (N < 0) return invalid("N < 0");
  if (!params_ok(prm)) return invalid("params");
  CamTable ct;
  if (!build_cam_table(cams, V, prm, prm->tile_size, &ct)) return invalid("cameras");
  if ((long long)N * V >= (1ll << 32)) return invalid("V*N must be < 2^32");
  if (!proj_ok(out, true)) return invalid("projection buffers (NULL or misaligned)");
  if (!out->rect && !rect8_fits(ct))
    return invalid("rect is required when a view is more than 255 tiles wide or high");
  if (N > 0 && (!means || !log_scales || !quats || !opacity_logits || !sh))
    return invalid("parameter pointers");
  if (N > 0 && !aligned(quats, 16)) return invalid("quats must be 16-byte aligned");
  return launch_preprocess(means, log_scales, quats, opacity_logits, sh, N, ct, prm, out,
                           (cudaStream_t)stream);
}

int gs_bin_sort(const gs_proj* proj, int N, const gs_camera* cams, int V, int tile_size,
                void* workspace,
                size_t workspace_bytes, long long pair_capacity, unsigned* sorted_vals,
                unsigned long long* sorted_keys, unsigned* tile_ranges, long long* num_pairs_dev,
                long long* num_pairs_host, int* status_dev, gs_stream stream) {
  if (N < 0) return invalid("N < 0");
  CamTable ct;
  if (tile_size != 0 && tile_size != 8 && tile_size != 16) return invalid("tile_size (8 or 16)");
  if (!build_cam_table(cams, V, nullptr, tile_size, &ct)) return invalid("cameras");
  if (!proj_ok(proj, false)) return invalid("projection buffers");
  if (!proj->rect && !(proj->rect8 && rect8_fits(ct)))
    return invalid("rect is required unless rect8 is set and every view is at most 255 tiles "
                   "wide and high");
  if (pair_capacity < 0 || pair_capacity >= (1ll << 32)) return invalid("pair_capacity");
  if (!tile_ranges || !num_pairs_dev || !status_dev) return invalid("output pointers");
  if (pair_capacity > 0 && !sorted_vals) return invalid("sorted_vals");
  if (!workspace || !aligned(workspace, 256)) return invalid("workspace (NULL or not 256-B aligned)");
  if (workspace_bytes < bin_sort_workspace_size((long long)N * V, pair_capacity, ct.total_tiles))
    return invalid("workspace too small");
  return launch_bin_sort(proj, N, ct, workspace, workspace_bytes, pair_capacity, sorted_vals,
                         sorted_keys, tile_ranges, num_pairs_dev, num_pairs_host, status_dev,
                         (cudaStream_t)stream);
}

namespace {
// The launch controls of the render calls, checked on the host (NULL = defaults).
const char* launch_opt_error(const gs_launch* opt, const gs_params* prm) {
  if (!opt) return nullptr;
  if (opt->ctas < 0) return "ctas < 0";
  if (opt->ctas > 0 && !opt->work_counter) return "persistent launch needs work_counter";
  const int ppt = opt->pixels_per_thread;
  if (ppt != 0 && ppt != 1 && ppt != 2 && ppt != 4) return "pixels_per_thread (0, 1, 2 or 4)";
  if (ppt == 4 && prm->tile_size == 8) return "pixels_per_thread 4 needs 16-pixel tiles";
  if (opt->batch != 0 && opt->batch != 256 && opt->batch != 128) return "batch (0, 128 or 256)";
  if (opt->batch == 128 && (prm->tile_size == 8 || prm->attr_dtype != GS_ATTR_F32))
    return "batch 128 needs F32 records and 16-pixel tiles";
  return nullptr;
}
}  // namespace

int gs_render_fwd(const gs_proj* proj, int N, const gs_camera* cams, int V, const gs_params* prm,
                  const unsigned* sorted_vals, const unsigned* tile_ranges, float* image,
                  float* final_T, unsigned* last_idx, float* entropy, const gs_launch* opt,
                  gs_stream stream) {
  if (N < 0) return invalid("N < 0");
  if (!params_ok(prm)) return invalid("params");
  CamTable ct;
  if (!build_cam_table(cams, V, prm, prm->tile_size, &ct)) return invalid("cameras");
  if (!proj_ok(proj, true)) return invalid("projection buffers");
  if (!tile_ranges || !image || !final_T || !last_idx) return invalid("output pointers");
  if (!aligned(tile_ranges, 8)) return invalid("tile_ranges must be 8-byte aligned");
  if (const char* why = launch_opt_error(opt, prm)) return invalid(why);
  return launch_render_fwd(proj, (long long)N * V, ct, prm, sorted_vals, tile_ranges, image,
                           final_T, last_idx, entropy, opt, (cudaStream_t)stream);
}

namespace {
int loss_impl(const float* image, const float* target, const float* entropy, const gs_camera* cams,
              int V, float lambda, float gamma, double* loss_dev, float* dL_dimage,
              float* dL_dentropy, void* workspace, size_t workspace_bytes, cudaStream_t st) {
  CamTable ct;
  if (!build_cam_table(cams, V, nullptr, 0, &ct)) return invalid("cameras");
  long long P = ct.c[V - 1].pix_off + (long long)ct.c[V - 1].W * ct.c[V - 1].H;
  if (!image || !target || !loss_dev || !dL_dimage) return invalid("pointers");
  if (gamma != 0.f && !entropy) return invalid("entropy is required when gamma != 0");
  if (!(gamma >= 0.f)) return invalid("gamma");
  if (!(lambda >= 0.f && lambda <= 1.f)) return invalid("lambda (0..1)");
  const int nb = loss_blocks(P);
  const int ns = lambda > 0.f ? ssim_blocks(ct) : 0;
  const size_t need = sizeof(double) * (size_t)(nb + ns) +
                      (lambda > 0.f ? ssim_workspace_bytes(P) + 256 : 0);
  if (!workspace || workspace_bytes < need) return invalid("workspace");
  double* partials = reinterpret_cast<double*>(workspace);
  LossViews lv;
  lv.V = V;
  for (int v = 0; v < V; ++v) {
    const double M = (double)ct.c[v].W * ct.c[v].H;
    lv.pix_off[v] = ct.c[v].pix_off;
    lv.w[v] = (float)(1.0 / (M * V));
    lv.g_img[v] = (float)((1.0 - (double)lambda) / (3.0 * M * V));
    lv.g_ent[v] = (float)((double)gamma / (M * V));
  }
  const int vec = aligned(image, 16) && aligned(target, 16) && aligned(dL_dimage, 16) &&
                  (gamma == 0.f || !entropy || aligned(entropy, 16)) &&
                  (!dL_dentropy || aligned(dL_dentropy, 16));
  loss_kernel<<<nb, kLossThreads, 0, st>>>(image, target, gamma != 0.f ? entropy : nullptr, lv, P,
                                           gamma, (float)(1.0 - (double)lambda), dL_dimage, dL_dentropy,
                                           partials, vec);
  count_launches(1);
  if (lambda > 0.f) {
    uintptr_t m = reinterpret_cast<uintptr_t>(partials + nb + ns);
    float* maps = reinterpret_cast<float*>((m + 255) & ~uintptr_t(255));
    const int e = launch_ssim(image, target, ct, lambda, maps, partials + nb, dL_dimage, st);
    if (e != GS_OK) return e;
  }
  loss_finalize_kernel<<<1, kLossThreads, 0, st>>>(partials, nb + ns, loss_dev);
  count_launches(1);
  return check_launch();
}
}  // namespace

int gs_loss_l1_entropy(const float* image, const float* target, const float* entropy,
                       const gs_camera* cams, int V, float gamma, double* loss_dev,
                       float* dL_dimage, float* dL_dentropy, void* workspace,
                       size_t workspace_bytes, gs_stream stream) {
  return loss_impl(image, target, entropy, cams, V, 0.f, gamma, loss_dev, dL_dimage, dL_dentropy,
                   workspace, workspace_bytes, (cudaStream_t)stream);
}

size_t gs_loss_base_workspace_size(const gs_camera* cams, int V) {
  CamTable ct;
  if (!build_cam_table(cams, V, nullptr, 0, &ct)) return 0;
  const long long P = ct.c[V - 1].pix_off + (long long)ct.c[V - 1].W * ct.c[V - 1].H;
  return sizeof(double) * (size_t)(loss_blocks(P) + ssim_blocks(ct)) + ssim_workspace_bytes(P) +
         256;
}

int gs_loss_base(const float* image, const float* target, const float* entropy,
                 const gs_camera* cams, int V, float lambda, float gamma, double* loss_dev,
                 float* dL_dimage, float* dL_dentropy, void* workspace, size_t workspace_bytes,
                 gs_stream stream) {
  return loss_impl(image, target, entropy, cams, V, lambda, gamma, loss_dev, dL_dimage,
                   dL_dentropy, workspace, workspace_bytes, (cudaStream_t)stream);
}

int gs_render_bwd(const gs_proj* proj, int N, const gs_camera* cams, int V, const gs_params* prm,
                  const unsigned* sorted_vals, const unsigned* tile_ranges, const float* final_T,
                  const unsigned* last_idx, const float* dL_dimage, const float* dL_dentropy,
                  const float* means, const float* log_scales, const float* quats,
                  const float* opacity_logits, const float* sh, float* grad2d, float* g_means,
                  float* g_log_scales, float* g_quats, float* g_opacity_logits, float* g_sh,
                  const gs_launch* opt, gs_stream stream) {
  if (N < 0) return invalid("N < 0");
  if (!params_ok(prm)) return invalid("params");
  CamTable ct;
  if (!build_cam_table(cams, V, prm, prm->tile_size, &ct)) return invalid("cameras");
  if (!proj_ok(proj, true)) return invalid("projection buffers");
  if (!tile_ranges || !final_T || !last_idx || !dL_dimage) return invalid("forward outputs");
  if (!grad2d || !aligned(grad2d, 16)) return invalid("grad2d (NULL or not 16-B aligned)");
  if (N > 0 && (!means || !log_scales || !quats || !opacity_logits || !sh)) return invalid("params");
  if (N > 0 && (!g_means || !g_log_scales || !g_quats || !g_opacity_logits || !g_sh))
    return invalid("gradient outputs");
  if (N > 0 && (!aligned(quats, 16) || !aligned(g_quats, 16))) return invalid("quat alignment");
  if (const char* why = launch_opt_error(opt, prm)) return invalid(why);
  cudaStream_t st = (cudaStream_t)stream;
  if (N == 0) return GS_OK;  // no Gaussians: no gradients
  if (!opt || !opt->grad2d_zeroed)
    GS_TRY_CUDA(cudaMemsetAsync(grad2d, 0, sizeof(float) * 12 * (size_t)N * V, st));
  // Beside the blending adjoint (bound by instruction issue, most of the
  // memory bandwidth free), on the side stream: the list of Gaussians some
  // view sees (in grad2d's pad floats, after its zeroing) and the zeroing of
  // every parameter gradient.  (Zeroing only the unseen Gaussians' gradients
  // inside the list kernel was slower where most Gaussians are unseen and
  // no faster where all are seen.)
  auto side_work = [&](cudaStream_t s) -> int {
    const int r = launch_adjoint_list(proj->tiles_touched, N, V, grad2d, s);
    if (r != GS_OK) return r;
    GS_TRY_CUDA(cudaMemsetAsync(g_sh, 0, sizeof(float) * 3 * (size_t)prm->sh_stride * N, s));
    GS_TRY_CUDA(cudaMemsetAsync(g_means, 0, sizeof(float) * 3 * (size_t)N, s));
    GS_TRY_CUDA(cudaMemsetAsync(g_log_scales, 0, sizeof(float) * 3 * (size_t)N, s));
    GS_TRY_CUDA(cudaMemsetAsync(g_quats, 0, sizeof(float) * 4 * (size_t)N, s));
    GS_TRY_CUDA(cudaMemsetAsync(g_opacity_logits, 0, sizeof(float) * (size_t)N, s));
    return GS_OK;
  };
  std::lock_guard<std::mutex> lock(g_side_mu);
  SideStream* ss = side_stream_locked(st);
  int rc = GS_OK;
  if (ss) {
    GS_TRY_CUDA(cudaEventRecord(ss->fork, st));
    GS_TRY_CUDA(cudaStreamWaitEvent(ss->s, ss->fork, 0));
    const int rs = side_work(ss->s);
    // (the side branch is joined back on every path from here)
    GS_TRY_CUDA(cudaEventRecord(ss->join, ss->s));
    if (rs == GS_OK)
      rc = launch_render_bwd(proj, (long long)N * V, ct, prm, sorted_vals, tile_ranges, final_T,
                             last_idx, dL_dimage, dL_dentropy, grad2d, opt, st);
    GS_TRY_CUDA(cudaStreamWaitEvent(st, ss->join, 0));
    if (rs != GS_OK) return rs;
  } else {
    rc = side_work(st);
    if (rc == GS_OK)
      rc = launch_render_bwd(proj, (long long)N * V, ct, prm, sorted_vals, tile_ranges, final_T,
                             last_idx, dL_dimage, dL_dentropy, grad2d, opt, st);
  }
  if (rc != GS_OK) return rc;
  return launch_preprocess_bwd(means, log_scales, quats, opacity_logits, sh, N, ct, prm,
                               proj->tiles_touched, grad2d, g_means, g_log_scales, g_quats,
                               g_opacity_logits, g_sh, st);
}

int gs_grad2d_attributes(const gs_proj* proj, int N, int V, const gs_params* prm,
                         const float* grad2d, float* out, gs_stream stream) {
  if (N < 0 || V < 1 || V > GS_MAX_VIEWS) return invalid("N or V");
  if (!params_ok(prm)) return invalid("params");
  if (!proj_ok(proj, true)) return invalid("projection buffers");
  if ((long long)N * V >= (1ll << 32)) return invalid("V*N must be < 2^32");
  if (N > 0 && (!grad2d || !aligned(grad2d, 16) || !out))
    return invalid("grad2d (16-B aligned) and out");
  return launch_grad2d_attributes(proj, (long long)N * V, prm, grad2d, out, (cudaStream_t)stream);
}

int gs_scale_reset(float* log_scales, long long n, float zeta, gs_stream stream) {
  if (!(zeta > 0.f && zeta < 1.f)) return invalid("zeta must be in (0, 1)");
  if (n < 0 || (n > 0 && !log_scales)) return invalid("log_scales");
  if (n == 0) return GS_OK;
  const float delta = (float)log((double)zeta);
  unsigned grid = (unsigned)std::min<long long>((n / 4 + 255) / 256 + 1, 152ll * 8);
  scale_reset_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(log_scales, n, delta);
  count_launches(1);
  return check_launch();
}

int gs_tile_queue(const unsigned* tile_ranges, long long total_tiles, unsigned* tile_order,
                  void* workspace, size_t workspace_bytes, gs_stream stream) {
  if (total_tiles < 0 || total_tiles >= (1ll << 31)) return invalid("total_tiles");
  if (total_tiles > 0 && (!tile_ranges || !tile_order)) return invalid("pointers");
  if (!workspace || !aligned(workspace, 256)) return invalid("workspace");
  return launch_tile_queue(tile_ranges, total_tiles, tile_order, workspace, workspace_bytes,
                           (cudaStream_t)stream);
}

}  // extern "C"
