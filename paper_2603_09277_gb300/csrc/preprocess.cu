// preprocess.cu -- per-Gaussian projection (forward) and its adjoint.
//
// Forward (Sec. 3, Background): Sigma = R S S^T R^T from the normalised
// quaternion and s = exp(log_scale); EWA splatting Sigma' = J W Sigma W^T J^T
// + dilation I with the perspective Jacobian J at the camera-space mean; the
// conic Sigma'^-1; opacity sigmoid(logit); real SH colour up to degree 3,
// + 0.5, clamped at 0; the 3-sigma radius and the rect of tiles (side 16 or
// 8) it meets.
//
// One thread per Gaussian loops over the views, so the view-independent
// part (activations, Sigma) is computed once.  Parameter loads are
// coalesced across the warp; quaternions and SH rows use 16-byte loads.
//
// Backward: hand-derived adjoint of the same steps, one thread per Gaussian
// that some view sees (a list built beside the blending adjoint), summing
// over views; the covariance part runs through the Cholesky factor of the
// 2D covariance (whitened form) and accumulates the log-scale and
// rotation-matrix gradients over views, pushed to the quaternion once.
#include <algorithm>

#include "gs_internal.cuh"

namespace gs {
namespace {

// Real SH basis up to degree 3 (orthonormal, Condon-Shortley phase), order
// (l, m), m = -l..l, at a unit direction.
constexpr float kY0 = 0.28209479177387814f;   // sqrt(1/(4 pi))
constexpr float kY1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
constexpr float kY2a = 1.0925484305920792f;   // sqrt(15/pi)/2
constexpr float kY2b = 0.31539156525252005f;  // sqrt(5/pi)/4
constexpr float kY2c = 0.54627421529603959f;  // sqrt(15/pi)/4
constexpr float kY3a = 0.59004358992664352f;  // sqrt(35/(2 pi))/4
constexpr float kY3b = 2.8906114426405538f;   // sqrt(105/pi)/2
constexpr float kY3c = 0.45704579946446572f;  // sqrt(21/(2 pi))/4
constexpr float kY3d = 0.3731763325901154f;   // sqrt(7/pi)/4
constexpr float kY3e = 1.4453057213202769f;   // sqrt(105/pi)/4


__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* Y) {
  Y[0] = kY0;
  if (deg < 1) return;
  Y[1] = -kY1 * y;
  Y[2] = kY1 * z;
  Y[3] = -kY1 * x;
  if (deg < 2) return;
  float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = kY2a * x * y;
  Y[5] = -kY2a * y * z;
  Y[6] = kY2b * (2.f * zz - xx - yy);
  Y[7] = -kY2a * x * z;
  Y[8] = kY2c * (xx - yy);
  if (deg < 3) return;
  Y[9] = -kY3a * y * (3.f * xx - yy);
  Y[10] = kY3b * x * y * z;
  Y[11] = -kY3c * y * (4.f * zz - xx - yy);
  Y[12] = kY3d * z * (2.f * zz - 3.f * xx - 3.f * yy);
  Y[13] = -kY3c * x * (4.f * zz - xx - yy);
  Y[14] = kY3e * z * (xx - yy);
  Y[15] = -kY3a * x * (xx - 3.f * yy);
}

// Gradient of each basis polynomial with respect to (x, y, z), contracted
// with coefficients c[k]: returns sum_k c[k] grad Y_k.
__device__ __forceinline__ float3 sh_basis_grad_dot(int deg, float x, float y, float z,
                                                    const float* c) {
  float gx = 0.f, gy = 0.f, gz = 0.f;
  if (deg < 1) return make_float3(0.f, 0.f, 0.f);
  gy += -kY1 * c[1];
  gz += kY1 * c[2];
  gx += -kY1 * c[3];
  if (deg >= 2) {
    gx += kY2a * y * c[4];
    gy += kY2a * x * c[4];
    gy += -kY2a * z * c[5];
    gz += -kY2a * y * c[5];
    gx += -2.f * kY2b * x * c[6];
    gy += -2.f * kY2b * y * c[6];
    gz += 4.f * kY2b * z * c[6];
    gx += -kY2a * z * c[7];
    gz += -kY2a * x * c[7];
    gx += 2.f * kY2c * x * c[8];
    gy += -2.f * kY2c * y * c[8];
  }
  if (deg >= 3) {
    float xx = x * x, yy = y * y, zz = z * z;
    gx += -6.f * kY3a * x * y * c[9];
    gy += -kY3a * (3.f * xx - 3.f * yy) * c[9];
    gx += kY3b * y * z * c[10];
    gy += kY3b * x * z * c[10];
    gz += kY3b * x * y * c[10];
    gx += 2.f * kY3c * x * y * c[11];
    gy += -kY3c * (4.f * zz - xx - 3.f * yy) * c[11];
    gz += -8.f * kY3c * y * z * c[11];
    gx += -6.f * kY3d * x * z * c[12];
    gy += -6.f * kY3d * y * z * c[12];
    gz += kY3d * (6.f * zz - 3.f * xx - 3.f * yy) * c[12];
    gx += -kY3c * (4.f * zz - 3.f * xx - yy) * c[13];
    gy += 2.f * kY3c * x * y * c[13];
    gz += -8.f * kY3c * x * z * c[13];
    gx += 2.f * kY3e * x * z * c[14];
    gy += -2.f * kY3e * y * z * c[14];
    gz += kY3e * (xx - yy) * c[14];
    gx += -kY3a * (3.f * xx - 3.f * yy) * c[15];
    gy += 6.f * kY3a * x * y * c[15];
  }
  return make_float3(gx, gy, gz);
}

// Where value e = 3k + channel of Gaussian g's SH lies: sh[g * gs + k * ks +
// channel].  Layout 0 keeps a Gaussian's coefficients together (gs = 3 *
// stride, ks = 3); layout 1 keeps each coefficient of all Gaussians together
// (gs = 3, ks = 3N), so that a warp's loads of one coefficient are
// contiguous and a degree below the stored one reads only its coefficients.
struct ShPtr {
  long long gs, ks;
  int vec;  // layout 0, 16-byte aligned array, stride a multiple of 4: 16-byte loads
};

inline ShPtr sh_ptr(const float* sh, const gs_params* prm, int N) {
  ShPtr L;
  if (prm->sh_layout == 1) {
    L.gs = 3;
    L.ks = 3ll * N;
    L.vec = 0;
  } else {
    L.gs = 3ll * prm->sh_stride;
    L.ks = 3;
    L.vec = (prm->sh_stride & 3) == 0 && (reinterpret_cast<uintptr_t>(sh) & 15) == 0;
  }
  return L;
}

__device__ __forceinline__ long long sh_index(const ShPtr& L, long long g, int e) {
  return g * L.gs + (long long)(e / 3) * L.ks + e % 3;
}

// Calls f(e, value) for the floats e = 3k + channel, e < 3K, of Gaussian
// g's SH, in ascending e.  With vec, 16-byte loads of the Gaussian's block:
// the last one may read up to 3 floats past 3K, which stay inside the block
// (3 * stride is a multiple of 4 and at least 3K) and are not passed on.
template <typename F>
__device__ __forceinline__ void for_sh_block(const float* sh, long long g, const ShPtr& L,
                                             int K, F&& f) {
  if (L.vec) {
    const float* p = sh + g * L.gs;
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      if (4 * i < 3 * K) {
        const float4 t = __ldg(reinterpret_cast<const float4*>(p) + i);
        f(4 * i, t.x);
        if (4 * i + 1 < 3 * K) f(4 * i + 1, t.y);
        if (4 * i + 2 < 3 * K) f(4 * i + 2, t.z);
        if (4 * i + 3 < 3 * K) f(4 * i + 3, t.w);
      }
    }
  } else {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (k < K) {
        const float* q = sh + g * L.gs + k * L.ks;
        f(3 * k, __ldg(q));
        f(3 * k + 1, __ldg(q + 1));
        f(3 * k + 2, __ldg(q + 2));
      }
    }
  }
}

// Rotation matrix of a unit quaternion (w, x, y, z), row-major.
__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float* R) {
  R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
  R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
  R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
}

struct Activated {
  float mean[3];
  float s[3];      // scales
  float q[4];      // unit quaternion
  float qnorm;     // |q| before normalisation
  float Rq[9];
  float Sig[6];    // Sigma: xx, xy, xz, yy, yz, zz
  float sigma;     // opacity
};

__device__ __forceinline__ Activated activate(const float* means, const float* log_scales,
                                              const float* quats, const float* opacity_logits,
                                              int g) {
  Activated a;
  a.mean[0] = __ldg(means + 3ll * g);
  a.mean[1] = __ldg(means + 3ll * g + 1);
  a.mean[2] = __ldg(means + 3ll * g + 2);
  for (int k = 0; k < 3; ++k) a.s[k] = expf(__ldg(log_scales + 3ll * g + k));
  float4 q = __ldg(reinterpret_cast<const float4*>(quats) + g);
  float n2 = q.x * q.x + q.y * q.y + q.z * q.z + q.w * q.w;
  a.qnorm = sqrtf(n2);
  float inv = rsqrtf(n2);
  a.q[0] = q.x * inv; a.q[1] = q.y * inv; a.q[2] = q.z * inv; a.q[3] = q.w * inv;
  quat_to_rot(a.q[0], a.q[1], a.q[2], a.q[3], a.Rq);
  float M[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[i * 3 + j] = a.Rq[i * 3 + j] * a.s[j];
  a.Sig[0] = M[0] * M[0] + M[1] * M[1] + M[2] * M[2];
  a.Sig[1] = M[0] * M[3] + M[1] * M[4] + M[2] * M[5];
  a.Sig[2] = M[0] * M[6] + M[1] * M[7] + M[2] * M[8];
  a.Sig[3] = M[3] * M[3] + M[4] * M[4] + M[5] * M[5];
  a.Sig[4] = M[3] * M[6] + M[4] * M[7] + M[5] * M[8];
  a.Sig[5] = M[6] * M[6] + M[7] * M[7] + M[8] * M[8];
  float o = __ldg(opacity_logits + g);
  a.sigma = 1.f / (1.f + expf(-o));
  return a;
}

// ---------------------------------------------------------------------------
// Error-free FP32 transformations (FP32x2 "double-float" arithmetic): the
// camera-space mean and the 2D mean are carried as unevaluated sums hi + lo,
// so that cancellation in R mean + t (scene coordinates far larger than the
// camera-space offset) does not cost pixel-level precision.
// ---------------------------------------------------------------------------
struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ F2 two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}

__device__ __forceinline__ F2 fast_two_sum(float a, float b) {  // |a| >= |b|
  float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// r0 m0 + r1 m1 + r2 m2 + t, accurate to about FP32 epsilon squared.
__device__ __forceinline__ F2 dot3_plus(float r0, float r1, float r2, const float* m, float t) {
  F2 p0 = two_prod(r0, m[0]), p1 = two_prod(r1, m[1]), p2 = two_prod(r2, m[2]);
  F2 s1 = two_sum(p0.hi, p1.hi);
  F2 s2 = two_sum(s1.hi, p2.hi);
  F2 s3 = two_sum(s2.hi, t);
  float err = __fadd_rn(__fadd_rn(__fadd_rn(p0.lo, p1.lo), __fadd_rn(p2.lo, s1.lo)),
                        __fadd_rn(s2.lo, s3.lo));
  return fast_two_sum(s3.hi, err);
}

// Camera-space depth, defined as the FP32 rounding of the FP64 value
// ((R20 mx + R21 my) + R22 mz) + t2 (products of FP32 values are exact in
// FP64, so the value does not depend on FMA contraction).
__device__ __forceinline__ float depth_fp64(const CamInfo& c, const float* m) {
  double z = __dadd_rn(__dadd_rn(__dadd_rn(__dmul_rn((double)c.R[6], (double)m[0]),
                                           __dmul_rn((double)c.R[7], (double)m[1])),
                                 __dmul_rn((double)c.R[8], (double)m[2])),
                       (double)c.t[2]);
  return __double2float_rn(z);
}

// The same value without FP64 arithmetic in all but rare cases (FP64 runs at
// a small fraction of the FP32 rate here).  With S the exact sum and A the
// sum of the four terms' magnitudes: error-free FP32 transformations give
// hi + lo with |hi + lo - S| <= 2^-44 A (six rounding-error terms, each at
// most 2^-24 A, summed in FP32) and hi = RN(hi + lo); the FP64 expression
// differs from S by at most 3 2^-53 A < 2^-51 A.  So when hi + lo lies more
// than tol = 2^-40 A inside both rounding midpoints around hi, the FP64 value
// lies strictly between them as well and rounds to hi.  Otherwise (hi + lo
// within about 2^-16 (A / |hi|) ulp of a midpoint, a non-normal or very large
// hi, or a non-finite term) the FP64 expression itself is evaluated.
__device__ __forceinline__ float depth_of(const CamInfo& c, const float* m) {
  const F2 p0 = two_prod(c.R[6], m[0]), p1 = two_prod(c.R[7], m[1]), p2 = two_prod(c.R[8], m[2]);
  const F2 s1 = two_sum(p0.hi, p1.hi);
  const F2 s2 = two_sum(s1.hi, p2.hi);
  const F2 s3 = two_sum(s2.hi, c.t[2]);
  const float err = __fadd_rn(__fadd_rn(__fadd_rn(p0.lo, p1.lo), __fadd_rn(p2.lo, s1.lo)),
                              __fadd_rn(s2.lo, s3.lo));
  const F2 z = two_sum(s3.hi, err);
  const float A = __fadd_rn(__fadd_rn(fabsf(p0.hi), fabsf(p1.hi)),
                            __fadd_rn(fabsf(p2.hi), fabsf(c.t[2])));
  const float tol = __fmul_rn(A, 0x1p-40f);
  const float a = fabsf(z.hi);
  const int bits = __float_as_int(a);
  const float up = __fsub_rn(__int_as_float(bits + 1), a);    // spacing above |hi|
  const float down = __fsub_rn(a, __int_as_float(bits - 1));  // spacing below |hi|
  const float l = z.hi < 0.f ? -z.lo : z.lo;                   // lo, away from zero
  const bool sure = a >= 0x1p-100f && a < 0x1p+120f && __fsub_rn(0.5f * up, l) > tol &&
                    __fadd_rn(0.5f * down, l) > tol;
  return sure ? z.hi : depth_fp64(c, m);
}

// (x.hi + x.lo) / (y.hi + y.lo) as a double-float, with the correctly rounded
// reciprocal iy = 1 / y.hi given: the quotient's high part is x.hi iy (within
// about an ulp of x.hi / y.hi), the FMA remainder and the low part correct
// it, so the double-float result keeps its accuracy; the two divisions by tz
// share the reciprocal.
__device__ __forceinline__ F2 div2_rcp(F2 x, F2 y, float iy) {
  const float q = __fmul_rn(x.hi, iy);
  float r = __fmaf_rn(-q, y.hi, x.hi);
  r = __fadd_rn(r, __fsub_rn(x.lo, __fmul_rn(q, y.lo)));
  return fast_two_sum(q, __fmul_rn(r, iy));
}

// f (u.hi + u.lo) + c as a double-float.
__device__ __forceinline__ F2 affine2(float f, F2 u, float c) {
  F2 p = two_prod(f, u.hi);
  F2 s = two_sum(p.hi, c);
  return fast_two_sum(s.hi, __fadd_rn(__fadd_rn(p.lo, __fmul_rn(f, u.lo)), s.lo));
}

// a d - b c with one rounding (Kahan's FMA form).
__device__ __forceinline__ float det2(float a, float b, float c, float d) {
  float w = __fmul_rn(b, c);
  float e = __fmaf_rn(-b, c, w);
  float f = __fmaf_rn(a, d, -w);
  return __fadd_rn(f, e);
}

struct Projected {
  bool ok;
  float tx, ty, tz, ux, uy;
  bool clx, cly;       // Jacobian clamp active in x / y
  float J00, J02, J11, J12;
  float T[6];          // J W (2x3)
  float A, B, C;       // Sigma' + dilation I
  float det;           // det(Sigma' + dilation I)
  float ca, cb, cc;    // conic
  float f11, f21, f22; // sqrt(log2(e)/2) L^-1 with L L^T = Sigma' + dilation I
  float l21, i11, i22; // L = [[l11, 0], [l21, l22]] and 1 / l11, 1 / l22
  float itz;           // 1 / tz
  F2 mx, my;           // 2D mean (double-float)
};

// EWA projection (Sec. 3).  Sigma' = N N^T with N = J W M (M = R S): the
// Cholesky factor of Sigma' + dilation I and its determinant are formed from
// N directly (rows n0, n1): det = |n0 x n1|^2 + d (|n0|^2 + |n1|^2) + d^2,
// which avoids squaring the condition number of Sigma'.
// From the camera-space position (p.tz, p.ux = tx / tz, p.uy = ty / tz): the
// clamped EWA Jacobian, Sigma' + dilation I, its Cholesky factor and the
// conic.  Shared by the projection and its adjoint; ADJ: the adjoint's form,
// with the inverse Cholesky diagonal from reciprocal square roots.
template <bool ADJ = false>
__device__ __forceinline__ void project_tail(const CamInfo& c, const Activated& a, float dilation,
                                             Projected& p) {
  const float itz = __frcp_rn(p.tz);  // (correctly rounded: the value of 1.f / tz)
  p.itz = itz;
  p.clx = p.ux < -c.limx || p.ux > c.limx;
  p.cly = p.uy < -c.limy || p.uy > c.limy;
  float uxc = fminf(fmaxf(p.ux, -c.limx), c.limx);
  float uyc = fminf(fmaxf(p.uy, -c.limy), c.limy);
  p.J00 = c.fx * itz;
  p.J02 = -c.fx * uxc * itz;
  p.J11 = c.fy * itz;
  p.J12 = -c.fy * uyc * itz;
  for (int j = 0; j < 3; ++j) {
    p.T[j] = p.J00 * c.R[j] + p.J02 * c.R[6 + j];
    p.T[3 + j] = p.J11 * c.R[3 + j] + p.J12 * c.R[6 + j];
  }
  // N = T M, M = Rq diag(s)
  float n0[3], n1[3];
  for (int j = 0; j < 3; ++j) {
    float mj0 = a.Rq[j] * a.s[j], mj1 = a.Rq[3 + j] * a.s[j], mj2 = a.Rq[6 + j] * a.s[j];
    n0[j] = p.T[0] * mj0 + p.T[1] * mj1 + p.T[2] * mj2;
    n1[j] = p.T[3] * mj0 + p.T[4] * mj1 + p.T[5] * mj2;
  }
  float s00 = n0[0] * n0[0] + n0[1] * n0[1] + n0[2] * n0[2];
  float s11 = n1[0] * n1[0] + n1[1] * n1[1] + n1[2] * n1[2];
  float s01 = n0[0] * n1[0] + n0[1] * n1[1] + n0[2] * n1[2];
  float cx0 = det2(n0[1], n0[2], n1[1], n1[2]);
  float cx1 = det2(n0[2], n0[0], n1[2], n1[0]);
  float cx2 = det2(n0[0], n0[1], n1[0], n1[1]);
  p.A = s00 + dilation;
  p.B = s01;
  p.C = s11 + dilation;
  p.det = (cx0 * cx0 + cx1 * cx1 + cx2 * cx2) + dilation * (s00 + s11) + dilation * dilation;
  p.ok = p.det > 0.f && p.A > 0.f;
  // L = [[l11, 0], [l21, l22]], L L^T = [[A, B], [B, C]]
  if constexpr (ADJ) {
    // 1 / l11 = A^-1/2 and 1 / l22 = l11 / sqrt(det) = A det^-1/2 A^-1/2
    const float i11 = rsqrtf(p.A);
    const float l21 = p.B * i11;
    const float i22 = rsqrtf(p.det) * (p.A * i11);
    const float i21 = -l21 * i11 * i22;
    p.l21 = l21;
    p.i11 = i11;
    p.i22 = i22;
    p.ca = i11 * i11 + i21 * i21;
    p.cb = i21 * i22;
    p.cc = i22 * i22;
    return;
  }
  // one correctly rounded reciprocal per diagonal entry, then products
  const float l11 = sqrtf(p.A);
  const float i11 = __frcp_rn(l11);
  const float l21 = p.B * i11;
  const float l22 = sqrtf(p.det) * i11;
  const float i22 = __frcp_rn(l22);
  const float i21 = -l21 * i11 * i22;
  const float kc = 0.8493218002880191f;  // sqrt(log2(e) / 2)
  p.f11 = kc * i11;
  p.f22 = kc * i22;
  p.f21 = kc * i21;
  // conic = L^-T L^-1
  p.l21 = l21;
  p.i11 = i11;
  p.i22 = i22;
  p.ca = i11 * i11 + i21 * i21;
  p.cb = i21 * i22;
  p.cc = i22 * i22;
}

__device__ __forceinline__ Projected project(const CamInfo& c, const Activated& a, float depth,
                                             float dilation) {
  Projected p;
  const float* m = a.mean;
  F2 tx = dot3_plus(c.R[0], c.R[1], c.R[2], m, c.t[0]);
  F2 ty = dot3_plus(c.R[3], c.R[4], c.R[5], m, c.t[1]);
  F2 tz = {depth, 0.f};
  p.tx = tx.hi;
  p.ty = ty.hi;
  p.tz = depth;
  const float itz = __frcp_rn(depth);
  F2 ux = div2_rcp(tx, tz, itz), uy = div2_rcp(ty, tz, itz);
  p.ux = ux.hi;
  p.uy = uy.hi;
  project_tail(c, a, dilation, p);
  p.mx = affine2(c.fx, ux, c.cx);
  p.my = affine2(c.fy, uy, c.cy);
  return p;
}

// The exact projection as a call of its own, for the adjoint's rare fallback
// (inlined a second time it would raise the adjoint's register pressure).
__device__ __noinline__ Projected project_exact(const CamInfo& c, const Activated& a,
                                                float dilation) {
  return project(c, a, depth_of(c, a.mean), dilation);
}

// The projection as its adjoint needs it: camera-space position and its
// ratios in plain FP32 (the adjoint's gradients are compared at 1e-4, the
// exact depth key and double-float mean serve the forward's list order and
// tile-relative means).  The one decision that must match the forward's, the
// Jacobian clamp of x/z and y/z, is taken from the exact projection whenever
// a ratio lies within 1e-5 (relative) of its limit.
__device__ __forceinline__ Projected project_adjoint(const CamInfo& c, const Activated& a,
                                                     float dilation) {
  const float* m = a.mean;
  const float tx = __fmaf_rn(c.R[2], m[2], __fmaf_rn(c.R[1], m[1], __fmaf_rn(c.R[0], m[0], c.t[0])));
  const float ty = __fmaf_rn(c.R[5], m[2], __fmaf_rn(c.R[4], m[1], __fmaf_rn(c.R[3], m[0], c.t[1])));
  const float tz = __fmaf_rn(c.R[8], m[2], __fmaf_rn(c.R[7], m[1], __fmaf_rn(c.R[6], m[0], c.t[2])));
  const float itz = __frcp_rn(tz);
  const float ux = tx * itz, uy = ty * itz;
  if (fabsf(fabsf(ux) - c.limx) <= 1e-5f * c.limx || fabsf(fabsf(uy) - c.limy) <= 1e-5f * c.limy)
    return project_exact(c, a, dilation);
  Projected p;
  p.tx = tx;
  p.ty = ty;
  p.tz = tz;
  p.ux = ux;
  p.uy = uy;
  project_tail<true>(c, a, dilation, p);
  return p;
}

// Templated on the staging dtype and the SH degree in use: with the degree a
// constant the basis values and the coefficient loop stay in registers (a
// runtime degree put them in local memory).
// Resident projection CTAs per SM the register budget targets: 4 (64
// registers, no spills) up to SH degree 1, 5 (48 registers) above.  Measured
// on cfg3 (degree 0): 562 us at 5, 486 us at 4; on cfg2 (degree 3): 43.7 us
// at 5, 47.5 us at 4.
template <int DEG>
constexpr int pre_ctas_per_sm() {
  return DEG <= 1 ? 4 : 5;
}
template <int DT, int DEG>
__global__ void __launch_bounds__(256, pre_ctas_per_sm<DEG>()) preprocess_kernel(
    const float* __restrict__ means, const float* __restrict__ log_scales,
    const float* __restrict__ quats, const float* __restrict__ opacity_logits,
    const float* __restrict__ sh, int N, const CamTable ct, float dilation, float near_z,
    const ShPtr shp, gs_proj out) {
  int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= N) return;
  Activated a = activate(means, log_scales, quats, opacity_logits, g);
  constexpr int sh_deg = DEG;
  constexpr int K = (DEG + 1) * (DEG + 1);
  // per Gaussian, not per view: log2 of the opacity and, at degree 0, the colour
  const float L2S = log2f(a.sigma);
  float col0[3] = {0.5f, 0.5f, 0.5f};
  if constexpr (DEG == 0) {
    float Y[16];
    sh_basis(0, 0.f, 0.f, 1.f, Y);
    for_sh_block(sh, g, shp, K, [&](int e, float v) { col0[e % 3] += Y[e / 3] * v; });
  }
  for (int v = 0; v < ct.V; ++v) {
    const CamInfo& c = ct.c[v];
    long long row = (long long)v * N + g;
    float depth = depth_of(c, a.mean);
    out.depth[row] = depth;
    bool vis = depth > near_z;
    Projected p;
    int x0 = 0, y0 = 0, x1 = 0, y1 = 0;
    float r = 0.f;
    if (vis) {
      p = project(c, a, depth, dilation);
      vis = p.ok && isfinite(p.mx.hi) && isfinite(p.my.hi) && isfinite(p.f11) &&
            isfinite(p.f21) && isfinite(p.f22) && isfinite(p.ca) && isfinite(p.cc);
    }
    if (vis) {
      // larger eigenvalue of [[A, B], [B, C]] in the cancellation-free form
      float hd = 0.5f * (p.A - p.C);
      float lam = 0.5f * (p.A + p.C) + sqrtf(hd * hd + p.B * p.B);
      r = ceilf(3.f * sqrtf(lam));
      const float inv_tile = 1.f / (float)ct.tile;  // exact: the side is a power of two
      const float mx = p.mx.hi, my = p.my.hi;
      float fx0 = floorf((mx - r) * inv_tile), fx1 = floorf((mx + r) * inv_tile) + 1.f;
      float fy0 = floorf((my - r) * inv_tile), fy1 = floorf((my + r) * inv_tile) + 1.f;
      x0 = (int)fminf(fmaxf(fx0, 0.f), (float)c.TX);
      x1 = (int)fminf(fmaxf(fx1, 0.f), (float)c.TX);
      y0 = (int)fminf(fmaxf(fy0, 0.f), (float)c.TY);
      y1 = (int)fminf(fmaxf(fy1, 0.f), (float)c.TY);
      vis = (x1 > x0) && (y1 > y0) && isfinite(r);
    }
    if (!vis) {
      if (out.rect) reinterpret_cast<int4*>(out.rect)[row] = make_int4(0, 0, 0, 0);
      out.tiles_touched[row] = 0u;
      if (out.radius) out.radius[row] = 0;
      continue;
    }
    // SH colour at the direction from the camera centre to the mean (at
    // degree 0 it does not depend on the view: taken once per Gaussian)
    float col[3] = {col0[0], col0[1], col0[2]};
    if constexpr (DEG > 0) {
      float vx = a.mean[0] - c.cp[0], vy = a.mean[1] - c.cp[1], vz = a.mean[2] - c.cp[2];
      float il = rsqrtf(vx * vx + vy * vy + vz * vz);
      float Y[16];
      sh_basis(sh_deg, vx * il, vy * il, vz * il, Y);
      for_sh_block(sh, g, shp, K, [&](int e, float v) { col[e % 3] += Y[e / 3] * v; });
    }
    float cr = col[0], cg = col[1], cbl = col[2];
    cr = fmaxf(cr, 0.f);
    cg = fmaxf(cg, 0.f);
    cbl = fmaxf(cbl, 0.f);

    Splat s;
    // 2D mean as integer + fraction (the fraction carries the low part)
    s.hx = rintf(p.mx.hi);
    s.hy = rintf(p.my.hi);
    s.lx = __fadd_rn(__fsub_rn(p.mx.hi, s.hx), p.mx.lo);
    s.ly = __fadd_rn(__fsub_rn(p.my.hi, s.hy), p.my.lo);
    s.f11 = p.f11;
    s.f21 = p.f21;
    s.f22 = p.f22;
    s.L2S = L2S;
    s.R = cr;
    s.G = cg;
    s.B = cbl;
    s.sigma = a.sigma;
    store_record<DT>(out.records, row, s);
    if (out.rect) reinterpret_cast<int4*>(out.rect)[row] = make_int4(x0, y0, x1, y1);
    if (out.rect8)  // (views of at most 255 tiles per side)
      out.rect8[row] =
          (unsigned)x0 | ((unsigned)y0 << 8) | ((unsigned)x1 << 16) | ((unsigned)y1 << 24);
    out.tiles_touched[row] = (unsigned)((x1 - x0) * (y1 - y0));
    if (out.radius) out.radius[row] = (int)r;
    if (out.mean2d)
      reinterpret_cast<float2*>(out.mean2d)[row] =
          make_float2(__fadd_rn(p.mx.hi, p.mx.lo), __fadd_rn(p.my.hi, p.my.lo));
    if (out.conic_opacity)
      reinterpret_cast<float4*>(out.conic_opacity)[row] = make_float4(p.ca, p.cb, p.cc, a.sigma);
    if (out.rgb) {
      out.rgb[3 * row] = cr;
      out.rgb[3 * row + 1] = cg;
      out.rgb[3 * row + 2] = cbl;
    }
  }
}

// ---------------------------------------------------------------------------
// Adjoint of the projection.  grad2d rows, summed over the pixels of every
// blended pair of the row: dd (dx, dy, dx^2, dx dy, dy^2, 1) and w (r, g, b),
// with dd = dL/dalpha alpha where alpha is not clamped and (dx, dy) the
// pixel centre minus the 2D mean.  Since alpha = sigma exp(-d^T K d / 2)
// (K the conic, d = pixel - mean):
//   dL/dsigma = sum dd / sigma,  dL/dK = -(1/2) sum dd d d^T
//   (so dL/da = -Sxx / 2, dL/db = -Sxy with b counted twice in d^T K d,
//   dL/dc = -Syy / 2),  dL/dmean = K (Sx, Sy).
// ---------------------------------------------------------------------------
// Per-lane sums of one Gaussian's adjoint over the views the lane takes:
// dL/dmean, dL/dlog-scale, dL/d(rotation matrix entries), the sum of dd
// (-> opacity) and dL/dSH for the K coefficients in use.
template <int DEG>
struct AdjAcc {
  static constexpr int K = (DEG + 1) * (DEG + 1);
  float gm[3], gls[3], gRq[9], gsig, gsh[3 * K];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < 3; ++i) gm[i] = gls[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 9; ++i) gRq[i] = 0.f;
    gsig = 0.f;
#pragma unroll
    for (int i = 0; i < 3 * K; ++i) gsh[i] = 0.f;
  }
  // sum over the L lanes of a group (butterfly, group-local mask)
  template <int L>
  __device__ __forceinline__ void reduce(unsigned mask) {
#pragma unroll
    for (int o = 1; o < L; o <<= 1) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        gm[i] += __shfl_xor_sync(mask, gm[i], o);
        gls[i] += __shfl_xor_sync(mask, gls[i], o);
      }
#pragma unroll
      for (int i = 0; i < 9; ++i) gRq[i] += __shfl_xor_sync(mask, gRq[i], o);
      gsig += __shfl_xor_sync(mask, gsig, o);
#pragma unroll
      for (int i = 0; i < 3 * K; ++i) gsh[i] += __shfl_xor_sync(mask, gsh[i], o);
    }
  }
};

// Adjoint of Gaussian g in view v (which sees it), added to acc.
// A Gaussian's SH coefficients for the adjoint's views: held in registers at
// degree 0 (3 floats, read once per Gaussian instead of twice per view; the
// 12 floats of degree 1 would spill), read from the block on each use above.
template <int DEG>
struct ShCoef {
  static constexpr int K = (DEG + 1) * (DEG + 1);
  static constexpr bool kCached = DEG == 0;
  float c[kCached ? 3 * K : 1];
  __device__ __forceinline__ void load(const float* __restrict__ sh, long long g, const ShPtr& L) {
    if constexpr (kCached) for_sh_block(sh, g, L, K, [&](int e, float v) { c[e] = v; });
  }
  // f(e, value) for e < 3K, like for_sh_block
  template <typename F>
  __device__ __forceinline__ void each(const float* __restrict__ sh, long long g, const ShPtr& L,
                                       F&& f) const {
    if constexpr (kCached) {
#pragma unroll
      for (int e = 0; e < 3 * K; ++e) f(e, c[e]);
    } else {
      for_sh_block(sh, g, L, K, f);
    }
  }
};

// SHREG: the SH gradient is summed in acc (a group of several lanes);
// otherwise (one lane per Gaussian, degree 3: 48 sums would halve the
// occupancy) it goes to g_sh directly: the first view that sees the
// Gaussian stores, later ones add.
template <int DEG, bool SHREG>
__device__ __forceinline__ void adjoint_view(
    int g, int v, const Activated& a, const float* __restrict__ sh, int N, const CamTable& ct,
    float dilation, const ShPtr& shp, const float* __restrict__ grad2d,
    AdjAcc<SHREG ? DEG : 0>& acc, bool first_view, bool vec_out, float* __restrict__ g_sh,
    const ShCoef<DEG>& shc) {
  constexpr int sh_deg = DEG;
  constexpr int K = AdjAcc<DEG>::K;
  float* gm = acc.gm;
  float* gls = acc.gls;
  float* gRq = acc.gRq;
  float& gsig = acc.gsig;
    long long row = (long long)v * N + g;
    const float4* G4 = reinterpret_cast<const float4*>(grad2d + row * 12);
    float4 G0 = G4[0], G1 = G4[1], G2 = G4[2];
    // G0 = (Sx, Sy, Sxx, Sxy), G1 = (Syy, S1, r, g), G2 = (b, pad, pad, pad)
    const CamInfo& c = ct.c[v];
    // (degree 3 keeps the exact projection: the FP32 head with its fallback
    // spills there, 31 -> 33 us on a 1M-Gaussian view)
    Projected p = DEG < 3 ? project_adjoint(c, a, dilation) : project(c, a, depth_of(c, a.mean), dilation);

    gsig += G1.y;  // sum dd; dL/dlogit = (sum dd / sigma) sigma (1 - sigma)
    const float gmx = p.ca * G0.x + p.cb * G0.y;  // dL/dmean2d = K (Sx, Sy)
    const float gmy = p.cb * G0.x + p.cc * G0.y;

    // --- colour -> SH coefficients and view direction
    float vx = a.mean[0] - c.cp[0], vy = a.mean[1] - c.cp[1], vz = a.mean[2] - c.cp[2];
    float il = rsqrtf(vx * vx + vy * vy + vz * vz);
    float dx = vx * il, dy = vy * il, dz = vz * il;
    float Y[16] = {};
    sh_basis(sh_deg, dx, dy, dz, Y);
    float raw[3] = {0.5f, 0.5f, 0.5f};
    shc.each(sh, g, shp, [&](int e, float v) { raw[e % 3] += Y[e / 3] * v; });
    float grgb[3] = {raw[0] < 0.f ? 0.f : G1.z, raw[1] < 0.f ? 0.f : G1.w,
                     raw[2] < 0.f ? 0.f : G2.x};
    float cdot[16] = {};  // SH[k] . grgb
    shc.each(sh, g, shp,
             [&](int e, float v) { cdot[e / 3] = __fmaf_rn(v, grgb[e % 3], cdot[e / 3]); });
    // dL/dSH[k][ch] = Y_k grgb_ch
    if constexpr (SHREG) {
#pragma unroll
      for (int e = 0; e < 3 * K; ++e) acc.gsh[e] = __fmaf_rn(Y[e / 3], grgb[e % 3], acc.gsh[e]);
    } else {
      float* gsh = g_sh + (long long)g * shp.gs;  // (vec_out: layout 0)
      if (vec_out) {
#pragma unroll
        for (int i = 0; i < 12; ++i) {
          if (4 * i < 3 * K) {
            float o[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
              const int e = 4 * i + j;
              o[j] = e < 3 * K ? Y[e / 3] * grgb[e % 3] : 0.f;
            }
            float4* q = reinterpret_cast<float4*>(gsh) + i;
            if (first_view) {
              *q = make_float4(o[0], o[1], o[2], o[3]);
            } else {
              const float4 t = *q;
              *q = make_float4(t.x + o[0], t.y + o[1], t.z + o[2], t.w + o[3]);
            }
          }
        }
      } else {
#pragma unroll
        for (int e = 0; e < 48; ++e) {
          if (e < 3 * K) {
            const float y = Y[e / 3] * grgb[e % 3];
            float& o = g_sh[sh_index(shp, g, e)];
            o = first_view ? y : o + y;
          }
        }
      }
      // (coefficients past K keep the zeros of the caller's zeroing)
    }
    if (sh_deg > 0) {
      float3 gd = sh_basis_grad_dot(sh_deg, dx, dy, dz, cdot);
      float dd = gd.x * dx + gd.y * dy + gd.z * dz;
      gm[0] += (gd.x - dx * dd) * il;
      gm[1] += (gd.y - dy * dd) * il;
      gm[2] += (gd.z - dz * dd) * il;
    }

    // --- conic -> (N, T), in whitened form.  With Sigma' + dilation I =
    // N N^T + d I = L L^T (L from the forward), Gk the gradient of the conic
    // as a symmetric matrix and G^ = L^-1 Gk L^-T, Z = L^-1 N, T^ = L^-1 T:
    //   dL/dN = -2 L^-T G^ Z,   dL/dM = -2 T^T G^ Z,
    //   dL/d log s_j = -2 Z_j^T G^ Z_j (Z_j = column j of Z).
    // Every factor is scaled by L^-1, so the condition number of Sigma' is
    // not squared as it would be through dL/dSigma' = -K Gk K.
    const float* T = p.T;
    // the projection's Cholesky factor of Sigma' + dilation I
    const float l21 = p.l21, i11 = p.i11, i22 = p.i22;
    const float i21 = -l21 * i11 * i22;
    float Th[6];
    for (int j = 0; j < 3; ++j) {
      Th[j] = T[j] * i11;
      Th[3 + j] = (T[3 + j] - l21 * Th[j]) * i22;
    }
    float Z[6];
    for (int j = 0; j < 3; ++j) {
      Z[j] = a.s[j] * (Th[0] * a.Rq[j] + Th[1] * a.Rq[3 + j] + Th[2] * a.Rq[6 + j]);
      Z[3 + j] = a.s[j] * (Th[3] * a.Rq[j] + Th[4] * a.Rq[3 + j] + Th[5] * a.Rq[6 + j]);
    }
    const float ga = -0.5f * G0.z, gbh = -0.5f * G0.w, gc = -0.5f * G1.x;
    const float G00 = i11 * i11 * ga;
    const float G01 = i11 * (i21 * ga + i22 * gbh);
    const float G11 = i21 * i21 * ga + 2.f * i21 * i22 * gbh + i22 * i22 * gc;
    float GZ[6];
    for (int j = 0; j < 3; ++j) {
      GZ[j] = G00 * Z[j] + G01 * Z[3 + j];
      GZ[3 + j] = G01 * Z[j] + G11 * Z[3 + j];
    }
    for (int j = 0; j < 3; ++j) {
      gls[j] += -2.f * (Z[j] * GZ[j] + Z[3 + j] * GZ[3 + j]);
      for (int i = 0; i < 3; ++i)
        gRq[i * 3 + j] += -2.f * a.s[j] * (Th[i] * GZ[j] + Th[3 + i] * GZ[3 + j]);
    }
    // dL/dT = dL/dN M^T with dL/dN = -2 L^-T G^ Z
    float gN[6];
    for (int j = 0; j < 3; ++j) {
      gN[j] = -2.f * (i11 * GZ[j] + i21 * GZ[3 + j]);
      gN[3 + j] = -2.f * i22 * GZ[3 + j];
    }
    float gT[6];
    for (int r = 0; r < 2; ++r)
      for (int i = 0; i < 3; ++i) {
        float acc = 0.f;
        for (int j = 0; j < 3; ++j) acc += gN[3 * r + j] * a.Rq[i * 3 + j] * a.s[j];
        gT[3 * r + i] = acc;
      }
    // --- T = J W
    float gJ00 = gT[0] * c.R[0] + gT[1] * c.R[1] + gT[2] * c.R[2];
    float gJ02 = gT[0] * c.R[6] + gT[1] * c.R[7] + gT[2] * c.R[8];
    float gJ11 = gT[3] * c.R[3] + gT[4] * c.R[4] + gT[5] * c.R[5];
    float gJ12 = gT[3] * c.R[6] + gT[4] * c.R[7] + gT[5] * c.R[8];
    // --- J(t) and the 2D mean(t)
    const float itz = p.itz;
    float gtx = 0.f, gty = 0.f, gtz = 0.f;
    gtz += -gJ00 * c.fx * itz * itz - gJ11 * c.fy * itz * itz;
    if (p.clx) {
      gtz += -gJ02 * p.J02 * itz;
    } else {
      gtx += -gJ02 * c.fx * itz * itz;
      gtz += -2.f * gJ02 * p.J02 * itz;
    }
    if (p.cly) {
      gtz += -gJ12 * p.J12 * itz;
    } else {
      gty += -gJ12 * c.fy * itz * itz;
      gtz += -2.f * gJ12 * p.J12 * itz;
    }
    gtx += gmx * c.fx * itz;
    gty += gmy * c.fy * itz;
    gtz += -(gmx * c.fx * p.ux + gmy * c.fy * p.uy) * itz;
    // --- t = W mean + t_w
    gm[0] += c.R[0] * gtx + c.R[3] * gty + c.R[6] * gtz;
    gm[1] += c.R[1] * gtx + c.R[4] * gty + c.R[7] * gtz;
    gm[2] += c.R[2] * gtx + c.R[5] * gty + c.R[8] * gtz;
  }

// Writes Gaussian g's gradients from the group's sums: lane `sub` == 0 the
// per-Gaussian ones, the K SH coefficients in use split over the group's L
// lanes as 16-byte stores where aligned, up to the end of the 32-byte sector
// holding the last of them (a partly written sector is filled from DRAM
// first); the coefficients past that keep the zeros of the caller's zeroing
// (with 16 coefficients stored per Gaussian and degree 0 in use, rewriting
// them was 15/16 of this kernel's SH writes).
template <int DEG, int L, bool SHREG>
__device__ __forceinline__ void adjoint_finish(
    int g, int sub, const Activated& a, const AdjAcc<DEG>& acc, const ShPtr& shp, bool vec_out,
    float* __restrict__ g_means, float* __restrict__ g_ls, float* __restrict__ g_quats,
    float* __restrict__ g_opac, float* __restrict__ g_sh) {
  constexpr int K = AdjAcc<DEG>::K;
  constexpr int kSectorFloats = (3 * K + 7) / 8 * 8;  // 3K rounded up to 32 bytes
  float* gsh = g_sh + (long long)g * shp.gs;  // (vec_out: layout 0, the block's start)
  if (!SHREG) {
  } else if (vec_out) {
#pragma unroll
    for (int i = 0; i < 12; ++i) {
      if (i % L == sub && 4 * i < kSectorFloats && 4 * i < shp.gs) {
        float o[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) o[j] = 4 * i + j < 3 * K ? acc.gsh[4 * i + j] : 0.f;
        reinterpret_cast<float4*>(gsh)[i] = make_float4(o[0], o[1], o[2], o[3]);
      }
    }
  } else {
#pragma unroll
    for (int e = 0; e < 48; ++e)
      if (e % L == sub && e < 3 * K) g_sh[sh_index(shp, g, e)] = acc.gsh[e];
  }
  if (sub != 0) return;
  const float* gm = acc.gm;
  const float* gls = acc.gls;
  const float* gRq = acc.gRq;
  const float gsig = acc.gsig;
  g_means[3ll * g] = gm[0];
  g_means[3ll * g + 1] = gm[1];
  g_means[3ll * g + 2] = gm[2];
  g_opac[g] = gsig * (1.f - a.sigma);

  for (int j = 0; j < 3; ++j) g_ls[3ll * g + j] = gls[j];
  const float* GR = gRq;
  // --- rotation matrix of the unit quaternion
  float w = a.q[0], x = a.q[1], y = a.q[2], z = a.q[3];
  float gw = 2.f * (-z * GR[1] + y * GR[2] + z * GR[3] - x * GR[5] - y * GR[6] + x * GR[7]);
  float gx = 2.f * (y * GR[1] + z * GR[2] + y * GR[3] - 2.f * x * GR[4] - w * GR[5] + z * GR[6] +
                    w * GR[7] - 2.f * x * GR[8]);
  float gy = 2.f * (-2.f * y * GR[0] + x * GR[1] + w * GR[2] + x * GR[3] + z * GR[5] - w * GR[6] +
                    z * GR[7] - 2.f * y * GR[8]);
  float gz = 2.f * (-2.f * z * GR[0] - w * GR[1] + x * GR[2] + w * GR[3] - 2.f * z * GR[4] +
                    y * GR[5] + x * GR[6] + y * GR[7]);
  // --- normalisation q / |q|
  float dotq = w * gw + x * gx + y * gy + z * gz;
  float iq = 1.f / a.qnorm;
  float4 gq = make_float4((gw - w * dotq) * iq, (gx - x * dotq) * iq, (gy - y * dotq) * iq,
                          (gz - z * dotq) * iq);
  reinterpret_cast<float4*>(g_quats)[g] = gq;
}

// Adjoint of one listed Gaussian by a group of L lanes (L = the views rounded
// up to a power of two, at most 8): lane `sub` takes views sub, sub + L, ...
// that see the Gaussian, the group sums its lanes' parts with shuffles and
// writes the gradients.  Every gradient starts at zero (the caller zeroes
// them), so the Gaussians no view sees keep zeros.
template <int DEG, int L>
__device__ __forceinline__ void adjoint_group(
    int g, int sub, unsigned mask, const float* __restrict__ means,
    const float* __restrict__ log_scales, const float* __restrict__ quats,
    const float* __restrict__ opacity_logits, const float* __restrict__ sh, int N,
    const CamTable& ct, float dilation, const ShPtr& shp,
    const unsigned* __restrict__ tiles_touched, const float* __restrict__ grad2d,
    float* __restrict__ g_means, float* __restrict__ g_ls, float* __restrict__ g_quats,
    float* __restrict__ g_opac, float* __restrict__ g_sh) {
  const bool vec_out = shp.vec && (reinterpret_cast<uintptr_t>(g_sh) & 15) == 0;
  const Activated a = activate(means, log_scales, quats, opacity_logits, g);
  constexpr bool SHREG = L > 1 || DEG < 3;
  AdjAcc<SHREG ? DEG : 0> acc;
  acc.zero();
  // the views (of this lane's share) that see the Gaussian, as a mask: the
  // loads are issued together instead of one memory latency per view ahead
  // of its moment row's
  unsigned long long seen = 0ull;
#pragma unroll 8
  for (int v = sub; v < ct.V; v += L)
    seen |= (unsigned long long)(tiles_touched[(long long)v * N + g] != 0u) << v;
  ShCoef<DEG> shc;
  shc.load(sh, g, shp);
  bool first = true;
  while (seen) {
    const int v = __ffsll((long long)seen) - 1;
    seen &= seen - 1ull;
    adjoint_view<DEG, SHREG>(g, v, a, sh, N, ct, dilation, shp, grad2d, acc, first, vec_out,
                             g_sh, shc);
    first = false;
  }
  acc.template reduce<L>(mask);
  adjoint_finish<SHREG ? DEG : 0, L, SHREG>(g, sub, a, acc, shp, vec_out, g_means, g_ls,
                                            g_quats, g_opac, g_sh);
}

// The adjoint runs over a list of the Gaussians some view sees, kept in the
// pad floats of grad2d (the blending adjoint writes floats 0..8 of a row):
// entry k is float 9 of row k and the count is float 11 of row 0, all as
// unsigned; grad2d is zeroed before.  A CTA ranks its visible threads by
// warp ballots and reserves their slots with one atomic (one per CTA keeps
// the shared counter from serialising), so the list is in no particular
// order (each entry is independent).  A Gaussian's views are tested in order
// up to the first that sees it.
constexpr int kListThreads = 256;
__global__ void __launch_bounds__(kListThreads) adjoint_list_kernel(
    const unsigned* __restrict__ tiles_touched, int N, int V, float* __restrict__ grad2d) {
  __shared__ unsigned s_cnt[kListThreads / 32];
  __shared__ unsigned s_base;
  unsigned* g2 = reinterpret_cast<unsigned*>(grad2d);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (long long base = (long long)blockIdx.x * kListThreads; base < N;
       base += (long long)gridDim.x * kListThreads) {
    const long long g = base + threadIdx.x;
    bool vis = false;
    if (g < N)
      for (int v = 0; v < V && !vis; ++v) vis = tiles_touched[(long long)v * N + g] != 0u;
    const unsigned b = __ballot_sync(0xffffffffu, vis);
    if (lane == 0) s_cnt[w] = __popc(b);
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned run = 0u;
      for (int k = 0; k < kListThreads / 32; ++k) {
        const unsigned c = s_cnt[k];
        s_cnt[k] = run;
        run += c;
      }
      s_base = run ? atomicAdd(g2 + 11, run) : 0u;
    }
    __syncthreads();
    if (vis) g2[12ll * (s_base + s_cnt[w] + __popc(b & ((1u << lane) - 1u))) + 9] = (unsigned)g;
    __syncthreads();  // s_cnt and s_base are rewritten by the next round
  }
}

// The adjoint over the listed Gaussians: a resident grid, one group of L
// lanes per Gaussian and iteration (a group's lanes share the Gaussian, so
// they leave the loop together; shuffles use the group's lanes only).
constexpr int kAdjThreads = 128;
// CTAs per SM the register budget allows: 2 where a group sums 48 SH
// gradients in registers, 3 with 27, else 4 (at most 128 registers)
#ifndef GS_ADJ_CTAS
#define GS_ADJ_CTAS 5  // CTAs per SM of the single-lane adjoint (measured: 4 -> 0.725 ms, 5 -> 0.689, 6 -> 0.723 on 8 views of 3M)
#endif
template <int DEG, int L>
constexpr int adj_ctas_per_sm() { return (DEG == 3 && L > 1) ? 2 : (DEG == 2 ? 3 : GS_ADJ_CTAS); }

template <int DEG, int L>
__global__ void __launch_bounds__(kAdjThreads, adj_ctas_per_sm<DEG, L>()) preprocess_bwd_kernel(
    const float* __restrict__ means, const float* __restrict__ log_scales,
    const float* __restrict__ quats, const float* __restrict__ opacity_logits,
    const float* __restrict__ sh, int N, const CamTable ct, float dilation, const ShPtr shp,
    const unsigned* __restrict__ tiles_touched, const float* __restrict__ grad2d,
    float* __restrict__ g_means, float* __restrict__ g_ls, float* __restrict__ g_quats,
    float* __restrict__ g_opac, float* __restrict__ g_sh) {
  const unsigned* g2 = reinterpret_cast<const unsigned*>(grad2d);
  const unsigned n = g2[11];
  const int lane = threadIdx.x & 31;
  const int sub = lane % L;
  const unsigned mask = (L == 32 ? 0xffffffffu : ((1u << L) - 1u)) << (lane - sub);
  const unsigned groups = gridDim.x * (kAdjThreads / L);
  for (unsigned i = (blockIdx.x * kAdjThreads + threadIdx.x) / L; i < n; i += groups) {
    if (!GS_IN_BOUNDS(i, N, 302)) break;  // the list holds at most N Gaussians
    const unsigned g = g2[12ll * i + 9];
    if (!GS_IN_BOUNDS(g, N, 301)) continue;
    adjoint_group<DEG, L>((int)g, sub, mask, means, log_scales, quats,
                          opacity_logits, sh, N, ct, dilation, shp, tiles_touched, grad2d,
                          g_means, g_ls, g_quats, g_opac, g_sh);
  }
}

template <int DEG, int L>
void launch_adjoint(const float* means, const float* log_scales, const float* quats,
                    const float* opacity_logits, const float* sh, int N, const CamTable& ct,
                    const gs_params* prm, const unsigned* tiles_touched, const float* grad2d,
                    float* g_means, float* g_ls, float* g_quats, float* g_opac, float* g_sh,
                    cudaStream_t st) {
  // a resident grid: enough groups for every listed Gaussian at most
  const long long want = ((long long)N * L + kAdjThreads - 1) / kAdjThreads;
  const int grid = (int)std::min<long long>(152ll * adj_ctas_per_sm<DEG, L>() * 2, want);
  preprocess_bwd_kernel<DEG, L><<<grid, kAdjThreads, 0, st>>>(
      means, log_scales, quats, opacity_logits, sh, N, ct, prm->dilation, sh_ptr(sh, prm, N),
      tiles_touched, grad2d, g_means, g_ls, g_quats, g_opac, g_sh);
}

// Largest group of lanes per Gaussian.  1 (one thread walks all of a
// Gaussian's views) is the form the timings chose: on 8 views of 3M
// Gaussians 0.78 ms against 1.39 ms for groups of 8 lanes, whose redundant
// activation and shuffle reduction cost more than their parallelism gains.
#ifndef GS_ADJ_MAX_LANES
#define GS_ADJ_MAX_LANES 1
#endif

template <int DEG>
void launch_adjoint_deg(const float* means, const float* log_scales, const float* quats,
                        const float* opacity_logits, const float* sh, int N, const CamTable& ct,
                        const gs_params* prm, const unsigned* tiles_touched, const float* grad2d,
                        float* g_means, float* g_ls, float* g_quats, float* g_opac, float* g_sh,
                        cudaStream_t st) {
  // lanes per Gaussian: the views rounded up to a power of two, at most 8
  if (ct.V <= 1 || GS_ADJ_MAX_LANES == 1)
    launch_adjoint<DEG, 1>(means, log_scales, quats, opacity_logits, sh, N, ct, prm,
                           tiles_touched, grad2d, g_means, g_ls, g_quats, g_opac, g_sh, st);
  else if (ct.V <= 2 || GS_ADJ_MAX_LANES == 2)
    launch_adjoint<DEG, 2>(means, log_scales, quats, opacity_logits, sh, N, ct, prm,
                           tiles_touched, grad2d, g_means, g_ls, g_quats, g_opac, g_sh, st);
  else if (ct.V <= 4 || GS_ADJ_MAX_LANES == 4)
    launch_adjoint<DEG, 4>(means, log_scales, quats, opacity_logits, sh, N, ct, prm,
                           tiles_touched, grad2d, g_means, g_ls, g_quats, g_opac, g_sh, st);
  else
    launch_adjoint<DEG, 8>(means, log_scales, quats, opacity_logits, sh, N, ct, prm,
                           tiles_touched, grad2d, g_means, g_ls, g_quats, g_opac, g_sh, st);
}

// The 2D gradients of Suppl. C per row from the moment rows of the blending
// adjoint.  The conic comes from the record's square-root factor F
// (F^T F = log2(e) / 2 conic, F lower triangular): a = 2 ln 2 (f11^2 + f21^2),
// b = 2 ln 2 f21 f22, c = 2 ln 2 f22^2.
template <int DT>
__global__ void __launch_bounds__(256) grad2d_attr_kernel(const void* __restrict__ recs,
                                                          const unsigned* __restrict__ tiles_touched,
                                                          const float* __restrict__ grad2d,
                                                          long long rows, float* __restrict__ out) {
  for (long long row = (long long)blockIdx.x * blockDim.x + threadIdx.x; row < rows;
       row += (long long)gridDim.x * blockDim.x) {
    float o[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (tiles_touched[row] != 0u) {
      const Splat s = load_record<DT>(recs, (unsigned)row);
      const float k2 = 1.3862943611198906f;  // 2 ln 2
      const float ca = k2 * __fmaf_rn(s.f11, s.f11, s.f21 * s.f21);
      const float cb = k2 * s.f21 * s.f22;
      const float cc = k2 * s.f22 * s.f22;
      const float4* G4 = reinterpret_cast<const float4*>(grad2d + 12 * row);
      const float4 G0 = G4[0], G1 = G4[1], G2 = G4[2];
      // G0 = (Sx, Sy, Sxx, Sxy), G1 = (Syy, S1, r, g), G2 = (b, pad, pad, pad)
      o[0] = ca * G0.x + cb * G0.y;  // dL/dmean2d = K (Sx, Sy)
      o[1] = cb * G0.x + cc * G0.y;
      o[2] = -0.5f * G0.z;           // dL/dK: d = -1/2 (a dx^2 + 2 b dx dy + c dy^2)
      o[3] = -G0.w;
      o[4] = -0.5f * G1.x;
      o[5] = G1.y / s.sigma;         // alpha = sigma exp(d): dL/dsigma = sum dd / sigma
      o[6] = G1.z;
      o[7] = G1.w;
      o[8] = G2.x;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) out[9 * row + k] = o[k];
  }
}

}  // namespace

GS_BOUNDS_READER(bounds_status_preprocess)

int launch_grad2d_attributes(const gs_proj* proj, long long rows, const gs_params* prm,
                             const float* grad2d, float* out, cudaStream_t st) {
  if (rows == 0) return GS_OK;
  const unsigned grid = (unsigned)std::min<long long>((rows + 255) / 256, 152ll * 8);
  switch (prm->attr_dtype) {
    case GS_ATTR_F32:
      grad2d_attr_kernel<GS_ATTR_F32><<<grid, 256, 0, st>>>(proj->records, proj->tiles_touched,
                                                            grad2d, rows, out);
      break;
    case GS_ATTR_F16:
      grad2d_attr_kernel<GS_ATTR_F16><<<grid, 256, 0, st>>>(proj->records, proj->tiles_touched,
                                                            grad2d, rows, out);
      break;
    case GS_ATTR_BF16:
      grad2d_attr_kernel<GS_ATTR_BF16><<<grid, 256, 0, st>>>(proj->records, proj->tiles_touched,
                                                             grad2d, rows, out);
      break;
    default:
      return GS_ERR_INVALID_ARG;
  }
  count_launches(1);
  return check_launch();
}

template <int DT>
void launch_preprocess_dt(int deg, dim3 grid, dim3 block, const float* means,
                          const float* log_scales, const float* quats,
                          const float* opacity_logits, const float* sh, int N, const CamTable& ct,
                          const gs_params* prm, const gs_proj& o, cudaStream_t st) {
#define GS_PRE_LAUNCH(D)                                                                   \
  preprocess_kernel<DT, D><<<grid, block, 0, st>>>(means, log_scales, quats, opacity_logits, \
                                                   sh, N, ct, prm->dilation, prm->near_z,    \
                                                   sh_ptr(sh, prm, N), o)
  switch (deg) {
    case 0: GS_PRE_LAUNCH(0); break;
    case 1: GS_PRE_LAUNCH(1); break;
    case 2: GS_PRE_LAUNCH(2); break;
    default: GS_PRE_LAUNCH(3); break;
  }
#undef GS_PRE_LAUNCH
}

int launch_preprocess(const float* means, const float* log_scales, const float* quats,
                      const float* opacity_logits, const float* sh, int N, const CamTable& ct,
                      const gs_params* prm, const gs_proj* out, cudaStream_t st) {
  if (N == 0) return GS_OK;
  dim3 block(256), grid((N + 255) / 256);
  gs_proj o = *out;
  if (!rect8_fits(ct)) o.rect8 = nullptr;
  {
    const int e = stage_event(GS_STAGE_PROJECTION, false, st);
    if (e != GS_OK) return e;
  }
  const int deg = prm->sh_degree;
  if (deg < 0 || deg > 3) return GS_ERR_INVALID_ARG;
  switch (prm->attr_dtype) {
    case GS_ATTR_F32:
      launch_preprocess_dt<GS_ATTR_F32>(deg, grid, block, means, log_scales, quats,
                                        opacity_logits, sh, N, ct, prm, o, st);
      break;
    case GS_ATTR_F16:
      launch_preprocess_dt<GS_ATTR_F16>(deg, grid, block, means, log_scales, quats,
                                        opacity_logits, sh, N, ct, prm, o, st);
      break;
    case GS_ATTR_BF16:
      launch_preprocess_dt<GS_ATTR_BF16>(deg, grid, block, means, log_scales, quats,
                                         opacity_logits, sh, N, ct, prm, o, st);
      break;
    default:
      return GS_ERR_INVALID_ARG;
  }
  count_launches(1);
  {
    const int e = stage_event(GS_STAGE_PROJECTION, true, st);
    if (e != GS_OK) return e;
  }
  return check_launch();
}

int launch_preprocess_bwd(const float* means, const float* log_scales, const float* quats,
                          const float* opacity_logits, const float* sh, int N, const CamTable& ct,
                          const gs_params* prm, const unsigned* tiles_touched, const float* grad2d,
                          float* g_means, float* g_ls, float* g_quats, float* g_opac, float* g_sh,
                          cudaStream_t st) {
  if (N == 0) return GS_OK;
  {
    const int e = stage_event(GS_STAGE_ADJOINT, false, st);
    if (e != GS_OK) return e;
  }
  switch (prm->sh_degree) {
    case 0: launch_adjoint_deg<0>(means, log_scales, quats, opacity_logits, sh, N, ct, prm,
                                  tiles_touched, grad2d, g_means, g_ls, g_quats, g_opac, g_sh, st);
      break;
    case 1: launch_adjoint_deg<1>(means, log_scales, quats, opacity_logits, sh, N, ct, prm,
                                  tiles_touched, grad2d, g_means, g_ls, g_quats, g_opac, g_sh, st);
      break;
    case 2: launch_adjoint_deg<2>(means, log_scales, quats, opacity_logits, sh, N, ct, prm,
                                  tiles_touched, grad2d, g_means, g_ls, g_quats, g_opac, g_sh, st);
      break;
    default: launch_adjoint_deg<3>(means, log_scales, quats, opacity_logits, sh, N, ct, prm,
                                   tiles_touched, grad2d, g_means, g_ls, g_quats, g_opac, g_sh, st);
      break;
  }
  count_launches(1);
  {
    const int e = stage_event(GS_STAGE_ADJOINT, true, st);
    if (e != GS_OK) return e;
  }
  return check_launch();
}

int launch_adjoint_list(const unsigned* tiles_touched, int N, int V, float* grad2d,
                        cudaStream_t st) {
  if (N == 0) return GS_OK;
  const int grid = (int)std::min<long long>(152ll * 8, ((long long)N + kListThreads - 1) / kListThreads);
  adjoint_list_kernel<<<grid, kListThreads, 0, st>>>(tiles_touched, N, V, grad2d);
  count_launches(1);
  return check_launch();
}

}  // namespace gs
