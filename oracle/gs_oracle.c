/*
 * gs_oracle.c -- plain FP64 CPU oracle for the differentiable square-tile
 * Gaussian rasterizer with the entropy term on blending weights
 * ("Speeding Up the Learning of 3D Gaussians with Much Shorter Gaussian
 * Lists", arXiv 2603.09277).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * load this file; only the tests, the smoke check and the bench's CPU
 * baseline leg do.  It shares no code, header, table or constant with the
 * CUDA library: every formula below is written out here from the paper (and,
 * where the paper is silent, from the readings listed in the design notes).
 *
 * Precision: everything is IEEE double.  The parameters arrive widened from
 * their stored FP32 values; the thresholds are FP32 numbers by definition;
 * the depth sort key is by definition the FP32 rounding of an FP64
 * camera-space depth.
 *
 * Differentiation:
 *  - compositing (alpha -> colour, entropy) uses the paper's closed forms
 *    (Sec. 4.4 and Suppl. B), with the inner sums written out directly
 *    (O(N^2) per pixel), never Algorithm 1's reverse recursion;
 *  - alpha -> opacity, exponent, inverse covariance, 2D mean uses Suppl. C;
 *  - the per-Gaussian projection (Sec. 3) is differentiated by the complex
 *    step method: the projection is written once over complex doubles, and
 *    d out / d x = Im(f(x + i h)) / h with h = 1e-30, which is exact to
 *    rounding for analytic code and needs no hand-derived adjoint.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (see __init__.py).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cx;

/* ------------------------------------------------------------------------ */
/* Camera and threshold parameters, passed from Python as flat double arrays. */
/*  cam[0..1]  width, height                                                   */
/*  cam[2..5]  fx, fy, cx, cy                                                  */
/*  cam[6..17] world->camera [R|t] row-major 3x4 (FP32-representable values)   */
/*  cam[18..20] camera centre in world space                                   */
/*  prm[0..5]  alpha_max, alpha_min, t_min, dilation, near_z, fov_clamp        */
/*             (the FP32 values, widened)                                      */
/*  prm[6]     tile side in pixels (16 as in 3DGS; 8 as in LiteGS and the      */
/*             paper's own runs, Sec. 5 "Effect of tile sizes")                */
/* ------------------------------------------------------------------------ */
typedef struct {
    int W, H;
    double fx, fy, cx, cy;
    double R[9], t[3], cp[3];
} cam_t;

typedef struct {
    double amax, amin, tmin, dil, near_z, fovc;
    int tile;
} prm_t;

static cam_t load_cam(const double* c) {
    cam_t k;
    k.W = (int)c[0];
    k.H = (int)c[1];
    k.fx = c[2]; k.fy = c[3]; k.cx = c[4]; k.cy = c[5];
    for (int r = 0; r < 3; ++r) {
        for (int j = 0; j < 3; ++j) k.R[r * 3 + j] = c[6 + r * 4 + j];
        k.t[r] = c[6 + r * 4 + 3];
    }
    for (int j = 0; j < 3; ++j) k.cp[j] = c[18 + j];
    return k;
}

static prm_t load_prm(const double* p) {
    prm_t q = {p[0], p[1], p[2], p[3], p[4], p[5], (int)p[6]};
    return q;
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics up to degree 3 (orthonormal on the unit sphere,  */
/* Condon-Shortley phase), written from the textbook closed forms with the   */
/* normalisation constants evaluated from their definitions.  Order is       */
/* (l, m) for l = 0..3, m = -l..l.                                           */
/* ------------------------------------------------------------------------ */
static void sh_basis_cx(int deg, cx x, cx y, cx z, cx* Y) {
    const double pi = 3.14159265358979323846;
    Y[0] = sqrt(1.0 / (4.0 * pi));
    if (deg < 1) return;
    const double k1 = sqrt(3.0 / (4.0 * pi));
    Y[1] = -k1 * y;
    Y[2] = k1 * z;
    Y[3] = -k1 * x;
    if (deg < 2) return;
    const double k2a = 0.5 * sqrt(15.0 / pi);
    const double k2b = 0.25 * sqrt(5.0 / pi);
    const double k2c = 0.25 * sqrt(15.0 / pi);
    Y[4] = k2a * x * y;
    Y[5] = -k2a * y * z;
    Y[6] = k2b * (2.0 * z * z - x * x - y * y);
    Y[7] = -k2a * x * z;
    Y[8] = k2c * (x * x - y * y);
    if (deg < 3) return;
    const double k3a = 0.25 * sqrt(35.0 / (2.0 * pi));
    const double k3b = 0.5 * sqrt(105.0 / pi);
    const double k3c = 0.25 * sqrt(21.0 / (2.0 * pi));
    const double k3d = 0.25 * sqrt(7.0 / pi);
    const double k3e = 0.25 * sqrt(105.0 / pi);
    Y[9] = -k3a * y * (3.0 * x * x - y * y);
    Y[10] = k3b * x * y * z;
    Y[11] = -k3c * y * (4.0 * z * z - x * x - y * y);
    Y[12] = k3d * z * (2.0 * z * z - 3.0 * x * x - 3.0 * y * y);
    Y[13] = -k3c * x * (4.0 * z * z - x * x - y * y);
    Y[14] = k3e * z * (x * x - y * y);
    Y[15] = -k3a * x * (x * x - 3.0 * y * y);
}

/* Exported for the spherical-harmonic pins (orthonormality by quadrature). */
void ora_sh_basis(int deg, const double* dirs, int n, double* Y /* n x 16 */) {
    for (int i = 0; i < n; ++i) {
        cx Yc[16];
        for (int k = 0; k < 16; ++k) Yc[k] = 0;
        sh_basis_cx(deg, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], Yc);
        for (int k = 0; k < 16; ++k) Y[16 * i + k] = creal(Yc[k]);
    }
}

/* ------------------------------------------------------------------------ */
/* Projection of one Gaussian (Sec. 3, Background): Sigma = R S S^T R^T,    */
/* EWA splatting to a 2D mean and covariance, inverse covariance (conic),   */
/* opacity, SH colour.  Written over complex doubles so that the complex    */
/* step gives exact derivatives; all decisions use real parts.              */
/* ------------------------------------------------------------------------ */
typedef struct {
    int culled;      /* 1: behind the near plane, singular, or no tile touched */
    float depth;     /* FP32 rounding of the FP64 camera-space depth           */
    int radius;      /* ceil(3 sqrt(lambda_max)) in pixels                     */
    int rect[4];     /* x0, y0, x1, y1 in tiles, half-open                     */
    int tiles;       /* (x1-x0)*(y1-y0)                                        */
    int clamped[3];  /* SH colour channel clamped at 0                         */
    int boundary;    /* 1: the rect could differ under FP32 rounding           */
    int rect_lo[4];  /* tiles in the rect under every admissible rounding      */
    int rect_hi[4];  /* tiles in the rect under some admissible rounding       */
} proj_int;

/* Tile rect from the four pixel-space edges mx - r, mx + r, my - r, my + r:
 * the half-open range of tiles (side `tile` px) whose pixels
 * [tile k, tile k + tile) meet [edge0, edge1], clamped to the tile grid. */
static void rect_of_edges(double l, double r, double t, double b, int TX, int TY, int tile,
                          int out[4]) {
    double x0 = floor(l / tile), x1 = floor(r / tile) + 1.0;
    double y0 = floor(t / tile), y1 = floor(b / tile) + 1.0;
    x0 = fmin(fmax(x0, 0.0), (double)TX);
    x1 = fmin(fmax(x1, 0.0), (double)TX);
    y0 = fmin(fmax(y0, 0.0), (double)TY);
    y1 = fmin(fmax(y1, 0.0), (double)TY);
    out[0] = (int)x0; out[1] = (int)y0; out[2] = (int)x1; out[3] = (int)y1;
}

/* Boundary bands for the FP32 path: a pixel-space rect edge within EPS_PX of
 * a tile boundary, or 3 sqrt(lambda) within EPS_R (relative) of an integer,
 * may round the other way in FP32.  The bands are wide next to the FP32
 * error of the projection (about 1e-4 px at 1237 px focal length). */
#define EPS_PX 2e-3
#define EPS_R 2e-5

static void project_one(const cx mu[3], const cx ls[3], const cx q[4], cx o,
                        const cx* sh /* K x 3 */, int deg,
                        const cam_t* c, const prm_t* p,
                        cx out[9], proj_int* pi) {
    memset(pi, 0, sizeof(*pi));
    for (int k = 0; k < 9; ++k) out[k] = 0;

    /* World -> camera.  The depth used for sorting and culling is computed
     * from the real FP32 inputs in FP64 in the fixed order
     * ((R20 mx + R21 my) + R22 mz) + t2 and rounded once to FP32. */
    double mr[3] = {creal(mu[0]), creal(mu[1]), creal(mu[2])};
    double tz_key = ((c->R[6] * mr[0] + c->R[7] * mr[1]) + c->R[8] * mr[2]) + c->t[2];
    pi->depth = (float)tz_key;
    cx tx = c->R[0] * mu[0] + c->R[1] * mu[1] + c->R[2] * mu[2] + c->t[0];
    cx ty = c->R[3] * mu[0] + c->R[4] * mu[1] + c->R[5] * mu[2] + c->t[1];
    cx tz = ((c->R[6] * mu[0] + c->R[7] * mu[1]) + c->R[8] * mu[2]) + c->t[2];
    if (!((double)pi->depth > p->near_z)) { pi->culled = 1; return; }

    /* 3D covariance Sigma = R S S^T R^T from the normalised quaternion
     * (w, x, y, z) and s = exp(log_scale). */
    cx qn2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
    cx qinv = 1.0 / csqrt(qn2);
    cx w = q[0] * qinv, x = q[1] * qinv, y = q[2] * qinv, z = q[3] * qinv;
    cx Rq[9] = {
        1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y),
        2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
        2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)};
    cx s[3] = {cexp(ls[0]), cexp(ls[1]), cexp(ls[2])};
    cx M[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i * 3 + j] = Rq[i * 3 + j] * s[j];
    cx Sig[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cx acc = 0;
            for (int k = 0; k < 3; ++k) acc += M[i * 3 + k] * M[j * 3 + k];
            Sig[i * 3 + j] = acc;
        }

    /* EWA: Sigma' = J W Sigma W^T J^T with the perspective Jacobian J taken at
     * the camera-space mean, its x/z and y/z clamped to fov_clamp times the
     * half field of view; then the low-pass dilation on the diagonal. */
    double limx = p->fovc * (0.5 * c->W / c->fx);
    double limy = p->fovc * (0.5 * c->H / c->fy);
    cx ux = tx / tz, uy = ty / tz;
    cx uxc = creal(ux) < -limx ? (cx)(-limx) : (creal(ux) > limx ? (cx)limx : ux);
    cx uyc = creal(uy) < -limy ? (cx)(-limy) : (creal(uy) > limy ? (cx)limy : uy);
    cx J00 = c->fx / tz, J02 = -c->fx * uxc / tz;
    cx J11 = c->fy / tz, J12 = -c->fy * uyc / tz;
    cx T[6];
    for (int j = 0; j < 3; ++j) {
        T[j] = J00 * c->R[j] + J02 * c->R[6 + j];
        T[3 + j] = J11 * c->R[3 + j] + J12 * c->R[6 + j];
    }
    cx TS[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            cx acc = 0;
            for (int k = 0; k < 3; ++k) acc += T[i * 3 + k] * Sig[k * 3 + j];
            TS[i * 3 + j] = acc;
        }
    cx S2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            cx acc = 0;
            for (int k = 0; k < 3; ++k) acc += TS[i * 3 + k] * T[j * 3 + k];
            S2[i * 2 + j] = acc;
        }
    cx A = S2[0] + p->dil, B = S2[1], C = S2[3] + p->dil;
    cx det = A * C - B * B;
    if (!(creal(det) > 0.0)) { pi->culled = 1; return; }
    cx ca = C / det, cb = -B / det, cc = A / det;

    /* Pinhole projection of the mean (pixel centres at u + 0.5). */
    cx mx = c->fx * ux + c->cx, my = c->fy * uy + c->cy;

    /* 3-sigma radius from the larger eigenvalue of Sigma', and the tile rect. */
    double Ar = creal(A), Cr = creal(C), detr = creal(det);
    double mid = 0.5 * (Ar + Cr);
    double lam = mid + sqrt(fmax(mid * mid - detr, 0.0));
    double rf = 3.0 * sqrt(lam);
    double r = ceil(rf);
    int TX = (c->W + p->tile - 1) / p->tile, TY = (c->H + p->tile - 1) / p->tile;
    double mxr = creal(mx), myr = creal(my);
    rect_of_edges(mxr - r, mxr + r, myr - r, myr + r, TX, TY, p->tile, pi->rect);
    pi->radius = (int)r;
    pi->tiles = (pi->rect[2] - pi->rect[0]) * (pi->rect[3] - pi->rect[1]);
    /* Boundary flag: does a rounding of the radius within EPS_R, or of the
     * edges within EPS_PX, change the rect?  rect_lo / rect_hi bound every
     * rect reachable that way (intersection / union). */
    {
        double rs[3] = {r, ceil(rf * (1.0 - EPS_R)), ceil(rf * (1.0 + EPS_R))};
        memcpy(pi->rect_lo, pi->rect, sizeof pi->rect);
        memcpy(pi->rect_hi, pi->rect, sizeof pi->rect);
        for (int a = 0; a < 3; ++a) {
            double e[4] = {mxr - rs[a], mxr + rs[a], myr - rs[a], myr + rs[a]};
            for (int k = 0; k < 4; ++k)
                for (int sg = -1; sg <= 1; ++sg) {
                    double f[4] = {e[0], e[1], e[2], e[3]};
                    f[k] += sg * EPS_PX;
                    int r1[4];
                    rect_of_edges(f[0], f[1], f[2], f[3], TX, TY, p->tile, r1);
                    if (memcmp(r1, pi->rect, sizeof r1)) pi->boundary = 1;
                    for (int c = 0; c < 2; ++c) {
                        if (r1[c] > pi->rect_lo[c]) pi->rect_lo[c] = r1[c];
                        if (r1[c] < pi->rect_hi[c]) pi->rect_hi[c] = r1[c];
                        if (r1[c + 2] < pi->rect_lo[c + 2]) pi->rect_lo[c + 2] = r1[c + 2];
                        if (r1[c + 2] > pi->rect_hi[c + 2]) pi->rect_hi[c + 2] = r1[c + 2];
                    }
                }
        }
    }
    if (pi->tiles == 0) { pi->culled = 1; return; }

    /* View-dependent colour: real SH at the unit direction from the camera
     * centre to the mean, plus 0.5, clamped below at 0. */
    cx v[3] = {mu[0] - c->cp[0], mu[1] - c->cp[1], mu[2] - c->cp[2]};
    cx vinv = 1.0 / csqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    cx Y[16];
    for (int k = 0; k < 16; ++k) Y[k] = 0;
    sh_basis_cx(deg, v[0] * vinv, v[1] * vinv, v[2] * vinv, Y);
    int K = (deg + 1) * (deg + 1);
    cx rgb[3];
    for (int ch = 0; ch < 3; ++ch) {
        cx acc = 0;
        for (int k = 0; k < K; ++k) acc += Y[k] * sh[k * 3 + ch];
        acc += 0.5;
        if (creal(acc) < 0.0) { acc = 0; pi->clamped[ch] = 1; }
        rgb[ch] = acc;
    }

    cx sig = 1.0 / (1.0 + cexp(-o));

    out[0] = mx; out[1] = my;
    out[2] = ca; out[3] = cb; out[4] = cc;
    out[5] = sig;
    out[6] = rgb[0]; out[7] = rgb[1]; out[8] = rgb[2];
}

/* Gathers Gaussian i's parameters as complex numbers with zero imaginary part.
 * Parameters arrive as doubles (the stored FP32 values widened, or perturbed
 * values in finite-difference checks). */
static void load_gauss(int i, const double* means, const double* ls, const double* quats,
                       const double* opac, const double* sh, int Kst, int deg,
                       cx mu[3], cx l[3], cx q[4], cx* o, cx* shc) {
    for (int j = 0; j < 3; ++j) { mu[j] = means[3 * i + j]; l[j] = ls[3 * i + j]; }
    for (int j = 0; j < 4; ++j) q[j] = quats[4 * i + j];
    *o = opac[i];
    int K = (deg + 1) * (deg + 1);
    for (int k = 0; k < K; ++k)
        for (int ch = 0; ch < 3; ++ch) shc[k * 3 + ch] = sh[((size_t)i * Kst + k) * 3 + ch];
}

/* Per-Gaussian projection for one view.
 * out9 rows: mean2d x, y; conic a, b, c (d = -1/2 (a dx^2 + 2 b dx dy + c dy^2));
 * opacity; rgb.  Kst = SH coefficients stored per Gaussian, deg = degree used. */
void ora_preprocess(int N, const double* means, const double* ls, const double* quats,
                    const double* opac, const double* sh, int Kst, int deg,
                    const double* camv, const double* prmv,
                    double* out9, float* depth, int* radius, int* rect, int* tiles,
                    int* clamped, int* boundary, int* rect_lo, int* rect_hi) {
    cam_t c = load_cam(camv);
    prm_t p = load_prm(prmv);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < N; ++i) {
        cx mu[3], l[3], q[4], o, shc[48], out[9];
        load_gauss(i, means, ls, quats, opac, sh, Kst, deg, mu, l, q, &o, shc);
        proj_int pi;
        project_one(mu, l, q, o, shc, deg, &c, &p, out, &pi);
        for (int k = 0; k < 9; ++k) out9[9 * (size_t)i + k] = creal(out[k]);
        depth[i] = pi.depth;
        radius[i] = pi.culled ? 0 : pi.radius;
        for (int k = 0; k < 4; ++k) rect[4 * (size_t)i + k] = pi.culled ? 0 : pi.rect[k];
        tiles[i] = pi.culled ? 0 : pi.tiles;
        for (int k = 0; k < 3; ++k) clamped[3 * (size_t)i + k] = pi.clamped[k];
        boundary[i] = pi.boundary;
        for (int k = 0; k < 4; ++k) {
            /* a Gaussian culled for another reason never has a rect */
            int keep = pi.boundary || !pi.culled;
            rect_lo[4 * (size_t)i + k] = keep ? pi.rect_lo[k] : 0;
            rect_hi[4 * (size_t)i + k] = keep ? pi.rect_hi[k] : 0;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Per-tile Gaussian lists (Sec. 3: the splatting gives each pixel the list  */
/* of Gaussians whose rect covers its tile, sorted by depth).  Plain         */
/* collection and a comparison sort on (tile, depth key, Gaussian id).       */
/* ------------------------------------------------------------------------ */
typedef struct { int tile; uint32_t dkey; int id; } pair_t;

static int cmp_pair(const void* a, const void* b) {
    const pair_t* x = (const pair_t*)a;
    const pair_t* y = (const pair_t*)b;
    if (x->tile != y->tile) return x->tile < y->tile ? -1 : 1;
    if (x->dkey != y->dkey) return x->dkey < y->dkey ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

static uint32_t float_bits(float f) {
    uint32_t u;
    memcpy(&u, &f, 4);
    return u;
}

/* Returns the number of (tile, Gaussian) pairs.  With ids != NULL fills
 * tile_start[0..TX*TY] and ids[0..P) (the concatenated per-tile lists).
 * tile_mask (nullable, TX*TY bytes) keeps only the lists of the marked tiles
 * (the others are left empty); the returned count is then of kept pairs. */
long long ora_build_lists(int N, const int* rect, const int* tiles, const float* depth,
                          int TX, int TY, long long* tile_start, int* ids,
                          const unsigned char* tile_mask) {
    long long P = 0;
    for (int i = 0; i < N; ++i) {
        if (tiles[i] <= 0) continue;
        if (!tile_mask) { P += tiles[i]; continue; }
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i + 0]; tx < rect[4 * i + 2]; ++tx)
                P += tile_mask[ty * TX + tx] ? 1 : 0;
    }
    if (!ids) return P;
    pair_t* pr = (pair_t*)malloc(sizeof(pair_t) * (size_t)(P > 0 ? P : 1));
    long long k = 0;
    for (int i = 0; i < N; ++i) {
        if (tiles[i] <= 0) continue;
        for (int ty = rect[4 * i + 1]; ty < rect[4 * i + 3]; ++ty)
            for (int tx = rect[4 * i + 0]; tx < rect[4 * i + 2]; ++tx) {
                if (tile_mask && !tile_mask[ty * TX + tx]) continue;
                pr[k].tile = ty * TX + tx;
                pr[k].dkey = float_bits(depth[i]);
                pr[k].id = i;
                ++k;
            }
    }
    qsort(pr, (size_t)P, sizeof(pair_t), cmp_pair);
    for (int t = 0; t <= TX * TY; ++t) tile_start[t] = 0;
    for (long long j = 0; j < P; ++j) tile_start[pr[j].tile + 1]++;
    for (int t = 0; t < TX * TY; ++t) tile_start[t + 1] += tile_start[t];
    for (long long j = 0; j < P; ++j) ids[j] = pr[j].id;
    free(pr);
    return P;
}

/* ------------------------------------------------------------------------ */
/* Front-to-back compositing of one pixel (Sec. 3 and Sec. 4.3).             */
/*  alpha_hat = min(alpha_max, sigma g); entries with alpha_hat < alpha_min  */
/*  are skipped; the walk stops before blending an entry that would take T   */
/*  below t_min.  w_i = T_i alpha_i, C = sum w c (black background),         */
/*  H = -sum_{i=1}^{N+1} w log w with w_{N+1} = T_{N+1} (natural log).       */
/* ------------------------------------------------------------------------ */
typedef struct {
    int id;
    double ah, araw, T, dx, dy, g;
} blend_t;

static double rel(double a, double b) { return fabs(a - b) / fabs(b); }

/* Walks one pixel; fills bl (if not NULL) with the blended entries. */
/* Threshold band of the first_near output: list positions from the first
 * entry whose threshold test lies within this relative distance may be
 * decided differently by an FP32 implementation. */
#define NEAR_BAND 1e-3

static int walk_pixel(double px, double py, const int* ids, long long s, long long e,
                      const double* P9, const prm_t* p, blend_t* bl,
                      double C[3], double* Tout, double* Hout, int* last, int* neval,
                      double* margin, int* first_near) {
    double T = 1.0, swl = 0.0;
    int nb = 0;
    C[0] = C[1] = C[2] = 0.0;
    *last = 0;
    *neval = 0;
    *first_near = -1;
    double mg = INFINITY;
    for (long long j = s; j < e; ++j) {
        const double* g = P9 + 9 * (size_t)ids[j];
        double dx = px - g[0], dy = py - g[1];
        double d = -0.5 * (g[2] * dx * dx + 2.0 * g[3] * dx * dy + g[4] * dy * dy);
        double gd = exp(d);
        double araw = g[5] * gd;
        ++*neval;
        double me = fmin(rel(araw, p->amin), rel(araw, p->amax));
        mg = fmin(mg, me);
        if (me < NEAR_BAND && *first_near < 0) *first_near = (int)(j - s);
        double ah = fmin(p->amax, araw);
        if (ah < p->amin) continue;
        double testT = T * (1.0 - ah);
        mg = fmin(mg, rel(testT, p->tmin));
        if (rel(testT, p->tmin) < NEAR_BAND && *first_near < 0) *first_near = (int)(j - s);
        if (testT < p->tmin) break;
        double w = ah * T;
        for (int ch = 0; ch < 3; ++ch) C[ch] += w * g[6 + ch];
        swl += w * log(w);
        if (bl) {
            bl[nb].id = ids[j];
            bl[nb].ah = ah; bl[nb].araw = araw; bl[nb].T = T;
            bl[nb].dx = dx; bl[nb].dy = dy; bl[nb].g = gd;
        }
        ++nb;
        T = testT;
        *last = (int)(j - s + 1);
    }
    *Tout = T;
    *Hout = -(swl + T * log(T));
    *margin = mg;
    return nb;
}

/* Renders one view.  mask (nullable, H*W bytes) restricts the pixels computed;
 * other pixels are left untouched.  image: H*W*3, others H*W. */
void ora_render_fwd(int W, int H, const long long* tile_start, const int* ids,
                    const double* P9, const double* prmv, const unsigned char* mask,
                    double* image, double* finalT, int* last, double* entropy,
                    int* nblend, int* neval, double* margin, int* first_near) {
    prm_t p = load_prm(prmv);
    int TX = (W + p.tile - 1) / p.tile;
#pragma omp parallel for schedule(dynamic, 64)
    for (int pix = 0; pix < W * H; ++pix) {
        if (mask && !mask[pix]) continue;
        int u = pix % W, v = pix / W;
        int tile = (v / p.tile) * TX + (u / p.tile);
        double C[3], T, Hv, mg;
        int lst, ne, fn;
        int nb = walk_pixel(u + 0.5, v + 0.5, ids, tile_start[tile], tile_start[tile + 1], P9, &p,
                            NULL, C, &T, &Hv, &lst, &ne, &mg, &fn);
        for (int ch = 0; ch < 3; ++ch) image[3 * (size_t)pix + ch] = C[ch];
        finalT[pix] = T;
        last[pix] = lst;
        entropy[pix] = Hv;
        nblend[pix] = nb;
        neval[pix] = ne;
        margin[pix] = mg;
        first_near[pix] = fn;
    }
}

/* ------------------------------------------------------------------------ */
/* Entropy gradient of one pixel's weight distribution, three ways.          */
/* Input: the blended alphas a[0..n) in order; weights follow from          */
/* T_1 = 1, T_{i+1} = T_i (1 - a_i), w_i = T_i a_i, w_{n+1} = T_{n+1}.       */
/* ------------------------------------------------------------------------ */
static void weights_of(int n, const double* a, double* T /* n+1 */, double* w /* n+1 */) {
    T[0] = 1.0;
    for (int i = 0; i < n; ++i) {
        w[i] = T[i] * a[i];
        T[i + 1] = T[i] * (1.0 - a[i]);
    }
    w[n] = T[n];
}

double ora_entropy(int n, const double* a) {
    double* T = (double*)malloc(sizeof(double) * (n + 1));
    double* w = (double*)malloc(sizeof(double) * (n + 1));
    weights_of(n, a, T, w);
    double H = 0.0;
    for (int i = 0; i <= n; ++i) H -= w[i] * log(w[i]);
    free(T);
    free(w);
    return H;
}

/* Direct chain-rule sum (Suppl. B, "General formula" before R is introduced):
 * dH/da_i = (-log w_i - 1) T_i + sum_{k>i}^{n+1} (-log w_k - 1)(-w_k / (1 - a_i)). */
void ora_dH_da_direct(int n, const double* a, double* out) {
    double* T = (double*)malloc(sizeof(double) * (n + 1));
    double* w = (double*)malloc(sizeof(double) * (n + 1));
    weights_of(n, a, T, w);
    for (int i = 0; i < n; ++i) {
        double acc = (-log(w[i]) - 1.0) * T[i];
        for (int k = i + 1; k <= n; ++k) acc += (-log(w[k]) - 1.0) * (-w[k] / (1.0 - a[i]));
        out[i] = acc;
    }
    free(T);
    free(w);
}

/* Closed form of Sec. 4.4 with R_{i+1} = sum_{k=i+1}^{n+1} (log w_k + 1) w_k
 * evaluated as an explicit sum for every i. */
void ora_dH_da_closed(int n, const double* a, double* out) {
    double* T = (double*)malloc(sizeof(double) * (n + 1));
    double* w = (double*)malloc(sizeof(double) * (n + 1));
    weights_of(n, a, T, w);
    for (int i = 0; i < n; ++i) {
        double R = 0.0;
        for (int k = i + 1; k <= n; ++k) R += (log(w[k]) + 1.0) * w[k];
        out[i] = (-log(w[i]) - 1.0) * T[i] + R / (1.0 - a[i]);
    }
    free(T);
    free(w);
}

/* Algorithm 1 (Sec. 4.4): one reverse sweep carrying R. */
void ora_dH_da_alg1(int n, const double* a, double* out) {
    double* T = (double*)malloc(sizeof(double) * (n + 1));
    double* w = (double*)malloc(sizeof(double) * (n + 1));
    weights_of(n, a, T, w);
    double R = (log(w[n]) + 1.0) * w[n];
    for (int i = n - 1; i >= 0; --i) {
        out[i] = (-log(w[i]) - 1.0) * T[i] + R / (1.0 - a[i]);
        R = (log(w[i]) + 1.0) * w[i] + R;
    }
    free(T);
    free(w);
}

/* ------------------------------------------------------------------------ */
/* Backward of one view's compositing.  Given dL/dC (H*W*3) and dL/dH (H*W,  */
/* nullable), accumulates per-Gaussian gradients into grad9 (N*9, same row   */
/* meaning as out9): colour and entropy parts of dL/dalpha from the closed   */
/* forms with inner sums written out (O(n^2) per pixel), then Suppl. C:      */
/* dsigma = dalpha g, dd = dalpha sigma g, dconic = dd (-1/2 delta delta^T), */
/* dmean2d = dd conic delta, delta = x - mu'.  The min() clamp at alpha_max  */
/* passes no gradient.  mask (nullable) restricts the contributing pixels.   */
/* ------------------------------------------------------------------------ */
void ora_render_bwd(int W, int H, const long long* tile_start, const int* ids,
                    const double* P9, const double* prmv, const unsigned char* mask,
                    const double* dL_dC, const double* dL_dH, double* grad9) {
    prm_t p = load_prm(prmv);
    int TX = (W + p.tile - 1) / p.tile;
    long long maxlen = 0;
    int TY = (H + p.tile - 1) / p.tile;
    for (int t = 0; t < TX * TY; ++t)
        if (tile_start[t + 1] - tile_start[t] > maxlen) maxlen = tile_start[t + 1] - tile_start[t];
#pragma omp parallel
    {
        blend_t* bl = (blend_t*)malloc(sizeof(blend_t) * (size_t)(maxlen + 1));
        double* w = (double*)malloc(sizeof(double) * (size_t)(maxlen + 2));
#pragma omp for schedule(dynamic, 64)
        for (int pix = 0; pix < W * H; ++pix) {
            if (mask && !mask[pix]) continue;
            int u = pix % W, v = pix / W;
            int tile = (v / p.tile) * TX + (u / p.tile);
            double C[3], Tf, Hv, mg;
            int lst, ne, fn;
            int n = walk_pixel(u + 0.5, v + 0.5, ids, tile_start[tile], tile_start[tile + 1], P9,
                               &p, bl, C, &Tf, &Hv, &lst, &ne, &mg, &fn);
            const double* gC = dL_dC + 3 * (size_t)pix;
            double gH = dL_dH ? dL_dH[pix] : 0.0;
            for (int b = 0; b < n; ++b) w[b] = bl[b].ah * bl[b].T;
            w[n] = Tf;
            for (int b = 0; b < n; ++b) {
                const double* g = P9 + 9 * (size_t)bl[b].id;
                double om = 1.0 - bl[b].ah;
                /* colour: dC/da_b = T_b c_b - sum_{k>b} w_k c_k / (1 - a_b) */
                double dA = 0.0;
                for (int ch = 0; ch < 3; ++ch) {
                    double tail = 0.0;
                    for (int k = b + 1; k < n; ++k) tail += w[k] * P9[9 * (size_t)bl[k].id + 6 + ch];
                    dA += gC[ch] * (bl[b].T * g[6 + ch] - tail / om);
                }
                /* entropy: direct chain-rule sum over k >= b including background */
                if (gH != 0.0) {
                    double dH = (-log(w[b]) - 1.0) * bl[b].T;
                    for (int k = b + 1; k <= n; ++k) dH += (-log(w[k]) - 1.0) * (-w[k] / om);
                    dA += gH * dH;
                }
                double* G = grad9 + 9 * (size_t)bl[b].id;
                for (int ch = 0; ch < 3; ++ch) {
#pragma omp atomic
                    G[6 + ch] += w[b] * gC[ch];
                }
                if (bl[b].araw > p.amax) continue; /* clamped: no gradient to sigma g */
                double dsig = dA * bl[b].g;
                double dd = dA * bl[b].araw;
                double dx = bl[b].dx, dy = bl[b].dy;
                double da = dd * (-0.5 * dx * dx);
                double db = dd * (-dx * dy);
                double dc = dd * (-0.5 * dy * dy);
                double dmx = dd * (g[2] * dx + g[3] * dy);
                double dmy = dd * (g[3] * dx + g[4] * dy);
#pragma omp atomic
                G[0] += dmx;
#pragma omp atomic
                G[1] += dmy;
#pragma omp atomic
                G[2] += da;
#pragma omp atomic
                G[3] += db;
#pragma omp atomic
                G[4] += dc;
#pragma omp atomic
                G[5] += dsig;
            }
        }
        free(bl);
        free(w);
    }
}

/* ------------------------------------------------------------------------ */
/* Backward of the projection by the complex step: for every Gaussian with  */
/* gmask set (nullable = all) and every parameter x_j,                       */
/*   dL/dx_j += sum_k Im(out_k(x + i h e_j)) / h * grad9_k.                  */
/* Accumulates (+=) into the gradient arrays so that views can be summed.    */
/* ------------------------------------------------------------------------ */
void ora_preprocess_bwd(int N, const double* means, const double* ls, const double* quats,
                        const double* opac, const double* sh, int Kst, int deg,
                        const double* camv, const double* prmv, const double* grad9,
                        const unsigned char* gmask, double* g_means, double* g_ls,
                        double* g_quats, double* g_opac, double* g_sh) {
    cam_t c = load_cam(camv);
    prm_t p = load_prm(prmv);
    const double h = 1e-30;
    int K = (deg + 1) * (deg + 1);
#pragma omp parallel for schedule(dynamic, 256)
    for (int i = 0; i < N; ++i) {
        if (gmask && !gmask[i]) continue;
        const double* G = grad9 + 9 * (size_t)i;
        int any = 0;
        for (int k = 0; k < 9; ++k) any |= (G[k] != 0.0);
        if (!any) continue;
        cx mu[3], l[3], q[4], o, shc[48], out[9];
        load_gauss(i, means, ls, quats, opac, sh, Kst, deg, mu, l, q, &o, shc);
        proj_int pi;
        /* 11 geometric/opacity parameters, then the K*3 SH coefficients */
        int nparam = 11 + 3 * K;
        for (int j = 0; j < nparam; ++j) {
            cx* slot;
            if (j < 3) slot = &mu[j];
            else if (j < 6) slot = &l[j - 3];
            else if (j < 10) slot = &q[j - 6];
            else if (j == 10) slot = &o;
            else slot = &shc[j - 11];
            cx saved = *slot;
            *slot = creal(saved) + I * h;
            project_one(mu, l, q, o, shc, deg, &c, &p, out, &pi);
            *slot = saved;
            double acc = 0.0;
            if (!pi.culled)
                for (int k = 0; k < 9; ++k) acc += cimag(out[k]) / h * G[k];
            if (j < 3) g_means[3 * (size_t)i + j] += acc;
            else if (j < 6) g_ls[3 * (size_t)i + j - 3] += acc;
            else if (j < 10) g_quats[4 * (size_t)i + j - 6] += acc;
            else if (j == 10) g_opac[i] += acc;
            else {
                int kk = (j - 11) / 3, ch = (j - 11) % 3;
                g_sh[((size_t)i * Kst + kk) * 3 + ch] += acc;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Loss of one view (Sec. 3 eq. base with lambda = 0, plus Sec. 4.3):        */
/*   L_v = (1/(3M)) sum |C - C*| + gamma (1/M) sum_j H_j, M = H*W,          */
/* scaled by view_weight; writes dL/dC and dL/dH.  Returns L_v * weight.     */
/* sign(0) = 0.                                                             */
/* ------------------------------------------------------------------------ */
double ora_loss(int M, const double* image, const float* target, const double* entropy,
                double gamma, double view_weight, double* dL_dC, double* dL_dH) {
    double l1 = 0.0, hs = 0.0;
    for (int j = 0; j < M; ++j) {
        for (int ch = 0; ch < 3; ++ch) {
            double r = image[3 * (size_t)j + ch] - (double)target[3 * (size_t)j + ch];
            l1 += fabs(r);
            double sg = r > 0.0 ? 1.0 : (r < 0.0 ? -1.0 : 0.0);
            dL_dC[3 * (size_t)j + ch] = view_weight * sg / (3.0 * M);
        }
        hs += entropy[j];
        dL_dH[j] = view_weight * gamma / M;
    }
    return view_weight * (l1 / (3.0 * M) + gamma * hs / M);
}

/* ------------------------------------------------------------------------ */
/* SSIM of one view (the D-SSIM term of L_base, Sec. 3 Eq. base; the paper   */
/* does not define it: the reading is 3DGS's, D-SSIM = 1 - SSIM with the     */
/* 11x11 Gaussian window of sigma 1.5 (normalised), zero padding outside the */
/* image, C1 = 0.01^2, C2 = 0.03^2, SSIM = mean over pixels and channels).   */
/* Per pixel q and channel, over the 121 window samples (padding included as */
/* zeros): mu_x = E[x], sigma_x^2 = E[(x - mu_x)^2], sigma_xy likewise;       */
/* S = (2 mu_x mu_y + C1)(2 sigma_xy + C2) / ((mu_x^2 + mu_y^2 + C1)         */
/*     (sigma_x^2 + sigma_y^2 + C2)).                                         */
/* grad (nullable, H*W*3): d SSIM / d image, from                             */
/*   dS(q)/dx(p) = G(q-p) [dS/dmu_x + 2 (x(p) - mu_x(q)) dS/dsigma_x^2        */
/*                         + (y(p) - mu_y(q)) dS/dsigma_xy],                  */
/* (d sigma_x^2(q) / dx(p) = 2 G(q-p)(x(p) - mu_x(q)) since the weights sum  */
/* to 1), summed over the windows q that contain p, divided by 3 H W.        */
/* ------------------------------------------------------------------------ */
#define SSIM_R 5
#define SSIM_C1 (0.01 * 0.01)
#define SSIM_C2 (0.03 * 0.03)

static void ssim_window(double g[2 * SSIM_R + 1]) {
    double s = 0.0;
    for (int k = -SSIM_R; k <= SSIM_R; ++k) {
        g[k + SSIM_R] = exp(-(double)(k * k) / (2.0 * 1.5 * 1.5));
        s += g[k + SSIM_R];
    }
    for (int k = 0; k < 2 * SSIM_R + 1; ++k) g[k] /= s;
}

double ora_ssim(int W, int H, const double* img, const float* tgt, double* grad) {
    double g[2 * SSIM_R + 1];
    ssim_window(g);
    const size_t M = (size_t)W * H;
    /* per pixel and channel: mu_x, mu_y, dS/dmu_x, dS/dsigma_x^2, dS/dsigma_xy */
    double* maps = grad ? (double*)malloc(sizeof(double) * 5 * 3 * M) : NULL;
    double total = 0.0;
#pragma omp parallel for reduction(+ : total) schedule(static)
    for (long long q = 0; q < (long long)M; ++q) {
        int u = (int)(q % W), v = (int)(q / W);
        for (int ch = 0; ch < 3; ++ch) {
            double mx = 0, my = 0;
            for (int dy = -SSIM_R; dy <= SSIM_R; ++dy)
                for (int dx = -SSIM_R; dx <= SSIM_R; ++dx) {
                    int uu = u + dx, vv = v + dy;
                    if (uu < 0 || uu >= W || vv < 0 || vv >= H) continue;
                    double w = g[dy + SSIM_R] * g[dx + SSIM_R];
                    size_t k = 3 * ((size_t)vv * W + uu) + ch;
                    mx += w * img[k];
                    my += w * (double)tgt[k];
                }
            double sxx = 0, syy = 0, sxy = 0;
            for (int dy = -SSIM_R; dy <= SSIM_R; ++dy)
                for (int dx = -SSIM_R; dx <= SSIM_R; ++dx) {
                    int uu = u + dx, vv = v + dy;
                    double w = g[dy + SSIM_R] * g[dx + SSIM_R];
                    double a = -mx, b = -my;  /* padding samples are zero */
                    if (!(uu < 0 || uu >= W || vv < 0 || vv >= H)) {
                        size_t k = 3 * ((size_t)vv * W + uu) + ch;
                        a = img[k] - mx;
                        b = (double)tgt[k] - my;
                    }
                    sxx += w * a * a;
                    syy += w * b * b;
                    sxy += w * a * b;
                }
            double A1 = 2 * mx * my + SSIM_C1, A2 = 2 * sxy + SSIM_C2;
            double B1 = mx * mx + my * my + SSIM_C1, B2 = sxx + syy + SSIM_C2;
            double D = B1 * B2, S = A1 * A2 / D;
            total += S;
            if (maps) {
                double* m = maps + 15 * (size_t)q + 5 * ch;
                m[0] = mx;
                m[1] = my;
                m[2] = (2 * my * A2 - S * 2 * mx * B2) / D;  /* dS/dmu_x, sigmas fixed */
                m[3] = -S / B2;                              /* dS/dsigma_x^2 */
                m[4] = 2 * A1 / D;                           /* dS/dsigma_xy */
            }
        }
    }
    if (grad) {
#pragma omp parallel for schedule(static)
        for (long long p = 0; p < (long long)M; ++p) {
            int u = (int)(p % W), v = (int)(p / W);
            for (int ch = 0; ch < 3; ++ch) {
                double xp = img[3 * (size_t)p + ch], yp = (double)tgt[3 * (size_t)p + ch];
                double acc = 0.0;
                for (int dy = -SSIM_R; dy <= SSIM_R; ++dy)
                    for (int dx = -SSIM_R; dx <= SSIM_R; ++dx) {
                        int uu = u + dx, vv = v + dy;  /* window centre q containing p */
                        if (uu < 0 || uu >= W || vv < 0 || vv >= H) continue;
                        double w = g[dy + SSIM_R] * g[dx + SSIM_R];
                        const double* m = maps + 15 * ((size_t)vv * W + uu) + 5 * ch;
                        acc += w * (m[2] + 2 * (xp - m[0]) * m[3] + (yp - m[1]) * m[4]);
                    }
                grad[3 * (size_t)p + ch] = acc / (3.0 * M);
            }
        }
        free(maps);
    }
    return total / (3.0 * M);
}

/* Scale reset (Sec. 4.2): s <- zeta s for every Gaussian, i.e. the stored
 * log-scale gains log(zeta). */
void ora_scale_reset(int n, const float* log_scales, double zeta, double* out) {
    for (int i = 0; i < n; ++i) out[i] = (double)log_scales[i] + log(zeta);
}

int ora_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
