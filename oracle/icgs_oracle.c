/*
 * icgs_oracle.c -- plain, slow FP64 CPU oracle for instant colorization of Gaussian splats
 * (arXiv 2604.17155, Sec. 3 and Alg. 1).
 *
 * TEST INFRASTRUCTURE. Only the test-suite, the smoke check and the benchmark's CPU-baseline leg
 * may load or call this file. It shares no code, header, table or constant generator with the
 * CUDA library, and the library never calls it.
 *
 * What it computes, per camera j (everything in double precision):
 *   - the projection of every Gaussian (Eq. 1; the paper renders "following Kerbl et al.", so the
 *     3DGS conventions are taken: EWA first-order Jacobian with the 1.3*tan(fov/2) clamp, 0.3 px^2
 *     dilation, alpha = min(0.99, o exp(-q/2)), skip alpha < 1/255, stop before a Gaussian when
 *     T(1-alpha) < 1e-4);
 *   - for every pixel, the front-to-back alpha-blend of Eq. 2 over the depth-ordered list of the
 *     Gaussians whose candidate box contains the pixel, giving the per-pixel visibility
 *     V_{i,x,y} = alpha_i T_i of Eq. 4;
 *   - the per-image sums of Eq. 5 and Eq. 6: V_i^j = sum V_{i,x,y} and S_i^{j,k} = sum V_{i,x,y} t_k
 *     (so that C_hat = S / V is never formed);
 *   - the render of Eq. 1-3 for given SH coefficients, and the adjoint walk used for gradients.
 *   - the real orthonormal spherical-harmonic basis of Eq. 3 by the associated-Legendre recurrence.
 * The fold into normal equations and the regularised solve (Eq. 13-14) are written in numpy in
 * oracle.py.
 *
 * Decisions that must be taken identically on both sides are taken in a fixed precision here:
 * the depth used for ordering (and for the near-plane test) is the float32 key
 * fma(W22, z, fma(W21, y, fma(W20, x, W23))), each step one correctly rounded fused multiply-add
 * in float32 (C99 fmaf); ties are broken by the Gaussian index. Everything else here is double
 * with no contraction (compile with -ffp-contract=off). Threshold decisions on alpha and T
 * are taken in double. A renderer that computes alpha and T in lower precision can take a decision
 * that falls close to its threshold the other way; walk_pixel records, per Gaussian, an upper bound
 * on how much weight such flips can move (its "stake"; see walk_pixel), so a test can tell a
 * threshold flip from an arithmetic error.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
  int32_t width, height;
  double fx, fy, cx, cy;
  double w2c[12]; /* row-major [R|t] */
  double near_z;
} ocam_t;

typedef struct {
  int32_t visible;
  double mx, my;             /* projected mean in pixels */
  double cxx, cxy, cyy;      /* 2D covariance incl. dilation */
  double ca, cb, cc;         /* conic = inverse 2D covariance */
  double depth;              /* camera-space z */
  float key;                 /* float32 depth key (fused multiply-adds): the ordering key */
  double opacity;
  double qthr;               /* 2 ln(255 o): alpha >= 1/255 <=> q <= qthr (ignoring the 0.99 cap) */
  int32_t x0, x1, y0, y1;    /* candidate pixel box, inclusive */
} oproj_t;

#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX 0.99
#define T_MIN 1e-4
#define DILATION 0.3

/* Test-only scale factors of the two thresholds (1 = the renderer's values). A test moves a
 * threshold by a relative amount within the stake margin to flip, on purpose, every decision that
 * lies that close to it, and checks the result against the stake-derived bound. */
static double g_alpha_min_scale = 1.0, g_t_min_scale = 1.0;

/* Rotation matrix of the unit quaternion (w,x,y,z) (Hamilton convention). */
static void quat_to_rot(const float* qf, double R[9]) {
  double w = qf[0], x = qf[1], y = qf[2], z = qf[3];
  double n = sqrt(w * w + x * x + y * y + z * z);
  w /= n; x /= n; y /= n; z /= n;
  R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

/* Project Gaussian (mean, scale, quat, opacity) into camera c (Eq. 1 with the 3DGS model). */
static void project_one(const float* mean, const float* scale, const float* quat, float opac,
                        const ocam_t* c, oproj_t* p) {
  memset(p, 0, sizeof(*p));
  const double* W = c->w2c;
  double x = mean[0], y = mean[1], z = mean[2];
  double tx = ((W[0] * x + W[1] * y) + W[2] * z) + W[3];
  double ty = ((W[4] * x + W[5] * y) + W[6] * z) + W[7];
  double tz = ((W[8] * x + W[9] * y) + W[10] * z) + W[11];
  /* the ordering key: three float32 fused multiply-adds (W holds float32 values exactly) */
  const float key = fmaf((float)W[10], mean[2], fmaf((float)W[9], mean[1], fmaf((float)W[8], mean[0], (float)W[11])));
  p->depth = tz;
  p->key = key;
  p->opacity = opac;
  if (!(key > (float)c->near_z)) return;         /* behind the near plane (on the key) */
  if (!((double)opac * 255.0 >= 1.0)) return;    /* alpha < 1/255 everywhere */

  /* 3D covariance Sigma = R S S^T R^T */
  double R[9];
  quat_to_rot(quat, R);
  double M[9];
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) M[r * 3 + k] = R[r * 3 + k] * (double)scale[k];
  double S3[9];
  for (int r = 0; r < 3; ++r)
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
      for (int l = 0; l < 3; ++l) s += M[r * 3 + l] * M[k * 3 + l];
      S3[r * 3 + k] = s;
    }

  /* Jacobian of the pinhole projection at the (clamped) camera-space mean */
  double limx = 1.3 * ((double)c->width / (2.0 * c->fx));
  double limy = 1.3 * ((double)c->height / (2.0 * c->fy));
  double ux = tx / tz, uy = ty / tz;
  if (ux < -limx) ux = -limx;
  if (ux > limx) ux = limx;
  if (uy < -limy) uy = -limy;
  if (uy > limy) uy = limy;
  double J[6] = {c->fx / tz, 0.0, -c->fx * ux / tz, 0.0, c->fy / tz, -c->fy * uy / tz};
  /* T = J Wrot (2x3) */
  double T[6];
  for (int r = 0; r < 2; ++r)
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
      for (int l = 0; l < 3; ++l) s += J[r * 3 + l] * W[l * 4 + k];
      T[r * 3 + k] = s;
    }
  /* Sigma' = T Sigma T^T + 0.3 I */
  double C2[4];
  for (int r = 0; r < 2; ++r)
    for (int k = 0; k < 2; ++k) {
      double s = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) s += T[r * 3 + a] * S3[a * 3 + b] * T[k * 3 + b];
      C2[r * 2 + k] = s;
    }
  double a = C2[0] + DILATION, b = 0.5 * (C2[1] + C2[2]), cyy = C2[3] + DILATION;
  double det = a * cyy - b * b;
  if (!(det > 0.0)) return;
  p->cxx = a; p->cxy = b; p->cyy = cyy;
  p->ca = cyy / det; p->cb = -b / det; p->cc = a / det;
  p->mx = c->fx * tx / tz + c->cx;
  p->my = c->fy * ty / tz + c->cy;
  p->qthr = 2.0 * log(255.0 * (double)opac);

  /* candidate box: the disc of radius sqrt(lambda_max * qthr) contains every pixel centre with
     alpha >= 1/255; one extra pixel on each side keeps it a superset under rounding */
  double lmax = 0.5 * (a + cyy) + sqrt(0.25 * (a - cyy) * (a - cyy) + b * b);
  double rad = sqrt(lmax * (p->qthr > 0.0 ? p->qthr : 0.0));
  double fx0 = ceil(p->mx - rad - 0.5) - 1.0, fx1 = floor(p->mx + rad - 0.5) + 1.0;
  double fy0 = ceil(p->my - rad - 0.5) - 1.0, fy1 = floor(p->my + rad - 0.5) + 1.0;
  if (fx0 < 0.0) fx0 = 0.0;
  if (fy0 < 0.0) fy0 = 0.0;
  if (fx1 > c->width - 1) fx1 = c->width - 1;
  if (fy1 > c->height - 1) fy1 = c->height - 1;
  if (fx0 > fx1 || fy0 > fy1) return;
  p->x0 = (int32_t)fx0; p->x1 = (int32_t)fx1; p->y0 = (int32_t)fy0; p->y1 = (int32_t)fy1;
  p->visible = 1;
}

static void project_all(int64_t n, const float* means, const float* scales, const float* quats,
                        const float* opac, const ocam_t* cam, oproj_t* P) {
  for (int64_t i = 0; i < n; ++i)
    project_one(means + 3 * i, scales + 3 * i, quats + 4 * i, opac[i], cam, P + i);
}

/* ---------------------------------------------------------------------------------------------
 * Depth order: (float32 depth key, index) ascending.
 * ------------------------------------------------------------------------------------------- */
typedef struct { float key; int32_t idx; } okey_t;
static int cmp_key(const void* A, const void* B) {
  const okey_t* a = (const okey_t*)A;
  const okey_t* b = (const okey_t*)B;
  if (a->key < b->key) return -1;
  if (a->key > b->key) return 1;
  return (a->idx > b->idx) - (a->idx < b->idx);
}

/* Visible Gaussians in depth order; returns the count. */
static int64_t depth_order(int64_t n, const oproj_t* P, int32_t* order) {
  okey_t* tmp = (okey_t*)malloc(sizeof(okey_t) * (size_t)(n > 0 ? n : 1));
  int64_t m = 0;
  for (int64_t i = 0; i < n; ++i)
    if (P[i].visible) { tmp[m].key = P[i].key; tmp[m].idx = (int32_t)i; ++m; }
  qsort(tmp, (size_t)m, sizeof(okey_t), cmp_key);
  for (int64_t k = 0; k < m; ++k) order[k] = tmp[k].idx;
  free(tmp);
  return m;
}

/* ---------------------------------------------------------------------------------------------
 * Per-pixel front-to-back walk (Eq. 2 and Eq. 4).
 * ------------------------------------------------------------------------------------------- */
typedef struct {
  int32_t i;
  double alpha, w, T;   /* T = transmittance in front of this Gaussian, w = alpha*T */
  double e;             /* exp(-q/2), so alpha = min(0.99, o*e) */
  int32_t clamped;      /* alpha hit the 0.99 cap */
} ocontrib_t;

/* Stake bookkeeping of one pixel's walk. A decision is "near" its threshold when alpha lies within
 * relative margin delta_a of 1/255, or T(1 - alpha) within delta_t (+ the T perturbation already at
 * stake, below) of 1e-4. Each entry is an upper bound on |dV|, the change of the pixel's weight of
 * that Gaussian when any set of near decisions is taken the other way:
 *   own[i]  the Gaussian's own near decision: alpha_hi T' for an alpha decision (alpha_hi =
 *           (1 + delta_a)/255 bounds alpha there), alpha T' for a stop decision;
 *   up[i]   near decisions in front of it: rel * w for a contributor, where rel bounds
 *           |T_other / T - 1| (each alpha flip scales T by (1 - alpha)^(+-1), so rel grows by the
 *           factor 1 + alpha_hi / (1 - alpha_hi); a stop in front at stake adds 1, since the other
 *           side may then drop the Gaussian); and, behind a stop at stake, T' min(alpha, 0.99) for
 *           every Gaussian the other side could still take (alpha >= (1 - delta_a)/255);
 *   tw[i]   the same amounts times the pixel's target norm |t_p|_2, for the bound on the
 *           coefficients (the pair's right-hand side moves by dV t_p).
 * T' = T (1 + rel) bounds the other side's transmittance. */
typedef struct {
  double delta_a, delta_t;
  double* own;
  double* up;
  double* tw;
  double tnorm;
  int hits;      /* stake entries added in this pixel */
} ostake_t;

static void stake_add(ostake_t* sk, double* arr, int32_t i, double v) {
  arr[i] += v;
  if (sk->tw) sk->tw[i] += v * sk->tnorm;
  sk->hits++;
}

/* Walks `list` (indices in depth order) for the pixel with centre (pxc, pyc). Writes the
 * contributors to `out` and returns their number. With `sk`, near decisions add their stake. */
static int walk_pixel(const oproj_t* P, const int32_t* list, int len, double pxc, double pyc,
                      ocontrib_t* out, ostake_t* sk) {
  const double amin = ALPHA_MIN * g_alpha_min_scale, tmin = T_MIN * g_t_min_scale;
  double T = 1.0;
  int m = 0;
  double rel = 0.0; /* bound on |T_other / T - 1| behind the Gaussians walked so far */
  for (int k = 0; k < len; ++k) {
    const oproj_t* g = P + list[k];
    double dx = pxc - g->mx, dy = pyc - g->my;
    double q = g->ca * dx * dx + 2.0 * g->cb * dx * dy + g->cc * dy * dy;
    double e = exp(-0.5 * q);
    double oe = g->opacity * e;
    double alpha = oe < ALPHA_MAX ? oe : ALPHA_MAX;
    const double rel_front = rel; /* in front of this Gaussian: its own decisions do not count */
    if (sk && fabs(alpha - amin) <= sk->delta_a * amin) {
      const double a_hi = amin * (1.0 + sk->delta_a);
      stake_add(sk, sk->own, list[k], a_hi * T * (1.0 + rel_front));
      rel = (1.0 + rel) * (1.0 + a_hi / (1.0 - a_hi)) - 1.0;
    }
    if (alpha < amin) continue;
    double test_T = T * (1.0 - alpha);
    int stop_at_stake = 0;
    if (sk && fabs(test_T - tmin) <= (sk->delta_t + rel_front) * tmin) {
      stake_add(sk, sk->own, list[k], alpha * T * (1.0 + rel_front));
      rel += 1.0;
      stop_at_stake = 1;
    }
    if (test_T < tmin) {
      if (sk && stop_at_stake) {
        /* the other side may go on: everything behind that it could take is at stake */
        for (int r = k + 1; r < len; ++r) {
          const oproj_t* h = P + list[r];
          double ex = pxc - h->mx, ey = pyc - h->my;
          double qq = h->ca * ex * ex + 2.0 * h->cb * ex * ey + h->cc * ey * ey;
          double aa = h->opacity * exp(-0.5 * qq);
          if (aa >= amin * (1.0 - sk->delta_a))
            stake_add(sk, sk->up, list[r], T * (1.0 + rel_front) * (aa < ALPHA_MAX ? aa : ALPHA_MAX));
        }
      }
      break;
    }
    out[m].i = list[k];
    out[m].alpha = alpha;
    out[m].T = T;
    out[m].w = alpha * T;
    out[m].e = e;
    out[m].clamped = oe >= ALPHA_MAX;
    if (sk && rel_front > 0.0) stake_add(sk, sk->up, list[k], rel_front * out[m].w);
    ++m;
    T = test_T;
  }
  return m;
}

/* Builds, strip by strip, the candidate list of every pixel (Gaussians whose candidate box
 * contains it, in depth order) and calls `visit` on each pixel selected by `mask`. */
typedef void (*visit_fn)(void* ctx, int32_t px, int32_t py, const int32_t* list, int len);

#define STRIP 16
static void for_each_pixel(const ocam_t* cam, int64_t nvis, const int32_t* order, const oproj_t* P,
                           const uint8_t* mask, visit_fn visit, void* ctx) {
  int W = cam->width, H = cam->height;
  int64_t* start = (int64_t*)malloc(sizeof(int64_t) * ((size_t)W * STRIP + 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * ((size_t)W * STRIP));
  for (int ys = 0; ys < H; ys += STRIP) {
    int ye = ys + STRIP < H ? ys + STRIP : H;
    int64_t npx = (int64_t)W * (ye - ys);
    if (mask) { /* strips without a selected pixel need no lists */
      int any = 0;
      for (int64_t p = 0; p < npx && !any; ++p) any = mask[(int64_t)ys * W + p] != 0;
      if (!any) continue;
    }
    memset(start, 0, sizeof(int64_t) * (size_t)(npx + 1));
    for (int64_t r = 0; r < nvis; ++r) {
      const oproj_t* g = P + order[r];
      int y0 = g->y0 > ys ? g->y0 : ys, y1 = g->y1 < ye - 1 ? g->y1 : ye - 1;
      for (int y = y0; y <= y1; ++y)
        for (int x = g->x0; x <= g->x1; ++x) start[(int64_t)(y - ys) * W + x + 1] += 1;
    }
    for (int64_t p = 0; p < npx; ++p) start[p + 1] += start[p];
    int32_t* lists = (int32_t*)malloc(sizeof(int32_t) * (size_t)(start[npx] > 0 ? start[npx] : 1));
    memcpy(fill, start, sizeof(int64_t) * (size_t)npx);
    for (int64_t r = 0; r < nvis; ++r) {
      const oproj_t* g = P + order[r];
      int y0 = g->y0 > ys ? g->y0 : ys, y1 = g->y1 < ye - 1 ? g->y1 : ye - 1;
      for (int y = y0; y <= y1; ++y)
        for (int x = g->x0; x <= g->x1; ++x) {
          int64_t p = (int64_t)(y - ys) * W + x;
          lists[fill[p]++] = order[r];
        }
    }
    for (int y = ys; y < ye; ++y)
      for (int x = 0; x < W; ++x) {
        if (mask && !mask[(int64_t)y * W + x]) continue;
        int64_t p = (int64_t)(y - ys) * W + x;
        visit(ctx, x, y, lists + start[p], (int)(start[p + 1] - start[p]));
      }
    free(lists);
  }
  free(start);
  free(fill);
}

/* Same visitor, but every pixel's list is every visible Gaussian (brute force, no boxes). */
static void for_each_pixel_bruteforce(const ocam_t* cam, int64_t nvis, const int32_t* order,
                                      const uint8_t* mask, visit_fn visit, void* ctx) {
  for (int y = 0; y < cam->height; ++y)
    for (int x = 0; x < cam->width; ++x) {
      if (mask && !mask[(int64_t)y * cam->width + x]) continue;
      visit(ctx, x, y, order, (int)nvis);
    }
}

/* ---------------------------------------------------------------------------------------------
 * Visitors
 * ------------------------------------------------------------------------------------------- */
typedef struct {
  const ocam_t* cam;
  const oproj_t* P;
  int32_t K;
  const double* targets;     /* [H,W,K] */
  double* V;                 /* [n] */
  double* S;                 /* [n,K] */
  ostake_t stake;            /* stake arrays (own NULL: no bookkeeping) */
  uint8_t* pix_flag;         /* [H,W] or NULL: 1 where the pixel's walk has a near decision (or,
                                with `dirty`, a contributor marked dirty) */
  double* flag_w;            /* [n] or NULL: each Gaussian's weight in such pixels */
  const uint8_t* dirty;      /* [n] or NULL: Gaussians whose sums a flip elsewhere may have moved */
  int64_t pairs;
  ocontrib_t* scratch;
  /* render */
  const double* colors;      /* [n,K] */
  double* image;             /* [H,W,K] */
  /* weight listing */
  int64_t cap, count;
  int32_t* out_pix;
  int32_t* out_gid;
  double* out_w;
  double* out_T;             /* or NULL */
  /* adjoint */
  const double* a;           /* [n,K] dL/dS */
  const double* beta;        /* [n]   dL/dV */
  double* grad_t;            /* [H,W,K] */
  double* grad_o;            /* [n] */
} octx_t;

static void visit_accumulate(void* vctx, int32_t px, int32_t py, const int32_t* list, int len) {
  octx_t* c = (octx_t*)vctx;
  const double* t = c->targets + ((int64_t)py * c->cam->width + px) * c->K;
  ostake_t sk = c->stake;
  const int with_stake = sk.own != NULL && sk.up != NULL;
  if (with_stake) {
    double nn = 0.0;
    for (int k = 0; k < c->K; ++k) nn += t[k] * t[k];
    sk.tnorm = sqrt(nn);
  }
  sk.hits = 0;
  int m = walk_pixel(c->P, list, len, px + 0.5, py + 0.5, c->scratch, with_stake ? &sk : NULL);
  int flagged = sk.hits > 0;
  for (int r = 0; r < m && !flagged && c->dirty; ++r) flagged = c->dirty[c->scratch[r].i] != 0;
  if (flagged) {
    if (c->pix_flag) c->pix_flag[(int64_t)py * c->cam->width + px] = 1;
    if (c->flag_w)
      for (int r = 0; r < m; ++r) c->flag_w[c->scratch[r].i] += c->scratch[r].w;
  }
  for (int r = 0; r < m; ++r) {
    int32_t i = c->scratch[r].i;
    double w = c->scratch[r].w;
    c->V[i] += w;
    for (int k = 0; k < c->K; ++k) c->S[(int64_t)i * c->K + k] += w * t[k];
  }
  c->pairs += m;
}

static void visit_render(void* vctx, int32_t px, int32_t py, const int32_t* list, int len) {
  octx_t* c = (octx_t*)vctx;
  int m = walk_pixel(c->P, list, len, px + 0.5, py + 0.5, c->scratch, NULL);
  double* img = c->image + ((int64_t)py * c->cam->width + px) * c->K;
  for (int r = 0; r < m; ++r)
    for (int k = 0; k < c->K; ++k) img[k] += c->scratch[r].w * c->colors[(int64_t)c->scratch[r].i * c->K + k];
  c->pairs += m;
}

static void visit_weights(void* vctx, int32_t px, int32_t py, const int32_t* list, int len) {
  octx_t* c = (octx_t*)vctx;
  int m = walk_pixel(c->P, list, len, px + 0.5, py + 0.5, c->scratch, NULL);
  for (int r = 0; r < m; ++r) {
    if (c->count < c->cap) {
      c->out_pix[c->count] = py * c->cam->width + px;
      c->out_gid[c->count] = c->scratch[r].i;
      c->out_w[c->count] = c->scratch[r].w;
      if (c->out_T) c->out_T[c->count] = c->scratch[r].T;
    }
    c->count++;
  }
}

/* Adjoint of F = sum_pixels sum_n g_n w_n with g_n = beta_i + sum_k a_ik t_k (the pixel's
 * contribution to L through V and S): dF/dt_k = sum_n w_n a_{i_n k};
 * dF/dalpha_n = g_n T_n - (sum_{l>n} g_l w_l) / (1 - alpha_n); dalpha/do = e unless capped. */
static void visit_adjoint(void* vctx, int32_t px, int32_t py, const int32_t* list, int len) {
  octx_t* c = (octx_t*)vctx;
  int m = walk_pixel(c->P, list, len, px + 0.5, py + 0.5, c->scratch, NULL);
  int K = c->K;
  const double* t = c->targets + ((int64_t)py * c->cam->width + px) * K;
  double* gt = c->grad_t + ((int64_t)py * c->cam->width + px) * K;
  double suffix = 0.0;
  for (int r = m - 1; r >= 0; --r) {
    const ocontrib_t* q = c->scratch + r;
    const double* a = c->a + (int64_t)q->i * K;
    double g = c->beta[q->i];
    for (int k = 0; k < K; ++k) {
      g += a[k] * t[k];
      gt[k] += q->w * a[k];
    }
    double dalpha = g * q->T - suffix / (1.0 - q->alpha);
    if (!q->clamped) c->grad_o[q->i] += dalpha * q->e;
    suffix += g * q->w;
  }
  c->pairs += m;
}

/* Common driver: project, order, walk. */
static int run_camera(int64_t n, const float* means, const float* scales, const float* quats,
                      const float* opac, const ocam_t* cam, const uint8_t* mask, int brute,
                      visit_fn visit, octx_t* ctx) {
  oproj_t* P = (oproj_t*)malloc(sizeof(oproj_t) * (size_t)(n > 0 ? n : 1));
  int32_t* order = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  ocontrib_t* scratch = (ocontrib_t*)malloc(sizeof(ocontrib_t) * (size_t)(n > 0 ? n : 1));
  if (!P || !order || !scratch) { free(P); free(order); free(scratch); return -1; }
  project_all(n, means, scales, quats, opac, cam, P);
  int64_t nvis = depth_order(n, P, order);
  ctx->cam = cam;
  ctx->P = P;
  ctx->scratch = scratch;
  if (brute)
    for_each_pixel_bruteforce(cam, nvis, order, mask, visit, ctx);
  else
    for_each_pixel(cam, nvis, order, P, mask, visit, ctx);
  free(P);
  free(order);
  free(scratch);
  return 0;
}

/* ---------------------------------------------------------------------------------------------
 * Exported entry points (called through ctypes from oracle.py)
 * ------------------------------------------------------------------------------------------- */

/* Per-Gaussian projection record, 16 doubles each:
 * visible, mx, my, cov_xx, cov_xy, cov_yy, conic_a, conic_b, conic_c, depth, key, qthr, x0, x1, y0, y1 */
int icgso_project(int64_t n, const float* means, const float* scales, const float* quats,
                  const float* opac, const ocam_t* cam, double* out) {
  for (int64_t i = 0; i < n; ++i) {
    oproj_t p;
    project_one(means + 3 * i, scales + 3 * i, quats + 4 * i, opac[i], cam, &p);
    double* o = out + 16 * i;
    o[0] = p.visible; o[1] = p.mx; o[2] = p.my; o[3] = p.cxx; o[4] = p.cxy; o[5] = p.cyy;
    o[6] = p.ca; o[7] = p.cb; o[8] = p.cc; o[9] = p.depth; o[10] = p.key; o[11] = p.qthr;
    o[12] = p.x0; o[13] = p.x1; o[14] = p.y0; o[15] = p.y1;
  }
  return 0;
}

/* V_i = sum_pixels alpha_i T_i (Eq. 4-5), S_ik = sum_pixels alpha_i T_i t_k (numerator of Eq. 6).
 * V, S and the stakes (walk_pixel; stake_own or stake_up NULL: none; stake_tw may be NULL) are accumulated
 * into (the caller zeroes them). delta_a, delta_t: the relative margins of the alpha and stop
 * decisions. pix_flag [H,W] (may be NULL) is set to 1 at every pixel whose walk has a near decision
 * or, with dirty [n] (may be NULL), a contributor marked dirty; flag_w [n] (may be NULL) accumulates
 * each Gaussian's weight in those pixels. Returns the number of (pixel, Gaussian) pairs with nonzero weight, or -1 on
 * allocation failure. */
int64_t icgso_accumulate(int64_t n, const float* means, const float* scales, const float* quats,
                         const float* opac, const ocam_t* cam, int32_t K, const double* targets,
                         const uint8_t* mask, int32_t brute, double delta_a, double delta_t, double* V,
                         double* S, double* stake_own, double* stake_up, double* stake_tw,
                         uint8_t* pix_flag, double* flag_w, const uint8_t* dirty) {
  octx_t ctx;
  memset(&ctx, 0, sizeof ctx);
  ctx.K = K; ctx.targets = targets; ctx.V = V; ctx.S = S;
  ctx.stake.delta_a = delta_a; ctx.stake.delta_t = delta_t;
  ctx.stake.own = stake_own; ctx.stake.up = stake_up; ctx.stake.tw = stake_own ? stake_tw : NULL;
  ctx.pix_flag = pix_flag; ctx.flag_w = flag_w; ctx.dirty = dirty;
  if (run_camera(n, means, scales, quats, opac, cam, mask, brute, visit_accumulate, &ctx)) return -1;
  return ctx.pairs;
}

/* img_k = sum_i alpha_i T_i colors_ik (Eq. 1-2 with the per-Gaussian colour of this camera).
 * `image` is accumulated into. Returns the number of contributing pairs. */
int64_t icgso_render(int64_t n, const float* means, const float* scales, const float* quats,
                     const float* opac, const ocam_t* cam, int32_t K, const double* colors,
                     const uint8_t* mask, int32_t brute, double* image) {
  octx_t ctx;
  memset(&ctx, 0, sizeof ctx);
  ctx.K = K; ctx.colors = colors; ctx.image = image;
  if (run_camera(n, means, scales, quats, opac, cam, mask, brute, visit_render, &ctx)) return -1;
  return ctx.pairs;
}

/* Lists every (pixel, Gaussian, weight) with nonzero weight, and the transmittance in front of the
 * Gaussian (T may be NULL), up to `cap` entries; returns the total count (call again with a larger
 * cap if it exceeds cap). */
int64_t icgso_weights(int64_t n, const float* means, const float* scales, const float* quats,
                      const float* opac, const ocam_t* cam, const uint8_t* mask, int32_t brute,
                      int64_t cap, int32_t* pix, int32_t* gid, double* w, double* T) {
  octx_t ctx;
  memset(&ctx, 0, sizeof ctx);
  ctx.cap = cap; ctx.out_pix = pix; ctx.out_gid = gid; ctx.out_w = w; ctx.out_T = T;
  if (run_camera(n, means, scales, quats, opac, cam, mask, brute, visit_weights, &ctx)) return -1;
  return ctx.count;
}

/* Adjoint walk of one camera for given a = dL/dS [n,K] and beta = dL/dV [n]:
 * grad_t [H,W,K] += dL/dt and grad_o [n] += dL/dopacity (both accumulated into). */
int64_t icgso_adjoint(int64_t n, const float* means, const float* scales, const float* quats,
                      const float* opac, const ocam_t* cam, int32_t K, const double* targets,
                      const double* a, const double* beta, double* grad_t, double* grad_o) {
  octx_t ctx;
  memset(&ctx, 0, sizeof ctx);
  ctx.K = K; ctx.targets = targets; ctx.a = a; ctx.beta = beta; ctx.grad_t = grad_t; ctx.grad_o = grad_o;
  if (run_camera(n, means, scales, quats, opac, cam, NULL, 0, visit_adjoint, &ctx)) return -1;
  return ctx.pairs;
}

/* Test-only: scales the alpha threshold 1/255 and the stop threshold 1e-4 by the given factors
 * (1, 1 restores them). Not thread-safe: call it while no walk is running. */
void icgso_set_threshold_scale(double alpha_scale, double t_scale) {
  g_alpha_min_scale = alpha_scale;
  g_t_min_scale = t_scale;
}

/* Real orthonormal spherical harmonics (Eq. 3), degree 0..L, index l*l + l + m (m = -l..l):
 *   m > 0: sqrt(2) N_lm P_l^m(cos th) cos(m ph);  m < 0: sqrt(2) N_l|m| P_l^|m|(cos th) sin(|m| ph);
 *   m = 0: N_l0 P_l(cos th);  N_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!),
 * with the associated Legendre functions P_l^m taken WITHOUT the Condon-Shortley phase, so that
 * the degree-1 functions are +sqrt(3/(4 pi)) * (y, z, x). Directions need not be unit length. */
int icgso_sh_basis(int32_t L, int64_t m, const double* dirs, double* out) {
  if (L < 0 || L > 16) return -1;
  int B = (L + 1) * (L + 1);
  double P[17][17];
  for (int64_t s = 0; s < m; ++s) {
    double x = dirs[3 * s], y = dirs[3 * s + 1], z = dirs[3 * s + 2];
    double r = sqrt(x * x + y * y + z * z);
    double ct = z / r;
    double st = sqrt(x * x + y * y) / r;
    double ph = atan2(y, x);
    for (int mm = 0; mm <= L; ++mm) {
      /* P_m^m = (2m-1)!! st^m */
      double pmm = 1.0;
      for (int k = 1; k <= mm; ++k) pmm *= (2.0 * k - 1.0) * st;
      P[mm][mm] = pmm;
      if (mm + 1 <= L) P[mm + 1][mm] = ct * (2.0 * mm + 1.0) * pmm;
      for (int l = mm + 2; l <= L; ++l)
        P[l][mm] = ((2.0 * l - 1.0) * ct * P[l - 1][mm] - (l + mm - 1.0) * P[l - 2][mm]) / (l - mm);
    }
    double* o = out + (int64_t)s * B;
    for (int l = 0; l <= L; ++l)
      for (int mm = -l; mm <= l; ++mm) {
        int am = mm < 0 ? -mm : mm;
        double ratio = 1.0; /* (l-am)!/(l+am)! */
        for (int k = l - am + 1; k <= l + am; ++k) ratio /= (double)k;
        double N = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * ratio);
        double v;
        if (mm > 0) v = sqrt(2.0) * N * P[l][am] * cos(am * ph);
        else if (mm < 0) v = sqrt(2.0) * N * P[l][am] * sin(am * ph);
        else v = N * P[l][0];
        o[l * l + l + mm] = v;
      }
  }
  return 0;
}
