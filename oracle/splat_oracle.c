/*
 * FP64 CPU oracle of the MP-aware differentiable Gaussian splatting path.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link or call this
 * file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark use it. It shares no code with the CUDA kernels.
 *
 * What it computes, in plain double precision, one view at a time:
 *
 *   project   the 3D Gaussian of each record to a 2D conic (EWA splatting,
 *             the rasterisation the paper inherits from 3DGS, Sec. IV-D
 *             "during rasterization");
 *   render    for every pixel, front-to-back alpha compositing of colour,
 *             depth, opacity and motion probability over ALL Gaussians in
 *             (depth, id) order; the per-pixel static weight w(u) of Eq. (20)
 *             and the MP-weighted L1 photometric and depth losses of
 *             Eqs. (21), (22) with the lambda_1, lambda_2 of Sec. V-A(c);
 *   backward  the hand-derived adjoint of all of the above with respect to
 *             every Gaussian parameter and to the left-perturbation twist of
 *             the world-to-camera pose (joint optimisation of Gaussians and
 *             poses, Eq. (27));
 *   binning   the (tile, Gaussian) pair list sorted by (tile, depth, id).
 *
 * The paper does not print the rasteriser's equations or constants. The
 * readings used here are those of the published 3D Gaussian splatting
 * rasteriser, restated: alpha = min(0.99, o exp(-d^T Q d / 2)); a Gaussian
 * with alpha below 1/255 is skipped; compositing stops before the
 * contribution that would take the transmittance under 1e-4; 0.3 px^2 is
 * added to the 2D covariance's diagonal; means with camera z <= 0.2 m are
 * culled; the EWA Jacobian is evaluated with x/z and y/z clamped to 1.3
 * times the half field of view; a Gaussian is binned to the tiles its
 * alpha >= 1/255 ellipse reaches. The same constants are the defaults of the
 * C ABI's raster config.
 *
 * The depth order is decided on an FP32 depth key that both this oracle and
 * the CUDA path evaluate bit-identically (see depth_key). Other decisions
 * that floating point takes are flagged when the FP64 quantity lies within
 * the error an FP32 evaluation can have of its threshold: alpha skip, clamp
 * and the transmittance stop by a propagated bound (exponent_margin), tile
 * bounds, radius, residual signs and the near plane by a relative 1e-5. A
 * test can then tell an FP32-vs-FP64 rounding disagreement from a bug.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- layouts shared with the Python wrapper (oracle/__init__.py) ---- */

/* Gaussian parameters, FP64, one row of G_STRIDE per Gaussian. */
enum { G_MX = 0, G_MY, G_MZ, G_LOGIT, G_QW, G_QX, G_QY, G_QZ, G_S0, G_S1, G_S2,
       G_MP, G_CR, G_CG, G_CB, G_STRIDE };

/* Camera: fx, fy, cx, cy, width, height. Pose: 3x4 row-major [R | t], world->camera. */
enum { CAM_FX = 0, CAM_FY, CAM_CX, CAM_CY, CAM_W, CAM_H };

/* Raster constants. */
enum { RC_TILE = 0, RC_ALPHA_MIN, RC_ALPHA_MAX, RC_T_MIN, RC_DILATION, RC_Z_NEAR,
       RC_GUARD, RC_N };

/* Loss constants: lambda_pho, lambda_depth, weight_mode (0: normalised w =
 * (O - R_MP)/O, 1: unnormalised w = O - R_MP), weight_grad (0: w is a
 * constant in the adjoint), o_eps (normalised w is 0 where O <= o_eps). */
enum { LC_LPHO = 0, LC_LDEPTH, LC_WMODE, LC_WGRAD, LC_OEPS, LC_N };

/* Projection record per Gaussian. */
enum { PJ_VIS = 0, PJ_U, PJ_V, PJ_Z, PJ_A, PJ_B, PJ_C, PJ_O, PJ_SA, PJ_SB, PJ_SC,
       PJ_LMAX, PJ_R, PJ_X0, PJ_Y0, PJ_X1, PJ_Y1, PJ_FLAG, PJ_PX, PJ_PY, PJ_ZKEY, PJ_EX, PJ_EY,
       PJ_CTHR, PJ_STRIDE };

/* Per-pixel output: colour (3), depth, opacity, rendered MP, final
 * transmittance, number of contributors, id of the last contributor (-1),
 * static weight w(u) of Eq. (20) (0 without targets). */
enum { PX_CR = 0, PX_CG, PX_CB, PX_D, PX_O, PX_RMP, PX_T, PX_N, PX_LAST, PX_W, PX_STRIDE };

/* Gradient per Gaussian, same layout as G_*. */

/* Flag bits. */
#define FL_ZNEAR    1   /* depth within margin of the near plane           */
#define FL_CLAMP    2   /* x/z or y/z within margin of the frustum guard    */
#define FL_RADIUS   4   /* bounding radius within margin of an integer      */
#define FL_RECT     8   /* (u +- r)/tile within margin of an integer        */
#define FL_OPAC    16   /* opacity within margin of alpha_min               */
#define FL_ALPHA   32   /* pixel: some o*G within margin of alpha_min        */
#define FL_AMAX    64   /* pixel: some o*G within margin of alpha_max        */
#define FL_TSTOP  128   /* pixel: transmittance test within margin of t_min  */
#define FL_ZTIE   256   /* unused (depth order is decided on the FP32 key)   */
#define FL_OEPS   512   /* pixel: opacity within margin of o_eps             */
#define FL_SIGN  1024   /* pixel: a loss residual within margin of zero      */

#define MARGIN 1e-5

static int near_rel(double x, double thr) { return fabs(x - thr) <= MARGIN * fabs(thr); }

static int near_int(double x) {
  double f = x - floor(x + 0.5);
  return fabs(f) <= MARGIN * fmax(1.0, fabs(x));
}

/* Rotation matrix of the unit quaternion n = q/|q| (Hamilton convention,
 * scalar first), row-major. */
static void quat_rot(const double *q, double *R, double *nq, double *qn) {
  double len = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double w = q[0] / len, x = q[1] / len, y = q[2] / len, z = q[3] / len;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
  if (nq) { nq[0] = w; nq[1] = x; nq[2] = y; nq[3] = z; }
  if (qn) *qn = len;
}

/* C = A * B for 3x3 row-major. */
static void mm3(const double *A, const double *B, double *C) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      double s = 0;
      for (int k = 0; k < 3; k++) s += A[3 * i + k] * B[3 * k + j];
      C[3 * i + j] = s;
    }
}
static void tr3(const double *A, double *T) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) T[3 * j + i] = A[3 * i + j];
}

/* Everything projection computes for one Gaussian, kept for the adjoint. */
struct proj_s;
typedef struct proj_s {
  int vis, flags;
  double p[3];          /* camera-space mean                        */
  double tx, ty;        /* clamped x/z, y/z                          */
  int clx, cly;         /* 1 if the guard clamp was active           */
  double J[6];          /* 2x3 projection Jacobian                   */
  double Rq[9];         /* rotation of the Gaussian                  */
  double nq[4], qlen;   /* unit quaternion and |q|                   */
  double S[3];          /* exp(log-scale)                            */
  double Sig[9];        /* world covariance                          */
  double Sc[9];         /* camera covariance                         */
  double A, B, C;       /* 2D covariance after dilation              */
  double a, b, c;       /* conic = inverse 2D covariance             */
  double o, u, v, lmax, rext;
  double cthr;          /* 2 ln(o / alpha_min): alpha >= alpha_min iff q(d) <= cthr */
  double ex, ey;        /* half extents of the bounding box of that ellipse */
  double cond;          /* condition number of the dilated 2D covariance   */
  float zkey;           /* FP32 depth key that decides the depth order      */
  int r, x0, y0, x1, y1;
} proj_t;

/* Depth order key. The order of two Gaussians whose depths differ by less
 * than the rounding of a 32-bit float is not decided by the depth itself,
 * so the order is defined on this FP32 key (ties by id): the camera z of the
 * record's FP32 mean under the pose rounded to FP32, evaluated in FP32 in
 * exactly this order, without fused multiply-adds. The CUDA path evaluates
 * the same expression, so both sides take the decision identically. */
static float depth_key(const double *g, const double *pose) {
  float r20 = (float)pose[8], r21 = (float)pose[9], r22 = (float)pose[10], tz = (float)pose[11];
  float mx = (float)g[G_MX], my = (float)g[G_MY], mz = (float)g[G_MZ];
  volatile float a = r20 * mx;
  volatile float b = r21 * my;
  volatile float c = r22 * mz;
  volatile float ab = a + b;
  volatile float abc = ab + c;
  volatile float z = abc + tz;
  return z;
}

static int tile_reached(const proj_t *p, int tx, int ty, double tile, int W, int H, double *margin);

static void project_one(const double *g, const double *cam, const double *pose,
                        const double *rc, proj_t *P) {
  memset(P, 0, sizeof(*P));
  const double *Rw = pose; /* rows at 0,4,8; t at 3,7,11 */
  double R[9] = {pose[0], pose[1], pose[2], pose[4], pose[5], pose[6], pose[8], pose[9], pose[10]};
  double t[3] = {pose[3], pose[7], pose[11]};
  (void)Rw;
  for (int i = 0; i < 3; i++)
    P->p[i] = R[3 * i] * g[G_MX] + R[3 * i + 1] * g[G_MY] + R[3 * i + 2] * g[G_MZ] + t[i];
  P->zkey = depth_key(g, pose);
  double x = P->p[0], y = P->p[1], z = P->p[2];
  if (near_rel(z, rc[RC_Z_NEAR])) P->flags |= FL_ZNEAR;
  if (!(z > rc[RC_Z_NEAR])) return;

  double fx = cam[CAM_FX], fy = cam[CAM_FY];
  double limx = rc[RC_GUARD] * 0.5 * cam[CAM_W] / fx;
  double limy = rc[RC_GUARD] * 0.5 * cam[CAM_H] / fy;
  double txz = x / z, tyz = y / z;
  if (near_rel(fabs(txz), limx) || near_rel(fabs(tyz), limy)) P->flags |= FL_CLAMP;
  P->clx = (txz > limx || txz < -limx);
  P->cly = (tyz > limy || tyz < -limy);
  P->tx = txz > limx ? limx : (txz < -limx ? -limx : txz);
  P->ty = tyz > limy ? limy : (tyz < -limy ? -limy : tyz);
  double *J = P->J;
  J[0] = fx / z; J[1] = 0; J[2] = -fx * P->tx / z;
  J[3] = 0; J[4] = fy / z; J[5] = -fy * P->ty / z;

  quat_rot(g + G_QW, P->Rq, P->nq, &P->qlen);
  for (int i = 0; i < 3; i++) P->S[i] = exp(g[G_S0 + i]);
  double M[9], Mt[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) M[3 * i + j] = P->Rq[3 * i + j] * P->S[j];
  tr3(M, Mt);
  mm3(M, Mt, P->Sig);
  double Rt[9], tmp[9];
  tr3(R, Rt);
  mm3(R, P->Sig, tmp);
  mm3(tmp, Rt, P->Sc);
  /* Sigma' = J Sc J^T (2x2) */
  double JS[6];
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 3; j++) {
      double s = 0;
      for (int k = 0; k < 3; k++) s += J[3 * i + k] * P->Sc[3 * k + j];
      JS[3 * i + j] = s;
    }
  double S2[4];
  for (int i = 0; i < 2; i++)
    for (int j = 0; j < 2; j++) {
      double s = 0;
      for (int k = 0; k < 3; k++) s += JS[3 * i + k] * J[3 * j + k];
      S2[2 * i + j] = s;
    }
  P->A = S2[0] + rc[RC_DILATION];
  P->B = S2[1];
  P->C = S2[3] + rc[RC_DILATION];
  double det = P->A * P->C - P->B * P->B;
  if (!(det > 0)) return;
  P->a = P->C / det;
  P->b = -P->B / det;
  P->c = P->A / det;
  {
    double m2 = 0.5 * (P->A + P->C), hd = sqrt(0.25 * (P->A - P->C) * (P->A - P->C) + P->B * P->B);
    P->cond = (m2 + hd) / fmax(m2 - hd, 1e-300);
  }

  P->o = 1.0 / (1.0 + exp(-g[G_LOGIT]));
  if (near_rel(P->o, rc[RC_ALPHA_MIN])) P->flags |= FL_OPAC;
  if (!(P->o > rc[RC_ALPHA_MIN])) return;

  P->u = fx * x / z + cam[CAM_CX];
  P->v = fy * y / z + cam[CAM_CY];
  double mid = 0.5 * (P->A + P->C);
  double disc = mid * mid - det;
  P->lmax = mid + sqrt(disc > 0.1 ? disc : 0.1);
  /* Outside |d| <= sqrt(2 lmax ln(o/alpha_min)) the Gaussian's alpha is below
   * alpha_min, so it cannot contribute there. */
  P->cthr = 2.0 * log(P->o / rc[RC_ALPHA_MIN]);
  P->rext = sqrt(P->lmax * P->cthr);
  P->r = (int)ceil(P->rext);
  /* Bounding box of the ellipse q(d) = d^T Q d <= cthr outside of which the
   * Gaussian's alpha is below alpha_min: half extents sqrt(cthr Sigma'_xx),
   * sqrt(cthr Sigma'_yy). Its tile range is the candidate range; binning
   * keeps the candidate tiles the ellipse actually reaches (tile_reached). */
  P->ex = sqrt(P->cthr * P->A);
  P->ey = sqrt(P->cthr * P->C);
  double tile = rc[RC_TILE];
  int tx = (int)ceil(cam[CAM_W] / tile), ty = (int)ceil(cam[CAM_H] / tile);
  double ex[4] = {(P->u - P->ex) / tile, (P->v - P->ey) / tile, (P->u + P->ex) / tile,
                  (P->v + P->ey) / tile};
  for (int i = 0; i < 4; i++)
    if (near_int(ex[i])) P->flags |= FL_RECT;
  int x0 = (int)floor(ex[0]), y0 = (int)floor(ex[1]);
  int x1 = (int)floor(ex[2]) + 1, y1 = (int)floor(ex[3]) + 1;
  P->x0 = x0 < 0 ? 0 : (x0 > tx ? tx : x0);
  P->y0 = y0 < 0 ? 0 : (y0 > ty ? ty : y0);
  P->x1 = x1 < 0 ? 0 : (x1 > tx ? tx : x1);
  P->y1 = y1 < 0 ? 0 : (y1 > ty ? ty : y1);
  if ((P->x1 - P->x0) * (P->y1 - P->y0) <= 0) return;
  P->vis = 1;
}

/* Flags FL_RECT on a visible Gaussian if any of its candidate-tile decisions
 * lies within FP32 rounding of the threshold. */
static void flag_tile_decisions(proj_t *P, const double *cam, const double *rc) {
  if (!P->vis) return;
  for (int y = P->y0; y < P->y1; y++)
    for (int x = P->x0; x < P->x1; x++) {
      double m;
      tile_reached(P, x, y, rc[RC_TILE], (int)cam[CAM_W], (int)cam[CAM_H], &m);
      if (m < 1.0) P->flags |= FL_RECT;
    }
}

/* Projection of all Gaussians into out[n * PJ_STRIDE]. */
void oracle_project(int64_t n, const double *G, const double *cam, const double *pose,
                    const double *rc, double *out) {
  for (int64_t i = 0; i < n; i++) {
    proj_t P;
    project_one(G + i * G_STRIDE, cam, pose, rc, &P);
    flag_tile_decisions(&P, cam, rc);
    double *o = out + i * PJ_STRIDE;
    o[PJ_VIS] = P.vis; o[PJ_U] = P.u; o[PJ_V] = P.v; o[PJ_Z] = P.p[2];
    o[PJ_A] = P.a; o[PJ_B] = P.b; o[PJ_C] = P.c; o[PJ_O] = P.o;
    o[PJ_SA] = P.A; o[PJ_SB] = P.B; o[PJ_SC] = P.C; o[PJ_LMAX] = P.lmax;
    o[PJ_R] = P.r; o[PJ_X0] = P.x0; o[PJ_Y0] = P.y0; o[PJ_X1] = P.x1; o[PJ_Y1] = P.y1;
    o[PJ_FLAG] = P.flags; o[PJ_PX] = P.p[0]; o[PJ_PY] = P.p[1]; o[PJ_ZKEY] = (double)P.zkey;
    o[PJ_EX] = P.ex; o[PJ_EY] = P.ey; o[PJ_CTHR] = P.cthr;
  }
}

/* Bound on the error of an FP32 evaluation of the exponent ln(o G) at pixel
 * offset (dx, dy): the projected centre carries a few ulps of its own
 * magnitude (2^-22 |u|), the conic a relative error growing with the 2D
 * covariance's condition number. Decisions of alpha against a threshold
 * closer than this are flagged. */
static double exponent_margin(const proj_t *p, double dx, double dy, double power) {
  double gx = fabs(p->a * dx + p->b * dy), gy = fabs(p->b * dx + p->c * dy);
  double ecoord = ldexp(1.0, -22) * fmax(fmax(fabs(p->u), fabs(p->v)), 1.0);
  return (gx + gy) * ecoord + fabs(power) * (1e-6 + 4e-7 * p->cond) + 2e-6;
}

/* ---- depth order: (FP32 depth key, id) ---- */

typedef struct { float z; int64_t id; } zkey_t;

static int cmp_zkey(const void *pa, const void *pb) {
  const zkey_t *a = (const zkey_t *)pa, *b = (const zkey_t *)pb;
  if (a->z < b->z) return -1;
  if (a->z > b->z) return 1;
  return (a->id > b->id) - (a->id < b->id);
}

/* ---- binning ---- */

/* Does the ellipse q(d) <= cthr reach the pixel-centre rectangle of tile
 * (tx, ty) (pixels 16 tx .. 16 tx + 15 clipped to the image)? The minimum of
 * the positive-definite q over the rectangle is 0 if the centre is inside,
 * else it lies on one of the four edges, where q is a 1-D quadratic whose
 * minimiser is clamped to the edge. *margin receives the distance of that
 * minimum to cthr relative to the FP32 error bound of its evaluation (< 1:
 * the decision is within FP32 rounding). */
static int tile_reached(const proj_t *p, int tx, int ty, double tile, int W, int H, double *margin) {
  double xl = tx * tile - p->u, xh = fmin(tx * tile + tile - 1, W - 1) - p->u;
  double yl = ty * tile - p->v, yh = fmin(ty * tile + tile - 1, H - 1) - p->v;
  double qmin;
  if (xl <= 0 && xh >= 0 && yl <= 0 && yh >= 0) {
    qmin = 0.0;
  } else {
    double a = p->a, b = p->b, c = p->c;
    double best = INFINITY;
    double X[2] = {xl, xh}, Y[2] = {yl, yh};
    for (int k = 0; k < 2; k++) {
      double x = X[k];
      double y = -b * x / c;
      y = y < yl ? yl : (y > yh ? yh : y);
      double q = a * x * x + 2 * b * x * y + c * y * y;
      if (q < best) best = q;
      double yy = Y[k];
      double xx = -b * yy / a;
      xx = xx < xl ? xl : (xx > xh ? xh : xx);
      q = a * xx * xx + 2 * b * xx * yy + c * yy * yy;
      if (q < best) best = q;
    }
    qmin = best;
  }
  double ecoord = ldexp(1.0, -22) * fmax(fmax(fabs(p->u), fabs(p->v)), 1.0);
  double err = 2.0 * sqrt(fmax(qmin, 0.0) * fmax(p->a, p->c)) * ecoord * 2.0 + 1e-5 * p->cthr * (1.0 + p->cond * 0.1) + 1e-6;
  if (margin) *margin = fabs(qmin - p->cthr) / err;
  return qmin <= p->cthr;
}

/* Pairs (tile, id) of every visible Gaussian and every tile of its rect,
 * sorted by (tile, depth key, id). Writes up to cap pairs, returns the total.
 * tie_flag[k] = 1 where pair k and pair k-1 share a tile and an equal depth
 * key (their order is then decided by the id). */
typedef struct { int64_t tile; float z; int64_t id; } bkey_t;

static int cmp_bkey(const void *pa, const void *pb) {
  const bkey_t *a = (const bkey_t *)pa, *b = (const bkey_t *)pb;
  if (a->tile != b->tile) return (a->tile > b->tile) - (a->tile < b->tile);
  if (a->z < b->z) return -1;
  if (a->z > b->z) return 1;
  return (a->id > b->id) - (a->id < b->id);
}

int64_t oracle_binning(int64_t n, const double *G, const double *cam, const double *pose,
                       const double *rc, int64_t cap, int64_t *tiles, int64_t *ids,
                       int32_t *tie_flag) {
  int tx = (int)ceil(cam[CAM_W] / rc[RC_TILE]);
  proj_t *P = (proj_t *)malloc(sizeof(proj_t) * (size_t)(n > 0 ? n : 1));
  int64_t total = 0;
  const int W = (int)cam[CAM_W], H = (int)cam[CAM_H];
  for (int64_t i = 0; i < n; i++) {
    project_one(G + i * G_STRIDE, cam, pose, rc, &P[i]);
    if (P[i].vis) total += (int64_t)(P[i].x1 - P[i].x0) * (P[i].y1 - P[i].y0);
  }
  bkey_t *keys = (bkey_t *)malloc(sizeof(bkey_t) * (size_t)(total > 0 ? total : 1));
  int64_t k = 0;
  for (int64_t i = 0; i < n; i++) {
    if (!P[i].vis) continue;
    for (int y = P[i].y0; y < P[i].y1; y++)
      for (int x = P[i].x0; x < P[i].x1; x++) {
        double m;
        if (!tile_reached(&P[i], x, y, rc[RC_TILE], W, H, &m)) continue;
        keys[k].tile = (int64_t)y * tx + x;
        keys[k].z = P[i].zkey;
        keys[k].id = i;
        k++;
      }
  }
  total = k;
  qsort(keys, (size_t)total, sizeof(bkey_t), cmp_bkey);
  for (int64_t j = 0; j < total && j < cap; j++) {
    tiles[j] = keys[j].tile;
    ids[j] = keys[j].id;
    tie_flag[j] = (j > 0 && keys[j].tile == keys[j - 1].tile && keys[j].z == keys[j - 1].z);
  }
  free(keys);
  free(P);
  return total;
}

/* ---- render, loss and adjoint ---- */

typedef struct { int64_t id; double alpha, T, G, dx, dy; int clamped; } contrib_t;

/* Candidate lists: a pixel's candidates are the visible Gaussians whose
 * bounding square |dx|, |dy| <= r (r >= sqrt(lambda_max cthr)) holds the
 * pixel, in (depth, id) order. Outside that square alpha < alpha_min
 * exactly, so restricting to it does not change any value; with accel = 0
 * every visible Gaussian is tested. */
typedef struct { int64_t *start; int64_t *ids; int cw, ch, cell; } cells_t;

static void build_cells(int64_t n, const proj_t *P, const int64_t *order, int W, int H,
                        int cell, int accel, cells_t *cs) {
  cs->cell = accel ? cell : (W > H ? W : H);
  cs->cw = (W + cs->cell - 1) / cs->cell;
  cs->ch = (H + cs->cell - 1) / cs->cell;
  int nc = cs->cw * cs->ch;
  cs->start = (int64_t *)calloc((size_t)nc + 1, sizeof(int64_t));
  for (int pass = 0; pass < 2; pass++) {
    int64_t *fill = NULL;
    if (pass == 1) {
      for (int c = 0; c < nc; c++) cs->start[c + 1] += cs->start[c];
      cs->ids = (int64_t *)malloc(sizeof(int64_t) * (size_t)(cs->start[nc] > 0 ? cs->start[nc] : 1));
      fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nc);
      for (int c = 0; c < nc; c++) fill[c] = cs->start[c];
    }
    for (int64_t oi = 0; oi < n; oi++) {
      int64_t i = order[oi];
      const proj_t *p = &P[i];
      if (!p->vis) continue;
      int px0 = 0, py0 = 0, px1 = W - 1, py1 = H - 1;
      if (accel) {
        px0 = (int)ceil(p->u - p->r); px1 = (int)floor(p->u + p->r);
        py0 = (int)ceil(p->v - p->r); py1 = (int)floor(p->v + p->r);
        if (px0 < 0) px0 = 0;
        if (py0 < 0) py0 = 0;
        if (px1 > W - 1) px1 = W - 1;
        if (py1 > H - 1) py1 = H - 1;
        if (px0 > px1 || py0 > py1) continue;
      }
      for (int cy = py0 / cs->cell; cy <= py1 / cs->cell; cy++)
        for (int cx = px0 / cs->cell; cx <= px1 / cs->cell; cx++) {
          int c = cy * cs->cw + cx;
          if (pass == 0) cs->start[c + 1]++;
          else cs->ids[fill[c]++] = i;
        }
    }
    free(fill);
  }
}

/* The adjoint of one pixel's front-to-back compositing, back to front:
 * given the upstream gradients gF of its six composited channels and its
 * contributor list, ADDS each contributor's gradients of (u, v, a, b, c, o,
 * z, colour) to g2 (10 per Gaussian). With S the channels' sums over the
 * contributors behind k, d/d alpha_k = sum_ch gF_ch (f_ch T_k - S_ch /
 * (1 - alpha_k)); a clamped alpha passes nothing to its exponent. */
static void adjoint_pixel(const contrib_t *list, int64_t nl, const proj_t *P, const double *G,
                          const double *gF, double *g2, double *g2abs) {
  double S[6] = {0, 0, 0, 0, 0, 0}; /* sum over later contributors */
  for (int64_t k = nl - 1; k >= 0; k--) {
    const contrib_t *e = &list[k];
    const proj_t *p = &P[e->id];
    const double *g = G + e->id * G_STRIDE;
    double f[6] = {g[G_CR], g[G_CG], g[G_CB], p->p[2], 1.0, g[G_MP]};
    double wk = e->alpha * e->T;
    double dal = 0;
    for (int ch = 0; ch < 6; ch++)
      dal += gF[ch] * (f[ch] * e->T - S[ch] / (1.0 - e->alpha));
    double *gg = g2 + e->id * 10;
    double t[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    t[7] = gF[0] * wk;
    t[8] = gF[1] * wk;
    t[9] = gF[2] * wk;
    t[6] = gF[3] * wk;
    if (!e->clamped) {
      t[5] = dal * e->G;
      double dpw = dal * e->alpha;
      t[0] = dpw * (-(p->a * e->dx + p->b * e->dy));
      t[1] = dpw * (-(p->b * e->dx + p->c * e->dy));
      t[2] = dpw * (-0.5 * e->dx * e->dx);
      t[3] = dpw * (-e->dx * e->dy);
      t[4] = dpw * (-0.5 * e->dy * e->dy);
    }
    for (int k = 0; k < 10; k++) gg[k] += t[k];
    if (g2abs)
      for (int k = 0; k < 10; k++) g2abs[e->id * 10 + k] += fabs(t[k]);
    for (int ch = 0; ch < 6; ch++) S[ch] += f[ch] * wk;
  }
}

/* The chain of one Gaussian's 2D gradients gg[10] (u, v, a, b, c, o, z,
 * colour) to its parameters (ADDED to out[G_STRIDE], if non-NULL) and to the
 * pose twist (ADDED to pg[6]): conic to 2D covariance, EWA covariance and
 * Jacobian to the camera-space mean and covariance, camera transform, scale
 * and rotation (through the quaternion's normalisation). Linear in gg. */
static void chain_gauss(const proj_t *p, const double *R, double fx, double fy, const double *gg, double *out,
                        double *pg) {
  double x = p->p[0], y = p->p[1], z = p->p[2];
  /* conic -> 2D covariance: dL/dSigma' = -Q Gq Q (symmetric matrix form) */
  double Q[4] = {p->a, p->b, p->b, p->c};
  double Gq[4] = {gg[2], 0.5 * gg[3], 0.5 * gg[3], gg[4]};
  double QG[4], dS2[4];
  for (int r = 0; r < 2; r++)
    for (int s = 0; s < 2; s++)
      QG[2 * r + s] = Q[2 * r] * Gq[s] + Q[2 * r + 1] * Gq[2 + s];
  for (int r = 0; r < 2; r++)
    for (int s = 0; s < 2; s++)
      dS2[2 * r + s] = -(QG[2 * r] * Q[s] + QG[2 * r + 1] * Q[2 + s]);
  const double *J = p->J;
  /* dL/dSc = J^T dS2 J */
  double dSc[9];
  for (int r = 0; r < 3; r++)
    for (int s = 0; s < 3; s++) {
      double acc2 = 0;
      for (int k = 0; k < 2; k++)
        for (int l = 0; l < 2; l++) acc2 += J[3 * k + r] * dS2[2 * k + l] * J[3 * l + s];
      dSc[3 * r + s] = acc2;
    }
  /* dL/dJ = 2 dS2 J Sc */
  double JSc[6], dJ[6];
  for (int r = 0; r < 2; r++)
    for (int s = 0; s < 3; s++) {
      double acc2 = 0;
      for (int k = 0; k < 3; k++) acc2 += J[3 * r + k] * p->Sc[3 * k + s];
      JSc[3 * r + s] = acc2;
    }
  for (int r = 0; r < 2; r++)
    for (int s = 0; s < 3; s++) dJ[3 * r + s] = 2.0 * (dS2[2 * r] * JSc[s] + dS2[2 * r + 1] * JSc[3 + s]);
  /* dL/dp (camera-space mean) */
  double dp[3] = {0, 0, 0};
  dp[0] += gg[0] * fx / z;
  dp[2] += gg[0] * (-fx * x / (z * z));
  dp[1] += gg[1] * fy / z;
  dp[2] += gg[1] * (-fy * y / (z * z));
  dp[2] += gg[6];
  dp[2] += dJ[0] * (-fx / (z * z));
  dp[2] += dJ[4] * (-fy / (z * z));
  if (!p->clx) {
    dp[0] += dJ[2] * (-fx / (z * z));
    dp[2] += dJ[2] * (2.0 * fx * x / (z * z * z));
  } else {
    dp[2] += dJ[2] * (fx * p->tx / (z * z));
  }
  if (!p->cly) {
    dp[1] += dJ[5] * (-fy / (z * z));
    dp[2] += dJ[5] * (2.0 * fy * y / (z * z * z));
  } else {
    dp[2] += dJ[5] * (fy * p->ty / (z * z));
  }
  /* pose: rho += dp; phi += p x dp + covariance term */
  pg[0] += dp[0]; pg[1] += dp[1]; pg[2] += dp[2];
  pg[3] += y * dp[2] - z * dp[1];
  pg[4] += z * dp[0] - x * dp[2];
  pg[5] += x * dp[1] - y * dp[0];
  double Am[9];
  mm3(p->Sc, dSc, Am);
  pg[3] += 2.0 * (Am[5] - Am[7]);
  pg[4] += 2.0 * (Am[6] - Am[2]);
  pg[5] += 2.0 * (Am[1] - Am[3]);

  if (!out) return;
  /* mean: p = R mu + t */
  for (int k = 0; k < 3; k++)
    out[G_MX + k] += R[k] * dp[0] + R[3 + k] * dp[1] + R[6 + k] * dp[2];
  /* world covariance: dSig = R^T dSc R */
  double Rt[9], tmp[9], dSig[9];
  tr3(R, Rt);
  mm3(Rt, dSc, tmp);
  mm3(tmp, R, dSig);
  /* Sig = M M^T, M = Rq diag(S): dM = 2 dSig M */
  double M[9], dM[9];
  for (int r = 0; r < 3; r++)
    for (int s = 0; s < 3; s++) M[3 * r + s] = p->Rq[3 * r + s] * p->S[s];
  mm3(dSig, M, dM);
  for (int k = 0; k < 9; k++) dM[k] *= 2.0;
  double dRq[9];
  for (int s = 0; s < 3; s++) {
    double dSs = 0;
    for (int r = 0; r < 3; r++) {
      dSs += p->Rq[3 * r + s] * dM[3 * r + s];
      dRq[3 * r + s] = dM[3 * r + s] * p->S[s];
    }
    out[G_S0 + s] += dSs * p->S[s];
  }
  double w = p->nq[0], qx = p->nq[1], qy = p->nq[2], qz = p->nq[3];
  double dn[4];
  dn[0] = dRq[1] * (-2 * qz) + dRq[2] * (2 * qy) + dRq[3] * (2 * qz) + dRq[5] * (-2 * qx) +
          dRq[6] * (-2 * qy) + dRq[7] * (2 * qx);
  dn[1] = dRq[1] * (2 * qy) + dRq[2] * (2 * qz) + dRq[3] * (2 * qy) + dRq[4] * (-4 * qx) +
          dRq[5] * (-2 * w) + dRq[6] * (2 * qz) + dRq[7] * (2 * w) + dRq[8] * (-4 * qx);
  dn[2] = dRq[0] * (-4 * qy) + dRq[1] * (2 * qx) + dRq[2] * (2 * w) + dRq[3] * (2 * qx) +
          dRq[5] * (2 * qz) + dRq[6] * (-2 * w) + dRq[7] * (2 * qz) + dRq[8] * (-4 * qy);
  dn[3] = dRq[0] * (-4 * qz) + dRq[1] * (-2 * w) + dRq[2] * (2 * qx) + dRq[3] * (2 * w) +
          dRq[4] * (-4 * qz) + dRq[5] * (2 * qy) + dRq[6] * (2 * qx) + dRq[7] * (2 * qy);
  double ndn = w * dn[0] + qx * dn[1] + qy * dn[2] + qz * dn[3];
  out[G_QW] += (dn[0] - w * ndn) / p->qlen;
  out[G_QX] += (dn[1] - qx * ndn) / p->qlen;
  out[G_QY] += (dn[2] - qy * ndn) / p->qlen;
  out[G_QZ] += (dn[3] - qz * ndn) / p->qlen;
  out[G_LOGIT] += gg[5] * p->o * (1.0 - p->o);
  out[G_CR] += gg[7];
  out[G_CG] += gg[8];
  out[G_CB] += gg[9];
}

/* Render one view: out_px[P * PX_STRIDE], out_flags[P]; if targets
 * (P x 4: r, g, b, depth) is given, the loss goes to *loss and, if grads /
 * pose_grad are non-NULL, the adjoint is ADDED to grads[n * G_STRIDE] and
 * written to pose_grad[6] = (rho, phi) of the left-perturbation twist.
 * wfix (P, or NULL) replaces the static weight w(u) by given constants, so
 * that finite differences can check the stop-gradient adjoint.
 * grad_mag (n * G_STRIDE, or NULL; with grads) receives, per parameter, the
 * sum over pixels and 2D words of |term| |d parameter / d word|: the size of
 * the terms the gradient sums, which bounds its rounding error in any
 * arithmetic that rounds each term relatively (added, like grads).
 * upstream (P x 6, or NULL) replaces the loss: the adjoint is that of
 * sum_u upstream[u] . (C_r, C_g, C_b, D, O, R_MP)(u), a caller's gradient of
 * its own function of the composited channels (targets are then unused).
 * Returns 0, or -1 on allocation failure. */
int oracle_render(int64_t n, const double *G, const double *cam, const double *pose,
                  const double *rc, const double *lc, const double *targets, const double *wfix,
                  const double *upstream, int accel, double *out_px, int32_t *out_flags, double *loss,
                  double *grads, double *pose_grad, double *grad_mag) {
  int W = (int)cam[CAM_W], H = (int)cam[CAM_H];
  proj_t *P = (proj_t *)malloc(sizeof(proj_t) * (size_t)(n > 0 ? n : 1));
  zkey_t *zk = (zkey_t *)malloc(sizeof(zkey_t) * (size_t)(n > 0 ? n : 1));
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!P || !zk || !order) return -1;
  int64_t nv = 0;
  for (int64_t i = 0; i < n; i++) {
    project_one(G + i * G_STRIDE, cam, pose, rc, &P[i]);
    if (P[i].vis) { zk[nv].z = P[i].zkey; zk[nv].id = i; nv++; }
  }
  qsort(zk, (size_t)nv, sizeof(zkey_t), cmp_zkey);
  for (int64_t k = 0; k < nv; k++) order[k] = zk[k].id;
  cells_t cs;
  build_cells(nv, P, order, W, H, 8, accel, &cs);

  if (upstream) targets = NULL;
  const int want_grad = (targets != NULL || upstream != NULL) && (grads != NULL || pose_grad != NULL);
  /* per-Gaussian accumulated 2D gradients: u, v, a, b, c, o, z, cr, cg, cb */
  double *g2 = want_grad ? (double *)calloc((size_t)(n > 0 ? n : 1) * 10, sizeof(double)) : NULL;
  /* with grad_mag: the per-Gaussian sums of the 2D terms' magnitudes */
  if (!want_grad) grad_mag = NULL;
  double *g2abs = grad_mag ? (double *)calloc((size_t)(n > 0 ? n : 1) * 10, sizeof(double)) : NULL;
  int64_t cap = 256;
  contrib_t *list = (contrib_t *)malloc(sizeof(contrib_t) * (size_t)cap);
  double L = 0.0;
  const double amin = rc[RC_ALPHA_MIN], amax = rc[RC_ALPHA_MAX], tmin = rc[RC_T_MIN];

  for (int j = 0; j < H; j++)
    for (int i = 0; i < W; i++) {
      int c = (j / cs.cell) * cs.cw + (i / cs.cell);
      double T = 1.0, acc[6] = {0, 0, 0, 0, 0, 0};
      double eT = 0.0; /* bound on the relative FP32 error of T */
      int flags = 0;
      int64_t nl = 0, last = -1;
      for (int64_t q = cs.start[c]; q < cs.start[c + 1]; q++) {
        int64_t id = cs.ids[q];
        const proj_t *p = &P[id];
        double dx = p->u - i, dy = p->v - j;
        double power = -0.5 * (p->a * dx * dx + p->c * dy * dy) - p->b * dx * dy;
        double Gv = exp(power);
        double ag = p->o * Gv;
        double em = exponent_margin(p, dx, dy, power);
        double lag = power + log(p->o);
        if (fabs(lag - log(amin)) <= em) flags |= FL_ALPHA;
        if (fabs(lag - log(amax)) <= em) flags |= FL_AMAX;
        if (ag < amin) continue;
        int clamped = ag > amax;
        double alpha = clamped ? amax : ag;
        double testT = T * (1.0 - alpha);
        double eTk = eT + (clamped ? 0.0 : alpha / (1.0 - alpha) * em) + 1e-6;
        if (fabs(log(testT) - log(tmin)) <= eTk) flags |= FL_TSTOP;
        if (testT < tmin) break;
        eT = eTk;
        const double *g = G + id * G_STRIDE;
        double wgt = alpha * T;
        acc[0] += g[G_CR] * wgt;
        acc[1] += g[G_CG] * wgt;
        acc[2] += g[G_CB] * wgt;
        acc[3] += p->p[2] * wgt;
        acc[4] += wgt;
        acc[5] += g[G_MP] * wgt;
        if (nl == cap) {
          cap *= 2;
          list = (contrib_t *)realloc(list, sizeof(contrib_t) * (size_t)cap);
        }
        list[nl].id = id; list[nl].alpha = alpha; list[nl].T = T; list[nl].G = Gv;
        list[nl].dx = dx; list[nl].dy = dy; list[nl].clamped = clamped;
        nl++;
        last = id;
        T = testT;
      }
      int64_t pix = (int64_t)j * W + i;
      double *o = out_px + pix * PX_STRIDE;
      for (int k = 0; k < 6; k++) o[k] = acc[k];
      o[PX_T] = T; o[PX_N] = (double)nl; o[PX_LAST] = (double)last; o[PX_W] = 0.0;

      if (upstream && want_grad && nl > 0) {
        /* the caller's upstream gradients of the six composited channels */
        double gF[6];
        for (int k = 0; k < 6; k++) gF[k] = upstream[pix * 6 + k];
        adjoint_pixel(list, nl, P, G, gF, g2, g2abs);
      }
      if (targets) {
        const double *tg = targets + pix * 4;
        double O = acc[4], Rm = acc[5];
        double w = 0.0;
        if (lc[LC_WMODE] == 0) {
          if (near_rel(O, lc[LC_OEPS])) flags |= FL_OEPS;
          if (O > lc[LC_OEPS]) w = (O - Rm) / O;
        } else {
          w = O - Rm;
        }
        if (wfix) w = wfix[pix];
        o[PX_W] = w;
        double rcol[3], sc[3], rd = acc[3] - tg[3], sd;
        double l1 = 0;
        for (int k = 0; k < 3; k++) {
          rcol[k] = acc[k] - tg[k];
          if (fabs(rcol[k]) <= MARGIN * fmax(fabs(acc[k]), fabs(tg[k]))) flags |= FL_SIGN;
          sc[k] = (rcol[k] > 0) - (rcol[k] < 0);
          l1 += fabs(rcol[k]);
        }
        int dvalid = tg[3] > 0;
        if (dvalid && fabs(rd) <= MARGIN * fmax(fabs(acc[3]), fabs(tg[3]))) flags |= FL_SIGN;
        sd = dvalid ? (double)((rd > 0) - (rd < 0)) : 0.0;
        double lw = lc[LC_LPHO] * l1 + (dvalid ? lc[LC_LDEPTH] * fabs(rd) : 0.0);
        /* a target with negative red marks a pixel without valid colour: it is
         * left out of both loss terms, as a pixel without valid depth is left
         * out of the depth term */
        const int pvalid = tg[0] >= 0;
        if (!pvalid) lw = 0.0;
        L += w * lw;

        if (want_grad && nl > 0 && pvalid) {
          /* upstream gradients of the six composited channels */
          double gF[6];
          for (int k = 0; k < 3; k++) gF[k] = lc[LC_LPHO] * w * sc[k];
          gF[3] = lc[LC_LDEPTH] * w * sd;
          gF[4] = 0.0;
          gF[5] = 0.0;
          if (lc[LC_WGRAD] != 0 && !wfix) {
            if (lc[LC_WMODE] == 0) {
              if (O > lc[LC_OEPS]) { gF[4] += lw * Rm / (O * O); gF[5] += -lw / O; }
            } else {
              gF[4] += lw; gF[5] += -lw;
            }
          }
          adjoint_pixel(list, nl, P, G, gF, g2, g2abs);
        }
      }
      out_flags[pix] = flags;
    }
  if (loss) *loss = L;

  if (want_grad) {
    double R[9] = {pose[0], pose[1], pose[2], pose[4], pose[5], pose[6], pose[8], pose[9], pose[10]};
    double pg[6] = {0, 0, 0, 0, 0, 0};
    double fx = cam[CAM_FX], fy = cam[CAM_FY];
    for (int64_t id = 0; id < n; id++) {
      const proj_t *p = &P[id];
      if (!p->vis) continue;
      chain_gauss(p, R, fx, fy, g2 + id * 10, grads ? grads + id * G_STRIDE : NULL, pg);
      if (grad_mag) {
        /* |J| times the sum of the pixel terms' magnitudes: the chain of
         * each unit 2D word, taken in absolute value */
        double *mag = grad_mag + id * G_STRIDE;
        for (int k = 0; k < 10; k++) {
          const double a = g2abs[id * 10 + k];
          if (a == 0.0) continue;
          double e[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0}, col[G_STRIDE], pcol[6] = {0, 0, 0, 0, 0, 0};
          for (int c = 0; c < G_STRIDE; c++) col[c] = 0.0;
          e[k] = 1.0;
          chain_gauss(p, R, fx, fy, e, col, pcol);
          for (int c = 0; c < G_STRIDE; c++) mag[c] += fabs(col[c]) * a;
        }
      }
    }
    if (pose_grad)
      for (int k = 0; k < 6; k++) pose_grad[k] = pg[k];
  }
  free(list);
  free(g2);
  free(g2abs);
  free(cs.start);
  free(cs.ids);
  free(order);
  free(zk);
  free(P);
  return 0;
}

/* Render one pixel (i, j) by testing every Gaussian: the per-pixel form of
 * oracle_render for spot checks at sizes where a whole image is too slow.
 * out[PX_STRIDE]; returns the flags. */
int oracle_render_pixel(int64_t n, const double *G, const double *cam, const double *pose,
                        const double *rc, int i, int j, double *out) {
  zkey_t *zk = (zkey_t *)malloc(sizeof(zkey_t) * (size_t)(n > 0 ? n : 1));
  proj_t *P = (proj_t *)malloc(sizeof(proj_t) * (size_t)(n > 0 ? n : 1));
  int64_t nv = 0;
  for (int64_t k = 0; k < n; k++) {
    project_one(G + k * G_STRIDE, cam, pose, rc, &P[k]);
    if (P[k].vis) { zk[nv].z = P[k].zkey; zk[nv].id = k; nv++; }
  }
  qsort(zk, (size_t)nv, sizeof(zkey_t), cmp_zkey);
  double T = 1.0, acc[6] = {0, 0, 0, 0, 0, 0}, eT = 0.0;
  int flags = 0, nl = 0;
  int64_t last = -1;
  for (int64_t q = 0; q < nv; q++) {
    const proj_t *p = &P[zk[q].id];
    const double *g = G + zk[q].id * G_STRIDE;
    double dx = p->u - i, dy = p->v - j;
    double power = -0.5 * (p->a * dx * dx + p->c * dy * dy) - p->b * dx * dy;
    double ag = p->o * exp(power);
    double em = exponent_margin(p, dx, dy, power);
    double lag = power + log(p->o);
    if (fabs(lag - log(rc[RC_ALPHA_MIN])) <= em) flags |= FL_ALPHA;
    if (fabs(lag - log(rc[RC_ALPHA_MAX])) <= em) flags |= FL_AMAX;
    if (ag < rc[RC_ALPHA_MIN]) continue;
    int clamped = ag > rc[RC_ALPHA_MAX];
    double alpha = clamped ? rc[RC_ALPHA_MAX] : ag;
    double testT = T * (1.0 - alpha);
    double eTk = eT + (clamped ? 0.0 : alpha / (1.0 - alpha) * em) + 1e-6;
    if (fabs(log(testT) - log(rc[RC_T_MIN])) <= eTk) flags |= FL_TSTOP;
    if (testT < rc[RC_T_MIN]) break;
    eT = eTk;
    double wgt = alpha * T;
    acc[0] += g[G_CR] * wgt; acc[1] += g[G_CG] * wgt; acc[2] += g[G_CB] * wgt;
    acc[3] += p->p[2] * wgt; acc[4] += wgt; acc[5] += g[G_MP] * wgt;
    T = testT;
    nl++;
    last = zk[q].id;
  }
  for (int k = 0; k < 6; k++) out[k] = acc[k];
  out[PX_T] = T; out[PX_N] = nl; out[PX_LAST] = (double)last; out[PX_W] = 0.0;
  free(zk);
  free(P);
  return flags;
}

/* ---- forward-mode pose Jacobian and the IRLS normal equations ----
 *
 * Levenberg-Marquardt pose refinement (Sec. V-A(c)) of the MP-weighted L1
 * objective of Eqs. (20)-(22). The paper names the method only; the reading:
 * each channel residual r_i of a pixel (colour r, g, b with coefficient
 * c_i = lambda_pho w(u); depth with lambda_depth w(u) where D_gt > 0; w(u)
 * held constant, as in the stop-gradient adjoint) enters a weighted least
 * squares problem with the iteratively-reweighted weight
 * W_i = c_i / max(|r_i|, delta), whose gradient equals that of c_i |r_i|
 * wherever |r_i| > delta. The Gauss-Newton model needs J_i = d r_i / d xi,
 * the derivative of the rendered channel along the twist xi = (rho, phi) of
 * the left perturbation T <- exp(xi^) T, at the current discrete decisions
 * (which Gaussians contribute, the alpha clamp, where the walk stops).
 *   H = sum_i W_i J_i J_i^T,   g = sum_i W_i r_i J_i,   L = sum_u w(u) l(u). */

/* d(u, v, a, b, c, z) / d xi_k of one projected Gaussian, k = 0..5 (conic in
 * natural units: power = -(a dx^2 + c dy^2)/2 - b dx dy). */
static void project_tangents(const proj_t *P, const double *cam, double tan[6][6]) {
  const double fx = cam[CAM_FX], fy = cam[CAM_FY];
  const double x = P->p[0], y = P->p[1], z = P->p[2];
  const double *J = P->J;
  for (int k = 0; k < 6; k++) {
    double dp[3] = {0, 0, 0}, dSc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (k < 3) {
      dp[k] = 1.0;
    } else {
      double ph[3] = {0, 0, 0};
      ph[k - 3] = 1.0;
      /* camera mean: phi x p; camera covariance: [phi]x Sc - Sc [phi]x */
      dp[0] = ph[1] * z - ph[2] * y;
      dp[1] = ph[2] * x - ph[0] * z;
      dp[2] = ph[0] * y - ph[1] * x;
      double Kx[9] = {0, -ph[2], ph[1], ph[2], 0, -ph[0], -ph[1], ph[0], 0};
      double A1[9], A2[9];
      mm3(Kx, P->Sc, A1);
      mm3(P->Sc, Kx, A2);
      for (int e = 0; e < 9; e++) dSc[e] = A1[e] - A2[e];
    }
    /* the guard clamp freezes x/z (y/z) in the Jacobian */
    double dtx = P->clx ? 0.0 : (dp[0] * z - x * dp[2]) / (z * z);
    double dty = P->cly ? 0.0 : (dp[1] * z - y * dp[2]) / (z * z);
    double dJ[6] = {-fx * dp[2] / (z * z), 0.0, -fx * (dtx * z - P->tx * dp[2]) / (z * z),
                    0.0, -fy * dp[2] / (z * z), -fy * (dty * z - P->ty * dp[2]) / (z * z)};
    /* d(J Sc J^T) */
    double dS2[4];
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++) {
        double s = 0;
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++)
            s += dJ[3 * i + a] * P->Sc[3 * a + b] * J[3 * j + b] + J[3 * i + a] * dSc[3 * a + b] * J[3 * j + b] +
                 J[3 * i + a] * P->Sc[3 * a + b] * dJ[3 * j + b];
        dS2[2 * i + j] = s;
      }
    /* conic Q = (2D covariance)^-1: dQ = -Q dS2 Q */
    double Q[4] = {P->a, P->b, P->b, P->c}, QdS[4], dQ[4];
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++) QdS[2 * i + j] = Q[2 * i] * dS2[j] + Q[2 * i + 1] * dS2[2 + j];
    for (int i = 0; i < 2; i++)
      for (int j = 0; j < 2; j++) dQ[2 * i + j] = -(QdS[2 * i] * Q[j] + QdS[2 * i + 1] * Q[2 + j]);
    tan[k][0] = fx * (dp[0] * z - x * dp[2]) / (z * z);
    tan[k][1] = fy * (dp[1] * z - y * dp[2]) / (z * z);
    tan[k][2] = dQ[0];
    tan[k][3] = dQ[1];
    tan[k][4] = dQ[3];
    tan[k][5] = dp[2];
  }
}

/* Render one view with the tangents of colour and depth and reduce the
 * normal equations. targets (P x 4) required. out_px[P * PX_STRIDE] or NULL,
 * out_J[P * 24] or NULL (per pixel: channels r, g, b, depth, each 6 twist
 * components), out_flags[P] (as oracle_render), normal[28] = L, H (upper
 * triangle, row-major, 21), g (6). Returns 0, or -1 on allocation failure. */
int oracle_render_jac(int64_t n, const double *G, const double *cam, const double *pose,
                      const double *rc, const double *lc, const double *targets, double delta,
                      double *out_px, double *out_J, int32_t *out_flags, double *normal) {
  int W = (int)cam[CAM_W], H = (int)cam[CAM_H];
  proj_t *P = (proj_t *)malloc(sizeof(proj_t) * (size_t)(n > 0 ? n : 1));
  zkey_t *zk = (zkey_t *)malloc(sizeof(zkey_t) * (size_t)(n > 0 ? n : 1));
  int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  double (*tan)[6][6] = (double (*)[6][6])malloc(sizeof(double) * 36 * (size_t)(n > 0 ? n : 1));
  if (!P || !zk || !order || !tan) return -1;
  int64_t nv = 0;
  for (int64_t i = 0; i < n; i++) {
    project_one(G + i * G_STRIDE, cam, pose, rc, &P[i]);
    if (P[i].vis) {
      zk[nv].z = P[i].zkey; zk[nv].id = i; nv++;
      project_tangents(&P[i], cam, tan[i]);
    }
  }
  qsort(zk, (size_t)nv, sizeof(zkey_t), cmp_zkey);
  for (int64_t k = 0; k < nv; k++) order[k] = zk[k].id;
  cells_t cs;
  build_cells(nv, P, order, W, H, 8, 1, &cs);

  const double amin = rc[RC_ALPHA_MIN], amax = rc[RC_ALPHA_MAX], tmin = rc[RC_T_MIN];
  double L = 0.0, Hm[36], gv[6];
  for (int k = 0; k < 36; k++) Hm[k] = 0.0;
  for (int k = 0; k < 6; k++) gv[k] = 0.0;

  for (int j = 0; j < H; j++)
    for (int i = 0; i < W; i++) {
      int c = (j / cs.cell) * cs.cw + (i / cs.cell);
      double T = 1.0, acc[6] = {0, 0, 0, 0, 0, 0}, eT = 0.0;
      double dT[6] = {0, 0, 0, 0, 0, 0}, dC[4][6];
      for (int a = 0; a < 4; a++)
        for (int k = 0; k < 6; k++) dC[a][k] = 0.0;
      int flags = 0;
      int64_t nl = 0, last = -1;
      for (int64_t q = cs.start[c]; q < cs.start[c + 1]; q++) {
        int64_t id = cs.ids[q];
        const proj_t *p = &P[id];
        double dx = p->u - i, dy = p->v - j;
        double power = -0.5 * (p->a * dx * dx + p->c * dy * dy) - p->b * dx * dy;
        double ag = p->o * exp(power);
        double em = exponent_margin(p, dx, dy, power);
        double lag = power + log(p->o);
        if (fabs(lag - log(amin)) <= em) flags |= FL_ALPHA;
        if (fabs(lag - log(amax)) <= em) flags |= FL_AMAX;
        if (ag < amin) continue;
        int clamped = ag > amax;
        double alpha = clamped ? amax : ag;
        double testT = T * (1.0 - alpha);
        double eTk = eT + (clamped ? 0.0 : alpha / (1.0 - alpha) * em) + 1e-6;
        if (fabs(log(testT) - log(tmin)) <= eTk) flags |= FL_TSTOP;
        if (testT < tmin) break;
        eT = eTk;
        const double *g = G + id * G_STRIDE;
        double wgt = alpha * T;
        acc[0] += g[G_CR] * wgt;
        acc[1] += g[G_CG] * wgt;
        acc[2] += g[G_CB] * wgt;
        acc[3] += p->p[2] * wgt;
        acc[4] += wgt;
        acc[5] += g[G_MP] * wgt;
        /* tangents: alpha' = alpha power' (0 where clamped); the weight
         * alpha T has tangent alpha' T + alpha T'; T' of the next entry is
         * T' (1 - alpha) - T alpha' */
        for (int k = 0; k < 6; k++) {
          const double *t = tan[id][k];
          double dpow = -0.5 * (t[2] * dx * dx + t[4] * dy * dy) - t[3] * dx * dy -
                        (p->a * dx + p->b * dy) * t[0] - (p->b * dx + p->c * dy) * t[1];
          double da = clamped ? 0.0 : alpha * dpow;
          double dw = da * T + alpha * dT[k];
          dC[0][k] += g[G_CR] * dw;
          dC[1][k] += g[G_CG] * dw;
          dC[2][k] += g[G_CB] * dw;
          dC[3][k] += p->p[2] * dw + wgt * t[5];
          dT[k] = dT[k] * (1.0 - alpha) - T * da;
        }
        nl++;
        last = id;
        T = testT;
      }
      int64_t pix = (int64_t)j * W + i;
      if (out_px) {
        double *o = out_px + pix * PX_STRIDE;
        for (int k = 0; k < 6; k++) o[k] = acc[k];
        o[PX_T] = T; o[PX_N] = (double)nl; o[PX_LAST] = (double)last; o[PX_W] = 0.0;
      }
      if (out_J)
        for (int a = 0; a < 4; a++)
          for (int k = 0; k < 6; k++) out_J[pix * 24 + a * 6 + k] = dC[a][k];
      const double *tg = targets + pix * 4;
      double O = acc[4], Rm = acc[5], w = 0.0;
      if (lc[LC_WMODE] == 0) {
        if (near_rel(O, lc[LC_OEPS])) flags |= FL_OEPS;
        if (O > lc[LC_OEPS]) w = (O - Rm) / O;
      } else {
        w = O - Rm;
      }
      if (out_px) out_px[pix * PX_STRIDE + PX_W] = w;
      out_flags[pix] = flags;
      if (!(tg[0] >= 0)) continue;
      const int dvalid = tg[3] > 0;
      double l1 = 0.0;
      for (int a = 0; a < 4; a++) {
        double r = acc[a] - tg[a];
        double cc = a < 3 ? lc[LC_LPHO] * w : (dvalid ? lc[LC_LDEPTH] * w : 0.0);
        if (a < 3) l1 += fabs(r);
        if (cc == 0.0) continue;
        double Wt = cc / fmax(fabs(r), delta);
        for (int k = 0; k < 6; k++) {
          gv[k] += Wt * r * dC[a][k];
          for (int m = k; m < 6; m++) Hm[6 * k + m] += Wt * dC[a][k] * dC[a][m];
        }
      }
      L += w * (lc[LC_LPHO] * l1 + (dvalid ? lc[LC_LDEPTH] * fabs(acc[3] - tg[3]) : 0.0));
    }
  normal[0] = L;
  int e = 1;
  for (int k = 0; k < 6; k++)
    for (int m = k; m < 6; m++) normal[e++] = Hm[6 * k + m];
  for (int k = 0; k < 6; k++) normal[22 + k] = gv[k];
  free(cs.start);
  free(cs.ids);
  free(tan);
  free(order);
  free(zk);
  free(P);
  return 0;
}
