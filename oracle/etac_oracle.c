/*
 * etac_oracle.c -- plain, slow FP64 restatement of the ETac tactile step.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load this library.  It shares no code, header, table or helper with the
 * CUDA library; both read the same seeded input arrays and nothing else.
 *
 * What it computes, per environment and per elastomer pad (ETac, Sec. III-A):
 *   1. contact detection with signed distance fields between the pad's surface nodes and the
 *      environment's rigid objects (Sec. III-A "Overview"): analytic primitives or closed
 *      triangle meshes (exact distance to the nearest surface point, sign by the winding
 *      number); phi = min over objects, node active iff phi < 0;
 *   2. the penalty-style local displacement of an active node: it is moved onto the object
 *      surface along the outward SDF normal, u_hat = -phi * grad(phi) (Sec. III-A, Table I:
 *      3-D element displacement);
 *   3. decay-based linear propagation to every passive node, Eq. 1 and the propagation
 *      matrix Omega[i,j] = exp(-alpha |p_j - p_i|), giving Omega * U_a;
 *   4. the residual network Phi (Sec. III-A 2): per-node shared MLP on [P, N, U_hat] (n x 9,
 *      passive displacements zero), channel max-pool to a 64-d global feature, a global MLP,
 *      broadcast + concat to n x 128, shared MLP decoder to n x 3, passive rows kept;
 *   5. Eq. 4: U_p = Omega U_a + Phi_p; active nodes keep u_hat.
 * Everything is written literally (no factoring, no tiling) in double precision.  A pad
 * with no active node outputs zero displacement.
 *
 * orc_regress is the real-to-sim taxel regressor of the appendix ("Modeling Real Sensors"),
 * which maps a pad's displacement field to its sensor's eight taxel outputs.
 *
 * orc_backward is the hand-derived reverse mode of the same steps (mask held fixed,
 * ReLU'(0) = 0, max-pool gradient routed to the lowest-index maximiser).  Pose gradients
 * are taken with respect to each object's world translation and a world-frame rotation
 * increment applied on the left about the object's origin.
 *
 * Hidden widths (64), ReLU activations, one global layer and the [local; global] concat
 * order are readings of Sec. III-A 2, which fixes only the 9 / 64 / 128 / 3 sizes.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define H 64          /* hidden width */
#define NIN 9         /* per-node input: position, normal, displacement */

enum { OBJ_NONE = 0, OBJ_SPHERE = 1, OBJ_BOX = 2, OBJ_CYLINDER = 3, OBJ_CAPSULE = 4, OBJ_MESH = 5 };
enum { MODE_FULL = 0, MODE_LINEAR_ONLY = 1, MODE_RESIDUAL_ONLY = 2, MODE_PENETRATION_ONLY = 3 };
/* the terms of Eq. 4 a mode keeps: the Eq. 1 propagation, the residual network; the
 * penetration-only mode keeps neither (active nodes u_hat, passive nodes zero) */
static int with_propagation(int mode) { return mode == MODE_FULL || mode == MODE_LINEAR_ONLY; }
static int with_residual(int mode) { return mode == MODE_FULL || mode == MODE_RESIDUAL_ONLY; }

typedef struct {
  int num_types;
  const int32_t* type_n;      /* [T] nodes per pad type                       */
  const double* type_pos;     /* [sum n, 3] undeformed node positions (pad frame) */
  const double* type_nrm;     /* [sum n, 3] undeformed unit normals          */
  int num_envs, pads_per_env, max_objects;
  const int32_t* pad_type;    /* [E*P] */
  const int32_t* obj_type;    /* [E*K] */
  const double* obj_dims;     /* [E*K*3] */
  const double* obj_pose;     /* [E*K*7] t, q(xyzw) world */
  const double* pad_pose;     /* [E*P*7] world */
  /* closed triangle meshes for OBJ_MESH objects (obj_dims[0] holds the mesh index) */
  int num_meshes;
  const int32_t* mesh_tri_off;  /* [M+1] first triangle of each mesh                  */
  const double* mesh_tri;       /* [sum T, 3, 3] vertices of each triangle, object frame,
                                 * counter-clockwise seen from outside                   */
} orc_scene;

/* parameter views into the flat vector: alpha, then W (row-major out x in) and b per layer */
typedef struct {
  double alpha;
  const double *W1, *b1, *W2, *b2, *Wg, *bg, *Wd, *bd, *W4, *b4;
} orc_params;

size_t orc_param_count(void) {
  return 1 + (H * NIN + H) + (H * H + H) + (H * H + H) + (H * 2 * H + H) + (3 * H + 3);
}

static void view_params(const double* th, orc_params* p) {
  const double* c = th;
  p->alpha = c[0]; c += 1;
  p->W1 = c; c += H * NIN; p->b1 = c; c += H;
  p->W2 = c; c += H * H;   p->b2 = c; c += H;
  p->Wg = c; c += H * H;   p->bg = c; c += H;
  p->Wd = c; c += H * 2 * H; p->bd = c; c += H;
  p->W4 = c; c += 3 * H;   p->b4 = c;
}

/* ----------------------------------------------------------------- rigid motions */

/* rotation matrix of a quaternion (x, y, z, w) after normalising it */
static void quat_to_mat(const double* q, double R[3][3]) {
  double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  double x = q[0] / n, y = q[1] / n, z = q[2] / n, w = q[3] / n;
  R[0][0] = 1 - 2 * (y * y + z * z); R[0][1] = 2 * (x * y - z * w); R[0][2] = 2 * (x * z + y * w);
  R[1][0] = 2 * (x * y + z * w); R[1][1] = 1 - 2 * (x * x + z * z); R[1][2] = 2 * (y * z - x * w);
  R[2][0] = 2 * (x * z - y * w); R[2][1] = 2 * (y * z + x * w); R[2][2] = 1 - 2 * (x * x + y * y);
}

static void mat_vec(double R[3][3], const double* v, double* o) {
  for (int a = 0; a < 3; ++a) o[a] = R[a][0] * v[0] + R[a][1] * v[1] + R[a][2] * v[2];
}

static void mat_t_vec(double R[3][3], const double* v, double* o) {
  for (int a = 0; a < 3; ++a) o[a] = R[0][a] * v[0] + R[1][a] * v[1] + R[2][a] * v[2];
}

static void cross(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}

/* ----------------------------------------------------------------- signed distances */

/* Exact SDF of a primitive in its own frame at point q: returns phi, writes the outward
 * gradient g and the Hessian Hs (only needed inside, where the node is active).  deg is set
 * when the gradient is undefined (q on a sphere centre / capsule or cylinder axis); the
 * caller then uses the fallback direction. */
static double sdf(int type, const double* dims, const double* q, double* g, double Hs[3][3],
                  int* deg) {
  *deg = 0;
  memset(Hs, 0, sizeof(double) * 9);
  g[0] = g[1] = g[2] = 0.0;
  if (type == OBJ_SPHERE) {
    double L = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    if (L > 0) {
      for (int a = 0; a < 3; ++a) g[a] = q[a] / L;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Hs[a][b] = ((a == b) - g[a] * g[b]) / L;
    } else {
      *deg = 1;
    }
    return L - dims[0];
  }
  if (type == OBJ_BOX) {
    double d[3], mx = -INFINITY, out2 = 0.0;
    int am = 0, outside = 0;
    for (int a = 0; a < 3; ++a) {
      d[a] = fabs(q[a]) - dims[a];
      if (d[a] > mx) { mx = d[a]; am = a; }   /* strict: ties keep the lowest axis */
      if (d[a] > 0) { outside = 1; out2 += d[a] * d[a]; }
    }
    if (outside) {
      double o = sqrt(out2);
      for (int a = 0; a < 3; ++a) g[a] = d[a] > 0 ? d[a] * (q[a] >= 0 ? 1.0 : -1.0) / o : 0.0;
      return o;
    }
    g[am] = q[am] >= 0 ? 1.0 : -1.0;
    return mx;
  }
  if (type == OBJ_CYLINDER) {
    double rho = sqrt(q[0] * q[0] + q[1] * q[1]);
    double dr = rho - dims[0], dz = fabs(q[2]) - dims[1];
    double sz = q[2] >= 0 ? 1.0 : -1.0;
    if (dr > 0 || dz > 0) {
      double er = dr > 0 ? dr : 0.0, ez = dz > 0 ? dz : 0.0, o = sqrt(er * er + ez * ez);
      if (rho > 0) { g[0] = er * q[0] / rho / o; g[1] = er * q[1] / rho / o; }
      g[2] = ez * sz / o;
      return o;
    }
    if (dr >= dz) {  /* ties go to the radial direction */
      if (rho > 0) {
        double nx = q[0] / rho, ny = q[1] / rho;
        g[0] = nx; g[1] = ny;
        Hs[0][0] = (1 - nx * nx) / rho; Hs[0][1] = -nx * ny / rho;
        Hs[1][0] = -nx * ny / rho;      Hs[1][1] = (1 - ny * ny) / rho;
      } else {
        *deg = 1;
      }
      return dr;
    }
    g[2] = sz;
    return dz;
  }
  if (type == OBJ_CAPSULE) {
    double h = dims[1];
    double cz = q[2] < -h ? -h : (q[2] > h ? h : q[2]);
    int side = (q[2] > -h && q[2] < h);
    double v[3] = {q[0], q[1], q[2] - cz};
    double L = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    if (L > 0) {
      for (int a = 0; a < 3; ++a) g[a] = v[a] / L;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double P = (a == b) ? ((side && a == 2) ? 0.0 : 1.0) : 0.0;
          Hs[a][b] = (P - g[a] * g[b]) / L;
        }
    } else {
      *deg = 1;
    }
    return L - dims[0];
  }
  return INFINITY;
}

/* ----------------------------------------------------------------- triangle meshes */

/* The object-mesh contact of Sec. III-A ("Overview"): signed distance from a node to a
 * closed triangle mesh, |phi| = distance to the nearest point of the surface, negative
 * inside.  Written as the plain definition: every triangle is visited. */

/* Closest point of segment [a, b] to p: the projection parameter clamped to [0, 1]. */
static double seg_closest(const double* p, const double* a, const double* b, double* cp,
                          double* t_out) {
  double ab[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  double ap[3] = {p[0] - a[0], p[1] - a[1], p[2] - a[2]};
  double L2 = ab[0] * ab[0] + ab[1] * ab[1] + ab[2] * ab[2];
  double t = L2 > 0 ? (ap[0] * ab[0] + ap[1] * ab[1] + ap[2] * ab[2]) / L2 : 0.0;
  t = t < 0 ? 0 : (t > 1 ? 1 : t);
  double d2 = 0.0;
  for (int k = 0; k < 3; ++k) {
    cp[k] = a[k] + t * ab[k];
    d2 += (p[k] - cp[k]) * (p[k] - cp[k]);
  }
  *t_out = t;
  return d2;
}

/* Closest point of triangle (a, b, c) to p.  If the orthogonal projection of p onto the
 * triangle's plane falls inside the triangle (all barycentric weights >= 0, to within
 * 1e-12) it is that
 * projection; otherwise the nearest point lies on the boundary, the closest of the three
 * edge segments' points.  Writes the point to cp, the feature that holds it to *feat
 * (0 face, 1 edge, 2 vertex) and the unit direction of the chosen edge to edir; returns the
 * squared distance. */
static double tri_closest(const double* p, const double* a, const double* b, const double* c,
                          double* cp, int* feat, double* edir) {
  double e0[3], e1[3], n[3], ap[3];
  for (int k = 0; k < 3; ++k) { e0[k] = b[k] - a[k]; e1[k] = c[k] - a[k]; ap[k] = p[k] - a[k]; }
  cross(e0, e1, n);
  double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  if (nn > 0) {
    double s = (ap[0] * n[0] + ap[1] * n[1] + ap[2] * n[2]) / nn;
    double q[3] = {p[0] - s * n[0], p[1] - s * n[1], p[2] - s * n[2]};
    /* barycentric weights of q from the sub-triangle areas (signed, along n) */
    double qa[3] = {a[0] - q[0], a[1] - q[1], a[2] - q[2]};
    double qb[3] = {b[0] - q[0], b[1] - q[1], b[2] - q[2]};
    double qc[3] = {c[0] - q[0], c[1] - q[1], c[2] - q[2]};
    double xa[3], xb[3], xc[3];
    cross(qb, qc, xa);
    cross(qc, qa, xb);
    cross(qa, qb, xc);
    double wa = (xa[0] * n[0] + xa[1] * n[1] + xa[2] * n[2]) / nn;
    double wb = (xb[0] * n[0] + xb[1] * n[1] + xb[2] * n[2]) / nn;
    double wc = (xc[0] * n[0] + xc[1] * n[1] + xc[2] * n[2]) / nn;
    /* a projection on a shared edge of two coplanar triangles counts as the face's point
     * on both (the tolerance absorbs the rounding of the weights there) */
    if (wa >= -1e-12 && wb >= -1e-12 && wc >= -1e-12) {
      for (int k = 0; k < 3; ++k) cp[k] = q[k];
      *feat = 0;
      return s * s * nn;
    }
  }
  const double* ends[3][2] = {{a, b}, {b, c}, {c, a}};
  double best = INFINITY, tb = 0.0;
  int eb = 0;
  for (int e = 0; e < 3; ++e) {
    double cq[3], t;
    double d2 = seg_closest(p, ends[e][0], ends[e][1], cq, &t);
    if (d2 < best) { best = d2; tb = t; eb = e; memcpy(cp, cq, sizeof cq); }
  }
  *feat = (tb > 0 && tb < 1) ? 1 : 2;
  double L = 0.0;
  for (int k = 0; k < 3; ++k) { edir[k] = ends[eb][1][k] - ends[eb][0][k]; L += edir[k] * edir[k]; }
  L = sqrt(L);
  for (int k = 0; k < 3; ++k) edir[k] = L > 0 ? edir[k] / L : 0.0;
  return best;
}

/* Signed solid angle of triangle (a, b, c) seen from p (van Oosterom and Strackee, 1983).
 * Its sign is that of (a-p).((b-p)x(c-p)): positive when p lies behind the triangle, on the
 * side opposite to its normal (b-a)x(c-a), as every point inside a closed mesh does for
 * triangles wound counter-clockwise seen from outside. */
static double solid_angle(const double* p, const double* a, const double* b, const double* c) {
  double A[3], B[3], C[3], bc[3];
  for (int k = 0; k < 3; ++k) { A[k] = a[k] - p[k]; B[k] = b[k] - p[k]; C[k] = c[k] - p[k]; }
  double la = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
  double lb = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
  double lc = sqrt(C[0] * C[0] + C[1] * C[1] + C[2] * C[2]);
  cross(B, C, bc);
  double num = A[0] * bc[0] + A[1] * bc[1] + A[2] * bc[2];
  double den = la * lb * lc + (A[0] * B[0] + A[1] * B[1] + A[2] * B[2]) * lc +
               (A[0] * C[0] + A[1] * C[1] + A[2] * C[2]) * lb +
               (B[0] * C[0] + B[1] * C[1] + B[2] * C[2]) * la;
  return 2.0 * atan2(num, den);
}

/* Signed distance to mesh `mi` at q (object frame).  The sign comes from the winding
 * number, the total solid angle over 4 pi: 1 inside a closed, consistently oriented mesh,
 * 0 outside; inside iff it exceeds 1/2.  The gradient is the outward unit direction
 * between q and its nearest surface point; the Hessian is zero when that point is interior
 * to a face, (I - e e^T - g g^T)/dist on an edge of direction e and (I - g g^T)/dist at a
 * vertex, times the sign.  Ties between triangles keep the lowest index. */
static double mesh_sdf(const orc_scene* sc, int mi, const double* q, double* g, double Hs[3][3]) {
  memset(Hs, 0, sizeof(double) * 9);
  g[0] = g[1] = g[2] = 0.0;
  if (mi < 0 || mi >= sc->num_meshes) return INFINITY;
  double best = INFINITY, wind = 0.0, bc[3] = {0, 0, 0}, be[3] = {0, 0, 0};
  int bf = 0;
  for (int t = sc->mesh_tri_off[mi]; t < sc->mesh_tri_off[mi + 1]; ++t) {
    const double* v = sc->mesh_tri + 9 * (size_t)t;
    double cp[3], ed[3] = {0, 0, 0};
    int f;
    double d2 = tri_closest(q, v, v + 3, v + 6, cp, &f, ed);
    if (d2 < best) { best = d2; bf = f; memcpy(bc, cp, sizeof bc); memcpy(be, ed, sizeof be); }
    wind += solid_angle(q, v, v + 3, v + 6);
  }
  double sgn = wind / (4.0 * M_PI) > 0.5 ? -1.0 : 1.0;
  double d = sqrt(best);
  if (d > 0) {
    for (int a = 0; a < 3; ++a) g[a] = sgn * (q[a] - bc[a]) / d;
    if (bf > 0)
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double P = (a == b) - g[a] * g[b] - (bf == 1 ? be[a] * be[b] : 0.0);
          Hs[a][b] = sgn * P / d;
        }
  }
  return sgn * d;
}

/* ----------------------------------------------------------------- per-pad state */

typedef struct {
  int n, m;
  const double *pos, *nrm;
  double Rp[3][3], tp[3];
  unsigned char* act;   /* [n] */
  double* phi;          /* [n] */
  double* uhat;         /* [n*3] pad frame, zero for passive nodes */
  double* gobj;         /* [n*3] outward normal in the object frame at the chosen object */
  double* Hs;           /* [n*9] SDF Hessian (object frame) */
  double* xw;           /* [n*3] world position of the node */
  int* kobj;            /* [n] chosen object (-1 if none) */
  /* network activations (all nodes) */
  double *a1, *a2, *f;  /* [n*H] */
  double g0[H], ag[H], g[H];
  int amax[H];
  double *a3;           /* [n*H] */
} pad_state;

static void pad_alloc(pad_state* s, int n) {
  s->n = n;
  s->act = (unsigned char*)calloc(n, 1);
  s->phi = (double*)calloc(n, sizeof(double));
  s->uhat = (double*)calloc(3 * n, sizeof(double));
  s->gobj = (double*)calloc(3 * n, sizeof(double));
  s->Hs = (double*)calloc(9 * n, sizeof(double));
  s->xw = (double*)calloc(3 * n, sizeof(double));
  s->kobj = (int*)calloc(n, sizeof(int));
  s->a1 = (double*)calloc((size_t)H * n, sizeof(double));
  s->a2 = (double*)calloc((size_t)H * n, sizeof(double));
  s->f = (double*)calloc((size_t)H * n, sizeof(double));
  s->a3 = (double*)calloc((size_t)H * n, sizeof(double));
}

static void pad_free(pad_state* s) {
  free(s->act); free(s->phi); free(s->uhat); free(s->gobj); free(s->Hs); free(s->xw);
  free(s->kobj); free(s->a1); free(s->a2); free(s->f); free(s->a3);
}

static double relu(double x) { return x > 0 ? x : 0.0; }

/* Contact detection + local displacement for every node of pad `pi` (steps 1-2). */
static void pad_contact(const orc_scene* sc, int pi, pad_state* s,
                        const unsigned char* mask_ovr, const double* uhat_ovr, long base) {
  int e = pi / sc->pads_per_env, K = sc->max_objects;
  quat_to_mat(sc->pad_pose + 7 * pi + 3, s->Rp);
  for (int a = 0; a < 3; ++a) s->tp[a] = sc->pad_pose[7 * pi + a];
  double Ro[8][3][3];
  for (int k = 0; k < K && k < 8; ++k) quat_to_mat(sc->obj_pose + 7 * (e * K + k) + 3, Ro[k]);
  s->m = 0;
  for (int i = 0; i < s->n; ++i) {
    const double* p = s->pos + 3 * i;
    double x[3];
    mat_vec(s->Rp, p, x);
    for (int a = 0; a < 3; ++a) x[a] += s->tp[a];
    for (int a = 0; a < 3; ++a) s->xw[3 * i + a] = x[a];
    double best = INFINITY, bg[3] = {0, 0, 0}, bH[3][3];
    int bk = -1, bdeg = 0;
    memset(bH, 0, sizeof bH);
    for (int k = 0; k < K; ++k) {
      int o = e * K + k, ty = sc->obj_type[o];
      if (ty == OBJ_NONE) continue;
      const double* to = sc->obj_pose + 7 * o;
      double r[3] = {x[0] - to[0], x[1] - to[1], x[2] - to[2]}, q[3], gg[3], HH[3][3];
      int deg;
      mat_t_vec(Ro[k], r, q);
      double ph = ty == OBJ_MESH
                      ? (deg = 0, mesh_sdf(sc, (int)sc->obj_dims[3 * o], q, gg, HH))
                      : sdf(ty, sc->obj_dims + 3 * o, q, gg, HH, &deg);
      if (ph < best) {  /* strict: ties keep the lowest object index */
        best = ph; bk = k; bdeg = deg;
        memcpy(bg, gg, sizeof bg);
        memcpy(bH, HH, sizeof bH);
      }
    }
    if (bk >= 0 && bdeg) {
      /* undefined SDF gradient: push the node back along its own inward normal */
      double nw[3];
      mat_vec(s->Rp, s->nrm + 3 * i, nw);
      mat_t_vec(Ro[bk], nw, bg);
      for (int a = 0; a < 3; ++a) bg[a] = -bg[a];
      memset(bH, 0, sizeof bH);
    }
    s->phi[i] = best;
    s->kobj[i] = bk;
    int act = best < 0.0;
    if (mask_ovr) act = mask_ovr[base + i] != 0;
    s->act[i] = (unsigned char)act;
    for (int a = 0; a < 3; ++a) s->gobj[3 * i + a] = bg[a];
    memcpy(s->Hs + 9 * i, bH, sizeof bH);
    double u[3] = {0, 0, 0};
    if (act) {
      if (uhat_ovr) {
        for (int a = 0; a < 3; ++a) u[a] = uhat_ovr[3 * (base + i) + a];
      } else if (bk >= 0) {
        double nwd[3];
        mat_vec(Ro[bk], bg, nwd);
        mat_t_vec(s->Rp, nwd, u);
        for (int a = 0; a < 3; ++a) u[a] *= -best;
      }
      s->m++;
    }
    for (int a = 0; a < 3; ++a) s->uhat[3 * i + a] = u[a];
  }
}

/* Residual network forward on all n nodes (step 4). */
static void pad_network(const orc_params* P, pad_state* s) {
  int n = s->n;
  for (int c = 0; c < H; ++c) { s->g0[c] = -INFINITY; s->amax[c] = 0; }
  for (int i = 0; i < n; ++i) {
    double X[NIN];
    for (int a = 0; a < 3; ++a) {
      X[a] = s->pos[3 * i + a];
      X[3 + a] = s->nrm[3 * i + a];
      X[6 + a] = s->uhat[3 * i + a];
    }
    double z1[H];
    for (int c = 0; c < H; ++c) {
      double acc = P->b1[c];
      for (int k = 0; k < NIN; ++k) acc += P->W1[c * NIN + k] * X[k];
      s->a1[(size_t)i * H + c] = acc;
      z1[c] = relu(acc);
    }
    for (int c = 0; c < H; ++c) {
      double acc = P->b2[c];
      for (int k = 0; k < H; ++k) acc += P->W2[c * H + k] * z1[k];
      s->a2[(size_t)i * H + c] = acc;
      double fv = relu(acc);
      s->f[(size_t)i * H + c] = fv;
      if (fv > s->g0[c]) { s->g0[c] = fv; s->amax[c] = i; }  /* lowest index on ties */
    }
  }
  for (int c = 0; c < H; ++c) {
    double acc = P->bg[c];
    for (int k = 0; k < H; ++k) acc += P->Wg[c * H + k] * s->g0[k];
    s->ag[c] = acc;
    s->g[c] = relu(acc);
  }
  for (int i = 0; i < n; ++i) {
    if (s->act[i]) continue;
    for (int c = 0; c < H; ++c) {
      double acc = P->bd[c];
      for (int k = 0; k < H; ++k) acc += P->Wd[c * 2 * H + k] * s->f[(size_t)i * H + k];
      for (int k = 0; k < H; ++k) acc += P->Wd[c * 2 * H + H + k] * s->g[k];
      s->a3[(size_t)i * H + c] = acc;
    }
  }
}

static void pad_forward(const orc_scene* sc, const orc_params* P, int mode, int pi, long base,
                        const unsigned char* mask_ovr, const double* uhat_ovr, pad_state* s,
                        double* disp) {
  int n = s->n;
  pad_contact(sc, pi, s, mask_ovr, uhat_ovr, base);
  double* U = disp + 3 * base;
  if (s->m == 0) {
    memset(U, 0, sizeof(double) * 3 * n);
    return;
  }
  for (int i = 0; i < n; ++i)
    for (int a = 0; a < 3; ++a) U[3 * i + a] = s->act[i] ? s->uhat[3 * i + a] : 0.0;
  if (with_propagation(mode)) {
    /* Eq. 1 summed over the active nodes: Omega U_a */
    for (int i = 0; i < n; ++i) {
      if (s->act[i]) continue;
      const double* pi_ = s->pos + 3 * i;
      double l[3] = {0, 0, 0};
      for (int j = 0; j < n; ++j) {
        if (!s->act[j]) continue;
        const double* pj = s->pos + 3 * j;
        double dx = pj[0] - pi_[0], dy = pj[1] - pi_[1], dz = pj[2] - pi_[2];
        double w = exp(-P->alpha * sqrt(dx * dx + dy * dy + dz * dz));
        for (int a = 0; a < 3; ++a) l[a] += w * s->uhat[3 * j + a];
      }
      for (int a = 0; a < 3; ++a) U[3 * i + a] += l[a];
    }
  }
  if (with_residual(mode)) {
    pad_network(P, s);
    for (int i = 0; i < n; ++i) {
      if (s->act[i]) continue;
      for (int a = 0; a < 3; ++a) {
        double acc = P->b4[a];
        for (int c = 0; c < H; ++c) acc += P->W4[a * H + c] * relu(s->a3[(size_t)i * H + c]);
        U[3 * i + a] += acc;
      }
    }
  }
}

static long pad_base(const orc_scene* sc, int pi, const long* offs) { (void)sc; return offs[pi]; }

static long* make_offsets(const orc_scene* sc, long* total) {
  int np = sc->num_envs * sc->pads_per_env;
  long* offs = (long*)malloc(sizeof(long) * (np + 1));
  offs[0] = 0;
  for (int p = 0; p < np; ++p) offs[p + 1] = offs[p] + sc->type_n[sc->pad_type[p]];
  *total = offs[np];
  return offs;
}

static const double* type_ptr(const orc_scene* sc, const double* arr, int t) {
  long o = 0;
  for (int u = 0; u < t; ++u) o += sc->type_n[u];
  return arr + 3 * o;
}

/* Forward over every pad.  Outputs (any may be NULL): disp [N*3], active mask [N], phi [N]
 * (min signed distance, +inf without objects), penetration max(0,-phi) [N], active count
 * per pad [E*P].  mask_ovr / uhat_ovr replace the contact result when given. */
int orc_forward(const orc_scene* sc, const double* theta, int mode,
                const unsigned char* mask_ovr, const double* uhat_ovr, double* disp,
                unsigned char* mask, double* phi, double* pen, int32_t* active_count,
                int nthreads) {
  orc_params P;
  if (sc->max_objects > 8) return 1;
  view_params(theta, &P);
  long N;
  long* offs = make_offsets(sc, &N);
  int np = sc->num_envs * sc->pads_per_env;
  double* D = disp ? disp : (double*)malloc(sizeof(double) * 3 * (N > 0 ? N : 1));
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int p = 0; p < np; ++p) {
    int t = sc->pad_type[p];
    pad_state s;
    pad_alloc(&s, sc->type_n[t]);
    s.pos = type_ptr(sc, sc->type_pos, t);
    s.nrm = type_ptr(sc, sc->type_nrm, t);
    long base = pad_base(sc, p, offs);
    pad_forward(sc, &P, mode, p, base, mask_ovr, uhat_ovr, &s, D);
    for (int i = 0; i < s.n; ++i) {
      if (mask) mask[base + i] = s.act[i];
      if (phi) phi[base + i] = s.phi[i];
      if (pen) pen[base + i] = s.phi[i] < 0 ? -s.phi[i] : 0.0;
    }
    if (active_count) active_count[p] = s.m;
    pad_free(&s);
  }
  if (!disp) free(D);
  free(offs);
  return 0;
}

/* Reverse mode of orc_forward for a given upstream gradient grad_disp [N*3].  Outputs (any
 * may be NULL, all overwritten): grad_obj_pose [E*K*6] (d/dt world, then d/d omega with the
 * rotation increment exp([omega]x) applied on the left about the object origin),
 * grad_uhat [N*3] (active nodes, pad frame), grad_pen [N] (active nodes, through
 * u_hat = pen * n), grad_params [orc_param_count()]. */
int orc_backward(const orc_scene* sc, const double* theta, int mode,
                 const unsigned char* mask_ovr, const double* uhat_ovr,
                 const double* grad_disp, double* grad_obj_pose, double* grad_uhat,
                 double* grad_pen, double* grad_params, int nthreads) {
  orc_params P;
  if (sc->max_objects > 8) return 1;
  view_params(theta, &P);
  long N;
  long* offs = make_offsets(sc, &N);
  int np = sc->num_envs * sc->pads_per_env, K = sc->max_objects;
  size_t npar = orc_param_count();
  int nth = 1;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
  nth = omp_get_max_threads();
#endif
  double* gpar_t = (double*)calloc((size_t)nth * npar, sizeof(double));
  double* gpose_p = (double*)calloc((size_t)np * K * 6 + 1, sizeof(double));
  double* D = (double*)malloc(sizeof(double) * 3 * (N > 0 ? N : 1));
#ifdef _OPENMP
#pragma omp parallel for schedule(static, 1)
#endif
  for (int p = 0; p < np; ++p) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* gp = gpar_t + (size_t)tid * npar;
    orc_params G;
    view_params(gp, &G);
    double *gW1 = (double*)G.W1, *gb1 = (double*)G.b1, *gW2 = (double*)G.W2,
           *gb2 = (double*)G.b2, *gWg = (double*)G.Wg, *gbg = (double*)G.bg,
           *gWd = (double*)G.Wd, *gbd = (double*)G.bd, *gW4 = (double*)G.W4,
           *gb4 = (double*)G.b4;
    int t = sc->pad_type[p], e = p / sc->pads_per_env;
    pad_state s;
    pad_alloc(&s, sc->type_n[t]);
    s.pos = type_ptr(sc, sc->type_pos, t);
    s.nrm = type_ptr(sc, sc->type_nrm, t);
    long base = pad_base(sc, p, offs);
    int n = s.n;
    pad_forward(sc, &P, mode, p, base, mask_ovr, uhat_ovr, &s, D);
    const double* Gd = grad_disp + 3 * base;
    double* gu = (double*)calloc(3 * (size_t)n, sizeof(double));
    if (s.m > 0) {
      for (int i = 0; i < n; ++i)
        if (s.act[i])
          for (int a = 0; a < 3; ++a) gu[3 * i + a] += Gd[3 * i + a];
      if (with_propagation(mode)) {
        for (int i = 0; i < n; ++i) {
          if (s.act[i]) continue;
          const double* pi_ = s.pos + 3 * i;
          for (int j = 0; j < n; ++j) {
            if (!s.act[j]) continue;
            const double* pj = s.pos + 3 * j;
            double dx = pj[0] - pi_[0], dy = pj[1] - pi_[1], dz = pj[2] - pi_[2];
            double d = sqrt(dx * dx + dy * dy + dz * dz);
            double w = exp(-P.alpha * d);
            double dot = 0.0;
            for (int a = 0; a < 3; ++a) {
              gu[3 * j + a] += w * Gd[3 * i + a];
              dot += Gd[3 * i + a] * s.uhat[3 * j + a];
            }
            gp[0] += -d * w * dot;
          }
        }
      }
      if (with_residual(mode)) {
        double* gf = (double*)calloc((size_t)H * n, sizeof(double));
        double gg[H], gag[H], gg0[H];
        memset(gg, 0, sizeof gg);
        for (int i = 0; i < n; ++i) {
          if (s.act[i]) continue;
          const double* gr = Gd + 3 * i;
          double z3[H], ga3[H];
          for (int c = 0; c < H; ++c) z3[c] = relu(s.a3[(size_t)i * H + c]);
          for (int a = 0; a < 3; ++a) {
            gb4[a] += gr[a];
            for (int c = 0; c < H; ++c) gW4[a * H + c] += gr[a] * z3[c];
          }
          for (int c = 0; c < H; ++c) {
            double gz = 0.0;
            for (int a = 0; a < 3; ++a) gz += P.W4[a * H + c] * gr[a];
            ga3[c] = s.a3[(size_t)i * H + c] > 0 ? gz : 0.0;
          }
          for (int c = 0; c < H; ++c) {
            gbd[c] += ga3[c];
            for (int k = 0; k < H; ++k) {
              gWd[c * 2 * H + k] += ga3[c] * s.f[(size_t)i * H + k];
              gWd[c * 2 * H + H + k] += ga3[c] * s.g[k];
            }
          }
          for (int k = 0; k < H; ++k) {
            double a = 0.0, b = 0.0;
            for (int c = 0; c < H; ++c) {
              a += P.Wd[c * 2 * H + k] * ga3[c];
              b += P.Wd[c * 2 * H + H + k] * ga3[c];
            }
            gf[(size_t)i * H + k] += a;
            gg[k] += b;
          }
        }
        for (int c = 0; c < H; ++c) gag[c] = s.ag[c] > 0 ? gg[c] : 0.0;
        for (int c = 0; c < H; ++c) {
          gbg[c] += gag[c];
          for (int k = 0; k < H; ++k) gWg[c * H + k] += gag[c] * s.g0[k];
        }
        for (int k = 0; k < H; ++k) {
          double a = 0.0;
          for (int c = 0; c < H; ++c) a += P.Wg[c * H + k] * gag[c];
          gg0[k] = a;
        }
        for (int c = 0; c < H; ++c) gf[(size_t)s.amax[c] * H + c] += gg0[c];
        for (int i = 0; i < n; ++i) {
          double ga2[H], ga1[H], z1[H], X[NIN];
          int any = 0;
          for (int c = 0; c < H; ++c) {
            ga2[c] = s.a2[(size_t)i * H + c] > 0 ? gf[(size_t)i * H + c] : 0.0;
            any |= ga2[c] != 0.0;
          }
          if (!any) continue;
          for (int c = 0; c < H; ++c) z1[c] = relu(s.a1[(size_t)i * H + c]);
          for (int a = 0; a < 3; ++a) {
            X[a] = s.pos[3 * i + a];
            X[3 + a] = s.nrm[3 * i + a];
            X[6 + a] = s.uhat[3 * i + a];
          }
          for (int c = 0; c < H; ++c) {
            gb2[c] += ga2[c];
            for (int k = 0; k < H; ++k) gW2[c * H + k] += ga2[c] * z1[k];
          }
          for (int k = 0; k < H; ++k) {
            double a = 0.0;
            for (int c = 0; c < H; ++c) a += P.W2[c * H + k] * ga2[c];
            ga1[k] = s.a1[(size_t)i * H + k] > 0 ? a : 0.0;
          }
          for (int c = 0; c < H; ++c) {
            gb1[c] += ga1[c];
            for (int k = 0; k < NIN; ++k) gW1[c * NIN + k] += ga1[c] * X[k];
          }
          if (s.act[i])
            for (int a = 0; a < 3; ++a) {
              double acc = 0.0;
              for (int c = 0; c < H; ++c) acc += P.W1[c * NIN + 6 + a] * ga1[c];
              gu[3 * i + a] += acc;
            }
        }
        free(gf);
      }
    }
    /* displacement -> penetration and object pose */
    double Ro[3][3];
    for (int i = 0; i < n; ++i) {
      long gi = base + i;
      if (grad_uhat)
        for (int a = 0; a < 3; ++a) grad_uhat[3 * gi + a] = s.act[i] ? gu[3 * i + a] : 0.0;
      if (grad_pen) grad_pen[gi] = 0.0;
      if (!s.act[i] || s.m == 0) continue;
      int k = s.kobj[i];
      if (k < 0 || uhat_ovr) continue;
      quat_to_mat(sc->obj_pose + 7 * (e * K + k) + 3, Ro);
      const double* gobj = s.gobj + 3 * i;
      double nw[3], npd[3], v[3];
      mat_vec(Ro, gobj, nw);
      mat_t_vec(s.Rp, nw, npd);
      if (grad_pen) grad_pen[gi] = npd[0] * gu[3 * i] + npd[1] * gu[3 * i + 1] + npd[2] * gu[3 * i + 2];
      mat_vec(s.Rp, gu + 3 * i, v);           /* dL/d(world displacement) */
      double vo[3], Av[3], sw[3];
      mat_t_vec(Ro, v, vo);                   /* object frame */
      double gdv = gobj[0] * vo[0] + gobj[1] * vo[1] + gobj[2] * vo[2];
      const double* Hs = s.Hs + 9 * i;
      for (int a = 0; a < 3; ++a) {
        Av[a] = gobj[a] * gdv;
        for (int b = 0; b < 3; ++b) Av[a] += s.phi[i] * Hs[3 * a + b] * vo[b];
      }
      mat_vec(Ro, Av, sw);
      const double* to = sc->obj_pose + 7 * (e * K + k);
      double r[3] = {s.xw[3 * i] - to[0], s.xw[3 * i + 1] - to[1], s.xw[3 * i + 2] - to[2]};
      double c1[3], c2[3];
      cross(r, sw, c1);
      cross(nw, v, c2);
      double* gpo = gpose_p + ((size_t)p * K + k) * 6;
      for (int a = 0; a < 3; ++a) {
        gpo[a] += sw[a];
        gpo[3 + a] += c1[a] - s.phi[i] * c2[a];
      }
    }
    free(gu);
    pad_free(&s);
  }
  if (grad_params) {
    memset(grad_params, 0, sizeof(double) * npar);
    for (int t = 0; t < nth; ++t)
      for (size_t q = 0; q < npar; ++q) grad_params[q] += gpar_t[(size_t)t * npar + q];
  }
  if (grad_obj_pose) {
    memset(grad_obj_pose, 0, sizeof(double) * (size_t)sc->num_envs * K * 6);
    for (int p = 0; p < np; ++p) {
      int e = p / sc->pads_per_env;
      for (int q = 0; q < K * 6; ++q)
        grad_obj_pose[(size_t)e * K * 6 + q] += gpose_p[(size_t)p * K * 6 + q];
    }
  }
  free(gpar_t);
  free(gpose_p);
  free(D);
  free(offs);
  return 0;
}

/* Margin of the max-pool's discrete choice (Sec. III-A 2: g0_c = max over the pad's n nodes of
 * f_ic).  For every pad p and channel c: top2[2 (64 p + c)] = the node holding the largest f_ic
 * and top2[... + 1] = the node holding the second largest (ties to the lower index; -1 when the
 * pad has one node), gap[64 p + c] = (f_top1 - f_top2) / f_top1 (INFINITY when f_top1 <= 0 or
 * the pad has one node).  The reverse mode routes a channel's gradient to its top node, so a
 * small gap flags a choice that a lower-precision evaluation of f may take differently.  The
 * contact step (and mask_ovr / uhat_ovr) are those of orc_forward; pads without contact are
 * reported too (their output is zero, so nothing is routed). */
int orc_pool_margin(const orc_scene* sc, const double* theta, const unsigned char* mask_ovr,
                    const double* uhat_ovr, int32_t* top2, double* gap, int nthreads) {
  orc_params P;
  if (sc->max_objects > 8) return 1;
  view_params(theta, &P);
  long N;
  long* offs = make_offsets(sc, &N);
  int np = sc->num_envs * sc->pads_per_env;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int p = 0; p < np; ++p) {
    int t = sc->pad_type[p];
    pad_state s;
    pad_alloc(&s, sc->type_n[t]);
    s.pos = type_ptr(sc, sc->type_pos, t);
    s.nrm = type_ptr(sc, sc->type_nrm, t);
    pad_contact(sc, p, &s, mask_ovr, uhat_ovr, offs[p]);
    pad_network(&P, &s);
    for (int c = 0; c < H; ++c) {
      int i1 = -1, i2 = -1;
      for (int i = 0; i < s.n; ++i) {
        double v = s.f[(size_t)i * H + c];
        if (i1 < 0 || v > s.f[(size_t)i1 * H + c]) {
          i2 = i1;
          i1 = i;
        } else if (i2 < 0 || v > s.f[(size_t)i2 * H + c]) {
          i2 = i;
        }
      }
      double f1 = s.f[(size_t)i1 * H + c];
      top2[2 * ((size_t)p * H + c)] = i1;
      top2[2 * ((size_t)p * H + c) + 1] = i2;
      gap[(size_t)p * H + c] =
          (i2 < 0 || !(f1 > 0.0)) ? INFINITY : (f1 - s.f[(size_t)i2 * H + c]) / f1;
    }
    pad_free(&s);
  }
  free(offs);
  return 0;
}

/* |x| / s, the margin of a ReLU or comparison decision on x relative to the scale s of the
 * terms it sums (INFINITY when s == 0: nothing to decide) */
static double rel_margin(double x, double s) { return s > 0.0 ? fabs(x) / s : INFINITY; }

/* Margins of every discrete decision that the reverse mode of the residual network takes
 * (Sec. III-A 2), per pad, as the smallest relative margin of each kind:
 *   margin[5 p + 0]  ReLU of E1 and E2 at passive nodes (the decoder path), and ReLU of the
 *                    decoder's hidden layer D1 at passive nodes;
 *   margin[5 p + 1]  ReLU of E1 and E2 at active nodes that hold a channel's maximum;
 *   margin[5 p + 2]  ReLU of the global layer G1;
 *   margin[5 p + 3]  max-pool: (f_top1 - f_top2) / f_top1 for channels whose top two nodes
 *                    include an active node (with f_top1 > 0);
 *   margin[5 p + 4]  the same for channels whose top two nodes are both passive.
 * A ReLU margin is |a| / (|b| + sum_k |w_k x_k|) for pre-activation a = b + sum_k w_k x_k.
 * Pads without contact output zero and take no decision: INFINITY throughout.  The contact
 * step (and mask_ovr / uhat_ovr) are those of orc_forward. */
int orc_decision_margin(const orc_scene* sc, const double* theta, const unsigned char* mask_ovr,
                        const double* uhat_ovr, double* margin, int nthreads) {
  orc_params P;
  if (sc->max_objects > 8) return 1;
  view_params(theta, &P);
  long N;
  long* offs = make_offsets(sc, &N);
  int np = sc->num_envs * sc->pads_per_env;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int p = 0; p < np; ++p) {
    int t = sc->pad_type[p];
    pad_state s;
    pad_alloc(&s, sc->type_n[t]);
    s.pos = type_ptr(sc, sc->type_pos, t);
    s.nrm = type_ptr(sc, sc->type_nrm, t);
    pad_contact(sc, p, &s, mask_ovr, uhat_ovr, offs[p]);
    double mg[5] = {INFINITY, INFINITY, INFINITY, INFINITY, INFINITY};
    if (s.m > 0) {
      pad_network(&P, &s);
      unsigned char* holds_max = (unsigned char*)calloc(s.n, 1);
      for (int c = 0; c < H; ++c) holds_max[s.amax[c]] = 1;
      for (int i = 0; i < s.n; ++i) {
        if (s.act[i] && !holds_max[i]) continue;   /* its features reach no output */
        int kind = s.act[i] ? 1 : 0;
        double X[NIN], z1[H];
        for (int a = 0; a < 3; ++a) {
          X[a] = s.pos[3 * i + a];
          X[3 + a] = s.nrm[3 * i + a];
          X[6 + a] = s.uhat[3 * i + a];
        }
        for (int c = 0; c < H; ++c) {
          double sc1 = fabs(P.b1[c]);
          for (int k = 0; k < NIN; ++k) sc1 += fabs(P.W1[c * NIN + k] * X[k]);
          double a1 = s.a1[(size_t)i * H + c];
          z1[c] = relu(a1);
          double mv = rel_margin(a1, sc1);
          if (mv < mg[kind]) mg[kind] = mv;
        }
        for (int c = 0; c < H; ++c) {
          double sc2 = fabs(P.b2[c]);
          for (int k = 0; k < H; ++k) sc2 += fabs(P.W2[c * H + k] * z1[k]);
          double mv = rel_margin(s.a2[(size_t)i * H + c], sc2);
          if (mv < mg[kind]) mg[kind] = mv;
        }
        if (!s.act[i])
          for (int c = 0; c < H; ++c) {
            double sc3 = fabs(P.bd[c]);
            for (int k = 0; k < H; ++k) sc3 += fabs(P.Wd[c * 2 * H + k] * s.f[(size_t)i * H + k]);
            for (int k = 0; k < H; ++k) sc3 += fabs(P.Wd[c * 2 * H + H + k] * s.g[k]);
            double mv = rel_margin(s.a3[(size_t)i * H + c], sc3);
            if (mv < mg[0]) mg[0] = mv;
          }
      }
      free(holds_max);
      for (int c = 0; c < H; ++c) {
        double scg = fabs(P.bg[c]);
        for (int k = 0; k < H; ++k) scg += fabs(P.Wg[c * H + k] * s.g0[k]);
        double mv = rel_margin(s.ag[c], scg);
        if (mv < mg[2]) mg[2] = mv;
        /* top two nodes of channel c (ties to the lower index) */
        int i1 = -1, i2 = -1;
        for (int i = 0; i < s.n; ++i) {
          double v = s.f[(size_t)i * H + c];
          if (i1 < 0 || v > s.f[(size_t)i1 * H + c]) {
            i2 = i1;
            i1 = i;
          } else if (i2 < 0 || v > s.f[(size_t)i2 * H + c]) {
            i2 = i;
          }
        }
        double f1 = s.f[(size_t)i1 * H + c];
        if (i2 >= 0 && f1 > 0.0) {
          double gp = (f1 - s.f[(size_t)i2 * H + c]) / f1;
          int kind = (s.act[i1] || s.act[i2]) ? 3 : 4;
          if (gp < mg[kind]) mg[kind] = gp;
        }
      }
    }
    for (int q = 0; q < 5; ++q) margin[5 * (size_t)p + q] = mg[q];
    pad_free(&s);
  }
  free(offs);
  return 0;
}

/* Signed distance, outward gradient [n*3] and Hessian [n*9] of mesh `mesh` of the scene at n
 * object-frame points q [n*3] (the same routine the contact step calls for OBJ_MESH). */
int orc_mesh_sdf(const orc_scene* sc, int mesh, long n, const double* q, double* phi,
                 double* grad, double* hess) {
  if (mesh < 0 || mesh >= sc->num_meshes) return 1;
  for (long i = 0; i < n; ++i) {
    double g[3], Hs[3][3];
    phi[i] = mesh_sdf(sc, mesh, q + 3 * i, g, Hs);
    if (grad) memcpy(grad + 3 * i, g, sizeof g);
    if (hess) memcpy(hess + 9 * i, Hs, sizeof Hs);
  }
  return 0;
}

/* ----------------------------------------------------------------- taxel regressor */

/* Real-to-sim taxel regressor (appendix "Modeling Real Sensors"): a PointNet-style network
 * from a pad's simulated displacement field to the outputs of the real sensor's eight
 * pressure taxels, with residual connections and attention pooling in place of max pooling.
 * The appendix fixes the attention MLP ([256, 128, 1], tanh) and the softmax; the encoder
 * widths, the residual layer and the head are readings (the figure is not in the text):
 *   x_i = [p_i, n_i, U_i]                           (9, pad frame)
 *   h1 = relu(R1 x + b), h2 = relu(R2 h1 + b), h3 = relu(R3 h2 + b)   (64, 128, 256)
 *   f_i = h3 + relu(R4 h3 + b)                      (256, residual)
 *   a_i = A2 tanh(A1 f_i + b) + b                   (attention score)
 *   alpha = softmax over the pad's nodes of a       (computed as exp(a_i - max a) / sum)
 *   g = sum_i alpha_i f_i
 *   y = H2 relu(H1 g + b) + b                       (8 taxels)
 * Parameters: W (row-major, out x in) then b for R1, R2, R3, R4, A1, A2, H1, H2. */
#define RT 8
static const int reg_dims[8][2] = {{64, 9}, {128, 64}, {256, 128}, {256, 256},
                                   {128, 256}, {1, 128}, {128, 256}, {RT, 128}};

size_t orc_regressor_param_count(void) {
  size_t n = 0;
  for (int l = 0; l < 8; ++l) n += (size_t)reg_dims[l][0] * reg_dims[l][1] + reg_dims[l][0];
  return n;
}

/* y = W x + b for layer l of the flat regressor vector */
static void reg_layer(const double* rp, int l, const double* x, double* y) {
  size_t off = 0;
  for (int k = 0; k < l; ++k) off += (size_t)reg_dims[k][0] * reg_dims[k][1] + reg_dims[k][0];
  int o = reg_dims[l][0], in = reg_dims[l][1];
  const double* W = rp + off;
  const double* b = W + (size_t)o * in;
  for (int r = 0; r < o; ++r) {
    double acc = b[r];
    for (int c = 0; c < in; ++c) acc += W[(size_t)r * in + c] * x[c];
    y[r] = acc;
  }
}

/* disp [N*3] (pad frame) -> taxels [pads*8]; attn [N] (optional) receives the softmax
 * weights of every node within its pad. */
int orc_regress(const orc_scene* sc, const double* disp, const double* rp, double* taxels,
                double* attn, int nthreads) {
  long N;
  long* offs = make_offsets(sc, &N);
  int np = sc->num_envs * sc->pads_per_env;
#ifdef _OPENMP
  if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
  for (int p = 0; p < np; ++p) {
    int t = sc->pad_type[p], n = sc->type_n[t];
    const double* pos = type_ptr(sc, sc->type_pos, t);
    const double* nrm = type_ptr(sc, sc->type_nrm, t);
    long base = offs[p];
    double* f = (double*)malloc(sizeof(double) * 256 * (size_t)(n > 0 ? n : 1));
    double* a = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
      double x[9], h1[64], h2[128], h3[256], h4[256], s1[128], s;
      for (int k = 0; k < 3; ++k) {
        x[k] = pos[3 * i + k];
        x[3 + k] = nrm[3 * i + k];
        x[6 + k] = disp[3 * (base + i) + k];
      }
      reg_layer(rp, 0, x, h1);
      for (int k = 0; k < 64; ++k) h1[k] = relu(h1[k]);
      reg_layer(rp, 1, h1, h2);
      for (int k = 0; k < 128; ++k) h2[k] = relu(h2[k]);
      reg_layer(rp, 2, h2, h3);
      for (int k = 0; k < 256; ++k) h3[k] = relu(h3[k]);
      reg_layer(rp, 3, h3, h4);
      for (int k = 0; k < 256; ++k) f[(size_t)i * 256 + k] = h3[k] + relu(h4[k]);
      reg_layer(rp, 4, f + (size_t)i * 256, s1);
      for (int k = 0; k < 128; ++k) s1[k] = tanh(s1[k]);
      reg_layer(rp, 5, s1, &s);
      a[i] = s;
    }
    double mx = -INFINITY, Z = 0.0, g[256], z[128], y[RT];
    for (int i = 0; i < n; ++i) mx = a[i] > mx ? a[i] : mx;
    for (int i = 0; i < n; ++i) { a[i] = exp(a[i] - mx); Z += a[i]; }
    for (int k = 0; k < 256; ++k) g[k] = 0.0;
    for (int i = 0; i < n; ++i) {
      double al = a[i] / Z;
      if (attn) attn[base + i] = al;
      for (int k = 0; k < 256; ++k) g[k] += al * f[(size_t)i * 256 + k];
    }
    reg_layer(rp, 6, g, z);
    for (int k = 0; k < 128; ++k) z[k] = relu(z[k]);
    reg_layer(rp, 7, z, y);
    for (int k = 0; k < RT; ++k) taxels[(size_t)p * RT + k] = n > 0 ? y[k] : 0.0;
    free(f);
    free(a);
  }
  free(offs);
  return 0;
}
