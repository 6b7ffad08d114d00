/*
 * Correctness oracle: a plain, slow FP64 full-grid S-model discrete velocity
 * method on an unstructured hex mesh (Chikitkin, Kornev & Titarev,
 * arXiv:1912.04582).
 *
 * TEST INFRASTRUCTURE ONLY.  It is linked by the tests, by the package entry
 * point's smoke check and by the benchmark's CPU-baseline leg, and by nothing
 * else.  It shares no code with the CUDA library: geometry, face matching,
 * moments, equilibrium, boundary values and the update are written here from
 * the paper, in its order:
 *
 *   Section 2   model equation, macroparameters [n, u, T, q], Shakhov operator,
 *               diffuse-wall / symmetry / free-stream boundary conditions;
 *   Section 3   velocity grid and quadrature, finite-volume form (ode_system),
 *               CIR upwind flux (exact-flux), explicit Euler (expl-scheme-final),
 *               Algorithm 1 (time step) and Algorithm 2 (computeJ);
 *               the implicit scheme (linear-system, diagonal_term): one LU-SGS
 *               pass per step over the cells in index order.
 *
 * Readings of points the paper leaves open (each is also listed with its
 * reason in the design notes):
 *   - units: R_g = 1/2, m = 1 (so 2 R_g T = T), nu = p / mu(T) with
 *     mu = (Kn / sqrt(pi)) T^omega, i.e. nu = sqrt(pi)/(2 Kn) n T^(1-omega);
 *   - Shakhov coefficient: the factor printed in the shakhov_integral equation
 *     is read as (2/5)(1-Pr) / (p R_g T) with q = (m/2) int v v^2 f, so that the
 *     heat flux of f^S is (1-Pr) q (the S-model's defining property);
 *   - velocity nodes xi_i = ((N-1-i) lo + i hi) / (N-1), i = 0..N-1 (equal to
 *     lo + i*dxi, written so that a grid with lo = -hi is exactly symmetric);
 *     every node has weight dxi_1 dxi_2 dxi_3;
 *   - face area vector = (1/2)(p2 - p0) x (p3 - p1) of the quad (exact for a
 *     bilinear face), cell volume = (1/3) sum_faces centroid . area vector;
 *   - the time step is one value per solve: dt = CFL / max_i [nu_i +
 *     (1/(2|V_i|)) sum_l |A_l| xi_max] taken on the initial state;
 *   - residual = ||U^{n+1} - U^n||_{2,V} / (dt ||U^n||_{2,V}) with U the
 *     conserved moments (n, n u, sum w xi^2 f) and a volume-weighted L2 norm.
 *
 * Storage: f[cell][i1][i2][i3], i3 fastest (N1 x N2 x N3 per cell).
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define ORC_FREESTREAM 0
#define ORC_ZEROGRAD 1
#define ORC_SYMMETRY 2
#define ORC_WALL 3
#define ORC_MAX_GROUPS 4096

static const double ORC_PI = 3.14159265358979323846;

/* Quads of a VTK-ordered hexahedron, outward by the right-hand rule. */
static const int HEX_FACE[6][4] = {
    {0, 4, 7, 3}, {1, 2, 6, 5}, {0, 1, 5, 4}, {3, 7, 6, 2}, {0, 3, 2, 1}, {4, 5, 6, 7}};

typedef struct {
  int64_t owner;  /* cell whose local order defines the area vector          */
  int64_t nb;     /* neighbour cell, or -1 on the boundary                   */
  int32_t group;  /* boundary group, -1 for interior faces                   */
  int32_t sym_axis; /* for symmetry faces: the axis of the normal            */
  double area;    /* |A_j|                                                   */
  double e[3];    /* unit normal pointing from owner to neighbour / outside  */
} orc_face;

typedef struct orc {
  int64_t nc, nf, nnode;
  int N[3];
  double lo[3], hi[3];
  double *xi[3];
  double w;       /* quadrature weight dxi1 dxi2 dxi3 */
  double xi_max;  /* max over nodes of |xi| */
  double Pr, omega, Kn;
  double *vol;
  orc_face *face;
  int64_t *cell_face; /* [nc][6] global face of local face l */
  int8_t *cell_sign;  /* [nc][6] +1 if the cell is the owner, -1 otherwise */
  int32_t bc_type[ORC_MAX_GROUPS];
  double bc_par[ORC_MAX_GROUPS][8];
  int32_t bc_set[ORC_MAX_GROUPS];
  int32_t max_group;
  double *f, *fnew;
  double *ghost_scale; /* per face: wall density n_w (boundary wall faces only) */
  double *wall_hat;    /* per group: unit-density wall Maxwellian over the grid  */
  double *free_max;    /* per group: free-stream Maxwellian over the grid        */
  char err[256];
} orc;

/* ----------------------------------------------------------------------- */
/* compensated (Neumaier) summation                                        */
typedef struct { double s, c; } ksum;
static void ks_add(ksum *k, double x) {
  double t = k->s + x;
  if (fabs(k->s) >= fabs(x)) k->c += (k->s - t) + x;
  else k->c += (x - t) + k->s;
  k->s = t;
}
static double ks_val(const ksum *k) { return k->s + k->c; }

/* ----------------------------------------------------------------------- */
/* grid (Section 3)                                                         */
static int make_grid(orc *P, const int32_t *N, const double *lo, const double *hi) {
  P->nnode = 1;
  double dxi[3];
  double m2 = 0.0;
  for (int a = 0; a < 3; ++a) {
    if (N[a] < 2 || !(hi[a] > lo[a])) return -1;
    P->N[a] = N[a];
    P->lo[a] = lo[a];
    P->hi[a] = hi[a];
    P->xi[a] = (double *)malloc(sizeof(double) * N[a]);
    for (int i = 0; i < N[a]; ++i)
      P->xi[a][i] = ((double)(N[a] - 1 - i) * lo[a] + (double)i * hi[a]) / (double)(N[a] - 1);
    dxi[a] = (hi[a] - lo[a]) / (double)(N[a] - 1);
    P->nnode *= N[a];
    double am = fabs(lo[a]) > fabs(hi[a]) ? fabs(lo[a]) : fabs(hi[a]);
    m2 += am * am;
  }
  P->w = dxi[0] * dxi[1] * dxi[2];
  P->xi_max = sqrt(m2);
  return 0;
}

/* ----------------------------------------------------------------------- */
/* geometry                                                                */
static void quad_area(const double *xyz, const int64_t *v, double A[3], double c[3]) {
  const double *p0 = xyz + 3 * v[0], *p1 = xyz + 3 * v[1], *p2 = xyz + 3 * v[2],
               *p3 = xyz + 3 * v[3];
  double d1[3], d2[3];
  for (int k = 0; k < 3; ++k) {
    d1[k] = p2[k] - p0[k];
    d2[k] = p3[k] - p1[k];
    c[k] = 0.25 * (p0[k] + p1[k] + p2[k] + p3[k]);
  }
  A[0] = 0.5 * (d1[1] * d2[2] - d1[2] * d2[1]);
  A[1] = 0.5 * (d1[2] * d2[0] - d1[0] * d2[2]);
  A[2] = 0.5 * (d1[0] * d2[1] - d1[1] * d2[0]);
}

typedef struct { int64_t key[4]; int64_t cell; int32_t lf; } face_key;

static int cmp_i64(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return (x > y) - (x < y);
}
static int cmp_key(const void *a, const void *b) {
  const face_key *x = (const face_key *)a, *y = (const face_key *)b;
  for (int k = 0; k < 4; ++k) {
    if (x->key[k] != y->key[k]) return (x->key[k] > y->key[k]) - (x->key[k] < y->key[k]);
  }
  if (x->cell != y->cell) return (x->cell > y->cell) - (x->cell < y->cell);
  return x->lf - y->lf;
}

static int build_mesh(orc *P, int64_t n_vert, const double *xyz, int64_t nc, const int64_t *hex8,
                      int64_t nb, const int64_t *bface, const int32_t *bgroup) {
  P->nc = nc;
  if (nc <= 0) { snprintf(P->err, sizeof P->err, "empty mesh"); return -1; }
  for (int64_t i = 0; i < 8 * nc; ++i)
    if (hex8[i] < 0 || hex8[i] >= n_vert) { snprintf(P->err, sizeof P->err, "bad vertex id"); return -1; }
  face_key *keys = (face_key *)malloc(sizeof(face_key) * 6 * nc);
  for (int64_t c = 0; c < nc; ++c)
    for (int l = 0; l < 6; ++l) {
      face_key *k = &keys[6 * c + l];
      for (int q = 0; q < 4; ++q) k->key[q] = hex8[8 * c + HEX_FACE[l][q]];
      qsort(k->key, 4, sizeof(int64_t), cmp_i64);
      k->cell = c;
      k->lf = l;
    }
  qsort(keys, 6 * nc, sizeof(face_key), cmp_key);
  P->cell_face = (int64_t *)malloc(sizeof(int64_t) * 6 * nc);
  P->cell_sign = (int8_t *)malloc((size_t)(6 * nc));
  for (int64_t i = 0; i < 6 * nc; ++i) P->cell_face[i] = -1;
  P->face = (orc_face *)malloc(sizeof(orc_face) * 6 * nc);
  int64_t nf = 0;
  /* boundary lookup: (cell, lf) -> group */
  int32_t *bmark = (int32_t *)malloc(sizeof(int32_t) * 6 * nc);
  for (int64_t i = 0; i < 6 * nc; ++i) bmark[i] = -1;
  for (int64_t b = 0; b < nb; ++b) {
    int64_t c = bface[2 * b], l = bface[2 * b + 1];
    if (c < 0 || c >= nc || l < 0 || l > 5 || bgroup[b] < 0 || bgroup[b] >= ORC_MAX_GROUPS ||
        bmark[6 * c + l] >= 0) {
      snprintf(P->err, sizeof P->err, "bad boundary face entry %lld", (long long)b);
      free(keys); free(bmark); return -1;
    }
    bmark[6 * c + l] = bgroup[b];
    if (bgroup[b] > P->max_group) P->max_group = bgroup[b];
  }
  int64_t i = 0;
  while (i < 6 * nc) {
    int64_t j = i + 1;
    while (j < 6 * nc && memcmp(keys[j].key, keys[i].key, sizeof keys[i].key) == 0) ++j;
    int64_t cnt = j - i;
    if (cnt > 2) { snprintf(P->err, sizeof P->err, "face shared by >2 cells"); free(keys); free(bmark); return -1; }
    orc_face *F = &P->face[nf];
    int64_t oc = keys[i].cell;
    int ol = keys[i].lf;
    int64_t v[4];
    for (int q = 0; q < 4; ++q) v[q] = hex8[8 * oc + HEX_FACE[ol][q]];
    double A[3], cc[3];
    quad_area(xyz, v, A, cc);
    double an = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
    F->owner = oc;
    F->area = an;
    for (int k = 0; k < 3; ++k) F->e[k] = A[k] / an;
    F->sym_axis = -1;
    P->cell_face[6 * oc + ol] = nf;
    P->cell_sign[6 * oc + ol] = 1;
    if (cnt == 2) {
      if (bmark[6 * oc + ol] >= 0 || bmark[6 * keys[i + 1].cell + keys[i + 1].lf] >= 0) {
        snprintf(P->err, sizeof P->err, "interior face listed as boundary"); free(keys); free(bmark); return -1;
      }
      F->nb = keys[i + 1].cell;
      F->group = -1;
      P->cell_face[6 * F->nb + keys[i + 1].lf] = nf;
      P->cell_sign[6 * F->nb + keys[i + 1].lf] = -1;
    } else {
      if (bmark[6 * oc + ol] < 0) {
        snprintf(P->err, sizeof P->err, "unmatched face without boundary group"); free(keys); free(bmark); return -1;
      }
      F->nb = -1;
      F->group = bmark[6 * oc + ol];
    }
    ++nf;
    i = j;
  }
  P->nf = nf;
  free(keys);
  free(bmark);
  /* volumes: divergence theorem over each cell's own six quads */
  P->vol = (double *)malloc(sizeof(double) * nc);
  for (int64_t c = 0; c < nc; ++c) {
    double s = 0.0;
    for (int l = 0; l < 6; ++l) {
      int64_t v[4];
      for (int q = 0; q < 4; ++q) v[q] = hex8[8 * c + HEX_FACE[l][q]];
      double A[3], cc[3];
      quad_area(xyz, v, A, cc);
      s += cc[0] * A[0] + cc[1] * A[1] + cc[2] * A[2];
    }
    P->vol[c] = s / 3.0;
    if (!(P->vol[c] > 0.0)) { snprintf(P->err, sizeof P->err, "non-positive cell volume"); return -1; }
  }
  return 0;
}

/* ----------------------------------------------------------------------- */
/* Maxwellian on the grid (Section 2): n (2 pi R_g T)^{-3/2} exp(-|xi-u|^2/(2 R_g T)), R_g = 1/2 */
static void maxwellian(const orc *P, double n, const double *u, double T, double *out) {
  const double c = n / pow(ORC_PI * T, 1.5);
  int64_t idx = 0;
  for (int i1 = 0; i1 < P->N[0]; ++i1)
    for (int i2 = 0; i2 < P->N[1]; ++i2)
      for (int i3 = 0; i3 < P->N[2]; ++i3, ++idx) {
        double v1 = P->xi[0][i1] - u[0], v2 = P->xi[1][i2] - u[1], v3 = P->xi[2][i3] - u[2];
        out[idx] = c * exp(-(v1 * v1 + v2 * v2 + v3 * v3) / T);
      }
}

/* ----------------------------------------------------------------------- */
/* Algorithm 2, lines 2-9: macroparameters of one cell.  a = [n, u1,u2,u3, T, q1,q2,q3] */
static void macro(const orc *P, const double *f, double a[8]) {
  ksum s0 = {0, 0}, s1[3] = {{0, 0}, {0, 0}, {0, 0}}, s2 = {0, 0};
  int64_t idx = 0;
  for (int i1 = 0; i1 < P->N[0]; ++i1)
    for (int i2 = 0; i2 < P->N[1]; ++i2)
      for (int i3 = 0; i3 < P->N[2]; ++i3, ++idx) {
        double x1 = P->xi[0][i1], x2 = P->xi[1][i2], x3 = P->xi[2][i3];
        double g = f[idx];
        ks_add(&s0, g);
        ks_add(&s1[0], x1 * g);
        ks_add(&s1[1], x2 * g);
        ks_add(&s1[2], x3 * g);
        ks_add(&s2, (x1 * x1 + x2 * x2 + x3 * x3) * g);
      }
  const double w = P->w;
  double n = w * ks_val(&s0);
  double u[3];
  for (int a2 = 0; a2 < 3; ++a2) u[a2] = w * ks_val(&s1[a2]) / n;
  double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double Rg = 0.5;
  double T = (w * ks_val(&s2) - n * uu) / (3.0 * n * Rg);
  ksum q[3] = {{0, 0}, {0, 0}, {0, 0}};
  idx = 0;
  for (int i1 = 0; i1 < P->N[0]; ++i1)
    for (int i2 = 0; i2 < P->N[1]; ++i2)
      for (int i3 = 0; i3 < P->N[2]; ++i3, ++idx) {
        double v1 = P->xi[0][i1] - u[0], v2 = P->xi[1][i2] - u[1], v3 = P->xi[2][i3] - u[2];
        double v2s = v1 * v1 + v2 * v2 + v3 * v3;
        double g = f[idx];
        ks_add(&q[0], v1 * v2s * g);
        ks_add(&q[1], v2 * v2s * g);
        ks_add(&q[2], v3 * v2s * g);
      }
  a[0] = n;
  a[1] = u[0]; a[2] = u[1]; a[3] = u[2];
  a[4] = T;
  for (int a2 = 0; a2 < 3; ++a2) a[5 + a2] = 0.5 * w * ks_val(&q[a2]); /* m = 1 */
}

/* collision frequency nu = p / mu(T) (Section 2), nondimensional */
static double collision_nu(const orc *P, double n, double T) {
  return sqrt(ORC_PI) / (2.0 * P->Kn) * n * pow(T, 1.0 - P->omega);
}

/* Algorithm 2, lines 10-11: f^S at every node (written to out) */
static void shakhov(const orc *P, const double a[8], double *out) {
  const double Rg = 0.5;
  double n = a[0], T = a[4];
  const double *u = a + 1, *q = a + 5;
  double p = n * Rg * T; /* rho R_g T with m = 1 */
  double coef = 0.4 * (1.0 - P->Pr) / (p * Rg * T);
  double c = n / pow(2.0 * ORC_PI * Rg * T, 1.5);
  int64_t idx = 0;
  for (int i1 = 0; i1 < P->N[0]; ++i1)
    for (int i2 = 0; i2 < P->N[1]; ++i2)
      for (int i3 = 0; i3 < P->N[2]; ++i3, ++idx) {
        double v1 = P->xi[0][i1] - u[0], v2 = P->xi[1][i2] - u[1], v3 = P->xi[2][i3] - u[2];
        double v2s = v1 * v1 + v2 * v2 + v3 * v3;
        double fM = c * exp(-v2s / (2.0 * Rg * T));
        double qv = q[0] * v1 + q[1] * v2 + q[2] * v3;
        out[idx] = fM * (1.0 + coef * qv * (v2s / (2.0 * Rg * T) - 2.5));
      }
}

/* ----------------------------------------------------------------------- */
/* ghost value of face j at node (i1,i2,i3) given the owner's f (boundary) */
static double face_right_value(const orc *P, int64_t j, const double *fl, const double *fr,
                               int i1, int i2, int i3, int64_t idx) {
  const orc_face *F = &P->face[j];
  if (F->nb >= 0) return fr[idx];
  int g = F->group;
  switch (P->bc_type[g]) {
    case ORC_ZEROGRAD:
      return fl[idx];
    case ORC_SYMMETRY: {
      int ii[3] = {i1, i2, i3};
      int a = F->sym_axis;
      ii[a] = P->N[a] - 1 - ii[a];
      return fl[((int64_t)ii[0] * P->N[1] + ii[1]) * P->N[2] + ii[2]];
    }
    case ORC_FREESTREAM:
      return P->free_max[(int64_t)g * P->nnode + idx];
    case ORC_WALL:
      return P->ghost_scale[j] * P->wall_hat[(int64_t)g * P->nnode + idx];
  }
  return 0.0;
}

/* CIR flux of face j at one node (exact-flux equation):
 *   F = 1/2 xn (fL + fR) - 1/2 |xn| (fR - fL)  ==  xn^+ fL + xn^- fR                   */
static double face_flux(const orc *P, int64_t j, const double *f, int i1, int i2, int i3,
                        int64_t idx) {
  const orc_face *F = &P->face[j];
  const double *fl = f + F->owner * P->nnode;
  const double *fr = F->nb >= 0 ? f + F->nb * P->nnode : NULL;
  double xn = F->e[0] * P->xi[0][i1] + F->e[1] * P->xi[1][i2] + F->e[2] * P->xi[2][i3];
  double xp = xn > 0.0 ? xn : 0.0;
  double xm = xn < 0.0 ? xn : 0.0;
  double vl = fl[idx];
  double vr = face_right_value(P, j, fl, fr, i1, i2, i3, idx);
  return xp * vl + xm * vr;
}

/* ----------------------------------------------------------------------- */
/* public API                                                              */

orc *orc_create(int64_t n_vert, const double *xyz, int64_t n_cell, const int64_t *hex8,
                int64_t n_bface, const int64_t *bface, const int32_t *bgroup, const int32_t *N,
                const double *lo, const double *hi, double Pr, double omega, double Kn,
                char *err_out) {
  orc *P = (orc *)calloc(1, sizeof(orc));
  P->max_group = -1;
  if (make_grid(P, N, lo, hi) != 0) {
    if (err_out) snprintf(err_out, 256, "bad velocity grid");
    free(P);
    return NULL;
  }
  P->Pr = Pr;
  P->omega = omega;
  P->Kn = Kn;
  if (build_mesh(P, n_vert, xyz, n_cell, hex8, n_bface, bface, bgroup) != 0) {
    if (err_out) snprintf(err_out, 256, "%s", P->err);
    return NULL; /* leaks on error: test infrastructure */
  }
  P->f = (double *)calloc((size_t)(P->nc * P->nnode), sizeof(double));
  P->fnew = (double *)calloc((size_t)(P->nc * P->nnode), sizeof(double));
  P->ghost_scale = (double *)calloc((size_t)P->nf, sizeof(double));
  int ng = P->max_group + 1;
  if (ng < 1) ng = 1;
  P->wall_hat = (double *)calloc((size_t)(ng * P->nnode), sizeof(double));
  P->free_max = (double *)calloc((size_t)(ng * P->nnode), sizeof(double));
  return P;
}

void orc_destroy(orc *P) {
  if (!P) return;
  for (int a = 0; a < 3; ++a) free(P->xi[a]);
  free(P->vol); free(P->face); free(P->cell_face); free(P->cell_sign);
  free(P->f); free(P->fnew); free(P->ghost_scale); free(P->wall_hat); free(P->free_max);
  free(P);
}

const char *orc_error(orc *P) { return P->err; }

int orc_set_bc(orc *P, int32_t group, int32_t type, const double *par) {
  if (group < 0 || group > P->max_group || type < 0 || type > 3) return -1;
  P->bc_type[group] = type;
  for (int k = 0; k < 8; ++k) P->bc_par[group][k] = par[k];
  P->bc_set[group] = 1;
  double *dst;
  switch (type) {
    case ORC_FREESTREAM:
      maxwellian(P, par[0], par + 1, par[4], P->free_max + (int64_t)group * P->nnode);
      break;
    case ORC_WALL:
      dst = P->wall_hat + (int64_t)group * P->nnode;
      maxwellian(P, 1.0, par + 1, par[4], dst);
      break;
    default:
      break;
  }
  /* symmetry: the plane must be a coordinate plane and the grid symmetric about 0 */
  for (int64_t j = 0; j < P->nf; ++j) {
    orc_face *F = &P->face[j];
    if (F->nb >= 0 || F->group != group) continue;
    F->sym_axis = -1;
    if (type == ORC_SYMMETRY) {
      for (int a = 0; a < 3; ++a)
        if (fabs(fabs(F->e[a]) - 1.0) < 1e-12) F->sym_axis = a;
      if (F->sym_axis < 0 || P->lo[F->sym_axis] != -P->hi[F->sym_axis]) {
        snprintf(P->err, sizeof P->err, "symmetry needs an axis plane and a symmetric grid");
        return -2;
      }
    }
  }
  return 0;
}

static int check_bcs(orc *P) {
  for (int64_t j = 0; j < P->nf; ++j)
    if (P->face[j].nb < 0 && !P->bc_set[P->face[j].group]) {
      snprintf(P->err, sizeof P->err, "boundary group %d has no condition", P->face[j].group);
      return -1;
    }
  return 0;
}

int orc_init_maxwellian(orc *P, const double *n, const double *u, const double *T) {
  for (int64_t c = 0; c < P->nc; ++c) maxwellian(P, n[c], u + 3 * c, T[c], P->f + c * P->nnode);
  return check_bcs(P);
}

int orc_init_f(orc *P, const double *f) {
  memcpy(P->f, f, sizeof(double) * P->nc * P->nnode);
  return check_bcs(P);
}

int orc_get_f(const orc *P, double *out) {
  memcpy(out, P->f, sizeof(double) * P->nc * P->nnode);
  return 0;
}

/* per-cell macroparameters [n,u,T,q] -> out[nc][8] */
int orc_macro(const orc *P, double *out) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t c = 0; c < P->nc; ++c) macro(P, P->f + c * P->nnode, out + 8 * c);
  return 0;
}

/* geometry export for tests: vol[nc]; per face (owner, nb, group) and (area, e[3]) */
int orc_geometry(const orc *P, double *vol, int64_t *fcell, double *fgeo) {
  for (int64_t c = 0; c < P->nc; ++c) vol[c] = P->vol[c];
  for (int64_t j = 0; j < P->nf; ++j) {
    fcell[3 * j] = P->face[j].owner;
    fcell[3 * j + 1] = P->face[j].nb;
    fcell[3 * j + 2] = P->face[j].group;
    fgeo[4 * j] = P->face[j].area;
    for (int k = 0; k < 3; ++k) fgeo[4 * j + 1 + k] = P->face[j].e[k];
  }
  return 0;
}

int64_t orc_num_faces(const orc *P) { return P->nf; }

/* the fixed time step of a solve (taken on the current state) */
double orc_dt(const orc *P, double cfl) {
  double worst = 0.0;
  for (int64_t c = 0; c < P->nc; ++c) {
    double a[8];
    macro(P, P->f + c * P->nnode, a);
    double s = 0.0;
    for (int l = 0; l < 6; ++l) s += P->face[P->cell_face[6 * c + l]].area;
    double rate = collision_nu(P, a[0], a[4]) + s * P->xi_max / (2.0 * P->vol[c]);
    if (rate > worst) worst = rate;
  }
  return cfl / worst;
}

/* conserved moments U = (n, n u1, n u2, n u3, w sum |xi|^2 f) of one cell */
static void conserved(const orc *P, const double *f, double U[5]) {
  ksum s[5];
  memset(s, 0, sizeof s);
  int64_t idx = 0;
  for (int i1 = 0; i1 < P->N[0]; ++i1)
    for (int i2 = 0; i2 < P->N[1]; ++i2)
      for (int i3 = 0; i3 < P->N[2]; ++i3, ++idx) {
        double x1 = P->xi[0][i1], x2 = P->xi[1][i2], x3 = P->xi[2][i3];
        double g = f[idx];
        ks_add(&s[0], g);
        ks_add(&s[1], x1 * g);
        ks_add(&s[2], x2 * g);
        ks_add(&s[3], x3 * g);
        ks_add(&s[4], (x1 * x1 + x2 * x2 + x3 * x3) * g);
      }
  for (int k = 0; k < 5; ++k) U[k] = P->w * ks_val(&s[k]);
}

/* boundary conditions: wall density from impermeability (Section 2) */
static void set_wall_density(orc *P) {
  const int64_t nn = P->nnode;
#pragma omp parallel for schedule(dynamic, 8)
  for (int64_t j = 0; j < P->nf; ++j) {
    orc_face *F = &P->face[j];
    if (F->nb >= 0 || P->bc_type[F->group] != ORC_WALL) continue;
    const double *fl = P->f + F->owner * nn;
    const double *fw = P->wall_hat + (int64_t)F->group * nn;
    ksum out = {0, 0}, in = {0, 0};
    int64_t idx = 0;
    for (int i1 = 0; i1 < P->N[0]; ++i1)
      for (int i2 = 0; i2 < P->N[1]; ++i2)
        for (int i3 = 0; i3 < P->N[2]; ++i3, ++idx) {
          double xn = F->e[0] * P->xi[0][i1] + F->e[1] * P->xi[1][i2] + F->e[2] * P->xi[2][i3];
          if (xn > 0.0) ks_add(&out, xn * fl[idx]);
          else if (xn < 0.0) ks_add(&in, xn * fw[idx]);
        }
    P->ghost_scale[j] = -ks_val(&out) / ks_val(&in);
  }
}

/* Algorithm 1: one explicit time step (returns the residual) */
static double one_step(orc *P, double dt) {
  const int64_t nn = P->nnode;
  set_wall_density(P);
  double num = 0.0, den = 0.0;
  /* cell loop: R_i = J(f_i) - sum_l sign(i,l) |A_j| / |V_i| F_j ;  f_i += dt R_i */
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : num, den)
  for (int64_t c = 0; c < P->nc; ++c) {
    const double *fc = P->f + c * nn;
    double *fo = P->fnew + c * nn;
    double a[8];
    macro(P, fc, a);
    double nu = collision_nu(P, a[0], a[4]);
    shakhov(P, a, fo); /* fo temporarily holds f^S */
    int64_t idx = 0;
    for (int i1 = 0; i1 < P->N[0]; ++i1)
      for (int i2 = 0; i2 < P->N[1]; ++i2)
        for (int i3 = 0; i3 < P->N[2]; ++i3, ++idx) {
          double R = nu * (fo[idx] - fc[idx]);
          for (int l = 0; l < 6; ++l) {
            int64_t j = P->cell_face[6 * c + l];
            double Fj = face_flux(P, j, P->f, i1, i2, i3, idx);
            R -= (double)P->cell_sign[6 * c + l] * P->face[j].area / P->vol[c] * Fj;
          }
          fo[idx] = fc[idx] + dt * R;
        }
    double U0[5], U1[5];
    conserved(P, fc, U0);
    conserved(P, fo, U1);
    for (int k = 0; k < 5; ++k) {
      num += P->vol[c] * (U1[k] - U0[k]) * (U1[k] - U0[k]);
      den += P->vol[c] * U0[k] * U0[k];
    }
  }
  double *t = P->f;
  P->f = P->fnew;
  P->fnew = t;
  return sqrt(num) / (dt * sqrt(den));
}

int orc_step(orc *P, int32_t nsteps, double dt, double *residual) {
  double r = 0.0;
  for (int s = 0; s < nsteps; ++s) r = one_step(P, dt);
  if (residual) *residual = r;
  return 0;
}

/* building blocks exported for the pin tests */
int orc_cell_shakhov(const orc *P, const double *f, double *fs_out, double *a_out) {
  double a[8];
  macro(P, f, a);
  shakhov(P, a, fs_out);
  if (a_out) memcpy(a_out, a, sizeof a);
  return 0;
}

int orc_shakhov_from_macro(const orc *P, const double *a, double *fs_out) {
  shakhov(P, a, fs_out);
  return 0;
}

int orc_maxwellian(const orc *P, double n, const double *u, double T, double *out) {
  maxwellian(P, n, u, T, out);
  return 0;
}

double orc_nu(const orc *P, double n, double T) { return collision_nu(P, n, T); }

int orc_nodes(const orc *P, int32_t axis, double *out) {
  for (int i = 0; i < P->N[axis]; ++i) out[i] = P->xi[axis][i];
  return 0;
}

double orc_weight(const orc *P) { return P->w; }

/* wall densities n_w of the last step, per face (0 for non-wall faces) */
int orc_wall_density(const orc *P, double *out) {
  for (int64_t j = 0; j < P->nf; ++j) out[j] = P->ghost_scale[j];
  return 0;
}

/* ----------------------------------------------------------------------- */
/* Implicit step, Section 3 (linear-system and diagonal_term equations): the
 * right-hand side of the explicit scheme is taken at t^{n+1} and linearised,
 *   [I/dt - dR/df] (f^{n+1} - f^n) = R^n,
 * and the system is solved approximately by one symmetric Gauss-Seidel pass
 * (LU-SGS) over the cells in their index order.  With e_l outward from cell i
 * and the upwind flux xn^+ f_i + xn^- f_nb of Algorithm 1, the blocks are
 *   diagonal    D_i  = 1/dt + nu_i + (1/(2|V_i|)) sum_l |A_l| |xi.e_l|
 *                      (the diagonal_term equation; f^S held fixed),
 *   off-diagonal M_ij = (|A_l| / |V_i|) (xi.e_l)^-    (interior face l to j),
 * and boundary ghost values stay at their t^n values (they enter R^n only).
 *   forward : for i = 0 .. nc-1   D_i g_i   = R_i - sum_{j<i} M_ij g_j
 *   backward: for i = nc-1 .. 0   df_i      = g_i - D_i^{-1} sum_{j>i} M_ij df_j
 *   f^{n+1} = f^n + df.
 * Every operation is a node-by-node one, so the division by D_i is exact here
 * (the full-grid format). */

/* R^n of one cell at every node (Algorithm 1 without the Euler update) */
static void cell_rhs(const orc *P, int64_t c, double *R) {
  const int64_t nn = P->nnode;
  const double *fc = P->f + c * nn;
  double a[8];
  macro(P, fc, a);
  double nu = collision_nu(P, a[0], a[4]);
  shakhov(P, a, R); /* R temporarily holds f^S */
  int64_t idx = 0;
  for (int i1 = 0; i1 < P->N[0]; ++i1)
    for (int i2 = 0; i2 < P->N[1]; ++i2)
      for (int i3 = 0; i3 < P->N[2]; ++i3, ++idx) {
        double r = nu * (R[idx] - fc[idx]);
        for (int l = 0; l < 6; ++l) {
          int64_t j = P->cell_face[6 * c + l];
          double Fj = face_flux(P, j, P->f, i1, i2, i3, idx);
          r -= (double)P->cell_sign[6 * c + l] * P->face[j].area / P->vol[c] * Fj;
        }
        R[idx] = r;
      }
}

/* the neighbour blocks of cell c on one side of it:
 *   out = sum over interior faces l with (nb < c) == lower of M_c,nb x[nb]      */
static void offdiag_sum(const orc *P, int64_t c, const double *x, int lower, double *out) {
  const int64_t nn = P->nnode;
  for (int64_t k = 0; k < nn; ++k) out[k] = 0.0;
  for (int l = 0; l < 6; ++l) {
    int64_t j = P->cell_face[6 * c + l];
    const orc_face *F = &P->face[j];
    if (F->nb < 0) continue;
    int64_t nb = F->owner == c ? F->nb : F->owner;
    if ((nb < c) != (lower != 0)) continue;
    double s = (double)P->cell_sign[6 * c + l], k = F->area / P->vol[c];
    const double *xn_ = x + nb * nn;
    int64_t idx = 0;
    for (int i1 = 0; i1 < P->N[0]; ++i1)
      for (int i2 = 0; i2 < P->N[1]; ++i2)
        for (int i3 = 0; i3 < P->N[2]; ++i3, ++idx) {
          double xn = s * (F->e[0] * P->xi[0][i1] + F->e[1] * P->xi[1][i2] +
                           F->e[2] * P->xi[2][i3]);
          if (xn < 0.0) out[idx] += k * xn * xn_[idx];
        }
  }
}

/* the diagonal tensor D_i (diagonal_term equation) */
static void cell_diag(const orc *P, int64_t c, double dt, double *D) {
  double a[8];
  macro(P, P->f + c * P->nnode, a);
  double nu = collision_nu(P, a[0], a[4]);
  int64_t idx = 0;
  for (int i1 = 0; i1 < P->N[0]; ++i1)
    for (int i2 = 0; i2 < P->N[1]; ++i2)
      for (int i3 = 0; i3 < P->N[2]; ++i3, ++idx) {
        double s = 0.0;
        for (int l = 0; l < 6; ++l) {
          const orc_face *F = &P->face[P->cell_face[6 * c + l]];
          double xn = F->e[0] * P->xi[0][i1] + F->e[1] * P->xi[1][i2] + F->e[2] * P->xi[2][i3];
          s += F->area * fabs(xn);
        }
        D[idx] = 1.0 / dt + nu + s / (2.0 * P->vol[c]);
      }
}

static double one_step_lusgs(orc *P, double dt) {
  const int64_t nn = P->nnode, nc = P->nc;
  set_wall_density(P);
  double *g = P->fnew; /* R, then g, then df */
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t c = 0; c < nc; ++c) cell_rhs(P, c, g + c * nn);
  double *D = (double *)malloc(sizeof(double) * nn);
  double *S = (double *)malloc(sizeof(double) * nn);
  for (int64_t c = 0; c < nc; ++c) { /* forward sweep */
    cell_diag(P, c, dt, D);
    offdiag_sum(P, c, g, 1, S);
    double *gc = g + c * nn;
    for (int64_t k = 0; k < nn; ++k) gc[k] = (gc[k] - S[k]) / D[k];
  }
  for (int64_t c = nc - 1; c >= 0; --c) { /* backward sweep */
    cell_diag(P, c, dt, D);
    offdiag_sum(P, c, g, 0, S);
    double *gc = g + c * nn;
    for (int64_t k = 0; k < nn; ++k) gc[k] -= S[k] / D[k];
  }
  free(D);
  free(S);
  double num = 0.0, den = 0.0;
  for (int64_t c = 0; c < nc; ++c) {
    double *fc = P->f + c * nn, *dc = g + c * nn;
    double U0[5], U1[5];
    conserved(P, fc, U0);
    for (int64_t k = 0; k < nn; ++k) dc[k] = fc[k] + dc[k]; /* f^{n+1} */
    conserved(P, dc, U1);
    for (int k = 0; k < 5; ++k) {
      num += P->vol[c] * (U1[k] - U0[k]) * (U1[k] - U0[k]);
      den += P->vol[c] * U0[k] * U0[k];
    }
  }
  double *t = P->f;
  P->f = P->fnew;
  P->fnew = t;
  return sqrt(num) / (dt * sqrt(den));
}

int orc_step_lusgs(orc *P, int32_t nsteps, double dt, double *residual) {
  double r = 0.0;
  for (int s = 0; s < nsteps; ++s) r = one_step_lusgs(P, dt);
  if (residual) *residual = r;
  return 0;
}

/* R^n of every cell (the explicit right-hand side), for the pin tests */
int orc_rhs(orc *P, double *out) {
  set_wall_density(P);
  for (int64_t c = 0; c < P->nc; ++c) cell_rhs(P, c, out + c * P->nnode);
  return 0;
}

/* D_i of every cell (diagonal_term equation), for the pin tests */
int orc_lusgs_diag(const orc *P, double dt, double *out) {
  for (int64_t c = 0; c < P->nc; ++c) cell_diag(P, c, dt, out + c * P->nnode);
  return 0;
}
