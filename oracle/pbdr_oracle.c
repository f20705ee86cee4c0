/*
 * PBD-R reference oracle (FP64, serial).  TEST INFRASTRUCTURE ONLY: see the
 * header.  Every function follows the paper's definitions in the paper's
 * order; the passages are cited beside each one.  Where the paper is silent
 * (contact and friction formulas, neighbour search) the standard PBD reading
 * is written out and named.
 *
 * Build: cc -O2 -std=c11 -ffp-contract=off -fPIC -shared pbdr_oracle.c -lm
 */
#include "pbdr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* small FP64 vector helpers                                                */
/* ------------------------------------------------------------------------ */

static double dot3(const double *a, const double *b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static void cross3(const double *a, const double *b, double *o) {
  double t0 = a[1] * b[2] - a[2] * b[1];
  double t1 = a[2] * b[0] - a[0] * b[2];
  double t2 = a[0] * b[1] - a[1] * b[0];
  o[0] = t0;
  o[1] = t1;
  o[2] = t2;
}

static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* ------------------------------------------------------------------------ */
/* neighbour search (FP32 predicate).  The paper needs the set of particle  */
/* pairs of different object groups that may touch (Sec. III-A, constraint  */
/* (2)) but does not say how it is found; this is a uniform grid hashed with */
/* the Teschner et al. 2003 prime-XOR hash, plus the O(N^2) definition.     */
/* ------------------------------------------------------------------------ */

void orc_nbr_constants(float radius, float *Rn, float *Rn2, float *h, float *inv_h) {
  float rn = (float)(2.2 * (double)radius);
  float hh = (float)((double)rn * (1.0 + 1.0 / 1024.0));
  *Rn = rn;
  *Rn2 = rn * rn;
  *h = hh;
  *inv_h = (float)(1.0 / (double)hh);
}

uint32_t orc_table_size(int32_t n) {
  uint32_t want = (uint32_t)(n > 0 ? n : 1) * 2u;
  uint32_t t = 1;
  while (t < want) t <<= 1;
  return t;
}

static int32_t cell_coord(float x, float inv_h) {
  float u = floorf(x * inv_h);
  u = fminf(fmaxf(u, -1.0e9f), 1.0e9f);
  return (int32_t)u;
}

static uint32_t cell_hash(int32_t ix, int32_t iy, int32_t iz) {
  return ((uint32_t)ix * 73856093u) ^ ((uint32_t)iy * 19349663u) ^
         ((uint32_t)iz * 83492791u);
}

void orc_cell_keys(int32_t n, const float *x, float inv_h, uint32_t T, uint32_t *key) {
  for (int32_t p = 0; p < n; ++p) {
    int32_t ix = cell_coord(x[3 * p + 0], inv_h);
    int32_t iy = cell_coord(x[3 * p + 1], inv_h);
    int32_t iz = cell_coord(x[3 * p + 2], inv_h);
    key[p] = cell_hash(ix, iy, iz) & (T - 1u);
  }
}

/* counting sort: stable, so ids stay ascending within a key */
void orc_sort_keys(int32_t n, const uint32_t *key, uint32_t T,
                   uint32_t *sorted_key, uint32_t *sorted_id) {
  uint32_t *start = (uint32_t *)calloc((size_t)T + 1, sizeof(uint32_t));
  for (int32_t p = 0; p < n; ++p) start[key[p] + 1]++;
  for (uint32_t k = 0; k < T; ++k) start[k + 1] += start[k];
  for (int32_t p = 0; p < n; ++p) {
    uint32_t at = start[key[p]]++;
    sorted_key[at] = key[p];
    sorted_id[at] = (uint32_t)p;
  }
  free(start);
}

/* squared distance in FP32: dx = x_q - x_p per axis, then (dx*dx + dy*dy) + dz*dz,
 * every operation rounded to nearest (no fused multiply-add) */
static int fp32_within(const float *xp, const float *xq, float Rn2) {
  float dx = xq[0] - xp[0];
  float dy = xq[1] - xp[1];
  float dz = xq[2] - xp[2];
  float d2 = dx * dx + dy * dy;
  d2 = d2 + dz * dz;
  return d2 < Rn2;
}

int64_t orc_neighbors_brute(int32_t n, const float *x, const int32_t *body,
                            float Rn2, int32_t *off, int32_t *idx, int64_t cap) {
  int64_t cnt = 0;
  for (int32_t p = 0; p < n; ++p) {
    off[p] = (int32_t)(cnt < INT32_MAX ? cnt : INT32_MAX);
    for (int32_t q = 0; q < n; ++q) {
      if (q == p || body[q] == body[p]) continue;
      if (!fp32_within(x + 3 * p, x + 3 * q, Rn2)) continue;
      if (cnt < cap) idx[cnt] = q;
      cnt++;
    }
  }
  off[n] = (int32_t)(cnt < INT32_MAX ? cnt : INT32_MAX);
  return cnt;
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}

int64_t orc_neighbors_grid(int32_t n, const float *x, const int32_t *body,
                           float Rn2, float inv_h, int32_t *off, int32_t *idx,
                           int64_t cap) {
  uint32_t T = orc_table_size(n);
  uint32_t *key = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  uint32_t *skey = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  uint32_t *sid = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
  int32_t *cstart = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
  int32_t *cend = (int32_t *)malloc(sizeof(int32_t) * (size_t)T);
  int32_t *cand = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  orc_cell_keys(n, x, inv_h, T, key);
  orc_sort_keys(n, key, T, skey, sid);
  for (uint32_t k = 0; k < T; ++k) cstart[k] = cend[k] = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (i == 0 || skey[i] != skey[i - 1]) cstart[skey[i]] = i;
    if (i == n - 1 || skey[i] != skey[i + 1]) cend[skey[i]] = i + 1;
  }
  int64_t cnt = 0;
  for (int32_t p = 0; p < n; ++p) {
    off[p] = (int32_t)(cnt < INT32_MAX ? cnt : INT32_MAX);
    int32_t ix = cell_coord(x[3 * p + 0], inv_h);
    int32_t iy = cell_coord(x[3 * p + 1], inv_h);
    int32_t iz = cell_coord(x[3 * p + 2], inv_h);
    uint32_t buckets[27];
    int nbk = 0;
    for (int dz = -1; dz <= 1; ++dz)
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          uint32_t b = cell_hash(ix + dx, iy + dy, iz + dz) & (T - 1u);
          int dup = 0;
          for (int k = 0; k < nbk; ++k) dup |= (buckets[k] == b);
          if (!dup) buckets[nbk++] = b;
        }
    int32_t nc = 0;
    for (int k = 0; k < nbk; ++k) {
      for (int32_t i = cstart[buckets[k]]; i < cend[buckets[k]]; ++i) {
        int32_t q = (int32_t)sid[i];
        if (q == p || body[q] == body[p]) continue;
        if (!fp32_within(x + 3 * p, x + 3 * q, Rn2)) continue;
        cand[nc++] = q;
      }
    }
    qsort(cand, (size_t)nc, sizeof(int32_t), cmp_i32);
    for (int32_t k = 0; k < nc; ++k) {
      if (cnt < cap) idx[cnt] = cand[k];
      cnt++;
    }
  }
  off[n] = (int32_t)(cnt < INT32_MAX ? cnt : INT32_MAX);
  free(key); free(skey); free(sid); free(cstart); free(cend); free(cand);
  return cnt;
}

/* ------------------------------------------------------------------------ */
/* shape matching (Sec. III-A constraint (3), Sec. III-C; Mueller et al.    */
/* 2005): rest offsets, optimal rotation, goals                              */
/* ------------------------------------------------------------------------ */

void orc_rest_shape(int32_t n, int32_t nb, const int32_t *body_off,
                    const double *inv_mass, const double *x0, double *rest,
                    double *body_mass) {
  (void)n;
  for (int32_t b = 0; b < nb; ++b) {
    double M = 0.0, c[3] = {0.0, 0.0, 0.0};
    for (int32_t p = body_off[b]; p < body_off[b + 1]; ++p) {
      double m = 1.0 / inv_mass[p];
      M += m;
      for (int k = 0; k < 3; ++k) c[k] += m * x0[3 * p + k];
    }
    for (int k = 0; k < 3; ++k) c[k] /= M;
    body_mass[b] = M;
    for (int32_t p = body_off[b]; p < body_off[b + 1]; ++p)
      for (int k = 0; k < 3; ++k) rest[3 * p + k] = x0[3 * p + k] - c[k];
  }
}

/* cyclic Jacobi eigen-decomposition of a symmetric 3x3 S: S = V diag(lam) V^T,
 * V's columns are the eigenvectors */
static void sym_eig3(const double *S_in, double *lam, double *V) {
  double S[9];
  memcpy(S, S_in, sizeof(S));
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = S[1] * S[1] + S[2] * S[2] + S[5] * S[5];
    double diag = S[0] * S[0] + S[4] * S[4] + S[8] * S[8];
    if (off <= 1e-36 * diag || off == 0.0) break;
    for (int p = 0; p < 2; ++p) {
      for (int q = p + 1; q < 3; ++q) {
        double apq = S[3 * p + q];
        if (apq == 0.0) continue;
        double app = S[3 * p + p], aqq = S[3 * q + q];
        double theta = (aqq - app) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
        double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
        /* S <- J^T S J with J the rotation in the (p,q) plane */
        for (int k = 0; k < 3; ++k) { /* columns p,q */
          double skp = S[3 * k + p], skq = S[3 * k + q];
          S[3 * k + p] = c * skp - s * skq;
          S[3 * k + q] = s * skp + c * skq;
        }
        for (int k = 0; k < 3; ++k) { /* rows p,q */
          double spk = S[3 * p + k], sqk = S[3 * q + k];
          S[3 * p + k] = c * spk - s * sqk;
          S[3 * q + k] = s * spk + c * sqk;
        }
        for (int k = 0; k < 3; ++k) {
          double vkp = V[3 * k + p], vkq = V[3 * k + q];
          V[3 * k + p] = c * vkp - s * vkq;
          V[3 * k + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  for (int i = 0; i < 3; ++i) lam[i] = S[4 * i];
}

void orc_polar_rotation(const double *A, const double *Rprev, double *R) {
  double AtA[9], lam[3], V[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * k + i] * A[3 * k + j];
      AtA[3 * i + j] = s;
    }
  sym_eig3(AtA, lam, V);
  /* eigenpairs in descending order */
  int ord[3] = {0, 1, 2};
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (lam[ord[j]] > lam[ord[i]]) { int t = ord[i]; ord[i] = ord[j]; ord[j] = t; }
  double v[3][3], u[3][3], Av[3][3];
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) v[i][k] = V[3 * k + ord[i]];
  /* rank <= 1 (sigma_2 <= 1e-6 sigma_1, i.e. within the rounding of the
   * eigenvalues of A^T A): the rotation is not unique */
  if (!(lam[ord[0]] > 0.0) || !(lam[ord[1]] > 1e-12 * lam[ord[0]])) {
    memcpy(R, Rprev, 9 * sizeof(double));
    return;
  }
  /* right-handed V */
  double c12[3];
  cross3(v[0], v[1], c12);
  if (dot3(c12, v[2]) < 0) for (int k = 0; k < 3; ++k) v[2][k] = -v[2][k];
  for (int i = 0; i < 2; ++i)
    for (int r = 0; r < 3; ++r)
      Av[i][r] = A[3 * r + 0] * v[i][0] + A[3 * r + 1] * v[i][1] + A[3 * r + 2] * v[i][2];
  double n0 = norm3(Av[0]);
  for (int k = 0; k < 3; ++k) u[0][k] = Av[0][k] / n0;
  double pr = dot3(u[0], Av[1]);
  for (int k = 0; k < 3; ++k) u[1][k] = Av[1][k] - pr * u[0][k];
  double n1 = norm3(u[1]);
  for (int k = 0; k < 3; ++k) u[1][k] /= n1;
  cross3(u[0], u[1], u[2]);
  /* R = U V^T: the maximiser of tr(R^T A) over proper rotations */
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c)
      R[3 * r + c] = u[0][r] * v[0][c] + u[1][r] * v[1][c] + u[2][r] * v[2][c];
}

/* ------------------------------------------------------------------------ */
/* momentum conservation constraint (Sec. III-C)                             */
/* ------------------------------------------------------------------------ */

void orc_body_inertia(int32_t n, const double *x, const double *mass,
                      const double *c, double *I) {
  for (int i = 0; i < 9; ++i) I[i] = 0.0;
  for (int32_t p = 0; p < n; ++p) {
    double r[3] = {x[3 * p] - c[0], x[3 * p + 1] - c[1], x[3 * p + 2] - c[2]};
    double rr = dot3(r, r);
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        I[3 * i + j] += mass[p] * ((i == j ? rr : 0.0) - r[i] * r[j]);
  }
}

/* centre of mass, linear momentum P = sum m v and angular momentum
 * L = sum (x - c) x m v of one body state (Sec. III-C definitions) */
static void body_momenta(int32_t n, const double *mass, const double *x,
                         const double *v, double *c, double *P, double *L) {
  double M = 0.0;
  for (int k = 0; k < 3; ++k) c[k] = P[k] = L[k] = 0.0;
  for (int32_t p = 0; p < n; ++p) {
    M += mass[p];
    for (int k = 0; k < 3; ++k) c[k] += mass[p] * x[3 * p + k];
  }
  for (int k = 0; k < 3; ++k) c[k] /= M;
  for (int32_t p = 0; p < n; ++p) {
    double r[3] = {x[3 * p] - c[0], x[3 * p + 1] - c[1], x[3 * p + 2] - c[2]};
    double mv[3] = {mass[p] * v[3 * p], mass[p] * v[3 * p + 1], mass[p] * v[3 * p + 2]};
    double rxmv[3];
    cross3(r, mv, rxmv);
    for (int k = 0; k < 3; ++k) {
      P[k] += mv[k];
      L[k] += rxmv[k];
    }
  }
}

/* solve the 3x3 system I w = b by the adjugate; returns 0 if I is singular */
static int solve3(const double *I, const double *b, double *w) {
  double a = I[0], bb = I[1], c = I[2], d = I[3], e = I[4], f = I[5], g = I[6], h = I[7], k = I[8];
  double A00 = e * k - f * h, A01 = c * h - bb * k, A02 = bb * f - c * e;
  double A10 = f * g - d * k, A11 = a * k - c * g, A12 = c * d - a * f;
  double A20 = d * h - e * g, A21 = bb * g - a * h, A22 = a * e - bb * d;
  double det = a * A00 + bb * A10 + c * A20;
  double tr = (a + e + k) / 3.0;
  if (!(fabs(det) > 1e-12 * tr * tr * tr) || !(tr > 0.0)) {
    w[0] = w[1] = w[2] = 0.0;
    return 0;
  }
  w[0] = (A00 * b[0] + A01 * b[1] + A02 * b[2]) / det;
  w[1] = (A10 * b[0] + A11 * b[1] + A12 * b[2]) / det;
  w[2] = (A20 * b[0] + A21 * b[1] + A22 * b[2]) / det;
  return 1;
}

void orc_enforce_momentum(int32_t n, const double *mass, const double *xb,
                          const double *vb, const double *xa, const double *va,
                          double dt, uint32_t flags, double *x_out, double *v_out) {
  double cb[3], Pb[3], Lb[3], ca[3], Pa[3], La[3];
  double M = 0.0;
  for (int32_t p = 0; p < n; ++p) M += mass[p];
  body_momenta(n, mass, xb, vb, cb, Pb, Lb);
  body_momenta(n, mass, xa, va, ca, Pa, La);
  /* linear: sum m (v_asm + dv) = P_bsm  =>  dv = (P_bsm - P_asm)/M */
  double dv[3] = {0.0, 0.0, 0.0};
  if (!(flags & ORC_NO_LINMOM))
    for (int k = 0; k < 3; ++k) dv[k] = (Pb[k] - Pa[k]) / M;
  /* angular: L_asm - L_bsm = I w, I about c_asm from the post-shape-matching positions */
  double w[3] = {0.0, 0.0, 0.0};
  if (!(flags & ORC_NO_ANGMOM)) {
    double I[9], dL[3] = {La[0] - Lb[0], La[1] - Lb[1], La[2] - Lb[2]};
    orc_body_inertia(n, xa, mass, ca, I);
    solve3(I, dL, w);
  }
  for (int32_t p = 0; p < n; ++p) {
    double r[3] = {xa[3 * p] - ca[0], xa[3 * p + 1] - ca[1], xa[3 * p + 2] - ca[2]};
    double wxr[3];
    cross3(w, r, wxr);
    for (int k = 0; k < 3; ++k) {
      double corr = dv[k] - wxr[k];
      double xn = xa[3 * p + k] + corr * dt;
      double vn = va[3 * p + k] + corr;
      x_out[3 * p + k] = xn;
      v_out[3 * p + k] = vn;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* contacts (Sec. III-A constraints (1) and (2); contact step of Algorithm 1).  */
/* The paper gives no formulas; this is standard position-based contact with */
/* Coulomb friction: normal push-out by the penetration, friction removes    */
/* the tangential displacement of this substep up to mu times the            */
/* penetration (static = kinetic coefficient mu).                            */
/* ------------------------------------------------------------------------ */

static void ground_correction(const orc_scene *s, const double *x, const double *xi,
                              double *out) {
  const double *nrm = s->plane;
  double pen = s->radius - (dot3(nrm, x) - s->plane[3]);
  out[0] = out[1] = out[2] = 0.0;
  if (!(pen > 0.0)) return;
  double del[3] = {x[0] - xi[0], x[1] - xi[1], x[2] - xi[2]};
  double dn = dot3(del, nrm);
  double dtan[3] = {del[0] - dn * nrm[0], del[1] - dn * nrm[1], del[2] - dn * nrm[2]};
  double lt = norm3(dtan);
  double f = 0.0;
  if (lt > 0.0) f = fmin(s->friction * pen / lt, 1.0);
  for (int k = 0; k < 3; ++k) out[k] = pen * nrm[k] - f * dtan[k];
}

/* correction of particle p from its contact with q */
static int pair_correction(const orc_scene *s, int32_t p, int32_t q, const double *x,
                           const double *xi, double *out) {
  double diff[3] = {x[3 * p] - x[3 * q], x[3 * p + 1] - x[3 * q + 1], x[3 * p + 2] - x[3 * q + 2]};
  double d = norm3(diff);
  double r2 = 2.0 * s->radius;
  out[0] = out[1] = out[2] = 0.0;
  if (!(d > 0.0) || !(d < r2)) return 0;
  double pen = r2 - d;
  double nh[3] = {diff[0] / d, diff[1] / d, diff[2] / d};
  double sw = s->inv_mass[p] / (s->inv_mass[p] + s->inv_mass[q]);
  double del[3];
  for (int k = 0; k < 3; ++k)
    del[k] = (x[3 * p + k] - xi[3 * p + k]) - (x[3 * q + k] - xi[3 * q + k]);
  double dn = dot3(del, nh);
  double dtan[3] = {del[0] - dn * nh[0], del[1] - dn * nh[1], del[2] - dn * nh[2]};
  double lt = norm3(dtan);
  double f = 0.0;
  if (lt > 0.0) f = fmin(s->friction * pen / lt, 1.0);
  for (int k = 0; k < 3; ++k) out[k] = sw * (pen * nh[k] - f * dtan[k]);
  return 1;
}

/* ------------------------------------------------------------------------ */
/* one substep: Algorithm 1                                                  */
/* ------------------------------------------------------------------------ */

int orc_substep(const orc_scene *s, double *x, double *v, double *rot, int use_brute) {
  const int32_t N = s->num_particles, B = s->num_bodies;
  const double dt = s->dt;
  size_t n3 = (size_t)(N > 0 ? N : 1) * 3;
  double *xi = (double *)malloc(sizeof(double) * n3);   /* X_init */
  double *X = (double *)malloc(sizeof(double) * n3);    /* X_i */
  double *V = (double *)malloc(sizeof(double) * n3);    /* V_i */
  double *Xb = (double *)malloc(sizeof(double) * n3);   /* X_bsm */
  double *Vb = (double *)malloc(sizeof(double) * n3);   /* V_bsm */
  double *Xa = (double *)malloc(sizeof(double) * n3);   /* X_asm */
  double *Va = (double *)malloc(sizeof(double) * n3);   /* V_asm */
  double *mass = (double *)malloc(sizeof(double) * (size_t)(N > 0 ? N : 1));
  float *xf = (float *)malloc(sizeof(float) * n3);
  int32_t *body = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N > 0 ? N : 1));
  int32_t *off = (int32_t *)malloc(sizeof(int32_t) * (size_t)(N + 1));
  int64_t cap = (int64_t)N * 8 + 64;
  int32_t *nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
  if (!xi || !X || !V || !Xb || !Vb || !Xa || !Va || !mass || !xf || !body || !off || !nbr) {
    free(xi); free(X); free(V); free(Xb); free(Vb); free(Xa); free(Va);
    free(mass); free(xf); free(body); free(off); free(nbr);
    return -1;
  }
  for (int32_t p = 0; p < N; ++p) mass[p] = 1.0 / s->inv_mass[p];
  for (int32_t b = 0; b < B; ++b)
    for (int32_t p = s->body_off[b]; p < s->body_off[b + 1]; ++p) body[p] = b;

  /* integration step (integration step of Algorithm 1): v~ = v_init + dt w f_ext(x),
   * x~ = x_init + dt v~.  Gravity gives w m g = g.  A constant force F at the
   * CoM gives every particle F/M; a constant torque tau gives the rigid angular
   * acceleration alpha = I^-1 tau, i.e. alpha x (x_init - c), with c and I of
   * the substep's initial positions. */
  memcpy(xi, x, sizeof(double) * 3 * (size_t)N);
  for (int32_t b = 0; b < B; ++b) {
    int32_t p0 = s->body_off[b], nb = s->body_off[b + 1] - p0;
    double aF[3] = {0.0, 0.0, 0.0}, alpha[3] = {0.0, 0.0, 0.0}, c[3] = {0.0, 0.0, 0.0};
    if (s->force)
      for (int k = 0; k < 3; ++k) aF[k] = s->force[3 * b + k] / s->body_mass[b];
    if (s->torque) {
      double M = 0.0;
      for (int32_t p = p0; p < p0 + nb; ++p) {
        M += mass[p];
        for (int k = 0; k < 3; ++k) c[k] += mass[p] * xi[3 * p + k];
      }
      for (int k = 0; k < 3; ++k) c[k] /= M;
      double I[9];
      orc_body_inertia(nb, xi + 3 * p0, mass + p0, c, I);
      solve3(I, s->torque + 3 * b, alpha);
    }
    for (int32_t p = p0; p < p0 + nb; ++p) {
      double r[3] = {xi[3 * p] - c[0], xi[3 * p + 1] - c[1], xi[3 * p + 2] - c[2]};
      double axr[3];
      cross3(alpha, r, axr);
      for (int k = 0; k < 3; ++k) {
        double a = s->gravity[k] + aF[k] + axr[k];
        V[3 * p + k] = v[3 * p + k] + dt * a;
        X[3 * p + k] = xi[3 * p + k] + dt * V[3 * p + k];
      }
    }
  }

  /* neighbour candidates on the predicted positions, FP32 predicate */
  float Rn, Rn2, h, inv_h;
  orc_nbr_constants((float)s->radius, &Rn, &Rn2, &h, &inv_h);
  for (size_t k = 0; k < 3 * (size_t)N; ++k) xf[k] = (float)X[k];
  for (;;) {
    int64_t need = use_brute ? orc_neighbors_brute(N, xf, body, Rn2, off, nbr, cap)
                             : orc_neighbors_grid(N, xf, body, Rn2, inv_h, off, nbr, cap);
    if (need <= cap) break;
    free(nbr);
    cap = need;
    nbr = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
    if (!nbr) {
      free(xi); free(X); free(V); free(Xb); free(Vb); free(Xa); free(Va);
      free(mass); free(xf); free(body); free(off);
      return -1;
    }
  }

  /* solver iterations (solver loop of Algorithm 1) */
  for (int32_t it = 0; it < s->iterations; ++it) {
    /* contacts from X_i (Jacobi): dX_PG + dX_PP */
    for (int32_t p = 0; p < N; ++p) {
      double dpg[3], dpp[3] = {0.0, 0.0, 0.0}, t[3];
      ground_correction(s, X + 3 * p, xi + 3 * p, dpg);
      int active = 0;
      for (int32_t k = off[p]; k < off[p + 1]; ++k) {
        if (pair_correction(s, p, nbr[k], X, xi, t)) {
          active++;
          for (int j = 0; j < 3; ++j) dpp[j] += t[j];
        }
      }
      if ((s->flags & ORC_CONTACT_AVG) && active > 0)
        for (int j = 0; j < 3; ++j) dpp[j] /= (double)active;
      for (int j = 0; j < 3; ++j) {
        double dc = dpg[j] + dpp[j];
        Xb[3 * p + j] = X[3 * p + j] + dc;
        if (s->flags & ORC_STD_VELOCITY)
          Vb[3 * p + j] = (Xb[3 * p + j] - xi[3 * p + j]) / dt;
        else
          Vb[3 * p + j] = V[3 * p + j] + dc / dt;   /* V_i + dX/dt (Sec. III-B) */
      }
    }
    /* shape matching per body on X_bsm (or X_i), then momentum enforcement */
    for (int32_t b = 0; b < B; ++b) {
      int32_t p0 = s->body_off[b], nb = s->body_off[b + 1] - p0;
      const double *src = (s->flags & ORC_SM_FROM_XI) ? X : Xb;
      double M = s->body_mass[b], c[3] = {0.0, 0.0, 0.0}, A[9] = {0};
      for (int32_t p = p0; p < p0 + nb; ++p)
        for (int k = 0; k < 3; ++k) c[k] += mass[p] * src[3 * p + k];
      for (int k = 0; k < 3; ++k) c[k] /= M;
      for (int32_t p = p0; p < p0 + nb; ++p)
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            A[3 * i + j] += mass[p] * (src[3 * p + i] - c[i]) * s->rest[3 * p + j];
      double R[9];
      orc_polar_rotation(A, rot + 9 * b, R);
      memcpy(rot + 9 * b, R, sizeof(R));
      for (int32_t p = p0; p < p0 + nb; ++p) {
        const double *q = s->rest + 3 * p;
        for (int i = 0; i < 3; ++i) {
          double goal = R[3 * i] * q[0] + R[3 * i + 1] * q[1] + R[3 * i + 2] * q[2] + c[i];
          double dsm = goal - src[3 * p + i];
          Xa[3 * p + i] = Xb[3 * p + i] + dsm;
          if (s->flags & ORC_STD_VELOCITY)
            Va[3 * p + i] = (Xa[3 * p + i] - xi[3 * p + i]) / dt;
          else
            Va[3 * p + i] = Vb[3 * p + i] + dsm / dt;
        }
      }
      orc_enforce_momentum(nb, mass + p0, Xb + 3 * p0, Vb + 3 * p0, Xa + 3 * p0,
                           Va + 3 * p0, dt, s->flags, X + 3 * p0, V + 3 * p0);
    }
  }
  memcpy(x, X, sizeof(double) * 3 * (size_t)N);
  memcpy(v, V, sizeof(double) * 3 * (size_t)N);
  free(xi); free(X); free(V); free(Xb); free(Vb); free(Xa); free(Va);
  free(mass); free(xf); free(body); free(off); free(nbr);
  return 0;
}
