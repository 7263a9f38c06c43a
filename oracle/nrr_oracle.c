/*
 * nrr_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).
 *
 * What it computes, and where the paper states it (arXiv 2501.14030):
 *   - the Hamiltonian constraint for the non-singular part u of the conformal
 *     factor, lap(u) + (1/8) A~_ij A~^ij (psi_singular + u)^-7 = 0   (Sec. 2)
 *   - the hyperbolic relaxation system du/dt = v - eta u,
 *     dv/dt = c^2 [lap(u) + source]                                   (Sec. 2)
 *   - wave speed proportional to the local grid spacing under the CFL limit,
 *     on SinhSymTP coordinates                                        (Sec. 2)
 *   - the driver order RHS -> BC -> RK substep, residual H and its L2 norm
 *     with a stop test                                                (Alg. 1)
 *   - centred finite differences of selectable order                  (Sec. 4)
 * The paper defers the coordinate map, the Bowen-York curvature, the
 * boundary conditions, eta, c and the norm to its predecessor; the readings
 * used here are listed in the repository design notes and restated at each
 * function below.
 *
 * Style: straight loops over padded grid functions, no blocking, no fusion.
 * OpenMP pragmas only parallelise independent per-point loops; every
 * reduction is sequential so results do not depend on the thread count.
 */
#include "nrr_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_PI 3.14159265358979323846

struct or_grid {
  or_desc d;
  int ng, s[3];
  long npts;
  double xxmin[3], dxx[3];
  double dsmin_global;
  double *xx[3];                 /* per point coordinate values            */
  double *x, *y, *z, *r;         /* Cartesian position and radius          */
  double *h[3];                  /* orthogonal scale factors               */
  double *gl[3];                 /* (1/J) d_i (J / h_i^2)                  */
  double *jac;                   /* J = h0 h1 h2                           */
  double *dsmin, *c;             /* local spacing and wave speed           */
  double *drdxx0;                /* dr/dxx0 at fixed xx1, xx2              */
  int *kind, *image;
  double w1[13], w2[13];         /* FD weights, offset k stored at k+ng    */
};

/* ------------------------------------------------------------------------ */
/* Finite-difference weights: Fornberg's recursion (Math. Comp. 51, 1988),  */
/* written out for nodes x_j = -m..m about z = 0.  c[j][k] is the weight of */
/* node j for the k-th derivative using nodes 0..i.                         */
/* ------------------------------------------------------------------------ */
int or_fd_weights(int order, int deriv, double *w) {
  if (order < 2 || order > 12 || (order & 1) || deriv < 0 || deriv > 2)
    return -1;
  int m = order / 2, n = order; /* n+1 nodes */
  double xs[13], c[13][3];
  for (int j = 0; j <= n; j++) {
    xs[j] = (double)(j - m);
    for (int k = 0; k < 3; k++) c[j][k] = 0.0;
  }
  double z = 0.0;
  double c1 = 1.0, c4 = xs[0] - z;
  c[0][0] = 1.0;
  for (int i = 1; i <= n; i++) {
    int mn = i < deriv ? i : deriv;
    double c2 = 1.0, c5 = c4;
    c4 = xs[i] - z;
    for (int j = 0; j < i; j++) {
      double c3 = xs[i] - xs[j];
      c2 *= c3;
      if (j == i - 1) {
        for (int k = mn; k >= 1; k--)
          c[i][k] = c1 * (k * c[i - 1][k - 1] - c5 * c[i - 1][k]) / c2;
        c[i][0] = -c1 * c5 * c[i - 1][0] / c2;
      }
      for (int k = mn; k >= 1; k--)
        c[j][k] = (c4 * c[j][k] - k * c[j][k - 1]) / c3;
      c[j][0] = c4 * c[j][0] / c3;
    }
    c1 = c2;
  }
  for (int j = 0; j <= n; j++) w[j] = c[j][deriv];
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Coordinate maps.  SinhSymTP (named in Sec. 2; map from its predecessor): */
/*   A(xx0) = AMAX sinh(xx0/w)/sinh(1/w), Z = sqrt(A^2 + b^2),              */
/*   x = A sin(th) cos(ph), y = A sin(th) sin(ph), z = Z cos(th).           */
/* Spherical: xx0 = r.  Cartesian: identity.                                */
/* ------------------------------------------------------------------------ */
typedef struct {
  double x, y, z, r;
  double h[3], gl[3];
  double drdxx0;
} point_geom;

static void geom_sinhsymtp(const or_desc *d, double x0, double x1, double x2,
                           point_geom *o) {
  double w = d->sinhwaa, b = d->bscale;
  double A = d->amax * sinh(x0 / w) / sinh(1.0 / w);
  double Ap = d->amax * cosh(x0 / w) / (w * sinh(1.0 / w));
  double App = d->amax * sinh(x0 / w) / (w * w * sinh(1.0 / w));
  double st = sin(x1), ct = cos(x1);
  double Z = sqrt(A * A + b * b);
  double V1 = sqrt(A * A + b * b * st * st);
  o->x = A * st * cos(x2);
  o->y = A * st * sin(x2);
  o->z = Z * ct;
  o->r = sqrt(o->x * o->x + o->y * o->y + o->z * o->z);
  /* |d(x,y,z)/d xx_i| */
  o->h[0] = Ap * V1 / Z;
  o->h[1] = V1;
  o->h[2] = A * st;
  /* (1/J) d_i (J/h_i^2) with J = h0 h1 h2, derived by hand:
   *   J/h0^2 = A Z sin(th)/A',  J/h1^2 = A A' sin(th)/Z,  J/h2^2 indep. of ph */
  o->gl[0] = (Z * Z + A * A - A * Z * Z * App / (Ap * Ap)) / (Ap * A * V1 * V1);
  o->gl[1] = ct / (st * V1 * V1);
  o->gl[2] = 0.0;
  /* r^2 = A^2 + b^2 cos^2(th)  =>  dr/dxx0 = A A'/r */
  o->drdxx0 = A * Ap / o->r;
}

static void geom_spherical(double x0, double x1, double x2, point_geom *o) {
  double st = sin(x1), ct = cos(x1);
  o->x = x0 * st * cos(x2);
  o->y = x0 * st * sin(x2);
  o->z = x0 * ct;
  o->r = fabs(x0);
  o->h[0] = 1.0;
  o->h[1] = x0;
  o->h[2] = x0 * st;
  o->gl[0] = 2.0 / x0;
  o->gl[1] = ct / (x0 * x0 * st);
  o->gl[2] = 0.0;
  o->drdxx0 = 1.0;
}

/* SinhSpherical: spherical coordinates with r = AMAX sinh(xx0/w)/sinh(1/w)
 * (xx0 in [0,1]).  h = (r', r, r sin th); with J = r' r^2 sin th,
 *   J/h0^2 = r^2 sin th / r'  =>  g0 = 2/(r r') - r''/r'^3,
 *   J/h1^2 = r' sin th        =>  g1 = cot th / r^2.                        */
static void geom_sinhspherical(const or_desc *d, double x0, double x1,
                               double x2, point_geom *o) {
  double w = d->sinhwaa;
  double r = d->amax * sinh(x0 / w) / sinh(1.0 / w);
  double rp = d->amax * cosh(x0 / w) / (w * sinh(1.0 / w));
  double rpp = r / (w * w);
  double st = sin(x1), ct = cos(x1);
  o->x = r * st * cos(x2);
  o->y = r * st * sin(x2);
  o->z = r * ct;
  o->r = fabs(r);
  o->h[0] = rp;
  o->h[1] = r;
  o->h[2] = r * st;
  o->gl[0] = 2.0 / (r * rp) - rpp / (rp * rp * rp);
  o->gl[1] = ct / (r * r * st);
  o->gl[2] = 0.0;
  o->drdxx0 = rp;
}

/* SinhCylindrical, stored as (rho, z, ph) so that the periodic direction is
 * the third: rho = AMAX sinh(xx0/w)/sinh(1/w) (xx0 in [0,1]),
 * z = ZMAX sinh(xx1/wz)/sinh(1/wz) (xx1 in [-1,1]), ph = xx2;
 * x = rho cos ph, y = rho sin ph.  h = (rho', z', rho); with
 * J = rho' z' rho,
 *   J/h0^2 = z' rho / rho'  =>  g0 = 1/(rho rho') - rho''/rho'^3,
 *   J/h1^2 = rho' rho / z'  =>  g1 = -z''/z'^3,
 *   J/h2^2 independent of ph => g2 = 0.                                    */
static void geom_sinhcylindrical(const or_desc *d, double x0, double x1,
                                 double x2, point_geom *o) {
  double w = d->sinhwaa, wz = d->sinhwz;
  double rho = d->amax * sinh(x0 / w) / sinh(1.0 / w);
  double rhop = d->amax * cosh(x0 / w) / (w * sinh(1.0 / w));
  double rhopp = rho / (w * w);
  double z = d->zmax * sinh(x1 / wz) / sinh(1.0 / wz);
  double zp = d->zmax * cosh(x1 / wz) / (wz * sinh(1.0 / wz));
  double zpp = z / (wz * wz);
  o->x = rho * cos(x2);
  o->y = rho * sin(x2);
  o->z = z;
  o->r = sqrt(rho * rho + z * z);
  o->h[0] = rhop;
  o->h[1] = zp;
  o->h[2] = rho;
  o->gl[0] = 1.0 / (rho * rhop) - rhopp / (rhop * rhop * rhop);
  o->gl[1] = -zpp / (zp * zp * zp);
  o->gl[2] = 0.0;
  o->drdxx0 = rhop;  /* d rho / d xx0; the radiation condition uses both */
}

static void geom_cartesian(double x0, double x1, double x2, point_geom *o) {
  o->x = x0;
  o->y = x1;
  o->z = x2;
  o->r = sqrt(x0 * x0 + x1 * x1 + x2 * x2);
  for (int i = 0; i < 3; i++) {
    o->h[i] = 1.0;
    o->gl[i] = 0.0;
  }
  o->drdxx0 = 0.0;
}

static void geom_at(const or_desc *d, double x0, double x1, double x2,
                    point_geom *o) {
  if (d->coord == OR_SINHSYMTP)
    geom_sinhsymtp(d, x0, x1, x2, o);
  else if (d->coord == OR_SPHERICAL)
    geom_spherical(x0, x1, x2, o);
  else if (d->coord == OR_SINHSPHERICAL)
    geom_sinhspherical(d, x0, x1, x2, o);
  else if (d->coord == OR_SINHCYLINDRICAL)
    geom_sinhcylindrical(d, x0, x1, x2, o);
  else
    geom_cartesian(x0, x1, x2, o);
}

/* Inverse map to the canonical domain (xx0 >= 0, th in [0,pi], ph in
 * [-pi,pi)).  Used only to locate inner-boundary images. */
static void cart_to_xx(const or_desc *d, double x, double y, double z,
                       double xx[3]) {
  double rho2 = x * x + y * y, rho = sqrt(rho2);
  xx[2] = atan2(y, x);
  if (d->coord == OR_SINHSYMTP) {
    double b = d->bscale, w = d->sinhwaa;
    /* A^2 solves X^2 - q X - rho^2 b^2 = 0, q = rho^2 + z^2 - b^2. */
    double q = rho2 + z * z - b * b;
    double disc = sqrt(q * q + 4.0 * rho2 * b * b);
    double A2 = q >= 0.0 ? 0.5 * (q + disc) : 2.0 * rho2 * b * b / (disc - q);
    double A = sqrt(A2), Z = sqrt(A2 + b * b);
    xx[0] = w * asinh(A * sinh(1.0 / w) / d->amax);
    xx[1] = atan2(rho * Z, z * A);
  } else if (d->coord == OR_SINHSPHERICAL) {
    double w = d->sinhwaa;
    xx[0] = w * asinh(sqrt(rho2 + z * z) * sinh(1.0 / w) / d->amax);
    xx[1] = atan2(rho, z);
  } else if (d->coord == OR_SINHCYLINDRICAL) {
    xx[0] = d->sinhwaa * asinh(rho * sinh(1.0 / d->sinhwaa) / d->amax);
    xx[1] = d->sinhwz * asinh(z * sinh(1.0 / d->sinhwz) / d->zmax);
  } else {
    xx[0] = sqrt(rho2 + z * z);
    xx[1] = atan2(rho, z);
  }
}

static void grid_dims(const or_desc *d, double xxmin[3], double xxmax[3]) {
  if (d->coord == OR_CARTESIAN) {
    for (int i = 0; i < 3; i++) {
      xxmin[i] = -d->xmax;
      xxmax[i] = d->xmax;
    }
    return;
  }
  xxmin[0] = 0.0;
  xxmax[0] = (d->coord == OR_SINHSYMTP || d->coord == OR_SINHSPHERICAL ||
              d->coord == OR_SINHCYLINDRICAL) ? 1.0 : d->rmax;
  xxmin[1] = 0.0;
  xxmax[1] = OR_PI;
  if (d->coord == OR_SINHCYLINDRICAL) {
    xxmin[1] = -1.0;
    xxmax[1] = 1.0;
  }
  xxmin[2] = -OR_PI;
  xxmax[2] = OR_PI;
}

static long pidx(const or_grid *g, int i0, int i1, int i2) {
  return (long)i0 + (long)g->s[0] * ((long)i1 + (long)g->s[1] * (long)i2);
}

static int in_interior(const or_grid *g, int i, int dir) {
  return i >= g->ng && i < g->ng + g->d.n[dir];
}

void or_grid_free(or_grid *g) {
  if (!g) return;
  double *arrs[] = {g->xx[0], g->xx[1], g->xx[2], g->x,  g->y,     g->z,
                    g->r,     g->h[0],  g->h[1],  g->h[2], g->gl[0], g->gl[1],
                    g->gl[2], g->jac,   g->dsmin, g->c,    g->drdxx0};
  for (size_t i = 0; i < sizeof(arrs) / sizeof(arrs[0]); i++) free(arrs[i]);
  free(g->kind);
  free(g->image);
  free(g);
}

or_grid *or_grid_new(const or_desc *d, char *err, int errlen) {
#define FAIL(...)                                   \
  do {                                              \
    if (err) snprintf(err, (size_t)errlen, __VA_ARGS__); \
    or_grid_free(g);                                \
    return NULL;                                    \
  } while (0)
  or_grid *g = (or_grid *)calloc(1, sizeof(or_grid));
  if (!g) return NULL;
  g->d = *d;
  if (d->order < 2 || d->order > 12 || (d->order & 1))
    FAIL("unsupported FD order %d", d->order);
  if (d->coord < OR_SINHSYMTP || d->coord > OR_SINHCYLINDRICAL)
    FAIL("unknown coordinate system %d", d->coord);
  if (d->coord == OR_SINHCYLINDRICAL &&
      !(d->amax > 0 && d->sinhwaa > 0 && d->zmax > 0 && d->sinhwz > 0))
    FAIL("SinhCylindrical needs amax, sinhwaa, zmax, sinhwz > 0");
  g->ng = d->order / 2;
  for (int i = 0; i < 3; i++) {
    if (d->n[i] < 1) FAIL("n[%d] must be positive", i);
    g->s[i] = d->n[i] + 2 * g->ng;
  }
  if (d->coord != OR_CARTESIAN && (d->n[2] & 1))
    FAIL("n2 must be even for the ph -> ph + pi image");
  g->npts = (long)g->s[0] * g->s[1] * g->s[2];
  double xxmax[3];
  grid_dims(d, g->xxmin, xxmax);
  for (int i = 0; i < 3; i++) g->dxx[i] = (xxmax[i] - g->xxmin[i]) / d->n[i];
  or_fd_weights(d->order, 1, g->w1);
  or_fd_weights(d->order, 2, g->w2);

  long n = g->npts;
  double **arrs[] = {&g->xx[0], &g->xx[1], &g->xx[2], &g->x,  &g->y,
                     &g->z,     &g->r,     &g->h[0],  &g->h[1], &g->h[2],
                     &g->gl[0], &g->gl[1], &g->gl[2], &g->jac, &g->dsmin,
                     &g->c,     &g->drdxx0};
  for (size_t i = 0; i < sizeof(arrs) / sizeof(arrs[0]); i++) {
    *arrs[i] = (double *)calloc((size_t)n, sizeof(double));
    if (!*arrs[i]) FAIL("out of memory");
  }
  g->kind = (int *)calloc((size_t)n, sizeof(int));
  g->image = (int *)calloc((size_t)n, sizeof(int));
  if (!g->kind || !g->image) FAIL("out of memory");

  /* Geometry at every padded point. */
  for (int i2 = 0; i2 < g->s[2]; i2++)
    for (int i1 = 0; i1 < g->s[1]; i1++)
      for (int i0 = 0; i0 < g->s[0]; i0++) {
        long p = pidx(g, i0, i1, i2);
        int ii[3] = {i0, i1, i2};
        double xx[3];
        for (int k = 0; k < 3; k++) {
          xx[k] = g->xxmin[k] + ((double)(ii[k] - g->ng) + 0.5) * g->dxx[k];
          g->xx[k][p] = xx[k];
        }
        point_geom pg;
        geom_at(d, xx[0], xx[1], xx[2], &pg);
        g->x[p] = pg.x;
        g->y[p] = pg.y;
        g->z[p] = pg.z;
        g->r[p] = pg.r;
        double ds = INFINITY;
        for (int k = 0; k < 3; k++) {
          g->h[k][p] = pg.h[k];
          g->gl[k][p] = pg.gl[k];
          double dsk = fabs(pg.h[k]) * g->dxx[k];
          if (dsk < ds) ds = dsk;
        }
        g->jac[p] = pg.h[0] * pg.h[1] * pg.h[2];
        g->dsmin[p] = ds;
        g->drdxx0[p] = pg.drdxx0;
        /* Classification: interior; outer ghost (evolved by the radiation
         * condition); inner ghost (a copy of its image point). */
        int inside = in_interior(g, i0, 0) && in_interior(g, i1, 1) &&
                     in_interior(g, i2, 2);
        if (inside)
          g->kind[p] = OR_INTERIOR;
        else if (d->coord == OR_CARTESIAN)
          g->kind[p] = OR_OUTER;
        else if (d->coord == OR_SINHCYLINDRICAL)
          /* rho < 0 and ph outside [-pi, pi) are images; every other
           * ghost lies beyond the cylinder's side or its ends */
          g->kind[p] = (i0 >= g->ng && in_interior(g, i2, 2)) ? OR_OUTER
                                                               : OR_INNER;
        else if (i0 >= g->ng + d->n[0] && in_interior(g, i1, 1) &&
                 in_interior(g, i2, 2))
          g->kind[p] = OR_OUTER;
        else
          g->kind[p] = OR_INNER;
        g->image[p] = (int)p;
      }

  /* Smallest spacing over the interior sets the time step; the wave speed is
   * the local spacing in units of it (Sec. 2: c proportional to the local
   * grid spacing, CFL satisfied everywhere). */
  g->dsmin_global = INFINITY;
  for (long p = 0; p < n; p++)
    if (g->kind[p] == OR_INTERIOR && g->dsmin[p] < g->dsmin_global)
      g->dsmin_global = g->dsmin[p];
  for (long p = 0; p < n; p++) g->c[p] = g->dsmin[p] / g->dsmin_global;

  /* Inner-boundary images by Cartesian matching: map the ghost's Cartesian
   * position back into the canonical coordinate domain, take the nearest
   * grid index and require that point's Cartesian position to agree. */
  for (long p = 0; p < n; p++) {
    if (g->kind[p] != OR_INNER) continue;
    double xx[3];
    cart_to_xx(d, g->x[p], g->y[p], g->z[p], xx);
    int ii[3];
    for (int k = 0; k < 3; k++) {
      double f = (xx[k] - g->xxmin[k]) / g->dxx[k] - 0.5;
      double fr = floor(f + 0.5);
      if (fabs(f - fr) > 1e-6)
        FAIL("ghost %ld: coordinate %d not on the grid (%.9f)", p, k, f);
      int k_int = (int)fr;
      if (k == 2) k_int = ((k_int % d->n[2]) + d->n[2]) % d->n[2];
      ii[k] = k_int + g->ng;
    }
    /* (a SinhCylindrical image may lie beyond the ends in z: i1 spans the
     * padded range there) */
    int i1_ok = d->coord == OR_SINHCYLINDRICAL ? (ii[1] >= 0 && ii[1] < g->s[1])
                                               : in_interior(g, ii[1], 1);
    if (ii[0] < g->ng || ii[0] >= g->s[0] || !i1_ok || !in_interior(g, ii[2], 2))
      FAIL("ghost %ld: image index out of range", p);
    long q = pidx(g, ii[0], ii[1], ii[2]);
    double scale = 1.0 + g->r[p];
    double dist = fabs(g->x[q] - g->x[p]) + fabs(g->y[q] - g->y[p]) +
                  fabs(g->z[q] - g->z[p]);
    if (dist > 1e-9 * scale)
      FAIL("ghost %ld: image Cartesian mismatch %.3e", p, dist);
    if (g->kind[q] == OR_INNER) FAIL("ghost %ld: image is itself a ghost", p);
    g->image[p] = (int)q;
  }
  return g;
#undef FAIL
}

void or_grid_info(const or_grid *g, int *ints, double *dbls) {
  ints[0] = g->ng;
  ints[1] = g->s[0];
  ints[2] = g->s[1];
  ints[3] = g->s[2];
  ints[4] = (int)g->npts;
  for (int k = 0; k < 3; k++) {
    dbls[k] = g->xxmin[k];
    dbls[3 + k] = g->dxx[k];
  }
  dbls[6] = g->dsmin_global;
}

void *or_grid_field(or_grid *g, const char *name) {
  static const char *names[] = {"xx0", "xx1", "xx2", "x",  "y",  "z",
                                "r",   "h0",  "h1",  "h2", "g0", "g1",
                                "g2",  "jac", "dsmin", "c", "drdxx0"};
  double *ptrs[] = {g->xx[0], g->xx[1], g->xx[2], g->x,     g->y,
                    g->z,     g->r,     g->h[0],  g->h[1],  g->h[2],
                    g->gl[0], g->gl[1], g->gl[2], g->jac,   g->dsmin,
                    g->c,     g->drdxx0};
  for (size_t i = 0; i < sizeof(names) / sizeof(names[0]); i++)
    if (!strcmp(name, names[i])) return ptrs[i];
  if (!strcmp(name, "kind")) return g->kind;
  if (!strcmp(name, "image")) return g->image;
  return NULL;
}

/* ------------------------------------------------------------------------ */
/* Source: Brandt-Bruegmann punctures (Sec. 2).  Conformal trace-free       */
/* curvature of Bowen-York form, per puncture a with n = (x - x_a)/r_a:     */
/*  A^ij = 3/(2 r^2) [P^i n^j + P^j n^i - (delta^ij - n^i n^j) P.n]         */
/*       + 3/r^3 [(S x n)^i n^j + (S x n)^j n^i]                            */
/* summed over punctures; aa = sum_ij (A^ij)^2 in Cartesian components;     */
/* psi_singular = 1 + sum_a m_a / (2 r_a).                                  */
/* ------------------------------------------------------------------------ */
void or_bowen_york(int np, const or_puncture *p, const double *x, double *aa,
                   double *psi_s) {
  double A[3][3] = {{0.0}};
  double psi = 1.0;
  for (int a = 0; a < np; a++) {
    double dx[3], r2 = 0.0;
    for (int i = 0; i < 3; i++) {
      dx[i] = x[i] - p[a].x[i];
      r2 += dx[i] * dx[i];
    }
    double r = sqrt(r2);
    double nn[3] = {dx[0] / r, dx[1] / r, dx[2] / r};
    double Pn = p[a].P[0] * nn[0] + p[a].P[1] * nn[1] + p[a].P[2] * nn[2];
    double Sxn[3] = {p[a].S[1] * nn[2] - p[a].S[2] * nn[1],
                     p[a].S[2] * nn[0] - p[a].S[0] * nn[2],
                     p[a].S[0] * nn[1] - p[a].S[1] * nn[0]};
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) {
        double delta = (i == j) ? 1.0 : 0.0;
        double momentum = 1.5 / (r * r) *
                          (p[a].P[i] * nn[j] + p[a].P[j] * nn[i] -
                           (delta - nn[i] * nn[j]) * Pn);
        double spin = 3.0 / (r * r * r) * (Sxn[i] * nn[j] + Sxn[j] * nn[i]);
        A[i][j] += momentum + spin;
      }
    psi += p[a].m / (2.0 * r);
  }
  double s = 0.0;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) s += A[i][j] * A[i][j];
  *aa = s;
  *psi_s = psi;
}

/* (1/8) aa (psi_s + u)^-7 = beta (1 + alpha u)^-7 with alpha = 1/psi_s and
 * beta = aa alpha^7 / 8: the same term, regular at the punctures. */
int or_source(const or_grid *g, int np, const or_puncture *p, double *alpha,
              double *beta) {
  for (long q = 0; q < g->npts; q++) {
    double x[3] = {g->x[q], g->y[q], g->z[q]}, aa, psi_s;
    or_bowen_york(np, p, x, &aa, &psi_s);
    alpha[q] = 1.0 / psi_s;
    beta[q] = 0.125 * aa * pow(alpha[q], 7.0);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Flat Laplacian in orthogonal coordinates (Sec. 2, the hat-nabla^2 term): */
/*   lap u = sum_i [ h_i^-2 d_i^2 u + (1/J) d_i(J/h_i^2) d_i u ]            */
/* with centred differences of the grid's order, at interior points.        */
/* ------------------------------------------------------------------------ */
static double laplacian_at(const or_grid *g, const double *u, int i0, int i1,
                           int i2) {
  long p = pidx(g, i0, i1, i2);
  long stride[3] = {1, g->s[0], (long)g->s[0] * g->s[1]};
  double lap = 0.0;
  for (int dir = 0; dir < 3; dir++) {
    double d1 = 0.0, d2 = 0.0;
    for (int k = -g->ng; k <= g->ng; k++) {
      double f = u[p + k * stride[dir]];
      d1 += g->w1[k + g->ng] * f;
      d2 += g->w2[k + g->ng] * f;
    }
    d1 /= g->dxx[dir];
    d2 /= g->dxx[dir] * g->dxx[dir];
    double hh = g->h[dir][p];
    lap += d2 / (hh * hh) + g->gl[dir][p] * d1;
  }
  return lap;
}

void or_laplacian(const or_grid *g, const double *u, double *lap) {
#pragma omp parallel for collapse(2)
  for (int i2 = 0; i2 < g->s[2]; i2++)
    for (int i1 = 0; i1 < g->s[1]; i1++)
      for (int i0 = 0; i0 < g->s[0]; i0++) {
        long p = pidx(g, i0, i1, i2);
        lap[p] = g->kind[p] == OR_INTERIOR ? laplacian_at(g, u, i0, i1, i2)
                                           : 0.0;
      }
}

void or_fill_inner_ghosts(const or_grid *g, double *f) {
  for (long p = 0; p < g->npts; p++)
    if (g->kind[p] == OR_INNER) f[p] = f[g->image[p]];
}

/* Radiation (Sommerfeld) condition with zero asymptotic value at an outer
 * ghost: df/dt = -c (d_r f + f/r).  Curvilinear: d_r f from the second-order
 * backward difference along xx0 over dr/dxx0.  Cartesian: d_r f =
 * sum_i (x^i/r) D_i f, one-sided inward along directions in which the point
 * lies outside, centred otherwise. */
static double radiation_df(const or_grid *g, const double *f, int i0, int i1,
                           int i2) {
  long p = pidx(g, i0, i1, i2);
  if (g->d.coord == OR_SINHCYLINDRICAL) {
    /* d_r f = (rho/r) d_rho f + (z/r) d_z f with d_rho = (1/rho') d_xx0 and
     * d_z = (1/z') d_xx1; each difference one-sided inward where the point
     * lies beyond that direction's outer boundary, centred otherwise (an
     * xx0 neighbour at rho < 0 is an inner ghost, filled from its image). */
    int ii[2] = {i0, i1};
    long stride[2] = {1, g->s[0]};
    double scale[2] = {g->x[p] * cos(g->xx[2][p]) + g->y[p] * sin(g->xx[2][p]),
                       g->z[p]};  /* rho and z */
    double dr = 0.0;
    for (int dir = 0; dir < 2; dir++) {
      long st = stride[dir];
      double D;
      if (ii[dir] >= g->ng + g->d.n[dir])
        D = (3.0 * f[p] - 4.0 * f[p - st] + f[p - 2 * st]) / (2.0 * g->dxx[dir]);
      else if (ii[dir] < g->ng)
        D = -(3.0 * f[p] - 4.0 * f[p + st] + f[p + 2 * st]) / (2.0 * g->dxx[dir]);
      else
        D = (f[p + st] - f[p - st]) / (2.0 * g->dxx[dir]);
      dr += scale[dir] / g->r[p] * D / g->h[dir][p];
    }
    return dr + f[p] / g->r[p];
  }
  if (g->d.coord != OR_CARTESIAN) {
    double db = (3.0 * f[p] - 4.0 * f[p - 1] + f[p - 2]) / (2.0 * g->dxx[0]);
    return db / g->drdxx0[p] + f[p] / g->r[p];
  }
  int ii[3] = {i0, i1, i2};
  long stride[3] = {1, g->s[0], (long)g->s[0] * g->s[1]};
  double pos[3] = {g->x[p], g->y[p], g->z[p]};
  double dr = 0.0;
  for (int dir = 0; dir < 3; dir++) {
    long st = stride[dir];
    double D;
    if (ii[dir] >= g->ng + g->d.n[dir])
      D = (3.0 * f[p] - 4.0 * f[p - st] + f[p - 2 * st]) / (2.0 * g->dxx[dir]);
    else if (ii[dir] < g->ng)
      D = -(3.0 * f[p] - 4.0 * f[p + st] + f[p + 2 * st]) / (2.0 * g->dxx[dir]);
    else
      D = (f[p + st] - f[p - st]) / (2.0 * g->dxx[dir]);
    dr += pos[dir] / g->r[p] * D;
  }
  return dr + f[p] / g->r[p];
}

/* Right-hand side of the relaxation system (Sec. 2) followed by the
 * boundary conditions on it (Alg. 1: RHS, then BC): interior points first,
 * outer ghosts by the radiation condition, inner ghosts copy their image. */
void or_rhs(const or_grid *g, const double *alpha, const double *beta,
            double eta, const double *u, const double *v, double *ku,
            double *kv) {
#pragma omp parallel for collapse(2)
  for (int i2 = 0; i2 < g->s[2]; i2++)
    for (int i1 = 0; i1 < g->s[1]; i1++)
      for (int i0 = 0; i0 < g->s[0]; i0++) {
        long p = pidx(g, i0, i1, i2);
        if (g->kind[p] == OR_INTERIOR) {
          double lap = laplacian_at(g, u, i0, i1, i2);
          double src = beta[p] * pow(1.0 + alpha[p] * u[p], -7.0);
          ku[p] = v[p] - eta * u[p];
          kv[p] = g->c[p] * g->c[p] * (lap + src);
        } else if (g->kind[p] == OR_OUTER) {
          ku[p] = -g->c[p] * radiation_df(g, u, i0, i1, i2);
          kv[p] = -g->c[p] * radiation_df(g, v, i0, i1, i2);
        }
      }
  for (long p = 0; p < g->npts; p++)
    if (g->kind[p] == OR_INNER) {
      ku[p] = ku[g->image[p]];
      kv[p] = kv[g->image[p]];
    }
}

/* a = -d/du of the source term beta (1 + alpha u)^-7, i.e.
 * 7 alpha beta (1 + alpha u)^-8, at every point. */
void or_linear_coefficient(const or_grid *g, const double *alpha,
                           const double *beta, const double *u, double *a) {
  for (long p = 0; p < g->npts; p++)
    a[p] = 7.0 * alpha[p] * beta[p] * pow(1.0 + alpha[p] * u[p], -8.0);
}

/* Right-hand side of the relaxation system of the correction equation with
 * the same boundary handling as or_rhs. */
void or_linear_rhs(const or_grid *g, const double *a, const double *rhat,
                   double eta, const double *d, const double *w, double *kd,
                   double *kw) {
#pragma omp parallel for collapse(2)
  for (int i2 = 0; i2 < g->s[2]; i2++)
    for (int i1 = 0; i1 < g->s[1]; i1++)
      for (int i0 = 0; i0 < g->s[0]; i0++) {
        long p = pidx(g, i0, i1, i2);
        if (g->kind[p] == OR_INTERIOR) {
          double lap = laplacian_at(g, d, i0, i1, i2);
          kd[p] = w[p] - eta * d[p];
          kw[p] = g->c[p] * g->c[p] * (lap - a[p] * d[p] + rhat[p]);
        } else if (g->kind[p] == OR_OUTER) {
          kd[p] = -g->c[p] * radiation_df(g, d, i0, i1, i2);
          kw[p] = -g->c[p] * radiation_df(g, w, i0, i1, i2);
        }
      }
  for (long p = 0; p < g->npts; p++)
    if (g->kind[p] == OR_INNER) {
      kd[p] = kd[g->image[p]];
      kw[p] = kw[g->image[p]];
    }
}

/* Classical RK4 (method of lines), the substep loop of Alg. 1. */
void or_rk4_step(const or_grid *g, const double *alpha, const double *beta,
                 double eta, double dt, double *u, double *v) {
  long n = g->npts;
  double *buf = (double *)malloc(sizeof(double) * (size_t)n * 10);
  double *ku[4], *kv[4], *us = buf + 8 * n, *vs = buf + 9 * n;
  for (int s = 0; s < 4; s++) {
    ku[s] = buf + (2 * s) * n;
    kv[s] = buf + (2 * s + 1) * n;
  }
  static const double a[4] = {0.0, 0.5, 0.5, 1.0};
  for (int s = 0; s < 4; s++) {
    const double *uin = u, *vin = v;
    if (s > 0) {
      for (long p = 0; p < n; p++) {
        us[p] = u[p] + a[s] * dt * ku[s - 1][p];
        vs[p] = v[p] + a[s] * dt * kv[s - 1][p];
      }
      uin = us;
      vin = vs;
    }
    or_rhs(g, alpha, beta, eta, uin, vin, ku[s], kv[s]);
  }
  for (long p = 0; p < n; p++) {
    u[p] += dt / 6.0 * (ku[0][p] + 2.0 * ku[1][p] + 2.0 * ku[2][p] + ku[3][p]);
    v[p] += dt / 6.0 * (kv[0][p] + 2.0 * kv[1][p] + 2.0 * kv[2][p] + kv[3][p]);
  }
  free(buf);
}

/* Residual H: left-hand side of the Hamiltonian constraint (Sec. 2, Alg. 1
 * "H"), at interior points; zero elsewhere. */
void or_residual(const or_grid *g, const double *alpha, const double *beta,
                 const double *u, double *H) {
#pragma omp parallel for collapse(2)
  for (int i2 = 0; i2 < g->s[2]; i2++)
    for (int i1 = 0; i1 < g->s[1]; i1++)
      for (int i0 = 0; i0 < g->s[0]; i0++) {
        long p = pidx(g, i0, i1, i2);
        if (g->kind[p] != OR_INTERIOR) {
          H[p] = 0.0;
          continue;
        }
        double lap = laplacian_at(g, u, i0, i1, i2);
        H[p] = lap + beta[p] * pow(1.0 + alpha[p] * u[p], -7.0);
      }
}

/* L2 norm of H (Alg. 1): volume-weighted mean over interior points inside
 * r < r_int, with the reference-metric volume element J dxx0 dxx1 dxx2
 * (the constant cell volume cancels in the ratio). */
double or_residual_norm(const or_grid *g, const double *H, double r_int) {
  double num = 0.0, den = 0.0;
  for (long p = 0; p < g->npts; p++) {
    if (g->kind[p] != OR_INTERIOR || !(g->r[p] < r_int)) continue;
    double w = fabs(g->jac[p]);
    num += H[p] * H[p] * w;
    den += w;
  }
  return den > 0.0 ? sqrt(num / den) : 0.0;
}

/* The relaxation loop of Alg. 1: evaluate H and its norm every check_every
 * steps (and before the first), stop below tol, otherwise take RK4 steps. */
int or_relax(const or_grid *g, const double *alpha, const double *beta,
             const or_relax_params *prm, double *u, double *v,
             or_relax_result *res) {
  double *H = (double *)malloc(sizeof(double) * (size_t)g->npts);
  if (!H) return -1;
  or_fill_inner_ghosts(g, u);
  or_fill_inner_ghosts(g, v);
  long it = 0;
  int every = prm->check_every > 0 ? prm->check_every : 1;
  res->status = OR_NOT_CONVERGED;
  for (;;) {
    if (it % every == 0) {
      or_residual(g, alpha, beta, u, H);
      double nrm = or_residual_norm(g, H, prm->r_int);
      res->norm = nrm;
      if (!isfinite(nrm)) {
        res->status = OR_DIVERGED;
        break;
      }
      if (nrm < prm->tol) {
        res->status = OR_CONVERGED;
        break;
      }
    }
    if (it >= prm->max_iters) break;
    or_rk4_step(g, alpha, beta, prm->eta, prm->dt, u, v);
    it++;
  }
  res->iters = it;
  free(H);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Brute force on tiny grids: Newton's method for the discrete steady state */
/* (every padded point is an unknown): interior H = 0; outer ghosts         */
/* d_r u + u/r = 0 (the radiation condition at rest); inner ghosts          */
/* u - u_image = 0.  Dense Jacobian, LU with partial pivoting.              */
/* ------------------------------------------------------------------------ */
static int lu_solve(double *Am, double *b, int n) {
  for (int k = 0; k < n; k++) {
    int piv = k;
    double best = fabs(Am[(long)k * n + k]);
    for (int i = k + 1; i < n; i++)
      if (fabs(Am[(long)i * n + k]) > best) {
        best = fabs(Am[(long)i * n + k]);
        piv = i;
      }
    if (best == 0.0) return -1;
    if (piv != k) {
      for (int j = 0; j < n; j++) {
        double t = Am[(long)k * n + j];
        Am[(long)k * n + j] = Am[(long)piv * n + j];
        Am[(long)piv * n + j] = t;
      }
      double t = b[k];
      b[k] = b[piv];
      b[piv] = t;
    }
    double inv = 1.0 / Am[(long)k * n + k];
    for (int i = k + 1; i < n; i++) {
      double f = Am[(long)i * n + k] * inv;
      if (f == 0.0) continue;
      Am[(long)i * n + k] = 0.0;
      for (int j = k + 1; j < n; j++) Am[(long)i * n + j] -= f * Am[(long)k * n + j];
      b[i] -= f * b[k];
    }
  }
  for (int i = n - 1; i >= 0; i--) {
    double s = b[i];
    for (int j = i + 1; j < n; j++) s -= Am[(long)i * n + j] * b[j];
    b[i] = s / Am[(long)i * n + i];
  }
  return 0;
}

int or_newton(const or_grid *g, const double *alpha, const double *beta,
              double *u, int max_it, double step_tol, double *final_step) {
  int n = (int)g->npts;
  if (g->npts > 6000) return -2;
  double *J = (double *)malloc(sizeof(double) * (size_t)n * (size_t)n);
  double *F = (double *)malloc(sizeof(double) * (size_t)n);
  if (!J || !F) {
    free(J);
    free(F);
    return -1;
  }
  long stride[3] = {1, g->s[0], (long)g->s[0] * g->s[1]};
  double step = INFINITY;
  int it;
  for (it = 0; it < max_it; it++) {
    memset(J, 0, sizeof(double) * (size_t)n * (size_t)n);
    for (int i2 = 0; i2 < g->s[2]; i2++)
      for (int i1 = 0; i1 < g->s[1]; i1++)
        for (int i0 = 0; i0 < g->s[0]; i0++) {
          long p = pidx(g, i0, i1, i2);
          double *row = J + p * (long)n;
          if (g->kind[p] == OR_INTERIOR) {
            double lap = laplacian_at(g, u, i0, i1, i2);
            double base = 1.0 + alpha[p] * u[p];
            F[p] = lap + beta[p] * pow(base, -7.0);
            for (int dir = 0; dir < 3; dir++) {
              double hh = g->h[dir][p];
              for (int k = -g->ng; k <= g->ng; k++) {
                double wgt = g->w2[k + g->ng] /
                                 (g->dxx[dir] * g->dxx[dir] * hh * hh) +
                             g->gl[dir][p] * g->w1[k + g->ng] / g->dxx[dir];
                row[p + k * stride[dir]] += wgt;
              }
            }
            row[p] += -7.0 * alpha[p] * beta[p] * pow(base, -8.0);
          } else if (g->kind[p] == OR_OUTER) {
            F[p] = radiation_df(g, u, i0, i1, i2);
            /* radiation_df is linear in f: differentiate by probing it with
             * unit vectors on its (at most 7-point) support. */
            long supp[7];
            int ns = 0;
            supp[ns++] = p;
            if (g->d.coord != OR_CARTESIAN &&
                g->d.coord != OR_SINHCYLINDRICAL) {
              supp[ns++] = p - 1;
              supp[ns++] = p - 2;
            } else {
              int ii[3] = {i0, i1, i2};
              int ndir = g->d.coord == OR_CARTESIAN ? 3 : 2;
              for (int dir = 0; dir < ndir; dir++) {
                long st = stride[dir];
                if (ii[dir] >= g->ng + g->d.n[dir]) {
                  supp[ns++] = p - st;
                  supp[ns++] = p - 2 * st;
                } else if (ii[dir] < g->ng) {
                  supp[ns++] = p + st;
                  supp[ns++] = p + 2 * st;
                } else {
                  supp[ns++] = p + st;
                  supp[ns++] = p - st;
                }
              }
            }
            double *e = (double *)calloc((size_t)n, sizeof(double));
            for (int s = 0; s < ns; s++) {
              e[supp[s]] = 1.0;
              row[supp[s]] = radiation_df(g, e, i0, i1, i2);
              e[supp[s]] = 0.0;
            }
            free(e);
          } else {
            F[p] = u[p] - u[g->image[p]];
            row[p] += 1.0;
            row[g->image[p]] += -1.0;
          }
        }
    for (int p = 0; p < n; p++) F[p] = -F[p];
    if (lu_solve(J, F, n) != 0) {
      free(J);
      free(F);
      return -3;
    }
    double umax = 0.0;
    step = 0.0;
    for (int p = 0; p < n; p++) {
      u[p] += F[p];
      if (fabs(F[p]) > step) step = fabs(F[p]);
      if (fabs(u[p]) > umax) umax = fabs(u[p]);
    }
    if (step <= step_tol * (umax > 0.0 ? umax : 1.0)) {
      it++;
      break;
    }
  }
  if (final_step) *final_step = step;
  free(J);
  free(F);
  return it;
}

void or_grid_set_speed_reference(or_grid *g, double ds_ref) {
  g->dsmin_global = ds_ref;
  for (long p = 0; p < g->npts; p++) g->c[p] = g->dsmin[p] / ds_ref;
}

/* ------------------------------------------------------------------------ */
/* Two overlapping patches (Sec. 5: several patches of one solve; Sec. 6:   */
/* multipatch grids with interpolation between patches).                    */
/* ------------------------------------------------------------------------ */
struct or_link {
  long n;       /* receivers                                              */
  int q;        /* interpolation points per direction                     */
  long *recv;   /* receiver flat index in the receiving patch             */
  long *donor;  /* [n][q^3] donor flat indices (images of inner ghosts)   */
  double *w;    /* [n][q^3] products of the three Lagrange weights        */
};

void or_link_free(or_link *l) {
  if (!l) return;
  free(l->recv);
  free(l->donor);
  free(l->w);
  free(l);
}

long or_link_count(const or_link *l) { return l->n; }

void or_link_get(const or_link *l, long *recv, long *donor, double *w) {
  long m = (long)l->q * l->q * l->q;
  memcpy(recv, l->recv, sizeof(long) * (size_t)l->n);
  memcpy(donor, l->donor, sizeof(long) * (size_t)(l->n * m));
  memcpy(w, l->w, sizeof(double) * (size_t)(l->n * m));
}

/* Lagrange weights of the q nodes base, base+1, ... at position f (all in
 * units of the grid index): w_j = prod_{m != j} (f - t_m) / (t_j - t_m). */
static void lagrange_weights(int q, int base, double f, double *w) {
  for (int j = 0; j < q; j++) {
    double num = 1.0, den = 1.0;
    for (int m = 0; m < q; m++) {
      if (m == j) continue;
      num *= f - (double)(base + m);
      den *= (double)(j - m);
    }
    w[j] = num / den;
  }
}

or_link *or_link_new(const or_grid *rg, const or_grid *dg, int kind,
                     double hole, int q, char *err, int errlen) {
#define LFAIL(...)                                       \
  do {                                                   \
    if (err) snprintf(err, (size_t)errlen, __VA_ARGS__); \
    or_link_free(l);                                     \
    return NULL;                                         \
  } while (0)
  or_link *l = (or_link *)calloc(1, sizeof(or_link));
  if (!l) return NULL;
  if (q < 2 || q > 6 || (q & 1)) LFAIL("q must be 2, 4 or 6");
  if (q / 2 > dg->ng) LFAIL("q/2 exceeds the donor's ghost width");
  if (kind == 0 && rg->d.coord != OR_CARTESIAN)
    LFAIL("ghost receivers need a Cartesian receiving patch");
  if (kind != 0 && kind != 1) LFAIL("unknown receiver kind");
  long m = (long)q * q * q;
  long n = 0;
  for (long p = 0; p < rg->npts; p++) {
    int take = kind == 0 ? rg->kind[p] == OR_OUTER
                         : rg->kind[p] == OR_INTERIOR &&
                               fmax(fabs(rg->x[p]), fmax(fabs(rg->y[p]), fabs(rg->z[p]))) < hole;
    n += take;
  }
  l->n = n;
  l->q = q;
  l->recv = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n : 1));
  l->donor = (long *)malloc(sizeof(long) * (size_t)(n > 0 ? n * m : 1));
  l->w = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n * m : 1));
  if (!l->recv || !l->donor || !l->w) LFAIL("out of memory");
  long r = 0;
  for (long p = 0; p < rg->npts; p++) {
    int take = kind == 0 ? rg->kind[p] == OR_OUTER
                         : rg->kind[p] == OR_INTERIOR &&
                               fmax(fabs(rg->x[p]), fmax(fabs(rg->y[p]), fabs(rg->z[p]))) < hole;
    if (!take) continue;
    /* the receiver's position in the donor's coordinates, as a fractional
     * padded index (cell centre i at i) */
    double xx[3];
    if (dg->d.coord == OR_CARTESIAN) {
      xx[0] = rg->x[p];
      xx[1] = rg->y[p];
      xx[2] = rg->z[p];
    } else {
      cart_to_xx(&dg->d, rg->x[p], rg->y[p], rg->z[p], xx);
    }
    int base[3];
    double wd[3][6];
    for (int d = 0; d < 3; d++) {
      double f = (xx[d] - dg->xxmin[d]) / dg->dxx[d] - 0.5 + dg->ng;
      base[d] = (int)floor(f) - (q / 2 - 1);
      if (base[d] < 0 || base[d] + q - 1 >= dg->s[d])
        LFAIL("receiver %ld: donor stencil leaves the donor (direction %d)", p, d);
      lagrange_weights(q, base[d], f, wd[d]);
    }
    long k = 0;
    for (int c = 0; c < q; c++)
      for (int b = 0; b < q; b++)
        for (int a = 0; a < q; a++, k++) {
          long dp = pidx(dg, base[0] + a, base[1] + b, base[2] + c);
          if (dg->kind[dp] == OR_INNER) dp = dg->image[dp];
          l->donor[r * m + k] = dp;
          l->w[r * m + k] = wd[0][a] * wd[1][b] * wd[2][c];
        }
    l->recv[r++] = p;
  }
  return l;
#undef LFAIL
}

void or_link_apply(const or_link *l, const double *f_donor, double *f_recv) {
  long m = (long)l->q * l->q * l->q;
  for (long r = 0; r < l->n; r++) {
    double s = 0.0;
    for (long k = 0; k < m; k++) s += l->w[r * m + k] * f_donor[l->donor[r * m + k]];
    f_recv[l->recv[r]] = s;
  }
}

int or_link_conflict(const or_link *l, const or_link *other) {
  long m = (long)other->q * other->q * other->q;
  for (long r = 0; r < l->n; r++)
    for (long k = 0; k < other->n * m; k++)
      if (other->donor[k] == l->recv[r]) return 1;
  return 0;
}

void or_patch_rk4_step(const or_grid *a, const double *alpha_a,
                       const double *beta_a, const or_grid *b,
                       const double *alpha_b, const double *beta_b,
                       const or_link *la, const or_link *lb, double eta,
                       double dt, double *ua, double *va, double *ub,
                       double *vb) {
  const or_grid *gs[2] = {a, b};
  const double *al[2] = {alpha_a, alpha_b}, *be[2] = {beta_a, beta_b};
  double *u[2] = {ua, ub}, *v[2] = {va, vb};
  double *ku[2][4], *kv[2][4], *us[2], *vs[2];
  for (int i = 0; i < 2; i++) {
    long n = gs[i]->npts;
    double *buf = (double *)malloc(sizeof(double) * (size_t)n * 10);
    for (int s = 0; s < 4; s++) {
      ku[i][s] = buf + (2 * s) * n;
      kv[i][s] = buf + (2 * s + 1) * n;
    }
    us[i] = buf + 8 * n;
    vs[i] = buf + 9 * n;
  }
  static const double c[4] = {0.0, 0.5, 0.5, 1.0};
  for (int s = 0; s < 4; s++) {
    for (int i = 0; i < 2; i++) {
      const double *uin = u[i], *vin = v[i];
      if (s > 0) {
        for (long p = 0; p < gs[i]->npts; p++) {
          us[i][p] = u[i][p] + c[s] * dt * ku[i][s - 1][p];
          vs[i][p] = v[i][p] + c[s] * dt * kv[i][s - 1][p];
        }
        uin = us[i];
        vin = vs[i];
      }
      or_rhs(gs[i], al[i], be[i], eta, uin, vin, ku[i][s], kv[i][s]);
    }
    /* receivers of a from b, receivers of b from a, then the inner ghosts
     * again (a receiver may be the image of an inner ghost) */
    or_link_apply(la, ku[1][s], ku[0][s]);
    or_link_apply(la, kv[1][s], kv[0][s]);
    or_link_apply(lb, ku[0][s], ku[1][s]);
    or_link_apply(lb, kv[0][s], kv[1][s]);
    for (int i = 0; i < 2; i++) {
      or_fill_inner_ghosts(gs[i], ku[i][s]);
      or_fill_inner_ghosts(gs[i], kv[i][s]);
    }
  }
  for (int i = 0; i < 2; i++) {
    for (long p = 0; p < gs[i]->npts; p++) {
      u[i][p] += dt / 6.0 * (ku[i][0][p] + 2.0 * ku[i][1][p] + 2.0 * ku[i][2][p] + ku[i][3][p]);
      v[i][p] += dt / 6.0 * (kv[i][0][p] + 2.0 * kv[i][1][p] + 2.0 * kv[i][2][p] + kv[i][3][p]);
    }
    free(ku[i][0]);
  }
}

double or_patch_norm(const or_grid *a, const double *Ha, const or_link *la,
                     const or_grid *b, const double *Hb, const or_link *lb,
                     double r_int) {
  const or_grid *gs[2] = {a, b};
  const double *H[2] = {Ha, Hb};
  const or_link *ls[2] = {la, lb};
  double num = 0.0, den = 0.0;
  for (int i = 0; i < 2; i++) {
    char *recv = (char *)calloc((size_t)gs[i]->npts, 1);
    for (long r = 0; r < ls[i]->n; r++) recv[ls[i]->recv[r]] = 1;
    for (long p = 0; p < gs[i]->npts; p++) {
      if (gs[i]->kind[p] != OR_INTERIOR || recv[p] || !(gs[i]->r[p] < r_int)) continue;
      double w = fabs(gs[i]->jac[p]);
      num += H[i][p] * H[i][p] * w;
      den += w;
    }
    free(recv);
  }
  return den > 0.0 ? sqrt(num / den) : 0.0;
}

int or_patch_relax(const or_grid *a, const double *alpha_a,
                   const double *beta_a, const or_grid *b,
                   const double *alpha_b, const double *beta_b,
                   const or_link *la, const or_link *lb,
                   const or_relax_params *prm, double *ua, double *va,
                   double *ub, double *vb, or_relax_result *res) {
  double *Ha = (double *)malloc(sizeof(double) * (size_t)a->npts);
  double *Hb = (double *)malloc(sizeof(double) * (size_t)b->npts);
  if (!Ha || !Hb) {
    free(Ha);
    free(Hb);
    return -1;
  }
  long it = 0;
  int every = prm->check_every > 0 ? prm->check_every : 1;
  res->status = OR_NOT_CONVERGED;
  for (;;) {
    if (it % every == 0) {
      or_residual(a, alpha_a, beta_a, ua, Ha);
      or_residual(b, alpha_b, beta_b, ub, Hb);
      double nrm = or_patch_norm(a, Ha, la, b, Hb, lb, prm->r_int);
      res->norm = nrm;
      if (!isfinite(nrm)) {
        res->status = OR_DIVERGED;
        break;
      }
      if (nrm < prm->tol) {
        res->status = OR_CONVERGED;
        break;
      }
    }
    if (it >= prm->max_iters) break;
    or_patch_rk4_step(a, alpha_a, beta_a, b, alpha_b, beta_b, la, lb, prm->eta,
                      prm->dt, ua, va, ub, vb);
    it++;
  }
  res->iters = it;
  free(Ha);
  free(Hb);
  return 0;
}
