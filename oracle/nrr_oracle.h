/*
 * nrr_oracle.h -- plain FP64 CPU oracle for the hyperbolic-relaxation solve of
 * the binary-black-hole puncture Hamiltonian constraint (arXiv 2501.14030,
 * Sec. 2, Eqs. for u and for the relaxation system; Alg. 1).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the independent checker of the
 * CUDA path.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
 * leg may load it.  It shares no code, header, table or constant generator
 * with the CUDA library; neither includes the other.
 *
 * Every array is a padded 3-D grid function of s0*s1*s2 doubles, index
 * p = i0 + s0*(i1 + s1*i2), i0 fastest, s_d = n_d + 2*ng, ng = order/2.
 * Cell-centred sampling: xx_d[i] = xxmin_d + (i - ng + 1/2) * dxx_d.
 */
#ifndef NRR_ORACLE_H
#define NRR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_SINHSYMTP = 0, OR_SPHERICAL = 1, OR_CARTESIAN = 2, OR_SINHSPHERICAL = 3,
       OR_SINHCYLINDRICAL = 4 };
enum { OR_INTERIOR = 0, OR_OUTER = 1, OR_INNER = 2 };
enum { OR_CONVERGED = 0, OR_NOT_CONVERGED = 1, OR_DIVERGED = 2 };

typedef struct {
  int coord;       /* OR_SINHSYMTP / OR_SPHERICAL / OR_CARTESIAN /
                      OR_SINHSPHERICAL / OR_SINHCYLINDRICAL            */
  int n[3];        /* interior points per direction                      */
  int order;       /* centred finite-difference order: 2,4,6,8,10,12     */
  double amax;     /* SinhSymTP / SinhSpherical outer extent; SinhCylindrical
                      outer cylindrical radius                            */
  double bscale;   /* SinhSymTP focal half-distance                       */
  double sinhwaa;  /* sinh width of xx0                                   */
  double rmax;     /* Spherical outer radius                              */
  double xmax;     /* Cartesian half-width                                */
  double zmax;     /* SinhCylindrical half-height                         */
  double sinhwz;   /* SinhCylindrical sinh width of xx1 (the z direction) */
} or_desc;

typedef struct {
  double m;        /* bare mass                                           */
  double x[3];     /* position                                            */
  double P[3];     /* linear momentum                                     */
  double S[3];     /* spin angular momentum                               */
} or_puncture;

typedef struct {
  double eta;      /* damping factor of the relaxation system             */
  double dt;       /* time step                                           */
  double tol;      /* stop when the residual norm falls below this       */
  double r_int;    /* radius of the norm's integration region             */
  long max_iters;  /* RK4 steps allowed                                   */
  int check_every; /* residual is evaluated every this many steps         */
} or_relax_params;

typedef struct {
  long iters;
  double norm;
  int status;      /* OR_CONVERGED / OR_NOT_CONVERGED / OR_DIVERGED       */
} or_relax_result;

typedef struct or_grid or_grid;

/* Geometry: coordinates, scale factors, Laplacian coefficients, wave speed,
 * ghost classification and the inner-boundary image of every inner ghost,
 * found by matching Cartesian coordinates.  NULL on error (message in err). */
or_grid *or_grid_new(const or_desc *d, char *err, int errlen);
void or_grid_free(or_grid *g);
/* ints: ng, s0, s1, s2, npts(low 31 bits); dbls: xxmin[3], dxx[3], dsmin_global */
void or_grid_info(const or_grid *g, int *ints, double *dbls);
/* Named per-point arrays: "x","y","z","r","h0","h1","h2","g0","g1","g2",
 * "jac","dsmin","c","drdxx0","xx0","xx1","xx2" (doubles); "kind","image"
 * (ints).  Returns NULL for an unknown name. */
void *or_grid_field(or_grid *g, const char *name);

/* Centred FD weights at offsets -order/2..order/2 for derivative `deriv`. */
int or_fd_weights(int order, int deriv, double *w);

/* Bowen-York conformal extrinsic curvature contraction and psi_singular at x. */
void or_bowen_york(int np, const or_puncture *p, const double *x,
                   double *aa, double *psi_s);
/* alpha = 1/psi_s and beta = aa * alpha^7 / 8 at every padded point. */
int or_source(const or_grid *g, int np, const or_puncture *p,
              double *alpha, double *beta);

void or_fill_inner_ghosts(const or_grid *g, double *f);
void or_laplacian(const or_grid *g, const double *u, double *lap);
void or_rhs(const or_grid *g, const double *alpha, const double *beta,
            double eta, const double *u, const double *v,
            double *ku, double *kv);
void or_rk4_step(const or_grid *g, const double *alpha, const double *beta,
                 double eta, double dt, double *u, double *v);
void or_residual(const or_grid *g, const double *alpha, const double *beta,
                 const double *u, double *H);
double or_residual_norm(const or_grid *g, const double *H, double r_int);
int or_relax(const or_grid *g, const double *alpha, const double *beta,
             const or_relax_params *prm, double *u, double *v,
             or_relax_result *res);

/* Defect correction (FP32 relaxation inside an FP64 outer loop): the
 * linearisation of H at u, H(u + d) ~ H(u) + lap(d) - a d, with
 * a = 7 alpha beta (1 + alpha u)^-8, and the relaxation system of the
 * correction equation lap(d) - a d + rhat = 0:
 *   dd/dt = w - eta d,  dw/dt = c^2 [lap(d) - a d + rhat]
 * with the same boundary conditions as (u, v). */
void or_linear_coefficient(const or_grid *g, const double *alpha,
                           const double *beta, const double *u, double *a);
void or_linear_rhs(const or_grid *g, const double *a, const double *rhat,
                   double eta, const double *d, const double *w,
                   double *kd, double *kw);

/* Newton's method with a dense LU on the discrete steady-state system. */
int or_newton(const or_grid *g, const double *alpha, const double *beta,
              double *u, int max_it, double step_tol, double *final_step);

/* Wave speed reference of a patch that is part of a multi-patch system:
 * c = (local spacing) / ds_ref, with ds_ref the smallest spacing over all
 * patches, so that one time step dt = cfl ds_ref runs every patch at the
 * same Courant number (Sec. 2: c proportional to the local spacing). */
void or_grid_set_speed_reference(or_grid *g, double ds_ref);

/* Two overlapping patches (Sec. 5 multiple patches; Sec. 6 multipatch
 * grids): values at the receiver points of one patch are interpolated from
 * a donor patch by tensor-product Lagrange interpolation of q points per
 * direction in the donor's coordinates xx.  Receivers: kind 0 = every ghost
 * point of a Cartesian patch (the inner box's boundary); kind 1 = interior
 * points of the patch with max(|x|,|y|,|z|) < hole (the outer patch's hole
 * inside the box).  Donor points are evolved points of the donor (inner
 * ghosts replaced by their images).  NULL on error (message in err). */
typedef struct or_link or_link;
or_link *or_link_new(const or_grid *recv, const or_grid *donor, int kind,
                     double hole, int q, char *err, int errlen);
void or_link_free(or_link *l);
long or_link_count(const or_link *l);
/* receiver flat indices (n), donor flat indices (n*q^3), weights (n*q^3) */
void or_link_get(const or_link *l, long *recv, long *donor, double *w);
/* f_recv[r] = sum_j w[r][j] f_donor[donor[r][j]] at every receiver. */
void or_link_apply(const or_link *l, const double *f_donor, double *f_recv);
/* 1 if a receiver of `l` is a donor point of `other` (the coupling would
 * then read interpolated values to interpolate), else 0. */
int or_link_conflict(const or_link *l, const or_link *other);

/* One RK4 step of the two-patch system: each stage evaluates both patches'
 * right-hand sides with their boundary conditions, then sets the
 * right-hand side at the receivers of each link from the donor's (la: the
 * receivers of patch a, donor b; lb the converse), then the inner ghosts
 * of both copy their images again. */
void or_patch_rk4_step(const or_grid *a, const double *alpha_a,
                       const double *beta_a, const or_grid *b,
                       const double *alpha_b, const double *beta_b,
                       const or_link *la, const or_link *lb, double eta,
                       double dt, double *ua, double *va, double *ub,
                       double *vb);
/* Norm of the two-patch residual: sqrt((sum H^2 J over the interior points
 * of both patches with r < r_int that are not receivers) / (sum J)). */
double or_patch_norm(const or_grid *a, const double *Ha, const or_link *la,
                     const or_grid *b, const double *Hb, const or_link *lb,
                     double r_int);
/* The relaxation loop of Alg. 1 on the two-patch system (norm every
 * check_every steps and before the first). */
int or_patch_relax(const or_grid *a, const double *alpha_a,
                   const double *beta_a, const or_grid *b,
                   const double *alpha_b, const double *beta_b,
                   const or_link *la, const or_link *lb,
                   const or_relax_params *prm, double *ua, double *va,
                   double *ub, double *vb, or_relax_result *res);

#ifdef __cplusplus
}
#endif
#endif
