// nrr_internal.h -- device buffers of one grid and the kernel launchers that
// the C-ABI layer (nrr_api.cu) drives.
#pragma once

#include <cuda_runtime.h>

#include "../../include/nrr.h"
#include "nrr_common.cuh"

namespace nrr {

// Sets the calling thread's message returned by nrr_last_error().
void set_last_error(const char *msg);

// The one check of a grid descriptor that every entry point taking one
// uses: known coordinates, FD order 4/8/10, sizes (curvilinear: even n2,
// n0 and n1 >= fd_order/2; Cartesian: n >= 2; each n <= 65536 and the
// padded plane s0*s1 below 2^31, computed in 64 bits) and positive map
// parameters.  NRR_OK, or NRR_ERR_INVALID_ARG with nrr_last_error() set.
nrr_status check_grid_desc(const nrr_grid_desc *d);
// Padded sizes, coordinate ranges and spacings of a checked descriptor.
Geo grid_geo(const nrr_grid_desc *d);

// The driver's cuTensorMapEncodeTiled (as a plain pointer), or null.
void *tensor_map_encoder();

// Stage kinds of the fused RK4 stage kernel (classical RK4: k1..k4 with
// weights 1/6, 1/3, 1/3, 1/6 and stage offsets 1/2, 1/2, 1):
//   FIRST: acc = y + b dt k;  out = y + a dt k        (input state: y)
//   MID:   acc += b dt k;     out = y + a dt k        (input: stage state)
//   LAST:  out = acc + b dt k                         (out is y's buffer)
//   RAW:   out = k                                    (one RHS evaluation)
enum StageKind { STAGE_FIRST = 0, STAGE_MID = 1, STAGE_LAST = 2, STAGE_RAW = 3 };

// Number of folded stencil coefficients per column: one centre weight, ng
// forward and ng backward weights in xx0 and xx1, ng symmetric weights in xx2.
inline int ncoef(int ng) { return 5 * ng + 1; }

// Per-column arrays of a curvilinear grid in one precision.
template <typename R>
struct ColumnSet {
  R *coef = nullptr;   // [ncoef][ncol] c^2-scaled Laplacian weights
  R *somm = nullptr;   // [3][ncol]: c, 1/(2 dxx0 dr/dxx0), 1/r; SinhCylindrical
                       // [4][ncol]: c, rho/(2 dxx0 r rho'), 1/r, z/(2 dxx1 r z')
  R *c2inv = nullptr;  // [ncol] 1/c^2
};

// Grid functions of one precision: RK4 state y, two stage states s/t, the
// accumulator a (each u and v), and the constant sources alpha and
// c^2 beta.
template <typename R>
struct FieldSet {
  R *y[2] = {nullptr, nullptr};
  R *s[2] = {nullptr, nullptr};
  R *t[2] = {nullptr, nullptr};
  R *a[2] = {nullptr, nullptr};
  R *alpha = nullptr;
  R *bc2 = nullptr;
  R *fu = nullptr;  // forcing of the u equation (linear mode only)
  int lin = 0;      // 1: increment equation of the defect correction, with
                    // (alpha, bc2, fu) = (c^2 a, f_v, f_u)
};

struct LaunchCfg {
  int block = 128;  // threads per block (Cartesian and residual kernels)
  int zc = 2;       // curvilinear stages: phi planes per thread (variant 0)
                    // or per block chunk (variant 1)
  int variant = 0;  // curvilinear stages: 0 column kernel, 1 tiled kernel,
                    // 2 persistent column kernel, 3 tensor-copy tiled
                    // kernel, 4 multi-stage cooperative kernel, 5 its
                    // tensor-copy tiled form, 6 two stages per launch
                    // (FP32, small SinhSymTP grids); Cartesian
                    // stages: 0 column kernel, 1 tensor-copy tiled kernel
  int pdl = 1;      // stage kernels: programmatic dependent launch (the next
                    // stage's blocks start while this one drains)
};

// Cartesian grids use constant coefficients (uniform spacing, so the wave
// speed c = spacing / reference spacing is one constant: 1 on its own, other
// values in a multi-patch system).  c^2 is folded into the weights.
struct CartCoef {
  double cc;          // centre weight, all three directions
  double a[3][6];     // a[dir][k] for k = 1..ng, symmetric
  double speed;       // c, multiplies the radiation condition
};

// ----------------------------------------------------------------- set-up
// Column geometry (curvilinear): scale factors, Laplacian first-derivative
// coefficients, radius, dr/dxx0, volume factor and local spacing.
void launch_column_geometry(const Geo &g, double *h, double *gl, double *rad,
                            double *drdxx0, double *jac, double *dsmin,
                            cudaStream_t st);
void launch_min_interior(const Geo &g, const double *dsmin, double *out,
                         cudaStream_t st);
// Folded, c^2-scaled coefficients and boundary factors.  w1/w2 = FD weights
// for k = 0..ng (closed forms).
void launch_column_coefs(const Geo &g, const double *h, const double *gl,
                         const double *rad, const double *drdxx0,
                         const double *dsmin, const double *dsmin_global,
                         const double *w1, const double *w2,
                         ColumnSet<double> c64, ColumnSet<float> c32,
                         cudaStream_t st);

struct PunctureDev {
  double m, x[3], P[3], S[3];
};
struct PunctureSet {
  int n;
  PunctureDev p[8];
};
// alpha = 1/psi_s, c^2 beta at every padded point (FP64 and FP32 copies);
// sets *bad if a puncture coincides with a grid point.
void launch_source(const Geo &g, const PunctureSet &ps, const double *dsmin,
                   const double *dsmin_global, double *alpha, double *bc2,
                   float *alpha32, float *bc2_32, int *bad, cudaStream_t st);

// ---------------------------------------------------------------- stencil
template <typename R>
struct StageArgs {
  const R *su, *sv;  // stage input state (u is differentiated)
  const R *bu, *bv;  // base state y (FIRST/MID)
  R *au, *av;        // accumulator
  R *ou, *ov;        // stage output (or k for RAW)
  const R *alpha, *bc2;
  ColumnSet<R> col;
  CartCoef cart;
  R eta, wa, wb;     // damping, a_s dt, b_s dt
  const R *fu;       // forcing of the u equation (lin only)
  int *err;          // device flag set by a stage kernel whose bounded wait
                     // for an asynchronous copy expired (nullable)
  int lin;           // 1: increment equation of the defect correction:
                     //    k_u = v - eta u + f_u, k_v = c^2 lap u - alpha u + bc2
                     //    with alpha = c^2 a, bc2 = f_v (forcings also added
                     //    on the outer shell)
};

template <typename R>
void launch_stage(const Geo &g, int kind, const StageArgs<R> &a,
                  const LaunchCfg &cfg, cudaStream_t st);

// Arguments of RK4 stage `stage` (0..3) of one field set: classical RK4,
// k1 = F(y); k2 = F(y + dt/2 k1); k3 = F(y + dt/2 k2); k4 = F(y + dt k3);
// y += dt/6 (k1 + 2 k2 + 2 k3 + k4), through the buffers y -> s -> t -> s -> y
// with the accumulator a.
template <typename R>
StageArgs<R> rk4_stage_args(const FieldSet<R> &f, const ColumnSet<R> &c,
                            const CartCoef &cart, int *err, int stage,
                            double dt, double eta) {
  StageArgs<R> a{};
  a.alpha = f.alpha;
  a.bc2 = f.bc2;
  a.err = err;
  a.col = c;
  a.cart = cart;
  a.eta = (R)eta;
  a.lin = f.lin;
  a.fu = f.fu;
  a.au = f.a[0];
  a.av = f.a[1];
  a.bu = f.y[0];
  a.bv = f.y[1];
  switch (stage) {
    case 0:  // in y; acc = y + dt/6 k1; s = y + dt/2 k1
      a.su = f.y[0]; a.sv = f.y[1];
      a.ou = f.s[0]; a.ov = f.s[1];
      a.wa = (R)(0.5 * dt); a.wb = (R)(dt / 6.0);
      break;
    case 1:  // in s; acc += dt/3 k2; t = y + dt/2 k2
      a.su = f.s[0]; a.sv = f.s[1];
      a.ou = f.t[0]; a.ov = f.t[1];
      a.wa = (R)(0.5 * dt); a.wb = (R)(dt / 3.0);
      break;
    case 2:  // in t; acc += dt/3 k3; s = y + dt k3
      a.su = f.t[0]; a.sv = f.t[1];
      a.ou = f.s[0]; a.ov = f.s[1];
      a.wa = (R)dt; a.wb = (R)(dt / 3.0);
      break;
    default:  // in s; y = acc + dt/6 k4
      a.su = f.s[0]; a.sv = f.s[1];
      a.ou = f.y[0]; a.ov = f.y[1];
      a.wa = (R)0; a.wb = (R)(dt / 6.0);
      break;
  }
  return a;
}

// The FP64 device data of one grid, for drivers outside nrr_api.cu (the
// multi-patch system).  Pointers are owned by the grid.
struct GridView {
  Geo geo;
  cudaStream_t stream;     // the grid's work stream
  FieldSet<double> f64;
  ColumnSet<double> c64;
  CartCoef cart;
  LaunchCfg cfg64;         // FP64 stage launch shape
  LaunchCfg res_cfg;       // residual kernels
  const double *jac, *rad; // per column (curvilinear grids)
  double *scratch;         // s0*s1*s2 doubles free for the caller
  double *partials;        // residual partial sums (residual_blocks pairs)
  int *err;                // stage kernels' bounded-wait flag
  double dsmin;            // the wave speed's reference spacing
  bool have_source;
  FieldSet<float> dc32;    // defect correction: the FP32 increment fields
  ColumnSet<float> c32;
  LaunchCfg cfg32;         // FP32 stage launch shape
};
GridView grid_view(nrr_grid *g);

// Defect correction driven from outside a grid's own relaxation loop (the
// two-patch system), on stream st: the start of one outer iteration (the FP64
// right-hand side at the current state as the defect, the FP32 coefficient
// and forcings from it, the increment at rest) and its end (the FP64 state
// plus the FP32 increment).
void dc_outer_prep(nrr_grid *g, double eta, cudaStream_t st);
void dc_outer_update(nrr_grid *g, cudaStream_t st);

// `steps` RK4 steps (stage arguments FIRST, MID, MID, LAST) in one
// cooperative launch of a multi-stage curvilinear kernel (variant 5: the
// tensor-copy tiled form where the grid allows it, else variant 4's
// column form); `count` is a device word for its grid barriers (reset by
// this call).
template <typename R>
cudaError_t launch_stage_steps(const Geo &g, const StageArgs<R> (&sa)[4], int steps,
                               unsigned *count, const LaunchCfg &cfg,
                               cudaStream_t st);

// Two RK4 stages per launch (stage variant 6; FP32 SinhSymTP grids of FD
// order 8 with n0 % 32 == 0, n1 % 4 == 0 and n2 <= 16): stage2_ok tells
// whether a grid is eligible; launch_stage2_steps takes `steps` RK4 steps
// (2 launches each), the state alternating between f.y and f.s from step to
// step, so an even count leaves it in f.y.
bool stage2_ok(const Geo &g);
cudaError_t launch_stage2_steps(const Geo &g, const FieldSet<float> &f,
                                const ColumnSet<float> &c, double dt, double eta,
                                int64_t steps, int pdl, cudaStream_t st);

// Residual H (c^-2 times the scaled operator) at interior points and the
// per-block partial sums of H^2 J and J over r < r_int.  h_out nullable.
template <typename R>
void launch_residual(const Geo &g, const R *u, const R *alpha, const R *bc2,
                     ColumnSet<R> col, const CartCoef &cart, const double *jac,
                     const double *rad, double r_int, double *h_out,
                     double *partials, int *nblocks_out, const LaunchCfg &cfg,
                     cudaStream_t st, int lin = 0);
int residual_blocks(const Geo &g, const LaunchCfg &cfg);
// sqrt(sum num / sum den) of nblocks partial pairs into out[0]; out[1] = num,
// out[2] = den.  Fixed summation order.
void launch_norm_finalize(const double *partials, int nblocks, double *out,
                          cudaStream_t st);

// Fill inner ghosts of a padded grid function from their images.
template <typename R>
void launch_fill_ghosts(const Geo &g, R *f, cudaStream_t st);
// Precision conversion of whole padded arrays.
void launch_convert(const double *src, float *dst, int64_t n, cudaStream_t st);
void launch_convert(const float *src, double *dst, int64_t n, cudaStream_t st);
void launch_scale(double *f, double s, int64_t n, cudaStream_t st);
// Defect correction: FP32 coefficient c^2 a and forcings (f_u, f_v) = the
// FP64 right-hand side at (u, v); and the FP64 update (u, v) += (d, w).
void launch_dc_prepare(const Geo &g, const double *u, const double *alpha,
                       const double *bc2, const double *ku, const double *kv,
                       float *ac2, float *fu, float *fv, cudaStream_t st);
void launch_dc_update(double *u, double *v, const float *d, const float *w,
                      int64_t n, cudaStream_t st);

}  // namespace nrr
