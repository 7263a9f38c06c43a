// nrr_setup.cu -- device set-up of one grid (arXiv 2501.14030, Alg. 1 set-up:
// coordinate arrays, reference-metric precompute, constant source terms).
//
// Curvilinear grids (SinhSymTP, Spherical, SinhSpherical, SinhCylindrical)
// have a reference metric that does not depend on phi, so everything except the source lives in per-column
// arrays indexed col = i0 + s0*i1.
#include <cuda_runtime.h>

#include <cmath>

#include "nrr_internal.h"

namespace nrr {

namespace {

struct ColGeom {
  double h[3], gl[2], r, drdxx0;
};

// Scale factors h_i = |d(x,y,z)/d xx_i| and the first-derivative terms of
// the flat Laplacian, (1/J) d_i (J/h_i^2), J = h0 h1 h2 (Sec. 2, the
// reference-metric Laplacian).  SinhSymTP with A(xx0), Z = sqrt(A^2+b^2),
// V = sqrt(A^2 + b^2 sin^2 th):
//   h0 = A' V / Z, h1 = V, h2 = A sin th,
//   g0 = (Z^2 + A^2 - A Z^2 A''/A'^2) / (A' A V^2),  g1 = cot th / V^2.
// Spherical: h = (1, r, r sin th), g0 = 2/r, g1 = cot th / r^2.
// SinhSpherical, r = amax sinh(xx0/w)/sinh(1/w): h = (r', r, r sin th),
//   g0 = 2/(r r') - r''/r'^3, g1 = cot th / r^2.
// SinhCylindrical, columns (rho(xx0), z(xx1)) with sinh-stretched rho and z:
//   h = (rho', z', rho), g0 = 1/(rho rho') - rho''/rho'^3, g1 = -z''/z'^3.
__device__ ColGeom column_geom(const Geo &g, double xx0, double th) {
  ColGeom o;
  if (g.coord == SINHCYLINDRICAL) {
    const double w = g.sinhwaa, wz = g.sinhwz;
    const double rho = g.amax * sinh(xx0 / w) / sinh(1.0 / w);
    const double rhop = g.amax * cosh(xx0 / w) / (w * sinh(1.0 / w));
    const double rhopp = rho / (w * w);
    const double z = g.zmax * sinh(th / wz) / sinh(1.0 / wz);
    const double zp = g.zmax * cosh(th / wz) / (wz * sinh(1.0 / wz));
    const double zpp = z / (wz * wz);
    o.h[0] = rhop;
    o.h[1] = zp;
    o.h[2] = rho;
    o.gl[0] = 1.0 / (rho * rhop) - rhopp / (rhop * rhop * rhop);
    o.gl[1] = -zpp / (zp * zp * zp);
    o.r = sqrt(rho * rho + z * z);
    o.drdxx0 = rhop;
    return o;
  }
  double st, ct;
  sincos(th, &st, &ct);
  if (g.coord == SINHSYMTP) {
    double w = g.sinhwaa, b = g.bscale;
    double sh1 = sinh(1.0 / w);
    double sx, cx;
    sx = sinh(xx0 / w);
    cx = cosh(xx0 / w);
    double A = g.amax * sx / sh1;
    double Ap = g.amax * cx / (w * sh1);
    double App = A / (w * w);
    double Z2 = A * A + b * b;
    double V2 = A * A + b * b * st * st;
    double V = sqrt(V2);
    o.h[0] = Ap * V / sqrt(Z2);
    o.h[1] = V;
    o.h[2] = A * st;
    o.gl[0] = (Z2 + A * A - A * Z2 * App / (Ap * Ap)) / (Ap * A * V2);
    o.gl[1] = ct / (st * V2);
    o.r = sqrt(A * A + b * b * ct * ct);
    o.drdxx0 = A * Ap / o.r;
  } else if (g.coord == SINHSPHERICAL) {
    double w = g.sinhwaa;
    double sh1 = sinh(1.0 / w);
    double r = g.amax * sinh(xx0 / w) / sh1;
    double rp = g.amax * cosh(xx0 / w) / (w * sh1);
    double rpp = r / (w * w);
    o.h[0] = rp;
    o.h[1] = r;
    o.h[2] = r * st;
    o.gl[0] = 2.0 / (r * rp) - rpp / (rp * rp * rp);
    o.gl[1] = ct / (r * r * st);
    o.r = fabs(r);
    o.drdxx0 = rp;
  } else {
    double r = xx0;
    o.h[0] = 1.0;
    o.h[1] = r;
    o.h[2] = r * st;
    o.gl[0] = 2.0 / r;
    o.gl[1] = ct / (r * r * st);
    o.r = fabs(r);
    o.drdxx0 = 1.0;
  }
  return o;
}

__global__ void column_geometry_kernel(Geo g, double *h, double *gl,
                                       double *rad, double *drdxx0,
                                       double *jac, double *dsmin) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= g.ncol) return;
  int i0 = col % g.s0, i1 = col / g.s0;
  double xx0 = g.xxmin[0] + (i0 - g.ng + 0.5) * g.dxx[0];
  double th = g.xxmin[1] + (i1 - g.ng + 0.5) * g.dxx[1];
  ColGeom o = column_geom(g, xx0, th);
  double ds = INFINITY;
  for (int d = 0; d < 3; d++) {
    h[d * g.ncol + col] = o.h[d];
    ds = fmin(ds, fabs(o.h[d]) * g.dxx[d]);
  }
  gl[col] = o.gl[0];
  gl[g.ncol + col] = o.gl[1];
  rad[col] = o.r;
  drdxx0[col] = o.drdxx0;
  jac[col] = fabs(o.h[0] * o.h[1] * o.h[2]);
  dsmin[col] = ds;
}

// Minimum over interior columns; min is exact, so the order is irrelevant.
__global__ void min_interior_kernel(Geo g, const double *dsmin, double *out) {
  __shared__ double sm[256];
  double m = INFINITY;
  int nint = g.n0 * g.n1;
  for (int e = threadIdx.x; e < nint; e += blockDim.x) {
    int i0 = e % g.n0 + g.ng, i1 = e / g.n0 + g.ng;
    m = fmin(m, dsmin[i0 + g.s0 * i1]);
  }
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] = fmin(sm[threadIdx.x], sm[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sm[0];
}

struct Weights {
  double w1[7], w2[7];  // k = 0..ng
};

// Fold the metric, the FD weights and c^2 into one weight per stencil point:
//   c^2 [ h_d^-2 w2_k / dxx_d^2 +- g_d w1_k / dxx_d ]
// so that c^2 lap(u) = sum over stencil points of weight * u.
__global__ void column_coefs_kernel(Geo g, const double *h, const double *gl,
                                    const double *rad, const double *drdxx0,
                                    const double *dsmin,
                                    const double *dsmin_global, Weights w,
                                    ColumnSet<double> c64,
                                    ColumnSet<float> c32) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= g.ncol) return;
  const int ng = g.ng, nc = g.ncol;
  double c = dsmin[col] / dsmin_global[0];
  double c2 = c * c;
  double ghat[3], gf[2];
  for (int d = 0; d < 3; d++) {
    double hd = h[d * nc + col];
    ghat[d] = 1.0 / (hd * hd * g.dxx[d] * g.dxx[d]);
  }
  gf[0] = gl[col] / g.dxx[0];
  gf[1] = gl[nc + col] / g.dxx[1];
  double vals[31];
  vals[0] = c2 * w.w2[0] * (ghat[0] + ghat[1] + ghat[2]);
  for (int k = 1; k <= ng; k++) {
    vals[k] = c2 * (ghat[0] * w.w2[k] + gf[0] * w.w1[k]);
    vals[ng + k] = c2 * (ghat[0] * w.w2[k] - gf[0] * w.w1[k]);
    vals[2 * ng + k] = c2 * (ghat[1] * w.w2[k] + gf[1] * w.w1[k]);
    vals[3 * ng + k] = c2 * (ghat[1] * w.w2[k] - gf[1] * w.w1[k]);
    vals[4 * ng + k] = c2 * (ghat[2] * w.w2[k]);
  }
  int nco = 5 * ng + 1;
  for (int j = 0; j < nco; j++) {
    c64.coef[j * nc + col] = vals[j];
    c32.coef[j * nc + col] = (float)vals[j];
  }
  double sm[3] = {c, 1.0 / (2.0 * g.dxx[0] * drdxx0[col]), 1.0 / rad[col]};
  if (g.coord == SINHCYLINDRICAL) {
    // d_r f = (rho/r)(1/rho') D_xx0 f + (z/r)(1/z') D_xx1 f, both D with
    // the 1/(2 dxx) of the second-order differences folded in: row 1 holds
    // the rho factor, row 3 (SinhCylindrical only) the z factor
    const int i1 = col / g.s0;
    const double xx1 = g.xxmin[1] + (i1 - ng + 0.5) * g.dxx[1];
    const double z = g.zmax * sinh(xx1 / g.sinhwz) / sinh(1.0 / g.sinhwz);
    const double rho = h[2 * nc + col];
    sm[1] = rho / (rad[col] * 2.0 * g.dxx[0] * h[col]);
    const double kz = z / (rad[col] * 2.0 * g.dxx[1] * h[nc + col]);
    c64.somm[3 * nc + col] = kz;
    c32.somm[3 * nc + col] = (float)kz;
  }
  for (int j = 0; j < 3; j++) {
    c64.somm[j * nc + col] = sm[j];
    c32.somm[j * nc + col] = (float)sm[j];
  }
  c64.c2inv[col] = 1.0 / c2;
  c32.c2inv[col] = (float)(1.0 / c2);
}

// Cartesian position of a padded point.
__device__ void cart_position(const Geo &g, int i0, int i1, int i2,
                              double x[3]) {
  double xx0 = g.xxmin[0] + (i0 - g.ng + 0.5) * g.dxx[0];
  double xx1 = g.xxmin[1] + (i1 - g.ng + 0.5) * g.dxx[1];
  double xx2 = g.xxmin[2] + (i2 - g.ng + 0.5) * g.dxx[2];
  if (g.coord == CARTESIAN) {
    x[0] = xx0;
    x[1] = xx1;
    x[2] = xx2;
    return;
  }
  double st, ct, sp, cp;
  sincos(xx1, &st, &ct);
  sincos(xx2, &sp, &cp);
  if (g.coord == SINHCYLINDRICAL) {
    const double rho = g.amax * sinh(xx0 / g.sinhwaa) / sinh(1.0 / g.sinhwaa);
    x[0] = rho * cp;
    x[1] = rho * sp;
    x[2] = g.zmax * sinh(xx1 / g.sinhwz) / sinh(1.0 / g.sinhwz);
    return;
  }
  if (g.coord == SINHSYMTP) {
    double A = g.amax * sinh(xx0 / g.sinhwaa) / sinh(1.0 / g.sinhwaa);
    double Z = sqrt(A * A + g.bscale * g.bscale);
    x[0] = A * st * cp;
    x[1] = A * st * sp;
    x[2] = Z * ct;
  } else {
    const double r = g.coord == SINHSPHERICAL
                         ? g.amax * sinh(xx0 / g.sinhwaa) / sinh(1.0 / g.sinhwaa)
                         : xx0;
    x[0] = r * st * cp;
    x[1] = r * st * sp;
    x[2] = r * ct;
  }
}

// Bowen-York curvature of each puncture (n = unit vector from the puncture):
//   A^ij = 3/(2r^2)[P^i n^j + P^j n^i - (delta^ij - n^i n^j) P.n]
//        + 3/r^3 [(S x n)^i n^j + (S x n)^j n^i],
// summed; A~A~ = sum_ij (A^ij)^2.  psi_s = 1 + sum m/(2r).
// Stored: alpha = 1/psi_s and c^2 beta, beta = A~A~ alpha^7 / 8.
__global__ void source_kernel(Geo g, PunctureSet ps, const double *dsmin,
                              const double *dsmin_global, double *alpha,
                              double *bc2, float *alpha32, float *bc2_32,
                              int *bad) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= g.npts) return;
  int i0 = (int)(p % g.s0);
  int i1 = (int)((p / g.s0) % g.s1);
  int i2 = (int)(p / g.ncol);
  double x[3];
  cart_position(g, i0, i1, i2, x);
  double A[6] = {0, 0, 0, 0, 0, 0};  // xx, yy, zz, xy, xz, yz
  double psi = 1.0;
  for (int a = 0; a < ps.n; a++) {
    const PunctureDev &q = ps.p[a];
    double d0 = x[0] - q.x[0], d1 = x[1] - q.x[1], d2 = x[2] - q.x[2];
    double r = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
    if (!(r > 0.0)) {
      *bad = 1;
      r = 1e-300;
    }
    double ir = 1.0 / r;
    double n[3] = {d0 * ir, d1 * ir, d2 * ir};
    double Pn = q.P[0] * n[0] + q.P[1] * n[1] + q.P[2] * n[2];
    double sxn[3] = {q.S[1] * n[2] - q.S[2] * n[1],
                     q.S[2] * n[0] - q.S[0] * n[2],
                     q.S[0] * n[1] - q.S[1] * n[0]};
    double cm = 1.5 * ir * ir, cs = 3.0 * ir * ir * ir;
    const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
    for (int c = 0; c < 6; c++) {
      int i = ii[c], j = jj[c];
      double delta = (i == j) ? 1.0 : 0.0;
      A[c] += cm * (q.P[i] * n[j] + q.P[j] * n[i] - (delta - n[i] * n[j]) * Pn) +
              cs * (sxn[i] * n[j] + sxn[j] * n[i]);
    }
    psi += q.m * 0.5 * ir;
  }
  double aa = A[0] * A[0] + A[1] * A[1] + A[2] * A[2] +
              2.0 * (A[3] * A[3] + A[4] * A[4] + A[5] * A[5]);
  double al = 1.0 / psi;
  double al2 = al * al, al4 = al2 * al2;
  double beta = 0.125 * aa * al4 * al2 * al;
  double c2 = 1.0;
  if (g.coord != CARTESIAN) {
    double c = dsmin[i0 + g.s0 * i1] / dsmin_global[0];
    c2 = c * c;
  } else {
    // uniform spacing: c = spacing / reference spacing, exactly 1 unless the
    // grid is a patch of a multi-patch system with a smaller reference
    double c = fmin(g.dxx[0], fmin(g.dxx[1], g.dxx[2])) / dsmin_global[0];
    c2 = c * c;
  }
  alpha[p] = al;
  bc2[p] = c2 * beta;
  alpha32[p] = (float)al;
  bc2_32[p] = (float)(c2 * beta);
}

}  // namespace

void launch_column_geometry(const Geo &g, double *h, double *gl, double *rad,
                            double *drdxx0, double *jac, double *dsmin,
                            cudaStream_t st) {
  int nb = (g.ncol + 127) / 128;
  column_geometry_kernel<<<nb, 128, 0, st>>>(g, h, gl, rad, drdxx0, jac, dsmin);
}

void launch_min_interior(const Geo &g, const double *dsmin, double *out,
                         cudaStream_t st) {
  min_interior_kernel<<<1, 256, 0, st>>>(g, dsmin, out);
}

void launch_column_coefs(const Geo &g, const double *h, const double *gl,
                         const double *rad, const double *drdxx0,
                         const double *dsmin, const double *dsmin_global,
                         const double *w1, const double *w2,
                         ColumnSet<double> c64, ColumnSet<float> c32,
                         cudaStream_t st) {
  Weights w;
  for (int k = 0; k < 7; k++) {
    w.w1[k] = k <= g.ng ? w1[k] : 0.0;
    w.w2[k] = k <= g.ng ? w2[k] : 0.0;
  }
  int nb = (g.ncol + 127) / 128;
  column_coefs_kernel<<<nb, 128, 0, st>>>(g, h, gl, rad, drdxx0, dsmin,
                                          dsmin_global, w, c64, c32);
}

void launch_source(const Geo &g, const PunctureSet &ps, const double *dsmin,
                   const double *dsmin_global, double *alpha, double *bc2,
                   float *alpha32, float *bc2_32, int *bad, cudaStream_t st) {
  int64_t nb = (g.npts + 255) / 256;
  source_kernel<<<(unsigned)nb, 256, 0, st>>>(g, ps, dsmin, dsmin_global,
                                              alpha, bc2, alpha32, bc2_32, bad);
}

}  // namespace nrr
