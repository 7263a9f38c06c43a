// nrr_common.cuh -- grid descriptor and index rules shared by host and device
// code of libnrr.
//
// Layout: padded grid functions, flat index p = i0 + s0*(i1 + s1*i2), i0
// fastest, s_d = n_d + 2*ng.  Per-column arrays (curvilinear grids, where the
// reference metric does not depend on phi) have index col = i0 + s0*i1.
#pragma once

#include <cstdint>

#if defined(__CUDACC__)
#define NRR_HD __host__ __device__ __forceinline__
#else
#define NRR_HD inline
#endif

namespace nrr {

enum Coord { SINHSYMTP = 0, SPHERICAL = 1, CARTESIAN = 2, SINHSPHERICAL = 3,
             SINHCYLINDRICAL = 4 };

// Spherical-like maps (radius odd in xx0): the xx0 < 0 image also reflects
// theta.
NRR_HD bool spherical_like(int coord) {
  return coord == SPHERICAL || coord == SINHSPHERICAL;
}

// Everything a kernel needs to know about one grid, passed by value.
struct Geo {
  int coord;
  int n0, n1, n2;
  int ng;
  int s0, s1, s2;
  int64_t npts;   // s0*s1*s2
  int ncol;       // s0*s1
  double xxmin[3];
  double dxx[3];
  double amax, bscale, sinhwaa;
  double zmax, sinhwz;  // SinhCylindrical: z = zmax sinh(xx1/sinhwz)/sinh(1/sinhwz)
};

NRR_HD int64_t flat(const Geo &g, int i0, int i1, int i2) {
  return (int64_t)i0 + (int64_t)g.s0 * ((int64_t)i1 + (int64_t)g.s1 * i2);
}

// Wrap a phi index into the interior range [ng, ng+n2).
NRR_HD int wrap_phi(const Geo &g, int i2) {
  int k = (i2 - g.ng) % g.n2;
  if (k < 0) k += g.n2;
  return k + g.ng;
}

// Inner-boundary image of a padded point on a curvilinear grid, by the
// symmetries of the coordinate map (cell-centred sampling makes each image
// an exact grid point):
//   SinhSymTP: (xx0,th,ph) with xx0<0 -> (-xx0, th, ph+pi)   [A odd, Z even]
//              th<0 -> (-th, ph+pi); th>pi -> (2pi-th, ph+pi)
//   Spherical, SinhSpherical: r<0 -> (-r, pi-th, ph+pi); theta rules as above
//   SinhCylindrical (rho, z, ph): rho<0 -> (-rho, z, ph+pi); points beyond
//              the ends in z are evolved (outer), not images
//   phi periodic.
// Evolved points (interior and the outer shell) map to themselves.
NRR_HD void image_of(const Geo &g, int &i0, int &i1, int &i2) {
  int flip = 0;
  if (i0 < g.ng) {
    i0 = 2 * g.ng - 1 - i0;
    flip ^= 1;
    if (spherical_like(g.coord)) i1 = g.n1 + 2 * g.ng - 1 - i1;
  }
  if (g.coord == SINHCYLINDRICAL) {
    i2 = wrap_phi(g, i2 + (flip ? g.n2 / 2 : 0));
    return;
  }
  if (i1 < g.ng) {
    i1 = 2 * g.ng - 1 - i1;
    flip ^= 1;
  } else if (i1 >= g.n1 + g.ng) {
    i1 = 2 * g.n1 + 2 * g.ng - 1 - i1;
    flip ^= 1;
  }
  i2 = wrap_phi(g, i2 + (flip ? g.n2 / 2 : 0));
}

// Centred finite-difference weights of order 2m, closed forms:
//   first derivative  w_k = (-1)^(k+1) (m!)^2 / (k (m-k)! (m+k)!),  w_-k = -w_k
//   second derivative w_k = 2 (-1)^(k+1) (m!)^2 / (k^2 (m-k)! (m+k)!),
//                     w_0 = -2 sum_{k=1..m} 1/k^2.
inline double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; i++) f *= i;
  return f;
}
inline double fd_first(int m, int k) {  // k in [1, m]
  double v = factorial(m) * factorial(m) /
             ((double)k * factorial(m - k) * factorial(m + k));
  return (k & 1) ? v : -v;
}
inline double fd_second(int m, int k) {  // k in [0, m]
  if (k == 0) {
    double s = 0.0;
    for (int j = 1; j <= m; j++) s += 1.0 / ((double)j * j);
    return -2.0 * s;
  }
  double v = 2.0 * factorial(m) * factorial(m) /
             ((double)k * k * factorial(m - k) * factorial(m + k));
  return (k & 1) ? v : -v;
}

}  // namespace nrr
