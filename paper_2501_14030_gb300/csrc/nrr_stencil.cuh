// nrr_stencil.cuh -- device building blocks of the relaxation hot path
// (arXiv 2501.14030, Sec. 2 relaxation system; Alg. 1 RHS, BC, RK, H), shared
// by the single-grid kernels (nrr_stencil.cu) and the batched kernels
// (nrr_batch.cu).
#pragma once

#include <cuda_runtime.h>

#include "nrr_async.cuh"
#include "nrr_debug.cuh"
#include "nrr_internal.h"

namespace nrr {
namespace dev {

// In the NRR_DEBUG build every helper below first checks the address against
// the library's registered allocations (nrr_debug.cuh) and skips the access
// if it lies outside them; in the release build the check is absent.
#if NRR_DEBUG
#define NRR_DBG_LOAD(p) \
  if (!dbg_ok((p), sizeof(*(p)))) return decltype(+*(p))(0)
#define NRR_DBG_STORE(p) \
  if (!dbg_ok((p), sizeof(*(p)))) return
#else
#define NRR_DBG_LOAD(p) (void)0
#define NRR_DBG_STORE(p) (void)0
#endif

// Solve-constant data (folded stencil weights, boundary factors): the
// read-only path.  These are the only arrays a stage kernel reads before
// pdl_wait().
template <typename R>
__device__ __forceinline__ R ldc(const R *p) {
  NRR_DBG_LOAD(p);
  return __ldg(p);
}

// Everything a preceding kernel may have written (stage and base state, the
// accumulator, the defect correction's coefficient and forcings): plain
// coherent loads.  A read-only load counts as invariant for the whole
// kernel, so the compiler may issue it ahead of the griddepcontrol.wait
// statement -- before the preceding stage has finished writing -- and with
// programmatic dependent launch that reads stale state.  A plain load stays
// behind the wait's memory clobber.
template <typename R>
__device__ __forceinline__ R ld(const R *p) {
  NRR_DBG_LOAD(p);
  return *p;
}

// Stores of the stage and residual kernels to global memory.
template <typename R>
__device__ __forceinline__ void st(R *p, R v) {
  NRR_DBG_STORE(p);
  *p = v;
}

// Loads of state written earlier in the same launch (the multi-stage kernel
// below, after a grid barrier) go through L2 (ld.global.cg); everything
// else with plain loads (ld above).
template <bool COH, typename R>
__device__ __forceinline__ R lds(const R *p) {
  if constexpr (COH) {
    NRR_DBG_LOAD(p);
    return __ldcg(p);
  } else {
    return ld(p);
  }
}

// A product or sum rounded on its own: the compiler may not fuse it with a
// neighbouring operation into an FMA, so that the result does not depend on
// how the surrounding code was optimised (the debug build must agree with
// the release build bit for bit).
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }

// Programmatic dependent launch: a stage kernel launched with the
// programmatic-serialisation attribute may start while the preceding kernel
// on its stream drains.  Before pdl_wait() it reads only data that no kernel
// of the solve writes (column weights, geometry); pdl_wait() returns once the
// preceding grid has completed and its writes are visible.  pdl_trigger()
// lets the next kernel begin launching as soon as every block of this one
// has started.  Both are no-ops for a kernel launched without the attribute.
__device__ __forceinline__ void pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The linear (defect-correction increment) mode exists only in FP32; in FP64
// the tests below fold to constants and the FP64 pipe never sees them.
template <typename R>
__device__ __forceinline__ bool linear_mode(int lin) {
  return sizeof(R) == 4 && lin;
}

// Reciprocal of s = 1 + alpha u (a normal number near 1) by refinement of the
// hardware approximation: in single precision one Newton-Raphson step
// t <- t + t (1 - s t) (quadratic) suffices; in double precision one
// third-order step replaces two Newton steps.
__device__ __forceinline__ double recip(double s) {
  double t;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(t) : "d"(s));
  // third-order (Householder) step 1/s = t / (1 - e) ~ t (1 + e + e^2) with
  // e = 1 - s t: the seed's relative error (measured below 2^-20 on sm_103a)
  // cubes to below 2^-60, so the result is within one ulp of 1/s.
  double e = fma(-s, t, 1.0);
  return fma(t, fma(e, e, e), t);
}
__device__ __forceinline__ float recip(float s) {
  float t;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(t) : "f"(s));
  float e = fmaf(-s, t, 1.0f);
  return fmaf(t, e, t);
}

// The source term added to acc (both c^2-scaled).  Nonlinear:
// beta c^2 (1 + alpha u)^-7 with (al, bc2) = (alpha, c^2 beta).  Linear (the
// increment equation of the defect correction): f_v - c^2 a d with
// (al, bc2) = (c^2 a, f_v).  `lin` is uniform across the launch.
template <typename R>
__device__ __forceinline__ R add_source(R acc, R u0, R al, R bc2, int lin) {
  if (linear_mode<R>(lin)) return acc + fma(-al, u0, bc2);
  R t = recip(fma(al, u0, R(1)));
  R t2 = t * t;
  R t4 = t2 * t2;
  R q = bc2 * t;
  q = q * t2;
  return fma(q, t4, acc);
}

// c^2 [lap(u) + source] at ZC interior points of one column (i0, i1) of a
// curvilinear grid, planes pl[0..ZC).  zo[] holds the element offsets
// (ncol x plane) of the wrapped phi planes pl[0]-NG .. pl[ZC-1]+NG, ho[]
// those of the planes phi + pi of pl[].  Indices are 32-bit: a grid holds
// at most 2^31 points.  One
// accumulation chain per point -- centre, xx0, xx1, phi, then the source --
// in the order every curvilinear stage kernel uses: on the FP64 pipe (a
// warp instruction every 64 cycles per SM sub-partition) latency is hidden
// by the other warps, and a second chain would cost its own multiply and
// the add that joins the two.
//
// CYL (SinhCylindrical, columns (rho, z)): the second direction is z, whose
// ghost rows beyond both ends are evolved outer points read as stored
// instead of theta reflections.
template <typename R, int NG, int ZC, bool COH = false, bool CYL = false>
__device__ __forceinline__ void curvi_operator(
    const Geo &g, const R *__restrict__ su, const R (&w)[5 * NG + 1], int col,
    int i0, int i1, const int (&zo)[ZC + 2 * NG], const int (&ho)[ZC],
    const R (&u0)[ZC], const R (&al)[ZC], const R (&bc)[ZC], R (&out)[ZC],
    int lin) {
  const int s0 = g.s0;
  R a0[ZC];
#pragma unroll
  for (int j = 0; j < ZC; j++) a0[j] = w[0] * u0[j];
  // xx0: the + side stays inside the padded box; the - side may cross
  // xx0 = 0 and read the reflected point at phi + pi.
  const int rrow = s0 * (spherical_like(g.coord) ? g.n1 + 2 * NG - 1 - i1 : i1);
#pragma unroll
  for (int k = 1; k <= NG; k++) {
    const int im = i0 - k;
    const bool refl = im < NG;
    const int rcol = (2 * NG - 1 - im) + rrow;
#pragma unroll
    for (int j = 0; j < ZC; j++) {
      const R *pc = su + (col + zo[NG + j]);
      R up = lds<COH>(pc + k);
      R um = refl ? lds<COH>(su + (rcol + ho[j])) : lds<COH>(pc - k);
      a0[j] = fma(w[k], up, a0[j]);
      a0[j] = fma(w[NG + k], um, a0[j]);
    }
  }
  // theta: reflections through the axis, again with phi + pi.
#pragma unroll
  for (int k = 1; k <= NG; k++) {
    const int ip = i1 + k, im = i1 - k;
    const bool rp = !CYL && ip >= g.n1 + NG, rm = !CYL && im < NG;
    const int cp = i0 + s0 * (rp ? 2 * g.n1 + 2 * NG - 1 - ip : ip);
    const int cm = i0 + s0 * (rm ? 2 * NG - 1 - im : im);
#pragma unroll
    for (int j = 0; j < ZC; j++) {
      R up = lds<COH>(su + (cp + (rp ? ho[j] : zo[NG + j])));
      R um = lds<COH>(su + (cm + (rm ? ho[j] : zo[NG + j])));
      a0[j] = fma(w[2 * NG + k], up, a0[j]);
      a0[j] = fma(w[3 * NG + k], um, a0[j]);
    }
  }
  // phi: periodic.
#pragma unroll
  for (int k = 1; k <= NG; k++) {
#pragma unroll
    for (int j = 0; j < ZC; j++) {
      R sp = lds<COH>(su + (col + zo[NG + j + k]));
      R sm = lds<COH>(su + (col + zo[NG + j - k]));
      a0[j] = fma(w[4 * NG + k], sp + sm, a0[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < ZC; j++)
    out[j] = add_source(a0[j], u0[j], al[j], bc[j], lin);
}

// phi index into [NG, NG+n2) by adding or subtracting periods (offsets are a
// few planes, so this is one or two compare-and-adds, no division).
template <int NG>
__device__ __forceinline__ int wrap_plane(const Geo &g, int z) {
  while (z < NG) z += g.n2;
  while (z >= NG + g.n2) z -= g.n2;
  return z;
}

// Plane offsets of one thread: zo[j] = ncol x (phi plane z0-NG+j, wrapped;
// planes past the last one are clamped so that loads stay in range), ho[j]
// = ncol x (the plane at phi + pi of plane z0+j).  Each plane is wrapped on
// its own: an incremental form (previous plane plus one) made the stage
// kernel slower.
template <int NG, int ZC>
__device__ __forceinline__ void plane_offsets(const Geo &g, int z0, int (&zo)[ZC + 2 * NG],
                                              int (&ho)[ZC]) {
  const int nc = g.ncol, last = NG + g.n2 - 1;
#pragma unroll
  for (int j = 0; j < ZC + 2 * NG; j++) zo[j] = nc * wrap_plane<NG>(g, min(z0 - NG + j, last + NG));
#pragma unroll
  for (int j = 0; j < ZC; j++) ho[j] = nc * wrap_plane<NG>(g, min(z0 + j, last) + g.n2 / 2);
}

template <typename R, int KIND, bool COH = false>
__device__ __forceinline__ void stage_epilogue(const StageArgs<R> &a, int64_t p,
                                               R ku, R kv) {
  if (KIND == STAGE_FIRST) {
    R yu = lds<COH>(a.bu + p), yv = lds<COH>(a.bv + p);
    st(a.au + p, fma(a.wb, ku, yu));
    st(a.av + p, fma(a.wb, kv, yv));
    st(a.ou + p, fma(a.wa, ku, yu));
    st(a.ov + p, fma(a.wa, kv, yv));
  } else if (KIND == STAGE_MID) {
    R yu = lds<COH>(a.bu + p), yv = lds<COH>(a.bv + p);
    st(a.au + p, fma(a.wb, ku, ld(a.au + p)));
    st(a.av + p, fma(a.wb, kv, ld(a.av + p)));
    st(a.ou + p, fma(a.wa, ku, yu));
    st(a.ov + p, fma(a.wa, kv, yv));
  } else if (KIND == STAGE_LAST) {
    st(a.ou + p, fma(a.wb, ku, ld(a.au + p)));
    st(a.ov + p, fma(a.wb, kv, ld(a.av + p)));
  } else {
    st(a.ou + p, ku);
    st(a.ov + p, kv);
  }
}

// One work item of the curvilinear stage kernel: column e of the evolved
// points on ZC consecutive phi planes from z0.  Columns e < n0 n1 are the
// interior ones (i0 fastest); the NG n1 columns after them form the outer
// shell i0 >= n0+ng.  Numbering the shell last keeps the short radiation
// path out of the interior warps (except the one warp at the seam).
// SinhCylindrical outer shell, item s of NG n1 + 2 NG (n0 + NG) columns: first
// the side beyond rho = amax (i0 >= n0+NG, interior i1), then the rows beyond
// both ends in z (i1 < NG or i1 >= n1+NG, i0 from NG).  Radiation condition
// df/dt = -c (d_r f + f/r) with d_r f = (rho/r)(1/rho') D_xx0 f +
// (z/r)(1/z') D_xx1 f; each second-order difference one-sided inward where
// the point lies beyond that direction's boundary, centred otherwise.  At
// i0 = NG the centred xx0 difference reaches the rho < 0 image: the same
// column at phi + pi.
template <typename R, int NG, int KIND, int ZC>
__device__ __forceinline__ void stage_cyl_shell(const Geo &g, const StageArgs<R> &a,
                                                int s, int z0) {
  const int nside = NG * g.n1;
  int i0, i1;
  if (s < nside) {
    i0 = g.n0 + NG + s % NG;
    i1 = NG + s / NG;
  } else {
    const int t = s - nside, wdt = g.n0 + NG, row = t / wdt;
    i0 = NG + t % wdt;
    i1 = row < NG ? row : g.n1 + row;
  }
  const int col = i0 + g.s0 * i1;
  const int nc = g.ncol, s0 = g.s0;
  const int zend = NG + g.n2;
  const R c = ldc(a.col.somm + col), kr = ldc(a.col.somm + nc + col),
          rinv = ldc(a.col.somm + 2 * nc + col), kz = ldc(a.col.somm + 3 * nc + col);
  const bool out0 = i0 >= g.n0 + NG;
  const int side1 = i1 >= g.n1 + NG ? 1 : (i1 < NG ? -1 : 0);
  pdl_wait();
#pragma unroll
  for (int j = 0; j < ZC; j++) {
    const int z = z0 + j;
    if (z >= zend) break;
    const int64_t p = col + (int64_t)nc * z;
    const int64_t pm = i0 == NG ? col + (int64_t)nc * wrap_plane<NG>(g, z + g.n2 / 2)
                                : p - 1;
    R k2[2];
#pragma unroll
    for (int f = 0; f < 2; f++) {
      const R *q = f == 0 ? a.su : a.sv;
      const R f0 = ld(q + p);
      const R d0 = out0 ? fma(R(3), f0, fma(R(-4), ld(q + p - 1), ld(q + p - 2)))
                        : ld(q + p + 1) - ld(q + pm);
      R d1;
      if (side1 > 0)
        d1 = fma(R(3), f0, fma(R(-4), ld(q + p - s0), ld(q + p - 2 * s0)));
      else if (side1 < 0)
        d1 = -fma(R(3), f0, fma(R(-4), ld(q + p + s0), ld(q + p + 2 * s0)));
      else
        d1 = ld(q + p + s0) - ld(q + p - s0);
      k2[f] = mul_rn(-c, fma(kr, d0, fma(kz, d1, mul_rn(rinv, f0))));
    }
    if (linear_mode<R>(a.lin)) {
      k2[0] += ld(a.fu + p);
      k2[1] += ld(a.bc2 + p);
    }
    stage_epilogue<R, KIND>(a, p, k2[0], k2[1]);
  }
}

template <typename R, int NG, int KIND, int ZC, bool COH = false, bool CYL = false>
__device__ __forceinline__ void stage_curvi_item(const Geo &g, const StageArgs<R> &a,
                                                 int e, int z0) {
  const int nint = g.n0 * g.n1;
  const bool shell = e >= nint;
  if constexpr (CYL) {
    if (shell) {
      stage_cyl_shell<R, NG, KIND, ZC>(g, a, e - nint, z0);
      return;
    }
  }
  const int i0 = shell ? g.n0 + NG + (e - nint) % NG : e % g.n0 + NG;
  const int i1 = (shell ? (e - nint) / NG : e / g.n0) + NG;
  const int col = i0 + g.s0 * i1;
  const int nc = g.ncol;
  const int zend = NG + g.n2;
  if (shell) {
    // Radiation condition, df/dt = -c (d_r f + f/r), d_r from the
    // second-order backward difference along xx0.
    R c = ldc(a.col.somm + col), kdb = ldc(a.col.somm + nc + col),
      rinv = ldc(a.col.somm + 2 * nc + col);
    pdl_wait();
#pragma unroll
    for (int j = 0; j < ZC; j++) {
      if (z0 + j >= zend) break;
      int64_t p = col + (int64_t)nc * (z0 + j);
      R u0 = lds<COH>(a.su + p), u1 = lds<COH>(a.su + p - 1),
        u2 = lds<COH>(a.su + p - 2);
      R v0 = lds<COH>(a.sv + p), v1 = lds<COH>(a.sv + p - 1),
        v2 = lds<COH>(a.sv + p - 2);
      R du = fma(R(3), u0, fma(R(-4), u1, u2));
      R dv = fma(R(3), v0, fma(R(-4), v1, v2));
      R ku = mul_rn(-c, fma(kdb, du, mul_rn(rinv, u0)));
      R kv = mul_rn(-c, fma(kdb, dv, mul_rn(rinv, v0)));
      if (linear_mode<R>(a.lin)) {
        ku += ld(a.fu + p);
        kv += ld(a.bc2 + p);
      }
      stage_epilogue<R, KIND, COH>(a, p, ku, kv);
    }
    return;
  }
  R w[5 * NG + 1];
#pragma unroll
  for (int j = 0; j < 5 * NG + 1; j++) w[j] = ldc(a.col.coef + (int64_t)j * nc + col);
  int zo[ZC + 2 * NG], ho[ZC];
  plane_offsets<NG, ZC>(g, z0, zo, ho);
  pdl_wait();
  R u0[ZC], v0[ZC], al[ZC], bc[ZC], kv[ZC];
#pragma unroll
  for (int j = 0; j < ZC; j++) {
    const int p = col + zo[NG + j];
    u0[j] = lds<COH>(a.su + p);
    v0[j] = lds<COH>(a.sv + p);
    al[j] = ld(a.alpha + p);
    bc[j] = ld(a.bc2 + p);
  }
  // Operands of the RK4 update, loaded before any store so that the loads
  // overlap the stencil's.
  R yb[2][ZC], ac[2][ZC], fu[ZC];
#pragma unroll
  for (int j = 0; j < ZC; j++) {
    const int p = col + zo[NG + j];
    if (KIND == STAGE_FIRST || KIND == STAGE_MID) {
      yb[0][j] = lds<COH>(a.bu + p);
      yb[1][j] = lds<COH>(a.bv + p);
    }
    if (KIND == STAGE_MID || KIND == STAGE_LAST) {
      ac[0][j] = ld(a.au + p);
      ac[1][j] = ld(a.av + p);
    }
    fu[j] = linear_mode<R>(a.lin) ? ld(a.fu + p) : R(0);
  }
  curvi_operator<R, NG, ZC, COH, CYL>(g, a.su, w, col, i0, i1, zo, ho, u0, al, bc,
                                      kv, a.lin);
  // Plane z0 + j (< zend) is its own wrapped plane, so its offset is
  // zo[NG + j].
#pragma unroll
  for (int j = 0; j < ZC; j++) {
    if (z0 + j >= zend) break;
    const int p = col + zo[NG + j];
    R ku = fma(-a.eta, u0[j], v0[j]);
    if (linear_mode<R>(a.lin)) ku += fu[j];
    if (KIND == STAGE_FIRST) {
      st(a.au + p, fma(a.wb, ku, yb[0][j]));
      st(a.av + p, fma(a.wb, kv[j], yb[1][j]));
      st(a.ou + p, fma(a.wa, ku, yb[0][j]));
      st(a.ov + p, fma(a.wa, kv[j], yb[1][j]));
    } else if (KIND == STAGE_MID) {
      st(a.au + p, fma(a.wb, ku, ac[0][j]));
      st(a.av + p, fma(a.wb, kv[j], ac[1][j]));
      st(a.ou + p, fma(a.wa, ku, yb[0][j]));
      st(a.ov + p, fma(a.wa, kv[j], yb[1][j]));
    } else if (KIND == STAGE_LAST) {
      st(a.ou + p, fma(a.wb, ku, ac[0][j]));
      st(a.ov + p, fma(a.wb, kv[j], ac[1][j]));
    } else {
      st(a.ou + p, ku);
      st(a.ov + p, kv[j]);
    }
  }
}


// Deterministic block sum of two FP64 values (warp shuffles in a fixed
// pattern, then the warps in order).
__device__ __forceinline__ void block_sum2(double &x, double &y, double *out) {
  __shared__ double sx[32], sy[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    x += __shfl_down_sync(0xffffffffu, x, o);
    y += __shfl_down_sync(0xffffffffu, y, o);
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    sx[wid] = x;
    sy[wid] = y;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tx = 0.0, ty = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) {
      tx += sx[i];
      ty += sy[i];
    }
    out[0] = tx;
    out[1] = ty;
  }
}

// Residual of the curvilinear operator at one interior column e (counted i0
// fastest over the n0 x n1 interior columns) on planes [z0, z1): H at each
// point (written to h_out if given) and the sums of H^2 wt and wt with the
// column's norm weight wt.
template <typename R, int NG, bool CYL = false>
__device__ __forceinline__ void residual_curvi_item(
    const Geo &g, const R *__restrict__ su, const R *__restrict__ alpha,
    const R *__restrict__ bc2, const ColumnSet<R> &col_set, double wt, int e,
    int z0, int z1, int lin, double *h_out, double &num, double &den) {
  const int i0 = e % g.n0 + NG, i1 = e / g.n0 + NG;
  const int col = i0 + g.s0 * i1;
  const int nc = g.ncol;
  R w[5 * NG + 1];
#pragma unroll
  for (int j = 0; j < 5 * NG + 1; j++)
    w[j] = ldc(col_set.coef + (int64_t)j * nc + col);
  R c2inv = ldc(col_set.c2inv + col);
  for (int i2 = z0; i2 < z1; i2++) {
    int zo[1 + 2 * NG], ho[1];
    plane_offsets<NG, 1>(g, i2, zo, ho);
    const int p = col + nc * i2;
    R u0[1] = {ld(su + p)}, al[1] = {ld(alpha + p)}, bc[1] = {ld(bc2 + p)}, op[1];
    curvi_operator<R, NG, 1, false, CYL>(g, su, w, col, i0, i1, zo, ho, u0, al, bc,
                                         op, lin);
    double H = (double)(op[0] * c2inv);
    if (h_out) h_out[p] = H;
    num = fma(H * H, wt, num);
    den += wt;
  }
}

}  // namespace dev
}  // namespace nrr

namespace nrr {
namespace dev {

// ---------------------------------------------------------------------------
// Tiled stage: one block = a tile of 32 (i0) x TY (i1) interior columns and a
// chunk of ZC phi planes.  Per plane the block stages the tile with its
// NG-wide halo into shared memory (inner-boundary halo cells read from their
// images, so the phi + pi planes of reflected cells come in here), each
// thread keeps the 2NG+1 phi neighbours of its column in a register queue,
// and the folded column weights are loaded once per thread.  The loads of
// plane i2 + 1 (staged cells and operands, into registers) are issued before
// plane i2 is computed; one barrier per plane.  Extra blocks
// (tile_x == number of interior tiles) evolve the outer shell with the
// radiation condition.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int tiles_x(const Geo &g) { return (g.n0 + 31) / 32; }
template <int TY>
__host__ __device__ __forceinline__ int tiles_y(const Geo &g) { return (g.n1 + TY - 1) / TY; }
__host__ __device__ __forceinline__ int chunks_z(const Geo &g, int zc) { return (g.n2 + zc - 1) / zc; }

// Outer-shell rows of the tiled stage kernels: lane tx < NG of a tile row
// evolves column (n0 + NG + tx, i1) on planes [z0, z1) with the radiation
// condition df/dt = -c (d_r f + f/r).
template <typename R, int NG, int KIND, bool COH = false>
__device__ __forceinline__ void stage_shell_rows(const Geo &g, const StageArgs<R> &a,
                                                 int tx, int i1, int z0, int z1) {
  if (tx >= NG || i1 >= g.n1 + NG) return;
  const int nc = g.ncol;
  const int i0 = g.n0 + NG + tx;
  const int col = i0 + g.s0 * i1;
  const R c = ldc(a.col.somm + col), kdb = ldc(a.col.somm + nc + col),
          rinv = ldc(a.col.somm + 2 * nc + col);
  pdl_wait();
#pragma unroll 4
  for (int i2 = z0; i2 < z1; i2++) {
    const int64_t p = col + (int64_t)nc * i2;
    R u0 = lds<COH>(a.su + p), u1 = lds<COH>(a.su + p - 1), u2 = lds<COH>(a.su + p - 2);
    R v0 = lds<COH>(a.sv + p), v1 = lds<COH>(a.sv + p - 1), v2 = lds<COH>(a.sv + p - 2);
    R ku = mul_rn(-c, fma(kdb, fma(R(3), u0, fma(R(-4), u1, u2)), mul_rn(rinv, u0)));
    R kv = mul_rn(-c, fma(kdb, fma(R(3), v0, fma(R(-4), v1, v2)), mul_rn(rinv, v0)));
    if (linear_mode<R>(a.lin)) {
      ku += ld(a.fu + p);
      kv += ld(a.bc2 + p);
    }
    stage_epilogue<R, KIND, COH>(a, p, ku, kv);
  }
}

template <typename R, int NG, int KIND, int TY>
__device__ __forceinline__ void stage_tile_block(const Geo &g, const StageArgs<R> &a,
                                                 int tile_x, int tile_y, int chunk,
                                                 int zc, R (*tile)[TY + 2 * NG][32 + 2 * NG]) {
  constexpr int TW = 32 + 2 * NG, TH = TY + 2 * NG;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int nc = g.ncol;
  const int z0 = NG + chunk * zc;
  const int z1 = min(z0 + zc, NG + g.n2);
  const int i1 = NG + tile_y * TY + ty;
  if (tile_x == tiles_x(g)) {
    stage_shell_rows<R, NG, KIND>(g, a, tx, i1, z0, z1);
    return;
  }
  const int i0 = NG + tile_x * 32 + tx;
  const bool active = i0 < g.n0 + NG && i1 < g.n1 + NG;
  const int col = i0 + g.s0 * i1;
  constexpr int NT = 32 * TY;                   // threads of the block
  constexpr int NST = (TW * TH + NT - 1) / NT;  // staged cells per thread
  // The staged cells of this thread (flat index threadIdx.x + k NT of the
  // TH x TW tile with halo): in-plane offset of the cell's source -- its
  // image for an inner-boundary halo cell -- and whether that source lies on
  // the plane phi + pi; -1 for cells past the padded box, which no evolved
  // point reads.  Computed once; every plane reuses them.
  int soff[NST];
  unsigned flip = 0;
  {
    const int j0b = tile_x * 32, j1b = tile_y * TY;
#pragma unroll
    for (int k = 0; k < NST; k++) {
      const int cidx = threadIdx.x + k * NT;
      soff[k] = -1;
      if (cidx < TW * TH) {
        const int cy = cidx / TW, cx = cidx - cy * TW;
        int j0 = j0b + cx, j1 = j1b + cy;
        if (j0 < g.s0 && j1 < g.s1) {
          unsigned f = 0;
          if (j0 < NG) {
            j0 = 2 * NG - 1 - j0;
            f = 1;
            if (spherical_like(g.coord)) j1 = g.n1 + 2 * NG - 1 - j1;
          }
          if (j1 < NG) {
            j1 = 2 * NG - 1 - j1;
            f ^= 1;
          } else if (j1 >= g.n1 + NG) {
            j1 = 2 * g.n1 + 2 * NG - 1 - j1;
            f ^= 1;
          }
          soff[k] = j0 + g.s0 * j1;
          flip |= f << k;
        }
      }
    }
  }
  R w[5 * NG + 1];
  R q[2 * NG + 1];
  if (active) {
#pragma unroll
    for (int j = 0; j < 5 * NG + 1; j++) w[j] = ldc(a.col.coef + (int64_t)j * nc + col);
  }
  pdl_wait();
  if (active) {
#pragma unroll
    for (int k = 0; k < 2 * NG; k++)
      q[k + 1] = ld(a.su + col + (int64_t)nc * wrap_plane<NG>(g, z0 - NG + k));
  }
  // Registers holding the next plane: its staged cells and this thread's
  // operands.  Plane i2 + 1 is fetched before plane i2 is computed, so its
  // loads are in flight during the arithmetic.
  R sreg[NST];
  R nv = R(0), nal = R(0), nbc = R(0), nyb0 = R(0), nyb1 = R(0), nac0 = R(0),
    nac1 = R(0), nfu = R(0), nq = R(0);
#define NRR_TILE_FETCH(PL)                                                       \
  do {                                                                           \
    const int pl_ = (PL);                                                        \
    const R *base_ = a.su + (int64_t)nc * pl_;                                   \
    const R *bflip_ = a.su + (int64_t)nc * wrap_plane<NG>(g, pl_ + g.n2 / 2);    \
    _Pragma("unroll") for (int k = 0; k < NST; k++) if (soff[k] >= 0)            \
        sreg[k] = ld(((flip >> k) & 1u ? bflip_ : base_) + soff[k]);             \
    if (active) {                                                                \
      const int64_t p_ = col + (int64_t)nc * pl_;                                \
      nv = ld(a.sv + p_);                                                        \
      nal = ld(a.alpha + p_);                                                    \
      nbc = ld(a.bc2 + p_);                                                      \
      if (KIND == STAGE_FIRST || KIND == STAGE_MID) {                            \
        nyb0 = ld(a.bu + p_);                                                    \
        nyb1 = ld(a.bv + p_);                                                    \
      }                                                                          \
      if (KIND == STAGE_MID || KIND == STAGE_LAST) {                             \
        nac0 = ld(a.au + p_);                                                         \
        nac1 = ld(a.av + p_);                                                         \
      }                                                                          \
      if (linear_mode<R>(a.lin)) nfu = ld(a.fu + p_);                            \
      nq = ld(a.su + col + (int64_t)nc * wrap_plane<NG>(g, pl_ + NG));           \
    }                                                                            \
  } while (0)
  NRR_TILE_FETCH(z0);
  int buf = 0;
  for (int i2 = z0; i2 < z1; i2++, buf ^= 1) {
    // Commit plane i2.  The barrier of the previous iteration ordered every
    // thread's reads of tile[buf] (two planes back) before these writes.
    R *flat_ = &tile[buf][0][0];
#pragma unroll
    for (int k = 0; k < NST; k++)
      if (soff[k] >= 0) flat_[threadIdx.x + k * NT] = sreg[k];
    const R v0 = nv, al = nal, bc = nbc, yb0 = nyb0, yb1 = nyb1, ac0 = nac0,
            ac1 = nac1, fu = nfu;
#pragma unroll
    for (int k = 0; k < 2 * NG; k++) q[k] = q[k + 1];
    q[2 * NG] = nq;
    __syncthreads();
    if (i2 + 1 < z1) NRR_TILE_FETCH(i2 + 1);
    if (active) {
      const int64_t p = col + (int64_t)nc * i2;
      const R(&t)[TH][TW] = tile[buf];
      const R u0 = t[ty + NG][tx + NG];
      R a0 = w[0] * u0;
#pragma unroll
      for (int k = 1; k <= NG; k++) {
        a0 = fma(w[k], t[ty + NG][tx + NG + k], a0);
        a0 = fma(w[NG + k], t[ty + NG][tx + NG - k], a0);
      }
#pragma unroll
      for (int k = 1; k <= NG; k++) {
        a0 = fma(w[2 * NG + k], t[ty + NG + k][tx + NG], a0);
        a0 = fma(w[3 * NG + k], t[ty + NG - k][tx + NG], a0);
      }
#pragma unroll
      for (int k = 1; k <= NG; k++) a0 = fma(w[4 * NG + k], q[NG + k] + q[NG - k], a0);
      const R kv = add_source(a0, u0, al, bc, a.lin);
      R ku = fma(-a.eta, u0, v0);
      if (linear_mode<R>(a.lin)) ku += fu;
      if (KIND == STAGE_FIRST) {
        st(a.au + p, fma(a.wb, ku, yb0));
        st(a.av + p, fma(a.wb, kv, yb1));
        st(a.ou + p, fma(a.wa, ku, yb0));
        st(a.ov + p, fma(a.wa, kv, yb1));
      } else if (KIND == STAGE_MID) {
        st(a.au + p, fma(a.wb, ku, ac0));
        st(a.av + p, fma(a.wb, kv, ac1));
        st(a.ou + p, fma(a.wa, ku, yb0));
        st(a.ov + p, fma(a.wa, kv, yb1));
      } else if (KIND == STAGE_LAST) {
        st(a.ou + p, fma(a.wb, ku, ac0));
        st(a.ov + p, fma(a.wb, kv, ac1));
      } else {
        st(a.ou + p, ku);
        st(a.ov + p, kv);
      }
    }
  }
#undef NRR_TILE_FETCH
}


// ---------------------------------------------------------------------------
// TMA-fed tiled stage (same work split as stage_tile_block, order 8): the
// planes of a block's chunk stream, PZ at a time, through a ring of NS
// shared-memory slots, each filled by tiled tensor copies -- one
// (32 + 2 NG) x (TY + 2 NG) x PZ box of u with its halo and one 32 x TY x PZ
// box per operand array -- that complete on the slot's mbarrier.  One
// thread fills all NS slots at the start and refills each as soon as the
// block has finished reading it (maps: ArenaSrc or FieldSrc).  Each
// thread evaluates PZ points of its column per slot; it fetches only the
// inner-boundary image cells itself, one slot ahead, overwriting the box's
// unmaintained ghost cells.  Requires n0 % 32 == 0, n1 % TY == 0 and the
// chunk's plane count a multiple of PZ (checked on the host).  In the FIRST
// stage the base state is the input state (bu == su, bv == sv).
// ---------------------------------------------------------------------------
// Where the tensor copies come from.  ArenaSrc: one pair of 4-D maps
// (i0, i1, i2, field) per solve over a precision's field arena, the field
// index being the 4th coordinate (batches).  FieldSrc: one 3-D map per array
// (single grids); it must stay a __grid_constant__ kernel parameter, since a
// tensor copy names its map by address.
struct ArenaSrc {
  const CUtensorMap *map_u;   // box (32 + 2 NG, TY + 2 NG, PZ, 1)
  const CUtensorMap *map_op;  // box (32, TY, PZ, 1)
  const void *base;           // field 0 of this solve in the arena
  int64_t stride;             // elements between consecutive fields
  // (p - base) is a whole number f of fields, f at most a few dozen: the
  // FP32 quotient is within about 2e-7 f of f (three roundings of 2^-24),
  // so rounding recovers f exactly without a 64-bit integer division.
  template <typename R>
  __device__ __forceinline__ int field(const R *p) const {
    return __float2int_rn((float)(p - static_cast<const R *>(base)) / (float)stride);
  }
  __device__ __forceinline__ void load_u(void *dst, uint64_t *bar, int x, int y,
                                         int z, int f) const {
    tma_load_4d(dst, map_u, bar, x, y, z, f);
  }
  __device__ __forceinline__ void load_op(int, void *dst, uint64_t *bar, int x,
                                          int y, int z, int f) const {
    tma_load_4d(dst, map_op, bar, x, y, z, f);
  }
  // u without halo (the planes entering the phi queue): the operand box of
  // the u field
  __device__ __forceinline__ void load_ph(void *dst, uint64_t *bar, int x, int y,
                                          int z, int f) const {
    tma_load_4d(dst, map_op, bar, x, y, z, f);
  }
};
struct FieldSrc {
  CUtensorMap u;      // su, box (32 + 2 NG, TY + 2 NG, PZ)
  CUtensorMap op[8];  // operand arrays by TmaOp slot, box (32, TY, PZ)
  CUtensorMap ph;     // su, box (32, TY, PZ): planes entering the phi queue
  template <typename R>
  __device__ __forceinline__ int field(const R *) const { return 0; }
  __device__ __forceinline__ void load_u(void *dst, uint64_t *bar, int x, int y,
                                         int z, int) const {
    tma_load_3d(dst, &u, bar, x, y, z);
  }
  __device__ __forceinline__ void load_op(int o, void *dst, uint64_t *bar, int x,
                                          int y, int z, int) const {
    tma_load_3d(dst, &op[o], bar, x, y, z);
  }
  __device__ __forceinline__ void load_ph(void *dst, uint64_t *bar, int x, int y,
                                          int z, int) const {
    tma_load_3d(dst, &ph, bar, x, y, z);
  }
};

// One ring slot.  Every member is a tensor-copy destination and starts on a
// 128-byte boundary (checked where the ring is used).  PH: the slot also
// carries, without halo, the PZ planes of u that enter the phi queue (NG
// planes ahead of the slot's own), so that no thread loads them itself.
template <typename R, int NG, int TY, int PZ, bool PH = false>
struct TmaSlot {
  R u[PZ][TY + 2 * NG][32 + 2 * NG];  // PZ planes of u with halo
  R op[8][PZ][TY][32];                // operand rows, slots below
};
template <typename R, int NG, int TY, int PZ>
struct TmaSlot<R, NG, TY, PZ, true> {
  R u[PZ][TY + 2 * NG][32 + 2 * NG];
  R op[8][PZ][TY][32];
  R ph[PZ][TY][32];  // phi-queue planes of u, no halo
};
// Shared-memory destinations of tensor copies: 128-byte aligned slots and
// members, so that a ring of slots keeps every copy aligned.
template <typename R, int NG, int TY, int PZ, bool PH>
constexpr bool tma_slot_aligned() {
  return sizeof(TmaSlot<R, NG, TY, PZ, PH>) % 128 == 0 &&
         (PZ * (TY + 2 * NG) * (32 + 2 * NG) * sizeof(R)) % 128 == 0 &&
         (PZ * TY * 32 * sizeof(R)) % 128 == 0;
}
enum TmaOp { OP_SV = 0, OP_AL, OP_BC, OP_FU, OP_BU, OP_BV, OP_AU, OP_AV };

template <typename R, int NG, int KIND, int TY, int NS, int PZ, typename Src,
          bool COH = false, bool PH = false>
__device__ __forceinline__ void stage_tma_block(const Geo &g, const StageArgs<R> &a,
                                                 int tile_x, int tile_y, int chunk,
                                                 int zc, const Src &src,
                                                 TmaSlot<R, NG, TY, PZ, PH> *ring,
                                                 uint64_t *full, int *err) {
  // With PH the phi box of a slot (planes i2 + NG .. i2 + NG + PZ - 1,
  // wrapped) must not straddle the periodic seam: PZ == 2 with even NG, even
  // n2 and slots starting on even local planes keep it whole.
  static_assert(!PH || (PZ == 2 && NG % 2 == 0), "phi box needs PZ 2, even NG");
  static_assert(tma_slot_aligned<R, NG, TY, PZ, PH>(),
                "tensor-copy destinations must start on 128-byte boundaries");
  static_assert((NG * sizeof(R)) % 16 == 0,
                "operand boxes start at x = NG: 16-byte aligned");
  constexpr int TW = 32 + 2 * NG, TH = TY + 2 * NG;
  constexpr int NT = 32 * TY;
  constexpr int NST = (TW * TH + NT - 1) / NT;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int nc = g.ncol;
  const int z0 = NG + chunk * zc;
  const int z1 = min(z0 + zc, NG + g.n2);
  const int i1 = NG + tile_y * TY + ty;
  if (tile_x == tiles_x(g)) {
    stage_shell_rows<R, NG, KIND, COH>(g, a, tx, i1, z0, z1);
    return;
  }
  const int nslots = (z1 - z0) / PZ;
  const int i0 = NG + tile_x * 32 + tx;
  const int col = i0 + g.s0 * i1;
  const int j0b = tile_x * 32, j1b = tile_y * TY;
  const bool use_fu = linear_mode<R>(a.lin);
  constexpr bool use_b = KIND == STAGE_MID;
  constexpr bool use_acc = KIND == STAGE_MID || KIND == STAGE_LAST;
  // Image cells of this thread (tile cells whose source is not the cell
  // itself): offset of the image in its plane and whether it lies on the
  // plane phi + pi; -1 for the other cells.
  int soff[NST];
  unsigned flip = 0;
  bool has_img = false;
#pragma unroll
  for (int k = 0; k < NST; k++) {
    const int cidx = threadIdx.x + k * NT;
    soff[k] = -1;
    if (cidx < TW * TH) {
      const int cy = cidx / TW, cx = cidx - cy * TW;
      int j0 = j0b + cx, j1 = j1b + cy;
      if (j0 < NG || j1 < NG || j1 >= g.n1 + NG) {
        unsigned f = 0;
        if (j0 < NG) {
          j0 = 2 * NG - 1 - j0;
          f = 1;
          if (spherical_like(g.coord)) j1 = g.n1 + 2 * NG - 1 - j1;
        }
        if (j1 < NG) {
          j1 = 2 * NG - 1 - j1;
          f ^= 1;
        } else if (j1 >= g.n1 + NG) {
          j1 = 2 * g.n1 + 2 * NG - 1 - j1;
          f ^= 1;
        }
        soff[k] = j0 + g.s0 * j1;
        flip |= f << k;
        has_img = true;
      }
    }
  }
  if (threadIdx.x == 0) {
    for (int k = 0; k < NS; k++) mbar_init_count(&full[k], 1);
    mbar_init_fence();
  }
  __syncthreads();
  pdl_wait();
  // Operands this stage reads (slot mask) and their field indices (the 4th
  // tensor coordinate); thread 0 issues every copy.
  const unsigned opmask = (1u << OP_SV) | (1u << OP_AL) | (1u << OP_BC) |
                          (use_fu ? 1u << OP_FU : 0u) |
                          (use_b ? (1u << OP_BU) | (1u << OP_BV) : 0u) |
                          (use_acc ? (1u << OP_AU) | (1u << OP_AV) : 0u);
  const uint32_t slot_bytes =
      (uint32_t)(PZ * (TW * TH + (__popc(opmask) + (PH ? 1 : 0)) * TY * 32) * sizeof(R));
  // Source coordinate (field index for an arena) of u (fidx[8]) and of
  // each operand: thread 0 only.
  int fidx[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  auto issue = [&](int pl, int sl) {
    mbar_arrive_expect(&full[sl], slot_bytes);
    fence_proxy_async_smem();
    src.load_u(&ring[sl].u[0][0][0], &full[sl], j0b, j1b, pl, fidx[8]);
#pragma unroll
    for (int o = 0; o < 8; o++)
      if ((opmask >> o) & 1u)
        src.load_op(o, &ring[sl].op[o][0][0][0], &full[sl], NG + j0b, NG + j1b,
                    pl, fidx[o]);
    if constexpr (PH)
      src.load_ph(&ring[sl].ph[0][0][0], &full[sl], NG + j0b, NG + j1b,
                  wrap_plane<NG>(g, pl + NG), fidx[8]);
  };
  if (threadIdx.x == 0) {
    const R *optr[8] = {a.sv, a.alpha, a.bc2, a.fu, a.bu, a.bv, a.au, a.av};
#pragma unroll
    for (int o = 0; o < 8; o++)
      if ((opmask >> o) & 1u) fidx[o] = src.field(optr[o]);
    fidx[8] = src.field(a.su);
    for (int k = 0; k < NS && k < nslots; k++) issue(z0 + PZ * k, k);
  }
  // The column's folded weights are loaded while the first copies are in
  // flight: a block that starts after the preceding stage has finished
  // would otherwise wait for them before issuing any copy.  Plain loads, so
  // that the compiler keeps them behind the copies.
  R w[5 * NG + 1];
#pragma unroll
  for (int j = 0; j < 5 * NG + 1; j++) w[j] = ld(a.col.coef + (int64_t)j * nc + col);
  // phi queue of this column (planes i2 - NG .. i2 + NG of the slot's first
  // plane i2) and the image cells of the next slot
  R q[2 * NG + PZ];
#pragma unroll
  for (int k = 0; k < 2 * NG; k++)
    q[k + PZ] = lds<COH>(a.su + col + (int64_t)nc * wrap_plane<NG>(g, z0 - NG + k));
  R nq[PZ];
  if constexpr (!PH) {
#pragma unroll
    for (int j = 0; j < PZ; j++)
      nq[j] = lds<COH>(a.su + col + (int64_t)nc * wrap_plane<NG>(g, z0 + NG + j));
  }
  R ireg[PZ][NST];
  auto fetch_images = [&](int pl) {
    if (!has_img) return;
#pragma unroll
    for (int j = 0; j < PZ; j++) {
      const R *base = a.su + (int64_t)nc * (pl + j);
      const R *bflip = a.su + (int64_t)nc * wrap_plane<NG>(g, pl + j + g.n2 / 2);
#pragma unroll
      for (int k = 0; k < NST; k++)
        if (soff[k] >= 0) ireg[j][k] = lds<COH>(((flip >> k) & 1u ? bflip : base) + soff[k]);
    }
  };
  fetch_images(z0);
  // The loop runs over rounds of NS slots, unrolled, so that slot indices
  // and addresses are compile-time constants; `phase` is the parity of the
  // round's barrier phases.
  for (int base = 0, phase = 0; base < nslots; base += NS, phase ^= 1) {
#pragma unroll
    for (int sl = 0; sl < NS; sl++) {
      const int it = base + sl;
      if (it >= nslots) break;
      const int i2 = z0 + PZ * it;
      const bool ok = mbar_wait_parity(&full[sl], (uint32_t)phase);
      TmaSlot<R, NG, TY, PZ, PH> &S = ring[sl];
      if (has_img) {
#pragma unroll
        for (int j = 0; j < PZ; j++) {
          R *flat_u = &S.u[j][0][0];
#pragma unroll
          for (int k = 0; k < NST; k++)
            if (soff[k] >= 0) flat_u[threadIdx.x + k * NT] = ireg[j][k];
        }
        // these cells are refilled by tensor copies when the slot comes round
        fence_proxy_async_smem();
      }
#pragma unroll
      for (int k = 0; k < 2 * NG; k++) q[k] = q[k + PZ];
      if constexpr (PH) {
#pragma unroll
        for (int j = 0; j < PZ; j++) q[2 * NG + j] = S.ph[j][ty][tx];
      } else {
#pragma unroll
        for (int j = 0; j < PZ; j++) q[2 * NG + j] = nq[j];
      }
      if (__syncthreads_or(!ok)) {
        // A copy did not complete in time: record it, let the copies still in
        // flight (slots it .. it + NS - 1) land, bounded, and leave.
        if (threadIdx.x == 0) {
          atomicExch(err, 1);
          for (int j = it; j < nslots && j < it + NS; j++)
            mbar_wait_parity(&full[j % NS], (uint32_t)((j / NS) & 1));
        }
        __syncthreads();
        return;
      }
      if (it + 1 < nslots) {
        fetch_images(i2 + PZ);
        if constexpr (!PH) {
#pragma unroll
          for (int j = 0; j < PZ; j++)
            nq[j] = lds<COH>(a.su + col + (int64_t)nc * wrap_plane<NG>(g, i2 + PZ + NG + j));
        }
      }
#pragma unroll
      for (int j = 0; j < PZ; j++) {
        const int64_t p = col + (int64_t)nc * (i2 + j);
        const R(&t)[TH][TW] = S.u[j];
        const R u0 = t[ty + NG][tx + NG];
        const R v0 = S.op[OP_SV][j][ty][tx], al = S.op[OP_AL][j][ty][tx],
                bc = S.op[OP_BC][j][ty][tx];
        R a0 = w[0] * u0;
#pragma unroll
        for (int k = 1; k <= NG; k++) {
          a0 = fma(w[k], t[ty + NG][tx + NG + k], a0);
          a0 = fma(w[NG + k], t[ty + NG][tx + NG - k], a0);
        }
#pragma unroll
        for (int k = 1; k <= NG; k++) {
          a0 = fma(w[2 * NG + k], t[ty + NG + k][tx + NG], a0);
          a0 = fma(w[3 * NG + k], t[ty + NG - k][tx + NG], a0);
        }
        // q[NG + j] is the centre plane i2 + j
#pragma unroll
        for (int k = 1; k <= NG; k++)
          a0 = fma(w[4 * NG + k], q[NG + j + k] + q[NG + j - k], a0);
        const R kv = add_source(a0, u0, al, bc, a.lin);
        R ku = fma(-a.eta, u0, v0);
        if (use_fu) ku += S.op[OP_FU][j][ty][tx];
        if (KIND == STAGE_FIRST) {
          st(a.au + p, fma(a.wb, ku, u0));
          st(a.av + p, fma(a.wb, kv, v0));
          st(a.ou + p, fma(a.wa, ku, u0));
          st(a.ov + p, fma(a.wa, kv, v0));
        } else if (KIND == STAGE_MID) {
          st(a.au + p, fma(a.wb, ku, S.op[OP_AU][j][ty][tx]));
          st(a.av + p, fma(a.wb, kv, S.op[OP_AV][j][ty][tx]));
          st(a.ou + p, fma(a.wa, ku, S.op[OP_BU][j][ty][tx]));
          st(a.ov + p, fma(a.wa, kv, S.op[OP_BV][j][ty][tx]));
        } else if (KIND == STAGE_LAST) {
          st(a.ou + p, fma(a.wb, ku, S.op[OP_AU][j][ty][tx]));
          st(a.ov + p, fma(a.wb, kv, S.op[OP_AV][j][ty][tx]));
        } else {
          st(a.ou + p, ku);
          st(a.ov + p, kv);
        }
      }
      // Refill this slot as soon as every thread is done with it, so that
      // NS copies are in flight while the block waits for the next one.
      if (it + NS < nslots) {
        __syncthreads();
        if (threadIdx.x == 0) issue(i2 + PZ * NS, sl);
      }
    }
  }
}

}  // namespace dev
}  // namespace nrr
