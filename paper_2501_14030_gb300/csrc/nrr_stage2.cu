// nrr_stage2.cu -- two RK4 stages per launch for small FP32 grids (stage
// variant 6; arXiv 2501.14030 Alg. 1's RHS -> BC -> RK substeps, two of them
// fused in time).
//
// At 128x128x16 and below an FP32 stage takes a few microseconds, a large
// part of it launch ramp and latency rather than data movement.  Here one
// block owns a 32 x 4 tile of (i0, i1) columns with every phi plane of the
// grid, so that the phi + pi images of the inner boundary and the periodic
// phi neighbours stay inside the block, and evaluates two consecutive RK4
// stages:
//   stage A on the tile and a halo of NG columns on each side (region R1),
//     from the stage input staged with a halo of 2 NG (region R0) in shared
//     memory; its output stays in shared memory, and R1's inner-boundary
//     ghost cells copy their images, which lie inside R1;
//   stage B on the tile (and, for the last tile of a row, the outer-shell
//     columns of its rows) from stage A's output.
// Launch 0 fuses stages 1 and 2 (FIRST + MID) and writes the accumulator and
// the second stage's output; launch 1 fuses stages 3 and 4 (MID + LAST).
// Launch 1 reads the base state y in its halo while other blocks finish the
// step: its new state goes to the other state buffer, so the state alternates
// between two buffers from step to step (an even number of steps returns it
// to the first).  Every point is evaluated by the same arithmetic, in the
// same order, as the per-stage kernels, so the results are bitwise equal.
//
// Eligible grids: SinhSymTP, FD order 8, n0 % 32 == 0, n1 % 4 == 0,
// n2 <= 16 (shared memory holds every plane).
#include <cuda_runtime.h>

#include "nrr_internal.h"
#include "nrr_stencil.cuh"

namespace nrr {

namespace {

using namespace dev;

constexpr int NG2 = 4;                    // FD order 8
constexpr int TY2 = 4;                    // tile rows
constexpr int TX2 = 32;                   // tile columns
constexpr int NZ2 = 16;                   // most phi planes
constexpr int R1W = TX2 + 2 * NG2, R1H = TY2 + 2 * NG2;  // 40 x 12
constexpr int R0W = TX2 + 4 * NG2, R0H = TY2 + 4 * NG2;  // 48 x 20
constexpr int BW = TX2 + NG2;             // stage-B columns incl. the shell
constexpr int NT2 = 512;                  // threads per block
constexpr int NCO = 5 * NG2 + 1;          // folded weights per column

// Arguments of one fused launch.
struct Stage2Args {
  const float *in_u, *in_v;    // stage A input (launch 0: y; launch 1: t)
  const float *yu, *yv;        // base state y
  float *au, *av;              // accumulator
  float *ou, *ov;              // launch 0: t; launch 1: the new state
  const float *alpha, *bc2, *fu;
  ColumnSet<float> col;
  float eta;
  float waA, wbA, waB, wbB;    // a_s dt and b_s dt of stages A and B
  int lin;
};

// Shared memory of one block (floats), for nz planes:
//   U0[nz][R0H][R0W]     stage A's input u with halo 2 NG
//   S1[2][nz][R1H][R1W]  stage A's output (u, v) with halo NG
//   AC[2][nz][TY2][BW]   accumulator after stage A at stage B's cells
//   WB[NCO][TY2][BW]     folded weights of stage B's columns
__host__ __device__ constexpr int smem_floats(int nz) {
  return nz * R0H * R0W + 2 * nz * R1H * R1W + 2 * nz * TY2 * BW + NCO * TY2 * BW;
}

__device__ __forceinline__ bool evolved_col(const Geo &g, int j0, int j1) {
  return j0 >= NG2 && j0 < g.n0 + 2 * NG2 && j1 >= NG2 && j1 < g.n1 + NG2;
}

// Image of padded cell (j0, j1) on plane offset flip (SinhSymTP rules: xx0 <
// 0 -> (-xx0, th, ph + pi); th < 0 or th > pi -> reflected, ph + pi).
__device__ __forceinline__ void image2(const Geo &g, int &j0, int &j1, int &flip) {
  flip = 0;
  if (j0 < NG2) {
    j0 = 2 * NG2 - 1 - j0;
    flip ^= 1;
  }
  if (j1 < NG2) {
    j1 = 2 * NG2 - 1 - j1;
    flip ^= 1;
  } else if (j1 >= g.n1 + NG2) {
    j1 = 2 * g.n1 + 2 * NG2 - 1 - j1;
    flip ^= 1;
  }
}

// Local plane index in [0, nz) (the stencil reaches NG planes, more than one
// period when nz < NG).
__device__ __forceinline__ int zwrap(int z, int nz) {
  while (z < 0) z += nz;
  while (z >= nz) z -= nz;
  return z;
}

template <int PAIR>
__global__ void __launch_bounds__(NT2, 1)
    stage2_kernel(Geo g, Stage2Args a) {
  extern __shared__ __align__(16) float sm2[];
  pdl_trigger();
  const int nz = g.n2;
  float *U0 = sm2;
  float *S1 = U0 + nz * R0H * R0W;
  float *AC = S1 + 2 * nz * R1H * R1W;
  float *WB = AC + 2 * nz * TY2 * BW;
  const int t = threadIdx.x;
  const int c0 = NG2 + blockIdx.x * TX2, c1 = NG2 + blockIdx.y * TY2;  // tile origin
  const bool last_x = c0 + TX2 == g.n0 + NG2;  // this tile's rows own the shell
  const int nc = g.ncol;
  // ---- solve-constant data first (before the wait)
  // stage A: thread t < R1W * R1H owns R1 column (t % R1W, t / R1W)
  const int a_x = t % R1W, a_y = t / R1W;
  const int aj0 = c0 - NG2 + a_x, aj1 = c1 - NG2 + a_y;
  const bool a_act = t < R1W * R1H && evolved_col(g, aj0, aj1);
  const bool a_shell = aj0 >= g.n0 + NG2;
  const int acol = aj0 + g.s0 * aj1;
  float wA[NCO];
  float sc = 0.f, skdb = 0.f, srinv = 0.f;
  if (a_act) {
    if (a_shell) {
      sc = ldc(a.col.somm + acol);
      skdb = ldc(a.col.somm + nc + acol);
      srinv = ldc(a.col.somm + 2 * nc + acol);
    } else {
#pragma unroll
      for (int j = 0; j < NCO; j++) wA[j] = ldc(a.col.coef + (int64_t)j * nc + acol);
    }
  }
  // stage B's weights into shared memory
  for (int i = t; i < NCO * TY2 * BW; i += NT2) {
    const int j = i / (TY2 * BW), r = (i / BW) % TY2, x = i % BW;
    const int j0 = c0 + x, j1 = c1 + r;
    WB[i] = x < TX2 ? ldc(a.col.coef + (int64_t)j * nc + j0 + g.s0 * j1) : 0.f;
  }
  pdl_wait();
  // ---- U0: the stage input u over R0 (images for inner-boundary cells);
  // unrolled so that several loads are in flight before their stores
#pragma unroll 8
  for (int i = t; i < nz * R0H * R0W; i += NT2) {
    const int z = i / (R0H * R0W), r = (i / R0W) % R0H, x = i % R0W;
    int j0 = c0 - 2 * NG2 + x, j1 = c1 - 2 * NG2 + r, flip;
    if (j0 < 0 || j1 < 0 || j0 >= g.s0 || j1 >= g.s1) continue;  // never read
    image2(g, j0, j1, flip);
    const int zz = flip ? zwrap(z + nz / 2, nz) : z;
    U0[i] = ld(a.in_u + j0 + (int64_t)g.s0 * j1 + (int64_t)nc * (zz + NG2));
  }
  __syncthreads();
  // ---- stage A over R1's evolved columns, every plane
  if (a_act) {
    const int ux = a_x + NG2, uy = a_y + NG2;  // position in U0
#pragma unroll 4
    for (int z = 0; z < nz; z++) {
      const int64_t p = acol + (int64_t)nc * (z + NG2);
      const float *Uz = U0 + z * R0H * R0W;
      const float u0 = Uz[uy * R0W + ux];
      const float v0 = ld(a.in_v + p);
      const float yb0 = PAIR == 0 ? u0 : ld(a.yu + p);
      const float yb1 = PAIR == 0 ? v0 : ld(a.yv + p);
      float ku, kv;
      if (a_shell) {
        const float u1 = Uz[uy * R0W + ux - 1], u2 = Uz[uy * R0W + ux - 2];
        const float v1 = ld(a.in_v + p - 1), v2 = ld(a.in_v + p - 2);
        ku = -sc * fmaf(skdb, fmaf(3.f, u0, fmaf(-4.f, u1, u2)), srinv * u0);
        kv = -sc * fmaf(skdb, fmaf(3.f, v0, fmaf(-4.f, v1, v2)), srinv * v0);
        if (linear_mode<float>(a.lin)) {
          ku += ld(a.fu + p);
          kv += ld(a.bc2 + p);
        }
      } else {
        float a0 = wA[0] * u0;
#pragma unroll
        for (int k = 1; k <= NG2; k++) {
          a0 = fmaf(wA[k], Uz[uy * R0W + ux + k], a0);
          a0 = fmaf(wA[NG2 + k], Uz[uy * R0W + ux - k], a0);
        }
#pragma unroll
        for (int k = 1; k <= NG2; k++) {
          a0 = fmaf(wA[2 * NG2 + k], Uz[(uy + k) * R0W + ux], a0);
          a0 = fmaf(wA[3 * NG2 + k], Uz[(uy - k) * R0W + ux], a0);
        }
#pragma unroll
        for (int k = 1; k <= NG2; k++) {
          const float sp = U0[zwrap(z + k, nz) * R0H * R0W + uy * R0W + ux];
          const float sm = U0[zwrap(z - k, nz) * R0H * R0W + uy * R0W + ux];
          a0 = fmaf(wA[4 * NG2 + k], sp + sm, a0);
        }
        kv = add_source(a0, u0, ld(a.alpha + p), ld(a.bc2 + p), a.lin);
        ku = fmaf(-a.eta, u0, v0);
        if (linear_mode<float>(a.lin)) ku += ld(a.fu + p);
      }
      float *S1z = S1 + z * R1H * R1W + a_y * R1W + a_x;
      S1z[0] = fmaf(a.waA, ku, yb0);
      S1z[nz * R1H * R1W] = fmaf(a.waA, kv, yb1);
      // the accumulator at stage B's cells (tile columns and, for the last
      // tile of a row, the shell columns)
      const int bx = aj0 - c0, by = aj1 - c1;
      if (bx >= 0 && bx < BW && by >= 0 && by < TY2 && (bx < TX2 || last_x)) {
        const float accu = PAIR == 0 ? yb0 : ld(a.au + p);
        const float accv = PAIR == 0 ? yb1 : ld(a.av + p);
        float *ACz = AC + z * TY2 * BW + by * BW + bx;
        ACz[0] = fmaf(a.wbA, ku, accu);
        ACz[nz * TY2 * BW] = fmaf(a.wbA, kv, accv);
      }
    }
  }
  __syncthreads();
  // ---- R1's inner-boundary ghost cells copy their images (inside R1)
  for (int i = t; i < nz * R1H * R1W; i += NT2) {
    const int z = i / (R1H * R1W), r = (i / R1W) % R1H, x = i % R1W;
    int j0 = c0 - NG2 + x, j1 = c1 - NG2 + r, flip;
    if (j0 < 0 || j1 < 0 || j0 >= g.s0 || j1 >= g.s1) continue;
    if (j0 >= NG2 && j1 >= NG2 && j1 < g.n1 + NG2) continue;  // evolved
    image2(g, j0, j1, flip);
    const int src = (flip ? zwrap(z + nz / 2, nz) : z) * R1H * R1W +
                    (j1 - (c1 - NG2)) * R1W + (j0 - (c0 - NG2));
    S1[i] = S1[src];
    S1[i + nz * R1H * R1W] = S1[src + nz * R1H * R1W];
  }
  __syncthreads();
  // ---- stage B at the tile's cells (and the shell columns of the last tile)
  const int nbx = last_x ? BW : TX2;
#pragma unroll 4
  for (int i = t; i < nz * TY2 * nbx; i += NT2) {
    const int z = i / (TY2 * nbx), by = (i / nbx) % TY2, bx = i % nbx;
    const int j0 = c0 + bx, j1 = c1 + by;
    const int64_t p = j0 + (int64_t)g.s0 * j1 + (int64_t)nc * (z + NG2);
    const float *S1z = S1 + z * R1H * R1W;
    const int sx = bx + NG2, sy = by + NG2;
    const float u0 = S1z[sy * R1W + sx];
    const float v0 = S1z[nz * R1H * R1W + sy * R1W + sx];
    float ku, kv;
    if (bx >= TX2) {
      const int col = j0 + g.s0 * j1;
      const float c = ldc(a.col.somm + col), kdb = ldc(a.col.somm + nc + col),
                  rinv = ldc(a.col.somm + 2 * nc + col);
      const float u1 = S1z[sy * R1W + sx - 1], u2 = S1z[sy * R1W + sx - 2];
      const float v1 = S1z[nz * R1H * R1W + sy * R1W + sx - 1],
                  v2 = S1z[nz * R1H * R1W + sy * R1W + sx - 2];
      ku = -c * fmaf(kdb, fmaf(3.f, u0, fmaf(-4.f, u1, u2)), rinv * u0);
      kv = -c * fmaf(kdb, fmaf(3.f, v0, fmaf(-4.f, v1, v2)), rinv * v0);
      if (linear_mode<float>(a.lin)) {
        ku += ld(a.fu + p);
        kv += ld(a.bc2 + p);
      }
    } else {
      const float *w = WB + by * BW + bx;  // weight j at w[j * TY2 * BW]
      float a0 = w[0] * u0;
#pragma unroll
      for (int k = 1; k <= NG2; k++) {
        a0 = fmaf(w[k * TY2 * BW], S1z[sy * R1W + sx + k], a0);
        a0 = fmaf(w[(NG2 + k) * TY2 * BW], S1z[sy * R1W + sx - k], a0);
      }
#pragma unroll
      for (int k = 1; k <= NG2; k++) {
        a0 = fmaf(w[(2 * NG2 + k) * TY2 * BW], S1z[(sy + k) * R1W + sx], a0);
        a0 = fmaf(w[(3 * NG2 + k) * TY2 * BW], S1z[(sy - k) * R1W + sx], a0);
      }
#pragma unroll
      for (int k = 1; k <= NG2; k++) {
        const float sp = S1[zwrap(z + k, nz) * R1H * R1W + sy * R1W + sx];
        const float sm = S1[zwrap(z - k, nz) * R1H * R1W + sy * R1W + sx];
        a0 = fmaf(w[(4 * NG2 + k) * TY2 * BW], sp + sm, a0);
      }
      kv = add_source(a0, u0, ld(a.alpha + p), ld(a.bc2 + p), a.lin);
      ku = fmaf(-a.eta, u0, v0);
      if (linear_mode<float>(a.lin)) ku += ld(a.fu + p);
    }
    const float *ACz = AC + z * TY2 * BW + by * BW + bx;
    const float acu = ACz[0], acv = ACz[nz * TY2 * BW];
    if (PAIR == 0) {
      // stage 2 (MID): accumulator and its output t
      st(a.au + p, fmaf(a.wbB, ku, acu));
      st(a.av + p, fmaf(a.wbB, kv, acv));
      st(a.ou + p, fmaf(a.waB, ku, ld(a.yu + p)));
      st(a.ov + p, fmaf(a.waB, kv, ld(a.yv + p)));
    } else {
      // stage 4 (LAST): the new state
      st(a.ou + p, fmaf(a.wbB, ku, acu));
      st(a.ov + p, fmaf(a.wbB, kv, acv));
    }
  }
}

}  // namespace

bool stage2_ok(const Geo &g) {
  return g.coord == SINHSYMTP && g.ng == NG2 && g.n0 % TX2 == 0 && g.n1 % TY2 == 0 &&
         g.n2 <= NZ2 && g.n2 >= 2 && g.n2 % 2 == 0;
}

cudaError_t launch_stage2_steps(const Geo &g, const FieldSet<float> &f,
                                const ColumnSet<float> &c, double dt, double eta,
                                int64_t steps, int pdl, cudaStream_t st) {
  const size_t smem = (size_t)smem_floats(g.n2) * sizeof(float);
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(stage2_kernel<0>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(smem_floats(NZ2) * sizeof(float)));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(stage2_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(smem_floats(NZ2) * sizeof(float)));
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const dim3 grid(g.n0 / TX2, g.n1 / TY2);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(NT2);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl ? 1 : 0;
  Stage2Args a{};
  a.alpha = f.alpha;
  a.bc2 = f.bc2;
  a.fu = f.fu;
  a.col = c;
  a.eta = (float)eta;
  a.lin = f.lin;
  for (int64_t s = 0; s < steps; s++) {
    // the state alternates between the y and s buffers
    float *yu = (s & 1) ? f.s[0] : f.y[0], *yv = (s & 1) ? f.s[1] : f.y[1];
    float *nu = (s & 1) ? f.y[0] : f.s[0], *nv = (s & 1) ? f.y[1] : f.s[1];
    // stages 1 and 2: y -> accumulator, t
    a.in_u = yu, a.in_v = yv, a.yu = yu, a.yv = yv;
    a.au = f.a[0], a.av = f.a[1];
    a.ou = f.t[0], a.ov = f.t[1];
    a.waA = (float)(0.5 * dt), a.wbA = (float)(dt / 6.0);
    a.waB = (float)(0.5 * dt), a.wbB = (float)(dt / 3.0);
    cudaError_t e = cudaLaunchKernelEx(&cfg, stage2_kernel<0>, g, a);
    if (e != cudaSuccess) return e;
    // stages 3 and 4: t, y, accumulator -> the new state
    a.in_u = f.t[0], a.in_v = f.t[1];
    a.ou = nu, a.ov = nv;
    a.waA = (float)dt, a.wbA = (float)(dt / 3.0);
    a.waB = 0.f, a.wbB = (float)(dt / 6.0);
    e = cudaLaunchKernelEx(&cfg, stage2_kernel<1>, g, a);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace nrr
