// nrr_mlp.cu -- the warm-start surrogate: a multilayer perceptron from
// puncture parameters to the coarse-grid solution u, trained on the device.
//
// Layers l = 0..L-1: Z_l = A_{l-1} W_l^T + b_l with A_{-1} the (zero-padded)
// inputs; A_l = GELU(Z_l) for the hidden layers, the last layer is linear.
// BF16 operands, FP32 accumulation (tcgen05 GEMM), FP32 master weights,
// AdamW.  The loss is the mean squared error of the normalised outputs.
// Every contraction runs on the tensor-core GEMM in the TN form
// D = A B^T with K-major operands, so each layer keeps its weights in both
// layouts (W^T for the forward and the input gradient, W for ...) and the
// elementwise kernels also write transposed activations for the
// weight-gradient GEMMs.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/nrr.h"
#include "nrr_debug.cuh"
#include "nrr_internal.h"

namespace nrr {
nrr_status gemm_bf16_tn(const void *A, const void *B, float *D, int M, int N,
                        int K, int ldd, cudaStream_t st, char *msg, int msglen,
                        int bn, int splits, float *ws, size_t ws_bytes,
                        int persistent);
nrr_status gemm_check_error(cudaStream_t st, char *msg, int msglen);
void gemm_plan(int M, int N, int K, int *bn, int *splits, int *persistent);
size_t gemm_workspace_bytes(int M, int N, int splits);
}  // namespace nrr

using namespace nrr;
typedef __nv_bfloat16 bf16;

namespace {

nrr_status mfail(nrr_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return s;
}

#define MCUDA(call)                                                        \
  do {                                                                     \
    cudaError_t e_ = (call);                                               \
    if (e_ != cudaSuccess)                                                 \
      return mfail(NRR_ERR_CUDA, "%s: %s (%s:%d)", #call,                  \
                   cudaGetErrorString(e_), __FILE__, __LINE__);            \
  } while (0)
#define MTRY(expr)                \
  do {                            \
    nrr_status s_ = (expr);       \
    if (s_ != NRR_OK) return s_;  \
  } while (0)

// GELU(x) = x Phi(x), Phi the standard normal distribution function.
__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
// d/dx GELU = Phi(x) + x phi(x).
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// Tiled transpose-and-store helper: a 32x32 tile of values v (row r, col c
// of a [rows][cols] matrix) is also written to the [cols][rows] matrix.
// Block 32x8; each thread handles 4 rows of the tile.
template <typename F>
__device__ __forceinline__ void tile_apply(int rows, int cols, F f,
                                           bf16 *out_t) {
  __shared__ bf16 tile[32][33];
  const int c = blockIdx.x * 32 + threadIdx.x;
  for (int k = 0; k < 4; k++) {
    const int r = blockIdx.y * 32 + threadIdx.y + 8 * k;
    bf16 v = __float2bfloat16(0.f);
    if (r < rows && c < cols) v = f(r, c);
    tile[threadIdx.y + 8 * k][threadIdx.x] = v;
  }
  __syncthreads();
  if (!out_t) return;
  const int rt = blockIdx.x * 32 + threadIdx.y;  // row of the transposed
  const int ct = blockIdx.y * 32 + threadIdx.x;
  for (int k = 0; k < 4; k++) {
    const int rr = rt + 8 * k;
    if (rr < cols && ct < rows)
      out_t[(int64_t)rr * rows + ct] = tile[threadIdx.x][threadIdx.y + 8 * k];
  }
}

// Z += b; A = bf16(GELU(Z)) and A^T.
__global__ void bias_gelu_kernel(float *Z, const float *b, bf16 *A, bf16 *At,
                                 int rows, int cols) {
  tile_apply(
      rows, cols,
      [&](int r, int c) {
        float z = Z[(int64_t)r * cols + c] + b[c];
        Z[(int64_t)r * cols + c] = z;
        bf16 a = __float2bfloat16(gelu(z));
        A[(int64_t)r * cols + c] = a;
        return a;
      },
      At);
}

// Last layer: Z += b (FP32 output).
__global__ void bias_kernel(float *Z, const float *b, int rows, int cols) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < (int64_t)rows * cols) Z[i] += b[i % cols];
}

// Mean squared error gradient dZ = 2 (Z - Y) / (rows cols) in FP32 and BF16
// (and its transpose), with per-block partial sums of (Z - Y)^2.
__global__ void mse_grad_kernel(const float *Z, const float *Y, float *dz32,
                                bf16 *dz, bf16 *dzt, int rows, int cols,
                                double *partials) {
  __shared__ double red[256];
  const float scale = 2.0f / ((float)rows * (float)cols);
  double sq = 0.0;
  tile_apply(
      rows, cols,
      [&](int r, int c) {
        const int64_t i = (int64_t)r * cols + c;
        float d = Z[i] - Y[i];
        sq += (double)d * d;
        float g = scale * d;
        dz32[i] = g;
        bf16 gb = __float2bfloat16(g);
        dz[i] = gb;
        return gb;
      },
      dzt);
  const int t = threadIdx.y * 32 + threadIdx.x;
  red[t] = sq;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (t < s) red[t] += red[t + s];
    __syncthreads();
  }
  if (t == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = red[0];
}

// out: the loss slot, or (step != nullptr) the base of a ring of `cap`
// slots indexed by the device step counter.
__global__ void loss_finalize_kernel(const double *partials, int n,
                                     double denom, double *out,
                                     const int64_t *step, int cap) {
  if (step) out += *step % cap;
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += partials[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] / denom;
}

// dZ = dA * GELU'(Z) in FP32 and BF16 (+ transpose).
__global__ void gelu_backward_kernel(const float *dA, const float *Z,
                                     float *dz32, bf16 *dz, bf16 *dzt,
                                     int rows, int cols) {
  tile_apply(
      rows, cols,
      [&](int r, int c) {
        const int64_t i = (int64_t)r * cols + c;
        float g = dA[i] * gelu_grad(Z[i]);
        dz32[i] = g;
        bf16 gb = __float2bfloat16(g);
        dz[i] = gb;
        return gb;
      },
      dzt);
}

// db[c] = sum_r dz[r][c] (fixed order over rows).
__global__ void colsum_kernel(const float *dz, float *db, int rows, int cols) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float s = 0.f;
  for (int r = 0; r < rows; r++) s += dz[(int64_t)r * cols + c];
  db[c] = s;
}

// Minibatch assembly: rows order[0..rows) of X (n_in wide, zero-padded to
// in_pad) as BF16 and transposed BF16; of Y normalised by (mean, std).
// order: the rows of this minibatch, or (step != nullptr) of every
// minibatch, rows * (*step) entries in.
__global__ void gather_inputs_kernel(const float *X, const int32_t *order,
                                     int n_in, int in_pad, int rows,
                                     bf16 *xb, bf16 *xt, const int64_t *step) {
  if (step) order += *step * rows;
  tile_apply(
      rows, in_pad,
      [&](int r, int c) {
        float v = c < n_in ? X[(int64_t)order[r] * n_in + c] : 0.f;
        bf16 b = __float2bfloat16(v);
        xb[(int64_t)r * in_pad + c] = b;
        return b;
      },
      xt);
}
__global__ void gather_targets_kernel(const float *Y, const int32_t *order,
                                      const float *mean, const float *std,
                                      int n_out, int rows, float *yb,
                                      const int64_t *step) {
  if (step) order += *step * rows;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)rows * n_out) return;
  const int r = (int)(i / n_out), c = (int)(i % n_out);
  yb[i] = (Y[(int64_t)order[r] * n_out + c] - mean[c]) / std[c];
}

// out[order[r]][c] = Z[r][c] std[c] + mean[c] for the first `valid` rows.
__global__ void denorm_kernel(const float *Z, const float *mean,
                              const float *std, int n_out, int valid,
                              int64_t row0, float *out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)valid * n_out) return;
  const int c = (int)(i % n_out);
  out[row0 * n_out + i] = Z[i] * std[c] + mean[c];
}

// Per-column mean and standard deviation over n rows (two passes, fixed
// order); std floored at 1e-3 of the largest.
__global__ void column_stats_kernel(const float *Y, int64_t n, int cols,
                                    float *mean, float *std) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  double s = 0.0;
  for (int64_t r = 0; r < n; r++) s += Y[r * cols + c];
  double mu = s / (double)n, q = 0.0;
  for (int64_t r = 0; r < n; r++) {
    double d = Y[r * cols + c] - mu;
    q += d * d;
  }
  mean[c] = (float)mu;
  std[c] = (float)sqrt(q / (double)n);
}
__global__ void std_floor_kernel(float *std, int cols) {
  __shared__ float red[256];
  float m = 0.f;
  for (int c = threadIdx.x; c < cols; c += blockDim.x) m = fmaxf(m, std[c]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if ((int)threadIdx.x < k) red[threadIdx.x] = fmaxf(red[threadIdx.x], red[threadIdx.x + k]);
    __syncthreads();
  }
  const float floor_v = fmaxf(1e-3f * red[0], 1e-30f);
  for (int c = threadIdx.x; c < cols; c += blockDim.x) std[c] = fmaxf(std[c], floor_v);
}

// AdamW step on one layer's weights [dout][din] and biases [dout]; writes
// the BF16 copies W^T ([dout][din]) and W ([din][dout]).
struct AdamArgs {
  float lr, beta1, beta2, eps, wd, c1, c2;  // c1 = 1/(1-beta1^t), c2 likewise
};
// corr (nullable): per-step bias corrections (c1, c2) indexed by the device
// step counter, in place of a.c1 and a.c2.
__global__ void adamw_kernel(float *p, const float *g, float *m, float *v,
                             int64_t n, AdamArgs a, int dout, int din,
                             int is_weight, bf16 *wt, bf16 *w, const float2 *corr,
                             const int64_t *step) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (corr) {
    const float2 c = corr[*step];
    a.c1 = c.x;
    a.c2 = c.y;
  }
  float gi = g[i];
  float mi = a.beta1 * m[i] + (1.f - a.beta1) * gi;
  float vi = a.beta2 * v[i] + (1.f - a.beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  float upd = (mi * a.c1) / (sqrtf(vi * a.c2) + a.eps);
  float pi = p[i];
  if (is_weight) pi -= a.lr * a.wd * pi;
  pi -= a.lr * upd;
  p[i] = pi;
  if (is_weight) {
    bf16 b = __float2bfloat16(pi);
    wt[i] = b;
    const int o = (int)(i / din), k = (int)(i % din);
    w[(int64_t)k * dout + o] = b;
  }
}

__global__ void step_advance_kernel(int64_t *step) { *step += 1; }

// BF16 copies of one layer's weights in both layouts.
__global__ void weights_to_bf16_kernel(const float *p, int dout, int din,
                                       bf16 *wt, bf16 *w) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)dout * din) return;
  bf16 b = __float2bfloat16(p[i]);
  wt[i] = b;
  w[(int64_t)(i % din) * dout + i / din] = b;
}

dim3 tile_grid(int rows, int cols) { return dim3((cols + 31) / 32, (rows + 31) / 32); }

}  // namespace

struct nrr_surrogate {
  int n_in = 0, in_pad = 64, hidden = 0, depth = 0, n_out = 0, batch = 0;
  int L = 0;
  std::vector<int> din, dout;
  std::vector<int64_t> offW, offB;  // internal packed offsets
  int64_t nparam = 0;
  int64_t step = 0;
  int device = 0;
  cudaStream_t stream = nullptr, user_stream = nullptr;
  cudaEvent_t order_ev = nullptr;
  std::vector<void *> allocs;
  float *param = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  std::vector<bf16 *> wt, w;  // per layer BF16 copies
  bf16 *xb = nullptr, *xt = nullptr;
  std::vector<float *> z;
  std::vector<bf16 *> a, at;
  float *da = nullptr, *dz32 = nullptr, *yb = nullptr;
  float *ws = nullptr;  // split-K partial products
  size_t ws_bytes = 0;
  bf16 *dzb = nullptr, *dzt = nullptr;
  float *mean = nullptr, *stdv = nullptr;
  int32_t *order_id = nullptr;  // identity order
  double *partials = nullptr, *loss = nullptr;
  int loss_cap = 0;
};

namespace {

template <typename T>
nrr_status malloc_s(nrr_surrogate *s, T **p, size_t count) {
  void *ptr = nullptr;
  cudaError_t e = cudaMalloc(&ptr, std::max<size_t>(count, 1) * sizeof(T));
  if (e != cudaSuccess)
    return mfail(NRR_ERR_OOM, "cudaMalloc of %zu bytes: %s", count * sizeof(T),
                 cudaGetErrorString(e));
  s->allocs.push_back(ptr);
  dbg_register(ptr, std::max<size_t>(count, 1) * sizeof(T));
  *p = static_cast<T *>(ptr);
  return NRR_OK;
}

nrr_status sbegin(nrr_surrogate *s) {
  MCUDA(cudaSetDevice(s->device));
  MCUDA(cudaEventRecord(s->order_ev, s->user_stream));
  MCUDA(cudaStreamWaitEvent(s->stream, s->order_ev, 0));
  return NRR_OK;
}

nrr_status gemm(nrr_surrogate *s, const void *A, const void *B, float *D, int M,
                int N, int K) {
  char msg[256];
  nrr_status st = gemm_bf16_tn(A, B, D, M, N, K, N, s->stream, msg, sizeof msg, 0, 0,
                               s->ws, s->ws_bytes, -1);
  if (st != NRR_OK) set_last_error(msg);
  return st;
}

// Forward pass of `rows` = batch rows already gathered into xb/xt.
nrr_status forward(nrr_surrogate *s) {
  const int B = s->batch;
  for (int l = 0; l < s->L; l++) {
    const void *in = l == 0 ? (const void *)s->xb : (const void *)s->a[l - 1];
    MTRY(gemm(s, in, s->wt[l], s->z[l], B, s->dout[l], s->din[l]));
    const float *b = s->param + s->offB[l];
    if (l < s->L - 1)
      bias_gelu_kernel<<<tile_grid(B, s->dout[l]), dim3(32, 8), 0, s->stream>>>(
          s->z[l], b, s->a[l], s->at[l], B, s->dout[l]);
    else
      bias_kernel<<<(unsigned)(((int64_t)B * s->dout[l] + 255) / 256), 256, 0,
                    s->stream>>>(s->z[l], b, B, s->dout[l]);
  }
  MCUDA(cudaGetLastError());
  return NRR_OK;
}

// Backward pass from the normalised targets yb; gradients into s->grad; the
// batch loss into loss_slot (device).
// step (nullable): the device step counter of a captured training step; the
// loss then goes to loss_slot[*step % s->loss_cap].
nrr_status backward(nrr_surrogate *s, double *loss_slot, const int64_t *step = nullptr) {
  const int B = s->batch, Lm = s->L - 1;
  dim3 tg = tile_grid(B, s->dout[Lm]);
  mse_grad_kernel<<<tg, dim3(32, 8), 0, s->stream>>>(
      s->z[Lm], s->yb, s->dz32, s->dzb, s->dzt, B, s->dout[Lm], s->partials);
  loss_finalize_kernel<<<1, 256, 0, s->stream>>>(s->partials, (int)(tg.x * tg.y),
                                                 (double)B * s->dout[Lm], loss_slot,
                                                 step, s->loss_cap);
  for (int l = Lm; l >= 0; l--) {
    const int dout = s->dout[l], din = s->din[l];
    const void *act_t = l == 0 ? (const void *)s->xt : (const void *)s->at[l - 1];
    // dW^T[dout][din] = dZ^T[dout][B] . A_{l-1}^T[din][B]^T
    MTRY(gemm(s, s->dzt, act_t, s->grad + s->offW[l], dout, din, B));
    colsum_kernel<<<(dout + 255) / 256, 256, 0, s->stream>>>(
        s->dz32, s->grad + s->offB[l], B, dout);
    if (l > 0) {
      // dA[B][din] = dZ[B][dout] . W[din][dout]^T
      MTRY(gemm(s, s->dzb, s->w[l], s->da, B, din, dout));
      gelu_backward_kernel<<<tile_grid(B, din), dim3(32, 8), 0, s->stream>>>(
          s->da, s->z[l - 1], s->dz32, s->dzb, s->dzt, B, din);
    }
  }
  MCUDA(cudaGetLastError());
  return NRR_OK;
}

// step (nullable): the minibatch is order[*step * batch ..] (a captured
// training step), else order[0 .. batch).
nrr_status gather(nrr_surrogate *s, const float *X, const float *Y,
                  const int32_t *order, const int64_t *step = nullptr) {
  const int B = s->batch;
  gather_inputs_kernel<<<tile_grid(B, s->in_pad), dim3(32, 8), 0, s->stream>>>(
      X, order, s->n_in, s->in_pad, B, s->xb, s->xt, step);
  if (Y)
    gather_targets_kernel<<<(unsigned)(((int64_t)B * s->n_out + 255) / 256), 256,
                            0, s->stream>>>(Y, order, s->mean, s->stdv, s->n_out,
                                            B, s->yb, step);
  MCUDA(cudaGetLastError());
  return NRR_OK;
}

// AdamW's bias corrections after `step` updates.
float2 bias_corrections(int64_t step) {
  return make_float2((float)(1.0 / (1.0 - std::pow(0.9, (double)step))),
                     (float)(1.0 / (1.0 - std::pow(0.999, (double)step))));
}

// corr, step (nullable): a captured training step reads its corrections from
// corr[*step]; otherwise the host counter s->step advances here.
nrr_status adam_step(nrr_surrogate *s, double lr, double wd,
                     const float2 *corr = nullptr, const int64_t *step = nullptr) {
  AdamArgs a;
  a.lr = (float)lr;
  a.beta1 = 0.9f;
  a.beta2 = 0.999f;
  a.eps = 1e-8f;
  a.wd = (float)wd;
  a.c1 = a.c2 = 0.f;
  if (!corr) {
    s->step++;
    const float2 c = bias_corrections(s->step);
    a.c1 = c.x;
    a.c2 = c.y;
  }
  for (int l = 0; l < s->L; l++) {
    int64_t nw = (int64_t)s->dout[l] * s->din[l];
    adamw_kernel<<<(unsigned)((nw + 255) / 256), 256, 0, s->stream>>>(
        s->param + s->offW[l], s->grad + s->offW[l], s->m + s->offW[l],
        s->v + s->offW[l], nw, a, s->dout[l], s->din[l], 1, s->wt[l], s->w[l], corr,
        step);
    adamw_kernel<<<(s->dout[l] + 255) / 256, 256, 0, s->stream>>>(
        s->param + s->offB[l], s->grad + s->offB[l], s->m + s->offB[l],
        s->v + s->offB[l], s->dout[l], a, 0, 1, 0, nullptr, nullptr, corr, step);
  }
  MCUDA(cudaGetLastError());
  return NRR_OK;
}

// Logical packed layout (per layer W[dout][din_logical] then b[dout]) <->
// internal layout (layer 0 padded to in_pad columns).
int64_t logical_size(const nrr_surrogate *s) {
  int64_t n = 0;
  for (int l = 0; l < s->L; l++) {
    int dl = l == 0 ? s->n_in : s->din[l];
    n += (int64_t)s->dout[l] * dl + s->dout[l];
  }
  return n;
}

void logical_to_internal(const nrr_surrogate *s, const float *src,
                         std::vector<float> &dst) {
  dst.assign((size_t)s->nparam, 0.f);
  int64_t off = 0;
  for (int l = 0; l < s->L; l++) {
    int dl = l == 0 ? s->n_in : s->din[l];
    for (int o = 0; o < s->dout[l]; o++)
      for (int k = 0; k < dl; k++)
        dst[s->offW[l] + (int64_t)o * s->din[l] + k] = src[off + (int64_t)o * dl + k];
    off += (int64_t)s->dout[l] * dl;
    for (int o = 0; o < s->dout[l]; o++) dst[s->offB[l] + o] = src[off + o];
    off += s->dout[l];
  }
}

void internal_to_logical(const nrr_surrogate *s, const std::vector<float> &src,
                         float *dst) {
  int64_t off = 0;
  for (int l = 0; l < s->L; l++) {
    int dl = l == 0 ? s->n_in : s->din[l];
    for (int o = 0; o < s->dout[l]; o++)
      for (int k = 0; k < dl; k++)
        dst[off + (int64_t)o * dl + k] = src[s->offW[l] + (int64_t)o * s->din[l] + k];
    off += (int64_t)s->dout[l] * dl;
    for (int o = 0; o < s->dout[l]; o++) dst[off + o] = src[s->offB[l] + o];
    off += s->dout[l];
  }
}

nrr_status check_gemm(nrr_surrogate *s) {
  char msg[256];
  nrr_status st = gemm_check_error(s->stream, msg, sizeof msg);
  if (st != NRR_OK) set_last_error(msg);
  return st;
}

}  // namespace

extern "C" {

nrr_status nrr_surrogate_create(int n_in, int hidden, int depth, int n_out,
                                int batch, const float *init_params,
                                void *stream, nrr_surrogate **out) {
  if (!out) return mfail(NRR_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  if (n_in < 1 || n_in > 64 || hidden < 64 || hidden % 128 || depth < 1 ||
      depth > 16 || n_out < 128 || n_out % 128 || batch < 128 || batch % 128 ||
      !init_params)
    return mfail(NRR_ERR_INVALID_ARG,
                 "need 1 <= n_in <= 64, hidden and n_out multiples of 128, "
                 "batch a multiple of 128, 1 <= depth <= 16, initial parameters");
  nrr_surrogate *s = new (std::nothrow) nrr_surrogate();
  if (!s) return mfail(NRR_ERR_OOM, "host allocation failed");
  s->n_in = n_in;
  s->hidden = hidden;
  s->depth = depth;
  s->n_out = n_out;
  s->batch = batch;
  s->L = depth + 1;
  s->user_stream = static_cast<cudaStream_t>(stream);
  nrr_status st = [&]() -> nrr_status {
    MCUDA(cudaGetDevice(&s->device));
    MCUDA(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    MCUDA(cudaEventCreateWithFlags(&s->order_ev, cudaEventDisableTiming));
    MTRY(sbegin(s));
    for (int l = 0; l < s->L; l++) {
      s->din.push_back(l == 0 ? s->in_pad : hidden);
      s->dout.push_back(l == s->L - 1 ? n_out : hidden);
    }
    int64_t off = 0;
    for (int l = 0; l < s->L; l++) {
      s->offW.push_back(off);
      off += (int64_t)s->dout[l] * s->din[l];
      s->offB.push_back(off);
      off += s->dout[l];
    }
    s->nparam = off;
    MTRY(malloc_s(s, &s->param, off));
    MTRY(malloc_s(s, &s->grad, off));
    MTRY(malloc_s(s, &s->m, off));
    MTRY(malloc_s(s, &s->v, off));
    MCUDA(cudaMemsetAsync(s->m, 0, off * 4, s->stream));
    MCUDA(cudaMemsetAsync(s->v, 0, off * 4, s->stream));
    MCUDA(cudaMemsetAsync(s->grad, 0, off * 4, s->stream));
    for (int l = 0; l < s->L; l++) {
      bf16 *a1, *a2;
      MTRY(malloc_s(s, &a1, (size_t)s->dout[l] * s->din[l]));
      MTRY(malloc_s(s, &a2, (size_t)s->dout[l] * s->din[l]));
      s->wt.push_back(a1);
      s->w.push_back(a2);
      float *zl;
      MTRY(malloc_s(s, &zl, (size_t)batch * s->dout[l]));
      s->z.push_back(zl);
      if (l < s->L - 1) {
        bf16 *al, *atl;
        MTRY(malloc_s(s, &al, (size_t)batch * s->dout[l]));
        MTRY(malloc_s(s, &atl, (size_t)batch * s->dout[l]));
        s->a.push_back(al);
        s->at.push_back(atl);
      }
    }
    const int widest = std::max(n_out, hidden);
    MTRY(malloc_s(s, &s->xb, (size_t)batch * s->in_pad));
    MTRY(malloc_s(s, &s->xt, (size_t)batch * s->in_pad));
    MTRY(malloc_s(s, &s->da, (size_t)batch * widest));
    MTRY(malloc_s(s, &s->dz32, (size_t)batch * widest));
    MTRY(malloc_s(s, &s->dzb, (size_t)batch * widest));
    MTRY(malloc_s(s, &s->dzt, (size_t)batch * widest));
    MTRY(malloc_s(s, &s->yb, (size_t)batch * n_out));
    MTRY(malloc_s(s, &s->mean, n_out));
    MTRY(malloc_s(s, &s->stdv, n_out));
    MTRY(malloc_s(s, &s->order_id, batch));
    // split-K workspace of the largest split GEMM of a training step (the
    // weight gradients contract over the batch, the input gradients and
    // the forward over a layer's width)
    for (int l = 0; l < s->L; l++) {
      const int shapes[3][3] = {{batch, s->dout[l], s->din[l]},
                                {s->dout[l], s->din[l], batch},
                                {batch, s->din[l], s->dout[l]}};
      for (const auto &sh : shapes) {
        int bn = 0, sp = 0, pers = -1;
        gemm_plan(sh[0], sh[1], sh[2], &bn, &sp, &pers);
        s->ws_bytes = std::max(s->ws_bytes, gemm_workspace_bytes(sh[0], sh[1], sp));
      }
    }
    if (s->ws_bytes) MTRY(malloc_s(s, &s->ws, s->ws_bytes / sizeof(float)));
    MTRY(malloc_s(s, &s->partials, (size_t)((n_out + 31) / 32) * ((batch + 31) / 32) + 64));
    s->loss_cap = 1 << 16;
    MTRY(malloc_s(s, &s->loss, (size_t)s->loss_cap));
    std::vector<float> ones(n_out, 1.f), zeros(n_out, 0.f);
    std::vector<int32_t> ident(batch);
    for (int i = 0; i < batch; i++) ident[i] = i;
    MCUDA(cudaMemcpyAsync(s->stdv, ones.data(), n_out * 4, cudaMemcpyHostToDevice, s->stream));
    MCUDA(cudaMemcpyAsync(s->mean, zeros.data(), n_out * 4, cudaMemcpyHostToDevice, s->stream));
    MCUDA(cudaMemcpyAsync(s->order_id, ident.data(), batch * 4, cudaMemcpyHostToDevice, s->stream));
    std::vector<float> internal;
    logical_to_internal(s, init_params, internal);
    MCUDA(cudaMemcpyAsync(s->param, internal.data(), internal.size() * 4,
                          cudaMemcpyHostToDevice, s->stream));
    for (int l = 0; l < s->L; l++) {
      int64_t nw = (int64_t)s->dout[l] * s->din[l];
      weights_to_bf16_kernel<<<(unsigned)((nw + 255) / 256), 256, 0, s->stream>>>(
          s->param + s->offW[l], s->dout[l], s->din[l], s->wt[l], s->w[l]);
    }
    MCUDA(cudaGetLastError());
    MCUDA(cudaStreamSynchronize(s->stream));
    return NRR_OK;
  }();
  if (st != NRR_OK) {
    std::string msg = nrr_last_error();
    nrr_surrogate_destroy(s);
    set_last_error(msg.c_str());
    return st;
  }
  *out = s;
  return NRR_OK;
}

nrr_status nrr_surrogate_destroy(nrr_surrogate *s) {
  if (!s) return NRR_OK;
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (void *p : s->allocs) {
    dbg_unregister(p);
    cudaFree(p);
  }
  if (s->order_ev) cudaEventDestroy(s->order_ev);
  if (s->stream) cudaStreamDestroy(s->stream);
  delete s;
  return NRR_OK;
}

int64_t nrr_surrogate_num_params(const nrr_surrogate *s) {
  return s ? logical_size(s) : 0;
}

nrr_status nrr_surrogate_fit_scaling(nrr_surrogate *s, const float *Y, int64_t n) {
  if (!s || !Y || n < 1) return mfail(NRR_ERR_INVALID_ARG, "bad arguments");
  MTRY(sbegin(s));
  column_stats_kernel<<<(s->n_out + 127) / 128, 128, 0, s->stream>>>(Y, n, s->n_out,
                                                                     s->mean, s->stdv);
  std_floor_kernel<<<1, 256, 0, s->stream>>>(s->stdv, s->n_out);
  MCUDA(cudaGetLastError());
  MCUDA(cudaStreamSynchronize(s->stream));
  return NRR_OK;
}

nrr_status nrr_surrogate_train(nrr_surrogate *s, const float *X, const float *Y,
                               int64_t n, const int32_t *order, int64_t steps,
                               double lr, double weight_decay, float *loss_out) {
  if (!s || !X || !Y || !order || n < s->batch || steps < 0 || !(lr > 0.0))
    return mfail(NRR_ERR_INVALID_ARG, "bad arguments (n >= batch, lr > 0)");
  MTRY(sbegin(s));
  // Two or more steps: the first runs from the host (it also sets up what a
  // capture may not: the error flag, kernel attributes, tensor maps); then
  // one training step (gather, forward, backward, AdamW, counter advance) is
  // captured as a CUDA graph and replayed for the others.  Its minibatch
  // offset, loss slot and AdamW corrections come from a device step counter
  // and a per-step table, so every replay issues the same kernels with the
  // same arguments as a step launched from the host.
  cudaGraphExec_t exec = nullptr;
  int64_t *d_step = nullptr;
  float2 *d_corr = nullptr;
  struct Release {
    cudaGraphExec_t *e;
    int64_t **st;
    float2 **c;
    cudaStream_t stream;
    ~Release() {
      if (*e || *st || *c) cudaStreamSynchronize(stream);
      if (*e) cudaGraphExecDestroy(*e);
      if (*st) cudaFree(*st);
      if (*c) cudaFree(*c);
    }
  } release{&exec, &d_step, &d_corr, s->stream};
  int64_t t_first = 0;  // steps already taken from the host
  if (steps >= 2) {
    std::vector<float2> corr((size_t)steps);
    for (int64_t t = 0; t < steps; t++) corr[(size_t)t] = bias_corrections(s->step + 1 + t);
    MCUDA(cudaMalloc(&d_step, sizeof(int64_t)));
    MCUDA(cudaMalloc(&d_corr, corr.size() * sizeof(float2)));
    MCUDA(cudaMemcpyAsync(d_corr, corr.data(), corr.size() * sizeof(float2),
                          cudaMemcpyHostToDevice, s->stream));
    MTRY(gather(s, X, Y, order));
    MTRY(forward(s));
    MTRY(backward(s, s->loss));
    MTRY(adam_step(s, lr, weight_decay));
    t_first = 1;
    const int64_t one = 1;
    MCUDA(cudaMemcpyAsync(d_step, &one, sizeof one, cudaMemcpyHostToDevice, s->stream));
    MCUDA(cudaStreamSynchronize(s->stream));
    cudaGraph_t graph = nullptr;
    MCUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    nrr_status cs = [&]() -> nrr_status {
      MTRY(gather(s, X, Y, order, d_step));
      MTRY(forward(s));
      MTRY(backward(s, s->loss, d_step));
      MTRY(adam_step(s, lr, weight_decay, d_corr, d_step));
      step_advance_kernel<<<1, 1, 0, s->stream>>>(d_step);
      return NRR_OK;
    }();
    const cudaError_t ce = cudaStreamEndCapture(s->stream, &graph);
    if (cs != NRR_OK) {
      if (graph) cudaGraphDestroy(graph);
      return cs;
    }
    if (ce != cudaSuccess)
      return mfail(NRR_ERR_CUDA, "training step capture: %s", cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess)
      return mfail(NRR_ERR_CUDA, "training step graph: %s", cudaGetErrorString(ie));
  }
  for (int64_t t0 = 0; t0 < steps; t0 += s->loss_cap) {
    const int64_t chunk = std::min<int64_t>(s->loss_cap, steps - t0);
    for (int64_t t = 0; t < chunk; t++) {
      if (t0 + t < t_first) continue;
      if (exec) {
        MCUDA(cudaGraphLaunch(exec, s->stream));
        continue;
      }
      MTRY(gather(s, X, Y, order + (t0 + t) * s->batch));
      MTRY(forward(s));
      MTRY(backward(s, s->loss + t));
      MTRY(adam_step(s, lr, weight_decay));
    }
    if (loss_out) {
      std::vector<double> h(chunk);
      MCUDA(cudaMemcpyAsync(h.data(), s->loss, chunk * sizeof(double),
                            cudaMemcpyDeviceToHost, s->stream));
      MCUDA(cudaStreamSynchronize(s->stream));
      for (int64_t t = 0; t < chunk; t++) loss_out[t0 + t] = (float)h[t];
    }
  }
  if (exec) s->step += steps - t_first;  // the replays' AdamW updates
  MCUDA(cudaStreamSynchronize(s->stream));
  return check_gemm(s);
}

nrr_status nrr_surrogate_predict(nrr_surrogate *s, const float *X, int64_t n,
                                 float *out) {
  if (!s || !X || !out || n < 1) return mfail(NRR_ERR_INVALID_ARG, "bad arguments");
  MTRY(sbegin(s));
  std::vector<int32_t> ord(s->batch);
  int32_t *d_ord = s->order_id;
  for (int64_t r0 = 0; r0 < n; r0 += s->batch) {
    const int valid = (int)std::min<int64_t>(s->batch, n - r0);
    for (int i = 0; i < s->batch; i++) ord[i] = (int32_t)(r0 + std::min(i, valid - 1));
    // the identity slot doubles as the row list of this chunk
    MCUDA(cudaMemcpyAsync(d_ord, ord.data(), s->batch * 4, cudaMemcpyHostToDevice,
                          s->stream));
    MTRY(gather(s, X, nullptr, d_ord));
    MTRY(forward(s));
    denorm_kernel<<<(unsigned)(((int64_t)valid * s->n_out + 255) / 256), 256, 0,
                    s->stream>>>(s->z[s->L - 1], s->mean, s->stdv, s->n_out, valid,
                                 r0, out);
    MCUDA(cudaGetLastError());
    MCUDA(cudaStreamSynchronize(s->stream));  // ord is reused
  }
  std::vector<int32_t> ident(s->batch);
  for (int i = 0; i < s->batch; i++) ident[i] = i;
  MCUDA(cudaMemcpyAsync(d_ord, ident.data(), s->batch * 4, cudaMemcpyHostToDevice,
                        s->stream));
  MCUDA(cudaStreamSynchronize(s->stream));
  return check_gemm(s);
}

nrr_status nrr_surrogate_gradients(nrr_surrogate *s, const float *X,
                                   const float *Y, float *grads, double *loss) {
  if (!s || !X || !Y || !grads) return mfail(NRR_ERR_INVALID_ARG, "null argument");
  MTRY(sbegin(s));
  MTRY(gather(s, X, Y, s->order_id));
  MTRY(forward(s));
  MTRY(backward(s, s->loss));
  std::vector<float> g((size_t)s->nparam);
  double l = 0.0;
  MCUDA(cudaMemcpyAsync(g.data(), s->grad, g.size() * 4, cudaMemcpyDeviceToHost, s->stream));
  MCUDA(cudaMemcpyAsync(&l, s->loss, sizeof l, cudaMemcpyDeviceToHost, s->stream));
  MCUDA(cudaStreamSynchronize(s->stream));
  MTRY(check_gemm(s));
  internal_to_logical(s, g, grads);
  if (loss) *loss = l;
  return NRR_OK;
}

nrr_status nrr_surrogate_get_params(nrr_surrogate *s, float *params) {
  if (!s || !params) return mfail(NRR_ERR_INVALID_ARG, "null argument");
  MTRY(sbegin(s));
  std::vector<float> p((size_t)s->nparam);
  MCUDA(cudaMemcpyAsync(p.data(), s->param, p.size() * 4, cudaMemcpyDeviceToHost, s->stream));
  MCUDA(cudaStreamSynchronize(s->stream));
  internal_to_logical(s, p, params);
  return NRR_OK;
}

}  // extern "C"
