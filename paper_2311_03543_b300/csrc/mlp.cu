// Learned cost model kernels: a 3-layer perceptron (8 -> 64 -> 64 ->
// 2 * COMPAR_V_COUNT, ReLU) that predicts, for each of the COMPAR_V_COUNT
// variant ids, log2 of the run time and
// log10 of the relative error of a call from the call's context.  The paper's
// runtime selects variants with performance models it calls machine-learning
// models and expects more training to select better (Sec. 3.2, Sec. 5).
//
//   mlp_forward_kernel : inference for many rows and ensemble members.
//   mlp_train_kernel   : the whole training loop on the device, one CTA per
//                        ensemble member: per step, forward over a batch of up
//                        to 128 rows (one row per thread), masked-MSE loss,
//                        backward (weight gradients as small smem GEMMs), Adam.
//                        With apply == 0 it runs one step and returns the
//                        gradients instead of updating (used for gradient checks).
//
// Parameter layout per member (floats): W1[64][8] b1[64] W2[64][64] b2[64]
// W3[2 * COMPAR_V_COUNT][64] b3[2 * COMPAR_V_COUNT] — weights stored (out, in),
// row-major.
#include <cuda_runtime.h>

#include <cstdint>

#include "common.h"

namespace compar {
namespace {

constexpr int kIn = 8, kH = 64, kOut = 2 * COMPAR_V_COUNT;
constexpr int oW1 = 0, ob1 = oW1 + kH * kIn, oW2 = ob1 + kH, ob2 = oW2 + kH * kH,
              oW3 = ob2 + kH, ob3 = oW3 + kOut * kH, kP = ob3 + kOut;
constexpr int kB = 128;       // rows per training step (one per thread)
constexpr int kPad = kH + 1;  // padded activation rows in shared memory

__device__ __forceinline__ void forward_row(const float* __restrict__ p, const float* x,
                                            float* h1, float* h2, float* y) {
#pragma unroll 4
  for (int i = 0; i < kH; ++i) {
    float z = p[ob1 + i];
#pragma unroll
    for (int j = 0; j < kIn; ++j) z = fmaf(p[oW1 + i * kIn + j], x[j], z);
    h1[i] = fmaxf(z, 0.f);
  }
#pragma unroll 2
  for (int i = 0; i < kH; ++i) {
    float z = p[ob2 + i];
#pragma unroll 16
    for (int j = 0; j < kH; ++j) z = fmaf(p[oW2 + i * kH + j], h1[j], z);
    h2[i] = fmaxf(z, 0.f);
  }
#pragma unroll
  for (int o = 0; o < kOut; ++o) {
    float z = p[ob3 + o];
#pragma unroll 16
    for (int j = 0; j < kH; ++j) z = fmaf(p[oW3 + o * kH + j], h2[j], z);
    y[o] = z;
  }
}

// Y[e][r][o] for every member e (blockIdx.y) and row r.
__global__ void __launch_bounds__(128) mlp_forward_kernel(const float* __restrict__ params,
                                                          const float* __restrict__ X, int rows,
                                                          float* __restrict__ Y) {
  __shared__ float p[kP];
  const int e = blockIdx.y;
  for (int i = threadIdx.x; i < kP; i += blockDim.x) p[i] = params[e * kP + i];
  __syncthreads();
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= rows) return;
  float x[kIn], h1[kH], h2[kH], y[kOut];
#pragma unroll
  for (int j = 0; j < kIn; ++j) x[j] = X[r * kIn + j];
  forward_row(p, x, h1, h2, y);
#pragma unroll
  for (int o = 0; o < kOut; ++o) Y[(static_cast<int64_t>(e) * rows + r) * kOut + o] = y[o];
}

// Inference for a few rows (a selection decision): one 64-thread block per
// (row, member); thread j computes hidden unit j of each layer, so a row's
// forward pass takes three short dependent steps instead of one long serial
// loop.
__global__ void __launch_bounds__(64) mlp_forward_small_kernel(const float* __restrict__ params,
                                                               const float* __restrict__ X,
                                                               int rows, float* __restrict__ Y) {
  __shared__ float x[kIn], h1[kH], h2[kH];
  const int r = blockIdx.x, e = blockIdx.y, j = threadIdx.x;
  const float* p = params + static_cast<int64_t>(e) * kP;
  if (j < kIn) x[j] = X[r * kIn + j];
  __syncthreads();
  float z = p[ob1 + j];
#pragma unroll
  for (int i = 0; i < kIn; ++i) z = fmaf(p[oW1 + j * kIn + i], x[i], z);
  h1[j] = fmaxf(z, 0.f);
  __syncthreads();
  z = p[ob2 + j];
#pragma unroll 16
  for (int i = 0; i < kH; ++i) z = fmaf(p[oW2 + j * kH + i], h1[i], z);
  h2[j] = fmaxf(z, 0.f);
  __syncthreads();
  if (j < kOut) {
    z = p[ob3 + j];
#pragma unroll 16
    for (int i = 0; i < kH; ++i) z = fmaf(p[oW3 + j * kH + i], h2[i], z);
    Y[(static_cast<int64_t>(e) * rows + r) * kOut + j] = z;
  }
}

__device__ __forceinline__ float block_sum(float v, float* red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x % 32, warp = threadIdx.x / 32;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.f;
  for (int w = 0; w < static_cast<int>(blockDim.x / 32); ++w) s += red[w];
  return s;
}

struct TrainArgs {
  float* params;        // [E][kP] in/out
  float* adam_m;        // [E][kP]
  float* adam_v;        // [E][kP]
  const float* X;       // [rows][kIn]
  const float* T;       // [rows][kOut]
  const float* M;       // [rows][kOut] mask
  const int* idx;       // [E][steps][batch]
  int steps, batch;
  float lr, beta1, beta2, eps;
  int step0;            // Adam step counter of the first step (1-based)
  int apply;            // 0: one step, gradients to `grads`, params untouched
  float* grads;         // [E][kP] when apply == 0
  float* loss;          // [E][steps]
};

__global__ void __launch_bounds__(kB) mlp_train_kernel(TrainArgs a) {
  extern __shared__ float sm[];
  float* p = sm;                      // kP
  float* g = p + kP;                  // kP gradients
  float* xs = g + kP;                 // [kB][kIn]
  float* h1 = xs + kB * kIn;          // [kB][kPad]  (later dz1)
  float* h2 = h1 + kB * kPad;         // [kB][kPad]  (later dz2)
  float* dy = h2 + kB * kPad;         // [kB][kOut]
  float* red = dy + kB * kOut;        // 32

  const int e = blockIdx.x;
  const int t = threadIdx.x;
  const int B = a.batch;
  float* gp = a.params + static_cast<int64_t>(e) * kP;
  float* gm = a.adam_m + static_cast<int64_t>(e) * kP;
  float* gv = a.adam_v + static_cast<int64_t>(e) * kP;
  for (int i = t; i < kP; i += kB) p[i] = gp[i];
  __syncthreads();

  for (int s = 0; s < a.steps; ++s) {
    // ---------------------------------------------------------- forward
    const bool live = t < B;
    const int row = live ? a.idx[(static_cast<int64_t>(e) * a.steps + s) * B + t] : 0;
    float x[kIn], y[kOut];
    float a1[kH], a2[kH];
#pragma unroll
    for (int j = 0; j < kIn; ++j) x[j] = live ? a.X[static_cast<int64_t>(row) * kIn + j] : 0.f;
    forward_row(p, x, a1, a2, y);
    float msum = 0.f, lsum = 0.f, d[kOut];
#pragma unroll
    for (int o = 0; o < kOut; ++o) {
      const float mk = live ? a.M[static_cast<int64_t>(row) * kOut + o] : 0.f;
      const float diff = live ? y[o] - a.T[static_cast<int64_t>(row) * kOut + o] : 0.f;
      d[o] = mk * diff;
      msum += mk;
      lsum += mk * diff * diff;
    }
#pragma unroll
    for (int j = 0; j < kIn; ++j) xs[t * kIn + j] = x[j];
#pragma unroll
    for (int j = 0; j < kH; ++j) {
      h1[t * kPad + j] = live ? a1[j] : 0.f;
      h2[t * kPad + j] = live ? a2[j] : 0.f;
    }
    const float den = fmaxf(1.f, block_sum(msum, red));
    const float loss = block_sum(lsum, red) / den;
    if (t == 0 && a.loss) a.loss[static_cast<int64_t>(e) * a.steps + s] = loss;
    const float scale = 2.f / den;
#pragma unroll
    for (int o = 0; o < kOut; ++o) dy[t * kOut + o] = d[o] * scale;
    __syncthreads();

    // ---------------------------------------------------------- dW3, db3
    for (int q = t; q < kOut * kH + kOut; q += kB) {
      float acc = 0.f;
      if (q < kOut * kH) {
        const int o = q / kH, j = q % kH;
        for (int r = 0; r < B; ++r) acc = fmaf(dy[r * kOut + o], h2[r * kPad + j], acc);
        g[oW3 + q] = acc;
      } else {
        const int o = q - kOut * kH;
        for (int r = 0; r < B; ++r) acc += dy[r * kOut + o];
        g[ob3 + o] = acc;
      }
    }
    __syncthreads();
    // dz2 = (W3^T dy) * [z2 > 0], written over h2
    {
      float dyr[kOut];
#pragma unroll
      for (int o = 0; o < kOut; ++o) dyr[o] = dy[t * kOut + o];
      for (int j = 0; j < kH; ++j) {
        float acc = 0.f;
#pragma unroll
        for (int o = 0; o < kOut; ++o) acc = fmaf(p[oW3 + o * kH + j], dyr[o], acc);
        const float hv = h2[t * kPad + j];
        h2[t * kPad + j] = hv > 0.f ? acc : 0.f;
      }
    }
    __syncthreads();
    // ---------------------------------------------------------- dW2, db2
    for (int q = t; q < kH * kH + kH; q += kB) {
      float acc = 0.f;
      if (q < kH * kH) {
        const int i = q / kH, j = q % kH;
        for (int r = 0; r < B; ++r) acc = fmaf(h2[r * kPad + i], h1[r * kPad + j], acc);
        g[oW2 + q] = acc;
      } else {
        const int i = q - kH * kH;
        for (int r = 0; r < B; ++r) acc += h2[r * kPad + i];
        g[ob2 + i] = acc;
      }
    }
    __syncthreads();
    // dz1 = (W2^T dz2) * [z1 > 0], written over h1
    {
      float dz1[kH];
      for (int j = 0; j < kH; ++j) dz1[j] = 0.f;
      for (int i = 0; i < kH; ++i) {
        const float dz2 = h2[t * kPad + i];
#pragma unroll 16
        for (int j = 0; j < kH; ++j) dz1[j] = fmaf(p[oW2 + i * kH + j], dz2, dz1[j]);
      }
      for (int j = 0; j < kH; ++j) {
        const float hv = h1[t * kPad + j];
        h1[t * kPad + j] = hv > 0.f ? dz1[j] : 0.f;
      }
    }
    __syncthreads();
    // ---------------------------------------------------------- dW1, db1
    for (int q = t; q < kH * kIn + kH; q += kB) {
      float acc = 0.f;
      if (q < kH * kIn) {
        const int i = q / kIn, j = q % kIn;
        for (int r = 0; r < B; ++r) acc = fmaf(h1[r * kPad + i], xs[r * kIn + j], acc);
        g[oW1 + q] = acc;
      } else {
        const int i = q - kH * kIn;
        for (int r = 0; r < B; ++r) acc += h1[r * kPad + i];
        g[ob1 + i] = acc;
      }
    }
    __syncthreads();
    // ---------------------------------------------------------- Adam / output
    if (!a.apply) {
      for (int i = t; i < kP; i += kB) a.grads[static_cast<int64_t>(e) * kP + i] = g[i];
      break;
    }
    const int step = a.step0 + s;
    const float c1 = 1.f - powf(a.beta1, static_cast<float>(step));
    const float c2 = 1.f - powf(a.beta2, static_cast<float>(step));
    for (int i = t; i < kP; i += kB) {
      const float gi = g[i];
      const float m = a.beta1 * gm[i] + (1.f - a.beta1) * gi;
      const float v = a.beta2 * gv[i] + (1.f - a.beta2) * gi * gi;
      gm[i] = m;
      gv[i] = v;
      p[i] -= a.lr * (m / c1) / (sqrtf(v / c2) + a.eps);
    }
    __syncthreads();
  }
  if (a.apply)
    for (int i = t; i < kP; i += kB) gp[i] = p[i];
}

constexpr size_t kTrainSmem =
    sizeof(float) * (2 * kP + kB * kIn + 2 * kB * kPad + kB * kOut + 32);

}  // namespace

int mlp_param_count() { return kP; }

int mlp_forward_device(const float* d_params, int members, const float* d_X, int rows,
                       float* d_Y, cudaStream_t s) {
  if (rows <= 0 || members <= 0) return COMPAR_OK;
  if (rows <= 64) {
    mlp_forward_small_kernel<<<dim3(rows, members), 64, 0, s>>>(d_params, d_X, rows, d_Y);
  } else {
    dim3 grid((rows + 127) / 128, members);
    mlp_forward_kernel<<<grid, 128, 0, s>>>(d_params, d_X, rows, d_Y);
  }
  COMPAR_CUDA_TRY(cudaGetLastError());
  count_launch();
  return COMPAR_OK;
}

int mlp_train_device(float* d_params, float* d_m, float* d_v, int members, const float* d_X,
                     const float* d_T, const float* d_M, const int* d_idx, int steps, int batch,
                     float lr, int step0, int apply, float* d_grads, float* d_loss,
                     cudaStream_t s) {
  if (members <= 0 || steps <= 0 || batch <= 0 || batch > kB) return COMPAR_ERR_INVALID;
  COMPAR_CUDA_TRY(smem_opt_in(reinterpret_cast<const void*>(mlp_train_kernel),
                              static_cast<int>(kTrainSmem)));
  TrainArgs a{};
  a.params = d_params;
  a.adam_m = d_m;
  a.adam_v = d_v;
  a.X = d_X;
  a.T = d_T;
  a.M = d_M;
  a.idx = d_idx;
  a.steps = steps;
  a.batch = batch;
  a.lr = lr;
  a.beta1 = 0.9f;
  a.beta2 = 0.999f;
  a.eps = 1e-8f;
  a.step0 = step0;
  a.apply = apply;
  a.grads = d_grads;
  a.loss = d_loss;
  mlp_train_kernel<<<members, kB, kTrainSmem, s>>>(a);
  COMPAR_CUDA_TRY(cudaGetLastError());
  count_launch();
  return COMPAR_OK;
}

}  // namespace compar
