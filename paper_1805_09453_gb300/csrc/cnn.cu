// Learned warm start for the EMD solve: a 4-level encoder-decoder CNN that
// maps a density pair (f0, f1) to an initial dual potential phi_0, with
// hand-written inference and training kernels (BF16 or FP32 weights and
// activations, FP32 accumulation, FP32 gradients, FP32 master weights).
//
// The dual of the Beckmann problem (section 4.2) is a potential phi with
// |grad phi| <= 1; the saddle point's p is the gradient of such a potential,
// so a predicted phi_0 gives the dual start p_0 = proj(grad phi_0).
//
// Architecture (C = base width; 3x3 convolutions with zero padding; ReLU
// after every convolution but the last; 2x2 average pooling; nearest 2x
// upsampling; skip connections by channel concatenation [upsampled, skip]):
//   enc1: 3 -> C -> C              (N)     -> skip1
//   enc2: C -> 2C -> 2C            (N/2)   -> skip2
//   enc3: 2C -> 4C -> 4C           (N/4)   -> skip3
//   mid : 4C -> 8C -> 8C           (N/8)
//   dec3: [up(8C), skip3] 12C -> 4C -> 4C    (N/4)
//   dec2: [up(4C), skip2]  6C -> 2C -> 2C    (N/2)
//   dec1: [up(2C), skip1]  3C -> C -> C      (N)
//   head: C -> 1                   phi = prior + head (FP32), mean removed
// Input channels: (f0 - f1)/16, (f0 + f1)/16 and a prior potential phi_c
// (the EMD potential solved on a coarser grid and interpolated, see
// emd_coarse_start; zero when none is given).  The output is a correction:
// phi = phi_c + head, mean removed.  The head starts at zero, so an untrained
// network returns the prior itself.
//
// Loss (per sample, averaged over the batch), e = phi - t with both sides
// mean-free and D the unscaled forward difference with zero last slots:
//   |e|^2 / |t|^2  +  |D e|^2 / |D t|^2.
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

#include "gp_internal.cuh"

namespace {

template <typename T>
__device__ __forceinline__ float ldf(const T* p) {
  if constexpr (sizeof(T) == 2) return __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(p));
  else return (float)*p;
}
template <typename T>
__device__ __forceinline__ void stf(T* p, float v) {
  if constexpr (sizeof(T) == 2) *reinterpret_cast<__nv_bfloat16*>(p) = __float2bfloat16(v);
  else *p = (T)v;
}

constexpr int TS = 16;   // spatial tile edge (one output pixel per thread)
constexpr int COT = 16;  // output channels per CTA (per thread)
constexpr int CIT = 8;   // input channels staged per step
constexpr int HP = TS + 2;

// Y[b, co, p] = act(bias[co] + sum_ci sum_t W[co, ci, t] X[b, ci, p + o_t]),
// o_t = (t / 3 - 1, t % 3 - 1), zero outside the grid.
// FLIP: the weights are read as W[ci][co][8 - t] with the roles of Cin and
// Cout exchanged: the adjoint of a convolution is the convolution with the
// transposed, flipped kernel (the data gradient).
template <typename TX, typename TW, typename TY, bool RELU, bool FLIP>
__global__ void __launch_bounds__(TS* TS) k_conv3x3(const TX* __restrict__ X, long xbs, int Cin,
                                                     const TW* __restrict__ W, const float* __restrict__ bias,
                                                     TY* __restrict__ Y, long ybs, int Cout, int H, int Wd) {
  __shared__ float xs[CIT][HP][HP];
  __shared__ __align__(16) float ws[CIT][9][COT];
  const int tiles_x = (Wd + TS - 1) / TS;
  const int tx0 = (blockIdx.x % tiles_x) * TS, ty0 = (blockIdx.x / tiles_x) * TS;
  const int co0 = blockIdx.y * COT, b = blockIdx.z;
  const int lx = threadIdx.x % TS, ly = threadIdx.x / TS;
  const int x = tx0 + lx, y = ty0 + ly;
  float acc[COT];
#pragma unroll
  for (int c = 0; c < COT; ++c) acc[c] = 0.f;
  const TX* Xb = X + (long)b * xbs;
  const long plane = (long)H * Wd;
  for (int ci0 = 0; ci0 < Cin; ci0 += CIT) {
    for (int idx = threadIdx.x; idx < CIT * HP * HP; idx += TS * TS) {
      const int c = idx / (HP * HP), rem = idx % (HP * HP);
      const int yy = ty0 + rem / HP - 1, xx = tx0 + rem % HP - 1;
      float v = 0.f;
      if (ci0 + c < Cin && yy >= 0 && yy < H && xx >= 0 && xx < Wd) v = ldf(Xb + (long)(ci0 + c) * plane + (long)yy * Wd + xx);
      xs[c][rem / HP][rem % HP] = v;
    }
    for (int idx = threadIdx.x; idx < CIT * 9 * COT; idx += TS * TS) {
      const int co = idx % COT, t = (idx / COT) % 9, ci = idx / (COT * 9);
      float v = 0.f;
      if (co0 + co < Cout && ci0 + ci < Cin) {
        if (FLIP) v = ldf(W + ((long)(ci0 + ci) * Cout + (co0 + co)) * 9 + (8 - t));
        else v = ldf(W + ((long)(co0 + co) * Cin + (ci0 + ci)) * 9 + t);
      }
      ws[ci][t][co] = v;
    }
    __syncthreads();
    const int nci = min(CIT, Cin - ci0);
    for (int ci = 0; ci < nci; ++ci) {
      float xv[9];
#pragma unroll
      for (int t = 0; t < 9; ++t) xv[t] = xs[ci][ly + t / 3][lx + t % 3];
#pragma unroll
      for (int t = 0; t < 9; ++t) {
#pragma unroll
        for (int c4 = 0; c4 < COT / 4; ++c4) {
          const float4 w = *reinterpret_cast<const float4*>(&ws[ci][t][4 * c4]);
          acc[4 * c4 + 0] = fmaf(w.x, xv[t], acc[4 * c4 + 0]);
          acc[4 * c4 + 1] = fmaf(w.y, xv[t], acc[4 * c4 + 1]);
          acc[4 * c4 + 2] = fmaf(w.z, xv[t], acc[4 * c4 + 2]);
          acc[4 * c4 + 3] = fmaf(w.w, xv[t], acc[4 * c4 + 3]);
        }
      }
    }
    __syncthreads();
  }
  if (x < Wd && y < H) {
#pragma unroll
    for (int c = 0; c < COT; ++c) {
      const int co = co0 + c;
      if (co < Cout) {
        float v = acc[c] + (bias ? bias[co] : 0.f);
        if (RELU) v = fmaxf(v, 0.f);
        stf(Y + (long)b * ybs + (long)co * plane + (long)y * Wd + x, v);
      }
    }
  }
}

// Weight and bias gradients: dW[co, ci, t] += sum_{b, p} dY[b, co, p] X[b, ci, p + o_t],
// db[co] += sum_{b, p} dY[b, co, p].  CTA: 16 output x 16 input channels, one
// thread per (co, ci) pair holding its 9 taps in registers; the CTA loops over
// spatial tiles (strided by gridDim.x) and over the batch, and adds its
// partial sums with one atomic per tap at the end.
constexpr int WG_CO = 16, WG_CI = 16;
constexpr int XSTR = HP * HP + 1, GSTR = TS * TS + 1;  // odd channel strides: no bank conflicts
template <typename TX>
__global__ void __launch_bounds__(256) k_conv3x3_wgrad(const float* __restrict__ dY, long dybs, int Cout,
                                                       const TX* __restrict__ X, long xbs, int Cin, int H, int Wd,
                                                       int B, float* __restrict__ dW, float* __restrict__ db) {
  __shared__ float gs[WG_CO * GSTR];
  __shared__ float xs[WG_CI * XSTR];
  const int tiles_x = (Wd + TS - 1) / TS, tiles = tiles_x * ((H + TS - 1) / TS);
  const int co0 = blockIdx.y * WG_CO, ci0 = blockIdx.z * WG_CI;
  const int co = threadIdx.x / WG_CI, ci = threadIdx.x % WG_CI;
  const long plane = (long)H * Wd;
  float acc[9];
#pragma unroll
  for (int t = 0; t < 9; ++t) acc[t] = 0.f;
  float bacc = 0.f;
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int tx0 = (tile % tiles_x) * TS, ty0 = (tile / tiles_x) * TS;
    for (int b = 0; b < B; ++b) {
      for (int idx = threadIdx.x; idx < WG_CO * TS * TS; idx += 256) {
        const int c = idx / (TS * TS), rem = idx % (TS * TS), yy = ty0 + rem / TS, xx = tx0 + rem % TS;
        float v = 0.f;
        if (co0 + c < Cout && yy < H && xx < Wd) v = dY[(long)b * dybs + (long)(co0 + c) * plane + (long)yy * Wd + xx];
        gs[c * GSTR + rem] = v;
      }
      for (int idx = threadIdx.x; idx < WG_CI * HP * HP; idx += 256) {
        const int c = idx / (HP * HP), rem = idx % (HP * HP);
        const int yy = ty0 + rem / HP - 1, xx = tx0 + rem % HP - 1;
        float v = 0.f;
        if (ci0 + c < Cin && yy >= 0 && yy < H && xx >= 0 && xx < Wd)
          v = ldf(X + (long)b * xbs + (long)(ci0 + c) * plane + (long)yy * Wd + xx);
        xs[c * XSTR + rem] = v;
      }
      __syncthreads();
      const float* xc = xs + ci * XSTR;
      for (int py = 0; py < TS; ++py) {
        // 3x3 window sliding along the row: three new values per pixel
        float w0[3], w1[3], w2[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
          w0[r] = xc[(py + r) * HP + 0];
          w1[r] = xc[(py + r) * HP + 1];
        }
#pragma unroll 4
        for (int px = 0; px < TS; ++px) {
#pragma unroll
          for (int r = 0; r < 3; ++r) w2[r] = xc[(py + r) * HP + px + 2];
          const float g = gs[co * GSTR + py * TS + px];
          bacc += g;
#pragma unroll
          for (int r = 0; r < 3; ++r) {
            acc[3 * r + 0] = fmaf(g, w0[r], acc[3 * r + 0]);
            acc[3 * r + 1] = fmaf(g, w1[r], acc[3 * r + 1]);
            acc[3 * r + 2] = fmaf(g, w2[r], acc[3 * r + 2]);
            w0[r] = w1[r];
            w1[r] = w2[r];
          }
        }
      }
      __syncthreads();
    }
  }
  if (co0 + co < Cout && ci0 + ci < Cin) {
#pragma unroll
    for (int t = 0; t < 9; ++t) atomicAdd(&dW[((long)(co0 + co) * Cin + (ci0 + ci)) * 9 + t], acc[t]);
    if (ci == 0 && blockIdx.z == 0) atomicAdd(&db[co0 + co], bacc);
  }
}

// 2x2 average pooling (H even) and its adjoint (accumulated into dX).
template <typename T>
__global__ void k_pool2(const T* __restrict__ X, long xbs, T* __restrict__ Y, long ybs, int C, int H, int B) {
  const int Ho = H / 2;
  const long n = (long)B * C * Ho * Ho;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int x = i % Ho, y = (i / Ho) % Ho, c = (i / ((long)Ho * Ho)) % C, b = i / ((long)Ho * Ho * C);
    const T* p = X + (long)b * xbs + (long)c * H * H + (long)(2 * y) * H + 2 * x;
    stf(Y + (long)b * ybs + (long)c * Ho * Ho + (long)y * Ho + x,
        0.25f * ((ldf(p) + ldf(p + 1)) + (ldf(p + H) + ldf(p + H + 1))));
  }
}
__global__ void k_pool2_bwd_acc(const float* __restrict__ dY, long dybs, float* __restrict__ dX, long dxbs, int C,
                                int H, int B) {
  const int Ho = H / 2;
  const long n = (long)B * C * H * H;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int x = i % H, y = (i / H) % H, c = (i / ((long)H * H)) % C, b = i / ((long)H * H * C);
    dX[(long)b * dxbs + (long)c * H * H + (long)y * H + x] +=
        0.25f * dY[(long)b * dybs + (long)c * Ho * Ho + (long)(y / 2) * Ho + x / 2];
  }
}
// nearest 2x upsampling (side H -> 2H) and its adjoint
template <typename T>
__global__ void k_up2(const T* __restrict__ X, long xbs, T* __restrict__ Y, long ybs, int C, int H, int B) {
  const int Ho = 2 * H;
  const long n = (long)B * C * Ho * Ho;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int x = i % Ho, y = (i / Ho) % Ho, c = (i / ((long)Ho * Ho)) % C, b = i / ((long)Ho * Ho * C);
    Y[(long)b * ybs + (long)c * Ho * Ho + (long)y * Ho + x] = X[(long)b * xbs + (long)c * H * H + (long)(y / 2) * H + x / 2];
  }
}
__global__ void k_up2_bwd(const float* __restrict__ dY, long dybs, float* __restrict__ dX, long dxbs, int C, int H,
                          int B) {
  const int Ho = 2 * H;
  const long n = (long)B * C * H * H;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const int x = i % H, y = (i / H) % H, c = (i / ((long)H * H)) % C, b = i / ((long)H * H * C);
    const float* p = dY + (long)b * dybs + (long)c * Ho * Ho + (long)(2 * y) * Ho + 2 * x;
    dX[(long)b * dxbs + (long)c * H * H + (long)y * H + x] = (p[0] + p[1]) + (p[Ho] + p[Ho + 1]);
  }
}
// d *= (Y > 0): the ReLU adjoint, Y the stored forward output.
template <typename T>
__global__ void k_relu_bwd(float* __restrict__ d, long dbs, const T* __restrict__ Y, long ybs, long per, int B) {
  const long n = (long)B * per;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long b = i / per, j = i % per;
    if (!(ldf(Y + b * ybs + j) > 0.f)) d[b * dbs + j] = 0.f;
  }
}

// FP64 sum over one plane of NN values, one CTA: out = sum x (mode 0) or sum x^2 (mode 1).
__global__ void k_plane_sum(const float* __restrict__ x, long xbs, long NN, int mode, double* __restrict__ out) {
  __shared__ double sh[256];
  const float* p = x + blockIdx.x * xbs;
  double s = 0.0;
  for (long i = threadIdx.x; i < NN; i += blockDim.x) {
    const double v = p[i];
    s += mode ? v * v : v;
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}
// Input channels of one sample: (f0 - f1)/16, (f0 + f1)/16, prior (0 if null).
template <typename T>
__global__ void k_cnn_input(const float* __restrict__ f0, const float* __restrict__ f1, const float* __restrict__ prior,
                            T* __restrict__ X, long NN) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < NN; i += (long)gridDim.x * blockDim.x) {
    const float a = f0[i], c = f1[i];
    stf(X + i, (a - c) * 0.0625f);
    stf(X + NN + i, (a + c) * 0.0625f);
    stf(X + 2 * NN + i, prior ? prior[i] : 0.f);
  }
}
// phi += prior (one sample)
__global__ void k_add(float* __restrict__ phi, const float* __restrict__ prior, long NN) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < NN; i += (long)gridDim.x * blockDim.x) phi[i] += prior[i];
}
// ROF through the same network: *sum = sum I (FP64); the inputs a = 8 (I - mean),
// b = -a (so that the input channels are I - mean and 0) and the prior
// u_prior - mean; the start is u = mean + phi.
__global__ void k_sum64(const float* __restrict__ x, long n, double* __restrict__ sum) {
  double s = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) s += x[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(sum, s);
}
__global__ void k_rof_net_inputs(const float* __restrict__ I, const float* __restrict__ uprior,
                                 const double* __restrict__ sum, float* __restrict__ a, float* __restrict__ b,
                                 float* __restrict__ pr, long NN) {
  const float mean = (float)(*sum / (double)NN);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < NN; i += (long)gridDim.x * blockDim.x) {
    const float c = I[i] - mean;
    a[i] = 8.f * c;
    b[i] = -8.f * c;
    if (uprior) pr[i] = uprior[i] - mean;
  }
}
__global__ void k_rof_from_net(const float* __restrict__ phi, const double* __restrict__ sum, float* __restrict__ u,
                               long NN) {
  const float mean = (float)(*sum / (double)NN);
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < NN; i += (long)gridDim.x * blockDim.x)
    u[i] = mean + phi[i];
}
// x[b] -= sum[b] / NN for B planes of NN values
__global__ void k_sub_mean(float* __restrict__ x, long NN, int B, const double* __restrict__ sum) {
  const long n = (long)B * NN;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    x[i] -= (float)(sum[i / NN] / (double)NN);
}

// Loss sums of sample b (one CTA per sample), phi mean-free, target mean
// tsum[b] / NN.  out[4b .. 4b+3] = |e|^2, |t_c|^2, |D e|^2, |D t|^2.
__global__ void k_loss_sums(const float* __restrict__ phi, const float* __restrict__ tgt, int N,
                            const double* __restrict__ tsum, double* __restrict__ out) {
  __shared__ double sh[4][256];
  const long NN = (long)N * N, off = blockIdx.x * NN;
  const double mt = tsum[blockIdx.x] / (double)NN;
  double a[4] = {0.0, 0.0, 0.0, 0.0};
  for (long i = threadIdx.x; i < NN; i += blockDim.x) {
    const int r = (int)(i / N), c = (int)(i % N);
    const double t = (double)tgt[off + i] - mt;
    const double e = (double)phi[off + i] - t;
    a[0] += e * e;
    a[1] += t * t;
    if (c < N - 1) {
      const double t1 = (double)tgt[off + i + 1] - mt, e1 = (double)phi[off + i + 1] - t1;
      a[2] += (e1 - e) * (e1 - e);
      a[3] += (t1 - t) * (t1 - t);
    }
    if (r < N - 1) {
      const double t1 = (double)tgt[off + i + N] - mt, e1 = (double)phi[off + i + N] - t1;
      a[2] += (e1 - e) * (e1 - e);
      a[3] += (t1 - t) * (t1 - t);
    }
  }
  for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] = a[q];
  __syncthreads();
  for (int k = 128; k > 0; k >>= 1) {
    if (threadIdx.x < k)
      for (int q = 0; q < 4; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x < 4) out[4 * blockIdx.x + threadIdx.x] = sh[threadIdx.x][0];
}
// dL/dphi = (2 e / |t_c|^2 + 2 L e / |D t|^2) / B, L = D^T D the 5-point
// graph Laplacian (degree times the value minus the neighbours).  Both
// terms have zero sum, so they are also the gradient with respect to the
// head's output before its mean was removed.
__global__ void k_loss_grad(const float* __restrict__ phi, const float* __restrict__ tgt, int N, int B,
                            const double* __restrict__ tsum, const double* __restrict__ sums, float* __restrict__ dphi) {
  const long NN = (long)N * N, n = (long)B * NN;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const long b = i / NN, j = i % NN;
    const int r = (int)(j / N), c = (int)(j % N);
    const double mt = tsum[b] / (double)NN;
    const float* P = phi + b * NN;
    const float* T = tgt + b * NN;
    auto ev = [&](long k) { return (double)P[k] - ((double)T[k] - mt); };
    const double e = ev(j);
    double lap = 0.0;
    if (c > 0) lap += e - ev(j - 1);
    if (c < N - 1) lap += e - ev(j + 1);
    if (r > 0) lap += e - ev(j - N);
    if (r < N - 1) lap += e - ev(j + N);
    const double s0 = fmax(sums[4 * b + 1], 1e-300), s1 = fmax(sums[4 * b + 3], 1e-300);
    dphi[i] = (float)((2.0 * e / s0 + 2.0 * lap / s1) / (double)B);
  }
}

// Adam with bias correction on the FP32 master weights; the compute copy
// (BF16 or FP32) is refreshed in the same pass.
template <typename T>
__global__ void k_adam(float* __restrict__ w, float* __restrict__ m, float* __restrict__ v, const float* __restrict__ g,
                       T* __restrict__ wc, long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    stf(wc + i, wi);
  }
}
template <typename T>
__global__ void k_copy_params(const float* __restrict__ w, T* __restrict__ wc, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) stf(wc + i, w[i]);
}
// p_0 = proj(grad phi_0): forward differences (h = 1/N, zero last slots) and
// the pointwise projection onto the unit disc (sections 3.2, 4.2).
__global__ void k_warm_dual(const float* __restrict__ phi, float* __restrict__ p, int N) {
  const long NN = (long)N * N;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < NN; i += (long)gridDim.x * blockDim.x) {
    const int r = (int)(i / N), c = (int)(i % N);
    float gx = c < N - 1 ? (phi[i + 1] - phi[i]) * N : 0.f;
    float gy = r < N - 1 ? (phi[i + N] - phi[i]) * N : 0.f;
    const float n2 = gx * gx + gy * gy;
    if (n2 > 1.f) {
      const float s = rsqrtf(n2);
      gx *= s;
      gy *= s;
    }
    p[i] = gx;
    p[NN + i] = gy;
  }
}

inline int g1d(long n) { return (int)std::min<long>((n + 255) / 256, 8192); }

// ----------------------------------------------------------------- network
struct Conv {
  int cin, cout;
  long woff, boff;  // offsets of W [cout][cin][3][3] and b [cout] in the parameter vector
  long imoff;       // offset of its tensor-core weight images (BF16 mode)
};

// Activations of one sample, with their channel counts and pyramid level
// (side N >> level).  K1..K3 are the decoders' concatenation inputs: the
// encoder writes its skip output into their upper channels and the decoder
// writes the upsampled field into the lower ones.
enum { X0, A1, K1, A2, K2, A3, K3, P1, P2, P3, M1, M2, D3a, D3b, D2a, D2b, D1a, D1b, NACT };

struct Dims {
  long ch[NACT];
  int lev[NACT];
};

Dims act_dims(int C) {
  Dims d;
  const long ch[NACT] = {3, C, 3 * C, 2 * C, 6 * C, 4 * C, 12 * C, C, 2 * C, 4 * C, 8 * C, 8 * C, 4 * C, 4 * C, 2 * C, 2 * C, C, C};
  const int lev[NACT] = {0, 0, 0, 1, 1, 2, 2, 1, 2, 3, 3, 3, 2, 2, 1, 1, 0, 0};
  for (int i = 0; i < NACT; ++i) {
    d.ch[i] = ch[i];
    d.lev[i] = lev[i];
  }
  return d;
}

// The 15 convolutions in forward order; parameters stored conv by conv,
// weights W[cout][cin][3][3] then biases b[cout].
std::vector<Conv> build_convs(int C, long* nparam) {
  const int spec[15][2] = {{3, C},         {C, C},         {C, 2 * C},      {2 * C, 2 * C}, {2 * C, 4 * C},
                           {4 * C, 4 * C}, {4 * C, 8 * C}, {8 * C, 8 * C},  {12 * C, 4 * C}, {4 * C, 4 * C},
                           {6 * C, 2 * C}, {2 * C, 2 * C}, {3 * C, C},      {C, C},         {C, 1}};
  std::vector<Conv> v;
  long off = 0;
  for (auto& s : spec) {
    Conv c{s[0], s[1], off, 0, 0};
    off += (long)s[0] * s[1] * 9;
    c.boff = off;
    off += s[1];
    v.push_back(c);
  }
  *nparam = off;
  return v;
}

}  // namespace

struct gp_cnn_s {
  gp_handle h = nullptr;
  int device = 0;
  int C = 0;
  bool bf16 = true;
  std::vector<Conv> convs;
  long nparam = 0;
  float *w = nullptr, *m = nullptr, *v = nullptr, *g = nullptr;  // master weights, Adam moments, gradients
  void* wc = nullptr;                                            // compute copy of the weights
  void* wimg = nullptr;  // the convolutions' tensor-core weight images (BF16 mode)
  long step = 0;
  int cap_B = 0, cap_N = 0;
  void* act[NACT] = {};
  float* grd[NACT] = {};
  float *phi = nullptr, *dphi = nullptr, *tgt = nullptr, *pw = nullptr, *prior = nullptr;
  double* dsc = nullptr;  // per-sample FP64 scalars
  int* tc_err = nullptr;  // timeout flag of the tensor-core convolutions (BF16 mode)
  std::string err;
};

namespace {

gp_status cfail(gp_cnn n, gp_status s, const std::string& msg) {
  n->err = msg;
  return s;
}
#define CN_CUDA(n, expr)                                                                       \
  do {                                                                                         \
    cudaError_t e_ = (expr);                                                                   \
    if (e_ != cudaSuccess) return cfail(n, GP_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

struct DevGuard {
  int prev = -1;
  bool ok = false;
  explicit DevGuard(int d) {
    if (cudaGetDevice(&prev) != cudaSuccess) return;
    ok = cudaSetDevice(d) == cudaSuccess;
  }
  ~DevGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

void free_bufs(gp_cnn n) {
  for (int i = 0; i < NACT; ++i) {
    cudaFree(n->act[i]);
    cudaFree(n->grd[i]);
    n->act[i] = nullptr;
    n->grd[i] = nullptr;
  }
  cudaFree(n->phi);
  cudaFree(n->dphi);
  cudaFree(n->tgt);
  cudaFree(n->pw);
  cudaFree(n->prior);
  cudaFree(n->dsc);
  n->phi = n->dphi = n->tgt = n->pw = n->prior = nullptr;
  n->dsc = nullptr;
  n->cap_B = n->cap_N = 0;
}

// The tensor-core convolutions' timeout flag (BF16 mode): read (synchronising
// the stream) and cleared; a wait that timed out fails the call.
gp_status tc_flag(gp_cnn n, cudaStream_t st) {
  int f = 0;
  CN_CUDA(n, cudaMemcpyAsync(&f, n->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CN_CUDA(n, cudaStreamSynchronize(st));
  if (!f) return GP_OK;
  CN_CUDA(n, cudaMemsetAsync(n->tc_err, 0, sizeof(int), st));
  return cfail(n, GP_ERR_CUDA, "tensor-core convolution: a wait timed out");
}

// Activation, gradient and scratch buffers for batches of up to B samples of side N.
gp_status reserve(gp_cnn n, int B, int N) {
  if (n->cap_N == N && n->cap_B >= B) return GP_OK;
  free_bufs(n);
  const Dims d = act_dims(n->C);
  const size_t es = n->bf16 ? 2 : 4;
  for (int i = 0; i < NACT; ++i) {
    const size_t per = (size_t)d.ch[i] * (size_t)(N >> d.lev[i]) * (size_t)(N >> d.lev[i]);
    CN_CUDA(n, cudaMalloc(&n->act[i], (size_t)B * per * es));
    CN_CUDA(n, cudaMalloc((void**)&n->grd[i], (size_t)B * per * 4));
  }
  const size_t NN = (size_t)N * N;
  CN_CUDA(n, cudaMalloc((void**)&n->phi, (size_t)B * NN * 4));
  CN_CUDA(n, cudaMalloc((void**)&n->dphi, (size_t)B * NN * 4));
  CN_CUDA(n, cudaMalloc((void**)&n->tgt, (size_t)B * NN * 4));
  CN_CUDA(n, cudaMalloc((void**)&n->pw, 2 * NN * 4));
  CN_CUDA(n, cudaMalloc((void**)&n->prior, NN * 4));
  CN_CUDA(n, cudaMalloc((void**)&n->dsc, (size_t)(8 * B + 8) * sizeof(double)));
  n->cap_B = B;
  n->cap_N = N;
  return GP_OK;
}

template <typename T>
struct Net {
  gp_cnn n;
  cudaStream_t st;
  Dims d;
  int B, N;
  Net(gp_cnn nn, int b, int N_, cudaStream_t s) : n(nn), st(s), d(act_dims(nn->C)), B(b), N(N_) {}
  int side(int l) const { return N >> l; }
  long plane(int l) const { return (long)side(l) * side(l); }
  long bs(int a) const { return d.ch[a] * plane(d.lev[a]); }
  T* ptr(int a, long ch0 = 0) const { return reinterpret_cast<T*>(n->act[a]) + ch0 * plane(d.lev[a]); }
  float* gptr(int a, long ch0 = 0) const { return n->grd[a] + ch0 * plane(d.lev[a]); }
  const T* W(int i) const { return reinterpret_cast<const T*>(n->wc) + n->convs[i].woff; }
  const void* img(int i) const { return reinterpret_cast<const __nv_bfloat16*>(n->wimg) + n->convs[i].imoff; }
  const float* Bv(int i) const { return n->w + n->convs[i].boff; }
  dim3 cgrid(int l, int cout) const {
    const int t = (side(l) + TS - 1) / TS;
    return dim3(t * t, (cout + COT - 1) / COT, B);
  }

  template <typename TO, bool RELU>
  void conv(int i, const T* x, long xbs, TO* y, long ybs, int l) const {
    const Conv& c = n->convs[i];
    if constexpr (sizeof(T) == 2) {  // BF16 mode: implicit GEMM on the tensor cores
      gp::conv3x3_tc(x, xbs, c.cin, img(i), Bv(i), y, ybs, c.cout, side(l), side(l), B, RELU, sizeof(TO) == 4,
                     n->tc_err, st);
    } else {
      k_conv3x3<T, T, TO, RELU, false><<<cgrid(l, c.cout), TS * TS, 0, st>>>(x, xbs, c.cin, W(i), Bv(i), y, ybs,
                                                                             c.cout, side(l), side(l));
    }
  }
  void pool(int src, long sch0, int dst, int C, int l) const {  // level l -> l + 1
    k_pool2<T><<<g1d((long)B * C * plane(l + 1)), 256, 0, st>>>(ptr(src, sch0), bs(src), ptr(dst), bs(dst), C, side(l), B);
  }
  void up(int src, int dst, int C, int l) const {  // level l -> l - 1, into channels [0, C) of dst
    k_up2<T><<<g1d((long)B * C * plane(l - 1)), 256, 0, st>>>(ptr(src), bs(src), ptr(dst), bs(dst), C, side(l), B);
  }
  void forward() const {
    const int C = n->C;
    conv<T, true>(0, ptr(X0), bs(X0), ptr(A1), bs(A1), 0);
    conv<T, true>(1, ptr(A1), bs(A1), ptr(K1, 2 * C), bs(K1), 0);  // skip1
    pool(K1, 2 * C, P1, C, 0);
    conv<T, true>(2, ptr(P1), bs(P1), ptr(A2), bs(A2), 1);
    conv<T, true>(3, ptr(A2), bs(A2), ptr(K2, 4 * C), bs(K2), 1);  // skip2
    pool(K2, 4 * C, P2, 2 * C, 1);
    conv<T, true>(4, ptr(P2), bs(P2), ptr(A3), bs(A3), 2);
    conv<T, true>(5, ptr(A3), bs(A3), ptr(K3, 8 * C), bs(K3), 2);  // skip3
    pool(K3, 8 * C, P3, 4 * C, 2);
    conv<T, true>(6, ptr(P3), bs(P3), ptr(M1), bs(M1), 3);
    conv<T, true>(7, ptr(M1), bs(M1), ptr(M2), bs(M2), 3);
    up(M2, K3, 8 * C, 3);
    conv<T, true>(8, ptr(K3), bs(K3), ptr(D3a), bs(D3a), 2);
    conv<T, true>(9, ptr(D3a), bs(D3a), ptr(D3b), bs(D3b), 2);
    up(D3b, K2, 4 * C, 2);
    conv<T, true>(10, ptr(K2), bs(K2), ptr(D2a), bs(D2a), 1);
    conv<T, true>(11, ptr(D2a), bs(D2a), ptr(D2b), bs(D2b), 1);
    up(D2b, K1, 2 * C, 1);
    conv<T, true>(12, ptr(K1), bs(K1), ptr(D1a), bs(D1a), 0);
    conv<T, true>(13, ptr(D1a), bs(D1a), ptr(D1b), bs(D1b), 0);
    conv<float, false>(14, ptr(D1b), bs(D1b), n->phi, plane(0), 0);
  }
  // Backward of conv i: dy (FP32, ReLU adjoint applied) -> weight and bias
  // gradients (accumulated) and the input gradient dx (overwritten; skipped
  // when null).  xa names the conv's input activation.
  void conv_bwd(int i, const float* dy, long dybs, int xa, long xch0, float* dx, int l) const {
    const Conv& c = n->convs[i];
    const int t = (side(l) + TS - 1) / TS, tiles = t * t;
    const int cg = (c.cout + WG_CO - 1) / WG_CO, kg = (c.cin + WG_CI - 1) / WG_CI;
    const int gx = std::max(1, std::min(tiles, (4 * 152 + cg * kg - 1) / (cg * kg)));
    if constexpr (sizeof(T) == 2) {  // BF16 mode: weight gradient on the tensor cores
      gp::conv3x3_wgrad_tc(dy, dybs, c.cout, ptr(xa, xch0), bs(xa), c.cin, side(l), side(l), B, n->g + c.woff,
                           n->g + c.boff, n->tc_err, st);
    } else {
      k_conv3x3_wgrad<T><<<dim3(gx, cg, kg), 256, 0, st>>>(dy, dybs, c.cout, ptr(xa, xch0), bs(xa), c.cin, side(l),
                                                          side(l), B, n->g + c.woff, n->g + c.boff);
    }
    if (dx) {
      if constexpr (sizeof(T) == 2) {  // BF16 mode: data gradient on the tensor cores
        gp::conv3x3_dgrad_tc(dy, dybs, c.cout, img(i), dx, bs(xa), c.cin, side(l), side(l), B, n->tc_err, st);
      } else {
        k_conv3x3<float, T, float, false, true><<<cgrid(l, c.cin), TS * TS, 0, st>>>(dy, dybs, c.cout, W(i), nullptr,
                                                                                    dx, bs(xa), c.cin, side(l), side(l));
      }
    }
  }
  void relu_bwd(int a, long ch0, long C) const {
    k_relu_bwd<T><<<g1d((long)B * C * plane(d.lev[a])), 256, 0, st>>>(gptr(a, ch0), bs(a), ptr(a, ch0), bs(a),
                                                                     C * plane(d.lev[a]), B);
  }
  void pool_bwd(int src, int dst, long dch0, int C, int l) const {  // src at level l + 1 -> dst slice at level l
    k_pool2_bwd_acc<<<g1d((long)B * C * plane(l)), 256, 0, st>>>(gptr(src), bs(src), gptr(dst, dch0), bs(dst), C,
                                                                side(l), B);
  }
  void up_bwd(int src, int dst, int C, int l) const {  // channels [0, C) of src at level l - 1 -> dst at level l
    k_up2_bwd<<<g1d((long)B * C * plane(l)), 256, 0, st>>>(gptr(src), bs(src), gptr(dst), bs(dst), C, side(l), B);
  }
  void backward() const {
    const int C = n->C;
    conv_bwd(14, n->dphi, plane(0), D1b, 0, gptr(D1b), 0);
    relu_bwd(D1b, 0, C);
    conv_bwd(13, gptr(D1b), bs(D1b), D1a, 0, gptr(D1a), 0);
    relu_bwd(D1a, 0, C);
    conv_bwd(12, gptr(D1a), bs(D1a), K1, 0, gptr(K1), 0);
    up_bwd(K1, D2b, 2 * C, 1);
    relu_bwd(D2b, 0, 2 * C);
    conv_bwd(11, gptr(D2b), bs(D2b), D2a, 0, gptr(D2a), 1);
    relu_bwd(D2a, 0, 2 * C);
    conv_bwd(10, gptr(D2a), bs(D2a), K2, 0, gptr(K2), 1);
    up_bwd(K2, D3b, 4 * C, 2);
    relu_bwd(D3b, 0, 4 * C);
    conv_bwd(9, gptr(D3b), bs(D3b), D3a, 0, gptr(D3a), 2);
    relu_bwd(D3a, 0, 4 * C);
    conv_bwd(8, gptr(D3a), bs(D3a), K3, 0, gptr(K3), 2);
    up_bwd(K3, M2, 8 * C, 3);
    relu_bwd(M2, 0, 8 * C);
    conv_bwd(7, gptr(M2), bs(M2), M1, 0, gptr(M1), 3);
    relu_bwd(M1, 0, 8 * C);
    conv_bwd(6, gptr(M1), bs(M1), P3, 0, gptr(P3), 3);
    pool_bwd(P3, K3, 8 * C, 4 * C, 2);  // skip3: its decoder slice plus the pooled path
    relu_bwd(K3, 8 * C, 4 * C);
    conv_bwd(5, gptr(K3, 8 * C), bs(K3), A3, 0, gptr(A3), 2);
    relu_bwd(A3, 0, 4 * C);
    conv_bwd(4, gptr(A3), bs(A3), P2, 0, gptr(P2), 2);
    pool_bwd(P2, K2, 4 * C, 2 * C, 1);
    relu_bwd(K2, 4 * C, 2 * C);
    conv_bwd(3, gptr(K2, 4 * C), bs(K2), A2, 0, gptr(A2), 1);
    relu_bwd(A2, 0, 2 * C);
    conv_bwd(2, gptr(A2), bs(A2), P1, 0, gptr(P1), 1);
    pool_bwd(P1, K1, 2 * C, C, 0);
    relu_bwd(K1, 2 * C, C);
    conv_bwd(1, gptr(K1, 2 * C), bs(K1), A1, 0, gptr(A1), 0);
    relu_bwd(A1, 0, C);
    conv_bwd(0, gptr(A1), bs(A1), X0, 0, nullptr, 0);
  }
};

gp_status check_dev(gp_cnn n, const void* p, const char* what) {
  cudaPointerAttributes a;
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess ||
      !(a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == n->device))) {
    cudaGetLastError();
    return cfail(n, GP_ERR_ARG, std::string(what) + " must be a device pointer of the handle's device");
  }
  return GP_OK;
}

gp_status check_batch(gp_cnn n, int B, const float* const* f0, const float* const* f1, const float* const* prior,
                      int N) {
  if (B < 1 || !f0 || !f1) return cfail(n, GP_ERR_ARG, "bad batch arguments");
  if (N < 8 || N > 8192 || N % 8) return cfail(n, GP_ERR_ARG, "N must be a multiple of 8 in [8, 8192] (three 2x2 poolings)");
  for (int b = 0; b < B; ++b) {
    gp_status r;
    if ((r = check_dev(n, f0[b], "f0[b]")) != GP_OK || (r = check_dev(n, f1[b], "f1[b]")) != GP_OK) return r;
    if (prior && prior[b] && (r = check_dev(n, prior[b], "prior[b]")) != GP_OK) return r;
  }
  return GP_OK;
}

// Input features and the forward pass of B samples; n->phi receives
// prior + head output, mean removed.
template <typename T>
gp_status forward_impl(gp_cnn n, int B, const float* const* f0, const float* const* f1, const float* const* prior,
                       int N, cudaStream_t st) {
  Net<T> net(n, B, N, st);
  const long NN = (long)N * N;
  for (int b = 0; b < B; ++b)
    k_cnn_input<T><<<g1d(NN), 256, 0, st>>>(f0[b], f1[b], prior ? prior[b] : nullptr, net.ptr(X0) + b * net.bs(X0), NN);
  net.forward();
  if (prior)
    for (int b = 0; b < B; ++b)
      if (prior[b]) k_add<<<g1d(NN), 256, 0, st>>>(n->phi + b * NN, prior[b], NN);
  k_plane_sum<<<B, 256, 0, st>>>(n->phi, NN, NN, 0, n->dsc);
  k_sub_mean<<<g1d(B * NN), 256, 0, st>>>(n->phi, NN, B, n->dsc);
  CN_CUDA(n, cudaGetLastError());
  return GP_OK;
}

gp_status forward(gp_cnn n, int B, const float* const* f0, const float* const* f1, const float* const* prior, int N,
                  cudaStream_t st) {
  gp_status r = reserve(n, B, N);
  if (r != GP_OK) return r;
  return n->bf16 ? forward_impl<__nv_bfloat16>(n, B, f0, f1, prior, N, st)
                 : forward_impl<float>(n, B, f0, f1, prior, N, st);
}

template <typename T>
void backward_impl(gp_cnn n, int B, int N, cudaStream_t st) {
  Net<T>(n, B, N, st).backward();
}

// BF16 mode: the tensor-core weight images of every convolution, from the compute copy.
gp_status pack_images(gp_cnn n, cudaStream_t st) {
  for (const Conv& c : n->convs)
    CN_CUDA(n, gp::conv3x3_tc_pack(reinterpret_cast<const __nv_bfloat16*>(n->wc) + c.woff, c.cin, c.cout,
                                   reinterpret_cast<__nv_bfloat16*>(n->wimg) + c.imoff, st));
  return GP_OK;
}

gp_status refresh_copy(gp_cnn n, cudaStream_t st) {
  if (n->bf16) k_copy_params<__nv_bfloat16><<<g1d(n->nparam), 256, 0, st>>>(n->w, (__nv_bfloat16*)n->wc, n->nparam);
  else k_copy_params<float><<<g1d(n->nparam), 256, 0, st>>>(n->w, (float*)n->wc, n->nparam);
  CN_CUDA(n, cudaGetLastError());
  return n->bf16 ? pack_images(n, st) : GP_OK;
}

}  // namespace

// =================================================================== ABI
extern "C" {

GP_API gp_status gp_cnn_create(gp_handle h, int base_channels, int bf16, unsigned long long seed, gp_cnn* out) {
  if (!h || !out) return GP_ERR_ARG;
  *out = nullptr;
  if (base_channels < 1 || base_channels > 256) return GP_ERR_ARG;
  gp_cnn n = new gp_cnn_s;
  n->h = h;
  n->device = gp::handle_device(h);
  n->C = base_channels;
  n->bf16 = bf16 != 0;
  n->convs = build_convs(n->C, &n->nparam);
  size_t nimg = 0;
  for (Conv& c : n->convs) {
    c.imoff = (long)nimg;
    nimg += gp::conv3x3_tc_image_elems(c.cin, c.cout);
  }
  DevGuard g(n->device);
  const size_t P = (size_t)n->nparam;
  if (!g.ok || cudaMalloc((void**)&n->w, P * 4) || cudaMalloc((void**)&n->m, P * 4) ||
      cudaMalloc((void**)&n->v, P * 4) || cudaMalloc((void**)&n->g, P * 4) ||
      cudaMalloc(&n->wc, P * (n->bf16 ? 2 : 4)) || (n->bf16 && cudaMalloc(&n->wimg, nimg * 2)) ||
      cudaMalloc((void**)&n->tc_err, sizeof(int)) ||
      cudaMemset(n->tc_err, 0, sizeof(int))) {
    cudaGetLastError();
    gp_cnn_destroy(n);
    return GP_ERR_CUDA;
  }
  // He-uniform weights from a 64-bit LCG, zero biases, zero head (the
  // untrained network returns its prior)
  std::vector<float> w(P, 0.f);
  unsigned long long s = seed;
  for (size_t ci = 0; ci + 1 < n->convs.size(); ++ci) {
    const Conv& c = n->convs[ci];
    const double lim = sqrt(6.0 / (9.0 * c.cin));
    for (long i = 0; i < (long)c.cin * c.cout * 9; ++i) {
      s = s * 6364136223846793005ull + 1442695040888963407ull;
      const double u = (double)(s >> 11) * (1.0 / 9007199254740992.0);
      w[c.woff + i] = (float)((2.0 * u - 1.0) * lim);
    }
  }
  if (gp_cnn_set_params(n, w.data()) != GP_OK) {
    gp_cnn_destroy(n);
    return GP_ERR_CUDA;
  }
  *out = n;
  return GP_OK;
}

GP_API gp_status gp_cnn_destroy(gp_cnn n) {
  if (!n) return GP_ERR_ARG;
  DevGuard g(n->device);
  free_bufs(n);
  cudaFree(n->w);
  cudaFree(n->m);
  cudaFree(n->v);
  cudaFree(n->g);
  cudaFree(n->wc);
  cudaFree(n->wimg);
  cudaFree(n->tc_err);
  delete n;
  return GP_OK;
}

GP_API const char* gp_cnn_last_error(gp_cnn n) { return n ? n->err.c_str() : "null network"; }

GP_API long long gp_cnn_num_params(gp_cnn n) { return n ? (long long)n->nparam : -1; }

GP_API gp_status gp_cnn_get_params(gp_cnn n, float* w) {
  if (!n || !w) return GP_ERR_ARG;
  DevGuard g(n->device);
  CN_CUDA(n, cudaMemcpy(w, n->w, (size_t)n->nparam * 4, cudaMemcpyDeviceToHost));
  return GP_OK;
}

GP_API gp_status gp_cnn_set_params(gp_cnn n, const float* w) {
  if (!n || !w) return GP_ERR_ARG;
  n->err.clear();
  DevGuard g(n->device);
  const size_t P = (size_t)n->nparam;
  CN_CUDA(n, cudaMemcpy(n->w, w, P * 4, cudaMemcpyHostToDevice));
  CN_CUDA(n, cudaMemset(n->m, 0, P * 4));
  CN_CUDA(n, cudaMemset(n->v, 0, P * 4));
  CN_CUDA(n, cudaMemset(n->g, 0, P * 4));
  n->step = 0;
  gp_status r = refresh_copy(n, nullptr);
  if (r != GP_OK) return r;
  CN_CUDA(n, cudaDeviceSynchronize());
  return GP_OK;
}

GP_API gp_status gp_cnn_forward(gp_cnn n, int B, const float* const* f0, const float* const* f1,
                                const float* const* prior, int N, float* phi, void* stream) {
  if (!n) return GP_ERR_ARG;
  n->err.clear();
  DevGuard g(n->device);
  gp_status r = check_batch(n, B, f0, f1, prior, N);
  if (r != GP_OK) return r;
  if ((r = check_dev(n, phi, "phi")) != GP_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  if ((r = forward(n, B, f0, f1, prior, N, st)) != GP_OK) return r;
  CN_CUDA(n, cudaMemcpyAsync(phi, n->phi, (size_t)B * N * N * 4, cudaMemcpyDeviceToDevice, st));
  return GP_OK;
}

GP_API gp_status gp_cnn_loss_grad(gp_cnn n, int B, const float* const* f0, const float* const* f1,
                                  const float* const* prior, const float* const* phi_target, int N, double* loss,
                                  float* grad, void* stream) {
  if (!n) return GP_ERR_ARG;
  n->err.clear();
  DevGuard g(n->device);
  gp_status r = check_batch(n, B, f0, f1, prior, N);
  if (r != GP_OK) return r;
  if (!phi_target) return cfail(n, GP_ERR_ARG, "phi_target is null");
  for (int b = 0; b < B; ++b)
    if ((r = check_dev(n, phi_target[b], "phi_target[b]")) != GP_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  if ((r = forward(n, B, f0, f1, prior, N, st)) != GP_OK) return r;
  const long NN = (long)N * N;
  for (int b = 0; b < B; ++b)
    CN_CUDA(n, cudaMemcpyAsync(n->tgt + b * NN, phi_target[b], NN * 4, cudaMemcpyDeviceToDevice, st));
  double* tsum = n->dsc;
  double* sums = n->dsc + B;
  k_plane_sum<<<B, 256, 0, st>>>(n->tgt, NN, NN, 0, tsum);
  k_loss_sums<<<B, 256, 0, st>>>(n->phi, n->tgt, N, tsum, sums);
  k_loss_grad<<<g1d(B * NN), 256, 0, st>>>(n->phi, n->tgt, N, B, tsum, sums, n->dphi);
  CN_CUDA(n, cudaMemsetAsync(n->g, 0, (size_t)n->nparam * 4, st));
  if (n->bf16) backward_impl<__nv_bfloat16>(n, B, N, st);
  else backward_impl<float>(n, B, N, st);
  CN_CUDA(n, cudaGetLastError());
  if (loss) {
    std::vector<double> hs(4 * (size_t)B);
    CN_CUDA(n, cudaMemcpyAsync(hs.data(), sums, hs.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    CN_CUDA(n, cudaStreamSynchronize(st));
    double L = 0.0;
    for (int b = 0; b < B; ++b) L += hs[4 * b] / fmax(hs[4 * b + 1], 1e-300) + hs[4 * b + 2] / fmax(hs[4 * b + 3], 1e-300);
    *loss = L / B;
  }
  if (grad) {
    CN_CUDA(n, cudaMemcpyAsync(grad, n->g, (size_t)n->nparam * 4, cudaMemcpyDeviceToHost, st));
    CN_CUDA(n, cudaStreamSynchronize(st));
  }
  if ((loss || grad) && n->bf16) return tc_flag(n, st);
  return GP_OK;
}

GP_API gp_status gp_cnn_adam_step(gp_cnn n, double lr, void* stream) {
  if (!n) return GP_ERR_ARG;
  n->err.clear();
  if (!(lr > 0) || !isfinite(lr)) return cfail(n, GP_ERR_ARG, "lr must be finite and > 0");
  DevGuard g(n->device);
  cudaStream_t st = (cudaStream_t)stream;
  n->step++;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = (float)(1.0 - pow(0.9, (double)n->step)), c2 = (float)(1.0 - pow(0.999, (double)n->step));
  if (n->bf16)
    k_adam<__nv_bfloat16><<<g1d(n->nparam), 256, 0, st>>>(n->w, n->m, n->v, n->g, (__nv_bfloat16*)n->wc, n->nparam,
                                                          (float)lr, b1, b2, 1e-8f, c1, c2);
  else
    k_adam<float><<<g1d(n->nparam), 256, 0, st>>>(n->w, n->m, n->v, n->g, (float*)n->wc, n->nparam, (float)lr, b1, b2,
                                                  1e-8f, c1, c2);
  CN_CUDA(n, cudaGetLastError());
  return n->bf16 ? pack_images(n, st) : GP_OK;
}

GP_API gp_status emd_solve_learned(gp_handle h, gp_cnn n, const float* f0, const float* f1, float* m, float* p,
                                   float* phi, int N, int coarse_factor, const gp_opts* coarse_opts,
                                   const gp_opts* opts, gp_report* report, int* start_used, void* stream) {
  if (!h || !n || n->h != h) return GP_ERR_ARG;
  n->err.clear();
  const auto t0 = std::chrono::steady_clock::now();
  DevGuard g(n->device);
  gp_status r = check_batch(n, 1, &f0, &f1, nullptr, N);
  if (r != GP_OK) return r;
  if (coarse_factor < 0 || coarse_factor == 1) return cfail(n, GP_ERR_ARG, "coarse_factor must be 0 (none) or >= 2");
  gp_opts o;
  gp_default_opts(&o);
  if (opts) o = *opts;
  if (o.warm_start) return cfail(n, GP_ERR_ARG, "opts.warm_start must be 0: the start is chosen here");
  if ((r = reserve(n, 1, N)) != GP_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  const float* prior = nullptr;
  if (coarse_factor) {
    gp_opts oc;
    gp_default_opts(&oc);
    oc.tol_rel_gap = 1e-4;
    oc.max_iters = 100000;
    oc.use_graph = o.use_graph;
    if (coarse_opts) oc = *coarse_opts;
    gp_report rc;
    r = emd_coarse_start(h, f0, f1, N, coarse_factor, &oc, n->prior, &rc, stream);
    if (r != GP_OK && r != GP_ERR_MAXITER) return cfail(n, r, std::string("coarse start: ") + gp_last_error(h));
    prior = n->prior;
  }
  if ((r = forward(n, 1, &f0, &f1, prior ? &prior : nullptr, N, st)) != GP_OK) return r;
  float* p0 = p ? p : n->pw;
  // Candidates: the learned start, the prior alone, the zero start; the one
  // with the smallest duality gap at n = 0 is kept.
  gp_opts probe = o;
  probe.max_iters = 0;
  double best = INFINITY;
  int choice = 0;
  const float* cand[2] = {n->phi, prior};
  for (int c = 0; c < 2; ++c) {
    if (!cand[c]) continue;
    k_warm_dual<<<g1d((long)N * N), 256, 0, st>>>(cand[c], p0, N);
    CN_CUDA(n, cudaGetLastError());
    probe.warm_start = 1;
    gp_report rw;
    r = emd_solve(h, f0, f1, m, p0, nullptr, N, &probe, &rw, stream);
    if (r != GP_OK && r != GP_ERR_MAXITER) return cfail(n, r, std::string("start probe: ") + gp_last_error(h));
    if (rw.rel_gap < best) {
      best = rw.rel_gap;
      choice = c == 0 ? 1 : 2;
    }
  }
  probe.warm_start = 0;
  gp_report rz;
  r = emd_solve(h, f0, f1, m, nullptr, nullptr, N, &probe, &rz, stream);
  if (r != GP_OK && r != GP_ERR_MAXITER) return cfail(n, r, std::string("zero probe: ") + gp_last_error(h));
  if (!(best < rz.rel_gap)) choice = 0;
  if (choice == 0) CN_CUDA(n, cudaMemsetAsync(p0, 0, 2 * (size_t)N * N * 4, st));
  else k_warm_dual<<<g1d((long)N * N), 256, 0, st>>>(choice == 1 ? n->phi : prior, p0, N);
  o.warm_start = 1;
  gp_report rep;
  r = emd_solve(h, f0, f1, m, p0, phi, N, &o, &rep, stream);
  if (r != GP_OK && !(r == GP_ERR_MAXITER || r == GP_ERR_DIVERGED || r == GP_ERR_NONFINITE))
    return cfail(n, r, gp_last_error(h));
  if (r != GP_OK) n->err = gp_last_error(h);
  if (n->bf16) {
    const gp_status q = tc_flag(n, st);
    if (q != GP_OK) return q;
  }
  rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (report) *report = rep;
  if (start_used) *start_used = choice;
  return r;
}


GP_API gp_status rof_solve_learned(gp_handle h, gp_cnn n, const float* I, float* u, float* p, int N, double lambda,
                                   int coarse_factor, const gp_opts* coarse_opts, const gp_opts* opts,
                                   gp_report* report, int* start_used, void* stream) {
  if (!h || !n || n->h != h) return GP_ERR_ARG;
  n->err.clear();
  const auto t0 = std::chrono::steady_clock::now();
  DevGuard g(n->device);
  gp_status r = check_batch(n, 1, &I, &I, nullptr, N);
  if (r != GP_OK) return r;
  if ((r = check_dev(n, u, "u")) != GP_OK) return r;
  if (p && (r = check_dev(n, p, "p")) != GP_OK) return r;
  if (coarse_factor < 0 || coarse_factor == 1) return cfail(n, GP_ERR_ARG, "coarse_factor must be 0 (none) or >= 2");
  if (!(lambda > 0)) return cfail(n, GP_ERR_ARG, "lambda must be > 0");
  gp_opts o;
  gp_default_opts(&o);
  if (opts) o = *opts;
  if (o.warm_start) return cfail(n, GP_ERR_ARG, "opts.warm_start must be 0: the start is chosen here");
  if ((r = reserve(n, 1, N)) != GP_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  const long NN = (long)N * N;
  // scratch: the two network inputs (tgt, dphi), the centred prior, the learned u, the probe p
  float* buf = nullptr;
  CN_CUDA(n, cudaMalloc(&buf, 4 * (size_t)NN * sizeof(float)));
  struct Free {
    float* b;
    ~Free() { cudaFree(b); }
  } fr{buf};
  float* pr = buf;
  float* ul = buf + NN;
  float* pp = buf + 2 * NN;
  const float* uprior = nullptr;
  const float* pprior = nullptr;
  if (coarse_factor) {
    gp_opts oc;
    gp_default_opts(&oc);
    oc.tol_rel_gap = 1e-4;
    oc.max_iters = 100000;
    oc.use_graph = o.use_graph;
    if (coarse_opts) oc = *coarse_opts;
    gp_report rc;
    r = rof_coarse_start(h, I, N, coarse_factor, lambda, &oc, n->prior, n->pw, &rc, stream);
    if (r != GP_OK && r != GP_ERR_MAXITER) return cfail(n, r, std::string("coarse start: ") + gp_last_error(h));
    uprior = n->prior;
    pprior = n->pw;
  }
  CN_CUDA(n, cudaMemsetAsync(n->dsc, 0, sizeof(double), st));
  k_sum64<<<g1d(NN), 256, 0, st>>>(I, NN, n->dsc);
  k_rof_net_inputs<<<g1d(NN), 256, 0, st>>>(I, uprior, n->dsc, n->tgt, n->dphi, pr, NN);
  CN_CUDA(n, cudaGetLastError());
  const float* fa = n->tgt;
  const float* fb = n->dphi;
  const float* prc = pr;
  if ((r = forward(n, 1, &fa, &fb, uprior ? &prc : nullptr, N, st)) != GP_OK) return r;
  k_rof_from_net<<<g1d(NN), 256, 0, st>>>(n->phi, n->dsc, ul, NN);
  CN_CUDA(n, cudaGetLastError());
  // Candidates: learned u (with the prior's p, else p = 0), the prior alone, zero;
  // the smallest duality gap at n = 0 decides.
  auto load = [&](const float* uc, const float* pc) -> gp_status {
    CN_CUDA(n, cudaMemcpyAsync(u, uc, NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (pc) CN_CUDA(n, cudaMemcpyAsync(pp, pc, 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
    else CN_CUDA(n, cudaMemsetAsync(pp, 0, 2 * NN * sizeof(float), st));
    return GP_OK;
  };
  gp_opts probe = o;
  probe.max_iters = 0;
  probe.warm_start = 1;
  double best = INFINITY;
  int choice = 0;
  const float* cu[2] = {ul, uprior};
  for (int c = 0; c < 2; ++c) {
    if (!cu[c]) continue;
    if ((r = load(cu[c], pprior)) != GP_OK) return r;
    gp_report rw;
    r = rof_solve(h, I, u, pp, N, lambda, &probe, &rw, stream);
    if (r != GP_OK && r != GP_ERR_MAXITER) return cfail(n, r, std::string("start probe: ") + gp_last_error(h));
    if (rw.rel_gap < best) {
      best = rw.rel_gap;
      choice = c == 0 ? 1 : 2;
    }
  }
  probe.warm_start = 0;
  gp_report rz;
  r = rof_solve(h, I, u, nullptr, N, lambda, &probe, &rz, stream);
  if (r != GP_OK && r != GP_ERR_MAXITER) return cfail(n, r, std::string("zero probe: ") + gp_last_error(h));
  if (!(best < rz.rel_gap)) choice = 0;
  gp_report rep;
  if (choice == 0) {
    r = rof_solve(h, I, u, p, N, lambda, &o, &rep, stream);
  } else {
    if ((r = load(choice == 1 ? ul : uprior, pprior)) != GP_OK) return r;
    o.warm_start = 1;
    r = rof_solve(h, I, u, pp, N, lambda, &o, &rep, stream);
    if (p) CN_CUDA(n, cudaMemcpyAsync(p, pp, 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  }
  if (r != GP_OK && !(r == GP_ERR_MAXITER || r == GP_ERR_DIVERGED || r == GP_ERR_NONFINITE))
    return cfail(n, r, gp_last_error(h));
  if (r != GP_OK) n->err = gp_last_error(h);
  CN_CUDA(n, cudaStreamSynchronize(st));
  if (n->bf16) {
    const gp_status q = tc_flag(n, st);
    if (q != GP_OK) return q;
  }
  rep.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (report) *report = rep;
  if (start_used) *start_used = choice;
  return r;
}

}  // extern "C"
