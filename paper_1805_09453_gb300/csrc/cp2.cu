// CP2: the accelerated primal-dual hybrid gradient method the paper compares
// G-prox PDHG with for ROF (section 4.1, Tables 4-5).  For the saddle problem
//   L(u, p) = (grad u, p) + lambda/2 ||u - I||^2 - chi(|p| <= 1)
// one iteration is
//   p_{n+1}   = proj(p_n + sigma_n grad ubar_n)                      (k_cp2_dual)
//   u_{n+1}   = (u_n + tau_n div p_{n+1} + tau_n lambda I) / (1 + tau_n lambda)
//   ubar_{n+1} = u_{n+1} + theta_n (u_{n+1} - u_n)                   (k_cp2_primal)
// with theta_n = 1 / sqrt(1 + 2 lambda tau_n), tau_{n+1} = theta_n tau_n,
// sigma_{n+1} = sigma_n / theta_n (the step sequence is computed on the host
// in FP64 and passed per launch).  No linear solve: two pointwise/stencil
// passes over HBM per iteration (dual: read ubar, p, write p; primal: read u,
// p, I, write u, ubar), the same discrete grad / div as the G-prox kernels.
#include "gp_internal.cuh"
#include "stencil.cuh"

namespace gp {
namespace {

__global__ void __launch_bounds__(256) k_cp2_dual(const float* __restrict__ ub, float* __restrict__ p, int N,
                                                  float invh, float sigma) {
  const size_t NN = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    const float c = ub[idx];
    const float gx = j < N - 1 ? (ub[idx + 1] - c) * invh : 0.f;  // forward differences, zero-flux slots
    const float gy = i < N - 1 ? (ub[idx + N] - c) * invh : 0.f;
    float px, py;
    proj2(p[idx] + sigma * gx, p[NN + idx] + sigma * gy, px, py);
    p[idx] = px;
    p[NN + idx] = py;
  }
}

__global__ void __launch_bounds__(256) k_cp2_primal(float* __restrict__ u, float* __restrict__ ub,
                                                    const float* __restrict__ p, const float* __restrict__ I, int N,
                                                    float invh, float tau, float lt, float inv1lt, float theta) {
  const size_t NN = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    // backward-difference divergence (= -grad^T); the last slot of each component is ignored
    const float d = ((j < N - 1 ? p[idx] : 0.f) - (j > 0 ? p[idx - 1] : 0.f) + (i < N - 1 ? p[NN + idx] : 0.f) -
                     (i > 0 ? p[NN + idx - N] : 0.f)) *
                    invh;
    const float uo = u[idx];
    const float un = (uo + tau * d + lt * I[idx]) * inv1lt;
    u[idx] = un;
    ub[idx] = un + theta * (un - uo);
  }
}

int grid_of(size_t n) {
  const size_t b = (n + 255) / 256;
  return (int)(b < 65535 * 8 ? b : 65535 * 8);
}

}  // namespace

cudaError_t launch_cp2_dual(const float* ubar, float* p, int N, float sigma, cudaStream_t st) {
  k_cp2_dual<<<grid_of((size_t)N * N), 256, 0, st>>>(ubar, p, N, (float)N, sigma);
  return cudaGetLastError();
}

cudaError_t launch_cp2_primal(float* u, float* ubar, const float* p, const float* I, int N, double tau, double lambda,
                              double theta, cudaStream_t st) {
  const double lt = tau * lambda;
  k_cp2_primal<<<grid_of((size_t)N * N), 256, 0, st>>>(u, ubar, p, I, N, (float)N, (float)tau, (float)lt,
                                                       (float)(1.0 / (1.0 + lt)), (float)theta);
  return cudaGetLastError();
}

}  // namespace gp
