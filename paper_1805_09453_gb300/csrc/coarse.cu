// emd_coarse_start: the EMD dual potential solved on a grid `factor` times
// coarser and interpolated back to N x N, as a start (or network prior) for
// the fine solve.
//
// Restriction: block means of the densities (the same total mass on the
// coarse grid, h_c = factor / N).  The coarse problem is solved with
// emd_solve; its potential phi_c = Lap^{-1} div p (section 4.2's dual
// variable, |grad phi| <= 1 at the saddle point) is interpolated bilinearly
// between cell centres, constant beyond the outermost coarse centres.
#include <math.h>

#include <string>

#include "gp_internal.cuh"

namespace {

// c[I][J] = mean of f over the factor x factor block of coarse cell (I, J)
__global__ void k_restrict_mean(const float* __restrict__ f, float* __restrict__ c, int N, int k) {
  const int n = N / k;
  const long nn = (long)n * n;
  const float w = 1.f / ((float)k * (float)k);
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < nn; idx += (long)gridDim.x * blockDim.x) {
    const int I = (int)(idx / n), J = (int)(idx % n);
    float s = 0.f;
    for (int a = 0; a < k; ++a) {
      const float* row = f + (long)(I * k + a) * N + (long)J * k;
      for (int b = 0; b < k; ++b) s += row[b];
    }
    c[idx] = s * w;
  }
}

// Cell-centred bilinear interpolation from n x n to N = n k: fine centre j
// sits at coarse coordinate (j + 1/2)/k - 1/2, clamped to [0, n - 1].
__device__ __forceinline__ void lerp_coord(int j, int n, int k, int& i0, int& i1, float& t) {
  float x = ((float)j + 0.5f) / (float)k - 0.5f;
  x = fminf(fmaxf(x, 0.f), (float)(n - 1));
  i0 = min((int)x, n - 1);
  i1 = min(i0 + 1, n - 1);
  t = x - (float)i0;
}

__global__ void k_upsample_bilinear(const float* __restrict__ c, float* __restrict__ f, int N, int k) {
  const int n = N / k;
  const long NN = (long)N * N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < NN; idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    int r0, r1, c0, c1;
    float ty, tx;
    lerp_coord(i, n, k, r0, r1, ty);
    lerp_coord(j, n, k, c0, c1, tx);
    const float a = c[(long)r0 * n + c0] * (1.f - tx) + c[(long)r0 * n + c1] * tx;
    const float b = c[(long)r1 * n + c0] * (1.f - tx) + c[(long)r1 * n + c1] * tx;
    f[idx] = a * (1.f - ty) + b * ty;
  }
}

// Interpolated dual field -> a feasible start: zero structural slots (x: last
// column, y: last row), then |p| <= 1 pointwise.
__global__ void k_dual_feasible(float* __restrict__ p, int N) {
  const long NN = (long)N * N;
  for (long idx = blockIdx.x * (long)blockDim.x + threadIdx.x; idx < NN; idx += (long)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    float px = j < N - 1 ? p[idx] : 0.f;
    float py = i < N - 1 ? p[NN + idx] : 0.f;
    const float nrm = sqrtf(px * px + py * py);
    if (nrm > 1.f) {
      px /= nrm;
      py /= nrm;
    }
    p[idx] = px;
    p[NN + idx] = py;
  }
}

inline int g1d(long n) { return (int)std::min<long>((n + 255) / 256, 8192); }

}  // namespace

extern "C" GP_API gp_status emd_coarse_start(gp_handle h, const float* f0, const float* f1, int N, int factor,
                                             const gp_opts* opts, float* phi, gp_report* report, void* stream) {
  if (!h) return GP_ERR_ARG;
  if (factor < 2 || N % factor != 0 || N / factor < 2) return GP_ERR_ARG;
  if (!f0 || !f1 || !phi) return GP_ERR_ARG;
  gp_opts o;
  gp_default_opts(&o);
  if (opts) o = *opts;
  if (o.warm_start) return GP_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(gp::handle_device(h)) != cudaSuccess) return GP_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = N / factor;
  const size_t nn = (size_t)n * n;
  float* buf = nullptr;  // c0, c1 (n^2 each), m (2 n^2), phi_c (n^2)
  gp_status r = GP_OK;
  if (cudaMalloc(&buf, 5 * nn * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    r = GP_ERR_CUDA;
  } else {
    float *c0 = buf, *c1 = buf + nn, *mc = buf + 2 * nn, *pc = buf + 4 * nn;
    k_restrict_mean<<<g1d((long)nn), 256, 0, st>>>(f0, c0, N, factor);
    k_restrict_mean<<<g1d((long)nn), 256, 0, st>>>(f1, c1, N, factor);
    if (cudaGetLastError() != cudaSuccess) r = GP_ERR_CUDA;
    gp_report rc;
    if (r == GP_OK) r = emd_solve(h, c0, c1, mc, nullptr, pc, n, &o, &rc, stream);
    if (r == GP_OK || r == GP_ERR_MAXITER) {
      k_upsample_bilinear<<<g1d((long)N * N), 256, 0, st>>>(pc, phi, N, factor);
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) r = GP_ERR_CUDA;
      if (report) *report = rc;
    }
    cudaFree(buf);
  }
  if (prev >= 0) cudaSetDevice(prev);
  return r;
}

// rof_coarse_start: the ROF pair (u, p) solved on a grid `factor` times
// coarser and interpolated back.  The image is restricted by block means; the
// coarse problem is the same continuum energy (section 3.1, the same lambda,
// h_c = factor / N), solved with rof_solve; u_c and both components of p_c
// are interpolated bilinearly between cell centres, and the interpolated p is
// made feasible (zero slots, |p| <= 1).
extern "C" GP_API gp_status rof_coarse_start(gp_handle h, const float* I, int N, int factor, double lambda,
                                             const gp_opts* opts, float* u, float* p, gp_report* report,
                                             void* stream) {
  if (!h) return GP_ERR_ARG;
  if (factor < 2 || N % factor != 0 || N / factor < 2) return GP_ERR_ARG;
  if (!I || !u || !p || !(lambda > 0)) return GP_ERR_ARG;
  gp_opts o;
  gp_default_opts(&o);
  if (opts) o = *opts;
  if (o.warm_start) return GP_ERR_ARG;
  int prev = -1;
  cudaGetDevice(&prev);
  if (cudaSetDevice(gp::handle_device(h)) != cudaSuccess) return GP_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)stream;
  const int n = N / factor;
  const size_t nn = (size_t)n * n;
  float* buf = nullptr;  // I_c, u_c (n^2 each), p_c (2 n^2)
  gp_status r = GP_OK;
  if (cudaMalloc(&buf, 4 * nn * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    r = GP_ERR_CUDA;
  } else {
    float *ic = buf, *uc = buf + nn, *pc = buf + 2 * nn;
    k_restrict_mean<<<g1d((long)nn), 256, 0, st>>>(I, ic, N, factor);
    if (cudaGetLastError() != cudaSuccess) r = GP_ERR_CUDA;
    gp_report rc;
    if (r == GP_OK) r = rof_solve(h, ic, uc, pc, n, lambda, &o, &rc, stream);
    if (r == GP_OK || r == GP_ERR_MAXITER) {
      const long NN = (long)N * N;
      k_upsample_bilinear<<<g1d(NN), 256, 0, st>>>(uc, u, N, factor);
      k_upsample_bilinear<<<g1d(NN), 256, 0, st>>>(pc, p, N, factor);
      k_upsample_bilinear<<<g1d(NN), 256, 0, st>>>(pc + nn, p + NN, N, factor);
      k_dual_feasible<<<g1d(NN), 256, 0, st>>>(p, N);
      if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(st) != cudaSuccess) r = GP_ERR_CUDA;
      if (report) *report = rc;
    }
    cudaFree(buf);
  }
  if (prev >= 0) cudaSetDevice(prev);
  return r;
}
