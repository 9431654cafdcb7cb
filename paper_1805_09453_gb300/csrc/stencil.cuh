// Launchers of the fused stencil kernels and reductions (stencil.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace gp {

struct RofParams {
  int N;
  float invh, invh2;  // 1/h, 1/h^2
  float lt;           // lambda * tau
  float tau, sigma;
};

struct EmdParams {
  int N;
  float invh;
  float tau, sigma;
};

// Pointwise projection of the dual variable onto the unit disc (the
// proximal step of the dual's constraint |p| <= 1, sections 3.1 / 3.2).
__device__ __forceinline__ void proj2(float qx, float qy, float& px, float& py) {
  const float n2 = qx * qx + qy * qy;
  if (n2 > 1.f) {
    const float s = rsqrtf(n2);
    px = qx * s;
    py = qy * s;
  } else {
    px = qx;
    py = qy;
  }
}

// rb: row-block height of the fused kernels (4, 8, 16 or 32; anything else -> 16)
dim3 fused_grid(int N, int V, int rb);
int reduce_blocks_1d(size_t n);

cudaError_t launch_rof_fused(const float* gu, const float* u, const float* pin, const float* I, float* pout, float* r,
                             double* part, const RofParams& P, bool vec, bool gap, int rb, cudaStream_t st);
cudaError_t launch_emd_fused(const float* gq, const float* sin_, const float* pin, const float* g, float* sout,
                             float* pout, float* d, float* m, float* e, double* part, const EmdParams& P, bool vec,
                             bool gap, int rb, cudaStream_t st);
// r = -div p + Lap phi in FP64 (the dual potential's residual), stored FP32.
cudaError_t launch_dual_residual(const float* p, const float* phi, float* r, int N, cudaStream_t st);
// EMD dual bound inputs (sum phi (f1 - f0), max |D phi|) for phi = hi + lo, two
// FP32 planes, in FP64 with forward differences.
cudaError_t launch_emd_dual_hilo(const float* hi, const float* lo, const float* f0, const float* f1, int N,
                                 double* part, int nblk, cudaStream_t st);
cudaError_t launch_rof_stats(const float* I, int N, double* part, int nblk, cudaStream_t st);
cudaError_t launch_sq_dev(const float* I, size_t NN, float mean, double* part, int nblk, cudaStream_t st);
cudaError_t launch_rof_gap(const float* u, const float* p, const float* I, int N, double* part, int nblk,
                           cudaStream_t st);
cudaError_t launch_emd_primal(const float* m, const float* p, const float* f0, const float* f1, float* e, int N,
                              double* part, int nblk, cudaStream_t st);
// EMD feasibility certificate: rho = (f0 - f1) - div m (FP64, stored FP32) and
// sum |rho|; then sum |m + grad c| and sum |(f0 - f1) - div(m + grad c)|.
cudaError_t launch_emd_residual64(const float* m, const float* f0, const float* f1, float* rho, int N, double* part,
                                 int nblk, cudaStream_t st);
cudaError_t launch_emd_corrected(const float* m, const float* gc, const float* f0, const float* f1, int N,
                                 double* part, int nblk, cudaStream_t st);
cudaError_t launch_mass_stats(const float* f0, const float* f1, size_t NN, double* part, int nblk, cudaStream_t st);
cudaError_t launch_final_reduce(const double* part, int nblk, int nq, unsigned maxmask, double* out, cudaStream_t st);
cudaError_t launch_rof_init(const float* I, const float* u, const float* pbar, float* p, float* r, const RofParams& P,
                            cudaStream_t st);
cudaError_t launch_emd_init(const float* m0, const float* pbar, float* p, float* s, const float* g, float* d,
                            const EmdParams& P, cudaStream_t st);
cudaError_t launch_sub(const float* a, const float* b, float* out, size_t n, cudaStream_t st);
// Ergodic averages: sum += x (FP64 sums of FP32 planes); out = sum * scale;
// EMD flux m = s_sum * scale + grad q over two planes (n2 = 2 N^2).
cudaError_t launch_accumulate(double* sum, const float* x, size_t n, cudaStream_t st);
cudaError_t launch_scale_sum(const double* sum, float* out, size_t n, double scale, cudaStream_t st);
cudaError_t launch_emd_average_flux(const double* s_sum, const float* gq, float* m, size_t n2, double scale,
                                    cudaStream_t st);
cudaError_t launch_grad(const float* x, float* g, int N, cudaStream_t st);
// Refined split-precision solves: r = b - inv_scale (alpha - Lap) x in FP64; x += y.
cudaError_t launch_helmholtz_residual(const float* b, const float* x, float* r, int N, double alpha, double inv_scale,
                                     cudaStream_t st);
cudaError_t launch_add_inplace(float* x, const float* y, size_t n, cudaStream_t st);
// out = x - mean(x), the mean reduced on the device; part holds reduce_blocks_1d(n)
// doubles, sum one double.
cudaError_t launch_center(const float* x, float* out, size_t n, double* part, double* sum, cudaStream_t st);
// 3-D (N^3 volumes, (z, y, x), vector fields as three volumes; see stencil.cu).
cudaError_t launch_rof3_pstep(const float* gu, const float* pin, float* pout, int N, float sigma, cudaStream_t st);
cudaError_t launch_rof3_rhs(const float* pout, const float* pin, const float* gu, const float* I, float* r, int N,
                            float lt, float tau, cudaStream_t st);
cudaError_t launch_emd3_step(const float* gq, const float* sin_, const float* pin, float* sout, float* pout, float* m,
                             int N, float tau, float sigma, cudaStream_t st);
cudaError_t launch_emd3_rhs(const float* sout, const float* g, float* d, int N, cudaStream_t st);
cudaError_t launch_div3(const float* v, float* e, int N, float scale, cudaStream_t st);
cudaError_t launch_rof3_gap(const float* u, const float* gu, const float* I, const float* p, int N, double* part,
                            int nblk, cudaStream_t st);
cudaError_t launch_emd3_primal(const float* m, const float* g, int N, double* part, int nblk, cudaStream_t st);
cudaError_t launch_emd3_dual(const float* phi, const float* gphi, const float* f0, const float* f1, int N,
                             double* part, int nblk, cudaStream_t st);
cudaError_t launch_rof3_stats(const float* I, int N, double* part, int nblk, cudaStream_t st);
// CP2 (cp2.cu): p = proj(p + sigma grad ubar); then u' = (u + tau div p + tau lambda I) / (1 + tau lambda),
// ubar = u' + theta (u' - u), u = u'.
cudaError_t launch_cp2_dual(const float* ubar, float* p, int N, float sigma, cudaStream_t st);
cudaError_t launch_cp2_primal(float* u, float* ubar, const float* p, const float* I, int N, double tau, double lambda,
                              double theta, cudaStream_t st);
cudaError_t launch_copy_field(const float* a, float* b, int N, cudaStream_t st);

}  // namespace gp
