// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "gprox.h"

namespace gp {

// ---------------------------------------------------------------- helpers
__host__ __device__ inline int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Neumaier (compensated) FP32 accumulator: per-thread partial sums whose
// error does not grow with the number of terms; each thread's result is
// widened to FP64 before the cross-thread reduction.
struct CSum {
  float s, c;
  __device__ __forceinline__ CSum() : s(0.f), c(0.f) {}
  __device__ __forceinline__ void add(float x) {
    float t = s + x;
    if (fabsf(s) >= fabsf(x)) c += (s - t) + x;
    else c += (x - t) + s;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

// Per-solve cosine-transform plan (one per grid size N, owned by the handle).
struct DctPlan {
  int N = 0;
  bool fft = false;          // power-of-two fast transform available
  float2* tw = nullptr;      // e^{-2 pi i m / N}, m < N          (fft)
  float2* wq = nullptr;      // e^{-i pi k / (2N)}, k <= N/2       (fft)
  float* mu = nullptr;       // (4/h^2) sin^2(pi k / 2N), k < N
  float* C = nullptr;        // orthonormal DCT-II matrix, N x N   (dense)
  float* CT = nullptr;       // its transpose (tensor-core path)
  float* E = nullptr;        // derivative synthesis C D^T: E[k][j] = N (C[k][j+1] - C[k][j]), 0 at j = N-1
  float* ET = nullptr;       // its transpose
  // C, C^T, E, E^T split into hi / lo BF16 in the tensor-core tile layout
  // (128 x 64 tiles, hi slab then lo slab, 32 KiB per tile; 4 N^2 bytes each)
  void* Cs = nullptr;
  void* CTs = nullptr;
  void* Es = nullptr;
  void* ETs = nullptr;
  // the same in hi / lo FP16, scaled by a power of two (FP16 split mode), and
  // that mode's scale / maximum slots (32 floats, see tc_gemm.cu)
  void* Cs16 = nullptr;
  void* CTs16 = nullptr;
  void* Es16 = nullptr;
  void* ETs16 = nullptr;
  float* tc16 = nullptr;
  int* err = nullptr;  // fast sizes: set to 1 by a transform kernel whose bulk copy never landed
};

// Launchers (dct.cu)
cudaError_t dct_plan_init(DctPlan& p, int N);
void dct_plan_free(DctPlan& p);
// One pass of the fast solve x = scale * (alpha - Lap)^{-1} b:
//   pass 0: tmp = row DCT-II of b          (in = b,   out = tmp)
//   pass 1: column solve in place on tmp    (out = tmp)
//   pass 2: x = row inverse DCT-II of tmp   (in = tmp, out = x)
// tmp (N*N floats) holds spectra in a 4-row-interleaved layout; b may alias x.
cudaError_t dct_fft_pass(const DctPlan& p, int pass, const float* in, float* out, float alpha, float scale,
                         cudaStream_t st);
// Gradient solve: after pass 0 (tmp = row spectra of b),
//   dct_grad_cols(tmp -> A, B)  and  dct_grad_rows(A, B -> gx, gy [, phi])
// give gx, gy = forward-difference gradient of x = scale (alpha - Lap)^{-1} b,
// taken in the spectral domain, and optionally x itself (phi).  A may alias
// tmp; A and B are N*N each.
cudaError_t dct_grad_cols(const DctPlan& p, const float* in, float* A, float* B, float alpha, float scale,
                          cudaStream_t st);
cudaError_t dct_grad_rows(const DctPlan& p, const float* A, const float* B, float* gx, float* gy, float* phi,
                          cudaStream_t st);
// At N = 4096 (fftreg.cu) the gradient solve runs register-resident
// transforms on pair-interleaved spectra (rows 2q, 2q + 1 as N float2 per row
// pair) instead of the 4-row layout: its forward row pass is rows_fwd_4k
// (not dct_fft_pass 0), and dct_grad_cols / dct_grad_rows take and give that
// layout; cudaErrorNotSupported (nothing launched) for other plans or when
// the column pass's tensor maps cannot be made.
bool grad4k_supported(const DctPlan& p);
cudaError_t rows_fwd_4k(const DctPlan& p, const float* in, float* out, cudaStream_t st);
cudaError_t grad_cols_4k(const DctPlan& p, const float* in, float* A, float* B, float alpha, float scale,
                         cudaStream_t st);
cudaError_t grad_rows_4k(const DctPlan& p, const float* A, const float* B, float* gx, float* gy, float* phi,
                         cudaStream_t st);
// One non-gap step fused with its solve's row syntheses and the next solve's
// forward row pass (A, B: the column pass's outputs; out: the next row
// spectra, pair-interleaved).  ROF: p_in, I -> p_out; EMD: s_in, p_in, g ->
// s_out, p_out.  All pointers 16-byte aligned.
struct EmdParams;
struct RofParams;
cudaError_t rof_rows_step_4k(const DctPlan& p, const float* A, const float* B, const float* pin, const float* I,
                             float* pout, float* out, const RofParams& P, cudaStream_t st);
cudaError_t emd_rows_step_4k(const DctPlan& p, const float* A, const float* B, const float* sin_, const float* pin,
                             const float* g, float* sout, float* pout, float* out, const EmdParams& P,
                             cudaStream_t st);
// One non-gap iteration's stencil (k_emd_fused / k_rof_fused arithmetic)
// fused with the forward row pass of the next solve: writes s', p' (EMD) or
// p' (ROF) and, instead of the right-hand side itself, its row spectra `out`
// in the interleaved layout of pass 0.  Fast sizes only; all pointers
// 16-byte aligned.
struct EmdParams;
struct RofParams;
cudaError_t dct_emd_step_fwd(const DctPlan& p, const float* gq, const float* sin_, const float* pin, const float* g,
                             float* sout, float* pout, float* out, const EmdParams& P, cudaStream_t st);
cudaError_t dct_rof_step_fwd(const DctPlan& p, const float* gu, const float* pin, const float* I, float* pout,
                             float* out, const RofParams& P, cudaStream_t st);
// 3-D volumes (z, y, x), x fastest, power-of-two N in [16, 512]: one pass of
// line transforms along `axis` (0 x, 1 y, 2 z); mode 0 forward DCT-II, 1 plain
// cosine synthesis, 2 forward-difference synthesis (in may equal out); and the
// spectral gain X *= scale / ((alpha + mu_x + mu_y + mu_z) N^3).
cudaError_t dct3_lines(const DctPlan& p, const float* in, float* out, int axis, int mode, cudaStream_t st);
cudaError_t dct3_gain(const DctPlan& p, float* X, float alpha, float scale, cudaStream_t st);
cudaError_t solve_grad3(const DctPlan& p, const float* b, float* g3, float* u, float* W0, float* W1, float* W2,
                        float alpha, float scale, cudaStream_t st, int* nlaunch);
// Build C (and C^T) for a plan that lacks them (tensor-core path).
cudaError_t dct_plan_dense(DctPlan& p);
// Split-precision (hi + lo BF16, or FP16 with power-of-two scales) tensor-core
// form, N % 128 == 0: four tcgen05 GEMMs (FP16: each product staged in FP32
// and split with its own scale, x used as the staging plane); tmp holds
// 2*N*N floats; *err is set to 1 if a wait timed out.
bool tc_solve_supported(int N);
// Warm-start network (BF16 mode): 3x3 convolutions as tcgen05 implicit GEMMs
// (cnn_tc.cu).  A convolution's BF16 weights W [Cout][Cin][3][3] are first
// packed into two tensor-core images (conv3x3_tc_image_elems elements, 16-byte
// aligned): the forward image, then the data-gradient (flipped, transposed)
// image.  *err is set to 1 if a wait timed out.
size_t conv3x3_tc_image_elems(int Cin, int Cout);
cudaError_t conv3x3_tc_pack(const void* W, int Cin, int Cout, void* img, cudaStream_t st);
// Y = act(conv(X) + bias): X BF16, Y BF16 (or FP32 when y_fp32).
cudaError_t conv3x3_tc(const void* X, long xbs, int Cin, const void* img, const float* bias, void* Y, long ybs, int Cout,
                       int H, int Wd, int B, bool relu, bool y_fp32, int* err, cudaStream_t st);
// Weight and bias gradients (accumulated into dW [Cout][Cin][3][3] and db, which may be null):
// dY FP32 as a hi + lo BF16 pair, X BF16.
cudaError_t conv3x3_wgrad_tc(const float* dY, long dybs, int Cout, const void* X, long xbs, int Cin, int H, int Wd,
                             int B, float* dW, float* db, int* err, cudaStream_t st);
// Data gradient dX (written, FP32) from dY (FP32, hi + lo BF16) and the data-gradient image.
cudaError_t conv3x3_dgrad_tc(const float* dY, long dybs, int Cout, const void* img, float* dX, long dxbs, int Cin,
                             int H, int Wd, int B, int* err, cudaStream_t st);
cudaError_t dct_solve_tc(const DctPlan& p, const float* b, float* x, float* tmp, float alpha, float scale, int* err,
                         cudaStream_t st, bool fp16);
// Gradient of the split-precision solve, taken in the spectral domain with
// tensor-core GEMMs (7, or 8 with phi): gx = C^T Q E, gy = E^T Q C with
// Q = gain .* (C b C^T).  tmp holds 2*N*N floats; gy doubles as scratch.
cudaError_t dct_plan_grad_dense(DctPlan& p);
// Pre-split tile copies of the dense matrices the plan has (tensor-core path;
// fp16: the scaled FP16 copies and the mode's slot array).
cudaError_t dct_plan_tc_split(DctPlan& p, cudaStream_t st, bool fp16);
cudaError_t dct_grad_tc(const DctPlan& p, const float* b, float* gx, float* gy, float* phi, float* tmp, float alpha,
                        float scale, int* err, cudaStream_t st, bool fp16);
// Dense-matrix form (any N): tmp must hold 2*N*N floats.
cudaError_t dct_solve_dense_fp32(const DctPlan& p, const float* b, float* x, float* tmp,
                                 float alpha, float scale, cudaStream_t st);

// Device ordinal a handle was created on (api.cu).
int handle_device(gp_handle h);

// Error text of the last failed handle-free call on this thread (static_solve.cu).
const char* static_last_error();

// Reduction helpers (stencil.cu)
constexpr int kRedThreads = 256;
constexpr int kMaxQ = 4;

}  // namespace gp
