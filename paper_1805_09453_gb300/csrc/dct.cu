// Neumann Helmholtz / Poisson solve (alpha - Lap) x = b in the cosine basis.
//
// The even reflection of Appendix A (arXiv 1805.09453) makes every function
// on [0,1]^2 a cosine series, in which the 5-point Neumann Laplacian (the
// grad / div pair of the discretisation) is diagonal:
//     -Lap = C^T diag(mu_k + mu_l) C,  mu_k = (4/h^2) sin^2(pi k / 2N),
// with C the orthonormal DCT-II.  The solve is therefore
//     x = T^{-1} [ (T b T^T) / (alpha + mu_k + mu_l) ] T^{-T}
// for the unnormalised DCT-II T (the normalisations of C cancel).
//
// Fast path (power-of-two N, FP32): three HBM passes over the grid
//   1. rows:    DCT-II of every row                 (k_dct_rows_fwd)
//   2. columns: DCT-II, divide by the eigenvalue, inverse DCT-II of every
//               column, all in shared memory         (k_dct_cols_solve)
//   3. rows:    inverse DCT-II of every row          (k_dct_rows_inv)
// Each length-N DCT-II is one length-N complex FFT shared by two real
// sequences (z = a + i b) after Makhoul's even/odd reordering
//     v_n = x_{2n},  v_{N-1-n} = x_{2n+1},   X_k = Re(e^{-i pi k / 2N} V_k).
// The complex FFT is a self-sorting (Stockham) radix-16 transform in padded
// shared memory; each thread holds one 16-point butterfly in registers.
//
// Dense path (any N): four FP32 GEMMs with the orthonormal DCT-II matrix.
#include <math.h>

#include <vector>

#include "gp_internal.cuh"

namespace gp {
namespace {

constexpr float kRsqrt2 = 0.70710678118654752440f;
constexpr float kSqrt2 = 1.41421356237309504880f;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// Shared-memory padding: one slot per 16 complex values keeps the strided
// butterfly stores of the first Stockham stage free of bank conflicts.
__device__ __forceinline__ int padi(int a) { return a + (a >> 4); }

// e^{DIR 2 pi i m / 16} times a, for m known at compile time after unrolling.
template <int DIR>
__device__ __forceinline__ float2 mul_root16(float2 a, int m) {
  m &= 15;
  if (m == 0) return a;
  if (m == 8) return make_float2(-a.x, -a.y);
  if (m == 4) return DIR < 0 ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
  if (m == 12) return DIR < 0 ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
  const float C1 = 0.92387953251128675613f;  // cos(pi/8)
  const float C2 = 0.70710678118654752440f;  // cos(pi/4)
  const float C3 = 0.38268343236508977173f;  // cos(3pi/8)
  const float c[16] = {1.f, C1, C2, C3, 0.f, -C3, -C2, -C1, -1.f, -C1, -C2, -C3, 0.f, C3, C2, C1};
  const float s[16] = {0.f, C3, C2, C1, 1.f, C1, C2, C3, 0.f, -C3, -C2, -C1, -1.f, -C1, -C2, -C3};
  return cmul(a, make_float2(c[m], DIR < 0 ? -s[m] : s[m]));
}

__host__ __device__ constexpr int brev_small(int i, int R) {
  int r = 0;
  for (int b = 1; b < R; b <<= 1) r = (r << 1) | ((i & b) ? 1 : 0);
  return r;
}

// In-register R-point DFT (R = 2, 4, 8, 16), natural order in and out:
// iterative radix-2 decimation in time on bit-reversed input.
template <int R, int DIR>
__device__ __forceinline__ void dft_reg(float2* v) {
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int j = brev_small(i, R);
    if (j > i) {
      float2 t = v[i];
      v[i] = v[j];
      v[j] = t;
    }
  }
#pragma unroll
  for (int half = 1; half < R; half <<= 1) {
#pragma unroll
    for (int i = 0; i < R; i += 2 * half) {
#pragma unroll
      for (int k = 0; k < half; ++k) {
        const float2 b = mul_root16<DIR>(v[i + k + half], k * (8 / half));
        const float2 a = v[i + k];
        v[i + k] = cadd(a, b);
        v[i + k + half] = csub(a, b);
      }
    }
  }
}

// One self-sorting Stockham stage of radix R over a length-N complex array
// in (padded) shared memory, TPF threads per transform.
template <int N, int R, int DIR, int TPF>
__device__ __forceinline__ void fft_stage(float2* buf, const int Ns, const int t,
                                          const float2* __restrict__ tw) {
  constexpr int NB = N / R;
  constexpr int BPT = NB / TPF;
  static_assert(BPT >= 1 && NB % TPF == 0, "threads per transform must divide N/R");
  float2 v[BPT][R];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int j = t + b * TPF;
#pragma unroll
    for (int r = 0; r < R; ++r) v[b][r] = buf[padi(j + r * NB)];
  }
  __syncthreads();
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int j = t + b * TPF;
    const int k = j & (Ns - 1);
    if (Ns > 1) {
      const int step = NB / Ns;  // N / (Ns R)
#pragma unroll
      for (int r = 1; r < R; ++r) {
        float2 w = __ldg(&tw[r * k * step]);
        if (DIR > 0) w.y = -w.y;
        v[b][r] = cmul(v[b][r], w);
      }
    }
    dft_reg<R, DIR>(v[b]);
    const int base = (j - k) * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) buf[padi(base + r * Ns)] = v[b][r];
  }
  __syncthreads();
}

// Length-2^LOG2N complex FFT in shared memory (unnormalised), natural order.
// DIR = -1: forward e^{-i...}; DIR = +1: inverse without the 1/N factor.
template <int LOG2N, int DIR, int TPF>
__device__ __forceinline__ void fft_smem(float2* buf, int t, const float2* __restrict__ tw) {
  constexpr int N = 1 << LOG2N;
  constexpr int S16 = LOG2N / 4;
  constexpr int REM = 1 << (LOG2N % 4);
  int Ns = 1;
#pragma unroll
  for (int s = 0; s < S16; ++s) {
    fft_stage<N, 16, DIR, TPF>(buf, Ns, t, tw);
    Ns *= 16;
  }
  if constexpr (REM > 1) fft_stage<N, REM, DIR, TPF>(buf, Ns, t, tw);
}

// Makhoul position of sample n inside the reordered sequence v.
__device__ __forceinline__ int mk_pos(int n, int N) { return (n & 1) ? (N - 1 - (n >> 1)) : (n >> 1); }

// ----------------------------------------------------------------- pass 1
template <int LOG2N, int TPF, int FPC>
__global__ void __launch_bounds__(TPF* FPC) k_dct_rows_fwd(const float* __restrict__ in,
                                                         float* __restrict__ out,
                                                         const float2* __restrict__ tw,
                                                         const float2* __restrict__ wq) {
  constexpr int N = 1 << LOG2N;
  constexpr int PADN = N + N / 16;
  extern __shared__ float2 smem[];
  const int f = threadIdx.x / TPF, t = threadIdx.x % TPF;
  float2* buf = smem + f * PADN;
  const size_t ra = (size_t)(2 * (blockIdx.x * FPC + f)) * N;
  const float* __restrict__ xa = in + ra;
  const float* __restrict__ xb = xa + N;
  for (int j = 4 * t; j < N; j += 4 * TPF) {
    const float4 a = *reinterpret_cast<const float4*>(xa + j);
    const float4 b = *reinterpret_cast<const float4*>(xb + j);
    const int hj = j >> 1;
    buf[padi(hj)] = make_float2(a.x, b.x);
    buf[padi(N - 1 - hj)] = make_float2(a.y, b.y);
    buf[padi(hj + 1)] = make_float2(a.z, b.z);
    buf[padi(N - 2 - hj)] = make_float2(a.w, b.w);
  }
  __syncthreads();
  fft_smem<LOG2N, -1, TPF>(buf, t, tw);
  float* __restrict__ oa = out + ra;
  float* __restrict__ ob = oa + N;
  for (int k = t; k <= N / 2; k += TPF) {
    if (k == 0) {
      const float2 z = buf[0];
      oa[0] = z.x;
      ob[0] = z.y;
    } else if (k == N / 2) {
      const float2 z = buf[padi(N / 2)];
      oa[N / 2] = z.x * kRsqrt2;
      ob[N / 2] = z.y * kRsqrt2;
    } else {
      const float2 A = buf[padi(k)], B = buf[padi(N - k)];
      const float2 va = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
      const float2 vb = make_float2(0.5f * (A.y + B.y), -0.5f * (A.x - B.x));
      const float2 w = __ldg(&wq[k]);
      const float2 ya = cmul(w, va), yb = cmul(w, vb);
      oa[k] = ya.x;
      oa[N - k] = -ya.y;
      ob[k] = yb.x;
      ob[N - k] = -yb.y;
    }
  }
}

// Spectral factor of the solve at frequency (k, l): scale / ((alpha + mu_k + mu_l) N^2),
// 0 for the constant mode when alpha == 0.
__device__ __forceinline__ float spec_gain(int k, int l, const float* __restrict__ mu, float mul,
                                           float alpha, float sN2) {
  const float den = alpha + __ldg(&mu[k]) + mul;
  return den > 0.f ? sN2 / den : 0.f;
}

// ----------------------------------------------------------------- pass 2
template <int LOG2N, int TPF, int FPC>
__global__ void __launch_bounds__(TPF* FPC) k_dct_cols_solve(float* __restrict__ data,
                                                           const float2* __restrict__ tw,
                                                           const float2* __restrict__ wq,
                                                           const float* __restrict__ mu, float alpha,
                                                           float sN2) {
  constexpr int N = 1 << LOG2N;
  constexpr int PADN = N + N / 16;
  extern __shared__ float2 smem[];
  const int col0 = blockIdx.x * (2 * FPC);
  for (int idx = threadIdx.x; idx < N * FPC; idx += TPF * FPC) {
    const int n = idx / FPC, f = idx % FPC;
    const float2 v = *reinterpret_cast<const float2*>(data + (size_t)n * N + col0 + 2 * f);
    smem[f * PADN + padi(mk_pos(n, N))] = v;
  }
  __syncthreads();
  const int f = threadIdx.x / TPF, t = threadIdx.x % TPF;
  float2* buf = smem + f * PADN;
  fft_smem<LOG2N, -1, TPF>(buf, t, tw);
  const int la = col0 + 2 * f, lb = la + 1;
  const float mua = __ldg(&mu[la]), mub = __ldg(&mu[lb]);
  for (int k = t; k <= N / 2; k += TPF) {
    if (k == 0 || k == N / 2) {
      const int p = padi(k);
      const float2 z = buf[p];
      buf[p] = make_float2(z.x * spec_gain(k, la, mu, mua, alpha, sN2),
                           z.y * spec_gain(k, lb, mu, mub, alpha, sN2));
    } else {
      const float2 A = buf[padi(k)], B = buf[padi(N - k)];
      const float2 va = make_float2(0.5f * (A.x + B.x), 0.5f * (A.y - B.y));
      const float2 vb = make_float2(0.5f * (A.y + B.y), -0.5f * (A.x - B.x));
      const float2 w = __ldg(&wq[k]);
      const float2 ya = cmul(w, va), yb = cmul(w, vb);
      // forward spectra X[k] = Re y, X[N-k] = -Im y, then the eigenvalue gain
      const float gak = spec_gain(k, la, mu, mua, alpha, sN2);
      const float gan = spec_gain(N - k, la, mu, mua, alpha, sN2);
      const float gbk = spec_gain(k, lb, mu, mub, alpha, sN2);
      const float gbn = spec_gain(N - k, lb, mu, mub, alpha, sN2);
      const float2 wc = make_float2(w.x, -w.y);
      // inverse pre-step: V = conj(w) (X[k] - i X[N-k])
      const float2 ua = cmul(wc, make_float2(ya.x * gak, ya.y * gan));
      const float2 ub = cmul(wc, make_float2(yb.x * gbk, yb.y * gbn));
      buf[padi(k)] = make_float2(ua.x - ub.y, ua.y + ub.x);
      buf[padi(N - k)] = make_float2(ua.x + ub.y, -ua.y + ub.x);
    }
  }
  __syncthreads();
  fft_smem<LOG2N, +1, TPF>(buf, t, tw);
  for (int idx = threadIdx.x; idx < N * FPC; idx += TPF * FPC) {
    const int n = idx / FPC, ff = idx % FPC;
    *reinterpret_cast<float2*>(data + (size_t)n * N + col0 + 2 * ff) = smem[ff * PADN + padi(mk_pos(n, N))];
  }
}

// ----------------------------------------------------------------- pass 3
template <int LOG2N, int TPF, int FPC>
__global__ void __launch_bounds__(TPF* FPC) k_dct_rows_inv(const float* __restrict__ in,
                                                         float* __restrict__ out,
                                                         const float2* __restrict__ tw,
                                                         const float2* __restrict__ wq) {
  constexpr int N = 1 << LOG2N;
  constexpr int PADN = N + N / 16;
  extern __shared__ float2 smem[];
  const int f = threadIdx.x / TPF, t = threadIdx.x % TPF;
  float2* buf = smem + f * PADN;
  const size_t ra = (size_t)(2 * (blockIdx.x * FPC + f)) * N;
  const float* __restrict__ xa = in + ra;
  const float* __restrict__ xb = xa + N;
  for (int k = t; k <= N / 2; k += TPF) {
    if (k == 0) {
      buf[0] = make_float2(xa[0], xb[0]);
    } else if (k == N / 2) {
      buf[padi(N / 2)] = make_float2(kSqrt2 * xa[N / 2], kSqrt2 * xb[N / 2]);
    } else {
      const float2 w = __ldg(&wq[k]);
      const float2 wc = make_float2(w.x, -w.y);
      const float2 ua = cmul(wc, make_float2(xa[k], -xa[N - k]));
      const float2 ub = cmul(wc, make_float2(xb[k], -xb[N - k]));
      buf[padi(k)] = make_float2(ua.x - ub.y, ua.y + ub.x);
      buf[padi(N - k)] = make_float2(ua.x + ub.y, -ua.y + ub.x);
    }
  }
  __syncthreads();
  fft_smem<LOG2N, +1, TPF>(buf, t, tw);
  float* __restrict__ oa = out + ra;
  float* __restrict__ ob = oa + N;
  for (int j = 4 * t; j < N; j += 4 * TPF) {
    const int hj = j >> 1;
    const float2 z0 = buf[padi(hj)], z1 = buf[padi(N - 1 - hj)];
    const float2 z2 = buf[padi(hj + 1)], z3 = buf[padi(N - 2 - hj)];
    *reinterpret_cast<float4*>(oa + j) = make_float4(z0.x, z1.x, z2.x, z3.x);
    *reinterpret_cast<float4*>(ob + j) = make_float4(z0.y, z1.y, z2.y, z3.y);
  }
}

// Launch configuration per size: threads per transform (TPF = N/16 / split)
// and transforms per CTA for the row passes (FPR) and the column pass (FPCc).
template <int LOG2N>
struct FftCfg {
  static constexpr int N = 1 << LOG2N;
  static constexpr int TPF = N / 16;
  static constexpr int FPR = (TPF >= 256) ? 1 : (256 / TPF < N / 2 ? 256 / TPF : N / 2);
  static constexpr int FPC = (N >= 4096) ? 2 : (TPF >= 128 ? 2 : (256 / TPF < 8 ? 256 / TPF : 8));
};

template <int LOG2N>
cudaError_t launch_fft_pass(const DctPlan& p, int pass, const float* in, float* out, float alpha, float scale,
                            cudaStream_t st) {
  using Cfg = FftCfg<LOG2N>;
  constexpr int N = Cfg::N;
  constexpr int PADN = N + N / 16;
  const size_t smR = (size_t)Cfg::FPR * PADN * sizeof(float2);
  const size_t smC = (size_t)Cfg::FPC * PADN * sizeof(float2);
  cudaError_t e;
  if (pass == 0) {
    auto k = k_dct_rows_fwd<LOG2N, Cfg::TPF, Cfg::FPR>;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smR))) return e;
    k<<<N / 2 / Cfg::FPR, Cfg::TPF * Cfg::FPR, smR, st>>>(in, out, p.tw, p.wq);
  } else if (pass == 1) {
    auto k = k_dct_cols_solve<LOG2N, Cfg::TPF, Cfg::FPC>;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smC))) return e;
    const float sN2 = (float)((double)scale / ((double)N * (double)N));
    k<<<N / 2 / Cfg::FPC, Cfg::TPF * Cfg::FPC, smC, st>>>(out, p.tw, p.wq, p.mu, alpha, sN2);
  } else {
    auto k = k_dct_rows_inv<LOG2N, Cfg::TPF, Cfg::FPR>;
    if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smR))) return e;
    k<<<N / 2 / Cfg::FPR, Cfg::TPF * Cfg::FPR, smR, st>>>(in, out, p.tw, p.wq);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------ dense path
// D = op(A) * op(B), all N x N row-major; op = transpose when the flag is set.
template <bool TA, bool TB>
__global__ void __launch_bounds__(256) k_gemm_nn(const float* __restrict__ A, const float* __restrict__ B,
                                                 float* __restrict__ D, int N) {
  __shared__ float As[32][33];
  __shared__ float Bs[32][33];
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 32 x 8
  const int row0 = blockIdx.y * 32, col0 = blockIdx.x * 32;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < N; k0 += 32) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = ty + 8 * q;
      // As[r][c] = op(A)[row0 + r][k0 + c]
      {
        const int gi = row0 + r, gk = k0 + tx;
        float v = 0.f;
        if (gi < N && gk < N) v = TA ? A[(size_t)gk * N + gi] : A[(size_t)gi * N + gk];
        As[r][tx] = v;
      }
      // Bs[r][c] = op(B)[k0 + r][col0 + c]
      {
        const int gk = k0 + r, gj = col0 + tx;
        float v = 0.f;
        if (gk < N && gj < N) v = TB ? B[(size_t)gj * N + gk] : B[(size_t)gk * N + gj];
        Bs[r][tx] = v;
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const float bv = Bs[kk][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(As[ty + 8 * q][kk], bv, acc[q]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int gi = row0 + ty + 8 * q, gj = col0 + tx;
    if (gi < N && gj < N) D[(size_t)gi * N + gj] = acc[q];
  }
}

__global__ void k_spec_scale_dense(float* __restrict__ X, const float* __restrict__ mu, int N, float alpha,
                                   float scale) {
  const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (size_t)N * N) return;
  const int k = (int)(idx / N), l = (int)(idx % N);
  const float den = alpha + mu[k] + mu[l];
  X[idx] = den > 0.f ? X[idx] * (scale / den) : 0.f;
}

}  // namespace

cudaError_t dct_solve_dense_fp32(const DctPlan& p, const float* b, float* x, float* tmp, float alpha,
                                 float scale, cudaStream_t st) {
  const int N = p.N;
  float* t0 = tmp;
  float* t1 = tmp + (size_t)N * N;
  dim3 g(ceil_div(N, 32), ceil_div(N, 32));
  k_gemm_nn<false, true><<<g, 256, 0, st>>>(b, p.C, t0, N);   // b C^T   (rows)
  k_gemm_nn<false, false><<<g, 256, 0, st>>>(p.C, t0, t1, N);  // C (.)    (columns)
  const size_t NN = (size_t)N * N;
  k_spec_scale_dense<<<(unsigned)((NN + 255) / 256), 256, 0, st>>>(t1, p.mu, N, alpha, scale);
  k_gemm_nn<true, false><<<g, 256, 0, st>>>(p.C, t1, t0, N);   // C^T (.)
  k_gemm_nn<false, false><<<g, 256, 0, st>>>(t0, p.C, x, N);   // (.) C
  return cudaGetLastError();
}

cudaError_t dct_fft_pass(const DctPlan& p, int pass, const float* in, float* out, float alpha, float scale,
                         cudaStream_t st) {
  if (!p.fft) return cudaErrorInvalidValue;
  switch (p.N) {
    case 16: return launch_fft_pass<4>(p, pass, in, out, alpha, scale, st);
    case 32: return launch_fft_pass<5>(p, pass, in, out, alpha, scale, st);
    case 64: return launch_fft_pass<6>(p, pass, in, out, alpha, scale, st);
    case 128: return launch_fft_pass<7>(p, pass, in, out, alpha, scale, st);
    case 256: return launch_fft_pass<8>(p, pass, in, out, alpha, scale, st);
    case 512: return launch_fft_pass<9>(p, pass, in, out, alpha, scale, st);
    case 1024: return launch_fft_pass<10>(p, pass, in, out, alpha, scale, st);
    case 2048: return launch_fft_pass<11>(p, pass, in, out, alpha, scale, st);
    case 4096: return launch_fft_pass<12>(p, pass, in, out, alpha, scale, st);
    case 8192: return launch_fft_pass<13>(p, pass, in, out, alpha, scale, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t dct_plan_init(DctPlan& p, int N) {
  p.N = N;
  p.fft = (N >= 16 && N <= 8192 && (N & (N - 1)) == 0);
  const double PI = 3.14159265358979323846;
  const double h = 1.0 / N;
  std::vector<float> mu(N);
  for (int k = 0; k < N; ++k) {
    const double s = sin(PI * k / (2.0 * N));
    mu[k] = (float)(4.0 / (h * h) * s * s);
  }
  cudaError_t e;
  if ((e = cudaMalloc(&p.mu, sizeof(float) * N))) return e;
  if ((e = cudaMemcpy(p.mu, mu.data(), sizeof(float) * N, cudaMemcpyHostToDevice))) return e;
  if (p.fft) {
    std::vector<float2> tw(N), wq(N / 2 + 1);
    for (int m = 0; m < N; ++m) tw[m] = make_float2((float)cos(2 * PI * m / N), (float)-sin(2 * PI * m / N));
    for (int k = 0; k <= N / 2; ++k) wq[k] = make_float2((float)cos(PI * k / (2.0 * N)), (float)-sin(PI * k / (2.0 * N)));
    if ((e = cudaMalloc(&p.tw, sizeof(float2) * N))) return e;
    if ((e = cudaMalloc(&p.wq, sizeof(float2) * (N / 2 + 1)))) return e;
    if ((e = cudaMemcpy(p.tw, tw.data(), sizeof(float2) * N, cudaMemcpyHostToDevice))) return e;
    if ((e = cudaMemcpy(p.wq, wq.data(), sizeof(float2) * (N / 2 + 1), cudaMemcpyHostToDevice))) return e;
  }
  // The dense matrix serves the sizes without a fast transform.
  if (!p.fft) {
    std::vector<float> C((size_t)N * N);
    for (int k = 0; k < N; ++k) {
      const double s = (k == 0) ? sqrt(1.0 / N) : sqrt(2.0 / N);
      for (int n = 0; n < N; ++n) C[(size_t)k * N + n] = (float)(s * cos(PI * k * (2.0 * n + 1.0) / (2.0 * N)));
    }
    if ((e = cudaMalloc(&p.C, sizeof(float) * (size_t)N * N))) return e;
    if ((e = cudaMemcpy(p.C, C.data(), sizeof(float) * (size_t)N * N, cudaMemcpyHostToDevice))) return e;
  }
  return cudaSuccess;
}

void dct_plan_free(DctPlan& p) {
  if (p.tw) cudaFree(p.tw);
  if (p.wq) cudaFree(p.wq);
  if (p.mu) cudaFree(p.mu);
  if (p.C) cudaFree(p.C);
  p = DctPlan();
}

}  // namespace gp
