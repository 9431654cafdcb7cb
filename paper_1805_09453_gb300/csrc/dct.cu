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
// Between passes the spectra live in a 4-row-interleaved layout so that the
// row passes (4 rows per CTA) and the column pass (2 columns per CTA) all
// move contiguous, full-sector blocks; at N >= 512 (gradient form) and
// N >= 2048 (plain solve) the column passes move them with bulk tensor
// copies.
//
// Gradient variant (ROF and EMD steps): the column and last row pass also
// synthesise the forward differences of the solution directly from its
// spectrum, so that the gradient keeps FP32 relative precision at any N
// (differencing an FP32 potential loses about log2(N) bits).  Inside a chunk
// of steps the forward row pass of the next solve runs in the same CTAs as
// the step's stencil (k_rof_step_rows_fwd, k_emd_step_rows_fwd).
//
// Dense path (any N): four FP32 GEMMs with the orthonormal DCT-II matrix.
#include <math.h>

#include <vector>

#include "fft_common.cuh"
#include "gp_internal.cuh"
#include "stencil.cuh"
#include "tma.cuh"

namespace gp {
namespace {

constexpr float kRsqrt2 = 0.70710678118654752440f;
constexpr float kSqrt2 = 1.41421356237309504880f;

// Shared-memory padding: one slot per 16 complex values keeps the strided
// butterfly stores of the first Stockham stage free of bank conflicts.
__device__ __forceinline__ int padi(int a) { return a + (a >> 4); }

// Twiddles w_r = e^{DIR 2 pi i r m / N}, r < R, from at most four table loads
// (w1, w2, w4, w8); the others are products of two or three of them.
template <int R, int DIR>
__device__ __forceinline__ void stage_twiddles(const float2* __restrict__ tw, int m, float2 (&w)[R]) {
  w[0] = make_float2(1.f, 0.f);
  if constexpr (R >= 2) w[1] = __ldg(&tw[m]);
  if constexpr (R >= 4) {
    w[2] = __ldg(&tw[2 * m]);
    w[3] = cmul(w[1], w[2]);
  }
  if constexpr (R >= 8) {
    w[4] = __ldg(&tw[4 * m]);
#pragma unroll
    for (int r = 5; r < 8; ++r) w[r] = cmul(w[r - 4], w[4]);
  }
  if constexpr (R >= 16) {
    w[8] = __ldg(&tw[8 * m]);
#pragma unroll
    for (int r = 9; r < 16; ++r) w[r] = cmul(w[r - 8], w[8]);
  }
  if constexpr (DIR > 0) {
#pragma unroll
    for (int r = 1; r < R; ++r) w[r].y = -w[r].y;
  }
}

// One self-sorting Stockham stage of radix R over a length-N complex array
// in (padded) shared memory, TPF threads per transform.  Padded addresses
// are formed once per butterfly and advanced by compile-time strides: with
// NB and Ns multiples of 16, padi(a + r*S) = padi(a) + r*(S + S/16); for the
// first stage (Ns = 1) the store index is 16j + r, whose padded form is
// padi(16j) + r.
// Barrier of a transform's threads: the whole CTA (bar == 0) or named barrier
// `bar` shared by the NT threads of one transform group (NT a multiple of 32).
__device__ __forceinline__ void gsync(int bar, int nt) {
  if (bar == 0) __syncthreads();
  else asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
}

template <int N, int R, int DIR, int TPF>
__device__ __forceinline__ void fft_stage(float2* buf, const int Ns, const int t,
                                          const float2* __restrict__ tw, int bar = 0) {
  constexpr int NB = N / R;
  constexpr int BPT = NB / TPF;
  static_assert(BPT >= 1 && NB % TPF == 0, "threads per transform must divide N/R");
  constexpr int LD = (NB % 16 == 0) ? NB + NB / 16 : 0;  // padded load stride (0: generic path)
  float2 v[BPT][R];
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int j = t + b * TPF;
    if constexpr (LD != 0) {
      const float2* src = buf + padi(j);
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = src[r * LD];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) v[b][r] = buf[padi(j + r * NB)];
    }
  }
  gsync(bar, TPF);
#pragma unroll
  for (int b = 0; b < BPT; ++b) {
    const int j = t + b * TPF;
    const int k = j & (Ns - 1);
    if (Ns > 1) {
      float2 w[R];
      stage_twiddles<R, DIR>(tw, k * (NB / Ns), w);
#pragma unroll
      for (int r = 1; r < R; ++r) v[b][r] = cmul(v[b][r], w[r]);
    }
    dft_reg<R, DIR>(v[b]);
    const int base = (j - k) * R + k;
    if (Ns == 1 && R == 16) {
      float2* dst = buf + padi(base);
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r] = v[b][r];
    } else if (Ns % 16 == 0) {
      float2* dst = buf + padi(base);
      const int SS = Ns + Ns / 16;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * SS] = v[b][r];
    } else {
#pragma unroll
      for (int r = 0; r < R; ++r) buf[padi(base + r * Ns)] = v[b][r];
    }
  }
  gsync(bar, TPF);
}

// Length-2^LOG2N complex FFT in shared memory (unnormalised), natural order.
// DIR = -1: forward e^{-i...}; DIR = +1: inverse without the 1/N factor.
// bar: 0 = __syncthreads, else the named barrier of this transform's TPF threads.
template <int LOG2N, int DIR, int TPF>
__device__ __forceinline__ void fft_smem(float2* buf, int t, const float2* __restrict__ tw, int bar = 0) {
  constexpr int N = 1 << LOG2N;
  constexpr int S16 = LOG2N / 4;
  constexpr int REM = 1 << (LOG2N % 4);
  int Ns = 1;
#pragma unroll
  for (int s = 0; s < S16; ++s) {
    fft_stage<N, 16, DIR, TPF>(buf, Ns, t, tw, bar);
    Ns *= 16;
  }
  if constexpr (REM > 1) fft_stage<N, REM, DIR, TPF>(buf, Ns, t, tw, bar);
}

// Base twiddles (w1, w2, w4, w8 of e^{-2 pi i m / N}) of thread t's butterfly
// in radix-16 stages 1 .. S16-1 (stage 0 has none).  With N/16 threads per
// transform every thread owns one butterfly per stage, so these are the same
// for every transform a kernel runs: kernels with several FFTs load them once
// into registers instead of gathering them from the table in every stage.
template <int LOG2N>
struct StageTw {
  static constexpr int N = 1 << LOG2N, S16 = LOG2N / 4, NS = S16 > 1 ? S16 - 1 : 1;
  float2 w[NS][4];
  __device__ __forceinline__ void load(const float2* __restrict__ tw, int t) {
    int Ns = 16;
#pragma unroll
    for (int s = 0; s + 1 < S16; ++s) {
      const int m = (t & (Ns - 1)) * ((N / 16) / Ns);
      w[s][0] = __ldg(&tw[m]);
      w[s][1] = __ldg(&tw[2 * m]);
      w[s][2] = __ldg(&tw[4 * m]);
      w[s][3] = __ldg(&tw[8 * m]);
      Ns *= 16;
    }
  }
};

// fft_smem with the base twiddles of the radix-16 stages 1 .. S16-1 supplied
// by get(s, q) (q = 0..3: w1, w2, w4, w8 of stage s); TPF = N/16.
template <int LOG2N, int DIR, int TPF, typename GetTw>
__device__ __forceinline__ void fft_smem_tw_impl(float2* buf, int t, const float2* __restrict__ tw, GetTw get,
                                                 int bar) {
  constexpr int N = 1 << LOG2N;
  constexpr int S16 = LOG2N / 4;
  constexpr int REM = 1 << (LOG2N % 4);
  constexpr int NB = N / 16;
  static_assert(TPF == NB, "stored twiddles need one radix-16 butterfly per thread");
  fft_stage<N, 16, DIR, TPF>(buf, 1, t, tw, bar);  // stage 0: no twiddles
  int Ns = 16;
#pragma unroll
  for (int s = 1; s < S16; ++s) {
    float2 v[16];
    const float2* src = buf + padi(t);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = src[r * (NB + NB / 16)];
    gsync(bar, TPF);
    const int k = t & (Ns - 1);
    float2 w[16];
    w[0] = make_float2(1.f, 0.f);
    w[1] = get(s, 0);
    w[2] = get(s, 1);
    w[3] = cmul(w[1], w[2]);
    w[4] = get(s, 2);
#pragma unroll
    for (int r = 5; r < 8; ++r) w[r] = cmul(w[r - 4], w[4]);
    w[8] = get(s, 3);
#pragma unroll
    for (int r = 9; r < 16; ++r) w[r] = cmul(w[r - 8], w[8]);
#pragma unroll
    for (int r = 1; r < 16; ++r) {
      if (DIR > 0) w[r].y = -w[r].y;
      v[r] = cmul(v[r], w[r]);
    }
    dft_reg<16, DIR>(v);
    const int base = (t - k) * 16 + k;
    float2* dst = buf + padi(base);
    const int SS = Ns + Ns / 16;
#pragma unroll
    for (int r = 0; r < 16; ++r) dst[r * SS] = v[r];
    gsync(bar, TPF);
    Ns *= 16;
  }
  if constexpr (REM > 1) fft_stage<N, REM, DIR, TPF>(buf, Ns, t, tw, bar);
}

// ... with the twiddles in registers
template <int LOG2N, int DIR, int TPF>
__device__ __forceinline__ void fft_smem_tw(float2* buf, int t, const float2* __restrict__ tw,
                                            const StageTw<LOG2N>& stw, int bar = 0) {
  fft_smem_tw_impl<LOG2N, DIR, TPF>(buf, t, tw, [&](int s, int q) { return stw.w[s - 1][q]; }, bar);
}

// ... with the twiddles in a shared-memory table twsm[(s - 1) * 4 + q][t]
// (filled by fill_stage_tw), for kernels without registers to spare.
template <int LOG2N, int DIR, int TPF>
__device__ __forceinline__ void fft_smem_tws(float2* buf, int t, const float2* __restrict__ tw,
                                             const float2* twsm, int bar = 0) {
  fft_smem_tw_impl<LOG2N, DIR, TPF>(buf, t, tw, [&](int s, int q) { return twsm[((s - 1) * 4 + q) * TPF + t]; },
                                    bar);
}

template <int LOG2N>
__host__ __device__ constexpr int stage_tw_entries() { return (LOG2N / 4 > 1 ? LOG2N / 4 - 1 : 0) * 4 * ((1 << LOG2N) / 16); }

// twsm[(s - 1) * 4 + q][t] = tw[2^q m(s, t)], filled by all `nthr` threads of the CTA.
template <int LOG2N>
__device__ __forceinline__ void fill_stage_tw(float2* twsm, const float2* __restrict__ tw, int tid, int nthr) {
  constexpr int N = 1 << LOG2N, TPF = N / 16;
  for (int e = tid; e < stage_tw_entries<LOG2N>(); e += nthr) {
    const int t = e % TPF, q = (e / TPF) % 4, s = e / (4 * TPF) + 1;
    int Ns = 1;
    for (int i = 0; i < s; ++i) Ns *= 16;
    const int m = (t & (Ns - 1)) * ((N / 16) / Ns);
    twsm[e] = __ldg(&tw[m << q]);
  }
}

// Makhoul position of sample n inside the reordered sequence v.
__device__ __forceinline__ int mk_pos(int n, int N) { return (n & 1) ? (N - 1 - (n >> 1)) : (n >> 1); }

// Offset of element (row i, column l) in the 4-row-interleaved layout of the
// intermediate spectra: each block of 4 rows is stored column by column, 4
// values per column.  A row pass (4 rows per CTA) then reads or writes one
// contiguous 16N-byte block, and a column pass (2 columns per CTA) moves 32
// contiguous bytes per block (one cache line per lane for thread loads, so
// at N >= 512 the column passes hand those to bulk tensor copies).
__device__ __forceinline__ size_t b4(int i, int l, int N) {
  return (size_t)(i >> 2) * 4 * N + (size_t)l * 4 + (i & 3);
}

// Forward post-step of a two-real-sequence FFT for the pair (k, N-k),
// 0 < k < N/2: spectra of the real part (a) and imaginary part (b).
__device__ __forceinline__ void fwd_post(float2 zk, float2 zn, float2 w, float& ak, float& an, float& bk, float& bn) {
  const float2 va = make_float2(0.5f * (zk.x + zn.x), 0.5f * (zk.y - zn.y));
  const float2 vb = make_float2(0.5f * (zk.y + zn.y), -0.5f * (zk.x - zn.x));
  const float2 ya = cmul(w, va), yb = cmul(w, vb);
  ak = ya.x;
  an = -ya.y;
  bk = yb.x;
  bn = -yb.y;
}

// Unnormalised-inverse pre-step for the pair (k, N-k), 0 < k < N/2: the
// values Z[k], Z[N-k] whose inverse FFT (Makhoul order) is S_c(P) + i S_c(Q),
// S_c(X)[j] = X_0 + 2 sum_{l>=1} X_l cos(pi l (2j+1) / 2N).
__device__ __forceinline__ void inv_pre(float pk, float pn, float qk, float qn, float2 w, float2& zk, float2& zn) {
  const float2 wc = make_float2(w.x, -w.y);
  const float2 ua = cmul(wc, make_float2(pk, -pn));
  const float2 ub = cmul(wc, make_float2(qk, -qn));
  zk = make_float2(ua.x - ub.y, ua.y + ub.x);
  zn = make_float2(ua.x + ub.y, -ua.y + ub.x);
}

// ------------------------------------------------- spectral gradients
// Forward differences of a cosine series, taken in the spectral domain so that
// no two nearly equal FP32 values are ever subtracted.  For one dimension,
// with theta_l = pi l / N,
//     N (S_c(X)[j+1] - S_c(X)[j]) = N (S_c(P)[j] - (-1)^j S_c(Q)[j]),
//     P_l = -2 sin^2(theta_l / 2) X_l,   Q_l = sin(theta_l) X_{N-l},  Q_0 = 0,
// and the right side vanishes at j = N-1 (the zero-flux slot).  Both
// syntheses are one complex Makhoul inverse.  For the pair (k, N-k) with
// w = e^{-i pi k / 2N} = (c, -s):
//     P_k = -2 s^2 X_k,  P_{N-k} = -2 c^2 X_{N-k},  Q_k = 2sc X_{N-k},  Q_{N-k} = 2sc X_k;
// k = N/2: P = -X, Q = X;  k = 0: P = Q = 0.
__device__ __forceinline__ void deriv_pre(float xk, float xn, float2 w, float2& zk, float2& zn) {
  const float c = w.x, s = -w.y;
  const float sc2 = 2.f * s * c;
  inv_pre(-2.f * s * s * xk, -2.f * c * c * xn, sc2 * xn, sc2 * xk, w, zk, zn);
}

// Spectral factor of the solve at frequency (k, l): scale / ((alpha + mu_k + mu_l) N^2),
// 0 for the constant mode when alpha == 0.
__device__ __forceinline__ float spec_gain(int k, const float* __restrict__ mu, float mul, float alpha, float sN2) {
  const float den = alpha + __ldg(&mu[k]) + mul;
  return den > 0.f ? __fdividef(sN2, den) : 0.f;  // den >= pi^2 (or alpha) is far from the fast-divide limits
}

template <int LOG2N>
struct FftCfg {
  static constexpr int N = 1 << LOG2N;
  static constexpr int PADN = N + N / 16;
  static constexpr int TPF = N / 16;  // threads per transform
};

// Makhoul scatter of 4 consecutive samples x[j..j+3] (j % 4 == 0) of two real
// rows into the complex buffer z = a + i b.
__device__ __forceinline__ void scatter4(float2* buf, int j, int N, float4 a, float4 b) {
  const int hj = j >> 1;
  buf[padi(hj)] = make_float2(a.x, b.x);
  buf[padi(N - 1 - hj)] = make_float2(a.y, b.y);
  buf[padi(hj + 1)] = make_float2(a.z, b.z);
  buf[padi(N - 2 - hj)] = make_float2(a.w, b.w);
}

// Second half of the forward row pass: the two Makhoul-ordered complex
// buffers in shared memory (rows 4rb, 4rb+1 in buffer 0, 4rb+2, 4rb+3 in
// buffer 1) are transformed and their spectra written to the interleaved
// layout.  Called after a barrier that publishes the buffers.
template <int LOG2N>
__device__ __forceinline__ void rows_fwd_tail(float2* smem, float* __restrict__ out, int rb,
                                              const float2* __restrict__ tw, const float2* __restrict__ wq) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, PADN = C::PADN, TPF = C::TPF;
  const int f = threadIdx.x / TPF, t = threadIdx.x % TPF;
  // each slot's transform on its own barrier; the post-step reads both buffers
  fft_smem<LOG2N, -1, TPF>(smem + f * PADN, t, tw, TPF >= 32 ? f + 1 : 0);
  if (TPF >= 32) __syncthreads();
  float* __restrict__ o = out + (size_t)rb * 4 * N;
  const float2* b0 = smem;
  const float2* b1 = smem + PADN;
  #pragma unroll
  for (int kk = 0; kk <= (N / 2) / (2 * TPF); ++kk) {
    if (kk == (N / 2) / (2 * TPF) && threadIdx.x != 0) break;
    const int k = threadIdx.x + kk * 2 * TPF;
    if (k == 0 || k == N / 2) {
      const float sc = k == 0 ? 1.f : kRsqrt2;
      const float2 z0 = b0[padi(k)], z1 = b1[padi(k)];
      *reinterpret_cast<float4*>(o + 4 * k) = make_float4(sc * z0.x, sc * z0.y, sc * z1.x, sc * z1.y);
    } else {
      const float2 w = __ldg(&wq[k]);
      float4 vk, vn;
      fwd_post(b0[padi(k)], b0[padi(N - k)], w, vk.x, vn.x, vk.y, vn.y);
      fwd_post(b1[padi(k)], b1[padi(N - k)], w, vk.z, vn.z, vk.w, vn.w);
      *reinterpret_cast<float4*>(o + 4 * k) = vk;
      *reinterpret_cast<float4*>(o + 4 * (N - k)) = vn;
    }
  }
}

// The same for a CTA of TPF threads holding one row pair (rows i0, i0 + 1,
// i0 even) in one buffer: its spectra fill half of each 4-row group.
template <int LOG2N>
__device__ __forceinline__ void rows_fwd_tail_pair(float2* buf, float* __restrict__ out, int i0,
                                                   const float2* __restrict__ tw, const float2* __restrict__ wq) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, TPF = C::TPF;
  const int t = threadIdx.x;
  fft_smem<LOG2N, -1, TPF>(buf, t, tw);
  float* __restrict__ o = out + b4(i0, 0, N);
#pragma unroll
  for (int kk = 0; kk <= (N / 2) / TPF; ++kk) {
    if (kk == (N / 2) / TPF && t != 0) break;
    const int k = t + kk * TPF;
    if (k == 0 || k == N / 2) {
      const float sc = k == 0 ? 1.f : kRsqrt2;
      const float2 z = buf[padi(k)];
      *reinterpret_cast<float2*>(o + 4 * k) = make_float2(sc * z.x, sc * z.y);
    } else {
      float ak, an, bk, bn;
      fwd_post(buf[padi(k)], buf[padi(N - k)], __ldg(&wq[k]), ak, an, bk, bn);
      *reinterpret_cast<float2*>(o + 4 * k) = make_float2(ak, bk);
      *reinterpret_cast<float2*>(o + 4 * (N - k)) = make_float2(an, bn);
    }
  }
}

// ------------------------------------------------------- row pass, forward
// CTA = one block of 4 rows (two transforms of two rows each); input
// row-major, output spectra in the 4-row-interleaved layout.
template <int LOG2N>
__global__ void __launch_bounds__(2 * FftCfg<LOG2N>::TPF, (LOG2N == 12 ? 2 : 1))
    k_dct_rows_fwd(const float* __restrict__ in, float* __restrict__ out, const float2* __restrict__ tw,
                   const float2* __restrict__ wq) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, PADN = C::PADN, TPF = C::TPF;
  extern __shared__ float2 smem[];
  const int f = threadIdx.x / TPF, t = threadIdx.x % TPF;
  float2* buf = smem + f * PADN;
  const int rb = blockIdx.x;
  const float* __restrict__ xa = in + (size_t)(4 * rb + 2 * f) * N;
  const float* __restrict__ xb = xa + N;
#pragma unroll
  for (int ii = 0; ii < N / (4 * TPF); ++ii) {
    const int j = 4 * t + ii * 4 * TPF;
    scatter4(buf, j, N, *reinterpret_cast<const float4*>(xa + j), *reinterpret_cast<const float4*>(xb + j));
  }
  __syncthreads();
  rows_fwd_tail<LOG2N>(smem, out, rb, tw, wq);
}

// ------------------------------------- stencil fused with the forward row pass
// One non-gap iteration's pointwise / stencil update (the same arithmetic as
// k_rof_fused and k_emd_fused, sections 3.1 / 3.2) run by the CTA of the
// forward row pass of the next solve: the block's rows are updated (dual
// and auxiliary variables to HBM), the new right-hand side is scattered in
// Makhoul order straight into the transform buffer(s) (one per row pair),
// and the block then transforms it.  The right-hand side never travels through HBM, and the
// transform's shared-memory work overlaps other blocks' streaming.  The row
// above the block is recomputed from its inputs, so blocks are independent.
// Thread layout: a CTA of RPC rows (2 or 4) has NT = RPC/2 * N/16 threads,
// each owning 4 consecutive columns in N/(4 NT) chunks (j0 = 4 tid + 4 NT c),
// walking the block's rows downwards.
// Requires every pointer 16-byte aligned (state buffers).

__device__ __forceinline__ void ld4(float* d, const float* __restrict__ p) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  d[0] = t.x; d[1] = t.y; d[2] = t.z; d[3] = t.w;
}
__device__ __forceinline__ void st4(float* __restrict__ p, const float* s) {
  *reinterpret_cast<float4*>(p) = make_float4(s[0], s[1], s[2], s[3]);
}

// EMD (section 3.2, affine Leray form): with m = s + grad q,
//   p' = proj(p + sigma m),  s' = m - tau (2 p' - p),  d' = g - div s'.
template <int LOG2N, int RPC>
__global__ void __launch_bounds__(RPC / 2 * FftCfg<LOG2N>::TPF, (LOG2N == 12 ? 8 / RPC : 1))
    k_emd_step_rows_fwd(const float* __restrict__ gq, const float* __restrict__ sin_, const float* __restrict__ pin,
                        const float* __restrict__ g, float* __restrict__ sout, float* __restrict__ pout,
                        float* __restrict__ out, const float2* __restrict__ tw, const float2* __restrict__ wq,
                        EmdParams P) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, PADN = C::PADN, NT = RPC / 2 * C::TPF;
  constexpr size_t NN = (size_t)N * N;
  extern __shared__ float2 smem[];
  const int rb = blockIdx.x, i0 = RPC * rb;
  const float* __restrict__ gx_ = gq;
  const float* __restrict__ gy_ = gq + NN;
  const float* __restrict__ sx_ = sin_;
  const float* __restrict__ sy_ = sin_ + NN;
  const float* __restrict__ px_ = pin;
  const float* __restrict__ py_ = pin + NN;
#pragma unroll 1
  for (int ch = 0; ch < N / (4 * NT); ++ch) {
    const int j0 = 4 * ((int)threadIdx.x + ch * NT);
    float syu[4];  // s'_y of the row above
    if (i0 > 0) {
      const size_t ro = (size_t)(i0 - 1) * N + j0;
      float gx[4], gy[4], sx[4], sy[4], px[4], py[4];
      ld4(gx, gx_ + ro); ld4(gy, gy_ + ro); ld4(sx, sx_ + ro); ld4(sy, sy_ + ro); ld4(px, px_ + ro); ld4(py, py_ + ro);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const bool xr = j0 + c < N - 1;
        const float mx = xr ? sx[c] + gx[c] : 0.f, my = sy[c] + gy[c];
        float p1x, p1y;
        proj2(px[c] + P.sigma * mx, py[c] + P.sigma * my, p1x, p1y);
        syu[c] = my - P.tau * (2.f * p1y - py[c]);
      }
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) syu[c] = 0.f;
    }
    float dprev[4];  // d' of the block's even row, written with its odd partner
#pragma unroll 1
    for (int r = 0; r < RPC; ++r) {
      const int i = i0 + r;
      const size_t ro = (size_t)i * N + j0;
      float gx[5], gy[5], sx[5], sy[5], px[5], py[5];  // [0]: column j0 - 1
      ld4(&gx[1], gx_ + ro); ld4(&gy[1], gy_ + ro); ld4(&sx[1], sx_ + ro);
      ld4(&sy[1], sy_ + ro); ld4(&px[1], px_ + ro); ld4(&py[1], py_ + ro);
      if (j0 > 0) {
        gx[0] = gx_[ro - 1]; gy[0] = gy_[ro - 1]; sx[0] = sx_[ro - 1];
        sy[0] = sy_[ro - 1]; px[0] = px_[ro - 1]; py[0] = py_[ro - 1];
      } else {
        gx[0] = gy[0] = sx[0] = sy[0] = px[0] = py[0] = 0.f;
      }
      float gv[4];
      ld4(gv, g + ro);
      float p1x[5], p1y[5], snx[5], sny[5];
#pragma unroll
      for (int c = 0; c <= 4; ++c) {
        const bool xr = j0 - 1 + c < N - 1, yd = i < N - 1;
        const float mx = xr ? sx[c] + gx[c] : 0.f, my = yd ? sy[c] + gy[c] : 0.f;
        proj2(px[c] + P.sigma * mx, py[c] + P.sigma * my, p1x[c], p1y[c]);
        if (!xr) p1x[c] = 0.f;
        if (!yd) p1y[c] = 0.f;
        snx[c] = xr ? mx - P.tau * (2.f * p1x[c] - px[c]) : 0.f;
        sny[c] = yd ? my - P.tau * (2.f * p1y[c] - py[c]) : 0.f;
      }
      float od[4];
#pragma unroll
      for (int c = 1; c <= 4; ++c) {
        const bool xl = j0 + c - 1 > 0, yu = i > 0;
        const float divs = (snx[c] - (xl ? snx[c - 1] : 0.f) + sny[c] - (yu ? syu[c - 1] : 0.f)) * P.invh;
        od[c - 1] = gv[c - 1] - divs;
      }
      st4(sout + ro, &snx[1]);
      st4(sout + NN + ro, &sny[1]);
      st4(pout + ro, &p1x[1]);
      st4(pout + NN + ro, &p1y[1]);
#pragma unroll
      for (int c = 0; c < 4; ++c) syu[c] = sny[c + 1];
      if (r & 1) {
        scatter4(smem + (r >> 1) * PADN, j0, N, make_float4(dprev[0], dprev[1], dprev[2], dprev[3]),
                 make_float4(od[0], od[1], od[2], od[3]));
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) dprev[c] = od[c];
      }
    }
  }
  __syncthreads();
  if constexpr (RPC == 4) rows_fwd_tail<LOG2N>(smem, out, rb, tw, wq);
  else rows_fwd_tail_pair<LOG2N>(smem, out, i0, tw, wq);
}

// ROF (section 3.1): p' = proj(p + sigma grad u), pbar = 2 p' - p,
//   r' = lambda tau I + tau div pbar - div grad u.
template <int LOG2N, int RPC>
__global__ void __launch_bounds__(RPC / 2 * FftCfg<LOG2N>::TPF, (LOG2N == 12 ? 8 / RPC : 1))
    k_rof_step_rows_fwd(const float* __restrict__ gu, const float* __restrict__ pin, const float* __restrict__ I,
                        float* __restrict__ pout, float* __restrict__ out, const float2* __restrict__ tw,
                        const float2* __restrict__ wq, RofParams P) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, PADN = C::PADN, NT = RPC / 2 * C::TPF;
  constexpr size_t NN = (size_t)N * N;
  extern __shared__ float2 smem[];
  const int rb = blockIdx.x, i0 = RPC * rb;
  const float* __restrict__ gx_ = gu;
  const float* __restrict__ gy_ = gu + NN;
  const float* __restrict__ px_ = pin;
  const float* __restrict__ py_ = pin + NN;
#pragma unroll 1
  for (int ch = 0; ch < N / (4 * NT); ++ch) {
    const int j0 = 4 * ((int)threadIdx.x + ch * NT);
    float pbu[4], gyu[4];  // pbar_y and (grad u)_y of the row above
    if (i0 > 0) {
      const size_t ro = (size_t)(i0 - 1) * N + j0;
      float gx[4], px[4], py[4];
      ld4(gx, gx_ + ro); ld4(gyu, gy_ + ro); ld4(px, px_ + ro); ld4(py, py_ + ro);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        float p1x, p1y;
        proj2(px[c] + P.sigma * gx[c], py[c] + P.sigma * gyu[c], p1x, p1y);
        pbu[c] = 2.f * p1y - py[c];
      }
    } else {
#pragma unroll
      for (int c = 0; c < 4; ++c) pbu[c] = gyu[c] = 0.f;
    }
    float rprev[4];
#pragma unroll 1
    for (int r = 0; r < RPC; ++r) {
      const int i = i0 + r;
      const size_t ro = (size_t)i * N + j0;
      float gx[5], gy[5], px[5], py[5];  // [0]: column j0 - 1
      ld4(&gx[1], gx_ + ro); ld4(&gy[1], gy_ + ro); ld4(&px[1], px_ + ro); ld4(&py[1], py_ + ro);
      if (j0 > 0) {
        gx[0] = gx_[ro - 1]; gy[0] = gy_[ro - 1]; px[0] = px_[ro - 1]; py[0] = py_[ro - 1];
      } else {
        gx[0] = gy[0] = px[0] = py[0] = 0.f;
      }
      float Iv[4];
      ld4(Iv, I + ro);
      float p1x[5], p1y[5], pbx[5], pby[5];
#pragma unroll
      for (int c = 0; c <= 4; ++c) {
        const bool xr = j0 - 1 + c < N - 1, yd = i < N - 1;
        proj2(px[c] + P.sigma * gx[c], py[c] + P.sigma * gy[c], p1x[c], p1y[c]);
        if (!xr) p1x[c] = 0.f;
        if (!yd) p1y[c] = 0.f;
        pbx[c] = 2.f * p1x[c] - (xr ? px[c] : 0.f);
        pby[c] = 2.f * p1y[c] - (yd ? py[c] : 0.f);
      }
      float rv[4];
#pragma unroll
      for (int c = 1; c <= 4; ++c) {
        const bool xl = j0 + c - 1 > 0, yu = i > 0;
        const float dpb = (pbx[c] - (xl ? pbx[c - 1] : 0.f) + pby[c] - (yu ? pbu[c - 1] : 0.f)) * P.invh;
        const float lap = (gx[c] - (xl ? gx[c - 1] : 0.f) + gy[c] - (yu ? gyu[c - 1] : 0.f)) * P.invh;
        rv[c - 1] = P.lt * Iv[c - 1] + P.tau * dpb - lap;
      }
      st4(pout + ro, &p1x[1]);
      st4(pout + NN + ro, &p1y[1]);
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        pbu[c] = pby[c + 1];
        gyu[c] = gy[c + 1];
      }
      if (r & 1) {
        scatter4(smem + (r >> 1) * PADN, j0, N, make_float4(rprev[0], rprev[1], rprev[2], rprev[3]),
                 make_float4(rv[0], rv[1], rv[2], rv[3]));
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) rprev[c] = rv[c];
      }
    }
  }
  __syncthreads();
  if constexpr (RPC == 4) rows_fwd_tail<LOG2N>(smem, out, rb, tw, wq);
  else rows_fwd_tail_pair<LOG2N>(smem, out, i0, tw, wq);
}

// Load the two columns (2cp, 2cp+1) of the interleaved layout into one
// Makhoul-ordered complex buffer (column 2cp real, 2cp+1 imaginary): one
// thread per 4-row block reads both columns (32 contiguous bytes) and writes
// four complex values.
template <int N, int TPF>
__device__ __forceinline__ void load_cols(float2* buf, const float* __restrict__ src, int cp, int t) {
  #pragma unroll
  for (int ii = 0; ii < (N / 4) / TPF; ++ii) {
    const int rb = t + ii * TPF;
    const float* p = src + (size_t)rb * 4 * N + (size_t)(2 * cp) * 4;
    const float4 a = *reinterpret_cast<const float4*>(p);
    const float4 b = *reinterpret_cast<const float4*>(p + 4);
    const int n = 4 * rb;
    buf[padi(mk_pos(n, N))] = make_float2(a.x, b.x);
    buf[padi(mk_pos(n + 1, N))] = make_float2(a.y, b.y);
    buf[padi(mk_pos(n + 2, N))] = make_float2(a.z, b.z);
    buf[padi(mk_pos(n + 3, N))] = make_float2(a.w, b.w);
  }
}

// Store the synthesised columns (real part -> column 2cp, imaginary -> 2cp+1).
template <int N, int TPF>
__device__ __forceinline__ void store_cols(const float2* buf, float* __restrict__ dst, int cp, int t) {
  #pragma unroll
  for (int ii = 0; ii < (N / 4) / TPF; ++ii) {
    const int rb = t + ii * TPF;
    const int n = 4 * rb;
    const float2 z0 = buf[padi(mk_pos(n, N))], z1 = buf[padi(mk_pos(n + 1, N))];
    const float2 z2 = buf[padi(mk_pos(n + 2, N))], z3 = buf[padi(mk_pos(n + 3, N))];
    float* p = dst + (size_t)rb * 4 * N + (size_t)(2 * cp) * 4;
    *reinterpret_cast<float4*>(p) = make_float4(z0.x, z1.x, z2.x, z3.x);
    *reinterpret_cast<float4*>(p + 4) = make_float4(z0.y, z1.y, z2.y, z3.y);
  }
}

// Forward column transform + gain: leaves the gained spectra of both columns
// in `buf` as the inverse pre-step values (plain synthesis) when X == nullptr,
// or stores them in X[k] = (X_a[k], X_b[k]) when X != nullptr.
template <int N, int TPF>
__device__ __forceinline__ void col_spectrum(float2* buf, float2* X, int cp, int t, const float2* __restrict__ wq,
                                             const float* __restrict__ mu, float alpha, float sN2) {
  const int la = 2 * cp, lb = la + 1;
  const float mua = __ldg(&mu[la]), mub = __ldg(&mu[lb]);
  #pragma unroll
  for (int kk = 0; kk <= (N / 2) / TPF; ++kk) {  // k = t + kk TPF covers [0, N/2]; k = N/2 only for t = 0
    if (kk == (N / 2) / TPF && t != 0) break;
    const int k = t + kk * TPF;
    if (k == 0 || k == N / 2) {
      const int pk = padi(k);
      const float2 z = buf[pk];
      const float ga = spec_gain(k, mu, mua, alpha, sN2), gb = spec_gain(k, mu, mub, alpha, sN2);
      if (X) {
        const float sc = k == 0 ? 1.f : kRsqrt2;
        X[k] = make_float2(sc * z.x * ga, sc * z.y * gb);
      } else {
        buf[pk] = make_float2(z.x * ga, z.y * gb);  // k = N/2: the 1/sqrt2 and sqrt2 cancel
      }
    } else {
      const float2 w = __ldg(&wq[k]);
      float ak, an, bk, bn;
      fwd_post(buf[padi(k)], buf[padi(N - k)], w, ak, an, bk, bn);
      ak *= spec_gain(k, mu, mua, alpha, sN2);
      an *= spec_gain(N - k, mu, mua, alpha, sN2);
      bk *= spec_gain(k, mu, mub, alpha, sN2);
      bn *= spec_gain(N - k, mu, mub, alpha, sN2);
      if (X) {
        X[k] = make_float2(ak, bk);
        X[N - k] = make_float2(an, bn);
      } else {
        float2 zk, zn;
        inv_pre(ak, an, bk, bn, w, zk, zn);
        buf[padi(k)] = zk;
        buf[padi(N - k)] = zn;
      }
    }
  }
}

// ------------------------------------------------------ column pass, solve
// CTA = one column pair; in place on the interleaved spectra: forward DCT-II
// along the column, divide by the eigenvalue, inverse.
template <int LOG2N>
__global__ void __launch_bounds__(FftCfg<LOG2N>::TPF, (LOG2N == 12 ? 4 : 1)) k_dct_cols_solve(float* __restrict__ data,
                                                                      const float2* __restrict__ tw,
                                                                      const float2* __restrict__ wq,
                                                                      const float* __restrict__ mu, float alpha,
                                                                      float sN2) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, TPF = C::TPF;
  extern __shared__ float2 smem[];
  const int cp = blockIdx.x, t = threadIdx.x;
  StageTw<LOG2N> stw;
  stw.load(tw, t);
  load_cols<N, TPF>(smem, data, cp, t);
  __syncthreads();
  fft_smem_tw<LOG2N, -1, TPF>(smem, t, tw, stw);
  col_spectrum<N, TPF>(smem, nullptr, cp, t, wq, mu, alpha, sN2);
  __syncthreads();
  fft_smem_tw<LOG2N, +1, TPF>(smem, t, tw, stw);
  store_cols<N, TPF>(smem, data, cp, t);
}

// ------------------------------------------------------- row pass, inverse
// CTA = one block of 4 rows: interleaved spectra in, row-major x out.
template <int LOG2N>
__global__ void __launch_bounds__(2 * FftCfg<LOG2N>::TPF, (LOG2N == 12 ? 2 : 1))
    k_dct_rows_inv(const float* __restrict__ in, float* __restrict__ out, const float2* __restrict__ tw,
                   const float2* __restrict__ wq) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, PADN = C::PADN, TPF = C::TPF;
  extern __shared__ float2 smem[];
  const int rb = blockIdx.x;
  const float* __restrict__ src = in + (size_t)rb * 4 * N;
  float2* b0 = smem;
  float2* b1 = smem + PADN;
  #pragma unroll
  for (int kk = 0; kk <= (N / 2) / (2 * TPF); ++kk) {
    if (kk == (N / 2) / (2 * TPF) && threadIdx.x != 0) break;
    const int k = threadIdx.x + kk * 2 * TPF;
    const float4 vk = *reinterpret_cast<const float4*>(src + 4 * k);
    if (k == 0) {
      b0[0] = make_float2(vk.x, vk.y);
      b1[0] = make_float2(vk.z, vk.w);
    } else if (k == N / 2) {
      b0[padi(k)] = make_float2(kSqrt2 * vk.x, kSqrt2 * vk.y);
      b1[padi(k)] = make_float2(kSqrt2 * vk.z, kSqrt2 * vk.w);
    } else {
      const float4 vn = *reinterpret_cast<const float4*>(src + 4 * (N - k));
      const float2 w = __ldg(&wq[k]);
      float2 zk, zn;
      inv_pre(vk.x, vn.x, vk.y, vn.y, w, zk, zn);
      b0[padi(k)] = zk;
      b0[padi(N - k)] = zn;
      inv_pre(vk.z, vn.z, vk.w, vn.w, w, zk, zn);
      b1[padi(k)] = zk;
      b1[padi(N - k)] = zn;
    }
  }
  __syncthreads();
  const int f = threadIdx.x / TPF, t = threadIdx.x % TPF;
  float2* buf = smem + f * PADN;
  fft_smem<LOG2N, +1, TPF>(buf, t, tw, TPF >= 32 ? f + 1 : 0);  // the post-step reads only this slot's buffer
  float* __restrict__ oa = out + (size_t)(4 * rb + 2 * f) * N;
  float* __restrict__ ob = oa + N;
  #pragma unroll
  for (int ii = 0; ii < N / (4 * TPF); ++ii) {
    const int j = 4 * t + ii * 4 * TPF;
    const int hj = j >> 1;
    const float2 z0 = buf[padi(hj)], z1 = buf[padi(N - 1 - hj)];
    const float2 z2 = buf[padi(hj + 1)], z3 = buf[padi(N - 2 - hj)];
    *reinterpret_cast<float4*>(oa + j) = make_float4(z0.x, z1.x, z2.x, z3.x);
    *reinterpret_cast<float4*>(ob + j) = make_float4(z0.y, z1.y, z2.y, z3.y);
  }
}

// --------------------------------------------------- column pass, gradient
// CTA = one column pair.  After the forward transform and the gain, three
// syntheses along the column:
//   A[:, pair] = S_c(X)                      (plain; feeds the x-derivative and phi)
//   B[:, a]    = D_y S_c(X_a),  B[:, b] = D_y S_c(X_b)
// `in` may alias A.  Shared memory: transform buffer(s), gained spectra.
// PAR (small N, where one CTA's chain of transforms is the latency): three
// groups of TPF threads run the three syntheses at once in their own
// buffers, each synchronising on its own named barrier.
template <int LOG2N, bool PAR>
__global__ void __launch_bounds__((PAR ? 3 : 1) * FftCfg<LOG2N>::TPF, (LOG2N == 12 && !PAR ? 3 : 1))
    k_dct_cols_grad(const float* __restrict__ in, float* A, float* B, const float2* __restrict__ tw,
                    const float2* __restrict__ wq, const float* __restrict__ mu, float alpha, float sN2) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, PADN = C::PADN, TPF = C::TPF;
  extern __shared__ float2 smem[];
  const int grp = PAR ? (int)threadIdx.x / TPF : 0, t = (int)threadIdx.x % TPF;
  float2* buf = smem + grp * PADN;
  float2* X = smem + (PAR ? 3 : 1) * PADN;  // gained spectra of the two columns, N complex
  const int cp = blockIdx.x;
  const float fN = (float)N;
  StageTw<LOG2N> stw;
  stw.load(tw, t);
  if (grp == 0) {
    const int bar0 = PAR ? 1 : 0;
    load_cols<N, TPF>(buf, in, cp, t);
    gsync(bar0, TPF);
    fft_smem_tw<LOG2N, -1, TPF>(buf, t, tw, stw, bar0);
    col_spectrum<N, TPF>(buf, X, cp, t, wq, mu, alpha, sN2);
  }
  __syncthreads();
  const int bar = PAR ? grp + 1 : 0;
  for (int pass = PAR ? grp : 0; pass < (PAR ? grp + 1 : 3); ++pass) {
#pragma unroll
    for (int kk = 0; kk <= (N / 2) / TPF; ++kk) {  // k = t + kk TPF covers [0, N/2]; k = N/2 only for t = 0
      if (kk == (N / 2) / TPF && t != 0) break;
      const int k = t + kk * TPF;
      const float2 xk = X[k];
      if (pass == 0) {
        if (k == 0) {
          buf[0] = xk;
        } else if (k == N / 2) {
          buf[padi(k)] = make_float2(kSqrt2 * xk.x, kSqrt2 * xk.y);
        } else {
          const float2 xn = X[N - k];
          float2 zk, zn;
          inv_pre(xk.x, xn.x, xk.y, xn.y, __ldg(&wq[k]), zk, zn);
          buf[padi(k)] = zk;
          buf[padi(N - k)] = zn;
        }
      } else {
        const float x0 = pass == 1 ? xk.x : xk.y;
        if (k == 0) {
          buf[0] = make_float2(0.f, 0.f);
        } else if (k == N / 2) {
          buf[padi(k)] = make_float2(-kSqrt2 * x0, kSqrt2 * x0);
        } else {
          const float2 xn2 = X[N - k];
          float2 zk, zn;
          deriv_pre(x0, pass == 1 ? xn2.x : xn2.y, __ldg(&wq[k]), zk, zn);
          buf[padi(k)] = zk;
          buf[padi(N - k)] = zn;
        }
      }
    }
    gsync(bar, TPF);
    fft_smem_tw<LOG2N, +1, TPF>(buf, t, tw, stw, bar);
    if (pass == 0) {
      store_cols<N, TPF>(buf, A, cp, t);
    } else {
      // D_y of column (2cp + pass - 1): one float4 (4 rows) per row block
      const int col = 2 * cp + pass - 1;
#pragma unroll
      for (int ii = 0; ii < (N / 4) / TPF; ++ii) {
        const int rb = t + ii * TPF;
        float v[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int n = 4 * rb + r;
          const float2 z = buf[padi(mk_pos(n, N))];
          v[r] = (n == N - 1) ? 0.f : fN * (z.x - ((n & 1) ? -z.y : z.y));
        }
        *reinterpret_cast<float4*>(B + (size_t)rb * 4 * N + (size_t)col * 4) = make_float4(v[0], v[1], v[2], v[3]);
      }
    }
    gsync(bar, TPF);
  }
}

// ------------------------------------- column pass, gradient, bulk tensor copies
// The interleaved spectra seen as a 3-D tensor {4 rows, N columns, N/4 row
// blocks} (strides 16 B and 16N B): a column pair is 32 B per row block, so a
// thread-per-row-block load or store touches one cache line per lane (32
// lines per warp instruction).  Here the tensor-memory-access engine moves
// the column pair in (one box of up to 256 row blocks per copy, counted on an
// mbarrier) and each synthesis out (staged in the transform buffer, one bulk
// tensor store per box), and the threads only touch shared memory.
// Same computation as k_dct_cols_grad.  tm_in: box {4, 2, BOXR} over `in`;
// tm_a: box {4, 2, BOXR} over A; tm_b: box {4, 1, BOXR} over B.  PAR (N = 512,
// 1024): three groups of TPF threads run the three syntheses at once, each in
// its own buffer on its own named barrier, each staging and storing its own
// output.  A copy that never lands (bounded wait) poisons the column pair with
// NaN and sets *err, so the solve reports a non-finite iterate instead of
// hanging.
template <int LOG2N, bool PAR>
__global__ void __launch_bounds__((PAR ? 3 : 1) * FftCfg<LOG2N>::TPF, (LOG2N == 12 ? 3 : 1))
    k_dct_cols_grad_tma(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_a,
                        const __grid_constant__ CUtensorMap tm_b, const float2* __restrict__ tw,
                        const float2* __restrict__ wq, const float* __restrict__ mu, float alpha, float sN2,
                        int* __restrict__ err) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, PADN = C::PADN, TPF = C::TPF;
  constexpr int NG = PAR ? 3 : 1;
  constexpr int BOXR = N / 4 < 256 ? N / 4 : 256, NBOX = (N / 4) / BOXR;
  constexpr int RBT = (N / 4) / TPF;  // row blocks per thread
  extern __shared__ __align__(128) float2 smem_tma[];
  const int grp = PAR ? (int)threadIdx.x / TPF : 0, t = (int)threadIdx.x % TPF;
  float2* buf = smem_tma + grp * PADN;
  float2* X = smem_tma + NG * PADN;  // staged column pair, then the gained spectra
  uint64_t* mbar = reinterpret_cast<uint64_t*>(X + N);
  float* stage = reinterpret_cast<float*>(buf);
  const int cp = blockIdx.x;
  const float fN = (float)N;
  const uint32_t bar = smem_addr(mbar);
  const int gbar = PAR ? grp + 1 : 0;  // this group's barrier
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)(N * 8))
                 : "memory");
#pragma unroll
    for (int q = 0; q < NBOX; ++q) tma_load_3d(smem_addr(X) + q * BOXR * 32, &tm_in, 0, 2 * cp, q * BOXR, bar);
  }
  StageTw<LOG2N> stw;
  stw.load(tw, t);
  if (grp == 0) {
    float poison = 1.f;
    if (!mbar_try(bar, 0)) {
      poison = __int_as_float(0x7fc00000);
      atomicExch(err, 1);
    }
    const float* Xs = reinterpret_cast<const float*>(X);
#pragma unroll
    for (int ii = 0; ii < RBT; ++ii) {
      const int rb = t + ii * TPF;
      const float4 a = *reinterpret_cast<const float4*>(Xs + rb * 8);
      const float4 b = *reinterpret_cast<const float4*>(Xs + rb * 8 + 4);
      const int n = 4 * rb;
      buf[padi(mk_pos(n, N))] = make_float2(poison * a.x, poison * b.x);
      buf[padi(mk_pos(n + 1, N))] = make_float2(poison * a.y, poison * b.y);
      buf[padi(mk_pos(n + 2, N))] = make_float2(poison * a.z, poison * b.z);
      buf[padi(mk_pos(n + 3, N))] = make_float2(poison * a.w, poison * b.w);
    }
    gsync(gbar, TPF);
    fft_smem_tw<LOG2N, -1, TPF>(buf, t, tw, stw, gbar);
    col_spectrum<N, TPF>(buf, X, cp, t, wq, mu, alpha, sN2);
  }
  __syncthreads();
#pragma unroll 1
  for (int pass = PAR ? grp : 0; pass < (PAR ? grp + 1 : 3); ++pass) {
#pragma unroll
    for (int kk = 0; kk <= (N / 2) / TPF; ++kk) {  // k = t + kk TPF covers [0, N/2]; k = N/2 only for t = 0
      if (kk == (N / 2) / TPF && t != 0) break;
      const int k = t + kk * TPF;
      const float2 xk = X[k];
      if (pass == 0) {
        if (k == 0) {
          buf[0] = xk;
        } else if (k == N / 2) {
          buf[padi(k)] = make_float2(kSqrt2 * xk.x, kSqrt2 * xk.y);
        } else {
          const float2 xn = X[N - k];
          float2 zk, zn;
          inv_pre(xk.x, xn.x, xk.y, xn.y, __ldg(&wq[k]), zk, zn);
          buf[padi(k)] = zk;
          buf[padi(N - k)] = zn;
        }
      } else {
        const float x0 = pass == 1 ? xk.x : xk.y;
        if (k == 0) {
          buf[0] = make_float2(0.f, 0.f);
        } else if (k == N / 2) {
          buf[padi(k)] = make_float2(-kSqrt2 * x0, kSqrt2 * x0);
        } else {
          const float2 xn2 = X[N - k];
          float2 zk, zn;
          deriv_pre(x0, pass == 1 ? xn2.x : xn2.y, __ldg(&wq[k]), zk, zn);
          buf[padi(k)] = zk;
          buf[padi(N - k)] = zn;
        }
      }
    }
    gsync(gbar, TPF);
    fft_smem_tw<LOG2N, +1, TPF>(buf, t, tw, stw, gbar);
    // this thread's row blocks: read out of the transform buffer, then staged
    // over it as {row block, column(s), 4 rows} for the tensor store
    float4 va[RBT], vb[RBT];
#pragma unroll
    for (int ii = 0; ii < RBT; ++ii) {
      const int n = 4 * (t + ii * TPF);
      const float2 z0 = buf[padi(mk_pos(n, N))], z1 = buf[padi(mk_pos(n + 1, N))];
      const float2 z2 = buf[padi(mk_pos(n + 2, N))], z3 = buf[padi(mk_pos(n + 3, N))];
      if (pass == 0) {
        va[ii] = make_float4(z0.x, z1.x, z2.x, z3.x);
        vb[ii] = make_float4(z0.y, z1.y, z2.y, z3.y);
      } else {  // D_y: N (S_c(P) - (-1)^n S_c(Q)), zero-flux slot at n = N-1
        va[ii] = make_float4(fN * (z0.x - z0.y), fN * (z1.x + z1.y), fN * (z2.x - z2.y),
                             n + 3 == N - 1 ? 0.f : fN * (z3.x + z3.y));
      }
    }
    gsync(gbar, TPF);
#pragma unroll
    for (int ii = 0; ii < RBT; ++ii) {
      const int rb = t + ii * TPF;
      if (pass == 0) {
        *reinterpret_cast<float4*>(stage + rb * 8) = va[ii];
        *reinterpret_cast<float4*>(stage + rb * 8 + 4) = vb[ii];
      } else {
        *reinterpret_cast<float4*>(stage + rb * 4) = va[ii];
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    gsync(gbar, TPF);
    if (t == 0) {
#pragma unroll
      for (int q = 0; q < NBOX; ++q) {
        if (pass == 0)
          tma_store_3d(&tm_a, 0, 2 * cp, q * BOXR, smem_addr(stage) + q * BOXR * 32);
        else
          tma_store_3d(&tm_b, 0, 2 * cp + pass - 1, q * BOXR, smem_addr(stage) + q * BOXR * 16);
      }
      asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");  // the buffer is reused next pass
    }
    gsync(gbar, TPF);
  }
  if (t == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Column pass of the plain solve on bulk tensor copies, in place on the
// interleaved spectra (same computation as k_dct_cols_solve): the column
// pair arrives staged in the transform buffer, each thread takes its row
// blocks into registers before the Makhoul scatter overwrites it, and the
// result leaves the same way through a staging copy and a tensor store.
// tm: box {4, 2, BOXR} over `data`.
template <int LOG2N>
__global__ void __launch_bounds__(FftCfg<LOG2N>::TPF, (LOG2N == 12 ? 4 : 1))
    k_dct_cols_solve_tma(const __grid_constant__ CUtensorMap tm, const float2* __restrict__ tw,
                         const float2* __restrict__ wq, const float* __restrict__ mu, float alpha, float sN2,
                         int* __restrict__ err) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, PADN = C::PADN, TPF = C::TPF;
  constexpr int BOXR = N / 4 < 256 ? N / 4 : 256, NBOX = (N / 4) / BOXR;
  constexpr int RBT = (N / 4) / TPF;
  extern __shared__ __align__(128) float2 smem_tma[];
  float2* buf = smem_tma;
  float* stage = reinterpret_cast<float*>(buf);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem_tma + PADN);
  const int cp = blockIdx.x, t = threadIdx.x;
  const uint32_t bar = smem_addr(mbar);
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (t == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)(N * 8))
                 : "memory");
#pragma unroll
    for (int q = 0; q < NBOX; ++q) tma_load_3d(smem_addr(stage) + q * BOXR * 32, &tm, 0, 2 * cp, q * BOXR, bar);
  }
  StageTw<LOG2N> stw;
  stw.load(tw, t);
  float poison = 1.f;
  if (!mbar_try(bar, 0)) {
    poison = __int_as_float(0x7fc00000);
    atomicExch(err, 1);
  }
  float4 va[RBT], vb[RBT];
#pragma unroll
  for (int ii = 0; ii < RBT; ++ii) {
    const int rb = t + ii * TPF;
    va[ii] = *reinterpret_cast<const float4*>(stage + rb * 8);
    vb[ii] = *reinterpret_cast<const float4*>(stage + rb * 8 + 4);
  }
  __syncthreads();
#pragma unroll
  for (int ii = 0; ii < RBT; ++ii) {
    const int n = 4 * (t + ii * TPF);
    buf[padi(mk_pos(n, N))] = make_float2(poison * va[ii].x, poison * vb[ii].x);
    buf[padi(mk_pos(n + 1, N))] = make_float2(poison * va[ii].y, poison * vb[ii].y);
    buf[padi(mk_pos(n + 2, N))] = make_float2(poison * va[ii].z, poison * vb[ii].z);
    buf[padi(mk_pos(n + 3, N))] = make_float2(poison * va[ii].w, poison * vb[ii].w);
  }
  __syncthreads();
  fft_smem_tw<LOG2N, -1, TPF>(buf, t, tw, stw);
  col_spectrum<N, TPF>(buf, nullptr, cp, t, wq, mu, alpha, sN2);
  __syncthreads();
  fft_smem_tw<LOG2N, +1, TPF>(buf, t, tw, stw);
#pragma unroll
  for (int ii = 0; ii < RBT; ++ii) {
    const int n = 4 * (t + ii * TPF);
    const float2 z0 = buf[padi(mk_pos(n, N))], z1 = buf[padi(mk_pos(n + 1, N))];
    const float2 z2 = buf[padi(mk_pos(n + 2, N))], z3 = buf[padi(mk_pos(n + 3, N))];
    va[ii] = make_float4(z0.x, z1.x, z2.x, z3.x);
    vb[ii] = make_float4(z0.y, z1.y, z2.y, z3.y);
  }
  __syncthreads();
#pragma unroll
  for (int ii = 0; ii < RBT; ++ii) {
    const int rb = t + ii * TPF;
    *reinterpret_cast<float4*>(stage + rb * 8) = va[ii];
    *reinterpret_cast<float4*>(stage + rb * 8 + 4) = vb[ii];
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (t == 0) {
#pragma unroll
    for (int q = 0; q < NBOX; ++q) tma_store_3d(&tm, 0, 2 * cp, q * BOXR, smem_addr(stage) + q * BOXR * 32);
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
}

// ------------------------------------------------------ row pass, gradient
// CTA = one block of 4 rows (two transform slots).  Per slot f (rows
// r0 = 4 rb + 2f and r0 + 1):
//   gx[r0] = D_x S_c(A[r0]),  gx[r0+1] = D_x S_c(A[r0+1]),  gy[r0, r0+1] = S_c(B[r0, r0+1]),
//   and phi[r0, r0+1] = S_c(A[r0, r0+1]) when phi != nullptr.
// A, B interleaved; gx, gy, phi row-major; gx has its zero slot at j = N-1.
// PAR (small N): one group of TPF threads per (slot, pass), all at once, each
// in its own buffer on its own named barrier; blockDim = 2 npass TPF.
template <int LOG2N, bool PAR>
__global__ void __launch_bounds__((PAR ? 8 : 2) * FftCfg<LOG2N>::TPF, (LOG2N == 12 && !PAR ? 2 : 1))
    k_dct_rows_grad(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ gx,
                    float* __restrict__ gy, float* __restrict__ phi, const float2* __restrict__ tw,
                    const float2* __restrict__ wq) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, PADN = C::PADN, TPF = C::TPF;
  extern __shared__ float2 smem[];
  const int npass = phi ? 4 : 3;
  const int grp = (int)threadIdx.x / TPF, t = (int)threadIdx.x % TPF;
  const int f = PAR ? grp / npass : grp;
  float2* buf = smem + grp * PADN;
  float2* twsm = smem + (PAR ? 2 * npass : 2) * PADN;
  fill_stage_tw<LOG2N>(twsm, tw, threadIdx.x, blockDim.x);
  __syncthreads();
  const int rb = blockIdx.x;
  const int r0 = 4 * rb + 2 * f;
  const float fN = (float)N;
  const int bar = PAR ? grp + 1 : 0;
  const int p0 = PAR ? grp % npass : 0;
  for (int pass = p0; pass < (PAR ? p0 + 1 : npass); ++pass) {
    // pass 0: D_x of A row r0; 1: D_x of A row r0+1; 2: plain of B rows r0, r0+1; 3: plain of A rows
    const float* __restrict__ src = (pass == 2 ? B : A) + (size_t)rb * 4 * N;
    if constexpr (!PAR) {
      // both slots' pre-steps at once: one float4 (the block's 4 rows at column k) per load
      float2* b0 = smem;
      float2* b1 = smem + PADN;
#pragma unroll
      for (int kk = 0; kk <= (N / 2) / (2 * TPF); ++kk) {  // k = tid + kk 2TPF covers [0, N/2]
        if (kk == (N / 2) / (2 * TPF) && threadIdx.x != 0) break;
        const int k = (int)threadIdx.x + kk * 2 * TPF;
        const float4 xk = *reinterpret_cast<const float4*>(src + 4 * k);
        if (pass < 2) {
          const float a0 = pass == 0 ? xk.x : xk.y, a1 = pass == 0 ? xk.z : xk.w;
          if (k == 0) {
            b0[0] = make_float2(0.f, 0.f);
            b1[0] = make_float2(0.f, 0.f);
          } else if (k == N / 2) {
            b0[padi(k)] = make_float2(-kSqrt2 * a0, kSqrt2 * a0);
            b1[padi(k)] = make_float2(-kSqrt2 * a1, kSqrt2 * a1);
          } else {
            const float4 xn = *reinterpret_cast<const float4*>(src + 4 * (N - k));
            const float2 w = __ldg(&wq[k]);
            float2 zk, zn;
            deriv_pre(a0, pass == 0 ? xn.x : xn.y, w, zk, zn);
            b0[padi(k)] = zk;
            b0[padi(N - k)] = zn;
            deriv_pre(a1, pass == 0 ? xn.z : xn.w, w, zk, zn);
            b1[padi(k)] = zk;
            b1[padi(N - k)] = zn;
          }
        } else {
          if (k == 0) {
            b0[0] = make_float2(xk.x, xk.y);
            b1[0] = make_float2(xk.z, xk.w);
          } else if (k == N / 2) {
            b0[padi(k)] = make_float2(kSqrt2 * xk.x, kSqrt2 * xk.y);
            b1[padi(k)] = make_float2(kSqrt2 * xk.z, kSqrt2 * xk.w);
          } else {
            const float4 xn = *reinterpret_cast<const float4*>(src + 4 * (N - k));
            const float2 w = __ldg(&wq[k]);
            float2 zk, zn;
            inv_pre(xk.x, xn.x, xk.y, xn.y, w, zk, zn);
            b0[padi(k)] = zk;
            b0[padi(N - k)] = zn;
            inv_pre(xk.z, xn.z, xk.w, xn.w, w, zk, zn);
            b1[padi(k)] = zk;
            b1[padi(N - k)] = zn;
          }
        }
      }
    } else {
      // one slot's pre-step per thread group (each group in its own buffer)
#pragma unroll
      for (int kk = 0; kk <= (N / 2) / TPF; ++kk) {  // k = t + kk TPF covers [0, N/2]; k = N/2 only for t = 0
        if (kk == (N / 2) / TPF && t != 0) break;
        const int k = t + kk * TPF;
        const float2 xk2 = *reinterpret_cast<const float2*>(src + 4 * k + 2 * f);
        if (pass < 2) {
          const float xk = pass == 0 ? xk2.x : xk2.y;
          if (k == 0) {
            buf[0] = make_float2(0.f, 0.f);
          } else if (k == N / 2) {
            buf[padi(k)] = make_float2(-kSqrt2 * xk, kSqrt2 * xk);
          } else {
            const float2 xn2 = *reinterpret_cast<const float2*>(src + 4 * (N - k) + 2 * f);
            float2 zk, zn;
            deriv_pre(xk, pass == 0 ? xn2.x : xn2.y, __ldg(&wq[k]), zk, zn);
            buf[padi(k)] = zk;
            buf[padi(N - k)] = zn;
          }
        } else {
          if (k == 0) {
            buf[0] = xk2;
          } else if (k == N / 2) {
            buf[padi(k)] = make_float2(kSqrt2 * xk2.x, kSqrt2 * xk2.y);
          } else {
            const float2 xn2 = *reinterpret_cast<const float2*>(src + 4 * (N - k) + 2 * f);
            float2 zk, zn;
            inv_pre(xk2.x, xn2.x, xk2.y, xn2.y, __ldg(&wq[k]), zk, zn);
            buf[padi(k)] = zk;
            buf[padi(N - k)] = zn;
          }
        }
      }
    }
    gsync(bar, (PAR ? 1 : 2) * TPF);
    // the transform and the post-step touch only this slot's buffer: each
    // slot synchronises on its own barrier (the pre-step above writes both
    // buffers, so it and the end of the pass stay CTA-wide)
    fft_smem_tws<LOG2N, +1, TPF>(buf, t, tw, twsm, PAR ? bar : (TPF >= 32 ? f + 1 : 0));
    if (pass < 2) {
      float* __restrict__ o = gx + (size_t)(r0 + pass) * N;
#pragma unroll
      for (int ii = 0; ii < N / (4 * TPF); ++ii) {
        const int j = 4 * t + ii * 4 * TPF;
        const int hj = j >> 1;
        const float2 z0 = buf[padi(hj)], z1 = buf[padi(N - 1 - hj)];
        const float2 z2 = buf[padi(hj + 1)], z3 = buf[padi(N - 2 - hj)];
        float4 v = make_float4(fN * (z0.x - z0.y), fN * (z1.x + z1.y), fN * (z2.x - z2.y), fN * (z3.x + z3.y));
        if (j + 4 == N) v.w = 0.f;  // zero-flux slot
        *reinterpret_cast<float4*>(o + j) = v;
      }
    } else {
      float* __restrict__ oa = (pass == 2 ? gy : phi) + (size_t)r0 * N;
      float* __restrict__ ob = oa + N;
#pragma unroll
      for (int ii = 0; ii < N / (4 * TPF); ++ii) {
        const int j = 4 * t + ii * 4 * TPF;
        const int hj = j >> 1;
        const float2 z0 = buf[padi(hj)], z1 = buf[padi(N - 1 - hj)];
        const float2 z2 = buf[padi(hj + 1)], z3 = buf[padi(N - 2 - hj)];
        *reinterpret_cast<float4*>(oa + j) = make_float4(z0.x, z1.x, z2.x, z3.x);
        *reinterpret_cast<float4*>(ob + j) = make_float4(z0.y, z1.y, z2.y, z3.y);
      }
    }
    gsync(bar, (PAR ? 1 : 2) * TPF);
  }
}

template <typename K>
cudaError_t set_smem(K k, size_t bytes) {
  return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Tensor map of an interleaved-spectra plane as {4 rows, N columns, N/4 row
// blocks}, box {4, ncols, min(256, N/4)}; false when the CUDA driver's encoder is
// unavailable or refuses.
template <int LOG2N>
cudaError_t launch_fft_pass(const DctPlan& p, int pass, const float* in, float* out, float alpha, float scale,
                            cudaStream_t st) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, PADN = C::PADN, TPF = C::TPF;
  const size_t sm1 = (size_t)PADN * sizeof(float2), sm2 = 2 * sm1;
  cudaError_t e;
  if (pass == 0) {
    if ((e = set_smem(k_dct_rows_fwd<LOG2N>, sm2))) return e;
    k_dct_rows_fwd<LOG2N><<<N / 4, 2 * TPF, sm2, st>>>(in, out, p.tw, p.wq);
  } else if (pass == 1) {
    const float sN2 = (float)((double)scale / ((double)N * (double)N));
    if constexpr (LOG2N >= 11) {
      CUtensorMap tm;
      if (p.err && encode_b4_map(&tm, out, N, 2)) {
        const size_t sm = sm1 + 16;
        if ((e = set_smem(k_dct_cols_solve_tma<LOG2N>, sm))) return e;
        k_dct_cols_solve_tma<LOG2N><<<N / 2, TPF, sm, st>>>(tm, p.tw, p.wq, p.mu, alpha, sN2, p.err);
        return cudaGetLastError();
      }
    }
    if ((e = set_smem(k_dct_cols_solve<LOG2N>, sm1))) return e;
    k_dct_cols_solve<LOG2N><<<N / 2, TPF, sm1, st>>>(out, p.tw, p.wq, p.mu, alpha, sN2);
  } else {
    if ((e = set_smem(k_dct_rows_inv<LOG2N>, sm2))) return e;
    k_dct_rows_inv<LOG2N><<<N / 4, 2 * TPF, sm2, st>>>(in, out, p.tw, p.wq);
  }
  return cudaGetLastError();
}

template <int LOG2N>
cudaError_t launch_grad_cols(const DctPlan& p, const float* in, float* A, float* B, float alpha, float scale,
                             cudaStream_t st) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, PADN = C::PADN, TPF = C::TPF;
  if constexpr (LOG2N == 12) return grad_cols_4k(p, in, A, B, alpha, scale, st);  // pair-interleaved spectra
  if constexpr (LOG2N >= 9) {
    constexpr bool PART = LOG2N == 9 || LOG2N == 10;
    CUtensorMap tm_in, tm_a, tm_b;
    if (p.err && encode_b4_map(&tm_in, in, N, 2) && encode_b4_map(&tm_a, A, N, 2) && encode_b4_map(&tm_b, B, N, 1)) {
      const size_t sm = (size_t)((PART ? 3 : 1) * PADN + N) * sizeof(float2) + 16;
      cudaError_t e;
      if ((e = set_smem(k_dct_cols_grad_tma<LOG2N, PART>, sm))) return e;
      const float sN2 = (float)((double)scale / ((double)N * (double)N));
      k_dct_cols_grad_tma<LOG2N, PART>
          <<<N / 2, (PART ? 3 : 1) * TPF, sm, st>>>(tm_in, tm_a, tm_b, p.tw, p.wq, p.mu, alpha, sN2, p.err);
      return cudaGetLastError();
    }
  }
  // small N (one CTA's transform chain is the latency): the three syntheses in
  // parallel groups; named barriers need whole warps per group (TPF >= 32)
  constexpr bool PAR = LOG2N == 9 || LOG2N == 10;
  const size_t sm = (size_t)(PAR ? 3 : 1) * PADN * sizeof(float2) + (size_t)N * sizeof(float2);
  cudaError_t e;
  if ((e = set_smem(k_dct_cols_grad<LOG2N, PAR>, sm))) return e;
  const float sN2 = (float)((double)scale / ((double)N * (double)N));
  k_dct_cols_grad<LOG2N, PAR><<<N / 2, (PAR ? 3 : 1) * TPF, sm, st>>>(in, A, B, p.tw, p.wq, p.mu, alpha, sN2);
  return cudaGetLastError();
}

template <int LOG2N>
cudaError_t launch_grad_rows(const DctPlan& p, const float* A, const float* B, float* gx, float* gy, float* phi,
                             cudaStream_t st) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, PADN = C::PADN, TPF = C::TPF;
  constexpr bool PAR = LOG2N == 9 || LOG2N == 10;  // as in the column pass
  if constexpr (LOG2N == 12) return grad_rows_4k(p, A, B, gx, gy, phi, st);
  const int groups = PAR ? 2 * (phi ? 4 : 3) : 2;
  const size_t sm = ((size_t)groups * PADN + stage_tw_entries<LOG2N>()) * sizeof(float2);
  cudaError_t e;
  if ((e = set_smem(k_dct_rows_grad<LOG2N, PAR>, sm))) return e;
  k_dct_rows_grad<LOG2N, PAR><<<N / 4, groups * TPF, sm, st>>>(A, B, gx, gy, phi, p.tw, p.wq);
  return cudaGetLastError();
}

// Rows per CTA of the fused step kernels.  EMD: 2 (one transform of TPF
// threads, four CTAs per SM at N = 4096, so that co-resident CTAs drift out
// of phase and one's stencil streaming overlaps another's transform; 158 ->
// 151 us at 4096^2).  ROF, with fewer bytes per point, loses more to the
// extra recomputed row above each 2-row block than it gains (107 -> 116 us):
// 4.
constexpr int kEmdStepRowsPerCta = 2;
constexpr int kRofStepRowsPerCta = 4;

template <int LOG2N>
cudaError_t launch_emd_step_fwd(const DctPlan& p, const float* gq, const float* sin_, const float* pin,
                                const float* g, float* sout, float* pout, float* out, const EmdParams& P,
                                cudaStream_t st) {
  using C = FftCfg<LOG2N>;
  constexpr int RPC = kEmdStepRowsPerCta;
  const size_t sm = RPC / 2 * (size_t)C::PADN * sizeof(float2);
  cudaError_t e;
  if ((e = set_smem(k_emd_step_rows_fwd<LOG2N, RPC>, sm))) return e;
  k_emd_step_rows_fwd<LOG2N, RPC>
      <<<C::N / RPC, RPC / 2 * C::TPF, sm, st>>>(gq, sin_, pin, g, sout, pout, out, p.tw, p.wq, P);
  return cudaGetLastError();
}

template <int LOG2N>
cudaError_t launch_rof_step_fwd(const DctPlan& p, const float* gu, const float* pin, const float* I, float* pout,
                                float* out, const RofParams& P, cudaStream_t st) {
  using C = FftCfg<LOG2N>;
  constexpr int RPC = kRofStepRowsPerCta;
  const size_t sm = RPC / 2 * (size_t)C::PADN * sizeof(float2);
  cudaError_t e;
  if ((e = set_smem(k_rof_step_rows_fwd<LOG2N, RPC>, sm))) return e;
  k_rof_step_rows_fwd<LOG2N, RPC><<<C::N / RPC, RPC / 2 * C::TPF, sm, st>>>(gu, pin, I, pout, out, p.tw, p.wq, P);
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

// ------------------------------------------------------------- 3-D lines
// Volumes (z, y, x), x fastest, N^3.  One pass transforms every line along
// `axis` (0: x, 1: y, 2: z): MODE 0 the forward DCT-II, MODE 1 the plain
// cosine synthesis S_c, MODE 2 the forward-difference synthesis
// N (S_c(P) - (-1)^j S_c(Q)) of the spectral gradient (zero-flux slot at
// j = N - 1).  A CTA takes 16 lines adjacent in their fastest other
// coordinate (x for the y and z lines, y for the x lines), staged in shared
// memory, so that every global access moves 16 consecutive floats or more;
// two lines share one complex FFT (MODE 0 / 1), or one line per FFT (MODE 2,
// S_c(P) + i S_c(Q)).  In place is allowed: a CTA reads all its lines
// before it writes them.
constexpr int kLines3 = 16;

template <int LOG2N, int MODE>
__global__ void k_dct3_lines(const float* in, float* out, int axis,
                             const float2* __restrict__ tw, const float2* __restrict__ wq) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N, PADN = C::PADN, TPF = C::TPF;
  constexpr int NF = MODE == 2 ? kLines3 : kLines3 / 2;  // FFTs per CTA
  extern __shared__ float2 sm3[];
  float* stg = reinterpret_cast<float*>(sm3 + NF * PADN);  // [line][n], row stride SN
  constexpr int SN = N + 1;  // odd stride: the 16 lines of a y / z column fall into 16 banks
  const int f = (int)threadIdx.x / TPF, t = (int)threadIdx.x % TPF;
  const int nthr = (int)blockDim.x;
  const size_t NN = (size_t)N * N;
  const int L0 = (int)blockIdx.x * kLines3;
  const int outer = L0 / N, inner0 = L0 % N;
  const size_t base = axis == 0 ? (size_t)L0 * N : (size_t)outer * (axis == 1 ? NN : (size_t)N) + inner0;
  const size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)N : NN);
  // load: element e of the CTA's block -> line l, position n
  for (int e = (int)threadIdx.x; e < kLines3 * N; e += nthr) {
    int l, n;
    if (axis == 0) { l = e / N; n = e % N; }
    else { l = e % kLines3; n = e / kLines3; }
    const size_t g = axis == 0 ? base + (size_t)l * N + n : base + (size_t)l + (size_t)n * stride;
    stg[l * SN + n] = in[g];
  }
  __syncthreads();
  float2* buf = sm3 + f * PADN;
  const float fN = (float)N;
  if (MODE == 0) {
    const float* xa = stg + (2 * f) * SN;
    const float* xb = xa + SN;
    for (int n = t; n < N; n += TPF) buf[padi(mk_pos(n, N))] = make_float2(xa[n], xb[n]);
  } else {
    // pre-step from the line spectra (MODE 1: lines 2f, 2f+1; MODE 2: line f)
    const float* xa = stg + (MODE == 1 ? 2 * f : f) * SN;
    const float* xb = xa + SN;
    for (int k = t; k <= N / 2; k += TPF) {
      if (MODE == 1) {
        if (k == 0) buf[0] = make_float2(xa[0], xb[0]);
        else if (k == N / 2) buf[padi(k)] = make_float2(kSqrt2 * xa[k], kSqrt2 * xb[k]);
        else {
          float2 zk, zn;
          inv_pre(xa[k], xa[N - k], xb[k], xb[N - k], __ldg(&wq[k]), zk, zn);
          buf[padi(k)] = zk;
          buf[padi(N - k)] = zn;
        }
      } else {
        if (k == 0) buf[0] = make_float2(0.f, 0.f);
        else if (k == N / 2) buf[padi(k)] = make_float2(-kSqrt2 * xa[k], kSqrt2 * xa[k]);
        else {
          float2 zk, zn;
          deriv_pre(xa[k], xa[N - k], __ldg(&wq[k]), zk, zn);
          buf[padi(k)] = zk;
          buf[padi(N - k)] = zn;
        }
      }
    }
  }
  __syncthreads();
  if (MODE == 0) fft_smem<LOG2N, -1, TPF>(buf, t, tw, 0);
  else fft_smem<LOG2N, +1, TPF>(buf, t, tw, 0);
  // results back into the staging lines (each FFT group writes only its own lines)
  if (MODE == 0) {
    float* xa = stg + (2 * f) * SN;
    float* xb = xa + SN;
    for (int k = t; k <= N / 2; k += TPF) {
      if (k == 0 || k == N / 2) {
        const float sc = k == 0 ? 1.f : kRsqrt2;
        const float2 z = buf[padi(k)];
        xa[k] = sc * z.x;
        xb[k] = sc * z.y;
      } else {
        float ak, an, bk, bn;
        fwd_post(buf[padi(k)], buf[padi(N - k)], __ldg(&wq[k]), ak, an, bk, bn);
        xa[k] = ak;
        xa[N - k] = an;
        xb[k] = bk;
        xb[N - k] = bn;
      }
    }
  } else if (MODE == 1) {
    float* xa = stg + (2 * f) * SN;
    float* xb = xa + SN;
    for (int n = t; n < N; n += TPF) {
      const float2 z = buf[padi(mk_pos(n, N))];
      xa[n] = z.x;
      xb[n] = z.y;
    }
  } else {
    float* xa = stg + f * SN;
    for (int n = t; n < N; n += TPF) {
      const float2 z = buf[padi(mk_pos(n, N))];
      xa[n] = n == N - 1 ? 0.f : fN * (z.x - ((n & 1) ? -z.y : z.y));
    }
  }
  __syncthreads();
  for (int e = (int)threadIdx.x; e < kLines3 * N; e += nthr) {
    int l, n;
    if (axis == 0) { l = e / N; n = e % N; }
    else { l = e % kLines3; n = e / kLines3; }
    const size_t g = axis == 0 ? base + (size_t)l * N + n : base + (size_t)l + (size_t)n * stride;
    out[g] = stg[l * SN + n];
  }
}

// Spectral gain of the 3-D solve: X *= sN3 / (alpha + mu_x + mu_y + mu_z), 0 for
// the constant mode when alpha == 0.
__global__ void k_gain3(float* __restrict__ X, const float* __restrict__ mu, int N, float alpha, float sN3) {
  const size_t NN = (size_t)N * N, n3 = NN * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
    const int kx = (int)(i % N), ky = (int)((i / N) % N), kz = (int)(i / NN);
    const float den = alpha + __ldg(&mu[kx]) + __ldg(&mu[ky]) + __ldg(&mu[kz]);
    X[i] = den > 0.f ? X[i] * (sN3 / den) : 0.f;
  }
}

template <int LOG2N>
cudaError_t launch_dct3_lines(const DctPlan& p, const float* in, float* out, int axis, int mode, cudaStream_t st) {
  using C = FftCfg<LOG2N>;
  constexpr int N = C::N;
  const int nf = mode == 2 ? kLines3 : kLines3 / 2;
  const size_t sm = (size_t)nf * C::PADN * sizeof(float2) + (size_t)kLines3 * (N + 1) * sizeof(float);
  const int grid = N * N / kLines3, thr = nf * C::TPF;
  cudaError_t e;
  if (mode == 0) {
    if ((e = set_smem(k_dct3_lines<LOG2N, 0>, sm))) return e;
    k_dct3_lines<LOG2N, 0><<<grid, thr, sm, st>>>(in, out, axis, p.tw, p.wq);
  } else if (mode == 1) {
    if ((e = set_smem(k_dct3_lines<LOG2N, 1>, sm))) return e;
    k_dct3_lines<LOG2N, 1><<<grid, thr, sm, st>>>(in, out, axis, p.tw, p.wq);
  } else {
    if ((e = set_smem(k_dct3_lines<LOG2N, 2>, sm))) return e;
    k_dct3_lines<LOG2N, 2><<<grid, thr, sm, st>>>(in, out, axis, p.tw, p.wq);
  }
  return cudaGetLastError();
}

}  // namespace

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_tiled_fn() {
  static EncodeTiledFn fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(f);
  }();
  return fn;
}

bool encode_b4_map(CUtensorMap* m, const float* base, int N, int ncols) {
  EncodeTiledFn fn = encode_tiled_fn();
  if (!fn || ((uintptr_t)base & 15u)) return false;
  const cuuint64_t dims[3] = {4, (cuuint64_t)N, (cuuint64_t)(N / 4)};
  const cuuint64_t strides[2] = {16, (cuuint64_t)N * 16};
  const cuuint32_t box[3] = {4, (cuuint32_t)ncols, (cuuint32_t)(N / 4 < 256 ? N / 4 : 256)};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool encode_pairs_map(CUtensorMap* m, const float* base, int N) {
  EncodeTiledFn fn = encode_tiled_fn();
  if (!fn || ((uintptr_t)base & 15u) || N < 512) return false;
  const cuuint64_t dims[3] = {4, (cuuint64_t)N / 2, (cuuint64_t)N / 2};
  const cuuint64_t strides[2] = {16, (cuuint64_t)N * 8};
  const cuuint32_t box[3] = {4, 1, 256};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

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

#define GP_FFT_DISPATCH(N, CALL)   \
  switch (N) {                     \
    case 16: return CALL(4);       \
    case 32: return CALL(5);       \
    case 64: return CALL(6);       \
    case 128: return CALL(7);      \
    case 256: return CALL(8);      \
    case 512: return CALL(9);      \
    case 1024: return CALL(10);    \
    case 2048: return CALL(11);    \
    case 4096: return CALL(12);    \
    case 8192: return CALL(13);    \
    default: return cudaErrorInvalidValue; \
  }

cudaError_t dct_fft_pass(const DctPlan& p, int pass, const float* in, float* out, float alpha, float scale,
                         cudaStream_t st) {
  if (!p.fft) return cudaErrorInvalidValue;
#define GP_CALL(L) launch_fft_pass<L>(p, pass, in, out, alpha, scale, st)
  GP_FFT_DISPATCH(p.N, GP_CALL)
#undef GP_CALL
}

cudaError_t dct_grad_cols(const DctPlan& p, const float* in, float* A, float* B, float alpha, float scale,
                          cudaStream_t st) {
  if (!p.fft) return cudaErrorInvalidValue;
#define GP_CALL(L) launch_grad_cols<L>(p, in, A, B, alpha, scale, st)
  GP_FFT_DISPATCH(p.N, GP_CALL)
#undef GP_CALL
}

cudaError_t dct_grad_rows(const DctPlan& p, const float* A, const float* B, float* gx, float* gy, float* phi,
                          cudaStream_t st) {
  if (!p.fft) return cudaErrorInvalidValue;
#define GP_CALL(L) launch_grad_rows<L>(p, A, B, gx, gy, phi, st)
  GP_FFT_DISPATCH(p.N, GP_CALL)
#undef GP_CALL
}

cudaError_t dct_emd_step_fwd(const DctPlan& p, const float* gq, const float* sin_, const float* pin, const float* g,
                             float* sout, float* pout, float* out, const EmdParams& P, cudaStream_t st) {
  if (!p.fft || P.N != p.N || grad4k_supported(p)) return cudaErrorInvalidValue;  // 4096: emd_rows_step_4k
#define GP_CALL(L) launch_emd_step_fwd<L>(p, gq, sin_, pin, g, sout, pout, out, P, st)
  GP_FFT_DISPATCH(p.N, GP_CALL)
#undef GP_CALL
}

cudaError_t dct_rof_step_fwd(const DctPlan& p, const float* gu, const float* pin, const float* I, float* pout,
                             float* out, const RofParams& P, cudaStream_t st) {
  if (!p.fft || P.N != p.N || grad4k_supported(p)) return cudaErrorInvalidValue;  // 4096: rof_rows_step_4k
#define GP_CALL(L) launch_rof_step_fwd<L>(p, gu, pin, I, pout, out, P, st)
  GP_FFT_DISPATCH(p.N, GP_CALL)
#undef GP_CALL
}

cudaError_t dct3_lines(const DctPlan& p, const float* in, float* out, int axis, int mode, cudaStream_t st) {
  if (!p.fft || p.N > 512) return cudaErrorInvalidValue;
  switch (p.N) {
    case 16: return launch_dct3_lines<4>(p, in, out, axis, mode, st);
    case 32: return launch_dct3_lines<5>(p, in, out, axis, mode, st);
    case 64: return launch_dct3_lines<6>(p, in, out, axis, mode, st);
    case 128: return launch_dct3_lines<7>(p, in, out, axis, mode, st);
    case 256: return launch_dct3_lines<8>(p, in, out, axis, mode, st);
    case 512: return launch_dct3_lines<9>(p, in, out, axis, mode, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t dct3_gain(const DctPlan& p, float* X, float alpha, float scale, cudaStream_t st) {
  const int N = p.N;
  const size_t n3 = (size_t)N * N * N;
  const float sN3 = (float)((double)scale / ((double)N * N * N));
  const size_t blocks = (n3 + 255) / 256;
  k_gain3<<<(unsigned)(blocks < 65535 * 16 ? blocks : 65535 * 16), 256, 0, st>>>(X, p.mu, N, alpha, sN3);
  return cudaGetLastError();
}

// g3 = grad x and (u != nullptr) u = x for x = scale (alpha - Lap)^{-1} b on an
// N^3 grid: three forward line passes, the spectral gain, then the
// syntheses, sharing S_z X between the x, y components and u:
//   gz = S_x S_y D_z X,  gx = D_x S_y S_z X,  u = S_x S_y S_z X,  gy = S_x D_y S_z X.
// W0..W2 are N^3 scratch volumes; b is not written (it may alias u).
// Returns the number of line / gain launches through *nlaunch.
cudaError_t solve_grad3(const DctPlan& p, const float* b, float* g3, float* u, float* W0, float* W1, float* W2,
                        float alpha, float scale, cudaStream_t st, int* nlaunch) {
  const size_t n3 = (size_t)p.N * p.N * p.N;
  float* gx = g3;
  float* gy = g3 + n3;
  float* gz = g3 + 2 * n3;
  cudaError_t e;
#define GP_L3(IN, OUT, AX, MODE) \
  if ((e = dct3_lines(p, IN, OUT, AX, MODE, st))) return e
  GP_L3(b, W0, 0, 0);
  GP_L3(W0, W0, 1, 0);
  GP_L3(W0, W0, 2, 0);
  if ((e = dct3_gain(p, W0, alpha, scale, st))) return e;
  GP_L3(W0, W1, 2, 1);  // S_z X
  GP_L3(W0, W2, 2, 2);  // D_z X
  GP_L3(W2, W2, 1, 1);
  GP_L3(W2, gz, 0, 1);
  GP_L3(W1, W2, 1, 1);  // S_y S_z X
  GP_L3(W2, gx, 0, 2);
  if (u) GP_L3(W2, u, 0, 1);
  GP_L3(W1, W1, 1, 2);  // D_y S_z X
  GP_L3(W1, gy, 0, 1);
#undef GP_L3
  if (nlaunch) *nlaunch = u ? 13 : 12;
  return cudaSuccess;
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
    if ((e = cudaMalloc(&p.err, sizeof(int)))) return e;
    if ((e = cudaMemset(p.err, 0, sizeof(int)))) return e;
    std::vector<float2> tw(N), wq(N / 2 + 1);
    for (int m = 0; m < N; ++m) tw[m] = make_float2((float)cos(2 * PI * m / N), (float)-sin(2 * PI * m / N));
    for (int k = 0; k <= N / 2; ++k) wq[k] = make_float2((float)cos(PI * k / (2.0 * N)), (float)-sin(PI * k / (2.0 * N)));
    if ((e = cudaMalloc(&p.tw, sizeof(float2) * N))) return e;
    if ((e = cudaMalloc(&p.wq, sizeof(float2) * (N / 2 + 1)))) return e;
    if ((e = cudaMemcpy(p.tw, tw.data(), sizeof(float2) * N, cudaMemcpyHostToDevice))) return e;
    if ((e = cudaMemcpy(p.wq, wq.data(), sizeof(float2) * (N / 2 + 1), cudaMemcpyHostToDevice))) return e;
  }
  // The dense matrix serves the sizes without a fast transform.
  if (!p.fft) return dct_plan_dense(p);
  return cudaSuccess;
}

cudaError_t dct_plan_dense(DctPlan& p) {
  if (p.C && p.CT) return cudaSuccess;
  const int N = p.N;
  const double PI = 3.14159265358979323846;
  std::vector<float> C((size_t)N * N), CT((size_t)N * N);
  for (int k = 0; k < N; ++k) {
    const double s = (k == 0) ? sqrt(1.0 / N) : sqrt(2.0 / N);
    for (int n = 0; n < N; ++n) {
      const float v = (float)(s * cos(PI * k * (2.0 * n + 1.0) / (2.0 * N)));
      C[(size_t)k * N + n] = v;
      CT[(size_t)n * N + k] = v;
    }
  }
  cudaError_t e;
  if (!p.C) {
    if ((e = cudaMalloc(&p.C, sizeof(float) * (size_t)N * N))) return e;
    if ((e = cudaMemcpy(p.C, C.data(), sizeof(float) * (size_t)N * N, cudaMemcpyHostToDevice))) return e;
  }
  if (!p.CT) {
    if ((e = cudaMalloc(&p.CT, sizeof(float) * (size_t)N * N))) return e;
    if ((e = cudaMemcpy(p.CT, CT.data(), sizeof(float) * (size_t)N * N, cudaMemcpyHostToDevice))) return e;
  }
  return cudaSuccess;
}

// E[k][j] = N (C[k][j+1] - C[k][j]) = -2N s_k sin(pi k (j+1) / N) sin(pi k / 2N)
// (product form: no cancellation), j < N-1; the last column is the zero slot.
cudaError_t dct_plan_grad_dense(DctPlan& p) {
  if (p.E && p.ET) return cudaSuccess;
  const int N = p.N;
  const double PI = 3.14159265358979323846;
  std::vector<float> E((size_t)N * N), ET((size_t)N * N);
  for (int k = 0; k < N; ++k) {
    const double s = (k == 0) ? sqrt(1.0 / N) : sqrt(2.0 / N);
    const double sh = sin(PI * k / (2.0 * N));
    for (int j = 0; j < N; ++j) {
      const float v = j == N - 1 ? 0.f : (float)(-2.0 * N * s * sin(PI * k * (j + 1.0) / N) * sh);
      E[(size_t)k * N + j] = v;
      ET[(size_t)j * N + k] = v;
    }
  }
  cudaError_t e;
  if (!p.E) {
    if ((e = cudaMalloc(&p.E, sizeof(float) * (size_t)N * N))) return e;
    if ((e = cudaMemcpy(p.E, E.data(), sizeof(float) * (size_t)N * N, cudaMemcpyHostToDevice))) return e;
  }
  if (!p.ET) {
    if ((e = cudaMalloc(&p.ET, sizeof(float) * (size_t)N * N))) return e;
    if ((e = cudaMemcpy(p.ET, ET.data(), sizeof(float) * (size_t)N * N, cudaMemcpyHostToDevice))) return e;
  }
  return cudaSuccess;
}

void dct_plan_free(DctPlan& p) {
  if (p.tw) cudaFree(p.tw);
  if (p.wq) cudaFree(p.wq);
  if (p.mu) cudaFree(p.mu);
  if (p.C) cudaFree(p.C);
  if (p.CT) cudaFree(p.CT);
  if (p.E) cudaFree(p.E);
  if (p.ET) cudaFree(p.ET);
  if (p.Cs) cudaFree(p.Cs);
  if (p.CTs) cudaFree(p.CTs);
  if (p.Es) cudaFree(p.Es);
  if (p.ETs) cudaFree(p.ETs);
  if (p.Cs16) cudaFree(p.Cs16);
  if (p.CTs16) cudaFree(p.CTs16);
  if (p.Es16) cudaFree(p.Es16);
  if (p.ETs16) cudaFree(p.ETs16);
  if (p.tc16) cudaFree(p.tc16);
  if (p.err) cudaFree(p.err);
  p = DctPlan();
}

}  // namespace gp
