// The gradient-form cosine solve and the stencil step at N = 4096, with
// register-resident transforms (the spectral gradient of (alpha - Lap)^{-1} b,
// Appendix A of arXiv 1805.09453: the cosine basis diagonalises the Neumann
// Laplacian; the G-prox PDHG updates of sections 3.1 / 3.2).
//
// Transform.  The length-4096 complex FFT is three radix-16 stages
// (4096 = 16 * 16 * 16) whose butterflies stay in registers, 16 complex values
// per thread of a 256-thread CTA, with two exchanges through a padded
// shared-memory buffer (layout [16][16][17]: every exchange store and load is
// free of bank conflicts).  Only the forward transform is compiled; the
// unnormalised inverse is conj(fft(conj(x))), with the conjugations folded
// into the callers' pre- and post-steps.
//
// Index maps of one transform: thread th owns the transform index
//   t = pair_t(th) = 32 w + l (lane l < 16 of warp w),  271 - 32 w - l (l >= 16),
// so that lanes l and l ^ 16 own t and 255 - t; with t = a + 16 b:
//   entry:   v[r] = x[t + 256 r]
//   stage A: DFT over r, twiddle e^{-2 pi i t k0 / 4096}; exchange [k0][b][a]
//   stage B: thread th = a' + 16 k0: DFT over b, twiddle e^{-2 pi i a' c / 256};
//            exchange [c][k0][a']
//   stage C: the thread owning t = k0 + 16 c: DFT over a
//   exit:    v[d] = X[t + 256 d]
// The Makhoul order of a length-N real sequence puts sample 2m at position
// m and sample 2m + 1 at position N - 1 - m; so a thread's positions
// t + 256 d (d < 8) and its partner's 255 - t + 256 (15 - d) are the samples
// 2p and 2p + 1, p = t + 256 d: one shuffle per pair of samples lets every
// load and store of samples move two neighbours at once.
//
// Layout.  Between the passes, spectra live "pair-interleaved": rows 2q and
// 2q + 1 of a plane are stored as one block of N float2 (row 2q, row 2q + 1)
// per spectral index, so a row pair is one contiguous 32 KB block (the row
// passes load and store it coalesced) and a column pair over all rows is
// a 3-D tensor {4 floats, N/2 column pairs, N/2 row pairs} that the column
// pass moves with bulk tensor copies (box {4, 1, 256}: 4 KB).
//
// Kernels (N = 4096 only; other sizes use the shared-memory passes of dct.cu):
//   k_rows_fwd_4k      rows: forward DCT-II of a row-major plane -> row spectra
//   k_cols_grad_4k     columns: forward DCT-II, gain, plain and D_y syntheses
//   k_rows_grad_4k     rows: D_x and plain syntheses -> grad (and phi)
//   k_rof_rows_step_4k rows: the syntheses, the ROF stencil step and the next
//                      forward row transform in one pass (grad u never in HBM)
//   k_emd_rows_step_4k the same for the EMD step
#include <math.h>

#include <algorithm>

#include "fft_common.cuh"
#include "gp_internal.cuh"
#include "stencil.cuh"
#include "tma.cuh"

namespace gp {
namespace {

constexpr int kN = 4096;
constexpr int kT = 256;                 // threads of one transform (= CTA)
constexpr int kPairs = kN / 2;          // row pairs
constexpr int kExStride = 17;           // padded row of the exchange buffer
constexpr int kExPlane = 16 * kExStride;
constexpr int kExSize = 16 * kExPlane;  // float2 entries (34816 B)
constexpr size_t kExBytes = (size_t)kExSize * 8;
constexpr size_t kPlaneRowPair = 2 * (size_t)kN;  // floats per row pair of a pair-interleaved plane

__device__ __forceinline__ int pair_t(int th) {
  const int w = th >> 5, l = th & 31;
  return l < 16 ? 32 * w + l : 271 - 32 * w - l;
}

__device__ __forceinline__ float shfl16(float x) { return __shfl_xor_sync(0xffffffffu, x, 16); }

// Stage twiddle bases: stage A e^{-2 pi i t q / 4096}, stage B
// e^{-2 pi i 16 a q / 4096}, q = 1, 2, 4, 8; the other powers are products.
struct Tw4k {
  float2 a[4], b[4];
  __device__ __forceinline__ void load(const float2* __restrict__ tw, int t, int a_b) {
    a[0] = __ldg(&tw[t]);
    a[1] = __ldg(&tw[2 * t]);
    a[2] = __ldg(&tw[4 * t]);
    a[3] = __ldg(&tw[8 * t]);
    const int m = 16 * a_b;
    b[0] = __ldg(&tw[m]);
    b[1] = __ldg(&tw[2 * m]);
    b[2] = __ldg(&tw[4 * m]);
    b[3] = __ldg(&tw[8 * m]);
  }
};

// v[r] *= w^r (r = 1..15), w^1, w^2, w^4, w^8 given.
__device__ __forceinline__ void twiddle16(float2 (&v)[16], const float2 (&base)[4]) {
  float2 w[16];
  w[1] = base[0];
  w[2] = base[1];
  w[3] = cmul(w[1], w[2]);
  w[4] = base[2];
#pragma unroll
  for (int r = 5; r < 8; ++r) w[r] = cmul(w[r - 4], w[4]);
  w[8] = base[3];
#pragma unroll
  for (int r = 9; r < 16; ++r) w[r] = cmul(w[r - 8], w[8]);
#pragma unroll
  for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], w[r]);
}

// Length-4096 forward complex FFT (e^{-2 pi i n k / N}, unnormalised) of the
// CTA, index maps in the file header.  Three CTA barriers; on return the
// exchange buffer is still being read: synchronise before writing it again.
__device__ __forceinline__ void fft4k(float2 (&v)[16], float2* __restrict__ ex, int th,
                                      const float2* __restrict__ twt) {
  const int t = pair_t(th);
  const int ta = t & 15, tb = t >> 4;    // stage A / C coordinates of t
  const int sa = th & 15, sk = th >> 4;  // stage B: (a', k0)
  Tw4k tw;  // reloaded per transform (L1 hits): no registers held between transforms
  tw.load(twt, t, sa);
  dft_reg<16, -1>(v);
  twiddle16(v, tw.a);
#pragma unroll
  for (int k0 = 0; k0 < 16; ++k0) ex[k0 * kExPlane + tb * kExStride + ta] = v[k0];
  __syncthreads();
#pragma unroll
  for (int b = 0; b < 16; ++b) v[b] = ex[sk * kExPlane + b * kExStride + sa];
  __syncthreads();
  dft_reg<16, -1>(v);
  twiddle16(v, tw.b);
#pragma unroll
  for (int c = 0; c < 16; ++c) ex[c * kExPlane + sk * kExStride + sa] = v[c];
  __syncthreads();
#pragma unroll
  for (int a = 0; a < 16; ++a) v[a] = ex[tb * kExPlane + ta * kExStride + a];
  dft_reg<16, -1>(v);
}

// Makhoul twiddle w_k = e^{-i pi k / 2N} for k = t + 256 d: w_t e^{-i pi d / 32}
// (w_t from the table, the second factor a compile-time constant).
__device__ __forceinline__ float2 wq_k(float2 wt, int d) {
  const float C[16] = {1.f, 0.99518472667219693f, 0.98078528040323043f, 0.95694033573220882f,
                       0.92387953251128674f, 0.88192126434835505f, 0.83146961230254524f, 0.77301045336273699f,
                       0.70710678118654757f, 0.63439328416364549f, 0.55557023301960218f, 0.47139673682599764f,
                       0.38268343236508978f, 0.29028467725446239f, 0.19509032201612828f, 0.098017140329560604f};
  const float S[16] = {0.f, 0.098017140329560604f, 0.19509032201612828f, 0.29028467725446239f,
                       0.38268343236508978f, 0.47139673682599764f, 0.55557023301960218f, 0.63439328416364549f,
                       0.70710678118654757f, 0.77301045336273699f, 0.83146961230254524f, 0.88192126434835505f,
                       0.92387953251128674f, 0.95694033573220882f, 0.98078528040323043f, 0.99518472667219693f};
  return cmul(wt, make_float2(C[d], -S[d]));
}

// Inverse Makhoul pre-step for one spectral index k, 0 <= k < N: the value
// Z[k] whose unnormalised inverse FFT (Makhoul order) is S_c(P) + i S_c(Q),
// S_c(X)[j] = X_0 + 2 sum_{l>=1} X_l cos(pi l (2j+1) / 2N), given
// P = P_k, Pn = P_{N-k}, Q = Q_k, Qn = Q_{N-k} (P_N = Q_N = 0) and w = w_k:
//   Z[k] = conj(w) (P - i Pn) + i conj(w) (Q - i Qn),
// returned conjugated, ready for the forward transform.
__device__ __forceinline__ float2 inv_pre_k(float P, float Pn, float Q, float Qn, float2 w) {
  const float2 ua = make_float2(w.x * P - w.y * Pn, -w.y * P - w.x * Pn);
  const float2 ub = make_float2(w.x * Q - w.y * Qn, -w.y * Q - w.x * Qn);
  return make_float2(ua.x - ub.y, -(ua.y + ub.x));
}

// The same for the forward difference N (S_c(X)[j+1] - S_c(X)[j]) of a cosine
// series, written N (S_c(P)[j] - (-1)^j S_c(Q)[j]) with theta_l = pi l / N,
// P_l = -2 sin^2(theta_l / 2) X_l, Q_l = sin(theta_l) X_{N-l}, Q_0 = 0; with
// w_k = (c, -s): P_k = -2 s^2 X_k, P_{N-k} = -2 c^2 X_{N-k}, Q_k = 2sc X_{N-k},
// Q_{N-k} = 2sc X_k.
__device__ __forceinline__ float2 deriv_pre_k(float x, float xn, float2 w) {
  const float c = w.x, s = -w.y, sc2 = 2.f * s * c;
  return inv_pre_k(-2.f * s * s * x, -2.f * c * c * xn, sc2 * xn, sc2 * x, w);
}

// mu_k = (4/h^2) sin^2(pi k / 2N) from w_k = e^{-i pi k / 2N}: 4 N^2 (Im w_k)^2.
__device__ __forceinline__ float mu_of_w(float2 w) { return 4.f * (float)kN * (float)kN * w.y * w.y; }

__device__ __forceinline__ float gain4k(float muk, float mul, float alpha, float sN2) {
  const float den = alpha + muk + mul;
  return den > 0.f ? __fdividef(sN2, den) : 0.f;  // den >= pi^2 (or alpha): far from the fast-divide limits
}

// After an inverse transform (v = conj of the Makhoul-ordered synthesis
// S_c(P) + i S_c(Q)), the synthesis at the samples 2p and 2p + 1 of position
// p = t + 256 D, D < 8: the thread's own v[D] and its partner lane's
// v[15 - D].  Call from converged code (the shuffle needs the whole warp).
struct SynPair {
  float2 e, o;  // S_c(P) + i S_c(Q) at samples 2p (even) and 2p + 1 (odd)
};
template <int D>
__device__ __forceinline__ SynPair syn_pair(const float2 (&v)[16]) {
  const float qx = shfl16(v[15 - D].x), qy = shfl16(v[15 - D].y);
  return SynPair{make_float2(v[D].x, -v[D].y), make_float2(qx, -qy)};
}
// D_x / D_y value pair at samples (2p, 2p + 1): N (S_c(P) - (-1)^j S_c(Q)),
// zero-flux slot at j = N - 1.
__device__ __forceinline__ float2 deriv_pair(const SynPair& sp, int p) {
  const float fN = (float)kN;
  return make_float2(fN * (sp.e.x - sp.e.y), 2 * p + 1 == kN - 1 ? 0.f : fN * (sp.o.x + sp.o.y));
}

// The sample pairs of the last inverse transform handed to emit(p, SynPair)
// for p = t + 256 d, d < 8.
template <typename Emit>
__device__ __forceinline__ void emit_pairs(const float2 (&v)[16], int t, Emit emit) {
  emit(t, syn_pair<0>(v));
  emit(t + kT, syn_pair<1>(v));
  emit(t + 2 * kT, syn_pair<2>(v));
  emit(t + 3 * kT, syn_pair<3>(v));
  emit(t + 4 * kT, syn_pair<4>(v));
  emit(t + 5 * kT, syn_pair<5>(v));
  emit(t + 6 * kT, syn_pair<6>(v));
  emit(t + 7 * kT, syn_pair<7>(v));
}

// Forward-transform input from two real rows held as pair-interleaved samples:
// get(m) returns (row0[2m], row0[2m+1], row1[2m], row1[2m+1]) for m < N/2;
// the Makhoul-ordered complex input z = row0 + i row1 lands in v (the odd
// samples through the partner lane).
template <typename Get>
__device__ __forceinline__ void gather_pairs(float2 (&v)[16], int t, Get get) {
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const float4 L = get(t + kT * r);
    v[r] = make_float2(L.x, L.z);
    v[15 - r] = make_float2(shfl16(L.y), shfl16(L.w));
  }
}

// Forward Makhoul post-step of two packed real sequences: Zs holds the
// transform Z (float2[N], written by the caller, then a barrier); returns in
// v[d] the DCT-II pair (X_a[k], X_b[k]), k = t + 256 d, times gain(w_k) when G.
template <bool G, typename Gain>
__device__ __forceinline__ void post_pairs(float2 (&v)[16], const float2* Zs, int t, float2 wt, Gain gain) {
#pragma unroll
  for (int d = 0; d < 16; ++d) {
    const int k = t + kT * d;
    const float2 z = v[d], zp = Zs[(kN - k) & (kN - 1)];
    const float2 va = make_float2(0.5f * (z.x + zp.x), 0.5f * (z.y - zp.y));   // spectrum of the real part
    const float2 vb = make_float2(0.5f * (z.y + zp.y), -0.5f * (z.x - zp.x));  // of the imaginary part
    const float2 w = wq_k(wt, d);
    float2 x = make_float2(w.x * va.x - w.y * va.y, w.x * vb.x - w.y * vb.y);
    if constexpr (G) {
      const float2 gn = gain(w);
      x.x *= gn.x;
      x.y *= gn.y;
    }
    v[d] = x;
  }
}

// Row-pair pre-step from a pair-interleaved block (ld(k) = (row 0, row 1) at
// spectral index k): MODE 0 / 1: D_x synthesis of row 0 / 1; MODE 2: plain
// synthesis of both rows.
template <int MODE, typename Ld>
__device__ __forceinline__ void pre_pairs(float2 (&v)[16], int t, float2 wt, Ld ld) {
#pragma unroll
  for (int d = 0; d < 16; ++d) {
    const int k = t + kT * d;
    const float2 xk = ld(k);
    const float2 xn = k == 0 ? make_float2(0.f, 0.f) : ld(kN - k);
    const float2 w = wq_k(wt, d);
    if (MODE == 0) v[d] = deriv_pre_k(xk.x, xn.x, w);
    else if (MODE == 1) v[d] = deriv_pre_k(xk.y, xn.y, w);
    else v[d] = inv_pre_k(xk.x, xn.x, xk.y, xn.y, w);
  }
}

__device__ __forceinline__ float2 ldg2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }
__device__ __forceinline__ float4 ld4g(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
__device__ __forceinline__ void st4g(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void prefetch_l2(const float* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// ------------------------------------------------------- row pass, forward
// CTA = one row pair (rows 2 rp, 2 rp + 1) of a row-major plane; output: its
// row spectra, pair-interleaved (float2 per spectral index).
__global__ void __launch_bounds__(kT, 3)
    k_rows_fwd_4k(const float* __restrict__ in, float* __restrict__ out, const float2* __restrict__ tw,
                  const float2* __restrict__ wq) {
  extern __shared__ __align__(128) float sf4k[];
  float2* ex = reinterpret_cast<float2*>(sf4k);
  float2* Zs = ex + kExSize;
  const int th = threadIdx.x, t = pair_t(th), rp = blockIdx.x;
  const float* r0 = in + (size_t)(2 * rp) * kN;
  const float* r1 = r0 + kN;
  float2 v[16];
  gather_pairs(v, t, [&](int m) {
    const float2 a = ldg2(r0 + 2 * m), b = ldg2(r1 + 2 * m);
    return make_float4(a.x, a.y, b.x, b.y);
  });
  fft4k(v, ex, th, tw);
#pragma unroll
  for (int d = 0; d < 16; ++d) Zs[t + kT * d] = v[d];
  __syncthreads();
  post_pairs<false>(v, Zs, t, __ldg(&wq[t]), [](float2) { return make_float2(1.f, 1.f); });
  float* o = out + (size_t)rp * kPlaneRowPair;
#pragma unroll
  for (int d = 0; d < 16; ++d) *reinterpret_cast<float2*>(o + 2 * (t + kT * d)) = v[d];
}

// ------------------------------------------------ column pass, gradient form
// CTA = one column pair (2cp, 2cp + 1) of the pair-interleaved row spectra
// `in`; forward DCT-II along the columns, gain 1 / (alpha + mu_k + mu_l)
// (times sN2), then three syntheses written by bulk tensor stores:
//   A[:, pair] = S_c(X)  (plain),  B[:, col] = D_y S_c(X_col) for each column
// (A and B pair-interleaved; `in` may alias A).  Shared memory: the exchange
// buffer (between transforms it stages the outputs for the tensor stores);
// the column pair as float4 per row pair (staged by the tensor copy, then the
// forward spectra Z, then the gained spectra X); the mbarrier.  A copy that
// never lands (bounded wait) poisons the pair with NaN and sets *err.
constexpr size_t kColsSmem = kExBytes + (size_t)kN * 8 + 16;

__global__ void __launch_bounds__(kT, 2)
    k_cols_grad_4k(const __grid_constant__ CUtensorMap tm_in, const __grid_constant__ CUtensorMap tm_a,
                   const __grid_constant__ CUtensorMap tm_b, const float2* __restrict__ tw,
                   const float2* __restrict__ wq, const float* __restrict__ mu, float alpha, float sN2,
                   int* __restrict__ err) {
  extern __shared__ __align__(128) float sc4k[];
  float2* ex = reinterpret_cast<float2*>(sc4k);
  float4* stage = reinterpret_cast<float4*>(sc4k);  // output staging over ex, between transforms
  float* R2 = sc4k + 2 * kExSize;                    // N float2
  uint64_t* mbar = reinterpret_cast<uint64_t*>(R2 + 2 * kN);
  const int th = threadIdx.x, t = pair_t(th), cp = blockIdx.x;
  const uint32_t bar = smem_addr(mbar);
  if (th == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (th == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"((uint32_t)(kN * 8))
                 : "memory");
#pragma unroll
    for (int q = 0; q < 8; ++q) tma_load_3d(smem_addr(R2) + q * 4096, &tm_in, 0, cp, q * 256, bar);
  }
  const float2 wt = __ldg(&wq[t]);
  const float mua = __ldg(&mu[2 * cp]), mub = __ldg(&mu[2 * cp + 1]);
  float poison = 1.f;
  if (!mbar_try(bar, 0)) {
    poison = __int_as_float(0x7fc00000);
    atomicExch(err, 1);
  }
  // R2 as float4 per row pair q: (a[2q], a[2q+1], b[2q], b[2q+1])
  const float4* S4 = reinterpret_cast<const float4*>(R2);
  float2 v[16];
  gather_pairs(v, t, [&](int m) {
    const float4 L = S4[m];
    return make_float4(poison * L.x, poison * L.y, poison * L.z, poison * L.w);
  });
  fft4k(v, ex, th, tw);
  // forward post-step on the owned indices k = t + 256 d (the staged input
  // was consumed before the transform's first barrier)
  float2* Zs = reinterpret_cast<float2*>(R2);
#pragma unroll
  for (int d = 0; d < 16; ++d) Zs[t + kT * d] = v[d];
  __syncthreads();
  post_pairs<true>(v, Zs, t, wt, [&](float2 w) {
    const float muk = mu_of_w(w);
    return make_float2(gain4k(muk, mua, alpha, sN2), gain4k(muk, mub, alpha, sN2));
  });
  __syncthreads();
  float2* Xs = Zs;  // gained spectra X[k] = (X_a[k], X_b[k])
#pragma unroll
  for (int d = 0; d < 16; ++d) Xs[t + kT * d] = v[d];
  __syncthreads();
  const auto ldx = [&](int k) { return Xs[k]; };
  // plain synthesis of both columns -> A
  pre_pairs<2>(v, t, wt, ldx);
  fft4k(v, ex, th, tw);
  __syncthreads();  // every stage-C read of ex is done before the staging overwrites it
  emit_pairs(v, t, [&](int p, const SynPair& sp) { stage[p] = make_float4(sp.e.x, sp.o.x, sp.e.y, sp.o.y); });
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (th == 0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) tma_store_3d(&tm_a, 0, cp, q * 256, smem_addr(stage) + q * 4096);
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }
  // D_y of column a (kept in registers), then of column b -> B
  float2 Da[8];
  pre_pairs<0>(v, t, wt, ldx);
  if (th == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  __syncthreads();  // the store has read the staging area before the transform rewrites it
  fft4k(v, ex, th, tw);
  {
    int d = 0;
    emit_pairs(v, t, [&](int p, const SynPair& sp) { Da[d++] = deriv_pair(sp, p); });
  }
  pre_pairs<1>(v, t, wt, ldx);
  __syncthreads();  // the previous transform's reads of ex are done
  fft4k(v, ex, th, tw);
  __syncthreads();
  {
    int d = 0;
    emit_pairs(v, t, [&](int p, const SynPair& sp) {
      const float2 db = deriv_pair(sp, p);
      stage[p] = make_float4(Da[d].x, Da[d].y, db.x, db.y);
      ++d;
    });
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  if (th == 0) {
#pragma unroll
    for (int q = 0; q < 8; ++q) tma_store_3d(&tm_b, 0, cp, q * 256, smem_addr(stage) + q * 4096);
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
}

// --------------------------------------------------- row pass, gradient form
// Persistent CTAs, each walking row pairs rp (rows i0 = 2 rp, i0 + 1) of the
// pair-interleaved column syntheses A (plain) and B (D_y):
//   gx[i] = D_x S_c(A[i]) (i = i0, i0 + 1),  gy[i0, i0+1] = S_c(B[i0, i0+1]),
//   phi[i0, i0+1] = S_c(A[i0, i0+1]) when phi != nullptr.
// gx, gy, phi row-major; gx has its zero slot at j = N - 1.  The next pair's
// blocks are prefetched into L2 while this pair is transformed.
__global__ void __launch_bounds__(kT, 2)
    k_rows_grad_4k(const float* __restrict__ A, const float* __restrict__ B, float* __restrict__ gx,
                   float* __restrict__ gy, float* __restrict__ phi, const float2* __restrict__ tw,
                   const float2* __restrict__ wq) {
  __shared__ __align__(16) float2 ex[kExSize];
  const int th = threadIdx.x, t = pair_t(th);
  const float2 wt = __ldg(&wq[t]);
#pragma unroll 1
  for (int rp = blockIdx.x; rp < kPairs; rp += gridDim.x) {
    const int i0 = 2 * rp, nxt = rp + gridDim.x;
    const float* Ab = A + (size_t)rp * kPlaneRowPair;
    const float* Bb = B + (size_t)rp * kPlaneRowPair;
    if (th == 0 && nxt < kPairs) {
      prefetch_l2(A + (size_t)nxt * kPlaneRowPair, (uint32_t)(kPlaneRowPair * 4));
      prefetch_l2(B + (size_t)nxt * kPlaneRowPair, (uint32_t)(kPlaneRowPair * 4));
    }
    const auto lda = [&](int k) { return ldg2(Ab + 2 * k); };
    const auto ldb = [&](int k) { return ldg2(Bb + 2 * k); };
    float2 v[16];
#pragma unroll 1
    for (int pass = 0; pass < (phi ? 4 : 3); ++pass) {
      // 0 / 1: D_x of row i0 / i0 + 1; 2: plain of the B rows; 3: plain of the A rows (phi)
      if (pass == 0) pre_pairs<0>(v, t, wt, lda);
      else if (pass == 1) pre_pairs<1>(v, t, wt, lda);
      else if (pass == 2) pre_pairs<2>(v, t, wt, ldb);
      else pre_pairs<2>(v, t, wt, lda);
      __syncthreads();  // the previous transform's reads of ex are done
      fft4k(v, ex, th, tw);
      if (pass < 2) {
        float* o = gx + (size_t)(i0 + pass) * kN;
        emit_pairs(v, t, [&](int p, const SynPair& sp) { *reinterpret_cast<float2*>(o + 2 * p) = deriv_pair(sp, p); });
      } else {
        float* o = (pass == 2 ? gy : phi) + (size_t)i0 * kN;
        emit_pairs(v, t, [&](int p, const SynPair& sp) {
          *reinterpret_cast<float2*>(o + 2 * p) = make_float2(sp.e.x, sp.o.x);
          *reinterpret_cast<float2*>(o + kN + 2 * p) = make_float2(sp.e.y, sp.o.y);
        });
      }
    }
  }
}

// ------------------------------------------- fused row pass: syntheses + step
// One non-gap G-prox PDHG step fused with the row syntheses of its solve and
// the forward row transform of the next solve.  Persistent CTAs, each owning
// a contiguous band of row pairs and walking it downwards; per pair:
//   D_x syntheses of the two A rows -> gradient x rows (shared memory),
//   plain synthesis of the B rows   -> gradient y rows (shared memory),
//   the stencil step of both rows (the same arithmetic as k_rof_fused /
//   k_emd_fused of stencil.cu) with the row above taken from a per-column
//   carry; its dual (and EMD auxiliary) variables to HBM,
//   the forward transform of the two new right-hand-side rows -> their row
//   spectra, pair-interleaved.
// The band's first row above is synthesised once (two extra transforms).
// Shared memory: ex (the gradient y rows between the transforms and the
// step), two gradient x rows (then the new right-hand sides, then Z), and
// the carry (two floats per column).
constexpr size_t kStepSmem = kExBytes + 2 * (size_t)kN * 4 + 2 * (size_t)kN * 4;

__device__ __forceinline__ void band_of(int b, int G, int& rp0, int& rp1) {
  rp0 = (int)(((long long)b * kPairs) / G);
  rp1 = (int)(((long long)(b + 1) * kPairs) / G);
}

// D_x synthesis of row MODE (0 / 1) of the pair-interleaved block Xb into the
// shared row buffer `row`.
template <int MODE>
__device__ __forceinline__ void synth_dx_row(float2 (&v)[16], const float* Xb, float* row, float2* ex, int th, int t,
                                             float2 wt, const float2* __restrict__ tw) {
  pre_pairs<MODE>(v, t, wt, [&](int k) { return ldg2(Xb + 2 * k); });
  __syncthreads();  // the previous transform's reads of ex are done
  fft4k(v, ex, th, tw);
  emit_pairs(v, t, [&](int p, const SynPair& sp) { *reinterpret_cast<float2*>(row + 2 * p) = deriv_pair(sp, p); });
}

// Plain synthesis of both rows of Xb into ex viewed as float[2][N] (after the
// transform's reads of ex).
__device__ __forceinline__ void synth_plain_rows(float2 (&v)[16], const float* Xb, float2* ex, int th, int t,
                                                 float2 wt, const float2* __restrict__ tw) {
  pre_pairs<2>(v, t, wt, [&](int k) { return ldg2(Xb + 2 * k); });
  __syncthreads();
  fft4k(v, ex, th, tw);
  __syncthreads();  // every stage-C read of ex is done before the rows overwrite it
  float* rows = reinterpret_cast<float*>(ex);
  emit_pairs(v, t, [&](int p, const SynPair& sp) {
    *reinterpret_cast<float2*>(rows + 2 * p) = make_float2(sp.e.x, sp.o.x);
    *reinterpret_cast<float2*>(rows + kN + 2 * p) = make_float2(sp.e.y, sp.o.y);
  });
}

// Forward transform of the two rows r0, r1 (shared, natural order, adjacent)
// with the pair-interleaved row spectra written to `out`; r0 / r1 then hold Z.
__device__ __forceinline__ void forward_rows_out(float2 (&v)[16], float* r0, float* out, float2* ex, int th, int t,
                                                 float2 wt, const float2* __restrict__ tw) {
  const float* r1 = r0 + kN;
  gather_pairs(v, t, [&](int m) {
    const float2 a = *reinterpret_cast<const float2*>(r0 + 2 * m);
    const float2 b = *reinterpret_cast<const float2*>(r1 + 2 * m);
    return make_float4(a.x, a.y, b.x, b.y);
  });
  fft4k(v, ex, th, tw);  // its first barrier: every gather read of r0 / r1 is done
  float2* Zs = reinterpret_cast<float2*>(r0);
#pragma unroll
  for (int d = 0; d < 16; ++d) Zs[t + kT * d] = v[d];
  __syncthreads();
  post_pairs<false>(v, Zs, t, wt, [](float2) { return make_float2(1.f, 1.f); });
#pragma unroll
  for (int d = 0; d < 16; ++d) *reinterpret_cast<float2*>(out + 2 * (t + kT * d)) = v[d];
}

__global__ void __launch_bounds__(kT, 2)
    k_rof_rows_step_4k(const float* __restrict__ A, const float* __restrict__ B, const float* __restrict__ pin,
                       const float* __restrict__ I, float* __restrict__ pout, float* __restrict__ out,
                       const float2* __restrict__ tw, const float2* __restrict__ wq, RofParams P) {
  extern __shared__ __align__(128) float sr4k[];
  float2* ex = reinterpret_cast<float2*>(sr4k);
  float* gyr = sr4k;                // over ex: gradient y rows [2][N] between transforms
  float* gxr = sr4k + 2 * kExSize;  // gradient x rows [2][N], then the right-hand sides, then Z
  float* pbu = gxr + 2 * kN;        // carry: pbar_y of the row above
  float* gyu = pbu + kN;            // carry: (grad u)_y of the row above
  constexpr size_t NN = (size_t)kN * kN;
  const int th = threadIdx.x, t = pair_t(th);
  const float2 wt = __ldg(&wq[t]);
  int rp0, rp1;
  band_of(blockIdx.x, gridDim.x, rp0, rp1);
  float2 v[16];
  // carry of the band's first row above: row 2 rp0 - 1 (the second row of pair rp0 - 1)
  if (rp0 > 0) {
    const int ia = 2 * rp0 - 1;
    synth_dx_row<1>(v, A + (size_t)(rp0 - 1) * kPlaneRowPair, gxr, ex, th, t, wt, tw);
    synth_plain_rows(v, B + (size_t)(rp0 - 1) * kPlaneRowPair, ex, th, t, wt, tw);
    __syncthreads();
    const float* gyrow = gyr + kN;  // the pair's second row
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j0 = 4 * (th + kT * c);
      const size_t ro = (size_t)ia * kN + j0;
      const float4 px = ld4g(pin + ro), py = ld4g(pin + NN + ro);
      const float pxa[4] = {px.x, px.y, px.z, px.w}, pya[4] = {py.x, py.y, py.z, py.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float g1 = gxr[j0 + q], g2 = gyrow[j0 + q];
        float p1x, p1y;
        proj2(pxa[q] + P.sigma * g1, pya[q] + P.sigma * g2, p1x, p1y);
        pbu[j0 + q] = 2.f * p1y - pya[q];  // row ia < N - 1
        gyu[j0 + q] = g2;
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) pbu[4 * (th + kT * c) + q] = gyu[4 * (th + kT * c) + q] = 0.f;
  }
#pragma unroll 1
  for (int rp = rp0; rp < rp1; ++rp) {
    const int i0 = 2 * rp;
    if (th == 0 && rp + 1 < rp1) {  // the next pair's blocks into L2 while this pair is transformed
      prefetch_l2(A + (size_t)(rp + 1) * kPlaneRowPair, (uint32_t)(kPlaneRowPair * 4));
      prefetch_l2(B + (size_t)(rp + 1) * kPlaneRowPair, (uint32_t)(kPlaneRowPair * 4));
    }
    __syncthreads();  // the previous pair's reads of gxr (its Z) are done
    const float* Ab = A + (size_t)rp * kPlaneRowPair;
    synth_dx_row<0>(v, Ab, gxr, ex, th, t, wt, tw);
    synth_dx_row<1>(v, Ab, gxr + kN, ex, th, t, wt, tw);
    synth_plain_rows(v, B + (size_t)rp * kPlaneRowPair, ex, th, t, wt, tw);
    __syncthreads();  // gradient rows complete
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
      const int i = i0 + s;
      const bool yd = i < kN - 1, yu = i > 0;
      const float* gxrow = gxr + s * kN;
      const float* gyrow = gyr + s * kN;
      float rv[4][4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j0 = 4 * (th + kT * c);
        const size_t ro = (size_t)i * kN + j0;
        float gxv[5], gyv[5], pnx[5], pny[5];  // [0]: column j0 - 1
        {
          const float4 a = *reinterpret_cast<const float4*>(gxrow + j0);
          const float4 b = *reinterpret_cast<const float4*>(gyrow + j0);
          const float4 px = ld4g(pin + ro), py = ld4g(pin + NN + ro);
          gxv[1] = a.x; gxv[2] = a.y; gxv[3] = a.z; gxv[4] = a.w;
          gyv[1] = b.x; gyv[2] = b.y; gyv[3] = b.z; gyv[4] = b.w;
          pnx[1] = px.x; pnx[2] = px.y; pnx[3] = px.z; pnx[4] = px.w;
          pny[1] = py.x; pny[2] = py.y; pny[3] = py.z; pny[4] = py.w;
          if (j0 > 0) {
            gxv[0] = gxrow[j0 - 1]; gyv[0] = gyrow[j0 - 1];
            pnx[0] = __ldg(pin + ro - 1); pny[0] = __ldg(pin + NN + ro - 1);
          } else {
            gxv[0] = gyv[0] = pnx[0] = pny[0] = 0.f;
          }
        }
        const float4 Iq = ld4g(I + ro);
        const float Iv[4] = {Iq.x, Iq.y, Iq.z, Iq.w};
        float p1x[5], p1y[5], pbx[5], pby[5];
#pragma unroll
        for (int q = 0; q <= 4; ++q) {
          const int j = j0 - 1 + q;
          const bool xr = j < kN - 1;
          proj2(pnx[q] + P.sigma * gxv[q], pny[q] + P.sigma * gyv[q], p1x[q], p1y[q]);
          if (!xr) p1x[q] = 0.f;
          if (!yd) p1y[q] = 0.f;
          pbx[q] = 2.f * p1x[q] - (xr ? pnx[q] : 0.f);
          pby[q] = 2.f * p1y[q] - (yd ? pny[q] : 0.f);
        }
#pragma unroll
        for (int q = 1; q <= 4; ++q) {
          const int j = j0 + q - 1;
          const bool xl = j > 0;
          const float dpb = (pbx[q] - (xl ? pbx[q - 1] : 0.f) + pby[q] - (yu ? pbu[j] : 0.f)) * P.invh;
          const float lap = (gxv[q] - (xl ? gxv[q - 1] : 0.f) + gyv[q] - (yu ? gyu[j] : 0.f)) * P.invh;
          rv[c][q - 1] = P.lt * Iv[q - 1] + P.tau * dpb - lap;
          pbu[j] = pby[q];  // this thread's own columns: read above, rewritten here
          gyu[j] = gyv[q];
        }
        st4g(pout + ro, p1x[1], p1x[2], p1x[3], p1x[4]);
        st4g(pout + NN + ro, p1y[1], p1y[2], p1y[3], p1y[4]);
      }
      __syncthreads();  // every read of this gradient row is done: its slot takes the right-hand side
      float* rrow = gxr + s * kN;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        *reinterpret_cast<float4*>(rrow + 4 * (th + kT * c)) = make_float4(rv[c][0], rv[c][1], rv[c][2], rv[c][3]);
    }
    __syncthreads();  // both right-hand-side rows complete; the y rows in ex are consumed
    forward_rows_out(v, gxr, out + (size_t)rp * kPlaneRowPair, ex, th, t, wt, tw);
  }
}

__global__ void __launch_bounds__(kT, 2)
    k_emd_rows_step_4k(const float* __restrict__ A, const float* __restrict__ B, const float* __restrict__ sin_,
                       const float* __restrict__ pin, const float* __restrict__ g, float* __restrict__ sout,
                       float* __restrict__ pout, float* __restrict__ out, const float2* __restrict__ tw,
                       const float2* __restrict__ wq, EmdParams P) {
  extern __shared__ __align__(128) float se4k[];
  float2* ex = reinterpret_cast<float2*>(se4k);
  float* gyr = se4k;                // over ex: gradient y rows [2][N] between transforms
  float* gxr = se4k + 2 * kExSize;  // gradient x rows [2][N], then the right-hand sides, then Z
  float* syu = gxr + 2 * kN;        // carry: new s_y of the row above
  constexpr size_t NN = (size_t)kN * kN;
  const int th = threadIdx.x, t = pair_t(th);
  const float2 wt = __ldg(&wq[t]);
  int rp0, rp1;
  band_of(blockIdx.x, gridDim.x, rp0, rp1);
  float2 v[16];
  if (rp0 > 0) {
    const int ia = 2 * rp0 - 1;
    synth_dx_row<1>(v, A + (size_t)(rp0 - 1) * kPlaneRowPair, gxr, ex, th, t, wt, tw);
    synth_plain_rows(v, B + (size_t)(rp0 - 1) * kPlaneRowPair, ex, th, t, wt, tw);
    __syncthreads();
    const float* gyrow = gyr + kN;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j0 = 4 * (th + kT * c);
      const size_t ro = (size_t)ia * kN + j0;
      const float4 sx = ld4g(sin_ + ro), sy = ld4g(sin_ + NN + ro), px = ld4g(pin + ro), py = ld4g(pin + NN + ro);
      const float sxa[4] = {sx.x, sx.y, sx.z, sx.w}, sya[4] = {sy.x, sy.y, sy.z, sy.w};
      const float pxa[4] = {px.x, px.y, px.z, px.w}, pya[4] = {py.x, py.y, py.z, py.w};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const bool xr = j0 + q < kN - 1;
        const float mx = xr ? sxa[q] + gxr[j0 + q] : 0.f, my = sya[q] + gyrow[j0 + q];
        float p1x, p1y;
        proj2(pxa[q] + P.sigma * mx, pya[q] + P.sigma * my, p1x, p1y);
        syu[j0 + q] = my - P.tau * (2.f * p1y - pya[q]);  // row ia < N - 1
      }
    }
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c)
#pragma unroll
      for (int q = 0; q < 4; ++q) syu[4 * (th + kT * c) + q] = 0.f;
  }
#pragma unroll 1
  for (int rp = rp0; rp < rp1; ++rp) {
    const int i0 = 2 * rp;
    if (th == 0 && rp + 1 < rp1) {
      prefetch_l2(A + (size_t)(rp + 1) * kPlaneRowPair, (uint32_t)(kPlaneRowPair * 4));
      prefetch_l2(B + (size_t)(rp + 1) * kPlaneRowPair, (uint32_t)(kPlaneRowPair * 4));
    }
    __syncthreads();
    const float* Ab = A + (size_t)rp * kPlaneRowPair;
    synth_dx_row<0>(v, Ab, gxr, ex, th, t, wt, tw);
    synth_dx_row<1>(v, Ab, gxr + kN, ex, th, t, wt, tw);
    synth_plain_rows(v, B + (size_t)rp * kPlaneRowPair, ex, th, t, wt, tw);
    __syncthreads();
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
      const int i = i0 + s;
      const bool yd = i < kN - 1, yu = i > 0;
      const float* gxrow = gxr + s * kN;
      const float* gyrow = gyr + s * kN;
      float dv[4][4];
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int j0 = 4 * (th + kT * c);
        const size_t ro = (size_t)i * kN + j0;
        float gxv[5], gyv[5], sxv[5], syv[5], pxv[5], pyv[5];
        {
          const float4 a = *reinterpret_cast<const float4*>(gxrow + j0);
          const float4 b = *reinterpret_cast<const float4*>(gyrow + j0);
          const float4 sx = ld4g(sin_ + ro), sy = ld4g(sin_ + NN + ro), px = ld4g(pin + ro),
                       py = ld4g(pin + NN + ro);
          gxv[1] = a.x; gxv[2] = a.y; gxv[3] = a.z; gxv[4] = a.w;
          gyv[1] = b.x; gyv[2] = b.y; gyv[3] = b.z; gyv[4] = b.w;
          sxv[1] = sx.x; sxv[2] = sx.y; sxv[3] = sx.z; sxv[4] = sx.w;
          syv[1] = sy.x; syv[2] = sy.y; syv[3] = sy.z; syv[4] = sy.w;
          pxv[1] = px.x; pxv[2] = px.y; pxv[3] = px.z; pxv[4] = px.w;
          pyv[1] = py.x; pyv[2] = py.y; pyv[3] = py.z; pyv[4] = py.w;
          if (j0 > 0) {
            gxv[0] = gxrow[j0 - 1]; gyv[0] = gyrow[j0 - 1];
            sxv[0] = __ldg(sin_ + ro - 1); syv[0] = __ldg(sin_ + NN + ro - 1);
            pxv[0] = __ldg(pin + ro - 1); pyv[0] = __ldg(pin + NN + ro - 1);
          } else {
            gxv[0] = gyv[0] = sxv[0] = syv[0] = pxv[0] = pyv[0] = 0.f;
          }
        }
        const float4 gq = ld4g(g + ro);
        const float gv[4] = {gq.x, gq.y, gq.z, gq.w};
        float p1x[5], p1y[5], snx[5], sny[5];
#pragma unroll
        for (int q = 0; q <= 4; ++q) {
          const int j = j0 - 1 + q;
          const bool xr = j < kN - 1;
          const float mx = xr ? sxv[q] + gxv[q] : 0.f, my = yd ? syv[q] + gyv[q] : 0.f;
          proj2(pxv[q] + P.sigma * mx, pyv[q] + P.sigma * my, p1x[q], p1y[q]);
          if (!xr) p1x[q] = 0.f;
          if (!yd) p1y[q] = 0.f;
          snx[q] = xr ? mx - P.tau * (2.f * p1x[q] - pxv[q]) : 0.f;
          sny[q] = yd ? my - P.tau * (2.f * p1y[q] - pyv[q]) : 0.f;
        }
#pragma unroll
        for (int q = 1; q <= 4; ++q) {
          const int j = j0 + q - 1;
          const bool xl = j > 0;
          const float divs = (snx[q] - (xl ? snx[q - 1] : 0.f) + sny[q] - (yu ? syu[j] : 0.f)) * P.invh;
          dv[c][q - 1] = gv[q - 1] - divs;
          syu[j] = sny[q];
        }
        st4g(sout + ro, snx[1], snx[2], snx[3], snx[4]);
        st4g(sout + NN + ro, sny[1], sny[2], sny[3], sny[4]);
        st4g(pout + ro, p1x[1], p1x[2], p1x[3], p1x[4]);
        st4g(pout + NN + ro, p1y[1], p1y[2], p1y[3], p1y[4]);
      }
      __syncthreads();
      float* rrow = gxr + s * kN;
#pragma unroll
      for (int c = 0; c < 4; ++c)
        *reinterpret_cast<float4*>(rrow + 4 * (th + kT * c)) = make_float4(dv[c][0], dv[c][1], dv[c][2], dv[c][3]);
    }
    __syncthreads();
    forward_rows_out(v, gxr, out + (size_t)rp * kPlaneRowPair, ex, th, t, wt, tw);
  }
}

int persistent_grid(int per_sm, int cap) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 148;
  }
  return std::min(cap, per_sm * std::max(sms, 1));
}

}  // namespace

bool grad4k_supported(const DctPlan& p) { return p.N == kN && p.fft && p.err; }

cudaError_t rows_fwd_4k(const DctPlan& p, const float* in, float* out, cudaStream_t st) {
  if (p.N != kN) return cudaErrorNotSupported;
  const size_t sm = kExBytes + (size_t)kN * 8;
  cudaError_t e = cudaFuncSetAttribute(k_rows_fwd_4k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_rows_fwd_4k<<<kPairs, kT, sm, st>>>(in, out, p.tw, p.wq);
  return cudaGetLastError();
}

cudaError_t grad_cols_4k(const DctPlan& p, const float* in, float* A, float* B, float alpha, float scale,
                         cudaStream_t st) {
  if (!grad4k_supported(p)) return cudaErrorNotSupported;
  CUtensorMap tm_in, tm_a, tm_b;
  if (!encode_pairs_map(&tm_in, in, kN) || !encode_pairs_map(&tm_a, A, kN) || !encode_pairs_map(&tm_b, B, kN))
    return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(k_cols_grad_4k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kColsSmem);
  if (e != cudaSuccess) return e;
  const float sN2 = (float)((double)scale / ((double)kN * (double)kN));
  k_cols_grad_4k<<<kN / 2, kT, kColsSmem, st>>>(tm_in, tm_a, tm_b, p.tw, p.wq, p.mu, alpha, sN2, p.err);
  return cudaGetLastError();
}

cudaError_t grad_rows_4k(const DctPlan& p, const float* A, const float* B, float* gx, float* gy, float* phi,
                         cudaStream_t st) {
  if (p.N != kN) return cudaErrorNotSupported;
  k_rows_grad_4k<<<persistent_grid(2, kPairs), kT, 0, st>>>(A, B, gx, gy, phi, p.tw, p.wq);
  return cudaGetLastError();
}

cudaError_t rof_rows_step_4k(const DctPlan& p, const float* A, const float* B, const float* pin, const float* I,
                             float* pout, float* out, const RofParams& P, cudaStream_t st) {
  if (p.N != kN || P.N != kN) return cudaErrorNotSupported;
  cudaError_t e =
      cudaFuncSetAttribute(k_rof_rows_step_4k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStepSmem);
  if (e != cudaSuccess) return e;
  k_rof_rows_step_4k<<<persistent_grid(2, kPairs), kT, kStepSmem, st>>>(A, B, pin, I, pout, out, p.tw, p.wq, P);
  return cudaGetLastError();
}

cudaError_t emd_rows_step_4k(const DctPlan& p, const float* A, const float* B, const float* sin_, const float* pin,
                             const float* g, float* sout, float* pout, float* out, const EmdParams& P,
                             cudaStream_t st) {
  if (p.N != kN || P.N != kN) return cudaErrorNotSupported;
  cudaError_t e =
      cudaFuncSetAttribute(k_emd_rows_step_4k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kStepSmem);
  if (e != cudaSuccess) return e;
  k_emd_rows_step_4k<<<persistent_grid(2, kPairs), kT, kStepSmem, st>>>(A, B, sin_, pin, g, sout, pout, out, p.tw,
                                                                         p.wq, P);
  return cudaGetLastError();
}

}  // namespace gp
