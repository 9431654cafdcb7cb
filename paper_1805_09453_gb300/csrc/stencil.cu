// Pointwise / stencil part of one G-prox PDHG iteration, fused per problem,
// and the FP64 objective / gap reductions.
//
// Discretisation (shared with the cosine solve): forward-difference grad with
// zero last slots, div = -grad^T, Lap = div grad, h = 1/N.
//
// ROF (section 3.1).  Given u_{n+1} (output of the solve) and p_n:
//     p_{n+1} = proj(p_n + sigma grad u_{n+1}),  pbar = 2 p_{n+1} - p_n,
//     r_{n+1} = lambda tau I + tau div pbar - Lap u_{n+1}
// (the right-hand side of the next u-step), one HBM pass: read u, p, I,
// write p', r.
//
// EMD (section 3.2) in the variables s_n = m_n - tau pbar_n and d_n = div pbar_n.
// Given q_n = Lap^{-1} d_n (output of the solve):
//     m_{n+1} = m_n - tau (pbar_n - grad q_n) = s_n + tau grad q_n
//     p_{n+1} = proj(p_n + sigma m_{n+1}),  pbar_{n+1} = 2 p_{n+1} - p_n
//     s_{n+1} = m_{n+1} - tau pbar_{n+1},    d_{n+1} = div pbar_{n+1}
// one HBM pass: read q, s, p, write s', p', d.  This is the Leray-projected
// update of the paper algebraically rearranged so that pbar never has to be
// stored; m is written only on gap-check iterations.
//
// Thread layout: a thread owns V consecutive cells of a row (V = 4 with
// 128-bit loads when N % 4 == 0 and pointers are 16-byte aligned, else 1)
// and walks RB rows down, carrying the previous row's values in registers;
// the left neighbour column and the row above the strip are recomputed.
#include "gp_internal.cuh"
#include "stencil.cuh"

namespace gp {
namespace {

template <int V>
__device__ __forceinline__ void ldv(float* d, const float* __restrict__ p) {
  if constexpr (V == 4) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    d[0] = t.x; d[1] = t.y; d[2] = t.z; d[3] = t.w;
  } else {
#pragma unroll
    for (int c = 0; c < V; ++c) d[c] = p[c];
  }
}

template <int V>
__device__ __forceinline__ void stv(float* __restrict__ p, const float* s) {
  if constexpr (V == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(s[0], s[1], s[2], s[3]);
  } else {
#pragma unroll
    for (int c = 0; c < V; ++c) p[c] = s[c];
  }
}

// Row window: w[0] = col j0-1, w[1..V] = cols j0..j0+V-1, w[V+1] = col j0+V
// (out-of-grid entries are 0 and never used).
template <int V>
__device__ __forceinline__ void load_row(float (&w)[V + 2], const float* __restrict__ base, int row, int N,
                                         int j0) {
  if (row < 0 || row >= N) {
#pragma unroll
    for (int c = 0; c < V + 2; ++c) w[c] = 0.f;
    return;
  }
  const float* r = base + (size_t)row * N;
  ldv<V>(&w[1], r + j0);
  w[0] = j0 > 0 ? r[j0 - 1] : 0.f;
  w[V + 1] = j0 + V < N ? r[j0 + V] : 0.f;
}

// Block reduction of NQ doubles; op bit q set = max, else sum.  Thread 0 writes
// the block's partials to part[block * NQ + q].
template <int NQ>
__device__ __forceinline__ void block_reduce_store(double (&v)[NQ], unsigned maxmask, double* __restrict__ part) {
  __shared__ double sh[32][NQ];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nthreads = blockDim.x * blockDim.y;
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  (void)nthreads;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double x = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_down_sync(0xffffffffu, x, o);
      x = ((maxmask >> q) & 1u) ? fmax(x, y) : x + y;
    }
    v[q] = x;
  }
  const int w = tid >> 5;
  (void)warp;
  if ((tid & 31) == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[w][q] = v[q];
  }
  __syncthreads();
  if (tid < 32) {
    const int nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double x = lane < nw ? sh[lane][q] : (((maxmask >> q) & 1u) ? -1e300 : 0.0);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double y = __shfl_down_sync(0xffffffffu, x, o);
        x = ((maxmask >> q) & 1u) ? fmax(x, y) : x + y;
      }
      if (lane == 0) part[(size_t)(blockIdx.y * gridDim.x + blockIdx.x) * NQ + q] = x;
    }
  }
}

// ------------------------------------------------------------------ ROF
// Given grad u_{n+1} (spectral gradient of the solve: two planes, zero slots)
// and p_n:  p_{n+1} = proj(p_n + sigma grad u_{n+1}), pbar = 2 p_{n+1} - p_n,
//           r_{n+1} = lambda tau I + tau div pbar - div grad u_{n+1}.
// GAP steps also read u_{n+1} for the fidelity term of the objective.
template <int V, int RB, bool GAP>
__global__ void __launch_bounds__(128) k_rof_fused(const float* __restrict__ gu, const float* __restrict__ u,
                                                   const float* __restrict__ pin, const float* __restrict__ I,
                                                   float* __restrict__ pout, float* __restrict__ r,
                                                   double* __restrict__ part, RofParams P) {
  const int N = P.N;
  const size_t NN = (size_t)N * N;
  const int j0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  const int i0 = blockIdx.y * RB;
  CSum s_tv, s_fid, s_id, s_dd;
  if (j0 < N) {
    const float* __restrict__ gux = gu;
    const float* __restrict__ guy = gu + NN;
    const float* __restrict__ pxin = pin;
    const float* __restrict__ pyin = pin + NN;
    float pby_up[V], p1y_up[V], gy_up[V];  // row above: pbar_y, p_{n+1,y}, (grad u)_y
    if (i0 > 0) {
      const size_t ro = (size_t)(i0 - 1) * N;
      float gxv[V], gyv[V], pnx[V], pny[V];
      ldv<V>(gxv, gux + ro + j0);
      ldv<V>(gyv, guy + ro + j0);
      ldv<V>(pnx, pxin + ro + j0);
      ldv<V>(pny, pyin + ro + j0);
#pragma unroll
      for (int c = 0; c < V; ++c) {
        float px1, py1;
        proj2(pnx[c] + P.sigma * gxv[c], pny[c] + P.sigma * gyv[c], px1, py1);
        pby_up[c] = 2.f * py1 - pny[c];
        p1y_up[c] = py1;
        gy_up[c] = gyv[c];
      }
    } else {
#pragma unroll
      for (int c = 0; c < V; ++c) { pby_up[c] = 0.f; p1y_up[c] = 0.f; gy_up[c] = 0.f; }
    }
    const int iend = min(i0 + RB, N);
    for (int i = i0; i < iend; ++i) {
      const size_t ro = (size_t)i * N;
      float gxv[V + 1], gyv[V + 1], pnx[V + 1], pny[V + 1];
      ldv<V>(&gxv[1], gux + ro + j0);
      ldv<V>(&gyv[1], guy + ro + j0);
      ldv<V>(&pnx[1], pxin + ro + j0);
      ldv<V>(&pny[1], pyin + ro + j0);
      if (j0 > 0) {
        gxv[0] = gux[ro + j0 - 1]; gyv[0] = guy[ro + j0 - 1];
        pnx[0] = pxin[ro + j0 - 1]; pny[0] = pyin[ro + j0 - 1];
      } else {
        gxv[0] = gyv[0] = pnx[0] = pny[0] = 0.f;
      }
      float Iv[V], uv[V];
      ldv<V>(Iv, I + ro + j0);
      if constexpr (GAP) ldv<V>(uv, u + ro + j0);
      float p1x[V + 1], p1y[V + 1], pbx[V + 1], pby[V + 1];
#pragma unroll
      for (int c = 0; c <= V; ++c) {
        const int j = j0 - 1 + c;
        const bool xr = j < N - 1, yd = i < N - 1;
        proj2(pnx[c] + P.sigma * gxv[c], pny[c] + P.sigma * gyv[c], p1x[c], p1y[c]);
        if (!xr) p1x[c] = 0.f;
        if (!yd) p1y[c] = 0.f;
        pbx[c] = 2.f * p1x[c] - (xr ? pnx[c] : 0.f);
        pby[c] = 2.f * p1y[c] - (yd ? pny[c] : 0.f);
      }
      float rv[V];
#pragma unroll
      for (int c = 1; c <= V; ++c) {
        const int j = j0 + c - 1;
        const bool xl = j > 0, yu = i > 0;
        const float dpb = (pbx[c] - (xl ? pbx[c - 1] : 0.f) + pby[c] - (yu ? pby_up[c - 1] : 0.f)) * P.invh;
        const float lap = (gxv[c] - (xl ? gxv[c - 1] : 0.f) + gyv[c] - (yu ? gy_up[c - 1] : 0.f)) * P.invh;
        rv[c - 1] = P.lt * Iv[c - 1] + P.tau * dpb - lap;
        if constexpr (GAP) {
          s_tv.add(sqrtf(gxv[c] * gxv[c] + gyv[c] * gyv[c]));
          const float e = uv[c - 1] - Iv[c - 1];
          s_fid.add(e * e);
          const float d1 = (p1x[c] - (xl ? p1x[c - 1] : 0.f) + p1y[c] - (yu ? p1y_up[c - 1] : 0.f)) * P.invh;
          s_id.add(Iv[c - 1] * d1);
          s_dd.add(d1 * d1);
        }
      }
      stv<V>(pout + ro + j0, &p1x[1]);
      stv<V>(pout + NN + ro + j0, &p1y[1]);
      stv<V>(r + ro + j0, rv);
#pragma unroll
      for (int c = 0; c < V; ++c) {
        pby_up[c] = pby[c + 1];
        p1y_up[c] = p1y[c + 1];
        gy_up[c] = gyv[c + 1];
      }
    }
  }
  if constexpr (GAP) {
    double v[4] = {s_tv.value(), s_fid.value(), s_id.value(), s_dd.value()};
    block_reduce_store<4>(v, 0u, part);
  }
}

// ------------------------------------------------------------------ EMD
// Affine form of the Leray step: with g = f0 - f1 and s_n = m_n - tau pbar_n,
//     q_n = Lap^{-1} (g - div s_n),   m_{n+1} = s_n + grad q_n.
// For a feasible m_n (div m_n = g) this is m_n - tau (pbar_n - grad Lap^{-1} div pbar_n),
// the update of section 3.2; in floating point it re-imposes div m = g at
// every step instead of carrying each step's solve error forward.  grad q_n
// comes from the spectral gradient of the cosine solve (two planes, zero slots).
template <int V, int RB, bool GAP>
__global__ void __launch_bounds__(128) k_emd_fused(const float* __restrict__ gq, const float* __restrict__ sin_,
                                                   const float* __restrict__ pin, const float* __restrict__ g,
                                                   float* __restrict__ sout, float* __restrict__ pout,
                                                   float* __restrict__ d, float* __restrict__ m,
                                                   float* __restrict__ e, double* __restrict__ part, EmdParams P) {
  const int N = P.N;
  const size_t NN = (size_t)N * N;
  const int j0 = (blockIdx.x * blockDim.x + threadIdx.x) * V;
  const int i0 = blockIdx.y * RB;
  CSum s_m, s_mass;
  if (j0 < N) {
    const float* __restrict__ gqx = gq;
    const float* __restrict__ gqy = gq + NN;
    const float* __restrict__ sx = sin_;
    const float* __restrict__ sy = sin_ + NN;
    const float* __restrict__ px = pin;
    const float* __restrict__ py = pin + NN;
    float sy_up[V], p1y_up[V], my_up[V];  // row above: new s_y, new p_y, m_y
    if (i0 > 0) {
      const size_t ro = (size_t)(i0 - 1) * N;
      float gxv[V], gyv[V], sxv[V], syv[V], pxv[V], pyv[V];
      ldv<V>(gxv, gqx + ro + j0);
      ldv<V>(gyv, gqy + ro + j0);
      ldv<V>(sxv, sx + ro + j0);
      ldv<V>(syv, sy + ro + j0);
      ldv<V>(pxv, px + ro + j0);
      ldv<V>(pyv, py + ro + j0);
#pragma unroll
      for (int c = 0; c < V; ++c) {
        const bool xr = j0 + c < N - 1;
        const float mx = xr ? sxv[c] + gxv[c] : 0.f, my = syv[c] + gyv[c];
        float p1x, p1y;
        proj2(pxv[c] + P.sigma * mx, pyv[c] + P.sigma * my, p1x, p1y);
        sy_up[c] = my - P.tau * (2.f * p1y - pyv[c]);
        p1y_up[c] = p1y;
        my_up[c] = my;
      }
    } else {
#pragma unroll
      for (int c = 0; c < V; ++c) { sy_up[c] = 0.f; p1y_up[c] = 0.f; my_up[c] = 0.f; }
    }
    const int iend = min(i0 + RB, N);
    for (int i = i0; i < iend; ++i) {
      const size_t ro = (size_t)i * N;
      float gxv[V + 1], gyv[V + 1], sxv[V + 1], syv[V + 1], pxv[V + 1], pyv[V + 1];
      ldv<V>(&gxv[1], gqx + ro + j0);
      ldv<V>(&gyv[1], gqy + ro + j0);
      ldv<V>(&sxv[1], sx + ro + j0);
      ldv<V>(&syv[1], sy + ro + j0);
      ldv<V>(&pxv[1], px + ro + j0);
      ldv<V>(&pyv[1], py + ro + j0);
      if (j0 > 0) {
        gxv[0] = gqx[ro + j0 - 1]; gyv[0] = gqy[ro + j0 - 1];
        sxv[0] = sx[ro + j0 - 1]; syv[0] = sy[ro + j0 - 1];
        pxv[0] = px[ro + j0 - 1]; pyv[0] = py[ro + j0 - 1];
      } else {
        gxv[0] = gyv[0] = sxv[0] = syv[0] = pxv[0] = pyv[0] = 0.f;
      }
      float gv[V];
      ldv<V>(gv, g + ro + j0);
      float mxv[V + 1], myv[V + 1], p1x[V + 1], p1y[V + 1], snx[V + 1], sny[V + 1];
#pragma unroll
      for (int c = 0; c <= V; ++c) {
        const int j = j0 - 1 + c;
        const bool xr = j < N - 1, yd = i < N - 1;
        mxv[c] = xr ? sxv[c] + gxv[c] : 0.f;
        myv[c] = yd ? syv[c] + gyv[c] : 0.f;
        proj2(pxv[c] + P.sigma * mxv[c], pyv[c] + P.sigma * myv[c], p1x[c], p1y[c]);
        if (!xr) p1x[c] = 0.f;
        if (!yd) p1y[c] = 0.f;
        snx[c] = xr ? mxv[c] - P.tau * (2.f * p1x[c] - pxv[c]) : 0.f;
        sny[c] = yd ? myv[c] - P.tau * (2.f * p1y[c] - pyv[c]) : 0.f;
      }
      float od[V], omx[V], omy[V], oe[V];
#pragma unroll
      for (int c = 1; c <= V; ++c) {
        const int j = j0 + c - 1;
        const bool xl = j > 0, yu = i > 0;
        const float divs = (snx[c] - (xl ? snx[c - 1] : 0.f) + sny[c] - (yu ? sy_up[c - 1] : 0.f)) * P.invh;
        od[c - 1] = gv[c - 1] - divs;
        if constexpr (GAP) {
          const float mx = mxv[c], my = myv[c];
          omx[c - 1] = mx;
          omy[c - 1] = my;
          oe[c - 1] = -(p1x[c] - (xl ? p1x[c - 1] : 0.f) + p1y[c] - (yu ? p1y_up[c - 1] : 0.f)) * P.invh;
          s_m.add(sqrtf(mx * mx + my * my));
          const float dm = (mx - (xl ? mxv[c - 1] : 0.f) + my - (yu ? my_up[c - 1] : 0.f)) * P.invh;
          s_mass.add(fabsf(dm - gv[c - 1]));
        }
      }
      stv<V>(sout + ro + j0, &snx[1]);
      stv<V>(sout + NN + ro + j0, &sny[1]);
      stv<V>(pout + ro + j0, &p1x[1]);
      stv<V>(pout + NN + ro + j0, &p1y[1]);
      stv<V>(d + ro + j0, od);
      if constexpr (GAP) {
        stv<V>(m + ro + j0, omx);
        stv<V>(m + NN + ro + j0, omy);
        stv<V>(e + ro + j0, oe);
      }
#pragma unroll
      for (int c = 0; c < V; ++c) {
        sy_up[c] = sny[c + 1];
        p1y_up[c] = p1y[c + 1];
        my_up[c] = myv[c + 1];
      }
    }
  }
  if constexpr (GAP) {
    double v[2] = {s_m.value(), s_mass.value()};
    block_reduce_store<2>(v, 0u, part);
  }
}

// Double-FP32 arithmetic for the dual bound's per-point work: a value is a
// pair hi + lo (|lo| <= ulp(hi) / 2, about 48 significant bits) built from
// the error-free transformations (Knuth's TwoSum and the FMA form of
// TwoProduct), with the intrinsics' explicit rounding so that no addition
// or product is contracted or reassociated.  GB300's FP64 rate is a small
// fraction of its FP32 rate, and FP64 per grid point made the EMD gap check
// cost more than an iteration.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DF df_fast(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DF df_add(DF x, DF y) {
  const DF s = df_two_sum(x.hi, y.hi);
  return df_fast(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}
__device__ __forceinline__ DF df_mul(DF x, float b) {  // x * b
  const float p = __fmul_rn(x.hi, b);
  return df_fast(p, __fmaf_rn(x.lo, b, __fmaf_rn(x.hi, b, -p)));
}
__device__ __forceinline__ DF df_sq(DF x) {  // x * x
  const float p = __fmul_rn(x.hi, x.hi);
  return df_fast(p, __fmaf_rn(__fmul_rn(2.f, x.hi), x.lo, __fmaf_rn(x.hi, x.hi, -p)));
}

// Residual of the dual potential's equation (0 - Lap) phi = -div p, to about
// 48 bits from the stored FP32 arrays: r = -div p + Lap phi with div p by
// forward differences with zero last slots and Lap the 5-point Neumann
// stencil (h = 1/N), i.e. r = N (N l - d) with l = sum (phi_nb - phi) over
// the neighbours and d = (px - px_left) + (py - py_up).  Neighbouring
// differences are exact pairs, the sums are pair sums, and r is rounded once.
// Taking div p here (not from an FP32 plane of it) makes phi_hi + phi_lo the
// potential of the p given, to the second solve's accuracy.
__global__ void __launch_bounds__(256) k_dual_residual(const float* __restrict__ p, const float* __restrict__ phi,
                                                       float* __restrict__ r, int N) {
  const size_t NN = (size_t)N * N;
  const float n = (float)N;  // exact for N <= 2^24
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const unsigned row = (unsigned)(idx / (unsigned)N), col = (unsigned)(idx % (unsigned)N);
    const bool xr = col + 1 < (unsigned)N, xl = col > 0, yd = row + 1 < (unsigned)N, yu = row > 0;
    const DF dv = df_add(df_two_sum(xr ? p[idx] : 0.f, -(xl ? p[idx - 1] : 0.f)),
                         df_two_sum(yd ? p[NN + idx] : 0.f, -(yu ? p[NN + idx - N] : 0.f)));
    const float c = phi[idx];
    DF lap = {0.f, 0.f};
    if (xl) lap = df_add(lap, df_two_sum(phi[idx - 1], -c));
    if (xr) lap = df_add(lap, df_two_sum(phi[idx + 1], -c));
    if (yu) lap = df_add(lap, df_two_sum(phi[idx - N], -c));
    if (yd) lap = df_add(lap, df_two_sum(phi[idx + N], -c));
    const DF t = df_add(df_mul(lap, n), {-dv.hi, -dv.lo});
    const DF rr = df_mul(t, n);
    r[idx] = __fadd_rn(rr.hi, rr.lo);
  }
}

// EMD dual bound inputs for a potential held as two FP32 planes,
// phi = hi + lo: sum phi (f1 - f0) and max |D phi|^2 (forward differences,
// h = 1/N, zero last slots), both in pair arithmetic: the neighbouring
// differences of each plane are exact pairs and the squares and sums keep
// about 48 bits, so the maximum is within ~1e-13 relative and is raised by
// 2^-40 to bound it from above.  Both inputs of the bound are then exact,
// or an upper bound, for the phi the planes represent, and weak duality
// holds for the bound as computed.
__global__ void __launch_bounds__(256) k_emd_dual_hilo(const float* __restrict__ hi, const float* __restrict__ lo,
                                                       const float* __restrict__ f0, const float* __restrict__ f1,
                                                       int N, double* __restrict__ part) {
  DF sum = {0.f, 0.f}, g2m = {0.f, 0.f};
  const size_t NN = (size_t)N * N;
  const float n = (float)N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const unsigned row = (unsigned)(idx / (unsigned)N), col = (unsigned)(idx % (unsigned)N);
    const float h0 = hi[idx], l0 = lo[idx];
    const DF t = df_two_sum(f1[idx], -f0[idx]);
    const float pr = __fmul_rn(h0, t.hi);
    const float pe = __fmaf_rn(h0, t.lo, __fmaf_rn(l0, t.hi, __fmaf_rn(h0, t.hi, -pr)));
    sum = df_add(sum, df_fast(pr, pe));
    DF gx = {0.f, 0.f}, gy = {0.f, 0.f};
    if (col + 1 < (unsigned)N)
      gx = df_mul(df_add(df_two_sum(hi[idx + 1], -h0), df_two_sum(lo[idx + 1], -l0)), n);
    if (row + 1 < (unsigned)N)
      gy = df_mul(df_add(df_two_sum(hi[idx + N], -h0), df_two_sum(lo[idx + N], -l0)), n);
    const DF g2 = df_add(df_sq(gx), df_sq(gy));
    if (g2.hi > g2m.hi || (g2.hi == g2m.hi && g2.lo > g2m.lo)) g2m = g2;
  }
  double v[2] = {(double)sum.hi + (double)sum.lo, sqrt((double)g2m.hi + (double)g2m.lo) * (1.0 + 0x1p-40)};
  block_reduce_store<2>(v, 2u, part);
}

// ROF step-rule statistics: sum |grad I|, sum |grad I|^2, sum I.
__global__ void __launch_bounds__(256) k_rof_stats(const float* __restrict__ I, int N, float invh,
                                                   double* __restrict__ part) {
  CSum a, b, c;
  const size_t NN = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    const float v = I[idx];
    const float gx = j < N - 1 ? (I[idx + 1] - v) * invh : 0.f;
    const float gy = i < N - 1 ? (I[idx + N] - v) * invh : 0.f;
    const float g2 = gx * gx + gy * gy;
    a.add(sqrtf(g2));
    b.add(g2);
    c.add(v);
  }
  double v[3] = {a.value(), b.value(), c.value()};
  block_reduce_store<3>(v, 0u, part);
}

__global__ void __launch_bounds__(256) k_sq_dev(const float* __restrict__ I, size_t NN, float mean,
                                                double* __restrict__ part) {
  CSum a;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const float e = I[idx] - mean;
    a.add(e * e);
  }
  double v[1] = {a.value()};
  block_reduce_store<1>(v, 0u, part);
}

// Sum (or max) of per-block partials in a fixed order: deterministic.
__global__ void __launch_bounds__(256) k_final_reduce(const double* __restrict__ part, int nblk, int nq,
                                                      unsigned maxmask, double* __restrict__ out) {
  __shared__ double sh[256];
  for (int q = 0; q < nq; ++q) {
    const bool mx = (maxmask >> q) & 1u;
    double acc = mx ? -1e300 : 0.0;
    for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
      const double x = part[(size_t)b * nq + q];
      acc = mx ? fmax(acc, x) : acc + x;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
      if (threadIdx.x < s) sh[threadIdx.x] = mx ? fmax(sh[threadIdx.x], sh[threadIdx.x + s]) : sh[threadIdx.x] + sh[threadIdx.x + s];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[q] = sh[0];
    __syncthreads();
  }
}

// ROF state set-up: r = lambda tau I + tau div pbar - Lap u; zero the p slots.
__global__ void k_rof_init(const float* __restrict__ I, const float* __restrict__ u, const float* __restrict__ pbar,
                           float* __restrict__ p, float* __restrict__ r, RofParams P) {
  const int N = P.N;
  const size_t NN = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    const bool xr = j < N - 1, xl = j > 0, yd = i < N - 1, yu = i > 0;
    const float dx = (xr ? pbar[idx] : 0.f) - (xl ? pbar[idx - 1] : 0.f);
    const float dy = (yd ? pbar[NN + idx] : 0.f) - (yu ? pbar[NN + idx - N] : 0.f);
    const float uo = u[idx];
    float lap = 0.f;
    if (xr) lap += u[idx + 1] - uo;
    if (xl) lap += u[idx - 1] - uo;
    if (yd) lap += u[idx + N] - uo;
    if (yu) lap += u[idx - N] - uo;
    r[idx] = P.lt * I[idx] + P.tau * (dx + dy) * P.invh - lap * P.invh2;
    if (!xr) p[idx] = 0.f;
    if (!yd) p[NN + idx] = 0.f;
  }
}

// EMD state set-up: s = m0 - tau pbar0 (slots 0); zero the p slots.
__global__ void k_emd_init(const float* __restrict__ m0, const float* __restrict__ pbar, float* __restrict__ p,
                           float* __restrict__ s, EmdParams P) {
  const int N = P.N;
  const size_t NN = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    const bool xr = j < N - 1, yd = i < N - 1;
    s[idx] = xr ? m0[idx] - P.tau * pbar[idx] : 0.f;
    s[NN + idx] = yd ? m0[NN + idx] - P.tau * pbar[NN + idx] : 0.f;
    if (!xr) p[idx] = 0.f;
    if (!yd) p[NN + idx] = 0.f;
  }
}

// d = g - div s (right-hand side of the affine Leray step)
__global__ void k_affine_rhs(const float* __restrict__ s, const float* __restrict__ g, float* __restrict__ d, int N,
                             float invh) {
  const size_t NN = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    const bool xr = j < N - 1, xl = j > 0, yd = i < N - 1, yu = i > 0;
    const float dv = ((xr ? s[idx] : 0.f) - (xl ? s[idx - 1] : 0.f) + (yd ? s[NN + idx] : 0.f) -
                      (yu ? s[NN + idx - N] : 0.f)) * invh;
    d[idx] = g[idx] - dv;
  }
}

// out = a - b
__global__ void k_sub(const float* __restrict__ a, const float* __restrict__ b, float* __restrict__ out, size_t n) {
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x)
    out[idx] = a[idx] - b[idx];
}

// g = grad x (two planes, zero slots)
__global__ void k_grad(const float* __restrict__ x, float* __restrict__ g, int N, float invh) {
  const size_t NN = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    g[idx] = j < N - 1 ? (x[idx + 1] - x[idx]) * invh : 0.f;
    g[NN + idx] = i < N - 1 ? (x[idx + N] - x[idx]) * invh : 0.f;
  }
}

// Copy a vector field (x plane, y plane), zeroing its structural slots.
__global__ void k_copy_field(const float* __restrict__ a, float* __restrict__ b, int N) {
  const size_t NN = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    b[idx] = j < N - 1 ? a[idx] : 0.f;
    b[NN + idx] = i < N - 1 ? a[NN + idx] : 0.f;
  }
}

// Generic (unfused) ROF gap terms of (u, p): sum |grad u|, sum (u - I)^2,
// sum I div p, sum (div p)^2.
__global__ void __launch_bounds__(256) k_rof_gap(const float* __restrict__ u, const float* __restrict__ p,
                                                 const float* __restrict__ I, int N, float invh,
                                                 double* __restrict__ part) {
  CSum a, b, c, e;
  const size_t NN = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    const bool xr = j < N - 1, xl = j > 0, yd = i < N - 1, yu = i > 0;
    const float uo = u[idx];
    const float gx = xr ? (u[idx + 1] - uo) * invh : 0.f;
    const float gy = yd ? (u[idx + N] - uo) * invh : 0.f;
    a.add(sqrtf(gx * gx + gy * gy));
    const float r = uo - I[idx];
    b.add(r * r);
    const float dv = ((xr ? p[idx] : 0.f) - (xl ? p[idx - 1] : 0.f) + (yd ? p[NN + idx] : 0.f) -
                      (yu ? p[NN + idx - N] : 0.f)) * invh;
    c.add(I[idx] * dv);
    e.add(dv * dv);
  }
  double v[4] = {a.value(), b.value(), c.value(), e.value()};
  block_reduce_store<4>(v, 0u, part);
}

// Generic EMD primal terms of m: sum |m|, sum |div m - (f0 - f1)|; and
// e = -div p for the dual potential.
__global__ void __launch_bounds__(256) k_emd_primal(const float* __restrict__ m, const float* __restrict__ p,
                                                    const float* __restrict__ f0, const float* __restrict__ f1,
                                                    float* __restrict__ e, int N, float invh,
                                                    double* __restrict__ part) {
  CSum a, b;
  const size_t NN = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    const bool xr = j < N - 1, xl = j > 0, yd = i < N - 1, yu = i > 0;
    const float mx = xr ? m[idx] : 0.f, my = yd ? m[NN + idx] : 0.f;
    a.add(sqrtf(mx * mx + my * my));
    const float dm = (mx - (xl ? m[idx - 1] : 0.f) + my - (yu ? m[NN + idx - N] : 0.f)) * invh;
    b.add(fabsf(dm - (f0[idx] - f1[idx])));
    e[idx] = -((xr ? p[idx] : 0.f) - (xl ? p[idx - 1] : 0.f) + (yd ? p[NN + idx] : 0.f) -
               (yu ? p[NN + idx - N] : 0.f)) * invh;
  }
  double v[2] = {a.value(), b.value()};
  block_reduce_store<2>(v, 0u, part);
}

// Feasibility certificate of an EMD flux (the constraint div m = f0 - f1 of
// section 3.2).  rho = (f0 - f1) - div m, evaluated in FP64 from the stored
// FP32 arrays (so it is the exact residual of the m a caller receives, not
// one blurred by FP32 cancellation in the divergence), is written as FP32 for
// the correcting solve; sum |rho| is reduced in FP64.
__global__ void __launch_bounds__(256) k_emd_residual64(const float* __restrict__ m, const float* __restrict__ f0,
                                                        const float* __restrict__ f1, float* __restrict__ rho,
                                                        int N, double invh, double* __restrict__ part) {
  double a = 0.0;
  const size_t NN = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    const double mx = j < N - 1 ? (double)m[idx] : 0.0, my = i < N - 1 ? (double)m[NN + idx] : 0.0;
    const double mxl = j > 0 ? (double)m[idx - 1] : 0.0, myu = i > 0 ? (double)m[NN + idx - N] : 0.0;
    const double r = ((double)f0[idx] - (double)f1[idx]) - ((mx - mxl) + (my - myu)) * invh;
    rho[idx] = (float)r;
    a += fabs(r);
  }
  double v[1] = {a};
  block_reduce_store<1>(v, 0u, part);
}

// The corrected flux m~ = m + grad c (grad c: two planes with zero slots, from
// the spectral gradient of c = Lap^{-1} rho): sum |m~| (FP32 terms, compensated
// sums: the objective has no 1/h amplification) and the residual left after
// the correction, sum |(f0 - f1) - div m~|, in FP64.
__global__ void __launch_bounds__(256) k_emd_corrected(const float* __restrict__ m, const float* __restrict__ gc,
                                                       const float* __restrict__ f0, const float* __restrict__ f1,
                                                       int N, double invh, double* __restrict__ part) {
  CSum a;
  double b = 0.0;
  const size_t NN = (size_t)N * N;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const int i = (int)(idx / N), j = (int)(idx % N);
    const bool xr = j < N - 1, yd = i < N - 1, xl = j > 0, yu = i > 0;
    const double mx = xr ? (double)m[idx] + (double)gc[idx] : 0.0;
    const double my = yd ? (double)m[NN + idx] + (double)gc[NN + idx] : 0.0;
    const double mxl = xl ? (double)m[idx - 1] + (double)gc[idx - 1] : 0.0;
    const double myu = yu ? (double)m[NN + idx - N] + (double)gc[NN + idx - N] : 0.0;
    const float fx = (float)mx, fy = (float)my;
    a.add(sqrtf(fx * fx + fy * fy));
    b += fabs(((double)f0[idx] - (double)f1[idx]) - ((mx - mxl) + (my - myu)) * invh);
  }
  double v[2] = {a.value(), b};
  block_reduce_store<2>(v, 0u, part);
}

// sum f0, sum f1, sum |f0 - f1|
__global__ void __launch_bounds__(256) k_mass_stats(const float* __restrict__ f0, const float* __restrict__ f1,
                                                    size_t NN, double* __restrict__ part) {
  CSum a, b, c;
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < NN; idx += (size_t)gridDim.x * blockDim.x) {
    const float x = f0[idx], y = f1[idx];
    a.add(x);
    b.add(y);
    c.add(fabsf(x - y));
  }
  double v[3] = {a.value(), b.value(), c.value()};
  block_reduce_store<3>(v, 0u, part);
}

inline int grid_1d(size_t n, int threads) {
  const size_t b = (n + threads - 1) / threads;
  return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

// Residual of the Helmholtz equation in FP64 from the stored FP32 solution:
// r = b - inv_scale (alpha x - Lap x), Lap the 5-point Neumann stencil
// (neighbours outside the grid omitted), h = 1/N.  The FP32 rounding of the
// result is relative to r itself, which is small when x is close.
__global__ void __launch_bounds__(256) k_helmholtz_residual(const float* __restrict__ b, const float* __restrict__ x,
                                                            float* __restrict__ r, int N, double alpha,
                                                            double inv_scale) {
  const size_t NN = (size_t)N * N;
  const double n2 = (double)N * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < NN; i += (size_t)gridDim.x * blockDim.x) {
    const int row = (int)(i / N), col = (int)(i % N);
    const double xc = x[i];
    double lap = 0.0;
    if (col > 0) lap += (double)x[i - 1] - xc;
    if (col < N - 1) lap += (double)x[i + 1] - xc;
    if (row > 0) lap += (double)x[i - N] - xc;
    if (row < N - 1) lap += (double)x[i + N] - xc;
    r[i] = (float)((double)b[i] - inv_scale * (alpha * xc - n2 * lap));
  }
}

// Mean removal on the device (no host round trip): sum x, then out = x - sum / n.
__global__ void __launch_bounds__(256) k_sum(const float* __restrict__ x, size_t n, double* __restrict__ part) {
  CSum a;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    a.add(x[i]);
  double v[1] = {a.value()};
  block_reduce_store<1>(v, 0u, part);
}
__global__ void __launch_bounds__(256) k_center(const float* __restrict__ x, float* __restrict__ out, size_t n,
                                                const double* __restrict__ sum) {
  const float mean = (float)(*sum / (double)n);
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = x[i] - mean;
}

// x += y
__global__ void __launch_bounds__(256) k_add_inplace(float* __restrict__ x, const float* __restrict__ y, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    x[i] += y[i];
}

// ------------------------------------------------------------------- 3-D
// The d = 3 instance of the updates above (Algorithm 2 for general d;
// sections 3.1 / 3.2): volumes (z, y, x), x fastest, n3 = N^3 points;
// vector fields are three consecutive volumes (x, y, z components) with
// structurally zero last slots; forward differences, div = -grad^T.
__device__ __forceinline__ void proj3(float qx, float qy, float qz, float& px, float& py, float& pz) {
  const float n2 = qx * qx + qy * qy + qz * qz;
  if (n2 > 1.f) {
    const float s = rsqrtf(n2);
    px = qx * s;
    py = qy * s;
    pz = qz * s;
  } else {
    px = qx;
    py = qy;
    pz = qz;
  }
}

struct Idx3 {
  int x, y, z;
  size_t sy, sz;  // strides of y and z
};
__device__ __forceinline__ Idx3 idx3(size_t i, int N) {
  const size_t NN = (size_t)N * N;
  return Idx3{(int)(i % N), (int)((i / N) % N), (int)(i / NN), (size_t)N, NN};
}

// div v at point i (backward differences, each component's last slot ignored)
__device__ __forceinline__ float div3_at(const float* __restrict__ v, size_t n3, size_t i, const Idx3& c, int N,
                                         float invh) {
  const float* vx = v;
  const float* vy = v + n3;
  const float* vz = v + 2 * n3;
  return ((c.x < N - 1 ? vx[i] : 0.f) - (c.x > 0 ? vx[i - 1] : 0.f) + (c.y < N - 1 ? vy[i] : 0.f) -
          (c.y > 0 ? vy[i - c.sy] : 0.f) + (c.z < N - 1 ? vz[i] : 0.f) - (c.z > 0 ? vz[i - c.sz] : 0.f)) *
         invh;
}

// ROF: p_{n+1} = proj(p_n + sigma grad u_{n+1})
__global__ void __launch_bounds__(256) k_rof3_pstep(const float* __restrict__ gu, const float* __restrict__ pin,
                                                    float* __restrict__ pout, int N, float sigma) {
  const size_t n3 = (size_t)N * N * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
    const Idx3 c = idx3(i, N);
    float px, py, pz;
    proj3(pin[i] + sigma * gu[i], pin[n3 + i] + sigma * gu[n3 + i], pin[2 * n3 + i] + sigma * gu[2 * n3 + i], px,
          py, pz);
    pout[i] = c.x < N - 1 ? px : 0.f;
    pout[n3 + i] = c.y < N - 1 ? py : 0.f;
    pout[2 * n3 + i] = c.z < N - 1 ? pz : 0.f;
  }
}

// ROF: r_{n+1} = lambda tau I + tau div pbar_{n+1} - div grad u_{n+1}, pbar = 2 p_{n+1} - p_n
__global__ void __launch_bounds__(256) k_rof3_rhs(const float* __restrict__ pout, const float* __restrict__ pin,
                                                  const float* __restrict__ gu, const float* __restrict__ I,
                                                  float* __restrict__ r, int N, float invh, float lt, float tau) {
  const size_t n3 = (size_t)N * N * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
    const Idx3 c = idx3(i, N);
    auto pb = [&](int comp, size_t j) { return 2.f * pout[comp * n3 + j] - pin[comp * n3 + j]; };
    const float dpb = ((c.x < N - 1 ? pb(0, i) : 0.f) - (c.x > 0 ? pb(0, i - 1) : 0.f) +
                       (c.y < N - 1 ? pb(1, i) : 0.f) - (c.y > 0 ? pb(1, i - c.sy) : 0.f) +
                       (c.z < N - 1 ? pb(2, i) : 0.f) - (c.z > 0 ? pb(2, i - c.sz) : 0.f)) *
                      invh;
    r[i] = lt * I[i] + tau * dpb - div3_at(gu, n3, i, c, N, invh);
  }
}

// EMD (affine Leray form): m = s + grad q;  p' = proj(p + sigma m);
// s' = m - tau (2 p' - p); m written when requested (gap steps)
__global__ void __launch_bounds__(256) k_emd3_step(const float* __restrict__ gq, const float* __restrict__ sin_,
                                                   const float* __restrict__ pin, float* __restrict__ sout,
                                                   float* __restrict__ pout, float* __restrict__ m, int N, float tau,
                                                   float sigma) {
  const size_t n3 = (size_t)N * N * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
    const Idx3 c = idx3(i, N);
    const bool in[3] = {c.x < N - 1, c.y < N - 1, c.z < N - 1};
    float mv[3], pv[3], q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      mv[k] = in[k] ? sin_[k * n3 + i] + gq[k * n3 + i] : 0.f;
      pv[k] = pin[k * n3 + i];
      q[k] = pv[k] + sigma * mv[k];
    }
    float p1[3];
    proj3(q[0], q[1], q[2], p1[0], p1[1], p1[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      if (!in[k]) p1[k] = 0.f;
      pout[k * n3 + i] = p1[k];
      sout[k * n3 + i] = in[k] ? mv[k] - tau * (2.f * p1[k] - pv[k]) : 0.f;
      if (m) m[k * n3 + i] = mv[k];
    }
  }
}

// EMD: d = g - div s
__global__ void __launch_bounds__(256) k_emd3_rhs(const float* __restrict__ sout, const float* __restrict__ g,
                                                  float* __restrict__ d, int N, float invh) {
  const size_t n3 = (size_t)N * N * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x)
    d[i] = g[i] - div3_at(sout, n3, i, idx3(i, N), N, invh);
}

// e = scale * div v
__global__ void __launch_bounds__(256) k_div3(const float* __restrict__ v, float* __restrict__ e, int N, float invh,
                                              float scale) {
  const size_t n3 = (size_t)N * N * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x)
    e[i] = scale * div3_at(v, n3, i, idx3(i, N), N, invh);
}

// ROF gap terms: sum |grad u|, sum (u - I)^2, sum I div p, sum (div p)^2
__global__ void __launch_bounds__(256) k_rof3_gap(const float* __restrict__ u, const float* __restrict__ gu,
                                                  const float* __restrict__ I, const float* __restrict__ p, int N,
                                                  float invh, double* __restrict__ part) {
  const size_t n3 = (size_t)N * N * N;
  CSum a, b, c2, d;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
    const float gx = gu[i], gy = gu[n3 + i], gz = gu[2 * n3 + i];
    a.add(sqrtf(gx * gx + gy * gy + gz * gz));
    const float e = u[i] - I[i];
    b.add(e * e);
    const float dp = div3_at(p, n3, i, idx3(i, N), N, invh);
    c2.add(I[i] * dp);
    d.add(dp * dp);
  }
  double v[4] = {a.value(), b.value(), c2.value(), d.value()};
  block_reduce_store<4>(v, 0u, part);
}

// EMD primal terms: sum |m|, sum |div m - g|
__global__ void __launch_bounds__(256) k_emd3_primal(const float* __restrict__ m, const float* __restrict__ g, int N,
                                                     float invh, double* __restrict__ part) {
  const size_t n3 = (size_t)N * N * N;
  CSum a, b;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
    const float mx = m[i], my = m[n3 + i], mz = m[2 * n3 + i];
    a.add(sqrtf(mx * mx + my * my + mz * mz));
    b.add(fabsf(div3_at(m, n3, i, idx3(i, N), N, invh) - g[i]));
  }
  double v[2] = {a.value(), b.value()};
  block_reduce_store<2>(v, 0u, part);
}

// EMD dual bound terms: sum phi (f1 - f0), max |grad phi|
__global__ void __launch_bounds__(256) k_emd3_dual(const float* __restrict__ phi, const float* __restrict__ gphi,
                                                   const float* __restrict__ f0, const float* __restrict__ f1, int N,
                                                   double* __restrict__ part) {
  const size_t n3 = (size_t)N * N * N;
  CSum a;
  double mx = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
    a.add(phi[i] * (f1[i] - f0[i]));
    const float gx = gphi[i], gy = gphi[n3 + i], gz = gphi[2 * n3 + i];
    mx = fmax(mx, (double)sqrtf(gx * gx + gy * gy + gz * gz));
  }
  double v[2] = {a.value(), mx};
  block_reduce_store<2>(v, 2u, part);
}

// ROF step-rule statistics of I: sum |grad I|, sum |grad I|^2, sum I
__global__ void __launch_bounds__(256) k_rof3_stats(const float* __restrict__ I, int N, float invh,
                                                    double* __restrict__ part) {
  const size_t n3 = (size_t)N * N * N;
  CSum a, b, c2;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3; i += (size_t)gridDim.x * blockDim.x) {
    const Idx3 c = idx3(i, N);
    const float v = I[i];
    const float gx = c.x < N - 1 ? (I[i + 1] - v) * invh : 0.f;
    const float gy = c.y < N - 1 ? (I[i + c.sy] - v) * invh : 0.f;
    const float gz = c.z < N - 1 ? (I[i + c.sz] - v) * invh : 0.f;
    const float m2 = gx * gx + gy * gy + gz * gz;
    a.add(sqrtf(m2));
    b.add(m2);
    c2.add(v);
  }
  double v[3] = {a.value(), b.value(), c2.value()};
  block_reduce_store<3>(v, 0u, part);
}

}  // namespace

// Row-block heights the fused kernels are instantiated for (the autotuned
// tile shape); 0 selects the default.
constexpr int kRBDefault = 16;
inline int norm_rb(int rb) { return (rb == 4 || rb == 8 || rb == 16 || rb == 32) ? rb : kRBDefault; }

dim3 fused_grid(int N, int V, int rb) { return dim3(ceil_div(ceil_div(N, V), 128), ceil_div(N, norm_rb(rb))); }

#define GP_RB_SWITCH(rb, CALL) \
  switch (norm_rb(rb)) {      \
    case 4: CALL(4); break;   \
    case 8: CALL(8); break;   \
    case 32: CALL(32); break; \
    default: CALL(16); break; \
  }

cudaError_t launch_rof_fused(const float* gu, const float* u, const float* pin, const float* I, float* pout, float* r,
                             double* part, const RofParams& P, bool vec, bool gap, int rb, cudaStream_t st) {
  const int V = vec ? 4 : 1;
  dim3 g = fused_grid(P.N, V, vec ? rb : kRBDefault);  // the scalar kernel walks kRBDefault rows per block
  if (vec) {
#define GP_L(R)                                                                                  \
  if (gap) k_rof_fused<4, R, true><<<g, 128, 0, st>>>(gu, u, pin, I, pout, r, part, P);           \
  else k_rof_fused<4, R, false><<<g, 128, 0, st>>>(gu, u, pin, I, pout, r, part, P)
    GP_RB_SWITCH(rb, GP_L)
#undef GP_L
  } else {
    if (gap) k_rof_fused<1, kRBDefault, true><<<g, 128, 0, st>>>(gu, u, pin, I, pout, r, part, P);
    else k_rof_fused<1, kRBDefault, false><<<g, 128, 0, st>>>(gu, u, pin, I, pout, r, part, P);
  }
  return cudaGetLastError();
}

cudaError_t launch_emd_fused(const float* gq, const float* sin_, const float* pin, const float* g, float* sout,
                             float* pout, float* d, float* m, float* e, double* part, const EmdParams& P, bool vec,
                             bool gap, int rb, cudaStream_t st) {
  const int V = vec ? 4 : 1;
  dim3 gr = fused_grid(P.N, V, vec ? rb : kRBDefault);  // the scalar kernel walks kRBDefault rows per block
  if (vec) {
#define GP_L(R)                                                                                            \
  if (gap) k_emd_fused<4, R, true><<<gr, 128, 0, st>>>(gq, sin_, pin, g, sout, pout, d, m, e, part, P);     \
  else k_emd_fused<4, R, false><<<gr, 128, 0, st>>>(gq, sin_, pin, g, sout, pout, d, m, e, part, P)
    GP_RB_SWITCH(rb, GP_L)
#undef GP_L
  } else {
    if (gap) k_emd_fused<1, kRBDefault, true><<<gr, 128, 0, st>>>(gq, sin_, pin, g, sout, pout, d, m, e, part, P);
    else k_emd_fused<1, kRBDefault, false><<<gr, 128, 0, st>>>(gq, sin_, pin, g, sout, pout, d, m, e, part, P);
  }
  return cudaGetLastError();
}

int reduce_blocks_1d(size_t n) { return grid_1d(n, 256) < 1024 ? grid_1d(n, 256) : 1024; }

cudaError_t launch_dual_residual(const float* p, const float* phi, float* r, int N, cudaStream_t st) {
  k_dual_residual<<<grid_1d((size_t)N * N, 256), 256, 0, st>>>(p, phi, r, N);
  return cudaGetLastError();
}

cudaError_t launch_emd_dual_hilo(const float* hi, const float* lo, const float* f0, const float* f1, int N,
                                 double* part, int nblk, cudaStream_t st) {
  k_emd_dual_hilo<<<nblk, 256, 0, st>>>(hi, lo, f0, f1, N, part);
  return cudaGetLastError();
}

cudaError_t launch_rof_stats(const float* I, int N, double* part, int nblk, cudaStream_t st) {
  k_rof_stats<<<nblk, 256, 0, st>>>(I, N, (float)N, part);
  return cudaGetLastError();
}

cudaError_t launch_sq_dev(const float* I, size_t NN, float mean, double* part, int nblk, cudaStream_t st) {
  k_sq_dev<<<nblk, 256, 0, st>>>(I, NN, mean, part);
  return cudaGetLastError();
}

cudaError_t launch_rof_gap(const float* u, const float* p, const float* I, int N, double* part, int nblk,
                           cudaStream_t st) {
  k_rof_gap<<<nblk, 256, 0, st>>>(u, p, I, N, (float)N, part);
  return cudaGetLastError();
}

cudaError_t launch_emd_primal(const float* m, const float* p, const float* f0, const float* f1, float* e, int N,
                              double* part, int nblk, cudaStream_t st) {
  k_emd_primal<<<nblk, 256, 0, st>>>(m, p, f0, f1, e, N, (float)N, part);
  return cudaGetLastError();
}

cudaError_t launch_emd_residual64(const float* m, const float* f0, const float* f1, float* rho, int N, double* part,
                                 int nblk, cudaStream_t st) {
  k_emd_residual64<<<nblk, 256, 0, st>>>(m, f0, f1, rho, N, (double)N, part);
  return cudaGetLastError();
}

cudaError_t launch_emd_corrected(const float* m, const float* gc, const float* f0, const float* f1, int N,
                                 double* part, int nblk, cudaStream_t st) {
  k_emd_corrected<<<nblk, 256, 0, st>>>(m, gc, f0, f1, N, (double)N, part);
  return cudaGetLastError();
}

cudaError_t launch_mass_stats(const float* f0, const float* f1, size_t NN, double* part, int nblk, cudaStream_t st) {
  k_mass_stats<<<nblk, 256, 0, st>>>(f0, f1, NN, part);
  return cudaGetLastError();
}

cudaError_t launch_final_reduce(const double* part, int nblk, int nq, unsigned maxmask, double* out, cudaStream_t st) {
  k_final_reduce<<<1, 256, 0, st>>>(part, nblk, nq, maxmask, out);
  return cudaGetLastError();
}

cudaError_t launch_rof_init(const float* I, const float* u, const float* pbar, float* p, float* r, const RofParams& P,
                            cudaStream_t st) {
  const size_t NN = (size_t)P.N * P.N;
  k_rof_init<<<grid_1d(NN, 256), 256, 0, st>>>(I, u, pbar, p, r, P);
  return cudaGetLastError();
}

cudaError_t launch_emd_init(const float* m0, const float* pbar, float* p, float* s, const float* g, float* d,
                            const EmdParams& P, cudaStream_t st) {
  const size_t NN = (size_t)P.N * P.N;
  k_emd_init<<<grid_1d(NN, 256), 256, 0, st>>>(m0, pbar, p, s, P);
  k_affine_rhs<<<grid_1d(NN, 256), 256, 0, st>>>(s, g, d, P.N, P.invh);
  return cudaGetLastError();
}

// Ergodic averages (the iterate averages of the convergence theorems): FP64
// running sums of FP32 planes, and their readout.
__global__ void k_accumulate(double* __restrict__ sum, const float* __restrict__ x, size_t n) {
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x)
    sum[idx] += (double)x[idx];
}

// out = sum * scale (FP32)
__global__ void k_scale_sum(const double* __restrict__ sum, float* __restrict__ out, size_t n, double scale) {
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += (size_t)gridDim.x * blockDim.x)
    out[idx] = (float)(sum[idx] * scale);
}

// EMD average flux: m = s_sum * scale + grad q (two planes; the zero slots of
// s and of the spectral gradient carry over)
__global__ void k_emd_average_flux(const double* __restrict__ s_sum, const float* __restrict__ gq,
                                   float* __restrict__ m, size_t n2, double scale) {
  for (size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n2; idx += (size_t)gridDim.x * blockDim.x)
    m[idx] = (float)(s_sum[idx] * scale + (double)gq[idx]);
}

cudaError_t launch_accumulate(double* sum, const float* x, size_t n, cudaStream_t st) {
  k_accumulate<<<grid_1d(n, 256), 256, 0, st>>>(sum, x, n);
  return cudaGetLastError();
}

cudaError_t launch_scale_sum(const double* sum, float* out, size_t n, double scale, cudaStream_t st) {
  k_scale_sum<<<grid_1d(n, 256), 256, 0, st>>>(sum, out, n, scale);
  return cudaGetLastError();
}

cudaError_t launch_emd_average_flux(const double* s_sum, const float* gq, float* m, size_t n2, double scale,
                                    cudaStream_t st) {
  k_emd_average_flux<<<grid_1d(n2, 256), 256, 0, st>>>(s_sum, gq, m, n2, scale);
  return cudaGetLastError();
}

cudaError_t launch_sub(const float* a, const float* b, float* out, size_t n, cudaStream_t st) {
  k_sub<<<grid_1d(n, 256), 256, 0, st>>>(a, b, out, n);
  return cudaGetLastError();
}

cudaError_t launch_grad(const float* x, float* g, int N, cudaStream_t st) {
  k_grad<<<grid_1d((size_t)N * N, 256), 256, 0, st>>>(x, g, N, (float)N);
  return cudaGetLastError();
}

cudaError_t launch_copy_field(const float* a, float* b, int N, cudaStream_t st) {
  k_copy_field<<<grid_1d((size_t)N * N, 256), 256, 0, st>>>(a, b, N);
  return cudaGetLastError();
}


// ------------------------------------------------------------------ 3-D

cudaError_t launch_helmholtz_residual(const float* b, const float* x, float* r, int N, double alpha, double inv_scale,
                                     cudaStream_t st) {
  k_helmholtz_residual<<<grid_1d((size_t)N * N, 256), 256, 0, st>>>(b, x, r, N, alpha, inv_scale);
  return cudaGetLastError();
}
cudaError_t launch_center(const float* x, float* out, size_t n, double* part, double* sum, cudaStream_t st) {
  const int nb = reduce_blocks_1d(n);
  k_sum<<<nb, 256, 0, st>>>(x, n, part);
  k_final_reduce<<<1, 256, 0, st>>>(part, nb, 1, 0u, sum);
  k_center<<<grid_1d(n, 256), 256, 0, st>>>(x, out, n, sum);
  return cudaGetLastError();
}
cudaError_t launch_add_inplace(float* x, const float* y, size_t n, cudaStream_t st) {
  k_add_inplace<<<grid_1d(n, 256), 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}
cudaError_t launch_rof3_pstep(const float* gu, const float* pin, float* pout, int N, float sigma, cudaStream_t st) {
  k_rof3_pstep<<<grid_1d((size_t)N * N * N, 256), 256, 0, st>>>(gu, pin, pout, N, sigma);
  return cudaGetLastError();
}
cudaError_t launch_rof3_rhs(const float* pout, const float* pin, const float* gu, const float* I, float* r, int N,
                            float lt, float tau, cudaStream_t st) {
  k_rof3_rhs<<<grid_1d((size_t)N * N * N, 256), 256, 0, st>>>(pout, pin, gu, I, r, N, (float)N, lt, tau);
  return cudaGetLastError();
}
cudaError_t launch_emd3_step(const float* gq, const float* sin_, const float* pin, float* sout, float* pout, float* m,
                             int N, float tau, float sigma, cudaStream_t st) {
  k_emd3_step<<<grid_1d((size_t)N * N * N, 256), 256, 0, st>>>(gq, sin_, pin, sout, pout, m, N, tau, sigma);
  return cudaGetLastError();
}
cudaError_t launch_emd3_rhs(const float* sout, const float* g, float* d, int N, cudaStream_t st) {
  k_emd3_rhs<<<grid_1d((size_t)N * N * N, 256), 256, 0, st>>>(sout, g, d, N, (float)N);
  return cudaGetLastError();
}
cudaError_t launch_div3(const float* v, float* e, int N, float scale, cudaStream_t st) {
  k_div3<<<grid_1d((size_t)N * N * N, 256), 256, 0, st>>>(v, e, N, (float)N, scale);
  return cudaGetLastError();
}
cudaError_t launch_rof3_gap(const float* u, const float* gu, const float* I, const float* p, int N, double* part,
                            int nblk, cudaStream_t st) {
  k_rof3_gap<<<nblk, 256, 0, st>>>(u, gu, I, p, N, (float)N, part);
  return cudaGetLastError();
}
cudaError_t launch_emd3_primal(const float* m, const float* g, int N, double* part, int nblk, cudaStream_t st) {
  k_emd3_primal<<<nblk, 256, 0, st>>>(m, g, N, (float)N, part);
  return cudaGetLastError();
}
cudaError_t launch_emd3_dual(const float* phi, const float* gphi, const float* f0, const float* f1, int N,
                             double* part, int nblk, cudaStream_t st) {
  k_emd3_dual<<<nblk, 256, 0, st>>>(phi, gphi, f0, f1, N, part);
  return cudaGetLastError();
}
cudaError_t launch_rof3_stats(const float* I, int N, double* part, int nblk, cudaStream_t st) {
  k_rof3_stats<<<nblk, 256, 0, st>>>(I, N, (float)N, part);
  return cudaGetLastError();
}

}  // namespace gp
