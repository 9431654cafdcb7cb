// 3x3 convolutions of the warm-start network on the 5th-generation tensor
// cores (BF16 storage mode): forward pass, weight gradient and data gradient.
//
// Implicit GEMMs D = A B^T, FP32 accumulation in tensor memory, zero padding
// outside the grid, k = c * 9 + t over the 3 x 3 taps t = 3 (dy + 1) + dx + 1:
//   forward     D[p][co] = sum_k X_col[p][k]  Wf[co][k],   Wf[co][ci * 9 + t] = W[co][ci][t]
//   data grad   D[q][ci] = sum_k dY_col[q][k] Wd[ci][k],   Wd[ci][co * 9 + t] = W[co][ci][8 - t]
//   weight grad D[k][co] = sum_q X_col[k][q]  dY[co][q]    (q over the pixels; an extra
//               row of ones at k = 9 Cin gives the bias gradient sum_q dY[co][q])
// A CTA of 128 threads (one warpgroup) owns 128 accumulator rows (pixels, or
// taps for the weight gradient) and a tile of up to 256 columns; the K loop
// runs over slabs of 64 in two shared-memory stages, so that the gather of
// slab s overlaps the tensor core's work on slab s - 1: one thread issues the
// tcgen05.mma instructions (K = 16 each) and tcgen05.commit signals the
// stage's mbarrier, which the threads wait on before they overwrite it.
//
// Operand layouts (no swizzle, 8 x 8 core matrices of 128 contiguous bytes):
// * the im2col operand of the forward and data-gradient products is MN-major
//   (eight consecutive pixels of one tap in 16 bytes), so that it is gathered
//   as shifted row segments: one aligned 16-byte load plus, for dx = +-1, one
//   neighbouring word and three funnel shifts per eight elements;
// * the weights are packed, once per update, into K-major images laid out
//   exactly as a stage expects them (rows padded to 16, K to 64, zeros
//   beyond), so a stage's B slab is one contiguous block copied with cp.async;
// * the weight gradient's operands are both K-major along the pixels: shifted
//   row segments of X and plain rows of dY.
// FP32 operands (dY) enter as hi + lo BF16 pairs, two MMAs per step.  Every
// mbarrier wait is bounded; a timeout sets the error flag, waits (bounded)
// for the tensor core and frees the tensor memory.  Grids without the
// alignment the vector gathers need (a row length not a multiple of 8, or an
// unaligned base) take a scalar gather with the same layouts.
#include <cuda_bf16.h>
#include <stdint.h>

#include "gp_internal.cuh"

namespace gp {
namespace {

constexpr int CM = 128;               // accumulator rows per CTA
constexpr int CK = 64;                // K slab
constexpr int CTHREADS = 128;         // one warpgroup
constexpr int A_BYTES = CM * CK * 2;  // 16 KiB
constexpr int kSMs = 152;
constexpr uint32_t kConvWait = 1u << 22;

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// K-major: row r, column k; MN-major: row m (MN), column k.  Both put core
// matrix (row >> 3, k >> 3) at (row >> 3) * 1024 + (k >> 3) * 128, so one
// descriptor form (128 B between core matrices along K, 1024 B along MN)
// serves both; the instruction descriptor's transpose bit tells them apart.
__device__ __forceinline__ uint32_t kmaj(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ uint32_t mnmaj(int m, int k) {
  return (uint32_t)((m >> 3) * 1024 + (k >> 3) * 128 + (k & 7) * 16 + (m & 7) * 2);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = 1024;
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

// D = F32, A = B = BF16, B K-major, A K-major or MN-major (bit 15), M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_bf16(int n, bool a_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (a_mn ? (1u << 15) : 0u) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(CM >> 4) << 24);
}

__device__ __forceinline__ bool wait_bar(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kConvWait; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mma(uint32_t tmem, uint32_t a, uint32_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
      "l"(sdesc(a)), "l"(sdesc(b)), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_wait_all() {
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ void st_out(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_out(__nv_bfloat16* p, float v) { *p = __float2bfloat16(v); }

// Tensor-memory allocation (warp 0), the two stage barriers, and the teardown.
__device__ __forceinline__ uint32_t tc_setup(uint64_t* bar, uint32_t* slot, int tcols) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(slot)),
                 "r"((uint32_t)tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar + 1)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  return *slot;
}
__device__ __forceinline__ void tc_teardown(uint32_t tmem, int tcols) {
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)tcols));
  }
}
// 16 accumulator columns of this thread's lane (warp w: lanes 32w .. 32w + 31).
__device__ __forceinline__ void tmem_ld16(uint32_t tmem, int c0, float* v) {
  uint32_t r[16];
  const uint32_t taddr = tmem + ((uint32_t)((threadIdx.x >> 5) * 32) << 16) + (uint32_t)c0;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int c = 0; c < 16; ++c) v[c] = __uint_as_float(r[c]);
}

// Eight consecutive elements row[x0 + dx .. x0 + dx + 7] of one grid row,
// zero outside [0, Wd): x0 % 8 == 0, x0 + 8 <= Wd, the row 16-byte aligned.
// BF16 pairs are 32-bit words (the lower address in the low half), so a
// shift by one element is a 16-bit funnel shift across neighbouring words.
// The loads (issued for all of a slab's items before any is used) and the
// combination are separate steps.
__device__ __forceinline__ void row8_load(const __nv_bfloat16* row, int x0, int dx, int Wd, uint4& c, uint32_t& nb) {
  c = __ldg(reinterpret_cast<const uint4*>(row + x0));
  nb = 0u;
  if (dx < 0 && x0 > 0) nb = __ldg(reinterpret_cast<const uint32_t*>(row + x0 - 2));
  if (dx > 0 && x0 + 8 < Wd) nb = __ldg(reinterpret_cast<const uint32_t*>(row + x0 + 8));
}
__device__ __forceinline__ uint4 row8_combine(const uint4& c, uint32_t nb, int dx) {
  if (dx == 0) return c;
  if (dx < 0)
    return make_uint4(__funnelshift_r(nb, c.x, 16), __funnelshift_r(c.x, c.y, 16), __funnelshift_r(c.y, c.z, 16),
                      __funnelshift_r(c.z, c.w, 16));
  return make_uint4(__funnelshift_r(c.x, c.y, 16), __funnelshift_r(c.y, c.z, 16), __funnelshift_r(c.z, c.w, 16),
                    __funnelshift_r(c.w, nb, 16));
}
__device__ __forceinline__ void row8_load(const float* row, int x0, int dx, int Wd, float4& a, float4& b, float& nb) {
  a = __ldg(reinterpret_cast<const float4*>(row + x0));
  b = __ldg(reinterpret_cast<const float4*>(row + x0 + 4));
  nb = 0.f;
  if (dx < 0 && x0 > 0) nb = __ldg(row + x0 - 1);
  if (dx > 0 && x0 + 8 < Wd) nb = __ldg(row + x0 + 8);
}
__device__ __forceinline__ void row8_combine(const float4& a, const float4& b, float nb, int dx, float* o) {
  if (dx == 0) {
    o[0] = a.x, o[1] = a.y, o[2] = a.z, o[3] = a.w, o[4] = b.x, o[5] = b.y, o[6] = b.z, o[7] = b.w;
  } else if (dx < 0) {
    o[0] = nb, o[1] = a.x, o[2] = a.y, o[3] = a.z, o[4] = a.w, o[5] = b.x, o[6] = b.y, o[7] = b.z;
  } else {
    o[0] = a.y, o[1] = a.z, o[2] = a.w, o[3] = b.x, o[4] = b.y, o[5] = b.z, o[6] = b.w, o[7] = nb;
  }
}

// FP32 -> (hi, lo) BF16 with hi + lo = v to 16 significant bits.
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    const float2 back = __bfloat1622float2(hh);
    const __nv_bfloat162 ll = __floats2bfloat162_rn(v[2 * i] - back.x, v[2 * i + 1] - back.y);
    h[i] = *reinterpret_cast<const uint32_t*>(&hh);
    l[i] = *reinterpret_cast<const uint32_t*>(&ll);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}
__device__ __forceinline__ uint4 pack8(const float* v) {
  uint32_t h[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 hh = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    h[i] = *reinterpret_cast<const uint32_t*>(&hh);
  }
  return make_uint4(h[0], h[1], h[2], h[3]);
}
__device__ __forceinline__ float ldf(const __nv_bfloat16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ float ldf(const float* p) { return *p; }

// Rows padded to 16 and columns to 64: the image of an R x K matrix.
__host__ __device__ inline int pad16(int r) { return (r + 15) / 16 * 16; }
__host__ __device__ inline int pad64(int k) { return (k + 63) / 64 * 64; }

// Both K-major weight images of one convolution (element offsets: the
// forward image Wf, NPf x Kpf with NPf = pad16(Cout), Kpf = pad64(9 Cin), then
// the data-gradient image Wd, NPd x Kpd with NPd = pad16(Cin), Kpd =
// pad64(9 Cout)).  Slab s of an image holds columns [64 s, 64 s + 64) of all
// its rows as a stage's B operand: element (n >> 3) * 512 + ((k & 63) >> 3) *
// 64 + (n & 7) * 8 + (k & 7) after s * NP * 64.
__global__ void k_pack_conv(const __nv_bfloat16* __restrict__ W, int Cin, int Cout, __nv_bfloat16* __restrict__ img) {
  const int Kf = 9 * Cin, Kd = 9 * Cout;
  const int NPf = pad16(Cout), Kpf = pad64(Kf), NPd = pad16(Cin), Kpd = pad64(Kd);
  const long nf = (long)NPf * Kpf, nd = (long)NPd * Kpd;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < nf + nd; i += (long)gridDim.x * blockDim.x) {
    const bool fwd = i < nf;
    const long j = fwd ? i : i - nf;
    const int Kp = fwd ? Kpf : Kpd, NP = fwd ? NPf : NPd;
    const int n = (int)(j / Kp), k = (int)(j % Kp);
    __nv_bfloat16 v = __float2bfloat16(0.f);
    if (fwd) {
      if (n < Cout && k < Kf) v = W[(long)n * Kf + k];
    } else if (n < Cin && k < Kd) {
      const int co = k / 9, t = k - 9 * co;
      v = W[((long)co * Cin + n) * 9 + (8 - t)];
    }
    const long dst = (long)(k >> 6) * NP * 64 + (n >> 3) * 512 + ((k & 63) >> 3) * 64 + (n & 7) * 8 + (k & 7);
    img[(fwd ? 0 : nf) + dst] = v;
  }
}

// Forward (TX = BF16: A = im2col of the input) and data gradient (TX = FP32:
// A = im2col of the output gradient, hi + lo): D[p][n] for the 128 pixels p
// of tile blockIdx.x (row-major in the H x Wd plane), the image rows n in
// [n0, n0 + nloc) of column tile blockIdx.y, and sample blockIdx.z.  Cx is
// the im2col source's channel count (K = 9 Cx), img the weight image (NP rows,
// pad64(K) columns); outputs n < Ny are written, with bias and ReLU applied
// when given.
template <typename TX, typename TY, bool RELU>
__global__ void __launch_bounds__(CTHREADS) k_conv_tc(const TX* __restrict__ X, long xbs, int Cx,
                                                      const __nv_bfloat16* __restrict__ img, int NP, int nt, int tcols,
                                                      const float* __restrict__ bias, TY* __restrict__ Y, long ybs,
                                                      int Ny, int H, int Wd, int vec, int* __restrict__ err) {
  constexpr bool SPLIT = sizeof(TX) == 4;
  constexpr int NA = SPLIT ? 2 : 1;
  extern __shared__ __align__(1024) uint8_t smem[];
  const int n0 = blockIdx.y * nt;
  const int nloc = min(nt, NP - n0);
  const int stage = NA * A_BYTES + nt * 128;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * stage);
  const uint32_t tmem = tc_setup(bar, reinterpret_cast<uint32_t*>(bar + 2), tcols);
  const long plane = (long)H * Wd;
  const long m0 = (long)blockIdx.x * CM;
  const TX* Xb = X + (long)blockIdx.z * xbs;
  const int K = 9 * Cx, nslab = (K + CK - 1) / CK;
  // A items of this thread: pixel group pg (pixels p0 .. p0 + 7), column 8 j + kr of each slab
  const int kr = threadIdx.x & 7, pg = threadIdx.x >> 3;
  const long p0 = m0 + 8 * pg;
  const bool pin = p0 < plane;
  const int py = pin ? (int)(p0 / Wd) : 0, px = pin ? (int)(p0 % Wd) : 0;
  const uint32_t id = idesc_bf16(nloc, true);
  const __nv_bfloat16* imgc = img + (long)n0 * 64;
  uint32_t ph = 0u;  // bit b: the parity of stage b's next barrier phase
  bool ok = true;
  int s = 0;
  for (; s < nslab; ++s) {
    const int b = s & 1;
    uint8_t* As = smem + b * stage;
    uint8_t* Bs = As + NA * A_BYTES;
    const unsigned kb = (unsigned)(s * CK + kr);  // column 8 j of the slab is k = kb + 8 j
    if (s >= 2) {  // the tensor core has finished slab s - 2, which used this stage
      if (!wait_bar(su32(bar + b), (ph >> b) & 1u)) ok = false;
      ph ^= 1u << b;
    }
    if (ok) {  // B: the image's slab s, one contiguous block
      const __nv_bfloat16* src = imgc + (long)s * NP * 64;
      for (int i = threadIdx.x; i < nloc * 8; i += CTHREADS) cp16(su32(Bs) + 16 * i, src + 8 * i);
    }
    if (vec) {
      int dxj[8];
      if constexpr (!SPLIT) {
        uint4 c[8];
        uint32_t nb[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const unsigned k = kb + 8 * j, ch = k / 9, t = k - 9 * ch;
          const int yy = py + (int)(t / 3) - 1;
          dxj[j] = (int)(t % 3) - 1;
          c[j] = make_uint4(0u, 0u, 0u, 0u);
          nb[j] = 0u;
          if (pin && (int)ch < Cx && yy >= 0 && yy < H) row8_load(Xb + ch * plane + (long)yy * Wd, px, dxj[j], Wd, c[j], nb[j]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j)
          *reinterpret_cast<uint4*>(As + mnmaj(8 * pg, 8 * j + kr)) = row8_combine(c[j], nb[j], dxj[j]);
      } else {
        float4 a[8], bb[8];
        float nb[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const unsigned k = kb + 8 * j, ch = k / 9, t = k - 9 * ch;
          const int yy = py + (int)(t / 3) - 1;
          dxj[j] = (int)(t % 3) - 1;
          a[j] = bb[j] = make_float4(0.f, 0.f, 0.f, 0.f);
          nb[j] = 0.f;
          if (pin && (int)ch < Cx && yy >= 0 && yy < H)
            row8_load(Xb + ch * plane + (long)yy * Wd, px, dxj[j], Wd, a[j], bb[j], nb[j]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float o[8];
          row8_combine(a[j], bb[j], nb[j], dxj[j], o);
          uint4 hi, lo;
          split8(o, hi, lo);
          *reinterpret_cast<uint4*>(As + mnmaj(8 * pg, 8 * j + kr)) = hi;
          *reinterpret_cast<uint4*>(As + A_BYTES + mnmaj(8 * pg, 8 * j + kr)) = lo;
        }
      }
    } else {  // scalar gather, same layout
#pragma unroll 1
      for (int j = 0; j < 8; ++j) {
        const unsigned k = kb + 8 * j, c = k / 9, t = k - 9 * c;
        const int dy = (int)(t / 3) - 1, dx = (int)(t % 3) - 1;
        float o[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const long p = p0 + e;
          o[e] = 0.f;
          if (p < plane && (int)c < Cx) {
            const int y = (int)(p / Wd) + dy, x = (int)(p % Wd) + dx;
            if (y >= 0 && y < H && x >= 0 && x < Wd) o[e] = ldf(Xb + c * plane + (long)y * Wd + x);
          }
        }
        if constexpr (SPLIT) {
          uint4 hi, lo;
          split8(o, hi, lo);
          *reinterpret_cast<uint4*>(As + mnmaj(8 * pg, 8 * j + kr)) = hi;
          *reinterpret_cast<uint4*>(As + A_BYTES + mnmaj(8 * pg, 8 * j + kr)) = lo;
        } else {
          *reinterpret_cast<uint4*>(As + mnmaj(8 * pg, 8 * j + kr)) = pack8(o);
        }
      }
    }
    cp_wait_all();
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int j = 0; j < CK / 16; ++j)
#pragma unroll
        for (int a = 0; a < NA; ++a)
          mma(tmem, su32(As) + a * A_BYTES + j * 256, su32(Bs) + j * 256, id, (s > 0 || j > 0 || a > 0) ? 1u : 0u);
      commit(su32(bar + b));
    }
  }
  if (threadIdx.x == 0 && s >= 1) {  // the last commit covers every MMA issued
    const int b = (s - 1) & 1;
    if (!wait_bar(su32(bar + b), (ph >> b) & 1u)) {
      ok = false;
      wait_bar(su32(bar + b), (ph >> b) & 1u);  // once more (bounded) before the memory is released
    }
  }
  ok = __syncthreads_and(ok);
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;");
    const long p = m0 + threadIdx.x;  // accumulator lane = pixel
    TY* Yb = Y + (long)blockIdx.z * ybs;
    for (int c0 = 0; c0 < nloc; c0 += 16) {
      float v[16];
      tmem_ld16(tmem, c0, v);
      if (p < plane) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int n = n0 + c0 + c;
          if (n < Ny) {
            float x = v[c] + (bias ? __ldg(&bias[n]) : 0.f);
            if (RELU) x = fmaxf(x, 0.f);
            st_out(Yb + (long)n * plane + p, x);
          }
        }
      }
    }
  }
  tc_teardown(tmem, tcols);
}

// Weight and bias gradients: D[m][n] = sum_q A[m][q] B[n][q] over the pixels
// q in [q0, q1) of chunk blockIdx.z % chunks of sample blockIdx.z / chunks,
// the rows m of tile blockIdx.x (taps k = ci * 9 + t < K = 9 Cin; the row
// m = K is all ones; zero beyond) and the output channels n of tile
// blockIdx.y.  A = shifted rows of X, B = rows of dY (hi + lo), both K-major
// along q.  The tile is added to dW[co][k] and db[co] with FP32 atomics.
__global__ void __launch_bounds__(CTHREADS) k_conv_wgrad_tc(const float* __restrict__ dY, long dybs, int Cout,
                                                            const __nv_bfloat16* __restrict__ X, long xbs, int Cin,
                                                            int H, int Wd, int LQ, int chunks, int nt, int tcols,
                                                            int vec, float* __restrict__ dW, float* __restrict__ db,
                                                            int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  const int NPc = pad16(Cout);
  const int n0 = blockIdx.y * nt, nloc = min(nt, NPc - n0);
  const int stage = A_BYTES + 2 * nt * 128;
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * stage);
  const uint32_t tmem = tc_setup(bar, reinterpret_cast<uint32_t*>(bar + 2), tcols);
  const long plane = (long)H * Wd;
  const int K = 9 * Cin;
  const int smp = blockIdx.z / chunks, chunk = blockIdx.z % chunks;
  const long q0 = (long)chunk * LQ, q1 = q0 + LQ < plane ? q0 + LQ : plane;
  const float* dYb = dY + (long)smp * dybs;
  const __nv_bfloat16* Xb = X + (long)smp * xbs;
  // A items of this thread: rows ml[i] = (t & 7) + 8 (t >> 5) + 32 i (i < 4),
  // pixel groups g = gl + 4 h (h < 2) of each slab
  const int gl = (threadIdx.x >> 3) & 3;
  int ml[4], tcn[4], tdy[4], tdx[4];  // channel (-1: zero row, -2: ones row) and tap offsets
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    ml[i] = (threadIdx.x & 7) + 8 * (threadIdx.x >> 5) + 32 * i;
    const int m = blockIdx.x * CM + ml[i];
    tcn[i] = m < K ? m / 9 : (m == K ? -2 : -1);
    const int t = m < K ? m % 9 : 4;
    tdy[i] = t / 3 - 1;
    tdx[i] = t % 3 - 1;
  }
  const uint32_t id = idesc_bf16(nloc, false);
  const int nslab = (int)((q1 - q0 + CK - 1) / CK);
  const uint4 ones = make_uint4(0x3F803F80u, 0x3F803F80u, 0x3F803F80u, 0x3F803F80u);  // BF16 1.0 pairs
  uint32_t ph = 0u;  // bit b: the parity of stage b's next barrier phase
  bool ok = true;
  int s = 0;
  for (; s < nslab; ++s) {
    const int b = s & 1;
    uint8_t* As = smem + b * stage;
    uint8_t* Bh = As + A_BYTES;
    uint8_t* Bl = Bh + nt * 128;
    if (s >= 2) {
      if (!wait_bar(su32(bar + b), (ph >> b) & 1u)) ok = false;
      ph ^= 1u << b;
    }
    const long qs = q0 + (long)s * CK;
    uint4 ac[2][4];
    uint32_t an[2][4];
    if (vec) {  // A loads first; a group lies in one row and wholly inside or outside [q0, q1)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const unsigned q = (unsigned)(qs + 8 * (gl + 4 * h));
        const bool qin = q < (unsigned)q1;
        const int y = (int)(q / (unsigned)Wd), x0 = (int)(q % (unsigned)Wd);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int yy = y + tdy[i];
          ac[h][i] = (qin && tcn[i] == -2) ? ones : make_uint4(0u, 0u, 0u, 0u);
          an[h][i] = 0u;
          if (qin && tcn[i] >= 0 && yy >= 0 && yy < H)
            row8_load(Xb + tcn[i] * plane + (long)yy * Wd, x0, tdx[i], Wd, ac[h][i], an[h][i]);
        }
      }
    } else {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int g = gl + 4 * h;
        const long q = qs + 8 * g;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          float o[8];
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const long qe = q + e;
            o[e] = 0.f;
            if (qe < q1 && tcn[i] == -2) {
              o[e] = 1.f;
            } else if (qe < q1 && tcn[i] >= 0) {
              const int y = (int)(qe / Wd) + tdy[i], x = (int)(qe % Wd) + tdx[i];
              if (y >= 0 && y < H && x >= 0 && x < Wd) o[e] = __bfloat162float(Xb[tcn[i] * plane + (long)y * Wd + x]);
            }
          }
          *reinterpret_cast<uint4*>(As + kmaj(ml[i], 8 * g)) = pack8(o);
        }
      }
    }
    // B: rows r = 8 (it >> 6) + (it & 7), groups g = (it >> 3) & 7, four items' loads at a time
    for (int it0 = threadIdx.x; it0 < nloc * 8; it0 += 4 * CTHREADS) {
      float4 lo4[4], hi4[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int it = it0 + u * CTHREADS;
        const int r = 8 * (it >> 6) + (it & 7), g = (it >> 3) & 7;
        const int co = n0 + r;
        const long q = qs + 8 * g;
        lo4[u] = hi4[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (it < nloc * 8 && co < Cout && q < q1) {
          const float* src = dYb + (long)co * plane + q;
          if (vec) {
            lo4[u] = __ldg(reinterpret_cast<const float4*>(src));
            hi4[u] = __ldg(reinterpret_cast<const float4*>(src + 4));
          } else {
            float o[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) o[e] = q + e < q1 ? src[e] : 0.f;
            lo4[u] = make_float4(o[0], o[1], o[2], o[3]);
            hi4[u] = make_float4(o[4], o[5], o[6], o[7]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int it = it0 + u * CTHREADS;
        if (it < nloc * 8) {
          const int r = 8 * (it >> 6) + (it & 7), g = (it >> 3) & 7;
          const float o[8] = {lo4[u].x, lo4[u].y, lo4[u].z, lo4[u].w, hi4[u].x, hi4[u].y, hi4[u].z, hi4[u].w};
          uint4 hi, lo;
          split8(o, hi, lo);
          *reinterpret_cast<uint4*>(Bh + kmaj(r, 8 * g)) = hi;
          *reinterpret_cast<uint4*>(Bl + kmaj(r, 8 * g)) = lo;
        }
      }
    }
    if (vec) {
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int i = 0; i < 4; ++i)
          *reinterpret_cast<uint4*>(As + kmaj(ml[i], 8 * (gl + 4 * h))) = row8_combine(ac[h][i], an[h][i], tdx[i]);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int j = 0; j < CK / 16; ++j) {
        mma(tmem, su32(As) + j * 256, su32(Bh) + j * 256, id, (s > 0 || j > 0) ? 1u : 0u);
        mma(tmem, su32(As) + j * 256, su32(Bl) + j * 256, id, 1u);
      }
      commit(su32(bar + b));
    }
  }
  if (threadIdx.x == 0 && s >= 1) {
    const int b = (s - 1) & 1;
    if (!wait_bar(su32(bar + b), (ph >> b) & 1u)) {
      ok = false;
      wait_bar(su32(bar + b), (ph >> b) & 1u);
    }
  }
  ok = __syncthreads_and(ok);
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else if (s >= 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int m = blockIdx.x * CM + threadIdx.x;  // accumulator lane = tap row
    for (int c0 = 0; c0 < nloc; c0 += 16) {
      float v[16];
      tmem_ld16(tmem, c0, v);
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        const int co = n0 + c0 + c;
        if (co < Cout) {
          if (m < K) atomicAdd(&dW[(long)co * K + m], v[c]);
          else if (m == K && db) atomicAdd(&db[co], v[c]);
        }
      }
    }
  }
  tc_teardown(tmem, tcols);
}

inline bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; }

template <typename TX, typename TY, bool RELU>
cudaError_t launch_conv(const TX* X, long xbs, int Cx, const __nv_bfloat16* img, int NP, const float* bias, TY* Y,
                        long ybs, int Ny, int H, int Wd, int B, int* err, cudaStream_t st) {
  const long plane = (long)H * Wd;
  const long tiles = (plane + CM - 1) / CM;
  if (tiles > 0x7FFFFFFFL || B > 65535) return cudaErrorInvalidValue;
  // column tiles of at most 256, halved (down to 32) while the grid is short of two CTAs per SM
  int nt = NP < 256 ? NP : 256;
  while (nt > 32 && tiles * B * ((NP + nt - 1) / nt) < 2 * kSMs) nt = pad16(nt / 2);
  int tcols = 32;
  while (tcols < nt) tcols *= 2;
  const int NA = sizeof(TX) == 4 ? 2 : 1;
  const size_t sm = 2 * ((size_t)NA * A_BYTES + (size_t)nt * 128) + 64;
  cudaError_t e = cudaFuncSetAttribute(k_conv_tc<TX, TY, RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int vec = Wd % 8 == 0 && al16(X) && (xbs * (long)sizeof(TX)) % 16 == 0;
  dim3 grid((unsigned)tiles, (unsigned)((NP + nt - 1) / nt), (unsigned)B);
  k_conv_tc<TX, TY, RELU><<<grid, CTHREADS, sm, st>>>(X, xbs, Cx, img, NP, nt, tcols, bias, Y, ybs, Ny, H, Wd, vec,
                                                      err);
  return cudaGetLastError();
}

}  // namespace

size_t conv3x3_tc_image_elems(int Cin, int Cout) {
  return (size_t)pad16(Cout) * pad64(9 * Cin) + (size_t)pad16(Cin) * pad64(9 * Cout);
}

cudaError_t conv3x3_tc_pack(const void* W, int Cin, int Cout, void* img, cudaStream_t st) {
  const long n = (long)conv3x3_tc_image_elems(Cin, Cout);
  const int grid = (int)((n + 255) / 256 < 4096 ? (n + 255) / 256 : 4096);
  k_pack_conv<<<grid, 256, 0, st>>>(static_cast<const __nv_bfloat16*>(W), Cin, Cout,
                                    static_cast<__nv_bfloat16*>(img));
  return cudaGetLastError();
}

cudaError_t conv3x3_tc(const void* X, long xbs, int Cin, const void* img, const float* bias, void* Y, long ybs,
                       int Cout, int H, int Wd, int B, bool relu, bool y_fp32, int* err, cudaStream_t st) {
  const auto* x = static_cast<const __nv_bfloat16*>(X);
  const auto* w = static_cast<const __nv_bfloat16*>(img);
  const int NP = pad16(Cout);
  using bf = __nv_bfloat16;
  if (y_fp32)
    return relu ? launch_conv<bf, float, true>(x, xbs, Cin, w, NP, bias, static_cast<float*>(Y), ybs, Cout, H, Wd, B,
                                               err, st)
                : launch_conv<bf, float, false>(x, xbs, Cin, w, NP, bias, static_cast<float*>(Y), ybs, Cout, H, Wd, B,
                                                err, st);
  auto* y = static_cast<bf*>(Y);
  return relu ? launch_conv<bf, bf, true>(x, xbs, Cin, w, NP, bias, y, ybs, Cout, H, Wd, B, err, st)
              : launch_conv<bf, bf, false>(x, xbs, Cin, w, NP, bias, y, ybs, Cout, H, Wd, B, err, st);
}

cudaError_t conv3x3_dgrad_tc(const float* dY, long dybs, int Cout, const void* img, float* dX, long dxbs, int Cin,
                             int H, int Wd, int B, int* err, cudaStream_t st) {
  const auto* wd = static_cast<const __nv_bfloat16*>(img) + (size_t)pad16(Cout) * pad64(9 * Cin);
  return launch_conv<float, float, false>(dY, dybs, Cout, wd, pad16(Cin), nullptr, dX, dxbs, Cin, H, Wd, B, err, st);
}

cudaError_t conv3x3_wgrad_tc(const float* dY, long dybs, int Cout, const void* X, long xbs, int Cin, int H, int Wd,
                             int B, float* dW, float* db, int* err, cudaStream_t st) {
  const int K = 9 * Cin;
  const int mtiles = (K + 1 + CM - 1) / CM;  // the taps and the ones row
  const int NPc = pad16(Cout);
  const int nt = NPc < 128 ? NPc : 128;
  const int ntiles = (NPc + nt - 1) / nt;
  int tcols = 32;
  while (tcols < nt) tcols *= 2;
  const long plane = (long)H * Wd;
  // pixel chunks (multiples of 64, at least 256) for about four CTAs per SM
  const long per = (long)mtiles * ntiles * B;
  long chunks = (4L * kSMs + per - 1) / per;
  long LQ = (plane + chunks - 1) / chunks;
  LQ = pad64((int)(LQ < 256 ? 256 : LQ));
  chunks = (plane + LQ - 1) / LQ;
  if ((long)B * chunks > 65535 || ntiles > 65535 || plane > 0x7FFFFFFFL) return cudaErrorInvalidValue;
  const size_t sm = 2 * ((size_t)A_BYTES + 2 * (size_t)nt * 128) + 64;
  cudaError_t e = cudaFuncSetAttribute(k_conv_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const auto* x = static_cast<const __nv_bfloat16*>(X);
  const int vec = Wd % 8 == 0 && al16(X) && al16(dY) && (xbs * 2) % 16 == 0 && (dybs * 4) % 16 == 0;
  dim3 grid((unsigned)mtiles, (unsigned)ntiles, (unsigned)(B * chunks));
  k_conv_wgrad_tc<<<grid, CTHREADS, sm, st>>>(dY, dybs, Cout, x, xbs, Cin, H, Wd, (int)LQ, (int)chunks, nt, tcols, vec,
                                              dW, db, err);
  return cudaGetLastError();
}

}  // namespace gp
