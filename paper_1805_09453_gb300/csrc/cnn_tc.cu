// 3x3 convolution of the warm-start network on the 5th-generation tensor
// cores (BF16 storage mode): forward pass, weight gradient and data gradient.
//
// Implicit GEMM: Y[co][p] = act(bias[co] + sum_k W[co][k] X_col[p][k]) with
// k = ci * 9 + t over the Cin x 3 x 3 receptive field (t = 3 (dy + 1) +
// dx + 1, zero padding outside the grid), i.e. D = A B^T with
// A = X_col (M = 128 output pixels per CTA, K-major), B = W (N = the output
// channels padded to a multiple of 16, K-major: W[co][ci][3][3] is already
// [co][k]).  The K loop runs over slabs of 64: 128 threads gather the A slab
// (im2col) and the B slab into shared memory in the canonical no-swizzle
// K-major layout (8 x 8 core matrices, 128 B apart along K, 1024 B along
// M / N), one thread issues four tcgen05.mma (K = 16 each) accumulating in
// FP32 in tensor memory, and tcgen05.commit signals an mbarrier before the
// slab is overwritten.  The epilogue reads the accumulator with tcgen05.ld
// (warp w owns tensor-memory lanes 32w..32w+31, i.e. pixels), adds the bias,
// applies the ReLU and stores BF16 (or FP32 for the head) activations.
// Every mbarrier wait is bounded; a timeout sets the error flag, waits
// (bounded) for the tensor core and frees the tensor memory.
#include <cuda_bf16.h>
#include <stdint.h>

#include "gp_internal.cuh"

namespace gp {
namespace {

constexpr int CM = 128;               // output pixels per CTA (accumulator lanes)
constexpr int CK = 64;                // K slab
constexpr int CTHREADS = 128;         // one warpgroup
constexpr int A_BYTES = CM * CK * 2;  // 16 KiB
constexpr uint32_t kConvWait = 1u << 22;

__device__ __forceinline__ uint32_t su32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ uint32_t kmaj(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = 1024;
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

// D = F32, A = B = BF16, both K-major, M = 128, N = n.
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(CM >> 4) << 24);
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

__device__ __forceinline__ void st_out(float* p, float v) { *p = v; }
__device__ __forceinline__ void st_out(__nv_bfloat16* p, float v) { *p = __float2bfloat16(v); }

// One CTA: output pixels [m0, m0 + 128) of sample blockIdx.y (row-major over
// the H x Wd plane), all Cout channels (NP = Cout padded, 16..256).
template <typename TY, bool RELU>
__global__ void __launch_bounds__(CTHREADS) k_conv3x3_tc(const __nv_bfloat16* __restrict__ X, long xbs, int Cin,
                                                         const __nv_bfloat16* __restrict__ W,
                                                         const float* __restrict__ bias, TY* __restrict__ Y, long ybs,
                                                         int Cout, int NP, int tcols, int H, int Wd,
                                                         int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* As = smem;                        // 128 x 64 bf16
  uint8_t* Bs = smem + A_BYTES;              // NP x 64 bf16
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + (size_t)NP * CK * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long plane = (long)H * Wd;
  const long m0 = (long)blockIdx.x * CM;
  const int b = blockIdx.y;
  const __nv_bfloat16* Xb = X + (long)b * xbs;
  const int K = Cin * 9;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"((uint32_t)tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const uint32_t id = idesc_bf16(NP);
  // this thread's pixel (A row) for the gather
  const long pm = m0 + threadIdx.x;
  const bool pin = pm < plane;
  const int py = pin ? (int)(pm / Wd) : 0, px = pin ? (int)(pm % Wd) : 0;
  bool ok = true;
  uint32_t phase = 0;
  const int nslab = (K + CK - 1) / CK;
  for (int ks = 0; ks < nslab; ++ks) {
    const int k0 = ks * CK;
    // A slab: row threadIdx.x, 64 consecutive k
    for (int kk = 0; kk < CK; kk += 8) {
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + kk + e;
        float x = 0.f;
        if (pin && k < K) {
          const int ci = k / 9, t = k - 9 * ci;
          const int yy = py + t / 3 - 1, xx = px + t % 3 - 1;
          if (yy >= 0 && yy < H && xx >= 0 && xx < Wd) x = __bfloat162float(Xb[(long)ci * plane + (long)yy * Wd + xx]);
        }
        v[e] = __float2bfloat16(x);
      }
      *reinterpret_cast<uint4*>(As + kmaj(threadIdx.x, kk)) = *reinterpret_cast<const uint4*>(v);
    }
    // B slab: NP rows x 64 k (zero beyond Cout / K)
    for (int r = threadIdx.x; r < NP * (CK / 8); r += CTHREADS) {
      const int co = r / (CK / 8), kk = (r % (CK / 8)) * 8;
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + kk + e;
        v[e] = (co < Cout && k < K) ? W[(long)co * K + k] : __float2bfloat16(0.f);
      }
      *reinterpret_cast<uint4*>(Bs + kmaj(co, kk)) = *reinterpret_cast<const uint4*>(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int j = 0; j < CK / 16; ++j) {
        const uint32_t off = (uint32_t)j * 256;  // 16 k = two core matrices
        const uint64_t ad = sdesc(su32(As) + off), bd = sdesc(su32(Bs) + off);
        const uint32_t acc = (ks > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(id), "r"(acc));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                   : "memory");
    }
    // the slab's buffers are rewritten only after the tensor core has read them
    if (threadIdx.x == 0 && !wait_bar(su32(bar), phase)) {
      ok = false;
      wait_bar(su32(bar), phase);  // once more (bounded) before the memory is released
    }
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;");
    const long p = m0 + warp * 32 + lane;  // this thread's accumulator lane = pixel
    TY* Yb = Y + (long)b * ybs;
    for (int c0 = 0; c0 < NP; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
          "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (p < plane) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int co = c0 + c;
          if (co < Cout) {
            float v = __uint_as_float(r[c]) + (bias ? __ldg(&bias[co]) : 0.f);
            if (RELU) v = fmaxf(v, 0.f);
            st_out(Yb + (long)co * plane + p, v);
          }
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)tcols));
  }
}

template <typename TY, bool RELU>
cudaError_t launch(const __nv_bfloat16* X, long xbs, int Cin, const __nv_bfloat16* W, const float* bias, TY* Y,
                   long ybs, int Cout, int H, int Wd, int B, int* err, cudaStream_t st) {
  const int NP = (Cout + 15) / 16 * 16;
  if (NP > 256) return cudaErrorInvalidValue;
  int tcols = 32;
  while (tcols < NP) tcols *= 2;
  const size_t sm = (size_t)A_BYTES + (size_t)NP * CK * 2 + 64;
  cudaError_t e = cudaFuncSetAttribute(k_conv3x3_tc<TY, RELU>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long plane = (long)H * Wd;
  dim3 grid((unsigned)((plane + CM - 1) / CM), (unsigned)B);
  k_conv3x3_tc<TY, RELU><<<grid, CTHREADS, sm, st>>>(X, xbs, Cin, W, bias, Y, ybs, Cout, NP, tcols, H, Wd, err);
  return cudaGetLastError();
}

// Data gradient on the tensor cores: the adjoint of the convolution is the
// convolution with the transposed, flipped kernel,
//   dX[ci][q] = sum_co sum_t W[co][ci][8 - t] dY[co][q + o_t],
// so D = A B^T with A = dY_col (M = 128 pixels, k = co * 9 + t) and
// B[ci][k] = W[co][ci][8 - t] (N = up to 256 input channels per CTA,
// blockIdx.z tiles the rest).  dY is FP32 and enters as a hi + lo BF16 pair
// (two MMAs per step); dX is written (not accumulated), FP32.
__global__ void __launch_bounds__(CTHREADS) k_conv3x3_dgrad_tc(const float* __restrict__ dY, long dybs, int Cout,
                                                               const __nv_bfloat16* __restrict__ W,
                                                               float* __restrict__ dX, long dxbs, int Cin, int NP,
                                                               int tcols, int H, int Wd, int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* Ah = smem;                // 128 x 64 bf16
  uint8_t* Al = smem + A_BYTES;      // 128 x 64 bf16
  uint8_t* Bs = smem + 2 * A_BYTES;  // NP x 64 bf16
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + (size_t)NP * CK * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long plane = (long)H * Wd;
  const long m0 = (long)blockIdx.x * CM;
  const int b = blockIdx.y, ci0 = blockIdx.z * 256;
  const float* dYb = dY + (long)b * dybs;
  const int K = Cout * 9;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"((uint32_t)tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const uint32_t id = idesc_bf16(NP);
  const long pm = m0 + threadIdx.x;
  const bool pin = pm < plane;
  const int py = pin ? (int)(pm / Wd) : 0, px = pin ? (int)(pm % Wd) : 0;
  bool ok = true;
  uint32_t phase = 0;
  const int nslab = (K + CK - 1) / CK;
  for (int ks = 0; ks < nslab; ++ks) {
    const int k0 = ks * CK;
    for (int kk = 0; kk < CK; kk += 8) {
      __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + kk + e;
        float v = 0.f;
        if (pin && k < K) {
          const int co = k / 9, t = k - 9 * co;
          const int yy = py + t / 3 - 1, xx = px + t % 3 - 1;
          if (yy >= 0 && yy < H && xx >= 0 && xx < Wd) v = dYb[(long)co * plane + (long)yy * Wd + xx];
        }
        hi[e] = __float2bfloat16(v);
        lo[e] = __float2bfloat16(v - __bfloat162float(hi[e]));
      }
      *reinterpret_cast<uint4*>(Ah + kmaj(threadIdx.x, kk)) = *reinterpret_cast<const uint4*>(hi);
      *reinterpret_cast<uint4*>(Al + kmaj(threadIdx.x, kk)) = *reinterpret_cast<const uint4*>(lo);
    }
    for (int r = threadIdx.x; r < NP * (CK / 8); r += CTHREADS) {
      const int row = r / (CK / 8), kk = (r % (CK / 8)) * 8;
      const int ci = ci0 + row;
      __align__(16) __nv_bfloat16 v[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int k = k0 + kk + e;
        __nv_bfloat16 w = __float2bfloat16(0.f);
        if (ci < Cin && k < K) {
          const int co = k / 9, t = k - 9 * co;
          w = W[((long)co * Cin + ci) * 9 + (8 - t)];
        }
        v[e] = w;
      }
      *reinterpret_cast<uint4*>(Bs + kmaj(row, kk)) = *reinterpret_cast<const uint4*>(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int j = 0; j < CK / 16; ++j) {
        const uint32_t off = (uint32_t)j * 256;
        const uint64_t bd = sdesc(su32(Bs) + off);
        const uint32_t acc0 = (ks > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(sdesc(su32(Ah) + off)), "l"(bd), "r"(id), "r"(acc0));
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(sdesc(su32(Al) + off)), "l"(bd), "r"(id), "r"(1u));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                   : "memory");
    }
    if (threadIdx.x == 0 && !wait_bar(su32(bar), phase)) {
      ok = false;
      wait_bar(su32(bar), phase);  // once more (bounded) before the memory is released
    }
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;");
    const long p = m0 + warp * 32 + lane;
    float* dXb = dX + (long)b * dxbs;
    for (int c0 = 0; c0 < NP; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
          "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (p < plane) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int ci = ci0 + c0 + c;
          if (ci < Cin) dXb[(long)ci * plane + p] = __uint_as_float(r[c]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)tcols));
  }
}

// Weight and bias gradients on the tensor cores:
//   dW[co][k] += sum_q dY[co][q] X_col[k][q],  db[co] += sum_q dY[co][q],
// q over the pixels of one sample's chunk (blockIdx.z = sample * chunks +
// chunk), k = ci * 9 + t as in the forward pass.  D = A B^T with A = dY
// (M = 128 output channels per CTA, the pixels as the reduction axis, K-major)
// and B = X_col (N = NT taps per CTA).  dY is FP32: it enters as a hi + lo
// BF16 pair (two MMAs per step, 16 significant bits); X is BF16 already.  The
// CTA reduces its chunk in tensor memory and adds the tile to dW with FP32
// atomics.
constexpr int WCHUNK = 4096;  // pixels per CTA
__global__ void __launch_bounds__(CTHREADS) k_conv3x3_wgrad_tc(const float* __restrict__ dY, long dybs, int Cout,
                                                               const __nv_bfloat16* __restrict__ X, long xbs, int Cin,
                                                               int H, int Wd, int chunks, int NT, int tcols,
                                                               float* __restrict__ dW, float* __restrict__ db,
                                                               int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint8_t* Ah = smem;                  // 128 x 64 bf16
  uint8_t* Al = smem + A_BYTES;        // 128 x 64 bf16
  uint8_t* Bs = smem + 2 * A_BYTES;    // NT x 64 bf16
  uint64_t* bar = reinterpret_cast<uint64_t*>(Bs + (size_t)NT * CK * 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long plane = (long)H * Wd;
  const int K = Cin * 9;
  const int k0 = blockIdx.x * NT, co0 = blockIdx.y * CM;
  const int b = blockIdx.z / chunks, chunk = blockIdx.z % chunks;
  const long q0 = (long)chunk * WCHUNK;
  const long q1 = q0 + WCHUNK < plane ? q0 + WCHUNK : plane;
  const float* dYb = dY + (long)b * dybs;
  const __nv_bfloat16* Xb = X + (long)b * xbs;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"((uint32_t)tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tslot;
  const uint32_t id = idesc_bf16(NT);
  const int co = co0 + threadIdx.x;  // this thread's A row
  const bool bias = blockIdx.x == 0 && db != nullptr;  // the first tap tile's CTAs take db
  float bsum = 0.f;
  bool ok = true;
  uint32_t phase = 0;
  int ns = 0;
  for (long qs = q0; qs < q1; qs += CK, ++ns) {
    // A slabs: row threadIdx.x = channel co, 64 consecutive pixels, split hi / lo
    for (int kk = 0; kk < CK; kk += 8) {
      __align__(16) __nv_bfloat16 hi[8], lo[8];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const long q = qs + kk + e;
        const float v = (co < Cout && q < q1) ? dYb[(long)co * plane + q] : 0.f;
        bsum += v;
        hi[e] = __float2bfloat16(v);
        lo[e] = __float2bfloat16(v - __bfloat162float(hi[e]));
      }
      *reinterpret_cast<uint4*>(Ah + kmaj(threadIdx.x, kk)) = *reinterpret_cast<const uint4*>(hi);
      *reinterpret_cast<uint4*>(Al + kmaj(threadIdx.x, kk)) = *reinterpret_cast<const uint4*>(lo);
    }
    // B slab: NT taps x 64 pixels of the shifted input
    for (int r = threadIdx.x; r < NT * (CK / 8); r += CTHREADS) {
      const int kr = r / (CK / 8), kk = (r % (CK / 8)) * 8;
      const int k = k0 + kr;
      __align__(16) __nv_bfloat16 v[8];
      if (k < K) {
        const int ci = k / 9, t = k - 9 * ci, dy = t / 3 - 1, dx = t % 3 - 1;
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const long q = qs + kk + e;
          __nv_bfloat16 x = __float2bfloat16(0.f);
          if (q < q1) {
            const int py = (int)(q / Wd), px = (int)(q % Wd);
            const int yy = py + dy, xx = px + dx;
            if (yy >= 0 && yy < H && xx >= 0 && xx < Wd) x = Xb[(long)ci * plane + (long)yy * Wd + xx];
          }
          v[e] = x;
        }
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16(0.f);
      }
      *reinterpret_cast<uint4*>(Bs + kmaj(kr, kk)) = *reinterpret_cast<const uint4*>(v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll
      for (int j = 0; j < CK / 16; ++j) {
        const uint32_t off = (uint32_t)j * 256;
        const uint64_t bd = sdesc(su32(Bs) + off);
        const uint32_t acc0 = (ns > 0 || j > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(sdesc(su32(Ah) + off)), "l"(bd), "r"(id), "r"(acc0));
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
            "l"(sdesc(su32(Al) + off)), "l"(bd), "r"(id), "r"(1u));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
                   : "memory");
    }
    if (threadIdx.x == 0 && !wait_bar(su32(bar), phase)) {
      ok = false;
      wait_bar(su32(bar), phase);  // once more (bounded) before the memory is released
    }
    phase ^= 1u;
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
  }
  if (!ok) {
    if (threadIdx.x == 0) atomicExch(err, 1);
  } else if (ns > 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int row = co0 + warp * 32 + lane;  // accumulator lane = output channel
    for (int c0 = 0; c0 < NT; c0 += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
          "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < Cout) {
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int k = k0 + c0 + c;
          if (k < K) atomicAdd(&dW[(long)row * K + k], __uint_as_float(r[c]));
        }
      }
    }
    if (bias && co < Cout) atomicAdd(&db[co], bsum);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)tcols));
  }
}

}  // namespace

cudaError_t conv3x3_tc(const void* X, long xbs, int Cin, const void* W, const float* bias, void* Y, long ybs, int Cout,
                       int H, int Wd, int B, bool relu, bool y_fp32, int* err, cudaStream_t st) {
  const auto* x = static_cast<const __nv_bfloat16*>(X);
  const auto* w = static_cast<const __nv_bfloat16*>(W);
  if (y_fp32)
    return relu ? launch<float, true>(x, xbs, Cin, w, bias, static_cast<float*>(Y), ybs, Cout, H, Wd, B, err, st)
                : launch<float, false>(x, xbs, Cin, w, bias, static_cast<float*>(Y), ybs, Cout, H, Wd, B, err, st);
  auto* y = static_cast<__nv_bfloat16*>(Y);
  return relu ? launch<__nv_bfloat16, true>(x, xbs, Cin, w, bias, y, ybs, Cout, H, Wd, B, err, st)
              : launch<__nv_bfloat16, false>(x, xbs, Cin, w, bias, y, ybs, Cout, H, Wd, B, err, st);
}

}  // namespace gp

namespace gp {

cudaError_t conv3x3_wgrad_tc(const float* dY, long dybs, int Cout, const void* X, long xbs, int Cin, int H, int Wd,
                             int B, float* dW, float* db, int* err, cudaStream_t st) {
  const int K = Cin * 9;
  const int NT = K >= 256 ? 256 : (K + 15) / 16 * 16;
  int tcols = 32;
  while (tcols < NT) tcols *= 2;
  const long plane = (long)H * Wd;
  const int chunks = (int)((plane + WCHUNK - 1) / WCHUNK);
  const size_t sm = (size_t)2 * A_BYTES + (size_t)NT * CK * 2 + 64;
  const auto* x = static_cast<const __nv_bfloat16*>(X);
  dim3 grid((unsigned)((K + NT - 1) / NT), (unsigned)((Cout + CM - 1) / CM), (unsigned)(B * chunks));
  cudaError_t e = cudaFuncSetAttribute(k_conv3x3_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  k_conv3x3_wgrad_tc<<<grid, CTHREADS, sm, st>>>(dY, dybs, Cout, x, xbs, Cin, H, Wd, chunks, NT, tcols, dW, db, err);
  return cudaGetLastError();
}

}  // namespace gp

namespace gp {

cudaError_t conv3x3_dgrad_tc(const float* dY, long dybs, int Cout, const void* W, float* dX, long dxbs, int Cin,
                             int H, int Wd, int B, int* err, cudaStream_t st) {
  const int ntile = Cin < 256 ? Cin : 256;
  const int NP = (ntile + 15) / 16 * 16;
  int tcols = 32;
  while (tcols < NP) tcols *= 2;
  const size_t sm = (size_t)2 * A_BYTES + (size_t)NP * CK * 2 + 64;
  cudaError_t e = cudaFuncSetAttribute(k_conv3x3_dgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const long plane = (long)H * Wd;
  dim3 grid((unsigned)((plane + CM - 1) / CM), (unsigned)B, (unsigned)((Cin + 255) / 256));
  k_conv3x3_dgrad_tc<<<grid, CTHREADS, sm, st>>>(dY, dybs, Cout, static_cast<const __nv_bfloat16*>(W), dX, dxbs, Cin,
                                                 NP, tcols, H, Wd, err);
  return cudaGetLastError();
}

}  // namespace gp
