// Split-precision cosine-transform solve on the 5th-generation tensor cores.
//
// The dense form of the Neumann solve (Appendix A cosine basis),
//     x = C^T [ (C b C^T) / (alpha + mu_k + mu_l) ] C,   C = orthonormal DCT-II,
// is four N x N x N contractions.  Each runs as a tcgen05 GEMM whose FP32
// operands are split on the fly into a high and a low 16-bit part,
// x = x_hi + x_lo (x_hi = bf16(x), x_lo = bf16(x - x_hi)), and
//     A B^T ~= A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T
// is accumulated in FP32 in tensor memory (the dropped A_lo B_lo^T term is
// ~2^-16 relative; BF16 keeps FP32's exponent range, so no operand scaling
// is needed).  One CTA (256 threads) computes a 128 x 128 tile.  Operands
// come either as FP32 (loaded and split by the threads) or pre-split into
// 128 x 64 tiles of the canonical K-major layout without swizzle (the
// constant cosine / derivative matrices, split once per plan, and every
// intermediate product, which the epilogue writes in that form), copied by
// the bulk-copy engine.  The K loop runs over three shared-memory stages: the
// next slab's copies are in flight while the tensor core multiplies the
// current one; one thread issues the tcgen05.mma instructions, and
// tcgen05.commit signals the stage's mbarrier when they have read it.  The
// epilogue moves the accumulator out of tensor memory with tcgen05.ld (a warp
// reads its lane quadrant, two warps share the columns), applies the spectral
// gain when asked, and stores the tile (FP32 or split), transposed when asked,
// so
// that every operand of the next GEMM is again K-major:
//     G1: T1^T <- (b C^T)^T      G2: T2^T <- (gain .* (C T1))^T
//     G3: T3   <- C^T T2         G4: x    <- T3 C
// Every wait on an mbarrier is bounded; a timeout sets an error flag, waits
// (bounded) for the tensor core, frees the tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <algorithm>

#include "gp_internal.cuh"

namespace gp {
namespace {

constexpr int BM = 128, BN = 128, BK = 64;
constexpr int TILE_BYTES = BM * BK * 2;  // one 16-bit operand slab, 16 KiB
constexpr int STAGES = 3;                // shared-memory stages (a_hi, a_lo, b_hi, b_lo each)
constexpr int THREADS = 256;
constexpr int SMEM_BYTES = STAGES * 4 * TILE_BYTES + 128;  // stages, 2 x STAGES mbarriers, TMEM slot
constexpr uint32_t kWaitLimit = 1u << 22;  // try_wait rounds before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Canonical K-major layout without swizzle: 8 x 8 core matrices of 16-bit
// elements (8 rows x 16 bytes); core matrices adjacent along K are LBO = 128 B
// apart, adjacent along M/N are SBO = 1024 B apart.
__device__ __forceinline__ uint32_t kmajor_offset(int row, int k) {
  return (uint32_t)((row >> 3) * 1024 + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  const uint64_t lbo = 128, sbo = 1024;
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((lbo >> 4) << 16) | ((sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor: D = F32, A = B = BF16 (or F16), both K-major, M = 128, N = 128.
template <bool BF16>
__device__ __forceinline__ uint32_t instr_desc() {
  const uint32_t ab = BF16 ? 1u : 0u;
  return (1u << 4) | (ab << 7) | (ab << 10) | ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t limit) {
  for (uint32_t it = 0; it < limit; ++it) {
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

template <bool BF16>
__device__ __forceinline__ void split4(float4 v, uint2& hi, uint2& lo) {
  if constexpr (BF16) {
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
    const __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
    const __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
    hi = make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
    lo = make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
  } else {
    const __half2 h01 = __floats2half2_rn(v.x, v.y), h23 = __floats2half2_rn(v.z, v.w);
    const float2 f01 = __half22float2(h01), f23 = __half22float2(h23);
    const __half2 l01 = __floats2half2_rn(v.x - f01.x, v.y - f01.y);
    const __half2 l23 = __floats2half2_rn(v.z - f23.x, v.w - f23.y);
    hi = make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
    lo = make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
  }
}

// Load a 128 x 64 FP32 slab (rows r0.., columns k0.. of a row-major matrix with
// leading dimension ld), multiplied by `s`, split into hi / lo 16-bit slabs.
template <bool BF16>
__device__ __forceinline__ void load_split(const float* __restrict__ src, int ld, int r0, int k0, float s,
                                           uint8_t* hi, uint8_t* lo) {
  // 128 rows x 16 float4 = 2048 float4, 16 consecutive threads per row
#pragma unroll 4
  for (int idx = threadIdx.x; idx < BM * (BK / 4); idx += THREADS) {
    const int row = idx >> 4, q = idx & 15;
    float4 v = *reinterpret_cast<const float4*>(src + (size_t)(r0 + row) * ld + k0 + 4 * q);
    v.x *= s;
    v.y *= s;
    v.z *= s;
    v.w *= s;
    uint2 h, l;
    split4<BF16>(v, h, l);
    const uint32_t off = kmajor_offset(row, 4 * q);
    *reinterpret_cast<uint2*>(hi + off) = h;
    *reinterpret_cast<uint2*>(lo + off) = l;
  }
}

// The bulk-copy engine brings pre-split tiles (hi slab then lo slab,
// 2 x TILE_BYTES) into shared memory; the mbarrier counts the bytes.
__device__ __forceinline__ void expect_bytes(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_tile(uint32_t dst, const void* src, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"((uint32_t)(2 * TILE_BYTES)), "r"(bar)
               : "memory");
}

// Byte offset of tile (row block rb, K block kb) of an N x N operand in the
// pre-split layout: 128 x 64 tiles, row blocks outermost, hi then lo slab.
__host__ __device__ __forceinline__ size_t split_tile_offset(int rb, int kb, int N) {
  return ((size_t)rb * (size_t)(N / BK) + (size_t)kb) * (size_t)(2 * TILE_BYTES);
}

// M (N x N, row-major FP32) -> pre-split tiles of s M.  One thread per 4
// consecutive elements of a row.  BF16 keeps FP32's exponent range: s = 1.
// FP16 (5 exponent bits) takes a power of two from the largest |M| (amax,
// written by an earlier kernel): with amax = f 2^e, f in [0.5, 1),
// s = 2^(14 - e) puts |s M| below 2^14, far inside FP16's range, and keeps the
// low parts normal down to 2^-17 of the largest entry (smaller entries keep
// an absolute error below 2^-38 of it).  *scale_out receives s.
template <bool BF16>
__global__ void k_split_tiles(const float* __restrict__ M, uint8_t* __restrict__ out, int N,
                              const unsigned* __restrict__ amax, float* __restrict__ scale_out) {
  float sc = 1.f;
  if (!BF16 && amax) {
    const float a = __uint_as_float(__ldg(amax));
    if (a > 0.f && a <= 3.0e38f) {
      int e;
      frexpf(a, &e);
      sc = ldexpf(1.f, 14 - e);
    }
  }
  if (scale_out && blockIdx.x == 0 && threadIdx.x == 0) *scale_out = sc;
  const long n4 = (long)N * N / 4;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n4; i += (long)gridDim.x * blockDim.x) {
    const int r = (int)(i / (N / 4)), k = (int)(i % (N / 4)) * 4;
    float4 v = *reinterpret_cast<const float4*>(M + (size_t)r * N + k);
    v.x *= sc;
    v.y *= sc;
    v.z *= sc;
    v.w *= sc;
    uint2 h, l;
    split4<BF16>(v, h, l);
    uint8_t* tile = out + split_tile_offset(r / BM, k / BK, N);
    const uint32_t off = kmajor_offset(r % BM, k % BK);
    *reinterpret_cast<uint2*>(tile + off) = h;
    *reinterpret_cast<uint2*>(tile + TILE_BYTES + off) = l;
  }
}

// *amax = max(*amax, max |x|) over n floats (non-negative floats order as integers).
__global__ void k_amax(const float* __restrict__ x, size_t n, unsigned* __restrict__ amax) {
  float m = 0.f;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax, __float_as_uint(m));
}

// D(m0.., n0..) = epi( A(m0.., :) B(n0.., :)^T ), A: M x K, B: Nc x K, both
// row-major (K-major) FP32.  mode 0: D[m][n] stored; 1: D^T stored (D[n][m]).
// gain (mu != nullptr): D[m][n] *= gscale / (alpha + mu[m] + mu[n]), 0 when
// the denominator is 0.  Operand scales sa, sb are undone in the epilogue.
// PRE bit 0 (1): A (B) comes pre-split (k_split_tiles layout, pointer As / Bs)
// and is copied by the bulk-copy engine; an operand without its bit is loaded
// and split by the threads.  OSPLIT: the epilogue writes D (or D^T) as
// pre-split tiles for the next product instead of FP32.
template <bool BF16, int PRE, bool OSPLIT>
__global__ void __launch_bounds__(THREADS) k_tc_gemm_split(const float* __restrict__ A, const float* __restrict__ B,
                                                           const uint8_t* __restrict__ As,
                                                           const uint8_t* __restrict__ Bs, float* __restrict__ D,
                                                           int Nn, int K, int mode, const float* __restrict__ mu,
                                                           float alpha, float gscale, const float* __restrict__ sap,
                                                           const float* __restrict__ sbp, unsigned* __restrict__ amax,
                                                           int* __restrict__ err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + STAGES * 4 * TILE_BYTES);  // per stage: MMAs done
  uint64_t* full = bar + STAGES;                                                 // per stage: bulk copy landed
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem + STAGES * 4 * TILE_BYTES + 64);
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int st = 0; st < 2 * STAGES; ++st)
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar + st)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = instr_desc<BF16>();
  const float sa = sap ? __ldg(sap) : 1.f, sb = sbp ? __ldg(sbp) : 1.f;
  bool ok = true;
  uint32_t phase[STAGES], fphase[STAGES];  // parity of each stage's next MMA / bulk-copy completion
#pragma unroll
  for (int i = 0; i < STAGES; ++i) phase[i] = fphase[i] = 0u;
  int last = -1;  // stage of the last committed tile
  const int nk = K / BK;
  auto stage_ptr = [&](int st) { return smem + st * 4 * TILE_BYTES; };
  // bulk copies of tile kt's pre-split operands into stage kt % STAGES (thread 0)
  auto prefetch = [&](int kt) {
    if (PRE == 0 || threadIdx.x != 0) return;
    const int st = kt % STAGES;
    uint8_t* a_hi = stage_ptr(st);
    expect_bytes(smem_u32(full + st), (uint32_t)((PRE == 3 ? 2 : 1) * 2 * TILE_BYTES));
    if (PRE & 1) bulk_tile(smem_u32(a_hi), As + split_tile_offset(m0 / BM, kt, K), smem_u32(full + st));
    if (PRE & 2) bulk_tile(smem_u32(a_hi + 2 * TILE_BYTES), Bs + split_tile_offset(n0 / BN, kt, K), smem_u32(full + st));
  };
  // Pipeline over STAGES stages: iteration kt first frees the stage of tile
  // kt + 1 (its previous user, tile kt + 1 - STAGES, committed two iterations
  // ago) and starts that tile's bulk copies, then fills the thread-split
  // operand of tile kt, waits for tile kt's copies and issues its MMAs; the
  // tensor core works on tile kt while tile kt + 1 is in flight.
  prefetch(0);
  for (int kt = 0; kt < nk; ++kt) {
    const int st = kt % STAGES;
    uint8_t* a_hi = stage_ptr(st);
    uint8_t* a_lo = a_hi + TILE_BYTES;
    uint8_t* b_hi = a_hi + 2 * TILE_BYTES;
    uint8_t* b_lo = a_hi + 3 * TILE_BYTES;
    if (kt + 1 < nk) {
      const int sn = (kt + 1) % STAGES;
      if (kt + 1 >= STAGES) {
        if (!mbar_wait(smem_u32(bar + sn), phase[sn], kWaitLimit)) ok = false;
        phase[sn] ^= 1u;
      }
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
      prefetch(kt + 1);
    }
    if (!(PRE & 1)) load_split<BF16>(A, K, m0, kt * BK, sa, a_hi, a_lo);
    if (!(PRE & 2)) load_split<BF16>(B, K, n0, kt * BK, sb, b_hi, b_lo);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (PRE != 0 && threadIdx.x == 0) {
      if (!mbar_wait(smem_u32(full + st), fphase[st], kWaitLimit)) ok = false;
      fphase[st] ^= 1u;
    }
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;");
      const uint32_t ah = smem_u32(a_hi), al = smem_u32(a_lo), bh = smem_u32(b_hi), bl = smem_u32(b_lo);
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint32_t off = (uint32_t)kk * 256;  // 16 elements along K = two core matrices
        mma_f16(tmem, smem_desc(ah + off), smem_desc(bh + off), idesc, (kt > 0 || kk > 0) ? 1u : 0u);
        mma_f16(tmem, smem_desc(ah + off), smem_desc(bl + off), idesc, 1u);
        mma_f16(tmem, smem_desc(al + off), smem_desc(bh + off), idesc, 1u);
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(bar + st))
                   : "memory");
    }
    last = st;
  }
  // the last commit arrives when every MMA issued before it has completed
  if (ok && last >= 0) {
    if (!mbar_wait(smem_u32(bar + last), phase[last], kWaitLimit)) ok = false;
  }
  if (!__syncthreads_and(ok)) {
    if (threadIdx.x == 0) atomicExch(err, 1);
    // let the tensor core finish (bounded) before the memory is released
    if (last >= 0) mbar_wait(smem_u32(bar + last), phase[last], kWaitLimit);
    __syncthreads();
  } else {
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int quad = warp & 3;            // a warp reads the tensor-memory lanes of its quadrant
    const int m = m0 + quad * 32 + lane;  // this thread's accumulator row
    const float inv = 1.f / (sa * sb);  // powers of two: exact
    const float mum = mu ? __ldg(&mu[m]) : 0.f;
    float vmax = 0.f;
#pragma unroll 1
    for (int c0 = (warp >> 2) * (BN / 2); c0 < (warp >> 2) * (BN / 2) + BN / 2; c0 += 32) {
      uint32_t r[32];
      const uint32_t taddr = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
          "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
            "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]),
            "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
            "=r"(r[30]), "=r"(r[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      float v[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        float x = __uint_as_float(r[c]) * inv;
        if (mu) {
          const float den = alpha + mum + __ldg(&mu[n0 + c0 + c]);
          x = den > 0.f ? x * (gscale / den) : 0.f;
        }
        v[c] = x;
        vmax = fmaxf(vmax, fabsf(x));
      }
      if constexpr (OSPLIT) {
        uint8_t* Ds = reinterpret_cast<uint8_t*>(D);
        if (mode == 0) {  // operand row m, K index n: four consecutive K per 8-byte store
#pragma unroll
          for (int c = 0; c < 32; c += 4) {
            const int n = n0 + c0 + c;
            uint2 hv, lv;
            split4<BF16>(make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]), hv, lv);
            uint8_t* tile = Ds + split_tile_offset(m / BM, n / BK, Nn);
            const uint32_t off = kmajor_offset(m % BM, n % BK);
            *reinterpret_cast<uint2*>(tile + off) = hv;
            *reinterpret_cast<uint2*>(tile + TILE_BYTES + off) = lv;
          }
        } else {  // D^T: operand row n, K index m (consecutive across the warp's lanes)
#pragma unroll
          for (int c = 0; c < 32; ++c) {
            const int n = n0 + c0 + c;
            const __nv_bfloat16 hi = __float2bfloat16_rn(v[c]);
            const __nv_bfloat16 lo = __float2bfloat16_rn(v[c] - __bfloat162float(hi));
            uint8_t* tile = Ds + split_tile_offset(n / BM, m / BK, Nn);
            const uint32_t off = kmajor_offset(n % BM, m % BK);
            *reinterpret_cast<__nv_bfloat16*>(tile + off) = hi;
            *reinterpret_cast<__nv_bfloat16*>(tile + TILE_BYTES + off) = lo;
          }
        }
      } else if (mode == 0) {
        float* row = D + (size_t)m * Nn + n0 + c0;
#pragma unroll
        for (int c = 0; c < 32; c += 4) *reinterpret_cast<float4*>(row + c) = make_float4(v[c], v[c + 1], v[c + 2], v[c + 3]);
      } else {
#pragma unroll
        for (int c = 0; c < 32; ++c) D[(size_t)(n0 + c0 + c) * Nn + m] = v[c];
      }
    }
    if (amax) {  // max |D| for the power-of-two scale of the next split (non-negative floats order as integers)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
      if (lane == 0) atomicMax(amax, __float_as_uint(vmax));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN));
  }
}

template <bool BF16, int PRE, bool OSPLIT>
cudaError_t gemm_launch(const float* A, const float* B, const void* As, const void* Bs, void* D, int N, int mode,
                        const float* mu, float alpha, float gscale, const float* sap, const float* sbp,
                        unsigned* amax, int* err, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_tc_gemm_split<BF16, PRE, OSPLIT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
  if (e != cudaSuccess) return e;
  dim3 grid(N / BN, N / BM);
  k_tc_gemm_split<BF16, PRE, OSPLIT><<<grid, THREADS, SMEM_BYTES, st>>>(
      A, B, (const uint8_t*)As, (const uint8_t*)Bs, (float*)D, N, N, mode, mu, alpha, gscale, sap, sbp, amax, err);
  return cudaGetLastError();
}

// An operand of a product: FP32 (split on the fly) or pre-split tiles with
// their scale (device pointer; nullptr = 1).
struct Op {
  const float* f = nullptr;
  const void* s = nullptr;
  const float* sc = nullptr;
};
inline Op pre(const void* s, const float* sc = nullptr) { return Op{nullptr, s, sc}; }

// D (FP32, or pre-split tiles when dsplit) = epi(A B^T); amax (FP32 output
// only, may be nullptr) collects max |D|.
template <bool BF16>
cudaError_t gemm(Op A, Op B, void* D, bool dsplit, int N, int mode, const float* mu, float alpha, float gscale,
                 int* err, cudaStream_t st, unsigned* amax = nullptr) {
  const int pre_mask = (A.s ? 1 : 0) | (B.s ? 2 : 0);
#define GP_G(P)                                                                                                \
  return dsplit ? gemm_launch<BF16, P, true>(A.f, B.f, A.s, B.s, D, N, mode, mu, alpha, gscale, A.sc, B.sc,  \
                                              nullptr, err, st)                                                \
                : gemm_launch<BF16, P, false>(A.f, B.f, A.s, B.s, D, N, mode, mu, alpha, gscale, A.sc, B.sc, \
                                              amax, err, st)
  switch (pre_mask) {
    case 1: GP_G(1);
    case 2: GP_G(2);
    case 3: GP_G(3);
    default: GP_G(0);
  }
#undef GP_G
}

int split_blocks(int N) { return (int)std::min<long>(((long)N * N / 4 + 255) / 256, 8192); }

// FP32 M -> pre-split tiles (FP16: scaled by the power of two of *amax, stored in *scale_out).
template <bool BF16>
cudaError_t split(const float* M, void* out, int N, const unsigned* amax, float* scale_out, cudaStream_t st) {
  k_split_tiles<BF16><<<split_blocks(N), 256, 0, st>>>(M, (uint8_t*)out, N, amax, scale_out);
  return cudaGetLastError();
}

cudaError_t amax_of(const float* x, size_t n, unsigned* amax, cudaStream_t st) {
  const size_t b = (n + 255) / 256;
  k_amax<<<(unsigned)(b < 4096 ? b : 4096), 256, 0, st>>>(x, n, amax);
  return cudaGetLastError();
}

// Scale and max slots of the FP16 mode (DctPlan::tc16): scales at [i], maxima
// at [kAmax + i]: 0 b, 1..5 the intermediate products, 8 C / C^T, 9 E / E^T.
constexpr int kAmax = 16, kSlotC = 8, kSlotE = 9, kTc16Floats = 32;

}  // namespace

bool tc_solve_supported(int N) { return N >= 128 && N <= 8192 && N % 128 == 0; }

cudaError_t dct_plan_tc_split(DctPlan& p, cudaStream_t st, bool fp16) {
  const int N = p.N;
  const size_t bytes = (size_t)N * N * 4;
  const float* src[4] = {p.C, p.CT, p.E, p.ET};
  cudaError_t e;
  if (!fp16) {
    void** dst[4] = {&p.Cs, &p.CTs, &p.Es, &p.ETs};
    for (int i = 0; i < 4; ++i) {
      if (!src[i] || *dst[i]) continue;
      if ((e = cudaMalloc(dst[i], bytes))) return e;
      if ((e = split<true>(src[i], *dst[i], N, nullptr, nullptr, st))) return e;
    }
    return cudaSuccess;
  }
  if (!p.tc16) {
    if ((e = cudaMalloc(&p.tc16, kTc16Floats * sizeof(float)))) return e;
    if ((e = cudaMemsetAsync(p.tc16, 0, kTc16Floats * sizeof(float), st))) return e;
  }
  unsigned* am = reinterpret_cast<unsigned*>(p.tc16 + kAmax);
  void** dst[4] = {&p.Cs16, &p.CTs16, &p.Es16, &p.ETs16};
  const int slot[4] = {kSlotC, kSlotC, kSlotE, kSlotE};  // a matrix and its transpose share the maximum
  for (int i = 0; i < 4; ++i) {
    if (!src[i] || *dst[i]) continue;
    if ((e = cudaMalloc(dst[i], bytes))) return e;
    if ((e = amax_of(src[i], (size_t)N * N, am + slot[i], st))) return e;
    if ((e = split<false>(src[i], *dst[i], N, am + slot[i], p.tc16 + slot[i], st))) return e;
  }
  return cudaSuccess;
}

cudaError_t dct_solve_tc(const DctPlan& p, const float* b, float* x, float* tmp, float alpha, float scale, int* err,
                         cudaStream_t st, bool fp16) {
  const int N = p.N;
  if (!tc_solve_supported(N)) return cudaErrorInvalidValue;
  // intermediates are stored as pre-split tiles (4 bytes per element, as FP32)
  void* t0 = tmp;
  void* t1 = tmp + (size_t)N * N;
  cudaError_t e;
  if (!fp16) {
    if (!p.Cs || !p.CTs) return cudaErrorInvalidValue;
    if ((e = split<true>(b, t1, N, nullptr, nullptr, st))) return e;                                     // t1 = split(b)
    if ((e = gemm<true>(pre(t1), pre(p.Cs), t0, true, N, 1, nullptr, alpha, scale, err, st))) return e;  // T1^T = (b C^T)^T
    if ((e = gemm<true>(pre(p.Cs), pre(t0), t1, true, N, 1, p.mu, alpha, scale, err, st))) return e;   // T2^T = (gain .* C T1)^T
    if ((e = gemm<true>(pre(p.CTs), pre(t1), t0, true, N, 0, nullptr, alpha, scale, err, st))) return e;  // T3 = C^T T2
    return gemm<true>(pre(t0), pre(p.CTs), x, false, N, 0, nullptr, alpha, scale, err, st);            // x = T3 C
  }
  // FP16: each product is written in FP32 (x serves as the staging plane: b
  // is consumed first) with its max |.|, then split with its own scale
  if (!p.Cs16 || !p.CTs16 || !p.tc16) return cudaErrorInvalidValue;
  float* sc = p.tc16;
  unsigned* am = reinterpret_cast<unsigned*>(p.tc16 + kAmax);
  const float* sC = sc + kSlotC;
  if ((e = cudaMemsetAsync(am, 0, 8 * sizeof(unsigned), st))) return e;
  if ((e = amax_of(b, (size_t)N * N, am, st))) return e;
  if ((e = split<false>(b, t1, N, am, sc, st))) return e;
  if ((e = gemm<false>(pre(t1, sc), pre(p.Cs16, sC), x, false, N, 1, nullptr, alpha, scale, err, st, am + 1))) return e;
  if ((e = split<false>(x, t0, N, am + 1, sc + 1, st))) return e;
  if ((e = gemm<false>(pre(p.Cs16, sC), pre(t0, sc + 1), x, false, N, 1, p.mu, alpha, scale, err, st, am + 2))) return e;
  if ((e = split<false>(x, t1, N, am + 2, sc + 2, st))) return e;
  if ((e = gemm<false>(pre(p.CTs16, sC), pre(t1, sc + 2), x, false, N, 0, nullptr, alpha, scale, err, st, am + 3)))
    return e;
  if ((e = split<false>(x, t0, N, am + 3, sc + 3, st))) return e;
  return gemm<false>(pre(t0, sc + 3), pre(p.CTs16, sC), x, false, N, 0, nullptr, alpha, scale, err, st);
}

// Spectral gradient in the split-precision mode (the forward differences of
// the solution synthesised from its spectrum, as the FP32 path does, so that
// the solve's error is not amplified by 1/h):
//   X = C b^T,  Q = gain .* (C X^T) (and Q^T),  U = C^T Q,
//   gx = U E,  phi = U C (optional),  V^T = (Q C)^T,  gy = E^T V.
// X, Z = tmp; Q lives in gy until the last product; intermediates are
// pre-split tiles (FP16: staged in FP32 in gx, then in X, and split with
// their own scales).
cudaError_t dct_grad_tc(const DctPlan& p, const float* b, float* gx, float* gy, float* phi, float* tmp, float alpha,
                        float scale, int* err, cudaStream_t st, bool fp16) {
  const int N = p.N;
  if (!tc_solve_supported(N)) return cudaErrorInvalidValue;
  void* X = tmp;
  void* Z = tmp + (size_t)N * N;
  void* Q = gy;
  cudaError_t e;
  if (!fp16) {
    if (!p.Cs || !p.CTs || !p.ETs) return cudaErrorInvalidValue;
    if ((e = split<true>(b, Z, N, nullptr, nullptr, st))) return e;                                        // Z = split(b)
    if ((e = gemm<true>(pre(Z), pre(p.Cs), X, true, N, 1, nullptr, alpha, scale, err, st))) return e;      // X = C b^T
    if ((e = gemm<true>(pre(p.Cs), pre(X), Q, true, N, 0, p.mu, alpha, scale, err, st))) return e;        // Q
    if ((e = gemm<true>(pre(p.Cs), pre(X), Z, true, N, 1, p.mu, alpha, scale, err, st))) return e;        // Z = Q^T
    if ((e = gemm<true>(pre(p.CTs), pre(Z), X, true, N, 0, nullptr, alpha, scale, err, st))) return e;    // X = U = C^T Q
    if ((e = gemm<true>(pre(X), pre(p.ETs), gx, false, N, 0, nullptr, alpha, scale, err, st))) return e;  // gx = U E
    if (phi && (e = gemm<true>(pre(X), pre(p.CTs), phi, false, N, 0, nullptr, alpha, scale, err, st)))
      return e;                                                                                            // phi = U C
    if ((e = gemm<true>(pre(Q), pre(p.CTs), Z, true, N, 1, nullptr, alpha, scale, err, st))) return e;    // Z = (Q C)^T
    return gemm<true>(pre(p.ETs), pre(Z), gy, false, N, 0, nullptr, alpha, scale, err, st);               // gy = E^T V
  }
  if (!p.Cs16 || !p.CTs16 || !p.ETs16 || !p.tc16) return cudaErrorInvalidValue;
  float* sc = p.tc16;
  unsigned* am = reinterpret_cast<unsigned*>(p.tc16 + kAmax);
  const float* sC = sc + kSlotC;
  const float* sE = sc + kSlotE;
  float* F = gx;  // FP32 staging until gx is written
  if ((e = cudaMemsetAsync(am, 0, 8 * sizeof(unsigned), st))) return e;
  if ((e = amax_of(b, (size_t)N * N, am, st))) return e;
  if ((e = split<false>(b, Z, N, am, sc, st))) return e;
  if ((e = gemm<false>(pre(Z, sc), pre(p.Cs16, sC), F, false, N, 1, nullptr, alpha, scale, err, st, am + 1))) return e;
  if ((e = split<false>(F, X, N, am + 1, sc + 1, st))) return e;                                         // X
  if ((e = gemm<false>(pre(p.Cs16, sC), pre(X, sc + 1), F, false, N, 0, p.mu, alpha, scale, err, st, am + 2))) return e;
  if ((e = split<false>(F, Q, N, am + 2, sc + 2, st))) return e;                                         // Q
  if ((e = gemm<false>(pre(p.Cs16, sC), pre(X, sc + 1), F, false, N, 1, p.mu, alpha, scale, err, st, am + 3))) return e;
  if ((e = split<false>(F, Z, N, am + 3, sc + 3, st))) return e;                                         // Z = Q^T
  if ((e = gemm<false>(pre(p.CTs16, sC), pre(Z, sc + 3), F, false, N, 0, nullptr, alpha, scale, err, st, am + 4)))
    return e;
  if ((e = split<false>(F, X, N, am + 4, sc + 4, st))) return e;                                         // X = U
  if ((e = gemm<false>(pre(X, sc + 4), pre(p.ETs16, sE), gx, false, N, 0, nullptr, alpha, scale, err, st))) return e;
  if (phi && (e = gemm<false>(pre(X, sc + 4), pre(p.CTs16, sC), phi, false, N, 0, nullptr, alpha, scale, err, st)))
    return e;
  float* G = reinterpret_cast<float*>(X);  // U is consumed: X stages (Q C)^T
  if ((e = gemm<false>(pre(Q, sc + 2), pre(p.CTs16, sC), G, false, N, 1, nullptr, alpha, scale, err, st, am + 5)))
    return e;
  if ((e = split<false>(G, Z, N, am + 5, sc + 5, st))) return e;                                         // Z = (Q C)^T
  return gemm<false>(pre(p.ETs16, sE), pre(Z, sc + 5), gy, false, N, 0, nullptr, alpha, scale, err, st);  // gy = E^T V
}

}  // namespace gp
