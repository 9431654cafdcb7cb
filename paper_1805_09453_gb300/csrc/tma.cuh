// Bulk tensor copies (TMA) and mbarrier waits shared by the transform passes.
#pragma once

#include <cuda.h>  // CUtensorMap (the encoder is reached through the runtime's driver entry point)
#include <cuda_runtime.h>
#include <stdint.h>

namespace gp {

// Tensor map of an interleaved-spectra plane (rows in blocks of 4, each block
// stored column by column) seen as {4 rows, N columns, N/4 row blocks}
// (strides 16 B and 16N B), box {4, ncols, min(256, N/4)}; false when the
// driver's encoder is unavailable or refuses, or base is not 16-byte aligned.
bool encode_b4_map(CUtensorMap* m, const float* base, int N, int ncols);

// Tensor map of a pair-interleaved plane (rows 2q, 2q + 1 stored as N float2
// per row pair) seen as {4 floats, N/2 column pairs, N/2 row pairs} (strides
// 16 B and 8N B), box {4, 1, 256}; false as encode_b4_map.
bool encode_pairs_map(CUtensorMap* m, const float* base, int N);

namespace {

constexpr uint32_t kTmaWaitLimit = 1u << 22;  // try_wait rounds before a copy is declared lost

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Bounded wait on phase `parity` of the mbarrier at shared address `bar`:
// false if the phase did not complete within kTmaWaitLimit polls.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  for (uint32_t it = 0; it < kTmaWaitLimit; ++it) {
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

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void tma_store_3d(const CUtensorMap* tm, int c0, int c1, int c2, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.tile.bulk_group [%0, {%1, %2, %3}], [%4];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(c0), "r"(c1), "r"(c2), "r"(src)
               : "memory");
}

}  // namespace
}  // namespace gp
