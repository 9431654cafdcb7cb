// Complex helpers and the in-register small DFT shared by the transform
// kernels (dct.cu: shared-memory Stockham passes; fftreg.cu: register-resident
// passes).
#pragma once

#include <cuda_runtime.h>

namespace gp {
namespace {

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

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

}  // namespace
}  // namespace gp
