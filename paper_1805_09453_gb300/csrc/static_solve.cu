// dct2_poisson_static: the cosine-basis Helmholtz / Poisson solve of
// dct2_poisson for callers that cannot allocate device memory.
//
// Who needs it: code that may not call cudaMalloc -- a host framework that
// owns all device memory through its own pool and budget (a stray driver
// allocation would escape its accounting or fail once the pool has taken the
// memory), or a real-time loop in which an allocation and the device
// synchronisation it can cause are not allowed.  Such a caller passes only
// its input and output arrays; the solve's scratch and its transform tables
// live in the file-scope device arrays below.
//
// Costs and limits:
//  * every GPU that loads the library holds these arrays (4 MiB of scratch
//    plus ~16 KiB of tables) until the process exits;
//  * N must be a power of two in [16, kStaticMaxN]; larger or other sizes are
//    rejected with GP_ERR_ARG;
//  * all calls share the arrays, so calls that overlap on the GPU (different
//    streams, or different host threads) race and give wrong results.  No part
//    of the scratch needs to start at zero: every pass writes the whole region
//    a later pass reads; the tables are rewritten whenever N changes.
//  * a call made while its stream is capturing records the table kernel with
//    the solve, and from then on every call on that device rewrites the
//    tables too: a recorded call may later rewrite them at any time, so the
//    size they hold is no longer known on the host.
//  * the first call on a device looks up the arrays' device addresses
//    (cudaGetSymbolAddress, with that device current) and caches them; make
//    that first call before any stream capture.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include "gp_internal.cuh"

namespace {

constexpr int kStaticMaxN = 1024;
constexpr int kMaxDevices = 64;

// In host code these names are host-side stand-ins, not device addresses:
// the kernels are always given the addresses from cudaGetSymbolAddress.
static __device__ __align__(256) float g_scratch[kStaticMaxN * kStaticMaxN];
static __device__ __align__(256) float2 g_tw[kStaticMaxN];
static __device__ __align__(256) float2 g_wq[kStaticMaxN / 2 + 1];
static __device__ __align__(256) float g_mu[kStaticMaxN];

struct DeviceArrays {
  bool ready = false;
  int table_n = 0;        // size the tables currently hold (0: none)
  bool tables_shared = false;  // a stream capture recorded a table kernel: sizes no longer tracked
  float* scratch = nullptr;
  float2* tw = nullptr;
  float2* wq = nullptr;
  float* mu = nullptr;
};
DeviceArrays g_dev[kMaxDevices];

// Error text of the last failed handle-free call on this thread (fixed buffer:
// reporting an error allocates nothing either).
thread_local char g_err[256];

gp_status set_err(gp_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

// Transform tables of the fast solve for size N (same definitions as the
// handle's tables: e^{-2 pi i m/N}, e^{-i pi k/2N}, (4/h^2) sin^2(pi k/2N)).
__global__ void k_static_tables(float2* __restrict__ tw, float2* __restrict__ wq, float* __restrict__ mu, int N) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < N; m += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * m / N, &s, &c);
    tw[m] = make_float2((float)c, (float)-s);
    sincospi(m / (2.0 * N), &s, &c);
    mu[m] = (float)(4.0 * (double)N * (double)N * s * s);
    if (m <= N / 2) wq[m] = make_float2((float)c, (float)-s);
  }
}

bool device_ptr(const void* p, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeManaged || (a.type == cudaMemoryTypeDevice && a.device == dev);
}

}  // namespace

namespace gp {
const char* static_last_error() { return g_err; }
}  // namespace gp

extern "C" GP_API gp_status dct2_poisson_static(const float* b, float* x, int N, double alpha, void* stream) {
  g_err[0] = '\0';
  if (N < 16 || N > kStaticMaxN || (N & (N - 1)) != 0)
    return set_err(GP_ERR_ARG, "dct2_poisson_static: N = %d; it takes power-of-two N in [16, %d] (static scratch of %d^2 floats)",
                   N, kStaticMaxN, kStaticMaxN);
  if (!(alpha >= 0.0) || !isfinite(alpha)) return set_err(GP_ERR_ARG, "dct2_poisson_static: alpha must be finite and >= 0");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return set_err(GP_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return set_err(GP_ERR_ARG, "dct2_poisson_static: device %d beyond %d", dev, kMaxDevices);
  if (!b || !x || !device_ptr(b, dev) || !device_ptr(x, dev))
    return set_err(GP_ERR_ARG, "dct2_poisson_static: b and x must be device pointers of the current device");
  if (((uintptr_t)b & 15u) || ((uintptr_t)x & 15u))
    return set_err(GP_ERR_ARG, "dct2_poisson_static: b and x must be 16-byte aligned");
  DeviceArrays& D = g_dev[dev];
  if (!D.ready) {
    // once per device, with that device current: device addresses of the arrays
    if ((e = cudaGetSymbolAddress((void**)&D.scratch, g_scratch)) != cudaSuccess ||
        (e = cudaGetSymbolAddress((void**)&D.tw, g_tw)) != cudaSuccess ||
        (e = cudaGetSymbolAddress((void**)&D.wq, g_wq)) != cudaSuccess ||
        (e = cudaGetSymbolAddress((void**)&D.mu, g_mu)) != cudaSuccess)
      return set_err(GP_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    D.ready = true;
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if ((e = cudaStreamIsCapturing(st, &cs)) != cudaSuccess)
    return set_err(GP_ERR_CUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
  if (cs != cudaStreamCaptureStatusNone) D.tables_shared = true;
  if (D.tables_shared || D.table_n != N) {
    k_static_tables<<<(N + 255) / 256, 256, 0, st>>>(D.tw, D.wq, D.mu, N);
    if ((e = cudaGetLastError()) != cudaSuccess) return set_err(GP_ERR_CUDA, "table kernel: %s", cudaGetErrorString(e));
    D.table_n = D.tables_shared ? 0 : N;
  }
  gp::DctPlan p;
  p.N = N;
  p.fft = true;
  p.tw = D.tw;
  p.wq = D.wq;
  p.mu = D.mu;
  const float a = (float)alpha;
  if ((e = gp::dct_fft_pass(p, 0, b, D.scratch, a, 1.f, st)) != cudaSuccess ||
      (e = gp::dct_fft_pass(p, 1, D.scratch, D.scratch, a, 1.f, st)) != cudaSuccess ||
      (e = gp::dct_fft_pass(p, 2, D.scratch, x, a, 1.f, st)) != cudaSuccess)
    return set_err(GP_ERR_CUDA, "dct2_poisson_static: %s", cudaGetErrorString(e));
  return GP_OK;
}
