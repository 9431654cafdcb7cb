// C ABI of the library: handles, solver states, the solve loops and the
// duality-gap stopping test.  All device work is issued on the caller's
// stream; the host synchronises only when it needs the gap scalars.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <string>
#include <tuple>
#include <utility>
#include <vector>

#include "gp_internal.cuh"
#include "stencil.cuh"

using namespace gp;

enum { KIND_ROF = 1, KIND_EMD = 2 };

// Kernel classes recorded by the launch profiler.
enum {
  PK_DCT_ROWS_FWD = 0,
  PK_DCT_COLS,
  PK_DCT_ROWS_INV,
  PK_DCT_COLS_GRAD,
  PK_DCT_ROWS_GRAD,
  PK_DCT_DENSE,
  PK_DCT_TC,
  PK_ROF_FUSED,
  PK_EMD_FUSED,
  PK_REDUCE,
  PK_SETUP,
  PK_ROF_STEP_FWD,
  PK_EMD_STEP_FWD,
  PK_CP2_DUAL,
  PK_CP2_PRIMAL,
  PK_3D_LINES,
  PK_3D_STENCIL,
  PK_COUNT
};
static const char* kProfNames[PK_COUNT] = {"dct_rows_fwd", "dct_cols_solve", "dct_rows_inv", "dct_cols_grad",
                                           "dct_rows_grad", "dct_dense",     "dct_tc_split", "rof_fused",
                                           "emd_fused",     "reduce",        "setup",         "rof_step_fwd",
                                           "emd_step_fwd",  "cp2_dual",      "cp2_primal",
                                           "dct3_lines",    "stencil3"};
// Kernel launches behind one recorded launch of a class.
static const int kProfLaunches[PK_COUNT] = {1, 1, 1, 1, 1, 5, 4, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};

struct Profiler {
  bool on = false;
  struct Rec {
    int id;
    cudaEvent_t a, b;
  };
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  std::vector<Rec> recs;
  long long launches[PK_COUNT] = {0};
  double ms[PK_COUNT] = {0};
  bool resolved = true;
  cudaEvent_t next() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
};

struct gp_handle_s {
  int device = 0;
  std::string err;
  std::map<int, DctPlan> plans;
  float* ws = nullptr;  // solve scratch for dct2_poisson
  size_t ws_floats = 0;
  double* part = nullptr;  // per-block partial sums of handle-level reductions
  size_t part_cap = 0;
  double* dres = nullptr;  // device result scalars
  double* hres = nullptr;  // pinned host copy
  std::map<std::pair<int, int>, gp_state_s*> cache;  // solver workspaces keyed by (kind, N)
  Profiler prof;
  bool capturing = false;
  int* tc_err = nullptr;  // timeout flag of the tensor-core kernels
  std::map<std::string, int> tune;  // autotuned row-block heights, "rof_fused/N=.../sm=..." -> rb
  // batched solves: per-problem states, branch streams, fork/join events, results
  std::vector<gp_state_s*> batch;
  std::vector<cudaStream_t> aux;
  std::vector<cudaEvent_t> evs;
  double* bres_d = nullptr;
  double* bres_h = nullptr;
  float* v3 = nullptr;  // volumes of the 3-D solves
  size_t v3_cap = 0;
  float* rf = nullptr;  // scratch of the refined split-precision solves
  size_t rf_cap = 0;
  double* rfd = nullptr;  // partial sums and the sum of the split solves' mean removal
};

struct gp_state_s {
  gp_handle h = nullptr;
  int kind = 0, N = 0, n = 0, cur = 0;
  double lam = 0, tau = 0, sigma = 0;
  const float* I = nullptr;
  const float* f0 = nullptr;
  const float* f1 = nullptr;
  float* prim = nullptr;  // ROF: u (N^2); EMD: grad q (2 N^2), also grad phi at gap checks
  float* gu = nullptr;    // ROF: grad u (2 N^2)
  float* Ic = nullptr;    // ROF: the state's own copy of I (captured graphs never see the caller's pointer)
  float* r = nullptr;     // ROF: next right-hand side; EMD: d = g - div s (= tau div pbar)
  float* p[2] = {nullptr, nullptr};
  float* s[2] = {nullptr, nullptr};  // EMD only
  float* m = nullptr;                // EMD: flux of the current iterate (after a gap step)
  float* e = nullptr;                // EMD: -div p of the current iterate (after a gap step)
  float* phi = nullptr;              // EMD: dual potential
  float* g = nullptr;                // EMD: f0 - f1
  float* tmp = nullptr;              // solve scratch, 2 N^2
  float* rh = nullptr;               // fast sizes: row spectra of the next right-hand side, left by a
                                     // fused step kernel for the next step of the same chunk
  double* part = nullptr;            // this state's per-block partial sums
  bool vec = false;
  // ergodic averages (gp_state_average): FP64 running sums of the right-hand
  // sides (ROF: r; EMD: s (2 planes) and d) and of p over avg_n steps
  double* avg_sum = nullptr;
  long long avg_n = 0;
  int rb = 16;                  // row-block height of the fused kernel (autotuned tile shape)
  bool partials_valid = false;  // part holds the fused gap partials of the current iterate
  double mass_den = 0;          // EMD: sum |f0 - f1| (mass-residual normaliser)
  // EMD stopping test: FP64 sum of p over the current averaging window (2 N^2)
  // and the potential of the window's average (N^2), see run_loop
  double* pwin = nullptr;
  float* phiwin = nullptr;
  std::vector<void*> allocs;
  // CUDA graphs of k-step chunks, keyed by (k, cur, prec, gap_last)
  std::map<std::tuple<int, int, int, int>, cudaGraphExec_t> graphs;
};

int gp::handle_device(gp_handle h) { return h->device; }

namespace {

struct DeviceGuard {
  int prev = -1;
  bool ok = true;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    ok = cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

gp_status fail(gp_handle h, gp_status st, const std::string& msg) {
  if (h) h->err = msg;
  return st;
}

gp_status cuda_fail(gp_handle h, cudaError_t e, const char* where) {
  return fail(h, GP_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define GP_CUDA(h, expr)                                     \
  do {                                                       \
    cudaError_t _e = (expr);                                 \
    if (_e != cudaSuccess) return cuda_fail((h), _e, #expr); \
  } while (0)

// Launch through the profiler: when it is on (and no graph is being
// captured), CUDA events bracket the launch on its stream.
template <typename F>
cudaError_t plaunch(gp_handle h, int id, cudaStream_t st, F&& f, int nlaunch = 0) {
  Profiler& P = h->prof;
  const bool rec = P.on && !h->capturing;
  cudaEvent_t a = nullptr, b = nullptr;
  if (rec) {
    a = P.next();
    b = P.next();
    cudaEventRecord(a, st);
  }
  cudaError_t e = f();
  if (rec) {
    cudaEventRecord(b, st);
    P.recs.push_back({id, a, b});
    P.resolved = false;
  }
  if (P.on) P.launches[id] += nlaunch > 0 ? nlaunch : kProfLaunches[id];
  return e;
}

bool is_device_ptr(const void* p, int device) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == device;
}

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

gp_status check_ptr(gp_handle h, const void* p, const char* name) {
  if (!is_device_ptr(p, h->device))
    return fail(h, GP_ERR_ARG, std::string(name) + " is not a device pointer of the handle's device");
  if (((uintptr_t)p & 3u) != 0) return fail(h, GP_ERR_ARG, std::string(name) + " is not 4-byte aligned");
  return GP_OK;
}

gp_status get_plan(gp_handle h, int N, const DctPlan** out) {
  auto it = h->plans.find(N);
  if (it == h->plans.end()) {
    DctPlan p;
    cudaError_t e = dct_plan_init(p, N);
    if (e != cudaSuccess) {
      dct_plan_free(p);
      return cuda_fail(h, e, "dct_plan_init");
    }
    it = h->plans.emplace(N, p).first;
  }
  *out = &it->second;
  return GP_OK;
}

gp_status ensure_part(gp_handle h, size_t n) {
  if (n <= h->part_cap) return GP_OK;
  if (h->part) cudaFree(h->part);
  h->part = nullptr;
  h->part_cap = 0;
  GP_CUDA(h, cudaMalloc(&h->part, n * sizeof(double)));
  h->part_cap = n;
  return GP_OK;
}

gp_status ensure_res(gp_handle h) {
  if (!h->dres) GP_CUDA(h, cudaMalloc(&h->dres, 16 * sizeof(double)));
  if (!h->hres) GP_CUDA(h, cudaMallocHost(&h->hres, 16 * sizeof(double)));
  return GP_OK;
}

bool prec_split(int prec) { return prec >= GP_PREC_SPLIT_BF16 && prec <= GP_PREC_SPLIT_FP16_REFINED; }
bool prec_fp16(int prec) { return prec == GP_PREC_SPLIT_FP16 || prec == GP_PREC_SPLIT_FP16_REFINED; }
bool prec_refined(int prec) { return prec == GP_PREC_SPLIT_BF16_REFINED || prec == GP_PREC_SPLIT_FP16_REFINED; }
constexpr int kPrecMax = GP_PREC_SPLIT_FP16_REFINED;

// Scratch of the split solves' refinement and mean removal (handle-owned, grown on demand).
gp_status ensure_rf(gp_handle h, size_t floats) {
  if (!h->rfd) GP_CUDA(h, cudaMalloc(&h->rfd, 1040 * sizeof(double)));
  if (floats <= h->rf_cap) return GP_OK;
  if (h->rf) cudaFree(h->rf);
  h->rf = nullptr;
  h->rf_cap = 0;
  GP_CUDA(h, cudaMalloc(&h->rf, floats * sizeof(float)));
  h->rf_cap = floats;
  return GP_OK;
}

// The split-precision plan of size N (dense matrices, their split tiles) and
// the tensor-core timeout flag.
gp_status tc_prepare(gp_handle h, int N, bool grad, bool f16, cudaStream_t st, DctPlan** out) {
  DctPlan* pm = &h->plans[N];
  GP_CUDA(h, dct_plan_dense(*pm));
  if (grad) GP_CUDA(h, dct_plan_grad_dense(*pm));
  GP_CUDA(h, dct_plan_tc_split(*pm, st, f16));
  if (!h->tc_err) {
    GP_CUDA(h, cudaMalloc(&h->tc_err, sizeof(int)));
    GP_CUDA(h, cudaMemset(h->tc_err, 0, sizeof(int)));
  }
  *out = pm;
  return GP_OK;
}

// x = scale (alpha - Lap)^{-1} b with the plan of size N; `tmp` holds 2 N^2.
gp_status solve(gp_handle h, int N, const float* b, float* x, float* tmp, double alpha, double scale, int prec,
                bool allow_fast, cudaStream_t st) {
  const DctPlan* p = nullptr;
  gp_status s = get_plan(h, N, &p);
  if (s != GP_OK) return s;
  const float a = (float)alpha, sc = (float)scale;
  if (prec_split(prec)) {
    if (!tc_solve_supported(N)) return fail(h, GP_ERR_UNSUPPORTED, "split-precision solve needs N a multiple of 128");
    const bool f16 = prec_fp16(prec);
    DctPlan* pm = nullptr;
    if ((s = tc_prepare(h, N, false, f16, st, &pm)) != GP_OK) return s;
    const int nl = f16 ? 9 : 5;
    const size_t NN = (size_t)N * N;
    const float* b0 = b;
    if ((s = ensure_rf(h, 3 * NN)) != GP_OK) return s;
    if (alpha == 0.0) {
      // the constant mode is dropped: remove it before the GEMMs, whose
      // rounding of a large mean would leak into the other modes
      GP_CUDA(h, plaunch(h, PK_SETUP, st,
                         [&] { return launch_center(b, h->rf + 2 * NN, NN, h->rfd + 8, h->rfd, st); }, 3));
      b0 = h->rf + 2 * NN;
    } else if (prec_refined(prec) && b == x) {  // the residual needs b after x is written
      GP_CUDA(h, cudaMemcpyAsync(h->rf + 2 * NN, b, NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
      b0 = h->rf + 2 * NN;
    }
    GP_CUDA(h, plaunch(h, PK_DCT_TC, st, [&] { return dct_solve_tc(*pm, b0, x, tmp, a, sc, h->tc_err, st, f16); },
                       nl));
    if (prec_refined(prec)) {  // r = b - (alpha - Lap) x / scale in FP64; x += solve(r)
      float* r = h->rf;
      float* t = h->rf + NN;
      GP_CUDA(h, plaunch(h, PK_SETUP, st,
                         [&] { return launch_helmholtz_residual(b0, x, r, N, alpha, 1.0 / scale, st); }));
      GP_CUDA(h, plaunch(h, PK_DCT_TC, st, [&] { return dct_solve_tc(*pm, r, t, tmp, a, sc, h->tc_err, st, f16); },
                         nl));
      GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_add_inplace(x, t, NN, st); }));
    }
    return GP_OK;
  }
  if (prec != GP_PREC_FP32) return fail(h, GP_ERR_UNSUPPORTED, "precision mode not available for this size");
  if (p->fft && allow_fast) {
    GP_CUDA(h, plaunch(h, PK_DCT_ROWS_FWD, st, [&] { return dct_fft_pass(*p, 0, b, tmp, a, sc, st); }));
    GP_CUDA(h, plaunch(h, PK_DCT_COLS, st, [&] { return dct_fft_pass(*p, 1, tmp, tmp, a, sc, st); }));
    GP_CUDA(h, plaunch(h, PK_DCT_ROWS_INV, st, [&] { return dct_fft_pass(*p, 2, tmp, x, a, sc, st); }));
  } else {
    if (!p->C) return fail(h, GP_ERR_ARG, "no dense transform for this size");
    GP_CUDA(h, plaunch(h, PK_DCT_DENSE, st, [&] { return dct_solve_dense_fp32(*p, b, x, tmp, a, sc, st); }));
  }
  return GP_OK;
}

// g2 (two planes) = forward-difference gradient of x = scale (alpha - Lap)^{-1} b
// and, when want_phi, phi = x.  Fast sizes (and the split-precision tensor-core
// mode) take the gradient in the spectral domain; other sizes difference the
// dense solve's output (phi is then always written).  tmp holds 2 N^2.
// b_rows: b already holds the row spectra of the right-hand side (the
// interleaved output of the forward row pass; fast sizes, FP32 only).
// cscr / cdscr (optional, split modes at alpha == 0): an N^2 plane and 1032
// doubles of the caller's for the mean removal, so that concurrent solves of
// different states (batched branches) share no scratch.
gp_status solve_grad(gp_handle h, int N, const float* b, float* g2, float* phi, bool want_phi, float* tmp,
                     double alpha, double scale, int prec, cudaStream_t st, bool b_rows = false,
                     float* cscr = nullptr, double* cdscr = nullptr) {
  const DctPlan* p = nullptr;
  gp_status s = get_plan(h, N, &p);
  if (s != GP_OK) return s;
  if (prec != GP_PREC_FP32 && !prec_split(prec)) return fail(h, GP_ERR_ARG, "unknown prec");
  if (b_rows && !(p->fft && prec == GP_PREC_FP32)) return fail(h, GP_ERR_ARG, "row spectra need the FP32 fast path");
  const float a = (float)alpha, sc = (float)scale;
  const size_t NN = (size_t)N * N;
  if (p->fft && prec == GP_PREC_FP32) {
    float* A = tmp;
    float* B = tmp + NN;
    if (!b_rows)  // N = 4096: pair-interleaved spectra for the register-resident passes
      GP_CUDA(h, plaunch(h, PK_DCT_ROWS_FWD, st, [&] {
                return grad4k_supported(*p) ? rows_fwd_4k(*p, b, A, st) : dct_fft_pass(*p, 0, b, A, a, sc, st);
              }));
    const float* in = b_rows ? b : A;
    GP_CUDA(h, plaunch(h, PK_DCT_COLS_GRAD, st, [&] { return dct_grad_cols(*p, in, A, B, a, sc, st); }));
    GP_CUDA(h, plaunch(h, PK_DCT_ROWS_GRAD, st,
                       [&] { return dct_grad_rows(*p, A, B, g2, g2 + NN, want_phi ? phi : nullptr, st); }));
    return GP_OK;
  }
  if (prec_split(prec) && tc_solve_supported(N)) {
    // tensor-core GEMMs with the gradient synthesised from the spectrum
    const bool f16 = prec_fp16(prec), ref = prec_refined(prec);
    DctPlan* pm = nullptr;
    if ((s = tc_prepare(h, N, true, f16, st, &pm)) != GP_OK) return s;
    auto nl = [&](bool ph) { return f16 ? (ph ? 15 : 14) : (ph ? 8 : 7); };
    if ((s = ensure_rf(h, 6 * NN)) != GP_OK) return s;
    const float* b0 = b;
    if (alpha == 0.0) {  // as in solve(): the dropped constant mode leaves before the GEMMs
      float* c = cscr ? cscr : h->rf + 5 * NN;
      double* cd = cdscr ? cdscr : h->rfd;
      GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_center(b, c, NN, cd + 8, cd, st); }, 3));
      b0 = c;
    } else if (ref && (b == g2 || b == g2 + NN || (want_phi && b == phi))) {
      GP_CUDA(h, cudaMemcpyAsync(h->rf + 5 * NN, b, NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
      b0 = h->rf + 5 * NN;
    }
    if (!ref) {
      GP_CUDA(h, plaunch(
                     h, PK_DCT_TC, st,
                     [&] {
                       return dct_grad_tc(*pm, b0, g2, g2 + NN, want_phi ? phi : nullptr, tmp, a, sc, h->tc_err, st,
                                          f16);
                     },
                     nl(want_phi)));
      return GP_OK;
    }
    // One residual correction.  x0 = S b (the solve), r = b - (alpha - Lap) x0 / scale
    // in FP64 from the stored x0, then grad x = D x0 + G r and x = x0 + S r: D x0,
    // the forward differences of the stored x0, is exact up to one rounding of
    // each difference, and G r, the split gradient of the correction, errs only
    // relative to the correction.  (G b + G r would keep G's own error on b.)
    float* x0 = want_phi ? phi : h->rf;
    float* r = h->rf + NN;
    float* gg = h->rf + 2 * NN;
    float* ph1 = h->rf + 4 * NN;
    GP_CUDA(h, plaunch(h, PK_DCT_TC, st, [&] { return dct_solve_tc(*pm, b0, x0, tmp, a, sc, h->tc_err, st, f16); },
                       f16 ? 9 : 5));
    GP_CUDA(h, plaunch(h, PK_SETUP, st,
                       [&] { return launch_helmholtz_residual(b0, x0, r, N, alpha, 1.0 / scale, st); }));
    GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_grad(x0, g2, N, st); }));
    GP_CUDA(h, plaunch(
                   h, PK_DCT_TC, st,
                   [&] {
                     return dct_grad_tc(*pm, r, gg, gg + NN, want_phi ? ph1 : nullptr, tmp, a, sc, h->tc_err, st, f16);
                   },
                   nl(want_phi)));
    GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_add_inplace(g2, gg, 2 * NN, st); }));
    if (want_phi) GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_add_inplace(phi, ph1, NN, st); }));
    return GP_OK;
  }
  if (!phi) return fail(h, GP_ERR_ARG, "internal: the dense gradient solve needs a plane for the solution");
  if ((s = solve(h, N, b, phi, tmp, alpha, scale, prec, false, st)) != GP_OK) return s;
  GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_grad(phi, g2, N, st); }));  // differences of the solution
  return GP_OK;
}

size_t fused_blocks(int N, bool vec, int rb) {
  dim3 g = fused_grid(N, vec ? 4 : 1, rb);
  return (size_t)g.x * g.y;
}

size_t state_part_size(int N) {
  // Gap partials: the first region holds <= 4 values per block of either the
  // fused kernels (most blocks: vector layout with the smallest row block, or
  // the scalar layout) or the unfused 1-D reduction (a gap taken before any
  // step); the EMD dual partials (2 per 1-D block) follow it.
  const size_t nd = (size_t)reduce_blocks_1d((size_t)N * N);
  const size_t nb = std::max({fused_blocks(N, true, 4), fused_blocks(N, false, 16), nd});
  return nb * 4 + nd * 2;
}

// Copy `nq` reduced scalars to the host and wait for them.
gp_status fetch(gp_handle h, int nq, cudaStream_t st) {
  GP_CUDA(h, cudaMemcpyAsync(h->hres, h->dres, nq * sizeof(double), cudaMemcpyDeviceToHost, st));
  GP_CUDA(h, cudaStreamSynchronize(st));
  return GP_OK;
}

void drop_graphs(gp_state s) {
  for (auto& kv : s->graphs) cudaGraphExecDestroy(kv.second);
  s->graphs.clear();
}

void free_state(gp_state s) {
  if (!s) return;
  drop_graphs(s);
  if (s->avg_sum) cudaFree(s->avg_sum);
  if (s->pwin) cudaFree(s->pwin);
  if (s->phiwin) cudaFree(s->phiwin);
  for (void* p : s->allocs) cudaFree(p);
  delete s;
}

gp_status alloc_state(gp_handle h, int kind, int N, gp_state* out) {
  gp_state s = new gp_state_s();
  s->h = h;
  s->kind = kind;
  s->N = N;
  const size_t NN = (size_t)N * N;
  auto A = [&](float** dst, size_t n) -> cudaError_t {
    cudaError_t e = cudaMalloc(dst, n * sizeof(float));
    if (e == cudaSuccess) s->allocs.push_back(*dst);
    return e;
  };
  cudaError_t e = cudaSuccess;
  if (!e) e = A(&s->prim, kind == KIND_EMD ? 2 * NN : NN);
  if (!e) e = A(&s->r, NN);
  if (!e) e = A(&s->p[0], 2 * NN);
  if (!e) e = A(&s->p[1], 2 * NN);
  if (!e) e = A(&s->tmp, 2 * NN);
  if (!e && N >= 16 && N <= 8192 && (N & (N - 1)) == 0) e = A(&s->rh, NN);
  if (kind == KIND_ROF && !e) e = A(&s->gu, 2 * NN);
  if (kind == KIND_ROF && !e) e = A(&s->Ic, NN);
  if (kind == KIND_EMD) {
    if (!e) e = A(&s->s[0], 2 * NN);
    if (!e) e = A(&s->s[1], 2 * NN);
    if (!e) e = A(&s->m, 2 * NN);
    if (!e) e = A(&s->e, NN);
    if (!e) e = A(&s->phi, NN);
    if (!e) e = A(&s->g, NN);
  }
  if (!e) {
    e = cudaMalloc(&s->part, state_part_size(N) * sizeof(double));
    if (e == cudaSuccess) s->allocs.push_back(s->part);
  }
  if (e != cudaSuccess) {
    free_state(s);
    return cuda_fail(h, e, "state allocation");
  }
  *out = s;
  return GP_OK;
}

std::string tune_key(gp_handle h, const char* kernel, int N) {
  int maj = 0, mnr = 0;
  cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, h->device);
  cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, h->device);
  return std::string(kernel) + "/N=" + std::to_string(N) + "/sm=" + std::to_string(maj * 10 + mnr);
}

// Row-block height of the fused kernels: the autotuned one, else a default
// that keeps small grids from running a few long per-thread row chains (at
// 1024^2, 16-row blocks give 128 CTAs of 128 threads: latency-bound).
int tuned_rb(gp_handle h, const char* kernel, int N) {
  auto it = h->tune.find(tune_key(h, kernel, N));
  if (it != h->tune.end()) return it->second;
  return N <= 1024 ? 4 : (N <= 2048 ? 8 : 16);
}

// --------------------------------------------------------------- ROF state
gp_status rof_setup(gp_state s, const float* I, double lam, double tau, double sigma, const float* u0,
                    const float* p0, const float* pbar0, cudaStream_t st) {
  gp_handle h = s->h;
  const int N = s->N;
  const size_t NN = (size_t)N * N;
  if (s->lam != lam || s->tau != tau || s->sigma != sigma) drop_graphs(s);
  s->I = I;
  GP_CUDA(h, cudaMemcpyAsync(s->Ic, I, NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  s->lam = lam;
  s->tau = tau;
  s->sigma = sigma;
  s->n = 0;
  s->cur = 0;
  s->partials_valid = false;
  s->vec = N % 4 == 0;  // all fused-kernel operands are state buffers
  const int rb = tuned_rb(h, "rof_fused", N);
  if (rb != s->rb) drop_graphs(s);  // the graphs hold the previous tile shape
  s->rb = rb;
  if (u0) GP_CUDA(h, cudaMemcpyAsync(s->prim, u0, NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  else GP_CUDA(h, cudaMemsetAsync(s->prim, 0, NN * sizeof(float), st));
  if (p0) GP_CUDA(h, cudaMemcpyAsync(s->p[0], p0, 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  else GP_CUDA(h, cudaMemsetAsync(s->p[0], 0, 2 * NN * sizeof(float), st));
  // pbar0 is staged in p[1], which the first step overwrites
  const float* pb = s->p[0];
  if (pbar0) {
    GP_CUDA(h, cudaMemcpyAsync(s->p[1], pbar0, 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
    pb = s->p[1];
  }
  RofParams P{N, (float)N, (float)((double)N * N), (float)(lam * tau), (float)tau, (float)sigma};
  GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_rof_init(I, s->prim, pb, s->p[0], s->r, P, st); }));
  return GP_OK;
}

// Within a chunk of steps, every step but the last runs its stencil fused
// with the next solve's forward row pass (fast sizes, FP32): the right-hand
// side reaches the next step as row spectra in s->rh.  The last step of a
// chunk (the gap step, when there is one) writes the right-hand side itself,
// so a chunk always starts and ends with s->r current.
const DctPlan* fused_step_plan(gp_state s, int prec) {
  if (prec != GP_PREC_FP32 || !s->rh || !s->vec || s->avg_sum) return nullptr;
  auto it = s->h->plans.find(s->N);
  return it != s->h->plans.end() && it->second.fft ? &it->second : nullptr;
}

// N = 4096: the plan of the fused row pass (one kernel per non-gap step for
// the solve's row syntheses, the step and the next forward row pass), else null.
const DctPlan* step4k_plan(gp_state s, int prec) {
  if (prec != GP_PREC_FP32 || !s->rh || !s->vec || s->avg_sum) return nullptr;
  const DctPlan* p = nullptr;
  if (get_plan(s->h, s->N, &p) != GP_OK) return nullptr;
  return grad4k_supported(*p) ? p : nullptr;
}

gp_status rof_steps_direct(gp_state s, int n_steps, int prec, bool gap_last, cudaStream_t st) {
  gp_handle h = s->h;
  const int N = s->N;
  RofParams P{N, (float)N, (float)((double)N * N), (float)(s->lam * s->tau), (float)s->tau, (float)s->sigma};
  if (const DctPlan* p4 = step4k_plan(s, prec)) {
    // per step: the column pass of the solve, then either the fused row pass
    // (rows of the solve + step + next forward rows) or, on the last step of
    // the call, the gradient row pass and the unfused step (r and gap terms)
    const size_t NN = (size_t)N * N;
    float* A = s->tmp;
    float* B = s->tmp + NN;
    const float a = (float)(s->lam * s->tau);
    for (int k = 0; k < n_steps; ++k) {
      const bool last = k == n_steps - 1, g = gap_last && last;
      if (k == 0) GP_CUDA(h, plaunch(h, PK_DCT_ROWS_FWD, st, [&] { return rows_fwd_4k(*p4, s->r, A, st); }));
      GP_CUDA(h, plaunch(h, PK_DCT_COLS_GRAD, st,
                         [&] { return grad_cols_4k(*p4, k == 0 ? A : s->rh, A, B, a, 1.f, st); }));
      float* pin = s->p[s->cur];
      float* pout = s->p[1 - s->cur];
      if (!last) {
        GP_CUDA(h, plaunch(h, PK_ROF_STEP_FWD, st,
                           [&] { return rof_rows_step_4k(*p4, A, B, pin, s->Ic, pout, s->rh, P, st); }));
      } else {
        GP_CUDA(h, plaunch(h, PK_DCT_ROWS_GRAD, st,
                           [&] { return grad_rows_4k(*p4, A, B, s->gu, s->gu + NN, g ? s->prim : nullptr, st); }));
        GP_CUDA(h, plaunch(h, PK_ROF_FUSED, st, [&] {
                  return launch_rof_fused(s->gu, s->prim, pin, s->Ic, pout, s->r, s->part, P, s->vec, g, s->rb, st);
                }));
      }
      s->cur = 1 - s->cur;
      s->n++;
    }
    return GP_OK;
  }
  for (int k = 0; k < n_steps; ++k) {
    const bool g = gap_last && (k == n_steps - 1);
    const DctPlan* fp = fused_step_plan(s, prec);  // the plan exists after the first solve
    const bool rows_in = fp && k > 0;
    if (s->avg_sum)  // u_{n+1} = (lambda tau - Lap)^{-1} r_n is linear in r_n: sum the r_n
      GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_accumulate(s->avg_sum, s->r, (size_t)N * N, st); }));
    // grad u_{n+1} from the spectrum; u_{n+1} itself only when the step reports the objective
    gp_status r = solve_grad(h, N, rows_in ? s->rh : s->r, s->gu, s->prim, g, s->tmp, s->lam * s->tau, 1.0, prec, st,
                             rows_in);
    if (r != GP_OK) return r;
    float* pin = s->p[s->cur];
    float* pout = s->p[1 - s->cur];
    fp = fused_step_plan(s, prec);
    if (fp && k < n_steps - 1) {
      GP_CUDA(h, plaunch(h, PK_ROF_STEP_FWD, st,
                         [&] { return dct_rof_step_fwd(*fp, s->gu, pin, s->Ic, pout, s->rh, P, st); }));
    } else {
      GP_CUDA(h, plaunch(h, PK_ROF_FUSED, st, [&] {
                return launch_rof_fused(s->gu, s->prim, pin, s->Ic, pout, s->r, s->part, P, s->vec, g, s->rb, st);
              }));
    }
    if (s->avg_sum) {
      const size_t NN = (size_t)N * N;
      GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_accumulate(s->avg_sum + NN, pout, 2 * NN, st); }));
      s->avg_n++;
    }
    s->cur = 1 - s->cur;
    s->n++;
  }
  return GP_OK;
}

gp_status emd_steps_direct(gp_state s, int n_steps, int prec, bool gap_last, cudaStream_t st) {
  gp_handle h = s->h;
  const int N = s->N;
  EmdParams P{N, (float)N, (float)s->tau, (float)s->sigma};
  if (const DctPlan* p4 = step4k_plan(s, prec)) {  // as in rof_steps_direct
    const size_t NN = (size_t)N * N;
    float* A = s->tmp;
    float* B = s->tmp + NN;
    for (int k = 0; k < n_steps; ++k) {
      const bool last = k == n_steps - 1, g = gap_last && last;
      const int c = s->cur;
      // grad q, q = Lap^{-1} d  <=>  (0 - Lap) q = -d
      if (k == 0) GP_CUDA(h, plaunch(h, PK_DCT_ROWS_FWD, st, [&] { return rows_fwd_4k(*p4, s->r, A, st); }));
      GP_CUDA(h, plaunch(h, PK_DCT_COLS_GRAD, st,
                         [&] { return grad_cols_4k(*p4, k == 0 ? A : s->rh, A, B, 0.f, -1.f, st); }));
      if (!last) {
        GP_CUDA(h, plaunch(h, PK_EMD_STEP_FWD, st, [&] {
                  return emd_rows_step_4k(*p4, A, B, s->s[c], s->p[c], s->g, s->s[1 - c], s->p[1 - c], s->rh, P, st);
                }));
      } else {
        GP_CUDA(h, plaunch(h, PK_DCT_ROWS_GRAD, st,
                           [&] { return grad_rows_4k(*p4, A, B, s->prim, s->prim + NN, nullptr, st); }));
        GP_CUDA(h, plaunch(h, PK_EMD_FUSED, st, [&] {
                  return launch_emd_fused(s->prim, s->s[c], s->p[c], s->g, s->s[1 - c], s->p[1 - c], s->r, s->m, s->e,
                                          s->part, P, s->vec, g, s->rb, st);
                }));
      }
      s->cur = 1 - s->cur;
      s->n++;
    }
    return GP_OK;
  }
  for (int k = 0; k < n_steps; ++k) {
    const DctPlan* fp = fused_step_plan(s, prec);
    const bool rows_in = fp && k > 0;
    if (s->avg_sum) {  // m_{n+1} = s_n + grad Lap^{-1} d_n is affine in (s_n, d_n): sum both
      const size_t NN = (size_t)N * N;
      GP_CUDA(h, plaunch(h, PK_SETUP, st,
                         [&] { return launch_accumulate(s->avg_sum, s->s[s->cur], 2 * NN, st); }));
      GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_accumulate(s->avg_sum + 2 * NN, s->r, NN, st); }));
    }
    // grad q, q = Lap^{-1} d  <=>  (0 - Lap) q = -d
    gp_status r = solve_grad(h, N, rows_in ? s->rh : s->r, s->prim, s->phi, false, s->tmp, 0.0, -1.0, prec, st,
                             rows_in, s->s[1 - s->cur], s->part);
    if (r != GP_OK) return r;
    const bool g = gap_last && (k == n_steps - 1);
    const int c = s->cur;
    fp = fused_step_plan(s, prec);
    if (fp && k < n_steps - 1) {
      GP_CUDA(h, plaunch(h, PK_EMD_STEP_FWD, st, [&] {
                return dct_emd_step_fwd(*fp, s->prim, s->s[c], s->p[c], s->g, s->s[1 - c], s->p[1 - c], s->rh, P,
                                        st);
              }));
    } else {
      GP_CUDA(h, plaunch(h, PK_EMD_FUSED, st, [&] {
                return launch_emd_fused(s->prim, s->s[c], s->p[c], s->g, s->s[1 - c], s->p[1 - c], s->r, s->m, s->e,
                                        s->part, P, s->vec, g, s->rb, st);
              }));
    }
    if (s->avg_sum) {
      const size_t NN = (size_t)N * N;
      GP_CUDA(h, plaunch(h, PK_SETUP, st,
                         [&] { return launch_accumulate(s->avg_sum + 3 * NN, s->p[1 - c], 2 * NN, st); }));
      s->avg_n++;
    }
    s->cur = 1 - s->cur;
    s->n++;
  }
  return GP_OK;
}

// k iterations, optionally replayed from a CUDA graph of the same chunk.
gp_status run_steps(gp_state s, int k, int prec, bool gap_last, bool use_graph, cudaStream_t st) {
  gp_handle h = s->h;
  auto direct = [&](int kk) {
    return s->kind == KIND_ROF ? rof_steps_direct(s, kk, prec, gap_last, st)
                               : emd_steps_direct(s, kk, prec, gap_last, st);
  };
  if (k <= 0) return GP_OK;
  if (!use_graph || st == nullptr || h->prof.on) {
    gp_status r = direct(k);
    if (r == GP_OK) s->partials_valid = gap_last;
    return r;
  }
  const auto key = std::make_tuple(k, s->cur, prec, gap_last ? 1 : 0);
  auto it = s->graphs.find(key);
  if (it == s->graphs.end()) {
    // First use: run the chunk directly (creates plans, sets kernel
    // attributes), then capture the same chunk for the next calls.
    const int cur0 = s->cur;
    gp_status r = direct(k);
    if (r != GP_OK) return r;
    s->partials_valid = gap_last;
    const int cur1 = s->cur, n1 = s->n;
    const long long avg1 = s->avg_n;
    s->cur = cur0;
    cudaGraph_t g = nullptr;
    GP_CUDA(h, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    h->capturing = true;
    r = direct(k);
    h->capturing = false;
    cudaError_t e = cudaStreamEndCapture(st, &g);
    s->cur = cur1;
    s->n = n1;
    s->avg_n = avg1;  // the capture launched nothing
    if (r != GP_OK) {
      if (g) cudaGraphDestroy(g);
      return r;
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    s->graphs[key] = ex;
    return GP_OK;
  }
  GP_CUDA(h, cudaGraphLaunch(it->second, st));
  if (k & 1) s->cur = 1 - s->cur;
  s->n += k;
  if (s->avg_sum) s->avg_n += k;
  s->partials_valid = gap_last;
  return GP_OK;
}

// --------------------------------------------------------------- EMD state
gp_status emd_setup(gp_state s, const float* f0, const float* f1, double tau, double sigma, const float* m0,
                    const float* p0, const float* pbar0, cudaStream_t st) {
  gp_handle h = s->h;
  const int N = s->N;
  const size_t NN = (size_t)N * N;
  // the captured step graphs read only state buffers (g = f0 - f1 is formed here), so new
  // input pointers need no recapture; the step sizes are kernel arguments
  if (s->tau != tau || s->sigma != sigma) drop_graphs(s);
  s->f0 = f0;
  s->f1 = f1;
  s->tau = tau;
  s->sigma = sigma;
  s->n = 0;
  s->cur = 0;
  s->partials_valid = false;
  s->vec = N % 4 == 0;  // all fused-kernel operands are state buffers
  const int rb = tuned_rb(h, "emd_fused", N);
  if (rb != s->rb) drop_graphs(s);  // the graphs hold the previous tile shape
  s->rb = rb;
  GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_sub(f0, f1, s->g, NN, st); }));
  if (m0) {
    GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_copy_field(m0, s->m, N, st); }));
  } else {
    // Hodge split (section 3.2): Lap psi = f0 - f1 = g  <=>  (0 - Lap) psi = -g; m0 = grad psi
    gp_status r = solve_grad(h, N, s->g, s->m, s->phi, false, s->tmp, 0.0, -1.0, GP_PREC_FP32, st);
    if (r != GP_OK) return r;
  }
  if (p0) GP_CUDA(h, cudaMemcpyAsync(s->p[0], p0, 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  else GP_CUDA(h, cudaMemsetAsync(s->p[0], 0, 2 * NN * sizeof(float), st));
  const float* pb = s->p[0];
  if (pbar0) {
    GP_CUDA(h, cudaMemcpyAsync(s->p[1], pbar0, 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
    pb = s->p[1];
  }
  EmdParams P{N, (float)N, (float)tau, (float)sigma};
  GP_CUDA(h, plaunch(h, PK_SETUP, st,
                     [&] { return launch_emd_init(s->m, pb, s->p[0], s->s[0], s->g, s->r, P, st); }));
  return GP_OK;
}

void finish_report(gp_report* rep, double P, double D) {
  rep->primal = P;
  rep->dual = D;
  const double sc = fmax(fabs(P), fabs(D));
  rep->rel_gap = sc > 0 ? (P - D) / sc : 0.0;
}

// EMD dual bound of p, whose e = -div p (FP32) is in s->e (section 3.2 with
// the weak duality of section 2.1): any phi with max |D phi| <= 1 gives the
// lower bound h^2 sum phi (f1 - f0), so D = h^2 sum phi (f1 - f0) /
// max(1, max |D phi|) for phi = Lap^{-1} div p.  phi is held as two FP32
// planes, phi_hi from the FP32 cosine solve of e and phi_lo from a second
// solve of the residual -div p + Lap phi_hi taken in FP64 from p itself, and
// both sums are taken in FP64 from the planes: the bound is exact for the phi
// represented, and FP32 rounding no longer inflates max |D phi| (near the
// optimum |D phi| = 1 on the whole transport region, so the largest of
// millions of rounding errors would land in the normalisation).  Writes the
// two partial sums (sum, max) to dst; uses e, prim and tmp (free between
// steps; p may be in prim); phi_hi + phi_lo is left in phi.
gp_status emd_dual_enqueue(gp_state s, const float* p, float* phi, double* part, double* dst, cudaStream_t st) {
  gp_handle h = s->h;
  const int N = s->N;
  const size_t NN = (size_t)N * N;
  float* r = s->e;
  float* lo = s->prim;
  gp_status q = solve(h, N, s->e, phi, s->tmp, 0.0, 1.0, GP_PREC_FP32, true, st);
  if (q != GP_OK) return q;
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_dual_residual(p, phi, r, N, st); }));
  if ((q = solve(h, N, r, lo, s->tmp, 0.0, 1.0, GP_PREC_FP32, true, st)) != GP_OK) return q;
  const int nd = reduce_blocks_1d(NN);
  GP_CUDA(h, plaunch(h, PK_REDUCE, st,
                     [&] { return launch_emd_dual_hilo(phi, lo, s->f0, s->f1, N, part, nd, st); }));
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(part, nd, 2, 2u, dst, st); }));
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_add_inplace(phi, lo, NN, st); }));
  return GP_OK;
}

// Gap of the current iterate, in two halves so that a CUDA graph can hold the
// device half: state_gap_enqueue writes the four reduced scalars to `dst`
// (device); state_gap_finish turns their host copy into P, D and the gap.
// The fused partials are used when the last step left them, else the terms
// are recomputed with the unfused kernels.
gp_status state_gap_enqueue(gp_state s, double* dst, cudaStream_t st) {
  gp_handle h = s->h;
  const int N = s->N;
  const size_t NN = (size_t)N * N;
  const bool fused = s->partials_valid;
  const int nb = fused ? (int)fused_blocks(N, s->vec, s->vec ? s->rb : 16) : reduce_blocks_1d(NN);
  if (s->kind == KIND_ROF) {
    if (!fused)
      GP_CUDA(h, plaunch(h, PK_REDUCE, st,
                         [&] { return launch_rof_gap(s->prim, s->p[s->cur], s->Ic, N, s->part, nb, st); }));
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(s->part, nb, 4, 0u, dst, st); }));
    return GP_OK;
  }
  if (!fused)
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] {
              return launch_emd_primal(s->m, s->p[s->cur], s->f0, s->f1, s->e, N, s->part, nb, st);
            }));
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(s->part, nb, 2, 0u, dst, st); }));
  // phi = Lap^{-1} div p  <=>  (0 - Lap) phi = -div p = e
  return emd_dual_enqueue(s, s->p[s->cur], s->phi, s->part + (size_t)nb * 4, dst + 2, st);
}

void state_gap_finish(gp_state s, const double* v, gp_report* rep) {
  const double h2 = 1.0 / ((double)s->N * s->N);
  if (s->kind == KIND_ROF) {
    finish_report(rep, h2 * (v[0] + 0.5 * s->lam * v[1]), -h2 * v[2] - h2 * v[3] / (2.0 * s->lam));
    rep->mass_residual = 0.0;
    rep->primal_feasible = rep->primal;  // no constraint on u: every iterate is feasible
    rep->rel_gap_feasible = rep->rel_gap;
    rep->mass_residual_feasible = 0.0;
  } else {
    finish_report(rep, h2 * v[0], h2 * v[2] / fmax(1.0, v[3]));
    rep->mass_residual = s->mass_den > 0 ? v[1] / s->mass_den : v[1];
    rep->primal_feasible = rep->rel_gap_feasible = rep->mass_residual_feasible = NAN;  // not certified yet
  }
}

// EMD feasibility certificate of the current m (after state_gap filled P, D):
// D bounds the optimum from below for any p, P(m) from above only for a
// feasible m (section 3.2's constraint div m = f0 - f1), and an FP32 m is
// feasible only up to its rounding times 1/h.  The residual rho of the stored
// m is taken in FP64, c = Lap^{-1} rho solved (FP32 cosine solve: its relative
// error multiplies the already small rho), and the corrected flux
// m~ = m + grad c is feasible up to the residual the correction leaves, which
// is measured too.  Uses e, prim and tmp, which are free between chunks.
gp_status emd_certify(gp_state s, gp_report* rep, cudaStream_t st) {
  gp_handle h = s->h;
  const int N = s->N;
  const size_t NN = (size_t)N * N;
  const int nd = reduce_blocks_1d(NN);
  gp_status r = ensure_res(h);
  if (r != GP_OK) return r;
  GP_CUDA(h, plaunch(h, PK_REDUCE, st,
                     [&] { return launch_emd_residual64(s->m, s->f0, s->f1, s->e, N, s->part, nd, st); }));
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(s->part, nd, 1, 0u, h->dres, st); }));
  // grad c with Lap c = rho  <=>  (0 - Lap) c = -rho.  Sizes without the fast
  // transform difference the dense solve's output, which needs a plane: c
  // goes over rho in e (the dense solve consumes its input first).
  if ((r = solve_grad(h, N, s->e, s->prim, s->e, false, s->tmp, 0.0, -1.0, GP_PREC_FP32, st)) != GP_OK) return r;
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] {
            return launch_emd_corrected(s->m, s->prim, s->f0, s->f1, N, s->part + nd, nd, st);
          }));
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(s->part + nd, nd, 2, 0u, h->dres + 1, st); }));
  if ((r = fetch(h, 3, st)) != GP_OK) return r;
  const double h2 = 1.0 / ((double)N * N), den = s->mass_den > 0 ? s->mass_den : 1.0;
  rep->mass_residual = h->hres[0] / den;
  rep->primal_feasible = h2 * h->hres[1];
  rep->mass_residual_feasible = h->hres[2] / den;
  const double sc = fmax(fabs(rep->primal_feasible), fabs(rep->dual));
  rep->rel_gap_feasible = sc > 0 ? (rep->primal_feasible - rep->dual) / sc : 0.0;
  s->partials_valid = false;  // part now holds the certificate's sums
  return GP_OK;
}

gp_status state_gap(gp_state s, gp_report* rep, cudaStream_t st) {
  gp_handle h = s->h;
  gp_status r = ensure_res(h);
  if (r != GP_OK) return r;
  if ((r = state_gap_enqueue(s, h->dres, st)) != GP_OK) return r;
  if ((r = fetch(h, 4, st)) != GP_OK) return r;
  state_gap_finish(s, h->hres, rep);
  return GP_OK;
}

// sum f0, sum f1 and sum |f0 - f1| of an EMD pair (FP64).
gp_status mass_stats(gp_handle h, const float* f0, const float* f1, int N, double out[3], cudaStream_t st) {
  const size_t NN = (size_t)N * N;
  const int nb = reduce_blocks_1d(NN);
  gp_status r = ensure_part(h, (size_t)nb * 3);
  if (r != GP_OK) return r;
  if ((r = ensure_res(h)) != GP_OK) return r;
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_mass_stats(f0, f1, NN, h->part, nb, st); }));
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(h->part, nb, 3, 0u, h->dres, st); }));
  if ((r = fetch(h, 3, st)) != GP_OK) return r;
  for (int q = 0; q < 3; ++q) out[q] = h->hres[q];
  return GP_OK;
}

gp_status check_mass(gp_handle h, const double ms[3]) {
  if (!isfinite(ms[0]) || !isfinite(ms[1])) return fail(h, GP_ERR_NONFINITE, "non-finite density");
  const double sc = fmax(fabs(ms[0]), fabs(ms[1]));
  if (fabs(ms[0] - ms[1]) > 1e-3 * sc)
    return fail(h, GP_ERR_MASS, "f0 and f1 differ in total mass by more than 1e-3 relative");
  return GP_OK;
}

// ROF step rule (sections 3.1 and 4.1).
// Image norms of the ROF step rule (section 4.1), FP64 reductions on the GPU:
// out[0] = ||I||_TV = h^2 sum |grad I|, out[1] = ||grad I||_L2, out[2] = ||I - mean I||^2_L2.
gp_status rof_image_stats(gp_handle h, const float* I, int N, double out[3], cudaStream_t st) {
  const size_t NN = (size_t)N * N;
  const int nb = reduce_blocks_1d(NN);
  gp_status r = ensure_part(h, (size_t)nb * 3);
  if (r != GP_OK) return r;
  if ((r = ensure_res(h)) != GP_OK) return r;
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_rof_stats(I, N, h->part, nb, st); }));
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(h->part, nb, 3, 0u, h->dres, st); }));
  if ((r = fetch(h, 3, st)) != GP_OK) return r;
  const double h2 = 1.0 / ((double)N * N);
  out[0] = h2 * h->hres[0];
  out[1] = sqrt(h2 * h->hres[1]);
  const double mean = h->hres[2] / (double)NN;
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_sq_dev(I, NN, (float)mean, h->part, nb, st); }));
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(h->part, nb, 1, 0u, h->dres, st); }));
  if ((r = fetch(h, 1, st)) != GP_OK) return r;
  out[2] = h2 * h->hres[0];
  return GP_OK;
}

gp_status rof_rule(gp_handle h, const float* I, int N, double lambda, const gp_opts& o, double* tau_out,
                   cudaStream_t st) {
  double stats[3];
  gp_status r = rof_image_stats(h, I, N, stats, st);
  if (r != GP_OK) return r;
  if (!isfinite(stats[0]) || !isfinite(stats[2])) return fail(h, GP_ERR_NONFINITE, "non-finite image");
  const double eps = o.eps > 0 ? o.eps : 1e-3;
  const double tau = gp_rof_step_tau(stats, lambda, eps, GP_RULE_GRID_CAP | GP_RULE_FIDELITY_BOUND);
  *tau_out = tau * (o.tau_scale > 0 ? o.tau_scale : 1.0);
  return GP_OK;
}

struct Timer {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double s() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
};

gp_status check_opts(gp_handle h, const gp_opts* o) {
  if (o->max_iters < 0) return fail(h, GP_ERR_ARG, "max_iters < 0");
  if (o->gap_every < 0) return fail(h, GP_ERR_ARG, "gap_every < 0");
  if (o->prec < 0 || o->prec > kPrecMax) return fail(h, GP_ERR_ARG, "unknown prec");
  if (o->warm_start < 0 || o->warm_start > 1) return fail(h, GP_ERR_ARG, "unknown warm_start");
  return GP_OK;
}

gp_state cached_state(gp_handle h, int kind, int N, gp_status* st) {
  auto key = std::make_pair(kind, N);
  auto it = h->cache.find(key);
  if (it != h->cache.end()) {
    *st = GP_OK;
    return it->second;
  }
  gp_state s = nullptr;
  *st = alloc_state(h, kind, N, &s);
  if (*st != GP_OK) return nullptr;
  h->cache[key] = s;
  return s;
}

// Divergence: the relative gap stayed above 10x its running minimum for 5
// consecutive checks while above 1e-2.
struct DivergenceWatch {
  double best = INFINITY;
  int bad = 0;
  bool update(double g) {
    if (g < best) best = g;
    bad = (g > 10.0 * best && g > 1e-2) ? bad + 1 : 0;
    return bad >= 5;
  }
};

// Adaptive gap-check schedule (gap_every == 0 with a positive tolerance).
// While the relative gap is above 3 x the tolerance, its decay between the
// last two checks is fitted as g ~ c n^-a and the next check goes halfway to
// the iteration where that fit reaches the tolerance, as a chunk of
// 10 * 2^j iterations (at most 320).  Within 3 x the tolerance, and without
// a decrease to fit, the next check is 10 iterations on: the primal-dual gap
// is not monotone, and near the target it dips below the tolerance at
// isolated checks (EMD at 4096^2: first at iteration 30480, next at 31940),
// which sparse checks would step over.
constexpr int kAdaptiveMinChunk = 10, kAdaptiveMaxChunk = 320;
constexpr double kAdaptiveNear = 3.0;

int adaptive_chunk(int n_prev, double g_prev, int n, double g, double tol) {
  if (n_prev <= 0 || n <= n_prev || !(tol > 0) || !(g > kAdaptiveNear * tol) || !(g_prev > g))
    return kAdaptiveMinChunk;
  const double a = log(g_prev / g) / log((double)n / n_prev);
  if (!(a > 0)) return kAdaptiveMinChunk;
  const double half = 0.5 * (n * pow(g / tol, 1.0 / a) - n);
  int k = kAdaptiveMinChunk;
  while (2 * k <= kAdaptiveMaxChunk && 2 * k <= half) k *= 2;
  return k;
}

// EMD dual bound of the average of the p's summed in s->pwin (count n): p_bar
// into prim, e = -div p_bar, phi = Lap^{-1} div p_bar with its gradient (prim),
// D = h^2 sum phi (f1 - f0) / max(1, max |grad phi|).  A convex combination of
// feasible p's is feasible, so D bounds the optimum from below.  Uses prim,
// e, tmp and the partial sums (free between chunks).
gp_status emd_window_dual(gp_state s, long long n, double* D, cudaStream_t st) {
  gp_handle h = s->h;
  const int N = s->N;
  const size_t NN = (size_t)N * N;
  const int nd = reduce_blocks_1d(NN);
  gp_status r = ensure_res(h);
  if (r != GP_OK) return r;
  GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_scale_sum(s->pwin, s->prim, 2 * NN, 1.0 / (double)n, st); }));
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] {
            return launch_emd_primal(s->m, s->prim, s->f0, s->f1, s->e, N, s->part, nd, st);  // e = -div p_bar
          }));
  if ((r = emd_dual_enqueue(s, s->prim, s->phiwin, s->part, h->dres, st)) != GP_OK) return r;
  if ((r = fetch(h, 2, st)) != GP_OK) return r;
  *D = h->hres[0] / ((double)N * N) / fmax(1.0, h->hres[1]);
  s->partials_valid = false;
  return GP_OK;
}

// EMD stopping test with a tolerance (run_loop and the batched loop).  The
// dual bound is the best one met so far, over the iterates' p at the checks
// and over averages of those p's (windows that open once the gap is within
// 30 x tol and restart whenever the iteration count has doubled since their
// start); each is a lower bound of the optimum, and the last iterate's p
// lags it.  The open window's bound is also taken whenever the window has
// grown by a quarter since it was last taken (at least 100 iterations and 4
// samples apart), so that a window can certify before it restarts.  The
// current flux is certified (its corrected primal taken) at every window
// evaluation and whenever it is a candidate: the stored primal,
// less the rounding cost P - P(m~) the last certificate measured, within
// 2 x tol of the best bound (at most every 100 iterations unless within
// tol).  The solve stops once a certified gap meets tol.  The offset matters:
// the stored FP32 flux's primal can exceed the corrected one by more than
// tol (2e-5 relative on some 4096^2 pairs), which would keep every candidate
// test from passing.
struct EmdStop {
  double d_best = -INFINITY;
  double p_off = 0.0;  // P - P(m~) at the last certificate
  int win_start = -1, last_cert = -1000000;
  int win_eval = 0;    // iteration count from which the open window is taken again
  long long win_n = 0;
};

double rel_gap_of(double P, double D) {
  const double sc = fmax(fabs(P), fabs(D));
  return sc > 0 ? (P - D) / sc : 0.0;
}

gp_status emd_close_window(gp_state s, EmdStop& z, cudaStream_t st) {
  if (z.win_n == 0) return GP_OK;
  double Dw;
  gp_status q = emd_window_dual(s, z.win_n, &Dw, st);
  if (q == GP_OK && Dw > z.d_best) z.d_best = Dw;
  return q;
}

// After a plain check filled rep (P, the iterate's D, the plain gap).
gp_status emd_stop_check(gp_state s, EmdStop& z, double tol, gp_report* rep, cudaStream_t st, bool* certified,
                         bool* stop) {
  gp_handle h = s->h;
  const size_t NN = (size_t)s->N * s->N;
  gp_status r;
  *stop = false;
  if (rep->dual > z.d_best) z.d_best = rep->dual;
  if (z.win_start < 0 && rep->rel_gap <= 30.0 * tol) z.win_start = s->n;
  bool fresh = false;
  if (z.win_start >= 0) {
    if (s->n >= 2 * z.win_start && z.win_n > 0) {  // restart the window
      if ((r = emd_close_window(s, z, st)) != GP_OK) return r;
      z.win_n = 0;
      z.win_start = s->n;
      z.win_eval = s->n + 100;
      fresh = true;
    }
    if (!s->pwin) GP_CUDA(h, cudaMalloc(&s->pwin, 2 * NN * sizeof(double)));
    if (!s->phiwin) GP_CUDA(h, cudaMalloc(&s->phiwin, NN * sizeof(float)));
    if (z.win_n == 0) GP_CUDA(h, cudaMemsetAsync(s->pwin, 0, 2 * NN * sizeof(double), st));
    GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_accumulate(s->pwin, s->p[s->cur], 2 * NN, st); }));
    ++z.win_n;
    if (!fresh && z.win_n >= 4 && s->n >= z.win_eval) {  // take the open window's bound
      if ((r = emd_close_window(s, z, st)) != GP_OK) return r;
      const int grow = (s->n - z.win_start) / 4;
      z.win_eval = s->n + (grow > 100 ? grow : 100);
      fresh = true;
    }
  }
  rep->dual = z.d_best;
  rep->rel_gap = rel_gap_of(rep->primal, z.d_best);
  const double g_est = rel_gap_of(rep->primal - z.p_off, z.d_best);
  if (fresh || (g_est <= 2.0 * tol && (g_est <= tol || s->n - z.last_cert >= 100))) {
    z.last_cert = s->n;
    if (!fresh && (r = emd_close_window(s, z, st)) != GP_OK) return r;
    if ((r = emd_certify(s, rep, st)) != GP_OK) return r;
    z.p_off = fmax(0.0, rep->primal - rep->primal_feasible);
    rep->dual = z.d_best;
    rep->rel_gap = rel_gap_of(rep->primal, z.d_best);
    rep->rel_gap_feasible = rel_gap_of(rep->primal_feasible, z.d_best);
    *certified = true;
    *stop = rep->rel_gap_feasible <= tol;
  }
  return GP_OK;
}

// The certificate of the returned iterate when the last check did not take it.
gp_status emd_stop_final(gp_state s, EmdStop& z, bool stop_test, gp_report* rep, cudaStream_t st) {
  gp_status r;
  if (rep->dual > z.d_best) z.d_best = rep->dual;  // a solve with no check yet (max_iters == 0)
  if (stop_test && (r = emd_close_window(s, z, st)) != GP_OK) return r;
  if ((r = emd_certify(s, rep, st)) != GP_OK) return r;
  if (stop_test) {
    rep->dual = z.d_best;
    rep->rel_gap = rel_gap_of(rep->primal, z.d_best);
    rep->rel_gap_feasible = rel_gap_of(rep->primal_feasible, z.d_best);
  }
  return GP_OK;
}

// Chunked solve loop shared by rof_solve / emd_solve: run gap_every
// iterations (the last one with the fused gap reductions), check, repeat;
// gap_every == 0 takes the adaptive schedule above.
gp_status run_loop(gp_state s, const gp_opts& o, gp_report* rep, cudaStream_t st) {
  gp_handle h = s->h;
  DivergenceWatch watch;
  gp_status status = o.tol_rel_gap > 0 ? GP_ERR_MAXITER : GP_OK;
  rep->primal = rep->dual = rep->rel_gap = rep->mass_residual = NAN;
  rep->primal_feasible = rep->rel_gap_feasible = rep->mass_residual_feasible = NAN;
  const bool emd = s->kind == KIND_EMD;
  const bool stop_test = o.tol_rel_gap > 0;
  bool certified = false;  // the report's certificate belongs to the current iterate
  EmdStop z;
  gp_status r;
  if (o.max_iters == 0 && (r = state_gap(s, rep, st)) != GP_OK) return r;
  int k_next = o.gap_every > 0 ? o.gap_every : kAdaptiveMinChunk;
  int n_prev = -1;
  double g_prev = 0;
  while (s->n < o.max_iters) {
    const int k = std::min(k_next, o.max_iters - s->n);
    if ((r = run_steps(s, k, o.prec, true, o.use_graph != 0, st)) != GP_OK) return r;
    if ((r = state_gap(s, rep, st)) != GP_OK) return r;
    certified = false;
    if (!isfinite(rep->primal) || !isfinite(rep->dual)) {
      status = GP_ERR_NONFINITE;
      fail(h, status, "non-finite objective: the iteration broke down");
      break;
    }
    bool stop = false;
    if (emd && stop_test) {
      if ((r = emd_stop_check(s, z, o.tol_rel_gap, rep, st, &certified, &stop)) != GP_OK) return r;
    } else {
      stop = stop_test && rep->rel_gap <= o.tol_rel_gap;
    }
    if (stop) {
      status = GP_OK;
      break;
    }
    if (watch.update(rep->rel_gap)) {
      status = GP_ERR_DIVERGED;
      fail(h, status, "relative gap diverged");
      break;
    }
    if (o.gap_every == 0) {
      k_next = adaptive_chunk(n_prev, g_prev, s->n, rep->rel_gap, o.tol_rel_gap);
      n_prev = s->n;
      g_prev = rep->rel_gap;
    }
  }
  if (emd && !certified && status != GP_ERR_NONFINITE && isfinite(rep->dual) &&
      (r = emd_stop_final(s, z, stop_test, rep, st)) != GP_OK)
    return r;
  rep->iters = s->n;
  rep->tau = s->tau;
  rep->sigma = s->sigma;
  rep->status = status;
  return status;
}

// ------------------------------------------------------------ 3-D solves
gp_status ensure_v3(gp_handle h, size_t floats) {
  if (floats <= h->v3_cap) return GP_OK;
  if (h->v3) cudaFree(h->v3);
  h->v3 = nullptr;
  h->v3_cap = 0;
  GP_CUDA(h, cudaMalloc(&h->v3, floats * sizeof(float)));
  h->v3_cap = floats;
  return GP_OK;
}

gp_status check3(gp_handle h, int N, const gp_opts& o) {
  if (N < 16 || N > 512 || (N & (N - 1)) != 0)
    return fail(h, GP_ERR_ARG, "3-D solves take N a power of two in [16, 512]");
  if (o.prec != GP_PREC_FP32) return fail(h, GP_ERR_UNSUPPORTED, "3-D solves run the FP32 transform only");
  if (o.warm_start) return fail(h, GP_ERR_UNSUPPORTED, "3-D solves take no warm start");
  return GP_OK;
}

// x = scale (alpha - Lap)^{-1} b on N^3, its gradient into g3, x itself into u when u != nullptr.
gp_status solve3(gp_handle h, const DctPlan& p, const float* b, float* g3, float* u, float* W, double alpha,
                 double scale, cudaStream_t st) {
  const size_t n3 = (size_t)p.N * p.N * p.N;
  GP_CUDA(h, plaunch(h, PK_3D_LINES, st,
                     [&] {
                       return solve_grad3(p, b, g3, u, W, W + n3, W + 2 * n3, (float)alpha, (float)scale, st,
                                          nullptr);
                     },
                     u ? 13 : 12));
  return GP_OK;
}

// The chunked check loop of run_loop for the 3-D solves: step(k) runs k
// iterations, gap() fills rep's P, D and rel_gap for the current iterate.
template <typename Step, typename Gap>
gp_status loop3(gp_handle h, const gp_opts& o, gp_report* rep, Step&& step, Gap&& gap) {
  DivergenceWatch watch;
  gp_status status = o.tol_rel_gap > 0 ? GP_ERR_MAXITER : GP_OK;
  gp_status r;
  int n = 0;
  if (o.max_iters == 0 && (r = gap()) != GP_OK) return r;
  int k_next = o.gap_every > 0 ? o.gap_every : kAdaptiveMinChunk;
  int n_prev = -1;
  double g_prev = 0;
  while (n < o.max_iters) {
    const int k = std::min(k_next, o.max_iters - n);
    if ((r = step(k)) != GP_OK) return r;
    n += k;
    if ((r = gap()) != GP_OK) return r;
    if (!isfinite(rep->primal) || !isfinite(rep->dual)) {
      status = GP_ERR_NONFINITE;
      fail(h, status, "non-finite objective: the iteration broke down");
      break;
    }
    if (o.tol_rel_gap > 0 && rep->rel_gap <= o.tol_rel_gap) {
      status = GP_OK;
      break;
    }
    if (watch.update(rep->rel_gap)) {
      status = GP_ERR_DIVERGED;
      fail(h, status, "relative gap diverged");
      break;
    }
    if (o.gap_every == 0) {
      k_next = adaptive_chunk(n_prev, g_prev, n, rep->rel_gap, o.tol_rel_gap);
      n_prev = n;
      g_prev = rep->rel_gap;
    }
  }
  rep->iters = n;
  rep->status = status;
  return status;
}

bool solve_status_has_outputs(gp_status s) {
  return s == GP_OK || s == GP_ERR_MAXITER || s == GP_ERR_DIVERGED || s == GP_ERR_NONFINITE;
}

}  // namespace

// =================================================================== ABI
extern "C" {

int gp_abi_version(void) { return GP_ABI_VERSION; }

void gp_default_opts(gp_opts* o) {
  if (!o) return;
  o->max_iters = 1000;
  o->gap_every = 10;
  o->tol_rel_gap = 1e-5;
  o->tau = 0.0;
  o->sigma = 0.0;
  o->tau_scale = 1.0;
  o->eps = 1e-3;
  o->prec = GP_PREC_FP32;
  o->use_graph = 0;
  o->warm_start = 0;
}

gp_status gp_create(gp_handle* out, int device) {
  if (!out) return GP_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess) {
    cudaGetLastError();
    return GP_ERR_CUDA;
  }
  if (device < 0 || device >= n) return GP_ERR_ARG;
  gp_handle h = new gp_handle_s();
  h->device = device;
  *out = h;
  return GP_OK;
}

gp_status gp_destroy(gp_handle h) {
  if (!h) return GP_OK;
  DeviceGuard g(h->device);
  cudaDeviceSynchronize();
  for (auto& kv : h->cache) free_state(kv.second);
  for (gp_state b : h->batch) free_state(b);
  for (cudaStream_t a : h->aux) cudaStreamDestroy(a);
  for (cudaEvent_t e : h->evs) cudaEventDestroy(e);
  if (h->bres_d) cudaFree(h->bres_d);
  if (h->bres_h) cudaFreeHost(h->bres_h);
  for (auto& kv : h->plans) dct_plan_free(kv.second);
  for (cudaEvent_t e : h->prof.pool) cudaEventDestroy(e);
  if (h->ws) cudaFree(h->ws);
  if (h->v3) cudaFree(h->v3);
  if (h->rf) cudaFree(h->rf);
  if (h->rfd) cudaFree(h->rfd);
  if (h->tc_err) cudaFree(h->tc_err);
  if (h->part) cudaFree(h->part);
  if (h->dres) cudaFree(h->dres);
  if (h->hres) cudaFreeHost(h->hres);
  delete h;
  return GP_OK;
}

const char* gp_last_error(gp_handle h) { return h ? h->err.c_str() : static_last_error(); }

gp_status dct2_poisson(gp_handle h, const float* b, float* x, int N, double alpha, int prec, void* stream) {
  if (!h) return GP_ERR_ARG;
  h->err.clear();
  if (N < 1 || N > 8192) return fail(h, GP_ERR_ARG, "N out of range [1, 8192]");
  if (!(alpha >= 0.0) || !isfinite(alpha)) return fail(h, GP_ERR_ARG, "alpha must be finite and >= 0");
  if (prec < 0 || prec > kPrecMax) return fail(h, GP_ERR_ARG, "unknown prec");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, GP_ERR_CUDA, "cudaSetDevice failed");
  gp_status r;
  if ((r = check_ptr(h, b, "b")) != GP_OK) return r;
  if ((r = check_ptr(h, x, "x")) != GP_OK) return r;
  const DctPlan* p = nullptr;
  if ((r = get_plan(h, N, &p)) != GP_OK) return r;
  const bool aligned = aligned16(b) && aligned16(x);
  if ((p->fft || prec_split(prec)) && !aligned)
    return fail(h, GP_ERR_ARG, "b and x must be 16-byte aligned for this size / precision");
  const size_t need = 2 * (size_t)N * N;
  if (h->ws_floats < need) {
    if (h->ws) cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_floats = 0;
    GP_CUDA(h, cudaMalloc(&h->ws, need * sizeof(float)));
    h->ws_floats = need;
  }
  r = solve(h, N, b, x, h->ws, alpha, 1.0, prec, true, (cudaStream_t)stream);
  if (r == GP_OK && prec_split(prec)) {
    // the tensor-core kernels report a timed-out wait through a flag: check it
    int flag = 0;
    GP_CUDA(h, cudaMemcpyAsync(&flag, h->tc_err, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    GP_CUDA(h, cudaStreamSynchronize((cudaStream_t)stream));
    if (flag) return fail(h, GP_ERR_CUDA, "tensor-core solve: a wait timed out");
  }
  return r;
}

gp_status dct2_poisson_grad(gp_handle h, const float* b, float* g, int N, double alpha, int prec, void* stream) {
  if (!h) return GP_ERR_ARG;
  h->err.clear();
  if (N < 1 || N > 8192) return fail(h, GP_ERR_ARG, "N out of range [1, 8192]");
  if (!(alpha >= 0.0) || !isfinite(alpha)) return fail(h, GP_ERR_ARG, "alpha must be finite and >= 0");
  if (prec < 0 || prec > kPrecMax) return fail(h, GP_ERR_ARG, "unknown prec");
  DeviceGuard dg(h->device);
  if (!dg.ok) return fail(h, GP_ERR_CUDA, "cudaSetDevice failed");
  gp_status r;
  if ((r = check_ptr(h, b, "b")) != GP_OK) return r;
  if ((r = check_ptr(h, g, "g")) != GP_OK) return r;
  const DctPlan* p = nullptr;
  if ((r = get_plan(h, N, &p)) != GP_OK) return r;
  if (p->fft && !(aligned16(b) && aligned16(g)))
    return fail(h, GP_ERR_ARG, "b and g must be 16-byte aligned for power-of-two N");
  const size_t NN = (size_t)N * N;
  const size_t need = 3 * NN;  // 2 N^2 transform scratch + N^2 for the potential
  if (h->ws_floats < need) {
    if (h->ws) cudaFree(h->ws);
    h->ws = nullptr;
    h->ws_floats = 0;
    GP_CUDA(h, cudaMalloc(&h->ws, need * sizeof(float)));
    h->ws_floats = need;
  }
  return solve_grad(h, N, b, g, h->ws + 2 * NN, false, h->ws, alpha, 1.0, prec, (cudaStream_t)stream);
}

gp_status gp_state_create_rof(gp_handle h, gp_state* out, const float* I, int N, double lambda, double tau,
                              double sigma, const float* u0, const float* p0, const float* pbar0, void* stream) {
  if (!h || !out) return GP_ERR_ARG;
  h->err.clear();
  *out = nullptr;
  if (N < 1 || N > 8192) return fail(h, GP_ERR_ARG, "N out of range [1, 8192]");
  if (!(lambda > 0) || !(tau > 0) || !(sigma > 0)) return fail(h, GP_ERR_ARG, "lambda, tau, sigma must be > 0");
  DeviceGuard g(h->device);
  gp_status r;
  if ((r = check_ptr(h, I, "I")) != GP_OK) return r;
  if (u0 && (r = check_ptr(h, u0, "u0")) != GP_OK) return r;
  if (p0 && (r = check_ptr(h, p0, "p0")) != GP_OK) return r;
  if (pbar0 && (r = check_ptr(h, pbar0, "pbar0")) != GP_OK) return r;
  gp_state s = nullptr;
  if ((r = alloc_state(h, KIND_ROF, N, &s)) != GP_OK) return r;
  if ((r = rof_setup(s, I, lambda, tau, sigma, u0, p0, pbar0, (cudaStream_t)stream)) != GP_OK) {
    free_state(s);
    return r;
  }
  *out = s;
  return GP_OK;
}

gp_status gp_state_create_emd(gp_handle h, gp_state* out, const float* f0, const float* f1, int N, double tau,
                              double sigma, const float* m0, const float* p0, const float* pbar0, void* stream) {
  if (!h || !out) return GP_ERR_ARG;
  h->err.clear();
  *out = nullptr;
  if (N < 1 || N > 8192) return fail(h, GP_ERR_ARG, "N out of range [1, 8192]");
  if (!(tau > 0) || !(sigma > 0)) return fail(h, GP_ERR_ARG, "tau, sigma must be > 0");
  DeviceGuard g(h->device);
  gp_status r;
  if ((r = check_ptr(h, f0, "f0")) != GP_OK) return r;
  if ((r = check_ptr(h, f1, "f1")) != GP_OK) return r;
  if (m0 && (r = check_ptr(h, m0, "m0")) != GP_OK) return r;
  if (p0 && (r = check_ptr(h, p0, "p0")) != GP_OK) return r;
  if (pbar0 && (r = check_ptr(h, pbar0, "pbar0")) != GP_OK) return r;
  gp_state s = nullptr;
  if ((r = alloc_state(h, KIND_EMD, N, &s)) != GP_OK) return r;
  double ms[3];
  if ((r = mass_stats(h, f0, f1, N, ms, (cudaStream_t)stream)) != GP_OK || (r = check_mass(h, ms)) != GP_OK ||
      (r = emd_setup(s, f0, f1, tau, sigma, m0, p0, pbar0, (cudaStream_t)stream)) != GP_OK) {
    free_state(s);
    return r;
  }
  s->mass_den = ms[2];
  *out = s;
  return GP_OK;
}

gp_status pd_step(gp_handle h, gp_state s, int n_steps, int prec, void* stream) {
  if (!h || !s || s->h != h) return h ? fail(h, GP_ERR_ARG, "state does not belong to handle") : GP_ERR_ARG;
  h->err.clear();
  if (n_steps < 0) return fail(h, GP_ERR_ARG, "n_steps < 0");
  if (prec < 0 || prec > kPrecMax) return fail(h, GP_ERR_ARG, "unknown prec");
  DeviceGuard g(h->device);
  if (n_steps == 0) return GP_OK;
  // The last step of every call also leaves the gap partials (and, for EMD,
  // m and -div p) of the new iterate, so the state can be read or checked.
  return run_steps(s, n_steps, prec, true, false, (cudaStream_t)stream);
}

gp_status gp_state_read(gp_handle h, gp_state s, float* primal, float* p, void* stream) {
  if (!h || !s || s->h != h) return GP_ERR_ARG;
  h->err.clear();
  DeviceGuard g(h->device);
  gp_status r;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t NN = (size_t)s->N * s->N;
  if (primal) {
    if ((r = check_ptr(h, primal, "primal")) != GP_OK) return r;
    if (s->kind == KIND_ROF)
      GP_CUDA(h, cudaMemcpyAsync(primal, s->prim, NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
    else
      GP_CUDA(h, cudaMemcpyAsync(primal, s->m, 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  }
  if (p) {
    if ((r = check_ptr(h, p, "p")) != GP_OK) return r;
    GP_CUDA(h, cudaMemcpyAsync(p, s->p[s->cur], 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  }
  return GP_OK;
}

gp_status gp_state_average(gp_handle h, gp_state s, int enable, void* stream) {
  if (!h || !s || s->h != h) return h ? fail(h, GP_ERR_ARG, "state does not belong to handle") : GP_ERR_ARG;
  h->err.clear();
  DeviceGuard g(h->device);
  drop_graphs(s);  // captured chunks differ with and without the sums
  if (!enable) {
    if (s->avg_sum) cudaFree(s->avg_sum);
    s->avg_sum = nullptr;
    s->avg_n = 0;
    return GP_OK;
  }
  const size_t NN = (size_t)s->N * s->N;
  const size_t planes = s->kind == KIND_ROF ? 3 : 5;
  if (!s->avg_sum) GP_CUDA(h, cudaMalloc(&s->avg_sum, planes * NN * sizeof(double)));
  GP_CUDA(h, cudaMemsetAsync(s->avg_sum, 0, planes * NN * sizeof(double), (cudaStream_t)stream));
  s->avg_n = 0;
  return GP_OK;
}

gp_status gp_state_read_average(gp_handle h, gp_state s, float* primal, float* p, long long* count,
                                void* stream) {
  if (!h || !s || s->h != h) return h ? fail(h, GP_ERR_ARG, "state does not belong to handle") : GP_ERR_ARG;
  h->err.clear();
  if (count) *count = s->avg_n;
  if (!s->avg_sum || s->avg_n == 0) return fail(h, GP_ERR_ARG, "no averaged steps (gp_state_average, then pd_step)");
  DeviceGuard g(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  const int N = s->N;
  const size_t NN = (size_t)N * N;
  const double inv = 1.0 / (double)s->avg_n;
  gp_status r;
  if (p) {
    if ((r = check_ptr(h, p, "p")) != GP_OK) return r;
    const double* ps = s->avg_sum + (s->kind == KIND_ROF ? NN : 3 * NN);
    GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_scale_sum(ps, p, 2 * NN, inv, st); }));
  }
  if (primal) {
    if ((r = check_ptr(h, primal, "primal")) != GP_OK) return r;
    if (s->kind == KIND_ROF) {
      // mean of u_{n+1} = (lambda tau - Lap)^{-1} (mean of r_n), solved into `primal`
      GP_CUDA(h, plaunch(h, PK_SETUP, st, [&] { return launch_scale_sum(s->avg_sum, primal, NN, inv, st); }));
      if ((r = solve_grad(h, N, primal, s->gu, primal, true, s->tmp, s->lam * s->tau, 1.0, GP_PREC_FP32, st)) !=
          GP_OK)
        return r;
    } else {
      // mean of m_{n+1} = mean(s_n) + grad q, q = Lap^{-1} mean(d_n); `primal` plane 0 holds mean(d_n)
      // for the solve (plane 1 is scratch), then both planes the flux
      GP_CUDA(h, plaunch(h, PK_SETUP, st,
                         [&] { return launch_scale_sum(s->avg_sum + 2 * NN, primal, NN, inv, st); }));
      if ((r = solve_grad(h, N, primal, s->prim, primal + NN, false, s->tmp, 0.0, -1.0, GP_PREC_FP32, st)) != GP_OK)
        return r;
      GP_CUDA(h, plaunch(h, PK_SETUP, st,
                         [&] { return launch_emd_average_flux(s->avg_sum, s->prim, primal, 2 * NN, inv, st); }));
    }
  }
  return GP_OK;
}

gp_status gp_state_gap(gp_handle h, gp_state s, gp_report* rep, void* stream) {
  if (!h || !s || s->h != h || !rep) return GP_ERR_ARG;
  h->err.clear();
  DeviceGuard g(h->device);
  Timer t;
  memset(rep, 0, sizeof(*rep));
  gp_status r = state_gap(s, rep, (cudaStream_t)stream);
  rep->iters = s->n;
  rep->tau = s->tau;
  rep->sigma = s->sigma;
  rep->status = r;
  rep->seconds = t.s();
  return r;
}

gp_status gp_state_certify(gp_handle h, gp_state s, gp_report* rep, void* stream) {
  if (!h || !s || s->h != h || !rep) return GP_ERR_ARG;
  h->err.clear();
  DeviceGuard g(h->device);
  Timer t;
  memset(rep, 0, sizeof(*rep));
  gp_status r = state_gap(s, rep, (cudaStream_t)stream);
  if (r == GP_OK && s->kind == KIND_EMD && isfinite(rep->dual)) r = emd_certify(s, rep, (cudaStream_t)stream);
  rep->iters = s->n;
  rep->tau = s->tau;
  rep->sigma = s->sigma;
  rep->status = r;
  rep->seconds = t.s();
  return r;
}

gp_status gp_state_destroy(gp_state s) {
  if (!s) return GP_OK;
  DeviceGuard g(s->h->device);
  cudaDeviceSynchronize();
  free_state(s);
  return GP_OK;
}

gp_status rof_solve(gp_handle h, const float* I, float* u, float* p, int N, double lambda, const gp_opts* opts,
                    gp_report* report, void* stream) {
  if (!h) return GP_ERR_ARG;
  h->err.clear();
  Timer t;
  gp_opts o;
  gp_default_opts(&o);
  if (opts) o = *opts;
  gp_report rep;
  memset(&rep, 0, sizeof(rep));
  gp_status r = check_opts(h, &o);
  if (r != GP_OK) return r;
  if (N < 1 || N > 8192) return fail(h, GP_ERR_ARG, "N out of range [1, 8192]");
  if (!(lambda > 0) || !isfinite(lambda)) return fail(h, GP_ERR_ARG, "lambda must be finite and > 0");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, GP_ERR_CUDA, "cudaSetDevice failed");
  if ((r = check_ptr(h, I, "I")) != GP_OK) return r;
  if ((r = check_ptr(h, u, "u")) != GP_OK) return r;
  if (p && (r = check_ptr(h, p, "p")) != GP_OK) return r;
  if (o.warm_start && !p) return fail(h, GP_ERR_ARG, "warm_start needs p");
  cudaStream_t st = (cudaStream_t)stream;
  double tau = o.tau;
  if (!(tau > 0) && (r = rof_rule(h, I, N, lambda, o, &tau, st)) != GP_OK) return r;
  const double sigma = o.sigma > 0 ? o.sigma : 1.0 / tau;
  gp_state s = cached_state(h, KIND_ROF, N, &r);
  if (!s) return r;
  if ((r = rof_setup(s, I, lambda, tau, sigma, o.warm_start ? u : nullptr, o.warm_start ? p : nullptr, nullptr,
                     st)) != GP_OK)
    return r;
  gp_status status = run_loop(s, o, &rep, st);
  if (!solve_status_has_outputs(status)) return status;
  const size_t NN = (size_t)N * N;
  GP_CUDA(h, cudaMemcpyAsync(u, s->prim, NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (p) GP_CUDA(h, cudaMemcpyAsync(p, s->p[s->cur], 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  GP_CUDA(h, cudaStreamSynchronize(st));
  rep.seconds = t.s();
  if (report) *report = rep;
  return status;
}

gp_status rof_solve_cp2(gp_handle h, const float* I, float* u, float* p, int N, double lambda, const gp_opts* opts,
                        gp_report* report, void* stream) {
  if (!h) return GP_ERR_ARG;
  h->err.clear();
  Timer t;
  gp_opts o;
  gp_default_opts(&o);
  if (opts) o = *opts;
  gp_report rep;
  memset(&rep, 0, sizeof(rep));
  gp_status r = check_opts(h, &o);
  if (r != GP_OK) return r;
  if (N < 2 || N > 8192) return fail(h, GP_ERR_ARG, "N out of range [2, 8192]");
  if (!(lambda > 0) || !isfinite(lambda)) return fail(h, GP_ERR_ARG, "lambda must be finite and > 0");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, GP_ERR_CUDA, "cudaSetDevice failed");
  if ((r = check_ptr(h, I, "I")) != GP_OK) return r;
  if ((r = check_ptr(h, u, "u")) != GP_OK) return r;
  if (p && (r = check_ptr(h, p, "p")) != GP_OK) return r;
  if (o.warm_start && !p) return fail(h, GP_ERR_ARG, "warm_start needs p");
  cudaStream_t st = (cudaStream_t)stream;
  gp_state s = cached_state(h, KIND_ROF, N, &r);  // its planes: u (prim), ubar (gu), p (p[0]), partials
  if (!s) return r;
  const size_t NN = (size_t)N * N;
  float* us = s->prim;
  float* ub = s->gu;
  float* ps = s->p[0];
  if (o.warm_start) {
    GP_CUDA(h, cudaMemcpyAsync(us, u, NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
    GP_CUDA(h, cudaMemcpyAsync(ps, p, 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  } else {
    GP_CUDA(h, cudaMemsetAsync(us, 0, NN * sizeof(float), st));
    GP_CUDA(h, cudaMemsetAsync(ps, 0, 2 * NN * sizeof(float), st));
  }
  GP_CUDA(h, cudaMemcpyAsync(ub, us, NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  // section 4.1: tau0 = sigma0 = 1 / sqrt(||Lap||), ||Lap|| = 2 mu_{N-1} = (8 / h^2) sin^2(pi (N-1) / 2N)
  const double PI = 3.14159265358979323846;
  const double sn = sin(PI * (N - 1) / (2.0 * N));
  const double t0 = 1.0 / sqrt(8.0 * (double)N * N * sn * sn);
  const double ts = o.tau_scale > 0 ? o.tau_scale : 1.0;
  double tau = o.tau > 0 ? o.tau : t0 * ts, sigma = o.sigma > 0 ? o.sigma : t0 / ts;
  const int every = o.gap_every > 0 ? o.gap_every : 10;
  const int nb = reduce_blocks_1d(NN);
  if ((r = ensure_res(h)) != GP_OK) return r;
  gp_status status = o.tol_rel_gap > 0 ? GP_ERR_MAXITER : GP_OK;
  rep.primal = rep.dual = rep.rel_gap = NAN;
  const double h2 = 1.0 / ((double)N * N);
  auto gap = [&]() -> gp_status {
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_rof_gap(us, ps, I, N, s->part, nb, st); }));
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(s->part, nb, 4, 0u, h->dres, st); }));
    gp_status q = fetch(h, 4, st);
    if (q != GP_OK) return q;
    const double* v = h->hres;
    finish_report(&rep, h2 * (v[0] + 0.5 * lambda * v[1]), -h2 * v[2] - h2 * v[3] / (2.0 * lambda));
    return GP_OK;
  };
  int n = 0;
  if (o.max_iters == 0 && (r = gap()) != GP_OK) return r;
  while (n < o.max_iters) {
    const int k = std::min(every, o.max_iters - n);
    for (int q = 0; q < k; ++q) {
      const double theta = 1.0 / sqrt(1.0 + 2.0 * lambda * tau);
      GP_CUDA(h, plaunch(h, PK_CP2_DUAL, st, [&] { return launch_cp2_dual(ub, ps, N, (float)sigma, st); }));
      GP_CUDA(h, plaunch(h, PK_CP2_PRIMAL, st,
                         [&] { return launch_cp2_primal(us, ub, ps, I, N, tau, lambda, theta, st); }));
      tau *= theta;
      sigma /= theta;
    }
    n += k;
    if ((r = gap()) != GP_OK) return r;
    if (!isfinite(rep.primal) || !isfinite(rep.dual)) {
      status = fail(h, GP_ERR_NONFINITE, "non-finite objective: the iteration broke down");
      break;
    }
    if (o.tol_rel_gap > 0 && rep.rel_gap <= o.tol_rel_gap) {
      status = GP_OK;
      break;
    }
  }
  rep.iters = n;
  rep.tau = tau;
  rep.sigma = sigma;
  rep.status = status;
  rep.mass_residual = 0.0;
  rep.primal_feasible = rep.primal;  // no constraint on u
  rep.rel_gap_feasible = rep.rel_gap;
  rep.mass_residual_feasible = 0.0;
  GP_CUDA(h, cudaMemcpyAsync(u, us, NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (p) GP_CUDA(h, cudaMemcpyAsync(p, ps, 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  GP_CUDA(h, cudaStreamSynchronize(st));
  s->partials_valid = false;  // the state's partials now hold CP2's gap terms
  rep.seconds = t.s();
  if (report) *report = rep;
  return status;
}

gp_status rof_solve3d(gp_handle h, const float* I, float* u, float* p, int N, double lambda, const gp_opts* opts,
                      gp_report* report, void* stream) {
  if (!h) return GP_ERR_ARG;
  h->err.clear();
  Timer t;
  gp_opts o;
  gp_default_opts(&o);
  if (opts) o = *opts;
  gp_report rep;
  memset(&rep, 0, sizeof(rep));
  gp_status r = check_opts(h, &o);
  if (r != GP_OK || (r = check3(h, N, o)) != GP_OK) return r;
  if (!(lambda > 0) || !isfinite(lambda)) return fail(h, GP_ERR_ARG, "lambda must be finite and > 0");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, GP_ERR_CUDA, "cudaSetDevice failed");
  if ((r = check_ptr(h, I, "I")) != GP_OK) return r;
  if ((r = check_ptr(h, u, "u")) != GP_OK) return r;
  if (p && (r = check_ptr(h, p, "p")) != GP_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  const DctPlan* plan = nullptr;
  if ((r = get_plan(h, N, &plan)) != GP_OK) return r;
  const size_t n3 = (size_t)N * N * N;
  // volumes: grad u (3), p ping-pong (3 + 3), r, u, solve scratch (3)
  if ((r = ensure_v3(h, 14 * n3)) != GP_OK) return r;
  float* gu = h->v3;
  float* pp[2] = {gu + 3 * n3, gu + 6 * n3};
  float* rr = gu + 9 * n3;
  float* us = rr + n3;
  float* W = us + n3;
  const int nb = reduce_blocks_1d(n3);
  if ((r = ensure_part(h, (size_t)nb * 4)) != GP_OK) return r;
  if ((r = ensure_res(h)) != GP_OK) return r;
  const double h3 = 1.0 / (double)n3;
  // step rule of rof_solve with h^3 weights (sections 3.1 and 4.1)
  double tau = o.tau;
  if (!(tau > 0)) {
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_rof3_stats(I, N, h->part, nb, st); }));
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(h->part, nb, 3, 0u, h->dres, st); }));
    if ((r = fetch(h, 3, st)) != GP_OK) return r;
    const double tv = h3 * h->hres[0], grad_l2 = sqrt(h3 * h->hres[1]), mean = h->hres[2] / (double)n3;
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_sq_dev(I, n3, (float)mean, h->part, nb, st); }));
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(h->part, nb, 1, 0u, h->dres, st); }));
    if ((r = fetch(h, 1, st)) != GP_OK) return r;
    const double fid = 0.5 * lambda * h3 * h->hres[0];
    if (!isfinite(tv) || !isfinite(fid)) return fail(h, GP_ERR_NONFINITE, "non-finite image");
    const double eps = o.eps > 0 ? o.eps : 1e-3;
    tau = fmin(sqrt(lambda) * fmin(tv, fid) / sqrt(eps), grad_l2);
    if (!(tau > 0)) tau = 1.0;  // constant image
    tau *= o.tau_scale > 0 ? o.tau_scale : 1.0;
  }
  const double sigma = o.sigma > 0 ? o.sigma : 1.0 / tau;
  const float lt = (float)(lambda * tau);
  // u_0 = 0, p_0 = pbar_0 = 0: r_0 = lambda tau I
  GP_CUDA(h, cudaMemsetAsync(gu, 0, 3 * n3 * sizeof(float), st));
  GP_CUDA(h, cudaMemsetAsync(pp[0], 0, 3 * n3 * sizeof(float), st));
  GP_CUDA(h, cudaMemsetAsync(us, 0, n3 * sizeof(float), st));
  GP_CUDA(h, plaunch(h, PK_3D_STENCIL, st,
                     [&] { return launch_rof3_rhs(pp[0], pp[0], gu, I, rr, N, lt, (float)tau, st); }));
  int cur = 0;
  auto step = [&](int k) -> gp_status {
    for (int q = 0; q < k; ++q) {
      gp_status e = solve3(h, *plan, rr, gu, q == k - 1 ? us : nullptr, W, lambda * tau, 1.0, st);
      if (e != GP_OK) return e;
      float* pin = pp[cur];
      float* pout = pp[cur ^ 1];
      GP_CUDA(h, plaunch(h, PK_3D_STENCIL, st, [&] { return launch_rof3_pstep(gu, pin, pout, N, (float)sigma, st); }));
      GP_CUDA(h, plaunch(h, PK_3D_STENCIL, st,
                         [&] { return launch_rof3_rhs(pout, pin, gu, I, rr, N, lt, (float)tau, st); }));
      cur ^= 1;
    }
    return GP_OK;
  };
  auto gap = [&]() -> gp_status {
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_rof3_gap(us, gu, I, pp[cur], N, h->part, nb, st); }));
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(h->part, nb, 4, 0u, h->dres, st); }));
    gp_status e = fetch(h, 4, st);
    if (e != GP_OK) return e;
    const double* v = h->hres;
    finish_report(&rep, h3 * (v[0] + 0.5 * lambda * v[1]), -h3 * v[2] - h3 * v[3] / (2.0 * lambda));
    return GP_OK;
  };
  gp_status status = loop3(h, o, &rep, step, gap);
  if (!solve_status_has_outputs(status)) return status;
  rep.tau = tau;
  rep.sigma = sigma;
  rep.mass_residual = 0.0;
  rep.primal_feasible = rep.primal;  // no constraint on u
  rep.rel_gap_feasible = rep.rel_gap;
  rep.mass_residual_feasible = 0.0;
  GP_CUDA(h, cudaMemcpyAsync(u, us, n3 * sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (p) GP_CUDA(h, cudaMemcpyAsync(p, pp[cur], 3 * n3 * sizeof(float), cudaMemcpyDeviceToDevice, st));
  GP_CUDA(h, cudaStreamSynchronize(st));
  rep.seconds = t.s();
  if (report) *report = rep;
  return status;
}

gp_status emd_solve3d(gp_handle h, const float* f0, const float* f1, float* m, float* p, int N, const gp_opts* opts,
                      gp_report* report, void* stream) {
  if (!h) return GP_ERR_ARG;
  h->err.clear();
  Timer t;
  gp_opts o;
  gp_default_opts(&o);
  if (opts) o = *opts;
  gp_report rep;
  memset(&rep, 0, sizeof(rep));
  gp_status r = check_opts(h, &o);
  if (r != GP_OK || (r = check3(h, N, o)) != GP_OK) return r;
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, GP_ERR_CUDA, "cudaSetDevice failed");
  if ((r = check_ptr(h, f0, "f0")) != GP_OK) return r;
  if ((r = check_ptr(h, f1, "f1")) != GP_OK) return r;
  if ((r = check_ptr(h, m, "m")) != GP_OK) return r;
  if (p && (r = check_ptr(h, p, "p")) != GP_OK) return r;
  cudaStream_t st = (cudaStream_t)stream;
  const DctPlan* plan = nullptr;
  if ((r = get_plan(h, N, &plan)) != GP_OK) return r;
  const size_t n3 = (size_t)N * N * N;
  const int nb = reduce_blocks_1d(n3);
  if ((r = ensure_part(h, (size_t)nb * 4)) != GP_OK) return r;
  if ((r = ensure_res(h)) != GP_OK) return r;
  double ms[3];
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_mass_stats(f0, f1, n3, h->part, nb, st); }));
  GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(h->part, nb, 3, 0u, h->dres, st); }));
  if ((r = fetch(h, 3, st)) != GP_OK) return r;
  for (int q = 0; q < 3; ++q) ms[q] = h->hres[q];
  if ((r = check_mass(h, ms)) != GP_OK) return r;
  // volumes: g, d, s ping-pong (3 + 3), p ping-pong (3 + 3), grad q (3), m (3), phi, -div p, scratch (3)
  if ((r = ensure_v3(h, 25 * n3)) != GP_OK) return r;
  float* gg = h->v3;
  float* dd = gg + n3;
  float* ss[2] = {dd + n3, dd + 4 * n3};
  float* pp[2] = {dd + 7 * n3, dd + 10 * n3};
  float* gq = dd + 13 * n3;
  float* mm = gq + 3 * n3;
  float* phi = mm + 3 * n3;
  float* ee = phi + n3;
  float* W = ee + n3;
  // section 4.2: tau = sigma = 1 for bounded densities
  const double tau = o.tau > 0 ? o.tau : (o.tau_scale > 0 ? o.tau_scale : 1.0);
  const double sigma = o.sigma > 0 ? o.sigma : 1.0 / tau;
  // s_0 = 0, p_0 = 0, d_0 = g: the first step's solve gives m_0 = grad psi, Lap psi = f0 - f1
  GP_CUDA(h, plaunch(h, PK_3D_STENCIL, st, [&] { return launch_sub(f0, f1, gg, n3, st); }));
  GP_CUDA(h, cudaMemcpyAsync(dd, gg, n3 * sizeof(float), cudaMemcpyDeviceToDevice, st));
  GP_CUDA(h, cudaMemsetAsync(ss[0], 0, 3 * n3 * sizeof(float), st));
  GP_CUDA(h, cudaMemsetAsync(pp[0], 0, 3 * n3 * sizeof(float), st));
  // q = Lap^{-1} d  <=>  (0 - Lap) q = -d
  if (o.max_iters == 0 && (r = solve3(h, *plan, dd, mm, nullptr, W, 0.0, -1.0, st)) != GP_OK) return r;
  int cur = 0;
  auto step = [&](int k) -> gp_status {
    for (int q = 0; q < k; ++q) {
      gp_status e = solve3(h, *plan, dd, gq, nullptr, W, 0.0, -1.0, st);  // grad q, Lap q = d
      if (e != GP_OK) return e;
      float* mo = q == k - 1 ? mm : nullptr;
      const int c = cur;
      GP_CUDA(h, plaunch(h, PK_3D_STENCIL, st, [&] {
                return launch_emd3_step(gq, ss[c], pp[c], ss[c ^ 1], pp[c ^ 1], mo, N, (float)tau, (float)sigma, st);
              }));
      GP_CUDA(h, plaunch(h, PK_3D_STENCIL, st, [&] { return launch_emd3_rhs(ss[c ^ 1], gg, dd, N, st); }));
      cur ^= 1;
    }
    return GP_OK;
  };
  auto gap = [&]() -> gp_status {
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_emd3_primal(mm, gg, N, h->part, nb, st); }));
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(h->part, nb, 2, 0u, h->dres, st); }));
    // phi = Lap^{-1} div p  <=>  (0 - Lap) phi = -div p; grad phi into gq (free between chunks)
    GP_CUDA(h, plaunch(h, PK_3D_STENCIL, st, [&] { return launch_div3(pp[cur], ee, N, -1.f, st); }));
    gp_status e = solve3(h, *plan, ee, gq, phi, W, 0.0, 1.0, st);
    if (e != GP_OK) return e;
    double* pd = h->part + (size_t)nb * 2;
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_emd3_dual(phi, gq, f0, f1, N, pd, nb, st); }));
    GP_CUDA(h, plaunch(h, PK_REDUCE, st, [&] { return launch_final_reduce(pd, nb, 2, 2u, h->dres + 2, st); }));
    if ((e = fetch(h, 4, st)) != GP_OK) return e;
    const double* v = h->hres;
    const double h3 = 1.0 / (double)n3;
    finish_report(&rep, h3 * v[0], h3 * v[2] / fmax(1.0, v[3]));
    rep.mass_residual = ms[2] > 0 ? v[1] / ms[2] : v[1];
    return GP_OK;
  };
  gp_status status = loop3(h, o, &rep, step, gap);
  if (!solve_status_has_outputs(status)) return status;
  rep.tau = tau;
  rep.sigma = sigma;
  rep.primal_feasible = rep.rel_gap_feasible = rep.mass_residual_feasible = NAN;  // no certificate in 3-D
  GP_CUDA(h, cudaMemcpyAsync(m, mm, 3 * n3 * sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (p) GP_CUDA(h, cudaMemcpyAsync(p, pp[cur], 3 * n3 * sizeof(float), cudaMemcpyDeviceToDevice, st));
  GP_CUDA(h, cudaStreamSynchronize(st));
  rep.seconds = t.s();
  if (report) *report = rep;
  return status;
}

gp_status emd_solve(gp_handle h, const float* f0, const float* f1, float* m, float* p, float* phi, int N,
                    const gp_opts* opts, gp_report* report, void* stream) {
  if (!h) return GP_ERR_ARG;
  h->err.clear();
  Timer t;
  gp_opts o;
  gp_default_opts(&o);
  if (opts) o = *opts;
  gp_report rep;
  memset(&rep, 0, sizeof(rep));
  gp_status r = check_opts(h, &o);
  if (r != GP_OK) return r;
  if (N < 1 || N > 8192) return fail(h, GP_ERR_ARG, "N out of range [1, 8192]");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, GP_ERR_CUDA, "cudaSetDevice failed");
  if ((r = check_ptr(h, f0, "f0")) != GP_OK) return r;
  if ((r = check_ptr(h, f1, "f1")) != GP_OK) return r;
  if ((r = check_ptr(h, m, "m")) != GP_OK) return r;
  if (p && (r = check_ptr(h, p, "p")) != GP_OK) return r;
  if (phi && (r = check_ptr(h, phi, "phi")) != GP_OK) return r;
  if (o.warm_start && !p) return fail(h, GP_ERR_ARG, "warm_start needs p");
  cudaStream_t st = (cudaStream_t)stream;
  double ms[3];
  if ((r = mass_stats(h, f0, f1, N, ms, st)) != GP_OK) return r;
  if ((r = check_mass(h, ms)) != GP_OK) return r;
  // section 4.2: tau = sigma = 1 for bounded densities
  const double tau = o.tau > 0 ? o.tau : (o.tau_scale > 0 ? o.tau_scale : 1.0);
  const double sigma = o.sigma > 0 ? o.sigma : 1.0 / tau;
  gp_state s = cached_state(h, KIND_EMD, N, &r);
  if (!s) return r;
  if ((r = emd_setup(s, f0, f1, tau, sigma, nullptr, o.warm_start ? p : nullptr, nullptr, st)) != GP_OK) return r;
  s->mass_den = ms[2];
  gp_status status = run_loop(s, o, &rep, st);
  if (!solve_status_has_outputs(status)) return status;
  const size_t NN = (size_t)N * N;
  GP_CUDA(h, cudaMemcpyAsync(m, s->m, 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (p) GP_CUDA(h, cudaMemcpyAsync(p, s->p[s->cur], 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  if (phi) GP_CUDA(h, cudaMemcpyAsync(phi, s->phi, NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
  GP_CUDA(h, cudaStreamSynchronize(st));
  rep.seconds = t.s();
  if (report) *report = rep;
  return status;
}

// ------------------------------------------------------- batched EMD
// Independent EMD problems of mixed sizes.  Each between-check chunk of all
// active problems is one CUDA graph with one branch per problem (its k steps
// and its gap reductions), so small problems run concurrently and the launch
// cost is paid once per chunk; all gap scalars come back in one copy per
// chunk.  The graph is re-instantiated when the set of active problems
// shrinks.
gp_status emd_solve_batched(gp_handle h, int B, const float* const* f0, const float* const* f1, float* const* m,
                            float* const* p_out, const int* N, const gp_opts* opts, gp_report* reports, void* stream) {
  if (!h) return GP_ERR_ARG;
  h->err.clear();
  Timer t;
  gp_opts o;
  gp_default_opts(&o);
  if (opts) o = *opts;
  gp_status r = check_opts(h, &o);
  if (r != GP_OK) return r;
  if (B < 1 || !f0 || !f1 || !m || !N || !reports) return fail(h, GP_ERR_ARG, "bad batch arguments");
  if (o.warm_start) return fail(h, GP_ERR_ARG, "warm_start is not available for batched solves");
  // the FP16 split's scale slots and the refinement scratch are per plan and
  // per handle: concurrent branches would share them
  if (prec_fp16(o.prec) || prec_refined(o.prec))
    return fail(h, GP_ERR_UNSUPPORTED, "batched solves take the FP32 or the BF16 split transform");
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, GP_ERR_CUDA, "cudaSetDevice failed");
  cudaStream_t st = (cudaStream_t)stream;
  if (st == nullptr) return fail(h, GP_ERR_ARG, "batched solves need a non-default stream (graph capture)");
  for (int b = 0; b < B; ++b) {
    if (N[b] < 1 || N[b] > 8192) return fail(h, GP_ERR_ARG, "N out of range [1, 8192]");
    if ((r = check_ptr(h, f0[b], "f0[b]")) != GP_OK || (r = check_ptr(h, f1[b], "f1[b]")) != GP_OK ||
        (r = check_ptr(h, m[b], "m[b]")) != GP_OK || (p_out && (r = check_ptr(h, p_out[b], "p[b]")) != GP_OK))
      return r;
  }
  const double tau = o.tau > 0 ? o.tau : (o.tau_scale > 0 ? o.tau_scale : 1.0);
  const double sigma = o.sigma > 0 ? o.sigma : 1.0 / tau;
  // states (reused across calls with the same sizes) and branch streams
  while ((int)h->batch.size() < B) h->batch.push_back(nullptr);
  while ((int)h->aux.size() < B) {
    cudaStream_t a;
    GP_CUDA(h, cudaStreamCreateWithFlags(&a, cudaStreamNonBlocking));
    h->aux.push_back(a);
  }
  if (!h->evs.size()) {
    for (int i = 0; i < 2 * 256; ++i) {
      cudaEvent_t e;
      GP_CUDA(h, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      h->evs.push_back(e);
    }
  }
  if (B > 256) return fail(h, GP_ERR_ARG, "at most 256 problems per batch");
  for (int b = 0; b < B; ++b) {
    gp_state& s = h->batch[b];
    if (s && s->N != N[b]) {
      free_state(s);
      s = nullptr;
    }
    if (!s && (r = alloc_state(h, KIND_EMD, N[b], &s)) != GP_OK) return r;
    double ms[3];
    if ((r = mass_stats(h, f0[b], f1[b], N[b], ms, st)) != GP_OK || (r = check_mass(h, ms)) != GP_OK) return r;
    if ((r = emd_setup(s, f0[b], f1[b], tau, sigma, nullptr, nullptr, nullptr, st)) != GP_OK) return r;
    s->mass_den = ms[2];
    memset(&reports[b], 0, sizeof(gp_report));
    reports[b].status = o.tol_rel_gap > 0 ? GP_ERR_MAXITER : GP_OK;
  }
  if (!h->bres_h) {
    GP_CUDA(h, cudaMallocHost(&h->bres_h, 256 * 4 * sizeof(double)));
    GP_CUDA(h, cudaMalloc(&h->bres_d, 256 * 4 * sizeof(double)));
  }
  // Warm every size once outside capture (plans, kernel attributes).
  for (int b = 0; b < B; ++b) {
    const DctPlan* p = nullptr;
    if ((r = get_plan(h, N[b], &p)) != GP_OK) return r;
  }
  std::vector<int> active;
  for (int b = 0; b < B; ++b) active.push_back(b);
  std::vector<DivergenceWatch> watch(B);
  std::vector<char> certified(B, 0);  // problem b's report holds the certificate of its current iterate
  std::vector<EmdStop> stops(B);
  cudaGraphExec_t exec = nullptr;
  int exec_k = -1;
  bool first = true;
  while (!active.empty()) {
    const int done_iters = h->batch[active[0]]->n;
    if (done_iters >= o.max_iters) break;
    const int k = std::min(o.gap_every > 0 ? o.gap_every : kAdaptiveMinChunk, o.max_iters - done_iters);
    if (!exec || exec_k != k || first) {
      if (exec) cudaGraphExecDestroy(exec);
      exec = nullptr;
      if (first) {
        // one direct chunk: sets kernel attributes before any capture
        for (int b : active) {
          gp_state s = h->batch[b];
          if ((r = run_steps(s, k, o.prec, true, false, st)) != GP_OK) return r;
          if ((r = state_gap_enqueue(s, h->bres_d + 4 * b, st)) != GP_OK) return r;
        }
        GP_CUDA(h, cudaMemcpyAsync(h->bres_h, h->bres_d, 4 * B * sizeof(double), cudaMemcpyDeviceToHost, st));
        GP_CUDA(h, cudaStreamSynchronize(st));
        first = false;
      } else {
        const int n0 = h->batch[active[0]]->n;
        std::vector<int> cur0;
        for (int b : active) cur0.push_back(h->batch[b]->cur);
        cudaGraph_t gr = nullptr;
        GP_CUDA(h, cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        h->capturing = true;
        gp_status cr = GP_OK;
        cudaEventRecord(h->evs[0], st);
        for (size_t i = 0; i < active.size() && cr == GP_OK; ++i) {
          const int b = active[i];
          cudaStream_t a = h->aux[b];
          cudaStreamWaitEvent(a, h->evs[0], 0);
          cr = run_steps(h->batch[b], k, o.prec, true, false, a);
          if (cr == GP_OK) cr = state_gap_enqueue(h->batch[b], h->bres_d + 4 * b, a);
          cudaEventRecord(h->evs[1 + i], a);
          cudaStreamWaitEvent(st, h->evs[1 + i], 0);
        }
        if (cr == GP_OK)
          cudaMemcpyAsync(h->bres_h, h->bres_d, 4 * B * sizeof(double), cudaMemcpyDeviceToHost, st);
        h->capturing = false;
        cudaError_t e = cudaStreamEndCapture(st, &gr);
        for (size_t i = 0; i < active.size(); ++i) {
          h->batch[active[i]]->cur = cur0[i];
          h->batch[active[i]]->n = n0;
        }
        if (cr != GP_OK) {
          if (gr) cudaGraphDestroy(gr);
          return cr;
        }
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
        e = cudaGraphInstantiate(&exec, gr, 0);
        cudaGraphDestroy(gr);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
        exec_k = k;
        GP_CUDA(h, cudaGraphLaunch(exec, st));
        GP_CUDA(h, cudaStreamSynchronize(st));
        for (int b : active) {
          gp_state s = h->batch[b];
          if (k & 1) s->cur = 1 - s->cur;
          s->n += k;
          s->partials_valid = true;
        }
      }
    } else {
      GP_CUDA(h, cudaGraphLaunch(exec, st));
      GP_CUDA(h, cudaStreamSynchronize(st));
      for (int b : active) {
        gp_state s = h->batch[b];
        if (k & 1) s->cur = 1 - s->cur;
        s->n += k;
        s->partials_valid = true;
      }
    }
    std::vector<int> still;
    for (int b : active) {
      gp_state s = h->batch[b];
      gp_report& rep = reports[b];
      state_gap_finish(s, h->bres_h + 4 * b, &rep);
      certified[b] = false;
      rep.iters = s->n;
      rep.tau = s->tau;
      rep.sigma = s->sigma;
      rep.seconds = t.s();
      bool stop = false, met = false, cert = false;
      if (!isfinite(rep.primal) || !isfinite(rep.dual)) {
        rep.status = GP_ERR_NONFINITE;
        stop = true;
      } else if (o.tol_rel_gap > 0 && (r = emd_stop_check(s, stops[b], o.tol_rel_gap, &rep, st, &cert, &met)) != GP_OK) {
        return r;
      } else if ((certified[b] = cert, met)) {
        rep.status = GP_OK;  // the corrected, feasible flux's gap met the tolerance
        stop = true;
      } else if (watch[b].update(rep.rel_gap)) {
        rep.status = GP_ERR_DIVERGED;
        stop = true;
      }
      if (!stop) still.push_back(b);
    }
    if (still.size() != active.size() && exec) {
      cudaGraphExecDestroy(exec);
      exec = nullptr;
      first = false;
    }
    active.swap(still);
  }
  if (exec) cudaGraphExecDestroy(exec);
  for (int b = 0; b < B; ++b) {  // every report carries the certificate of the returned iterate
    gp_state s = h->batch[b];
    if (!certified[b] && reports[b].status != GP_ERR_NONFINITE && isfinite(reports[b].dual) &&
        (r = emd_stop_final(s, stops[b], o.tol_rel_gap > 0, &reports[b], st)) != GP_OK)
      return r;
  }
  gp_status worst = GP_OK;
  for (int b = 0; b < B; ++b) {
    gp_state s = h->batch[b];
    const size_t NN = (size_t)N[b] * N[b];
    GP_CUDA(h, cudaMemcpyAsync(m[b], s->m, 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (p_out) GP_CUDA(h, cudaMemcpyAsync(p_out[b], s->p[s->cur], 2 * NN * sizeof(float), cudaMemcpyDeviceToDevice, st));
    if (reports[b].status != GP_OK && worst == GP_OK) worst = (gp_status)reports[b].status;
  }
  GP_CUDA(h, cudaStreamSynchronize(st));
  for (int b = 0; b < B; ++b) reports[b].seconds = t.s();
  return worst;
}

// ------------------------------------------------------------ autotuner
namespace {

void tune_load(gp_handle h, const char* path) {
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[512];
  while (fgets(line, sizeof(line), f)) {
    char key[256];
    int rb = 0;
    if (sscanf(line, " \"%255[^\"]\" : %d", key, &rb) == 2 && rb > 0) h->tune[key] = rb;
  }
  fclose(f);
}

bool tune_save(gp_handle h, const char* path) {
  if (!path) return true;
  FILE* f = fopen(path, "w");
  if (!f) return false;
  fprintf(f, "{\n");
  size_t i = 0;
  for (auto& kv : h->tune) fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++i < h->tune.size() ? "," : "");
  fprintf(f, "}\n");
  fclose(f);
  return true;
}

}  // namespace

gp_status gp_autotune(gp_handle h, int N, const char* cache_path, void* stream) {
  if (!h) return GP_ERR_ARG;
  h->err.clear();
  if (N < 4 || N > 8192 || N % 4 != 0) return fail(h, GP_ERR_ARG, "autotune needs N % 4 == 0 in [4, 8192]");
  DeviceGuard g(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  tune_load(h, cache_path);
  const char* names[2] = {"rof_fused", "emd_fused"};
  const int kinds[2] = {KIND_ROF, KIND_EMD};
  const int cands[4] = {4, 8, 16, 32};
  const bool prof = h->prof.on;
  h->prof.on = false;
  for (int q = 0; q < 2; ++q) {
    const std::string key = tune_key(h, names[q], N);
    if (h->tune.count(key)) continue;
    gp_state s = nullptr;
    gp_status r = alloc_state(h, kinds[q], N, &s);
    if (r != GP_OK) return r;
    const size_t NN = (size_t)N * N;
    float* in = nullptr;
    cudaError_t e = cudaMalloc(&in, 2 * NN * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(in, 0, 2 * NN * sizeof(float), st);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    int best = 16;
    float best_ms = 1e30f;
    for (int c = 0; c < 4 && e == cudaSuccess; ++c) {
      const int rb = cands[c];
      // the fused kernel on zeroed operands (its cost does not depend on the values)
      auto launch = [&]() {
        if (kinds[q] == KIND_ROF) {
          RofParams P{N, (float)N, (float)((double)N * N), 1.f, 1.f, 1.f};
          return launch_rof_fused(s->tmp, in, s->p[0], in, s->p[1], s->r, s->part, P, true, false, rb, st);
        }
        EmdParams P{N, (float)N, 1.f, 1.f};
        return launch_emd_fused(s->prim, s->s[0], s->p[0], in, s->s[1], s->p[1], s->r, s->m, s->e, s->part, P, true,
                                false, rb, st);
      };
      for (int w = 0; w < 2 && e == cudaSuccess; ++w) e = launch();
      if (e != cudaSuccess) break;
      cudaEventRecord(e0, st);
      for (int it = 0; it < 5 && e == cudaSuccess; ++it) e = launch();
      cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < best_ms) {
        best_ms = ms;
        best = rb;
      }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (in) cudaFree(in);
    free_state(s);
    if (e != cudaSuccess) {
      h->prof.on = prof;
      return cuda_fail(h, e, "autotune");
    }
    h->tune[key] = best;
  }
  h->prof.on = prof;
  // states built before the tuning pick the new shapes up at their next set-up
  for (auto& kv : h->cache) drop_graphs(kv.second);
  if (!tune_save(h, cache_path)) return fail(h, GP_ERR_ARG, "cannot write the autotune cache file");
  return GP_OK;
}

gp_status gp_rof_image_stats(gp_handle h, const float* I, int N, double* out, void* stream) {
  if (!h) return GP_ERR_ARG;
  h->err.clear();
  if (N < 1 || N > 8192) return fail(h, GP_ERR_ARG, "N out of range [1, 8192]");
  if (!out) return fail(h, GP_ERR_ARG, "out is NULL");
  gp_status r = check_ptr(h, I, "I");
  if (r != GP_OK) return r;
  DeviceGuard g(h->device);
  if (!g.ok) return fail(h, GP_ERR_CUDA, "cudaSetDevice failed");
  return rof_image_stats(h, I, N, out, (cudaStream_t)stream);
}

double gp_rof_step_tau(const double* stats, double lambda, double eps, int flags) {
  if (!stats || !(lambda > 0) || !(eps > 0)) return NAN;
  const double tv = stats[0], grad_l2 = stats[1], fid = 0.5 * lambda * stats[2];
  const double T = (flags & GP_RULE_FIDELITY_BOUND) ? fmin(tv, fid) : tv;
  double tau = sqrt(lambda) * T / sqrt(eps);
  if (flags & GP_RULE_GRID_CAP) tau = fmin(tau, grad_l2);
  return tau > 0 ? tau : 1.0;  // a constant image: any step
}

double gp_emd_delta_tau(int N, double eps, int m_points) {
  if (N < 1 || !(eps > 0) || !(eps < 1)) return NAN;
  const double M = m_points ? (double)N * N : (double)N;
  return fmin(sqrt(1.0 / (eps * fabs(log(eps)))), 2.0 * pow(M, 0.25));
}

int gp_gap_schedule_next(int n_prev, double g_prev, int n, double g, double tol) {
  return adaptive_chunk(n_prev, g_prev, n, g, tol);
}

int gp_tuned_row_block(gp_handle h, const char* kernel, int N) {
  if (!h || !kernel) return 0;
  auto it = h->tune.find(tune_key(h, kernel, N));
  return it == h->tune.end() ? 0 : it->second;
}

// ------------------------------------------------------------ profiling
gp_status gp_profile(gp_handle h, int enable) {
  if (!h) return GP_ERR_ARG;
  Profiler& P = h->prof;
  if (enable) {
    P.used = 0;
    P.recs.clear();
    for (int i = 0; i < PK_COUNT; ++i) {
      P.launches[i] = 0;
      P.ms[i] = 0;
    }
    P.resolved = true;
  }
  P.on = enable != 0;
  return GP_OK;
}

int gp_profile_kernels(void) { return PK_COUNT; }

gp_status gp_profile_query(gp_handle h, int kernel, const char** name, double* total_ms, long long* launches) {
  if (!h || kernel < 0 || kernel >= PK_COUNT) return GP_ERR_ARG;
  DeviceGuard g(h->device);
  Profiler& P = h->prof;
  if (!P.resolved) {
    for (auto& rc : P.recs) {
      cudaError_t e = cudaEventSynchronize(rc.b);
      if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventSynchronize");
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, rc.a, rc.b) == cudaSuccess) P.ms[rc.id] += ms;
    }
    P.recs.clear();
    P.resolved = true;
  }
  if (name) *name = kProfNames[kernel];
  if (total_ms) *total_ms = P.ms[kernel];
  if (launches) *launches = P.launches[kernel];
  return GP_OK;
}

}  // extern "C"
