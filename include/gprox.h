/*
 * gprox.h -- C ABI of the GB300 (sm_103a) G-prox PDHG library.
 *
 * The library solves, on one GPU, the two problems of Jacobs, Leger, Li and
 * Osher, "Solving large-scale optimization problems with a convergence rate
 * independent of grid size" (arXiv 1805.09453), with their preconditioned
 * primal-dual method (Algorithm 2, "G-prox PDHG", section 3):
 *   - ROF total-variation denoising, section 3.1 (updates of u, p, pbar);
 *   - the L1 earth mover's / Beckmann problem, section 3.2 (Hodge split
 *     m = u + grad psi, Leray-projected u update, projected p update).
 *
 * Discretisation (the paper does not print one; every choice below is the
 * reading the library and its tests use):
 *   - N x N cell-centred grid on [0,1]^2, h = 1/N, row-major float32 planes,
 *     row index i = y (slow), column index j = x (fast);
 *   - grad = forward differences with a zero last slot (zero Neumann flux),
 *     div = -grad^T (backward differences), Laplacian = div grad (5-point
 *     Neumann).  Then K^T K = -Laplacian exactly and the cosine basis of the
 *     even reflection (Appendix A) diagonalises the u-step;
 *   - vector fields are two consecutive planes (x component, then y): the
 *     slots [i][N-1] of the x plane and [N-1][j] of the y plane are
 *     structurally zero; inputs there are ignored, outputs there are 0;
 *   - inner products, objectives and gaps are h^2-weighted (L2 on [0,1]^2).
 *
 * Conventions for every entry point:
 *   - array arguments are DEVICE pointers (cudaMalloc / torch CUDA memory) of
 *     float32, owned by the caller; the library never frees them.  Host
 *     pointers are rejected with GP_ERR_ARG.  Pointers must be 4-byte
 *     aligned; 16-byte alignment together with N % 4 == 0 selects the
 *     vectorised kernels, anything else the scalar ones (same results);
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  All work is ordered on that stream; solver calls synchronise
 *     it only at duality-gap checks and on return;
 *   - a handle owns its workspace, DCT tables and scratch; one handle must
 *     not be used by two host threads or two streams at the same time;
 *   - functions return a gp_status and never abort or throw.  On an error
 *     other than GP_ERR_MAXITER the output arrays are unspecified;
 *     gp_last_error(handle) returns a description of the last failure.
 */
#ifndef GPROX_H
#define GPROX_H

#ifdef __cplusplus
extern "C" {
#endif

#define GP_ABI_VERSION 2

#if defined(__GNUC__)
#define GP_API __attribute__((visibility("default")))
#else
#define GP_API
#endif

typedef enum gp_status {
  GP_OK = 0,
  GP_ERR_ARG = 1,         /* bad size, pointer, option or state */
  GP_ERR_CUDA = 2,        /* a CUDA runtime call failed */
  GP_ERR_MAXITER = 3,     /* tolerance not reached within max_iters (outputs hold the last iterate) */
  GP_ERR_NONFINITE = 4,   /* NaN / Inf met in an objective or gap reduction */
  GP_ERR_DIVERGED = 5,    /* relative gap grew 10x over 5 consecutive checks */
  GP_ERR_MASS = 6,        /* EMD densities differ in total mass by more than 1e-3 relative */
  GP_ERR_UNSUPPORTED = 7  /* option not available for these arguments (e.g. a precision mode at this N) */
} gp_status;

/* Arithmetic of the cosine-transform (Helmholtz / Poisson) solve. */
/* The split modes need N a multiple of 128 (GP_ERR_UNSUPPORTED otherwise).
 * Each operand x is stored as x_hi + x_lo in two 16-bit formats and a product
 * A B^T ~ A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T is accumulated in FP32:
 * BF16 parts carry 16 significant bits; FP16 parts carry 22, each operand
 * first multiplied by a power of two taken from its largest magnitude so
 * that it fits FP16's range (exact: the product is divided back).  The
 * REFINED modes add one step of residual correction to every solve:
 * r = b - (alpha - Lap) x / scale evaluated in FP64 from the stored x, then
 * x += solve(r) (two solves per call; an FP32-level result from the BF16
 * split). */
typedef enum gp_prec {
  GP_PREC_FP32 = 0,                /* FP32 fast cosine transform (power-of-two N) or FP32 dense transform */
  GP_PREC_SPLIT_BF16 = 1,          /* dense transform on tensor cores, hi+lo bf16 split, FP32 accumulate */
  GP_PREC_SPLIT_FP16 = 2,          /* dense transform on tensor cores, scaled hi+lo fp16 split, FP32 accumulate */
  GP_PREC_SPLIT_BF16_REFINED = 3,  /* GP_PREC_SPLIT_BF16 plus one residual-correction solve */
  GP_PREC_SPLIT_FP16_REFINED = 4   /* GP_PREC_SPLIT_FP16 plus one residual-correction solve */
} gp_prec;

typedef struct gp_opts {
  int max_iters;       /* iteration cap (>= 0; default 1000) */
  int gap_every;       /* duality-gap check every k iterations (>= 1; default 10); 0: adaptive
                          (rof_solve / emd_solve with tol_rel_gap > 0): while the gap is above
                          3 x tol_rel_gap, its decay over the last two checks, fitted as
                          g ~ n^-a, places the next check halfway to the predicted crossing, in
                          chunks of 10 * 2^j <= 320 iterations; within 3 x, every 10 (see
                          gp_gap_schedule_next); batched solves take 10 */
  double tol_rel_gap;  /* stop once (P - D) / max(|P|,|D|) <= tol; <= 0: run exactly max_iters */
  double tau;          /* primal step; <= 0 selects the paper's rule (ROF section 4.1, EMD tau = 1) */
  double sigma;        /* dual step; <= 0 selects 1 / tau */
  double tau_scale;    /* multiplier on the rule's tau (<= 0 means 1) */
  double eps;          /* ROF rule tolerance epsilon (default 1e-3) */
  int prec;            /* gp_prec of the cosine-transform solve */
  int use_graph;       /* replay the k iterations between gap checks as a CUDA graph */
  int warm_start;      /* 0: zero initial state; 1: take the caller's u / p (ROF) or p (EMD) arrays as the start */
} gp_opts;

typedef struct gp_report {
  int iters;             /* iterations run */
  int status;            /* gp_status of the solve */
  double primal;         /* P at the last check: ROF energy or EMD cost sum |m| h^2 */
  double dual;           /* D at the last check (a lower bound on the optimum).  EMD: for a p,
                            D = h^2 sum phi (f1 - f0) / max(1, max |D phi|), phi = Lap^{-1} div p
                            held as two FP32 planes (an FP32 solve plus a solve of its residual,
                            taken from p itself), the sum and max |D phi| (forward differences)
                            in double-FP32 pair arithmetic, the max raised by 2^-40 to bound its
                            rounding: a valid bound for the phi the planes hold */
  double rel_gap;        /* (P - D) / max(|P|, |D|) */
  double mass_residual;  /* EMD: h^2 sum |div m - (f0 - f1)| / h^2 sum |f0 - f1| (FP32 terms at a
                            plain check, FP64 at a certified one, see below); ROF: 0 */
  double tau, sigma;     /* step sizes used */
  double seconds;        /* host wall time of the call */
  /* Feasibility certificate (section 3.2: P(m) bounds the optimum from above
   * only for an m with div m = f0 - f1 exactly; D bounds it from below for
   * any p).  EMD: at the final check, and at the checks the stop test picks
   * (below), the residual rho = (f0 - f1) - div m of the returned FP32 m
   * is evaluated in FP64 (mass_residual then reports it), c = Lap^{-1} rho is
   * solved, and m~ = m + grad c is the corrected, feasible flux:
   *   primal_feasible        = h^2 sum |m~|  (>= the optimum)
   *   rel_gap_feasible       = (primal_feasible - D) / max(|primal_feasible|, |D|)
   *   mass_residual_feasible = h^2 sum |div m~ - (f0 - f1)| / h^2 sum |f0 - f1|
   * and a solve with tol_rel_gap > 0 returns GP_OK only once
   * rel_gap_feasible <= tol_rel_gap (so the optimum lies within that of
   * primal_feasible).  In that mode (EMD, tol_rel_gap > 0) `dual` is the best
   * lower bound met during the solve: the dual value of the iterate's p at
   * every check and of averages of those p's (a convex combination of
   * feasible p's is feasible; the averaging window opens once the gap is
   * within 30 x tol_rel_gap and restarts whenever the iteration count has
   * doubled since it opened), and rel_gap / rel_gap_feasible use it; the
   * last iterate's own dual value lags the optimum far more than its primal
   * does.  The flux is certified at every window restart and whenever the
   * stored primal, less the offset primal - primal_feasible of the last
   * certificate, is within 2 x tol_rel_gap of that bound (at most every 100
   * iterations unless within tol_rel_gap).  ROF (unconstrained): primal,
   * rel_gap and 0. */
  double primal_feasible;
  double rel_gap_feasible;
  double mass_residual_feasible;
} gp_report;

typedef struct gp_handle_s* gp_handle;
typedef struct gp_state_s* gp_state;

/* Library ABI version (GP_ABI_VERSION of the build). */
GP_API int gp_abi_version(void);

/* Fill `opts` with the defaults listed in gp_opts. */
GP_API void gp_default_opts(gp_opts* opts);

/* Create a handle bound to CUDA device `device`.  Allocates no device memory
 * yet (workspace grows on first use).  Returns GP_ERR_ARG for a NULL `out`
 * or a device index out of range. */
GP_API gp_status gp_create(gp_handle* out, int device);

/* Release a handle and all memory it owns (synchronises the device). NULL is a no-op. */
GP_API gp_status gp_destroy(gp_handle h);

/* Text of the last error on this handle ("" if none).  Valid until the next call on `h`.
 * gp_last_error(NULL) describes the last failed handle-free call
 * (dct2_poisson_static) of the calling thread. */
GP_API const char* gp_last_error(gp_handle h);

/*
 * dct2_poisson: solve (alpha - Laplacian) x = b on the N x N grid with zero
 * Neumann conditions -- the linear solve inside the G-prox u-step
 * (section 3.1: (lambda tau Id - Laplacian)^{-1}; section 3.2: the
 * Laplacian^{-1} of the Leray projection and of the Hodge split), done in the
 * cosine basis that the even reflection of Appendix A gives:
 *     x = C^T [ (C b C^T) / (alpha + mu_k + mu_l) ] C,
 *     mu_k = (4/h^2) sin^2(pi k / 2N),  C = orthonormal DCT-II.
 *   b      device, N*N float32, read only.
 *   x      device, N*N float32, written (may equal b).
 *   N      1 <= N <= 8192.
 *   alpha  >= 0.  alpha == 0: the constant mode of b is dropped and x has zero mean.
 *   prec   gp_prec.  GP_PREC_FP32 uses the fast transform when N is a power of
 *          two in [16, 8192], else the dense one.
 * Errors: GP_ERR_ARG (N, alpha, pointers), GP_ERR_UNSUPPORTED (prec), GP_ERR_CUDA.
 */
GP_API gp_status dct2_poisson(gp_handle h, const float* b, float* x, int N, double alpha,
                       int prec, void* stream);

/*
 * dct2_poisson_grad: g = grad x for x = (alpha - Laplacian)^{-1} b, the
 * forward-difference gradient of the discretisation (x plane then y plane;
 * zero slots).  Sections 3.1 / 3.2 use it for the Hodge split m0 = grad psi
 * and the Leray step (grad Lap^{-1} div).  For power-of-two N in [16, 8192]
 * the gradient is synthesised from the cosine spectrum of x, so it keeps FP32
 * relative precision at any N (differencing an FP32 x loses ~log2(N) bits);
 * other N difference the dense solve's output.
 *   b      device, N*N, read only.  g: device, 2*N*N, written.
 *   alpha  >= 0 (alpha == 0: constant mode dropped).
 * Errors as dct2_poisson.
 */
GP_API gp_status dct2_poisson_grad(gp_handle h, const float* b, float* g, int N, double alpha, int prec,
                                   void* stream);

/*
 * rof_solve: minimise the ROF energy ||u||_TV + lambda/2 ||u - I||^2
 * (section 3.1) with G-prox PDHG:
 *     u_{n+1} = (lambda tau - Lap)^{-1} (lambda tau I + tau div pbar_n - Lap u_n)
 *     p_{n+1} = (p_n + sigma grad u_{n+1}) / max(1, |p_n + sigma grad u_{n+1}|)
 *     pbar_{n+1} = 2 p_{n+1} - p_n
 * Step rule when opts->tau <= 0 (section 4.1 with the section-3.1 bound on
 * ||u*||_TV): tau = min(sqrt(lambda) T / sqrt(eps), ||grad I||_L2),
 * T = min(||I||_TV, lambda/2 ||I - mean I||^2), sigma = 1/tau.
 *   I       device, N*N, the image (read only).
 *   u       device, N*N, out: the last primal iterate (in: start if warm_start).
 *   p       device, 2*N*N (x plane, y plane), out: the last dual iterate
 *           (in: start if warm_start); may be NULL when warm_start == 0.
 *   lambda  > 0 fidelity weight.
 *   opts    NULL = defaults.  report: may be NULL.
 * Returns GP_OK when the tolerance was met (or max_iters ran with tol <= 0),
 * GP_ERR_MAXITER if not, GP_ERR_NONFINITE / GP_ERR_DIVERGED on breakdown.
 */
GP_API gp_status rof_solve(gp_handle h, const float* I, float* u, float* p, int N, double lambda,
                    const gp_opts* opts, gp_report* report, void* stream);

/*
 * rof_solve_cp2: the comparison method of section 4.1 (Tables 4-5), the
 * accelerated primal-dual hybrid gradient iteration ("CP2") for the same ROF
 * problem as rof_solve.  It takes no linear solve: per iteration
 *   p_{n+1} = proj(p_n + sigma_n grad ubar_n),
 *   u_{n+1} = (u_n + tau_n div p_{n+1} + tau_n lambda I) / (1 + tau_n lambda),
 *   ubar_{n+1} = u_{n+1} + theta_n (u_{n+1} - u_n),
 *   theta_n = 1/sqrt(1 + 2 lambda tau_n), tau_{n+1} = theta_n tau_n, sigma_{n+1} = sigma_n / theta_n,
 * exploiting the lambda-strong convexity of the fidelity term; it needs many
 * more iterations than G-prox PDHG, increasingly so as the grid refines.
 *   I, u, p  as rof_solve (u out; p may be NULL; warm_start: u and p in/out).
 *   opts     max_iters, tol_rel_gap, gap_every (0: 10), warm_start as
 *            rof_solve; tau / sigma > 0 set tau_0 / sigma_0, else both are
 *            1/sqrt(||Lap||) (section 4.1), tau_0 times / sigma_0 divided by
 *            tau_scale when that is > 0.  prec and use_graph are ignored.
 * The report's tau / sigma are the last step sizes; the gap is the ROF gap
 * of rof_solve.  N in [2, 8192].  Uses (and resets) the handle's cached ROF
 * buffers of size N.
 */
GP_API gp_status rof_solve_cp2(gp_handle h, const float* I, float* u, float* p, int N, double lambda,
                               const gp_opts* opts, gp_report* report, void* stream);

/*
 * emd_solve: L1 earth mover's distance min sum_x |m(x)| h^2 s.t. div m = f0 - f1
 * (section 3.2, isotropic 2-norm) with G-prox PDHG on m = u + grad psi:
 *     Lap psi = f0 - f1,  m_0 = grad psi
 *     m_{n+1} = m_n - tau (pbar_n - grad Lap^{-1} div pbar_n)     (Leray projection)
 *     p_{n+1} = proj(p_n + sigma m_{n+1}),  pbar_{n+1} = 2 p_{n+1} - p_n
 * Default steps tau = sigma = 1 (section 4.2, bounded densities).  The dual
 * bound is D = (phi, f1 - f0) / max(1, max |grad phi|) with phi = Lap^{-1} div p.
 *   f0, f1  device, N*N densities with equal total mass (|diff| <= 1e-3 relative
 *           else GP_ERR_MASS); a tiny mass mismatch is dropped with the constant mode.
 *   m       device, 2*N*N, out: the last flux iterate m_n.
 *   p       device, 2*N*N or NULL: out: last dual iterate; in: start if warm_start.
 *   phi     device, N*N or NULL: out: the dual potential Lap^{-1} div p_n of the last check.
 * Returns as rof_solve.
 */
GP_API gp_status emd_solve(gp_handle h, const float* f0, const float* f1, float* m, float* p, float* phi,
                    int N, const gp_opts* opts, gp_report* report, void* stream);

/*
 * rof_solve3d / emd_solve3d: the d = 3 instance of rof_solve / emd_solve
 * (Algorithm 2 is stated for general dimension d; sections 3.1 / 3.2 carry d
 * through their constants).  Volumes are N x N x N arrays indexed (z, y, x),
 * x fastest, h = 1/N, weights h^3; vector fields are three consecutive
 * volumes (x, y, z components), each with a zero last slot along its own
 * axis; grad = forward differences, div = -grad^T, the Laplacian the 7-point
 * Neumann stencil, solved in the cosine basis (gain 1/(alpha + mu_x + mu_y +
 * mu_z)) with one line transform per axis.  The iterations, step rules, gaps
 * and stopping tests are those of the two-dimensional entry points.
 *   N       power of two in [16, 512].
 *   I, f0, f1   device, N^3, read only.
 *   u       device, N^3, out (rof_solve3d).  m: device, 3 N^3, out.
 *   p       device, 3 N^3 or NULL, out: the last dual iterate.
 *   opts    max_iters, tol_rel_gap, gap_every (0: adaptive as rof_solve),
 *           tau, sigma, tau_scale, eps as the 2-D calls; prec must be
 *           GP_PREC_FP32; warm_start, use_graph are not supported (warm_start
 *           != 0 returns GP_ERR_UNSUPPORTED).
 * EMD reports the FP32 gap (primal, dual, rel_gap, mass_residual); its
 * feasibility fields are NaN and the stopping test uses rel_gap.  Buffers of
 * 14 (ROF) / 25 (EMD) N^3 floats are allocated on first use and kept by
 * the handle.  Returns as rof_solve.
 */
GP_API gp_status rof_solve3d(gp_handle h, const float* I, float* u, float* p, int N, double lambda,
                             const gp_opts* opts, gp_report* report, void* stream);
GP_API gp_status emd_solve3d(gp_handle h, const float* f0, const float* f1, float* m, float* p, int N,
                             const gp_opts* opts, gp_report* report, void* stream);

/*
 * emd_solve_batched: B independent EMD problems (section 3.2) of possibly
 * different sizes N[b], solved together.  Every chunk of gap_every
 * iterations of all unconverged problems runs as one CUDA graph with one
 * branch per problem (so small problems execute concurrently), the gap
 * checks included; a problem stops at its own tolerance.  Arrays are host
 * arrays of B device pointers; reports[B] receives one report per problem.
 *   B       1..256.  stream must be a non-default stream (graph capture).
 *   m[b]    out, 2*N[b]*N[b] floats: the last primal iterate of problem b.
 *   p       NULL, or B device pointers (each 2*N[b]*N[b] floats, out): the
 *           last dual iterate of each problem.
 *   opts    as emd_solve (warm_start unsupported).
 * Returns GP_OK if every problem met the tolerance, else the first non-OK
 * per-problem status (each report's `status` holds its own).
 */
GP_API gp_status emd_solve_batched(gp_handle h, int B, const float* const* f0, const float* const* f1,
                                   float* const* m, float* const* p, const int* N, const gp_opts* opts,
                                   gp_report* reports, void* stream);

/*
 * Explicit solver states for step-by-step driving (checkpoint / resume, tests,
 * external schedulers).  A state owns its device buffers and keeps pointers
 * to the caller's inputs (I, or f0 / f1), which must outlive it.
 *
 * gp_state_create_rof / _emd: u0 (or m0), p0, pbar0 may be NULL: defaults are
 * u0 = 0, m0 = grad psi, p0 = 0, pbar0 = p0.  tau > 0, sigma > 0 required.
 * EMD iterates stay on the affine set {div m = f0 - f1} (m = u + grad psi with
 * u divergence-free, section 3.2): the first step projects a caller's m0 onto
 * it, m0 + grad Lap^{-1}(f0 - f1 - div m0), which changes a feasible m0 by
 * nothing.  Each EMD step solves Lap q = (f0 - f1) - div(m_n - tau pbar_n) and
 * sets m_{n+1} = m_n - tau pbar_n + grad q: on the affine set this equals the
 * section-3.2 update m_n - tau (pbar_n - grad Lap^{-1} div pbar_n), and in
 * floating point it keeps solve errors from accumulating in div m.
 * pd_step runs n_steps >= 0 G-prox iterations (section 3, Algorithm 2) with
 * the cosine solve in precision `prec`; in FP32 at power-of-two N every step
 * of a call but the last hands its right-hand side to the next as row
 * spectra (the stencil runs in the next solve's forward row pass), and the
 * last step writes it and the gap terms, so calls of any length compose.
 * gp_state_read copies the current
 * primal (u: N*N, or m: 2*N*N) and p (2*N*N) into caller device buffers
 * (either may be NULL).  gp_state_gap evaluates P, D, gap (and the EMD mass
 * residual) of the current iterate and synchronises `stream`;
 * gp_state_certify does the same and, for EMD, adds the feasibility
 * certificate described under gp_report (one more cosine solve and two FP64
 * reductions; ROF: the certificate fields equal P, the gap and 0).
 */
GP_API gp_status gp_state_create_rof(gp_handle h, gp_state* out, const float* I, int N, double lambda,
                              double tau, double sigma, const float* u0, const float* p0,
                              const float* pbar0, void* stream);
GP_API gp_status gp_state_create_emd(gp_handle h, gp_state* out, const float* f0, const float* f1, int N,
                              double tau, double sigma, const float* m0, const float* p0,
                              const float* pbar0, void* stream);
GP_API gp_status pd_step(gp_handle h, gp_state s, int n_steps, int prec, void* stream);
GP_API gp_status gp_state_read(gp_handle h, gp_state s, float* primal, float* p, void* stream);
GP_API gp_status gp_state_gap(gp_handle h, gp_state s, gp_report* report, void* stream);
GP_API gp_status gp_state_certify(gp_handle h, gp_state s, gp_report* report, void* stream);
GP_API gp_status gp_state_destroy(gp_state s);

/*
 * Ergodic averages (the iterate averages u^n = (1/n) sum_{k=1..n} u_k,
 * p^n = (1/n) sum p_k in which the convergence theorems of sections 3.1 / 3.2
 * are stated).  gp_state_average(h, s, 1, stream) starts (or restarts) the
 * averages of state s: it allocates 3 (ROF) or 5 (EMD) FP64 planes of running
 * sums, zeroes them, and every later pd_step adds its iterate; while it is on,
 * the steps write their right-hand sides (no fused forward row pass).
 * gp_state_average(h, s, 0, stream) stops and frees the sums.
 * gp_state_read_average writes the averages of the steps taken since the
 * start into caller device buffers (either may be NULL): primal (u: N*N, or
 * m: 2*N*N) and p (2*N*N); *count (may be NULL) receives n.  The primal
 * average is taken through the solve's linearity: ROF u^n = (lambda tau -
 * Lap)^{-1} (mean of the right-hand sides), EMD m^n = mean(s) + grad Lap^{-1}
 * (mean(d)), one solve per read.  Errors: GP_ERR_ARG (no averaged step, bad
 * pointers).  Not in the paper's experiments (they report the last iterate).
 */
GP_API gp_status gp_state_average(gp_handle h, gp_state s, int enable, void* stream);
GP_API gp_status gp_state_read_average(gp_handle h, gp_state s, float* primal, float* p, long long* count,
                                       void* stream);

/*
 * dct2_poisson_static: dct2_poisson without any device allocation.  The paper
 * has no counterpart; this entry point serves callers that may not call
 * cudaMalloc -- a host framework that owns all device memory through its own
 * pool and budget, or a real-time loop in which an allocation (and the device
 * synchronisation it can cause) is not allowed.  The caller passes only b and
 * x; the scratch (one N x N plane) and the transform tables live in
 * file-scope static device arrays of a fixed size, which every GPU that loads
 * the library holds until the process exits (4 MiB + ~16 KiB).
 *   b, x    device pointers of the current device, N*N float32, 16-byte
 *           aligned; x may equal b.  Same result as dct2_poisson(GP_PREC_FP32).
 *   N       power of two in [16, 1024]; anything else returns GP_ERR_ARG
 *           (text in gp_last_error(NULL)).
 *   alpha   >= 0, as in dct2_poisson.
 *   stream  cudaStream_t as void*.
 * All calls share the static arrays: calls that overlap on the GPU (other
 * streams, other host threads) race and give wrong results.  Nothing in the
 * arrays needs to start at zero (each pass writes what the next one reads;
 * the tables are rewritten when N changes).  A call made while `stream` is
 * capturing records the table kernel with the solve, and from then on every
 * call on that device rewrites the tables as well.  The first call on a
 * device looks up the arrays' device addresses with that device current and
 * caches them; make that first call before any stream capture.
 */
GP_API gp_status dct2_poisson_static(const float* b, float* x, int N, double alpha, void* stream);

/*
 * gp_autotune: pick the tile shape of the fused stencil kernels (the height of
 * the row block each thread walks: 4, 8, 16 or 32 rows) for grids of size N
 * on this handle's device by timing each on scratch buffers; solves on this
 * handle use the fastest from then on.  Keyed by (kernel, N, SM version).
 * cache_path (may be NULL): a JSON file of {"kernel/N=../sm=..": rows} read
 * before tuning (keys found there are not re-timed) and rewritten after.
 * N % 4 == 0 required.  Allocates scratch for the duration of the call.
 * gp_tuned_row_block returns the chosen height for kernel "rof_fused" or
 * "emd_fused" (0 if not tuned).  The paper has no counterpart.
 */
GP_API gp_status gp_autotune(gp_handle h, int N, const char* cache_path, void* stream);
GP_API int gp_tuned_row_block(gp_handle h, const char* kernel, int N);

/*
 * gp_rof_image_stats: the image norms the ROF step rules take (section 4.1;
 * the rof_solve rule, and the rules of the paper's disc experiments), as FP64
 * reductions on the GPU: out[0] = ||I||_TV = h^2 sum |grad I| (isotropic,
 * forward differences), out[1] = ||grad I||_L2 = (h^2 sum |grad I|^2)^(1/2),
 * out[2] = ||I - mean(I)||^2_L2 = h^2 sum (I - mean)^2, h = 1/N.  I: device
 * pointer, N x N row-major FP32, read only; out: host array of 3 doubles.
 * Synchronises the stream.  Errors: GP_ERR_ARG (bad pointer or N),
 * GP_ERR_CUDA.
 */
GP_API gp_status gp_rof_image_stats(gp_handle h, const float* I, int N, double* out, void* stream);

/*
 * gp_gap_schedule_next: the adaptive gap-check schedule of gap_every == 0 as
 * a pure function, for callers driving pd_step / gp_state_gap themselves.
 * Given the previous check (iteration n_prev, relative gap g_prev; n_prev <= 0
 * if none) and the current one (n, g), returns the number of iterations to
 * run before the next check: 10 * 2^j <= 320, halfway to the iteration where
 * the fit g ~ c n^-a through the two checks reaches tol; 10 when there is no
 * decrease to fit, no previous check, or g <= 3 tol (the gap is not
 * monotone: near the target it dips below tol at isolated checks that sparse
 * checks would step over).  Host only, no GPU work.
 * The paper has no counterpart (it reports gaps per iteration).
 */
GP_API int gp_gap_schedule_next(int n_prev, double g_prev, int n, double g, double tol);

/*
 * Step rules of the paper's experiments, host only (no GPU work).
 * gp_rof_step_tau: section 4.1's ROF rule from the image norms of
 * gp_rof_image_stats (stats[0] = ||I||_TV, stats[1] = ||grad I||_L2,
 * stats[2] = ||I - mean I||^2_L2):
 *   tau = sqrt(lambda) T / sqrt(eps),  T = ||I||_TV, or, with
 *   GP_RULE_FIDELITY_BOUND, T = min(||I||_TV, lambda/2 ||I - mean I||^2)
 *   (section 3.1's a-priori bound on ||u*||_TV); with GP_RULE_GRID_CAP the
 *   result is capped by ||grad I||_L2 (the grid-dependent rule).  1 for a
 *   constant image; NaN for bad arguments.  rof_solve uses both flags.
 * gp_emd_delta_tau: section 4.2's rule for delta measures,
 *   tau = min(sqrt(1 / (eps |log eps|)), 2 M^(1/4)),
 *   M = N^2 grid points (m_points != 0) or N (the other reading, see the
 *   design notes).  NaN unless N >= 1 and 0 < eps < 1.
 */
#define GP_RULE_GRID_CAP 1
#define GP_RULE_FIDELITY_BOUND 2
GP_API double gp_rof_step_tau(const double* stats, double lambda, double eps, int flags);
GP_API double gp_emd_delta_tau(int N, double eps, int m_points);

/*
 * Launch profiler (tracing).  gp_profile(h, 1) clears the counters and starts
 * recording: every kernel the handle launches is bracketed by CUDA events on
 * its stream (CUDA-graph replay is disabled while recording); gp_profile(h, 0)
 * stops.  gp_profile_query returns, for kernel class `kernel` in
 * [0, gp_profile_kernels()), its name (static string), the summed device time
 * in ms and the number of kernel launches recorded (it waits for the recorded
 * events).  Classes: dct_rows_fwd, dct_cols_solve, dct_rows_inv (the three
 * passes of the fast cosine solve), dct_cols_grad, dct_rows_grad (the
 * gradient form's column and row passes), dct_dense, dct_tc_split,
 * rof_fused, emd_fused (the stencil steps that write the right-hand side),
 * reduce, setup, rof_step_fwd, emd_step_fwd (stencil steps fused with the
 * next forward row pass).  The paper has no counterpart (it reports
 * wall-clock totals only).
 */
GP_API gp_status gp_profile(gp_handle h, int enable);
GP_API int gp_profile_kernels(void);
GP_API gp_status gp_profile_query(gp_handle h, int kernel, const char** name, double* total_ms,
                                  long long* launches);

/*
 * emd_coarse_start: a start for the EMD solve from a coarser grid.  The
 * densities are restricted to (N/factor)^2 by block means (same total mass),
 * the coarse problem is solved with emd_solve(opts), and its dual potential
 * phi_c = Lap^{-1} div p (section 4.2: the dual variable is the gradient of
 * a potential with |grad phi| <= 1) is interpolated to N x N, bilinearly
 * between cell centres (fine centre j at coarse coordinate (j + 1/2)/factor
 * - 1/2, clamped to [0, N/factor - 1]).
 *   f0, f1  device, N*N; phi device N*N out.
 *   factor  >= 2 with N % factor == 0 and N / factor >= 2.
 *   opts    the coarse solve's options (warm_start must be 0); report (may
 *           be NULL) receives the coarse solve's report.
 * Returns the coarse solve's status (GP_ERR_MAXITER still writes phi).
 * Allocates 5 (N/factor)^2 floats of scratch for the call; synchronises the
 * stream.  The paper has no counterpart (it starts from zero).
 */
GP_API gp_status emd_coarse_start(gp_handle h, const float* f0, const float* f1, int N, int factor,
                                  const gp_opts* opts, float* phi, gp_report* report, void* stream);

/*
 * rof_coarse_start: a start for the ROF solve from a coarser grid.  I is
 * restricted to (N/factor)^2 by block means, the coarse problem (the same
 * continuum energy of section 3.1: the same lambda, h_c = factor / N) is
 * solved with rof_solve(opts), and u_c and both planes of p_c are
 * interpolated bilinearly between cell centres as emd_coarse_start does;
 * the interpolated p is then made feasible (zero structural slots, |p| <= 1).
 *   I       device, N*N.  u: device N*N out.  p: device 2*N*N out.
 *   factor  >= 2 with N % factor == 0 and N / factor >= 2.  lambda > 0.
 *   opts    the coarse solve's options (warm_start must be 0); report (may
 *           be NULL) receives the coarse solve's report.
 * Returns the coarse solve's status (GP_ERR_MAXITER still writes u and p).
 * Allocates 4 (N/factor)^2 floats of scratch for the call; synchronises the
 * stream.  The paper has no counterpart (it starts from zero).
 */
GP_API gp_status rof_coarse_start(gp_handle h, const float* I, int N, int factor, double lambda,
                                  const gp_opts* opts, float* u, float* p, gp_report* report, void* stream);

/*
 * Learned warm start for the EMD solve (section 4.2's dual potential).  A
 * 4-level encoder-decoder CNN maps (f0, f1, prior) to a potential phi_0; the
 * start is p_0 = proj(grad phi_0) (forward differences, unit-disc
 * projection), and the method's own duality gap decides between it and the
 * other starts.  The paper has no learned component: this is an addition on
 * top of its method.
 *
 * Network, base width C: 3x3 convolutions with zero padding, ReLU after all
 * but the last, 2x2 average pooling, nearest 2x upsampling, concatenated
 * skips [upsampled, skip]:
 *   3 -> C -> C | C -> 2C -> 2C | 2C -> 4C -> 4C | 4C -> 8C -> 8C |
 *   12C -> 4C -> 4C | 6C -> 2C -> 2C | 3C -> C -> C | C -> 1.
 * Inputs per cell: (f0 - f1)/16, (f0 + f1)/16 and a prior potential (e.g.
 * emd_coarse_start's; zero when the prior array or its entry is NULL).
 * Output: phi = prior + head output, mean removed (a correction of the prior;
 * gp_cnn_create zeroes the head, so a new network returns the prior).
 * Parameters (FP32, gp_cnn_num_params floats): conv by conv in that order,
 * weights W[cout][cin][3][3] (tap (dy, dx) at index 3 (dy + 1) + dx + 1,
 * correlation: y(p) = sum W x(p + (dy, dx))) followed by biases b[cout].
 * bf16 != 0: weights and activations are stored as BF16 (FP32 accumulation;
 * gradients, master weights and Adam moments FP32); bf16 == 0: all FP32.
 *
 * Loss for targets t (per sample, averaged over the batch), e = phi - t with
 * both mean-free, D the forward difference without the 1/h factor and with
 * zero last slots:  |e|^2 / |t|^2 + |D e|^2 / |D t|^2.
 *
 * All device arrays are float32 N x N row-major on the handle's device; f0,
 * f1, prior and phi_target are HOST arrays of B device pointers (prior may be
 * NULL); N must be a multiple of 8 in [8, 8192].  The network owns its
 * parameters and its activation buffers (grown on demand).  Errors:
 * GP_ERR_ARG for bad arguments, GP_ERR_CUDA for CUDA failures; text in
 * gp_cnn_last_error.
 *   gp_cnn_create      He-uniform weights from `seed`, zero biases, zero head.
 *   gp_cnn_get_params / gp_cnn_set_params   host float32 copies; set resets
 *                      the Adam moments and step count.
 *   gp_cnn_forward     phi: device, B*N*N.
 *   gp_cnn_loss_grad   forward + loss + backward; *loss (may be NULL) is the
 *                      loss, grad (host, num_params, may be NULL) receives
 *                      the parameter gradient, which also stays on the
 *                      device for gp_cnn_adam_step.  Synchronises when loss
 *                      or grad is requested.
 *   gp_cnn_adam_step   one Adam step (beta 0.9 / 0.999, eps 1e-8, bias
 *                      correction) with the last gradient.
 *   emd_solve_learned  emd_solve from the best of three starts: the learned
 *                      one (prior = emd_coarse_start(coarse_factor,
 *                      coarse_opts) when coarse_factor >= 2, no prior when
 *                      coarse_factor == 0; coarse_opts NULL: relative gap
 *                      1e-4, at most 100000 iterations, opts->use_graph),
 *                      the prior alone, and zero; the
 *                      start with the smallest duality gap at n = 0 is kept
 *                      (*start_used: 0 zero, 1 learned, 2 prior).  Other
 *                      arguments as emd_solve (p may be NULL);
 *                      opts->warm_start must be 0.  report->seconds includes
 *                      the coarse solve, the network and the gap probes.
 */
typedef struct gp_cnn_s* gp_cnn;
GP_API gp_status gp_cnn_create(gp_handle h, int base_channels, int bf16, unsigned long long seed, gp_cnn* out);
GP_API gp_status gp_cnn_destroy(gp_cnn net);
GP_API const char* gp_cnn_last_error(gp_cnn net);
GP_API long long gp_cnn_num_params(gp_cnn net);
GP_API gp_status gp_cnn_get_params(gp_cnn net, float* w);
GP_API gp_status gp_cnn_set_params(gp_cnn net, const float* w);
GP_API gp_status gp_cnn_forward(gp_cnn net, int B, const float* const* f0, const float* const* f1,
                                const float* const* prior, int N, float* phi, void* stream);
GP_API gp_status gp_cnn_loss_grad(gp_cnn net, int B, const float* const* f0, const float* const* f1,
                                  const float* const* prior, const float* const* phi_target, int N, double* loss,
                                  float* grad, void* stream);
GP_API gp_status gp_cnn_adam_step(gp_cnn net, double lr, void* stream);
GP_API gp_status emd_solve_learned(gp_handle h, gp_cnn net, const float* f0, const float* f1, float* m, float* p,
                                   float* phi, int N, int coarse_factor, const gp_opts* coarse_opts,
                                   const gp_opts* opts, gp_report* report, int* start_used, void* stream);

/*
 * rof_solve_learned: the same network as a warm start for rof_solve
 * (section 3.1; the strong convexity of Corollary 3.4 makes the primal
 * iterate the quantity a start should approximate).  The inputs per cell
 * are I - mean(I), 0 and the prior u_prior - mean(I) (rof_coarse_start's u
 * when coarse_factor >= 2, none when 0), i.e. gp_cnn_forward with
 * f0 = 8 (I - mean), f1 = -f0; the learned start is u_0 = mean(I) + phi
 * (a fidelity minimiser keeps the mean), paired with the prior's p (zero
 * without a prior).  The duality gap at n = 0 picks among the learned start,
 * the prior alone and zero (*start_used: 0 zero, 1 learned, 2 prior).
 * Training targets: u* - mean(I) of converged solves (see learn.py).
 * Arguments as rof_solve (u out, p may be NULL) and emd_solve_learned;
 * coarse_opts NULL: relative gap 1e-4, at most 100000 iterations.
 * Allocates 4 N^2 floats of scratch for the call.
 */
GP_API gp_status rof_solve_learned(gp_handle h, gp_cnn net, const float* I, float* u, float* p, int N,
                                   double lambda, int coarse_factor, const gp_opts* coarse_opts,
                                   const gp_opts* opts, gp_report* report, int* start_used, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GPROX_H */
