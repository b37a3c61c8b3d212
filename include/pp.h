/*
 * pp.h -- C ABI of the GB300 window solver for the second-order polarization
 * propagator (arXiv 2512.09811).
 *
 * What is computed
 *   The response matrix of Sec. 2.2, Eq. (m_eigen):
 *       [A B; B A] (X; Y) = omega [S 0; 0 -S] (X; Y)
 *   over the particle-hole manifold {a^+ i, i^+ a} with the MP2 ground state,
 *   to zeroth, first or second order in the fluctuation potential W_N:
 *     S = 1 + S(2),              S(2)_ia,jb = d_ab rho_oo[i,j] - d_ij rho_vv[a,b]
 *     A = A(0) + A(1) + A(2),    A(0) = (e_a - e_i) d_ij d_ab,  A(1) = <aj||ib>
 *     B = B(1) + B(2),           B(1) = <ab||ij>
 *   (Eqs. s(2), a(0)-a(2), b(0)-b(2); matrix elements are the symmetrised
 *   double commutators of Eq. (mkk_so) with the normalised MP2 state).  Two-
 *   electron integrals are density fitted: (pq|rs) = sum_Q B[Q,p,q] B[Q,r,s].
 *   Interior roots in a frequency window are found with the inverse-Krylov /
 *   weighted-Jacobi / folded-spectrum method of Sec. 2.5; oscillator strengths
 *   use the zeroth-order property vector F = mu (Eq. pp_adc).
 *
 * Conventions
 *   Indices are spin orbitals, occupied first.  An "ov block" is a row-major
 *   [nocc][nvir] array of doubles (element (i,a) at i*nvir + a).  A
 *   supervector is [2][nocc][nvir]: the X block followed by the Y block.
 *   Arrays of supervectors are [nvec][2][nocc][nvir], contiguous.
 *
 * Ownership
 *   pp_create copies every input; the caller keeps its buffers.  Output
 *   buffers are caller-allocated.  The context owns all device memory and
 *   pp_destroy frees it.  Host pointers may be pageable or pinned.
 *
 * Errors
 *   Every call returns a pp_status; no exception crosses the ABI.  On error
 *   pp_last_error(ctx) holds a one-line message (ctx may be NULL for errors of
 *   pp_create, in which case pp_last_error(NULL) returns the last create error
 *   of the calling thread).
 *
 * Threading
 *   A context is not thread-safe; use one context per host thread, or guard it.
 *   All device work of a context is issued on one CUDA stream (opt->cuda_stream,
 *   or a stream the context creates); calls return after that stream is idle
 *   unless stated otherwise.
 */
#ifndef PP_H
#define PP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pp_ctx pp_ctx;

typedef enum {
  PP_OK = 0,
  PP_EINVAL = 1,      /* bad argument: size, NULL pointer, non-finite input, e_occ >= e_vir */
  PP_ENOMEM = 2,      /* device or host allocation failed */
  PP_ECUDA = 3,       /* a CUDA runtime call failed; see pp_last_error */
  PP_ENOTCONV = 4,    /* solver hit max_iter; best estimates are written */
  PP_ETIMEOUT = 5,    /* a bounded device wait ran out */
  PP_EMETRIC = 6,     /* S is not positive definite */
  PP_EUNSTABLE = 7    /* complex RPA roots (A - B not positive) */
} pp_status;

typedef enum {
  PP_FP64 = 0,   /* every contraction in FP64 (the plain form) */
  PP_BF16 = 2,   /* amplitude contractions on BF16 tensor cores (tcgen05) with FP32
                    accumulation, the other contractions in FP32; Krylov basis, projected
                    problem, fold centres and residuals stay FP64 */
  PP_BF16X3 = 3  /* as PP_BF16 with every tensor-core operand split into a BF16 pair
                    (hi + lo, three products): 16-bit significands, about 2^-16
                    relative error per product, used to refine */
} pp_precision;

typedef struct {
  int prec;            /* pp_precision of the solver's sigma: PP_FP64, PP_BF16 (with refine)
                          or PP_BF16X3 throughout */
  int order;           /* 0, 1 or 2 */
  int block;           /* trial vectors per window per iteration (default 8) */
  int m_max;           /* subspace size before a thick restart (default 96, <= 112) */
  int max_iter;        /* outer iterations per window (default 200) */
  double res_tol;      /* convergence: |M x - theta Sigma x| / |x^T Sigma x| (default 1e-7) */
  double jacobi_floor; /* |D_p| >= jacobi_floor in the Jacobi splitting (default 1e-3 Ha) */
  int select;          /* 0: k lowest roots in [omega0, omega0+delta]; 1: k nearest omega0 */
  int refine;          /* PP_BF16 only: split-precision refinement steps (default on) */
  uint64_t seed;       /* reserved for random initial vectors */
  void *cuda_stream;   /* cudaStream_t to use, or NULL to create one */
  double workspace_gb; /* device memory for one chunk of the tensor-core sigma workspaces
                          (0 = automatic: half of the free memory at first use, keeping 8 GB
                          free, at least 12 GB) */
  int tda;             /* 1: Tamm-Dancoff form (Sec. 2.2 with B = 0): M = diag(A, A), so the
                          roots are those of A X = omega S X and the sigma products skip every
                          B term (the amplitude contraction included); 0 (default): full form */
  int graphs;          /* tensor-core sigma: 1 (default) replays each chunk shape met before as a
                          captured CUDA graph; 0 launches kernel by kernel */
} pp_options;

/* Fill *opt with the defaults above. */
void pp_default_options(pp_options *opt);

/*
 * Create a context for one dot (Sec. 2.2 inputs; density fitting as in Sec. 3).
 *   eps   [nocc+nvir]            orbital energies, occupied first, host; need
 *                                max(eps_occ) < min(eps_vir) and finite values
 *   B     [naux][n][n], n = nocc+nvir, host; B_dtype 0 = double, 1 = float;
 *         symmetric in the last two indices (only the blocks oo, ov, vv are read)
 *   mu    [3][nocc][nvir]        dipole integrals, host (may be NULL: no oscillator strengths)
 * Computes the per-dot intermediates (MP2 densities and the 3-index ring
 * intermediate, the Jacobi diagonal) on the device: in FP64 when opt->prec is
 * PP_FP64, otherwise on the tensor cores (split-BF16 amplitudes, FP32 sums; relative
 * error about 1e-6 in these second-order intermediates, which every later sigma of
 * the context, FP64 ones included, inherits).  Returns PP_EMETRIC if the diagonal
 * of S is not positive.
 */
pp_status pp_create(int nocc, int nvir, int naux, const double *eps, const void *B, int B_dtype,
                    const double *mu, const pp_options *opt, pp_ctx **out);

/*
 * sigma = M z and (if metric != NULL) metric = Sigma z for nvec supervectors
 * (the matrix-free product of the abstract and Sec. 2.5.2).
 *   Z, sigma, metric: [nvec][2][nocc][nvir] doubles; host pointers if
 *   on_device == 0, device pointers (of the context's device) if on_device == 1.
 * prec selects the arithmetic: PP_FP64 or PP_BF16 (tensor cores, FP32 accumulation).
 */
pp_status pp_sigma(pp_ctx *ctx, int nvec, const double *Z, double *sigma, double *metric,
                   int prec, int on_device);

/*
 * Allocation-free metric product: out = Sigma z for nvec supervectors, the same
 * product as pp_sigma's metric output (Sigma = diag(S, -S), S = 1 + S(2) as above),
 * computed in FP64.  The paper has no counterpart to this entry point: it serves
 * callers that must not allocate device memory when they need the product -- code
 * running inside another framework's device memory pool (a raw cudaMalloc/cudaFree
 * would escape the pool's budget and accounting) and latency-critical loops that
 * avoid cudaMalloc/cudaFree because they can synchronise the device.  It calls
 * neither, nor any allocating library routine.
 *   Z, out: [nvec][2][nocc][nvir] doubles in DEVICE memory of the current device
 *           (no host staging); Z and out must not overlap.
 *   nvec * nocc * nvir must not exceed PP_METRIC_NOALLOC_MAX_ELEMS: the two
 *           intermediate products live in one fixed 16 MiB array per device compiled
 *           into the library.  Larger batches return PP_EINVAL with the sizes in
 *           pp_last_error; split them, or use pp_sigma.  nvec must also not exceed
 *           PP_METRIC_NOALLOC_MAX_NVEC (the 2 nvec half-vectors are one grid dimension).
 *   The current device must be the context's device (the one current at pp_create),
 *           else PP_EINVAL; Z and out must be that device's memory.
 *   The array is shared by all contexts and calls on a device: calls that overlap in
 *   time on one device (several host threads, or streams running concurrently) race
 *   on it and may return wrong results, so serialise them.  Nothing in it needs to
 *   start at zero.
 *   Set-up: the first call on each device (nvec = 0 does only the set-up) looks the
 *   array's address up with that device current and has the runtime load the kernels
 *   the call launches; it can load the library's device code, so it must precede any
 *   stream capture on that device.  Later calls load nothing.
 * Runs on the context's stream and returns after that stream has finished the work.
 */
#define PP_METRIC_NOALLOC_MAX_ELEMS (1LL << 19)
#define PP_METRIC_NOALLOC_MAX_NVEC 32767
pp_status pp_metric_noalloc(pp_ctx *ctx, int nvec, const double *Z, double *out);

/*
 * diag(A) and diag(S), each [nocc][nvir] host doubles: the Jacobi splitting D
 * of Sec. 2.5.2 (D = diag(M) - omega diag(Sigma)).
 */
pp_status pp_diagonal(pp_ctx *ctx, double *diagA, double *diagS);

/*
 * Roots of Eq. (m_eigen) inside one window (Sec. 2.5: weighted-Jacobi inverse
 * Krylov basis, folded-spectrum Rayleigh-Ritz on (M - omega Sigma)^2).
 *   select 0 (options): the k lowest roots in [omega0, omega0 + delta]; more than 8 are
 *                       found 8 at a time, each group starting 2 res_tol above the last root
 *                       of the previous one (roots closer than that are reported once);
 *   select 1:           the k roots nearest omega0 (delta ignored), k <= 24.
 *   omega[k], osc[k], resid[k]: host outputs, ascending omega; osc is 0 if mu was NULL.
 *   vecs: NULL or host [k][2][nocc][nvir], normalised X^T S X - Y^T S Y = 1.
 *   *nfound: number of roots written (< k if the window holds fewer).
 * Returns PP_ENOTCONV (with best estimates written) if max_iter is reached.
 */
pp_status pp_solve_window(pp_ctx *ctx, double omega0, double delta, int k, double *omega,
                          double *osc, double *resid, double *vecs, int *nfound);

/*
 * All roots inside [omega0, omega0 + delta] by the contour filter of Sec. 4.4 (the Riesz
 * projector, the alternative interior method the paper names): the projector onto the roots
 * inside the circle through omega0 and omega0 + delta is applied to a block of trial vectors
 * with nquad trapezoidal points on the circle (complex shifted systems solved by conjugate-
 * orthogonal CG with the Jacobi diagonal), followed by Rayleigh-Ritz with the accurate sigma,
 * repeated until every Ritz pair in the window meets res_tol (at most min(max_iter, 60)
 * filter applications).  The block holds 1.5 times the diagonal's count of roots in the window
 * plus 4, at most 64 vectors (PP_EINVAL for wider windows).  Mixed contexts filter with the
 * BF16 sigma until the worst in-window residual gains less than 2x per filter application,
 * then with the split form; their Rayleigh-Ritz products are always split-form.
 *   omega, osc, resid: host outputs of capacity k, ascending; *nfound: the roots in the window
 *   (PP_EINVAL if more than k).  PP_ENOTCONV with the last estimates if the limit is reached.
 */
pp_status pp_solve_window_contour(pp_ctx *ctx, double omega0, double delta, int nquad, int k, double *omega,
                                  double *osc, double *resid, int *nfound);

/*
 * Several windows of one dot solved together: all windows' trial blocks go
 * through one sigma batch per iteration.  Outputs are concatenated per window
 * at offsets off[w] = sum_{u<w} k[u]; nfound[nwin].
 */
pp_status pp_solve_windows(pp_ctx *ctx, int nwin, const double *omega0, const double *delta,
                           const int *k, double *omega, double *osc, double *resid, int *nfound);

/*
 * Frequency-dependent linear response (Eq. pp_adc at real frequencies): the dipole
 * polarizability tensor
 *     alpha[f][c][c'] = F_c^T (M - omega_f Sigma)^-1 F_c',   F_c = (mu_c; mu_c),
 * which equals sum_n 2 omega_n (mu_c . (X_n + Y_n)) (mu_c' . (X_n + Y_n)) / (omega_n^2 - omega_f^2)
 * over the positive roots (so the trace / 3 is sum_n f_n / (omega_n^2 - omega_f^2)).  The
 * three systems per frequency are solved by preconditioned MINRES with the Jacobi diagonal
 * |diag(M - omega Sigma)| (floored at jacobi_floor) as preconditioner; mixed contexts refine
 * on the residual (split-BF16 residuals; BF16 corrections, switched to the split form once
 * an outer step gains less than 4x, as near a root), FP64 contexts run in FP64.
 *   omega[nfreq]: host frequencies (Ha); off resonance (a frequency at a root is singular).
 *   tol: relative residual |F - K x| / |F| to reach; max_iter: MINRES iterations per frequency.
 *   alpha: host [nfreq][3][3]; resid (may be NULL): host [nfreq], the final relative residual
 *   (largest of the three systems, accurate operator); iterations (may be NULL): host [nfreq].
 * Needs dipole integrals (mu at pp_create), else PP_EINVAL.  PP_ENOTCONV if a frequency
 * ends above 10 tol (its best estimate is written).  In mixed contexts the residual cannot
 * fall below the noise of the split-BF16 products (their rounding is not linear in x) times
 * |x| / |F|, which grows near a root: about 1e-5 between two roots 3 mHa apart at the
 * 16/64/192 dot, where the polarizability itself is still accurate to 4e-5.
 */
pp_status pp_polarizability(pp_ctx *ctx, int nfreq, const double *omega, double tol, int max_iter, double *alpha,
                            double *resid, int *iterations);

/*
 * Absorption spectrum of the roots in [w_lo, w_hi] (Sec. 3 spectra; Eq. pp_adc): the range is
 * cut into nwin equal windows solved together (Sec. 2.5, the context's options; select is
 * taken as 0 for this call), each for its kmax lowest roots; a window that returns kmax roots
 * is halved and its halves solved again (up to 8 times), and a root found by two windows on
 * their shared edge (within 2 res_tol) is kept once.  Then
 *     spec[g] = sum_n f_n (eta / pi) / ((grid[g] - omega_n)^2 + eta^2)
 * for the ngrid host frequencies in grid (Lorentzian of half width eta > 0; ngrid may be 0).
 *   omega, osc, resid: host outputs of capacity cap (ascending omega); *nroots receives the
 *   number of roots in the range -- if it exceeds cap nothing is written and PP_EINVAL is
 *   returned.  PP_ENOTCONV if a window reached max_iter (its best estimates are included).
 */
pp_status pp_spectrum(pp_ctx *ctx, double w_lo, double w_hi, int nwin, int kmax, double eta, int ngrid,
                      const double *grid, double *spec, int cap, double *omega, double *osc, double *resid,
                      int *nroots);

/*
 * The same batched solve driven one block iteration at a time (for callers that interleave
 * other work, and for timing single iterations).  pp_windows_begin places the windows in the
 * context's window slots (arguments as pp_solve_windows; an earlier batch that was not
 * collected is abandoned).  Each pp_windows_step runs one iteration of every unfinished
 * window -- Rayleigh-Ritz and the folded extraction, residuals, Jacobi directions, block
 * CGS2, and one sigma batch per precision phase for the new vectors of all windows (Sec.
 * 2.5) -- and returns after the context's stream is idle; *unfinished receives the windows
 * still running, *sigma_vectors the supervectors multiplied in this step and *sigma_calls
 * the sigma batches applied (any of them may be NULL).  A step with no unfinished window
 * does nothing.  pp_windows_end, once no window is unfinished, writes the results as
 * pp_solve_windows does and releases the slots (PP_EINVAL while windows are running;
 * PP_ENOTCONV if a window reached max_iter).
 */
pp_status pp_windows_begin(pp_ctx *ctx, int nwin, const double *omega0, const double *delta, const int *k);
pp_status pp_windows_step(pp_ctx *ctx, int *unfinished, long long *sigma_vectors, int *sigma_calls);
pp_status pp_windows_end(pp_ctx *ctx, double *omega, double *osc, double *resid, int *nfound);

/* Statistics of the last solve: outer iterations, sigma supervectors applied,
   milliseconds spent in sigma and in the whole solve. */
pp_status pp_last_stats(const pp_ctx *ctx, int *iterations, long long *sigma_vectors,
                        double *sigma_ms, double *solve_ms);

/*
 * Launch timing of the two tensor-core kernels (a profiling aid for the
 * roofline of the dominant contraction).  pp_profile(ctx, 1) resets the
 * counters and records CUDA events around every later launch on the context's
 * stream; pp_profile(ctx, 0) stops recording.  pp_profile_read returns, for
 * kernel id 0 (the amplitude contraction GEMM, Eq. (b(2)) ladder and ring
 * parts), id 1 (the amplitude slab generator, MP2 t of Sec. 2.2) or id 2 (the
 * launches of id 0 that ran in the split form, three BF16 products each), the number
 * of launches, their summed device milliseconds and their algorithmic FLOPs: each
 * contraction counted once, 2 M N K with K excluding the zero padding; the three BF16
 * products of the split (refinement) form count as one, and the generator counts one
 * Q-long product per amplitude (the exchange integral (id|jc) of t_ij^cd is the direct
 * integral of t_ij^dc).
 */
pp_status pp_profile(pp_ctx *ctx, int enable);
pp_status pp_profile_read(pp_ctx *ctx, int id, long long *launches, double *ms, double *flops);

/*
 * The tensor-core GEMM autotuner's table as text (one line per GEMM site and shape class:
 * the chosen tile width, pipeline depth and K split, and the measured milliseconds of each
 * tile configuration), preceded by the number of tunings run in this process.  Writes at most
 * cap bytes (NUL-terminated) to buf and returns the size needed.  The tuner runs the first
 * time a site meets a shape class; PP_AUTOTUNE=0 disables it, PP_TUNE_CACHE=<file> keeps the
 * table in a text file across processes.
 */
long long pp_autotune_report(char *buf, long long cap);

/* Number of CUDA kernels this library has launched in the process so far (all contexts). */
long long pp_kernel_launches(void);

/* Release everything the context owns.  NULL-safe. */
void pp_destroy(pp_ctx *ctx);

/* One-line description of the last error on ctx (or of the last failed pp_create). */
const char *pp_last_error(const pp_ctx *ctx);

/* ------------------------------------------------------------------------------------
 * Serving: window-solve requests for several dots, continuously batched on one GPU.
 *
 * Each dot is registered once (host copies of its inputs are kept).  A dot is made
 * resident -- its context (Sec. 2.2 intermediates) and its window slots on the device --
 * when a request for it is scheduled and its estimated device footprint fits hbm_budget
 * next to the resident dots; idle resident dots are evicted, least recently used first,
 * to make room, and a dot that still does not fit waits until one does.  Worker threads
 * advance resident dots one solver iteration at a time (the Sec. 2.5 window solver of
 * pp_solve_windows); before each iteration the dot's queued requests are admitted into
 * free window slots, so a request that arrives while others are running joins their
 * sigma batches at the next iteration, and a finished window frees its slot at once.
 * Dots are stepped by different workers on their own streams, so their work overlaps on
 * the device.  Each result equals the one pp_solve_window gives for the same request
 * within the solver tolerance (the iteration path differs with the batch).
 * ------------------------------------------------------------------------------------ */
typedef struct pp_server pp_server;

typedef struct {
  long long submitted, completed, failed;  /* requests (completed includes PP_ENOTCONV) */
  long long ctx_created, ctx_evicted;      /* dots made resident / evicted */
  long long steps;                         /* solver iterations run (all dots) */
  int max_concurrent_dots;                 /* most dots stepped at the same time */
  int max_windows_per_step;                /* most windows advanced by one step of one dot */
  int resident_dots;                       /* at the time of the call */
  long long resident_bytes;                /* estimated / measured device bytes of resident dots */
} pp_server_stats_t;

/*
 * hbm_budget: device bytes the resident dots may hold (an estimate per dot until it has
 * run, then its measured allocations).  opt: solver options for every dot (opt->cuda_stream
 * must be NULL: each dot gets its own stream; NULL = defaults; workspace_gb 0 means 12 GB
 * per dot here).  slots_per_dot: windows a
 * dot advances together (1..16).  nworkers: worker threads (0 = 4, at most 16).  The
 * current device is the server's device.
 */
pp_status pp_server_create(size_t hbm_budget, const pp_options *opt, int slots_per_dot, int nworkers,
                           pp_server **out);
/* Register a dot (arguments as pp_create; inputs are copied).  *dot_id numbers dots from 0.
   Returns PP_ENOMEM (message in pp_server_last_error) if the dot's estimated device footprint
   alone exceeds hbm_budget: such a dot could never be admitted. */
pp_status pp_server_add_dot(pp_server *srv, int nocc, int nvir, int naux, const double *eps, const void *B,
                            int B_dtype, const double *mu, int *dot_id);
/* Queue a window request (arguments as pp_solve_window, select rule from the options). */
pp_status pp_server_submit(pp_server *srv, int dot_id, double omega0, double delta, int k,
                           unsigned long long *req_id);
/*
 * Wait up to timeout_ms (0: poll, < 0: no limit) for a request.  Returns PP_ETIMEOUT while
 * it is not finished (it stays queued or running).  Otherwise writes omega/osc/resid (arrays
 * of the request's k; any may be NULL), *nfound, latency_ms[0] = finish - submit and
 * latency_ms[1] = admission - submit (may be NULL), forgets the request and returns its
 * status (PP_OK, PP_ENOTCONV, or the failure of its dot).
 */
pp_status pp_server_wait(pp_server *srv, unsigned long long req_id, int timeout_ms, double *omega,
                         double *osc, double *resid, int *nfound, double *latency_ms);
pp_status pp_server_stats(pp_server *srv, pp_server_stats_t *out);
/* Message of the last failed request returned by pp_server_wait. */
const char *pp_server_last_error(const pp_server *srv);
/* Stop the workers and free every dot.  No other call on srv may run concurrently. */
void pp_server_destroy(pp_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* PP_H */
