// Internal declarations of the GB300 polarization-propagator library.
// Layouts (all row-major, doubles unless stated):
//   eps  [n]            orbital energies, occupied first
//   gap  [o][v]         e_a - e_i
//   Bov  [Q][o][v]      B[Q,i,a];   Boo [Q][o][o];   Bvv [Q][v][v]
//   BvvP [v][Q][v]      BvvP[b][Q][d] = B[Q,b,d]     (one GEMM forms V B_Q for every Q)
//   BooT [o][o][Q]      BooT[i][k][Q] = B[Q,i,k]     (contraction over (k, Q))
//   GB   [2Q][o][v]     rows 0..Q-1: Bov + Gamma, rows Q..2Q-1: Bov
//   Gam  [Q][o][v]      Gamma_Q[j,a] = sum_kc t_jk^ac B[Q,k,c]
//   p_oo, q_oo [o][o]; p_vv, q_vv [v][v]: pair sums of the MP2 amplitudes
//   supervectors [nvec][2][o][v] = half-vectors V[2 nvec][o][v]
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pp.h"

struct PPError {
  pp_status st;
  std::string msg;
  PPError(pp_status s, std::string m) : st(s), msg(std::move(m)) {}
};

#define PP_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      throw PPError(e_ == cudaErrorMemoryAllocation ? PP_ENOMEM : PP_ECUDA,                  \
                    std::string(#call) + " -> " + cudaGetErrorString(e_));                   \
  } while (0)

// every kernel launch of the library is followed by PP_LAUNCH_CHECK, which also counts it
extern unsigned long long g_pp_launches;
#define PP_LAUNCH_CHECK(name)                                                                \
  do {                                                                                       \
    __atomic_fetch_add(&g_pp_launches, 1ull, __ATOMIC_RELAXED);                              \
    cudaError_t e_ = cudaGetLastError();                                                     \
    if (e_ != cudaSuccess) throw PPError(PP_ECUDA, std::string(name) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// grow-only device buffer (owns its allocation; not copyable)
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void ensure(size_t nbytes) {
    if (nbytes <= bytes) return;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    PP_CUDA(cudaMalloc(&p, nbytes));
    bytes = nbytes;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class T> T *as() const { return reinterpret_cast<T *>(p); }
};

// ---------------------------------------------------------------------------
// generic strided FP64 GEMM with an inner reduction batch and an outer batch:
//   C_b = alpha * sum_{t < nred} op(A_{b,t}) op(B_{b,t}) + beta * C_b
// op(A) is M x K with element (m,k) at A + b*a_batch + t*a_red + m*a_m + k*a_k;
// op(B) is K x N with element (k,n) at B + b*b_batch + t*b_red + k*b_k + n*b_n;
// C element (m,n) at C + b*c_batch + m*c_m + n*c_n.
// ---------------------------------------------------------------------------
template <class T> struct GemmS {
  int M = 0, N = 0, K = 0, nred = 1, nbatch = 1;
  // ksplit > 1 splits the reduction (over nred, or over K when nred == 1) across blocks and
  // accumulates alpha * partial into C atomically; it requires beta == 1 (C already holds
  // the addend, zero it first for a plain product)
  int ksplit = 1;
  const T *A = nullptr;
  long long a_m = 0, a_k = 0, a_red = 0, a_batch = 0;
  const T *B = nullptr;
  long long b_k = 0, b_n = 0, b_red = 0, b_batch = 0;
  T *C = nullptr;
  long long c_m = 0, c_n = 0, c_batch = 0;
  T alpha = 1, beta = 0;
};
using GemmF64 = GemmS<double>;
using GemmF32 = GemmS<float>;
void gemm_f64(const GemmF64 &g, cudaStream_t s);
void gemm_f32(const GemmF32 &g, cudaStream_t s);
// has the runtime load the FP64 GEMM kernel on the current device now (lazy module loading
// would otherwise load it, and may allocate for it, at its first launch)
void gemm_f64_preload();

// T slab in FP64: rows (i - i0, c) for i in [i0, i0+ni), columns (j, d):
// T[(ii*v + c)*ov + j*v + d] = t_ij^cd = ((ci|dj) - (cj|di)) / (e_i + e_j - e_c - e_d)
void tslab_f64(const double *Bov, const double *eps, int o, int v, int Q, int i0, int ni, double *T,
               cudaStream_t s);

// elementwise helpers (sigma_f64.cu)
void ew_copy_scale(double *y, const double *x, double a, long long n, cudaStream_t s);

// ---------------------------------------------------------------------------
// BF16 tensor-core (tcgen05) path, tc_gemm.cu
// ---------------------------------------------------------------------------
struct TcPlan;  // opaque

// ---------------------------------------------------------------------------
// window solver slots (solver.cu)
// ---------------------------------------------------------------------------
struct WindowBatch;  // opaque
struct WindowRun;    // opaque: the slots and k of a pp_windows_begin batch
struct WindowResult {
  int status = PP_OK;  // PP_OK or PP_ENOTCONV
  int iters = 0;
  std::vector<double> omega, osc, resid;  // nfound roots, ascending
  std::vector<double> vecs;               // [nfound][2 ov] when vectors were requested
};

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
struct pp_ctx {
  int o = 0, v = 0, Q = 0, n = 0;
  long long ov = 0;
  int device = 0;  // CUDA device current at pp_create; all of the context's memory lives there
  pp_options opt{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::string err;
  bool has_mu = false;

  // resident FP64 data
  DevBuf eps, gap, Bov, Boo, Bvv, BvvP, BooT, GB, Gam, mu;
  DevBuf p_oo, q_oo, p_vv, q_vv, diagA, diagS;

  // FP64 sigma workspaces
  DevBuf w_acc, w_cq, w_W, w_U, w_P, w_EF, w_tmp, w_T, w_Tw, w_V;
  int sig_chunk = 2;  // half-vectors per chunk (even)
  int slab_i = 1;     // occupied indices per T slab

  // BF16 tensor-core path (lazily built)
  TcPlan *tc = nullptr;

  // window slots of the solver (lazily built, reused across pp_solve_window calls)
  WindowBatch *wb = nullptr;
  // windows begun by pp_windows_begin and not yet collected by pp_windows_end
  WindowRun *run = nullptr;

  // stats of the last solve
  int st_iters = 0;
  long long st_sigvec = 0;
  double st_sigma_ms = 0.0, st_solve_ms = 0.0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
};

// sigma_f64.cu
void build_residency(pp_ctx *c, const double *Bd, const float *Bf);
void ensure_bvvp(pp_ctx *c);  // the permuted FP64 Bvv of the FP64 sigma (built on first use)
// per-dot intermediates (MP2 pair sums p_oo, q_oo, p_vv, q_vv, ring intermediate Gamma, then
// GB and the Jacobi diagonal): precompute_f64 in FP64; precompute_tc on the tensor cores
// (split-BF16 amplitude slabs and Gamma, FP32 pair sums), both via begin / finish
void precompute_begin(pp_ctx *c);
void precompute_finish(pp_ctx *c);
void precompute_f64(pp_ctx *c);
void precompute_tc(pp_ctx *c);
void sigma_f64(pp_ctx *c, int nvec, const double *Zd, double *sig_d, double *met_d);
// tc_gemm.cu
void sigma_bf16(pp_ctx *c, int nvec, const double *Zd, double *sig_d, double *met_d, bool split);
void tc_destroy(pp_ctx *c);
// solver.cu
pp_status solve_windows_impl(pp_ctx *c, int nwin, const double *omega0, const double *delta, const int *k,
                             double *omega, double *osc, double *resid, double *vecs, int *nfound);
// the context's cached slots with room for cap windows (rebuilt when too small or in use)
WindowBatch *window_batch(pp_ctx *c, int cap, bool vectors);
WindowBatch *window_batch_new(pp_ctx *c, int cap, bool vectors);  // owned by the caller
void window_batch_destroy(WindowBatch *wb);
int window_batch_add(WindowBatch *wb, double omega0, double delta, int k);  // slot, or -1 when full
bool window_batch_has_work(const WindowBatch *wb);
void window_batch_step(WindowBatch *wb);  // one iteration of every unfinished window
bool window_batch_finished(const WindowBatch *wb, int slot);
WindowResult window_batch_take(WindowBatch *wb, int slot);  // frees the slot
void window_batch_release(WindowBatch *wb, int slot);       // frees the slot, result dropped
int window_batch_capacity(const WindowBatch *wb);
size_t window_batch_bytes(const WindowBatch *wb);
// device bytes held by the tensor-core plan (tc_gemm.cu) and by a whole context (capi.cu)
size_t tc_plan_bytes(const pp_ctx *c);
long long tc_workspace_bytes(const pp_ctx *c);
size_t ctx_device_bytes(const pp_ctx *c);
int window_batch_used(const WindowBatch *wb);
// windows driven one block iteration at a time (solver.cu; C ABI pp_windows_*)
pp_status windows_begin(pp_ctx *c, int nwin, const double *omega0, const double *delta, const int *k);
pp_status windows_step(pp_ctx *c, int *unfinished, long long *sigma_vectors, int *sigma_calls);
pp_status windows_end(pp_ctx *c, double *omega, double *osc, double *resid, int *nfound);
void window_run_destroy(pp_ctx *c);
// absorption spectrum of a frequency range from stitched window solves (spectrum.cu)
pp_status spectrum_impl(pp_ctx *c, double w_lo, double w_hi, int nwin, int kmax, double eta, int ngrid,
                        const double *grid, double *spec, int cap, double *omega, double *osc, double *resid,
                        int *nroots);
// contour (Riesz projector) filter solver of one window (solver.cu)
pp_status riesz_impl(pp_ctx *c, double omega0, double delta, int nquad, int m0, int max_outer, double *omega,
                     double *osc, double *resid, int cap, int *nfound);
// frequency-dependent dipole polarizability by preconditioned MINRES (response.cu)
pp_status polarizability_impl(pp_ctx *c, int nfreq, const double *omega, double tol, int max_iter, double *alpha,
                              double *resid, int *iterations);
// dispatch of one sigma application (solver and C ABI)
void apply_sigma(pp_ctx *c, int nvec, const double *Zd, double *sig_d, double *met_d, int prec);
