// C ABI of the library (declared in include/pp.h).  Argument validation,
// host/device staging, and error translation: no exception crosses the ABI.
#include "pp_internal.h"

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

static thread_local std::string g_create_err;
unsigned long long g_pp_launches = 0;

extern "C" long long pp_kernel_launches(void) {
  return (long long)__atomic_load_n(&g_pp_launches, __ATOMIC_RELAXED);
}

extern "C" void pp_default_options(pp_options *opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->prec = PP_FP64;
  opt->order = 2;
  opt->block = 8;
  opt->m_max = 96;
  opt->max_iter = 200;
  opt->res_tol = 1e-7;
  opt->jacobi_floor = 1e-3;
  opt->select = 0;
  opt->refine = 1;
  opt->seed = 0;
  opt->cuda_stream = nullptr;
  opt->graphs = 1;
}

static bool all_finite(const double *x, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}

template <class F> static pp_status guarded(pp_ctx *c, F &&f) {
  try {
    return f();
  } catch (const PPError &e) {
    if (c) c->err = e.msg;
    return e.st;
  } catch (const std::bad_alloc &) {
    if (c) c->err = "host allocation failed";
    return PP_ENOMEM;
  } catch (...) {
    if (c) c->err = "unexpected internal error";
    return PP_ECUDA;
  }
}

extern "C" pp_status pp_create(int nocc, int nvir, int naux, const double *eps, const void *B,
                               int B_dtype, const double *mu, const pp_options *opt, pp_ctx **out) {
  if (out) *out = nullptr;
  if (!out || !eps || (!B && naux > 0) || nocc < 1 || nvir < 1 || naux < 0 ||
      (B_dtype != 0 && B_dtype != 1)) {
    g_create_err = "pp_create: bad argument";
    return PP_EINVAL;
  }
  const int n = nocc + nvir;
  if (!all_finite(eps, n)) {
    g_create_err = "pp_create: non-finite orbital energy";
    return PP_EINVAL;
  }
  double emax_o = eps[0], emin_v = eps[nocc];
  for (int i = 0; i < nocc; ++i) emax_o = std::fmax(emax_o, eps[i]);
  for (int a = 0; a < nvir; ++a) emin_v = std::fmin(emin_v, eps[nocc + a]);
  if (!(emax_o < emin_v)) {
    g_create_err = "pp_create: need max(eps_occ) < min(eps_vir)";
    return PP_EINVAL;
  }
  const size_t nB = (size_t)naux * n * n;
  if (B_dtype == 0) {
    if (!all_finite((const double *)B, nB)) {
      g_create_err = "pp_create: non-finite B";
      return PP_EINVAL;
    }
  } else {
    const float *f = (const float *)B;
    for (size_t i = 0; i < nB; ++i)
      if (!std::isfinite(f[i])) {
        g_create_err = "pp_create: non-finite B";
        return PP_EINVAL;
      }
  }
  if (mu && !all_finite(mu, (size_t)3 * nocc * nvir)) {
    g_create_err = "pp_create: non-finite mu";
    return PP_EINVAL;
  }
  pp_options o;
  if (opt) o = *opt;
  else pp_default_options(&o);
  if (o.order < 0 || o.order > 2 || (o.prec != PP_FP64 && o.prec != PP_BF16 && o.prec != PP_BF16X3) || o.block < 1 ||
      o.m_max < 4 || !(o.res_tol > 0) || !(o.jacobi_floor > 0) || (o.select != 0 && o.select != 1) ||
      !(o.workspace_gb >= 0) || o.workspace_gb > 1e5 || (o.tda != 0 && o.tda != 1) || (o.graphs != 0 && o.graphs != 1)) {
    g_create_err = "pp_create: bad options";
    return PP_EINVAL;
  }
  pp_ctx *c = new (std::nothrow) pp_ctx();
  if (!c) {
    g_create_err = "pp_create: host allocation failed";
    return PP_ENOMEM;
  }
  c->o = nocc;
  c->v = nvir;
  c->Q = naux;
  c->n = n;
  c->ov = (long long)nocc * nvir;
  c->opt = o;
  pp_status st = guarded(c, [&]() -> pp_status {
    PP_CUDA(cudaGetDevice(&c->device));
    if (o.cuda_stream) {
      c->stream = (cudaStream_t)o.cuda_stream;
    } else {
      PP_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
      c->own_stream = true;
    }
    PP_CUDA(cudaEventCreate(&c->ev0));
    PP_CUDA(cudaEventCreate(&c->ev1));
    cudaStream_t s = c->stream;
    c->eps.ensure(sizeof(double) * n);
    PP_CUDA(cudaMemcpyAsync(c->eps.p, eps, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    if (mu) {
      c->mu.ensure(sizeof(double) * 3 * c->ov);
      PP_CUDA(cudaMemcpyAsync(c->mu.p, mu, sizeof(double) * 3 * c->ov, cudaMemcpyHostToDevice, s));
      c->has_mu = true;
    }
    const char *log_env = std::getenv("PP_LOG");
    const bool log_on = log_env && log_env[0] && log_env[0] != '0';
    auto now = [] { return std::chrono::steady_clock::now(); };
    auto ms = [](std::chrono::steady_clock::time_point a, std::chrono::steady_clock::time_point b) {
      return std::chrono::duration<double, std::milli>(b - a).count();
    };
    auto t0 = now();
    if (naux > 0) {
      DevBuf full;
      const size_t bytes = nB * (B_dtype == 0 ? sizeof(double) : sizeof(float));
      full.ensure(bytes);
      PP_CUDA(cudaMemcpyAsync(full.p, B, bytes, cudaMemcpyHostToDevice, s));
      build_residency(c, B_dtype == 0 ? full.as<double>() : nullptr,
                      B_dtype == 1 ? full.as<float>() : nullptr);
      PP_CUDA(cudaStreamSynchronize(s));
      full.release();
    } else {
      // no auxiliary functions: all integrals vanish
      c->Q = 0;
      c->opt.order = 0;
      build_residency(c, nullptr, nullptr);
    }
    PP_CUDA(cudaStreamSynchronize(s));
    auto t1 = now();
    if (c->opt.prec == PP_FP64 || c->opt.order < 2 || c->Q == 0) precompute_f64(c);
    else precompute_tc(c);
    PP_CUDA(cudaStreamSynchronize(s));
    if (log_on)
      std::fprintf(stderr, "[pp] create: upload + residency %.1f ms, precompute %.1f ms\n", ms(t0, t1), ms(t1, now()));
    // the Jacobi diagonal of S must be positive (S positive definite needs it)
    std::vector<double> dS(c->ov);
    PP_CUDA(cudaMemcpy(dS.data(), c->diagS.p, sizeof(double) * c->ov, cudaMemcpyDeviceToHost));
    for (double x : dS)
      if (!(x > 0.0)) throw PPError(PP_EMETRIC, "diag(S) is not positive: S is not positive definite");
    return PP_OK;
  });
  if (st != PP_OK) {
    g_create_err = c->err;
    pp_destroy(c);
    return st;
  }
  *out = c;
  return PP_OK;
}

extern "C" pp_status pp_sigma(pp_ctx *c, int nvec, const double *Z, double *sigma, double *metric,
                              int prec, int on_device) {
  if (!c) return PP_EINVAL;
  if (nvec < 0 || (nvec > 0 && (!Z || !sigma)) || (prec != PP_FP64 && prec != PP_BF16 && prec != PP_BF16X3)) {
    c->err = "pp_sigma: bad argument";
    return PP_EINVAL;
  }
  if (nvec == 0) return PP_OK;
  return guarded(c, [&]() -> pp_status {
    cudaStream_t s = c->stream;
    const size_t bytes = sizeof(double) * 2 * (size_t)c->ov * nvec;
    if (on_device) {
      apply_sigma(c, nvec, Z, sigma, metric, prec);
      PP_CUDA(cudaStreamSynchronize(s));
      return PP_OK;
    }
    DevBuf z, sg, mt;
    z.ensure(bytes);
    sg.ensure(bytes);
    if (metric) mt.ensure(bytes);
    PP_CUDA(cudaMemcpyAsync(z.p, Z, bytes, cudaMemcpyHostToDevice, s));
    apply_sigma(c, nvec, z.as<double>(), sg.as<double>(), metric ? mt.as<double>() : nullptr, prec);
    PP_CUDA(cudaMemcpyAsync(sigma, sg.p, bytes, cudaMemcpyDeviceToHost, s));
    if (metric) PP_CUDA(cudaMemcpyAsync(metric, mt.p, bytes, cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    z.release();
    sg.release();
    mt.release();
    return PP_OK;
  });
}

extern "C" pp_status pp_diagonal(pp_ctx *c, double *dA, double *dS) {
  if (!c || !dA || !dS) return PP_EINVAL;
  return guarded(c, [&]() -> pp_status {
    PP_CUDA(cudaMemcpyAsync(dA, c->diagA.p, sizeof(double) * c->ov, cudaMemcpyDeviceToHost, c->stream));
    PP_CUDA(cudaMemcpyAsync(dS, c->diagS.p, sizeof(double) * c->ov, cudaMemcpyDeviceToHost, c->stream));
    PP_CUDA(cudaStreamSynchronize(c->stream));
    return PP_OK;
  });
}

extern "C" pp_status pp_solve_window(pp_ctx *c, double omega0, double delta, int k, double *omega,
                                     double *osc, double *resid, double *vecs, int *nfound) {
  if (!c) return PP_EINVAL;
  if (k < 1 || !omega || !osc || !resid || !nfound || !std::isfinite(omega0) || !(delta >= 0)) {
    c->err = "pp_solve_window: bad argument";
    return PP_EINVAL;
  }
  return guarded(c, [&]() -> pp_status {
    PP_CUDA(cudaEventRecord(c->ev0, c->stream));
    cudaEvent_t t0, t1;
    PP_CUDA(cudaEventCreate(&t0));
    PP_CUDA(cudaEventCreate(&t1));
    PP_CUDA(cudaEventRecord(t0, c->stream));
    pp_status st = solve_windows_impl(c, 1, &omega0, &delta, &k, omega, osc, resid, vecs, nfound);
    PP_CUDA(cudaEventRecord(t1, c->stream));
    PP_CUDA(cudaEventSynchronize(t1));
    float ms = 0.f;
    PP_CUDA(cudaEventElapsedTime(&ms, t0, t1));
    c->st_solve_ms = ms;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return st;
  });
}

extern "C" pp_status pp_solve_windows(pp_ctx *c, int nwin, const double *omega0, const double *delta,
                                      const int *k, double *omega, double *osc, double *resid,
                                      int *nfound) {
  if (!c) return PP_EINVAL;
  if (nwin < 1 || !omega0 || !delta || !k || !omega || !osc || !resid || !nfound) {
    c->err = "pp_solve_windows: bad argument";
    return PP_EINVAL;
  }
  for (int w = 0; w < nwin; ++w)
    if (k[w] < 1 || !std::isfinite(omega0[w]) || !(delta[w] >= 0)) {
      c->err = "pp_solve_windows: bad window";
      return PP_EINVAL;
    }
  return guarded(c, [&]() -> pp_status {
    cudaEvent_t t0, t1;
    PP_CUDA(cudaEventCreate(&t0));
    PP_CUDA(cudaEventCreate(&t1));
    PP_CUDA(cudaEventRecord(t0, c->stream));
    pp_status st = solve_windows_impl(c, nwin, omega0, delta, k, omega, osc, resid, nullptr, nfound);
    PP_CUDA(cudaEventRecord(t1, c->stream));
    PP_CUDA(cudaEventSynchronize(t1));
    float ms = 0.f;
    PP_CUDA(cudaEventElapsedTime(&ms, t0, t1));
    c->st_solve_ms = ms;
    cudaEventDestroy(t0);
    cudaEventDestroy(t1);
    return st;
  });
}

extern "C" pp_status pp_solve_window_contour(pp_ctx *c, double omega0, double delta, int nquad, int k, double *omega,
                                             double *osc, double *resid, int *nfound) {
  if (!c) return PP_EINVAL;
  if (!std::isfinite(omega0) || !(delta > 0) || nquad < 2 || nquad > 32 || k < 1 || !omega || !osc || !resid ||
      !nfound) {
    c->err = "pp_solve_window_contour: bad argument";
    return PP_EINVAL;
  }
  return guarded(c, [&]() -> pp_status {
    PP_CUDA(cudaEventRecord(c->ev0, c->stream));
    const int outer = std::max(1, std::min(c->opt.max_iter, 60));
    pp_status st = riesz_impl(c, omega0, delta, nquad, 0, outer, omega, osc, resid, k, nfound);
    PP_CUDA(cudaEventRecord(c->ev1, c->stream));
    PP_CUDA(cudaEventSynchronize(c->ev1));
    float ms = 0.f;
    PP_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    c->st_solve_ms = ms;
    return st;
  });
}

extern "C" pp_status pp_polarizability(pp_ctx *c, int nfreq, const double *omega, double tol, int max_iter,
                                       double *alpha, double *resid, int *iterations) {
  if (!c) return PP_EINVAL;
  if (nfreq < 1 || !omega || !alpha || !(tol > 0) || max_iter < 1 || !all_finite(omega, (size_t)nfreq)) {
    c->err = "pp_polarizability: bad argument";
    return PP_EINVAL;
  }
  return guarded(c, [&]() -> pp_status {
    return polarizability_impl(c, nfreq, omega, tol, max_iter, alpha, resid, iterations);
  });
}

extern "C" pp_status pp_spectrum(pp_ctx *c, double w_lo, double w_hi, int nwin, int kmax, double eta, int ngrid,
                                 const double *grid, double *spec, int cap, double *omega, double *osc,
                                 double *resid, int *nroots) {
  if (!c) return PP_EINVAL;
  if (!std::isfinite(w_lo) || !std::isfinite(w_hi) || !(w_hi > w_lo) || nwin < 1 || kmax < 1 || !(eta > 0) ||
      ngrid < 0 || (ngrid > 0 && (!grid || !spec)) || cap < 0 || !nroots || (cap > 0 && (!omega || !osc || !resid))) {
    c->err = "pp_spectrum: bad argument";
    return PP_EINVAL;
  }
  if (ngrid > 0 && !all_finite(grid, (size_t)ngrid)) {
    c->err = "pp_spectrum: non-finite grid point";
    return PP_EINVAL;
  }
  return guarded(c, [&]() -> pp_status {
    return spectrum_impl(c, w_lo, w_hi, nwin, kmax, eta, ngrid, grid, spec, cap, omega, osc, resid, nroots);
  });
}

extern "C" pp_status pp_windows_begin(pp_ctx *c, int nwin, const double *omega0, const double *delta,
                                      const int *k) {
  if (!c) return PP_EINVAL;
  if (nwin < 1 || !omega0 || !delta || !k) {
    c->err = "pp_windows_begin: bad argument";
    return PP_EINVAL;
  }
  for (int w = 0; w < nwin; ++w)
    if (k[w] < 1 || !std::isfinite(omega0[w]) || !(delta[w] >= 0)) {
      c->err = "pp_windows_begin: bad window";
      return PP_EINVAL;
    }
  return guarded(c, [&]() -> pp_status { return windows_begin(c, nwin, omega0, delta, k); });
}

extern "C" pp_status pp_windows_step(pp_ctx *c, int *unfinished, long long *sigma_vectors, int *sigma_calls) {
  if (!c) return PP_EINVAL;
  return guarded(c, [&]() -> pp_status {
    pp_status st = windows_step(c, unfinished, sigma_vectors, sigma_calls);
    PP_CUDA(cudaStreamSynchronize(c->stream));
    return st;
  });
}

extern "C" pp_status pp_windows_end(pp_ctx *c, double *omega, double *osc, double *resid, int *nfound) {
  if (!c) return PP_EINVAL;
  if (!omega || !osc || !resid || !nfound) {
    c->err = "pp_windows_end: bad argument";
    return PP_EINVAL;
  }
  return guarded(c, [&]() -> pp_status { return windows_end(c, omega, osc, resid, nfound); });
}

extern "C" pp_status pp_last_stats(const pp_ctx *c, int *iterations, long long *sigma_vectors,
                                   double *sigma_ms, double *solve_ms) {
  if (!c) return PP_EINVAL;
  if (iterations) *iterations = c->st_iters;
  if (sigma_vectors) *sigma_vectors = c->st_sigvec;
  if (sigma_ms) *sigma_ms = c->st_sigma_ms;
  if (solve_ms) *solve_ms = c->st_solve_ms;
  return PP_OK;
}

size_t ctx_device_bytes(const pp_ctx *c) {
  const DevBuf *bufs[] = {&c->eps, &c->gap, &c->Bov, &c->Boo, &c->Bvv, &c->BvvP, &c->BooT, &c->GB,
                          &c->Gam, &c->mu, &c->p_oo, &c->q_oo, &c->p_vv, &c->q_vv, &c->diagA,
                          &c->diagS, &c->w_acc, &c->w_cq, &c->w_W, &c->w_U, &c->w_P, &c->w_EF,
                          &c->w_tmp, &c->w_T, &c->w_Tw, &c->w_V};
  size_t n = tc_plan_bytes(c) + (c->wb ? window_batch_bytes(c->wb) : 0);
  for (const DevBuf *b : bufs) n += b->bytes;
  return n;
}

extern "C" void pp_destroy(pp_ctx *c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  tc_destroy(c);
  window_run_destroy(c);
  if (c->wb) window_batch_destroy(c->wb);
  c->wb = nullptr;
  DevBuf *bufs[] = {&c->eps, &c->gap, &c->Bov, &c->Boo, &c->Bvv, &c->BvvP, &c->BooT, &c->GB,
                    &c->Gam, &c->mu, &c->p_oo, &c->q_oo, &c->p_vv, &c->q_vv, &c->diagA,
                    &c->diagS, &c->w_acc, &c->w_cq, &c->w_W, &c->w_U, &c->w_P, &c->w_EF,
                    &c->w_tmp, &c->w_T, &c->w_Tw, &c->w_V};
  for (DevBuf *b : bufs) b->release();
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

extern "C" const char *pp_last_error(const pp_ctx *c) {
  if (!c) return g_create_err.c_str();
  return c->err.c_str();
}
