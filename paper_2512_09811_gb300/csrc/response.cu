// Frequency-dependent linear response (declared in include/pp.h as pp_polarizability).
//
// Eq. (pp_adc) gives the propagator as F^T (omega - M)^-1 F in the non-orthogonal basis of
// Eq. (m_eigen).  With the pencil (M, Sigma) and the zeroth-order property vectors
// F_c = (mu_c; mu_c) (c = x, y, z), the dipole polarizability at a real frequency omega is
//   alpha_cc'(omega) = F_c^T (M - omega Sigma)^-1 F_c'
//                    = sum_n 2 omega_n (mu_c . u_n)(mu_c' . u_n) / (omega_n^2 - omega^2),
// u_n = X_n + Y_n, so (1/3) tr alpha = sum_n f_n / (omega_n^2 - omega^2).  The three systems
// K x_c = F_c, K = M - omega Sigma (symmetric, indefinite between roots), are solved together
// by preconditioned MINRES (Paige and Saunders' short recurrences for symmetric indefinite
// systems), with the positive diagonal preconditioner |diag K| floored at jacobi_floor -- the
// Jacobi splitting of Sec. 2.5.2 -- and one sigma batch of three supervectors per iteration.
//
// Arithmetic.  FP64 contexts: one MINRES run with the FP64 sigma.  Mixed contexts: iterative
// refinement on the residual -- the outer residual r = F - K x is formed with the split-BF16
// sigma, and each correction K d = r is solved by MINRES to a relative residual of 1e-2 (or
// the requested tolerance, if that is looser); x += d.  The corrections use the BF16 sigma
// until an outer step reduces the residual by less than 4x (near a root, where cond(K) times
// the BF16 operator error nears 1), then the split form.
#include "pp_internal.h"

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace {

constexpr int NR = 3;  // right-hand sides: the three dipole components

__device__ __forceinline__ double lr_block_sum(double x, double *red) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = x;
  __syncthreads();
  x = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
  if (w == 0)
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  return x;
}

// F_c = (mu_c; mu_c), c < NR, each a supervector of length 2 ov
__global__ void k_lr_rhs(double *__restrict__ F, const double *__restrict__ mu, long long ov) {
  const long long L = 2 * ov, total = NR * L;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const long long c = p / L, e = p % L;
    F[p] = mu[c * ov + (e % ov)];
  }
}
// out = sig - omega met  (K v from the sigma and metric products)
__global__ void k_lr_apply(double *__restrict__ out, const double *__restrict__ sig, const double *__restrict__ met,
                           double omega, long long n) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x)
    out[p] = sig[p] - omega * met[p];
}
// y = r / |D|, D = diag(M - omega Sigma) = [dA - omega dS; dA + omega dS], |D| floored
__global__ void k_lr_prec(double *__restrict__ y, const double *__restrict__ r, const double *__restrict__ dA,
                          const double *__restrict__ dS, double omega, double floor_, long long ov) {
  const long long L = 2 * ov, total = NR * L;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const long long e = p % L, ia = e % ov;
    const double d = fabs((e < ov) ? dA[ia] - omega * dS[ia] : dA[ia] + omega * dS[ia]);
    y[p] = r[p] / fmax(d, floor_);
  }
}
// out[c] = a_c . b_c, one block per right-hand side
__global__ void __launch_bounds__(256) k_lr_dot(const double *__restrict__ a, const double *__restrict__ b,
                                                long long L, double *__restrict__ out) {
  __shared__ double red[8];
  const long long off = (long long)blockIdx.x * L;
  double s = 0.0;
  for (long long l = threadIdx.x; l < L; l += blockDim.x) s += a[off + l] * b[off + l];
  s = lr_block_sum(s, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}
// y_c = alpha_c x_c + beta_c y_c (per right-hand side coefficients in device memory)
__global__ void k_lr_axpby(double *__restrict__ y, const double *__restrict__ x, const double *__restrict__ coef,
                           long long L) {
  const long long total = NR * L;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(p / L);
    const double b = coef[NR + c];
    y[p] = coef[c] * x[p] + (b != 0.0 ? b * y[p] : 0.0);  // y is not read when b = 0
  }
}
// MINRES direction and iterate: wn = (v - e w1 - d w2) g, x += phi wn (coefficients per rhs)
__global__ void k_lr_wx(double *__restrict__ wn, const double *__restrict__ v, const double *__restrict__ w1,
                        const double *__restrict__ w2, double *__restrict__ x, const double *__restrict__ coef,
                        long long L) {
  const long long total = NR * L;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(p / L);
    const double g = coef[2 * NR + c];
    const double w = g != 0.0 ? (v[p] - coef[c] * w1[p] - coef[NR + c] * w2[p]) * g : 0.0;  // 0: frozen
    wn[p] = w;
    x[p] += coef[3 * NR + c] * w;
  }
}

inline unsigned ew_blocks(long long n) {
  return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16));
}

struct Lr {
  pp_ctx *c;
  cudaStream_t s;
  long long ov, L;
  DevBuf buf;
  double *F, *x, *r, *d, *v, *y, *r1, *r2, *w, *w1, *w2, *sg, *mt, *coef, *dots;

  explicit Lr(pp_ctx *ctx) : c(ctx), s(ctx->stream), ov(ctx->ov), L(2 * ctx->ov) {
    const size_t vec = (size_t)NR * L;
    buf.ensure(sizeof(double) * (13 * vec + 64));
    double *p = buf.as<double>();
    double **slots[] = {&F, &x, &r, &d, &v, &y, &r1, &r2, &w, &w1, &w2, &sg, &mt};
    for (double **q : slots) {
      *q = p;
      p += vec;
    }
    coef = p;
    dots = p + 32;
  }
  void dot(const double *a, const double *b, double *h) {
    k_lr_dot<<<NR, 256, 0, s>>>(a, b, L, dots);
    PP_LAUNCH_CHECK("k_lr_dot");
    PP_CUDA(cudaMemcpyAsync(h, dots, sizeof(double) * NR, cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
  }
  void set_coef(const double *h, int n) {
    PP_CUDA(cudaMemcpyAsync(coef, h, sizeof(double) * n, cudaMemcpyHostToDevice, s));
  }
  // out = K in = (M - omega Sigma) in, for the NR supervectors of in
  void apply(const double *in, double *out, double omega, int prec) {
    apply_sigma(c, NR, in, sg, mt, prec);
    k_lr_apply<<<ew_blocks(NR * L), 256, 0, s>>>(out, sg, mt, omega, NR * L);
    PP_LAUNCH_CHECK("k_lr_apply");
  }
  void prec(double *out, const double *in, double omega) {
    k_lr_prec<<<ew_blocks(NR * L), 256, 0, s>>>(out, in, c->diagA.as<double>(), c->diagS.as<double>(), omega,
                                                c->opt.jacobi_floor, ov);
    PP_LAUNCH_CHECK("k_lr_prec");
  }
  // MINRES for K dx = b (b in `rhs`), dx starts at zero; returns iterations; stops when every
  // right-hand side's preconditioned residual estimate is below tol relative to its start
  int minres(const double *rhs, double *dx, double omega, int prec_id, double tol, int max_it) {
    PP_CUDA(cudaMemsetAsync(dx, 0, sizeof(double) * NR * L, s));
    PP_CUDA(cudaMemsetAsync(w, 0, sizeof(double) * NR * L, s));
    PP_CUDA(cudaMemsetAsync(w1, 0, sizeof(double) * NR * L, s));
    PP_CUDA(cudaMemsetAsync(w2, 0, sizeof(double) * NR * L, s));
    PP_CUDA(cudaMemcpyAsync(r1, rhs, sizeof(double) * NR * L, cudaMemcpyDeviceToDevice, s));
    PP_CUDA(cudaMemcpyAsync(r2, rhs, sizeof(double) * NR * L, cudaMemcpyDeviceToDevice, s));
    prec(y, r1, omega);
    double h[NR], beta1[NR], beta[NR], oldb[NR], dbar[NR], epsln[NR], phibar[NR], cs[NR], sn[NR];
    dot(r1, y, h);
    for (int q = 0; q < NR; ++q) {
      if (!(h[q] >= 0.0)) throw PPError(PP_ECUDA, "pp_polarizability: preconditioner not positive");
      beta1[q] = beta[q] = std::sqrt(h[q]);
      oldb[q] = dbar[q] = epsln[q] = 0.0;
      phibar[q] = beta1[q];
      cs[q] = -1.0;
      sn[q] = 0.0;
    }
    // a right-hand side that has converged is frozen: all its coefficients are zero from then
    // on (its Lanczos recurrence would otherwise run on with a vanishing beta)
    bool conv[NR];
    for (int q = 0; q < NR; ++q) conv[q] = !(beta1[q] > 0.0);
    double cf[4 * NR];
    int it = 0;
    for (; it < max_it; ++it) {
      bool done = true;
      for (int q = 0; q < NR; ++q) {
        conv[q] = conv[q] || phibar[q] <= tol * beta1[q];
        done = done && conv[q];
      }
      if (done) break;
      // v = y / beta
      for (int q = 0; q < NR; ++q) {
        cf[q] = (!conv[q] && beta[q] > 0.0) ? 1.0 / beta[q] : 0.0;
        cf[NR + q] = 0.0;
      }
      set_coef(cf, 2 * NR);
      k_lr_axpby<<<ew_blocks(NR * L), 256, 0, s>>>(v, y, coef, L);
      PP_LAUNCH_CHECK("k_lr_axpby");
      // y = K v - (beta / oldb) r1
      apply(v, y, omega, prec_id);
      if (it > 0) {
        for (int q = 0; q < NR; ++q) {
          cf[q] = (!conv[q] && oldb[q] != 0.0) ? -beta[q] / oldb[q] : 0.0;
          cf[NR + q] = 1.0;
        }
        set_coef(cf, 2 * NR);
        k_lr_axpby<<<ew_blocks(NR * L), 256, 0, s>>>(y, r1, coef, L);
        PP_LAUNCH_CHECK("k_lr_axpby");
      }
      double alfa[NR];
      dot(v, y, alfa);
      // y -= (alfa / beta) r2; then r1 <- r2, r2 <- y (pointer rotation), y = P^-1 r2
      for (int q = 0; q < NR; ++q) {
        cf[q] = (!conv[q] && beta[q] > 0.0) ? -alfa[q] / beta[q] : 0.0;
        cf[NR + q] = 1.0;
      }
      set_coef(cf, 2 * NR);
      k_lr_axpby<<<ew_blocks(NR * L), 256, 0, s>>>(y, r2, coef, L);
      PP_LAUNCH_CHECK("k_lr_axpby");
      std::swap(r1, r2);  // r1 <- old r2
      std::swap(r2, y);   // r2 <- new residual vector; y is free
      prec(y, r2, omega);
      dot(r2, y, h);
      for (int q = 0; q < NR; ++q) {
        if (conv[q]) {
          cf[q] = cf[NR + q] = cf[2 * NR + q] = cf[3 * NR + q] = 0.0;
          continue;
        }
        oldb[q] = beta[q];
        beta[q] = std::sqrt(std::max(h[q], 0.0));
        const double oldeps = epsln[q];
        const double delta = cs[q] * dbar[q] + sn[q] * alfa[q];
        const double gbar = sn[q] * dbar[q] - cs[q] * alfa[q];
        epsln[q] = sn[q] * beta[q];
        dbar[q] = -cs[q] * beta[q];
        double gamma = std::sqrt(gbar * gbar + beta[q] * beta[q]);
        if (!(gamma > 0.0)) gamma = 1e-300;
        cs[q] = gbar / gamma;
        sn[q] = beta[q] / gamma;
        const double phi = cs[q] * phibar[q];
        phibar[q] = sn[q] * phibar[q];
        cf[q] = oldeps;
        cf[NR + q] = delta;
        cf[2 * NR + q] = 1.0 / gamma;
        cf[3 * NR + q] = phi;
      }
      // w1 <- w2, w2 <- w, w <- (v - oldeps w1 - delta w2) / gamma, dx += phi w
      std::swap(w1, w2);  // w1 <- old w2
      std::swap(w2, w);   // w2 <- old w; w (the old w1) is overwritten
      set_coef(cf, 4 * NR);
      k_lr_wx<<<ew_blocks(NR * L), 256, 0, s>>>(w, v, w1, w2, dx, coef, L);
      PP_LAUNCH_CHECK("k_lr_wx");
    }
    return it;
  }
};

}  // namespace

pp_status polarizability_impl(pp_ctx *c, int nfreq, const double *omega, double tol, int max_iter, double *alpha,
                              double *resid, int *iterations) {
  if (!c->has_mu) throw PPError(PP_EINVAL, "pp_polarizability: the context has no dipole integrals");
  Lr lr(c);
  cudaStream_t s = c->stream;
  const long long L = lr.L;
  k_lr_rhs<<<ew_blocks(NR * L), 256, 0, s>>>(lr.F, c->mu.as<double>(), c->ov);
  PP_LAUNCH_CHECK("k_lr_rhs");
  double fn[NR];
  lr.dot(lr.F, lr.F, fn);
  const bool mixed = c->opt.prec != PP_FP64;
  const int p_acc = mixed ? PP_BF16X3 : PP_FP64;
  pp_status st = PP_OK;
  for (int f = 0; f < nfreq; ++f) {
    const double w = omega[f];
    int its = 0;
    double rel = 0.0;
    if (!mixed) {
      its = lr.minres(lr.F, lr.x, w, PP_FP64, tol, max_iter);
    } else {
      PP_CUDA(cudaMemsetAsync(lr.x, 0, sizeof(double) * NR * L, s));
      PP_CUDA(cudaMemcpyAsync(lr.r, lr.F, sizeof(double) * NR * L, cudaMemcpyDeviceToDevice, s));
      const double inner = std::max(tol, 1e-2);
      // the BF16 corrections contract the residual by about cond(K) x (BF16 operator error);
      // near a root that factor approaches 1, and the corrections switch to the split form
      // (the operator of the residual itself) once an outer step gains less than 4x
      int p_inner = PP_BF16, stalls = 0;
      double rel_prev = 0.0;
      for (int outer = 0; outer < 20 && its < max_iter; ++outer) {
        if (outer > 0) {  // r = F - K x with the split sigma
          lr.apply(lr.x, lr.r, w, p_acc);
          const double cf[2 * NR] = {1, 1, 1, -1, -1, -1};
          lr.set_coef(cf, 2 * NR);
          k_lr_axpby<<<ew_blocks(NR * L), 256, 0, s>>>(lr.r, lr.F, lr.coef, L);  // r = F - K x
          PP_LAUNCH_CHECK("k_lr_axpby");
        }
        double rn[NR];
        lr.dot(lr.r, lr.r, rn);
        rel = 0.0;
        for (int q = 0; q < NR; ++q) rel = std::max(rel, std::sqrt(rn[q] / std::max(fn[q], 1e-300)));
        if (rel <= tol) break;
        if (outer > 0 && rel > 0.25 * rel_prev) {
          // the split-form corrections stall too once the residual reaches the noise of the
          // split products (their rounding is not linear in x), amplified by |x| / |F|
          if (p_inner == p_acc && ++stalls >= 2) break;
          p_inner = p_acc;
        }
        rel_prev = rel;
        its += lr.minres(lr.r, lr.d, w, p_inner, inner, max_iter - its);
        const double cf[2 * NR] = {1, 1, 1, 1, 1, 1};
        lr.set_coef(cf, 2 * NR);
        k_lr_axpby<<<ew_blocks(NR * L), 256, 0, s>>>(lr.x, lr.d, lr.coef, L);  // x += d
        PP_LAUNCH_CHECK("k_lr_axpby");
      }
    }
    // final residual with the accurate operator, and alpha = F^T x
    lr.apply(lr.x, lr.r, w, p_acc);
    const double cf[2 * NR] = {1, 1, 1, -1, -1, -1};
    lr.set_coef(cf, 2 * NR);
    k_lr_axpby<<<ew_blocks(NR * L), 256, 0, s>>>(lr.r, lr.F, lr.coef, L);
    PP_LAUNCH_CHECK("k_lr_axpby");
    double rn[NR];
    lr.dot(lr.r, lr.r, rn);
    rel = 0.0;
    for (int q = 0; q < NR; ++q) rel = std::max(rel, std::sqrt(rn[q] / std::max(fn[q], 1e-300)));
    for (int a = 0; a < NR; ++a) {
      // alpha[a][b] = F_a . x_b for every b: shift F_a against the three x blocks
      for (int b = 0; b < NR; ++b) {
        double h = 0.0;
        double *tmp = lr.dots + 8;
        k_lr_dot<<<1, 256, 0, s>>>(lr.F + a * L, lr.x + b * L, L, tmp);
        PP_LAUNCH_CHECK("k_lr_dot");
        PP_CUDA(cudaMemcpyAsync(&h, tmp, sizeof(double), cudaMemcpyDeviceToHost, s));
        PP_CUDA(cudaStreamSynchronize(s));
        alpha[(size_t)f * 9 + a * 3 + b] = h;
      }
    }
    if (resid) resid[f] = rel;
    if (iterations) iterations[f] = its;
    if (!(rel <= std::max(tol, 1e-14) * 10.0)) st = PP_ENOTCONV;
  }
  return st;
}
