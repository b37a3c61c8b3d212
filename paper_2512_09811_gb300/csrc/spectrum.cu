// Absorption spectrum of a frequency range (declared in include/pp.h as pp_spectrum).
//
// The roots inside [w_lo, w_hi] are found with the window solver of Sec. 2.5: the range is
// cut into nwin windows that are solved together, up to 16 at a time (all their trial
// vectors share each sigma batch); a window that returns kmax roots may hold more, so it is
// halved and its halves solved again.  Roots found twice -- on the shared edge of two windows -- are kept once.
// The spectrum is the Lorentzian-broadened sum of their oscillator strengths (Sec. 3; the
// pole sum of Eq. (pp_adc) at w + i eta, -Im / pi):
//   S(w) = sum_n f_n (eta / pi) / ((w - omega_n)^2 + eta^2),
// evaluated on the caller's frequency grid by k_spectrum.
#include "pp_internal.h"

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace {

// one thread per grid point (grid-stride), FP64 sums over the roots
__global__ void k_spectrum(const double *__restrict__ grid, int ngrid, const double *__restrict__ omega,
                           const double *__restrict__ f, int n, double eta, double *__restrict__ out) {
  const double c = eta / 3.14159265358979323846;
  const double e2 = eta * eta;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ngrid; g += gridDim.x * blockDim.x) {
    const double w = grid[g];
    double s = 0.0;
    for (int k = 0; k < n; ++k) {
      const double x = w - omega[k];
      s += f[k] * c / (x * x + e2);
    }
    out[g] = s;
  }
}

struct Root {
  double omega, osc, resid;
};

}  // namespace

pp_status spectrum_impl(pp_ctx *c, double w_lo, double w_hi, int nwin, int kmax, double eta, int ngrid,
                        const double *grid, double *spec, int cap, double *omega, double *osc, double *resid,
                        int *nroots) {
  struct Win {
    double a, b;
    int depth;
  };
  constexpr int kMaxDepth = 8;
  std::vector<Win> todo;
  const double width = (w_hi - w_lo) / nwin;
  for (int w = 0; w < nwin; ++w) todo.push_back({w_lo + w * width, (w + 1 == nwin) ? w_hi : w_lo + (w + 1) * width, 0});
  std::vector<Root> roots;
  pp_status worst = PP_OK;
  const int sel0 = c->opt.select;
  c->opt.select = 0;  // the k lowest roots of each window
  try {
    constexpr int kGroup = 16;  // windows solved together (each holds a Krylov basis)
    while (!todo.empty()) {
      std::vector<Win> rest;
      if ((int)todo.size() > kGroup) {
        rest.assign(todo.begin() + kGroup, todo.end());
        todo.resize(kGroup);
      }
      const int nw = (int)todo.size();
      std::vector<double> w0(nw), dw(nw), om((size_t)nw * kmax), of((size_t)nw * kmax), rs((size_t)nw * kmax);
      std::vector<int> kk(nw, kmax), nf(nw, 0);
      for (int w = 0; w < nw; ++w) {
        w0[w] = todo[w].a;
        dw[w] = todo[w].b - todo[w].a;
      }
      pp_status st = solve_windows_impl(c, nw, w0.data(), dw.data(), kk.data(), om.data(), of.data(), rs.data(),
                                        nullptr, nf.data());
      if (st != PP_OK) worst = st;
      std::vector<Win> next;
      for (int w = 0; w < nw; ++w) {
        if (nf[w] >= kmax && todo[w].depth < kMaxDepth) {  // the window may hold more roots
          const double mid = 0.5 * (todo[w].a + todo[w].b);
          next.push_back({todo[w].a, mid, todo[w].depth + 1});
          next.push_back({mid, todo[w].b, todo[w].depth + 1});
          continue;
        }
        for (int t = 0; t < nf[w]; ++t)
          roots.push_back({om[(size_t)w * kmax + t], of[(size_t)w * kmax + t], rs[(size_t)w * kmax + t]});
      }
      next.insert(next.end(), rest.begin(), rest.end());
      todo.swap(next);
    }
  } catch (...) {
    c->opt.select = sel0;
    throw;
  }
  c->opt.select = sel0;
  // a root on the edge shared by two windows is found by both: keep the better one
  std::sort(roots.begin(), roots.end(), [](const Root &x, const Root &y) { return x.omega < y.omega; });
  const double same = std::max(2.0 * c->opt.res_tol, 1e-12);
  std::vector<Root> uniq;
  for (const Root &r : roots) {
    if (!uniq.empty() && r.omega - uniq.back().omega <= same) {
      if (r.resid < uniq.back().resid) uniq.back() = r;
      continue;
    }
    uniq.push_back(r);
  }
  const int n = (int)uniq.size();
  *nroots = n;
  if (n > cap) {
    c->err = "pp_spectrum: " + std::to_string(n) + " roots in the range exceed cap = " + std::to_string(cap);
    return PP_EINVAL;
  }
  for (int t = 0; t < n; ++t) {
    omega[t] = uniq[t].omega;
    osc[t] = uniq[t].osc;
    resid[t] = uniq[t].resid;
  }
  if (ngrid > 0) {
    cudaStream_t s = c->stream;
    DevBuf d;
    d.ensure(sizeof(double) * ((size_t)2 * ngrid + 2 * (size_t)std::max(n, 1)));
    double *dg = d.as<double>(), *ds = dg + ngrid, *dw = ds + ngrid, *df = dw + std::max(n, 1);
    PP_CUDA(cudaMemcpyAsync(dg, grid, sizeof(double) * ngrid, cudaMemcpyHostToDevice, s));
    if (n > 0) {
      PP_CUDA(cudaMemcpyAsync(dw, omega, sizeof(double) * n, cudaMemcpyHostToDevice, s));
      PP_CUDA(cudaMemcpyAsync(df, osc, sizeof(double) * n, cudaMemcpyHostToDevice, s));
    }
    const int nb = std::max(1, std::min((ngrid + 255) / 256, 152 * 4));
    k_spectrum<<<nb, 256, 0, s>>>(dg, ngrid, dw, df, n, eta, ds);
    PP_LAUNCH_CHECK("k_spectrum");
    PP_CUDA(cudaMemcpyAsync(spec, ds, sizeof(double) * ngrid, cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
  }
  return worst;
}
