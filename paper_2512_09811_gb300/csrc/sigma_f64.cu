// Plain FP64 form of the matrix-free product sigma = M z (Sec. 2.2 matrix
// elements, density-fitted) and the per-dot second-order intermediates.
//
// With half-vectors V (an X or a Y block), the products are split as
//   A V = Delta*V + J(V) - KA(V) + A2(V)         B V = J(V) - KB(V) + B2(V)
//   J(V)_ia  = sum_Q B_Qia sum_jb B_Qjb V_jb                       ((ai|jb), (ai|bj))
//   KA(V)    = sum_Q Boo_Q V Bvv_Q                                  ((ab|ij))
//   KB(V)    = sum_Q Bov_Q V^T Bov_Q                                ((aj|bi))
//   A2(V)_ia = -1/2 [e_a (p_oo V) + q_oo V - e_i (V p_vv) + V q_vv]_ia
//   B2(V)    = -sum_Q [Bov_Q V^T Gam_Q + Gam_Q V^T Bov_Q] + sum_Q C_Q(T C_Q(V))
// where C_Q(V) = V Bvv_Q - Boo_Q V and T[(i,c),(j,d)] = t_ij^cd.  The last
// form gathers the particle and hole ladders and the (ki|bc)/(kj|ac) ring parts
// of Eq. (b(2)) into one contraction with the amplitudes; Gam carries the
// (kc|bi)/(kc|aj) ring parts.  sigma_X = A X + B Y and sigma_Y = B X + A Y.
#include "pp_internal.h"
#include "sigma_terms.cuh"

#include <algorithm>

namespace {

// weighted slab copies for the pair sums
// q_oo weight: row (k,d), column (j,c) -> e_k - e_d - e_c
__global__ void k_weight_oo(double *__restrict__ Tw, const double *__restrict__ T,
                            const double *__restrict__ eps, int o, int v, int i0, long long rows) {
  const long long ov = (long long)o * v;
  const long long total = rows * ov;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    long long rho = p / ov, col = p % ov;
    int k = i0 + (int)(rho / v), d = (int)(rho % v), c = (int)(col % v);
    Tw[p] = T[p] * (eps[k] - eps[o + d] - eps[o + c]);
  }
}
// q_vv weight: row (k,b), column (l,c) -> e_k + e_l - e_c
__global__ void k_weight_vv(double *__restrict__ Tw, const double *__restrict__ T,
                            const double *__restrict__ eps, int o, int v, int i0, long long rows) {
  const long long ov = (long long)o * v;
  const long long total = rows * ov;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    long long rho = p / ov, col = p % ov;
    int k = i0 + (int)(rho / v), l = (int)(col / v), c = (int)(col % v);
    Tw[p] = T[p] * (eps[k] + eps[l] - eps[o + c]);
  }
}

// resident-layout builders
__global__ void k_extract_blocks(const double *__restrict__ B, int n, int o, int v, int Q,
                                 double *__restrict__ Boo, double *__restrict__ Bov,
                                 double *__restrict__ Bvv) {
  const long long nn = (long long)n * n;
  const long long total = (long long)Q * nn;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    long long q = p / nn, rem = p % nn;
    int r = (int)(rem / n), s = (int)(rem % n);
    double x = B[p];
    if (r < o && s < o) Boo[(q * o + r) * o + s] = x;
    else if (r < o && s >= o) Bov[(q * o + r) * v + (s - o)] = x;
    else if (r >= o && s >= o) Bvv[(q * v + (r - o)) * v + (s - o)] = x;
  }
}
__global__ void k_extract_blocks_f32(const float *__restrict__ B, int n, int o, int v, int Q,
                                     double *__restrict__ Boo, double *__restrict__ Bov,
                                     double *__restrict__ Bvv) {
  const long long nn = (long long)n * n;
  const long long total = (long long)Q * nn;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    long long q = p / nn, rem = p % nn;
    int r = (int)(rem / n), s = (int)(rem % n);
    double x = (double)B[p];
    if (r < o && s < o) Boo[(q * o + r) * o + s] = x;
    else if (r < o && s >= o) Bov[(q * o + r) * v + (s - o)] = x;
    else if (r >= o && s >= o) Bvv[(q * v + (r - o)) * v + (s - o)] = x;
  }
}
__global__ void k_perm_bvv(const double *__restrict__ Bvv, double *__restrict__ BvvP, int v, int Q) {
  const long long total = (long long)Q * v * v;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    long long q = p / ((long long)v * v), rem = p % ((long long)v * v);
    long long b = rem / v, d = rem % v;
    BvvP[(b * Q + q) * v + d] = Bvv[p];
  }
}
__global__ void k_perm_boo(const double *__restrict__ Boo, double *__restrict__ BooT, int o, int Q) {
  const long long total = (long long)Q * o * o;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    long long q = p / ((long long)o * o), rem = p % ((long long)o * o);
    long long i = rem / o, k = rem % o;
    BooT[(i * o + k) * Q + q] = Boo[p];
  }
}
__global__ void k_gap(const double *__restrict__ eps, double *__restrict__ gap, int o, int v) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < o * v) gap[p] = eps[o + p % v] - eps[p / v];
}
__global__ void k_make_gb(double *__restrict__ GB, const double *__restrict__ Bov,
                          const double *__restrict__ Gam, long long qov, int second) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < qov;
       p += (long long)gridDim.x * blockDim.x) {
    GB[p] = Bov[p] + (second ? Gam[p] : 0.0);
    GB[qov + p] = Bov[p];
  }
}
// diag(A), diag(S) (the Jacobi splitting of Sec. 2.5.2)
__global__ void k_diag(const double *__restrict__ eps, const double *__restrict__ Bov,
                       const double *__restrict__ Boo, const double *__restrict__ Bvv,
                       const double *__restrict__ p_oo, const double *__restrict__ q_oo,
                       const double *__restrict__ p_vv, const double *__restrict__ q_vv, int o,
                       int v, int Q, int order, double *__restrict__ dA, double *__restrict__ dS) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= o * v) return;
  int i = p / v, a = p % v;
  double ea = eps[o + a], ei = eps[i];
  double da = ea - ei, ds = 1.0;
  if (order >= 1) {
    double jj = 0.0, kk = 0.0;
    for (int q = 0; q < Q; ++q) {
      double b = Bov[((long long)q * o + i) * v + a];
      jj += b * b;
      kk += Bvv[((long long)q * v + a) * v + a] * Boo[((long long)q * o + i) * o + i];
    }
    da += jj - kk;
  }
  if (order >= 2) {
    double poo = p_oo[i * o + i], qoo = q_oo[i * o + i];
    double pvv = p_vv[(long long)a * v + a], qvv = q_vv[(long long)a * v + a];
    da += -0.5 * (ea * poo + qoo) - 0.5 * (qvv - ei * pvv);
    ds += -0.5 * poo - 0.5 * pvv;
  }
  dA[p] = da;
  dS[p] = ds;
}

using sigma_detail::ew_grid;

__global__ void k_copy_scale(double *y, const double *x, double a, long long n) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x)
    y[p] = a * x[p];
}

}  // namespace

void ew_copy_scale(double *y, const double *x, double a, long long n, cudaStream_t s) {
  k_copy_scale<<<ew_grid(n), 256, 0, s>>>(y, x, a, n);
  PP_LAUNCH_CHECK("k_copy_scale");
}

// ---------------------------------------------------------------------------
// residency + per-dot precompute
// ---------------------------------------------------------------------------
void build_residency(pp_ctx *c, const double *Bd, const float *Bf) {
  const int o = c->o, v = c->v, Q = c->Q, n = c->n;
  cudaStream_t s = c->stream;
  c->Boo.ensure(sizeof(double) * (size_t)Q * o * o);
  c->Bov.ensure(sizeof(double) * (size_t)Q * o * v);
  c->Bvv.ensure(sizeof(double) * (size_t)Q * v * v);
  long long total = (long long)Q * n * n;
  if (Bd)
    k_extract_blocks<<<ew_grid(total), 256, 0, s>>>(Bd, n, o, v, Q, c->Boo.as<double>(),
                                                    c->Bov.as<double>(), c->Bvv.as<double>());
  else
    k_extract_blocks_f32<<<ew_grid(total), 256, 0, s>>>(Bf, n, o, v, Q, c->Boo.as<double>(),
                                                        c->Bov.as<double>(), c->Bvv.as<double>());
  PP_LAUNCH_CHECK("k_extract_blocks");
  // the permuted copy of Bvv serves only the FP64 sigma: contexts of the mixed form build it at
  // their first FP64 sigma (it is as large as Bvv itself)
  if (c->opt.prec == PP_FP64) ensure_bvvp(c);
  c->BooT.ensure(sizeof(double) * (size_t)Q * o * o);
  k_perm_boo<<<ew_grid((long long)Q * o * o), 256, 0, s>>>(c->Boo.as<double>(), c->BooT.as<double>(), o, Q);
  c->gap.ensure(sizeof(double) * (size_t)o * v);
  k_gap<<<(o * v + 255) / 256, 256, 0, s>>>(c->eps.as<double>(), c->gap.as<double>(), o, v);
  PP_LAUNCH_CHECK("residency");
}

void ensure_bvvp(pp_ctx *c) {
  const long long total = (long long)c->Q * c->v * c->v;
  if (c->BvvP.bytes >= sizeof(double) * (size_t)std::max<long long>(total, 1)) return;
  c->BvvP.ensure(sizeof(double) * (size_t)std::max<long long>(total, 1));
  if (total > 0) {
    k_perm_bvv<<<ew_grid(total), 256, 0, c->stream>>>(c->Bvv.as<double>(), c->BvvP.as<double>(), c->v, c->Q);
    PP_LAUNCH_CHECK("k_perm_bvv");
  }
}

static void choose_chunks(pp_ctx *c) {
  const long long o = c->o, v = c->v, Q = c->Q, ov = c->ov;
  // FP64 workspace per half-vector: W, U, P (each Q*ov) + E/F (2Q*o^2) + 6 ov
  long long per_half = 3 * Q * ov + 2 * Q * o * o + 8 * ov + Q;
  long long budget = 6LL << 30;  // bytes
  long long R = budget / (8 * per_half);
  R = std::max<long long>(2, std::min<long long>(R, 64));
  R &= ~1LL;
  c->sig_chunk = (int)R;
  long long slab_bytes = 256LL << 20;
  long long si = slab_bytes / (8 * v * ov);
  c->slab_i = (int)std::max<long long>(1, std::min<long long>(si, o));
}

// chunk sizes, and the per-dot intermediates allocated and zeroed
void precompute_begin(pp_ctx *c) {
  const int o = c->o, v = c->v, Q = c->Q;
  const long long ov = c->ov;
  cudaStream_t s = c->stream;
  choose_chunks(c);
  c->p_oo.ensure(sizeof(double) * o * o);
  c->q_oo.ensure(sizeof(double) * o * o);
  c->p_vv.ensure(sizeof(double) * (size_t)v * v);
  c->q_vv.ensure(sizeof(double) * (size_t)v * v);
  c->Gam.ensure(sizeof(double) * (size_t)std::max<long long>(1, Q * ov));
  PP_CUDA(cudaMemsetAsync(c->p_oo.p, 0, sizeof(double) * o * o, s));
  PP_CUDA(cudaMemsetAsync(c->q_oo.p, 0, sizeof(double) * o * o, s));
  PP_CUDA(cudaMemsetAsync(c->p_vv.p, 0, sizeof(double) * (size_t)v * v, s));
  PP_CUDA(cudaMemsetAsync(c->q_vv.p, 0, sizeof(double) * (size_t)v * v, s));
  PP_CUDA(cudaMemsetAsync(c->Gam.p, 0, sizeof(double) * (size_t)std::max<long long>(1, Q * ov), s));
}

void precompute_f64(pp_ctx *c) {
  const int o = c->o, v = c->v, Q = c->Q;
  const long long ov = c->ov;
  cudaStream_t s = c->stream;
  precompute_begin(c);
  if (c->opt.order >= 2) {
    const int si = c->slab_i;
    c->w_T.ensure(sizeof(double) * (size_t)si * v * ov);
    c->w_Tw.ensure(sizeof(double) * (size_t)si * v * ov);
    double *T = c->w_T.as<double>(), *Tw = c->w_Tw.as<double>();
    for (int i0 = 0; i0 < o; i0 += si) {
      const int ni = std::min(si, o - i0);
      const long long rows = (long long)ni * v;
      tslab_f64(c->Bov.as<double>(), c->eps.as<double>(), o, v, Q, i0, ni, T, s);
      // p_oo[i][j] += sum_c sum_rho T[rho][(i,c)] T[rho][(j,c)]
      GemmF64 g;
      g.M = o; g.N = o; g.K = (int)rows; g.nred = v;
      g.A = T; g.a_m = v; g.a_k = ov; g.a_red = 1;
      g.B = T; g.b_k = ov; g.b_n = v; g.b_red = 1;
      g.C = c->p_oo.as<double>(); g.c_m = o; g.c_n = 1; g.beta = 1.0;
      gemm_f64(g, s);
      k_weight_oo<<<ew_grid(rows * ov), 256, 0, s>>>(Tw, T, c->eps.as<double>(), o, v, i0, rows);
      PP_LAUNCH_CHECK("k_weight_oo");
      g.B = Tw; g.C = c->q_oo.as<double>();
      gemm_f64(g, s);
      // p_vv[a][b] += sum_k sum_(l,c) T[(k,a)][(l,c)] T[(k,b)][(l,c)]
      GemmF64 h;
      h.M = v; h.N = v; h.K = (int)ov; h.nred = ni;
      h.A = T; h.a_m = ov; h.a_k = 1; h.a_red = (long long)v * ov;
      h.B = T; h.b_k = 1; h.b_n = ov; h.b_red = (long long)v * ov;
      h.C = c->p_vv.as<double>(); h.c_m = v; h.c_n = 1; h.beta = 1.0;
      gemm_f64(h, s);
      k_weight_vv<<<ew_grid(rows * ov), 256, 0, s>>>(Tw, T, c->eps.as<double>(), o, v, i0, rows);
      PP_LAUNCH_CHECK("k_weight_vv");
      h.B = Tw; h.C = c->q_vv.as<double>();
      gemm_f64(h, s);
      // Gam[Q][row0 + rho] = sum_p T[rho][p] Bov[Q][p]
      GemmF64 gg;
      gg.M = (int)rows; gg.N = Q; gg.K = (int)ov;
      gg.A = T; gg.a_m = ov; gg.a_k = 1;
      gg.B = c->Bov.as<double>(); gg.b_k = 1; gg.b_n = ov;
      gg.C = c->Gam.as<double>() + (long long)i0 * v; gg.c_m = 1; gg.c_n = ov;
      gemm_f64(gg, s);
    }
    c->w_Tw.release();
  }
  precompute_finish(c);
}

// Bov + Gamma stacked over Bov for the exchange-type ring terms, and the Jacobi diagonal
void precompute_finish(pp_ctx *c) {
  const int o = c->o, v = c->v, Q = c->Q;
  const long long ov = c->ov;
  cudaStream_t s = c->stream;
  c->GB.ensure(sizeof(double) * 2 * (size_t)Q * ov);
  k_make_gb<<<ew_grid((long long)Q * ov), 256, 0, s>>>(c->GB.as<double>(), c->Bov.as<double>(),
                                                       c->Gam.as<double>(), (long long)Q * ov,
                                                       c->opt.order >= 2);
  c->diagA.ensure(sizeof(double) * ov);
  c->diagS.ensure(sizeof(double) * ov);
  k_diag<<<(unsigned)((ov + 127) / 128), 128, 0, s>>>(
      c->eps.as<double>(), c->Bov.as<double>(), c->Boo.as<double>(), c->Bvv.as<double>(),
      c->p_oo.as<double>(), c->q_oo.as<double>(), c->p_vv.as<double>(), c->q_vv.as<double>(), o, v,
      Q, c->opt.order, c->diagA.as<double>(), c->diagS.as<double>());
  PP_LAUNCH_CHECK("k_diag");
}

// ---------------------------------------------------------------------------
// sigma, FP64 (plain form): the ladder contraction materialises FP64 amplitude
// slabs T[(i,c) for i in the slab][(j,d)] and multiplies them into P.
// ---------------------------------------------------------------------------
void sigma_f64(pp_ctx *c, int nvec, const double *Zd, double *sig_d, double *met_d) {
  const int o = c->o, v = c->v, Q = c->Q;
  const long long ov = c->ov;
  if (c->opt.order >= 1) ensure_bvvp(c);
  const int Rmax = c->sig_chunk;
  c->w_acc.ensure(sizeof(double) * 2 * (size_t)Rmax * ov);
  c->w_tmp.ensure(sizeof(double) * 4 * (size_t)Rmax * ov);
  if (c->opt.order >= 1) {
    c->w_cq.ensure(sizeof(double) * (size_t)Q * Rmax);
    c->w_W.ensure(sizeof(double) * (size_t)Rmax * o * Q * v);
    c->w_EF.ensure(sizeof(double) * (size_t)Rmax * 2 * Q * o * o);
  }
  if (c->opt.order >= 2) {
    c->w_U.ensure(sizeof(double) * (size_t)Rmax * Q * ov);
    c->w_P.ensure(sizeof(double) * (size_t)Rmax * Q * ov);
    c->w_T.ensure(sizeof(double) * (size_t)c->slab_i * v * ov);
  }
  SigmaRes<double> res{c->gap.as<double>(), c->eps.as<double>(), c->Bov.as<double>(),
                       c->Boo.as<double>(), c->Bvv.as<double>(), c->BvvP.as<double>(),
                       c->BooT.as<double>(), c->GB.as<double>(), c->Gam.as<double>(),
                       c->p_oo.as<double>(), c->q_oo.as<double>(), c->p_vv.as<double>(),
                       c->q_vv.as<double>()};
  const int R_total = 2 * nvec;
  for (int r0 = 0; r0 < R_total; r0 += Rmax) {
    const int R = std::min(Rmax, R_total - r0);
    SigmaWork<double> wk{c->w_acc.as<double>(), c->w_acc.as<double>() + (long long)R * ov,
                         c->w_tmp.as<double>(), c->w_cq.as<double>(), c->w_W.as<double>(),
                         c->w_U.as<double>(), c->w_EF.as<double>()};
    SigmaHooks<double> hk;
    hk.amplitude = [&](int Rc, const double *Cmat, double *Bacc) {
      const long long qov = (long long)Q * ov;
      double *T = c->w_T.as<double>();
      double *P = c->w_P.as<double>();
      const int si = c->slab_i;
      for (int i0 = 0; i0 < o; i0 += si) {
        const int ni = std::min(si, o - i0);
        const long long rows = (long long)ni * v;
        tslab_f64(c->Bov.as<double>(), c->eps.as<double>(), o, v, Q, i0, ni, T, c->stream);
        GemmF64 p2;  // P[r][(i,c)][Q] = sum_p T[(i,c)][p] Cmat[r][Q][p]
        p2.M = (int)rows; p2.N = Q; p2.K = (int)ov; p2.nbatch = Rc;
        p2.A = T; p2.a_m = ov; p2.a_k = 1;
        p2.B = Cmat; p2.b_k = 1; p2.b_n = ov; p2.b_batch = qov;
        p2.C = P + (long long)i0 * v * Q; p2.c_m = Q; p2.c_n = 1; p2.c_batch = qov;
        gemm_f64(p2, c->stream);
      }
      apply_cq_of_p<double>(c, Rc, P, qov, (long long)Q, res, Bacc);
    };
    const double *V = Zd + (long long)r0 * ov;
    sigma_chunk<double>(c, R, V, V, sig_d + (long long)r0 * ov,
                        met_d ? met_d + (long long)r0 * ov : nullptr, res, wk, hk);
  }
}
