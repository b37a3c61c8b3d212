// Shared sigma pipeline, templated on the scalar type of the small contractions
// (double for the plain FP64 form, float for the tensor-core form).  The
// ladder/ring contraction with the MP2 amplitudes is supplied by the caller.
//
// For half-vectors V (X or Y blocks):
//   A V = Delta*V + J(V) - KA(V) + A2(V)         B V = J(V) - KB(V) + B2(V)
//   J(V)_ia  = sum_Q B_Qia sum_jb B_Qjb V_jb                       ((ai|jb), (ai|bj))
//   KA(V)    = sum_Q Boo_Q V Bvv_Q                                  ((ab|ij))
//   KB(V)    = sum_Q Bov_Q V^T Bov_Q                                ((aj|bi))
//   A2(V)_ia = -1/2 [e_a (p_oo V) + q_oo V - e_i (V p_vv) + V q_vv]_ia
//   B2(V)    = -sum_Q [Bov_Q V^T Gam_Q + Gam_Q V^T Bov_Q] + sum_Q C_Q(P_Q),
//   P_Q      = T C_Q(V),  C_Q(V) = V Bvv_Q - Boo_Q V,  T[(i,c),(j,d)] = t_ij^cd.
// The last form gathers the particle and hole ladders and the (ki|bc)/(kj|ac)
// ring parts of Eq. (b(2)) into one contraction with the amplitudes; Gam carries
// the (kc|bi)/(kc|aj) ring parts.  sigma_X = A X + B Y, sigma_Y = B X + A Y; in the
// Tamm-Dancoff form (B = 0) sigma_X = A X, sigma_Y = A Y and no B term is formed.
#pragma once
#include <functional>

#include "pp_internal.h"

template <class T> struct SigmaRes {
  const T *gap, *eps, *Bov, *Boo, *Bvv, *BvvP, *BooT, *GB, *Gam, *p_oo, *q_oo, *p_vv, *q_vv;
};
template <class T> struct SigmaWork {
  T *Aacc, *Bacc, *tmp, *cq, *W, *U, *EF;  // sized for R half-vectors
};
// Backend hooks for the large contractions.  w / ef return false to fall back to the
// strided SIMT GEMMs; amplitude(R, Cmat, Bacc) must add sum_Q C_Q(T C_Q(V)) into Bacc.
template <class T> struct SigmaHooks {
  std::function<bool(int R, const T *V, T *W)> w;                 // W[r][j][Q][d] = (V_r Bvv_Q)[j][d]
  std::function<bool(int R, const T *V, T *EF, bool second)> ef;  // E (and F) into EF[r][t][i][j]
  // Cmat == nullptr: C_Q(V) was already formed by first_order in the amplitude hook's own layout
  std::function<void(int R, const T *Cmat, T *Bacc)> amplitude;
  // the whole first-order block (W, KA, E/F, KB and, at second order, C_Q(V)) in one go;
  // returns false to fall back to the step-by-step contractions below
  std::function<bool(int R, T *Aacc, T *Bacc)> first_order;
};

namespace sigma_detail {

inline dim3 ew_grid(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return dim3((unsigned)b);
}

template <class T>
__global__ void k_gap_scale(T *__restrict__ out, const T *__restrict__ gap, const T *__restrict__ V,
                            long long ov, long long total) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x)
    out[p] = gap[p % ov] * V[p];
}
// acc += x
template <class T>
__global__ void k_add(T *__restrict__ acc, const T *__restrict__ x, long long total) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x)
    acc[p] += x[p];
}
// U[r][Q][j][d] <- W[r][j][Q][d] - U[r][Q][j][d]
template <class T>
__global__ void k_cmat(T *__restrict__ U, const T *__restrict__ W, int o, int v, int Q, long long total) {
  const long long qov = (long long)Q * o * v;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    long long r = p / qov, rem = p % qov;
    long long q = rem / ((long long)o * v);
    long long jd = rem % ((long long)o * v);
    long long j = jd / v, d = jd % v;
    U[p] = W[r * qov + (j * Q + q) * v + d] - U[p];
  }
}
template <class T>
__global__ void k_a2(T *__restrict__ acc, const T *__restrict__ t1, const T *__restrict__ t2,
                     const T *__restrict__ t3, const T *__restrict__ t4, const T *__restrict__ eps,
                     int o, int v, long long total) {
  const long long ov = (long long)o * v;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    long long ia = p % ov;
    int i = (int)(ia / v), a = (int)(ia % v);
    acc[p] += T(-0.5) * (eps[o + a] * t1[p] + t2[p] - eps[i] * t3[p] + t4[p]);
  }
}
// metric, written in double: S V = V - t1/2 - t3/2 (rho_oo = -p_oo/2, rho_vv = p_vv/2)
template <class T>
__global__ void k_metric(double *__restrict__ met, const double *__restrict__ V,
                         const T *__restrict__ t1, const T *__restrict__ t3, int second,
                         long long ov, long long total) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    long long r = p / ov;
    double s = (r & 1) ? -1.0 : 1.0;
    double val = V[p];
    if (second) val += -0.5 * (double)t1[p] - 0.5 * (double)t3[p];
    met[p] = s * val;
  }
}
// sigma[s][0] = Aacc[2s] + Bacc[2s+1];  sigma[s][1] = Bacc[2s] + Aacc[2s+1]
// (gap64 set: the diagonal term gap * V is added here in FP64 instead of living in Aacc;
// Bacc null: the Tamm-Dancoff form, sigma = (A X, A Y))
template <class T>
__global__ void k_combine(double *__restrict__ sig, const T *__restrict__ Aacc,
                          const T *__restrict__ Bacc, const double *__restrict__ gap64,
                          const double *__restrict__ V64, long long ov, long long total) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    long long r = p / ov, e = p % ov;
    double x = (double)Aacc[p] + (Bacc ? (double)Bacc[(r ^ 1) * ov + e] : 0.0);
    if (gap64) x += gap64[e] * V64[p];
    sig[p] = x;
  }
}
// FP32 sums may be split across blocks (atomic, order-dependent rounding); FP64 stays deterministic
template <class T> constexpr bool split_k() { return sizeof(T) == 4; }
template <class T> inline void gemm(const GemmS<T> &g, cudaStream_t s);
template <> inline void gemm<double>(const GemmS<double> &g, cudaStream_t s) { gemm_f64(g, s); }
template <> inline void gemm<float>(const GemmS<float> &g, cudaStream_t s) { gemm_f32(g, s); }

}  // namespace sigma_detail

// One chunk of R half-vectors V (type T, device), outputs in double.
template <class T>
void sigma_chunk(const pp_ctx *c, int R, const T *V, const double *V64, double *sig, double *met,
                 const SigmaRes<T> &res, const SigmaWork<T> &wk, const SigmaHooks<T> &hk) {
  using namespace sigma_detail;
  const int o = c->o, v = c->v, Q = c->Q, order = c->opt.order;
  const bool tda = c->opt.tda != 0;  // Tamm-Dancoff form: no B terms
  const long long ov = c->ov;
  cudaStream_t s = c->stream;
  T *Aacc = wk.Aacc, *Bacc = wk.Bacc;
  T *t1 = wk.tmp, *t2 = wk.tmp + (long long)R * ov, *t3 = wk.tmp + 2LL * R * ov, *t4 = wk.tmp + 3LL * R * ov;
  const long long tot = (long long)R * ov;
  // reduced precision: the dominant diagonal term gap * V is added in FP64 by k_combine
  const bool diag64 = sizeof(T) < sizeof(double);
  if (diag64) {
    PP_CUDA(cudaMemsetAsync(Aacc, 0, sizeof(T) * tot, s));
  } else {
    k_gap_scale<T><<<ew_grid(tot), 256, 0, s>>>(Aacc, res.gap, V, ov, tot);
    PP_LAUNCH_CHECK("k_gap_scale");
  }
  PP_CUDA(cudaMemsetAsync(Bacc, 0, sizeof(T) * tot, s));
  if (order >= 1) {
    T *cq = wk.cq;
    GemmS<T> g;  // cq[Q][r] = sum_p Bov[Q][p] V[r][p]
    g.M = Q; g.N = R; g.K = (int)ov;
    g.A = res.Bov; g.a_m = ov; g.a_k = 1;
    g.B = V; g.b_k = 1; g.b_n = ov;
    g.C = cq; g.c_m = R; g.c_n = 1;
    if (split_k<T>()) {  // few output tiles, long K: split K across blocks
      PP_CUDA(cudaMemsetAsync(cq, 0, sizeof(T) * (size_t)Q * R, s));
      g.beta = T(1);
      g.ksplit = 32;
    }
    gemm<T>(g, s);
    GemmS<T> j;  // J, the same term in both accumulators: formed once in Bacc (still zero),
    j.M = R; j.N = (int)ov; j.K = Q;  // then added to Aacc
    j.A = cq; j.a_m = 1; j.a_k = R;
    j.B = res.Bov; j.b_k = ov; j.b_n = 1;
    j.C = Bacc; j.c_m = ov; j.c_n = 1; j.beta = T(1);
    gemm<T>(j, s);
    k_add<T><<<ew_grid(tot), 256, 0, s>>>(Aacc, Bacc, tot);
    PP_LAUNCH_CHECK("k_add");
    if (hk.first_order && hk.first_order(R, Aacc, Bacc)) {
      if (order >= 2 && !tda) hk.amplitude(R, nullptr, Bacc);
    } else {
      if (!res.Boo || !res.Bvv || !res.BvvP || !res.GB || !res.Gam)
        throw PPError(PP_ECUDA, "sigma: step-by-step contractions need operands this form does not keep");
      T *W = wk.W;  // W[r][j][Q][d] = V_r BvvP
      const long long oQv = (long long)o * Q * v;
      if (!(hk.w && hk.w(R, V, W))) {
        GemmS<T> w;
        w.M = o; w.N = Q * v; w.K = v; w.nbatch = R;
        w.A = V; w.a_m = v; w.a_k = 1; w.a_batch = ov;
        w.B = res.BvvP; w.b_k = (long long)Q * v; w.b_n = 1;
        w.C = W; w.c_m = (long long)Q * v; w.c_n = 1; w.c_batch = oQv;
        gemm<T>(w, s);
      }
      GemmS<T> ka;  // KA: Aacc -= sum_Q sum_k Boo[Q][i][k] W[r][k][Q][a]
      ka.M = o; ka.N = v; ka.K = o; ka.nred = Q; ka.nbatch = R;
      ka.A = res.Boo; ka.a_m = o; ka.a_k = 1; ka.a_red = (long long)o * o;
      ka.B = W; ka.b_k = (long long)Q * v; ka.b_n = 1; ka.b_red = v; ka.b_batch = oQv;
      ka.C = Aacc; ka.c_m = v; ka.c_n = 1; ka.c_batch = ov; ka.alpha = T(-1); ka.beta = T(1);
      if (split_k<T>()) ka.ksplit = 16;
      gemm<T>(ka, s);
      if (!tda) {
      T *EF = wk.EF;  // E[r][Q][i][j] = sum_b Bov[Q][i][b] V[r][j][b]; F likewise with Gam
      const long long efb = 2LL * Q * o * o;
      if (!(hk.ef && hk.ef(R, V, EF, order >= 2))) {
        GemmS<T> e;
        e.M = Q * o; e.N = o; e.K = v; e.nbatch = R;
        e.A = res.Bov; e.a_m = v; e.a_k = 1;
        e.B = V; e.b_k = 1; e.b_n = v; e.b_batch = ov;
        e.C = EF; e.c_m = o; e.c_n = 1; e.c_batch = efb;
        gemm<T>(e, s);
        if (order >= 2) {
          e.A = res.Gam;
          e.C = EF + (long long)Q * o * o;
          gemm<T>(e, s);
        }
      }
      GemmS<T> kb;  // Bacc -= sum_t sum_j EF[r][t][i][j] GB[t][j][a]
      kb.M = o; kb.N = v; kb.K = o; kb.nbatch = R;
      kb.A = EF; kb.a_m = o; kb.a_k = 1; kb.a_red = (long long)o * o; kb.a_batch = efb;
      kb.b_k = v; kb.b_n = 1; kb.b_red = ov;
      kb.C = Bacc; kb.c_m = v; kb.c_n = 1; kb.c_batch = ov; kb.alpha = T(-1); kb.beta = T(1);
      if (order >= 2) {
        kb.nred = 2 * Q;
        kb.B = res.GB;
      } else {
        kb.nred = Q;
        kb.B = res.Bov;
      }
      if (split_k<T>()) kb.ksplit = 16;
      gemm<T>(kb, s);
      if (order >= 2) {
        T *U = wk.U;  // U[r][Q][l][b] = Boo_Q V_r, then C_Q(V) = W - U in place
        const long long qov = (long long)Q * ov;
        GemmS<T> u;
        u.M = Q * o; u.N = v; u.K = o; u.nbatch = R;
        u.A = res.Boo; u.a_m = o; u.a_k = 1;
        u.B = V; u.b_k = v; u.b_n = 1; u.b_batch = ov;
        u.C = U; u.c_m = v; u.c_n = 1; u.c_batch = qov;
        gemm<T>(u, s);
        k_cmat<T><<<ew_grid(R * qov), 256, 0, s>>>(U, W, o, v, Q, R * qov);
        PP_LAUNCH_CHECK("k_cmat");
        hk.amplitude(R, (const T *)U, Bacc);
      }
      }  // !tda
    }
  }
  if (order >= 2) {
    GemmS<T> a;  // t1 = p_oo V, t2 = q_oo V
    a.M = o; a.N = v; a.K = o; a.nbatch = R;
    a.A = res.p_oo; a.a_m = o; a.a_k = 1;
    a.B = V; a.b_k = v; a.b_n = 1; a.b_batch = ov;
    a.C = t1; a.c_m = v; a.c_n = 1; a.c_batch = ov;
    gemm<T>(a, s);
    a.A = res.q_oo; a.C = t2;
    gemm<T>(a, s);
    GemmS<T> b;  // t3 = V p_vv, t4 = V q_vv
    b.M = o; b.N = v; b.K = v; b.nbatch = R;
    b.A = V; b.a_m = v; b.a_k = 1; b.a_batch = ov;
    b.B = res.p_vv; b.b_k = v; b.b_n = 1;
    b.C = t3; b.c_m = v; b.c_n = 1; b.c_batch = ov;
    gemm<T>(b, s);
    b.B = res.q_vv; b.C = t4;
    gemm<T>(b, s);
    k_a2<T><<<ew_grid(tot), 256, 0, s>>>(Aacc, t1, t2, t3, t4, res.eps, o, v, tot);
    PP_LAUNCH_CHECK("k_a2");
  }
  k_combine<T><<<ew_grid(tot), 256, 0, s>>>(sig, Aacc, tda ? nullptr : Bacc, diag64 ? c->gap.as<double>() : nullptr,
                                            V64, ov, tot);
  PP_LAUNCH_CHECK("k_combine");
  if (met) {
    k_metric<T><<<ew_grid(tot), 256, 0, s>>>(met, V64, t1, t3, order >= 2, ov, tot);
    PP_LAUNCH_CHECK("k_metric");
  }
}

// Bacc += sum_Q C_Q(P_Q) = sum_Q (P_Q Bvv_Q - Boo_Q P_Q) for P with element (r, i, c, Q) at
// r*p_r + (i*v + c)*p_ic + Q (strided SIMT GEMMs)
template <class T>
void apply_cq_of_p(const pp_ctx *c, int R, const T *P, long long p_r, long long p_ic, const SigmaRes<T> &res,
                   T *Bacc) {
  using namespace sigma_detail;
  const int o = c->o, v = c->v, Q = c->Q;
  const long long ov = c->ov;
  GemmS<T> f1;  // Bacc += sum_c sum_Q P[r][i][c][Q] Bvv[Q][c][a]
  f1.M = o; f1.N = v; f1.K = Q; f1.nred = v; f1.nbatch = R;
  f1.A = P; f1.a_m = v * p_ic; f1.a_k = 1; f1.a_red = p_ic; f1.a_batch = p_r;
  f1.B = res.Bvv; f1.b_k = (long long)v * v; f1.b_n = 1; f1.b_red = v;
  f1.C = Bacc; f1.c_m = v; f1.c_n = 1; f1.c_batch = ov; f1.beta = T(1);
  gemm<T>(f1, c->stream);
  GemmS<T> f2;  // Bacc -= sum_k sum_Q BooT[i][k][Q] P[r][k][a][Q]
  f2.M = o; f2.N = v; f2.K = Q; f2.nred = o; f2.nbatch = R;
  f2.A = res.BooT; f2.a_m = (long long)o * Q; f2.a_k = 1; f2.a_red = Q;
  f2.B = P; f2.b_k = 1; f2.b_n = p_ic; f2.b_red = v * p_ic; f2.b_batch = p_r;
  f2.C = Bacc; f2.c_m = v; f2.c_n = 1; f2.c_batch = ov; f2.alpha = T(-1); f2.beta = T(1);
  gemm<T>(f2, c->stream);
}
