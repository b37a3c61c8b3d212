// FP64 contraction kernels of the plain form: a generic strided GEMM with an
// inner reduction batch, and the MP2-amplitude slab generator.
//
// GB300 executes FP64 on the CUDA cores at a small fraction of its tensor
// rate, so these kernels are compute bound by design: 64x64 output tiles,
// 16-deep K steps staged in shared memory, 4x4 register blocking per thread.
#include "pp_internal.h"

#include <algorithm>

namespace {

constexpr int TM = 64, TN = 64, TK = 16, NT = 256;

template <class T>
__global__ void __launch_bounds__(NT) k_gemm(GemmS<T> g) {
  __shared__ T As[TK][TM + 1];
  __shared__ T Bs[TK][TN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const long long m0 = (long long)blockIdx.y * TM, n0 = (long long)blockIdx.x * TN;
  const long long b = blockIdx.z / g.ksplit;
  const int ks = blockIdx.z % g.ksplit;
  // this block's share of the reduction: a range of t (nred > 1) or of K (nred == 1)
  int t_lo = 0, t_hi = g.nred, k_lo = 0, k_hi = g.K;
  if (g.ksplit > 1) {
    if (g.nred > 1) {
      t_lo = (int)((long long)g.nred * ks / g.ksplit);
      t_hi = (int)((long long)g.nred * (ks + 1) / g.ksplit);
    } else {
      const int nk = (g.K + TK - 1) / TK;
      k_lo = (int)((long long)nk * ks / g.ksplit) * TK;
      k_hi = min(g.K, (int)((long long)nk * (ks + 1) / g.ksplit) * TK);
    }
  }
  const T *A = g.A + b * g.a_batch;
  const T *B = g.B + b * g.b_batch;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  const bool a_mfast = (g.a_m == 1);
  const bool b_nfast = (g.b_n == 1);
  for (int t = t_lo; t < t_hi; ++t) {
    const T *At = A + (long long)t * g.a_red;
    const T *Bt = B + (long long)t * g.b_red;
    for (int k0 = k_lo; k0 < k_hi; k0 += TK) {
#pragma unroll
      for (int e = 0; e < (TK * TM) / NT; ++e) {
        int idx = tid + e * NT;
        int kk, mm;
        if (a_mfast) {
          mm = idx % TM;
          kk = idx / TM;
        } else {
          kk = idx % TK;
          mm = idx / TK;
        }
        long long gm = m0 + mm;
        int gk = k0 + kk;
        As[kk][mm] = (gm < g.M && gk < k_hi) ? At[gm * g.a_m + (long long)gk * g.a_k] : T(0);
      }
#pragma unroll
      for (int e = 0; e < (TK * TN) / NT; ++e) {
        int idx = tid + e * NT;
        int kk, nn;
        if (b_nfast) {
          nn = idx % TN;
          kk = idx / TN;
        } else {
          kk = idx % TK;
          nn = idx / TK;
        }
        long long gn = n0 + nn;
        int gk = k0 + kk;
        Bs[kk][nn] = (gn < g.N && gk < k_hi) ? Bt[(long long)gk * g.b_k + gn * g.b_n] : T(0);
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < TK; ++kk) {
        T a[4], bb[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx * 4 + j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
  T *C = g.C + b * g.c_batch;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    long long gm = m0 + ty * 4 + i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      long long gn = n0 + tx * 4 + j;
      if (gn >= g.N) continue;
      T *cp = C + gm * g.c_m + gn * g.c_n;
      if (g.ksplit > 1) {
        atomicAdd(cp, g.alpha * acc[i][j]);
        continue;
      }
      T val = g.alpha * acc[i][j];
      if (g.beta != T(0)) val += g.beta * (*cp);
      *cp = val;
    }
  }
}

// t_ij^cd for a slab of occupied i: two accumulators (direct and exchange)
__global__ void __launch_bounds__(NT) k_tslab_f64(const double *__restrict__ Bov,
                                                  const double *__restrict__ eps, int o, int v,
                                                  int Q, int i0, double *__restrict__ T) {
  __shared__ double A1[TK][TM + 1], B1[TK][TN + 1], A2[TK][TM + 1], B2[TK][TN + 1];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int ii = blockIdx.z / o, j = blockIdx.z % o;
  const int i = i0 + ii;
  const int c0 = blockIdx.y * TM, d0 = blockIdx.x * TN;
  const long long ov = (long long)o * v;
  double acc1[4][4], acc2[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int bq = 0; bq < 4; ++bq) acc1[a][bq] = acc2[a][bq] = 0.0;
  for (int q0 = 0; q0 < Q; q0 += TK) {
#pragma unroll
    for (int e = 0; e < (TK * TM) / NT; ++e) {
      int idx = tid + e * NT;
      int mm = idx % TM, kk = idx / TM;
      int q = q0 + kk;
      bool okq = q < Q;
      int c = c0 + mm, d = d0 + mm;
      const double *row = Bov + (long long)q * ov;
      A1[kk][mm] = (okq && c < v) ? row[(long long)i * v + c] : 0.0;
      A2[kk][mm] = (okq && c < v) ? row[(long long)j * v + c] : 0.0;
      B1[kk][mm] = (okq && d < v) ? row[(long long)j * v + d] : 0.0;
      B2[kk][mm] = (okq && d < v) ? row[(long long)i * v + d] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      double a1[4], a2[4], b1[4], b2[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        a1[r] = A1[kk][ty * 4 + r];
        a2[r] = A2[kk][ty * 4 + r];
        b1[r] = B1[kk][tx * 4 + r];
        b2[r] = B2[kk][tx * 4 + r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          acc1[r][s] = fma(a1[r], b1[s], acc1[r][s]);
          acc2[r][s] = fma(a2[r], b2[s], acc2[r][s]);
        }
    }
    __syncthreads();
  }
  const double eij = eps[i] + eps[j];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    int c = c0 + ty * 4 + r;
    if (c >= v) continue;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      int d = d0 + tx * 4 + s;
      if (d >= v) continue;
      double den = eij - eps[o + c] - eps[o + d];
      T[((long long)ii * v + c) * ov + (long long)j * v + d] = (acc1[r][s] - acc2[r][s]) / den;
    }
  }
}

}  // namespace

template <class T> static void gemm_launch(const GemmS<T> &g, cudaStream_t s, const char *name) {
  if (g.M <= 0 || g.N <= 0 || g.nbatch <= 0) return;
  if (g.ksplit > 1 && g.beta != T(1)) throw PPError(PP_EINVAL, std::string(name) + ": ksplit needs beta = 1");
  dim3 grid((g.N + TN - 1) / TN, (g.M + TM - 1) / TM, g.nbatch * std::max(1, g.ksplit));
  if (grid.y > 65535 || grid.z > 65535) throw PPError(PP_EINVAL, std::string(name) + ": grid too large");
  k_gemm<T><<<grid, NT, 0, s>>>(g);
  PP_LAUNCH_CHECK(name);
}
void gemm_f64(const GemmF64 &g, cudaStream_t s) { gemm_launch(g, s, "k_gemm_f64"); }
void gemm_f64_preload() {
  cudaFuncAttributes fa;
  PP_CUDA(cudaFuncGetAttributes(&fa, k_gemm<double>));
}
void gemm_f32(const GemmF32 &g, cudaStream_t s) { gemm_launch(g, s, "k_gemm_f32"); }

void tslab_f64(const double *Bov, const double *eps, int o, int v, int Q, int i0, int ni, double *T,
               cudaStream_t s) {
  dim3 grid((v + TN - 1) / TN, (v + TM - 1) / TM, ni * o);
  k_tslab_f64<<<grid, NT, 0, s>>>(Bov, eps, o, v, Q, i0, T);
  PP_LAUNCH_CHECK("k_tslab_f64");
}
