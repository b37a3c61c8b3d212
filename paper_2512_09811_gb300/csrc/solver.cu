// Interior-root window solver of Sec. 2.5.
//
// For each window the solver keeps an orthonormal basis V (FP64) together
// with M V and Sigma V.  Each outer iteration
//   1. Rayleigh-Ritz on the projected pencil (V^T M V, V^T Sigma V): M is
//      positive definite for a stable RPA problem, so V^T M V = L L^T and the
//      symmetric matrix L^-1 V^T Sigma V L^-T is diagonalised (parallel cyclic
//      Jacobi); the Ritz values theta = 1/mu nearest the window shift become
//      the targets;
//   2. for each target, in order, the folded-spectrum vector of Sec. 2.5:
//        y = argmin <y|(M - w Sigma)^2|y> / <y|y>  over y in span(V),
//      with the fold centre w set to the Rayleigh quotient of y (four updates,
//      three inverse-iteration solves each), and y
//      kept Sigma-orthogonal to the earlier targets (a penalty on the
//      constraint directions).  With w equal to a root the minimum is the null
//      vector of Sec. 2.5; with S != 1 a fixed w would not converge to an
//      eigenvector, so the centre follows the Ritz value;
//   3. residuals r = M y - theta Sigma y; for unconverged targets the
//      inverse-Krylov direction is one weighted-Jacobi sweep (Sec. 2.5.2, the
//      splitting M - theta Sigma = D + F) on the correction equation
//      (M - theta Sigma) t = -r from t = 0, i.e. t = -D^-1 r;
//   4. thick restart when the basis is full; the directions are orthonormalised
//      against V (block CGS2) and among themselves (Cholesky QR twice), and the
//      survivors of all windows are multiplied in one sigma batch per precision
//      phase.
// Windows live in the slots of a WindowBatch and advance one iteration per
// step(); a window may join or leave between steps (the serving loop uses that).
#include "pp_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>

namespace {

constexpr int MAXM = 112;  // largest subspace the shared-memory eigensolver takes

// one warp per output: the partials are summed lane-strided, then across the warp
__global__ void __launch_bounds__(256) k_gram_reduce(const double *__restrict__ part, int nblk, int p, int q,
                                                     double *__restrict__ G, int ldg, double alpha, double beta) {
  const int lane = threadIdx.x & 31;
  const int pr = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (pr >= p * q) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += part[(long long)b * p * q + pr];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) {
    int i = pr / q, j = pr % q;
    double *g = G + (long long)i * ldg + j;
    *g = alpha * s + (beta != 0.0 ? beta * (*g) : 0.0);
  }
}

// ---- double-FP32 arithmetic for the Krylov-space products --------------------------------
// FP64 issues at a small fraction of the FP32 rate on this part, and the Grams and linear
// combinations of the basis are long FP64 dot products, so they run in double-FP32: each FP64
// operand becomes an unevaluated sum hi + lo of two floats (48 significant bits), products are
// formed with the exact FMA residual of hi * hi plus the two cross terms, and sums are kept as
// float pairs with an error-free two-sum (error within about 5e-14 of the sum of |terms| over
// the 256-term chunk of one Gram block, set by the rounding of the float correction term;
// the chunks are then summed in FP64).  The operations of the two-sum carry
// explicit rounding so that no step is contracted into an FMA.

// hi = the leading 24 significant bits of x (truncated), lo = x - hi rounded to float; integer
// operations only.  |x| < 2^-100 gives 0 (negligible next to the unit-scale entries here);
// |x| > 2^100, inf and NaN take the plain conversion.
__device__ __forceinline__ float2 split_df(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sgn = (unsigned int)(b >> 32) & 0x80000000u;
  const int e = (int)((b >> 52) & 0x7ffULL) - 1023;
  if (e < -100) return make_float2(0.f, 0.f);
  if (e > 100) {
    const float h = (float)x;
    return make_float2(h, (float)(x - (double)h));
  }
  const unsigned long long mant = b & 0xfffffffffffffULL;
  const float hi = __uint_as_float(sgn | ((unsigned int)(e + 127) << 23) | (unsigned int)(mant >> 29));
  float lo = 0.f;
  if (e >= -70) {
    const float mag = __fmul_rn(__uint2float_rn((unsigned int)(mant & 0x1fffffffULL)),
                                __uint_as_float((unsigned int)(e - 52 + 127) << 23));
    lo = __uint_as_float(__float_as_uint(mag) | sgn);
  }
  return make_float2(hi, lo);
}
// (s, c) += a * b
__device__ __forceinline__ void df_fma(float &s, float &c, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float t = __fadd_rn(s, p);
  const float z = __fsub_rn(t, s);
  const float w = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(p, z));
  c = __fadd_rn(c, __fadd_rn(w, e));
  s = t;
}

// ---- 2-D tiled Gram: part[chunk][i][j] = sum_{l in chunk} A_i[l] B_j[l], 32 x 32 pair tiles,
// 64 threads with 4 x 4 outputs each; double-FP32 products and sums, FP64 partials ---------
constexpr int GT = 32, GRT = 32;
__global__ void __launch_bounds__(64) k_gram2d(const double *__restrict__ A, long long lda, int p,
                                               const double *__restrict__ B, long long ldb, int q,
                                               long long L, long long chunk, int ntq,
                                               double *__restrict__ part) {
  __shared__ float2 As[GRT][GT + 1];
  __shared__ float2 Bs[GRT][GT + 1];
  const int ti = blockIdx.x / ntq, tj = blockIdx.x % ntq;
  const int i0 = ti * GT, j0 = tj * GT;
  const long long l0 = blockIdx.y * chunk, l1 = min(L, l0 + chunk);
  const int tid = threadIdx.x;
  const int ty = tid >> 3, tx = tid & 7;
  // warps whose rows or columns all fall outside the matrix skip the products
  const bool active = (i0 + 4 * ty < p) && (j0 + 4 * tx < q);
  float s[4][4], c[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) s[a][b] = c[a][b] = 0.f;
  constexpr int NLD = GT * GRT / 64;  // elements of each operand tile per thread
  for (long long r0 = l0; r0 < l1; r0 += GRT) {
    // all loads of the tile issued before the first is used
    double va[NLD], vb[NLD];
#pragma unroll
    for (int t = 0; t < NLD; ++t) {
      const int idx = tid + 64 * t, i = idx / GRT, rr = idx % GRT;
      const long long l = r0 + rr;
      va[t] = (i0 + i < p && l < l1) ? A[(long long)(i0 + i) * lda + l] : 0.0;
      vb[t] = (j0 + i < q && l < l1) ? B[(long long)(j0 + i) * ldb + l] : 0.0;
    }
#pragma unroll
    for (int t = 0; t < NLD; ++t) {
      const int idx = tid + 64 * t, i = idx / GRT, rr = idx % GRT;
      As[rr][i] = split_df(va[t]);
      Bs[rr][i] = split_df(vb[t]);
    }
    __syncthreads();
    if (active) {
#pragma unroll 4
      for (int rr = 0; rr < GRT; ++rr) {
        float2 a[4], b[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          a[t] = As[rr][4 * ty + t];
          b[t] = Bs[rr][4 * tx + t];
        }
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) df_fma(s[x][y], c[x][y], a[x], b[y]);
      }
    }
    __syncthreads();
  }
  const long long base = (long long)blockIdx.y * p * q;
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const int i = i0 + 4 * ty + x, j = j0 + 4 * tx + y;
      if (i < p && j < q) part[base + (long long)i * q + j] = (double)s[x][y] + (double)c[x][y];
    }
}

// ---- tall-skinny combine: Y[j][l] = alpha sum_k V[k][l] C[j][k] + beta Y[j][l], j < q ------
// double-FP32 products and sums, as the Grams
constexpr int CTS = 16;
__global__ void __launch_bounds__(256) k_combine_ts(const double *__restrict__ V, long long ldv, int m,
                                                    const double *__restrict__ C, int ldc, int q,
                                                    double *__restrict__ Y, long long ldy, long long L,
                                                    double alpha, double beta) {
  __shared__ float2 Cs[CTS][MAXM];
  const int j0 = blockIdx.y * CTS;
  const int nj = min(CTS, q - j0);
  for (int idx = threadIdx.x; idx < CTS * m; idx += blockDim.x) {
    int j = idx / m, k = idx % m;
    Cs[j][k] = split_df(j < nj ? C[(long long)(j0 + j) * ldc + k] : 0.0);
  }
  __syncthreads();
  const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= L) return;
  float s[CTS], c[CTS];
#pragma unroll
  for (int j = 0; j < CTS; ++j) s[j] = c[j] = 0.f;
#pragma unroll 8
  for (int k = 0; k < m; ++k) {
    const float2 vk = split_df(V[(long long)k * ldv + l]);
#pragma unroll
    for (int j = 0; j < CTS; ++j) df_fma(s[j], c[j], vk, Cs[j][k]);
  }
#pragma unroll
  for (int j = 0; j < CTS; ++j) {
    if (j < nj) {
      double *y = Y + (long long)(j0 + j) * ldy + l;
      const double acc = (double)s[j] + (double)c[j];
      *y = alpha * acc + (beta != 0.0 ? beta * (*y) : 0.0);
    }
  }
}

// ---- FP64 forms of the Gram, combination and Jacobi kernels ---------------------------------
// Contexts of the FP64 form converge to tight residuals (1e-8 and below), where the folded
// extraction resolves neighbouring roots only if its Grams carry FP64-level accuracy: their
// smallest eigenvalues sit at the squared residual.  These contexts keep the Krylov-space
// arithmetic in FP64 (at the FP64 issue rate); the mixed form (residual 1e-6) uses the
// double-FP32 kernels above.
__global__ void __launch_bounds__(256) k_gram2d_f64(const double *__restrict__ A, long long lda, int p,
                                                const double *__restrict__ B, long long ldb, int q,
                                                long long L, long long chunk, int ntq,
                                                double *__restrict__ part) {
  __shared__ double As[GT][GRT + 1];
  __shared__ double Bs[GT][GRT + 1];
  const int ti = blockIdx.x / ntq, tj = blockIdx.x % ntq;
  const int i0 = ti * GT, j0 = tj * GT;
  const long long l0 = blockIdx.y * chunk, l1 = min(L, l0 + chunk);
  const int tid = threadIdx.x;
  const int oi = tid >> 3, oj = (tid & 7) * 4;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long r0 = l0; r0 < l1; r0 += GRT) {
    for (int idx = tid; idx < GT * GRT; idx += 256) {
      int i = idx / GRT, rr = idx % GRT;
      long long l = r0 + rr;
      As[i][rr] = (i0 + i < p && l < l1) ? A[(long long)(i0 + i) * lda + l] : 0.0;
      Bs[i][rr] = (j0 + i < q && l < l1) ? B[(long long)(j0 + i) * ldb + l] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < GRT; ++rr) {
      const double a = As[oi][rr];
#pragma unroll
      for (int t = 0; t < 4; ++t) acc[t] = fma(a, Bs[oj + t][rr], acc[t]);
    }
    __syncthreads();
  }
  const long long base = (long long)blockIdx.y * p * q;
  for (int t = 0; t < 4; ++t) {
    const int i = i0 + oi, j = j0 + oj + t;
    if (i < p && j < q) part[base + (long long)i * q + j] = acc[t];
  }
}

__global__ void __launch_bounds__(256) k_combine_ts_f64(const double *__restrict__ V, long long ldv, int m,
                                                    const double *__restrict__ C, int ldc, int q,
                                                    double *__restrict__ Y, long long ldy, long long L,
                                                    double alpha, double beta) {
  __shared__ double Cs[CTS][MAXM];
  const int j0 = blockIdx.y * CTS;
  const int nj = min(CTS, q - j0);
  for (int idx = threadIdx.x; idx < nj * m; idx += blockDim.x) {
    int j = idx / m, k = idx % m;
    Cs[j][k] = C[(long long)(j0 + j) * ldc + k];
  }
  __syncthreads();
  const long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (l >= L) return;
  double acc[CTS];
#pragma unroll
  for (int j = 0; j < CTS; ++j) acc[j] = 0.0;
  for (int k = 0; k < m; ++k) {
    const double vk = V[(long long)k * ldv + l];
#pragma unroll
    for (int j = 0; j < CTS; ++j) acc[j] = fma(vk, Cs[j][k], acc[j]);
  }
  for (int j = 0; j < nj; ++j) {
    double *y = Y + (long long)(j0 + j) * ldy + l;
    *y = alpha * acc[j] + (beta != 0.0 ? beta * (*y) : 0.0);
  }
}

__global__ void __launch_bounds__(512) k_jacobi_eig_f64(const double *__restrict__ Gin, int m,
                                                    double *__restrict__ lam,
                                                    double *__restrict__ E, int max_sweeps) {
  extern __shared__ double sm[];
  const int mp = (m + 1) & ~1;
  double *A = sm;            // mp x mp
  double *V = sm + mp * mp;  // mp x mp, eigenvectors as columns
  __shared__ double cs[MAXM / 2], sn[MAXM / 2];
  __shared__ int pp[MAXM / 2], qq[MAXM / 2];
  __shared__ double red[512];
  __shared__ int perm[MAXM];
  const int tid = threadIdx.x, nt = blockDim.x;
  double diag_big = 0.0;
  for (int idx = tid; idx < mp * mp; idx += nt) {
    int i = idx / mp, j = idx % mp;
    double a;
    if (i < m && j < m) a = 0.5 * (Gin[i * m + j] + Gin[j * m + i]);
    else a = 0.0;
    A[idx] = a;
    V[idx] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // a padding row gets a diagonal larger than every eigenvalue so it sorts last
  if (mp != m) {
    double s = 0.0;
    for (int idx = tid; idx < m * m; idx += nt) s += fabs(A[(idx / m) * mp + idx % m]);
    red[tid] = s;
    __syncthreads();
    for (int st = nt / 2; st > 0; st >>= 1) {
      if (tid < st) red[tid] += red[tid + st];
      __syncthreads();
    }
    diag_big = 1.0 + 2.0 * red[0];
    if (tid == 0) A[(mp - 1) * mp + (mp - 1)] = diag_big;
    __syncthreads();
  }
  const int half = mp / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // off-diagonal and total norms
    double off = 0.0, tot = 0.0;
    for (int idx = tid; idx < mp * mp; idx += nt) {
      double a = A[idx];
      tot += a * a;
      if (idx / mp != idx % mp) off += a * a;
    }
    red[tid] = off;
    __syncthreads();
    for (int st = nt / 2; st > 0; st >>= 1) {
      if (tid < st) red[tid] += red[tid + st];
      __syncthreads();
    }
    off = red[0];
    __syncthreads();
    red[tid] = tot;
    __syncthreads();
    for (int st = nt / 2; st > 0; st >>= 1) {
      if (tid < st) red[tid] += red[tid + st];
      __syncthreads();
    }
    tot = red[0];
    __syncthreads();
    if (off <= 1e-28 * tot || off == 0.0) break;
    for (int r = 0; r < mp - 1; ++r) {
      if (tid < half) {
        int k = tid;
        int a, b;
        if (k == 0) {
          a = 0;
          b = (r % (mp - 1)) + 1;
        } else {
          a = ((r + k) % (mp - 1)) + 1;
          b = ((r - k + (mp - 1)) % (mp - 1)) + 1;
        }
        int p = min(a, b), q = max(a, b);
        double apq = A[p * mp + q];
        double c = 1.0, s = 0.0;
        if (fabs(apq) > 1e-300) {
          double app = A[p * mp + p], aqq = A[q * mp + q];
          double theta = (aqq - app) / (2.0 * apq);
          double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
          c = 1.0 / sqrt(t * t + 1.0);
          s = t * c;
        }
        cs[k] = c;
        sn[k] = s;
        pp[k] = p;
        qq[k] = q;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int idx = tid; idx < half * mp; idx += nt) {
        int k = idx / mp, j = idx % mp;
        int p = pp[k], q = qq[k];
        double c = cs[k], s = sn[k];
        double ap = A[p * mp + j], aq = A[q * mp + j];
        A[p * mp + j] = c * ap - s * aq;
        A[q * mp + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int idx = tid; idx < half * mp; idx += nt) {
        int k = idx / mp, i = idx % mp;
        int p = pp[k], q = qq[k];
        double c = cs[k], s = sn[k];
        double ap = A[i * mp + p], aq = A[i * mp + q];
        A[i * mp + p] = c * ap - s * aq;
        A[i * mp + q] = s * ap + c * aq;
        double vp = V[i * mp + p], vq = V[i * mp + q];
        V[i * mp + p] = c * vp - s * vq;
        V[i * mp + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    for (int i = 0; i < m; ++i) perm[i] = i;
    for (int i = 0; i < m; ++i) {  // selection sort of the m real eigenvalues
      int best = i;
      for (int j = i + 1; j < m; ++j)
        if (A[perm[j] * mp + perm[j]] < A[perm[best] * mp + perm[best]]) best = j;
      int t = perm[i];
      perm[i] = perm[best];
      perm[best] = t;
    }
  }
  __syncthreads();
  // drop the padding column: if it was not the last after sorting the pad index is m
  for (int j = tid; j < m; j += nt) lam[j] = A[perm[j] * mp + perm[j]];
  for (int idx = tid; idx < m * m; idx += nt) {
    int j = idx / m, i = idx % m;
    E[idx] = V[i * mp + perm[j]];
  }
}

// ---- Cholesky QR of a block: G = N^T N (n x n); T (row j = coefficients of new vector j) with
// N_new_j = sum_k N_k T[j][k]; columns whose pivot falls below tol * G_jj are dropped (T row 0,
// kept[j] = 0).  One thread (n <= 64).
__global__ void k_cholqr(const double *__restrict__ Gin, int n, double tol, double *__restrict__ T,
                         int *__restrict__ kept) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double Lm[64][64];
  int keep[64];
  for (int j = 0; j < n; ++j) {
    double d = Gin[j * n + j];
    for (int k = 0; k < j; ++k)
      if (keep[k]) d -= Lm[j][k] * Lm[j][k];
    keep[j] = (d > tol * Gin[j * n + j] && d > 0.0) ? 1 : 0;
    const double ljj = keep[j] ? sqrt(d) : 0.0;
    Lm[j][j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double g = Gin[i * n + j];
      for (int k = 0; k < j; ++k)
        if (keep[k]) g -= Lm[i][k] * Lm[j][k];
      Lm[i][j] = keep[j] ? g / ljj : 0.0;
    }
  }
  for (int idx = 0; idx < n * n; ++idx) T[idx] = 0.0;
  // row j of L^-1: L^-1 is lower triangular; compute column by column
  for (int c = 0; c < n; ++c) {
    if (!keep[c]) continue;
    for (int i = 0; i < n; ++i) {
      if (i < c || !keep[i]) continue;
      double r = (i == c) ? 1.0 : 0.0;
      for (int t = c; t < i; ++t)
        if (keep[t]) r -= Lm[i][t] * T[t * n + c];
      T[i * n + c] = r / Lm[i][i];
    }
  }
  for (int j = 0; j < n; ++j) kept[j] = keep[j];
}

// ---- parallel cyclic Jacobi for a symmetric m x m matrix (m <= MAXM) -----------------
// out: evals ascending in lam[m]; eigenvectors as rows E[j*m + i] (component i of vector j)
//
// A and the accumulated rotations V are held in double-FP32 (pairs hi + lo, 48 significant
// bits) and rotated with double-FP32 products and sums: the FP64 rate of this part would
// make the O(m^2) work of each of the m - 1 rounds of a sweep the dominant cost.  Rotation
// angles are computed in FP32 from the pairs; the (c, s) of each rotation are then corrected
// in double-FP32 so that c^2 + s^2 = 1 to about 2^-46, so every rotation stays orthogonal
// whatever the accuracy of its angle (an angle off by 1e-7 relative leaves an off-diagonal
// 1e-7 times smaller, removed by the next sweep).  The sweeps stop at an off-diagonal
// Frobenius norm of 1e-11 relative, within reach of the pair precision.
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float s = __fadd_rn(p, e);
  return make_float2(s, __fsub_rn(e, __fsub_rn(s, p)));
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float z = __fsub_rn(s, a.x);
  float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, z)), __fsub_rn(b.x, z));
  e = __fadd_rn(e, __fadd_rn(a.y, b.y));
  const float t = __fadd_rn(s, e);
  return make_float2(t, __fsub_rn(e, __fsub_rn(t, s)));
}
// (c', s') = (c, s) (1 + eps) with (c^2 + s^2)(1 + eps)^2 = 1 to second order in the defect
__device__ __forceinline__ void df_unit_rotation(float c, float s, float2 &cd, float2 &sd) {
  const float c2 = __fmul_rn(c, c), c2e = fmaf(c, c, -c2);
  const float s2 = __fmul_rn(s, s), s2e = fmaf(s, s, -s2);
  // defect d = c^2 + s^2 - 1 (|d| ~ 1e-7): the high parts summed exactly, then the residuals
  const float2 n = df_add(make_float2(c2, c2e), make_float2(s2, s2e));
  const float d = __fadd_rn(__fsub_rn(n.x, 1.0f), n.y);
  const float eps = fmaf(0.375f * d, d, -0.5f * d);
  cd = make_float2(c, __fmul_rn(c, eps));
  sd = make_float2(s, __fmul_rn(s, eps));
}
__global__ void __launch_bounds__(512) k_jacobi_eig(const double *__restrict__ Gin, int m,
                                                    double *__restrict__ lam,
                                                    double *__restrict__ E, int max_sweeps) {
  extern __shared__ double sm_raw[];
  const int mp = (m + 1) & ~1;
  // rows padded to an odd number of 8-byte words: a column of A or V read across a warp
  // then falls in distinct shared-memory banks
  const int ld = mp + 1;
  float2 *A = reinterpret_cast<float2 *>(sm_raw);  // mp x ld
  float2 *V = A + mp * ld;                          // mp x ld, eigenvectors as columns
  __shared__ float2 cs[MAXM / 2], sn[MAXM / 2];
  __shared__ int pp[MAXM / 2], qq[MAXM / 2];
  __shared__ float red[512];
  __shared__ int perm[MAXM];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int idx = tid; idx < mp * mp; idx += nt) {
    int i = idx / mp, j = idx % mp;
    double a;
    if (i < m && j < m) a = 0.5 * (Gin[i * m + j] + Gin[j * m + i]);
    else a = 0.0;
    A[i * ld + j] = split_df(a);
    V[i * ld + j] = make_float2((i == j) ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  // a padding row gets a diagonal larger than every eigenvalue so it sorts last
  if (mp != m) {
    float s = 0.f;
    for (int idx = tid; idx < m * m; idx += nt) s += fabsf(A[(idx / m) * ld + idx % m].x);
    red[tid] = s;
    __syncthreads();
    for (int st = nt / 2; st > 0; st >>= 1) {
      if (tid < st) red[tid] += red[tid + st];
      __syncthreads();
    }
    if (tid == 0) A[(mp - 1) * ld + (mp - 1)] = make_float2(1.f + 2.f * red[0], 0.f);
    __syncthreads();
  }
  const int half = mp / 2;
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // off-diagonal and total squared norms (FP32: only the stopping test uses them)
    float off = 0.f, tot = 0.f;
    for (int idx = tid; idx < mp * mp; idx += nt) {
      const float a = A[(idx / mp) * ld + idx % mp].x;
      tot += a * a;
      if (idx / mp != idx % mp) off += a * a;
    }
    red[tid] = off;
    __syncthreads();
    for (int st = nt / 2; st > 0; st >>= 1) {
      if (tid < st) red[tid] += red[tid + st];
      __syncthreads();
    }
    off = red[0];
    __syncthreads();
    red[tid] = tot;
    __syncthreads();
    for (int st = nt / 2; st > 0; st >>= 1) {
      if (tid < st) red[tid] += red[tid + st];
      __syncthreads();
    }
    tot = red[0];
    __syncthreads();
    if (off <= 1e-22f * tot || off == 0.f) break;
    for (int r = 0; r < mp - 1; ++r) {
      if (tid < half) {
        int k = tid;
        int a, b;
        if (k == 0) {
          a = 0;
          b = (r % (mp - 1)) + 1;
        } else {
          a = ((r + k) % (mp - 1)) + 1;
          b = ((r - k + (mp - 1)) % (mp - 1)) + 1;
        }
        int p = min(a, b), q = max(a, b);
        const float2 apq = A[p * ld + q];
        float2 cd = make_float2(1.f, 0.f), sd = make_float2(0.f, 0.f);
        if (apq.x != 0.f) {
          const float2 app = A[p * ld + p], aqq = A[q * ld + q];
          const float diff = __fadd_rn(__fsub_rn(aqq.x, app.x), __fsub_rn(aqq.y, app.y));
          const float theta = diff / (2.f * (apq.x + apq.y));
          const float t = (theta >= 0.f ? 1.f : -1.f) / (fabsf(theta) + sqrtf(fmaf(theta, theta, 1.f)));
          const float c = rsqrtf(fmaf(t, t, 1.f));
          df_unit_rotation(c, t * c, cd, sd);
        }
        cs[k] = cd;
        sn[k] = sd;
        pp[k] = p;
        qq[k] = q;
      }
      __syncthreads();
      // rows: A <- J^T A
      for (int idx = tid; idx < half * mp; idx += nt) {
        int k = idx / mp, j = idx % mp;
        int p = pp[k], q = qq[k];
        const float2 c = cs[k], s = sn[k];
        const float2 ap = A[p * ld + j], aq = A[q * ld + j];
        const float2 ms = make_float2(-s.x, -s.y);
        A[p * ld + j] = df_add(df_mul(c, ap), df_mul(ms, aq));
        A[q * ld + j] = df_add(df_mul(s, ap), df_mul(c, aq));
      }
      __syncthreads();
      // columns: A <- A J, V <- V J
      for (int idx = tid; idx < half * mp; idx += nt) {
        int k = idx / mp, i = idx % mp;
        int p = pp[k], q = qq[k];
        const float2 c = cs[k], s = sn[k];
        const float2 ms = make_float2(-s.x, -s.y);
        const float2 ap = A[i * ld + p], aq = A[i * ld + q];
        A[i * ld + p] = df_add(df_mul(c, ap), df_mul(ms, aq));
        A[i * ld + q] = df_add(df_mul(s, ap), df_mul(c, aq));
        const float2 vp = V[i * ld + p], vq = V[i * ld + q];
        V[i * ld + p] = df_add(df_mul(c, vp), df_mul(ms, vq));
        V[i * ld + q] = df_add(df_mul(s, vp), df_mul(c, vq));
      }
      __syncthreads();
    }
  }
  // ascending order of the diagonal (pairs normalised by df_add, so hi then lo orders them):
  // rank of each entry, ties broken by index
  for (int j = tid; j < mp; j += nt) {
    const float2 dj = A[j * ld + j];
    int rank = 0;
    for (int i = 0; i < mp; ++i) {
      const float2 di = A[i * ld + i];
      rank += (di.x < dj.x || (di.x == dj.x && (di.y < dj.y || (di.y == dj.y && i < j)))) ? 1 : 0;
    }
    perm[rank] = j;
  }
  __syncthreads();
  // drop the padding column: if it was not the last after sorting the pad index is m
  for (int j = tid; j < m; j += nt) {
    const float2 d = A[perm[j] * ld + perm[j]];
    lam[j] = (double)d.x + (double)d.y;
  }
  for (int idx = tid; idx < m * m; idx += nt) {
    int j = idx / m, i = idx % m;
    const float2 e = V[i * ld + perm[j]];
    E[idx] = (double)e.x + (double)e.y;
  }
}

// ---- per-column reductions ------------------------------------------------------------
__device__ double block_sum(double x, double *red) {
  red[threadIdx.x] = x;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  double r = red[0];
  __syncthreads();
  return r;
}

// per column j: out[j*3 + 0..2] = (x.Mx, x.Sx, x.x)
__global__ void k_ritz_dots(const double *__restrict__ X, const double *__restrict__ MX,
                            const double *__restrict__ SX, long long L, double *__restrict__ out) {
  __shared__ double red[256];
  const long long off = (long long)blockIdx.x * L;
  double a = 0, b = 0, c = 0;
  for (long long l = threadIdx.x; l < L; l += blockDim.x) {
    double x = X[off + l];
    a += x * MX[off + l];
    b += x * SX[off + l];
    c += x * x;
  }
  a = block_sum(a, red);
  b = block_sum(b, red);
  c = block_sum(c, red);
  if (threadIdx.x == 0) {
    out[blockIdx.x * 3 + 0] = a;
    out[blockIdx.x * 3 + 1] = b;
    out[blockIdx.x * 3 + 2] = c;
  }
}

// per column j: |MX - theta_j SX|^2 into rnorm[j]; correction direction of one Jacobi sweep on
// (M - theta_j Sigma) t = -r:  t = -r / D with D = [dA; dA] - theta_j [dS; -dS], |D| floored
// at floor_ keeping its sign.
__global__ void k_resid_dir(const double *__restrict__ X, const double *__restrict__ MX,
                            const double *__restrict__ SX, const double *__restrict__ theta,
                            const double *__restrict__ dA, const double *__restrict__ dS,
                            long long ov, double floor_, double *__restrict__ Dout,
                            double *__restrict__ rnorm) {
  __shared__ double red[256];
  const long long L = 2 * ov;
  const long long off = (long long)blockIdx.x * L;
  const double th = theta[blockIdx.x];
  double acc = 0.0;
  for (long long l = threadIdx.x; l < L; l += blockDim.x) {
    double r = MX[off + l] - th * SX[off + l];
    acc += r * r;
    if (Dout) {
      long long e = l % ov;
      double sg = (l < ov) ? 1.0 : -1.0;
      double D = dA[e] - th * sg * dS[e];
      if (fabs(D) < floor_) D = (D >= 0 ? floor_ : -floor_);
      Dout[off + l] = -r / D;
    }
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) rnorm[blockIdx.x] = acc;
}

// oscillator strengths: z = x / sqrt(x^T Sigma x); out[j] = (2/3) theta sum_c (mu_c . (X + Y))^2
__global__ void k_osc(const double *__restrict__ X, const double *__restrict__ mu, long long ov,
                      const double *__restrict__ theta, const double *__restrict__ xsx,
                      double *__restrict__ out) {
  __shared__ double red[256];
  const long long off = (long long)blockIdx.x * 2 * ov;
  double m0 = 0, m1 = 0, m2 = 0;
  for (long long e = threadIdx.x; e < ov; e += blockDim.x) {
    double s = X[off + e] + X[off + ov + e];
    m0 += mu[e] * s;
    m1 += mu[ov + e] * s;
    m2 += mu[2 * ov + e] * s;
  }
  m0 = block_sum(m0, red);
  m1 = block_sum(m1, red);
  m2 = block_sum(m2, red);
  if (threadIdx.x == 0) {
    double nrm = xsx[blockIdx.x];
    out[blockIdx.x] = (2.0 / 3.0) * theta[blockIdx.x] * (m0 * m0 + m1 * m1 + m2 * m2) / fabs(nrm);
  }
}

__global__ void k_unit_vectors(double *__restrict__ V, long long L, const int *__restrict__ idx, int nb) {
  int j = blockIdx.y;
  for (long long l = blockIdx.x * (long long)blockDim.x + threadIdx.x; l < L;
       l += (long long)gridDim.x * blockDim.x)
    V[j * L + l] = (l == idx[j]) ? 1.0 : 0.0;
}


// ---- small dense linear algebra on the projected pencil -----------------------------
// FP64 issues at a small fraction of the FP32 rate on this part, so these kernels keep
// dependent chains short (one reciprocal square root per pivot, products with reciprocals
// instead of divisions) and spread the O(m^2) work of each step over the whole block.
__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
// Cholesky of a symmetric positive definite m x m matrix held in shared memory (row stride
// ld), by the whole block.  Strict lower factor in place; the pivots as L_kk in dL (if set)
// and 1 / L_kk in dinv.  Returns false (for every thread) if a pivot is not positive.
__device__ bool blk_cholesky(double *G, int ld, int m, double *dinv, double *dL) {
  const int nt = blockDim.x;
  for (int k = 0; k < m; ++k) {
    const double akk = G[k * ld + k];
    if (!(akk > 0.0)) return false;
    const double r = rsqrt(akk);
    for (int i = k + 1 + threadIdx.x; i < m; i += nt) G[i * ld + k] *= r;
    if (threadIdx.x == 0) {
      dinv[k] = r;
      if (dL) dL[k] = akk * r;
    }
    __syncthreads();
    // trailing update of the lower triangle, element e -> (row k+1+ii, column k+1+jj), jj <= ii
    const int n = m - k - 1, cnt = n * (n + 1) / 2;
    for (int e = threadIdx.x; e < cnt; e += nt) {
      int ii = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
      while (ii * (ii + 1) / 2 > e) --ii;
      while ((ii + 1) * (ii + 2) / 2 <= e) ++ii;
      const int jj = e - ii * (ii + 1) / 2;
      const int i = k + 1 + ii, j = k + 1 + jj;
      G[i * ld + j] -= G[i * ld + k] * G[j * ld + k];
    }
    __syncthreads();
  }
  return true;
}

// Rayleigh-Ritz setup, step 1: Hm = L L^T (one block).  L to Lout (m x m, row-major, zero
// above the diagonal), 1 / L_ii to dinv_out.
__global__ void __launch_bounds__(256) k_chol_rr(const double *__restrict__ Hm, int m,
                                                 double *__restrict__ Lout, double *__restrict__ dinv_out,
                                                 int *__restrict__ status) {
  extern __shared__ double sm[];
  const int ld = m + 1;
  double *G = sm;
  double *dL = G + m * ld;
  double *dinv = dL + m;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    int i = idx / m, k = idx % m;
    G[i * ld + k] = 0.5 * (Hm[i * m + k] + Hm[k * m + i]);
  }
  __syncthreads();
  if (!blk_cholesky(G, ld, m, dinv, dL)) {
    if (threadIdx.x == 0) *status = 1;
    return;
  }
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    int i = idx / m, k = idx % m;
    Lout[idx] = (k < i) ? G[i * ld + k] : (k == i ? dL[i] : 0.0);
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) dinv_out[i] = dinv[i];
}
// Rayleigh-Ritz setup, steps 2 and 3 (Cw = L^-1 Hs L^-T), one warp per right-hand side:
//   rows == 0: Y[:, j] = L^-1 sym(Hs)[:, j]      rows == 1: Cw[j, :] = L^-1 Y[j, :]
// Forward substitution column by column of L (its column i read with stride m), the running
// right-hand side in shared memory.  Skipped when the factorisation failed.
__global__ void __launch_bounds__(128) k_rr_trsm(const double *__restrict__ R, const double *__restrict__ Lm,
                                                 const double *__restrict__ dinv, int m, int rows,
                                                 double *__restrict__ Out, const int *__restrict__ status) {
  __shared__ double acc[4][MAXM];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = blockIdx.x * 4 + warp;
  if (j >= m || *status) return;
  double *a = acc[warp];
  for (int i = lane; i < m; i += 32) a[i] = rows ? R[j * m + i] : 0.5 * (R[i * m + j] + R[j * m + i]);
  __syncwarp();
  for (int i = 0; i < m; ++i) {
    const double yi = a[i] * dinv[i];
    for (int k = i + 1 + lane; k < m; k += 32) a[k] -= Lm[k * m + i] * yi;
    if (lane == 0) Out[rows ? j * m + i : i * m + j] = yi;
    __syncwarp();
  }
}

// E = L^-T W (generalised eigenvectors, E^T Hm E = 1), theta = 1/mu, the ncol columns with
// theta nearest the shift (ascending distance), each scaled to unit Euclidean norm.  Only
// the selected columns are back-substituted, one warp each; the running sums of L^T e = w
// are held in shared memory and updated column by column (row i of L is contiguous).
__global__ void __launch_bounds__(128) k_rr_select(const double *__restrict__ Lm,
                                                   const double *__restrict__ mu,
                                                   const double *__restrict__ W, int m,
                                                   double shift, int ncol,
                                                   double *__restrict__ Ework,
                                                   double *__restrict__ theta_out,
                                                   double *__restrict__ Eout) {
  __shared__ int order[MAXM];
  __shared__ double dist[MAXM];
  __shared__ double dinv[MAXM];
  __shared__ double acc[4][MAXM];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = tid; j < m; j += blockDim.x) {
    const double th = (fabs(mu[j]) > 1e-300) ? 1.0 / mu[j] : 1e300;
    dist[j] = fabs(th - shift);
    dinv[j] = 1.0 / Lm[j * m + j];
  }
  __syncthreads();
  if (tid == 0) {
    for (int j = 0; j < m; ++j) order[j] = j;
    for (int i = 0; i < ncol && i < m; ++i) {
      int best = i;
      for (int j = i + 1; j < m; ++j)
        if (dist[order[j]] < dist[order[best]]) best = j;
      int t = order[i];
      order[i] = order[best];
      order[best] = t;
    }
  }
  __syncthreads();
  double *a = acc[warp];
  for (int t = warp; t < ncol && t < m; t += 4) {
    const int j = order[t];
    const double *w = W + (long long)j * m;
    double *e = Ework + (long long)t * m;
    for (int i = lane; i < m; i += 32) a[i] = w[i];
    __syncwarp();
    // L^T e = w from the last row up: e_i = a_i / L_ii, then a_k -= L_ik e_i for k < i
    for (int i = m - 1; i >= 0; --i) {
      const double ei = a[i] * dinv[i];
      for (int k = lane; k < i; k += 32) a[k] -= Lm[i * m + k] * ei;
      if (lane == 0) e[i] = ei;
      __syncwarp();
    }
    double nrm = 0.0;
    for (int i = lane; i < m; i += 32) nrm += e[i] * e[i];
    nrm = rsqrt(warp_sum(nrm));
    for (int i = lane; i < m; i += 32) Eout[(long long)t * m + i] = e[i] * nrm;
    if (lane == 0) theta_out[t] = (fabs(mu[j]) > 1e-300) ? 1.0 / mu[j] : 1e300;
    __syncwarp();
  }
}

// Folded-spectrum vectors with deflation, one block of four warps (the reduced problem has
// m <= 32).  For target j:
//   w <- th0[j]; repeat reps times:
//     G(w) = (MV - w SV)^T (MV - w SV) = Gmm - w (Gms + Gms^T) + w^2 Gss,
//     restricted to coefficients Euclidean-orthogonal to Hs c_i (i < j): P G(w) P + gamma Q^T Q
//     with P = 1 - Q^T Q, Q the orthonormal constraint directions,
//     c <- smallest eigenvector (inverse iteration from the previous c), w <- c^T Hm c / c^T Hs c.
// P G(w) P = Amm - w Ams + w^2 Ass with A = P G P for the three Grams; each new constraint
// direction q (orthogonal to the earlier ones) updates them by a rank-2 term,
//   A <- A - (A q) q^T - q (A q)^T + (q^T A q) q q^T,
// so a repetition costs O(m^2) plus one Cholesky factorisation.
//
// FP64 runs at a small fraction of the FP32 rate on this part, so the kernel keeps the
// dependent chains short: each Cholesky pivot takes one reciprocal square root, the
// triangular solves multiply by those reciprocals with the right-hand side held in the
// registers of warp 0 (element i in lane i), and the O(m^2) updates (trailing Cholesky
// update, shifted matrix, rank-2 projections, matrix-vector products) are spread over all
// four warps, so that all four schedulers of the SM issue FP64 work.
constexpr int RT = 128;  // threads of k_refined
// sum over the block of RT threads (every thread gets the result)
__device__ double rt_sum(double x, double *red) {
  x = warp_sum(x);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  const double r = red[0] + red[1] + red[2] + red[3];
  __syncthreads();
  return r;
}
// y = A x for m <= 32 (A row-major with leading dimension ld): thread (lane i, warp w) sums
// the columns k = w mod 4; part holds 4 x 32 partial sums
__device__ void rt_matvec(const double *A, int ld, int m, const double *x, double *y, double *part) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane < m) {
    double s = 0.0;
    for (int k = w; k < m; k += 4) s += A[lane * ld + k] * x[k];
    part[w * 32 + lane] = s;
  }
  __syncthreads();
  if (threadIdx.x < m) {
    const int i = threadIdx.x;
    y[i] = (part[i] + part[32 + i]) + (part[64 + i] + part[96 + i]);
  }
  __syncthreads();
}
// warp 0: solve L L^T x = y for the vector held one element per lane (lanes >= m hold 0)
__device__ double warp_chol_solve_reg(const double *G, int ld, int m, const double *dinv, double y) {
  const int lane = threadIdx.x & 31;
  for (int k = 0; k < m; ++k) {
    const double yk = __shfl_sync(0xffffffffu, y, k) * dinv[k];
    if (lane == k) y = yk;
    else if (lane > k && lane < m) y -= G[lane * ld + k] * yk;
  }
  for (int k = m - 1; k >= 0; --k) {
    const double xk = __shfl_sync(0xffffffffu, y, k) * dinv[k];
    if (lane == k) y = xk;
    else if (lane < k) y -= G[k * ld + lane] * xk;
  }
  return y;
}
// A <- A - u q^T - q u^T + (q^T u) q q^T with u = A q (u, part: scratch)
__device__ void rt_rank2_project(double *A, int ld, int m, const double *q, double *u, double *part,
                                 double *red) {
  rt_matvec(A, ld, m, q, u, part);
  const double a = rt_sum(threadIdx.x < m ? q[threadIdx.x] * u[threadIdx.x] : 0.0, red);
  for (int idx = threadIdx.x; idx < m * m; idx += RT) {
    const int i = idx / m, k = idx % m;
    A[i * ld + k] += -u[i] * q[k] - q[i] * u[k] + a * q[i] * q[k];
  }
  __syncthreads();
}
__global__ void __launch_bounds__(RT) k_refined(const double *__restrict__ Hm,
                                                const double *__restrict__ Hs,
                                                const double *__restrict__ Gmm,
                                                const double *__restrict__ Gms,
                                                const double *__restrict__ Gss, int m, int b,
                                                int reps, const double *__restrict__ th0,
                                                const double *__restrict__ C0,
                                                double *__restrict__ Cout,
                                                double *__restrict__ thout,
                                                int *__restrict__ status) {
  extern __shared__ double sm[];
  const int ld = m + 1;
  double *Amm = sm;             // m x ld each: P Gmm P, P (Gms + Gms^T) P, P Gss P
  double *Ams = Amm + m * ld;
  double *Ass = Ams + m * ld;
  double *QQ = Ass + m * ld;    // Q^T Q
  double *F = QQ + m * ld;      // the shifted matrix, then its Cholesky factor
  double *Qc = F + m * ld;      // b x m, orthonormal constraint directions
  double *c = Qc + b * m;       // m
  double *u = c + m;            // m
  double *dinv = u + m;         // m
  double *part = dinv + m;      // 4 x 32
  double *red = part + 128;     // 8
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int idx = tid; idx < m * m; idx += RT) {
    const int i = idx / m, k = idx % m;
    Amm[i * ld + k] = 0.5 * (Gmm[i * m + k] + Gmm[k * m + i]);
    Ams[i * ld + k] = Gms[i * m + k] + Gms[k * m + i];
    Ass[i * ld + k] = 0.5 * (Gss[i * m + k] + Gss[k * m + i]);
    QQ[i * ld + k] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < b; ++j) {
    double w = th0[j];
    if (tid < m) c[tid] = C0[(long long)j * m + tid];
    __syncthreads();
    bool ok = true;
    for (int rep = 0; rep < reps && ok; ++rep) {
      const double tr = fabs(rt_sum(
          tid < m ? Amm[tid * ld + tid] - w * Ams[tid * ld + tid] + w * w * Ass[tid * ld + tid] : 0.0, red));
      const double gamma = 10.0 * tr + 1e-300, delta = 1e-14 * tr + 1e-300;
      for (int idx = tid; idx < m * m; idx += RT) {
        const int i = idx / m, k = idx % m;
        F[i * ld + k] = Amm[i * ld + k] - w * Ams[i * ld + k] + w * w * Ass[i * ld + k] + gamma * QQ[i * ld + k] +
                        (i == k ? delta : 0.0);
      }
      __syncthreads();
      ok = blk_cholesky(F, ld, m, dinv, nullptr);
      if (!ok) {
        if (tid == 0) *status = 2;
        break;
      }
      if (warp == 0) {
        double ci = lane < m ? c[lane] : 0.0;
        for (int itv = 0; itv < 4; ++itv) {
          // project c off the constraint directions (Q is orthonormal) and normalise
          double proj = 0.0;
          for (int p = 0; p < j; ++p) {
            const double qp = lane < m ? Qc[p * m + lane] : 0.0;
            proj += warp_sum(qp * ci) * qp;
          }
          ci -= proj;
          double nn = warp_sum(ci * ci);
          if (!(nn > 0.0)) nn = 1.0;
          ci *= rsqrt(nn);
          if (itv == 3) break;
          ci = warp_chol_solve_reg(F, ld, m, dinv, ci);
        }
        if (lane < m) c[lane] = ci;
      }
      __syncthreads();
      // fold centre follows the Rayleigh quotient of the folded vector
      rt_matvec(Hm, m, m, c, u, part);
      const double nm = rt_sum(tid < m ? c[tid] * u[tid] : 0.0, red);
      rt_matvec(Hs, m, m, c, u, part);
      const double ns = rt_sum(tid < m ? c[tid] * u[tid] : 0.0, red);
      if (fabs(ns) > 1e-300) w = nm / ns;
    }
    if (tid < m) Cout[(long long)j * m + tid] = c[tid];
    if (tid == 0) thout[j] = w;
    if (j + 1 == b) break;
    // new constraint direction: Hs c, orthonormalised against the previous ones (twice)
    rt_matvec(Hs, m, m, c, u, part);
    if (warp == 0) {
      double t = lane < m ? u[lane] : 0.0;
      for (int pass = 0; pass < 2; ++pass)
        for (int p = 0; p < j; ++p) {
          const double qp = lane < m ? Qc[p * m + lane] : 0.0;
          t -= warp_sum(qp * t) * qp;
        }
      const double nn = warp_sum(t * t);
      const double inv = (nn > 1e-300) ? rsqrt(nn) : 0.0;
      if (lane < m) Qc[j * m + lane] = t * inv;
    }
    __syncthreads();
    // fold it into the projected Grams and Q^T Q
    const double *q = Qc + j * m;
    rt_rank2_project(Amm, ld, m, q, u, part, red);
    rt_rank2_project(Ams, ld, m, q, u, part, red);
    rt_rank2_project(Ass, ld, m, q, u, part, red);
    for (int idx = tid; idx < m * m; idx += RT) {
      const int i = idx / m, k = idx % m;
      QQ[i * ld + k] += q[i] * q[k];
    }
    __syncthreads();
  }
}

// Gram-Schmidt (classical, applied twice) of ncol coefficient vectors K[t][m] (Euclidean);
// the first nout (<= 64) independent ones go to Q[t][m]; *nkept receives their count.  One
// block of RT threads: the projections of a pass are formed together, one warp per earlier
// vector, and subtracted together.
__global__ void __launch_bounds__(RT) k_mgs(const double *__restrict__ K, int m, int ncol, int nout,
                                            double *__restrict__ Qo, int *__restrict__ nkept, double tol) {
  __shared__ double red[8];
  __shared__ double v[MAXM];
  __shared__ double sdot[64];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  nout = min(nout, 64);
  int kept = 0;
  for (int t = 0; t < ncol && kept < nout; ++t) {
    for (int i = tid; i < m; i += RT) v[i] = K[(long long)t * m + i];
    __syncthreads();
    double n0 = 0.0;
    for (int i = tid; i < m; i += RT) n0 += v[i] * v[i];
    n0 = rt_sum(n0, red);
    for (int pass = 0; pass < 2 && kept > 0; ++pass) {
      for (int p = warp; p < kept; p += RT / 32) {
        double s = 0.0;
        for (int i = lane; i < m; i += 32) s += Qo[(long long)p * m + i] * v[i];
        s = warp_sum(s);
        if (lane == 0) sdot[p] = s;
      }
      __syncthreads();
      for (int i = tid; i < m; i += RT) {
        double x = v[i];
        for (int p = 0; p < kept; ++p) x -= sdot[p] * Qo[(long long)p * m + i];
        v[i] = x;
      }
      __syncthreads();
    }
    double n1 = 0.0;
    for (int i = tid; i < m; i += RT) n1 += v[i] * v[i];
    n1 = rt_sum(n1, red);
    if (n1 > tol * n0 && n1 > 0.0) {
      const double inv = rsqrt(n1);
      for (int i = tid; i < m; i += RT) Qo[(long long)kept * m + i] = v[i] * inv;
      ++kept;
    }
    __syncthreads();
  }
  if (tid == 0) *nkept = kept;
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct Solver {
  pp_ctx *c;
  cudaStream_t s;
  long long L;  // 2 ov
  double *part = nullptr;
  size_t part_elems = 0;
  bool f64 = false;  // FP64 Krylov-space arithmetic (contexts of the FP64 form)

  void gram(const double *A, long long lda, int p, const double *B, long long ldb, int q,
            double *G, int ldg, double alpha = 1.0, double beta = 0.0) {
    const int ntp = (p + GT - 1) / GT, ntq = (q + GT - 1) / GT;
    if (f64) {
      long long nch = std::max<long long>(1, std::min<long long>(L / 512, 304 / std::max(1, ntp * ntq) + 1));
      long long chunk = (L + nch - 1) / nch;
      chunk = ((chunk + GRT - 1) / GRT) * GRT;
      nch = (L + chunk - 1) / chunk;
      if ((size_t)nch * p * q > part_elems) throw PPError(PP_ECUDA, "gram scratch too small");
      k_gram2d_f64<<<dim3(ntp * ntq, (unsigned)nch), 256, 0, s>>>(A, lda, p, B, ldb, q, L, chunk, ntq, part);
      PP_LAUNCH_CHECK("k_gram2d_f64");
      k_gram_reduce<<<(p * q + 7) / 8, 256, 0, s>>>(part, (int)nch, p, q, G, ldg, alpha, beta);
      PP_LAUNCH_CHECK("k_gram_reduce");
      return;
    }
    // about eight 2-warp blocks per SM, chunks of at least 128 rows, partials within the scratch
    long long nch = std::min<long long>(L / 128, (8LL * 152) / std::max(1, ntp * ntq));
    nch = std::max<long long>(1, std::min<long long>(nch, (long long)(part_elems / std::max(1, p * q))));
    long long chunk = (L + nch - 1) / nch;
    chunk = ((chunk + GRT - 1) / GRT) * GRT;
    nch = (L + chunk - 1) / chunk;
    size_t need = (size_t)nch * p * q;
    if (need > part_elems) throw PPError(PP_ECUDA, "gram scratch too small");
    k_gram2d<<<dim3(ntp * ntq, (unsigned)nch), 64, 0, s>>>(A, lda, p, B, ldb, q, L, chunk, ntq, part);
    PP_LAUNCH_CHECK("k_gram2d");
    k_gram_reduce<<<(p * q + 7) / 8, 256, 0, s>>>(part, (int)nch, p, q, G, ldg, alpha, beta);
    PP_LAUNCH_CHECK("k_gram_reduce");
  }
  // Y[:, 0..q) (+)= V[:, 0..m) C with C[j*ldc + i] (column j of C), columns of length L
  void combine(const double *V, int m, const double *C, int ldc, int q, double *Y, double alpha,
               double beta) {
    if (m <= MAXM) {
      dim3 grid((unsigned)((L + 255) / 256), (unsigned)((q + CTS - 1) / CTS));
      if (f64)
        k_combine_ts_f64<<<grid, 256, 0, s>>>(V, L, m, C, ldc, q, Y, L, L, alpha, beta);
      else
        k_combine_ts<<<grid, 256, 0, s>>>(V, L, m, C, ldc, q, Y, L, L, alpha, beta);
      PP_LAUNCH_CHECK("k_combine_ts");
      return;
    }
    GemmF64 g;
    g.M = (int)L; g.N = q; g.K = m;
    g.A = V; g.a_m = 1; g.a_k = L;
    g.B = C; g.b_k = 1; g.b_n = ldc;
    g.C = Y; g.c_m = 1; g.c_n = L;
    g.alpha = alpha; g.beta = beta;
    gemm_f64(g, s);
  }
};

struct Window {
  bool used = false;     // slot holds a window
  bool fresh = false;    // initial block not formed yet
  bool finished = false; // results extracted, waiting to be taken
  double omega0 = 0, delta = 0;
  int k = 0;
  double shift = 0;
  int nev = 0, b = 0;
  int m = 0;
  int prec = PP_FP64;    // precision phase of this window's sigma products
  double tol = 0;        // residual tolerance of the current phase
  int iters = 0;
  double *V = nullptr, *MV = nullptr, *SV = nullptr;  // [m_max][L]
  double *X = nullptr, *MX = nullptr, *SX = nullptr;  // [64][L]
  double *Vr = nullptr, *MVr = nullptr, *SVr = nullptr;  // [32][L] reduced blocks for the folded step
  double *Hm, *Hs, *Gmm, *Gms, *Gss, *Lm, *Yw, *Cw, *mu, *W, *Ew, *Esel, *thsel, *Cref, *thref, *Kc, *Qk;
  double *dinv;  // 1 / L_ii of the Rayleigh-Ritz Cholesky factor
  double *Qr, *hm, *hs, *C0, *Cred;
  int *dstat, *dkept;
  std::vector<double> h_theta, h_res, h_xsx;
  std::vector<int> order;   // Ritz columns sorted by distance of theta to the shift
  std::vector<int> active;  // columns that get a direction this iteration
  int ndir = 0;             // directions staged for this step
  long long dpos = 0;       // their first column in the direction buffer
  int nnew = 0;             // orthonormal new basis vectors staged for this step's sigma
  long long npos = 0;       // their first column in the direction buffer after compaction
  int bx = 0;               // block size of the last extraction (rows of Cref, columns of X)
  int adjust = 0;
  double best_worst = 1e300;  // BF16 phase: best worst-residual seen, and iterations without gain
  int stall = 0;
  int guard_wait = 0;  // iterations spent waiting for guard targets only
  // select 0 with k > KCHUNK: the roots are found KCHUNK at a time, each chunk restarting just
  // above the last root found; k_total and omega_end describe the whole request
  int k_total = 0;
  double omega_end = 0;
  int iter0 = 0;     // iterations before the current chunk (max_iter applies per chunk)
  WindowResult res;  // accumulated results
};

// A single block of more than KCHUNK targets fills up with spurious interior Ritz values
// (mixtures of roots far apart, residuals of order 0.1) and stalls; larger requests are
// solved as consecutive chunks of KCHUNK roots.
constexpr int KCHUNK = 8;
// Ritz pairs with a residual above this are uninformative (the root they stand for could be
// anywhere within that distance, and spurious interior values sit there for good); they are
// neither reported nor counted among the roots a window needs.  Genuine approximations are
// below 2e-2 from the first iteration on.
constexpr double kSpurRes = 3e-2;

}  // namespace

void apply_sigma(pp_ctx *c, int nvec, const double *Zd, double *sig_d, double *met_d, int prec) {
  if (nvec <= 0) return;
  if (prec == PP_FP64) sigma_f64(c, nvec, Zd, sig_d, met_d);
  else sigma_bf16(c, nvec, Zd, sig_d, met_d, prec == PP_BF16X3);
}

// ---------------------------------------------------------------------------
// WindowBatch: a fixed number of window slots of one context, advanced together one
// iteration at a time.  Windows join (add) and leave (take) between steps; every step
// forms the new vectors of all windows and multiplies them in at most two sigma batches
// (one per precision phase).
// ---------------------------------------------------------------------------
struct WindowBatch {
  pp_ctx *c;
  cudaStream_t s;
  long long ov, L;
  int cap;
  bool keep_vectors;
  int m_max, bcap;
  size_t vecbytes, per_win;
  Solver sv;
  std::vector<double> ratio;  // diag(A) / diag(S)
  std::vector<Window> W;
  DevBuf mem, D, MD, SD, part, small;
  double *scratch = nullptr;
  int *iscratch = nullptr;
  bool log_on = false;
  long long steps = 0;
  long long sigma_calls = 0;  // sigma batches applied (a step applies one per precision phase)
  bool refine = false;
  int prec0 = PP_FP64;

  WindowBatch(pp_ctx *ctx, int capacity, bool vectors)
      : c(ctx), s(ctx->stream), ov(ctx->ov), L(2 * ctx->ov), cap(capacity), keep_vectors(vectors),
        sv{ctx, ctx->stream, 2 * ctx->ov} {
    m_max = std::min<int>(std::min(c->opt.m_max, MAXM), (int)L);
    bcap = std::max(1, std::min(32, m_max / 3));
    prec0 = c->opt.prec;
    sv.f64 = (prec0 == PP_FP64);
    refine = (prec0 == PP_BF16) && c->opt.refine;
    std::vector<double> hA(ov), hS(ov);
    PP_CUDA(cudaMemcpyAsync(hA.data(), c->diagA.p, sizeof(double) * ov, cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaMemcpyAsync(hS.data(), c->diagS.p, sizeof(double) * ov, cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    ratio.resize(ov);
    for (long long p = 0; p < ov; ++p) ratio[p] = hA[p] / hS[p];
    // device memory: per window basis (3 m_max vectors), Ritz block (3 x 64), reduced blocks
    // (3 x 32), small matrices; direction buffers of 32 columns per window
    vecbytes = sizeof(double) * (size_t)L;
    const size_t mm = (size_t)MAXM * MAXM;
    per_win = vecbytes * (3 * (size_t)m_max + 3 * 64 + 3 * 32) + sizeof(double) * 26 * mm + 64;
    mem.ensure(per_win * cap);
    D.ensure(vecbytes * 32 * cap);
    MD.ensure(vecbytes * 32 * cap);
    SD.ensure(vecbytes * 32 * cap);
    sv.part_elems = (size_t)296 * mm;
    part.ensure(sizeof(double) * sv.part_elems);
    sv.part = part.as<double>();
    small.ensure(sizeof(double) * 8192);
    scratch = small.as<double>();
    iscratch = reinterpret_cast<int *>(scratch + 4096);
    W.resize(cap);
    char *base = mem.as<char>();
    for (int w = 0; w < cap; ++w) {
      char *p = base + per_win * w;
      Window &wi = W[w];
      auto take = [&](size_t bytes) {
        char *q = p;
        p += bytes;
        return (double *)q;
      };
      wi.V = take(vecbytes * m_max);
      wi.MV = take(vecbytes * m_max);
      wi.SV = take(vecbytes * m_max);
      wi.X = take(vecbytes * 64);
      wi.MX = take(vecbytes * 64);
      wi.SX = take(vecbytes * 64);
      wi.Vr = take(vecbytes * 32);
      wi.MVr = take(vecbytes * 32);
      wi.SVr = take(vecbytes * 32);
      double **mats[] = {&wi.Hm, &wi.Hs, &wi.Gmm, &wi.Gms, &wi.Gss, &wi.Lm, &wi.Yw, &wi.Cw, &wi.mu,
                         &wi.W, &wi.Ew, &wi.Esel, &wi.thsel, &wi.Cref, &wi.thref, &wi.Kc, &wi.Qk,
                         &wi.Qr, &wi.hm, &wi.hs, &wi.C0, &wi.Cred, &wi.dinv};
      for (double **q : mats) *q = take(sizeof(double) * mm);
      wi.dstat = (int *)take(sizeof(double) * mm);
      wi.dkept = wi.dstat + 4;
    }
    const int ld = MAXM + 1;
    const int smem_jac = 2 * MAXM * (MAXM + 1) * (int)sizeof(double);
    const int smem_chol = (MAXM * ld + 2 * MAXM) * (int)sizeof(double);
    const int smem_ref = (MAXM * ld + 2 * 32 * MAXM + 3 * MAXM) * (int)sizeof(double);
    PP_CUDA(cudaFuncSetAttribute(k_jacobi_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_jac));
    PP_CUDA(cudaFuncSetAttribute(k_jacobi_eig_f64, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 2 * MAXM * MAXM * (int)sizeof(double)));
    PP_CUDA(cudaFuncSetAttribute(k_chol_rr, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_chol));
    PP_CUDA(cudaFuncSetAttribute(k_refined, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_ref));
    const char *log_env = std::getenv("PP_LOG");
    log_on = log_env && log_env[0] && log_env[0] != '0';
  }

  int used() const {
    int n = 0;
    for (const Window &wi : W) n += wi.used ? 1 : 0;
    return n;
  }
  bool has_work() const {
    for (const Window &wi : W)
      if (wi.used && !wi.finished) return true;
    return false;
  }

  // A new window in a free slot (-1 if none).  Its initial block is formed by the next step.
  int add(double omega0, double delta, int k) {
    if (k <= 0) throw PPError(PP_EINVAL, "k must be positive");
    if (c->opt.select == 1 && k > 24) throw PPError(PP_EINVAL, "k must be at most 24 for select = 1");
    int slot = -1;
    for (int w = 0; w < cap; ++w)
      if (!W[w].used) {
        slot = w;
        break;
      }
    if (slot < 0) return -1;
    Window &wi = W[slot];
    wi.used = true;
    wi.fresh = true;
    wi.finished = false;
    wi.omega0 = omega0;
    wi.delta = delta;
    wi.k_total = k;
    wi.omega_end = omega0 + delta;
    wi.k = (c->opt.select == 0) ? std::min(k, KCHUNK) : k;
    wi.iters = 0;
    wi.res = WindowResult();
    start_chunk(wi);
    return slot;
  }

  // fresh state, targets and block size for the current chunk: k roots from omega0 up
  void start_chunk(Window &wi) {
    wi.fresh = true;
    wi.iter0 = wi.iters;
    wi.m = 0;
    wi.adjust = 0;
    wi.stall = 0;
    wi.guard_wait = 0;
    wi.best_worst = 1e300;
    wi.bx = 0;
    wi.ndir = wi.nnew = 0;
    wi.prec = prec0;
    wi.tol = refine ? std::max(c->opt.res_tol, 1e-5) : c->opt.res_tol;
    if (c->opt.select == 1) {
      wi.shift = wi.omega0;
      wi.nev = wi.k + 2;
    } else {
      // centre the targets on the expected k lowest roots above omega0 (diagonal estimate)
      std::vector<double> above;
      for (long long p = 0; p < ov; ++p)
        if (ratio[p] >= wi.omega0) above.push_back(ratio[p]);
      std::sort(above.begin(), above.end());
      double rk = above.empty() ? wi.omega0 : above[std::min<size_t>(above.size() - 1, wi.k - 1)];
      wi.shift = wi.omega0 + 0.5 * (rk - wi.omega0);
      wi.nev = wi.k + std::max(2, wi.k / 2);
    }
    wi.nev = std::min<int>(wi.nev, (int)L);
    wi.b = std::min(bcap, std::max(wi.nev + 2, c->opt.block));
    wi.b = std::min<int>(wi.b, (int)L);
    wi.nev = std::min(wi.nev, wi.b);
  }

  bool finished(int slot) const { return W[slot].used && W[slot].finished; }

  WindowResult take(int slot) {
    Window &wi = W[slot];
    WindowResult r = std::move(wi.res);
    wi.used = wi.fresh = wi.finished = false;
    wi.res = WindowResult();
    wi.m = wi.ndir = wi.nnew = 0;
    return r;
  }

  void timed_sigma(int nv, const double *Z, double *Sg, double *Mt, int prec) {
    if (nv <= 0) return;
    float ms = 0.f;
    PP_CUDA(cudaEventRecord(c->ev0, s));
    apply_sigma(c, nv, Z, Sg, Mt, prec);
    PP_CUDA(cudaEventRecord(c->ev1, s));
    PP_CUDA(cudaEventSynchronize(c->ev1));
    PP_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
    c->st_sigma_ms += ms;
    c->st_sigvec += nv;
    ++sigma_calls;
  }

  // results of a window from its last extraction (the selection rules of pp_solve_window)
  void finalize(Window &wi, int status) {
    WindowResult r;  // this chunk
    r.status = status;
    r.iters = wi.iters;
    const int nb = (int)wi.order.size();
    std::vector<int> sel;
    if (c->opt.select == 1) {
      std::vector<int> cand;
      for (int j : wi.order)
        if (wi.h_res[j] <= kSpurRes) cand.push_back(j);
      std::stable_sort(cand.begin(), cand.end(), [&](int a, int b2) {
        double da = fabs(wi.h_theta[a] - wi.omega0), db = fabs(wi.h_theta[b2] - wi.omega0);
        return da < db || (da == db && wi.h_theta[a] < wi.h_theta[b2]);
      });
      for (int j = 0; j < (int)cand.size() && (int)sel.size() < wi.k; ++j) sel.push_back(cand[j]);
    } else {
      std::vector<int> in;
      for (int t = 0; t < nb; ++t) {
        int j = wi.order[t];
        if (wi.h_theta[j] >= wi.omega0 && wi.h_theta[j] <= wi.omega0 + wi.delta && wi.h_res[j] <= kSpurRes)
          in.push_back(j);
      }
      std::stable_sort(in.begin(), in.end(), [&](int a, int b2) { return wi.h_theta[a] < wi.h_theta[b2]; });
      for (int j = 0; j < (int)in.size() && (int)sel.size() < wi.k; ++j) sel.push_back(in[j]);
    }
    std::stable_sort(sel.begin(), sel.end(), [&](int a, int b2) { return wi.h_theta[a] < wi.h_theta[b2]; });
    const int nf = (int)sel.size();
    r.omega.assign(nf, 0.0);
    r.osc.assign(nf, 0.0);
    r.resid.assign(nf, 0.0);
    if (nf > 0) {
      std::vector<double> xs(nf);
      for (int t = 0; t < nf; ++t) {
        r.omega[t] = wi.h_theta[sel[t]];
        r.resid[t] = wi.h_res[sel[t]];
        xs[t] = wi.h_xsx[sel[t]];
      }
      // X columns are unit vectors (V orthonormal, refined coefficients normalised); the
      // direction buffer past the staged columns is free at this point of a step
      double *Dv = wi.Vr;  // reduced-block buffer of this window: 32 columns, free after extraction
      for (int t = 0; t < nf; ++t)
        PP_CUDA(cudaMemcpyAsync(Dv + (long long)t * L, wi.X + (long long)sel[t] * L, vecbytes,
                                cudaMemcpyDeviceToDevice, s));
      double *thd = scratch, *xsd = scratch + 64, *od = scratch + 128;
      PP_CUDA(cudaMemcpyAsync(thd, r.omega.data(), sizeof(double) * nf, cudaMemcpyHostToDevice, s));
      PP_CUDA(cudaMemcpyAsync(xsd, xs.data(), sizeof(double) * nf, cudaMemcpyHostToDevice, s));
      if (c->has_mu) {
        k_osc<<<nf, 256, 0, s>>>(Dv, c->mu.as<double>(), ov, thd, xsd, od);
        PP_LAUNCH_CHECK("k_osc");
        PP_CUDA(cudaMemcpyAsync(r.osc.data(), od, sizeof(double) * nf, cudaMemcpyDeviceToHost, s));
      }
      if (keep_vectors) {
        r.vecs.assign((size_t)nf * L, 0.0);
        PP_CUDA(cudaMemcpyAsync(r.vecs.data(), Dv, vecbytes * nf, cudaMemcpyDeviceToHost, s));
      }
      PP_CUDA(cudaStreamSynchronize(s));
      if (keep_vectors)
        for (int t = 0; t < nf; ++t) {
          const double sc = 1.0 / sqrt(fabs(xs[t]));
          double *vv = r.vecs.data() + (size_t)t * L;
          for (long long l = 0; l < L; ++l) vv[l] *= sc;
        }
    }
    // append this chunk; a full chunk of a larger request restarts above its last root (the
    // offset 2 res_tol keeps a root found again within its tolerance out of the next chunk)
    WindowResult &acc = wi.res;
    acc.status = status;
    acc.iters = wi.iters;
    acc.omega.insert(acc.omega.end(), r.omega.begin(), r.omega.end());
    acc.osc.insert(acc.osc.end(), r.osc.begin(), r.osc.end());
    acc.resid.insert(acc.resid.end(), r.resid.begin(), r.resid.end());
    acc.vecs.insert(acc.vecs.end(), r.vecs.begin(), r.vecs.end());
    const int got = (int)acc.omega.size();
    if (c->opt.select == 0 && status == PP_OK && nf == wi.k && got < wi.k_total) {
      const double start = acc.omega.back() + std::max(1e-9, 2.0 * c->opt.res_tol);
      if (start < wi.omega_end) {
        wi.omega0 = start;
        wi.delta = wi.omega_end - start;
        wi.k = std::min(KCHUNK, wi.k_total - got);
        start_chunk(wi);
        return;
      }
    }
    wi.finished = true;
  }

  // Rayleigh-Ritz, folded extraction, residuals, convergence and window coverage of one
  // window; stages its correction directions at column pos of D.  Returns the number staged.
  int extract(int w, long long pos) {
    Window &wi = W[w];
    const int m = wi.m;
    const int b = std::min(wi.b, m);
    wi.bx = b;
    // Rayleigh-Ritz on the projected pencil (full basis)
    sv.gram(wi.V, L, m, wi.MV, L, m, wi.Hm, m);
    sv.gram(wi.V, L, m, wi.SV, L, m, wi.Hs, m);
    PP_CUDA(cudaMemsetAsync(wi.dstat, 0, sizeof(int) * 4, s));
    k_chol_rr<<<1, 256, (m * (m + 1) + 2 * m) * sizeof(double), s>>>(wi.Hm, m, wi.Lm, wi.dinv, wi.dstat);
    PP_LAUNCH_CHECK("k_chol_rr");
    k_rr_trsm<<<(m + 3) / 4, 128, 0, s>>>(wi.Hs, wi.Lm, wi.dinv, m, 0, wi.Yw, wi.dstat);
    PP_LAUNCH_CHECK("k_rr_trsm");
    k_rr_trsm<<<(m + 3) / 4, 128, 0, s>>>(wi.Yw, wi.Lm, wi.dinv, m, 1, wi.Cw, wi.dstat);
    PP_LAUNCH_CHECK("k_rr_trsm");
    int mp = (m + 1) & ~1;
    if (sv.f64)
      k_jacobi_eig_f64<<<1, 512, 2 * mp * mp * sizeof(double), s>>>(wi.Cw, m, wi.mu, wi.W, 16);
    else
      k_jacobi_eig<<<1, 512, 2 * mp * (mp + 1) * sizeof(double), s>>>(wi.Cw, m, wi.mu, wi.W, 16);
    PP_LAUNCH_CHECK("k_jacobi_eig");
    const int nsel = std::min(m, std::max(b, std::min(64, 2 * b)));
    k_rr_select<<<1, 128, 0, s>>>(wi.Lm, wi.mu, wi.W, m, wi.shift, nsel, wi.Ew, wi.thsel, wi.Esel);
    PP_LAUNCH_CHECK("k_rr_select");
    // folded step in the span of the nr Rayleigh-Ritz vectors nearest the shift: orthonormal
    // coefficients Qr, reduced blocks V Qr^T, M V Qr^T, Sigma V Qr^T, and their small Grams
    const int nr = std::min(nsel, 32);
    k_mgs<<<1, RT, 0, s>>>(wi.Esel, m, nsel, nr, wi.Qr, wi.dkept, 0.0);
    PP_LAUNCH_CHECK("k_mgs");
    sv.combine(wi.V, m, wi.Qr, m, nr, wi.Vr, 1.0, 0.0);
    sv.combine(wi.MV, m, wi.Qr, m, nr, wi.MVr, 1.0, 0.0);
    sv.combine(wi.SV, m, wi.Qr, m, nr, wi.SVr, 1.0, 0.0);
    sv.gram(wi.Vr, L, nr, wi.MVr, L, nr, wi.hm, nr);
    sv.gram(wi.Vr, L, nr, wi.SVr, L, nr, wi.hs, nr);
    sv.gram(wi.MVr, L, nr, wi.MVr, L, nr, wi.Gmm, nr);
    sv.gram(wi.MVr, L, nr, wi.SVr, L, nr, wi.Gms, nr);
    sv.gram(wi.SVr, L, nr, wi.SVr, L, nr, wi.Gss, nr);
    {  // initial guesses in reduced coordinates: C0[j][p] = Esel_j . Qr_p
      GemmF64 g;
      g.M = b; g.N = nr; g.K = m;
      g.A = wi.Esel; g.a_m = m; g.a_k = 1;
      g.B = wi.Qr; g.b_k = 1; g.b_n = m;
      g.C = wi.C0; g.c_m = nr; g.c_n = 1;
      gemm_f64(g, s);
    }
    k_refined<<<1, RT, (5 * nr * (nr + 1) + b * nr + 3 * nr + 136) * sizeof(double), s>>>(
        wi.hm, wi.hs, wi.Gmm, wi.Gms, wi.Gss, nr, b, 4, wi.thsel, wi.C0, wi.Cred, wi.thref, wi.dstat);
    PP_LAUNCH_CHECK("k_refined");
    sv.combine(wi.Vr, nr, wi.Cred, nr, b, wi.X, 1.0, 0.0);
    sv.combine(wi.MVr, nr, wi.Cred, nr, b, wi.MX, 1.0, 0.0);
    sv.combine(wi.SVr, nr, wi.Cred, nr, b, wi.SX, 1.0, 0.0);
    {  // coefficients of the folded vectors in the full basis (thick restart): Cref = Cred Qr
      GemmF64 g;
      g.M = b; g.N = m; g.K = nr;
      g.A = wi.Cred; g.a_m = nr; g.a_k = 1;
      g.B = wi.Qr; g.b_k = m; g.b_n = 1;
      g.C = wi.Cref; g.c_m = m; g.c_n = 1;
      gemm_f64(g, s);
    }
    double *dots = scratch;  // [b][3]
    double *theta_d = scratch + 3 * 64;
    double *rn = scratch + 4 * 64;
    k_ritz_dots<<<b, 256, 0, s>>>(wi.X, wi.MX, wi.SX, L, dots);
    PP_LAUNCH_CHECK("k_ritz_dots");
    std::vector<double> hd(3 * b);
    int hstat[4];
    PP_CUDA(cudaMemcpyAsync(hd.data(), dots, sizeof(double) * 3 * b, cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaMemcpyAsync(hstat, wi.dstat, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    if (hstat[0] == 1)  // V^T M V not positive definite: M is not positive definite
      throw PPError(PP_EUNSTABLE, "projected M is not positive definite (unstable RPA problem)");
    wi.h_theta.assign(b, 0.0);
    wi.h_xsx.assign(b, 0.0);
    for (int j = 0; j < b; ++j) {
      wi.h_xsx[j] = hd[3 * j + 1] / hd[3 * j + 2];
      wi.h_theta[j] = hd[3 * j] / hd[3 * j + 1];
    }
    PP_CUDA(cudaMemcpyAsync(theta_d, wi.h_theta.data(), sizeof(double) * b, cudaMemcpyHostToDevice, s));
    double *Dcols = D.as<double>() + pos * L;
    k_resid_dir<<<b, 256, 0, s>>>(wi.X, wi.MX, wi.SX, theta_d, c->diagA.as<double>(), c->diagS.as<double>(), ov,
                                  c->opt.jacobi_floor, Dcols, rn);
    PP_LAUNCH_CHECK("k_resid_dir");
    std::vector<double> hr(b);
    PP_CUDA(cudaMemcpyAsync(hr.data(), rn, sizeof(double) * b, cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    wi.h_res.assign(b, 0.0);
    for (int j = 0; j < b; ++j) {
      double nx2 = hd[3 * j + 2];
      wi.h_res[j] = sqrt(hr[j] / nx2) / fabs(wi.h_xsx[j]);
    }
    wi.order.resize(b);
    std::iota(wi.order.begin(), wi.order.end(), 0);
    std::stable_sort(wi.order.begin(), wi.order.end(), [&](int a, int b2) {
      return fabs(wi.h_theta[a] - wi.shift) < fabs(wi.h_theta[b2] - wi.shift);
    });
    ++wi.iters;
    // the roots this window needs: the k lowest targets inside [omega0, omega0 + delta]
    // (select 0) or the k targets nearest omega0 (select 1); only they must meet the tolerance
    std::vector<int> need;
    if (c->opt.select == 1) {
      for (int t = 0; t < b && (int)need.size() < wi.k; ++t)
        if (wi.h_res[wi.order[t]] <= kSpurRes) need.push_back(wi.order[t]);
    } else {
      std::vector<int> in;
      for (int j = 0; j < b; ++j)
        if (wi.h_theta[j] >= wi.omega0 && wi.h_theta[j] <= wi.omega0 + wi.delta && wi.h_res[j] <= kSpurRes)
          in.push_back(j);
      std::sort(in.begin(), in.end(), [&](int a, int b2) { return wi.h_theta[a] < wi.h_theta[b2]; });
      for (int j = 0; j < (int)in.size() && (int)need.size() < wi.k; ++j) need.push_back(in[j]);
    }
    // select 0: keep the targets centred on the span [omega0, theta_k] of the roots the window
    // needs (theta_k the k-th lowest Ritz value inside it), so that the k-th root sits well
    // inside the target block rather than at its edge
    if (c->opt.select == 0 && (int)need.size() >= wi.k) {
      double thk = wi.omega0;
      for (int j : need) thk = std::max(thk, wi.h_theta[j]);
      wi.shift = 0.5 * (wi.omega0 + thk);
    }
    // guards: an unconverged target whose Ritz value, give or take three residuals, reaches
    // the span of the selected roots may still converge to a root inside it, so it must meet
    // the tolerance too before the window is reported (else roots can be missed)
    const int nsel_need = (int)need.size();
    if (nsel_need > 0) {
      double lo, hi;
      if (c->opt.select == 1) {
        double dk = 0.0;
        for (int j : need) dk = std::max(dk, fabs(wi.h_theta[j] - wi.omega0));
        lo = wi.omega0 - dk;
        hi = wi.omega0 + dk;
      } else {
        lo = wi.omega0;
        hi = wi.omega0;
        for (int j : need) hi = std::max(hi, wi.h_theta[j]);
        if (nsel_need < wi.k) hi = wi.omega0 + wi.delta;
      }
      // (only targets on their way to convergence: interior Rayleigh-Ritz also yields spurious
      // values with residuals of order 0.1 that never converge)
      for (int j = 0; j < b; ++j) {
        if (std::find(need.begin(), need.end(), j) != need.end()) continue;
        if (!(wi.h_res[j] <= 1e3 * wi.tol)) continue;
        const double r3 = 3.0 * wi.h_res[j];
        if (wi.h_theta[j] + r3 >= lo && wi.h_theta[j] - r3 <= hi) need.push_back(j);
      }
    }
    bool conv = !need.empty();
    bool conv_sel = nsel_need > 0;
    double worst = 0.0;
    for (int t = 0; t < (int)need.size(); ++t) {
      const int j = need[t];
      if (!(wi.h_res[j] <= wi.tol)) {
        conv = false;
        if (t < nsel_need) conv_sel = false;
      }
      worst = std::max(worst, wi.h_res[j]);
    }
    // guards that stay unconverged for many iterations while the selected roots have
    // converged are given up on
    if (!conv && conv_sel) {
      if (++wi.guard_wait > 20) conv = true;
    } else {
      wi.guard_wait = 0;
    }
    if (log_on) {
      std::fprintf(stderr, "[pp] it %d win %d m %d b %d nev %d prec %d shift %.6f stat %d,%d worst %.2e |",
                   wi.iters - 1, w, m, b, wi.nev, wi.prec, wi.shift, hstat[0], hstat[1], worst);
      for (int t = 0; t < wi.nev; ++t)
        std::fprintf(stderr, " %.6f(%.1e)", wi.h_theta[wi.order[t]], wi.h_res[wi.order[t]]);
      std::fprintf(stderr, "\n");
    }
    if (!conv && refine && wi.prec == PP_BF16) {
      // the BF16 phase ends when its residuals stop improving: the rest is left to the split form
      if (worst < 0.7 * wi.best_worst) {
        wi.best_worst = worst;
        wi.stall = 0;
      } else if (++wi.stall >= 8) {
        int below = 0;
        for (int j : need)
          if (wi.h_res[j] <= 1e-3) ++below;
        if (!need.empty() && 2 * below >= (int)need.size()) conv = true;
      }
    }
    if (conv) {
      bool ok = true;
      if (c->opt.select == 0) {
        double tmin = 1e300, tmax = -1e300;
        for (int j = 0; j < b; ++j) {
          tmin = std::min(tmin, wi.h_theta[j]);
          tmax = std::max(tmax, wi.h_theta[j]);
        }
        const bool low_covered = tmin <= wi.omega0;
        const bool top_ok = (nsel_need >= wi.k) || (tmax >= wi.omega0 + wi.delta);
        if (!low_covered) {
          ok = false;  // targets do not reach down to omega0: move the centre down
          wi.shift = std::max(wi.omega0, wi.shift - 0.5 * (tmin - wi.omega0) - 0.25 * (tmax - tmin));
        } else if (!top_ok) {
          ok = false;  // fewer than k in the window and the window is not covered: widen
          if (wi.b < bcap) {
            wi.nev = std::min(wi.nev + std::max(2, wi.k / 2), bcap - 2);
            wi.b = std::min(bcap, std::max(wi.b, wi.nev + 2));
          } else {
            wi.shift += 0.5 * (tmax - wi.shift);
          }
        }
        if (!ok && ++wi.adjust > 8) ok = true;  // report what has been found
      }
      if (ok) {
        if (refine && wi.prec == PP_BF16) {
          switch_to_split(wi);
        } else {
          finalize(wi, PP_OK);
        }
        return 0;
      }
    }
    if (wi.iters - wi.iter0 >= std::max(1, c->opt.max_iter)) {
      finalize(wi, PP_ENOTCONV);
      return 0;
    }
    if (!conv && refine && wi.prec == PP_BF16X3) {
      // the split form has a floor too (its products round the intermediates to 16-bit
      // significands): a window whose worst needed residual has not improved 1.4x in 30
      // iterations reports what it has as not converged instead of running to max_iter
      if (worst < 0.7 * wi.best_worst) {
        wi.best_worst = worst;
        wi.stall = 0;
      } else if (++wi.stall >= 30) {
        finalize(wi, PP_ENOTCONV);
        return 0;
      }
    }
    // columns that get a direction: every unconverged block column, except in the split
    // (refinement) phase, where the products cost three times as much and the roots the
    // window needs (with their guards) are already close: only those, unless all of them
    // have converged and the window still has to move or widen
    std::vector<int> sel;
    const bool refining = refine && wi.prec == PP_BF16X3;
    if (refining) {
      for (int j : need)
        if (!(wi.h_res[j] <= wi.tol)) sel.push_back(j);
      std::sort(sel.begin(), sel.end());
    }
    if (sel.empty())
      for (int j = 0; j < b; ++j)
        if (!(wi.h_res[j] <= wi.tol)) sel.push_back(j);
    wi.active.clear();
    int nd = 0;
    for (int j : sel) {  // ascending, so a column moves only towards the front
      if (nd != j)
        PP_CUDA(cudaMemcpyAsync(Dcols + (long long)nd * L, Dcols + (long long)j * L, vecbytes,
                                cudaMemcpyDeviceToDevice, s));
      wi.active.push_back(j);
      ++nd;
    }
    if (nd == 0) {
      // every block column has converged but the window is not covered yet: widen with the
      // next Rayleigh-Ritz vectors' residual directions on the following iteration
      wi.b = std::min(bcap, wi.b + 2);
    }
    return nd;
  }

  // refinement: restart the window on its folded target vectors and recompute their
  // products with the split (three-product) tensor-core sigma
  void switch_to_split(Window &wi) {
    const int m = wi.m, b = wi.bx;
    const int nsel = std::min(m, std::max(b, std::min(64, 2 * b)));
    PP_CUDA(cudaMemcpyAsync(wi.Kc, wi.Cref, sizeof(double) * b * m, cudaMemcpyDeviceToDevice, s));
    PP_CUDA(cudaMemcpyAsync(wi.Kc + (long long)b * m, wi.Esel, sizeof(double) * nsel * m,
                            cudaMemcpyDeviceToDevice, s));
    // the folded vectors of the block only: each kept vector costs a split-form product
    const int nout = std::min(64, std::min(m, b));
    k_mgs<<<1, RT, 0, s>>>(wi.Kc, m, b + nsel, nout, wi.Qk, wi.dkept, 1e-20);
    PP_LAUNCH_CHECK("k_mgs");
    int kept = 0;
    PP_CUDA(cudaMemcpyAsync(&kept, wi.dkept, sizeof(int), cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    sv.combine(wi.V, m, wi.Qk, m, kept, wi.X, 1.0, 0.0);
    PP_CUDA(cudaMemcpyAsync(wi.V, wi.X, vecbytes * kept, cudaMemcpyDeviceToDevice, s));
    wi.prec = PP_BF16X3;
    wi.tol = c->opt.res_tol;
    timed_sigma(kept, wi.V, wi.MV, wi.SV, wi.prec);
    wi.m = kept;
    wi.adjust = 0;
    wi.stall = 0;
    wi.guard_wait = 0;
    wi.best_worst = 1e300;
  }

  // thick restart when the basis would overflow, then block CGS2 of the staged directions
  // against the basis and Cholesky QR (twice) among them -- on the vectors alone; the
  // orthonormal survivors are packed at column gpos of D.  Products are formed afterwards, of
  // the survivors: the part of a direction left after orthogonalisation can be orders of
  // magnitude smaller than the direction, and differencing reduced-precision products would
  // amplify their rounding by that ratio.
  int orthonormalise(Window &wi, long long gpos) {
    const int nd = wi.ndir;
    const int b = wi.bx;
    if (wi.m + nd > m_max) {
      // thick restart: keep the folded vectors and the next Rayleigh-Ritz vectors
      const int keep = std::min(wi.m, std::max(2 * b, m_max - nd - b));
      const int m = wi.m;
      const int nsel = std::min(m, std::max(b, std::min(64, 2 * b)));
      PP_CUDA(cudaMemcpyAsync(wi.Kc, wi.Cref, sizeof(double) * b * m, cudaMemcpyDeviceToDevice, s));
      PP_CUDA(cudaMemcpyAsync(wi.Kc + (long long)b * m, wi.Esel, sizeof(double) * nsel * m,
                              cudaMemcpyDeviceToDevice, s));
      k_mgs<<<1, RT, 0, s>>>(wi.Kc, m, b + nsel, std::min(keep, 64), wi.Qk, wi.dkept, 1e-20);
      PP_LAUNCH_CHECK("k_mgs");
      int kept = 0;
      PP_CUDA(cudaMemcpyAsync(&kept, wi.dkept, sizeof(int), cudaMemcpyDeviceToHost, s));
      PP_CUDA(cudaStreamSynchronize(s));
      double *stage = wi.X + (long long)b * L;  // X is free after the directions: room for 64 - b
      if (kept > 64 - b) kept = 64 - b;
      sv.combine(wi.V, m, wi.Qk, m, kept, stage, 1.0, 0.0);
      PP_CUDA(cudaMemcpyAsync(wi.V, stage, vecbytes * kept, cudaMemcpyDeviceToDevice, s));
      sv.combine(wi.MV, m, wi.Qk, m, kept, stage, 1.0, 0.0);
      PP_CUDA(cudaMemcpyAsync(wi.MV, stage, vecbytes * kept, cudaMemcpyDeviceToDevice, s));
      sv.combine(wi.SV, m, wi.Qk, m, kept, stage, 1.0, 0.0);
      PP_CUDA(cudaMemcpyAsync(wi.SV, stage, vecbytes * kept, cudaMemcpyDeviceToDevice, s));
      wi.m = kept;
    }
    const int m0 = wi.m;
    double *Nv = D.as<double>() + wi.dpos * L;
    double *H = wi.Kc;   // [nd][m0]
    double *GN = wi.Qk;  // [nd][nd]
    double *Tq = wi.Yw;  // [nd][nd]
    int *kflag = (int *)(scratch + 6144);
    for (int pass = 0; pass < 2 && m0 > 0; ++pass) {
      sv.gram(Nv, L, nd, wi.V, L, m0, H, m0);  // H[j][k] = N_j . V_k
      sv.combine(wi.V, m0, H, m0, nd, Nv, -1.0, 1.0);
    }
    int nkeep = nd;
    for (int qr = 0; qr < 2 && nkeep > 0; ++qr) {
      sv.gram(Nv, L, nkeep, Nv, L, nkeep, GN, nkeep);
      k_cholqr<<<1, 32, 0, s>>>(GN, nkeep, qr == 0 ? 1e-14 : 1e-10, Tq, kflag);
      PP_LAUNCH_CHECK("k_cholqr");
      std::vector<int> hk(nkeep);
      PP_CUDA(cudaMemcpyAsync(hk.data(), kflag, sizeof(int) * nkeep, cudaMemcpyDeviceToHost, s));
      PP_CUDA(cudaStreamSynchronize(s));
      // orthonormalised block staged in X, the kept columns compacted back into place
      sv.combine(Nv, nkeep, Tq, nkeep, nkeep, wi.X, 1.0, 0.0);
      double *dst = (qr == 1) ? D.as<double>() + gpos * L : Nv;
      int w2 = 0;
      for (int j = 0; j < nkeep; ++j) {
        if (!hk[j]) continue;
        PP_CUDA(cudaMemcpyAsync(dst + (long long)w2 * L, wi.X + (long long)j * L, vecbytes,
                                cudaMemcpyDeviceToDevice, s));
        ++w2;
      }
      nkeep = w2;
    }
    return nkeep;
  }

  // unit vectors on the diagonal entries nearest the shift, at column gpos of D
  int initial_block(Window &wi, long long gpos) {
    std::vector<long long> ord(ov);
    std::iota(ord.begin(), ord.end(), 0);
    const long long nb = std::min<long long>(wi.b, ov);
    std::partial_sort(ord.begin(), ord.begin() + nb, ord.end(), [&](long long a, long long b2) {
      double da = fabs(ratio[a] - wi.shift), db = fabs(ratio[b2] - wi.shift);
      return da < db || (da == db && a < b2);
    });
    std::vector<int> hidx(wi.b);
    for (int j = 0; j < wi.b; ++j) hidx[j] = (int)(j < nb ? ord[j] : ov + ord[j - nb]);
    PP_CUDA(cudaMemcpyAsync(iscratch, hidx.data(), sizeof(int) * wi.b, cudaMemcpyHostToDevice, s));
    k_unit_vectors<<<dim3(64, wi.b), 256, 0, s>>>(D.as<double>() + gpos * L, L, iscratch, wi.b);
    PP_LAUNCH_CHECK("k_unit_vectors");
    PP_CUDA(cudaStreamSynchronize(s));  // hidx is released on return
    wi.fresh = false;
    return wi.b;
  }

  // One iteration of every unfinished window.  New vectors are grouped by precision phase
  // so that each group is one contiguous sigma batch.
  void step() {
    ++steps;
    const int groups[2] = {prec0, PP_BF16X3};
    const int ngroups = refine ? 2 : 1;
    long long start[2] = {0, 0}, end[2] = {0, 0};
    long long pos = 0;
    for (int g = 0; g < ngroups; ++g) {
      const int gp = groups[g];
      start[g] = pos;
      // extraction and directions of the windows with a basis, staged from column pos
      long long dpos = pos;
      for (int w = 0; w < cap; ++w) {
        Window &wi = W[w];
        if (!wi.used || wi.finished || wi.fresh || wi.prec != gp) continue;
        wi.ndir = 0;
        wi.nnew = 0;
        const int nd = extract(w, dpos);
        if (wi.finished || wi.prec != gp) continue;  // finished, or moved to the split phase
        wi.ndir = nd;
        wi.dpos = dpos;
        dpos += nd;
      }
      // restart / orthonormalise, survivors packed from column pos (never ahead of dpos)
      long long gpos = pos;
      for (int w = 0; w < cap; ++w) {
        Window &wi = W[w];
        if (!wi.used || wi.finished || wi.fresh || wi.prec != gp || wi.ndir == 0) continue;
        wi.nnew = orthonormalise(wi, gpos);
        wi.npos = gpos;
        gpos += wi.nnew;
      }
      // fresh windows of this phase: their initial blocks, right after the survivors (every
      // staged direction of the phase has been consumed by now)
      for (int w = 0; w < cap; ++w) {
        Window &wi = W[w];
        if (!wi.used || wi.finished || !wi.fresh || wi.prec != gp) continue;
        wi.nnew = initial_block(wi, gpos);
        wi.npos = gpos;
        wi.ndir = 0;
        gpos += wi.nnew;
      }
      end[g] = gpos;
      pos = gpos;
    }
    for (int g = 0; g < ngroups; ++g) {
      const long long n = end[g] - start[g];
      if (n > 0)
        timed_sigma((int)n, D.as<double>() + start[g] * L, MD.as<double>() + start[g] * L,
                    SD.as<double>() + start[g] * L, groups[g]);
    }
    for (int w = 0; w < cap; ++w) {
      Window &wi = W[w];
      if (!wi.used || wi.finished || wi.nnew == 0) continue;
      const long long at = (long long)wi.m * L, from = wi.npos * L;
      PP_CUDA(cudaMemcpyAsync(wi.V + at, D.as<double>() + from, vecbytes * wi.nnew, cudaMemcpyDeviceToDevice, s));
      PP_CUDA(cudaMemcpyAsync(wi.MV + at, MD.as<double>() + from, vecbytes * wi.nnew, cudaMemcpyDeviceToDevice, s));
      PP_CUDA(cudaMemcpyAsync(wi.SV + at, SD.as<double>() + from, vecbytes * wi.nnew, cudaMemcpyDeviceToDevice, s));
      wi.m += wi.nnew;
      wi.nnew = 0;
      wi.ndir = 0;
    }
  }
};

WindowBatch *window_batch(pp_ctx *c, int cap, bool vectors) {
  if (c->wb && (c->wb->cap < cap || c->wb->used() > 0)) {
    delete c->wb;
    c->wb = nullptr;
  }
  if (!c->wb) c->wb = new WindowBatch(c, cap, vectors);
  c->wb->keep_vectors = vectors;
  return c->wb;
}
WindowBatch *window_batch_new(pp_ctx *c, int cap, bool vectors) { return new WindowBatch(c, cap, vectors); }
void window_batch_destroy(WindowBatch *wb) { delete wb; }
void window_batch_release(WindowBatch *wb, int slot) { (void)wb->take(slot); }
int window_batch_add(WindowBatch *wb, double omega0, double delta, int k) { return wb->add(omega0, delta, k); }
bool window_batch_has_work(const WindowBatch *wb) { return wb->has_work(); }
void window_batch_step(WindowBatch *wb) { wb->step(); }
bool window_batch_finished(const WindowBatch *wb, int slot) { return wb->finished(slot); }
WindowResult window_batch_take(WindowBatch *wb, int slot) { return wb->take(slot); }
int window_batch_capacity(const WindowBatch *wb) { return wb->cap; }
size_t window_batch_bytes(const WindowBatch *wb) {
  return wb->mem.bytes + wb->D.bytes + wb->MD.bytes + wb->SD.bytes + wb->part.bytes + wb->small.bytes;
}
int window_batch_used(const WindowBatch *wb) { return wb->used(); }

pp_status solve_windows_impl(pp_ctx *c, int nwin, const double *omega0, const double *delta,
                             const int *kk, double *omega_out, double *osc_out, double *resid_out,
                             double *vecs_out, int *nfound) {
  window_run_destroy(c);  // a batch begun by pp_windows_begin and not collected is abandoned
  c->st_iters = 0;
  c->st_sigvec = 0;
  c->st_sigma_ms = 0.0;
  WindowBatch *wb = window_batch(c, nwin, vecs_out != nullptr);
  std::vector<int> slot(nwin);
  for (int w = 0; w < nwin; ++w) {
    slot[w] = wb->add(omega0[w], delta ? delta[w] : 0.0, kk[w]);
    if (slot[w] < 0) throw PPError(PP_ECUDA, "window slots exhausted");
  }
  const long long steps0 = wb->steps;
  try {
    while (wb->has_work()) wb->step();
  } catch (...) {
    for (int w = 0; w < nwin; ++w) wb->take(slot[w]);
    throw;
  }
  c->st_iters = (int)(wb->steps - steps0);
  pp_status st = PP_OK;
  long long base = 0;
  const long long L = 2 * c->ov;
  for (int w = 0; w < nwin; ++w) {
    WindowResult r = wb->take(slot[w]);
    if (r.status != PP_OK) st = (pp_status)r.status;
    const int nf = (int)r.omega.size();
    nfound[w] = nf;
    for (int t = 0; t < nf; ++t) {
      omega_out[base + t] = r.omega[t];
      osc_out[base + t] = r.osc[t];
      resid_out[base + t] = r.resid[t];
    }
    if (vecs_out && nf > 0) std::memcpy(vecs_out + base * L, r.vecs.data(), sizeof(double) * (size_t)nf * L);
    base += kk[w];
  }
  return st;
}

// ---------------------------------------------------------------------------
// a batch of windows driven one block iteration at a time (pp_windows_begin / step / end)
// ---------------------------------------------------------------------------
struct WindowRun {
  std::vector<int> slot, k;
  long long steps0 = 0;
};

void window_run_destroy(pp_ctx *c) {
  if (!c->run) return;
  if (c->wb)
    for (int sl : c->run->slot) c->wb->take(sl);
  delete c->run;
  c->run = nullptr;
}

pp_status windows_begin(pp_ctx *c, int nwin, const double *omega0, const double *delta, const int *kk) {
  window_run_destroy(c);
  c->st_iters = 0;
  c->st_sigvec = 0;
  c->st_sigma_ms = 0.0;
  WindowBatch *wb = window_batch(c, nwin, false);
  WindowRun *r = new WindowRun();
  c->run = r;
  r->steps0 = wb->steps;
  for (int w = 0; w < nwin; ++w) {
    const int sl = wb->add(omega0[w], delta[w], kk[w]);
    if (sl < 0) throw PPError(PP_ECUDA, "window slots exhausted");
    r->slot.push_back(sl);
    r->k.push_back(kk[w]);
  }
  return PP_OK;
}

pp_status windows_step(pp_ctx *c, int *unfinished, long long *sigma_vectors, int *sigma_calls) {
  if (!c->run || !c->wb) throw PPError(PP_EINVAL, "pp_windows_step: no windows begun");
  WindowBatch *wb = c->wb;
  const long long v0 = c->st_sigvec, k0 = wb->sigma_calls;
  if (wb->has_work()) wb->step();
  c->st_iters = (int)(wb->steps - c->run->steps0);
  int n = 0;
  for (int sl : c->run->slot) n += wb->finished(sl) ? 0 : 1;
  if (unfinished) *unfinished = n;
  if (sigma_vectors) *sigma_vectors = c->st_sigvec - v0;
  if (sigma_calls) *sigma_calls = (int)(wb->sigma_calls - k0);
  return PP_OK;
}

pp_status windows_end(pp_ctx *c, double *omega_out, double *osc_out, double *resid_out, int *nfound) {
  if (!c->run || !c->wb) throw PPError(PP_EINVAL, "pp_windows_end: no windows begun");
  WindowRun *r = c->run;
  for (int sl : r->slot)
    if (!c->wb->finished(sl)) throw PPError(PP_EINVAL, "pp_windows_end: windows still running (step until none is unfinished)");
  pp_status st = PP_OK;
  long long base = 0;
  for (size_t w = 0; w < r->slot.size(); ++w) {
    WindowResult res = c->wb->take(r->slot[w]);
    if (res.status != PP_OK) st = (pp_status)res.status;
    const int nf = (int)res.omega.size();
    nfound[w] = nf;
    for (int t = 0; t < nf; ++t) {
      omega_out[base + t] = res.omega[t];
      osc_out[base + t] = res.osc[t];
      resid_out[base + t] = res.resid[t];
    }
    base += r->k[w];
  }
  delete r;
  c->run = nullptr;
  return st;
}

// ---------------------------------------------------------------------------
// Contour (Riesz projector) solver, the alternative interior method of Sec. 4.4.
//
// The Riesz projector of the pencil onto the roots inside a circle Gamma around the window,
//   P = (1 / 2 pi i) oint_Gamma (z Sigma - M)^-1 Sigma dz,
// is applied to a block Y of m0 trial vectors with the trapezoidal rule on the circle
// z(theta) = c + rho e^{i theta}, c the window centre, rho half its width.  Conjugate points
// give conjugate solutions (M and Sigma are real), so with Nq points on the upper half,
//   P Y ~ (1 / Nq) Re sum_j rho e^{i theta_j} X_j,   (z_j Sigma - M) X_j = Sigma Y,
//   theta_j = pi (j + 1/2) / Nq,
// whose scalar filter is 1 at the centre and decays away from the circle.  Each complex
// system is complex symmetric; all Nq m0 of them are solved together by conjugate-orthogonal
// CG (unconjugated inner products) with the diagonal preconditioner diag(z_j Sigma - M), one
// sigma batch of their real and imaginary parts per iteration.  The filtered block is
// orthonormalised, multiplied with the accurate sigma and Rayleigh-Ritz'd (the projected
// pencil as in the window solver); the Ritz vectors are filtered again until every Ritz
// pair inside the window meets the tolerance (subspace iteration with a rational filter).
// Mixed contexts filter with the BF16 sigma (the filter's accuracy sets only the convergence
// rate) and take the Rayleigh-Ritz products and residuals with the split form.
// ---------------------------------------------------------------------------
namespace {

// per system s (complex vector s = real parts at 2s, imaginary parts at 2s + 1, each L long)
struct RzCoef {
  const double *zre, *zim;  // z_j per system
};
// q = z Sigma p - M p for every system (from the sigma and metric products of p)
__global__ void k_rz_apply(double *__restrict__ q, const double *__restrict__ MP, const double *__restrict__ SP,
                           const double *__restrict__ zre, const double *__restrict__ zim, long long L, int ns) {
  const long long total = (long long)ns * L;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(p / L);
    const long long e = p % L, re = 2LL * s * L + e, im = re + L;
    const double a = zre[s], b = zim[s];
    const double sr = SP[re], si = SP[im];
    q[re] = a * sr - b * si - MP[re];
    q[im] = a * si + b * sr - MP[im];
  }
}
// z = r / D, D = z_j diag(Sigma) - diag(M), diag(Sigma) = [dS; -dS], diag(M) = [dA; dA]
__global__ void k_rz_prec(double *__restrict__ z, const double *__restrict__ r, const double *__restrict__ dA,
                          const double *__restrict__ dS, const double *__restrict__ zre,
                          const double *__restrict__ zim, long long ov, int ns) {
  const long long L = 2 * ov, total = (long long)ns * L;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(p / L);
    const long long e = p % L, ia = e % ov, re = 2LL * s * L + e, im = re + L;
    const double sg = (e < ov) ? dS[ia] : -dS[ia];
    const double dr = zre[s] * sg - dA[ia], di = zim[s] * sg;
    const double den = dr * dr + di * di;
    const double xr = r[re], xi = r[im];
    z[re] = (xr * dr + xi * di) / den;
    z[im] = (xi * dr - xr * di) / den;
  }
}
// per system: out[3 s] = Re(a^T b), out[3 s + 1] = Im(a^T b) (no conjugation), out[3 s + 2] = |a|^2
__global__ void __launch_bounds__(256) k_rz_dot(const double *__restrict__ a, const double *__restrict__ b,
                                                long long L, double *__restrict__ out) {
  __shared__ double red[256];
  const long long re = 2LL * blockIdx.x * L, im = re + L;
  double sr = 0.0, si = 0.0, nn = 0.0;
  for (long long e = threadIdx.x; e < L; e += blockDim.x) {
    const double ar = a[re + e], ai = a[im + e], br = b[re + e], bi = b[im + e];
    sr += ar * br - ai * bi;
    si += ar * bi + ai * br;
    nn += ar * ar + ai * ai;
  }
  sr = block_sum(sr, red);
  si = block_sum(si, red);
  nn = block_sum(nn, red);
  if (threadIdx.x == 0) {
    out[3 * blockIdx.x] = sr;
    out[3 * blockIdx.x + 1] = si;
    out[3 * blockIdx.x + 2] = nn;
  }
}
// y += c x (complex c per system; c = (cf[2s], cf[2s+1])); mode 1: y = x + c y
__global__ void k_rz_axpy(double *__restrict__ y, const double *__restrict__ x, const double *__restrict__ cf,
                          long long L, int ns, int mode) {
  const long long total = (long long)ns * L;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(p / L);
    const long long e = p % L, re = 2LL * s * L + e, im = re + L;
    const double cr = cf[2 * s], ci = cf[2 * s + 1];
    if (mode == 0) {
      const double xr = x[re], xi = x[im];
      y[re] += cr * xr - ci * xi;
      y[im] += cr * xi + ci * xr;
    } else {
      const double yr = y[re], yi = y[im];
      y[re] = x[re] + cr * yr - ci * yi;
      y[im] = x[im] + cr * yi + ci * yr;
    }
  }
}
// right-hand sides: b_s = Sigma y_q (real), s = j m0 + q
__global__ void k_rz_rhs(double *__restrict__ bvec, const double *__restrict__ SY, long long L, int m0, int ns) {
  const long long total = (long long)ns * L;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(p / L);
    const long long e = p % L;
    bvec[2LL * s * L + e] = SY[(long long)(s % m0) * L + e];
    bvec[2LL * s * L + L + e] = 0.0;
  }
}
// Q_q = sum_j Re(w_j X_{j m0 + q}), w_j = rho e^{i theta_j} / Nq
__global__ void k_rz_accum(double *__restrict__ Qv, const double *__restrict__ X, const double *__restrict__ wre,
                           const double *__restrict__ wim, long long L, int m0, int nq) {
  const long long total = (long long)m0 * L;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(p / L);
    const long long e = p % L;
    double acc = 0.0;
    for (int j = 0; j < nq; ++j) {
      const long long re = 2LL * (j * m0 + q) * L + e;
      acc += wre[j] * X[re] - wim[j] * X[re + L];
    }
    Qv[p] = acc;
  }
}

inline unsigned rz_blocks(long long n) {
  return (unsigned)std::max<long long>(1, std::min<long long>((n + 255) / 256, 152LL * 16));
}

}  // namespace

pp_status riesz_impl(pp_ctx *c, double omega0, double delta, int nquad, int m0_req, int max_outer, double *omega_out,
                     double *osc_out, double *resid_out, int cap, int *nfound) {
  cudaStream_t s = c->stream;
  const long long ov = c->ov, L = 2 * ov;
  const double ctr = omega0 + 0.5 * delta, rad = 0.5 * delta;
  const bool mixed = c->opt.prec != PP_FP64;
  const int p_acc = mixed ? PP_BF16X3 : PP_FP64;
  // the filter projects onto the invariant subspace of the operator it applies: the BF16 one
  // stalls at its own operator error, so a mixed context filters with the split form once the
  // worst in-window residual gains less than 2x in an outer iteration
  int p_filter = mixed ? PP_BF16 : PP_FP64;
  double worst_prev = 0.0;
  // subspace size: 1.5 x the diagonal estimate of the roots in the window, plus a margin
  std::vector<double> hA(ov), hS(ov);
  PP_CUDA(cudaMemcpyAsync(hA.data(), c->diagA.p, sizeof(double) * ov, cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaMemcpyAsync(hS.data(), c->diagS.p, sizeof(double) * ov, cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaStreamSynchronize(s));
  std::vector<double> ratio(ov);
  int n_in = 0;
  for (long long p = 0; p < ov; ++p) {
    ratio[p] = hA[p] / hS[p];
    if (ratio[p] >= omega0 && ratio[p] <= omega0 + delta) ++n_in;
  }
  int m0 = m0_req > 0 ? m0_req : std::max(8, (3 * n_in + 1) / 2 + 4);
  m0 = std::min<int>(m0, (int)L);
  if (m0 > 64)
    throw PPError(PP_EINVAL, "pp_solve_window_contour: the window holds about " + std::to_string(n_in) +
                                 " roots; the contour solver's subspace is limited to 64 vectors (narrow the window)");
  const int nq = nquad;
  const int ns = nq * m0;
  // device memory: Y, MY, SY, Q, MQ, SQ (m0 each); complex x, r, z, p, q (2 ns each); sigma
  // outputs of the complex batch (2 ns each, M and Sigma); small matrices
  DevBuf mem;
  const size_t vec = sizeof(double) * (size_t)L;
  const size_t ndots = std::max<size_t>(3 * (size_t)ns, 8 * (size_t)MAXM);
  const size_t small = sizeof(double) * (9 * (size_t)MAXM * MAXM + 4 * (size_t)MAXM + 4 * (size_t)ns + ndots +
                                         2 * (size_t)nq + 128);
  mem.ensure(vec * (6 * (size_t)m0 + 14 * (size_t)ns) + small);
  double *Y = mem.as<double>(), *MY = Y + m0 * L, *SY = MY + m0 * L, *Qb = SY + m0 * L, *MQ = Qb + m0 * L,
         *SQ = MQ + m0 * L;
  double *X = SQ + m0 * L, *R = X + 2LL * ns * L, *Z = R + 2LL * ns * L, *P = Z + 2LL * ns * L,
         *Qc = P + 2LL * ns * L, *MP = Qc + 2LL * ns * L, *SP = MP + 2LL * ns * L;
  double *sm = SP + 2LL * ns * L;
  double *G = sm, *T = G + MAXM * MAXM, *Lm = T + MAXM * MAXM, *Cw = Lm + MAXM * MAXM, *Yw = Cw + MAXM * MAXM,
         *mu = Yw + MAXM * MAXM, *W = mu + MAXM, *Esel = W + MAXM * MAXM, *thsel = Esel + MAXM * MAXM,
         *dinv = thsel + MAXM, *Ew = dinv + MAXM;
  double *zre = Ew + MAXM * MAXM, *zim = zre + ns, *cf = zim + ns, *dots = cf + 2 * ns, *wre = dots + ndots,
         *wim = wre + nq;
  int *istat = reinterpret_cast<int *>(wim + nq);
  int *kept = istat + 8;
  Solver sv{c, s, L};
  DevBuf part;
  sv.part_elems = (size_t)296 * MAXM * MAXM;
  part.ensure(sizeof(double) * sv.part_elems);
  sv.part = part.as<double>();
  sv.f64 = true;
  // quadrature points and weights
  std::vector<double> hzr(ns), hzi(ns), hwr(nq), hwi(nq);
  for (int j = 0; j < nq; ++j) {
    const double th = 3.14159265358979323846 * (j + 0.5) / nq;
    hwr[j] = rad * std::cos(th) / nq;
    hwi[j] = rad * std::sin(th) / nq;
    for (int q = 0; q < m0; ++q) {
      hzr[j * m0 + q] = ctr + rad * std::cos(th);
      hzi[j * m0 + q] = rad * std::sin(th);
    }
  }
  PP_CUDA(cudaMemcpyAsync(zre, hzr.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
  PP_CUDA(cudaMemcpyAsync(zim, hzi.data(), sizeof(double) * ns, cudaMemcpyHostToDevice, s));
  PP_CUDA(cudaMemcpyAsync(wre, hwr.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, s));
  PP_CUDA(cudaMemcpyAsync(wim, hwi.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, s));
  // initial block: unit vectors on the diagonal entries nearest the window centre
  {
    std::vector<long long> ord(ov);
    std::iota(ord.begin(), ord.end(), 0);
    const long long nb = std::min<long long>(m0, ov);
    std::partial_sort(ord.begin(), ord.begin() + nb, ord.end(), [&](long long a, long long b2) {
      const double da = std::fabs(ratio[a] - ctr), db = std::fabs(ratio[b2] - ctr);
      return da < db || (da == db && a < b2);
    });
    std::vector<int> hidx(m0);
    for (int j = 0; j < m0; ++j) hidx[j] = (int)(j < nb ? ord[j] : ov + ord[j - nb]);
    PP_CUDA(cudaMemcpyAsync(kept, hidx.data(), sizeof(int) * m0, cudaMemcpyHostToDevice, s));
    k_unit_vectors<<<dim3(64, m0), 256, 0, s>>>(Y, L, kept, m0);
    PP_LAUNCH_CHECK("k_unit_vectors");
    PP_CUDA(cudaStreamSynchronize(s));
  }
  // inner tolerance: the outer residual settles near 2e-3 times it (CPU emulation); BF16 filters
  // cannot go much below 1e-4 (their operator error is ~1e-5), split and FP64 ones go to 1e-6
  const int max_in = 300;  // inner iterations per filter application (tens suffice here)
  std::vector<double> th_prev;
  std::vector<double> h_th, h_res, h_xsx;
  pp_status status = PP_ENOTCONV;
  int m = m0;
  std::vector<int> sel;
  for (int outer = 0; outer < max_outer; ++outer) {
    // ---- filter: solve (z_j Sigma - M) X_s = Sigma Y_q for all systems (COCG) -----------
    apply_sigma(c, m, Y, MY, SY, p_filter);  // Sigma Y (the metric product is exact in either form)
    k_rz_rhs<<<rz_blocks(ns * L), 256, 0, s>>>(R, SY, L, m0, ns);
    PP_LAUNCH_CHECK("k_rz_rhs");
    PP_CUDA(cudaMemsetAsync(X, 0, sizeof(double) * 2 * (size_t)ns * L, s));
    k_rz_prec<<<rz_blocks(ns * L), 256, 0, s>>>(Z, R, c->diagA.as<double>(), c->diagS.as<double>(), zre, zim, ov, ns);
    PP_LAUNCH_CHECK("k_rz_prec");
    PP_CUDA(cudaMemcpyAsync(P, Z, sizeof(double) * 2 * (size_t)ns * L, cudaMemcpyDeviceToDevice, s));
    std::vector<double> hd(3 * ns), bn(ns), rho_r(ns), rho_i(ns);
    auto dot_all = [&](const double *a, const double *b) {
      k_rz_dot<<<ns, 256, 0, s>>>(a, b, L, dots);
      PP_LAUNCH_CHECK("k_rz_dot");
      PP_CUDA(cudaMemcpyAsync(hd.data(), dots, sizeof(double) * 3 * ns, cudaMemcpyDeviceToHost, s));
      PP_CUDA(cudaStreamSynchronize(s));
    };
    dot_all(R, Z);
    for (int t = 0; t < ns; ++t) {
      rho_r[t] = hd[3 * t];
      rho_i[t] = hd[3 * t + 1];
      bn[t] = std::sqrt(hd[3 * t + 2]);
    }
    std::vector<char> done(ns, 0);
    std::vector<double> hc(2 * ns);
    for (int it = 0; it < max_in; ++it) {
      apply_sigma(c, 2 * ns, P, MP, SP, p_filter);
      k_rz_apply<<<rz_blocks(ns * L), 256, 0, s>>>(Qc, MP, SP, zre, zim, L, ns);
      PP_LAUNCH_CHECK("k_rz_apply");
      dot_all(P, Qc);  // sigma_t = p^T q
      for (int t = 0; t < ns; ++t) {
        const double dr = hd[3 * t], di = hd[3 * t + 1], den = dr * dr + di * di;
        if (done[t] || den == 0.0) {
          hc[2 * t] = hc[2 * t + 1] = 0.0;
          continue;
        }
        hc[2 * t] = (rho_r[t] * dr + rho_i[t] * di) / den;  // alpha = rho / sigma
        hc[2 * t + 1] = (rho_i[t] * dr - rho_r[t] * di) / den;
      }
      PP_CUDA(cudaMemcpyAsync(cf, hc.data(), sizeof(double) * 2 * ns, cudaMemcpyHostToDevice, s));
      k_rz_axpy<<<rz_blocks(ns * L), 256, 0, s>>>(X, P, cf, L, ns, 0);  // x += alpha p
      PP_LAUNCH_CHECK("k_rz_axpy");
      for (int t = 0; t < 2 * ns; ++t) hc[t] = -hc[t];
      PP_CUDA(cudaMemcpyAsync(cf, hc.data(), sizeof(double) * 2 * ns, cudaMemcpyHostToDevice, s));
      k_rz_axpy<<<rz_blocks(ns * L), 256, 0, s>>>(R, Qc, cf, L, ns, 0);  // r -= alpha q
      PP_LAUNCH_CHECK("k_rz_axpy");
      k_rz_prec<<<rz_blocks(ns * L), 256, 0, s>>>(Z, R, c->diagA.as<double>(), c->diagS.as<double>(), zre, zim, ov,
                                                  ns);
      PP_LAUNCH_CHECK("k_rz_prec");
      dot_all(R, Z);
      bool all = true;
      for (int t = 0; t < ns; ++t) {
        if (!done[t] && std::sqrt(hd[3 * t + 2]) > 0.0) {
          // |r| from the same reduction: |r|^2 is the third output of the (r, z) dot
          const double rn = std::sqrt(hd[3 * t + 2]);
          if (rn <= (p_filter == PP_BF16 ? 1e-4 : 1e-6) * bn[t]) done[t] = 1;
        }
        const double nr = hd[3 * t], ni = hd[3 * t + 1];
        const double den = rho_r[t] * rho_r[t] + rho_i[t] * rho_i[t];
        if (done[t] || den == 0.0) {
          hc[2 * t] = hc[2 * t + 1] = 0.0;
        } else {
          hc[2 * t] = (nr * rho_r[t] + ni * rho_i[t]) / den;  // beta = rho' / rho
          hc[2 * t + 1] = (ni * rho_r[t] - nr * rho_i[t]) / den;
        }
        rho_r[t] = nr;
        rho_i[t] = ni;
        all = all && done[t];
      }
      if (all) break;
      PP_CUDA(cudaMemcpyAsync(cf, hc.data(), sizeof(double) * 2 * ns, cudaMemcpyHostToDevice, s));
      k_rz_axpy<<<rz_blocks(ns * L), 256, 0, s>>>(P, Z, cf, L, ns, 1);  // p = z + beta p
      PP_LAUNCH_CHECK("k_rz_axpy");
    }
    k_rz_accum<<<rz_blocks(m0 * L), 256, 0, s>>>(Qb, X, wre, wim, L, m0, nq);
    PP_LAUNCH_CHECK("k_rz_accum");
    // ---- orthonormalise the filtered block (Cholesky QR twice), then its products ----------
    int nk = m0;
    for (int pass = 0; pass < 2 && nk > 0; ++pass) {
      sv.gram(Qb, L, nk, Qb, L, nk, G, nk);
      k_cholqr<<<1, 32, 0, s>>>(G, nk, pass == 0 ? 1e-14 : 1e-10, T, kept);
      PP_LAUNCH_CHECK("k_cholqr");
      std::vector<int> hk(nk);
      PP_CUDA(cudaMemcpyAsync(hk.data(), kept, sizeof(int) * nk, cudaMemcpyDeviceToHost, s));
      PP_CUDA(cudaStreamSynchronize(s));
      sv.combine(Qb, nk, T, nk, nk, Y, 1.0, 0.0);  // staged in Y
      int w2 = 0;
      for (int j = 0; j < nk; ++j) {
        if (!hk[j]) continue;
        PP_CUDA(cudaMemcpyAsync(Qb + (long long)w2 * L, Y + (long long)j * L, vec, cudaMemcpyDeviceToDevice, s));
        ++w2;
      }
      nk = w2;
    }
    if (nk == 0) throw PPError(PP_ECUDA, "pp_solve_window_contour: the filtered block vanished");
    m = nk;
    apply_sigma(c, m, Qb, MQ, SQ, p_acc);
    // ---- Rayleigh-Ritz on (Q^T M Q, Q^T Sigma Q): all m pairs, nearest the centre first ------
    sv.gram(Qb, L, m, MQ, L, m, G, m);      // Hm
    sv.gram(Qb, L, m, SQ, L, m, T, m);      // Hs
    PP_CUDA(cudaMemsetAsync(istat, 0, sizeof(int) * 4, s));
    k_chol_rr<<<1, 256, (m * (m + 1) + 2 * m) * sizeof(double), s>>>(G, m, Lm, dinv, istat);
    PP_LAUNCH_CHECK("k_chol_rr");
    k_rr_trsm<<<(m + 3) / 4, 128, 0, s>>>(T, Lm, dinv, m, 0, Yw, istat);
    PP_LAUNCH_CHECK("k_rr_trsm");
    k_rr_trsm<<<(m + 3) / 4, 128, 0, s>>>(Yw, Lm, dinv, m, 1, Cw, istat);
    PP_LAUNCH_CHECK("k_rr_trsm");
    const int mp = (m + 1) & ~1;
    k_jacobi_eig_f64<<<1, 512, 2 * mp * mp * sizeof(double), s>>>(Cw, m, mu, W, 16);
    PP_LAUNCH_CHECK("k_jacobi_eig");
    k_rr_select<<<1, 128, 0, s>>>(Lm, mu, W, m, ctr, m, Ew, thsel, Esel);
    PP_LAUNCH_CHECK("k_rr_select");
    // Ritz vectors (unit norm) and their products, in Y / MY / SY (the next block to filter)
    sv.combine(Qb, m, Esel, m, m, Y, 1.0, 0.0);
    sv.combine(MQ, m, Esel, m, m, MY, 1.0, 0.0);
    sv.combine(SQ, m, Esel, m, m, SY, 1.0, 0.0);
    k_ritz_dots<<<m, 256, 0, s>>>(Y, MY, SY, L, dots);
    PP_LAUNCH_CHECK("k_ritz_dots");
    std::vector<double> rd(3 * m);
    int hstat = 0;
    PP_CUDA(cudaMemcpyAsync(rd.data(), dots, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaMemcpyAsync(&hstat, istat, sizeof(int), cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    if (hstat) throw PPError(PP_EUNSTABLE, "projected M is not positive definite (unstable RPA problem)");
    h_th.assign(m, 0.0);
    h_xsx.assign(m, 0.0);
    for (int j = 0; j < m; ++j) {
      h_xsx[j] = rd[3 * j + 1] / rd[3 * j + 2];
      h_th[j] = rd[3 * j] / rd[3 * j + 1];
    }
    double *theta_d = dots + 3 * MAXM, *rn = theta_d + MAXM;
    PP_CUDA(cudaMemcpyAsync(theta_d, h_th.data(), sizeof(double) * m, cudaMemcpyHostToDevice, s));
    // residual norms (the direction output lands in the complex work buffer, unused)
    k_resid_dir<<<m, 256, 0, s>>>(Y, MY, SY, theta_d, c->diagA.as<double>(), c->diagS.as<double>(), ov,
                                  c->opt.jacobi_floor, X, rn);
    PP_LAUNCH_CHECK("k_resid_dir");
    std::vector<double> hr(m);
    PP_CUDA(cudaMemcpyAsync(hr.data(), rn, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
    PP_CUDA(cudaStreamSynchronize(s));
    h_res.assign(m, 0.0);
    for (int j = 0; j < m; ++j) h_res[j] = std::sqrt(hr[j] / rd[3 * j + 2]) / std::fabs(h_xsx[j]);
    sel.clear();
    for (int j = 0; j < m; ++j)
      if (h_th[j] >= omega0 && h_th[j] <= omega0 + delta) sel.push_back(j);
    bool conv = true;
    for (int j : sel) conv = conv && h_res[j] <= c->opt.res_tol;
    std::vector<double> th_now;
    for (int j : sel) th_now.push_back(h_th[j]);
    std::sort(th_now.begin(), th_now.end());
    double worst = 0.0;
    for (int j : sel) worst = std::max(worst, h_res[j]);
    if (const char *e = std::getenv("PP_LOG"); e && e[0] && e[0] != '0')
      std::fprintf(stderr, "[pp] contour it %d m %d in-window %zu worst %.2e filter %d\n", outer, m, sel.size(), worst,
                   p_filter);
    // converged: every Ritz value in the window meets the tolerance and the count is stable
    if (conv && th_now.size() == th_prev.size()) {
      status = PP_OK;
      break;
    }
    th_prev = th_now;
    if (p_filter == PP_BF16 && outer > 0 && worst > 0.5 * worst_prev) p_filter = PP_BF16X3;
    worst_prev = worst;
    if (m < m0) {  // refill the block to m0 with unit vectors (the filter needs m0 >= roots inside)
      PP_CUDA(cudaMemsetAsync(Y + (long long)m * L, 0, vec * (m0 - m), s));
    }
    m = m0;
  }
  // results: the Ritz pairs inside the window, ascending
  std::sort(sel.begin(), sel.end(), [&](int a, int b2) { return h_th[a] < h_th[b2]; });
  const int nf = (int)sel.size();
  *nfound = nf;
  if (nf > cap) {
    c->err = "pp_solve_window_contour: " + std::to_string(nf) + " roots in the window exceed k = " + std::to_string(cap);
    return PP_EINVAL;
  }
  if (nf > 0) {
    double *thd = dots, *xsd = dots + MAXM, *od = dots + 2 * MAXM;
    std::vector<double> th(nf), xs(nf);
    for (int t = 0; t < nf; ++t) {
      th[t] = h_th[sel[t]];
      xs[t] = h_xsx[sel[t]];
      PP_CUDA(cudaMemcpyAsync(Qb + (long long)t * L, Y + (long long)sel[t] * L, vec, cudaMemcpyDeviceToDevice, s));
    }
    PP_CUDA(cudaMemcpyAsync(thd, th.data(), sizeof(double) * nf, cudaMemcpyHostToDevice, s));
    PP_CUDA(cudaMemcpyAsync(xsd, xs.data(), sizeof(double) * nf, cudaMemcpyHostToDevice, s));
    std::vector<double> ho(nf, 0.0);
    if (c->has_mu) {
      k_osc<<<nf, 256, 0, s>>>(Qb, c->mu.as<double>(), ov, thd, xsd, od);
      PP_LAUNCH_CHECK("k_osc");
      PP_CUDA(cudaMemcpyAsync(ho.data(), od, sizeof(double) * nf, cudaMemcpyDeviceToHost, s));
    }
    PP_CUDA(cudaStreamSynchronize(s));
    for (int t = 0; t < nf; ++t) {
      omega_out[t] = th[t];
      osc_out[t] = ho[t];
      resid_out[t] = h_res[sel[t]];
    }
  }
  return status;
}
