// Tensor-core (tcgen05 / TMA / TMEM, sm_103a) form of the sigma product.
//
// Dominant contraction of Sec. 2.2's B(2) (and its ring/ladder parts):
//   P[(i,c), n] = sum_(j,d) t_ij^cd  C[n, (j,d)],   C = C_Q(V) for every (V, Q).
// The amplitudes are regenerated slab by slab on the tensor cores,
//   t_ij^cd = (sum_Q B_Qic B_Qjd - sum_Q B_Qjc B_Qid) / (e_i + e_j - e_c - e_d),
// with both products accumulated in TMEM by one CTA and combined in the
// epilogue (BF16 out), then consumed by a long-K BF16 GEMM whose FP32
// accumulator lives in TMEM.  Only one slab of t (a few occupied indices) is
// alive at any time, in an L2-sized staging buffer; t is never stored whole.
// Split-BF16 ("bf16x3") operands (hi + lo, three products) give products with 16-bit
// significands (about 2^-16 relative error each) for the refinement.
//
// Kernel structure (both kernels): 128 threads; warp 0 lane 0 issues TMA loads
// into a STAGES-deep ring of 128B-swizzled shared tiles, warp 1 lane 0 issues
// tcgen05.mma (M = 128, K = 16 per instruction) and commits each stage back to
// the producer; all four warps read the accumulator out of TMEM (tcgen05.ld,
// 32 lanes per warp).  Every mbarrier wait is bounded: on timeout the kernel
// raises an error flag, stops issuing, frees its TMEM and returns.
#include "pp_internal.h"
#include "sigma_terms.cuh"

#include <cuda.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

namespace tc {

// ---------------------------------------------------------------------------
// device helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// bounded wait on the given phase parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < (1u << 24); ++it) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(a), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row core groups 1024 B apart
__device__ __forceinline__ uint64_t sdesc(const void *p) {
  const uint64_t a = smem_u32(p);
  uint64_t d = 0;
  d |= (a >> 4) & 0x3FFFull;           // start address
  d |= (uint64_t)(16 >> 4) << 16;      // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
  d |= 1ull << 46;                     // descriptor version
  d |= 2ull << 61;                     // 128B swizzle
  return d;
}
// instruction descriptor: kind::f16, A/B BF16, D FP32, both K-major, M x N
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 32 consecutive FP32 columns of this warp's 32 TMEM lanes
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float *v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

constexpr int BM = 128, BK = 64;  // BK bf16 = 128 bytes = one swizzle atom row

// ---------------------------------------------------------------------------
// generic GEMM: C[M x N] (+)= alpha * sum_seg A_seg[M x K] B_seg[N x K]^T
// (A and B BF16 K-major via TMA; C FP32 row-major with leading dimension ldc)
// ---------------------------------------------------------------------------
struct alignas(64) GemmMaps {
  CUtensorMap a[3];
  CUtensorMap b[3];
};
// output element (row, col) goes to  (row / d_r) * s_r1 + (row % d_r) * s_r0
//                                   + (col / d_c) * s_c1 + (col % d_c) * s_c0
// as FP32 (C, optionally accumulated) or as a BF16 pair (Chi, and Clo = remainder if set)
struct GemmOut {
  long long d_r = 1LL << 40, s_r1 = 0, s_r0 = 0, d_c = 1LL << 40, s_c1 = 0, s_c0 = 1;
  float *C = nullptr;
  __nv_bfloat16 *Chi = nullptr, *Clo = nullptr;
  float alpha = 1.f;
  int accumulate = 0;
  // optional addend add_scale * (add_hi + add_lo)[row * add_ld + col], a BF16 pair in a
  // row-major layout of its own
  const __nv_bfloat16 *add_hi = nullptr, *add_lo = nullptr;
  long long add_ld = 0;
  float add_scale = 0.f;
};
struct GemmArgs {
  int M, N, nk, nseg;
  GemmOut out, out2;  // out2 is written too when out2.C or out2.Chi is set
  int *err;
  int ksplit = 1;     // > 1: blockIdx.z takes a share of the K steps and adds into out.C atomically
  int mt = 1, nt = 1; // M and N tiles; blockIdx.x enumerates them, M fastest
};
__device__ __forceinline__ void epi_store(const GemmOut &o, long long off, float x) {
  if (o.C) {
    o.C[off] = o.accumulate ? x + o.C[off] : x;
  } else {
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    o.Chi[off] = h;
    if (o.Clo) o.Clo[off] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}

__device__ __forceinline__ float addend(const GemmOut &o, long long aoff) {
  return o.add_scale * (__bfloat162float(o.add_hi[aoff]) + (o.add_lo ? __bfloat162float(o.add_lo[aoff]) : 0.f));
}
// 32 consecutive columns [col0, col0 + 32) of output row `row`: x = alpha acc (+ the addend)
// written as FP32 (optionally accumulated) or as a BF16 pair.  Columns that run contiguously
// (s_c0 == 1) in 16-byte-aligned groups go out 8 BF16 / 4 FP32 values per store.
__device__ __forceinline__ bool al16(const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15) == 0; }
__device__ void store_row32(const GemmOut &o, long long row, long long rbase, long long col0, const float *v,
                            int N) {
  const bool contig = o.s_c0 == 1 && (o.s_r0 % 8) == 0 && (o.s_r1 % 8) == 0 && (o.s_c1 % 8) == 0 &&
                      (o.d_c % 8) == 0 &&
                      (!o.add_hi || (al16(o.add_hi) && al16(o.add_lo) && (o.add_ld % 8) == 0));
  const long long abase = row * o.add_ld;
  if (!o.C && contig && al16(o.Chi) && al16(o.Clo)) {
    // a full chunk's addend is loaded before any of its stores, so that its eight 16-byte
    // loads are in flight together
    uint4 pah[4], pal[4];
    const bool pre = o.add_hi && col0 + 32 <= N;
    if (pre) {
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        pah[g] = *reinterpret_cast<const uint4 *>(o.add_hi + abase + col0 + 8 * g);
        pal[g] = o.add_lo ? *reinterpret_cast<const uint4 *>(o.add_lo + abase + col0 + 8 * g) : make_uint4(0, 0, 0, 0);
      }
    }
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      const long long col = col0 + 8 * g;
      if (col >= N) return;
      const long long off = rbase + (col / o.d_c) * o.s_c1 + (col % o.d_c);
      if (col + 8 > N) {  // ragged tail
        for (int q = 0; q < 8 && col + q < N; ++q)
          epi_store(o, off + q, o.alpha * v[8 * g + q] + (o.add_hi ? addend(o, abase + col + q) : 0.f));
        return;
      }
      float x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = o.alpha * v[8 * g + q];
      if (o.add_hi) {
        const uint4 ah = pre ? pah[g] : *reinterpret_cast<const uint4 *>(o.add_hi + abase + col);
        const uint4 al = pre ? pal[g]
                             : (o.add_lo ? *reinterpret_cast<const uint4 *>(o.add_lo + abase + col) : make_uint4(0, 0, 0, 0));
        const uint32_t hw[4] = {ah.x, ah.y, ah.z, ah.w}, lw[4] = {al.x, al.y, al.z, al.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float h0 = __uint_as_float(hw[q] << 16), h1 = __uint_as_float(hw[q] & 0xffff0000u);
          const float l0 = __uint_as_float(lw[q] << 16), l1 = __uint_as_float(lw[q] & 0xffff0000u);
          x[2 * q] += o.add_scale * (h0 + l0);
          x[2 * q + 1] += o.add_scale * (h1 + l1);
        }
      }
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const __nv_bfloat16 h0 = __float2bfloat16_rn(x[2 * q]), h1 = __float2bfloat16_rn(x[2 * q + 1]);
        const __nv_bfloat16 l0 = __float2bfloat16_rn(x[2 * q] - __bfloat162float(h0));
        const __nv_bfloat16 l1 = __float2bfloat16_rn(x[2 * q + 1] - __bfloat162float(h1));
        hw[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        lw[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
      }
      *reinterpret_cast<uint4 *>(o.Chi + off) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
      if (o.Clo) *reinterpret_cast<uint4 *>(o.Clo + off) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
    }
    return;
  }
  if (o.C && contig && al16(o.C) && !o.add_hi) {
    for (int g = 0; g < 8; ++g) {
      const long long col = col0 + 4 * g;
      if (col >= N) return;
      const long long off = rbase + (col / o.d_c) * o.s_c1 + (col % o.d_c);
      if (col + 4 > N) {
        for (int q = 0; q < 4 && col + q < N; ++q) epi_store(o, off + q, o.alpha * v[4 * g + q]);
        return;
      }
      float4 *dst = reinterpret_cast<float4 *>(o.C + off);
      float4 x = make_float4(o.alpha * v[4 * g], o.alpha * v[4 * g + 1], o.alpha * v[4 * g + 2], o.alpha * v[4 * g + 3]);
      if (o.accumulate) {
        const float4 y = *dst;
        x.x += y.x; x.y += y.y; x.z += y.z; x.w += y.w;
      }
      *dst = x;
    }
    return;
  }
  long long cb = col0 / o.d_c, cr = col0 % o.d_c;
  for (int j = 0; j < 32; ++j) {
    if (col0 + j >= N) return;
    const long long off = rbase + cb * o.s_c1 + cr * o.s_c0;
    epi_store(o, off, o.alpha * v[j] + (o.add_hi ? addend(o, abase + col0 + j) : 0.f));
    if (++cr == o.d_c) {
      cr = 0;
      ++cb;
    }
  }
}


template <int BN, int STAGES>
__global__ void __launch_bounds__(128, 1) k_gemm_bf16(const __grid_constant__ GemmMaps maps, GemmArgs args) {
  constexpr uint32_t A_BYTES = BM * BK * 2, B_BYTES = BN * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], acc_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // blockIdx.x walks the M tiles fastest: the CTAs resident at one time cover every M tile of
  // a few N tiles, so each B tile is fetched from DRAM once, and an A operand that fits in L2
  // (the host keeps the amplitude slab of a wide GEMM within 64 MB) is read from DRAM once
  const int m0 = (int)(blockIdx.x % (unsigned)args.mt) * BM, n0 = (int)(blockIdx.x / (unsigned)args.mt) * BN;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_bar, 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, BN);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const int total = args.nseg * args.nk;
  // this CTA's K steps (all of them unless the reduction is split across blockIdx.z; the host
  // keeps every share non-empty)
  const int kb0 = (int)((long long)total * blockIdx.z / args.ksplit);
  const int kb1 = (int)((long long)total * (blockIdx.z + 1) / args.ksplit);
  if (warp == 0 && lane == 0) {
    for (int kb = kb0; kb < kb1; ++kb) {
      const int s = (kb - kb0) % STAGES;
      const uint32_t ph = ((kb - kb0) / STAGES) & 1;
      if (!mbar_wait(&empty_bar[s], ph ^ 1)) {
        atomicExch(args.err, 1);
        abort_flag = 1;
        break;
      }
      const int seg = kb / args.nk, k = kb % args.nk;
      uint8_t *sa = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full_bar[s], STAGE_BYTES);
      tma_load_2d(sa, &maps.a[seg], k * BK, m0, &full_bar[s]);
      tma_load_2d(sa + A_BYTES, &maps.b[seg], k * BK, n0, &full_bar[s]);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(BM, BN);
    for (int kb = kb0; kb < kb1; ++kb) {
      const int s = (kb - kb0) % STAGES;
      const uint32_t ph = ((kb - kb0) / STAGES) & 1;
      if (!mbar_wait(&full_bar[s], ph)) {
        atomicExch(args.err, 2);
        abort_flag = 1;
        break;
      }
      tc_fence_after();
      uint8_t *sa = smem + s * STAGE_BYTES;
      const uint64_t ad = sdesc(sa), bd = sdesc(sa + A_BYTES);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k)
        mma_bf16(tmem, ad + 2 * k, bd + 2 * k, idesc, (kb > kb0 || k > 0) ? 1u : 0u);
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&acc_bar);
  }
  __syncwarp();
  const bool ok = mbar_wait(&acc_bar, 0);
  if (!ok && lane == 0) atomicExch(args.err, 3);
  tc_fence_after();
  if (ok) {
    const GemmOut &o = args.out;
    const GemmOut &o2 = args.out2;
    const bool two = (o2.C != nullptr) || (o2.Chi != nullptr);
    const int row = m0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    const long long rbase = (row / o.d_r) * o.s_r1 + (row % o.d_r) * o.s_r0;
    const long long rbase2 = two ? (row / o2.d_r) * o2.s_r1 + (row % o2.d_r) * o2.s_r0 : 0;
    for (int c0 = 0; c0 < BN; c0 += 32) {
      float v[32];
      tmem_ld32(trow + c0, v);
      if (row >= args.M) continue;
      const long long col = n0 + c0;
      if (args.ksplit > 1) {  // partial sums of a split reduction
        for (int jj = 0; jj < 32 && col + jj < args.N; ++jj) {
          const long long cc = col + jj;
          atomicAdd(o.C + rbase + (cc / o.d_c) * o.s_c1 + (cc % o.d_c) * o.s_c0, o.alpha * v[jj]);
        }
        continue;
      }
      store_row32(o, row, rbase, col, v, args.N);
      if (two) store_row32(o2, row, rbase2, col, v, args.N);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN);
}

// ---------------------------------------------------------------------------
// amplitude slab: T[(ii, c)][j*v + d] = t_{i j}^{c d}, i = i0 + ii, for c, d in 128-wide
// tiles.  Two accumulators: D1 = B_i[ct]^T B_j[dt], D2 = B_j[ct]^T B_i[dt], K = Q (padded).
// The TMA source is BovT[(i,c)][Q] (BF16, row stride ldq).
// ---------------------------------------------------------------------------
struct alignas(64) TgenMaps {
  CUtensorMap hi, lo;
};
struct TgenArgs {
  int o, v, nk, i0, ntile, nseg;  // ntile = ceil(v / 128); nseg 1 (hi.hi) or 3 (+ hi.lo + lo.hi)
  const double *eps;
  __nv_bfloat16 *Thi, *Tlo;  // Tlo may be null
  long long ldT;
  float *Tf;                  // optional FP32 copy [rows][ldf] (per-dot precompute)
  long long ldf;
  int *err;
};
template <int STAGES>
__global__ void __launch_bounds__(128, 1) k_tgen(const __grid_constant__ TgenMaps maps, TgenArgs args) {
  constexpr uint32_t TILE = BM * BK * 2, STAGE_BYTES = 4 * TILE;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  __shared__ __align__(8) uint64_t full_bar[STAGES], empty_bar[STAGES], acc_bar;
  __shared__ uint32_t tmem_slot;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ct = blockIdx.x / args.ntile, dt = blockIdx.x % args.ntile;
  const int j = blockIdx.y, ii = blockIdx.z, i = args.i0 + ii;
  const int v = args.v;
  const int c0 = ct * BM, d0 = dt * BM;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, 256);
  // the virtual orbital energies of this CTA's d tile, for the denominators of the epilogue
  // (FP32: this part issues FP64 at a small fraction of its FP32 rate, and the relative
  // error ~1e-7 of an FP32 denominator is far below the output's rounding)
  __shared__ float eps_d[BM];
  eps_d[threadIdx.x] = (d0 + (int)threadIdx.x < v) ? (float)args.eps[args.o + d0 + threadIdx.x] : 0.f;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const int total = args.nk * args.nseg;
  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < total; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!mbar_wait(&empty_bar[s], ph ^ 1)) {
        atomicExch(args.err, 11);
        break;
      }
      // segment 0: hi x hi, 1: hi x lo, 2: lo x hi
      const int seg = kb / args.nk;
      const CUtensorMap *ma = (seg == 2) ? &maps.lo : &maps.hi;
      const CUtensorMap *mb = (seg == 1) ? &maps.lo : &maps.hi;
      uint8_t *sa = smem + s * STAGE_BYTES;
      mbar_expect_tx(&full_bar[s], STAGE_BYTES);
      const int x = (kb % args.nk) * BK;
      tma_load_2d(sa, ma, x, i * v + c0, &full_bar[s]);             // A1 = B_i[ct]
      tma_load_2d(sa + TILE, mb, x, j * v + d0, &full_bar[s]);      // B1 = B_j[dt]
      tma_load_2d(sa + 2 * TILE, ma, x, j * v + c0, &full_bar[s]);  // A2 = B_j[ct]
      tma_load_2d(sa + 3 * TILE, mb, x, i * v + d0, &full_bar[s]);  // B2 = B_i[dt]
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_bf16(BM, BM);
    for (int kb = 0; kb < total; ++kb) {
      const int s = kb % STAGES;
      const uint32_t ph = (kb / STAGES) & 1;
      if (!mbar_wait(&full_bar[s], ph)) {
        atomicExch(args.err, 12);
        break;
      }
      tc_fence_after();
      uint8_t *sa = smem + s * STAGE_BYTES;
      const uint64_t a1 = sdesc(sa), b1 = sdesc(sa + TILE), a2 = sdesc(sa + 2 * TILE), b2 = sdesc(sa + 3 * TILE);
#pragma unroll
      for (int k = 0; k < BK / 16; ++k) {
        const uint32_t acc = (kb > 0 || k > 0) ? 1u : 0u;
        mma_bf16(tmem, a1 + 2 * k, b1 + 2 * k, idesc, acc);
        mma_bf16(tmem + BM, a2 + 2 * k, b2 + 2 * k, idesc, acc);
      }
      mma_commit(&empty_bar[s]);
    }
    mma_commit(&acc_bar);
  }
  __syncwarp();
  const bool ok = mbar_wait(&acc_bar, 0);
  if (!ok && lane == 0) atomicExch(args.err, 13);
  tc_fence_after();
  if (ok) {
    const int c = c0 + warp * 32 + lane;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    const int o = args.o;
    const float eij_c = (c < v) ? (float)(args.eps[i] + args.eps[j] - args.eps[o + c]) : 1.f;
    __nv_bfloat16 *hrow = args.Thi + ((long long)ii * v + c) * args.ldT + (long long)j * v;
    __nv_bfloat16 *lrow = args.Tlo ? args.Tlo + ((long long)ii * v + c) * args.ldT + (long long)j * v : nullptr;
    float *frow = args.Tf ? args.Tf + ((long long)ii * v + c) * args.ldf + (long long)j * v : nullptr;
    // full 32-column chunks go out 8 BF16 (or 4 FP32) values per 16-byte store; v % 8 == 0
    // keeps every such chunk 16-byte aligned (ldT and ldf are multiples of 8 and of 4)
    const bool vec = (v % 8) == 0 && (args.ldT % 8) == 0 && (!frow || (args.ldf % 4) == 0);
    for (int cc = 0; cc < BM; cc += 32) {
      float d1[32], d2[32];
      tmem_ld32(trow + cc, d1);
      tmem_ld32(trow + BM + cc, d2);
      if (c < v && vec && d0 + cc + 32 <= v) {
        float t[32];
#pragma unroll
        for (int q = 0; q < 32; ++q) t[q] = __fdividef(d1[q] - d2[q], eij_c - eps_d[cc + q]);
        const int dbase = d0 + cc;
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const float x0 = t[8 * g + 2 * q], x1 = t[8 * g + 2 * q + 1];
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
            hw[q] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            lw[q] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
          }
          *reinterpret_cast<uint4 *>(hrow + dbase + 8 * g) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          if (lrow) *reinterpret_cast<uint4 *>(lrow + dbase + 8 * g) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        if (frow)
#pragma unroll
          for (int g = 0; g < 8; ++g)
            *reinterpret_cast<float4 *>(frow + dbase + 4 * g) =
                make_float4(t[4 * g], t[4 * g + 1], t[4 * g + 2], t[4 * g + 3]);
      } else if (c < v) {
#pragma unroll
        for (int q = 0; q < 32; ++q) {
          const int d = d0 + cc + q;
          if (d < v) {
            const float t = __fdividef(d1[q] - d2[q], eij_c - eps_d[cc + q]);
            const __nv_bfloat16 h = __float2bfloat16_rn(t);
            hrow[d] = h;
            if (lrow) lrow[d] = __float2bfloat16_rn(t - __bfloat162float(h));
            if (frow) frow[d] = t;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 256);
}

// ---------------------------------------------------------------------------
// amplitude slab, persistent form used by the sigma product.
//
// The exchange integral of t_ij^cd is the direct integral of t_ij^dc, so the amplitudes
// are antisymmetric in (c, d): t_ij^dc = -t_ij^cd.  One work item is an (i, j) pair and an
// unordered pair of 128-wide virtual tiles (ct <= dt).  Its two accumulators are
//   D1[c][d] = sum_Q B_Qic B_Qjd,   D2[c][d] = sum_Q B_Qjc B_Qid      (c in ct, d in dt),
// t[c][d] = (D1 - D2)[c][d] / (e_i + e_j - e_c - e_d) is written as tile (ct, dt), and for
// ct < dt its negated transpose as tile (dt, ct) -- through shared memory, so that every
// row still leaves in 16-byte stores.  Half of the off-diagonal tile products of the
// two-accumulator-per-tile form are saved.
//
// Warp roles (192 threads, one CTA per SM, persistent over the items):
//   warp 0 lane 0  TMA producer, 2-stage ring of the four 128 x 64 operand tiles;
//   warp 1 lane 0  MMA issuer; two TMEM accumulator pairs (512 columns), so the epilogue
//                  of one item overlaps the main loop of the next;
//   warps 2-5      epilogue (warp w reads TMEM lanes 32 (w % 4) ...): denominators in FP32
//                  (relative error ~1e-7, far below the BF16 and BF16-pair roundings),
//                  BF16 (pair) stores of tile (ct, dt), the transposed tile via shared memory.
// Every mbarrier wait is bounded; after a timeout the CTA sets the error flag, skips the
// remaining work (the epilogue warps still pass the same named barriers) and frees TMEM.
// ---------------------------------------------------------------------------
struct TgenPArgs {
  int o, v, nk, i0, ni, nt, npairs, nseg;
  long long nitems;          // ni * o * npairs
  const float *eps;          // orbital energies (FP32 copy)
  __nv_bfloat16 *Thi, *Tlo;  // Tlo may be null (BF16 form)
  long long ldT;
  int *err;
};
constexpr int TGP_STAGES = 2;
constexpr uint32_t TGP_TILE = BM * BK * 2, TGP_STAGE = 4 * TGP_TILE;
constexpr int TGP_XLD = 132;  // words per row of the transpose buffer (128 + 4: conflict-free)
constexpr size_t tgenp_smem() { return (size_t)TGP_STAGES * TGP_STAGE + (size_t)BM * TGP_XLD * 4 + 1024; }

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void epi_bar() { asm volatile("bar.sync 1, 128;" ::: "memory"); }
// item -> (ii, j, ct, dt), pairs enumerated row by row of the upper triangle ct <= dt
__device__ __forceinline__ void tgp_item(const TgenPArgs &a, long long item, int &ii, int &j, int &ct, int &dt) {
  const int p = (int)(item % a.npairs);
  const long long ij = item / a.npairs;
  j = (int)(ij % a.o);
  ii = (int)(ij / a.o);
  int r = 0, rem = p;
  while (rem >= a.nt - r) {
    rem -= a.nt - r;
    ++r;
  }
  ct = r;
  dt = r + rem;
}

__global__ void __launch_bounds__(192, 1) k_tgen_p(const __grid_constant__ TgenMaps maps, TgenPArgs args) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint32_t *xbuf = reinterpret_cast<uint32_t *>(smem + TGP_STAGES * TGP_STAGE);
  __shared__ __align__(8) uint64_t full_bar[TGP_STAGES], empty_bar[TGP_STAGES], accf[2], acce[2], done_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ float eps_s[BM];
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TGP_STAGES; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 4);
    }
    mbar_init(&done_bar, 1);
    abort_flag = 0;
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(&tmem_slot, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const int steps = args.nk * args.nseg;
  const int v = args.v, o = args.o;
  if (warp == 0) {
    if (lane == 0) {
      long long kb = 0;
      for (long long item = blockIdx.x; item < args.nitems && !abort_flag; item += gridDim.x) {
        int ii, j, ct, dt;
        tgp_item(args, item, ii, j, ct, dt);
        const int i = args.i0 + ii, c0 = ct * BM, d0 = dt * BM;
        for (int st = 0; st < steps; ++st, ++kb) {
          const int s = (int)(kb % TGP_STAGES);
          const uint32_t ph = (uint32_t)((kb / TGP_STAGES) & 1);
          if (!mbar_wait(&empty_bar[s], ph ^ 1)) {
            atomicExch(args.err, 21);
            abort_flag = 1;
            break;
          }
          // segment 0: hi x hi, 1: hi x lo, 2: lo x hi
          const int seg = st / args.nk, x = (st % args.nk) * BK;
          const CUtensorMap *ma = (seg == 2) ? &maps.lo : &maps.hi;
          const CUtensorMap *mb = (seg == 1) ? &maps.lo : &maps.hi;
          uint8_t *sa = smem + s * TGP_STAGE;
          mbar_expect_tx(&full_bar[s], TGP_STAGE);
          tma_load_2d(sa, ma, x, i * v + c0, &full_bar[s]);                 // B_i[ct]
          tma_load_2d(sa + TGP_TILE, mb, x, j * v + d0, &full_bar[s]);      // B_j[dt]
          tma_load_2d(sa + 2 * TGP_TILE, ma, x, j * v + c0, &full_bar[s]);  // B_j[ct]
          tma_load_2d(sa + 3 * TGP_TILE, mb, x, i * v + d0, &full_bar[s]);  // B_i[dt]
        }
      }
      // before the CTA can exit, every load it issued must have landed (bounded waits)
      for (long long k2 = kb > TGP_STAGES ? kb - TGP_STAGES : 0; k2 < kb; ++k2)
        mbar_wait(&full_bar[k2 % TGP_STAGES], (uint32_t)((k2 / TGP_STAGES) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16(BM, BM);
      long long kb = 0;
      int it = 0;
      for (long long item = blockIdx.x; item < args.nitems && !abort_flag; item += gridDim.x, ++it) {
        const int b = it & 1;
        const uint32_t use = (uint32_t)(it >> 1);
        if (!mbar_wait(&acce[b], (use & 1) ^ 1)) {
          atomicExch(args.err, 22);
          abort_flag = 1;
          break;
        }
        tc_fence_after();
        const uint32_t d1 = tmem + b * 256, d2 = d1 + BM;
        bool ok = true;
        for (int st = 0; st < steps; ++st, ++kb) {
          const int s = (int)(kb % TGP_STAGES);
          const uint32_t ph = (uint32_t)((kb / TGP_STAGES) & 1);
          if (!mbar_wait(&full_bar[s], ph)) {
            atomicExch(args.err, 23);
            abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          uint8_t *sa = smem + s * TGP_STAGE;
          const uint64_t a1 = sdesc(sa), b1 = sdesc(sa + TGP_TILE), a2 = sdesc(sa + 2 * TGP_TILE),
                         b2 = sdesc(sa + 3 * TGP_TILE);
#pragma unroll
          for (int k = 0; k < BK / 16; ++k) {
            const uint32_t acc = (st > 0 || k > 0) ? 1u : 0u;
            mma_bf16(d1, a1 + 2 * k, b1 + 2 * k, idesc, acc);
            mma_bf16(d2, a2 + 2 * k, b2 + 2 * k, idesc, acc);
          }
          mma_commit(&empty_bar[s]);
        }
        if (!ok) break;
        mma_commit(&accf[b]);
      }
      // every MMA issued has completed before TMEM is freed (bounded wait)
      mma_commit(&done_bar);
      mbar_wait(&done_bar, 0);
    }
    __syncwarp();
  } else {
    // epilogue: 128 threads; TMEM lane quarter q = warp % 4, tile row r = 32 q + lane
    const int et = threadIdx.x - 64;  // 0..127
    const int q = warp & 3, r = 32 * q + lane;
    const uint32_t lane_off = (uint32_t)(32 * q) << 16;
    const bool vec = (v % 8) == 0 && (args.ldT % 8) == 0;
    int it = 0;
    for (long long item = blockIdx.x; item < args.nitems; item += gridDim.x, ++it) {
      int ii, j, ct, dt;
      tgp_item(args, item, ii, j, ct, dt);
      const int i = args.i0 + ii, c0 = ct * BM, d0 = dt * BM;
      const int b = it & 1;
      const uint32_t use = (uint32_t)(it >> 1);
      const bool xpose = ct != dt;
      epi_bar();  // the previous item's readers of eps_s and of the transpose buffer are done
      eps_s[et] = (d0 + et < v) ? args.eps[o + d0 + et] : 0.f;
      epi_bar();
      bool ok = __all_sync(0xffffffffu, !abort_flag);
      if (ok && !mbar_wait(&accf[b], use & 1)) {
        if (lane == 0) atomicExch(args.err, 24);
        abort_flag = 1;
        ok = false;
      }
      ok = __all_sync(0xffffffffu, ok);  // warp-uniform: tcgen05.ld is a warp-wide instruction
      tc_fence_after();
      const int c = c0 + r;
      if (ok) {
        const float eij_c = (c < v) ? (float)((double)args.eps[i] + (double)args.eps[j] - (double)args.eps[o + c]) : 1.f;
        __nv_bfloat16 *hrow = args.Thi + ((long long)ii * v + c) * args.ldT + (long long)j * v;
        __nv_bfloat16 *lrow = args.Tlo ? args.Tlo + ((long long)ii * v + c) * args.ldT + (long long)j * v : nullptr;
        const uint32_t t1 = tmem + lane_off + b * 256, t2 = t1 + BM;
        for (int cc = 0; cc < BM; cc += 32) {
          float a1[32], a2[32];
          tmem_ld32(t1 + cc, a1);
          tmem_ld32(t2 + cc, a2);
          uint32_t hw[16], lw[16];
#pragma unroll
          for (int q2 = 0; q2 < 16; ++q2) {
            const float x0 = __fdividef(a1[2 * q2] - a2[2 * q2], eij_c - eps_s[cc + 2 * q2]);
            const float x1 = __fdividef(a1[2 * q2 + 1] - a2[2 * q2 + 1], eij_c - eps_s[cc + 2 * q2 + 1]);
            const __nv_bfloat16 h0 = __float2bfloat16_rn(x0), h1 = __float2bfloat16_rn(x1);
            const __nv_bfloat16 l0 = __float2bfloat16_rn(x0 - __bfloat162float(h0));
            const __nv_bfloat16 l1 = __float2bfloat16_rn(x1 - __bfloat162float(h1));
            hw[q2] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
            lw[q2] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
          }
          if (c < v) {
            const int dbase = d0 + cc;
            if (vec && dbase + 32 <= v) {
#pragma unroll
              for (int g = 0; g < 4; ++g) {
                *reinterpret_cast<uint4 *>(hrow + dbase + 8 * g) =
                    make_uint4(hw[4 * g], hw[4 * g + 1], hw[4 * g + 2], hw[4 * g + 3]);
                if (lrow)
                  *reinterpret_cast<uint4 *>(lrow + dbase + 8 * g) =
                      make_uint4(lw[4 * g], lw[4 * g + 1], lw[4 * g + 2], lw[4 * g + 3]);
              }
            } else {
#pragma unroll
              for (int q2 = 0; q2 < 32; ++q2) {
                if (dbase + q2 < v) {
                  const uint32_t h = (q2 & 1) ? (hw[q2 >> 1] >> 16) : (hw[q2 >> 1] & 0xffffu);
                  const uint32_t l = (q2 & 1) ? (lw[q2 >> 1] >> 16) : (lw[q2 >> 1] & 0xffffu);
                  hrow[dbase + q2] = __ushort_as_bfloat16((unsigned short)h);
                  if (lrow) lrow[dbase + q2] = __ushort_as_bfloat16((unsigned short)l);
                }
              }
            }
          }
          if (xpose) {  // word (hi | lo << 16) of t[c][d] at xbuf[d_local][c_local]
#pragma unroll
            for (int q2 = 0; q2 < 32; ++q2) {
              const uint32_t h = (q2 & 1) ? (hw[q2 >> 1] >> 16) : (hw[q2 >> 1] & 0xffffu);
              const uint32_t l = (q2 & 1) ? (lw[q2 >> 1] >> 16) : (lw[q2 >> 1] & 0xffffu);
              xbuf[(cc + q2) * TGP_XLD + r] = h | (l << 16);
            }
          }
        }
      }
      // hand the accumulator pair back to the MMA issuer
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&acce[b]);
      if (xpose) {
        epi_bar();
        // thread et writes row d = d0 + et of tile (dt, ct): T[(ii, d)][(j, c)] = -t[c][d]
        const int d = d0 + et;
        if (ok && d < v) {
          __nv_bfloat16 *hrow = args.Thi + ((long long)ii * v + d) * args.ldT + (long long)j * v;
          __nv_bfloat16 *lrow = args.Tlo ? args.Tlo + ((long long)ii * v + d) * args.ldT + (long long)j * v : nullptr;
          const uint32_t *xr = xbuf + et * TGP_XLD;
          for (int g = 0; g < BM / 8; ++g) {
            const int cb = c0 + 8 * g;
            if (cb >= v) break;
            const uint4 w0 = *reinterpret_cast<const uint4 *>(xr + 8 * g);
            const uint4 w1 = *reinterpret_cast<const uint4 *>(xr + 8 * g + 4);
            const uint32_t ws[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
            if (vec && cb + 8 <= v) {
              uint32_t hh[4], ll[4];
#pragma unroll
              for (int p2 = 0; p2 < 4; ++p2) {
                hh[p2] = __byte_perm(ws[2 * p2], ws[2 * p2 + 1], 0x5410) ^ 0x80008000u;
                ll[p2] = __byte_perm(ws[2 * p2], ws[2 * p2 + 1], 0x7632) ^ 0x80008000u;
              }
              *reinterpret_cast<uint4 *>(hrow + cb) = make_uint4(hh[0], hh[1], hh[2], hh[3]);
              if (lrow) *reinterpret_cast<uint4 *>(lrow + cb) = make_uint4(ll[0], ll[1], ll[2], ll[3]);
            } else {
#pragma unroll
              for (int p2 = 0; p2 < 8; ++p2) {
                if (cb + p2 < v) {
                  hrow[cb + p2] = __ushort_as_bfloat16((unsigned short)((ws[p2] & 0xffffu) ^ 0x8000u));
                  if (lrow) lrow[cb + p2] = __ushort_as_bfloat16((unsigned short)((ws[p2] >> 16) ^ 0x8000u));
                }
              }
            }
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// ---------------------------------------------------------------------------
// conversions
// ---------------------------------------------------------------------------
// dst[r][k] (row stride ldd, zero for k >= ncol) = bf16 hi (or lo remainder) of src[r][k]
template <class S>
__global__ void k_to_bf16(const S *__restrict__ src, long long rows, long long ncol, long long lds,
                          __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo, long long ldd) {
  const long long total = rows * ldd;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    long long r = p / ldd, k = p % ldd;
    float x = (k < ncol) ? (float)src[r * lds + k] : 0.f;
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[p] = h;
    if (lo) lo[p] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}
// BovT[(i,a)][Q] (row stride ldq, zero padded) from Bov[Q][i][a] (double)
__global__ void k_bovT(const double *__restrict__ Bov, int Q, long long ov, __nv_bfloat16 *__restrict__ hi,
                       __nv_bfloat16 *__restrict__ lo, long long ldq) {
  const long long total = ov * ldq;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    long long ia = p / ldq, q = p % ldq;
    float x = (q < Q) ? (float)Bov[q * ov + ia] : 0.f;
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[p] = h;
    if (lo) lo[p] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}
// dst[a][c][q] = src[q][c][a] for q < Q (zero for Q <= q < Qp); src [Q][n1][n2] double, dst [n2][n1][Qp]
__global__ void k_perm_qlast(const double *__restrict__ src, int Q, int n1, int n2, long long Qp,
                             __nv_bfloat16 *__restrict__ hi, __nv_bfloat16 *__restrict__ lo) {
  const long long total = (long long)n2 * n1 * Qp;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    long long a = p / ((long long)n1 * Qp), rem = p % ((long long)n1 * Qp);
    long long c = rem / Qp, q = rem % Qp;
    float x = (q < Q) ? (float)src[(q * n1 + c) * n2 + a] : 0.f;
    __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[p] = h;
    lo[p] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}
__global__ void k_d2f(const double *__restrict__ s, float *__restrict__ d, long long n) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x)
    d[p] = (float)s[p];
}

// vT[(r,b)][k] = V[r][k][b] (k < o; zero up to ldk), V double [R][o][v], as a BF16 pair
__global__ void k_vT(const double *__restrict__ V, int R, int o, int v, long long ldk, __nv_bfloat16 *__restrict__ hi,
                     __nv_bfloat16 *__restrict__ lo) {
  const long long total = (long long)R * v * ldk;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const long long rb = p / ldk, k = p % ldk;
    const long long r = rb / v, b = rb % v;
    const float x = (k < o) ? (float)V[(r * o + k) * v + b] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[p] = h;
    if (lo) lo[p] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}
// bvvK[a][Q v + b] = Bvv[Q][a][b] (zero up to ldk), Bvv double [Q][v][v], as a BF16 pair: the
// operand of the exchange contraction sum_(Q,b) U_Q[i][b] Bvv_Q[b][a] (the same Bvv_Q element
// the W = V Bvv_Q contraction reads)
__global__ void k_bvv_k(const double *__restrict__ Bvv, int Q, int v, long long ldk, __nv_bfloat16 *__restrict__ hi,
                        __nv_bfloat16 *__restrict__ lo) {
  const long long total = (long long)v * ldk;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const long long a = p / ldk, qb = p % ldk;
    const float x = (qb < (long long)Q * v) ? (float)Bvv[((qb / v) * v + a) * v + qb % v] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[p] = h;
    lo[p] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}
// gbT[a][(t,j)] = GB[t][j][a] for t < nt (zero up to ldk), GB double [nt][o][v], as a BF16 pair
__global__ void k_gb_t(const double *__restrict__ GB, int nt, int o, int v, long long ldk, __nv_bfloat16 *__restrict__ hi,
                       __nv_bfloat16 *__restrict__ lo) {
  const long long total = (long long)v * ldk;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const long long a = p / ldk, tj = p % ldk;
    const float x = (tj < (long long)nt * o) ? (float)GB[tj * v + a] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    hi[p] = h;
    lo[p] = __float2bfloat16_rn(x - __bfloat162float(h));
  }
}
__global__ void k_f2d(const float *__restrict__ s, double *__restrict__ d, long long n) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x)
    d[p] = (double)s[p];
}
// orbital-energy weights of the pair sums, FP32 slab T[(k,x)][(l,c)], k = i0 + row / v:
// mode 0 (q_oo): e_k - e_x - e_c;  mode 1 (q_vv): e_k + e_l - e_c
__global__ void k_weight_f32(float *__restrict__ Tw, const float *__restrict__ T, const double *__restrict__ eps,
                             int o, int v, int i0, long long rows, int mode) {
  const long long ov = (long long)o * v;
  const long long total = rows * ov;
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    const long long row = p / ov, col = p % ov;
    const int k = i0 + (int)(row / v), x = (int)(row % v), l = (int)(col / v), cc = (int)(col % v);
    const double w = mode == 0 ? eps[k] - eps[o + x] - eps[o + cc] : eps[k] + eps[l] - eps[o + cc];
    Tw[p] = T[p] * (float)w;
  }
}

inline dim3 grid_for(long long n) {
  long long b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  if (b < 1) b = 1;
  return dim3((unsigned)b);
}

// ---------------------------------------------------------------------------
// host: tensor maps via the driver entry point (no link-time libcuda dependency)
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                  CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    PP_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) throw PPError(PP_ECUDA, "cuTensorMapEncodeTiled is unavailable");
    fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}
// rows x K bf16 matrix, K contiguous with row stride ld (elements); box 64 x box_rows
static CUtensorMap kmajor_map(const void *base, long long K, long long rows, long long ld, int box_rows) {
  if ((reinterpret_cast<uintptr_t>(base) & 15) || ((ld * 2) & 15) || (K % BK))
    throw PPError(PP_EINVAL, "tensor map: base, stride or K not aligned");
  CUtensorMap m;
  std::memset(&m, 0, sizeof(m));
  cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(base), dims, strides, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw PPError(PP_ECUDA, "cuTensorMapEncodeTiled failed");
  return m;
}

// Tile configurations of k_gemm_bf16: (BN, stages) = (256, 4), 197 KB of shared memory, one
// CTA per SM; (256, 2), 97 KB, two CTAs per SM (their two 256-column accumulators fill TMEM, so
// one CTA's epilogue overlaps the other's main loop); (128, 6), 193 KB, one CTA per SM; (128, 3),
// 97 KB, two CTAs per SM.  The autotuner below chooses among them per GEMM site and shape.
struct GemmCfg {
  int bn, stages;
};
// GEMM sites (the contractions the autotuner keys on)
enum GemmSite { SITE_GAMMA = 0, SITE_U, SITE_W, SITE_KA, SITE_EF, SITE_KB, SITE_SLAB, SITE_SUMP1, SITE_SUMP2 };
constexpr GemmCfg kGemmCfgs[] = {{256, 4}, {256, 2}, {128, 6}, {128, 3}};
constexpr int NGEMMCFG = 4;
constexpr int TGEN_STAGES = 3;
constexpr int GEMM_SHORT_STEPS = 24;  // nseg * K / BK at or below which the default is the 2-CTA form
constexpr size_t gemm_smem_cfg(int bn, int stages) { return (size_t)stages * (BM * BK * 2 + bn * BK * 2) + 1024; }
constexpr size_t tgen_smem() { return (size_t)TGEN_STAGES * 4 * BM * BK * 2 + 1024; }

template <int BN, int ST>
static void launch_gemm_t(const GemmMaps &m, const GemmArgs &a, dim3 grid, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    PP_CUDA(cudaFuncSetAttribute(k_gemm_bf16<BN, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)gemm_smem_cfg(BN, ST)));
    attr = true;
  }
  k_gemm_bf16<BN, ST><<<grid, 128, gemm_smem_cfg(BN, ST), s>>>(m, a);
  PP_LAUNCH_CHECK("k_gemm_bf16");
}
// shared-memory limits of every tile configuration and of the generators, set once before any
// capture of a stream (a stream being captured must see only kernel launches and copies)
template <int BN, int ST> static void gemm_attr_t() {
  PP_CUDA(cudaFuncSetAttribute(k_gemm_bf16<BN, ST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)gemm_smem_cfg(BN, ST)));
}
static void launch_gemm_cfg(int cfg, const GemmMaps &m, const GemmArgs &a, dim3 grid, cudaStream_t s) {
  switch (cfg) {
    case 0: launch_gemm_t<256, 4>(m, a, grid, s); break;
    case 1: launch_gemm_t<256, 2>(m, a, grid, s); break;
    case 2: launch_gemm_t<128, 6>(m, a, grid, s); break;
    default: launch_gemm_t<128, 3>(m, a, grid, s); break;
  }
}

// ---------------------------------------------------------------------------
// Autotuner of the tensor-core GEMMs.  The first time a GEMM site meets a shape class
// (octaves of M, N and K, the number of split segments, whether the output accumulates), it
// runs every tile configuration -- and, for accumulating outputs, the K-split the default rule
// picks and no split -- twice, timed with CUDA events on the launching stream, keeps the
// fastest, and reruns it for the result.  GEMMs whose output is overwritten are idempotent; an
// accumulating output is copied aside before the first candidate and restored before each run.
// The choices live in a process-wide table (pp_autotune_report prints it).  PP_AUTOTUNE=0 turns
// tuning off (the default rule below is then used everywhere); PP_TUNE_CACHE=<file> loads the
// table from, and appends new entries to, a text file.
// ---------------------------------------------------------------------------
struct TuneKey {
  int site, nseg, acc, dev, m, n, k;
  bool operator<(const TuneKey &o) const {
    return std::tie(site, nseg, acc, dev, m, n, k) < std::tie(o.site, o.nseg, o.acc, o.dev, o.m, o.n, o.k);
  }
};
struct TuneVal {
  int cfg = 0, ksplit = 1;
  float ms[2 * NGEMMCFG] = {0};  // measured time of each candidate (cfg, split choice)
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneVal> g_tune;
static thread_local bool g_tune_blocked = false;  // inside a stream capture: no timing runs
void tune_block(bool on) { g_tune_blocked = on; }
static long long g_tune_runs = 0;  // tunings performed in this process
static bool g_tune_init = false, g_tune_on = true;
static std::string g_tune_file;
static const char *kSiteName[] = {"gamma", "U", "W", "KA", "EF", "KB", "slab", "sumP1", "sumP2", "other"};

static int octave(long long x) {
  int b = 0;
  while ((1LL << b) < x && b < 62) ++b;
  return b;
}
static void tune_init_locked() {
  if (g_tune_init) return;
  g_tune_init = true;
  const char *e = std::getenv("PP_AUTOTUNE");
  g_tune_on = !(e && e[0] == '0');
  const char *f = std::getenv("PP_TUNE_CACHE");
  if (f && f[0]) {
    g_tune_file = f;
    if (FILE *fp = std::fopen(f, "r")) {
      TuneKey k;
      TuneVal v;
      while (std::fscanf(fp, "%d %d %d %d %d %d %d %d %d", &k.site, &k.nseg, &k.acc, &k.dev, &k.m, &k.n, &k.k,
                         &v.cfg, &v.ksplit) == 9)
        if (v.cfg >= 0 && v.cfg < NGEMMCFG && v.ksplit >= 1) g_tune[k] = v;
      std::fclose(fp);
    }
  }
}

// default K split of an accumulating output: about two waves of CTAs over few output tiles,
// each CTA taking at least 8 K steps
static int default_ksplit(long long tiles, long long steps) {
  long long ks = std::min<long long>(304 / std::max<long long>(tiles, 1), steps / 8);
  return (int)std::max<long long>(1, std::min<long long>(ks, 65535));
}
// K split of an accumulating GEMM, from its reduction length alone: each split sums at most
// ACC_STEPS K steps (4 ACC_STEPS MMA accumulations into one FP32 TMEM element) before its partial
// is added into the output.  It depends on K only, so one output element is summed in the same
// order whatever the chunk shape (M) around it -- the reduced-precision sigma of a vector does
// not change with the batch it is computed in -- and the FP32 rounding of the longest
// reductions (the exchange and P contractions, up to millions of terms) is that of chains of
// at most 4 ACC_STEPS accumulations (about 2e-6 relative), below the 2^-16 of the BF16-pair
// operands.  Short reductions fall back to the wave-filling rule.
constexpr long long ACC_STEPS = 512;
static int acc_ksplit(long long tiles, long long steps) {
  if (steps <= ACC_STEPS) return default_ksplit(tiles, steps);
  return (int)std::min<long long>((steps + ACC_STEPS - 1) / ACC_STEPS, 65535);
}

// out (+)= alpha * sum_seg A_seg B_seg^T; segments share M, N, K; output addressing per GemmOut.
// site names the contraction for the autotuner; acc_base / acc_bytes give the region an
// accumulating output writes (restored between tuning runs; without it such a GEMM is not tuned).
void gemm_bf16(int site, int M, int N, long long K, int nseg, const __nv_bfloat16 *const *A, long long lda,
               const __nv_bfloat16 *const *B, long long ldb, const GemmOut &out, int *err, cudaStream_t s,
               const GemmOut *out2 = nullptr, void *acc_base = nullptr, size_t acc_bytes = 0) {
  GemmMaps maps[2];  // B boxes of 256 and 128 rows
  bool built[2] = {false, false};
  auto maps_for = [&](int bn) -> const GemmMaps & {
    const int w = bn == 256 ? 0 : 1;
    if (!built[w]) {
      std::memset(&maps[w], 0, sizeof(GemmMaps));
      for (int g = 0; g < nseg; ++g) {
        maps[w].a[g] = kmajor_map(A[g], K, M, lda, BM);
        maps[w].b[g] = kmajor_map(B[g], K, N, ldb, bn);
      }
      built[w] = true;
    }
    return maps[w];
  };
  const bool acc = out.C && out.accumulate && !out2;
  const int nk = (int)(K / BK);
  auto args_for = [&](int bn, int ksplit, dim3 &grid) {
    GemmArgs a{M, N, nk, nseg, out, out2 ? *out2 : GemmOut{}, err};
    a.mt = (M + BM - 1) / BM;
    a.nt = (N + bn - 1) / bn;
    const long long tiles = (long long)a.mt * a.nt;
    if (tiles > 0x7fffffffLL) throw PPError(PP_EINVAL, "k_gemm_bf16: too many tiles");
    grid = dim3((unsigned)tiles, 1, 1);
    a.ksplit = ksplit;
    grid.z = (unsigned)ksplit;
    return a;
  };
  auto ks_for = [&](int bn) {
    if (!acc) return 1;
    const long long tiles = (long long)((M + BM - 1) / BM) * ((N + bn - 1) / bn);
    return acc_ksplit(tiles, (long long)nseg * nk);
  };
  auto run = [&](int cfg, int ksplit) {
    dim3 grid;
    const int bn = kGemmCfgs[cfg].bn;
    GemmArgs a = args_for(bn, ksplit, grid);
    launch_gemm_cfg(cfg, maps_for(bn), a, grid, s);
  };
  int dev = 0;
  PP_CUDA(cudaGetDevice(&dev));
  const TuneKey key{site, nseg, acc ? 1 : 0, dev, octave(M), octave(N), octave(K)};
  TuneVal chosen;
  bool have = false, tune = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_init_locked();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      chosen = it->second;
      have = true;
    } else {
      tune = g_tune_on && !g_tune_blocked && (!acc || (acc_base && acc_bytes));
    }
  }
  if (have) {
    // long accumulating reductions always take the K-derived split (the table is keyed by
    // size classes, and a stored split may come from another K); a stored split larger than
    // the reduction allows falls back to the rule
    int ks = chosen.ksplit;
    if ((long long)nseg * nk > ACC_STEPS || ((long long)ks * 8 > (long long)nseg * nk && ks > 1))
      ks = ks_for(kGemmCfgs[chosen.cfg].bn);
    run(chosen.cfg, acc ? ks : 1);
    return;
  }
  if (!tune) {  // the default rule
    const int ks = ks_for(256);
    run((ks == 1 && (long long)nseg * nk <= GEMM_SHORT_STEPS) ? 1 : 0, ks);
    return;
  }
  // tune: every configuration (and for accumulating outputs the default split and none)
  DevBuf snap;
  if (acc) {
    snap.ensure(acc_bytes);
    PP_CUDA(cudaMemcpyAsync(snap.p, acc_base, acc_bytes, cudaMemcpyDeviceToDevice, s));
  }
  cudaEvent_t e0, e1;
  PP_CUDA(cudaEventCreate(&e0));
  PP_CUDA(cudaEventCreate(&e1));
  TuneVal best;
  float best_ms = 1e30f;
  for (int cfg = 0; cfg < NGEMMCFG; ++cfg) {
    const int ksd = ks_for(kGemmCfgs[cfg].bn);
    // long accumulating reductions keep their K-derived split (the summation order must not
    // depend on the tile choice); short ones may also run unsplit
    const int nsplit = (acc && ksd > 1 && (long long)nseg * nk <= ACC_STEPS) ? 2 : 1;
    for (int sp = 0; sp < nsplit; ++sp) {
      const int ks = sp == 0 ? ksd : 1;
      float t = 1e30f;
      for (int rep = 0; rep < 2; ++rep) {
        if (acc) PP_CUDA(cudaMemcpyAsync(acc_base, snap.p, acc_bytes, cudaMemcpyDeviceToDevice, s));
        PP_CUDA(cudaEventRecord(e0, s));
        run(cfg, ks);
        PP_CUDA(cudaEventRecord(e1, s));
        PP_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        PP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        t = std::min(t, ms);
      }
      best.ms[2 * cfg + sp] = t;
      if (t < best_ms) {
        best_ms = t;
        best.cfg = cfg;
        best.ksplit = ks;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (acc) PP_CUDA(cudaMemcpyAsync(acc_base, snap.p, acc_bytes, cudaMemcpyDeviceToDevice, s));
  run(best.cfg, best.ksplit);
  PP_CUDA(cudaStreamSynchronize(s));  // the snapshot is freed on return
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = best;
  ++g_tune_runs;
  if (!g_tune_file.empty())
    if (FILE *fp = std::fopen(g_tune_file.c_str(), "a")) {
      std::fprintf(fp, "%d %d %d %d %d %d %d %d %d\n", key.site, key.nseg, key.acc, key.dev, key.m, key.n, key.k,
                   best.cfg, best.ksplit);
      std::fclose(fp);
    }
}

void tgen(const __nv_bfloat16 *bovT, const __nv_bfloat16 *bovT_lo, long long ldq, long long ov, int o, int v,
          int i0, int ni, const double *eps, __nv_bfloat16 *Thi, __nv_bfloat16 *Tlo, long long ldT, int *err,
          cudaStream_t s, float *Tf = nullptr, long long ldf = 0) {
  static bool attr = false;
  if (!attr) {
    PP_CUDA(cudaFuncSetAttribute(k_tgen<TGEN_STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tgen_smem()));
    attr = true;
  }
  TgenMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  maps.hi = kmajor_map(bovT, ldq, ov, ldq, BM);
  maps.lo = bovT_lo ? kmajor_map(bovT_lo, ldq, ov, ldq, BM) : maps.hi;
  const int nt = (v + BM - 1) / BM;
  TgenArgs a{o, v, (int)(ldq / BK), i0, nt, bovT_lo ? 3 : 1, eps, Thi, Tlo, ldT, Tf, ldf, err};
  dim3 grid(nt * nt, o, ni);
  k_tgen<TGEN_STAGES><<<grid, 128, tgen_smem(), s>>>(maps, a);
  PP_LAUNCH_CHECK("k_tgen");
}

void prepare_kernels() {
  static bool done = false;
  if (done) return;
  gemm_attr_t<256, 4>();
  gemm_attr_t<256, 2>();
  gemm_attr_t<128, 6>();
  gemm_attr_t<128, 3>();
  PP_CUDA(cudaFuncSetAttribute(k_tgen_p, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tgenp_smem()));
  PP_CUDA(cudaFuncSetAttribute(k_tgen<TGEN_STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tgen_smem()));
  done = true;
}

// persistent amplitude slab (sigma product): one CTA per SM over the (i, j, ct <= dt) items
void tgen_p(const __nv_bfloat16 *bovT, const __nv_bfloat16 *bovT_lo, long long ldq, long long ov, int o, int v,
            int i0, int ni, const float *eps, __nv_bfloat16 *Thi, __nv_bfloat16 *Tlo, long long ldT, int *err,
            cudaStream_t s, int nsm) {
  static bool attr = false;
  if (!attr) {
    PP_CUDA(cudaFuncSetAttribute(k_tgen_p, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tgenp_smem()));
    attr = true;
  }
  TgenMaps maps;
  std::memset(&maps, 0, sizeof(maps));
  maps.hi = kmajor_map(bovT, ldq, ov, ldq, BM);
  maps.lo = bovT_lo ? kmajor_map(bovT_lo, ldq, ov, ldq, BM) : maps.hi;
  const int nt = (v + BM - 1) / BM;
  TgenPArgs a;
  a.o = o;
  a.v = v;
  a.nk = (int)(ldq / BK);
  a.i0 = i0;
  a.ni = ni;
  a.nt = nt;
  a.npairs = nt * (nt + 1) / 2;
  a.nseg = bovT_lo ? 3 : 1;
  a.nitems = (long long)ni * o * a.npairs;
  a.eps = eps;
  a.Thi = Thi;
  a.Tlo = Tlo;
  a.ldT = ldT;
  a.err = err;
  const long long grid = std::min<long long>(a.nitems, std::max(1, nsm));
  if (grid <= 0) return;
  k_tgen_p<<<(unsigned)grid, 192, tgenp_smem(), s>>>(maps, a);
  PP_LAUNCH_CHECK("k_tgen_p");
}

}  // namespace tc

// ---------------------------------------------------------------------------
// plan: BF16 / FP32 resident copies and workspaces of the tensor-core form
// ---------------------------------------------------------------------------
// per-kernel launch timing of the tensor-core form (enabled by pp_profile)
// ids: 0 the amplitude-contraction GEMM (all launches), 1 the amplitude generator, 2 the
// amplitude-contraction GEMM launches of the split form (three BF16 products each)
constexpr int NPROF = 3;
struct KernelProfile {
  bool on = false;
  std::vector<cudaEvent_t> ev[NPROF];  // start/stop pairs per kernel id
  long long launches[NPROF] = {0, 0, 0};
  double flops[NPROF] = {0, 0, 0};
  double ms[NPROF] = {0, 0, 0};
};
struct ChunkGraph {
  cudaGraphExec_t exec;
  long long kernels;  // kernel nodes of the graph (launch accounting)
};
struct TcPlan {
  long long ldq = 0, ldT = 0, vp = 0, Qp = 0;
  bool ready = false;  // copies of the per-dot intermediates made (after the precompute)
  KernelProfile prof;
  int slab_i = 1, Rmax = 2;  // slab_i: occupied rows of the largest slab the buffers hold
  int slab_l2 = 1;           // occupied rows of a slab within 64 MB per BF16 part (stays in L2)
  int nsm = 152;             // SMs of the device (waves of the slab GEMM)
  // BF16 hi/lo operands (K-major, K padded to 64)
  DevBuf bovT_hi, bovT_lo;   // [(i,a)][ldq]       amplitude slab generator
  DevBuf bvv_hi, bvv_lo;     // [(Q,d)][vp]        W = V Bvv_Q
  DevBuf bov_hi, bov_lo;     // [(Q,i)][vp]        E = Bov_Q V^T
  DevBuf gam_hi, gam_lo;     // [(Q,i)][vp]        F = Gam_Q V^T
  DevBuf bvvT_hi, bvvT_lo;   // [a][(c,Qp)]        sum_Q P_Q Bvv_Q
  DevBuf booT_hi, booT_lo;   // [i][(k,Qp)]        sum_Q Boo_Q P_Q
  long long kbo = 0, kqv = 0, kef = 0;  // padded K of the U, KA and KB contractions
  DevBuf booK_hi, booK_lo;   // [(Q,l)][kbo]       U = Boo_Q V
  DevBuf bvvK_hi, bvvK_lo;   // [a][(Q,b)]         KA = sum_(Q,b) U_Q Bvv_Q
  DevBuf gbT_hi, gbT_lo;     // [a][(t,j)]         KB = sum_t EF_t GB_t
  // FP32 copies of the operands of the remaining SIMT contractions
  DevBuf f_eps, f_Bov, f_poo, f_qoo, f_pvv, f_qvv;
  // workspaces
  DevBuf w_V, w_acc, w_tmp, w_cq, w_W, w_U, w_EF;
  DevBuf v_hi, v_lo;         // [(r,j)][vp]
  DevBuf c_hi, c_lo;         // C_Q(V): [(r,Q)][ldT]
  DevBuf t_hi, t_lo;         // amplitude slab [rows][ldT]
  DevBuf p1_hi, p1_lo;       // P as [(r,i)][(c,Qp)]
  DevBuf p2_hi, p2_lo;       // P as [(r,a)][(k,Qp)]
  DevBuf vT_hi, vT_lo;       // V^T [(r,b)][kbo]
  DevBuf kaU_hi, kaU_lo;     // U as [(r,i)][(Q,b)]
  DevBuf efB_hi, efB_lo;     // E, F as [(r,i)][(t,j)]
  DevBuf err;
  // CUDA graphs of sigma chunks (key: R, form, metric) and their staging buffers
  std::map<long long, ChunkGraph> graph_exec;
  std::set<long long> graph_seen;
  size_t graph_sig = 0;
  DevBuf g_in, g_sig, g_met;
};

size_t tc_plan_bytes(const pp_ctx *c) {
  if (!c->tc) return 0;
  TcPlan *p = c->tc;
  const DevBuf *bufs[] = {&p->bovT_hi, &p->bovT_lo, &p->bvv_hi, &p->bvv_lo, &p->bov_hi, &p->bov_lo, &p->gam_hi,
                          &p->gam_lo, &p->bvvT_hi, &p->bvvT_lo, &p->booT_hi, &p->booT_lo, &p->f_eps,
                          &p->f_Bov, &p->f_poo,
                          &p->f_qoo, &p->f_pvv, &p->f_qvv, &p->w_V, &p->w_acc, &p->w_tmp, &p->w_cq, &p->w_W,
                          &p->w_U, &p->w_EF, &p->v_hi, &p->v_lo, &p->c_hi, &p->c_lo, &p->t_hi, &p->t_lo,
                          &p->p1_hi, &p->p1_lo, &p->p2_hi, &p->p2_lo, &p->err, &p->booK_hi, &p->booK_lo,
                          &p->bvvK_hi, &p->bvvK_lo, &p->gbT_hi, &p->gbT_lo, &p->vT_hi, &p->vT_lo,
                          &p->kaU_hi, &p->kaU_lo, &p->efB_hi, &p->efB_lo, &p->g_in, &p->g_sig, &p->g_met};
  size_t n = 0;
  for (const DevBuf *b : bufs) n += b->bytes;
  return n;
}

static void clear_chunk_graphs(TcPlan *p) {
  for (auto &kv : p->graph_exec) cudaGraphExecDestroy(kv.second.exec);
  p->graph_exec.clear();
  p->graph_seen.clear();
}
// the addresses a captured chunk reads and writes (a change means the workspaces moved)
static size_t chunk_buffers_signature(const TcPlan *p) {
  const DevBuf *bufs[] = {&p->w_V, &p->w_acc, &p->w_tmp, &p->w_cq, &p->v_hi, &p->v_lo, &p->kaU_hi, &p->kaU_lo,
                          &p->vT_hi, &p->vT_lo, &p->efB_hi, &p->efB_lo, &p->c_hi, &p->c_lo, &p->t_hi, &p->t_lo,
                          &p->p1_hi, &p->p1_lo, &p->p2_hi, &p->p2_lo, &p->g_in, &p->g_sig, &p->g_met};
  size_t h = 1469598103934665603ull;
  for (const DevBuf *b : bufs) h = (h ^ reinterpret_cast<uintptr_t>(b->p)) * 1099511628211ull;
  return h;
}

void tc_destroy(pp_ctx *c) {
  if (!c->tc) return;
  TcPlan *p = c->tc;
  DevBuf *bufs[] = {&p->bovT_hi, &p->bovT_lo, &p->bvv_hi, &p->bvv_lo, &p->bov_hi, &p->bov_lo, &p->gam_hi,
                    &p->gam_lo, &p->bvvT_hi, &p->bvvT_lo, &p->booT_hi, &p->booT_lo, &p->f_eps,
                    &p->f_Bov, &p->f_poo,
                    &p->f_qoo, &p->f_pvv, &p->f_qvv, &p->w_V, &p->w_acc, &p->w_tmp, &p->w_cq, &p->w_W,
                    &p->w_U, &p->w_EF, &p->v_hi, &p->v_lo, &p->c_hi, &p->c_lo, &p->t_hi, &p->t_lo,
                    &p->p1_hi, &p->p1_lo, &p->p2_hi, &p->p2_lo, &p->err, &p->booK_hi, &p->booK_lo,
                    &p->bvvK_hi, &p->bvvK_lo, &p->gbT_hi, &p->gbT_lo, &p->vT_hi, &p->vT_lo,
                    &p->kaU_hi, &p->kaU_lo, &p->efB_hi, &p->efB_lo, &p->g_in, &p->g_sig, &p->g_met};
  for (DevBuf *b : bufs) b->release();
  clear_chunk_graphs(p);
  for (auto &v : p->prof.ev)
    for (cudaEvent_t e : v) cudaEventDestroy(e);
  delete p;
  c->tc = nullptr;
}

static void prof_mark(KernelProfile &pr, int id, cudaStream_t s) {
  if (!pr.on) return;
  cudaEvent_t e;
  PP_CUDA(cudaEventCreate(&e));
  PP_CUDA(cudaEventRecord(e, s));
  pr.ev[id].push_back(e);
}
// fold recorded event pairs into the totals (synchronises on the last event)
static void prof_collect(KernelProfile &pr) {
  for (int id = 0; id < NPROF; ++id) {
    auto &v = pr.ev[id];
    for (size_t k = 0; k + 1 < v.size(); k += 2) {
      PP_CUDA(cudaEventSynchronize(v[k + 1]));
      float ms = 0.f;
      PP_CUDA(cudaEventElapsedTime(&ms, v[k], v[k + 1]));
      pr.ms[id] += ms;
      cudaEventDestroy(v[k]);
      cudaEventDestroy(v[k + 1]);
    }
    v.clear();
  }
}

static void f32_copy(DevBuf &dst, const DevBuf &src, long long n, cudaStream_t s) {
  dst.ensure(sizeof(float) * (size_t)std::max<long long>(n, 1));
  if (n > 0) {
    tc::k_d2f<<<tc::grid_for(n), 256, 0, s>>>(src.as<double>(), dst.as<float>(), n);
    PP_LAUNCH_CHECK("k_d2f");
  }
}
// rows x ncol double matrix (row stride lds) -> BF16 hi/lo [rows][ld] (zero padded)
static void bf16_pair(DevBuf &hi, DevBuf &lo, const double *src, long long rows, long long ncol, long long lds,
                      long long ld, cudaStream_t s) {
  const size_t n = (size_t)std::max<long long>(rows * ld, 1);
  hi.ensure(sizeof(__nv_bfloat16) * n);
  lo.ensure(sizeof(__nv_bfloat16) * n);
  if (rows * ld > 0) {
    tc::k_to_bf16<double><<<tc::grid_for(rows * ld), 256, 0, s>>>(src, rows, ncol, lds, hi.as<__nv_bfloat16>(),
                                                                  lo.as<__nv_bfloat16>(), ld);
    PP_LAUNCH_CHECK("k_to_bf16");
  }
}

static long long pad64(long long x) { return std::max<long long>(tc::BK, ((x + tc::BK - 1) / tc::BK) * tc::BK); }

// device bytes for one chunk of the tensor-core sigma workspaces
long long tc_workspace_bytes(const pp_ctx *c) {
  if (c->opt.workspace_gb > 0) return (long long)(c->opt.workspace_gb * (1LL << 30));
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return 12LL << 30;
  // half of the free memory (keeping 8 GB free), at least 12 GB: the chunk size R of the sigma
  // sets how often the amplitudes are regenerated and how wide the contraction GEMMs are
  const long long half = (long long)(free_b / 2), room = (long long)free_b - (8LL << 30);
  return std::max<long long>(12LL << 30, std::min<long long>(half, room));
}

// Stage 1 of the plan: everything that depends on B and eps only (the precompute needs it).
static TcPlan *tc_plan_operands(pp_ctx *c) {
  if (c->tc) return c->tc;
  TcPlan *p = new TcPlan();
  c->tc = p;
  const long long o = c->o, v = c->v, Q = c->Q, ov = c->ov;
  cudaStream_t s = c->stream;
  p->ldq = pad64(Q);
  p->ldT = pad64(ov);
  p->vp = pad64(v);
  p->Qp = pad64(Q);
  // FP32 copies of the operands of the SIMT contractions that remain in this form (the
  // Coulomb term and the A(2) pair-sum products); the exchange and amplitude contractions
  // read only their BF16 pairs, so no FP32 copy of Boo, Bvv, Gamma or GB is kept
  f32_copy(p->f_eps, c->eps, c->n, s);
  f32_copy(p->f_Bov, c->Bov, Q * ov, s);
  p->kbo = pad64(o);
  p->kqv = pad64(Q * v);
  p->kef = pad64(2 * Q * o);
  if (c->opt.order >= 1 && Q > 0) {
    bf16_pair(p->bvv_hi, p->bvv_lo, c->Bvv.as<double>(), Q * v, v, v, p->vp, s);
    bf16_pair(p->bov_hi, p->bov_lo, c->Bov.as<double>(), Q * o, v, v, p->vp, s);
    p->bvvK_hi.ensure(sizeof(__nv_bfloat16) * (size_t)v * p->kqv);
    p->bvvK_lo.ensure(sizeof(__nv_bfloat16) * (size_t)v * p->kqv);
    tc::k_bvv_k<<<tc::grid_for(v * p->kqv), 256, 0, s>>>(c->Bvv.as<double>(), (int)Q, (int)v, p->kqv,
                                                         p->bvvK_hi.as<__nv_bfloat16>(), p->bvvK_lo.as<__nv_bfloat16>());
    PP_LAUNCH_CHECK("k_bvv_k");
    bf16_pair(p->booK_hi, p->booK_lo, c->Boo.as<double>(), Q * o, o, o, p->kbo, s);
  }
  if (c->opt.order >= 2 && Q > 0) {
    p->bovT_hi.ensure(sizeof(__nv_bfloat16) * (size_t)ov * p->ldq);
    p->bovT_lo.ensure(sizeof(__nv_bfloat16) * (size_t)ov * p->ldq);
    tc::k_bovT<<<tc::grid_for(ov * p->ldq), 256, 0, s>>>(c->Bov.as<double>(), (int)Q, ov,
                                                         p->bovT_hi.as<__nv_bfloat16>(),
                                                         p->bovT_lo.as<__nv_bfloat16>(), p->ldq);
    PP_LAUNCH_CHECK("k_bovT");
    p->bvvT_hi.ensure(sizeof(__nv_bfloat16) * (size_t)v * v * p->Qp);
    p->bvvT_lo.ensure(sizeof(__nv_bfloat16) * (size_t)v * v * p->Qp);
    tc::k_perm_qlast<<<tc::grid_for(v * v * p->Qp), 256, 0, s>>>(c->Bvv.as<double>(), (int)Q, (int)v, (int)v,
                                                                 p->Qp, p->bvvT_hi.as<__nv_bfloat16>(),
                                                                 p->bvvT_lo.as<__nv_bfloat16>());
    PP_LAUNCH_CHECK("k_perm_qlast");
    p->booT_hi.ensure(sizeof(__nv_bfloat16) * (size_t)o * o * p->Qp);
    p->booT_lo.ensure(sizeof(__nv_bfloat16) * (size_t)o * o * p->Qp);
    tc::k_perm_qlast<<<tc::grid_for(o * o * p->Qp), 256, 0, s>>>(c->Boo.as<double>(), (int)Q, (int)o, (int)o,
                                                                 p->Qp, p->booT_hi.as<__nv_bfloat16>(),
                                                                 p->booT_lo.as<__nv_bfloat16>());
    PP_LAUNCH_CHECK("k_perm_qlast");
  }
  // chunk of R half-vectors: FP32 W, U, E/F plus BF16 C_Q(V) and two BF16 copies of P
  // bytes per half-vector of the chunk workspaces sigma_bf16 allocates: FP32 V, accumulators and
  // temporaries (7 ov) and c_Q; BF16 pairs (4 bytes per element) of V, V^T, U, E/F, C_Q(V) and
  // the two layouts of P
  const long long per_half = 4 * (7 * ov + Q) + 4 * (o * p->vp + v * p->kbo + o * p->kqv + o * p->kef) +
                             4 * Q * p->ldT + 8 * ov * p->Qp;
  long long R = tc_workspace_bytes(c) / std::max<long long>(per_half, 1);
  R = std::max<long long>(2, std::min<long long>(R, 64));
  R &= ~1LL;
  p->Rmax = (int)R;
  // the amplitude slab holds up to 512 MB per BF16 part; each sigma chunk picks its height
  // (choose_slab): within 64 MB per part when its C_Q(V) operand is large (the slab is the
  // GEMM's A operand and must stay in L2 while C_Q(V) streams past it once), larger only for
  // narrow chunks, whose few N tiles would otherwise leave most SMs idle
  p->slab_i = (int)std::max<long long>(1, std::min<long long>(o, (512LL << 20) / (2 * v * p->ldT)));
  p->slab_l2 = (int)std::max<long long>(1, std::min<long long>(o, (64LL << 20) / (2 * v * p->ldT)));
  {
    int dev = 0, nsm = 0;
    PP_CUDA(cudaGetDevice(&dev));
    PP_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (nsm > 0) p->nsm = nsm;
  }
  p->err.ensure(sizeof(int) * 4);
  PP_CUDA(cudaMemsetAsync(p->err.p, 0, sizeof(int) * 4, s));
  return p;
}

// Stage 2: FP32 / BF16 copies of the per-dot intermediates (made once the precompute is done).
static TcPlan *tc_plan(pp_ctx *c) {
  TcPlan *p = tc_plan_operands(c);
  if (p->ready) return p;
  const long long o = c->o, v = c->v, Q = c->Q, ov = c->ov;
  cudaStream_t s = c->stream;
  f32_copy(p->f_poo, c->p_oo, o * o, s);
  f32_copy(p->f_qoo, c->q_oo, o * o, s);
  f32_copy(p->f_pvv, c->p_vv, v * v, s);
  f32_copy(p->f_qvv, c->q_vv, v * v, s);
  if (c->opt.order >= 1 && Q > 0) {
    bf16_pair(p->gam_hi, p->gam_lo, c->Gam.as<double>(), Q * o, v, v, p->vp, s);
    p->gbT_hi.ensure(sizeof(__nv_bfloat16) * (size_t)v * p->kef);
    p->gbT_lo.ensure(sizeof(__nv_bfloat16) * (size_t)v * p->kef);
    tc::k_gb_t<<<tc::grid_for(v * p->kef), 256, 0, s>>>(c->GB.as<double>(), (int)(2 * Q), (int)o, (int)v, p->kef,
                                                        p->gbT_hi.as<__nv_bfloat16>(), p->gbT_lo.as<__nv_bfloat16>());
    PP_LAUNCH_CHECK("k_gb_t");
  }
  p->ready = true;
  return p;
}

static void throw_on_tc_error(TcPlan *p, cudaStream_t s) {
  int herr = 0;
  PP_CUDA(cudaMemcpyAsync(&herr, p->err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaStreamSynchronize(s));
  if (herr) {
    PP_CUDA(cudaMemsetAsync(p->err.p, 0, sizeof(int), s));
    throw PPError(PP_ETIMEOUT, "tensor-core kernel wait timed out (code " + std::to_string(herr) + ")");
  }
}

// Per-dot intermediates on the tensor cores (contexts of the mixed form).  Amplitude slabs
// T[(i,c)][(j,d)] = t_ij^cd come from the split-BF16 generator (FP32 accumulation, FP32 copy
// of the slab); the pair sums (Eq. s(2) densities and the A(2) weights) are FP32 split-K
// contractions of that copy; Gamma_Q[(i,c)] = sum_(j,d) t_ij^cd B_Q,jd is a split-BF16 GEMM.
// The results (relative error about 1e-6) are stored in the FP64 context fields.
void precompute_tc(pp_ctx *c) {
  const int o = c->o, v = c->v, Q = c->Q;
  const long long ov = c->ov;
  cudaStream_t s = c->stream;
  precompute_begin(c);
  if (c->opt.order >= 2 && Q > 0) {
    using bf = __nv_bfloat16;
    TcPlan *p = tc_plan_operands(c);
    const long long ldT = p->ldT;
    const int si = p->slab_l2;
    p->t_hi.ensure(sizeof(bf) * (size_t)si * v * ldT);
    p->t_lo.ensure(sizeof(bf) * (size_t)si * v * ldT);
    DevBuf T32, Tw32, acc, bk_hi, bk_lo;
    T32.ensure(sizeof(float) * (size_t)si * v * ov);
    Tw32.ensure(sizeof(float) * (size_t)si * v * ov);
    const long long nacc = 2LL * o * o + 2LL * v * v + (long long)Q * ov;
    acc.ensure(sizeof(float) * (size_t)nacc);
    PP_CUDA(cudaMemsetAsync(acc.p, 0, sizeof(float) * (size_t)nacc, s));
    float *poo = acc.as<float>(), *qoo = poo + o * o, *pvv = qoo + o * o, *qvv = pvv + (long long)v * v;
    float *gam = qvv + (long long)v * v;
    bf16_pair(bk_hi, bk_lo, c->Bov.as<double>(), Q, ov, ov, ldT, s);  // Bov as [Q][(j,d)], K-major
    bf *thi = p->t_hi.as<bf>(), *tlo = p->t_lo.as<bf>();
    float *T = T32.as<float>(), *Tw = Tw32.as<float>();
    int *err = p->err.as<int>();
    for (int i0 = 0; i0 < o; i0 += si) {
      const int ni = std::min(si, o - i0);
      const long long rows = (long long)ni * v;
      if (ldT > ov) {
        PP_CUDA(cudaMemset2DAsync(thi + ov, ldT * 2, 0, (ldT - ov) * 2, rows, s));
        PP_CUDA(cudaMemset2DAsync(tlo + ov, ldT * 2, 0, (ldT - ov) * 2, rows, s));
      }
      tc::tgen(p->bovT_hi.as<bf>(), p->bovT_lo.as<bf>(), p->ldq, ov, o, v, i0, ni, c->eps.as<double>(), thi, tlo,
               ldT, err, s, T, ov);
      // p_oo[i][j] += sum_c sum_rho T[rho][(i,c)] T[rho][(j,c)]   (split over c)
      GemmF32 g;
      g.M = o; g.N = o; g.K = (int)rows; g.nred = v;
      g.A = T; g.a_m = v; g.a_k = ov; g.a_red = 1;
      g.B = T; g.b_k = ov; g.b_n = v; g.b_red = 1;
      g.C = poo; g.c_m = o; g.c_n = 1; g.beta = 1.f;
      g.ksplit = std::min(v, 256);
      gemm_f32(g, s);
      tc::k_weight_f32<<<tc::grid_for(rows * ov), 256, 0, s>>>(Tw, T, c->eps.as<double>(), o, v, i0, rows, 0);
      PP_LAUNCH_CHECK("k_weight_f32");
      g.B = Tw; g.C = qoo;
      gemm_f32(g, s);
      // p_vv[a][b] += sum_k sum_(l,c) T[(k,a)][(l,c)] T[(k,b)][(l,c)]   (split over k, else K)
      GemmF32 h;
      h.M = v; h.N = v; h.K = (int)ov; h.nred = ni;
      h.A = T; h.a_m = ov; h.a_k = 1; h.a_red = (long long)v * ov;
      h.B = T; h.b_k = 1; h.b_n = ov; h.b_red = (long long)v * ov;
      h.C = pvv; h.c_m = v; h.c_n = 1; h.beta = 1.f;
      h.ksplit = ni > 1 ? ni : 16;
      gemm_f32(h, s);
      tc::k_weight_f32<<<tc::grid_for(rows * ov), 256, 0, s>>>(Tw, T, c->eps.as<double>(), o, v, i0, rows, 1);
      PP_LAUNCH_CHECK("k_weight_f32");
      h.B = Tw; h.C = qvv;
      gemm_f32(h, s);
      // Gamma[Q][i0 v + row] = sum_(j,d) T[row][(j,d)] Bov[Q][(j,d)]
      const bf *A[3] = {thi, thi, tlo};
      const bf *B[3] = {bk_hi.as<bf>(), bk_lo.as<bf>(), bk_hi.as<bf>()};
      tc::GemmOut out;
      out.C = gam + (long long)i0 * v;
      out.s_r0 = 1;
      out.s_c0 = ov;
      tc::gemm_bf16(tc::SITE_GAMMA, (int)rows, Q, ldT, 3, A, ldT, B, ldT, out, err, s);
    }
    const float *src[5] = {poo, qoo, pvv, qvv, gam};
    double *dst[5] = {c->p_oo.as<double>(), c->q_oo.as<double>(), c->p_vv.as<double>(), c->q_vv.as<double>(),
                      c->Gam.as<double>()};
    const long long cnt[5] = {(long long)o * o, (long long)o * o, (long long)v * v, (long long)v * v,
                              (long long)Q * ov};
    for (int t = 0; t < 5; ++t) {
      tc::k_f2d<<<tc::grid_for(cnt[t]), 256, 0, s>>>(src[t], dst[t], cnt[t]);
      PP_LAUNCH_CHECK("k_f2d");
    }
    throw_on_tc_error(p, s);
  }
  precompute_finish(c);
}

// Occupied rows per slab for one sigma chunk of NC = R Q columns.  The slab GEMM P = T C^T has
// ceil(ni v / 128) x ceil(NC / 256) tiles at one CTA per SM, so its time goes in whole waves of
// nsm CTAs; the persistent generator covers ni o npairs items (two 128 x 128 x Q products each,
// about 2 Q / ov of a GEMM tile's time at its lower efficiency) in waves of nsm CTAs.  The
// height (at most si_max) that minimises the waves over all slabs, plus a small per-slab
// launch cost, is taken.
static int choose_slab(int o, int v, int Q, long long NC, int si_max, int nsm) {
  const long long nt = (v + 127) / 128, npairs = nt * (nt + 1) / 2, ntn = (NC + 255) / 256;
  const double item = 2.0 * Q / ((double)o * v);
  double best = 1e300;
  int arg = si_max;
  for (int si = si_max; si >= 1; --si) {
    double cost = 0.0;
    for (int i0 = 0; i0 < o; i0 += si) {
      const long long ni = std::min(si, o - i0);
      const long long gt = (ni * v + 127) / 128 * ntn, tt = ni * o * npairs;
      cost += (double)((gt + nsm - 1) / nsm) + item * (double)((tt + nsm - 1) / nsm) + 0.05;
    }
    if (cost < best - 1e-9) {
      best = cost;
      arg = si;
    }
  }
  return arg;
}

static void ensure_zeroed(DevBuf &b, size_t bytes, cudaStream_t s) {
  if (bytes <= b.bytes) return;
  b.ensure(bytes);
  PP_CUDA(cudaMemsetAsync(b.p, 0, b.bytes, s));
}

// BF16 tensor-core sigma: amplitude contraction and the large first-order contractions on
// tcgen05; the remaining small contractions in FP32.  split = true uses hi/lo BF16 pairs
// (three products) for a result with about 2^-16 relative error per product.
void sigma_bf16(pp_ctx *c, int nvec, const double *Zd, double *sig_d, double *met_d, bool split) {
  TcPlan *p = tc_plan(c);
  tc::prepare_kernels();
  const int o = c->o, v = c->v, Q = c->Q;
  const long long ov = c->ov, vp = p->vp, Qp = p->Qp, ldT = p->ldT;
  cudaStream_t s = c->stream;
  const int Rmax = p->Rmax;
  const int nseg = split ? 3 : 1;
  using bf = __nv_bfloat16;
  p->w_V.ensure(sizeof(float) * (size_t)Rmax * ov);
  p->w_acc.ensure(sizeof(float) * 2 * (size_t)Rmax * ov);
  p->w_tmp.ensure(sizeof(float) * 4 * (size_t)Rmax * ov);
  if (c->opt.order >= 1) {
    p->w_cq.ensure(sizeof(float) * (size_t)Q * Rmax);
    p->v_hi.ensure(sizeof(bf) * (size_t)Rmax * o * vp);
    p->v_lo.ensure(sizeof(bf) * (size_t)Rmax * o * vp);
    // K paddings (and, at first order, the F half of EF) stay zero: never written
    ensure_zeroed(p->kaU_hi, sizeof(bf) * (size_t)Rmax * o * p->kqv, s);
    ensure_zeroed(p->kaU_lo, sizeof(bf) * (size_t)Rmax * o * p->kqv, s);
    p->vT_hi.ensure(sizeof(bf) * (size_t)Rmax * v * p->kbo);
    p->vT_lo.ensure(sizeof(bf) * (size_t)Rmax * v * p->kbo);
    ensure_zeroed(p->efB_hi, sizeof(bf) * (size_t)Rmax * o * p->kef, s);
    ensure_zeroed(p->efB_lo, sizeof(bf) * (size_t)Rmax * o * p->kef, s);
  }
  if (c->opt.order >= 2) {
    ensure_zeroed(p->c_hi, sizeof(bf) * (size_t)Rmax * Q * ldT, s);
    ensure_zeroed(p->c_lo, sizeof(bf) * (size_t)Rmax * Q * ldT, s);
    p->t_hi.ensure(sizeof(bf) * (size_t)p->slab_i * v * ldT);
    p->t_lo.ensure(sizeof(bf) * (size_t)p->slab_i * v * ldT);
    const size_t pbytes = sizeof(bf) * (size_t)Rmax * ov * Qp;  // padding columns stay zero
    ensure_zeroed(p->p1_hi, pbytes, s);
    ensure_zeroed(p->p1_lo, pbytes, s);
    ensure_zeroed(p->p2_hi, pbytes, s);
    ensure_zeroed(p->p2_lo, pbytes, s);
  }
  // gap, Boo, Bvv, BvvP, BooT, GB and Gamma in FP32 are only read by the step-by-step fallback of
  // sigma_chunk, which the first_order hook below replaces (it always returns true)
  SigmaRes<float> res{nullptr, p->f_eps.as<float>(), p->f_Bov.as<float>(), nullptr, nullptr, nullptr, nullptr, nullptr,
                      nullptr, p->f_poo.as<float>(), p->f_qoo.as<float>(), p->f_pvv.as<float>(), p->f_qvv.as<float>()};
  int *err = p->err.as<int>();
  const bf *vhi = p->v_hi.as<bf>(), *vlo = p->v_lo.as<bf>();
  auto seg3 = [&](const bf *hiA, const bf *loA, const bf *hiB, const bf *loB, const bf **A, const bf **B) {
    A[0] = hiA; B[0] = hiB;
    A[1] = hiA; B[1] = loB;
    A[2] = loA; B[2] = hiB;
  };
  const int R_total = 2 * nvec;
  // one chunk of R half-vectors: V64 in, sg_out / mt_out (mt_out may be null) out
  auto run_chunk = [&](const int R, const double *V64, double *sg_out, double *mt_out) {
    float *V = p->w_V.as<float>();
    tc::k_d2f<<<tc::grid_for((long long)R * ov), 256, 0, s>>>(V64, V, (long long)R * ov);
    PP_LAUNCH_CHECK("k_d2f");
    if (c->opt.order >= 1) {
      tc::k_to_bf16<double><<<tc::grid_for((long long)R * o * vp), 256, 0, s>>>(
          V64, (long long)R * o, v, v, p->v_hi.as<bf>(), p->v_lo.as<bf>(), vp);
      PP_LAUNCH_CHECK("k_to_bf16");
    }
    SigmaWork<float> wk{p->w_acc.as<float>(), p->w_acc.as<float>() + (long long)R * ov, p->w_tmp.as<float>(),
                        p->w_cq.as<float>(), nullptr, nullptr, nullptr};  // W, U, EF: first_order
    SigmaHooks<float> hk;
    // The first-order block on the tensor cores; its operands are written by the GEMMs that
    // produce them in the K-major layouts the next GEMM reads.  These contractions are small
    // next to the amplitude contraction and always run in the split form (three BF16
    // products, about 2^-16 per product), so the BF16 phase keeps its first-order terms at
    // that accuracy.
    hk.first_order = [&](int Rc, float *Aacc, float *Bacc) {
      const int nseg1 = 3;
      const int order = c->opt.order;
      const bool tda = c->opt.tda != 0;  // Tamm-Dancoff form: only U and KA (A terms)
      const long long kbo = p->kbo, kqv = p->kqv, kef = p->kef;
      bf *kuh = p->kaU_hi.as<bf>(), *kul = p->kaU_lo.as<bf>();
      bf *efh = p->efB_hi.as<bf>(), *efl = p->efB_lo.as<bf>();
      const bf *A[3], *B[3];
      // U[r][Q][l][b] = sum_k Boo[Q][l][k] V[r][k][b]: rows (Q,l), columns (r,b), K = k.  Written
      // as the BF16 pair [(r,l)][(Q,b)] (row stride kqv), with b contiguous so that each output
      // row leaves in 16-byte stores: the K-major operand of KA and the addend of C_Q(V)
      {
        tc::k_vT<<<tc::grid_for((long long)Rc * v * kbo), 256, 0, s>>>(V64, Rc, o, v, kbo, p->vT_hi.as<bf>(),
                                                                      p->vT_lo.as<bf>());
        PP_LAUNCH_CHECK("k_vT");
        seg3(p->booK_hi.as<bf>(), p->booK_lo.as<bf>(), p->vT_hi.as<bf>(), p->vT_lo.as<bf>(), A, B);
        tc::GemmOut ku;
        ku.Chi = kuh;
        ku.Clo = kul;
        ku.d_r = o;
        ku.s_r1 = v;
        ku.s_r0 = kqv;
        ku.d_c = v;
        ku.s_c1 = (long long)o * kqv;
        ku.s_c0 = 1;
        tc::gemm_bf16(tc::SITE_U, Q * o, Rc * v, kbo, nseg1, A, kbo, B, kbo, ku, err, s);
      }
      // W[r][j][Q][d] = sum_b V[r][j][b] Bvv[Q][b][d]: rows (r,j), columns (Q,d), written as
      // C_Q(V) = W - U (BF16 pair, [(r,Q)][(j,d)]) for the amplitude contraction; U[r][Q][j][d]
      // is element (r o + j, Q v + d) of the pair above, i.e. row * kqv + column
      if (order >= 2 && !tda) {
        seg3(vhi, vlo, p->bvv_hi.as<bf>(), p->bvv_lo.as<bf>(), A, B);
        tc::GemmOut cc;
        cc.Chi = p->c_hi.as<bf>();
        cc.Clo = split ? p->c_lo.as<bf>() : nullptr;
        cc.d_r = o;
        cc.s_r1 = (long long)Q * ldT;
        cc.s_r0 = v;
        cc.d_c = v;
        cc.s_c1 = ldT;
        cc.s_c0 = 1;
        cc.add_hi = kuh;
        cc.add_lo = kul;
        cc.add_ld = kqv;
        cc.add_scale = -1.f;
        tc::gemm_bf16(tc::SITE_W, Rc * o, Q * v, vp, nseg1, A, vp, B, vp, cc, err, s);
      }
      // KA: Aacc[r][i][a] -= sum_(Q,k) Boo[Q][i][k] W[r][k][Q][a] = sum_(Q,b) U[r][Q][i][b] Bvv[Q][b][a]
      // (rows (r,i), columns a, K = (Q,b))
      {
        seg3(kuh, kul, p->bvvK_hi.as<bf>(), p->bvvK_lo.as<bf>(), A, B);
        tc::GemmOut out;
        out.C = Aacc;
        out.s_r0 = v;
        out.s_c0 = 1;
        out.alpha = -1.f;
        out.accumulate = 1;
        tc::gemm_bf16(tc::SITE_KA, Rc * o, v, kqv, nseg1, A, kqv, B, kqv, out, err, s, nullptr, Aacc,
                      sizeof(float) * (size_t)Rc * ov);
      }
      if (tda) return true;
      // E and F: EF[(r,i)][(t,j)] = sum_b X_t[i][b] V[r][j][b], X = Bov (t < Q), Gamma (t >= Q)
      {
        tc::GemmOut out;
        out.Chi = efh;
        out.Clo = efl;
        out.d_r = o;
        out.s_r1 = o;
        out.s_r0 = kef;
        out.d_c = o;
        out.s_c1 = (long long)o * kef;
        out.s_c0 = 1;
        seg3(p->bov_hi.as<bf>(), p->bov_lo.as<bf>(), vhi, vlo, A, B);
        tc::gemm_bf16(tc::SITE_EF, Q * o, Rc * o, vp, nseg1, A, vp, B, vp, out, err, s);
        if (order >= 2) {
          out.Chi = efh + (long long)Q * o;
          out.Clo = efl ? efl + (long long)Q * o : nullptr;
          seg3(p->gam_hi.as<bf>(), p->gam_lo.as<bf>(), vhi, vlo, A, B);
          tc::gemm_bf16(tc::SITE_EF, Q * o, Rc * o, vp, nseg1, A, vp, B, vp, out, err, s);
        }
      }
      // KB: Bacc[r][i][a] -= sum_(t,j) EF[r][t][i][j] GB[t][j][a]   (rows (r,i), columns a)
      {
        seg3(efh, efl, p->gbT_hi.as<bf>(), p->gbT_lo.as<bf>(), A, B);
        tc::GemmOut out;
        out.C = Bacc;
        out.s_r0 = v;
        out.alpha = -1.f;
        out.accumulate = 1;
        tc::gemm_bf16(tc::SITE_KB, Rc * o, v, kef, nseg1, A, kef, B, kef, out, err, s, nullptr, Bacc,
                      sizeof(float) * (size_t)Rc * ov);
      }
      return true;
    };
    hk.amplitude = [&](int Rc, const float *Cmat, float *Bacc) {
      const long long NC = (long long)Rc * Q;
      bf *chi = p->c_hi.as<bf>(), *clo = p->c_lo.as<bf>();
      if (Cmat) {  // C_Q(V) from the step-by-step path: convert to the BF16 pair
        tc::k_to_bf16<float><<<tc::grid_for(NC * ldT), 256, 0, s>>>(Cmat, NC, ov, ov, chi, clo, ldT);
        PP_LAUNCH_CHECK("k_to_bf16");
      }
      bf *thi = p->t_hi.as<bf>();
      bf *tlo = split ? p->t_lo.as<bf>() : nullptr;
      bf *p1h = p->p1_hi.as<bf>(), *p1l = split ? p->p1_lo.as<bf>() : nullptr;
      bf *p2h = p->p2_hi.as<bf>(), *p2l = split ? p->p2_lo.as<bf>() : nullptr;
      const long long cq_bytes = NC * ldT * 2 * (split ? 2 : 1);  // the streamed operand
      const int si = choose_slab(o, v, Q, NC, cq_bytes <= (2LL << 30) ? p->slab_i : p->slab_l2, p->nsm);
      for (int i0 = 0; i0 < o; i0 += si) {
        const int ni = std::min(si, o - i0);
        const long long rows = (long long)ni * v;
        if (ldT > ov) {  // zero the K padding of the slab rows
          PP_CUDA(cudaMemset2DAsync(thi + ov, ldT * 2, 0, (ldT - ov) * 2, rows, s));
          if (tlo) PP_CUDA(cudaMemset2DAsync(tlo + ov, ldT * 2, 0, (ldT - ov) * 2, rows, s));
        }
        prof_mark(p->prof, 1, s);
        tc::tgen_p(p->bovT_hi.as<bf>(), split ? p->bovT_lo.as<bf>() : nullptr, p->ldq, ov, o, v, i0, ni,
                   p->f_eps.as<float>(), thi, tlo, ldT, err, s, p->nsm);
        prof_mark(p->prof, 1, s);
        if (p->prof.on) {  // algorithmic: one Q-long product per amplitude (the exchange
          p->prof.launches[1] += 1;  // integral of (c,d) is the direct one of (d,c)), split counted once
          p->prof.flops[1] += 2.0 * (double)Q * (double)rows * (double)ov;
        }
        // P = T C^T for this slab, written as BF16 pairs in two layouts:
        //   P1[r][i][c][q] (rows (r,i), K = (c,q)) and P2[r][c][i][q] (rows (r,c), K = (i,q))
        const bf *A[3] = {thi, thi, tlo};
        const bf *B[3] = {chi, clo, chi};
        tc::GemmOut o1, o2;
        o1.Chi = p1h + (long long)i0 * v * Qp;
        o1.Clo = p1l ? p1l + (long long)i0 * v * Qp : nullptr;
        o1.s_r0 = Qp;
        o1.d_c = Q;
        o1.s_c1 = ov * Qp;
        o2.Chi = p2h + (long long)i0 * Qp;
        o2.Clo = p2l ? p2l + (long long)i0 * Qp : nullptr;
        o2.d_r = v;
        o2.s_r1 = Qp;
        o2.s_r0 = (long long)o * Qp;
        o2.d_c = Q;
        o2.s_c1 = ov * Qp;
        prof_mark(p->prof, 0, s);
        if (split) prof_mark(p->prof, 2, s);
        tc::gemm_bf16(tc::SITE_SLAB, (int)rows, (int)NC, ldT, nseg, A, ldT, B, ldT, o1, err, s, &o2);
        prof_mark(p->prof, 0, s);
        if (split) prof_mark(p->prof, 2, s);
        if (p->prof.on) {  // algorithmic: the contraction once (the split form's three
          p->prof.launches[0] += 1;  // products are an emulation of one)
          p->prof.flops[0] += 2.0 * (double)rows * (double)NC * (double)ov;
          if (split) {
            p->prof.launches[2] += 1;
            p->prof.flops[2] += 2.0 * (double)rows * (double)NC * (double)ov;
          }
        }
      }
      // Bacc[(r,i)][a] += sum_(c,q) P1[(r,i)][(c,q)] Bvv[q][c][a]
      {
        const bf *A[3], *B[3];
        seg3(p->p1_hi.as<bf>(), p->p1_lo.as<bf>(), p->bvvT_hi.as<bf>(), p->bvvT_lo.as<bf>(), A, B);
        tc::GemmOut out;
        out.C = Bacc;
        out.s_r0 = v;
        out.accumulate = 1;
        tc::gemm_bf16(tc::SITE_SUMP1, Rc * o, v, (long long)v * Qp, nseg, A, (long long)v * Qp, B, (long long)v * Qp,
                      out, err, s, nullptr, Bacc, sizeof(float) * (size_t)Rc * ov);
      }
      // Bacc[r][i][a] -= sum_(k,q) P2[(r,a)][(k,q)] Boo[q][i][k]   (rows (r,a), columns i)
      {
        const bf *A[3], *B[3];
        seg3(p->p2_hi.as<bf>(), p->p2_lo.as<bf>(), p->booT_hi.as<bf>(), p->booT_lo.as<bf>(), A, B);
        tc::GemmOut out;
        out.C = Bacc;
        out.d_r = v;
        out.s_r1 = ov;
        out.s_r0 = 1;
        out.s_c0 = v;
        out.alpha = -1.f;
        out.accumulate = 1;
        tc::gemm_bf16(tc::SITE_SUMP2, Rc * v, o, (long long)o * Qp, nseg, A, (long long)o * Qp, B,
                      (long long)o * Qp, out, err, s, nullptr, Bacc, sizeof(float) * (size_t)Rc * ov);
      }
    };
    sigma_chunk<float>(c, R, V, V64, sg_out, mt_out, res, wk, hk);
  };
  // A chunk shape (R, form, metric or not) met for the second time is captured into a CUDA
  // graph that reads and writes fixed staging buffers; later chunks of that shape copy their
  // half-vectors in, replay the graph and copy the products out.  The first run of a shape
  // goes kernel by kernel (the GEMM autotuner settles its choices there: a capture cannot
  // time anything, so inside one the tuner uses its table or the default rule).  Not while
  // the profiling events are recorded.
  const bool graphs = c->opt.graphs != 0 && !p->prof.on;
  if (graphs) {
    p->g_in.ensure(sizeof(double) * (size_t)Rmax * ov);
    p->g_sig.ensure(sizeof(double) * (size_t)Rmax * ov);
    p->g_met.ensure(sizeof(double) * (size_t)Rmax * ov);
    const size_t sig = chunk_buffers_signature(p);  // after every buffer a capture reads is in place
    if (sig != p->graph_sig) {  // workspaces reallocated since the graphs were captured
      clear_chunk_graphs(p);
      p->graph_sig = sig;
    }
  }
  for (int r0 = 0; r0 < R_total; r0 += Rmax) {
    const int R = std::min(Rmax, R_total - r0);
    const double *V64 = Zd + (long long)r0 * ov;
    double *sg = sig_d + (long long)r0 * ov, *mt = met_d ? met_d + (long long)r0 * ov : nullptr;
    if (!graphs) {
      run_chunk(R, V64, sg, mt);
      continue;
    }
    const long long key = ((long long)R << 2) | (split ? 2 : 0) | (mt ? 1 : 0);
    auto it = p->graph_exec.find(key);
    const size_t bytes = sizeof(double) * (size_t)R * ov;
    if (it == p->graph_exec.end() && !p->graph_seen.count(key)) {
      p->graph_seen.insert(key);
      run_chunk(R, V64, sg, mt);
      continue;
    }
    double *gin = p->g_in.as<double>(), *gsg = p->g_sig.as<double>(), *gmt = mt ? p->g_met.as<double>() : nullptr;
    PP_CUDA(cudaMemcpyAsync(gin, V64, bytes, cudaMemcpyDeviceToDevice, s));
    if (it == p->graph_exec.end()) {
      cudaGraph_t g = nullptr;
      const unsigned long long launches0 = __atomic_load_n(&g_pp_launches, __ATOMIC_RELAXED);
      PP_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
      tc::tune_block(true);
      try {
        run_chunk(R, gin, gsg, gmt);
      } catch (...) {
        tc::tune_block(false);
        cudaStreamEndCapture(s, &g);
        if (g) cudaGraphDestroy(g);
        throw;
      }
      tc::tune_block(false);
      PP_CUDA(cudaStreamEndCapture(s, &g));
      cudaGraphExec_t ge = nullptr;
      const cudaError_t ie = cudaGraphInstantiate(&ge, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) throw PPError(PP_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(ie));
      // the kernels of the capture were counted once while recording; count them per replay
      const long long nk = (long long)(__atomic_load_n(&g_pp_launches, __ATOMIC_RELAXED) - launches0);
      __atomic_fetch_sub(&g_pp_launches, (unsigned long long)nk, __ATOMIC_RELAXED);
      it = p->graph_exec.emplace(key, ChunkGraph{ge, nk}).first;
    }
    PP_CUDA(cudaGraphLaunch(it->second.exec, s));
    __atomic_fetch_add(&g_pp_launches, (unsigned long long)it->second.kernels, __ATOMIC_RELAXED);
    PP_CUDA(cudaMemcpyAsync(sg, gsg, bytes, cudaMemcpyDeviceToDevice, s));
    if (mt) PP_CUDA(cudaMemcpyAsync(mt, gmt, bytes, cudaMemcpyDeviceToDevice, s));
  }
  int herr = 0;
  PP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PP_CUDA(cudaStreamSynchronize(s));
  if (herr) {
    PP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
    throw PPError(PP_ETIMEOUT, "tensor-core kernel wait timed out (code " + std::to_string(herr) + ")");
  }
}

// ---------------------------------------------------------------------------
// profiling entry points (C ABI)
// ---------------------------------------------------------------------------
extern "C" long long pp_autotune_report(char *buf, long long cap) {
  std::string r;
  {
    std::lock_guard<std::mutex> lk(tc::g_tune_mu);
    tc::tune_init_locked();
    r += "autotune " + std::string(tc::g_tune_on ? "on" : "off") + ", tunings " + std::to_string(tc::g_tune_runs) + "\n";
    for (const auto &kv : tc::g_tune) {
      const tc::TuneKey &k = kv.first;
      const tc::TuneVal &v = kv.second;
      char line[256];
      std::snprintf(line, sizeof(line), "%s nseg=%d acc=%d M~2^%d N~2^%d K~2^%d -> BN=%d stages=%d ksplit=%d |",
                    tc::kSiteName[std::min(k.site, 9)], k.nseg, k.acc, k.m, k.n, k.k, tc::kGemmCfgs[v.cfg].bn,
                    tc::kGemmCfgs[v.cfg].stages, v.ksplit);
      r += line;
      for (int c = 0; c < tc::NGEMMCFG; ++c) {
        std::snprintf(line, sizeof(line), " %.3f", v.ms[2 * c]);
        r += line;
      }
      r += " ms\n";
    }
  }
  if (buf && cap > 0) {
    const long long n = std::min<long long>(cap - 1, (long long)r.size());
    std::memcpy(buf, r.data(), (size_t)n);
    buf[n] = 0;
  }
  return (long long)r.size() + 1;
}
extern "C" pp_status pp_profile(pp_ctx *c, int enable) {
  if (!c) return PP_EINVAL;
  try {
    TcPlan *p = tc_plan(c);
    prof_collect(p->prof);
    p->prof.on = enable != 0;
    if (enable)
      for (int id = 0; id < NPROF; ++id) {
        p->prof.launches[id] = 0;
        p->prof.flops[id] = 0;
        p->prof.ms[id] = 0;
      }
    return PP_OK;
  } catch (const PPError &e) {
    c->err = e.msg;
    return e.st;
  }
}

extern "C" pp_status pp_profile_read(pp_ctx *c, int id, long long *launches, double *ms, double *flops) {
  if (!c || id < 0 || id >= NPROF) return PP_EINVAL;
  try {
    TcPlan *p = tc_plan(c);
    prof_collect(p->prof);
    if (launches) *launches = p->prof.launches[id];
    if (ms) *ms = p->prof.ms[id];
    if (flops) *flops = p->prof.flops[id];
    return PP_OK;
  } catch (const PPError &e) {
    c->err = e.msg;
    return e.st;
  }
}
