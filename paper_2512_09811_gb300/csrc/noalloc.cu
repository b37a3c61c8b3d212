// Allocation-free metric product Sigma z (declared in include/pp.h as pp_metric_noalloc).
//
// Who needs it: a caller that must not allocate device memory at the moment it wants
// the product.  Two common cases: code that runs inside another framework's device
// memory pool, where the pool owns the GPU's memory and a raw cudaMalloc/cudaFree
// would escape its budget and accounting; and latency-critical loops, where
// cudaMalloc and cudaFree are avoided because they can synchronise the whole device.
// pp_sigma (metric != NULL) computes the same product but takes its intermediate
// products from context workspaces that grow on demand, and stages host arrays through
// temporary device buffers.  This entry point does neither: its two intermediate
// products live in one fixed array compiled into the library, and it takes device
// pointers only.
//
// The array is shared by every call in the process on a given device (it is one
// per device, not one per context).  Calls that overlap in time on the same device --
// from two host threads, or on two contexts whose streams run concurrently -- race on
// it and may return wrong results; callers must serialise them.  No element of the
// array needs to start at zero: each call writes every element it reads before
// reading it.
//
// Set-up: the first call on each device (a call with nvec = 0 does only this) looks
// the array's device address up with cudaGetSymbolAddress, with that device current,
// caches it, and has the runtime load the two kernels a call launches.  This can load
// the library's device code, so the first call must come before any stream capture
// begins on that device; later calls load nothing.  The current device must be the
// context's device (checked: PP_EINVAL otherwise).
#include "pp_internal.h"

#include <mutex>
#include <string>

namespace {

// 2^21 doubles = 16 MiB per device, resident for the life of the process once loaded.
// One call needs 4 * nvec * nocc * nvir doubles (p_oo V and V p_vv for the 2 nvec
// half-vectors), so nvec * nocc * nvir <= 2^19 (PP_METRIC_NOALLOC_MAX_ELEMS).
constexpr long long kScratchDoubles = 1LL << 21;
static_assert(4LL * PP_METRIC_NOALLOC_MAX_ELEMS == kScratchDoubles, "header limit and array size disagree");
static __device__ __align__(256) double g_metric_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mu;
double *g_scratch_addr[kMaxDevices] = {nullptr};

__global__ void k_metric_noalloc(double *__restrict__ out, const double *__restrict__ V,
                                 const double *__restrict__ t1, const double *__restrict__ t3, int second,
                                 long long ov, long long total);

// Address of the array on the current device, looked up once per device; the same
// set-up step also has the runtime load this file's kernel and the FP64 GEMM kernel the
// call launches (under lazy module loading either would otherwise be loaded, and may take
// device memory, at its first launch), so that later calls load nothing.
double *scratch_on_current_device() {
  int dev = -1;
  PP_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw PPError(PP_EINVAL, "pp_metric_noalloc: device index out of range");
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    double *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_metric_scratch);
    if (e != cudaSuccess)
      throw PPError(PP_ECUDA, std::string("pp_metric_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, k_metric_noalloc);
    if (e != cudaSuccess)
      throw PPError(PP_ECUDA, std::string("pp_metric_noalloc: cudaFuncGetAttributes: ") + cudaGetErrorString(e));
    gemm_f64_preload();
    g_scratch_addr[dev] = p;
  }
  return g_scratch_addr[dev];
}

// out = (S X, -S Y) per supervector, S = 1 + S(2) with S(2)_ia,jb = d_ab rho_oo[i,j] -
// d_ij rho_vv[a,b] (Eq. s(2)).  The context holds the pair sums p_oo = -2 rho_oo and
// p_vv = 2 rho_vv, so S V = V - (p_oo V)/2 - (V p_vv)/2 = V - t1/2 - t3/2.
__global__ void k_metric_noalloc(double *__restrict__ out, const double *__restrict__ V,
                                 const double *__restrict__ t1, const double *__restrict__ t3, int second,
                                 long long ov, long long total) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < total;
       p += (long long)gridDim.x * blockDim.x) {
    double val = V[p];
    if (second) val += -0.5 * t1[p] - 0.5 * t3[p];
    out[p] = ((p / ov) & 1) ? -val : val;
  }
}

}  // namespace

extern "C" pp_status pp_metric_noalloc(pp_ctx *c, int nvec, const double *Z, double *out) {
  if (!c) return PP_EINVAL;
  if (nvec < 0 || (nvec > 0 && (!Z || !out))) {
    c->err = "pp_metric_noalloc: bad argument";
    return PP_EINVAL;
  }
  const long long ov = c->ov;
  if (nvec > PP_METRIC_NOALLOC_MAX_NVEC) {
    c->err = "pp_metric_noalloc: nvec = " + std::to_string(nvec) + " exceeds the limit of " +
             std::to_string(PP_METRIC_NOALLOC_MAX_NVEC) + " supervectors per call (split the batch)";
    return PP_EINVAL;
  }
  if ((long long)nvec * ov > PP_METRIC_NOALLOC_MAX_ELEMS) {
    c->err = "pp_metric_noalloc: nvec * nocc * nvir = " + std::to_string((long long)nvec * ov) +
             " exceeds the fixed scratch limit of " + std::to_string((long long)PP_METRIC_NOALLOC_MAX_ELEMS) +
             " (split the batch, or use pp_sigma)";
    return PP_EINVAL;
  }
  try {
    // the scratch array is looked up on the current device and the kernels launch on the
    // context's stream: both must be the context's device
    int dev = -1;
    PP_CUDA(cudaGetDevice(&dev));
    if (dev != c->device) {
      c->err = "pp_metric_noalloc: the current device (" + std::to_string(dev) +
               ") is not the context's device (" + std::to_string(c->device) + ")";
      return PP_EINVAL;
    }
    double *scratch = scratch_on_current_device();
    if (nvec == 0) return PP_OK;
    const long long R = 2LL * nvec;
    double *t1 = scratch, *t3 = scratch + R * ov;
    cudaStream_t s = c->stream;
    const int o = c->o, v = c->v;
    const bool second = c->opt.order >= 2;
    if (second) {
      GemmF64 a;  // t1[r][i][a] = sum_j p_oo[i][j] V[r][j][a]
      a.M = o; a.N = v; a.K = o; a.nbatch = (int)R;
      a.A = c->p_oo.as<double>(); a.a_m = o; a.a_k = 1;
      a.B = Z; a.b_k = v; a.b_n = 1; a.b_batch = ov;
      a.C = t1; a.c_m = v; a.c_n = 1; a.c_batch = ov;
      gemm_f64(a, s);
      GemmF64 b;  // t3[r][i][a] = sum_b V[r][i][b] p_vv[b][a]
      b.M = o; b.N = v; b.K = v; b.nbatch = (int)R;
      b.A = Z; b.a_m = v; b.a_k = 1; b.a_batch = ov;
      b.B = c->p_vv.as<double>(); b.b_k = v; b.b_n = 1;
      b.C = t3; b.c_m = v; b.c_n = 1; b.c_batch = ov;
      gemm_f64(b, s);
    }
    const long long total = R * ov;
    const long long nb = std::max<long long>(1, std::min<long long>((total + 255) / 256, 152LL * 16));
    k_metric_noalloc<<<(unsigned)nb, 256, 0, s>>>(out, Z, t1, t3, second ? 1 : 0, ov, total);
    PP_LAUNCH_CHECK("k_metric_noalloc");
    PP_CUDA(cudaStreamSynchronize(s));
    return PP_OK;
  } catch (const PPError &e) {
    c->err = e.msg;
    return e.st;
  }
}
