// noalloc.cu -- polarization readout of a caller-owned device state that
// allocates no device memory at all.
//
// Some callers cannot call cudaMalloc: code running inside a host application
// that owns every device allocation (a plugin handed a fixed pool), or a
// latency-critical loop where an allocation would synchronize the device.
// This entry point reduces N_up / N_dn of one spin of a device state they
// already own, writing (P, norm) to a device buffer they pass in.  Its only
// scratch -- one FP64 partial pair per reduction block and a ticket counter --
// lives in the file-scope device array below, of fixed size
// (kNoAllocMaxBlocks partial pairs, about 19.5 KiB), which every GPU that loads
// the library holds until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/spinrp.h"
#include "internal.h"

namespace {

constexpr int kNoAllocMaxBlocks = 1216;  // 8 blocks per SM on a 152-SM GB300
constexpr int kNoAllocThreads = 256;

struct NoAllocScratch {
  double2 partials[kNoAllocMaxBlocks];
  unsigned ticket;
};

}  // namespace

// Shared by every call on a device; holds the last call's partials.
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

template <typename C>
__global__ void __launch_bounds__(kNoAllocThreads)
noalloc_observe_kernel(const C *__restrict__ psi, int M, int site_pos, NoAllocScratch *scratch,
                       double *out) {
  __shared__ double s_up[kNoAllocThreads / 32], s_dn[kNoAllocThreads / 32];
  __shared__ int s_last;
  const uint64_t N = 1ull << M;
  double up = 0.0, dn = 0.0;
  for (uint64_t y = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; y < N;
       y += (uint64_t)gridDim.x * blockDim.x) {
    const C v = psi[y];
    const double p = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
    if ((y >> site_pos) & 1ull) up += p;
    else dn += p;
  }
  for (int o = 16; o; o >>= 1) {
    up += __shfl_xor_sync(0xffffffffu, up, o);
    dn += __shfl_xor_sync(0xffffffffu, dn, o);
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  if (lane == 0) s_up[warp] = up, s_dn[warp] = dn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double u = 0.0, d = 0.0;
    for (int w = 0; w < nw; ++w) u += s_up[w], d += s_dn[w];
    scratch->partials[blockIdx.x] = make_double2(u, d);
    __threadfence();
    s_last = atomicAdd(&scratch->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double u = 0.0, d = 0.0;
  for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    const double2 p = __ldcg(&scratch->partials[b]);
    u += p.x, d += p.y;
  }
  for (int o = 16; o; o >>= 1) {
    u += __shfl_xor_sync(0xffffffffu, u, o);
    d += __shfl_xor_sync(0xffffffffu, d, o);
  }
  __syncthreads();
  if (lane == 0) s_up[warp] = u, s_dn[warp] = d;
  __syncthreads();
  if (threadIdx.x == 0) {
    double U = 0.0, D = 0.0;
    for (int w = 0; w < nw; ++w) U += s_up[w], D += s_dn[w];
    out[0] = (U - D) / (U + D);
    out[1] = U + D;
    scratch->ticket = 0u;
  }
}

// Device address of g_noalloc_scratch.  In host code the array's name is
// only a host-side stand-in, never a device address, so the address is looked
// up with cudaGetSymbolAddress on the first call on a device (with that
// device current) and cached per device together with the unique ID of the
// context it was resolved in; a call made in a different context (the device
// was reset and its context recreated) looks it up again.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);
static std::mutex g_noalloc_mu;
static void *g_noalloc_addr[256];
static unsigned long long g_noalloc_ctx[256];
static CtxGetCurrentFn g_ctx_current = nullptr;
static CtxGetIdFn g_ctx_id = nullptr;

// Unique ID of the calling thread's current context (0 if none can be had).
static unsigned long long current_context_id() {
  if (!g_ctx_current || !g_ctx_id) {
    void *f1 = nullptr, *f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return 0;
    }
    g_ctx_current = (CtxGetCurrentFn)f1;
    g_ctx_id = (CtxGetIdFn)f2;
  }
  void *ctx = nullptr;
  unsigned long long id = 0;
  if (g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
  return id;
}

extern "C" int spinrp_polarization_noalloc(const void *psi, int M, int prec, int site,
                                           const int32_t *layout, int blocks, double *out,
                                           void *stream) {
  using spinrp::report_error;
  if (!psi || !out) return report_error(SPINRP_EINVAL, "polarization_noalloc: psi or out is NULL");
  if (M < 1 || M > spinrp::kMaxM)
    return report_error(SPINRP_EINVAL, "polarization_noalloc: M outside 1..34");
  if (prec != SPINRP_C64 && prec != SPINRP_C128)
    return report_error(SPINRP_EINVAL, "polarization_noalloc: unknown precision");
  if (site < 1 || site > M) return report_error(SPINRP_EINVAL, "polarization_noalloc: site outside 1..M");
  if (blocks < 0 || blocks > kNoAllocMaxBlocks)
    return report_error(SPINRP_EINVAL,
                        "polarization_noalloc: blocks exceeds the 1216 partials of the static scratch");
  const int site_pos = layout ? layout[site - 1] : site - 1;
  if (site_pos < 0 || site_pos >= M)
    return report_error(SPINRP_EINVAL, "polarization_noalloc: layout entry outside 0..M-1");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256)
    return report_error(SPINRP_ECUDA, "polarization_noalloc: cudaGetDevice failed");
  void *addr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    const unsigned long long ctx = current_context_id();
    if (!g_noalloc_addr[dev] || ctx == 0 || ctx != g_noalloc_ctx[dev]) {
      // first call on this device or in this context (with the device
      // current): resolve the symbol's address
      if (cudaGetSymbolAddress(&g_noalloc_addr[dev], g_noalloc_scratch) != cudaSuccess) {
        g_noalloc_addr[dev] = nullptr;
        cudaGetLastError();
        return report_error(SPINRP_ECUDA, "polarization_noalloc: cudaGetSymbolAddress failed");
      }
      // the lookup makes the device's context current if it was not yet
      g_noalloc_ctx[dev] = ctx ? ctx : current_context_id();
    }
    addr = g_noalloc_addr[dev];
  }
  NoAllocScratch *scratch = (NoAllocScratch *)addr;
  cudaStream_t s = (cudaStream_t)stream;
  // the ticket must start at zero (a clear, not an allocation)
  if (cudaMemsetAsync(&scratch->ticket, 0, sizeof(unsigned), s) != cudaSuccess)
    return report_error(SPINRP_ECUDA, "polarization_noalloc: clearing the ticket failed");
  const uint64_t N = 1ull << M;
  int nb = (int)((N + kNoAllocThreads - 1) / kNoAllocThreads);
  if (nb > kNoAllocMaxBlocks) nb = kNoAllocMaxBlocks;
  if (blocks > 0 && blocks < nb) nb = blocks;
  if (prec == SPINRP_C64)
    noalloc_observe_kernel<float2><<<nb, kNoAllocThreads, 0, s>>>((const float2 *)psi, M, site_pos, scratch, out);
  else
    noalloc_observe_kernel<double2><<<nb, kNoAllocThreads, 0, s>>>((const double2 *)psi, M, site_pos, scratch, out);
  if (cudaGetLastError() != cudaSuccess)
    return report_error(SPINRP_ECUDA, "polarization_noalloc: kernel launch failed");
  return SPINRP_OK;
}
