// Allocation-free variant of the fused SpMM + loss entry point.
//
// Some callers cannot call cudaMalloc at all: code embedded in a host
// application that owns every byte of device memory through its own pool or
// a fixed budget, and latency-critical paths where an allocation (and the
// device synchronisation it can imply) is not acceptable.  For them,
// cpra_op_loss_noalloc takes only inputs and outputs; the per-block partial
// sums of the loss kernel live in the file-scope device array below, which
// every GPU that loads this library holds until the process exits.
//
// Contract (also stated in cpra.h):
//   * S <= CPRA_NOALLOC_MAX_S (1024); larger S is rejected with
//     CPRA_EINVAL before anything is launched.  N is not limited (the kernel
//     strides over rows with at most kMaxBlocks blocks).
//   * The first call on a device looks the array's device address up with
//     cudaGetSymbolAddress (once per device, under a lock); make that first
//     call before any stream capture.  Under lazy module loading that call
//     is also when the device reserves the array; if it has no room, the
//     call returns CPRA_ENOMEM.
//   * All calls on a device share the one array and it keeps the contents
//     of the last call.  Nothing in it needs clearing: every call writes
//     each partial row it later reads.  Calls whose work overlaps on the GPU
//     (different streams without ordering, or concurrent host threads) race
//     on the array and give wrong results: order them on one stream.
#include <mutex>

#include "cpra.h"
#include "kernels.cuh"

namespace cpra {
namespace {

constexpr int kMaxS = CPRA_NOALLOC_MAX_S;
constexpr int kMaxBlocks = 512;
// per-block partial rows of 4S+1 floats (padded to a multiple of 4)
constexpr size_t kScratchBytes =
    (size_t)kMaxBlocks * (((size_t)4 * kMaxS + 1 + 3) / 4 * 4) * sizeof(float);  // about 8.4 MB

static __device__ __align__(256) unsigned char g_loss_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of g_loss_scratch on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_loss_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace cpra

using namespace cpra;

extern "C" cpra_status cpra_op_loss_noalloc(int64_t N, int32_t S, const int32_t* rowptr,
                                            const int32_t* col, const float* P, int64_t ldp,
                                            const float* lambda, int32_t problem, int32_t alpha,
                                            float gamma, float nu, int32_t diversity_kind,
                                            int32_t grad_kind, float* G, int64_t ldg,
                                            uint32_t* x_bits, float* terms, void* cuda_stream) {
  if (S > kMaxS) return CPRA_EINVAL;  // beyond the fixed scratch array
  if (N < 1 || S < 1 || !rowptr || !col || !P || !G || !terms) return CPRA_EINVAL;
  if (ldp < S || ldp % 4 || ldg < S || ldg % 4 || ldg > (S + 15) / 16 * 16) return CPRA_EINVAL;
  if (problem != CPRA_MIS && problem != CPRA_MAXCUT) return CPRA_EINVAL;
  if (problem == CPRA_MIS && !lambda) return CPRA_EINVAL;
  if (alpha < 2 || alpha % 2 || diversity_kind < 0 || diversity_kind > 1) return CPRA_EINVAL;
  if (grad_kind != 0 && grad_kind != 1) return CPRA_EINVAL;
  void* base = nullptr;
  const cudaError_t se = scratch_address(&base);
  if (se == cudaErrorMemoryAllocation) {
    cudaGetLastError();  // the failed reservation is not sticky: clear it
    return CPRA_ENOMEM;
  }
  if (se != cudaSuccess) return CPRA_ECUDA;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return CPRA_ECUDA;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  LossArgs a;
  a.N = N; a.S = S; a.ldp = ldp; a.ldg = ldg; a.rowptr = rowptr; a.col = col; a.P = P;
  a.lambda = lambda; a.problem = problem; a.alpha = alpha; a.div_kind = diversity_kind;
  a.grad_kind = grad_kind; a.gamma = gamma; a.nu = nu; a.G = G; a.dg = DT_F32;
  a.xbits = x_bits; a.pstride = loss_pstride(S);
  a.partials = static_cast<float*>(base);
  a.do_loss = 1;
  const int max_grid = sms * 4 < kMaxBlocks ? sms * 4 : kMaxBlocks;
  const int grid = loss_launch(a, max_grid, st);
  colsum_finalize(a.partials, grid, a.pstride, 4 * S + 1, terms, nullptr, 0, 0, nullptr, st);
  return cudaGetLastError() == cudaSuccess ? CPRA_OK : CPRA_ECUDA;
}
