// CUDA-core GEMM with FP32 accumulation for the dense GCN layers (Eq. GCN
// combine step).  Used for the all-FP32 form and as the fallback-free
// reference shape for the tensor-core kernels: 64 x 64 output tile per block,
// 16 x 16 threads with 4 x 4 outputs each, K staged through shared memory in
// slices of 16.  Operands may be K-major or MN-major, FP32 or BF16.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace cpra {

namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <typename T>
__device__ __forceinline__ float ld_el(const void* base, int64_t idx) {
  return to_f(static_cast<const T*>(base)[idx]);
}

__device__ __forceinline__ void st_el(void* base, int dt, int64_t idx, float v) {
  if (dt == DT_BF16) static_cast<bf16*>(base)[idx] = __float2bfloat16_rn(v);
  else static_cast<float*>(base)[idx] = v;
}

template <typename TA, typename TB>
__global__ void __launch_bounds__(256)
gemm_simt_kernel(GemmArgs g) {
  __shared__ float As[BK][BM + 4];
  __shared__ float Bs[BK][BN + 4];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int nval = g.n_valid > 0 ? g.n_valid : g.Nc;
  int64_t kbeg = 0, kend = g.K;
  if (g.epi == EPI_PARTIAL && gridDim.z > 1) {
    const int64_t per = ((g.K + gridDim.z - 1) / gridDim.z + BK - 1) / BK * BK;
    kbeg = per * blockIdx.z;
    kend = kbeg + per < g.K ? kbeg + per : g.K;
  }
  float acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;

  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    // A tile: BM x BK
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int id = threadIdx.x + t * 256;
      int mm, kk;
      if (g.a_kmajor) { mm = id / BK; kk = id % BK; }
      else { kk = id / BM; mm = id % BM; }
      const int64_t m = m0 + mm, k = k0 + kk;
      float v = 0.f;
      if (m < g.M && k < kend)
        v = ld_el<TA>(g.A, g.a_kmajor ? m * g.lda + k : k * g.lda + m);
      As[kk][mm] = v;
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int id = threadIdx.x + t * 256;
      int nn, kk;
      if (g.b_kmajor) { nn = id / BK; kk = id % BK; }
      else { kk = id / BN; nn = id % BN; }
      const int n = n0 + nn;
      const int64_t k = k0 + kk;
      float v = 0.f;
      if (n < nval && k < kend)
        v = ld_el<TB>(g.B, g.b_kmajor ? (int64_t)n * g.ldb + k : k * g.ldb + n);
      Bs[kk][nn] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = As[kk][ty + 16 * r];
#pragma unroll
      for (int c = 0; c < 4; ++c) b[c] = Bs[kk][tx + 16 * c];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fmaf(a[r], b[c], acc[r][c]);
    }
    __syncthreads();
  }

  if (g.epi == EPI_RELU_BITS || (g.epi == EPI_BIAS_RELU && g.out1)) {
    // lanes 0-15 of a warp hold row ty, lanes 16-31 row ty + 1, each 16
    // consecutive columns n0 + 16c + tx: one ballot gives both rows' masks
    const bool only_bits = g.epi == EPI_RELU_BITS;
    uint16_t* mb = static_cast<uint16_t*>(only_bits ? g.out0 : g.out1);
    const int64_t ldm = only_bits ? g.ld0 : g.ld1;
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int64_t m = m0 + ty + 16 * r;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int n = n0 + tx + 16 * c;
        bool bit = false;
        if (m < g.M && n < g.Nc) {
          float v = acc[r][c] + g.bias[n];
          v = v > 0.f ? v : 0.f;
          if (g.d0 == DT_BF16) v = __bfloat162float(__float2bfloat16_rn(v));
          bit = v > 0.f;
        }
        const unsigned b = __ballot_sync(0xffffffffu, bit);
        if (tx == 0 && m < g.M && n < g.Nc)
          mb[m * ldm + n / 16] = static_cast<uint16_t>(lane >= 16 ? b >> 16 : b & 0xffffu);
      }
    }
    if (only_bits) return;
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int64_t m = m0 + ty + 16 * r;
    if (m >= g.M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int n = n0 + tx + 16 * c;
      if (n >= g.Nc) continue;
      float v = acc[r][c];
      switch (g.epi) {
        case EPI_PARTIAL:
          static_cast<float*>(g.out0)[(int64_t)blockIdx.z * g.M * g.ld0 + m * g.ld0 + n] = v;
          break;
        case EPI_BIAS_RELU:
          v += g.bias[n];
          st_el(g.out0, g.d0, m * g.ld0 + n, v > 0.f ? v : 0.f);
          break;
        case EPI_BIAS:
          st_el(g.out0, g.d0, m * g.ld0 + n, n < nval ? v + g.bias[n] : 0.f);
          break;
        case EPI_BIAS_SIGMOID:
          if (g.addend && n < nval)
            v += g.d_add == DT_BF16
                     ? __bfloat162float(static_cast<const bf16*>(g.addend)[m * g.ld_add + n])
                     : static_cast<const float*>(g.addend)[m * g.ld_add + n];
          v = (n < nval) ? 1.0f / (1.0f + expf(-(v + g.bias[n]))) : 0.f;
          st_el(g.out0, g.d0, m * g.ld0 + n, v);
          break;
        case EPI_SPLIT:
          if (n < g.split) st_el(g.out0, g.d0, m * g.ld0 + n, v);
          else st_el(g.out1, g.d1, m * g.ld1 + (n - g.split), v * g.row_scale[m]);
          break;
      }
    }
  }
}

__global__ void splitk_reduce_kernel(const float* __restrict__ part, int splits, int M,
                                     int Nc, int64_t ldp, float* out, int64_t ldo) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)M * Nc) return;
  const int r = (int)(idx / Nc), c = (int)(idx % Nc);
  float t = 0.f;
  for (int z = 0; z < splits; ++z) t += part[(int64_t)z * M * ldp + (int64_t)r * ldp + c];
  out[(int64_t)r * ldo + c] = t;
}

}  // namespace

void gemm_simt_launch(const GemmArgs& g, cudaStream_t st) {
  dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.Nc + BN - 1) / BN),
            g.epi == EPI_PARTIAL ? (unsigned)g.splits : 1u);
  if (g.da == DT_BF16) {
    if (g.db == DT_BF16) gemm_simt_kernel<bf16, bf16><<<grid, 256, 0, st>>>(g);
    else gemm_simt_kernel<bf16, float><<<grid, 256, 0, st>>>(g);
  } else {
    if (g.db == DT_BF16) gemm_simt_kernel<float, bf16><<<grid, 256, 0, st>>>(g);
    else gemm_simt_kernel<float, float><<<grid, 256, 0, st>>>(g);
  }
}

void splitk_reduce(const float* part, int splits, int M, int Nc, int64_t ldp, float* out,
                   int64_t ldo, cudaStream_t st) {
  const int64_t n = (int64_t)M * Nc;
  splitk_reduce_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(part, splits, M, Nc, ldp,
                                                                     out, ldo);
}

}  // namespace cpra
