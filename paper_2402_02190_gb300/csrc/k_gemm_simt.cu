// CUDA-core GEMM with FP32 accumulation for the dense GCN layers (Eq. GCN
// combine step): the all-FP32 form and the shapes the tensor-core kernels do
// not take.  128 x 128 output tile per block, 16 x 16 threads with 8 x 8
// outputs each, K staged through double-buffered shared memory in slices of
// 16.  Operands may be K-major or MN-major, FP32 or BF16.
//
// The build compiles this file once per operand type pair, with
// -DCPRA_SIMT_DA=<DType of A> -DCPRA_SIMT_DB=<DType of B>, so that the four
// sets of kernel instances (each with its four operand layouts) compile in
// parallel; the (FP32, FP32) object also holds the host dispatch and the
// split-K reduction.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

#if !defined(CPRA_SIMT_DA) || !defined(CPRA_SIMT_DB)
#error "k_gemm_simt.cu is compiled with -DCPRA_SIMT_DA=<0|1> -DCPRA_SIMT_DB=<0|1>"
#endif

namespace cpra {

namespace {

constexpr int BM = 128, BN = 128, BK = 16;

template <typename T>
__device__ __forceinline__ float ld_el(const void* base, int64_t idx) {
  return to_f(static_cast<const T*>(base)[idx]);
}

__device__ __forceinline__ void st_el(void* base, int dt, int64_t idx, float v) {
  if (dt == DT_BF16) static_cast<bf16*>(base)[idx] = __float2bfloat16_rn(v);
  else static_cast<float*>(base)[idx] = v;
}

// Four consecutive values at idx (dtype dt): one vector store when the row
// and the address allow it.
__device__ __forceinline__ void st4(void* base, int dt, int64_t idx, const float* v, int n_ok) {
  if (n_ok == 4) {
    if (dt == DT_BF16) {
      if ((idx & 3) == 0) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
        uint2 w;
        w.x = *reinterpret_cast<uint32_t*>(&lo);
        w.y = *reinterpret_cast<uint32_t*>(&hi);
        *reinterpret_cast<uint2*>(static_cast<bf16*>(base) + idx) = w;
        return;
      }
    } else if ((idx & 3) == 0) {
      *reinterpret_cast<float4*>(static_cast<float*>(base) + idx) = make_float4(v[0], v[1], v[2], v[3]);
      return;
    }
  }
  for (int j = 0; j < n_ok; ++j) st_el(base, dt, idx + j, v[j]);
}

// One element of the epilogue (all but the partial and the split, which the
// caller handles); n < Nc.
__device__ __forceinline__ float epi_value(const GemmArgs& g, int64_t m, int n, int nval, float v) {
  switch (g.epi) {
    case EPI_BIAS_RELU:
    case EPI_RELU_BITS:
      v += g.bias[n];
      return v > 0.f ? v : 0.f;
    case EPI_BIAS:
      return n < nval ? v + g.bias[n] : 0.f;
    case EPI_BIAS_SIGMOID:
      if (g.addend && n < nval)
        v += g.d_add == DT_BF16
                 ? __bfloat162float(static_cast<const bf16*>(g.addend)[m * g.ld_add + n])
                 : static_cast<const float*>(g.addend)[m * g.ld_add + n];
      return (n < nval) ? 1.0f / (1.0f + expf(-(v + g.bias[n]))) : 0.f;
    default:
      return v;
  }
}

// 128 x 128 output tile per block of 256 threads; thread (tx, ty) of a
// 16 x 16 grid owns the 8 x 8 outputs at rows {4ty, 64 + 4ty} + 0..3 and
// columns {4tx, 64 + 4tx} + 0..3, read from shared memory as float4.  K is
// staged in slices of 16, double-buffered: the next slice is loaded into
// registers while the current one is multiplied.
template <typename TA, typename TB, bool AK, bool BKM>
__global__ void __launch_bounds__(256, 2)
gemm_simt_kernel(GemmArgs g) {
  __shared__ __align__(16) float As[2][BK][BM + 4];
  __shared__ __align__(16) float Bs[2][BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int n0 = blockIdx.y * BN;
  const int nval = g.n_valid > 0 ? g.n_valid : g.Nc;
  int64_t kbeg = 0, kend = g.K;
  if (g.epi == EPI_PARTIAL && gridDim.z > 1) {
    const int64_t per = ((g.K + gridDim.z - 1) / gridDim.z + BK - 1) / BK * BK;
    kbeg = per * blockIdx.z;
    kend = kbeg + per < g.K ? kbeg + per : g.K;
  }

  // element e of this thread's share of a 128 x 16 slice: index id = e*256 + tid,
  // laid out so that consecutive threads read consecutive addresses
  float ra[8], rb[8];
  auto load = [&](int64_t k0) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int id = e * 256 + tid;
      int mm, kk;
      if (AK) { mm = id / BK; kk = id % BK; }
      else { kk = id / BM; mm = id % BM; }
      const int64_t m = m0 + mm, k = k0 + kk;
      ra[e] = (m < g.M && k < kend) ? ld_el<TA>(g.A, AK ? m * g.lda + k : k * g.lda + m) : 0.f;
      int nn;
      if (BKM) { nn = id / BK; kk = id % BK; }
      else { kk = id / BN; nn = id % BN; }
      const int n = n0 + nn;
      const int64_t kb = k0 + kk;
      rb[e] = (n < nval && kb < kend)
                  ? ld_el<TB>(g.B, BKM ? (int64_t)n * g.ldb + kb : kb * g.ldb + n)
                  : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      const int id = e * 256 + tid;
      if (AK) As[buf][id % BK][id / BK] = ra[e];
      else As[buf][id / BM][id % BM] = ra[e];
      if (BKM) Bs[buf][id % BK][id / BK] = rb[e];
      else Bs[buf][id / BN][id % BN] = rb[e];
    }
  };

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  int buf = 0;
  if (kbeg < kend) {
    load(kbeg);
    store(0);
  }
  __syncthreads();
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
    const bool more = k0 + BK < kend;
    if (more) load(k0 + BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[8], b[8];
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][4 * ty]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + 4 * ty]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][4 * tx]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + 4 * tx]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
      b[0] = b0.x; b[1] = b0.y; b[2] = b0.z; b[3] = b0.w;
      b[4] = b1.x; b[5] = b1.y; b[6] = b1.z; b[7] = b1.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }

  // ReLU mask as bits: lanes 0-15 of a warp hold row 4ty + i of an even ty,
  // lanes 16-31 the same row of the odd ty; lane tx holds columns 4tx + j of
  // each half.  Four ballots (one per j) give both rows' 64 columns.
  if (g.epi == EPI_RELU_BITS || (g.epi == EPI_BIAS_RELU && g.out1)) {
    const bool only_bits = g.epi == EPI_RELU_BITS;
    uint16_t* mb = static_cast<uint16_t*>(only_bits ? g.out0 : g.out1);
    const int64_t ldm = only_bits ? g.ld0 : g.ld1;
    const int lane = tid & 31;
    const int base = lane & 16;  // this row's lanes start here
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int64_t m = m0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + (i - 4));
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        unsigned bal[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n = n0 + 64 * h + 4 * tx + j;
          bool bit = false;
          if (m < g.M && n < g.Nc) {
            float v = epi_value(g, m, n, nval, acc[i][4 * h + j]);
            if (g.d0 == DT_BF16) v = __bfloat162float(__float2bfloat16_rn(v));
            bit = v > 0.f;
          }
          bal[j] = __ballot_sync(0xffffffffu, bit);
        }
        // 16-column block q of this half comes from lanes 4q .. 4q+3 (of the row)
        if ((tx & 3) == 0) {
          const int q = tx >> 2;
          uint32_t word = 0;
#pragma unroll
          for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int j = 0; j < 4; ++j) word |= ((bal[j] >> (base + 4 * q + t)) & 1u) << (4 * t + j);
          const int nb = n0 + 64 * h + 16 * q;
          if (m < g.M && nb < g.Nc) mb[m * ldm + nb / 16] = static_cast<uint16_t>(word);
        }
      }
    }
    if (only_bits) return;
  }

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t m = m0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + (i - 4));
    if (m >= g.M) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = n0 + 64 * h + 4 * tx;
      if (n >= g.Nc) continue;
      const int n_ok = g.Nc - n < 4 ? g.Nc - n : 4;
      float v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = acc[i][4 * h + j];
      switch (g.epi) {
        case EPI_PARTIAL:
          st4(g.out0, DT_F32, (int64_t)blockIdx.z * g.M * g.ld0 + m * g.ld0 + n, v, n_ok);
          break;
        case EPI_SPLIT:  // split is a multiple of 16: the four columns sit on one side
          if (n < g.split) {
            st4(g.out0, g.d0, m * g.ld0 + n, v, n_ok);
          } else {
            const float sc = g.row_scale[m];
#pragma unroll
            for (int j = 0; j < 4; ++j) v[j] *= sc;
            st4(g.out1, g.d1, m * g.ld1 + (n - g.split), v, n_ok);
          }
          break;
        default:
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (j < n_ok) v[j] = epi_value(g, m, n + j, nval, v[j]);
          st4(g.out0, g.d0, m * g.ld0 + n, v, n_ok);
          break;
      }
    }
  }
}

// Split-K sums in a fixed order: thread (x, y) of a 32 x 32 block adds the
// splits z = y, y + 32, ... of output blockIdx.x * 32 + x (32 independent
// load chains per output instead of one), then row y = 0 adds the 32 slices
// in ascending order.
__global__ void splitk_reduce_kernel(const float* __restrict__ part, int splits, int M,
                                     int Nc, int64_t ldp, float* out, int64_t ldo) {
  __shared__ float sl[32][33];
  const int x = threadIdx.x, y = threadIdx.y;
  const int64_t idx = (int64_t)blockIdx.x * 32 + x;
  const bool valid = idx < (int64_t)M * Nc;
  const int r = valid ? (int)(idx / Nc) : 0, c = valid ? (int)(idx % Nc) : 0;
  float t = 0.f;
  if (valid)
    for (int z = y; z < splits; z += 32) t += part[(int64_t)z * M * ldp + (int64_t)r * ldp + c];
  sl[y][x] = t;
  __syncthreads();
  if (y == 0 && valid) {
    float u = 0.f;
    for (int k = 0; k < 32; ++k) u += sl[k][x];
    out[(int64_t)r * ldo + c] = u;
  }
}

// The same sums, in the same order for every output, four outputs per
// thread: thread (x, y) owns the 16-byte vector x of a 128-output group and
// the splits z = y, y + 32, ...; it issues up to 8 of those vector loads
// before adding any of them, so one L2 round trip covers 256 splits (the
// partials were just written and sit in L2).  The grid is a quarter of the
// scalar kernel's and each thread keeps eight loads in flight instead of one.
__global__ void __launch_bounds__(1024, 1)
splitk_reduce4_kernel(const float* __restrict__ part, int splits, int M, int Nc, int64_t ldp,
                      float* out, int64_t ldo) {
  __shared__ float4 sl[32][32];
  const int x = threadIdx.x, y = threadIdx.y;
  const int64_t q = (int64_t)blockIdx.x * 32 + x;  // vector index over M * Nc / 4
  const bool valid = q < (int64_t)M * Nc / 4;
  const int64_t e = valid ? 4 * q : 0;
  const int r = (int)(e / Nc), c = (int)(e % Nc);
  const float* src = part + (int64_t)r * ldp + c;
  const int64_t zs = (int64_t)M * ldp;
  float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid) {
    for (int z0 = y; z0 < splits; z0 += 32 * 8) {
      float4 v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int z = z0 + 32 * u;
        v[u] = z < splits ? *reinterpret_cast<const float4*>(src + (int64_t)z * zs)
                          : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (z0 + 32 * u < splits) {
          t.x += v[u].x;
          t.y += v[u].y;
          t.z += v[u].z;
          t.w += v[u].w;
        }
      }
    }
  }
  sl[y][x] = t;
  __syncthreads();
  if (y == 0 && valid) {
    float4 u = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int k = 0; k < 32; ++k) {
      const float4 s = sl[k][x];
      u.x += s.x;
      u.y += s.y;
      u.z += s.z;
      u.w += s.w;
    }
    *reinterpret_cast<float4*>(out + (int64_t)r * ldo + c) = u;
  }
}

}  // namespace

template <typename TA, typename TB>
void launch_layout(const GemmArgs& g, dim3 grid, cudaStream_t st) {
  if (g.a_kmajor) {
    if (g.b_kmajor) gemm_simt_kernel<TA, TB, true, true><<<grid, 256, 0, st>>>(g);
    else gemm_simt_kernel<TA, TB, true, false><<<grid, 256, 0, st>>>(g);
  } else {
    if (g.b_kmajor) gemm_simt_kernel<TA, TB, false, true><<<grid, 256, 0, st>>>(g);
    else gemm_simt_kernel<TA, TB, false, false><<<grid, 256, 0, st>>>(g);
  }
}

template <int D> struct SimtType { using T = float; };
template <> struct SimtType<DT_BF16> { using T = bf16; };

template <>
void gemm_simt_launch_typed<CPRA_SIMT_DA, CPRA_SIMT_DB>(const GemmArgs& g, dim3 grid,
                                                        cudaStream_t st) {
  launch_layout<SimtType<CPRA_SIMT_DA>::T, SimtType<CPRA_SIMT_DB>::T>(g, grid, st);
}

#if CPRA_SIMT_DA == DT_F32 && CPRA_SIMT_DB == DT_F32
void gemm_simt_launch(const GemmArgs& g, cudaStream_t st) {
  dim3 grid((unsigned)((g.M + BM - 1) / BM), (unsigned)((g.Nc + BN - 1) / BN),
            g.epi == EPI_PARTIAL ? (unsigned)g.splits : 1u);
  if (g.da == DT_BF16) {
    if (g.db == DT_BF16) gemm_simt_launch_typed<DT_BF16, DT_BF16>(g, grid, st);
    else gemm_simt_launch_typed<DT_BF16, DT_F32>(g, grid, st);
  } else {
    if (g.db == DT_BF16) gemm_simt_launch_typed<DT_F32, DT_BF16>(g, grid, st);
    else gemm_simt_launch_typed<DT_F32, DT_F32>(g, grid, st);
  }
}

void splitk_reduce(const float* part, int splits, int M, int Nc, int64_t ldp, float* out,
                   int64_t ldo, cudaStream_t st) {
  const int64_t n = (int64_t)M * Nc;
  const bool vec = Nc % 4 == 0 && ldp % 4 == 0 && ldo % 4 == 0 &&
                   reinterpret_cast<uintptr_t>(part) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(out) % 16 == 0;
  if (vec) {
    splitk_reduce4_kernel<<<(unsigned)((n / 4 + 31) / 32), dim3(32, 32), 0, st>>>(
        part, splits, M, Nc, ldp, out, ldo);
    return;
  }
  splitk_reduce_kernel<<<(unsigned)((n + 31) / 32), dim3(32, 32), 0, st>>>(part, splits, M, Nc,
                                                                           ldp, out, ldo);
}
#endif

}  // namespace cpra
