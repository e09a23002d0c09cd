// Row-gather SpMM for the GCN aggregate step (Eq. GCN, App. B.1) and its
// adjoint.  One power-of-two segment of LPR lanes owns one node row; each lane
// moves 16-byte vectors, CPL of them per row.  Neighbour rows are gathered
// four at a time so that every lane keeps 4*CPL independent 16-byte loads in
// flight.
#include "common.cuh"
#include "kernels.cuh"

namespace cpra {

template <typename TX, typename TY, int LPR, int CPL>
__global__ void __launch_bounds__(256)
spmm_rows_kernel(SpmmArgs a) {
  constexpr int VEC = V16<TX>::n;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LPR - 1);
  const unsigned smask = segment_mask<LPR>(lane);
  const int segs_per_warp = 32 / LPR;
  const int64_t segs_per_block = (int64_t)(blockDim.x >> 5) * segs_per_warp;
  const int64_t first = (int64_t)blockIdx.x * segs_per_block +
                        (threadIdx.x >> 5) * segs_per_warp + lane / LPR;
  const int64_t stride = (int64_t)gridDim.x * segs_per_block;
  const int nchunks = a.H / VEC;
  const TX* __restrict__ X = static_cast<const TX*>(a.X);
  TY* __restrict__ Y = static_cast<TY*>(a.Y);
  const TX* __restrict__ ADD = static_cast<const TX*>(a.add);
  const TX* __restrict__ MASK = static_cast<const TX*>(a.mask);

  float csum[CPL][VEC];
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int v = 0; v < VEC; ++v) csum[c][v] = 0.f;

  for (int64_t i = first; i < a.N; i += stride) {
    float acc[CPL][VEC];
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[c][v] = 0.f;

    const int beg = a.rowptr[i];
    const int end = a.rowptr[i + 1];
    for (int eb = beg; eb < end; eb += LPR) {
      const int e = eb + sub;
      const int jl = (e < end) ? a.col[e] : 0;
      const int cnt = min(LPR, end - eb);
      int k = 0;
      for (; k + 4 <= cnt; k += 4) {
        uint4 raw[4][CPL];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = __shfl_sync(smask, jl, k + u, LPR);
          const TX* row = X + (int64_t)j * a.ldx;
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const int ch = c * LPR + sub;
            raw[u][c] = (ch < nchunks) ? ldg_nc16(row + ch * VEC) : make_uint4(0, 0, 0, 0);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            float f[VEC];
            widen(raw[u][c], f, (const TX*)nullptr);
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[c][v] += f[v];
          }
      }
      for (; k < cnt; ++k) {
        const int j = __shfl_sync(smask, jl, k, LPR);
        const TX* row = X + (int64_t)j * a.ldx;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int ch = c * LPR + sub;
          if (ch < nchunks) {
            float f[VEC];
            widen(ldg_nc16(row + ch * VEC), f, (const TX*)nullptr);
#pragma unroll
            for (int v = 0; v < VEC; ++v) acc[c][v] += f[v];
          }
        }
      }
    }

    const float s = a.mean ? a.inv_deg[i] : 1.f;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int ch = c * LPR + sub;
      if (ch >= nchunks) continue;
      float o[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) o[v] = acc[c][v];
      if (ADD) {
        float ad[VEC];
        load16(ADD + i * a.ldadd + ch * VEC, ad);
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[v] += ad[v];
      }
#pragma unroll
      for (int v = 0; v < VEC; ++v) o[v] *= s;
      if (MASK) {
        float mk[VEC];
        load16(MASK + i * a.ldm + ch * VEC, mk);
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[v] = (mk[v] > 0.f) ? o[v] : 0.f;
      }
#pragma unroll
      for (int v = 0; v < VEC; ++v) csum[c][v] += o[v];
      storeN<VEC>(Y + i * a.ldy + ch * VEC, o);
    }
  }

  if (a.colsum_partials == nullptr) return;
  // Fixed-order block reduction of the per-lane column sums.
  __syncwarp();
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int v = 0; v < VEC; ++v)
#pragma unroll
      for (int off = LPR; off < 32; off <<= 1)
        csum[c][v] += __shfl_xor_sync(0xffffffffu, csum[c][v], off);
  extern __shared__ float red[];  // [warps][H]
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  if (lane < LPR) {
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int ch = c * LPR + sub;
      if (ch < nchunks)
#pragma unroll
        for (int v = 0; v < VEC; ++v) red[warp * a.H + ch * VEC + v] = csum[c][v];
    }
  }
  __syncthreads();
  for (int col = threadIdx.x; col < a.H; col += blockDim.x) {
    float t = 0.f;
    for (int w = 0; w < nwarps; ++w) t += red[w * a.H + col];
    a.colsum_partials[(int64_t)blockIdx.x * a.H + col] = t;
  }
}

template <typename TX, typename TY, int LPR, int CPL>
static int launch_t(const SpmmArgs& a, int max_grid, cudaStream_t st) {
  constexpr int threads = 256;
  const int segs_per_block = (threads / 32) * (32 / LPR);
  int64_t want = (a.N + segs_per_block - 1) / segs_per_block;
  int grid = (int)(want < max_grid ? want : max_grid);
  if (grid < 1) grid = 1;
  const size_t smem = a.colsum_partials ? (size_t)(threads / 32) * a.H * sizeof(float) : 0;
  spmm_rows_kernel<TX, TY, LPR, CPL><<<grid, threads, smem, st>>>(a);
  return grid;
}

template <typename TX, typename TY>
static int dispatch_lpr(const SpmmArgs& a, int max_grid, cudaStream_t st) {
  const int nch = a.H / V16<TX>::n;
  if (nch <= 2) return launch_t<TX, TY, 2, 1>(a, max_grid, st);
  if (nch <= 4) return launch_t<TX, TY, 4, 1>(a, max_grid, st);
  if (nch <= 8) return launch_t<TX, TY, 8, 1>(a, max_grid, st);
  if (nch <= 16) return launch_t<TX, TY, 16, 1>(a, max_grid, st);
  if (nch <= 32) return launch_t<TX, TY, 32, 1>(a, max_grid, st);
  if (nch <= 64) return launch_t<TX, TY, 32, 2>(a, max_grid, st);
  if (nch <= 128) return launch_t<TX, TY, 32, 4>(a, max_grid, st);
  return launch_t<TX, TY, 32, 8>(a, max_grid, st);
}

int spmm_launch(const SpmmArgs& a, int max_grid, cudaStream_t st) {
  if (a.dx == DT_BF16) {
    if (a.dy == DT_BF16) return dispatch_lpr<bf16, bf16>(a, max_grid, st);
    return dispatch_lpr<bf16, float>(a, max_grid, st);
  }
  if (a.dy == DT_BF16) return dispatch_lpr<float, bf16>(a, max_grid, st);
  return dispatch_lpr<float, float>(a, max_grid, st);
}

}  // namespace cpra
