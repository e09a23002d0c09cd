// Kernels of the warm-start network (a three-layer Eq. GCN that predicts the
// S initial logits of a CPRA run): node features, degrees, the binary
// cross-entropy against rounded CPRA solutions, fixed-order column sums and
// BF16 weight copies.  The layers themselves run on the SpMM and GEMM
// kernels of the training step.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace cpra {

namespace {

unsigned grid_for_rows(int64_t n, int per_block) {
  int64_t g = (n + per_block - 1) / per_block;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

// Feature k of node i: 1 (k = 0), deg_i / 8 (k = 1), and N(0,1) draws from
// the counter-based stream (seed, i, k) for k >= 2.
__global__ void ws_features_kernel(int64_t N, const int* __restrict__ rowptr, uint64_t seed, int F,
                                   float* __restrict__ out) {
  const int64_t total = N * F;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / F;
    const int k = (int)(e % F);
    float v;
    if (k == 0) v = 1.f;
    else if (k == 1) v = (float)(rowptr[i + 1] - rowptr[i]) * 0.125f;
    else v = normal_at(seed, 0x5753ull, (uint64_t)e);
    out[e] = v;
  }
}

__global__ void inv_degree_kernel(int64_t N, const int* __restrict__ rowptr, float* __restrict__ inv) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int d = rowptr[i + 1] - rowptr[i];
    inv[i] = d > 0 ? 1.f / (float)d : 0.f;
  }
}

// One warp per row: G_is = (sigmoid(z_is) - y_is) * inv_count (0 in the pad
// columns), y_is = bit (s mod 32) of word s/32 of row i; the row's loss
// softplus(z) - y z = max(z, 0) - y z + log1p(exp(-|z|)) is accumulated per
// lane and reduced per block in a fixed order into partial[block] (scaled by
// inv_count, so the partials sum to the mean).
template <typename TG>
__global__ void __launch_bounds__(256)
ws_bce_kernel(int64_t N, int S, int S_pad, const float* __restrict__ Z, int64_t ldz,
              const uint32_t* __restrict__ bits, int W, TG* __restrict__ G, int64_t ldg,
              float inv_count, float* __restrict__ partial) {
  __shared__ float red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t wstride = (int64_t)gridDim.x * 8;
  float acc = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * 8 + warp; i < N; i += wstride) {
    for (int s = lane; s < S_pad; s += 32) {
      float g = 0.f;
      if (s < S) {
        const float z = Z[i * ldz + s];
        const float y = (float)((bits[i * W + (s >> 5)] >> (s & 31)) & 1u);
        const float p = 1.f / (1.f + expf(-z));
        g = (p - y) * inv_count;
        acc += fmaxf(z, 0.f) - y * z + log1pf(expf(-fabsf(z)));
      }
      G[i * ldg + s] = from_f<TG>(g);
    }
  }
  for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < 8; ++w) t += red[w];
    partial[blockIdx.x] = t * inv_count;
  }
}

// Block b sums rows [b*rows_per, (b+1)*rows_per) of X column by column, in
// row order, into partial[b*C + c].
template <typename TX>
__global__ void rows_colsum_kernel(int64_t N, int C, const TX* __restrict__ X, int64_t ldx,
                                   int64_t rows_per, float* __restrict__ partial) {
  const int64_t r0 = (int64_t)blockIdx.x * rows_per;
  const int64_t r1 = r0 + rows_per < N ? r0 + rows_per : N;
  for (int c = threadIdx.x; c < C; c += blockDim.x) {
    float t = 0.f;
    for (int64_t r = r0; r < r1; ++r) t += to_f(X[r * ldx + c]);
    partial[(int64_t)blockIdx.x * C + c] = t;
  }
}

// BF16 copies of a row-major FP32 weight W [rows x cols] for both operand
// orientations: Ws [rows_pad x cols] and Wt [cols x rows_pad] (rows past
// `rows` are zero).
__global__ void weight_pair_kernel(const float* __restrict__ W, int rows, int cols, int rows_pad,
                                   bf16* __restrict__ Ws, bf16* __restrict__ Wt) {
  const int64_t total = (int64_t)rows_pad * cols;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), k = (int)(e % cols);
    const bf16 w = __float2bfloat16_rn(r < rows ? W[(int64_t)r * cols + k] : 0.f);
    Ws[e] = w;
    Wt[(int64_t)k * rows_pad + r] = w;
  }
}

}  // namespace

void ws_features_launch(int64_t N, const int* rowptr, uint64_t seed, int F, float* out,
                        cudaStream_t st) {
  ws_features_kernel<<<grid_for_rows(N * F, 256), 256, 0, st>>>(N, rowptr, seed, F, out);
}

void inv_degree_launch(int64_t N, const int* rowptr, float* inv, cudaStream_t st) {
  inv_degree_kernel<<<grid_for_rows(N, 256), 256, 0, st>>>(N, rowptr, inv);
}

int ws_bce_launch(int64_t N, int S, int S_pad, const float* Z, int64_t ldz, const uint32_t* bits,
                  void* G, int64_t ldg, int dg, float inv_count, float* partial, int max_grid,
                  cudaStream_t st) {
  int64_t want = (N + 7) / 8;
  const int grid = (int)(want < max_grid ? (want < 1 ? 1 : want) : max_grid);
  const int W = (S + 31) / 32;
  if (dg == DT_BF16)
    ws_bce_kernel<bf16><<<grid, 256, 0, st>>>(N, S, S_pad, Z, ldz, bits, W, static_cast<bf16*>(G),
                                              ldg, inv_count, partial);
  else
    ws_bce_kernel<float><<<grid, 256, 0, st>>>(N, S, S_pad, Z, ldz, bits, W,
                                               static_cast<float*>(G), ldg, inv_count, partial);
  return grid;
}

int rows_colsum_launch(int64_t N, int C, const void* X, int64_t ldx, int dx, float* partial,
                       int max_blocks, cudaStream_t st) {
  int64_t rows_per = (N + max_blocks - 1) / max_blocks;
  if (rows_per < 1) rows_per = 1;
  const int blocks = (int)((N + rows_per - 1) / rows_per);
  if (dx == DT_BF16)
    rows_colsum_kernel<bf16><<<blocks < 1 ? 1 : blocks, 128, 0, st>>>(
        N, C, static_cast<const bf16*>(X), ldx, rows_per, partial);
  else
    rows_colsum_kernel<float><<<blocks < 1 ? 1 : blocks, 128, 0, st>>>(
        N, C, static_cast<const float*>(X), ldx, rows_per, partial);
  return blocks < 1 ? 1 : blocks;
}

void weight_pair_launch(const float* W, int rows, int cols, int rows_pad, void* Ws, void* Wt,
                        cudaStream_t st) {
  weight_pair_kernel<<<grid_for_rows((int64_t)rows_pad * cols, 256), 256, 0, st>>>(
      W, rows, cols, rows_pad, static_cast<bf16*>(Ws), static_cast<bf16*>(Wt));
}

}  // namespace cpra
