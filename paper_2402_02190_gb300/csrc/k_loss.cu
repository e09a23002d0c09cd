// Fused SpMM + relaxed CPRA loss + rounding: the host-side dispatch to the
// per-problem kernel instances (the kernels are in loss_impl.cuh, compiled
// once per problem from k_loss_problem.cu), and the fixed-order finalize
// kernels that sum the per-block partial rows.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace cpra {

int64_t loss_pstride(int S) { return ((int64_t)4 * S + 1 + 3) / 4 * 4; }

int loss_launch(const LossArgs& a, int max_grid, cudaStream_t st) {
  if (max_grid > kLossMaxGrid) max_grid = kLossMaxGrid;
  // The staged kernel runs two 256-thread blocks per SM (shared memory), so
  // half of the usual per-SM block budget keeps every block resident.
  int staged_grid = max_grid / 2;
  if (staged_grid < 1) staged_grid = 1;
  if (!a.do_loss) return loss_launch_bits(a, (a.S + 3) / 4, max_grid, st);  // no gathers
  const int nch = (int)(a.ldg / 4);
  if (a.problem == 0 && a.w) return loss_launch_problem<3>(a, nch, max_grid, staged_grid, st);
  if (a.problem == 0) return loss_launch_problem<0>(a, nch, max_grid, staged_grid, st);
  if (a.problem == 2) return loss_launch_problem<2>(a, nch, max_grid, staged_grid, st);
  if (a.ew) return loss_launch_problem<4>(a, nch, max_grid, staged_grid, st);
  return loss_launch_problem<1>(a, nch, max_grid, staged_grid, st);
}

// ---------------------------------------------------------------- finalize
// Column sums of the per-block partial rows in a fixed order: 32 strided
// slices per column, then the slices in ascending order.
__global__ void colsum_finalize_kernel(const float* __restrict__ part, int nblocks,
                                       int64_t pstride, int ncols, float* out,
                                       float* out2, int copy_from, int copy_n,
                                       int* err_flag) {
  __shared__ float sl[32][33];
  const int cx = threadIdx.x;  // column within tile
  const int sy = threadIdx.y;  // slice
  const int col = blockIdx.x * 32 + cx;
  float t = 0.f;
  if (col < ncols)
    for (int b = sy; b < nblocks; b += 32) t += part[(int64_t)b * pstride + col];
  sl[sy][cx] = t;
  __syncthreads();
  if (sy == 0 && col < ncols) {
    float r = 0.f;
    for (int k = 0; k < 32; ++k) r += sl[k][cx];
    out[col] = r;
    if (out2 && col >= copy_from && col < copy_from + copy_n) out2[col - copy_from] = r;
    if (err_flag && !isfinite(r)) atomicOr(err_flag, 1);
  }
}

void colsum_finalize(const float* part, int nblocks, int64_t pstride, int ncols,
                     float* out, float* out2, int copy_from, int copy_n, int* err_flag,
                     cudaStream_t st) {
  dim3 block(32, 32);
  dim3 grid((ncols + 31) / 32);
  colsum_finalize_kernel<<<grid, block, 0, st>>>(part, nblocks, pstride, ncols, out, out2,
                                                 copy_from, copy_n, err_flag);
}

__global__ void eval_finalize_kernel(const unsigned long long* __restrict__ cnt, int S,
                                     int problem, const float* __restrict__ lambda,
                                     const double* __restrict__ wvalue, ShotEvalRec* out,
                                     long long* ham) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S) {
    const long long obj = (long long)cnt[s];
    const long long viol = (long long)cnt[S + s];
    const double value = wvalue ? wvalue[s] : (double)obj;
    double qubo;
    if (problem == 0) qubo = -value + (double)lambda[s] * (double)viol;
    else qubo = -value;
    out[s].objective = obj;
    out[s].violations = (problem == 0) ? viol : 0;
    out[s].qubo = qubo;
    out[s].value = value;
  }
  if (s == 0 && ham) *ham = (long long)cnt[2 * S];
}

void eval_finalize(const unsigned long long* counters, int S, int problem,
                   const float* lambda, void* out_records, long long* pair_hamming,
                   cudaStream_t st, const double* wvalue) {
  eval_finalize_kernel<<<(S + 255) / 256, 256, 0, st>>>(
      counters, S, problem, lambda, wvalue, static_cast<ShotEvalRec*>(out_records), pair_hamming);
}

}  // namespace cpra
