// Diverse bipartite matching (App. problem specification, Eq.
// matching-cost-function) on the relaxed matching P and on its rounding.
//
// The variables x_ij of an N1 x N2 matching live at node i*N2 + j.  The
// loss couples them only through line sums: the row sums R_i = sum_j x_ij,
// the column sums K_j = sum_i x_ij, the total T = sum x and the cross-field
// total U = sum M x.  With those known, every element's derivative is local:
//   dl/dx_ij = -C_ij + lambda_1 1[R_i > 1] + lambda_2 1[K_j > 1]
//              + lambda_3 1[pT - U > 0] (p - M_ij)
//              + lambda_4 1[qT - (T - U) > 0] (q - 1 + M_ij)
//            = -C_ij + rowc_i + colc_j + b + d M_ij
// with ReLU'(0) = 0.  So a training step first forms the line sums here
// (one thread per (line, shot), lines and shots in a fixed order, no
// atomics), then the loss kernel's problem-2 epilogue applies the formula
// per element next to the annealing and diversity terms.  Each shot s has
// its own instance (C_s, M_s, lambda_s, p_s, q_s): the penalty grid and the
// multi-instance form of CPRA (App. multi-instance) are both this layout.
//
// The rounded matchings are evaluated exactly the same way: line counts of
// the rounding bits, FP64 sums of C x and M x per row line, then one thread
// per shot adds the lines in order and applies the constraints in FP64.
//
// The GNN's own graph, the constraint graph (pairs adjacent when they share
// a row or a column), is aggregated through line sums as well: the
// neighbour sum of pair (r, k) is R_r + K_k - 2 x_(r,k), with R, K the line
// sums of the activation block (line_sums_kernel, O(N H) instead of the
// (N1 + N2 - 2) N H of a gathered SpMM).
#include "common.cuh"
#include "kernels.cuh"

namespace cpra {

namespace {

constexpr int kLineThreads = 128;

__global__ void __launch_bounds__(kLineThreads)
dbm_lines_kernel(DbmDev d, int S, const float* __restrict__ P, int64_t ldp) {
  const int s = blockIdx.y * kLineThreads + threadIdx.x;
  if (s >= S) return;
  const int b = blockIdx.x;
  const int64_t ld = d.ld;
  float* line = d.line + (int64_t)b * 3 * ld;
  if (b < d.N1) {
    const int64_t n0 = (int64_t)b * d.N2;
    float R = 0.f, U = 0.f;
    for (int j = 0; j < d.N2; ++j) {
      const float v = P[(n0 + j) * ldp + s];
      R += v;
      U = fmaf(d.M[(n0 + j) * ld + s], v, U);
    }
    d.rowc[(int64_t)b * ld + s] = R > 1.f ? d.lam4[4 * s + 0] : 0.f;
    line[s] = fmaxf(R - 1.f, 0.f);
    line[ld + s] = R;
    line[2 * ld + s] = U;
  } else {
    const int j = b - d.N1;
    float K = 0.f;
    for (int i = 0; i < d.N1; ++i) K += P[((int64_t)i * d.N2 + j) * ldp + s];
    d.colc[(int64_t)j * ld + s] = K > 1.f ? d.lam4[4 * s + 1] : 0.f;
    line[s] = fmaxf(K - 1.f, 0.f);
  }
}

// One warp per shot: lane l takes lines l, l + 32, ... and the lanes' partial
// sums meet in a fixed butterfly.
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ long long warp_sum(long long v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__global__ void dbm_shot_kernel(DbmDev d, int S) {
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s >= S) return;
  const int64_t ld = d.ld;
  float er = 0.f, ec = 0.f, T = 0.f, U = 0.f;
  for (int b = lane; b < d.N1; b += 32) {
    const float* line = d.line + (int64_t)b * 3 * ld;
    er += line[s];
    T += line[ld + s];
    U += line[2 * ld + s];
  }
  for (int b = d.N1 + lane; b < d.N1 + d.N2; b += 32) ec += d.line[(int64_t)b * 3 * ld + s];
  er = warp_sum(er);
  T = warp_sum(T);
  U = warp_sum(U);
  ec = warp_sum(ec);
  if (lane) return;
  const float l1 = d.lam4[4 * s + 0], l2 = d.lam4[4 * s + 1];
  const float l3 = d.lam4[4 * s + 2], l4 = d.lam4[4 * s + 3];
  const float p = d.pq[2 * s + 0], q = d.pq[2 * s + 1];
  const float g3 = p * T - U;          // same-field shortfall
  const float g4 = q * T - (T - U);    // different-field shortfall
  const float a3 = g3 > 0.f ? l3 : 0.f;
  const float a4 = g4 > 0.f ? l4 : 0.f;
  d.shot[s] = a3 * p + a4 * (q - 1.f);
  d.shot[ld + s] = a4 - a3;
  d.shot[2 * ld + s] = l1 * er + l2 * ec + l3 * fmaxf(g3, 0.f) + l4 * fmaxf(g4, 0.f);
}

// hi + lo += v with the rounding error of hi + v kept in lo (TwoSum).
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
  const float s = __fadd_rn(hi, v);
  const float bp = __fadd_rn(s, -hi);
  const float err = __fadd_rn(__fadd_rn(hi, -__fadd_rn(s, -bp)), __fadd_rn(v, -bp));
  hi = s;
  lo = __fadd_rn(lo, err);
}

__device__ __forceinline__ int bit_of(const uint32_t* __restrict__ bits, int W, int64_t n, int s) {
  return (int)((bits[n * W + (s >> 5)] >> (s & 31)) & 1u);
}

__global__ void __launch_bounds__(kLineThreads)
dbm_eval_lines_kernel(DbmDev d, int S, const uint32_t* __restrict__ bits) {
  const int s = blockIdx.y * kLineThreads + threadIdx.x;
  if (s >= S) return;
  const int W = (S + 31) / 32;
  const int b = blockIdx.x;
  const int64_t ld = d.ld;
  int cnt = 0;
  if (b < d.N1) {
    const int64_t n0 = (int64_t)b * d.N2;
    // sums of M x and C x as unevaluated FP32 pairs (hi + lo, Knuth's
    // TwoSum at every addition): the FP64 pipe of this part is slow, and
    // the pair carries about 48 bits, enough for the FP64 totals
    float Uh = 0.f, Ul = 0.f, Vh = 0.f, Vl = 0.f;
    for (int j = 0; j < d.N2; ++j) {
      const int x = bit_of(bits, W, n0 + j, s);
      const float m = d.M[(n0 + j) * ld + s], c = d.C[(n0 + j) * ld + s];
      cnt += x;
      two_sum_acc(Uh, Ul, x ? m : 0.f);
      two_sum_acc(Vh, Vl, x ? c : 0.f);
    }
    d.eU[(int64_t)b * ld + s] = (double)Uh + (double)Ul;
    d.eC[(int64_t)b * ld + s] = (double)Vh + (double)Vl;
  } else {
    const int j = b - d.N1;
    for (int i = 0; i < d.N1; ++i) cnt += bit_of(bits, W, (int64_t)i * d.N2 + j, s);
  }
  d.ecnt[(int64_t)b * ld + s] = cnt;
}

__global__ void dbm_eval_finalize_kernel(DbmDev d, int S, const unsigned long long* counters,
                                         ShotEvalRec* out, long long* ham) {
  const int s = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (s == 0 && lane == 0 && ham) *ham = (long long)counters[2 * S];
  if (s >= S) return;
  const int64_t ld = d.ld;
  long long T = 0, over = 0, ex_r = 0, ex_c = 0;
  double U = 0.0, value = 0.0;
  for (int b = lane; b < d.N1; b += 32) {
    const int c = d.ecnt[(int64_t)b * ld + s];
    T += c;
    if (c > 1) { ++over; ex_r += c - 1; }
    U += d.eU[(int64_t)b * ld + s];
    value += d.eC[(int64_t)b * ld + s];
  }
  for (int b = d.N1 + lane; b < d.N1 + d.N2; b += 32) {
    const int c = d.ecnt[(int64_t)b * ld + s];
    if (c > 1) { ++over; ex_c += c - 1; }
  }
  T = warp_sum(T);
  over = warp_sum(over);
  ex_r = warp_sum(ex_r);
  ex_c = warp_sum(ex_c);
  U = warp_sum(U);
  value = warp_sum(value);
  if (lane) return;
  const double p = (double)d.pq[2 * s + 0], q = (double)d.pq[2 * s + 1];
  const double Td = (double)T;
  const double g3 = p * Td - U;
  const double g4 = q * Td - (Td - U);
  const double pen = (double)d.lam4[4 * s + 0] * (double)ex_r +
                     (double)d.lam4[4 * s + 1] * (double)ex_c +
                     (double)d.lam4[4 * s + 2] * (g3 > 0.0 ? g3 : 0.0) +
                     (double)d.lam4[4 * s + 3] * (g4 > 0.0 ? g4 : 0.0);
  out[s].objective = T;
  out[s].violations = over + (g3 > 0.0 ? 1 : 0) + (g4 > 0.0 ? 1 : 0);
  out[s].qubo = -value + pen;
  out[s].value = value;
}

// One thread per (line, column): the line's sum in index order.
template <typename TX>
__global__ void line_sums_kernel(int N1, int N2, int H, const TX* __restrict__ X, int64_t ldx,
                                 float* __restrict__ R, float* __restrict__ K, int64_t ldl) {
  const int h = blockIdx.y * blockDim.x + threadIdx.x;
  if (h >= H) return;
  const int b = blockIdx.x;
  float t = 0.f;
  if (b < N1) {
    const TX* row = X + (int64_t)b * N2 * ldx + h;
#pragma unroll 10
    for (int k = 0; k < N2; ++k) t += to_f(row[(int64_t)k * ldx]);
    R[(int64_t)b * ldl + h] = t;
  } else {
    const int k = b - N1;
    const TX* col = X + (int64_t)k * ldx + h;
#pragma unroll 10
    for (int r = 0; r < N1; ++r) t += to_f(col[(int64_t)r * N2 * ldx]);
    K[(int64_t)k * ldl + h] = t;
  }
}

}  // namespace

void dbm_line_sums_launch(int N1, int N2, int H, const void* X, int64_t ldx, int dx, float* R,
                          float* K, int64_t ldl, cudaStream_t st) {
  const dim3 grid(N1 + N2, (H + 127) / 128);
  if (dx == DT_BF16)
    line_sums_kernel<bf16><<<grid, 128, 0, st>>>(N1, N2, H, static_cast<const bf16*>(X), ldx, R, K, ldl);
  else
    line_sums_kernel<float><<<grid, 128, 0, st>>>(N1, N2, H, static_cast<const float*>(X), ldx, R, K, ldl);
}

void dbm_sums_launch(const DbmDev& d, int S, const float* P, int64_t ldp, cudaStream_t st) {
  const dim3 grid(d.N1 + d.N2, (S + kLineThreads - 1) / kLineThreads);
  dbm_lines_kernel<<<grid, kLineThreads, 0, st>>>(d, S, P, ldp);
  dbm_shot_kernel<<<(S + 3) / 4, 128, 0, st>>>(d, S);  // a warp per shot
}

void dbm_eval_launch(const DbmDev& d, int S, const uint32_t* bits,
                     const unsigned long long* counters, void* out_records,
                     long long* pair_hamming, cudaStream_t st) {
  const dim3 grid(d.N1 + d.N2, (S + kLineThreads - 1) / kLineThreads);
  dbm_eval_lines_kernel<<<grid, kLineThreads, 0, st>>>(d, S, bits);
  dbm_eval_finalize_kernel<<<(S + 3) / 4, 128, 0, st>>>(  // a warp per shot
      d, S, counters, static_cast<ShotEvalRec*>(out_records), pair_hamming);
}

}  // namespace cpra
