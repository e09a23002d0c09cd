// Fused SpMM + relaxed CPRA loss + rounding/integer evaluation.
//
// For each node i a segment of LPR lanes gathers the neighbour rows P_j.
// (S floats each, 16 bytes per lane per vector) and accumulates
// Q_i = (A P)_i in registers; Q is never written.  The epilogue, still in
// registers, evaluates per shot s (Eq. CPRA-loss-function-GNN-penalty /
// -variation with the QUBOs of Table objective-functions):
//   MIS     cost -= P_is, pen += 1/2 P_is Q_is, dR/dP = -1 + lambda_s Q_is
//   MaxCut  cost += P_is Q_is - deg_i P_is,      dR/dP = 2 Q_is - deg_i
//   ann    += 1 - (2P_is - 1)^alpha,  dR/dP += -2 alpha gamma (2P_is-1)^(alpha-1)
//   Psi: row mean / variance over the S shots by segment shuffles (O(S) per
//   node, Prop. 3.2), dR/dP += nu * dPsi/dP_is
// and writes G = dR/dP * P (1 - P) (the sigmoid head's dR/dZ2).  The same
// gathered values give the rounding x = 1[P > 0.5f] (App. C.2) of both ends
// of every edge, so MIS violations / MaxCut cuts per shot are counted here
// too, exactly, with integer reductions (each edge at its lower endpoint).
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace cpra {

int64_t loss_pstride(int S) { return ((int64_t)4 * S + 1 + 3) / 4 * 4; }

template <int LPR, int CPL, int PROBLEM, typename TG, bool DO_LOSS>
__global__ void __launch_bounds__(256, 2)
loss_kernel(LossArgs a) {
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LPR - 1);
  const unsigned smask = segment_mask<LPR>(lane);
  const int segs_per_warp = 32 / LPR;
  const int64_t segs_per_block = (int64_t)(blockDim.x >> 5) * segs_per_warp;
  const int64_t first = (int64_t)blockIdx.x * segs_per_block +
                        (threadIdx.x >> 5) * segs_per_warp + lane / LPR;
  const int64_t stride = (int64_t)gridDim.x * segs_per_block;
  const int S = a.S;
  const int nchS = (S + 3) / 4;                       // chunks holding data
  const int nchG = DO_LOSS ? (int)(a.ldg / 4) : nchS;  // chunks written to G
  const float* __restrict__ P = a.P;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;

  extern __shared__ float red[];  // [nwarps][S] floats, reused
  __shared__ int icnt[2 * 1024];
  __shared__ unsigned long long ham_s;
  for (int k = threadIdx.x; k < 2 * S; k += blockDim.x) icnt[k] = 0;
  if (threadIdx.x == 0) ham_s = 0ull;
  __syncthreads();

  float lam[CPL][4];
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int s = (c * LPR + sub) * 4 + e;
      lam[c][e] = (PROBLEM == 0 && DO_LOSS && s < S) ? a.lambda[s] : 0.f;
    }

  float pc[CPL][4], pp[CPL][4], pa[CPL][4], pg[CPL][4];
  int cobj[CPL][4], cviol[CPL][4];
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      pc[c][e] = pp[c][e] = pa[c][e] = pg[c][e] = 0.f;
      cobj[c][e] = cviol[c][e] = 0;
    }
  float psi = 0.f;
  long long ham = 0;

  for (int64_t i = first; i < a.N; i += stride) {
    float p[CPL][4];
    bool xi[CPL][4];
    int kones = 0;
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int ch = c * LPR + sub;
      if (ch < nchS) {
        load16(P + i * a.ldp + ch * 4, p[c]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) p[c][e] = 0.f;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int s = ch * 4 + e;
        xi[c][e] = (s < S) && (p[c][e] > 0.5f);
        kones += xi[c][e] ? 1 : 0;
        if (PROBLEM == 0) cobj[c][e] += xi[c][e] ? 1 : 0;
      }
    }

    float q[CPL][4];
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) q[c][e] = 0.f;

    const int beg = a.rowptr[i];
    const int end = a.rowptr[i + 1];
    for (int eb = beg; eb < end; eb += LPR) {
      const int ee = eb + sub;
      const int jl = (ee < end) ? a.col[ee] : 0;
      const int cnt = min(LPR, end - eb);
      int k = 0;
      for (; k + 4 <= cnt; k += 4) {
        uint4 raw[4][CPL];
        int js[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          js[u] = __shfl_sync(smask, jl, k + u, LPR);
          const float* row = P + (int64_t)js[u] * a.ldp;
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const int ch = c * LPR + sub;
            raw[u][c] = (ch < nchS) ? ldg_nc16(row + ch * 4) : make_uint4(0, 0, 0, 0);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const bool upper = js[u] > i;
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            float f[4];
            widen(raw[u][c], f, (const float*)nullptr);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              q[c][e] += f[e];
              const bool xj = f[e] > 0.5f;
              if (PROBLEM == 0) cviol[c][e] += (upper && xi[c][e] && xj) ? 1 : 0;
              else cobj[c][e] += (upper && (xi[c][e] != xj) && (c * LPR + sub) * 4 + e < S) ? 1 : 0;
            }
          }
        }
      }
      for (; k < cnt; ++k) {
        const int j = __shfl_sync(smask, jl, k, LPR);
        const bool upper = j > i;
        const float* row = P + (int64_t)j * a.ldp;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int ch = c * LPR + sub;
          if (ch < nchS) {
            float f[4];
            widen(ldg_nc16(row + ch * 4), f, (const float*)nullptr);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              q[c][e] += f[e];
              const bool xj = f[e] > 0.5f;
              if (PROBLEM == 0) cviol[c][e] += (upper && xi[c][e] && xj) ? 1 : 0;
              else cobj[c][e] += (upper && (xi[c][e] != xj) && ch * 4 + e < S) ? 1 : 0;
            }
          }
        }
      }
    }

    // pairwise Hamming contribution k_i (S - k_i) (Prop. 3.2)
#pragma unroll
    for (int off = LPR / 2; off > 0; off >>= 1) kones += __shfl_xor_sync(smask, kones, off);
    if (sub == 0) ham += (long long)kones * (long long)(S - kones);

    if (a.xbits) {
      const int W = (S + 31) / 32;
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        uint32_t nib = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) nib |= (xi[c][e] ? 1u : 0u) << e;
        uint32_t word = nib << ((sub & 7) * 4);
        if constexpr (LPR >= 8) {
          word = seg_or<8>(word, smask);
        } else {
          word = seg_or<LPR>(word, smask);
        }
        const int widx = (c * LPR + (sub & ~7)) / 8;
        if ((sub & 7) == 0 && widx < W) a.xbits[i * W + widx] = word;
      }
    }

    if constexpr (DO_LOSS) {
      const float deg = (float)(end - beg);
      // Row statistics over the S shots: Psi is reported even when nu = 0.
      float mean = 0.f, rstd = 0.f;
      {
        float sum = 0.f, mx = -INFINITY, mn = INFINITY;
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if ((c * LPR + sub) * 4 + e < S) {
              sum += p[c][e];
              mx = fmaxf(mx, p[c][e]);
              mn = fminf(mn, p[c][e]);
            }
          }
        sum = seg_sum<LPR>(sum, smask);
        mx = seg_max<LPR>(mx, smask);
        mn = seg_min<LPR>(mn, smask);
        mean = sum / (float)S;
        float d2 = 0.f;
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if ((c * LPR + sub) * 4 + e < S) {
              const float d = p[c][e] - mean;
              d2 += d * d;
            }
        d2 = seg_sum<LPR>(d2, smask);
        const bool zero_var = (mx == mn);
        const float var = zero_var ? 0.f : d2 / (float)S;
        if (a.div_kind == 0) {
          rstd = zero_var ? 0.f : 1.0f / sqrtf(var);
          if (sub == 0) psi += -(float)S * sqrtf(var);
        } else {
          if (sub == 0) psi += -(float)S * (float)S * var;
        }
      }
      const float c_ann = -2.f * (float)a.alpha * a.gamma;
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int ch = c * LPR + sub;
        if (ch >= nchG) continue;
        float out[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int s = ch * 4 + e;
          const float pv = p[c][e], qv = q[c][e];
          float g;
          if (PROBLEM == 0) {
            g = -1.f + lam[c][e] * qv;
          } else {
            g = 2.f * qv - deg;
          }
          const float t = 2.f * pv - 1.f;
          float tp = t;  // t^(alpha-1)
          for (int r = 2; r < a.alpha; ++r) tp *= t;
          g += c_ann * tp;
          if (a.nu != 0.f) {
            const float d = pv - mean;
            g += a.nu * ((a.div_kind == 0) ? -d * rstd : -2.f * (float)S * d);
          }
          if (a.grad_kind == 0) g *= pv * (1.f - pv);
          if (s < S) {
            if (PROBLEM == 0) {
              pc[c][e] -= pv;
              pp[c][e] += 0.5f * pv * qv;
            } else {
              pc[c][e] += pv * qv - deg * pv;
            }
            pa[c][e] += 1.f - tp * t;
            pg[c][e] += g;
          } else {
            g = 0.f;
          }
          out[e] = g;
        }
        storeN<4>(static_cast<TG*>(a.G) + i * a.ldg + ch * 4, out);
      }
    }
  }

  // ---------------- block reductions (fixed order for floats) ----------------
  __syncwarp();
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int off = LPR; off < 32; off <<= 1) {
        cobj[c][e] += __shfl_xor_sync(0xffffffffu, cobj[c][e], off);
        cviol[c][e] += __shfl_xor_sync(0xffffffffu, cviol[c][e], off);
        if constexpr (DO_LOSS) {
          pc[c][e] += __shfl_xor_sync(0xffffffffu, pc[c][e], off);
          pp[c][e] += __shfl_xor_sync(0xffffffffu, pp[c][e], off);
          pa[c][e] += __shfl_xor_sync(0xffffffffu, pa[c][e], off);
          pg[c][e] += __shfl_xor_sync(0xffffffffu, pg[c][e], off);
        }
      }
  // integer counters: shared-memory atomics, then one global atomic per shot
  if (lane < LPR) {
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int s = (c * LPR + sub) * 4 + e;
        if (s < S) {
          if (cobj[c][e]) atomicAdd(&icnt[s], cobj[c][e]);
          if (cviol[c][e]) atomicAdd(&icnt[S + s], cviol[c][e]);
        }
      }
  }
  if (ham) atomicAdd(&ham_s, (unsigned long long)ham);
  if constexpr (DO_LOSS) {
    psi = seg_sum<32>(psi, 0xffffffffu);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * S; k += blockDim.x)
    if (icnt[k]) atomicAdd(&a.counters[k], (unsigned long long)icnt[k]);
  if (threadIdx.x == 0 && ham_s) atomicAdd(&a.counters[2 * S], ham_s);

  if constexpr (DO_LOSS) {
    float* outp = a.partials + (int64_t)blockIdx.x * a.pstride;
    // psi: one value per warp
    __syncthreads();
    if (lane == 0) red[warp] = psi;
    __syncthreads();
    if (threadIdx.x == 0) {
      float t = 0.f;
      for (int w = 0; w < nwarps; ++w) t += red[w];
      outp[3 * S] = t;
    }
    for (int qd = 0; qd < 4; ++qd) {
      __syncthreads();
      if (lane < LPR) {
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int s = (c * LPR + sub) * 4 + e;
            if (s < S) {
              const float v = qd == 0 ? pc[c][e] : qd == 1 ? pp[c][e] : qd == 2 ? pa[c][e] : pg[c][e];
              red[warp * S + s] = v;
            }
          }
      }
      __syncthreads();
      const int base = qd < 3 ? qd * S : 3 * S + 1;
      for (int s = threadIdx.x; s < S; s += blockDim.x) {
        float t = 0.f;
        for (int w = 0; w < nwarps; ++w) t += red[w * S + s];
        outp[base + s] = t;
      }
    }
  }
}

template <int LPR, int CPL, int PROBLEM, typename TG, bool DO_LOSS>
static int launch_loss_t(const LossArgs& a, int max_grid, cudaStream_t st) {
  constexpr int threads = 256;
  const int segs_per_block = (threads / 32) * (32 / LPR);
  int64_t want = (a.N + segs_per_block - 1) / segs_per_block;
  int grid = (int)(want < max_grid ? want : max_grid);
  if (grid < 1) grid = 1;
  const size_t smem = (size_t)(threads / 32) * (a.S > 0 ? a.S : 1) * sizeof(float);
  loss_kernel<LPR, CPL, PROBLEM, TG, DO_LOSS><<<grid, threads, smem, st>>>(a);
  return grid;
}

template <int PROBLEM, typename TG, bool DO_LOSS>
static int dispatch_loss(const LossArgs& a, int nch, int max_grid, cudaStream_t st) {
  if (nch <= 2) return launch_loss_t<2, 1, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  if (nch <= 4) return launch_loss_t<4, 1, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  if (nch <= 8) return launch_loss_t<8, 1, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  if (nch <= 16) return launch_loss_t<16, 1, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  if (nch <= 32) return launch_loss_t<32, 1, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  if (nch <= 64) return launch_loss_t<32, 2, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  if (nch <= 128) return launch_loss_t<32, 4, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  return launch_loss_t<32, 8, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
}

int loss_launch(const LossArgs& a, int max_grid, cudaStream_t st) {
  if (max_grid > kLossMaxGrid) max_grid = kLossMaxGrid;
  if (!a.do_loss) {
    const int nch = (a.S + 3) / 4;
    if (a.problem == 0) return dispatch_loss<0, float, false>(a, nch, max_grid, st);
    return dispatch_loss<1, float, false>(a, nch, max_grid, st);
  }
  const int nch = (int)(a.ldg / 4);
  if (a.problem == 0) {
    if (a.dg == DT_BF16) return dispatch_loss<0, bf16, true>(a, nch, max_grid, st);
    return dispatch_loss<0, float, true>(a, nch, max_grid, st);
  }
  if (a.dg == DT_BF16) return dispatch_loss<1, bf16, true>(a, nch, max_grid, st);
  return dispatch_loss<1, float, true>(a, nch, max_grid, st);
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

struct ShotEvalRec {
  long long objective;
  long long violations;
  double qubo;
};

__global__ void eval_finalize_kernel(const unsigned long long* __restrict__ cnt, int S,
                                     int problem, const float* __restrict__ lambda,
                                     ShotEvalRec* out, long long* ham) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < S) {
    const long long obj = (long long)cnt[s];
    const long long viol = (long long)cnt[S + s];
    double qubo;
    if (problem == 0) qubo = -(double)obj + (double)lambda[s] * (double)viol;
    else qubo = -(double)obj;
    out[s].objective = obj;
    out[s].violations = (problem == 0) ? viol : 0;
    out[s].qubo = qubo;
  }
  if (s == 0 && ham) *ham = (long long)cnt[2 * S];
}

void eval_finalize(const unsigned long long* counters, int S, int problem,
                   const float* lambda, void* out_records, long long* pair_hamming,
                   cudaStream_t st) {
  eval_finalize_kernel<<<(S + 255) / 256, 256, 0, st>>>(
      counters, S, problem, lambda, static_cast<ShotEvalRec*>(out_records), pair_hamming);
}

}  // namespace cpra
