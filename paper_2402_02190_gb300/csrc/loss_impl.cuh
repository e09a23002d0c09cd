// Fused SpMM + relaxed CPRA loss + rounding.
//
// For each node i the lanes owning row i gather the neighbour rows P_j (S
// floats each) and accumulate Q_i = (A P)_i in registers; Q is never written.
// The epilogue, still in registers, evaluates per shot s (Eq.
// CPRA-loss-function-GNN-penalty / -variation with the QUBOs of Table
// objective-functions):
//   MIS     cost -= P_is, pen += 1/2 P_is Q_is, dR/dP = -1 + lambda_s Q_is
//   MaxCut  cost += P_is Q_is - deg_i P_is,      dR/dP = 2 Q_is - deg_i
//   DBM     cost -= C_is P_is, pen = the shot's penalty (added once, at row
//           0), dR/dP from the line sums of k_dbm.cu; no neighbour gathers
//   ann    += 1 - (2P_is - 1)^alpha (summed as 4P(1-P)(1 + t^2 + ...), t = 2P-1,
//             free of cancellation near 0 and 1),
//             dR/dP += -2 alpha gamma (2P_is-1)^(alpha-1)
//   Psi: row mean / variance over the S shots by lane shuffles (O(S) per
//   node, Prop. 3.2), dR/dP += nu * dPsi/dP_is
// writes G = dR/dP * P (1 - P) (the sigmoid head's dR/dZ2), and packs the
// rounding x = 1[P > 0.5f] (App. C.2) of row i into bits; the exact integer
// evaluation of those bits runs in k_eval.cu.
//
// The epilogue is instantiated per problem: 0 MIS, 1 MaxCut, 2 DBM,
// 3 weighted MIS (node weights w in place of the unit reward), 4 MaxCut with
// edge weights A_ij (Q_i = sum_j A_ij P_j, and the weighted degree
// sum_j A_ij in place of deg_i).
//
// Two kernels share the per-row epilogue:
//   loss_kernel         rows of up to 64 shots (and bit packing alone):
//                       segments of LPR lanes per row, neighbour rows
//                       gathered straight into registers;
//   loss_kernel_staged  rows of more than 64 shots: one warp per row; each
//                       warp bulk-copies (cp.async.bulk on one mbarrier per
//                       row) a row's own and neighbour P rows into shared
//                       memory, two rows ahead, so the gathers are in flight
//                       whatever the warp's register budget.
//
// This header holds the kernels and their launch templates; each problem's
// instances are compiled in their own object (k_loss_problem.cu, built once
// per problem), and k_loss.cu dispatches to them.
#pragma once

#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace cpra {

namespace {

constexpr uint32_t kLossSpinLimit = 1u << 26;

template <int CPL>
struct ShotAcc {
  float pc[CPL][4], pp[CPL][4], pa[CPL][4], pg[CPL][4];
  float psi;
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) pc[c][e] = pp[c][e] = pa[c][e] = pg[c][e] = 0.f;
    psi = 0.f;
  }
};

// Rounded bits of row i: bit (s mod 32) of word s/32 is 1[P_is > 0.5f].
template <int LPR, int CPL>
__device__ __forceinline__ void store_bits(const LossArgs& a, int64_t i, int sub, unsigned smask,
                                           const float (&p)[CPL][4]) {
  const int S = a.S;
  const int W = (S + 31) / 32;
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    uint32_t nib = 0;
#pragma unroll
    for (int e = 0; e < 4; ++e)
      nib |= (((c * LPR + sub) * 4 + e < S && p[c][e] > 0.5f) ? 1u : 0u) << e;
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

// Everything after Q_i is known: row statistics, dR/dP and the per-shot
// partial sums; stores G.
template <int LPR, int CPL, int PROBLEM, typename TG>
__device__ __forceinline__ void row_epilogue(const LossArgs& a, int64_t i, int sub, unsigned smask,
                                             const float (&p)[CPL][4], const float (&q)[CPL][4],
                                             float deg, const float (&lam)[CPL][4],
                                             float gamma, ShotAcc<CPL>& acc) {
  const int S = a.S;
  const int nchG = (int)(a.ldg / 4);
  // Row statistics over the S shots: Psi is reported even when nu = 0.
  float sum = 0.f, mx = -INFINITY, mn = INFINITY;
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if ((c * LPR + sub) * 4 + e < S) {
        sum += p[c][e];
        mx = fmaxf(mx, p[c][e]);
        mn = fminf(mn, p[c][e]);
      }
  sum = seg_sum<LPR>(sum, smask);
  mx = seg_max<LPR>(mx, smask);
  mn = seg_min<LPR>(mn, smask);
  const float inv_S = 1.0f / (float)S;
  const float mean = sum * inv_S;
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
  const float var = zero_var ? 0.f : d2 * inv_S;
  float rstd = 0.f;
  if (a.div_kind == 0) {
    rstd = zero_var ? 0.f : rsqrtf(var);
    if (sub == 0) acc.psi += -(float)S * sqrtf(var);
  } else {
    if (sub == 0) acc.psi += -(float)S * (float)S * var;
  }
  const float c_ann = -2.f * (float)a.alpha * gamma;
  const bool alpha2 = a.alpha == 2;
  const bool use_nu = a.nu != 0.f;
  const bool scale_g = a.grad_kind == 0;
#pragma unroll
  for (int c = 0; c < CPL; ++c) {
    const int ch = c * LPR + sub;
    if (ch >= nchG) continue;
    float out[4];
    float wv[4] = {1.f, 1.f, 1.f, 1.f};  // weighted MIS: w_is; DBM: C_is
    if constexpr (PROBLEM == 3) load16(a.w + i * a.ldw + ch * 4, wv);
    // DBM: dl/dx = -C + rowc + colc + b + d M from the step's line sums
    float dm[4], dr[4], dk[4], db[4], dd[4], dp[4];
    if constexpr (PROBLEM == 2) {
      const int64_t ld = a.dbm.ld;
      const int64_t r = i / a.dbm.N2;
      const int64_t k = i - r * a.dbm.N2;
      load16(a.dbm.C + i * ld + ch * 4, wv);
      load16(a.dbm.M + i * ld + ch * 4, dm);
      load16(a.dbm.rowc + r * ld + ch * 4, dr);
      load16(a.dbm.colc + k * ld + ch * 4, dk);
      load16(a.dbm.shot + ch * 4, db);
      load16(a.dbm.shot + ld + ch * 4, dd);
      load16(a.dbm.shot + 2 * ld + ch * 4, dp);
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int s = ch * 4 + e;
      const float pv = p[c][e], qv = q[c][e];
      float g;
      if constexpr (PROBLEM == 0 || PROBLEM == 3) {
        g = -wv[e] + lam[c][e] * qv;
      } else if constexpr (PROBLEM == 2) {
        g = -wv[e] + dr[e] + dk[e] + db[e] + dd[e] * dm[e];
      } else {
        g = 2.f * qv - deg;
      }
      const float t = 2.f * pv - 1.f;
      const float pq1 = pv * (1.f - pv);  // the sigmoid derivative P(1-P)
      // t^(alpha-1) = t (t^2)^((alpha-2)/2); the annealing term
      // 1 - t^alpha = (1 - t^2)(1 + t^2 + ... + t^(alpha-2)) with
      // 1 - t^2 = 4 P (1 - P): no cancellation as P approaches 0 or 1
      float tp = t, sm4 = 4.f;
      if (!alpha2) {
        const float t2 = t * t;
        float pw = 1.f, sm = 1.f;
        for (int r = 2; r < a.alpha; r += 2) {
          pw *= t2;
          sm += pw;
        }
        tp = t * pw;
        sm4 = 4.f * sm;
      }
      g += c_ann * tp;
      if (use_nu) {
        const float d = pv - mean;
        g += a.nu * ((a.div_kind == 0) ? -d * rstd : -2.f * (float)S * d);
      }
      if (scale_g) g *= pq1;
      if (s < S) {
        if constexpr (PROBLEM == 0 || PROBLEM == 3) {
          acc.pc[c][e] -= wv[e] * pv;
          acc.pp[c][e] += 0.5f * pv * qv;
        } else if constexpr (PROBLEM == 2) {
          acc.pc[c][e] -= wv[e] * pv;
          if (i == 0) acc.pp[c][e] += dp[e];  // the shot's whole penalty, once
        } else {
          acc.pc[c][e] += pv * qv - deg * pv;
        }
        acc.pa[c][e] = fmaf(sm4, pq1, acc.pa[c][e]);
        acc.pg[c][e] += g;
      } else {
        g = 0.f;
      }
      out[e] = g;
    }
    storeN<4>(static_cast<TG*>(a.G) + i * a.ldg + ch * 4, out);
  }
}

// Block-level reduction of the float partials per shot, in a fixed order,
// into this block's partial row.
template <int LPR, int CPL>
__device__ __forceinline__ void block_reduce(const LossArgs& a, ShotAcc<CPL>& acc, float* red) {
  const int S = a.S;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (LPR - 1);
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  __syncthreads();
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e)
#pragma unroll
      for (int off = LPR; off < 32; off <<= 1) {
        acc.pc[c][e] += __shfl_xor_sync(0xffffffffu, acc.pc[c][e], off);
        acc.pp[c][e] += __shfl_xor_sync(0xffffffffu, acc.pp[c][e], off);
        acc.pa[c][e] += __shfl_xor_sync(0xffffffffu, acc.pa[c][e], off);
        acc.pg[c][e] += __shfl_xor_sync(0xffffffffu, acc.pg[c][e], off);
      }
  const float psi = seg_sum<32>(acc.psi, 0xffffffffu);
  float* outp = a.partials + (int64_t)blockIdx.x * a.pstride;
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
            const float v = qd == 0 ? acc.pc[c][e]
                            : qd == 1 ? acc.pp[c][e]
                            : qd == 2 ? acc.pa[c][e]
                                      : acc.pg[c][e];
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

template <int LPR, int CPL, int PROBLEM>
__device__ __forceinline__ void load_lambda(const LossArgs& a, int sub, float (&lam)[CPL][4]) {
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int s = (c * LPR + sub) * 4 + e;
      lam[c][e] = ((PROBLEM == 0 || PROBLEM == 3) && s < a.S) ? a.lambda[s] : 0.f;
    }
}

// ------------------------------------------------------------------ kernels
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
  const int nchS = (a.S + 3) / 4;
  const float* __restrict__ P = a.P;
  extern __shared__ float red[];  // [nwarps][S]

  const float gamma = a.sc ? a.sc->gamma : a.gamma;
  float lam[CPL][4];
  if constexpr (DO_LOSS) load_lambda<LPR, CPL, PROBLEM>(a, sub, lam);
  ShotAcc<CPL> acc;
  acc.zero();

  for (int64_t i = first; i < a.N; i += stride) {
    float p[CPL][4];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int ch = c * LPR + sub;
      if (ch < nchS) {
        load16(P + i * a.ldp + ch * 4, p[c]);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) p[c][e] = 0.f;
      }
    }
    if (a.xbits) store_bits<LPR, CPL>(a, i, sub, smask, p);
    if constexpr (!DO_LOSS) continue;

    float q[CPL][4];
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) q[c][e] = 0.f;

    int beg = 0, end = 0;
    if constexpr (PROBLEM != 2) csr_row(a.rowptr, i, a.N, beg, end);  // DBM: no neighbour rows
    for (int eb = beg; eb < end; eb += LPR) {
      const int ee = eb + sub;
      const int jl = (ee < end) ? csr_col(a.col, ee, a.N) : 0;
      float wl = 1.f;  // edge weight A_ij (problem 4)
      if constexpr (PROBLEM == 4) wl = (ee < end) ? a.ew[ee] : 0.f;
      const int cnt = min(LPR, end - eb);
      int k = 0;
      for (; k + 4 <= cnt; k += 4) {
        uint4 raw[4][CPL];
        float wu[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j = __shfl_sync(smask, jl, k + u, LPR);
          wu[u] = 1.f;
          if constexpr (PROBLEM == 4) wu[u] = __shfl_sync(smask, wl, k + u, LPR);
          const float* row = P + (int64_t)j * a.ldp;
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            const int ch = c * LPR + sub;
            raw[u][c] = (ch < nchS) ? ldg_nc16(row + ch * 4) : make_uint4(0, 0, 0, 0);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int c = 0; c < CPL; ++c) {
            float f[4];
            widen(raw[u][c], f, (const float*)nullptr);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if constexpr (PROBLEM == 4) q[c][e] = fmaf(wu[u], f[e], q[c][e]);
              else q[c][e] += f[e];
            }
          }
      }
      for (; k < cnt; ++k) {
        const int j = __shfl_sync(smask, jl, k, LPR);
        float wk = 1.f;
        if constexpr (PROBLEM == 4) wk = __shfl_sync(smask, wl, k, LPR);
        const float* row = P + (int64_t)j * a.ldp;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const int ch = c * LPR + sub;
          if (ch < nchS) {
            float f[4];
            widen(ldg_nc16(row + ch * 4), f, (const float*)nullptr);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if constexpr (PROBLEM == 4) q[c][e] = fmaf(wk, f[e], q[c][e]);
              else q[c][e] += f[e];
            }
          }
        }
      }
    }
    float deg = (float)(end - beg);
    if constexpr (PROBLEM == 4) deg = a.wdeg[i];  // sum_j A_ij
    row_epilogue<LPR, CPL, PROBLEM, TG>(a, i, sub, smask, p, q, deg, lam, gamma, acc);
  }
  if constexpr (DO_LOSS) block_reduce<LPR, CPL>(a, acc, red);
}

// ---- staged variant: whole P rows bulk-copied into a per-warp ring ----
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void ring_init(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ bool ring_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ bool ring_wait(uint64_t* b, uint32_t parity) {
  for (uint32_t it = 0; it < kLossSpinLimit; ++it)
    if (ring_try(b, parity)) return true;
  return false;
}
__device__ __forceinline__ void ring_expect(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void ring_copy(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(b))
      : "memory");
}

// One warp per row.  Each warp owns RS row slots; a row slot holds the row's
// own P row and up to CAP neighbour rows, all copied with cp.async.bulk on a
// single mbarrier (one wait per row).  While row r is processed, the rows
// r + wstride .. r + (RS-1) wstride are in flight.  Neighbours beyond CAP
// (high-degree rows) are gathered directly from global memory.  The CSR
// index loads run ahead of the copies (row offsets two rows ahead, column
// indices one row ahead), so issuing a row's copies never waits on them.
constexpr int kRS = 2;
template <int CPL, int PROBLEM, typename TG>
__global__ void __launch_bounds__(256, 2)
loss_kernel_staged(LossArgs a, int CAP, int rslot_bytes, int bars_bytes) {
  constexpr int LPR = 32;
  constexpr int RS = kRS;
  const int lane = threadIdx.x & 31;
  const int sub = lane;
  const unsigned smask = 0xffffffffu;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int nchS = (a.S + 3) / 4;
  const uint32_t row_bytes = (uint32_t)nchS * 16u;

  extern __shared__ __align__(128) unsigned char dsm[];
  uint64_t* bars = reinterpret_cast<uint64_t*>(dsm) + warp * RS;
  unsigned char* slot_area = dsm + bars_bytes;
  unsigned char* slots = slot_area + (size_t)warp * RS * rslot_bytes;
  if (lane == 0) {
    for (int k = 0; k < RS; ++k) ring_init(bars + k);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();

  const float gamma = a.sc ? a.sc->gamma : a.gamma;
  float lam[CPL][4];
  load_lambda<LPR, CPL, PROBLEM>(a, sub, lam);
  ShotAcc<CPL> acc;
  acc.zero();

  const int64_t wstride = (int64_t)gridDim.x * nwarps;
  const int64_t first = (int64_t)blockIdx.x * nwarps + warp;
  const float* __restrict__ P = a.P;

  // Lane 0 issues the copies of row r (CSR range beg..end, the first
  // neighbour indices in jl across the lanes) into row slot k.
  auto issue_row = [&](int64_t r, int beg, int end, int jl, int k) {
    if (r >= a.N) return;
    const int n = min(end - beg, CAP);
    unsigned char* base = slots + (size_t)k * rslot_bytes;
    if (lane == 0) {
      ring_expect(bars + k, (uint32_t)(1 + n) * row_bytes);
      ring_copy(base, P + r * a.ldp, row_bytes, bars + k);
    }
    for (int t = 0; t < n; ++t) {
      const int j = __shfl_sync(smask, jl, t);
      if (lane == 0) ring_copy(base + (size_t)(1 + t) * row_bytes, P + (int64_t)j * a.ldp, row_bytes, bars + k);
    }
  };
  auto load_cols = [&](int beg, int end) -> int {
    return (lane < min(end - beg, CAP)) ? csr_col(a.col, beg + lane, a.N) : 0;
  };
  auto read_row = [&](const unsigned char* src, float (&f)[CPL][4]) {
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int ch = c * LPR + sub;
      if (ch < nchS) {
        const float4 v = *reinterpret_cast<const float4*>(src + ch * 16);
        f[c][0] = v.x; f[c][1] = v.y; f[c][2] = v.z; f[c][3] = v.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) f[c][e] = 0.f;
      }
    }
  };

  // CSR ranges of the rows in the two slots
  int sbeg0 = 0, send0 = 0, sbeg1 = 0, send1 = 0;
  {
    const int64_t r0 = first, r1 = first + wstride;
    if (r0 < a.N) csr_row(a.rowptr, r0, a.N, sbeg0, send0);
    if (r1 < a.N) csr_row(a.rowptr, r1, a.N, sbeg1, send1);
    const int j0 = load_cols(sbeg0, send0), j1 = load_cols(sbeg1, send1);
    issue_row(r0, sbeg0, send0, j0, 0);
    issue_row(r1, sbeg1, send1, j1, 1);
  }
  // index pipeline: row `nxt` (next to issue) has its range and column
  // indices loaded; row nxt + wstride has its range loaded
  int64_t nxt = first + RS * wstride;
  int nbeg = 0, nend = 0, njl = 0, pbeg = 0, pend = 0;
  if (nxt < a.N) csr_row(a.rowptr, nxt, a.N, nbeg, nend);
  njl = load_cols(nbeg, nend);
  if (nxt + wstride < a.N) csr_row(a.rowptr, nxt + wstride, a.N, pbeg, pend);

  int k = 0;
  uint32_t par = 0;
  bool dead = false;
  for (int64_t i = first; i < a.N; i += wstride) {
    const int beg = k ? sbeg1 : sbeg0;
    const int end = k ? send1 : send0;
    const int n = min(end - beg, CAP);
    float wl = 1.f;  // weight of slot neighbour `lane` (problem 4), loaded before the wait
    if constexpr (PROBLEM == 4) wl = (lane < n) ? a.ew[beg + lane] : 0.f;
    if (!ring_wait(bars + k, par)) {
      dead = true;
      break;
    }
    const unsigned char* base = slots + (size_t)k * rslot_bytes;
    float p[CPL][4];
    read_row(base, p);
    float q[CPL][4];
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
      for (int e = 0; e < 4; ++e) q[c][e] = 0.f;
    for (int t = 0; t < n; ++t) {
      float f[CPL][4];
      read_row(base + (size_t)(1 + t) * row_bytes, f);
      if constexpr (PROBLEM == 4) {
        const float wt = __shfl_sync(smask, wl, t);
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
          for (int e = 0; e < 4; ++e) q[c][e] = fmaf(wt, f[c][e], q[c][e]);
      } else {
#pragma unroll
        for (int c = 0; c < CPL; ++c)
#pragma unroll
          for (int e = 0; e < 4; ++e) q[c][e] += f[c][e];
      }
    }
    __syncwarp();
    issue_row(nxt, nbeg, nend, njl, k);  // refill the slot just read
    if (k) { sbeg1 = nbeg; send1 = nend; } else { sbeg0 = nbeg; send0 = nend; }
    // advance the index pipeline; these loads complete behind this row's
    // epilogue
    nxt += wstride;
    nbeg = pbeg;
    nend = pend;
    njl = (nxt < a.N) ? load_cols(nbeg, nend) : 0;
    pbeg = pend = 0;
    if (nxt + wstride < a.N) csr_row(a.rowptr, nxt + wstride, a.N, pbeg, pend);
    if (++k == RS) {
      k = 0;
      par ^= 1u;
    }
    for (int e = beg + n; e < end; ++e) {  // neighbours beyond the slot capacity
      const float* row = P + (int64_t)csr_col(a.col, e, a.N) * a.ldp;
      float we = 1.f;
      if constexpr (PROBLEM == 4) we = a.ew[e];
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int ch = c * LPR + sub;
        if (ch < nchS) {
          float f[4];
          widen(ldg_nc16(row + ch * 4), f, (const float*)nullptr);
#pragma unroll
          for (int e2 = 0; e2 < 4; ++e2) {
            if constexpr (PROBLEM == 4) q[c][e2] = fmaf(we, f[e2], q[c][e2]);
            else q[c][e2] += f[e2];
          }
        }
      }
    }
    if (a.xbits) store_bits<LPR, CPL>(a, i, sub, smask, p);
    float deg = (float)(end - beg);
    if constexpr (PROBLEM == 4) deg = a.wdeg[i];  // sum_j A_ij
    row_epilogue<LPR, CPL, PROBLEM, TG>(a, i, sub, smask, p, q, deg, lam, gamma, acc);
  }
  if (dead) {
    if (lane == 0 && a.err_flag) atomicOr(a.err_flag, 2);
    // let this warp's own copies land before the block's shared memory is reused
    for (int t = 0; t < RS; ++t) {
      for (uint32_t it = 0; it < kLossSpinLimit && !ring_try(bars + k, par); ++it) {
      }
      if (++k == RS) {
        k = 0;
        par ^= 1u;
      }
    }
  }
  // After every warp is done with its slots, the slot area holds the block's
  // reduction scratch (block_reduce starts with a block-wide barrier).
  block_reduce<LPR, CPL>(a, acc, reinterpret_cast<float*>(slot_area));
}

template <int LPR, int CPL, int PROBLEM, typename TG, bool DO_LOSS>
int launch_loss_t(const LossArgs& a, int max_grid, cudaStream_t st) {
  constexpr int threads = 256;
  const int segs_per_block = (threads / 32) * (32 / LPR);
  int64_t want = (a.N + segs_per_block - 1) / segs_per_block;
  int grid = (int)(want < max_grid ? want : max_grid);
  if (grid < 1) grid = 1;
  const size_t smem = DO_LOSS ? (size_t)(threads / 32) * (a.S > 0 ? a.S : 1) * sizeof(float) : 0;
  loss_kernel<LPR, CPL, PROBLEM, TG, DO_LOSS><<<grid, threads, smem, st>>>(a);
  return grid;
}

constexpr int kStagedBudget = 104 * 1024;  // dynamic shared memory per block (2 blocks / SM)

template <int CPL, int PROBLEM, typename TG>
int launch_staged_t(const LossArgs& a, int max_grid, cudaStream_t st) {
  constexpr int threads = 256;
  constexpr int nwarps = threads / 32;
  constexpr int RS = kRS;
  const int row_bytes = (a.S + 3) / 4 * 16;
  const int bars_bytes = 128;  // nwarps * RS barriers
  int CAP = ((kStagedBudget - bars_bytes) / nwarps / RS) / row_bytes - 1;
  if (CAP > 32) CAP = 32;
  if (CAP < 1) return -1;
  const int rslot_bytes = (1 + CAP) * row_bytes;
  const size_t slot_area = (size_t)nwarps * RS * rslot_bytes;
  // reduction scratch aliased onto the slot area at the end
  const size_t scratch = (size_t)nwarps * a.S * 4;
  if (scratch > slot_area) return -1;
  const size_t smem = bars_bytes + slot_area;
  static bool attr_set = false;
  if (!attr_set) {
    if (cudaFuncSetAttribute(loss_kernel_staged<CPL, PROBLEM, TG>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kStagedBudget) != cudaSuccess) {
      cudaGetLastError();
      return -1;
    }
    attr_set = true;
  }
  int64_t want = (a.N + nwarps - 1) / nwarps;
  int grid = (int)(want < max_grid ? want : max_grid);
  if (grid < 1) grid = 1;
  loss_kernel_staged<CPL, PROBLEM, TG><<<grid, threads, smem, st>>>(a, CAP, rslot_bytes, bars_bytes);
  return grid;
}

template <int PROBLEM, typename TG, bool DO_LOSS>
int dispatch_loss(const LossArgs& a, int nch, int max_grid, int staged_grid, cudaStream_t st) {
  if (nch <= 2) return launch_loss_t<2, 1, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  if (nch <= 4) return launch_loss_t<4, 1, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  if (nch <= 8) return launch_loss_t<8, 1, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  if (nch <= 16) return launch_loss_t<16, 1, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  if constexpr (DO_LOSS && PROBLEM != 2) {
    int g = -1;
    if (nch <= 32) g = launch_staged_t<1, PROBLEM, TG>(a, staged_grid, st);
    else if (nch <= 64) g = launch_staged_t<2, PROBLEM, TG>(a, staged_grid, st);
    else if (nch <= 128) g = launch_staged_t<4, PROBLEM, TG>(a, staged_grid, st);
    else g = launch_staged_t<8, PROBLEM, TG>(a, staged_grid, st);
    if (g > 0) return g;
  }
  if (nch <= 32) return launch_loss_t<32, 1, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  if (nch <= 64) return launch_loss_t<32, 2, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  if (nch <= 128) return launch_loss_t<32, 4, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
  return launch_loss_t<32, 8, PROBLEM, TG, DO_LOSS>(a, max_grid, st);
}

}  // namespace

}  // namespace cpra
