// Row-gather SpMM for the GCN aggregate step (Eq. GCN, App. B.1) and its
// adjoint.  One power-of-two segment of LPR lanes owns one node row; each lane
// moves 16-byte vectors, CPL of them per row.  Neighbour rows are gathered
// four at a time so that every lane keeps 4*CPL independent 16-byte loads in
// flight.  Everything but the gathered operand is touched once, so those
// reads and the output rows carry an L2 evict-first hint: the gathered rows
// then stay in L2 longer and fewer of the repeated gathers reach HBM.
//
// The operand set of a launch is a template parameter (KIND), so the forward
// aggregation carries no add/mask/column-sum code and fits in fewer
// registers; the grid is the number of blocks that are resident at once.
#include <atomic>

#include "common.cuh"
#include "kernels.cuh"

namespace cpra {

namespace {

enum SpmmKind {
  KIND_MEAN = 0,             // Y = D^-1 A X                     (forward aggregation)
  KIND_ADD_MASK_COLSUM = 1,  // Y = (add + A X) * 1[mask > 0], column sums of Y
  KIND_ADD = 2,              // Y = add + A X
  KIND_ADD_ADAM = 3,         // g = add + A X; Adam step on the embedding row with g
  KIND_ADD_MASKBITS_COLSUM = 4,  // as KIND_ADD_MASK_COLSUM with the mask given as bits
};

// LMODE: 0 CSR gathers, 1 line sums, 2 either, chosen at run time
template <typename TX, typename TY, int LPR, int CPL, int KIND, int LMODE>
__global__ void __launch_bounds__(256, CPL > 1 ? 1
                            : KIND == KIND_MEAN ? (LMODE == 1 ? 6 : 5)
                            : KIND == KIND_ADD  ? 5
                                                : 4)
spmm_rows_kernel(SpmmArgs a) {
  if (a.nsl > 1) {  // column slice blockIdx.y of nsl: shift every operand
    const int chunks = a.h_full / 16, k = blockIdx.y;
    const int c0 = 16 * (chunks * k / a.nsl), c1 = 16 * (chunks * (k + 1) / a.nsl);
    const int ex = a.dx == DT_BF16 ? 2 : 4, ey = a.dy == DT_BF16 ? 2 : 4;
    a.H = c1 - c0;
    a.X = static_cast<const char*>(a.X) + (int64_t)c0 * ex;
    if (a.Y) a.Y = static_cast<char*>(a.Y) + (int64_t)c0 * ey;
    if (a.add) a.add = static_cast<const char*>(a.add) + (int64_t)c0 * ex;
    if (a.mask) a.mask = static_cast<const char*>(a.mask) + (int64_t)c0 * ex;
    if (a.mask_bits) a.mask_bits += c0 / 16;
    if (a.colsum_partials) a.colsum_partials += c0;
    if (a.line_r) {
      a.line_r += c0;
      a.line_k += c0;
    }
    if (a.emb) {
      a.emb += c0;
      a.emb_m += c0;
      a.emb_v += c0;
      a.shadow = static_cast<char*>(a.shadow) + (int64_t)c0 * ex;
    }
  }
  constexpr bool MEAN = KIND == KIND_MEAN;
  constexpr bool HAS_ADD = KIND != KIND_MEAN;
  constexpr bool HAS_MASK = KIND == KIND_ADD_MASK_COLSUM;
  constexpr bool MASK_BITS = KIND == KIND_ADD_MASKBITS_COLSUM;
  constexpr bool COLSUM = KIND == KIND_ADD_MASK_COLSUM || KIND == KIND_ADD_MASKBITS_COLSUM;
  constexpr bool ADAM = KIND == KIND_ADD_ADAM;
  // Neighbour rows per gather pass.  With one 16-byte chunk per lane (CPL =
  // 1) the mean aggregation, the masked adjoint (mask as bits) and the
  // embedding-gradient aggregation issue one predicated batch of PB rows, so
  // a row of degree <= PB costs one memory round trip (degree 5, H = 128,
  // N = 10^6: mean 0.261 -> 0.253 ms at five blocks per SM instead of six,
  // masked adjoint 0.354 -> 0.329 ms, embedding gradient with Adam 0.780 ->
  // 0.776 ms).  The other kinds, and wide rows (CPL > 1, already CPL loads
  // per neighbour and lane), gather full batches of four and then the
  // remainder one row at a time.  The line-sum instance gathers nothing.
  constexpr int PB = (CPL == 1 && LMODE != 1 &&
                      (KIND == KIND_MEAN || KIND == KIND_ADD_MASKBITS_COLSUM ||
                       KIND == KIND_ADD_ADAM))
                         ? 5
                         : 0;
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
  TY* Y = static_cast<TY*>(a.Y);
  const TX* ADD = static_cast<const TX*>(a.add);  // may alias Y (same row, read first)
  const TX* __restrict__ MASK = static_cast<const TX*>(a.mask);
  const uint64_t pol = l2_evict_first_policy();
  bool update = true;  // embedding Adam step (ADAM kind), off once early stopping fired
  float bc1 = a.bc1, bc2 = a.bc2;
  if constexpr (ADAM) {
    update = !(a.halt && *a.halt);
    if (a.sc) {
      bc1 = a.sc->bc1;
      bc2 = a.sc->bc2;
    }
  }

  float csum[CPL][VEC];
#pragma unroll
  for (int c = 0; c < CPL; ++c)
#pragma unroll
    for (int v = 0; v < VEC; ++v) csum[c][v] = 0.f;

  // CSR index pipeline: the current row's range and first LPR column
  // indices, and the next row's range, are loaded one iteration ahead, so the
  // gathers never wait on an index load.
  // Matching constraint graph (line sums given): no CSR traffic at all.
  const bool lines = LMODE == 2 ? a.line_r != nullptr : LMODE == 1;
  int beg = 0, end = 0, jl = 0, pbeg = 0, pend = 0;
  if (!lines && first < a.N) {
    csr_row(a.rowptr, first, a.N, beg, end);
    jl = (sub < end - beg) ? csr_col(a.col, beg + sub, a.N) : 0;
  }
  if (!lines && first + stride < a.N) csr_row(a.rowptr, first + stride, a.N, pbeg, pend);
  for (int64_t i = first; i < a.N; i += stride) {
    const int njl =
        (!lines && i + stride < a.N && sub < pend - pbeg) ? csr_col(a.col, pbeg + sub, a.N) : 0;
    int ppbeg = 0, ppend = 0;
    if (!lines && i + 2 * stride < a.N) csr_row(a.rowptr, i + 2 * stride, a.N, ppbeg, ppend);
    // the row's own operands first, so that they arrive with the gathers
    uint4 rad[CPL], rmk[CPL];
    uint32_t mbits[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int ch = c * LPR + sub;
      rad[c] = rmk[c] = make_uint4(0, 0, 0, 0);
      mbits[c] = 0u;
      if (ch < nchunks) {
        if constexpr (HAS_ADD) rad[c] = ld_stream16(ADD + i * a.ldadd + ch * VEC, pol);
        if constexpr (HAS_MASK) rmk[c] = ld_stream16(MASK + i * a.ldm + ch * VEC, pol);
        if constexpr (MASK_BITS)
          mbits[c] = (uint32_t)a.mask_bits[i * a.ldmb + (ch * VEC) / 16] >> ((ch * VEC) % 16);
      }
    }
    float acc[CPL][VEC];
#pragma unroll
    for (int c = 0; c < CPL; ++c)
#pragma unroll
      for (int v = 0; v < VEC; ++v) acc[c][v] = 0.f;

    if (lines) {
      // the neighbours of pair (r, k) are the other pairs of row line r and
      // of column line k: their sum is R_r + K_k - 2 x_(r,k)
      const int64_t r = i / a.line_n2;
      const int64_t k = i - r * a.line_n2;
      const float* __restrict__ LR = a.line_r + r * a.ldl;
      const float* __restrict__ LK = a.line_k + k * a.ldl;
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const int ch = c * LPR + sub;
        if (ch < nchunks) {
          float f[VEC];
          widen(ldg_nc16(X + i * a.ldx + ch * VEC), f, (const TX*)nullptr);
#pragma unroll
          for (int q = 0; q < VEC; q += 4) {
            float lr[4], lk[4];
            load16(LR + ch * VEC + q, lr);
            load16(LK + ch * VEC + q, lk);
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[c][q + v] = (lr[v] - f[q + v]) + (lk[v] - f[q + v]);
          }
        }
      }
    }
    for (int eb = beg; eb < end; eb += LPR) {
      const int e = eb + sub;
      const int jc = (eb == beg) ? jl : ((e < end) ? csr_col(a.col, e, a.N) : 0);
      const int cnt = min(LPR, end - eb);
      int k = 0;
      if constexpr (PB > 0) {
        for (; k < cnt; k += PB) {
          uint4 raw[PB > 0 ? PB : 1][CPL];
#pragma unroll
          for (int u = 0; u < PB; ++u) {
            const int j = __shfl_sync(smask, jc, (k + u) & (LPR - 1), LPR);
            const TX* row = X + (int64_t)j * a.ldx;
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
              const int ch = c * LPR + sub;
              raw[u][c] = (k + u < cnt && ch < nchunks) ? ldg_nc16(row + ch * VEC)
                                                        : make_uint4(0, 0, 0, 0);
            }
          }
#pragma unroll
          for (int u = 0; u < PB; ++u)
            if (k + u < cnt)
#pragma unroll
              for (int c = 0; c < CPL; ++c) {
                float f[VEC];
                widen(raw[u][c], f, (const TX*)nullptr);
#pragma unroll
                for (int v = 0; v < VEC; ++v) acc[c][v] += f[v];
              }
        }
      } else {
        for (; k + 4 <= cnt; k += 4) {
          uint4 raw[4][CPL];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = __shfl_sync(smask, jc, k + u, LPR);
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
          const int j = __shfl_sync(smask, jc, k, LPR);
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
    }

    float s = 1.f;
    if constexpr (MEAN) s = a.inv_deg[i];
#pragma unroll
    for (int c = 0; c < CPL; ++c) {
      const int ch = c * LPR + sub;
      if (ch >= nchunks) continue;
      float o[VEC];
#pragma unroll
      for (int v = 0; v < VEC; ++v) o[v] = acc[c][v];
      if constexpr (HAS_ADD) {
        float ad[VEC];
        widen(rad[c], ad, (const TX*)nullptr);
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[v] += ad[v];
      }
      if constexpr (MEAN) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[v] *= s;
      }
      if constexpr (HAS_MASK) {
        float mk[VEC];
        widen(rmk[c], mk, (const TX*)nullptr);
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[v] = (mk[v] > 0.f) ? o[v] : 0.f;
      }
      if constexpr (MASK_BITS) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) o[v] = ((mbits[c] >> v) & 1u) ? o[v] : 0.f;
      }
      if constexpr (COLSUM) {
#pragma unroll
        for (int v = 0; v < VEC; ++v) csum[c][v] += o[v];
      }
      if constexpr (ADAM) {
        // o is dR/dh^0 for this chunk: one Adam step on the FP32 master row,
        // its moments, and the activation-dtype copy the forward reads (the
        // copy is rewritten even when early stopping froze the update)
        const int64_t off = i * a.lde + ch * VEC;
        float th[VEC], m[VEC], vv[VEC];
#pragma unroll
        for (int q = 0; q < VEC; q += 4) {
          widen(ld_stream16(a.emb + off + q, pol), th + q, (const float*)nullptr);
          widen(ld_stream16(a.emb_m + off + q, pol), m + q, (const float*)nullptr);
          widen(ld_stream16(a.emb_v + off + q, pol), vv + q, (const float*)nullptr);
        }
        if (Y) storeN_stream<VEC>(Y + i * a.ldy + ch * VEC, o, pol);
        if (update) {
#pragma unroll
          for (int v = 0; v < VEC; ++v)
            th[v] = adam_update(th[v], m[v], vv[v], o[v], a.lr, a.beta1, a.beta2, a.eps, a.wd,
                                bc1, bc2);
          storeN_stream<VEC>(a.emb + off, th, pol);
          storeN_stream<VEC>(a.emb_m + off, m, pol);
          storeN_stream<VEC>(a.emb_v + off, vv, pol);
        }
        storeN_stream<VEC>(static_cast<TX*>(a.shadow) + i * a.lds + ch * VEC, th, pol);
      } else {
        storeN_stream<VEC>(Y + i * a.ldy + ch * VEC, o, pol);
      }
    }
    beg = pbeg;
    end = pend;
    jl = njl;
    pbeg = ppbeg;
    pend = ppend;
  }

  if constexpr (COLSUM) {
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
      a.colsum_partials[(int64_t)blockIdx.x * a.ldcs + col] = t;
    }
  }
}

// Resident blocks per SM for one kernel and dynamic shared size; `cache`
// (one per kernel instantiation) keeps the last answer as (smem << 8) | blocks.
template <typename K>
int resident_blocks(K kernel, int threads, size_t smem, std::atomic<long long>& cache) {
  const long long c = cache.load(std::memory_order_relaxed);
  if (c >= 0 && (size_t)(c >> 8) == smem) return (int)(c & 0xff);
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, threads, smem) != cudaSuccess ||
      blocks < 1) {
    cudaGetLastError();
    blocks = 1;
  }
  if (blocks > 255) blocks = 255;
  cache.store(((long long)smem << 8) | blocks, std::memory_order_relaxed);
  return blocks;
}

template <typename TX, typename TY, int LPR, int CPL, int KIND, int LMODE>
int launch_lines(const SpmmArgs& a, int num_sms, int max_grid, cudaStream_t st) {
  constexpr int threads = 256;
  const int segs_per_block = (threads / 32) * (32 / LPR);
  const size_t smem = (KIND == KIND_ADD_MASK_COLSUM || KIND == KIND_ADD_MASKBITS_COLSUM)
                           ? (size_t)(threads / 32) * a.H * sizeof(float)
                           : 0;
  auto kernel = spmm_rows_kernel<TX, TY, LPR, CPL, KIND, LMODE>;
  static std::atomic<long long> occ_cache{-1};
  const int64_t resident = (int64_t)resident_blocks(kernel, threads, smem, occ_cache) * num_sms;
  int64_t grid = (a.N + segs_per_block - 1) / segs_per_block;
  if (grid > resident) grid = resident;
  if (grid > max_grid) grid = max_grid;
  if (grid < 1) grid = 1;
  kernel<<<dim3((unsigned)grid, (unsigned)a.nsl), threads, smem, st>>>(a);
  return (int)grid;
}

// The aggregations (mean; add + mask) run the matching constraint graph's
// line-sum path as its own instance, so the CSR path carries none of its code
// or registers (mean aggregation at N = 10^6, H = 128: 0.267 -> 0.259 ms).  The
// embedding-Adam kind keeps one instance with the choice made at run time:
// split the same way it ran slower (0.777 -> 0.811 ms), from its schedule
// alone, at the same residency.
template <typename TX, typename TY, int LPR, int CPL, int KIND>
int launch_t(const SpmmArgs& a, int num_sms, int max_grid, cudaStream_t st) {
  if constexpr (KIND == KIND_ADD_ADAM)
    return launch_lines<TX, TY, LPR, CPL, KIND, 2>(a, num_sms, max_grid, st);
  else
    return a.line_r ? launch_lines<TX, TY, LPR, CPL, KIND, 1>(a, num_sms, max_grid, st)
                    : launch_lines<TX, TY, LPR, CPL, KIND, 0>(a, num_sms, max_grid, st);
}

template <typename TX, typename TY, int KIND>
int dispatch_lpr(const SpmmArgs& a, int num_sms, int max_grid, cudaStream_t st) {
  const int nch = a.H / V16<TX>::n;
  if (nch <= 2) return launch_t<TX, TY, 2, 1, KIND>(a, num_sms, max_grid, st);
  if (nch <= 4) return launch_t<TX, TY, 4, 1, KIND>(a, num_sms, max_grid, st);
  if (nch <= 8) return launch_t<TX, TY, 8, 1, KIND>(a, num_sms, max_grid, st);
  if (nch <= 16) return launch_t<TX, TY, 16, 1, KIND>(a, num_sms, max_grid, st);
  if (nch <= 32) return launch_t<TX, TY, 32, 1, KIND>(a, num_sms, max_grid, st);
  if (nch <= 64) return launch_t<TX, TY, 32, 2, KIND>(a, num_sms, max_grid, st);
  if (nch <= 128) return launch_t<TX, TY, 32, 4, KIND>(a, num_sms, max_grid, st);
  return launch_t<TX, TY, 32, 8, KIND>(a, num_sms, max_grid, st);
}

}  // namespace

namespace {
int spmm_launch_one(const SpmmArgs& a, int num_sms, int max_grid, cudaStream_t st) {
  const bool add = a.add != nullptr, mask = a.mask != nullptr, cs = a.colsum_partials != nullptr;
  const bool same = a.dx == a.dy;
  if (a.adam && (a.mean || !add || mask || cs)) return -1;
  if (a.mean && !add && !mask && !cs && same) {
    return a.dx == DT_BF16 ? dispatch_lpr<bf16, bf16, KIND_MEAN>(a, num_sms, max_grid, st)
                           : dispatch_lpr<float, float, KIND_MEAN>(a, num_sms, max_grid, st);
  }
  if (!a.mean && add && !mask && a.mask_bits && cs && same) {
    return a.dx == DT_BF16
               ? dispatch_lpr<bf16, bf16, KIND_ADD_MASKBITS_COLSUM>(a, num_sms, max_grid, st)
               : dispatch_lpr<float, float, KIND_ADD_MASKBITS_COLSUM>(a, num_sms, max_grid, st);
  }
  if (a.mask_bits) return -1;
  if (!a.mean && add && mask && cs && same) {
    return a.dx == DT_BF16
               ? dispatch_lpr<bf16, bf16, KIND_ADD_MASK_COLSUM>(a, num_sms, max_grid, st)
               : dispatch_lpr<float, float, KIND_ADD_MASK_COLSUM>(a, num_sms, max_grid, st);
  }
  if (!a.mean && add && !mask && !cs && a.dy == DT_F32 && a.adam) {
    if (!a.emb || !a.emb_m || !a.emb_v || !a.shadow) return -1;
    return a.dx == DT_BF16 ? dispatch_lpr<bf16, float, KIND_ADD_ADAM>(a, num_sms, max_grid, st)
                           : dispatch_lpr<float, float, KIND_ADD_ADAM>(a, num_sms, max_grid, st);
  }
  if (!a.mean && add && !mask && !cs && a.dy == DT_F32) {
    return a.dx == DT_BF16 ? dispatch_lpr<bf16, float, KIND_ADD>(a, num_sms, max_grid, st)
                           : dispatch_lpr<float, float, KIND_ADD>(a, num_sms, max_grid, st);
  }
  return -1;  // operand set not used by the training step
}
}  // namespace

// Rows wider than spmm_slice_width columns run as column slices, blockIdx.y
// = slice, in one launch (every operand set is column-separable: the
// aggregation, the mask, the column sums and the embedding update act column
// by column; the column-sum partial rows of all slices share one grid).
int spmm_launch(const SpmmArgs& a0, int num_sms, int max_grid, cudaStream_t st) {
  SpmmArgs a = a0;
  if (a.lde == 0) a.lde = a.H;
  if (a.ldcs == 0) a.ldcs = a.H;
  const int nsl = spmm_slices(a);
  if (nsl > 1 && a.H % 16) return -1;
  a.nsl = nsl;
  a.h_full = a.H;
  // the widest slice decides the lane layout and the shared memory
  if (nsl > 1) a.H = 16 * ((a.H / 16 + nsl - 1) / nsl);
  return spmm_launch_one(a, num_sms, max_grid, st);
}

#ifdef CPRA_CHECKED
void csr_check_collect_spmm(CsrCheck* r) { CPRA_CSR_CHECK_COLLECT(r); }
#endif

}  // namespace cpra
