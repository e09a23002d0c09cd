// Exact integer evaluation of the rounded shots from their packed bits
// (App. C.2 rounding, Table objective-functions, Prop. 3.2).
//
// x_bits holds, per node, W = ceil(S/32) words; bit (s mod 32) of word s/32
// is x_is.  A segment of G >= W lanes owns one node row, lane w its word w.
// For every edge (i, j) with j > i the lane combines x_i[w] and x_j[w]
// (AND for MIS violations, XOR for MaxCut cut edges) and adds the 32 bits to
// bit-sliced vertical counters (eight bit planes, one ripple-carry add per
// edge); the planes are flushed to per-shot shared-memory counters before
// they can overflow, in practice once per thread.  MIS set sizes add x_i[w] the same way; the pairwise
// Hamming sum adds k_i (S - k_i) with k_i = popcount of row i.  All sums are
// integers, so the result does not depend on the order of the atomics.
#include "common.cuh"
#include "kernels.cuh"

namespace cpra {

namespace {

// 32 counters of 8 bits each, stored as 8 bit planes (plane k holds bit k
// of every counter); flushed before the 256th addition.
struct Planes {
  uint32_t p[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  int n = 0;  // additions since the last flush (< 256)
  __device__ __forceinline__ void add(uint32_t x) {
#pragma unroll
    for (int k = 0; k < 7; ++k) {
      const uint32_t t = p[k] & x;
      p[k] ^= x;
      x = t;
    }
    p[7] ^= x;
    ++n;
  }
  // Adds the per-bit counts to cnt[0..31] and clears the planes.
  __device__ __forceinline__ void flush(int* cnt) {
    uint32_t any = 0u;
#pragma unroll
    for (int k = 0; k < 8; ++k) any |= p[k];
    if (any) {
#pragma unroll 4
      for (int b = 0; b < 32; ++b) {
        int c = 0;
#pragma unroll
        for (int k = 0; k < 8; ++k) c |= (int)((p[k] >> b) & 1u) << k;
        if (c) atomicAdd(cnt + b, c);
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) p[k] = 0u;
    n = 0;
  }
};
constexpr int kFlushAt = 255;

template <int G, int PROBLEM>
__global__ void __launch_bounds__(256)
eval_bits_kernel(int64_t N, int S, int W, const int* __restrict__ rowptr,
                 const int* __restrict__ col, const uint32_t* __restrict__ bits,
                 unsigned long long* counters) {
  __shared__ int scnt[2 * 1024];  // objective per shot, then violations per shot
  __shared__ unsigned long long ham_s;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (G - 1);
  const unsigned smask = segment_mask<G>(lane);
  const int segs_per_warp = 32 / G;
  const int64_t segs_per_block = (int64_t)(blockDim.x >> 5) * segs_per_warp;
  const int64_t first = (int64_t)blockIdx.x * segs_per_block +
                        (threadIdx.x >> 5) * segs_per_warp + lane / G;
  const int64_t stride = (int64_t)gridDim.x * segs_per_block;
  const int Wpad = W * 32;
  for (int k = threadIdx.x; k < 2 * Wpad; k += blockDim.x) scnt[k] = 0;
  if (threadIdx.x == 0) ham_s = 0ull;
  __syncthreads();

  const bool active = sub < W;
  int* cnt_obj = scnt + 32 * sub;
  int* cnt_viol = scnt + Wpad + 32 * sub;
  Planes obj, viol;
  long long ham = 0;
  constexpr int U = 8;  // neighbour words loaded together
  // CSR index pipeline: the current row's range and first U column indices,
  // and the next row's range, are loaded one iteration ahead
  int beg = 0, end = 0, jfirst = -1, pbeg = 0, pend = 0;
  if (first < N) {
    beg = rowptr[first];
    end = rowptr[first + 1];
    jfirst = ((sub % U) < end - beg) ? col[beg + (sub % U)] : -1;
  }
  if (first + stride < N) {
    pbeg = rowptr[first + stride];
    pend = rowptr[first + stride + 1];
  }
  for (int64_t i = first; i < N; i += stride) {
    const int njfirst =
        (i + stride < N && (sub % U) < pend - pbeg) ? col[pbeg + (sub % U)] : -1;
    int ppbeg = 0, ppend = 0;
    if (i + 2 * stride < N) {
      ppbeg = rowptr[i + 2 * stride];
      ppend = rowptr[i + 2 * stride + 1];
    }
    const uint32_t xi = active ? bits[i * W + sub] : 0u;
    if constexpr (PROBLEM == 2) end = beg;  // set sizes and the Hamming sum only
    for (int eb = beg; eb < end; eb += U) {
      // lanes of the segment hold up to U neighbour indices, then every lane
      // loads its word of each neighbour j > i (each edge once, at its lower
      // endpoint); all loads are in flight before any counter is updated
      const int e = eb + (sub % U);
      const int jl = (eb == beg) ? jfirst : ((e < end) ? col[e] : -1);
      const int cnt = min(U, end - eb);
      uint32_t xs[U];
      bool use[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int j = __shfl_sync(smask, jl, u % G, G);
        use[u] = (u < cnt) && (u < G) && (j > i);
        xs[u] = (use[u] && active) ? bits[(int64_t)j * W + sub] : 0u;
      }
      if (G < U) {  // segments narrower than U lanes: the rest one index at a time
        for (int u = G; u < cnt; ++u) {
          const int j = col[eb + u];
          if (j > i) {
            const uint32_t xj = active ? bits[(int64_t)j * W + sub] : 0u;
            if (PROBLEM == 0) {
              viol.add(xi & xj);
              if (viol.n == kFlushAt) viol.flush(cnt_viol);
            } else {
              obj.add(xi ^ xj);
              if (obj.n == kFlushAt) obj.flush(cnt_obj);
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (!use[u]) continue;
        if (PROBLEM == 0) {
          viol.add(xi & xs[u]);
          if (viol.n == kFlushAt) viol.flush(cnt_viol);
        } else {
          obj.add(xi ^ xs[u]);
          if (obj.n == kFlushAt) obj.flush(cnt_obj);
        }
      }
    }
    int k = __popc(xi);
#pragma unroll
    for (int off = G / 2; off > 0; off >>= 1) k += __shfl_xor_sync(smask, k, off);
    if (sub == 0) ham += (long long)k * (long long)(S - k);
    if (PROBLEM != 1) {
      obj.add(xi);
      if (obj.n == kFlushAt) obj.flush(cnt_obj);
    }
    beg = pbeg;
    end = pend;
    jfirst = njfirst;
    pbeg = ppbeg;
    pend = ppend;
  }
  if (active) {
    obj.flush(cnt_obj);
    viol.flush(cnt_viol);
  }
  if (ham) atomicAdd(&ham_s, (unsigned long long)ham);
  __syncthreads();
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    if (scnt[s]) atomicAdd(&counters[s], (unsigned long long)scnt[s]);
    if (scnt[Wpad + s]) atomicAdd(&counters[S + s], (unsigned long long)scnt[Wpad + s]);
  }
  if (threadIdx.x == 0 && ham_s) atomicAdd(&counters[2 * S], ham_s);
}

template <int G>
void launch_g(int64_t N, int S, int W, const int* rowptr, const int* col, const uint32_t* bits,
              int problem, unsigned long long* counters, int max_grid, cudaStream_t st) {
  constexpr int threads = 256;
  const int segs_per_block = (threads / 32) * (32 / G);
  int64_t want = (N + segs_per_block - 1) / segs_per_block;
  int grid = (int)(want < max_grid ? want : max_grid);
  if (grid < 1) grid = 1;
  if (problem == 0)
    eval_bits_kernel<G, 0><<<grid, threads, 0, st>>>(N, S, W, rowptr, col, bits, counters);
  else if (problem == 1)
    eval_bits_kernel<G, 1><<<grid, threads, 0, st>>>(N, S, W, rowptr, col, bits, counters);
  else
    eval_bits_kernel<G, 2><<<grid, threads, 0, st>>>(N, S, W, rowptr, col, bits, counters);
}

// Weighted MIS value per shot: block b sums w_is over its row range for the
// shots set in the rounding bits, in row order; then the blocks in order.
__global__ void weighted_value_kernel(int64_t N, int S, int W, const uint32_t* __restrict__ bits,
                                      const float* __restrict__ w, int64_t ldw, int64_t rows_per,
                                      double* __restrict__ part) {
  const int64_t r0 = (int64_t)blockIdx.x * rows_per;
  const int64_t r1 = r0 + rows_per < N ? r0 + rows_per : N;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    double t = 0.0;
    for (int64_t r = r0; r < r1; ++r)
      if ((bits[r * W + (s >> 5)] >> (s & 31)) & 1u) t += (double)w[r * ldw + s];
    part[(int64_t)blockIdx.x * S + s] = t;
  }
}

__global__ void weighted_value_finalize(int blocks, int S, const double* __restrict__ part,
                                        double* __restrict__ value) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  double t = 0.0;
  for (int b = 0; b < blocks; ++b) t += part[(int64_t)b * S + s];
  value[s] = t;
}

}  // namespace

void weighted_value_launch(int64_t N, int S, const uint32_t* bits, const float* w, int64_t ldw,
                           double* part, int max_blocks, double* value, cudaStream_t st) {
  int64_t rows_per = (N + max_blocks - 1) / max_blocks;
  if (rows_per < 1) rows_per = 1;
  const int blocks = (int)((N + rows_per - 1) / rows_per);
  weighted_value_kernel<<<blocks, 128, 0, st>>>(N, S, (S + 31) / 32, bits, w, ldw, rows_per, part);
  weighted_value_finalize<<<(S + 127) / 128, 128, 0, st>>>(blocks, S, part, value);
}

void eval_bits_launch(int64_t N, int S, const int* rowptr, const int* col, const uint32_t* bits,
                      int problem, unsigned long long* counters, int max_grid, cudaStream_t st) {
  const int W = (S + 31) / 32;
  if (W <= 1) launch_g<1>(N, S, W, rowptr, col, bits, problem, counters, max_grid, st);
  else if (W <= 2) launch_g<2>(N, S, W, rowptr, col, bits, problem, counters, max_grid, st);
  else if (W <= 4) launch_g<4>(N, S, W, rowptr, col, bits, problem, counters, max_grid, st);
  else if (W <= 8) launch_g<8>(N, S, W, rowptr, col, bits, problem, counters, max_grid, st);
  else if (W <= 16) launch_g<16>(N, S, W, rowptr, col, bits, problem, counters, max_grid, st);
  else launch_g<32>(N, S, W, rowptr, col, bits, problem, counters, max_grid, st);
}

}  // namespace cpra
