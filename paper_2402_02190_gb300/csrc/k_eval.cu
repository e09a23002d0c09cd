// Exact integer evaluation of the rounded shots from their packed bits
// (App. C.2 rounding, Table objective-functions, Prop. 3.2).
//
// x_bits holds, per node, W = ceil(S/32) words; bit (s mod 32) of word s/32
// is x_is.  A segment of L >= max(W, 8) lanes owns one node row: lane w
// holds word w of x_i, and the segment's lanes hold up to L column indices
// of the row at a time.  A ballot picks the neighbours j > i (each
// undirected edge once, at its lower endpoint); they are taken kU = 3 at a
// time, every lane combining x_i[w] with x_j[w] (AND for MIS violations,
// XOR for MaxCut cut edges).  A carry-save adder reduces the combined words
// to a 2-bit count per bit position, which one ripple add puts into
// bit-sliced vertical counters (eight bit planes: 32 counters of 8 bits per
// lane).  MIS set sizes add x_i[w] the same way; the pairwise Hamming sum
// adds k_i (S - k_i) with k_i = popcount of row i.  The planes are decoded
// by 8 x 8 bit-matrix transposes into 32 counts: before a counter can pass
// 255 by one lane alone (rare), and once at the end by the whole warp, whose
// segments first sum the counts of the same word with shuffles so that each
// shared-memory atomic instruction touches distinct per-shot counters.  All
// sums are integers, so the result does not depend on the order of the
// atomics.
//
// Rows, neighbour passes and chunks advance in step across the warp (their
// trip counts are warp maxima), so the segments of a warp never diverge and
// a row whose neighbours are done costs a warp nothing but its share of
// the slowest row's chunks.
#include "common.cuh"
#include "kernels.cuh"

namespace cpra {

namespace {

constexpr int kU = 3;          // neighbours per chunk (measured: 2, 3 and 4 within 2%)
constexpr int kMaxCount = 255; // counter capacity of eight bit planes

// Transposes the 8 x 8 bit matrix held in x (row k = byte k, column r = bit r
// of the byte): bit 8k + r moves to bit 8r + k.
__device__ __forceinline__ uint64_t transpose8x8(uint64_t x) {
  uint64_t t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
  x = x ^ t ^ (t << 7);
  t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
  x = x ^ t ^ (t << 14);
  t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
  x = x ^ t ^ (t << 28);
  return x;
}

// 32 counters of 8 bits each, stored as 8 bit planes (plane k holds bit k
// of every counter).
struct Planes {
  uint32_t p[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  int n = 0;  // largest value any counter can hold since the last flush
  // Adds the bits of `in` (bit-sliced value of planes k0 and up) with
  // carry propagation through the upper planes.
  __device__ __forceinline__ void ripple(uint32_t cy, int k0) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (k < k0) continue;
      const uint32_t t = p[k] & cy;
      p[k] ^= cy;
      cy = t;
    }
  }
  // Adds one word (each counter grows by its bit).
  __device__ __forceinline__ void add1(uint32_t x) {
    ripple(x, 0);
    n += 1;
  }
  // Adds the per-bit sum of v[0..KU-1] (KU <= 4); c bounds that sum.
  template <int KU>
  __device__ __forceinline__ void add_chunk(const uint32_t (&v)[KU], int c) {
    // carry-save reduction to ones + 2 twos + 4 fours
    uint32_t ones = v[0], twos = 0u, fours = 0u;
    if constexpr (KU == 2) {
      ones = v[0] ^ v[1];
      twos = v[0] & v[1];
    } else if constexpr (KU >= 3) {
      const uint32_t u = v[0] ^ v[1];
      const uint32_t s = u ^ v[2];
      const uint32_t c1 = (v[0] & v[1]) | (u & v[2]);  // v0 + v1 + v2 = s + 2 c1
      if constexpr (KU == 3) {
        ones = s;
        twos = c1;
      } else {
        ones = s ^ v[3];
        const uint32_t c2 = s & v[3];                    // s + v3 = ones + 2 c2
        twos = c1 ^ c2;
        fours = c1 & c2;
      }
    }
    // planes += ones + 2 twos + 4 fours
    uint32_t cy = p[0] & ones;
    p[0] ^= ones;
    uint32_t w = p[1] ^ twos;
    uint32_t nc = (p[1] & twos) | (w & cy);
    p[1] = w ^ cy;
    cy = nc;
    if constexpr (KU == 4) {
      w = p[2] ^ fours;
      nc = (p[2] & fours) | (w & cy);
      p[2] = w ^ cy;
      ripple(nc, 3);
    } else {
      ripple(cy, 2);
    }
    n += c;
  }
  // The 32 counts as four 64-bit words: byte q of the eight planes is an
  // 8 x 8 bit matrix (plane x bit) whose transpose holds the counts of bits
  // 8q .. 8q+7 as bytes.
  __device__ __forceinline__ uint64_t decode(int q) const {
    const uint32_t sel = (uint32_t)q | ((uint32_t)(q + 4) << 4);
    const uint32_t lo =
        __byte_perm(__byte_perm(p[0], p[1], sel), __byte_perm(p[2], p[3], sel), 0x5410);
    const uint32_t hi =
        __byte_perm(__byte_perm(p[4], p[5], sel), __byte_perm(p[6], p[7], sel), 0x5410);
    return transpose8x8(((uint64_t)hi << 32) | lo);
  }
  __device__ __forceinline__ void clear() {
#pragma unroll
    for (int k = 0; k < 8; ++k) p[k] = 0u;
    n = 0;
  }
  // One lane alone: adds its 32 counts to cnt[0..31] and clears the planes.
  __device__ __forceinline__ void flush(int* cnt) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint64_t x = decode(q);
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const int c = (int)((x >> (8 * r)) & 0xffu);
        if (c) atomicAdd(cnt + 8 * q + r, c);
      }
    }
    clear();
  }
  // The final flush, with every lane of the warp present: the decoded counts
  // of the 32/L segments that hold the same word are summed by shuffles (as
  // 16-bit pairs: at most 32 x 255 per count), then lane `seg` of the word
  // adds counts seg*L .. seg*L + L-1 to cnt, so no two lanes of one atomic
  // instruction share an address.
  template <int L>
  __device__ __forceinline__ void flush_warp(int* cnt, bool active, int seg) {
    uint32_t h[16];  // h[4q + 2m + o]: counts of bits 8q + 4m + o and 8q + 4m + o + 2
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint64_t x = active ? decode(q) : 0ull;
      const uint32_t x0 = (uint32_t)x, x1 = (uint32_t)(x >> 32);
      h[4 * q + 0] = x0 & 0x00ff00ffu;
      h[4 * q + 1] = (x0 >> 8) & 0x00ff00ffu;
      h[4 * q + 2] = x1 & 0x00ff00ffu;
      h[4 * q + 3] = (x1 >> 8) & 0x00ff00ffu;
    }
#pragma unroll
    for (int off = L; off < 32; off <<= 1)
#pragma unroll
      for (int m = 0; m < 16; ++m) h[m] += __shfl_xor_sync(0xffffffffu, h[m], off);
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      // bit t = 8q + 4m + 2a + o  ->  half a of h[4q + 2m + o]
      const int q = t >> 3, m = (t >> 2) & 1, a = (t >> 1) & 1, o = t & 1;
      const int c = (int)((h[4 * q + 2 * m + o] >> (16 * a)) & 0xffffu);
      if (active && t / L == seg && c) atomicAdd(cnt + t, c);
    }
    clear();
  }
};

template <int L, int PROBLEM>
__global__ void __launch_bounds__(256)
eval_bits_kernel(int64_t N, int S, int W, const int* __restrict__ rowptr,
                 const int* __restrict__ col, const uint32_t* __restrict__ bits,
                 unsigned long long* counters) {
  __shared__ int scnt[2 * 1024];  // objective per shot, then violations per shot
  __shared__ unsigned long long ham_s;
  const int lane = threadIdx.x & 31;
  const int sub = lane & (L - 1);
  const int seg = lane / L;
  const int64_t segs_per_block = (int64_t)(blockDim.x >> 5) * (32 / L);
  const int64_t first = (int64_t)blockIdx.x * segs_per_block + (threadIdx.x >> 5) * (32 / L) + seg;
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

  // CSR pipeline: the current row's range and first L column indices, and
  // the next row's range, are loaded one row ahead
  int beg = 0, end = 0, jfirst = -1, nbeg = 0, nend = 0;
  if (first < N) {
    csr_row(rowptr, first, N, beg, end);
    if constexpr (PROBLEM == 2) end = beg;  // set sizes and the Hamming sum only
    jfirst = (sub < end - beg) ? csr_col(col, beg + sub, N) : -1;
  }
  if (first + stride < N) {
    csr_row(rowptr, first + stride, N, nbeg, nend);
    if constexpr (PROBLEM == 2) nend = nbeg;
  }
  // rows in step across the warp: a segment whose rows are done runs the
  // last iterations with empty ranges and a zero row
  for (int64_t i = first; __any_sync(0xffffffffu, i < N); i += stride) {
    const bool row = i < N;
    const uint32_t xi = (row && active) ? bits[i * W + sub] : 0u;
    const int njfirst = (i + stride < N && sub < nend - nbeg) ? csr_col(col, nbeg + sub, N) : -1;
    int pbeg = 0, pend = 0;
    if (i + 2 * stride < N) {
      csr_row(rowptr, i + 2 * stride, N, pbeg, pend);
      if constexpr (PROBLEM == 2) pend = pbeg;
    }
    // Neighbour passes of L column indices, in step across the warp (every
    // lane takes part in each pass, so the ballot and the slot loop below
    // are warp-uniform; a segment past its row's end contributes nothing).
    for (int eb = beg;; eb += L) {
      if (!__any_sync(0xffffffffu, eb < end)) break;
      const int j = (eb == beg) ? jfirst : ((eb + sub < end) ? csr_col(col, eb + sub, N) : -1);
      // the segment's neighbours j > i, as a mask over its lanes
      uint32_t m = __ballot_sync(0xffffffffu, j > i) >> (seg * L);
      if constexpr (L < 32) m &= (1u << (L & 31)) - 1u;
      const int nv = __popc(m);
      const int nvmax = __reduce_max_sync(0xffffffffu, nv);
      for (int c0 = 0; c0 < nvmax; c0 += kU) {
        uint32_t v[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
          const int src = __ffs(m) - 1;  // next neighbour's lane, -1 when none is left
          m &= m - 1u;
          const int jj = __shfl_sync(0xffffffffu, j, src < 0 ? 0 : src, L);
          const uint32_t xj = (src >= 0 && active) ? bits[(int64_t)jj * W + sub] : 0u;
          v[u] = src < 0 ? 0u : (PROBLEM == 0 ? (xi & xj) : (xi ^ xj));
        }
        const int c = max(0, min(kU, nv - c0));
        Planes& pl = PROBLEM == 0 ? viol : obj;
        if (pl.n + c > kMaxCount && active) pl.flush(PROBLEM == 0 ? cnt_viol : cnt_obj);
        pl.add_chunk<kU>(v, c);
      }
    }
    int k = __popc(xi);
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1) k += __shfl_xor_sync(0xffffffffu, k, off);
    if (sub == 0) ham += (long long)k * (long long)(S - k);
    if (PROBLEM != 1 && row) {
      if (obj.n + 1 > kMaxCount && active) obj.flush(cnt_obj);
      obj.add1(xi);
    }
    beg = nbeg;
    end = nend;
    jfirst = njfirst;
    nbeg = pbeg;
    nend = pend;
  }
  // every lane of the warp takes part in the shuffles of the final flush
  obj.flush_warp<L>(cnt_obj, active, seg);
  if (PROBLEM == 0) viol.flush_warp<L>(cnt_viol, active, seg);
  if (ham) atomicAdd(&ham_s, (unsigned long long)ham);
  __syncthreads();
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    if (scnt[s]) atomicAdd(&counters[s], (unsigned long long)scnt[s]);
    if (scnt[Wpad + s]) atomicAdd(&counters[S + s], (unsigned long long)scnt[Wpad + s]);
  }
  if (threadIdx.x == 0 && ham_s) atomicAdd(&counters[2 * S], ham_s);
}

template <int L>
void launch_l(int64_t N, int S, int W, const int* rowptr, const int* col, const uint32_t* bits,
              int problem, unsigned long long* counters, int max_grid, cudaStream_t st) {
  constexpr int threads = 256;
  const int segs_per_block = (threads / 32) * (32 / L);
  int64_t want = (N + segs_per_block - 1) / segs_per_block;
  int grid = (int)(want < max_grid ? want : max_grid);
  if (grid < 1) grid = 1;
  if (problem == 0)
    eval_bits_kernel<L, 0><<<grid, threads, 0, st>>>(N, S, W, rowptr, col, bits, counters);
  else if (problem == 1)
    eval_bits_kernel<L, 1><<<grid, threads, 0, st>>>(N, S, W, rowptr, col, bits, counters);
  else
    eval_bits_kernel<L, 2><<<grid, threads, 0, st>>>(N, S, W, rowptr, col, bits, counters);
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

// Weighted MaxCut: the cut weight of each shot, the sum of A_ij over the
// edges j > i with x_is != x_js, in FP64.  Thread s of block b walks the rows
// of b's range in order (the threads of a warp read the same column indices
// and weights, and the same 32-shot bit words); the blocks are then added
// in order by weighted_value_finalize.
__global__ void weighted_cut_kernel(int64_t N, int S, int W, const int* __restrict__ rowptr,
                                    const int* __restrict__ col, const float* __restrict__ ew,
                                    const uint32_t* __restrict__ bits, int64_t rows_per,
                                    double* __restrict__ part) {
  const int64_t r0 = (int64_t)blockIdx.x * rows_per;
  const int64_t r1 = r0 + rows_per < N ? r0 + rows_per : N;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const int w = s >> 5, b = s & 31;
    double t = 0.0;
    for (int64_t r = r0; r < r1; ++r) {
      const uint32_t xr = (bits[r * W + w] >> b) & 1u;
      int beg, end;
      csr_row(rowptr, r, N, beg, end);
      for (int e = beg; e < end; ++e) {
        const int j = csr_col(col, e, N);
        if (j > r && ((bits[(int64_t)j * W + w] >> b) & 1u) != xr) t += (double)ew[e];
      }
    }
    part[(int64_t)blockIdx.x * S + s] = t;
  }
}

}  // namespace

void weighted_cut_launch(int64_t N, int S, const int* rowptr, const int* col, const float* ew,
                         const uint32_t* bits, double* part, int max_blocks, double* value,
                         cudaStream_t st) {
  int64_t rows_per = (N + max_blocks - 1) / max_blocks;
  if (rows_per < 1) rows_per = 1;
  const int blocks = (int)((N + rows_per - 1) / rows_per);
  weighted_cut_kernel<<<blocks, 128, 0, st>>>(N, S, (S + 31) / 32, rowptr, col, ew, bits,
                                              rows_per, part);
  weighted_value_finalize<<<(S + 127) / 128, 128, 0, st>>>(blocks, S, part, value);
}

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
  if (W <= 8) launch_l<8>(N, S, W, rowptr, col, bits, problem, counters, max_grid, st);
  else if (W <= 16) launch_l<16>(N, S, W, rowptr, col, bits, problem, counters, max_grid, st);
  else launch_l<32>(N, S, W, rowptr, col, bits, problem, counters, max_grid, st);
}

#ifdef CPRA_CHECKED
void csr_check_collect_eval(CsrCheck* r) { CPRA_CSR_CHECK_COLLECT(r); }
#endif

}  // namespace cpra
