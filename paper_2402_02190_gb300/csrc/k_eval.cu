// Exact integer evaluation of the rounded shots from their packed bits
// (App. C.2 rounding, Table objective-functions, Prop. 3.2).
//
// x_bits holds, per node, W = ceil(S/32) words; bit (s mod 32) of word s/32
// is x_is.  A segment of L >= max(W, 8) lanes owns one node row: lane w
// holds word w of x_i, and the segment's lanes hold up to L column indices
// of the row at a time.  Every counter is bit-sliced: plane k of a lane's
// counter holds bit k of the 32 per-shot counts of the lane's word, so one
// logic instruction updates 32 counters.
//
// Edges.  The column indices of a pass are taken in groups of at most 7
// slots; slot u of every segment reads the word of its row's u-th neighbour
// j (only j > i, so each undirected edge is seen once, at its lower
// endpoint) and combines it with x_i (AND for MIS violations, XOR for MaxCut
// cut edges).  A carry-save tree of full adders reduces the group to a
// 3-plane count (at most 7), which is added into a 4-plane low-order
// counter; the low-order counter is added into the 8-plane main counter
// only when its bound would pass 15, and the main counter goes to shared
// memory only when its bound would pass 255.  Set sizes (MIS) add x_i into
// a 3-plane low-order counter the same way; the pairwise Hamming sum adds
// k_i (S - k_i) with k_i = popcount of row i.  The bounds count slots and
// rows, not set bits, and are warp-uniform, so no branch diverges.
//
// Rows, neighbour passes and groups advance in step across the warp (their
// trip counts are warp maxima); a segment whose row is done reads nothing.
// At the end the main planes are decoded by 8 x 8 bit-matrix transposes into
// 32 counts, the segments of a warp sum the counts of the same word with
// shuffles, and each shared-memory atomic instruction touches distinct
// per-shot counters.  All sums are integers, so the result does not depend
// on the order of the atomics.
#include "common.cuh"
#include "kernels.cuh"

namespace cpra {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kMaxCount = 255;  // capacity of the 8-plane main counters

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

// Full adder on 32 bit positions: a + b + c = s + 2 cy.
__device__ __forceinline__ void full_add(uint32_t a, uint32_t b, uint32_t c, uint32_t& s,
                                         uint32_t& cy) {
  s = a ^ b ^ c;
  cy = (a & b) | (c & (a ^ b));
}

// acc += x, both bit-sliced (K and M <= K planes); the caller's bound keeps
// the sum below 2^K, so the carry out of the top plane is zero.
template <int K, int M>
__device__ __forceinline__ void add_planes(uint32_t (&acc)[K], const uint32_t (&x)[M]) {
  uint32_t cy = 0u;
#pragma unroll
  for (int k = 0; k < K; ++k) {
    if (k < M) {
      if (k == 0) {
        cy = acc[0] & x[0];
        acc[0] ^= x[0];
      } else {
        uint32_t s;
        full_add(acc[k], x[k], cy, s, cy);
        acc[k] = s;
      }
    } else if (k == K - 1) {
      acc[k] ^= cy;
    } else {
      const uint32_t t = acc[k] & cy;
      acc[k] ^= cy;
      cy = t;
    }
  }
}

template <int K>
__device__ __forceinline__ void clear_planes(uint32_t (&acc)[K]) {
#pragma unroll
  for (int k = 0; k < K; ++k) acc[k] = 0u;
}

// 32 counters of 8 bits each, stored as 8 bit planes (plane k holds bit k
// of every counter).
struct Planes {
  uint32_t p[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
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
    clear_planes(p);
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
      for (int m = 0; m < 16; ++m) h[m] += __shfl_xor_sync(kFull, h[m], off);
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      // bit t = 8q + 4m + 2a + o  ->  half a of h[4q + 2m + o]
      const int q = t >> 3, m = (t >> 2) & 1, a = (t >> 1) & 1, o = t & 1;
      const int c = (int)((h[4 * q + 2 * m + o] >> (16 * a)) & 0xffffu);
      if (active && t / L == seg && c) atomicAdd(cnt + t, c);
    }
    clear_planes(p);
  }
};

// V bit-sliced counters (one per word of a lane): K low-order planes and,
// with kMain, 8 main planes.  The bounds are shared by the V words and are
// warp-uniform.  Without main planes the low-order planes go to shared
// memory whenever their bound would pass 2^K - 1.
template <int K, int V, bool kMain>
struct Counter {
  Planes main[kMain ? V : 1];
  uint32_t low[V][K] = {};
  int n_main = 0, n_low = 0;
  // The low-order planes of word w as a Planes value (upper planes zero).
  __device__ __forceinline__ Planes low_planes(int w) const {
    Planes t;
#pragma unroll
    for (int k = 0; k < K; ++k) t.p[k] = low[w][k];
    return t;
  }
  // Empties the low-order planes: into the main planes (flushing those to
  // cnt, 32 counters per word, first if the sum could pass 255), or without
  // main planes straight to cnt.
  __device__ __forceinline__ void spill(int* cnt, bool active) {
    if constexpr (kMain) {
      if (n_main + n_low > kMaxCount) {
        if (active) {
#pragma unroll
          for (int w = 0; w < V; ++w) main[w].flush(cnt + 32 * w);
        }
        n_main = 0;
      }
#pragma unroll
      for (int w = 0; w < V; ++w) add_planes<8, K>(main[w].p, low[w]);
      n_main += n_low;
    } else {
      if (active) {
#pragma unroll
        for (int w = 0; w < V; ++w) low_planes(w).flush(cnt + 32 * w);
      }
    }
#pragma unroll
    for (int w = 0; w < V; ++w) clear_planes(low[w]);
    n_low = 0;
  }
  // Adds an M-plane count per word whose value is at most c.
  template <int M>
  __device__ __forceinline__ void add(const uint32_t (&x)[V][M], int c, int* cnt, bool active) {
    if (n_low + c > (1 << K) - 1) spill(cnt, active);
#pragma unroll
    for (int w = 0; w < V; ++w) add_planes<K, M>(low[w], x[w]);
    n_low += c;
  }
  template <int L>
  __device__ __forceinline__ void flush_warp(int* cnt, bool active, int seg) {
    if constexpr (kMain) {
      spill(cnt, active);
#pragma unroll
      for (int w = 0; w < V; ++w) main[w].template flush_warp<L>(cnt + 32 * w, active, seg);
    } else {
#pragma unroll
      for (int w = 0; w < V; ++w) low_planes(w).template flush_warp<L>(cnt + 32 * w, active, seg);
    }
  }
};

// The lane's V consecutive words of one row (V = 2 needs an even W, so the
// pair is 8-byte aligned).
template <int V>
__device__ __forceinline__ void load_words(const uint32_t* __restrict__ p, uint32_t (&x)[V]) {
  if constexpr (V == 1) {
    x[0] = *p;
  } else {
    const uint2 t = *reinterpret_cast<const uint2*>(p);
    x[0] = t.x;
    x[1] = t.y;
  }
}

// One group of at most G slots (G = 3, 5 or 7) starting at slot U0 of a
// pass; slots g..G-1 are empty.  Slot s of a pass is column index s/L held
// by lane s mod L of the segment; it counts if that neighbour j is > i.
// Each slot combines x_i with x_j word by word; the per-bit sum of the
// slots goes into c as a 2- or 3-plane count.
template <int L, int V, int CPL, int PROBLEM, int U0, int G>
__device__ __forceinline__ void edge_group(Counter<4, V, true>& c, int* cnt, bool active, bool act,
                                           int i, const uint32_t (&xi)[V], const int (&j)[CPL],
                                           int g, const uint32_t* __restrict__ bl, int W) {
  uint32_t v[V][G];
#pragma unroll
  for (int u = 0; u < G; ++u) {
    constexpr int kCP = L * CPL;
    const int s = U0 + u;
    int jj = -1;
    if (s < kCP) jj = __shfl_sync(kFull, j[(s / L) % CPL], s % L, L);
    const bool ok = u < g && jj > i && act;
    uint32_t xj[V];
#pragma unroll
    for (int w = 0; w < V; ++w) xj[w] = 0u;
    if (ok) load_words<V>(bl + (int64_t)jj * W, xj);
#pragma unroll
    for (int w = 0; w < V; ++w)
      v[w][u] = PROBLEM == 0 ? (xi[w] & xj[w]) : (ok ? (xi[w] ^ xj[w]) : 0u);
  }
  if constexpr (G == 3) {
    uint32_t x[V][2];
#pragma unroll
    for (int w = 0; w < V; ++w) full_add(v[w][0], v[w][1], v[w][2], x[w][0], x[w][1]);
    c.template add<2>(x, g, cnt, active);
  } else if constexpr (G == 5) {
    uint32_t x[V][3];
#pragma unroll
    for (int w = 0; w < V; ++w) {
      uint32_t s1, c1, c2;
      full_add(v[w][0], v[w][1], v[w][2], s1, c1);
      full_add(s1, v[w][3], v[w][4], x[w][0], c2);
      x[w][1] = c1 ^ c2;
      x[w][2] = c1 & c2;
    }
    c.template add<3>(x, g, cnt, active);
  } else {
    uint32_t x[V][3];
#pragma unroll
    for (int w = 0; w < V; ++w) {
      uint32_t s1, c1, s2, c2, c3;
      full_add(v[w][0], v[w][1], v[w][2], s1, c1);
      full_add(v[w][3], v[w][4], v[w][5], s2, c2);
      full_add(s1, s2, v[w][6], x[w][0], c3);
      full_add(c1, c2, c3, x[w][1], x[w][2]);
    }
    c.template add<3>(x, g, cnt, active);
  }
}

// The group starting at slot U0 of a pass of dpass slots (warp-uniform),
// with the smallest G that holds it, then the next group.
template <int L, int V, int CPL, int PROBLEM, int U0>
__device__ __forceinline__ void edge_groups(Counter<4, V, true>& c, int* cnt, bool active, bool act,
                                            int i, const uint32_t (&xi)[V], const int (&j)[CPL],
                                            int dpass, const uint32_t* __restrict__ bl, int W) {
  if constexpr (U0 < L * CPL) {
    if (U0 >= dpass) return;
    const int g = dpass - U0 < 7 ? dpass - U0 : 7;
    if (g <= 3)
      edge_group<L, V, CPL, PROBLEM, U0, 3>(c, cnt, active, act, i, xi, j, g, bl, W);
    else if (g <= 5)
      edge_group<L, V, CPL, PROBLEM, U0, 5>(c, cnt, active, act, i, xi, j, g, bl, W);
    else
      edge_group<L, V, CPL, PROBLEM, U0, 7>(c, cnt, active, act, i, xi, j, g, bl, W);
    edge_groups<L, V, CPL, PROBLEM, U0 + 7>(c, cnt, active, act, i, xi, j, dpass, bl, W);
  }
}

// L lanes per row, V words per lane; a pass holds CPL column indices per
// lane (L * CPL >= 8).
// 3 blocks of 256 threads per SM (at most 85 registers a thread): the MIS
// instances with two words per lane need 105-116 registers unbounded, and
// the third block's warps hide more of the neighbour-word latency than the
// registers save (measured: 0.086 -> 0.065 ms at N = 10^6, S = 256).
template <int L, int V, int PROBLEM>
__global__ void __launch_bounds__(256, 3)
eval_bits_kernel(int64_t N, int S, int W, const int* __restrict__ rowptr,
                 const int* __restrict__ col, const uint32_t* __restrict__ bits,
                 unsigned long long* counters, const EvalFinalize fin) {
  constexpr bool kEdges = PROBLEM != 2;  // DBM: set sizes and the Hamming sum only
  constexpr bool kSizes = PROBLEM != 1;  // MaxCut: cut edges only
  constexpr int CPL = L >= 8 ? 1 : 8 / L;
  constexpr int CP = L * CPL;            // column indices per pass
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

  const bool active = V * sub < W;
  const uint32_t* __restrict__ bl = bits + V * sub;  // this lane's words of every row
  int* cnt_size = scnt + 32 * V * sub;
  int* cnt_edge = scnt + (PROBLEM == 0 ? Wpad : 0) + 32 * V * sub;
  Counter<6, V, false> size;  // at most one count per row
  Counter<4, V, true> edge;
  long long ham = 0;

  // CSR pipeline: the current row's range and first CP column indices, and
  // the next row's range, are loaded one row ahead
  int beg = 0, end = 0, nbeg = 0, nend = 0;
  int jfirst[CPL];
#pragma unroll
  for (int q = 0; q < CPL; ++q) jfirst[q] = -1;
  if constexpr (kEdges) {
    if (first < N) {
      csr_row(rowptr, first, N, beg, end);
#pragma unroll
      for (int q = 0; q < CPL; ++q)
        if (sub + q * L < end - beg) jfirst[q] = csr_col(col, beg + sub + q * L, N);
    }
    if (first + stride < N) csr_row(rowptr, first + stride, N, nbeg, nend);
  }
  // rows in step across the warp: a segment whose rows are done runs the
  // last iterations with empty ranges and a zero row
  for (int64_t i = first; __any_sync(kFull, i < N); i += stride) {
    const bool row = i < N;
    const bool act = row && active;
    uint32_t xi[V];
#pragma unroll
    for (int w = 0; w < V; ++w) xi[w] = 0u;
    if (act) load_words<V>(bl + i * W, xi);
    if constexpr (kEdges) {
      const int ii = row ? (int)i : 0;  // column indices are int32, so is every row
      int njfirst[CPL];
      const bool nrow = i + stride < N;
#pragma unroll
      for (int q = 0; q < CPL; ++q)
        njfirst[q] = (nrow && sub + q * L < nend - nbeg) ? csr_col(col, nbeg + sub + q * L, N) : -1;
      int pbeg = 0, pend = 0;
      if (i + 2 * stride < N) csr_row(rowptr, i + 2 * stride, N, pbeg, pend);
      // neighbour passes of CP column indices, groups of at most 7 slots,
      // all warp-uniform
      for (int eb = beg;; eb += CP) {
        const int dmax = __reduce_max_sync(kFull, end - eb);
        if (dmax <= 0) break;
        int j[CPL];
#pragma unroll
        for (int q = 0; q < CPL; ++q)
          j[q] = (eb == beg) ? jfirst[q]
                             : ((eb + sub + q * L < end) ? csr_col(col, eb + sub + q * L, N) : -1);
        const int dpass = dmax < CP ? dmax : CP;
        edge_groups<L, V, CPL, PROBLEM, 0>(edge, cnt_edge, active, act, ii, xi, j, dpass, bl, W);
      }
      beg = nbeg;
      end = nend;
#pragma unroll
      for (int q = 0; q < CPL; ++q) jfirst[q] = njfirst[q];
      nbeg = pbeg;
      nend = pend;
    }
    int k = 0;
#pragma unroll
    for (int w = 0; w < V; ++w) k += __popc(xi[w]);
#pragma unroll
    for (int off = L / 2; off > 0; off >>= 1) k += __shfl_xor_sync(kFull, k, off);
    if (sub == 0) ham += (long long)k * (long long)(S - k);
    if constexpr (kSizes) {
      uint32_t x[V][1];
#pragma unroll
      for (int w = 0; w < V; ++w) x[w][0] = xi[w];
      size.template add<1>(x, 1, cnt_size, active);
    }
  }
  // every lane of the warp takes part in the shuffles of the final flush
  if constexpr (kSizes) size.template flush_warp<L>(cnt_size, active, seg);
  if constexpr (kEdges) edge.template flush_warp<L>(cnt_edge, active, seg);
  if (ham) atomicAdd(&ham_s, (unsigned long long)ham);
  __syncthreads();
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    if (scnt[s]) atomicAdd(&counters[s], (unsigned long long)scnt[s]);
    if (scnt[Wpad + s]) atomicAdd(&counters[S + s], (unsigned long long)scnt[Wpad + s]);
  }
  if (threadIdx.x == 0 && ham_s) atomicAdd(&counters[2 * S], ham_s);
  if constexpr (PROBLEM != 2) {
    if (fin.records) {
      // the block's additions are visible device-wide before its ticket;
      // the last block then sees every block's additions
      __shared__ bool last;
      __threadfence();
      __syncthreads();
      if (threadIdx.x == 0) {
        const unsigned long long t =
            atomicAdd(&counters[2 * S + 1], 1ull);
        last = t == (unsigned long long)gridDim.x - 1ull;
      }
      __syncthreads();
      if (last) {
        __threadfence();
        volatile unsigned long long* vc = counters;
        ShotEvalRec* rec = static_cast<ShotEvalRec*>(fin.records);
        for (int s = threadIdx.x; s < S; s += blockDim.x) {
          const long long obj = (long long)vc[s];
          const long long viol = (long long)vc[S + s];
          const double value = fin.wvalue ? fin.wvalue[s] : (double)obj;
          rec[s].objective = obj;
          rec[s].violations = PROBLEM == 0 ? viol : 0;
          rec[s].qubo = PROBLEM == 0 ? -value + (double)fin.lambda[s] * (double)viol : -value;
          rec[s].value = value;
          vc[s] = 0ull;
          vc[S + s] = 0ull;
        }
        if (threadIdx.x == 0) {
          if (fin.ham) *fin.ham = (long long)vc[2 * S];
          vc[2 * S] = 0ull;
          vc[2 * S + 1] = 0ull;
        }
      }
    }
  }
}

template <int L, int V, int PROBLEM>
void launch_lp(int64_t N, int S, int W, const int* rowptr, const int* col, const uint32_t* bits,
               unsigned long long* counters, int sms, cudaStream_t st, const EvalFinalize& fin) {
  // one wave of resident blocks: the rows are spread evenly over the
  // segments, so a second, partial wave would only add a tail
  static const int per_sm = [] {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, eval_bits_kernel<L, V, PROBLEM>, 256,
                                                      0) != cudaSuccess || b < 1)
      b = 1;
    return b;
  }();
  if (sms < 1) sms = 1;
  // small graphs: narrower blocks, so that the rows reach every SM
  int threads = 256;
  auto blocks = [&](int t) {
    const int64_t segs = (int64_t)(t / 32) * (32 / L);
    return (N + segs - 1) / segs;
  };
  while (threads > 64 && blocks(threads) < 2 * (int64_t)sms) threads /= 2;
  const int64_t want = blocks(threads);
  const int64_t wave = (int64_t)per_sm * sms;
  const int grid = (int)(want < wave ? (want > 0 ? want : 1) : wave);
  eval_bits_kernel<L, V, PROBLEM>
      <<<grid, threads, 0, st>>>(N, S, W, rowptr, col, bits, counters, fin);
}

template <int L, int V>
void launch_l(int64_t N, int S, int W, const int* rowptr, const int* col, const uint32_t* bits,
              int problem, unsigned long long* counters, int sms, cudaStream_t st,
              const EvalFinalize& fin) {
  if (problem == 0)
    launch_lp<L, V, 0>(N, S, W, rowptr, col, bits, counters, sms, st, fin);
  else if (problem == 1)
    launch_lp<L, V, 1>(N, S, W, rowptr, col, bits, counters, sms, st, fin);
  else
    launch_lp<L, V, 2>(N, S, W, rowptr, col, bits, counters, sms, st, fin);
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
                      int problem, unsigned long long* counters, int sms, cudaStream_t st,
                      const EvalFinalize* fin) {
  const int W = (S + 31) / 32;
  EvalFinalize f;
  if (fin && problem != 2) f = *fin;
  if (W % 2 == 0) {  // two words per lane
    if (W <= 4) launch_l<2, 2>(N, S, W, rowptr, col, bits, problem, counters, sms, st, f);
    else if (W <= 8) launch_l<4, 2>(N, S, W, rowptr, col, bits, problem, counters, sms, st, f);
    else if (W <= 16) launch_l<8, 2>(N, S, W, rowptr, col, bits, problem, counters, sms, st, f);
    else launch_l<16, 2>(N, S, W, rowptr, col, bits, problem, counters, sms, st, f);
  } else {
    if (W <= 8) launch_l<8, 1>(N, S, W, rowptr, col, bits, problem, counters, sms, st, f);
    else if (W <= 16) launch_l<16, 1>(N, S, W, rowptr, col, bits, problem, counters, sms, st, f);
    else launch_l<32, 1>(N, S, W, rowptr, col, bits, problem, counters, sms, st, f);
  }
}

#ifdef CPRA_CHECKED
void csr_check_collect_eval(CsrCheck* r) { CPRA_CSR_CHECK_COLLECT(r); }
#endif

}  // namespace cpra
