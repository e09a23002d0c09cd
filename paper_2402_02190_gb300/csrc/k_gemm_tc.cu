// Tensor-core dense layers of the BF16 form (Eq. GCN combine step, App. C.1):
// tcgen05.mma (kind::f16, BF16 operands, FP32 accumulation in TMEM) fed by
// TMA (cp.async.bulk.tensor, 128-byte swizzle), sm_103a.
//
// C[M x Nc] = A[M x K] * B[Nc x K]^T with both operands K-major.  Each CTA
// owns one n tile of width BN (the last one may be ragged: rows of B past Nc
// read as zeros and their columns are not stored) and a strided set of
// 128-row m tiles.  When the tile's weight slice B[BN x K] fits in shared
// memory it stays resident for the whole persistent kernel and only A
// streams through the ring of shared-memory stages; for wide layers (large
// K) each stage carries the matching 64-column block of B as well.  Roles
// per CTA (one CTA per SM):
//   warp 0      TMA producer (one elected lane)
//   warp 1      TMEM allocation + MMA issuer (one elected lane)
//   warps 2..17 epilogue: TMEM -> registers -> bias / activation / split ->
//               shared-memory staging -> TMA tensor store; four warps per
//               TMEM lane quarter, each owning a quarter of the columns
// Two TMEM accumulators alternate so the epilogue of tile i overlaps the
// MMAs of tile i+1.  Every mbarrier wait is bounded: on expiry the kernel
// records bit 1 in *err_flag, stops issuing, waits (bounded) for its own TMA
// copies, frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"
#include "tc_gemm.cuh"

namespace cpra {
namespace {

constexpr int kBM = 128;            // rows per tile (UMMA M)
constexpr int kBK = 64;             // K elements per stage (128 bytes of BF16)
constexpr int kStageBytes = kBM * kBK * 2;
constexpr int kEpiWarps = 16;   // four per TMEM lane quarter
constexpr int kThreads = 64 + 32 * kEpiWarps;
constexpr uint32_t kSpinLimit = 1u << 26;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t addr, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(addr), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the phase with the given parity.  Gives up after
// kSpinLimit polls or when another role has already given up.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag) {
  const uint32_t a = smem_u32(b);
  for (uint32_t it = 0; it < kSpinLimit; ++it) {
    if (mbar_try(a, parity)) return true;
    if ((it & 1023u) == 1023u && *abort_flag) return false;
  }
  return false;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar,
                                            int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
      : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t desc_kmajor_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);  // start address
  d |= static_cast<uint64_t>(1) << 16;                  // leading offset (unused here)
  d |= static_cast<uint64_t>(1024 >> 4) << 32;          // stride offset between 8-row groups
  d |= static_cast<uint64_t>(1) << 46;                  // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                  // 128-byte swizzle
  return d;
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void umma_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (issue only; pair
// with tmem_wait_ld before reading v).
__device__ __forceinline__ void tmem_ld16_issue(uint32_t taddr, uint32_t* r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  tmem_ld16_issue(taddr, r);
  tmem_wait_ld();
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct TcParams {
  int64_t M = 0;
  int Nc = 0, K = 0, n_kb = 0, BN = 0, n_tiles_n = 0, stages = 0, tmem_cols = 0, acc_stride = 0;
  int64_t m_tiles = 0;
  uint32_t idesc = 0;
  int stream_b = 0;  // 1: B blocks stream with the A stages (weights not resident)
  int epi = 0;
  const float* bias = nullptr;
  void* out0 = nullptr;
  int64_t ld0 = 0;
  int d0 = DT_BF16;
  void* out1 = nullptr;
  int64_t ld1 = 0;
  int d1 = DT_BF16;
  int split = 0;
  const float* row_scale = nullptr;
  int n_valid = 0;
  int* err_flag = nullptr;
  const void* addend = nullptr;
  int64_t ld_add = 0;
  int d_add = DT_BF16;
};

// Output staging: each epilogue warp owns two buffers of 32 rows x 16
// columns; a TMA tensor store writes a buffer out while the warp fills the
// other one.
constexpr int kStgBytes = 32 * 16 * 4;

// Staging of one 32-row x 16-column output box (lane = row) in the layout
// the tensor store reads with its swizzle mode, which spreads the 16-byte
// chunks of consecutive rows over all shared-memory banks: FP32 rows are 64
// bytes (64-byte swizzle: chunk c of row r at c ^ ((r >> 1) & 3)), BF16 rows
// 32 bytes (32-byte swizzle: chunk c at c ^ ((r >> 2) & 1)).  buf is at least
// 512-byte aligned.
__device__ __forceinline__ void stage_row_f32(uint8_t* buf, int r, const float* v) {
#pragma unroll
  for (int c = 0; c < 4; ++c)
    *reinterpret_cast<float4*>(buf + r * 64 + 16 * (c ^ ((r >> 1) & 3))) =
        make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
}
__device__ __forceinline__ void stage_row_bf16(uint8_t* buf, int r, const float* v) {
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    uint32_t w[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      __nv_bfloat162 h = __floats2bfloat162_rn(v[8 * c + 2 * q], v[8 * c + 2 * q + 1]);
      w[q] = *reinterpret_cast<uint32_t*>(&h);
    }
    *reinterpret_cast<uint4*>(buf + r * 32 + 16 * (c ^ ((r >> 2) & 1))) =
        make_uint4(w[0], w[1], w[2], w[3]);
  }
}
constexpr int kStgTotal = kEpiWarps * 2 * kStgBytes;

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, const void* src, int c0, int c1) {
  asm volatile(
      "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%2, %3}], [%1];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(smem_u32(src)), "r"(c0), "r"(c1)
      : "memory");
}

// Epilogue arithmetic of 16 consecutive columns n .. n+15 of one row;
// returns which output (0 / 1) they belong to and their column there.
template <int EPI>
__device__ __forceinline__ int epilogue16(const TcParams& p, int64_t row, int n, float* v,
                                          int* out_col) {
  *out_col = n;
  switch (EPI) {
    case EPI_BIAS_RELU:
    case EPI_RELU_BITS: {
      const float4* b4 = reinterpret_cast<const float4*>(p.bias + n);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 b = __ldg(b4 + j);
        v[4 * j + 0] = fmaxf(v[4 * j + 0] + b.x, 0.f);
        v[4 * j + 1] = fmaxf(v[4 * j + 1] + b.y, 0.f);
        v[4 * j + 2] = fmaxf(v[4 * j + 2] + b.z, 0.f);
        v[4 * j + 3] = fmaxf(v[4 * j + 3] + b.w, 0.f);
      }
      return 0;
    }
    case EPI_BIAS_SIGMOID: {
      if (p.addend && row < p.M) {  // per-element offset of the pre-activation
        float a[16];
        if (p.d_add == DT_BF16) {
          const bf16* src = static_cast<const bf16*>(p.addend) + row * p.ld_add + n;
          load16(src, a);
          load16(src + 8, a + 8);
        } else {
          const float* src = static_cast<const float*>(p.addend) + row * p.ld_add + n;
#pragma unroll
          for (int q = 0; q < 16; q += 4) load16(src + q, a + q);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] += a[k];
      }
      const float4* b4 = reinterpret_cast<const float4*>(p.bias + n);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 b = __ldg(b4 + j);
        const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = 4 * j + e;
          v[k] = (n + k < p.n_valid) ? __fdividef(1.0f, 1.0f + __expf(-(v[k] + bb[e]))) : 0.f;
        }
      }
      return 0;
    }
    case EPI_BIAS: {
      const float4* b4 = reinterpret_cast<const float4*>(p.bias + n);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 b = __ldg(b4 + j);
        const float bb[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int k = 4 * j + e;
          v[k] = (n + k < p.n_valid) ? v[k] + bb[e] : 0.f;
        }
      }
      return 0;
    }
    case EPI_SPLIT: {
      if (n < p.split) return 0;
      const float s = row < p.M ? p.row_scale[row] : 0.f;
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] *= s;
      *out_col = n - p.split;
      return 1;
    }
    default:
      return 0;
  }
}

// The epilogue role: NW warps, NW/4 per TMEM lane quarter (a warp may read
// the lanes of quarter warp & 3), `ew` this warp's index among them.  Per
// tile: TMEM -> registers -> bias / activation / split -> shared-memory
// staging -> TMA tensor store; the accumulator is handed back through
// tempty.
// Epilogue of 16 columns c .. c+15 (tile-relative; n0 + c < Nc) of one row
// per lane (row0 = the warp's first row): bias / activation / split, then
// either mask bits stored directly or a shared-memory staging buffer (two
// per warp, alternating through sb) written out by a TMA tensor store.
template <int EPI>
__device__ __forceinline__ void epilogue_chunk(const TcParams& p, const CUtensorMap* tmO0,
                                               const CUtensorMap* tmO1, uint8_t* stg, int& sb,
                                               int lane, int64_t row0, int n0, int c, float* v) {
  const int64_t row = row0 + lane;
  int col;
  const int which = epilogue16<EPI>(p, row, n0 + c, v, &col);
  if constexpr (EPI == EPI_BIAS_RELU) {
    // optional ReLU mask of the stored activation (dtype d0) as bits
    if (p.out1 && row < p.M) {
      uint32_t bits = 0;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float h = v[i];
        if (p.d0 == DT_BF16) h = __bfloat162float(__float2bfloat16_rn(h));
        bits |= (h > 0.f ? 1u : 0u) << i;
      }
      static_cast<uint16_t*>(p.out1)[row * p.ld1 + (n0 + c) / 16] = static_cast<uint16_t>(bits);
    }
  }
  if constexpr (EPI == EPI_RELU_BITS) {
    // mask of the activation as stored in dtype d0; no tile store
    uint32_t bits = 0;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float h = v[i];
      if (p.d0 == DT_BF16) h = __bfloat162float(__float2bfloat16_rn(h));
      bits |= (h > 0.f ? 1u : 0u) << i;
    }
    if (row < p.M)
      static_cast<uint16_t*>(p.out0)[row * p.ld0 + (n0 + c) / 16] = static_cast<uint16_t>(bits);
    return;
  }
  uint8_t* buf = stg + sb * kStgBytes;
  // the tensor store that last read this buffer must be done with it
  if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
  __syncwarp();
  if ((which ? p.d1 : p.d0) == DT_BF16) stage_row_bf16(buf, lane, v);
  else stage_row_f32(buf, lane, v);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) {  // rows past M are clipped by the tensor map
    tma_store_2d(which ? tmO1 : tmO0, buf, col, static_cast<int>(row0));
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  }
  sb ^= 1;
}

// The epilogue role: NW warps, NW/4 per TMEM lane quarter (a warp may read
// the lanes of quarter warp & 3), `ew` this warp's index among them.  Per
// tile: TMEM -> registers -> epilogue_chunk; the accumulator is handed back
// through tempty.
template <int EPI, int NW>
__device__ __forceinline__ void epilogue_role(const TcParams& p, const CUtensorMap* tmO0,
                                              const CUtensorMap* tmO1, uint8_t* Stg,
                                              uint64_t* tfull, uint64_t* tempty,
                                              volatile int* abort_flag, uint32_t tmem_base,
                                              int warp, int ew, int lane, int group, int groups,
                                              int n0) {
  const int quarter = warp & 3;                 // TMEM lanes this warp may read
  constexpr int parts = NW / 4;                 // column parts per lane quarter
  const int cq = ew >> 2;
  const int nch = p.BN / 16;                    // 16-column chunks, split between parts
  const int c_begin = 16 * (nch * cq / parts);
  const int c_end = 16 * (nch * (cq + 1) / parts);
  uint8_t* stg = Stg + static_cast<size_t>(ew) * 2 * kStgBytes;
  int sb = 0;
  int it = 0;
  for (int64_t mt = group; mt < p.m_tiles; mt += groups, ++it) {
    const int acc = it & 1;
    const uint32_t acc_par = (static_cast<uint32_t>(it) >> 1) & 1u;
    if (!mbar_wait(tfull + acc, acc_par, abort_flag)) {
      if (lane == 0) {
        *abort_flag = 1;
        if (p.err_flag) atomicOr(p.err_flag, 2);
      }
      break;
    }
    tc_fence_after();
    const int64_t row0 = mt * kBM + quarter * 32;
    const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                           static_cast<uint32_t>(acc * p.acc_stride);
    for (int c2 = c_begin; c2 < c_end; c2 += 32) {
      // two TMEM loads in flight per wait
      uint32_t r[2][16];
      const bool two = c2 + 16 < c_end;
      tmem_ld16_issue(taddr + static_cast<uint32_t>(c2), r[0]);
      if (two) tmem_ld16_issue(taddr + static_cast<uint32_t>(c2 + 16), r[1]);
      tmem_wait_ld();
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !two) break;
        const int c = c2 + 16 * h;
        if (n0 + c >= p.Nc) continue;  // ragged last n tile: nothing stored past Nc
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[h][i]);
        epilogue_chunk<EPI>(p, tmO0, tmO1, stg, sb, lane, row0, n0, c, v);
      }
    }
    tc_fence_before();
    __syncwarp();
    if (lane == 0) mbar_arrive(tempty + acc);
  }
  if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  __syncwarp();
}

template <int EPI>
__global__ void __launch_bounds__(kThreads, 1)
tc_gemm_nt_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                  const __grid_constant__ CUtensorMap tmO0,
                  const __grid_constant__ CUtensorMap tmO1, const TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t b_kb_bytes = static_cast<uint32_t>(p.BN) * kBK * 2;
  const bool sb_mode = p.stream_b != 0;
  // resident: [B: n_kb blocks][A stages]; streaming: stages of [A block | B block]
  const uint32_t stage_bytes = kStageBytes + (sb_mode ? b_kb_bytes : 0u);
  uint8_t* Bs = smem;
  uint8_t* As = sb_mode ? smem : Bs + static_cast<size_t>(p.n_kb) * b_kb_bytes;
  uint8_t* Stg = As + static_cast<size_t>(p.stages) * stage_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(Stg + kStgTotal);
  uint64_t* empty = full + p.stages;
  uint64_t* bfull = empty + p.stages;
  uint64_t* tfull = bfull + 1;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int n_tile = blockIdx.x % p.n_tiles_n;
  const int group = blockIdx.x / p.n_tiles_n;
  const int groups = gridDim.x / p.n_tiles_n;
  const int n0 = n_tile * p.BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(bfull, 1);
    mbar_init(tfull + 0, 1);
    mbar_init(tfull + 1, 1);
    mbar_init(tempty + 0, kEpiWarps);
    mbar_init(tempty + 1, kEpiWarps);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  auto give_up = [&]() {
    *abort_flag = 1;
    if (p.err_flag) atomicOr(p.err_flag, 2);
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      if (!sb_mode) {
        mbar_expect_tx(bfull, static_cast<uint32_t>(p.n_kb) * b_kb_bytes);
        for (int kb = 0; kb < p.n_kb; ++kb)
          tma_load_2d(Bs + static_cast<size_t>(kb) * b_kb_bytes, &tmB, bfull, kb * kBK, n0);
      }
      uint32_t armed = 0;        // bit s: stage s has been armed at least once
      uint32_t last_par = 0;     // bit s: parity of the last arming of stage s
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t mt = group; ok && mt < p.m_tiles; mt += groups) {
        for (int kb = 0; kb < p.n_kb; ++kb) {
          if (!mbar_wait(empty + stage, phase ^ 1u, abort_flag)) {
            give_up();
            ok = false;
            break;
          }
          uint8_t* st = As + static_cast<size_t>(stage) * stage_bytes;
          mbar_expect_tx(full + stage, stage_bytes);
          tma_load_2d(st, &tmA, full + stage, kb * kBK, static_cast<int>(mt * kBM));
          if (sb_mode) tma_load_2d(st + kStageBytes, &tmB, full + stage, kb * kBK, n0);
          armed |= 1u << stage;
          last_par = (last_par & ~(1u << stage)) | (phase << stage);
          if (++stage == p.stages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        // let our own copies land before the CTA's shared memory goes away
        for (int s = 0; s < p.stages; ++s)
          if (armed & (1u << s)) {
            const uint32_t a = smem_u32(full + s);
            for (uint32_t it = 0; it < kSpinLimit && !mbar_try(a, (last_par >> s) & 1u); ++it) {
            }
          }
        if (!sb_mode) {
          const uint32_t a = smem_u32(bfull);
          for (uint32_t it = 0; it < kSpinLimit && !mbar_try(a, 0); ++it) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      bool ok = sb_mode || mbar_wait(bfull, 0, abort_flag);
      if (!ok) give_up();
      int stage = 0;
      uint32_t phase = 0;
      int it = 0;
      for (int64_t mt = group; ok && mt < p.m_tiles; mt += groups, ++it) {
        const int acc = it & 1;
        const uint32_t acc_par = (static_cast<uint32_t>(it) >> 1) & 1u;
        if (!mbar_wait(tempty + acc, acc_par ^ 1u, abort_flag)) {
          give_up();
          break;
        }
        tc_fence_after();
        const uint32_t d_tmem = tmem_base + static_cast<uint32_t>(acc * p.acc_stride);
        for (int kb = 0; kb < p.n_kb; ++kb) {
          if (!mbar_wait(full + stage, phase, abort_flag)) {
            give_up();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t a0 = smem_u32(As + static_cast<size_t>(stage) * stage_bytes);
          const uint32_t b0 = sb_mode ? a0 + kStageBytes
                                      : smem_u32(Bs + static_cast<size_t>(kb) * b_kb_bytes);
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k)
            umma_bf16(d_tmem, desc_kmajor_sw128(a0 + 32 * k), desc_kmajor_sw128(b0 + 32 * k),
                      p.idesc, (kb | k) != 0 ? 1u : 0u);
          umma_commit(empty + stage);
          if (++stage == p.stages) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (ok) umma_commit(tfull + acc);
      }
    }
  } else {
    epilogue_role<EPI, kEpiWarps>(p, &tmO0, &tmO1, Stg, tfull, tempty, abort_flag, tmem_base, warp,
                                  warp - 2, lane, group, groups, n0);
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(p.tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------- FP32 form: split TF32
// C[M x Nc] = A[M x K] B[Nc x K]^T for FP32 operands, to FP32 accuracy, on
// the tensor cores (tcgen05.mma kind::tf32).  Every operand value x is
// split exactly into three TF32 values, x = x_hi + x_mid + x_lo, with
// x_hi = tf32(x), x_mid = tf32(x - x_hi), x_lo = x - x_hi - x_mid (round to
// nearest; 11 + 11 significant bits cover 22 of FP32's 24, and the last 2
// fit in x_lo).  Each k block sums the six products whose order of
// magnitude is at least 2^-22 of |A||B| (hi.hi, hi.mid, mid.hi, hi.lo,
// lo.hi, mid.mid; the three left out are below 2^-32) into fresh TMEM
// accumulators -- hi.hi in one, the five smaller products in another --
// and the accumulation warps add both block sums into FP32 registers with
// round-to-nearest.  The tensor core's own accumulation is thus limited to
// one 32-deep k block, and the large sum to four additions in it:
// accumulating whole tiles in TMEM measured 10-30x less accurate than FP32
// CUDA-core GEMMs whatever the split (two-way or three-way), which points
// at the rounding of the tensor core's accumulator rather than at the
// operands.  Two accumulator pairs alternate so the MMAs of block j+1
// overlap the read-out of block j.  The
// weights arrive split (K-major hi, mid and lo copies written with the
// weight shadows); A arrives raw through TMA and two converter warps split
// each stage in shared memory: hi in place, mid and lo beside it.  Roles
// per CTA (one per SM):
//   warp 0       TMA producer (A stage, B_hi, B_mid and B_lo blocks)
//   warp 1       TMEM allocation + MMA issuer
//   warps 2..3   converters (A -> A_hi, A_mid, A_lo)
//   warps 4..11  accumulation and epilogue, two per TMEM lane quarter:
//                each holds up to 64 columns of its 32 rows in registers
// Stages: [A_hi | A_mid | A_lo | B_hi | B_mid | B_lo], 32 K elements (128
// bytes per row) each, 128-byte swizzle; the split is element-wise, so the
// parts keep the swizzled layout of A.  Bounded waits as in the BF16 kernel.
constexpr int kBK3 = 32;            // FP32 K elements per stage (128 bytes)
constexpr int kBN3 = 128;           // widest n tile
constexpr int kConvWarps = 2;
constexpr int kEpiWarps3 = 8;
constexpr int kThreads3 = 64 + 32 * (kConvWarps + kEpiWarps3);
constexpr int kStgTotal3 = kEpiWarps3 * 2 * kStgBytes;
constexpr uint32_t kAStage3 = kBM * kBK3 * 4;  // 16 KB

__device__ __forceinline__ void umma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate)
      : "memory");
}

// 12 warps: at most 3 per SM sub-partition, so up to 168 registers per thread
template <int EPI>
__global__ void __launch_bounds__(kThreads3, 1)
tc3_gemm_nt_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmBh,
                   const __grid_constant__ CUtensorMap tmBm,
                   const __grid_constant__ CUtensorMap tmBl,
                   const __grid_constant__ CUtensorMap tmO0,
                   const __grid_constant__ CUtensorMap tmO1, const TcParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t b_bytes = static_cast<uint32_t>(p.BN) * kBK3 * 4;
  const uint32_t stage_bytes = 3 * kAStage3 + 3 * b_bytes;
  uint8_t* St = smem;
  uint8_t* Stg = St + static_cast<size_t>(p.stages) * stage_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(Stg + kStgTotal3);
  uint64_t* conv = full + p.stages;
  uint64_t* empty = conv + p.stages;
  uint64_t* tfull = empty + p.stages;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int n_tile = blockIdx.x % p.n_tiles_n;
  const int group = blockIdx.x / p.n_tiles_n;
  const int groups = gridDim.x / p.n_tiles_n;
  const int n0 = n_tile * p.BN;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(conv + s, kConvWarps);
      mbar_init(empty + s, 1);
    }
    mbar_init(tfull + 0, 1);
    mbar_init(tfull + 1, 1);
    mbar_init(tempty + 0, kEpiWarps3);
    mbar_init(tempty + 1, kEpiWarps3);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  auto give_up = [&]() {
    *abort_flag = 1;
    if (p.err_flag) atomicOr(p.err_flag, 2);
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer ----------------
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmBh)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmBm)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmBl)) : "memory");
      const uint32_t tx = kAStage3 + 3 * b_bytes;  // A raw + B_hi + B_mid + B_lo
      uint32_t armed = 0, last_par = 0;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t mt = group; ok && mt < p.m_tiles; mt += groups) {
        for (int kb = 0; kb < p.n_kb; ++kb) {
          if (!mbar_wait(empty + stage, phase ^ 1u, abort_flag)) {
            give_up();
            ok = false;
            break;
          }
          uint8_t* st = St + static_cast<size_t>(stage) * stage_bytes;
          mbar_expect_tx(full + stage, tx);
          tma_load_2d(st, &tmA, full + stage, kb * kBK3, static_cast<int>(mt * kBM));
          tma_load_2d(st + 3 * kAStage3, &tmBh, full + stage, kb * kBK3, n0);
          tma_load_2d(st + 3 * kAStage3 + b_bytes, &tmBm, full + stage, kb * kBK3, n0);
          tma_load_2d(st + 3 * kAStage3 + 2 * b_bytes, &tmBl, full + stage, kb * kBK3, n0);
          armed |= 1u << stage;
          last_par = (last_par & ~(1u << stage)) | (phase << stage);
          if (++stage == p.stages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        // let our own copies land before the CTA's shared memory goes away
        for (int s = 0; s < p.stages; ++s)
          if (armed & (1u << s)) {
            const uint32_t a = smem_u32(full + s);
            for (uint32_t it = 0; it < kSpinLimit && !mbar_try(a, (last_par >> s) & 1u); ++it) {
            }
          }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer ----------------
      int stage = 0;
      uint32_t phase = 0;
      uint32_t blk = 0;  // k blocks issued so far (all tiles)
      bool ok = true;
      for (int64_t mt = group; ok && mt < p.m_tiles; mt += groups) {
        for (int kb = 0; kb < p.n_kb; ++kb, ++blk) {
          const int b = static_cast<int>(blk & 1u);
          if (!mbar_wait(tempty + b, ((blk >> 1) & 1u) ^ 1u, abort_flag) ||
              !mbar_wait(conv + stage, phase, abort_flag)) {
            give_up();
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d_main = tmem_base + static_cast<uint32_t>(2 * b * p.acc_stride);
          const uint32_t d_corr = d_main + static_cast<uint32_t>(p.acc_stride);
          const uint32_t ah = smem_u32(St + static_cast<size_t>(stage) * stage_bytes);
          const uint32_t am = ah + kAStage3;
          const uint32_t al = ah + 2 * kAStage3;
          const uint32_t bh = ah + 3 * kAStage3;
          const uint32_t bm = bh + b_bytes;
          const uint32_t bl = bh + 2 * b_bytes;
#pragma unroll
          for (int k = 0; k < kBK3 / 8; ++k) {  // 8 TF32 elements = 32 bytes per MMA
            const uint32_t o = 32 * k;
            // fresh sums per k block: the small products, then hi.hi alone
            const uint32_t acc = k != 0 ? 1u : 0u;
            umma_tf32(d_corr, desc_kmajor_sw128(am + o), desc_kmajor_sw128(bm + o), p.idesc, acc);
            umma_tf32(d_corr, desc_kmajor_sw128(al + o), desc_kmajor_sw128(bh + o), p.idesc, 1u);
            umma_tf32(d_corr, desc_kmajor_sw128(ah + o), desc_kmajor_sw128(bl + o), p.idesc, 1u);
            umma_tf32(d_corr, desc_kmajor_sw128(am + o), desc_kmajor_sw128(bh + o), p.idesc, 1u);
            umma_tf32(d_corr, desc_kmajor_sw128(ah + o), desc_kmajor_sw128(bm + o), p.idesc, 1u);
            umma_tf32(d_main, desc_kmajor_sw128(ah + o), desc_kmajor_sw128(bh + o), p.idesc, acc);
          }
          umma_commit(empty + stage);
          umma_commit(tfull + b);
          if (++stage == p.stages) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
    }
  } else if (warp < 2 + kConvWarps) {
    // ---------------- converters ----------------
    const int ct = threadIdx.x - 64;  // 0 .. 32 * kConvWarps - 1
    int stage = 0;
    uint32_t phase = 0;
    bool ok = true;
    for (int64_t mt = group; ok && mt < p.m_tiles; mt += groups) {
      for (int kb = 0; kb < p.n_kb; ++kb) {
        if (!mbar_wait(full + stage, phase, abort_flag)) {
          if (lane == 0) give_up();
          ok = false;
          break;
        }
        float4* a = reinterpret_cast<float4*>(St + static_cast<size_t>(stage) * stage_bytes);
        float4* amid = a + kAStage3 / 16;
        float4* alo = a + 2 * (kAStage3 / 16);
#pragma unroll 4
        for (int i = ct; i < static_cast<int>(kAStage3 / 16); i += 32 * kConvWarps) {
          const float4 v = a[i];
          float4 h, m, l;
          split3(v.x, h.x, m.x, l.x);
          split3(v.y, h.y, m.y, l.y);
          split3(v.z, h.z, m.z, l.z);
          split3(v.w, h.w, m.w, l.w);
          a[i] = h;
          amid[i] = m;
          alo[i] = l;
        }
        // the MMAs read this stage through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(conv + stage);
        if (++stage == p.stages) {
          stage = 0;
          phase ^= 1u;
        }
      }
    }
  } else {
    // ---------------- accumulation and epilogue ----------------
    const int ew = warp - 2 - kConvWarps;
    const int quarter = warp & 3;                 // TMEM lanes this warp may read
    constexpr int parts = kEpiWarps3 / 4;         // column parts per lane quarter
    const int nch = p.BN / 16;
    const int ch0 = nch * (ew >> 2) / parts;      // this warp's 16-column chunks
    const int nmine = nch * ((ew >> 2) + 1) / parts - ch0;  // at most 4 (BN <= 128)
    uint8_t* stg = Stg + static_cast<size_t>(ew) * 2 * kStgBytes;
    int sb = 0;
    uint32_t blk = 0;
    bool ok = true;
    for (int64_t mt = group; ok && mt < p.m_tiles; mt += groups) {
      float acc[4][16];
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int i = 0; i < 16; ++i) acc[q][i] = 0.f;
      for (int kb = 0; kb < p.n_kb; ++kb, ++blk) {
        const int b = static_cast<int>(blk & 1u);
        if (!mbar_wait(tfull + b, (blk >> 1) & 1u, abort_flag)) {
          if (lane == 0) give_up();
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                               static_cast<uint32_t>(2 * b * p.acc_stride + 16 * ch0);
#pragma unroll
        for (int q = 0; q < 4; ++q) {  // main and correction sums of one chunk per wait
          if (q >= nmine) break;
          uint32_t rm[16], rc[16];
          tmem_ld16_issue(taddr + static_cast<uint32_t>(16 * q), rm);
          tmem_ld16_issue(taddr + static_cast<uint32_t>(p.acc_stride + 16 * q), rc);
          tmem_wait_ld();
#pragma unroll
          for (int i = 0; i < 16; ++i)
            acc[q][i] += __uint_as_float(rm[i]) + __uint_as_float(rc[i]);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty + b);
      }
      if (!ok) break;
      const int64_t row0 = mt * kBM + quarter * 32;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int c = 16 * (ch0 + q);
        if (q < nmine && n0 + c < p.Nc)  // ragged last n tile: nothing stored past Nc
          epilogue_chunk<EPI>(p, &tmO0, &tmO1, stg, sb, lane, row0, n0, c, acc[q]);
      }
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    __syncwarp();
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(p.tmem_cols)
                 : "memory");
  }
}

// ------------------------------------------------------- weight gradients
// C[M x Nc] = sum_k A[k, m] B[k, n] with A, B row-major over k (the node
// dimension): both operands are MN-major.  Shared-memory tiles hold 64 k-rows
// of 128 bytes (64 elements of m or n) per TMA box, 128-byte swizzle; 64-wide
// chunks along m / n are LBO = 8 KB apart and 8-row k groups SBO = 1 KB.
// Each CTA owns up to two 128-row m chunks (two TMEM accumulators sharing
// every B tile) times one n tile of width BN, over one contiguous slice of
// k; it writes its FP32 partial tile to part[split][m][n] and a separate
// kernel adds the slices in a fixed order.
constexpr int kWgK = 64;             // k rows per stage
constexpr int kBoxBytes = 64 * 128;  // one 64 x 64 BF16 box

__device__ __forceinline__ uint64_t desc_mnmajor_sw128(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr & 0x3FFFFu) >> 4);   // start address
  d |= static_cast<uint64_t>(kBoxBytes >> 4) << 16;       // leading offset: next 64-wide chunk
  d |= static_cast<uint64_t>(1024 >> 4) << 32;            // stride offset: next 8 k-rows
  d |= static_cast<uint64_t>(1) << 46;                    // descriptor version
  d |= static_cast<uint64_t>(2) << 61;                    // 128-byte swizzle
  return d;
}

struct WgParams {
  int M = 0, Nc = 0, BN = 0, mpc = 0, m_groups = 0, n_tiles = 0, splits = 0, stages = 0;
  int tmem_cols = 0, acc_stride = 0;
  int64_t k_blocks = 0;  // ceil(K / 64)
  uint32_t idesc = 0;
  float* part = nullptr;
  int* err_flag = nullptr;
};

__global__ void __launch_bounds__(kThreads, 1)
tc_wgrad_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const WgParams p) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t a_bytes = static_cast<uint32_t>(p.mpc) * 2 * kBoxBytes;  // 128 m per chunk
  const uint32_t b_bytes = static_cast<uint32_t>(p.BN / 64) * kBoxBytes;
  const uint32_t stage_bytes = a_bytes + b_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + static_cast<size_t>(p.stages) * stage_bytes);
  uint64_t* empty = full + p.stages;
  uint64_t* tfull = empty + p.stages;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tfull + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5;
  const int lane = threadIdx.x & 31;
  const int tile = blockIdx.x % (p.m_groups * p.n_tiles);
  const int split = blockIdx.x / (p.m_groups * p.n_tiles);
  const int mg = tile % p.m_groups;
  const int nt = tile / p.m_groups;
  const int m_base = mg * p.mpc * 128;
  const int n0 = nt * p.BN;
  const int64_t per = (p.k_blocks + p.splits - 1) / p.splits;
  const int64_t kb_begin = per * split;
  const int64_t kb_end = kb_begin + per < p.k_blocks ? kb_begin + per : p.k_blocks;
  const int64_t n_kb = kb_end > kb_begin ? kb_end - kb_begin : 0;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(full + s, 1);
      mbar_init(empty + s, 1);
    }
    mbar_init(tfull, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  auto give_up = [&]() {
    *abort_flag = 1;
    if (p.err_flag) atomicOr(p.err_flag, 2);
  };

  if (warp == 0) {
    if (lane == 0 && n_kb > 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
      // A boxes lying wholly past the last valid row m are not loaded: the
      // accumulator rows they would feed are never stored.
      int a_boxes = (p.M - m_base + 63) / 64;
      if (a_boxes > 2 * p.mpc) a_boxes = 2 * p.mpc;
      const uint32_t tx_bytes = static_cast<uint32_t>(a_boxes) * kBoxBytes + b_bytes;
      uint32_t armed = 0, last_par = 0;
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t kb = kb_begin; kb < kb_end; ++kb) {
        if (!mbar_wait(empty + stage, phase ^ 1u, abort_flag)) {
          give_up();
          ok = false;
          break;
        }
        uint8_t* st = smem + static_cast<size_t>(stage) * stage_bytes;
        mbar_expect_tx(full + stage, tx_bytes);
        const int krow = static_cast<int>(kb * kWgK);
        for (int j = 0; j < a_boxes; ++j)
          tma_load_2d(st + static_cast<size_t>(j) * kBoxBytes, &tmA, full + stage, m_base + 64 * j,
                      krow);
        for (int j = 0; j < p.BN / 64; ++j)
          tma_load_2d(st + a_bytes + static_cast<size_t>(j) * kBoxBytes, &tmB, full + stage,
                      n0 + 64 * j, krow);
        armed |= 1u << stage;
        last_par = (last_par & ~(1u << stage)) | (phase << stage);
        if (++stage == p.stages) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (!ok) {
        for (int s = 0; s < p.stages; ++s)
          if (armed & (1u << s)) {
            const uint32_t a = smem_u32(full + s);
            for (uint32_t it = 0; it < kSpinLimit && !mbar_try(a, (last_par >> s) & 1u); ++it) {
            }
          }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && n_kb > 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int64_t kb = 0; kb < n_kb; ++kb) {
        if (!mbar_wait(full + stage, phase, abort_flag)) {
          give_up();
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t s0 = smem_u32(smem + static_cast<size_t>(stage) * stage_bytes);
        const uint32_t b0 = s0 + a_bytes;
#pragma unroll
        for (int k = 0; k < kWgK / 16; ++k) {
          for (int mc = 0; mc < p.mpc; ++mc)
            umma_bf16(tmem_base + static_cast<uint32_t>(mc * p.acc_stride),
                      desc_mnmajor_sw128(s0 + mc * 2 * kBoxBytes + k * 2048),
                      desc_mnmajor_sw128(b0 + k * 2048), p.idesc, (kb | k) != 0 ? 1u : 0u);
        }
        umma_commit(empty + stage);
        if (++stage == p.stages) {
          stage = 0;
          phase ^= 1u;
        }
      }
      if (ok) umma_commit(tfull);
    }
  } else {
    const int ew = warp - 2;
    const int quarter = warp & 3;
    constexpr int parts = kEpiWarps / 4;
    const int cq = ew >> 2;
    const int nch = p.BN / 16;
    const int c_begin = 16 * (nch * cq / parts);
    const int c_end = 16 * (nch * (cq + 1) / parts);
    bool ok = true;
    if (n_kb > 0) {
      ok = mbar_wait(tfull, 0, abort_flag);
      if (!ok && lane == 0) give_up();
      tc_fence_after();
    }
    float* out = p.part + static_cast<int64_t>(split) * p.M * p.Nc;
    for (int mc = 0; ok && mc < p.mpc; ++mc) {
      const int m = m_base + mc * 128 + quarter * 32 + lane;
      const uint32_t taddr = tmem_base + (static_cast<uint32_t>(quarter * 32) << 16) +
                             static_cast<uint32_t>(mc * p.acc_stride);
      for (int c = c_begin; c < c_end; c += 16) {
        float v[16];
        if (n_kb > 0) {
          tmem_ld16(taddr + static_cast<uint32_t>(c), v);
        } else {
#pragma unroll
          for (int j = 0; j < 16; ++j) v[j] = 0.f;
        }
        if (m < p.M && n0 + c < p.Nc) storeN<16>(out + static_cast<int64_t>(m) * p.Nc + n0 + c, v);
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(p.tmem_cols)
                 : "memory");
  }
}

// ------------------------------------------------------------------- host
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_once;
bool g_ok = false;
bool g_tf32_ok = false;
int g_max_smem = 0;

void init_driver() {
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                       &q) != cudaSuccess ||
      q != cudaDriverEntryPointSuccess || fn == nullptr) {
    cudaGetLastError();
    return;
  }
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  cudaDeviceGetAttribute(&g_max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (major != 10 || minor != 3) return;  // this build carries sm_103a code only
  if (cudaFuncSetAttribute(tc_gemm_nt_kernel<EPI_BIAS_RELU>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, g_max_smem) != cudaSuccess ||
      cudaFuncSetAttribute(tc_gemm_nt_kernel<EPI_BIAS_SIGMOID>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, g_max_smem) != cudaSuccess ||
      cudaFuncSetAttribute(tc_gemm_nt_kernel<EPI_SPLIT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, g_max_smem) != cudaSuccess ||
      cudaFuncSetAttribute(tc_gemm_nt_kernel<EPI_RELU_BITS>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, g_max_smem) != cudaSuccess ||
      cudaFuncSetAttribute(tc_gemm_nt_kernel<EPI_BIAS>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, g_max_smem) != cudaSuccess ||
      cudaFuncSetAttribute(tc_wgrad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           g_max_smem) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  // the split-TF32 kernels of the FP32 form (optional: without them that
  // form stays on CUDA cores)
  g_tf32_ok =
      cudaFuncSetAttribute(tc3_gemm_nt_kernel<EPI_BIAS_RELU>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, g_max_smem) == cudaSuccess &&
      cudaFuncSetAttribute(tc3_gemm_nt_kernel<EPI_BIAS_SIGMOID>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, g_max_smem) == cudaSuccess &&
      cudaFuncSetAttribute(tc3_gemm_nt_kernel<EPI_SPLIT>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, g_max_smem) == cudaSuccess &&
      cudaFuncSetAttribute(tc3_gemm_nt_kernel<EPI_RELU_BITS>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, g_max_smem) == cudaSuccess &&
      cudaFuncSetAttribute(tc3_gemm_nt_kernel<EPI_BIAS>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, g_max_smem) == cudaSuccess;
  if (!g_tf32_ok) cudaGetLastError();
  g_ok = true;
}

// 2-D BF16 tensor map over a row-major matrix: inner extent `cols`
// elements, `rows` rows, row pitch `ld` elements; box kBK x box_rows.
bool make_map(CUtensorMap* m, const void* base, int64_t cols, int64_t rows, int64_t ld,
              int box_rows) {
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 2};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kBK), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// 2-D FP32 tensor map over a row-major matrix: inner extent `cols`
// elements, `rows` rows, row pitch `ld` elements; box kBK3 x box_rows
// (128 bytes of K per row, 128-byte swizzle).
bool make_map_f32(CUtensorMap* m, const void* base, int64_t cols, int64_t rows, int64_t ld,
                  int box_rows) {
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 4};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(kBK3), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Output tensor map: `cols` valid columns of dtype dt, `rows` rows, row pitch
// `ld` elements; box of 16 columns x 32 rows, no swizzle (epilogue staging).
bool make_out_map(CUtensorMap* m, const void* base, int dt, int64_t cols, int64_t rows,
                  int64_t ld) {
  const int esz = dt == DT_BF16 ? 2 : 4;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * esz};
  cuuint32_t box[2] = {16, 32};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(m, dt == DT_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                        2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE,
                        esz == 4 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B,
                        CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Shared memory a CTA needs with BN output columns (weights resident) and
// `stages` A stages (two at least).
size_t tc_smem_need(int bn, int64_t K, int stages = 2) {
  const int n_kb = static_cast<int>((K + kBK - 1) / kBK);
  return 1024 + static_cast<size_t>(n_kb) * bn * kBK * 2 + kStgTotal +
         static_cast<size_t>(stages) * kStageBytes + 256;
}

// Shared memory with BN columns when the weights stream with the A stages
// (two stages at least).
size_t tc_stream_smem_need(int bn, int stages = 2) {
  return 1024 + kStgTotal +
         static_cast<size_t>(stages) * (static_cast<size_t>(kStageBytes) + static_cast<size_t>(bn) * kBK * 2) +
         256;
}

struct NPlan {
  int bn = 0;
  bool stream = false;
};

// n tile of a product with Nc (a multiple of 16) output columns: the widest
// multiple of 16 up to min(Nc, 256) whose weight slice stays resident, as
// long as that keeps the tile at least min(Nc, 128) wide (narrower tiles
// waste the tensor pipe); otherwise streamed weights.  The last tile may be
// ragged.  With streamed weights and M, num_sms known, the tile width (from
// 128 to 256) minimises the persistent schedule's critical path: each n tile
// gets floor(num_sms / n_tiles) CTAs, which take its m tiles in turn, so the
// slowest CTA runs ceil(m_tiles / groups) tiles of cost ~ bn (a product with
// few m tiles, like the 2500-row DBM layers, otherwise leaves SMs idle for a
// whole tile).  bn = 0: no plan fits.
NPlan plan_n(int Nc, int64_t K, int64_t M = 0, int num_sms = 0, bool deep = false) {
  NPlan pl;
  const int cap = Nc < 256 ? Nc : 256;
  const int want = cap < 128 ? cap : 128;
  // A full-width tile whose resident weights leave only two A stages streams
  // its weights with the stages instead (from L2), which keeps three: each A
  // tile is read once, with a deeper pipeline.  At N = 10^6, K = 256, 256
  // outputs: the split input gradient 0.204 -> 0.164 ms, the sigmoid head
  // 0.258 -> 0.254 ms (against its two resident 128-wide tiles).
  if (cap == 256 && tc_smem_need(cap, K, 3) > static_cast<size_t>(g_max_smem) &&
      tc_smem_need(cap, K, 2) <= static_cast<size_t>(g_max_smem) &&
      tc_stream_smem_need(cap, 3) <= static_cast<size_t>(g_max_smem)) {
    pl.bn = cap;
    pl.stream = true;
    return pl;
  }
  // deep: resident weights with a pipeline at least four A stages deep, on
  // equal n tiles (for the sigmoid head, whose FP32 output favoured two
  // 128-wide tiles sharing each A tile through L2 over one 256-wide tile with
  // two resident stages: 0.283 -> 0.258 ms before the streamed case above).
  if (deep)
    for (int bn = cap; bn >= want; bn -= 16)
      if (Nc % bn == 0 && tc_smem_need(bn, K, 4) <= static_cast<size_t>(g_max_smem)) {
        pl.bn = bn;
        return pl;
      }
  for (int bn = cap; bn >= want; bn -= 16)
    if (tc_smem_need(bn, K) <= static_cast<size_t>(g_max_smem)) {
      pl.bn = bn;
      return pl;
    }
  for (int bn = cap; bn >= 16; bn -= 16)
    if (tc_stream_smem_need(bn) <= static_cast<size_t>(g_max_smem)) {
      pl.bn = bn;
      pl.stream = true;
      break;
    }
  if (pl.bn == 0 || M <= 0 || num_sms <= 0) return pl;
  const int64_t m_tiles = (M + kBM - 1) / kBM;
  int64_t best = -1;
  for (int bn = pl.bn; bn >= want; bn -= 16) {
    const int64_t n_tiles = (Nc + bn - 1) / bn;
    const int64_t groups = n_tiles >= num_sms ? 1 : num_sms / n_tiles;
    const int64_t rounds = n_tiles > num_sms ? (n_tiles + num_sms - 1) / num_sms : 1;
    const int64_t cost = rounds * ((m_tiles + groups - 1) / groups) * bn;
    if (best < 0 || cost < best) {
      best = cost;
      pl.bn = bn;
    }
  }
  return pl;
}

}  // namespace

bool tc_available() { return true; }

bool tc_prepare(int, std::string* msg) {
  std::call_once(g_once, init_driver);
  if (!g_ok && msg) *msg = "tensor-core path unavailable (driver entry point or device)";
  return g_ok;
}

bool tc_gemm_supported(const GemmArgs& g) {
  if (!g_ok) return false;
  if (g.da != DT_BF16 || g.db != DT_BF16 || !g.a_kmajor || !g.b_kmajor) return false;
  if (g.epi != EPI_BIAS_RELU && g.epi != EPI_BIAS_SIGMOID && g.epi != EPI_SPLIT &&
      g.epi != EPI_RELU_BITS && g.epi != EPI_BIAS)
    return false;
  if (g.K < kBK || g.K % 8 || g.lda % 8 || g.ldb % 8) return false;
  if (g.Nc % 16 || plan_n(g.Nc, g.K).bn == 0) return false;
  if (g.epi == EPI_SPLIT && g.split % 16) return false;
  if ((g.epi != EPI_RELU_BITS && g.ld0 % 8) || (g.epi == EPI_SPLIT && g.ld1 % 8)) return false;
  return true;
}

int tc_gemm_launch(const GemmArgs& g, int num_sms, cudaStream_t st) {
  TcParams p;
  p.M = g.M;
  p.Nc = g.Nc;
  p.K = static_cast<int>(g.K);
  const NPlan pl = plan_n(g.Nc, g.K, g.M, num_sms, g.epi == EPI_BIAS_SIGMOID);
  p.BN = pl.bn;
  p.stream_b = pl.stream ? 1 : 0;
  p.n_tiles_n = (g.Nc + p.BN - 1) / p.BN;
  p.n_kb = (p.K + kBK - 1) / kBK;
  p.m_tiles = (g.M + kBM - 1) / kBM;
  const size_t b_kb = static_cast<size_t>(p.BN) * kBK * 2;
  const size_t b_bytes = pl.stream ? 0 : static_cast<size_t>(p.n_kb) * b_kb;
  const size_t stage_bytes = kStageBytes + (pl.stream ? b_kb : 0);
  const size_t fixed = 1024 + b_bytes + kStgTotal + 256;
  int stages = static_cast<int>((static_cast<size_t>(g_max_smem) - fixed) / stage_bytes);
  stages = stages > 6 ? 6 : stages;
  p.stages = stages;
  size_t smem = fixed + static_cast<size_t>(stages) * stage_bytes;
  // at least 120 KB so that only one CTA (and one TMEM allocation) fits per SM
  if (smem < 120 * 1024) smem = 120 * 1024;
  p.acc_stride = (p.BN + 31) / 32 * 32;
  int cols = 32;
  while (cols < 2 * p.acc_stride) cols <<= 1;
  p.tmem_cols = cols;
  p.idesc = (1u << 4) | (1u << 7) | (1u << 10) | (static_cast<uint32_t>(p.BN >> 3) << 17) |
            (static_cast<uint32_t>(kBM >> 4) << 24);
  p.epi = g.epi;
  p.bias = g.bias;
  p.out0 = g.out0;
  p.ld0 = g.ld0;
  p.d0 = g.d0;
  p.out1 = g.out1;
  p.ld1 = g.ld1;
  p.d1 = g.d1;
  p.split = g.split;
  p.row_scale = g.row_scale;
  p.addend = g.addend;
  p.ld_add = g.ld_add;
  p.d_add = g.d_add;
  p.n_valid = g.n_valid > 0 ? g.n_valid : g.Nc;
  p.err_flag = g.err_flag;
  CUtensorMap ta, tb, to0, to1;
  const int64_t cols0 = g.epi == EPI_SPLIT ? g.split : g.Nc;
  bool ok = make_map(&ta, g.A, g.K, g.M, g.lda, kBM) && make_map(&tb, g.B, g.K, g.Nc, g.ldb, p.BN);
  if (ok) {
    if (g.epi == EPI_RELU_BITS) to0 = tb;  // bits are stored directly; map unused
    else ok = make_out_map(&to0, g.out0, g.d0, cols0, g.M, g.ld0);
  }
  if (ok) {
    if (g.epi == EPI_SPLIT) ok = make_out_map(&to1, g.out1, g.d1, g.Nc - g.split, g.M, g.ld1);
    else to1 = to0;
  }
  if (!ok) {
    gemm_simt_launch(g, st);  // descriptor rejected: same product on CUDA cores
    return 1;
  }
  int groups = num_sms / p.n_tiles_n;
  if (groups < 1) groups = 1;
  const int64_t max_groups = p.m_tiles;
  if (groups > max_groups) groups = static_cast<int>(max_groups);
  const int grid = groups * p.n_tiles_n;
  switch (g.epi) {
    case EPI_BIAS_RELU:
      tc_gemm_nt_kernel<EPI_BIAS_RELU><<<grid, kThreads, smem, st>>>(ta, tb, to0, to1, p);
      break;
    case EPI_BIAS_SIGMOID:
      tc_gemm_nt_kernel<EPI_BIAS_SIGMOID><<<grid, kThreads, smem, st>>>(ta, tb, to0, to1, p);
      break;
    case EPI_RELU_BITS:
      tc_gemm_nt_kernel<EPI_RELU_BITS><<<grid, kThreads, smem, st>>>(ta, tb, to0, to1, p);
      break;
    case EPI_BIAS:
      tc_gemm_nt_kernel<EPI_BIAS><<<grid, kThreads, smem, st>>>(ta, tb, to0, to1, p);
      break;
    default:
      tc_gemm_nt_kernel<EPI_SPLIT><<<grid, kThreads, smem, st>>>(ta, tb, to0, to1, p);
      break;
  }
  return 1;
}

bool tc3_gemm_supported(const GemmArgs& g) {
  if (!g_ok || !g_tf32_ok) return false;
  if (g.da != DT_F32 || g.db != DT_F32 || !g.a_kmajor || !g.b_kmajor || !g.B_mid || !g.B_lo)
    return false;
  if (g.epi != EPI_BIAS_RELU && g.epi != EPI_BIAS_SIGMOID && g.epi != EPI_SPLIT &&
      g.epi != EPI_RELU_BITS && g.epi != EPI_BIAS)
    return false;
  if (g.K < kBK3 || g.K % 4 || g.lda % 4 || g.ldb % 4 || g.Nc % 16) return false;
  if (g.epi == EPI_SPLIT && g.split % 16) return false;
  if ((g.epi != EPI_RELU_BITS && g.ld0 % 4) || (g.epi == EPI_SPLIT && g.ld1 % 4)) return false;
  // tensor maps need 16-byte aligned bases
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; };
  if (!al16(g.A) || !al16(g.B) || !al16(g.B_mid) || !al16(g.B_lo) ||
      (g.epi != EPI_RELU_BITS && !al16(g.out0)) ||
      (g.epi == EPI_SPLIT && !al16(g.out1)))
    return false;
  // at least two pipeline stages
  const int bn = g.Nc < kBN3 ? g.Nc : kBN3;
  const size_t stage_bytes = 3 * static_cast<size_t>(kAStage3) + 3 * static_cast<size_t>(bn) * kBK3 * 4;
  return static_cast<size_t>(g_max_smem) >= 1024 + kStgTotal3 + 256 + 2 * stage_bytes;
}

int tc3_gemm_launch(const GemmArgs& g, int num_sms, cudaStream_t st) {
  TcParams p;
  p.M = g.M;
  p.Nc = g.Nc;
  p.K = static_cast<int>(g.K);
  p.BN = g.Nc < kBN3 ? g.Nc : kBN3;
  p.stream_b = 1;
  p.n_tiles_n = (g.Nc + p.BN - 1) / p.BN;
  p.n_kb = (p.K + kBK3 - 1) / kBK3;
  p.m_tiles = (g.M + kBM - 1) / kBM;
  const size_t stage_bytes = 3 * static_cast<size_t>(kAStage3) + 3 * static_cast<size_t>(p.BN) * kBK3 * 4;
  const size_t fixed = 1024 + kStgTotal3 + 256;
  int stages = static_cast<int>((static_cast<size_t>(g_max_smem) - fixed) / stage_bytes);
  stages = stages > 4 ? 4 : stages;
  if (stages < 2) {  // excluded by tc3_gemm_supported
    flag_error_launch(g.err_flag, 4, st);
    return 1;
  }
  p.stages = stages;
  size_t smem = fixed + static_cast<size_t>(stages) * stage_bytes;
  if (smem < 120 * 1024) smem = 120 * 1024;  // one CTA (one TMEM allocation) per SM
  p.acc_stride = (p.BN + 31) / 32 * 32;
  int cols = 32;
  while (cols < 4 * p.acc_stride) cols <<= 1;  // two (main, correction) pairs
  p.tmem_cols = cols;
  // D FP32, A and B TF32, both K-major, N = BN, M = 128
  p.idesc = (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(p.BN >> 3) << 17) |
            (static_cast<uint32_t>(kBM >> 4) << 24);
  p.epi = g.epi;
  p.bias = g.bias;
  p.out0 = g.out0;
  p.ld0 = g.ld0;
  p.d0 = g.d0;
  p.out1 = g.out1;
  p.ld1 = g.ld1;
  p.d1 = g.d1;
  p.split = g.split;
  p.row_scale = g.row_scale;
  p.addend = g.addend;
  p.ld_add = g.ld_add;
  p.d_add = g.d_add;
  p.n_valid = g.n_valid > 0 ? g.n_valid : g.Nc;
  p.err_flag = g.err_flag;
  CUtensorMap ta, tbh, tbm, tbl, to0, to1;
  const int64_t cols0 = g.epi == EPI_SPLIT ? g.split : g.Nc;
  bool ok = make_map_f32(&ta, g.A, g.K, g.M, g.lda, kBM) &&
            make_map_f32(&tbh, g.B, g.K, g.Nc, g.ldb, p.BN) &&
            make_map_f32(&tbm, g.B_mid, g.K, g.Nc, g.ldb, p.BN) &&
            make_map_f32(&tbl, g.B_lo, g.K, g.Nc, g.ldb, p.BN);
  if (ok) {
    if (g.epi == EPI_RELU_BITS) to0 = tbh;  // bits are stored directly; map unused
    else ok = make_out_map(&to0, g.out0, g.d0, cols0, g.M, g.ld0);
  }
  if (ok) {
    if (g.epi == EPI_SPLIT) ok = make_out_map(&to1, g.out1, g.d1, g.Nc - g.split, g.M, g.ld1);
    else to1 = to0;
  }
  if (!ok) {
    // a rejected descriptor: B holds only the hi part here, so no CUDA-core
    // product could stand in; the step reports the failure
    flag_error_launch(g.err_flag, 4, st);
    return 1;
  }
  int groups = num_sms / p.n_tiles_n;
  if (groups < 1) groups = 1;
  if (groups > p.m_tiles) groups = static_cast<int>(p.m_tiles);
  const int grid = groups * p.n_tiles_n;
  switch (g.epi) {
    case EPI_BIAS_RELU:
      tc3_gemm_nt_kernel<EPI_BIAS_RELU><<<grid, kThreads3, smem, st>>>(ta, tbh, tbm, tbl, to0, to1, p);
      break;
    case EPI_BIAS_SIGMOID:
      tc3_gemm_nt_kernel<EPI_BIAS_SIGMOID><<<grid, kThreads3, smem, st>>>(ta, tbh, tbm, tbl, to0, to1, p);
      break;
    case EPI_RELU_BITS:
      tc3_gemm_nt_kernel<EPI_RELU_BITS><<<grid, kThreads3, smem, st>>>(ta, tbh, tbm, tbl, to0, to1, p);
      break;
    case EPI_BIAS:
      tc3_gemm_nt_kernel<EPI_BIAS><<<grid, kThreads3, smem, st>>>(ta, tbh, tbm, tbl, to0, to1, p);
      break;
    default:
      tc3_gemm_nt_kernel<EPI_SPLIT><<<grid, kThreads3, smem, st>>>(ta, tbh, tbm, tbl, to0, to1, p);
      break;
  }
  return 1;
}

namespace {

struct WgShape {
  int BN, n_tiles, mpc, m_groups, stages;
  uint32_t stage_bytes;
};

bool wg_shape(const GemmArgs& g, WgShape* s) {
  const int nc64 = (g.Nc + 63) / 64 * 64;
  s->BN = nc64 < 256 ? nc64 : 256;
  s->n_tiles = (g.Nc + s->BN - 1) / s->BN;
  const int m_chunks = static_cast<int>((g.M + 127) / 128);
  s->mpc = m_chunks < 2 ? m_chunks : 2;
  s->m_groups = (m_chunks + s->mpc - 1) / s->mpc;
  s->stage_bytes = static_cast<uint32_t>(s->mpc) * 2 * kBoxBytes +
                   static_cast<uint32_t>(s->BN / 64) * kBoxBytes;
  const size_t fixed = 1024 + 256;
  int st = static_cast<int>((static_cast<size_t>(g_max_smem) - fixed) / s->stage_bytes);
  s->stages = st > 8 ? 8 : st;
  return s->stages >= 2;
}

}  // namespace

bool tc_wgrad_supported(const GemmArgs& g) {
  if (!g_ok) return false;
  if (g.da != DT_BF16 || g.db != DT_BF16 || g.a_kmajor || g.b_kmajor) return false;
  if (g.epi != EPI_PARTIAL || g.lda % 8 || g.ldb % 8 || g.Nc % 16) return false;
  if (g.K < kWgK || g.M < 1) return false;
  WgShape s;
  return wg_shape(g, &s);
}

int tc_wgrad_launch(const GemmArgs& g, int num_sms, size_t part_floats, float* dst, int64_t ldo,
                    cudaStream_t st) {
  WgShape s;
  wg_shape(g, &s);
  WgParams p;
  p.M = static_cast<int>(g.M);
  p.Nc = g.Nc;
  p.BN = s.BN;
  p.mpc = s.mpc;
  p.m_groups = s.m_groups;
  p.n_tiles = s.n_tiles;
  p.stages = s.stages;
  p.acc_stride = s.BN;
  int cols = 32;
  while (cols < s.mpc * s.BN) cols <<= 1;
  p.tmem_cols = cols;
  p.k_blocks = (g.K + kWgK - 1) / kWgK;
  const int tiles = s.m_groups * s.n_tiles;
  int64_t splits = num_sms / tiles;
  if (splits < 1) splits = 1;
  if (splits > p.k_blocks) splits = p.k_blocks;
  const int64_t cap = static_cast<int64_t>(part_floats / (static_cast<size_t>(p.M) * p.Nc));
  if (splits > cap) splits = cap < 1 ? 1 : cap;
  p.splits = static_cast<int>(splits);
  p.idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
            (static_cast<uint32_t>(s.BN >> 3) << 17) | (static_cast<uint32_t>(128 >> 4) << 24);
  p.part = static_cast<float*>(g.out0);
  p.err_flag = g.err_flag;
  CUtensorMap ta, tb;
  if (!make_map(&ta, g.A, g.M, g.K, g.lda, kWgK) || !make_map(&tb, g.B, g.Nc, g.K, g.ldb, kWgK)) {
    gemm_simt_launch(g, st);
    splitk_reduce(static_cast<float*>(g.out0), g.splits, p.M, p.Nc, p.Nc, dst, ldo, st);
    return 2;
  }
  size_t smem = 1024 + static_cast<size_t>(s.stages) * s.stage_bytes + 256;
  if (smem < 120 * 1024) smem = 120 * 1024;
  const int grid = tiles * p.splits;
  // one split into a destination with row stride Nc: no partials to add
  // (the kernel's epilogue stores 16-byte vectors, so dst must be 16-byte aligned)
  const bool direct = p.splits == 1 && ldo == p.Nc && reinterpret_cast<uintptr_t>(dst) % 16 == 0;
  if (direct) p.part = dst;
  tc_wgrad_kernel<<<grid, kThreads, smem, st>>>(ta, tb, p);
  if (direct) return 1;
  splitk_reduce(p.part, p.splits, p.M, p.Nc, p.Nc, dst, ldo, st);
  return 2;
}

}  // namespace cpra
