// Device-side helpers shared by the CPRA kernels (sm_103a).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace cpra {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(bf16 x) { return __bfloat162float(x); }

template <typename T> __device__ __forceinline__ T from_f(float x);
template <> __device__ __forceinline__ float from_f<float>(float x) { return x; }
template <> __device__ __forceinline__ bf16 from_f<bf16>(float x) { return __float2bfloat16_rn(x); }

// x rounded to TF32 (10 mantissa bits, round to nearest, ties away from
// zero), as an FP32 value whose low 13 mantissa bits are zero.
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// x = hi + mid + lo exactly, each part a TF32 value: hi = tf32(x),
// mid = tf32(x - hi), lo = x - hi - mid (both differences are exact in FP32;
// lo has at most 2 significant bits left, so it is a TF32 value too).
__device__ __forceinline__ void split3(float x, float& hi, float& mid, float& lo) {
  hi = tf32_rna(x);
  const float r = x - hi;
  mid = tf32_rna(r);
  lo = tf32_rna(r - mid);
}

// Number of T elements in one 16-byte vector.
template <typename T> struct V16 { static constexpr int n = 16 / (int)sizeof(T); };

// Load one 16-byte vector of T (16-byte aligned) and widen to float.
__device__ __forceinline__ void load16(const float* p, float* out) {
  float4 v = *reinterpret_cast<const float4*>(p);
  out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
}
__device__ __forceinline__ void load16(const bf16* p, float* out) {
  uint4 v = *reinterpret_cast<const uint4*>(p);
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[k]);
    float2 f = __bfloat1622float2(h);
    out[2 * k] = f.x;
    out[2 * k + 1] = f.y;
  }
}
// Read-only, no-L1-allocate variants for gathered rows.
__device__ __forceinline__ uint4 ldg_nc16(const void* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
  return v;
}
__device__ __forceinline__ void widen(const uint4& v, float* out, const float*) {
  out[0] = __uint_as_float(v.x); out[1] = __uint_as_float(v.y);
  out[2] = __uint_as_float(v.z); out[3] = __uint_as_float(v.w);
}
__device__ __forceinline__ void widen(const uint4& v, float* out, const bf16*) {
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    __nv_bfloat162 h = *reinterpret_cast<const __nv_bfloat162*>(&w[k]);
    float2 f = __bfloat1622float2(h);
    out[2 * k] = f.x;
    out[2 * k + 1] = f.y;
  }
}

// Store N floats (N*sizeof(T) a multiple of 8 bytes, aligned) as T.
template <int N>
__device__ __forceinline__ void storeN(float* p, const float* v) {
#pragma unroll
  for (int k = 0; k < N; k += 4)
    *reinterpret_cast<float4*>(p + k) = make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
}
template <int N>
__device__ __forceinline__ void storeN(bf16* p, const float* v) {
  if constexpr (N % 8 == 0) {
#pragma unroll
    for (int k = 0; k < N; k += 8) {
      uint4 u;
      __nv_bfloat162 h0 = __floats2bfloat162_rn(v[k + 0], v[k + 1]);
      __nv_bfloat162 h1 = __floats2bfloat162_rn(v[k + 2], v[k + 3]);
      __nv_bfloat162 h2 = __floats2bfloat162_rn(v[k + 4], v[k + 5]);
      __nv_bfloat162 h3 = __floats2bfloat162_rn(v[k + 6], v[k + 7]);
      u.x = *reinterpret_cast<uint32_t*>(&h0);
      u.y = *reinterpret_cast<uint32_t*>(&h1);
      u.z = *reinterpret_cast<uint32_t*>(&h2);
      u.w = *reinterpret_cast<uint32_t*>(&h3);
      *reinterpret_cast<uint4*>(p + k) = u;
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; k += 4) {
      uint2 u;
      __nv_bfloat162 h0 = __floats2bfloat162_rn(v[k + 0], v[k + 1]);
      __nv_bfloat162 h1 = __floats2bfloat162_rn(v[k + 2], v[k + 3]);
      u.x = *reinterpret_cast<uint32_t*>(&h0);
      u.y = *reinterpret_cast<uint32_t*>(&h1);
      *reinterpret_cast<uint2*>(p + k) = u;
    }
  }
}

// L2 eviction hints for data touched once (streamed outputs and row reads):
// marking them evict-first keeps the gathered operand resident in L2 longer.
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// Coherent 16-byte load (the data may be rewritten later by the same kernel).
__device__ __forceinline__ uint4 ld_stream16(const void* p, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_stream16(void* p, const uint4& v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1,%2,%3,%4}, %5;" ::"l"(p), "r"(v.x),
               "r"(v.y), "r"(v.z), "r"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st_stream8(void* p, const uint2& v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1,%2}, %3;" ::"l"(p), "r"(v.x), "r"(v.y),
               "l"(pol)
               : "memory");
}
// storeN for N a multiple of 4, with the L2 hint.
template <int N>
__device__ __forceinline__ void storeN_stream(float* p, const float* v, uint64_t pol) {
#pragma unroll
  for (int k = 0; k < N; k += 4)
    st_stream16(p + k, make_uint4(__float_as_uint(v[k]), __float_as_uint(v[k + 1]),
                                  __float_as_uint(v[k + 2]), __float_as_uint(v[k + 3])),
                pol);
}
template <int N>
__device__ __forceinline__ void storeN_stream(bf16* p, const float* v, uint64_t pol) {
  static_assert(N % 4 == 0, "bf16 streamed stores move 4 or 8 elements");
  if constexpr (N % 8 == 0) {
#pragma unroll
    for (int k = 0; k < N; k += 8) {
      uint32_t w[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        __nv_bfloat162 h = __floats2bfloat162_rn(v[k + 2 * q], v[k + 2 * q + 1]);
        w[q] = *reinterpret_cast<uint32_t*>(&h);
      }
      st_stream16(p + k, make_uint4(w[0], w[1], w[2], w[3]), pol);
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; k += 4) {
      __nv_bfloat162 h0 = __floats2bfloat162_rn(v[k], v[k + 1]);
      __nv_bfloat162 h1 = __floats2bfloat162_rn(v[k + 2], v[k + 3]);
      st_stream8(p + k,
                 make_uint2(*reinterpret_cast<uint32_t*>(&h0), *reinterpret_cast<uint32_t*>(&h1)),
                 pol);
    }
  }
}

// One Adam step (Kingma & Ba) on one parameter with optional decoupled
// weight decay (AdamW), the optimiser of the Experiments section; the bias
// corrections bc1 = 1 - beta1^t and bc2 = 1 - beta2^t come from the host.
// Shared by the parameter update and the fused embedding update so that both
// round identically.
__device__ __forceinline__ float adam_update(float th, float& m, float& v, float g, float lr,
                                             float b1, float b2, float eps, float wd, float bc1,
                                             float bc2) {
  if (wd != 0.f) th = th * (1.f - lr * wd);
  m = b1 * m + (1.f - b1) * g;
  v = b2 * v + (1.f - b2) * g * g;
  const float mhat = m / bc1;
  const float vhat = v / bc2;
  return th - lr * mhat / (sqrtf(vhat) + eps);
}

// SplitMix64 (Steele, Lea & Flood 2014) as a counter-based generator.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}
// Uniform [0, 1) with 24 random bits from stream (seed, tag) at index idx.
__device__ __forceinline__ float u24(uint64_t seed, uint64_t tag, uint64_t idx) {
  const uint64_t h = splitmix64(seed ^ splitmix64(tag) ^ (idx * 0xD1B54A32D192ED03ull));
  return (float)(h >> 40) * (1.0f / 16777216.0f);  // [0, 1)
}

// A standard normal from two uniforms of the same stream (Box-Muller).
__device__ __forceinline__ float normal_at(uint64_t seed, uint64_t tag, uint64_t i) {
  const float u1 = u24(seed, tag, 2 * i) + (0.5f / 16777216.0f);
  const float u2 = u24(seed, tag, 2 * i + 1);
  return sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

// Sum over the lanes of an aligned power-of-two segment of width W.
template <int W>
__device__ __forceinline__ float seg_sum(float v, unsigned mask) {
#pragma unroll
  for (int off = W / 2; off > 0; off >>= 1) v += __shfl_xor_sync(mask, v, off);
  return v;
}
template <int W>
__device__ __forceinline__ float seg_max(float v, unsigned mask) {
#pragma unroll
  for (int off = W / 2; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(mask, v, off));
  return v;
}
template <int W>
__device__ __forceinline__ float seg_min(float v, unsigned mask) {
#pragma unroll
  for (int off = W / 2; off > 0; off >>= 1) v = fminf(v, __shfl_xor_sync(mask, v, off));
  return v;
}
template <int W>
__device__ __forceinline__ uint32_t seg_or(uint32_t v, unsigned mask) {
#pragma unroll
  for (int off = W / 2; off > 0; off >>= 1) v |= __shfl_xor_sync(mask, v, off);
  return v;
}

template <int LPR>
__device__ __forceinline__ unsigned segment_mask(int lane) {
  if constexpr (LPR == 32) {
    return 0xffffffffu;
  } else {
    return ((1u << LPR) - 1u) << ((lane / LPR) * LPR);
  }
}

// ------------------------------------------------------------------ CSR reads
// Every kernel that walks the graph reads its CSR through csr_row and
// csr_col.  The normal build loads what it is given (cpra_init_graph checks
// the graph on the host; the op-level calls document their contract).  The
// checked build (CPRA_CHECKED) tests each row range against
// 0 <= rowptr[i] <= rowptr[i+1] <= rowptr[N] and each column index against
// 0 <= col[e] < N before it is used: a failing row is read as empty and a
// failing index as node 0, so no access leaves the arrays, and the failure is
// counted in this translation unit's device words, which the host reads and
// clears through the translation unit's collector (CPRA_CSR_CHECK_COLLECT).
#ifdef CPRA_CHECKED
namespace {
__device__ unsigned long long g_csr_fail_count = 0;
__device__ long long g_csr_fail_row = 0x7fffffffffffffffLL;    // smallest bad row range
__device__ long long g_csr_fail_entry = 0x7fffffffffffffffLL;  // smallest bad column position
}  // namespace
#endif

__device__ __forceinline__ void csr_row(const int* rowptr, int64_t i, int64_t N, int& beg,
                                        int& end) {
  beg = rowptr[i];
  end = rowptr[i + 1];
#ifdef CPRA_CHECKED
  const int nnz = rowptr[N];
  if (!(0 <= beg && beg <= end && end <= nnz)) {
    atomicAdd(&g_csr_fail_count, 1ull);
    atomicMin(&g_csr_fail_row, (long long)i);
    beg = end = 0;
  }
#else
  (void)N;
#endif
}

__device__ __forceinline__ int csr_col(const int* col, int64_t e, int64_t N) {
  const int j = col[e];
#ifdef CPRA_CHECKED
  if (j < 0 || (int64_t)j >= N) {
    atomicAdd(&g_csr_fail_count, 1ull);
    atomicMin(&g_csr_fail_entry, (long long)e);
    return 0;
  }
#else
  (void)N;
#endif
  return j;
}

}  // namespace cpra

#ifdef CPRA_CHECKED
// Body of a translation unit's collector: adds its failure count into the
// CsrCheck *r, lowers r's smallest bad row and position, and clears the
// device words.  The caller synchronises the device first.
#define CPRA_CSR_CHECK_COLLECT(r)                                                         \
  do {                                                                                    \
    unsigned long long n_ = 0;                                                            \
    long long row_ = 0, ent_ = 0;                                                         \
    cudaMemcpyFromSymbol(&n_, g_csr_fail_count, sizeof(n_));                              \
    cudaMemcpyFromSymbol(&row_, g_csr_fail_row, sizeof(row_));                            \
    cudaMemcpyFromSymbol(&ent_, g_csr_fail_entry, sizeof(ent_));                          \
    (r)->count += n_;                                                                     \
    if (row_ < (r)->first_row) (r)->first_row = row_;                                     \
    if (ent_ < (r)->first_entry) (r)->first_entry = ent_;                                 \
    const unsigned long long zero_ = 0;                                                   \
    const long long none_ = 0x7fffffffffffffffLL;                                         \
    cudaMemcpyToSymbol(g_csr_fail_count, &zero_, sizeof(zero_));                          \
    cudaMemcpyToSymbol(g_csr_fail_row, &none_, sizeof(none_));                            \
    cudaMemcpyToSymbol(g_csr_fail_entry, &none_, sizeof(none_));                          \
  } while (0)
#endif
