// Optimiser, weight shadows, parameter initialisation and layout copies.
#include <math.h>

#include "common.cuh"
#include "kernels.cuh"

namespace cpra {

namespace {

__global__ void adam_kernel(int64_t n, float* __restrict__ th, float* __restrict__ m,
                            float* __restrict__ v, const float* __restrict__ g, float lr,
                            float b1, float b2, float eps, float wd, float bc1, float bc2,
                            const int* halt, const StepScalars* sc) {
  if (halt && *halt) return;  // early stopping froze the parameters
  if (sc) {
    bc1 = sc->bc1;
    bc2 = sc->bc2;
  }
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nth = (int64_t)gridDim.x * blockDim.x;
  // four parameters per thread and iteration when every array is 16-byte
  // aligned, the remainder one at a time
  const bool vec = ((reinterpret_cast<uintptr_t>(th) | reinterpret_cast<uintptr_t>(m) |
                     reinterpret_cast<uintptr_t>(v) | reinterpret_cast<uintptr_t>(g)) & 15u) == 0;
  int64_t done = 0;
  if (vec) {
    const int64_t n4 = n / 4;
    for (int64_t q = tid; q < n4; q += nth) {
      float4 t4 = reinterpret_cast<float4*>(th)[q], m4 = reinterpret_cast<float4*>(m)[q];
      float4 v4 = reinterpret_cast<float4*>(v)[q];
      const float4 g4 = reinterpret_cast<const float4*>(g)[q];
      t4.x = adam_update(t4.x, m4.x, v4.x, g4.x, lr, b1, b2, eps, wd, bc1, bc2);
      t4.y = adam_update(t4.y, m4.y, v4.y, g4.y, lr, b1, b2, eps, wd, bc1, bc2);
      t4.z = adam_update(t4.z, m4.z, v4.z, g4.z, lr, b1, b2, eps, wd, bc1, bc2);
      t4.w = adam_update(t4.w, m4.w, v4.w, g4.w, lr, b1, b2, eps, wd, bc1, bc2);
      reinterpret_cast<float4*>(th)[q] = t4;
      reinterpret_cast<float4*>(m)[q] = m4;
      reinterpret_cast<float4*>(v)[q] = v4;
    }
    done = n4 * 4;
  }
  for (int64_t i = done + tid; i < n; i += nth) {
    float mi = m[i], vi = v[i];
    th[i] = adam_update(th[i], mi, vi, g[i], lr, b1, b2, eps, wd, bc1, bc2);
    m[i] = mi;
    v[i] = vi;
  }
}

template <typename TD>
__global__ void copy_rows_kernel(int64_t N, int H, const float* __restrict__ src, TD* dst,
                                 int64_t ldd) {
  const int64_t total = N * H;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / H, c = i % H;
    dst[r * ldd + c] = from_f<TD>(src[i]);
  }
}

// BF16 copies of the dense weights in both orientations, 32 x 32 tiles
// through shared memory so that the transposed copies are written row by row
// too.  Tiles t < t1 cover Wcat1 (H1 x 2H0), the rest Wcat2 padded to S_pad rows.
__global__ void weight_shadows_kernel(const float* __restrict__ th, int H0, int H1, int S,
                                      int S_pad, bf16* W1s, bf16* W1t, bf16* W2s, bf16* W2t) {
  __shared__ bf16 tile[32][34];
  const int K1 = 2 * H0, K2 = 2 * H1;
  const int tc1 = (K1 + 31) / 32, tr1 = (H1 + 31) / 32;
  const int tc2 = (K2 + 31) / 32;
  const int64_t t1 = (int64_t)tr1 * tc1;
  const int64_t t = blockIdx.x;
  const float* src;
  bf16 *ds, *dt;
  int rows, cols, valid_rows, tcn;
  int64_t tt;
  if (t < t1) {
    src = th; ds = W1s; dt = W1t; rows = H1; valid_rows = H1; cols = K1; tt = t; tcn = tc1;
  } else {
    src = th + (int64_t)H1 * K1 + H1; ds = W2s; dt = W2t; rows = S_pad; valid_rows = S;
    cols = K2; tt = t - t1; tcn = tc2;
  }
  const int r0 = (int)(tt / tcn) * 32, c0 = (int)(tt % tcn) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int y = ty; y < 32; y += 8) {
    const int r = r0 + y, c = c0 + tx;
    if (r < rows && c < cols) {
      const bf16 w = __float2bfloat16_rn(r < valid_rows ? src[(int64_t)r * cols + c] : 0.f);
      ds[(int64_t)r * cols + c] = w;
      tile[y][tx] = w;
    }
  }
  __syncthreads();
  for (int y = ty; y < 32; y += 8) {  // transposed: row c of dt, columns r
    const int c = c0 + y, r = r0 + tx;
    if (r < rows && c < cols) dt[(int64_t)c * rows + r] = tile[tx][y];
  }
}

// The dense weights split exactly into three TF32 parts (split3) for the FP32
// form's tensor-core GEMMs, written like the BF16 shadows (32 x 32 tiles
// through shared memory, both orientations).
struct SplitOut {
  float* W1[3];
  float* W1t[3];
  float* W2[3];
  float* W2t[3];
};

__global__ void weight_split_kernel(const float* __restrict__ th, int H0, int H1, int S,
                                    int S_pad, SplitOut o) {
  __shared__ float tile[3][32][33];
  const int K1 = 2 * H0, K2 = 2 * H1;
  const int tc1 = (K1 + 31) / 32, tr1 = (H1 + 31) / 32;
  const int tc2 = (K2 + 31) / 32;
  const int64_t t1 = (int64_t)tr1 * tc1;
  const int64_t t = blockIdx.x;
  const float* src;
  float* const* ds;
  float* const* dt;
  int rows, cols, valid_rows, tcn;
  int64_t tt;
  if (t < t1) {
    src = th; ds = o.W1; dt = o.W1t; rows = H1; valid_rows = H1; cols = K1; tt = t; tcn = tc1;
  } else {
    src = th + (int64_t)H1 * K1 + H1; ds = o.W2; dt = o.W2t; rows = S_pad; valid_rows = S;
    cols = K2; tt = t - t1; tcn = tc2;
  }
  const int r0 = (int)(tt / tcn) * 32, c0 = (int)(tt % tcn) * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8 threads
  for (int y = ty; y < 32; y += 8) {
    const int r = r0 + y, c = c0 + tx;
    if (r < rows && c < cols) {
      float part[3];
      split3(r < valid_rows ? src[(int64_t)r * cols + c] : 0.f, part[0], part[1], part[2]);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ds[k][(int64_t)r * cols + c] = part[k];
        tile[k][y][tx] = part[k];
      }
    }
  }
  __syncthreads();
  for (int y = ty; y < 32; y += 8) {  // transposed: row c, columns r
    const int c = c0 + y, r = r0 + tx;
    if (r < rows && c < cols) {
#pragma unroll
      for (int k = 0; k < 3; ++k) dt[k][(int64_t)c * rows + r] = tile[k][tx][y];
    }
  }
}

__global__ void flag_error_kernel(int* flag, int bits) {
  if (flag) atomicOr(flag, bits);
}

__global__ void init_uniform_kernel(float* p, int64_t n, float bound, uint64_t seed,
                                    uint64_t tag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (2.f * u24(seed, tag, (uint64_t)i) - 1.f) * bound;
}

// Box-Muller transform of two counter-based uniforms.
__global__ void init_normal_kernel(float* p, int64_t n, uint64_t seed, uint64_t tag) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    p[i] = normal_at(seed, tag, (uint64_t)i);
  }
}

template <typename TS>
__global__ void upcast_rows_kernel(int64_t N, int S, const TS* __restrict__ src, int64_t lds,
                                   float* dst) {
  const int64_t total = N * S;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = i / S, c = i % S;
    dst[i] = to_f(src[r * lds + c]);
  }
}

__global__ void total_loss_kernel(const float* __restrict__ terms, const float* __restrict__ lambda,
                                  int S, float gamma, float nu, float* out) {
  __shared__ double part[256];
  double t = 0.0;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    const double pen = lambda ? (double)lambda[s] * (double)terms[S + s] : 0.0;
    t += (double)terms[s] + pen + (double)gamma * (double)terms[2 * S + s];
  }
  part[threadIdx.x] = t;
  for (int k = threadIdx.x; k < 3 * S + 1; k += blockDim.x) out[k] = terms[k];
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) r += part[k];
    r += (double)nu * (double)terms[3 * S];
    out[3 * S + 1] = (float)r;
  }
}

__global__ void scale_copy_kernel(int64_t n, float scale, const float* __restrict__ src,
                                  float* __restrict__ dst) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = scale * src[i];
}

inline unsigned grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return (unsigned)(g < 1 ? 1 : g);
}

}  // namespace

void adam_launch(int64_t n, float* theta, float* m, float* v, const float* g, float lr,
                 float beta1, float beta2, float eps, float wd, float bc1, float bc2,
                 const int* halt, const StepScalars* sc, cudaStream_t st) {
  adam_kernel<<<grid_for(n), 256, 0, st>>>(n, theta, m, v, g, lr, beta1, beta2, eps, wd, bc1,
                                           bc2, halt, sc);
}

namespace {

// One block: every thread computes the per-shot monitored values (they do not
// depend on one another); thread 0 then adds them in shot order with
// explicit roundings (no contraction into fused multiply-adds), so the
// decision is reproducible.
__global__ void early_stop_kernel(const float* __restrict__ terms, const float* __restrict__ lambda,
                                  int S, float tol, int patience, float ann_below,
                                  const StepScalars* sc, EarlyStopState* st) {
  // the per-shot values in parallel (they do not depend on one another),
  // then the two running sums in shot order on one thread
  __shared__ double ls_s[1024], an_s[1024];
  if (st->stopped) return;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    double ls = (double)terms[s];
    if (lambda) ls = __dadd_rn(ls, __dmul_rn((double)lambda[s], (double)terms[S + s]));
    ls_s[s] = ls;
    an_s[s] = (double)terms[2 * S + s];
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const float gamma = sc->gamma;
  const long long t = sc->t, updates = sc->updates;
  double l = 0.0, ann = 0.0;
  for (int s = 0; s < S; ++s) {
    l = __dadd_rn(l, ls_s[s]);
    ann = __dadd_rn(ann, an_s[s]);
  }
  const double phi = __dmul_rn((double)gamma, ann);
  if (ann_below > 0.f && ann < (double)ann_below) {  // the annealing term has vanished
    st->stopped = 1;
    st->stop_step = t;
    st->updates_at_stop = updates;
  } else if (patience > 0 && st->have_prev) {
    const double dl = __dadd_rn(l, -st->prev_l), dp = __dadd_rn(phi, -st->prev_phi);
    const bool stale = (dl > 0.0 || fabs(dl) <= (double)tol) && (dp > 0.0 || fabs(dp) <= (double)tol);
    st->count = stale ? st->count + 1 : 0;
    if (st->count >= patience) {
      st->stopped = 1;
      st->stop_step = t;
      st->updates_at_stop = updates;
    }
  }
  st->prev_l = l;
  st->prev_phi = phi;
  st->have_prev = 1;
}

}  // namespace

void early_stop_launch(const float* terms, const float* lambda, int S, float tol, int patience,
                       float ann_below, const StepScalars* sc, EarlyStopState* st,
                       cudaStream_t stream) {
  early_stop_kernel<<<1, 256, 0, stream>>>(terms, lambda, S, tol, patience, ann_below, sc, st);
}

namespace {

// The linear schedule gamma_t = gamma0 + (gamma1 - gamma0) * min(t, T-1) / (T-1)
// (one thread, explicit double roundings) and the Adam bias corrections
// 1 - beta^(updates + 1).
__global__ void step_scalars_kernel(StepScalars* sc, int from_device, long long t, long long updates,
                                    float gamma0, float gamma1, long long T, float beta1,
                                    float beta2) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  if (from_device) {
    t = sc->next_t;
    updates = sc->next_updates;
  }
  float g = gamma1;
  if (T > 1) {
    long long tt = t < 0 ? 0 : (t > T - 1 ? T - 1 : t);
    const double span = __dadd_rn((double)gamma1, -(double)gamma0);
    const double frac = __ddiv_rn(__dmul_rn(span, (double)tt), (double)(T - 1));
    g = (float)__dadd_rn((double)gamma0, frac);
  }
  const double u = (double)(updates + 1);
  sc->gamma = g;
  sc->bc1 = (float)(1.0 - pow((double)beta1, u));
  sc->bc2 = (float)(1.0 - pow((double)beta2, u));
  sc->t = t;
  sc->updates = updates;
  sc->next_t = t + 1;
  sc->next_updates = updates + 1;
}

}  // namespace

void step_scalars_launch(StepScalars* sc, int from_device, long long t, long long updates,
                         float gamma0, float gamma1, long long T, float beta1, float beta2,
                         cudaStream_t st) {
  step_scalars_kernel<<<1, 32, 0, st>>>(sc, from_device, t, updates, gamma0, gamma1, T, beta1,
                                        beta2);
}

namespace {
__global__ void fill_rows_kernel(int64_t N, int S, int64_t ld, float value, float* dst) {
  const int64_t total = N * ld;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = (e % ld) < S ? value : 0.f;
}
}  // namespace

void fill_rows_launch(int64_t N, int S, int64_t ld, float value, float* dst, cudaStream_t st) {
  fill_rows_kernel<<<grid_for(N * ld), 256, 0, st>>>(N, S, ld, value, dst);
}

void copy_rows_launch(int64_t N, int H, const float* src, void* dst, int64_t ldd, int ddst,
                      cudaStream_t st) {
  const unsigned grid = grid_for(N * H);
  if (ddst == DT_BF16)
    copy_rows_kernel<bf16><<<grid, 256, 0, st>>>(N, H, src, static_cast<bf16*>(dst), ldd);
  else
    copy_rows_kernel<float><<<grid, 256, 0, st>>>(N, H, src, static_cast<float*>(dst), ldd);
}

void weight_shadows_launch(const float* theta, int H0, int H1, int S, int S_pad, void* W1s,
                           void* W1t, void* W2s, void* W2t, cudaStream_t st) {
  const int64_t tiles = (int64_t)((H1 + 31) / 32) * ((2 * H0 + 31) / 32) +
                        (int64_t)((S_pad + 31) / 32) * ((2 * H1 + 31) / 32);
  weight_shadows_kernel<<<(unsigned)tiles, 256, 0, st>>>(
      theta, H0, H1, S, S_pad, static_cast<bf16*>(W1s), static_cast<bf16*>(W1t),
      static_cast<bf16*>(W2s), static_cast<bf16*>(W2t));
}

void weight_split_launch(const float* theta, int H0, int H1, int S, int S_pad, float* const* W1,
                         float* const* W1t, float* const* W2, float* const* W2t, cudaStream_t st) {
  const int64_t tiles = (int64_t)((H1 + 31) / 32) * ((2 * H0 + 31) / 32) +
                        (int64_t)((S_pad + 31) / 32) * ((2 * H1 + 31) / 32);
  SplitOut o;
  for (int k = 0; k < 3; ++k) {
    o.W1[k] = W1[k];
    o.W1t[k] = W1t[k];
    o.W2[k] = W2[k];
    o.W2t[k] = W2t[k];
  }
  weight_split_kernel<<<(unsigned)tiles, 256, 0, st>>>(theta, H0, H1, S, S_pad, o);
}

void flag_error_launch(int* flag, int bits, cudaStream_t st) {
  flag_error_kernel<<<1, 1, 0, st>>>(flag, bits);
}

void init_uniform_launch(float* p, int64_t n, float bound, uint64_t seed, uint64_t tag,
                         cudaStream_t st) {
  init_uniform_kernel<<<grid_for(n), 256, 0, st>>>(p, n, bound, seed, tag);
}

void init_normal_launch(float* p, int64_t n, uint64_t seed, uint64_t tag, cudaStream_t st) {
  init_normal_kernel<<<grid_for(n), 256, 0, st>>>(p, n, seed, tag);
}

void total_loss_launch(const float* terms, const float* lambda, int S, float gamma, float nu,
                       float* out, cudaStream_t st) {
  total_loss_kernel<<<1, 256, 0, st>>>(terms, lambda, S, gamma, nu, out);
}

void scale_copy_launch(int64_t n, float scale, const float* src, float* dst, cudaStream_t st) {
  scale_copy_kernel<<<grid_for(n), 256, 0, st>>>(n, scale, src, dst);
}

void upcast_rows_launch(int64_t N, int S, const void* src, int64_t lds, int dsrc, float* dst,
                        cudaStream_t st) {
  const unsigned grid = grid_for(N * S);
  if (dsrc == DT_BF16)
    upcast_rows_kernel<bf16><<<grid, 256, 0, st>>>(N, S, static_cast<const bf16*>(src), lds, dst);
  else
    upcast_rows_kernel<float><<<grid, 256, 0, st>>>(N, S, static_cast<const float*>(src), lds,
                                                    dst);
}

}  // namespace cpra
