// Warm-start network behind the C ABI (cpra.h): a three-layer Eq. GCN that
// maps fixed node features to S logits, trained with binary cross-entropy
// against rounded CPRA solutions.  Forward, adjoint and Adam run on the same
// SpMM, tensor-core / CUDA-core GEMM and optimiser kernels as the CPRA step;
// k_warm.cu adds the features, the cross-entropy and the weight copies.
//
// Buffers (act = the dense layers' dtype):
//   A0 = [X | M0] N x 2F   A1 = [H1 | M1] N x 2H   A2 = [H2 | M2] N x 2H
//   Z3 f32 N x S_pad (logits)   G3 act N x S_pad   GA2, GA1 act N x 2H
// with M_k = D^-1 A H_k, H_{k+1} = ReLU(A_k Wcat_{k+1}^T + b_{k+1}), logits
// Z3 = A2 Wcat3^T + b3.  The adjoint follows the CPRA step's: input
// gradients [G_Ha | G_M / deg] = G Wcat (one GEMM with a split epilogue),
// G_Z = (G_Ha + A G_M/deg) * 1[H > 0] with the bias gradient as column sums,
// weight gradients G^T A_k split over the node dimension.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "cpra.h"
#include "kernels.cuh"
#include "tc_gemm.cuh"

using namespace cpra;

struct cpra_ws {
  cpra_ws_config cfg{};
  int F = 0, H = 0, S = 0, S_pad = 0, act = DT_F32;
  int64_t max_N = 0, max_nnz = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 148;
  bool use_tc = false;
  // parameter blocks (FP32), each 16-float aligned; logical layout in cpra.h
  int64_t nparam = 0, nstore = 0;
  int64_t o_w1 = 0, o_b1 = 0, o_w2 = 0, o_b2 = 0, o_w3 = 0, o_b3 = 0;
  float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  void *W1s = nullptr, *W1t = nullptr, *W2s = nullptr, *W2t = nullptr, *W3s = nullptr,
       *W3t = nullptr;
  void *A0 = nullptr, *A1 = nullptr, *A2 = nullptr, *G3 = nullptr, *GA2 = nullptr,
       *GA1 = nullptr;
  float* Z3 = nullptr;
  float* inv_deg = nullptr;
  float* part = nullptr;  // per-block partial rows
  size_t part_floats = 0;
  float* wg_part = nullptr;
  size_t wg_part_floats = 0;
  float* loss_d = nullptr;
  int* err_flag = nullptr;
  int64_t steps = 0;
  void* mem = nullptr;
  std::string err;
};

namespace {

constexpr size_t kAlignW = 256;
constexpr int kMaxPartRows = 2048;

int64_t align16(int64_t x) { return (x + 15) / 16 * 16; }

std::string ws_validate(const cpra_ws_config* c) {
  if (!c) return "cfg is NULL";
  if (c->F < 16 || c->F % 16 || c->F > 1024) return "F must be a multiple of 16 in [16, 1024]";
  if (c->H < 16 || c->H % 16 || c->H > 1024) return "H must be a multiple of 16 in [16, 1024]";
  if (c->S < 1 || c->S > 1024) return "S must be in [1, 1024]";
  if (c->precision != CPRA_FP32 && c->precision != CPRA_BF16) return "precision must be FP32 or BF16";
  if (!(c->lr > 0.f) || !(c->beta1 >= 0.f && c->beta1 < 1.f) || !(c->beta2 >= 0.f && c->beta2 < 1.f) ||
      !(c->eps >= 0.f) || !(c->weight_decay >= 0.f))
    return "bad optimiser hyper-parameters";
  return "";
}

cpra_status ws_fail(cpra_ws* w, cpra_status s, const std::string& msg) {
  if (w) w->err = msg;
  return s;
}

void* act_at(void* base, int64_t elems, const cpra_ws* w) {
  return static_cast<char*>(base) + elems * (w->act == DT_BF16 ? 2 : 4);
}

struct WCarver {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + kAlignW - 1) / kAlignW * kAlignW;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

size_t ws_carve(cpra_ws* w, void* base) {
  WCarver cv{static_cast<char*>(base)};
  const int64_t N = w->max_N;
  const size_t a = w->act == DT_BF16 ? 2 : 4;
  w->theta = cv.take<float>(w->nstore);
  w->m = cv.take<float>(w->nstore);
  w->v = cv.take<float>(w->nstore);
  w->grad = cv.take<float>(w->nstore);
  w->W1s = cv.take<uint16_t>((size_t)w->H * 2 * w->F);
  w->W1t = cv.take<uint16_t>((size_t)w->H * 2 * w->F);
  w->W2s = cv.take<uint16_t>((size_t)w->H * 2 * w->H);
  w->W2t = cv.take<uint16_t>((size_t)w->H * 2 * w->H);
  w->W3s = cv.take<uint16_t>((size_t)w->S_pad * 2 * w->H);
  w->W3t = cv.take<uint16_t>((size_t)w->S_pad * 2 * w->H);
  w->A0 = cv.take<char>((size_t)N * 2 * w->F * a);
  w->A1 = cv.take<char>((size_t)N * 2 * w->H * a);
  w->A2 = cv.take<char>((size_t)N * 2 * w->H * a);
  w->Z3 = cv.take<float>((size_t)N * w->S_pad);
  w->G3 = cv.take<char>((size_t)N * w->S_pad * a);
  w->GA2 = cv.take<char>((size_t)N * 2 * w->H * a);
  w->GA1 = cv.take<char>((size_t)N * 2 * w->H * a);
  w->inv_deg = cv.take<float>(N);
  w->part_floats = (size_t)kMaxPartRows * std::max(w->H, w->S_pad);
  w->part = cv.take<float>(w->part_floats);
  const size_t slab = std::max({(size_t)w->S_pad * 2 * w->H, (size_t)w->H * 2 * w->H,
                                (size_t)w->H * 2 * w->F});
  w->wg_part_floats = slab * (size_t)(4 * w->num_sms);
  w->wg_part = cv.take<float>(w->wg_part_floats);
  w->loss_d = cv.take<float>(4);
  w->err_flag = cv.take<int>(4);
  return cv.off + kAlignW;
}

void ws_dense(cpra_ws* w, const GemmArgs& g0) {
  GemmArgs g = g0;
  g.err_flag = w->err_flag;
  if (w->use_tc && tc_gemm_supported(g)) tc_gemm_launch(g, w->num_sms, w->stream);
  else gemm_simt_launch(g, w->stream);
}

// dst[M x Nc] (row stride ldo) = A^T B over the first N rows.
void ws_wgrad(cpra_ws* w, int64_t N, const void* A, int64_t lda, int M, const void* B,
              int64_t ldb, int Nc, float* dst, int64_t ldo) {
  GemmArgs g;
  g.M = M; g.Nc = Nc; g.K = N;
  g.A = A; g.lda = lda; g.da = w->act; g.a_kmajor = 0;
  g.B = B; g.ldb = ldb; g.db = w->act; g.b_kmajor = 0;
  g.epi = EPI_PARTIAL; g.out0 = w->wg_part; g.ld0 = Nc;
  const int64_t tiles = ((int64_t)(M + 63) / 64) * ((Nc + 63) / 64);
  int64_t splits = std::max<int64_t>(1, (2 * (int64_t)w->num_sms + tiles - 1) / tiles);
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, N / 256));
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, (int64_t)(w->wg_part_floats / ((size_t)M * Nc))));
  g.splits = (int)splits;
  g.err_flag = w->err_flag;
  if (w->use_tc && tc_wgrad_supported(g)) {
    tc_wgrad_launch(g, w->num_sms, w->wg_part_floats, dst, ldo, w->stream);
    return;
  }
  gemm_simt_launch(g, w->stream);
  splitk_reduce(w->wg_part, g.splits, M, Nc, Nc, dst, ldo, w->stream);
}

void ws_shadows(cpra_ws* w) {
  if (w->act != DT_BF16) return;
  weight_pair_launch(w->theta + w->o_w1, w->H, 2 * w->F, w->H, w->W1s, w->W1t, w->stream);
  weight_pair_launch(w->theta + w->o_w2, w->H, 2 * w->H, w->H, w->W2s, w->W2t, w->stream);
  weight_pair_launch(w->theta + w->o_w3, w->S, 2 * w->H, w->S_pad, w->W3s, w->W3t, w->stream);
}

// One GCN layer k (1..3) forward: out = act(A_in Wcat_k^T + b_k).
void ws_layer(cpra_ws* w, int64_t N, const void* Ain, int K, int64_t o_wcat, const void* Ws, int Nout,
              int epi, void* out, int64_t ldo, int dout, int n_valid) {
  GemmArgs g;
  g.M = N; g.Nc = Nout; g.K = K;
  g.A = Ain; g.lda = K; g.da = w->act; g.a_kmajor = 1;
  if (w->act == DT_BF16) { g.B = Ws; g.db = DT_BF16; }
  else { g.B = w->theta + o_wcat; g.db = DT_F32; }
  g.ldb = K; g.b_kmajor = 1;
  g.epi = epi; g.bias = w->theta + (o_wcat == w->o_w1 ? w->o_b1 : o_wcat == w->o_w2 ? w->o_b2 : w->o_b3);
  g.out0 = out; g.ld0 = ldo; g.d0 = dout; g.n_valid = n_valid;
  ws_dense(w, g);
}

void ws_mean(cpra_ws* w, int64_t N, const int* rowptr, const int* col, void* block, int Hh) {
  SpmmArgs a;
  a.N = N; a.H = Hh; a.rowptr = rowptr; a.col = col; a.inv_deg = w->inv_deg;
  a.X = block; a.ldx = 2 * Hh; a.Y = act_at(block, Hh, w); a.ldy = 2 * Hh; a.mean = 1;
  a.dx = w->act; a.dy = w->act; a.err_flag = w->err_flag;
  spmm_launch(a, w->num_sms, w->num_sms * 8, w->stream);
}

cpra_status ws_forward(cpra_ws* w, int64_t N, const int* rowptr, const int* col, const float* feat,
                       float* logits, int64_t ld) {
  inv_degree_launch(N, rowptr, w->inv_deg, w->stream);
  copy_rows_launch(N, w->F, feat, w->A0, 2 * w->F, w->act, w->stream);
  ws_mean(w, N, rowptr, col, w->A0, w->F);
  ws_layer(w, N, w->A0, 2 * w->F, w->o_w1, w->W1s, w->H, EPI_BIAS_RELU, w->A1, 2 * w->H, w->act, w->H);
  ws_mean(w, N, rowptr, col, w->A1, w->H);
  ws_layer(w, N, w->A1, 2 * w->H, w->o_w2, w->W2s, w->H, EPI_BIAS_RELU, w->A2, 2 * w->H, w->act, w->H);
  ws_mean(w, N, rowptr, col, w->A2, w->H);
  ws_layer(w, N, w->A2, 2 * w->H, w->o_w3, w->W3s, w->S_pad, EPI_BIAS, logits, ld, DT_F32, w->S);
  return CPRA_OK;
}

// Adjoint of one hidden layer: G (act, N x Nout, row stride ldg) is dR/dZ of
// the layer above, Wcat that layer's weights (Nout x 2Hh), Wt its BF16
// transposed copy; writes [G_Ha | G_M/deg] into GA, then
// G_Z = (G_Ha + A G_M/deg) * 1[H > 0] in place (H = left half of Aact) and
// the bias gradient db.
cpra_status ws_hidden_adjoint(cpra_ws* w, int64_t N, const int* rowptr, const int* col, const void* G,
                              int64_t ldg, int Kg, int64_t o_wcat_above, const void* Wt_above,
                              void* GA, const void* Aact, float* db) {
  const int Hh = w->H;
  GemmArgs g;
  g.M = N; g.Nc = 2 * Hh;
  g.A = G; g.lda = ldg; g.da = w->act; g.a_kmajor = 1;
  if (w->act == DT_BF16) { g.K = Kg; g.B = Wt_above; g.ldb = Kg; g.db = DT_BF16; g.b_kmajor = 1; }
  else { g.K = Kg; g.B = w->theta + o_wcat_above; g.ldb = 2 * Hh; g.db = DT_F32; g.b_kmajor = 0; }
  g.epi = EPI_SPLIT; g.split = Hh;
  g.out0 = GA; g.ld0 = 2 * Hh; g.d0 = w->act;
  g.out1 = act_at(GA, Hh, w); g.ld1 = 2 * Hh; g.d1 = w->act;
  g.row_scale = w->inv_deg; g.n_valid = 2 * Hh;
  ws_dense(w, g);
  SpmmArgs a;
  a.N = N; a.H = Hh; a.rowptr = rowptr; a.col = col; a.inv_deg = w->inv_deg;
  a.X = act_at(GA, Hh, w); a.ldx = 2 * Hh;
  a.add = GA; a.ldadd = 2 * Hh;
  a.mask = Aact; a.ldm = 2 * Hh;
  a.Y = GA; a.ldy = 2 * Hh; a.mean = 0;
  a.dx = w->act; a.dy = w->act; a.err_flag = w->err_flag;
  a.colsum_partials = w->part;
  const int grid = spmm_launch(a, w->num_sms, std::min(w->num_sms * 8, kMaxPartRows), w->stream);
  if (grid < 0) return CPRA_EINVAL;
  colsum_finalize(w->part, grid, Hh, Hh, db, nullptr, 0, 0, nullptr, w->stream);
  return CPRA_OK;
}

cpra_status ws_sync_err(cpra_ws* w) {
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, w->err_flag, sizeof(int), cudaMemcpyDeviceToHost, w->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(w->stream);
  if (e != cudaSuccess) return ws_fail(w, CPRA_ECUDA, cudaGetErrorString(e));
  if (flag & 2) {
    cudaMemsetAsync(w->err_flag, 0, sizeof(int), w->stream);
    return ws_fail(w, CPRA_ETIMEOUT, "a bounded device-side wait gave up (tensor-core pipeline)");
  }
  return CPRA_OK;
}

}  // namespace

extern "C" {

void cpra_ws_config_default(cpra_ws_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->F = 16;
  c->H = 64;
  c->S = 32;
  c->precision = CPRA_BF16;
  c->lr = 1e-3f;
  c->beta1 = 0.9f;
  c->beta2 = 0.999f;
  c->eps = 1e-8f;
  c->weight_decay = 0.f;
  c->seed = 1;
}

int64_t cpra_ws_param_count(const cpra_ws_config* c) {
  if (!ws_validate(c).empty()) return 0;
  const int64_t F = c->F, H = c->H, S = c->S;
  return 2 * H * F + H + 2 * H * H + H + 2 * S * H + S;
}

cpra_status cpra_ws_create(cpra_ws** out, const cpra_ws_config* cfg, int64_t max_nodes,
                           int64_t max_nnz, void* cuda_stream) {
  if (!out) return CPRA_EINVAL;
  *out = nullptr;
  if (!ws_validate(cfg).empty() || max_nodes < 1 || max_nnz < 0 || max_nodes > 0x7fffffffLL ||
      max_nnz > 0x7fffffffLL)
    return CPRA_EINVAL;
  cpra_ws* w = new cpra_ws();
  w->cfg = *cfg;
  w->F = cfg->F; w->H = cfg->H; w->S = cfg->S; w->S_pad = (cfg->S + 15) / 16 * 16;
  w->act = cfg->precision == CPRA_BF16 ? DT_BF16 : DT_F32;
  w->max_N = max_nodes; w->max_nnz = max_nnz;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&w->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (w->act == DT_BF16) {
    std::string msg;
    w->use_tc = tc_prepare(w->num_sms, &msg);
  }
  // parameter blocks, 16-float aligned; b3 padded to S_pad for the epilogue's vector loads
  const int64_t F = w->F, H = w->H, S = w->S;
  w->nparam = 2 * H * F + H + 2 * H * H + H + 2 * S * H + S;
  w->o_w1 = 0;
  w->o_b1 = align16(w->o_w1 + 2 * H * F);
  w->o_w2 = align16(w->o_b1 + H);
  w->o_b2 = align16(w->o_w2 + 2 * H * H);
  w->o_w3 = align16(w->o_b2 + H);
  w->o_b3 = align16(w->o_w3 + 2 * S * H);
  w->nstore = align16(w->o_b3 + w->S_pad);
  if (cuda_stream) {
    w->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete w;
      return CPRA_ECUDA;
    }
    w->own_stream = true;
  }
  const size_t bytes = ws_carve(w, nullptr);
  if (cudaMalloc(&w->mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    if (w->own_stream) cudaStreamDestroy(w->stream);
    delete w;
    return CPRA_ENOMEM;
  }
  ws_carve(w, w->mem);
  cudaStream_t st = w->stream;
  cudaMemsetAsync(w->mem, 0, bytes, st);
  // U(+-1/sqrt(fan_in)) per block (fan_in of a layer = 2 x its input width)
  init_uniform_launch(w->theta + w->o_w1, 2 * H * F, 1.f / std::sqrt(2.f * F), cfg->seed, 101, st);
  init_uniform_launch(w->theta + w->o_b1, H, 1.f / std::sqrt(2.f * F), cfg->seed, 102, st);
  init_uniform_launch(w->theta + w->o_w2, 2 * H * H, 1.f / std::sqrt(2.f * H), cfg->seed, 103, st);
  init_uniform_launch(w->theta + w->o_b2, H, 1.f / std::sqrt(2.f * H), cfg->seed, 104, st);
  init_uniform_launch(w->theta + w->o_w3, 2 * S * H, 1.f / std::sqrt(2.f * H), cfg->seed, 105, st);
  init_uniform_launch(w->theta + w->o_b3, S, 1.f / std::sqrt(2.f * H), cfg->seed, 106, st);
  ws_shadows(w);
  if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
    cpra_ws_destroy(w);
    return CPRA_ECUDA;
  }
  *out = w;
  return CPRA_OK;
}

cpra_status cpra_ws_features(cpra_ws* w, int64_t N, const int32_t* rowptr, uint64_t graph_seed,
                             float* features) {
  if (!w || !rowptr || !features || N < 1) return ws_fail(w, CPRA_EINVAL, "bad arguments");
  ws_features_launch(N, rowptr, graph_seed, w->F, features, w->stream);
  return cudaGetLastError() == cudaSuccess ? CPRA_OK : ws_fail(w, CPRA_ECUDA, "features");
}

cpra_status cpra_ws_train_step(cpra_ws* w, int64_t N, int64_t nnz, const int32_t* rowptr,
                               const int32_t* col, const float* features,
                               const uint32_t* target_bits, float* loss_out) {
  if (!w || !rowptr || !col || !features || !target_bits || N < 1 || nnz < 0)
    return ws_fail(w, CPRA_EINVAL, "bad arguments");
  if (N > w->max_N || nnz > w->max_nnz) return ws_fail(w, CPRA_EINVAL, "graph larger than the network's buffers");
  cudaStream_t st = w->stream;
  const int H = w->H;
  ws_forward(w, N, rowptr, col, features, w->Z3, w->S_pad);
  // dR/dZ3 of the mean cross-entropy and the loss
  const int bgrid = ws_bce_launch(N, w->S, w->S_pad, w->Z3, w->S_pad, target_bits, w->G3, w->S_pad,
                                  w->act, 1.f / ((float)N * (float)w->S), w->part,
                                  std::min(w->num_sms * 8, kMaxPartRows), st);
  colsum_finalize(w->part, bgrid, 1, 1, w->loss_d, nullptr, 0, 0, nullptr, st);
  const int cblocks = rows_colsum_launch(N, w->S, w->G3, w->S_pad, w->act, w->part,
                                         std::min<int>(kMaxPartRows, (int)(w->part_floats / w->S_pad)), st);
  colsum_finalize(w->part, cblocks, w->S, w->S, w->grad + w->o_b3, nullptr, 0, 0, nullptr, st);
  ws_wgrad(w, N, w->G3, w->S_pad, w->S, w->A2, 2 * H, 2 * H, w->grad + w->o_w3, 2 * H);
  cpra_status s = ws_hidden_adjoint(w, N, rowptr, col, w->G3, w->S_pad,
                                    w->act == DT_BF16 ? w->S_pad : w->S, w->o_w3, w->W3t, w->GA2,
                                    w->A2, w->grad + w->o_b2);
  if (s != CPRA_OK) return ws_fail(w, s, "layer-3 adjoint");
  ws_wgrad(w, N, w->GA2, 2 * H, H, w->A1, 2 * H, 2 * H, w->grad + w->o_w2, 2 * H);
  s = ws_hidden_adjoint(w, N, rowptr, col, w->GA2, 2 * H, H, w->o_w2, w->W2t, w->GA1, w->A1,
                        w->grad + w->o_b1);
  if (s != CPRA_OK) return ws_fail(w, s, "layer-2 adjoint");
  ws_wgrad(w, N, w->GA1, 2 * H, H, w->A0, 2 * w->F, 2 * w->F, w->grad + w->o_w1, 2 * w->F);
  w->steps += 1;
  const double t = (double)w->steps;
  const float bc1 = (float)(1.0 - std::pow((double)w->cfg.beta1, t));
  const float bc2 = (float)(1.0 - std::pow((double)w->cfg.beta2, t));
  adam_launch(w->nstore, w->theta, w->m, w->v, w->grad, w->cfg.lr, w->cfg.beta1, w->cfg.beta2,
              w->cfg.eps, w->cfg.weight_decay, bc1, bc2, nullptr, nullptr, st);
  ws_shadows(w);
  if (cudaGetLastError() != cudaSuccess) return ws_fail(w, CPRA_ECUDA, "training kernels");
  if (loss_out) {
    if (cudaMemcpyAsync(loss_out, w->loss_d, sizeof(float), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return ws_fail(w, CPRA_ECUDA, "loss readback");
    return ws_sync_err(w);
  }
  return CPRA_OK;
}

cpra_status cpra_ws_predict(cpra_ws* w, int64_t N, int64_t nnz, const int32_t* rowptr,
                            const int32_t* col, const float* features, float* logits, int64_t ld) {
  if (!w || !rowptr || !col || !features || !logits || N < 1 || nnz < 0 || ld < w->S)
    return ws_fail(w, CPRA_EINVAL, "bad arguments");
  if (N > w->max_N || nnz > w->max_nnz) return ws_fail(w, CPRA_EINVAL, "graph larger than the network's buffers");
  if (ld % 4) return ws_fail(w, CPRA_EINVAL, "ld must be a multiple of 4");
  if (ld >= w->S_pad) {
    ws_forward(w, N, rowptr, col, features, logits, ld);
  } else {  // the epilogue writes S_pad columns: go through Z3
    ws_forward(w, N, rowptr, col, features, w->Z3, w->S_pad);
    if (cudaMemcpy2DAsync(logits, sizeof(float) * ld, w->Z3, sizeof(float) * w->S_pad,
                          sizeof(float) * w->S, N, cudaMemcpyDeviceToDevice, w->stream) != cudaSuccess)
      return ws_fail(w, CPRA_ECUDA, "logits copy");
  }
  return cudaGetLastError() == cudaSuccess ? CPRA_OK : ws_fail(w, CPRA_ECUDA, "forward kernels");
}

cpra_status cpra_ws_get_params(cpra_ws* w, int32_t which, float* host, size_t count) {
  if (!w || !host || (size_t)w->nparam != count || (which != 0 && which != 1))
    return ws_fail(w, CPRA_EINVAL, "bad arguments");
  const float* src = which == 0 ? w->theta : w->grad;
  const int64_t F = w->F, H = w->H, S = w->S;
  const int64_t offs[6] = {w->o_w1, w->o_b1, w->o_w2, w->o_b2, w->o_w3, w->o_b3};
  const int64_t lens[6] = {2 * H * F, H, 2 * H * H, H, 2 * S * H, S};
  float* p = host;
  for (int k = 0; k < 6; ++k) {
    if (cudaMemcpyAsync(p, src + offs[k], sizeof(float) * lens[k], cudaMemcpyDeviceToHost,
                        w->stream) != cudaSuccess)
      return ws_fail(w, CPRA_ECUDA, "params readback");
    p += lens[k];
  }
  return cudaStreamSynchronize(w->stream) == cudaSuccess ? CPRA_OK : ws_fail(w, CPRA_ECUDA, "sync");
}

cpra_status cpra_ws_set_params(cpra_ws* w, const float* host, size_t count) {
  if (!w || !host || (size_t)w->nparam != count) return ws_fail(w, CPRA_EINVAL, "bad arguments");
  const int64_t F = w->F, H = w->H, S = w->S;
  const int64_t offs[6] = {w->o_w1, w->o_b1, w->o_w2, w->o_b2, w->o_w3, w->o_b3};
  const int64_t lens[6] = {2 * H * F, H, 2 * H * H, H, 2 * S * H, S};
  const float* p = host;
  for (int k = 0; k < 6; ++k) {
    if (cudaMemcpyAsync(w->theta + offs[k], p, sizeof(float) * lens[k], cudaMemcpyHostToDevice,
                        w->stream) != cudaSuccess)
      return ws_fail(w, CPRA_ECUDA, "params upload");
    p += lens[k];
  }
  ws_shadows(w);
  return cudaStreamSynchronize(w->stream) == cudaSuccess ? CPRA_OK : ws_fail(w, CPRA_ECUDA, "sync");
}

void cpra_ws_destroy(cpra_ws* w) {
  if (!w) return;
  if (w->stream) cudaStreamSynchronize(w->stream);
  if (w->mem) cudaFree(w->mem);
  if (w->own_stream && w->stream) cudaStreamDestroy(w->stream);
  delete w;
}

}  // extern "C"
