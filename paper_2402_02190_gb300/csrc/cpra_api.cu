// C-ABI of the CPRA step: context management, graph validation and upload,
// workspace layout in HBM, and the per-step kernel schedule.
//
// Step schedule (one CUDA stream, no host synchronisation unless asked):
//   forward   SPMM  M1 = mean_agg(X0)              -> XM[:, H0:]
//             GEMM  H1 = relu([X0|M1] Wcat1^T + b1)  -> HM[:, :H1]
//             SPMM  M2 = mean_agg(H1)              -> HM[:, H1:]
//             GEMM  P  = sigmoid([H1|M2] Wcat2^T + b2)
//   loss      fused SpMM + loss + rounding/eval     -> G_Z2, per-shot terms, x bits, counts
//   adjoint   GEMM  [G_H1a | G_M2/deg] = G_Z2 Wcat2
//             SPMM  G_Z1 = (G_H1a + A G_M2/deg) * 1[H1 > 0]   (+ db1 column sums)
//             GEMM  dWcat2 = G_Z2^T [H1|M2],  dWcat1 = G_Z1^T [X0|M1]   (split-K)
//             GEMM  [G_X0a | G_M1/deg] = G_Z1 Wcat1;  SPMM dX0 = G_X0a + A G_M1/deg
//   update    Adam on theta (+ BF16 weight shadows), Adam on the embeddings
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cpra.h"
#include "kernels.cuh"
#include "tc_gemm.cuh"

using namespace cpra;

namespace {

enum KernelId {
  K_SPMM_AGG1 = 0,
  K_GEMM_L1,
  K_SPMM_AGG2,
  K_GEMM_L2,
  K_LOSS,
  K_LOSS_FIN,
  K_GEMM_DGRAD2,
  K_SPMM_BWD2,
  K_WGRAD2,
  K_WGRAD1,
  K_GEMM_DGRAD1,
  K_SPMM_BWD1,
  K_ADAM,
  K_ADAM_EMB,
  K_EVAL,
  K_RECOMPUTE_MASK,
  K_DBM_SUMS,
  K_COUNT_
};

const char* kKernelNames[K_COUNT_] = {
    "spmm_agg1",   "gemm_layer1", "spmm_agg2",  "gemm_layer2", "loss_fused",
    "loss_finalize", "gemm_dgrad2", "spmm_bwd2", "wgrad2",     "wgrad1",
    "gemm_dgrad1", "spmm_bwd1",   "adam",       "spmm_bwd1_adam_embedding", "round_eval",
    "recompute_layer1_mask", "dbm_line_sums"};  // the mask now comes with layer 1: id unused

constexpr size_t kAlign = 256;
constexpr int kWvBlocks = 512;  // weighted-MIS value partial rows

struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <typename T>
  T* take(size_t count) {
    off = (off + kAlign - 1) / kAlign * kAlign;
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

int round_up(int v, int m) { return (v + m - 1) / m * m; }

int device_sm_count() {
  int dev = 0, n = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 148;
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 148;
  return n > 0 ? n : 148;
}

struct ProfRec {
  int id;
  cudaEvent_t a, b;
};

// Message of the last failed cpra_init_graph on this thread.
thread_local std::string g_init_err;

}  // namespace

struct cpra_ctx {
  cpra_config cfg{};
  std::vector<float> lambda_h;
  int64_t N = 0, nnz = 0, nparam = 0;
  int S = 0, S_pad = 0, W = 0, H0 = 0, H1 = 0, act_dt = DT_F32;
  int num_sms = 148;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  void* ws = nullptr;
  size_t ws_bytes = 0;
  bool own_ws = false;

  int* rowptr = nullptr;
  int* col = nullptr;
  float* inv_deg = nullptr;
  float* lambda_d = nullptr;
  float* theta = nullptr;
  float* theta_m = nullptr;
  float* theta_v = nullptr;
  float* grad = nullptr;
  float* X0m = nullptr;
  float* X0_m = nullptr;
  float* X0_v = nullptr;
  float* gX0 = nullptr;
  void* XM = nullptr;
  void* HM = nullptr;
  float* P = nullptr;
  void* GZ2 = nullptr;
  void* GHM = nullptr;   // aliases HM when recompute
  void* GXM = nullptr;   // aliases XM when recompute
  uint16_t* relu_bits = nullptr;  // recompute: 1[H1 > 0] as bits, N x H1/16 (layer-1 epilogue)
  EarlyStopState* es = nullptr;   // early-stopping monitor (device)
  float* w_d = nullptr;           // weighted MIS: node weights N x S_pad (else null)
  double* wv_part = nullptr;      // weighted MIS: per-block value partials
  double* wvalue = nullptr;       // weighted MIS: per-shot value
  bool wmis = false;
  // MaxCut with edge weights A_ij (own allocation): weight per CSR entry,
  // weighted degree per node, per-block cut-weight partials, cut weight per shot
  void* ew_mem = nullptr;
  float* ew_d = nullptr;
  float* wdeg_d = nullptr;
  double* cut_part = nullptr;
  double* cutw = nullptr;
  // JSON-lines metrics log written by cpra_solve (cpra_set_metrics_log)
  FILE* metrics = nullptr;
  DbmDev dbm;                     // matching instances (problem DBM)
  void* dbm_mem = nullptr;        // own cudaMalloc behind dbm, null until cpra_set_dbm
  int64_t dbm_bytes = 0;
  // the graph is the matching's constraint graph: aggregations through line
  // sums line_R [N1 x ldl], line_K [N2 x ldl] (in the DBM allocation)
  bool line_agg = false;
  float* line_R = nullptr;
  float* line_K = nullptr;
  int64_t ldl = 0;
  void* init_logits = nullptr;    // warm start: N x S_pad act dtype, own cudaMalloc
  StepScalars* sc = nullptr;      // per-step gamma / bias corrections (device)
  // one captured training step, replayed by cpra_steps / cpra_solve
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_launches = 0;     // kernels per replay
  bool capturing = false;
  bool recompute = false;
  uint32_t* xbits = nullptr;
  float* loss_part = nullptr;
  int64_t pstride = 0;
  float* terms = nullptr;
  unsigned long long* counters = nullptr;
  void* eval_rec = nullptr;
  long long* ham_d = nullptr;
  float* colsum_part = nullptr;
  float* wg_part = nullptr;
  size_t wg_part_floats = 0;
  int* err_flag = nullptr;
  void* W1s = nullptr;
  void* W1t = nullptr;
  void* W2s = nullptr;
  void* W2t = nullptr;
  // FP32 form on the tensor cores: the weights' split-TF32 parts (hi, mid,
  // lo), K-major in both orientations
  float* W1p[3] = {nullptr, nullptr, nullptr};
  float* W1tp[3] = {nullptr, nullptr, nullptr};
  float* W2p[3] = {nullptr, nullptr, nullptr};
  float* W2tp[3] = {nullptr, nullptr, nullptr};

  int64_t opt_steps = 0;
  int64_t launches = 0;
  bool have_eval = false;
  bool fwd_valid = false;  // a cpra_forward whose activations are still in place
  bool use_tc = false;
  bool use_tc3 = false;  // FP32 form: split-TF32 tensor-core GEMMs
  std::string err;

  bool prof = false;
  std::vector<ProfRec> prof_ring;
  size_t prof_used = 0;
  double prof_ms[K_COUNT_] = {0};
  int64_t prof_n[K_COUNT_] = {0};
  std::vector<cudaEvent_t> prof_pool;
};

namespace {

cpra_status fail(cpra_ctx* c, cpra_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

cpra_status cuda_check(cpra_ctx* c, cudaError_t e, const char* what) {
  if (e == cudaSuccess) return CPRA_OK;
  return fail(c, CPRA_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// Offsets into the flat theta vector.
struct Layout {
  int64_t wcat1, b1, wcat2, b2, total;
};
Layout layout_of(int H0, int H1, int S) {
  Layout L;
  L.wcat1 = 0;
  L.b1 = (int64_t)H1 * 2 * H0;
  L.wcat2 = L.b1 + H1;
  L.b2 = L.wcat2 + (int64_t)S * 2 * H1;
  L.total = L.b2 + S;
  return L;
}

std::string validate_config(const cpra_config* cfg) {
  if (!cfg) return "cfg is NULL";
  if (cfg->problem != CPRA_MIS && cfg->problem != CPRA_MAXCUT && cfg->problem != CPRA_WMIS &&
      cfg->problem != CPRA_DBM)
    return "problem must be MIS, MAXCUT, WMIS or DBM";
  if (cfg->S < 1 || cfg->S > 1024) return "S must be in [1, 1024]";
  if (cfg->H0 < 16 || cfg->H0 > 4096 || cfg->H0 % 16) return "H0 must be a multiple of 16 in [16, 4096]";
  if (cfg->H1 < 16 || cfg->H1 > 4096 || cfg->H1 % 16) return "H1 must be a multiple of 16 in [16, 4096]";
  if (cfg->alpha < 2 || cfg->alpha > 32 || cfg->alpha % 2) return "alpha must be even, 2..32";
  if (cfg->precision != CPRA_FP32 && cfg->precision != CPRA_BF16) return "precision must be FP32 or BF16";
  if (cfg->diversity_kind != CPRA_DIV_STD && cfg->diversity_kind != CPRA_DIV_VAR) return "bad diversity_kind";
  if (cfg->keep_emb_grad != 0 && cfg->keep_emb_grad != 1) return "keep_emb_grad must be 0 or 1";
  if (cfg->recompute != 0 && cfg->recompute != 1) return "recompute must be 0 or 1";
  if (cfg->es_patience < 0 || !(cfg->es_tol >= 0.f) || !std::isfinite(cfg->es_tol))
    return "early stopping needs es_patience >= 0 and a finite es_tol >= 0";
  if ((cfg->problem == CPRA_MIS || cfg->problem == CPRA_WMIS) && cfg->lambda == nullptr)
    return "MIS needs lambda[S]";
  if (cfg->train_encoder != 0 && cfg->train_encoder != 1) return "train_encoder must be 0 or 1";
  if (cfg->fp32_engine != CPRA_FP32_TENSOR && cfg->fp32_engine != CPRA_FP32_CUDA_CORES)
    return "fp32_engine must be CPRA_FP32_TENSOR or CPRA_FP32_CUDA_CORES";
  if (!(cfg->es_ann_below >= 0.f) || !std::isfinite(cfg->es_ann_below))
    return "es_ann_below must be finite and >= 0";
  if (cfg->schedule_steps < 1) return "schedule_steps must be >= 1";
  if (!(cfg->lr > 0.f) || !(cfg->beta1 >= 0.f && cfg->beta1 < 1.f) ||
      !(cfg->beta2 >= 0.f && cfg->beta2 < 1.f) || !(cfg->eps >= 0.f) || !(cfg->weight_decay >= 0.f))
    return "bad optimiser hyper-parameters";
  if (!std::isfinite(cfg->nu) || !std::isfinite(cfg->gamma0) || !std::isfinite(cfg->gamma1))
    return "nu / gamma must be finite";
  return "";
}

// Rows [r0, r1) of the graph checks: column range, no self-loop, strictly
// increasing columns, and symmetry (i appears in row j for every j in row i).
// Returns the first failing row's message, or "".
std::string validate_rows(int64_t N, const int64_t* rowptr, const int32_t* col, int64_t r0,
                          int64_t r1) {
  for (int64_t i = r0; i < r1; ++i) {
    for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int64_t j = col[e];
      if (j < 0 || j >= N) return "column index out of range";
      if (j == i) return "self-loop at node " + std::to_string(i);
      if (e > rowptr[i] && col[e - 1] >= j) return "columns must be strictly increasing within a row";
      const int32_t* b = col + rowptr[j];
      const int32_t* en = col + rowptr[j + 1];
      if (!std::binary_search(b, en, (int32_t)i))
        return "graph is not symmetric: (" + std::to_string(i) + "," + std::to_string(j) + ")";
    }
  }
  return "";
}

// Runs check(r0, r1) over contiguous row ranges on up to 16 host threads
// (one for small graphs) and returns the message of the lowest failing
// range, so the result does not depend on the thread count.
template <typename F>
std::string for_row_ranges(int64_t N, int64_t nnz, F check) {
  unsigned hw = std::thread::hardware_concurrency();
  int64_t T = nnz < (1 << 18) ? 1 : std::min<int64_t>(16, hw ? hw : 1);
  T = std::max<int64_t>(1, std::min<int64_t>(T, N));
  std::vector<std::string> msg((size_t)T);
  std::vector<std::thread> pool;
  auto range = [&](int64_t k) {
    msg[(size_t)k] = check(N * k / T, N * (k + 1) / T);
  };
  for (int64_t k = 1; k < T; ++k) pool.emplace_back(range, k);
  range(0);
  for (auto& th : pool) th.join();
  for (const auto& m : msg)
    if (!m.empty()) return m;
  return "";
}

std::string validate_graph(int64_t N, const int64_t* rowptr, const int32_t* col) {
  if (N < 1 || N > 0x7fffffffLL) return "N must be in [1, 2^31-1]";
  if (!rowptr) return "rowptr is NULL";
  if (rowptr[0] != 0) return "rowptr[0] must be 0";
  for (int64_t i = 0; i < N; ++i)
    if (rowptr[i + 1] < rowptr[i]) return "rowptr must be non-decreasing";
  const int64_t nnz = rowptr[N];
  if (nnz >= 0x7fffffffLL) return "nnz must be < 2^31";
  if (nnz > 0 && !col) return "col is NULL";
  return for_row_ranges(N, nnz, [&](int64_t r0, int64_t r1) {
    return validate_rows(N, rowptr, col, r0, r1);
  });
}

// Split count of a weight gradient C[M x Nc] summed over the N node rows:
// about two of the CUDA-core kernel's 128 x 128 tiles per SM, at least 256
// rows per split; the tensor-core path splits into at most num_sms / tiles
// slices of its own 256 x 256 tiles.
int64_t wgrad_splits(const cpra_ctx* c, int64_t M, int64_t Nc) {
  const int64_t tiles = ((M + 127) / 128) * ((Nc + 127) / 128);
  int64_t splits = std::max<int64_t>(1, (2 * (int64_t)c->num_sms + tiles - 1) / tiles);
  return std::min<int64_t>(splits, std::max<int64_t>(1, c->N / 256));
}
size_t wgrad_part_floats(const cpra_ctx* c, int64_t M, int64_t Nc) {
  const int64_t tc_tiles = ((M + 255) / 256) * ((Nc + 255) / 256);
  const int64_t tc = std::max<int64_t>(1, (int64_t)c->num_sms / tc_tiles);
  return (size_t)(M * Nc * std::max(wgrad_splits(c, M, Nc), tc));
}

// Carves every device buffer; with base == nullptr only sizes the layout.
size_t carve(cpra_ctx* c, void* base) {
  Carver cv(base);
  const int64_t N = c->N;
  const size_t act = c->act_dt == DT_BF16 ? 2 : 4;
  c->rowptr = cv.take<int>(N + 1);
  c->col = cv.take<int>(std::max<int64_t>(c->nnz, 1));
  c->inv_deg = cv.take<float>(N);
  c->lambda_d = cv.take<float>(c->S);
  c->theta = cv.take<float>(c->nparam);
  c->theta_m = cv.take<float>(c->nparam);
  c->theta_v = cv.take<float>(c->nparam);
  c->grad = cv.take<float>(c->nparam);
  c->X0m = cv.take<float>(N * c->H0);
  c->X0_m = cv.take<float>(N * c->H0);
  c->X0_v = cv.take<float>(N * c->H0);
  c->gX0 = cv.take<float>(N * c->H0);
  c->XM = cv.take<char>((size_t)N * 2 * c->H0 * act);
  c->HM = cv.take<char>((size_t)N * 2 * c->H1 * act);
  c->P = cv.take<float>((size_t)N * c->S_pad);
  c->GZ2 = cv.take<char>((size_t)N * c->S_pad * act);
  if (c->recompute) {
    // The layer activations [H1|M2] and [X0|M1] are dead by the time the
    // backward writes the same-shaped gradient blocks (layer-2 weight
    // gradient first, layer-1 weight gradient before dG_X0), so each pair
    // shares one block; of H1 the layer-1 adjoint needs only its ReLU
    // mask, which the layer-1 GEMM's epilogue writes as bits.
    c->GHM = c->HM;
    c->GXM = c->XM;
    c->relu_bits = cv.take<uint16_t>((size_t)N * (c->H1 / 16));
  } else {
    c->GHM = cv.take<char>((size_t)N * 2 * c->H1 * act);
    c->GXM = cv.take<char>((size_t)N * 2 * c->H0 * act);
  }
  c->xbits = cv.take<uint32_t>((size_t)N * c->W);
  c->pstride = loss_pstride(c->S);
  c->loss_part = cv.take<float>((size_t)kLossMaxGrid * c->pstride);
  c->terms = cv.take<float>(4 * (size_t)c->S + 1);
  c->counters = cv.take<unsigned long long>(2 * (size_t)c->S + 2);  // + the last-block ticket
  c->eval_rec = cv.take<cpra_shot_eval>(c->S);
  c->ham_d = cv.take<long long>(1);
  c->colsum_part = cv.take<float>((size_t)kLossMaxGrid * c->H1);
  // split-K partials: room for the split count either weight-gradient path
  // picks (wgrad_splits) for the larger of the two gradients
  c->wg_part_floats = std::max(wgrad_part_floats(c, c->S_pad, 2 * c->H1),
                               wgrad_part_floats(c, c->H1, 2 * c->H0));
  c->wg_part = cv.take<float>(c->wg_part_floats);
  c->err_flag = cv.take<int>(4);
  c->es = cv.take<EarlyStopState>(1);
  if (c->wmis) {
    c->w_d = cv.take<float>((size_t)N * c->S_pad);
    c->wv_part = cv.take<double>((size_t)kWvBlocks * c->S);
    c->wvalue = cv.take<double>(c->S);
  } else {
    c->w_d = nullptr;
    c->wv_part = nullptr;
    c->wvalue = nullptr;
  }
  c->sc = cv.take<StepScalars>(1);
  c->W1s = cv.take<uint16_t>((size_t)c->H1 * 2 * c->H0);
  c->W1t = cv.take<uint16_t>((size_t)c->H1 * 2 * c->H0);
  c->W2s = cv.take<uint16_t>((size_t)c->S_pad * 2 * c->H1);
  c->W2t = cv.take<uint16_t>((size_t)c->S_pad * 2 * c->H1);
  if (c->use_tc3) {
    const size_t w1 = (size_t)c->H1 * 2 * c->H0, w2 = (size_t)c->S_pad * 2 * c->H1;
    for (int k = 0; k < 3; ++k) {
      c->W1p[k] = cv.take<float>(w1);
      c->W1tp[k] = cv.take<float>(w1);
      c->W2p[k] = cv.take<float>(w2);
      c->W2tp[k] = cv.take<float>(w2);
    }
  }
  return cv.off + kAlign;
}

void set_dims(cpra_ctx* c, int64_t N, int64_t nnz, const cpra_config* cfg) {
  c->N = N;
  c->nnz = nnz;
  c->S = cfg->S;
  c->S_pad = round_up(cfg->S, 16);
  c->W = (cfg->S + 31) / 32;
  c->H0 = cfg->H0;
  c->H1 = cfg->H1;
  c->act_dt = cfg->precision == CPRA_BF16 ? DT_BF16 : DT_F32;
  // the split-TF32 engine of the FP32 form (its weight shadows are part of
  // the workspace; tc_prepare at init may still turn it off)
  c->use_tc3 = (c->act_dt == DT_F32) && cfg->fp32_engine == CPRA_FP32_TENSOR && tc_available();
  c->nparam = layout_of(cfg->H0, cfg->H1, cfg->S).total;
  c->recompute = cfg->recompute != 0;
  c->wmis = cfg->problem == CPRA_WMIS;
}

// ---------------------------------------------------------------- profiling
// NVTX ranges in the "cpra" domain: one per ABI call that launches work and
// one per kernel region of a step (named as cpra_kernel_name names them), so
// that a timeline profiler shows the step's structure.  Without a profiler
// attached a range costs an indirect call.  A captured step (cpra_steps)
// opens its kernel ranges once, while it is captured, not on each replay.
nvtxDomainHandle_t nvtx_domain() {
  static nvtxDomainHandle_t d = nvtxDomainCreateA("cpra");
  return d;
}

struct NvtxRange {
  explicit NvtxRange(const char* name) {
    nvtxEventAttributes_t a;
    std::memset(&a, 0, sizeof(a));
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    nvtxDomainRangePushEx(nvtx_domain(), &a);
  }
  ~NvtxRange() { nvtxDomainRangePop(nvtx_domain()); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

struct Region {
  NvtxRange range;
  cpra_ctx* c;
  int id;
  size_t slot = (size_t)-1;
  Region(cpra_ctx* ctx, int kid) : range(kKernelNames[kid]), c(ctx), id(kid) {
    if (!c->prof || c->capturing) return;
    if (c->prof_used == c->prof_ring.size()) {
      // flush: synchronise and accumulate
      cudaStreamSynchronize(c->stream);
      for (size_t k = 0; k < c->prof_used; ++k) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->prof_ring[k].a, c->prof_ring[k].b) == cudaSuccess) {
          c->prof_ms[c->prof_ring[k].id] += ms;
          c->prof_n[c->prof_ring[k].id] += 1;
        }
      }
      c->prof_used = 0;
    }
    slot = c->prof_used++;
    c->prof_ring[slot].id = id;
    cudaEventRecord(c->prof_ring[slot].a, c->stream);
  }
  ~Region() {
    if (slot != (size_t)-1) cudaEventRecord(c->prof_ring[slot].b, c->stream);
  }
};

float gamma_at(const cpra_config& cfg, int64_t t);

// One JSON line of the metrics log per evaluation: the step index t, gamma_t,
// the steps since the previous evaluation and their wall time (with this
// evaluation), the time since the solve began, the step's loss terms per
// shot and Psi, the rounded shots' objective, violations and value, and
// sum_i k_i (S - k_i).
cpra_status write_metrics(cpra_ctx* c, int64_t t, int64_t n_steps, double seconds, double elapsed,
                          const cpra_shot_eval* rec, int64_t ham) {
  const int S = c->S;
  std::vector<float> terms(3 * (size_t)S + 1);
  cpra_status st = cuda_check(c, cudaMemcpyAsync(terms.data(), c->terms, sizeof(float) * terms.size(),
                                                 cudaMemcpyDeviceToHost, c->stream),
                              "metrics terms readback");
  if (st == CPRA_OK) st = cuda_check(c, cudaStreamSynchronize(c->stream), "metrics sync");
  if (st != CPRA_OK) return st;
  FILE* f = c->metrics;
  std::fprintf(f, "{\"t\": %lld, \"gamma\": %.9g, \"steps\": %lld, \"seconds\": %.6f, "
               "\"elapsed\": %.6f, \"psi\": %.9g, \"pair_hamming\": %lld",
               (long long)t, (double)gamma_at(c->cfg, t), (long long)n_steps, seconds, elapsed,
               (double)terms[3 * (size_t)S], (long long)ham);
  const char* names[3] = {"cost", "pen", "ann"};
  for (int k = 0; k < 3; ++k) {
    std::fprintf(f, ", \"%s\": [", names[k]);
    for (int s = 0; s < S; ++s)
      std::fprintf(f, s ? ", %.9g" : "%.9g", (double)terms[(size_t)k * S + s]);
    std::fputc(']', f);
  }
  std::fputs(", \"objective\": [", f);
  for (int s = 0; s < S; ++s) std::fprintf(f, s ? ", %lld" : "%lld", (long long)rec[s].objective);
  std::fputs("], \"violations\": [", f);
  for (int s = 0; s < S; ++s) std::fprintf(f, s ? ", %lld" : "%lld", (long long)rec[s].violations);
  std::fputs("], \"value\": [", f);
  for (int s = 0; s < S; ++s) std::fprintf(f, s ? ", %.17g" : "%.17g", rec[s].value);
  std::fputs("]}\n", f);
  if (std::fflush(f) != 0 || std::ferror(f)) return fail(c, CPRA_EINVAL, "metrics log write failed");
  return CPRA_OK;
}

void refresh_shadows(cpra_ctx* c) {
  if (c->act_dt == DT_BF16) {
    weight_shadows_launch(c->theta, c->H0, c->H1, c->S, c->S_pad, c->W1s, c->W1t, c->W2s,
                          c->W2t, c->stream);
    c->launches += 1;
  } else if (c->use_tc3) {
    weight_split_launch(c->theta, c->H0, c->H1, c->S, c->S_pad, c->W1p, c->W1tp, c->W2p, c->W2tp,
                        c->stream);
    c->launches += 1;
  }
}

void refresh_emb_shadow(cpra_ctx* c) {
  copy_rows_launch(c->N, c->H0, c->X0m, c->XM, 2 * c->H0, c->act_dt, c->stream);
  c->launches += 1;
}

// Early-stopping state: reset, and read back (fixing the host's Adam step
// count, which runs ahead of the device once the parameters froze).
void reset_early_stop(cpra_ctx* c) {
  EarlyStopState h{};
  h.stop_step = -1;
  cudaMemcpyAsync(c->es, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream);
  cudaStreamSynchronize(c->stream);
}
cpra_status read_early_stop(cpra_ctx* c, EarlyStopState* h) {
  cudaError_t e = cudaMemcpyAsync(h, c->es, sizeof(*h), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return CPRA_ECUDA;
  if (h->stopped) c->opt_steps = h->updates_at_stop;
  return CPRA_OK;
}
bool es_on(const cpra_ctx* c) { return c->cfg.es_patience > 0 || c->cfg.es_ann_below > 0.f; }
const int* halt_flag(const cpra_ctx* c) { return es_on(c) ? &c->es->stopped : nullptr; }

float gamma_at(const cpra_config& cfg, int64_t t) {
  if (cfg.schedule_steps <= 1) return cfg.gamma1;
  const int64_t tt = std::min<int64_t>(std::max<int64_t>(t, 0), cfg.schedule_steps - 1);
  return (float)((double)cfg.gamma0 +
                 ((double)cfg.gamma1 - (double)cfg.gamma0) * (double)tt /
                     (double)(cfg.schedule_steps - 1));
}

size_t act_bytes(const cpra_ctx* c) { return c->act_dt == DT_BF16 ? 2 : 4; }
char* act_off(void* base, int64_t elems, const cpra_ctx* c) {
  return static_cast<char*>(base) + elems * (int64_t)act_bytes(c);
}

// Dense layer dispatch: tensor cores (BF16 form) or CUDA cores.
void dense(cpra_ctx* c, const GemmArgs& g0) {
  GemmArgs g = g0;
  g.err_flag = c->err_flag;
  if (g.B_lo) {  // split-TF32 operands, accepted by tc3_gemm_supported at the call site
    c->launches += tc3_gemm_launch(g, c->num_sms, c->stream);
    return;
  }
  if (c->use_tc && tc_gemm_supported(g)) {
    c->launches += tc_gemm_launch(g, c->num_sms, c->stream);
  } else {
    gemm_simt_launch(g, c->stream);
    c->launches += 1;
  }
}

// FP32 form: the same product with the weights' split-TF32 parts (hi, mid,
// lo; K-major, row pitch ldb) when the tensor-core kernel takes this shape;
// g keeps its CUDA-core form otherwise.
void use_split_tf32(const cpra_ctx* c, GemmArgs& g, float* const* parts, int64_t K, int64_t ldb) {
  if (!c->use_tc3) return;
  GemmArgs t = g;
  t.B = parts[0];
  t.B_mid = parts[1];
  t.B_lo = parts[2];
  t.K = K;
  t.ldb = ldb;
  t.db = DT_F32;
  t.b_kmajor = 1;
  if (tc3_gemm_supported(t)) g = t;
}

// Weight gradient C[M x Nc] = A^T B over K = N rows, split-K with a fixed-
// order reduction into dst (row stride ldo).
void wgrad(cpra_ctx* c, const void* A, int64_t lda, int M, const void* B, int64_t ldb, int Nc,
           float* dst, int64_t ldo) {
  GemmArgs g;
  g.M = M;
  g.Nc = Nc;
  g.K = c->N;
  g.A = A;
  g.lda = lda;
  g.da = c->act_dt;
  g.a_kmajor = 0;
  g.B = B;
  g.ldb = ldb;
  g.db = c->act_dt;
  g.b_kmajor = 0;
  g.epi = EPI_PARTIAL;
  g.out0 = c->wg_part;
  g.ld0 = Nc;
  int64_t splits = wgrad_splits(c, M, Nc);
  const int64_t cap = (int64_t)(c->wg_part_floats / ((size_t)M * Nc));
  splits = std::min<int64_t>(splits, std::max<int64_t>(1, cap));
  g.splits = (int)splits;
  g.err_flag = c->err_flag;
  if (c->use_tc && tc_wgrad_supported(g)) {
    c->launches += tc_wgrad_launch(g, c->num_sms, c->wg_part_floats, dst, ldo, c->stream);
    return;
  }
  gemm_simt_launch(g, c->stream);
  splitk_reduce(c->wg_part, g.splits, M, Nc, Nc, dst, ldo, c->stream);
  c->launches += 2;
}

// On the matching constraint graph an aggregation reads line sums of its
// operand instead of gathering neighbour rows: form them first.
void use_line_sums(cpra_ctx* c, SpmmArgs& a) {
  if (!c->line_agg) return;
  dbm_line_sums_launch(c->dbm.N1, c->dbm.N2, a.H, a.X, a.ldx, a.dx, c->line_R, c->line_K, c->ldl,
                       c->stream);
  a.line_r = c->line_R;
  a.line_k = c->line_K;
  a.line_n2 = c->dbm.N2;
  a.ldl = c->ldl;
  c->launches += 1;
}

cpra_status run_forward_and_loss(cpra_ctx* c, float gamma, bool do_loss,
                                 const StepScalars* sc = nullptr) {
  const bool dbm = c->cfg.problem == CPRA_DBM;
  if (dbm && !c->dbm_mem) return fail(c, CPRA_ESTATE, "DBM context: call cpra_set_dbm first");
  const int64_t N = c->N;
  const int H0 = c->H0, H1 = c->H1;
  const int max_grid = c->num_sms * 8;
  const Layout L = layout_of(H0, H1, c->S);
  {  // M1 = mean_agg(X0)
    Region r(c, K_SPMM_AGG1);
    SpmmArgs a;
    a.N = N; a.H = H0; a.rowptr = c->rowptr; a.col = c->col; a.inv_deg = c->inv_deg;
    a.X = c->XM; a.ldx = 2 * H0; a.Y = act_off(c->XM, H0, c); a.ldy = 2 * H0; a.mean = 1;
    a.dx = c->act_dt; a.dy = c->act_dt; a.err_flag = c->err_flag;
    use_line_sums(c, a);
    if (spmm_launch(a, c->num_sms, max_grid, c->stream) < 0) return CPRA_EINVAL;
    c->launches += 1;
  }
  {  // H1 = relu([X0|M1] Wcat1^T + b1)
    Region r(c, K_GEMM_L1);
    GemmArgs g;
    g.M = N; g.Nc = H1; g.K = 2 * H0;
    g.A = c->XM; g.lda = 2 * H0; g.da = c->act_dt; g.a_kmajor = 1;
    if (c->act_dt == DT_BF16) { g.B = c->W1s; g.db = DT_BF16; }
    else { g.B = c->theta + L.wcat1; g.db = DT_F32; }
    g.ldb = 2 * H0; g.b_kmajor = 1;
    g.epi = EPI_BIAS_RELU; g.bias = c->theta + L.b1;
    g.out0 = c->HM; g.ld0 = 2 * H1; g.d0 = c->act_dt; g.n_valid = H1;
    // recompute: H1's block is overwritten by the backward, so its ReLU mask
    // (all the layer-1 adjoint needs of it) is kept as bits, 1/16 of H1
    if (c->recompute) { g.out1 = c->relu_bits; g.ld1 = H1 / 16; }
    if (c->act_dt == DT_F32) use_split_tf32(c, g, c->W1p, 2 * H0, 2 * H0);
    dense(c, g);
  }
  {  // M2 = mean_agg(H1)
    Region r(c, K_SPMM_AGG2);
    SpmmArgs a;
    a.N = N; a.H = H1; a.rowptr = c->rowptr; a.col = c->col; a.inv_deg = c->inv_deg;
    a.X = c->HM; a.ldx = 2 * H1; a.Y = act_off(c->HM, H1, c); a.ldy = 2 * H1; a.mean = 1;
    a.dx = c->act_dt; a.dy = c->act_dt; a.err_flag = c->err_flag;
    use_line_sums(c, a);
    if (spmm_launch(a, c->num_sms, max_grid, c->stream) < 0) return CPRA_EINVAL;
    c->launches += 1;
  }
  {  // P = sigmoid([H1|M2] Wcat2^T + b2)
    Region r(c, K_GEMM_L2);
    GemmArgs g;
    g.M = N; g.Nc = c->S_pad; g.K = 2 * H1;
    g.A = c->HM; g.lda = 2 * H1; g.da = c->act_dt; g.a_kmajor = 1;
    if (c->act_dt == DT_BF16) { g.B = c->W2s; g.db = DT_BF16; }
    else { g.B = c->theta + L.wcat2; g.db = DT_F32; }
    g.ldb = 2 * H1; g.b_kmajor = 1;
    g.epi = EPI_BIAS_SIGMOID; g.bias = c->theta + L.b2;
    g.out0 = c->P; g.ld0 = c->S_pad; g.d0 = DT_F32; g.n_valid = c->S;
    if (c->init_logits) { g.addend = c->init_logits; g.ld_add = c->S_pad; g.d_add = c->act_dt; }
    if (c->act_dt == DT_F32) use_split_tf32(c, g, c->W2p, 2 * H1, 2 * H1);
    dense(c, g);
  }
  if (dbm && do_loss) {  // matching line sums R, K, T, U and the per-shot coefficients
    Region r(c, K_DBM_SUMS);
    dbm_sums_launch(c->dbm, c->S, c->P, c->S_pad, c->stream);
    c->launches += 2;
  }
  int grid = 0;
  {  // fused SpMM + loss + rounding bits
    Region r(c, K_LOSS);
    LossArgs a;
    a.N = N; a.S = c->S; a.ldp = c->S_pad; a.ldg = c->S_pad;
    a.rowptr = c->rowptr; a.col = c->col; a.P = c->P; a.lambda = c->lambda_d;
    // weighted MIS: MIS with weights
    a.problem = dbm ? 2 : c->cfg.problem == CPRA_MAXCUT ? 1 : 0;
    a.dbm = c->dbm;
    a.w = c->w_d; a.ldw = c->S_pad;
    a.ew = c->ew_d; a.wdeg = c->wdeg_d;
    a.alpha = c->cfg.alpha; a.div_kind = c->cfg.diversity_kind;
    a.grad_kind = 0; a.gamma = gamma; a.sc = do_loss ? sc : nullptr; a.nu = c->cfg.nu;
    a.G = c->GZ2; a.dg = c->act_dt; a.xbits = c->xbits;
    a.partials = c->loss_part; a.pstride = c->pstride; a.err_flag = c->err_flag;
    a.do_loss = do_loss ? 1 : 0;
    grid = loss_launch(a, c->num_sms * 4, c->stream);
    c->launches += 1;
  }
  if (do_loss) {  // per-shot loss terms, db2
    Region r(c, K_LOSS_FIN);
    colsum_finalize(c->loss_part, grid, c->pstride, 4 * c->S + 1, c->terms, c->grad + L.b2,
                    3 * c->S + 1, c->S, c->err_flag, c->stream);
    c->launches += 1;
  }
  {  // exact integer evaluation of the rounded shots
    Region r(c, K_EVAL);
    // shot values first (they read only the bits): the evaluation's last
    // block puts them into the records
    if (c->w_d) {  // weighted MIS: the value of each shot in weight units
      weighted_value_launch(N, c->S, c->xbits, c->w_d, c->S_pad, c->wv_part, kWvBlocks,
                            c->wvalue, c->stream);
      c->launches += 2;
    }
    if (c->ew_d) {  // weighted MaxCut: the cut weight of each shot
      weighted_cut_launch(N, c->S, c->rowptr, c->col, c->ew_d, c->xbits, c->cut_part, kWvBlocks,
                          c->cutw, c->stream);
      c->launches += 2;
    }
    if (dbm) {  // matchings: line counts, constraints and rewards (the set size and
                // pair-Hamming counters of the evaluation are problem-independent;
                // the pair counts come from the line counts, so no edges here)
      cudaMemsetAsync(c->counters, 0, (2 * (size_t)c->S + 2) * sizeof(unsigned long long),
                      c->stream);
      eval_bits_launch(N, c->S, c->rowptr, c->col, c->xbits, 2, c->counters, c->num_sms,
                       c->stream);
      dbm_eval_launch(c->dbm, c->S, c->xbits, c->counters, c->eval_rec, c->ham_d, c->stream);
      c->launches += 3;
    } else {
      // the counters are zero here (set at creation, reset by the last block
      // of every evaluation), and the launch writes the records itself
      EvalFinalize fin;
      fin.lambda = c->lambda_d;
      fin.wvalue = c->w_d ? c->wvalue : c->ew_d ? c->cutw : nullptr;
      fin.records = c->eval_rec;
      fin.ham = c->ham_d;
      eval_bits_launch(N, c->S, c->rowptr, c->col, c->xbits,
                       c->cfg.problem == CPRA_MAXCUT ? 1 : 0, c->counters, c->num_sms, c->stream,
                       &fin);
      c->launches += 1;
    }
  }
  c->have_eval = true;
  return CPRA_OK;
}

// Adam bias corrections for the next optimiser step t = opt_steps + 1.
void adam_bias(const cpra_ctx* c, float* bc1, float* bc2) {
  const double t = (double)(c->opt_steps + 1);
  *bc1 = (float)(1.0 - std::pow((double)c->cfg.beta1, t));
  *bc2 = (float)(1.0 - std::pow((double)c->cfg.beta2, t));
}

// Adjoint of the last forward: dR/dtheta into c->grad and, with emb_grad,
// dR/dh^0 into c->gX0.  With fuse_adam the last aggregation also takes the
// Adam step on the embeddings (and stores dR/dh^0 only when keep_emb_grad).
cpra_status run_backward(cpra_ctx* c, bool emb_grad, bool fuse_adam = false) {
  const int64_t N = c->N;
  const int H0 = c->H0, H1 = c->H1;
  const int max_grid = c->num_sms * 8;
  const Layout L = layout_of(H0, H1, c->S);
  const bool bf = c->act_dt == DT_BF16;
  // The layer-2 weight gradient goes first: with recompute the gradient block
  // [G_H1a | G_M2/deg] below overwrites [H1|M2].
  {
    Region r(c, K_WGRAD2);  // dWcat2 = G_Z2^T [H1|M2]
    wgrad(c, c->GZ2, c->S_pad, c->S, c->HM, 2 * H1, 2 * H1, c->grad + L.wcat2, 2 * H1);
  }
  if (!c->cfg.train_encoder) return CPRA_OK;  // head only: db2 and dWcat2 are all it needs
  {  // [G_H1a | G_M2/deg] = G_Z2 Wcat2
    Region r(c, K_GEMM_DGRAD2);
    GemmArgs g;
    g.M = N; g.Nc = 2 * H1;
    g.A = c->GZ2; g.lda = c->S_pad; g.da = c->act_dt; g.a_kmajor = 1;
    if (bf) { g.K = c->S_pad; g.B = c->W2t; g.ldb = c->S_pad; g.db = DT_BF16; g.b_kmajor = 1; }
    else { g.K = c->S; g.B = c->theta + L.wcat2; g.ldb = 2 * H1; g.db = DT_F32; g.b_kmajor = 0; }
    g.epi = EPI_SPLIT; g.split = H1;
    g.out0 = c->GHM; g.ld0 = 2 * H1; g.d0 = c->act_dt;
    g.out1 = act_off(c->GHM, H1, c); g.ld1 = 2 * H1; g.d1 = c->act_dt;
    g.row_scale = c->inv_deg; g.n_valid = 2 * H1;
    // (the split-TF32 form reads G_Z2 over its padded width: pad columns are 0)
    if (!bf) use_split_tf32(c, g, c->W2tp, c->S_pad, c->S_pad);
    dense(c, g);
  }
  {  // G_Z1 = (G_H1a + sum_j G_M2_j/deg_j) * 1[H1 > 0], db1 = colsum(G_Z1)
    Region r(c, K_SPMM_BWD2);
    SpmmArgs a;
    a.N = N; a.H = H1; a.rowptr = c->rowptr; a.col = c->col; a.inv_deg = c->inv_deg;
    a.X = act_off(c->GHM, H1, c); a.ldx = 2 * H1;
    a.add = c->GHM; a.ldadd = 2 * H1;
    if (c->recompute) { a.mask_bits = c->relu_bits; a.ldmb = H1 / 16; }
    else { a.mask = c->HM; a.ldm = 2 * H1; }
    a.Y = c->GHM; a.ldy = 2 * H1; a.mean = 0;
    a.dx = c->act_dt; a.dy = c->act_dt; a.err_flag = c->err_flag;
    a.colsum_partials = c->colsum_part;
    use_line_sums(c, a);
    const int grid = spmm_launch(a, c->num_sms, std::min(max_grid, kLossMaxGrid), c->stream);
    if (grid < 0) return CPRA_EINVAL;
    colsum_finalize(c->colsum_part, grid, H1, H1, c->grad + L.b1, nullptr, 0, 0, nullptr,
                    c->stream);
    c->launches += 2;
  }
  {
    Region r(c, K_WGRAD1);  // dWcat1 = G_Z1^T [X0|M1]
    wgrad(c, c->GHM, 2 * H1, H1, c->XM, 2 * H0, 2 * H0, c->grad + L.wcat1, 2 * H0);
  }
  if (emb_grad) {
    {  // [G_X0a | G_M1/deg] = G_Z1 Wcat1
      Region r(c, K_GEMM_DGRAD1);
      GemmArgs g;
      g.M = N; g.Nc = 2 * H0; g.K = H1;
      g.A = c->GHM; g.lda = 2 * H1; g.da = c->act_dt; g.a_kmajor = 1;
      if (bf) { g.B = c->W1t; g.ldb = H1; g.db = DT_BF16; g.b_kmajor = 1; }
      else { g.B = c->theta + L.wcat1; g.ldb = 2 * H0; g.db = DT_F32; g.b_kmajor = 0; }
      g.epi = EPI_SPLIT; g.split = H0;
      g.out0 = c->GXM; g.ld0 = 2 * H0; g.d0 = c->act_dt;
      g.out1 = act_off(c->GXM, H0, c); g.ld1 = 2 * H0; g.d1 = c->act_dt;
      g.row_scale = c->inv_deg; g.n_valid = 2 * H0;
      if (!bf) use_split_tf32(c, g, c->W1tp, H1, H1);
      dense(c, g);
    }
    {  // dX0 = G_X0a + sum_j G_M1_j/deg_j  [then Adam on h^0]
      Region r(c, fuse_adam ? K_ADAM_EMB : K_SPMM_BWD1);
      SpmmArgs a;
      a.N = N; a.H = H0; a.rowptr = c->rowptr; a.col = c->col; a.inv_deg = c->inv_deg;
      a.X = act_off(c->GXM, H0, c); a.ldx = 2 * H0;
      a.add = c->GXM; a.ldadd = 2 * H0;
      a.Y = c->gX0; a.ldy = H0; a.mean = 0;
      if (fuse_adam) {
        a.adam = 1;
        a.halt = halt_flag(c);
        a.sc = c->sc;
        if (!c->cfg.keep_emb_grad) a.Y = nullptr;
        a.emb = c->X0m; a.emb_m = c->X0_m; a.emb_v = c->X0_v;
        a.shadow = c->XM; a.lds = 2 * H0;
        a.lr = c->cfg.lr; a.beta1 = c->cfg.beta1; a.beta2 = c->cfg.beta2;
        a.eps = c->cfg.eps; a.wd = c->cfg.weight_decay;
        adam_bias(c, &a.bc1, &a.bc2);
      }
      a.dx = c->act_dt; a.dy = DT_F32; a.err_flag = c->err_flag;
      use_line_sums(c, a);
    if (spmm_launch(a, c->num_sms, max_grid, c->stream) < 0) return CPRA_EINVAL;
      c->launches += 1;
    }
    // With recompute the gradient block overwrote the embedding copy that
    // the forward reads; the fused update rewrites it, otherwise restore it.
    if (c->recompute && !fuse_adam) refresh_emb_shadow(c);
  }
  return CPRA_OK;
}

// Adam on theta (+ BF16 shadows); the embeddings take their Adam step inside
// the last backward aggregation (run_backward with fuse_adam).
cpra_status run_update(cpra_ctx* c) {
  float bc1, bc2;
  adam_bias(c, &bc1, &bc2);
  {
    Region r(c, K_ADAM);
    // head only: Adam on the trailing [Wcat2 | b2] block; layer 1 keeps its values
    const int64_t off = c->cfg.train_encoder ? 0 : layout_of(c->H0, c->H1, c->S).wcat2;
    adam_launch(c->nparam - off, c->theta + off, c->theta_m + off, c->theta_v + off, c->grad + off,
                c->cfg.lr, c->cfg.beta1,
                c->cfg.beta2, c->cfg.eps, c->cfg.weight_decay, bc1, bc2, halt_flag(c), c->sc,
                c->stream);
    c->launches += 1;
    refresh_shadows(c);
  }
  return CPRA_OK;
}

cpra_status check_err_flag(cpra_ctx* c) {
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_check(c, e, "error-flag readback");
  if (flag & 2) {
    cudaMemsetAsync(c->err_flag, 0, sizeof(int), c->stream);
    return fail(c, CPRA_ETIMEOUT, "a bounded device-side wait gave up (tensor-core pipeline)");
  }
  if (flag & 4) {
    cudaMemsetAsync(c->err_flag, 0, sizeof(int), c->stream);
    return fail(c, CPRA_ECUDA, "a tensor-core GEMM could not be set up (its product is missing)");
  }
  if (flag & 1) {
    cudaMemsetAsync(c->err_flag, 0, sizeof(int), c->stream);
    return fail(c, CPRA_ENUMERIC, "non-finite loss term");
  }
  return CPRA_OK;
}

// Edge weights: MaxCut only, finite, symmetric (A_ij = A_ji for the two CSR
// entries of each edge; columns are sorted, so the reverse entry is found by
// binary search).
std::string validate_edge_weights(int64_t N, const int64_t* rowptr, const int32_t* col,
                                  const float* w, int32_t problem) {
  if (problem != CPRA_MAXCUT) return "edge weights apply to CPRA_MAXCUT only (w must be NULL)";
  return for_row_ranges(N, rowptr[N], [&](int64_t r0, int64_t r1) -> std::string {
    for (int64_t i = r0; i < r1; ++i)
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) {
        if (!std::isfinite(w[e])) return "edge weights must be finite";
        const int32_t j = col[e];
        const int32_t* b = col + rowptr[j];
        const int32_t* f = col + rowptr[j + 1];
        const int32_t* it = std::lower_bound(b, f, static_cast<int32_t>(i));
        if (it == f || *it != i || w[rowptr[j] + (it - b)] != w[e])
          return "edge weights must be symmetric (A_ij == A_ji)";
      }
    return std::string();
  });
}

}  // namespace

// ======================================================================= ABI
extern "C" {

void cpra_config_default(cpra_config* cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->problem = CPRA_MIS;
  cfg->S = 8;
  cfg->H0 = 16;
  cfg->H1 = 16;
  cfg->alpha = 2;
  cfg->precision = CPRA_FP32;
  cfg->recompute = 0;
  cfg->train_embedding = 1;
  cfg->keep_emb_grad = 0;
  cfg->diversity_kind = CPRA_DIV_STD;
  cfg->lambda = nullptr;
  cfg->nu = 0.f;
  cfg->gamma0 = -2.f;
  cfg->gamma1 = 0.1f;
  cfg->schedule_steps = 3000;
  cfg->lr = 1e-3f;
  cfg->beta1 = 0.9f;
  cfg->beta2 = 0.999f;
  cfg->eps = 1e-8f;
  cfg->weight_decay = 0.f;
  cfg->seed = 1;
  cfg->mem_cap_bytes = 0;
  cfg->es_tol = 1e-5f;
  cfg->es_patience = 0;
  cfg->es_ann_below = 0.f;
  cfg->train_encoder = 1;
  cfg->fp32_engine = CPRA_FP32_TENSOR;
}

int64_t cpra_param_count_for(int32_t H0, int32_t H1, int32_t S) {
  return 2 * (int64_t)H1 * H0 + H1 + 2 * (int64_t)S * H1 + S;
}

size_t cpra_workspace_bytes(int64_t N, int64_t nnz, const cpra_config* cfg) {
  if (!validate_config(cfg).empty() || N < 1 || nnz < 0) return 0;
  cpra_ctx tmp;
  tmp.num_sms = device_sm_count();
  set_dims(&tmp, N, nnz, cfg);
  return carve(&tmp, nullptr);
}

cpra_status cpra_init_graph(cpra_ctx** out, int64_t N, const int64_t* rowptr,
                            const int32_t* col, const float* w, const cpra_config* cfg,
                            void* dev_workspace, size_t workspace_bytes, void* cuda_stream) {
  if (!out) return CPRA_EINVAL;
  *out = nullptr;
  cpra_ctx* c = new (std::nothrow) cpra_ctx();
  if (!c) return CPRA_ENOMEM;
  auto bail = [&](cpra_status s) {
    g_init_err = c->err;
    cpra_destroy(c);
    return s;
  };
  std::string msg = validate_config(cfg);
  if (!msg.empty()) { fail(c, CPRA_EINVAL, msg); return bail(CPRA_EINVAL); }
  msg = validate_graph(N, rowptr, col);
  if (!msg.empty()) { fail(c, CPRA_EINVAL, msg); return bail(CPRA_EINVAL); }
  if (w != nullptr) {
    msg = validate_edge_weights(N, rowptr, col, w, cfg->problem);
    if (!msg.empty()) { fail(c, CPRA_EINVAL, msg); return bail(CPRA_EINVAL); }
  }
  c->cfg = *cfg;
  c->num_sms = device_sm_count();
  set_dims(c, N, rowptr[N], cfg);
  c->lambda_h.assign((size_t)c->S, 0.f);
  if (cfg->problem == CPRA_DBM)  // the matching penalty carries its own lambdas
    c->lambda_h.assign((size_t)c->S, 1.f);
  else if (cfg->lambda)
    std::memcpy(c->lambda_h.data(), cfg->lambda, sizeof(float) * c->S);
  c->cfg.lambda = nullptr;
  c->use_tc = (c->act_dt == DT_BF16) && tc_available();

  const size_t need = carve(c, nullptr);
  if (cfg->mem_cap_bytes && need > cfg->mem_cap_bytes) {
    fail(c, CPRA_ENOMEM, "workspace of " + std::to_string(need) + " bytes exceeds mem_cap_bytes");
    return bail(CPRA_ENOMEM);
  }
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cuda_check(c, cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking), "stream") != CPRA_OK)
      return bail(CPRA_ECUDA);
    c->own_stream = true;
  }
  if (dev_workspace) {
    if (workspace_bytes < need) {
      fail(c, CPRA_EINVAL, "workspace too small: need " + std::to_string(need));
      return bail(CPRA_EINVAL);
    }
    c->ws = dev_workspace;
    c->ws_bytes = workspace_bytes;
  } else {
    cudaError_t e = cudaMalloc(&c->ws, need);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(c, CPRA_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
      return bail(CPRA_ENOMEM);
    }
    c->own_ws = true;
    c->ws_bytes = need;
  }
  // align the carve base
  char* base = reinterpret_cast<char*>(
      (reinterpret_cast<uintptr_t>(c->ws) + kAlign - 1) / kAlign * kAlign);
  carve(c, base);

  // graph upload (int32 row pointers, inverse degrees)
  std::vector<int> rp32((size_t)N + 1);
  std::vector<float> invd((size_t)N);
  for (int64_t i = 0; i <= N; ++i) rp32[i] = (int)rowptr[i];
  for (int64_t i = 0; i < N; ++i) {
    const int64_t d = rowptr[i + 1] - rowptr[i];
    invd[i] = d > 0 ? (float)(1.0 / (double)d) : 0.f;
  }
  cudaStream_t st = c->stream;
  cpra_status s = CPRA_OK;
  s = cuda_check(c, cudaMemcpyAsync(c->rowptr, rp32.data(), sizeof(int) * (N + 1), cudaMemcpyHostToDevice, st), "upload rowptr");
  if (s == CPRA_OK && c->nnz > 0)
    s = cuda_check(c, cudaMemcpyAsync(c->col, col, sizeof(int) * c->nnz, cudaMemcpyHostToDevice, st), "upload col");
  if (s == CPRA_OK)
    s = cuda_check(c, cudaMemcpyAsync(c->inv_deg, invd.data(), sizeof(float) * N, cudaMemcpyHostToDevice, st), "upload inv_deg");
  if (s == CPRA_OK)
    s = cuda_check(c, cudaMemcpyAsync(c->lambda_d, c->lambda_h.data(), sizeof(float) * c->S, cudaMemcpyHostToDevice, st), "upload lambda");
  if (s != CPRA_OK) return bail(s);
  std::vector<float> wdeg_h;
  if (w != nullptr) {  // MaxCut edge weights, their weighted degrees (FP64 sums), cut partials
    wdeg_h.assign((size_t)N, 0.f);
    for (int64_t i = 0; i < N; ++i) {
      double t = 0.0;
      for (int64_t e = rowptr[i]; e < rowptr[i + 1]; ++e) t += (double)w[e];
      wdeg_h[i] = (float)t;
    }
    const size_t ew_b = (sizeof(float) * (size_t)c->nnz + 255) / 256 * 256;
    const size_t wd_b = (sizeof(float) * (size_t)N + 255) / 256 * 256;
    const size_t cp_b = sizeof(double) * (size_t)kWvBlocks * c->S;
    cudaError_t e = cudaMalloc(&c->ew_mem, ew_b + wd_b + cp_b + sizeof(double) * c->S);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(c, CPRA_ENOMEM, std::string("cudaMalloc (edge weights): ") + cudaGetErrorString(e));
      return bail(CPRA_ENOMEM);
    }
    char* b = static_cast<char*>(c->ew_mem);
    c->ew_d = reinterpret_cast<float*>(b);
    c->wdeg_d = reinterpret_cast<float*>(b + ew_b);
    c->cut_part = reinterpret_cast<double*>(b + ew_b + wd_b);
    c->cutw = c->cut_part + (size_t)kWvBlocks * c->S;
    if (c->nnz > 0)
      s = cuda_check(c, cudaMemcpyAsync(c->ew_d, w, sizeof(float) * c->nnz, cudaMemcpyHostToDevice, st), "upload w");
    if (s == CPRA_OK)
      s = cuda_check(c, cudaMemcpyAsync(c->wdeg_d, wdeg_h.data(), sizeof(float) * N, cudaMemcpyHostToDevice, st), "upload weighted degrees");
    if (s != CPRA_OK) return bail(s);
  }
  // zero everything that must start at zero (pads included)
  const size_t act = act_bytes(c);
  cudaMemsetAsync(c->theta_m, 0, sizeof(float) * c->nparam, st);
  cudaMemsetAsync(c->theta_v, 0, sizeof(float) * c->nparam, st);
  cudaMemsetAsync(c->grad, 0, sizeof(float) * c->nparam, st);
  cudaMemsetAsync(c->X0_m, 0, sizeof(float) * N * c->H0, st);
  cudaMemsetAsync(c->X0_v, 0, sizeof(float) * N * c->H0, st);
  cudaMemsetAsync(c->gX0, 0, sizeof(float) * N * c->H0, st);
  cudaMemsetAsync(c->P, 0, sizeof(float) * N * c->S_pad, st);
  cudaMemsetAsync(c->GZ2, 0, act * N * c->S_pad, st);
  cudaMemsetAsync(c->err_flag, 0, sizeof(int) * 4, st);
  reset_early_stop(c);
  cudaMemsetAsync(c->terms, 0, sizeof(float) * (4 * c->S + 1), st);
  cudaMemsetAsync(c->counters, 0, sizeof(unsigned long long) * (2 * (size_t)c->S + 2), st);
  if (c->w_d) fill_rows_launch(N, c->S, c->S_pad, 1.f, c->w_d, st);  // weights 1 until set
  // parameters: U(+-1/sqrt(fan_in)) for weights and biases, N(0,1) embeddings
  const Layout L = layout_of(c->H0, c->H1, c->S);
  const uint64_t seed = cfg->seed;
  init_uniform_launch(c->theta + L.wcat1, L.b1 - L.wcat1, 1.f / std::sqrt((float)c->H0), seed, 1, st);
  init_uniform_launch(c->theta + L.b1, c->H1, 1.f / std::sqrt((float)c->H0), seed, 2, st);
  init_uniform_launch(c->theta + L.wcat2, L.b2 - L.wcat2, 1.f / std::sqrt((float)c->H1), seed, 3, st);
  init_uniform_launch(c->theta + L.b2, c->S, 1.f / std::sqrt((float)c->H1), seed, 4, st);
  init_normal_launch(c->X0m, N * c->H0, seed, 5, st);
  c->launches += 5;
  if (c->use_tc || c->use_tc3) {
    std::string tmsg;
    if (!tc_prepare(c->num_sms, &tmsg)) {
      c->use_tc = false;
      c->use_tc3 = false;  // shadows stay carved, unused
    }
  }
  refresh_shadows(c);
  refresh_emb_shadow(c);
  s = cuda_check(c, cudaStreamSynchronize(st), "init");
  if (s == CPRA_OK) s = cuda_check(c, cudaGetLastError(), "init kernels");
  if (s != CPRA_OK) return bail(s);
  *out = c;
  return CPRA_OK;
}

namespace {

// The kernels of one training step after its scalars are in c->sc:
// forward + loss, early-stopping monitor, adjoint with the fused embedding
// update, parameter Adam.  Launches only (no host synchronisation), so the
// sequence can be captured into a CUDA graph.
cpra_status launch_step_body(cpra_ctx* c) {
  cpra_status s = run_forward_and_loss(c, 0.f, true, c->sc);
  if (s != CPRA_OK) return s;
  if (es_on(c)) {
    early_stop_launch(c->terms, c->cfg.problem != CPRA_MAXCUT ? c->lambda_d : nullptr, c->S,
                      c->cfg.es_tol, c->cfg.es_patience, c->cfg.es_ann_below, c->sc, c->es,
                      c->stream);
    c->launches += 1;
  }
  const bool emb = c->cfg.train_embedding != 0 && c->cfg.train_encoder != 0;
  s = run_backward(c, emb, /*fuse_adam=*/emb);
  if (s != CPRA_OK) return s;
  return run_update(c);
}

void launch_step_scalars(cpra_ctx* c, bool from_device, int64_t t) {
  step_scalars_launch(c->sc, from_device ? 1 : 0, (long long)t, (long long)c->opt_steps,
                      c->cfg.gamma0, c->cfg.gamma1, (long long)c->cfg.schedule_steps,
                      c->cfg.beta1, c->cfg.beta2, c->stream);
  c->launches += 1;
}

void drop_graph(cpra_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->gexec = nullptr;
  c->graph = nullptr;
}

// Captures one step (scalars read from the device counters + body) on the
// context stream.
cpra_status capture_step(cpra_ctx* c) {
  drop_graph(c);
  const int64_t before = c->launches;
  c->capturing = true;
  cudaError_t e = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  cpra_status s = CPRA_OK;
  if (e == cudaSuccess) {
    launch_step_scalars(c, true, 0);
    s = launch_step_body(c);
    e = cudaStreamEndCapture(c->stream, &c->graph);
  }
  c->capturing = false;
  c->graph_launches = c->launches - before;
  c->launches = before;
  if (s != CPRA_OK) {
    drop_graph(c);
    return s;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&c->gexec, c->graph, 0);
  if (e != cudaSuccess) {
    drop_graph(c);
    return cuda_check(c, e, "step graph capture");
  }
  return CPRA_OK;
}

}  // namespace

cpra_status cpra_step(cpra_ctx* c, int64_t t, float* loss_terms_out) {
  NvtxRange range("cpra_step");
  if (!c) return CPRA_EINVAL;
  c->fwd_valid = false;
  launch_step_scalars(c, false, t);
  cpra_status s = launch_step_body(c);
  if (s != CPRA_OK) return s;
  c->opt_steps += 1;
  c->have_eval = true;
  s = cuda_check(c, cudaGetLastError(), "step kernels");
  if (s != CPRA_OK) return s;
  if (loss_terms_out) {
    s = cuda_check(c, cudaMemcpyAsync(loss_terms_out, c->terms, sizeof(float) * (3 * c->S + 1),
                                      cudaMemcpyDeviceToHost, c->stream), "terms readback");
    if (s != CPRA_OK) return s;
    s = check_err_flag(c);
    if (s != CPRA_OK) return s;
  }
  return CPRA_OK;
}

cpra_status cpra_steps(cpra_ctx* c, int64_t t0, int64_t n) {
  NvtxRange range("cpra_steps");
  if (!c || n < 0) return c ? fail(c, CPRA_EINVAL, "cpra_steps: n < 0") : CPRA_EINVAL;
  if (n == 0) return CPRA_OK;
  // the first step runs directly: it sets the device counters to (t0 + 1,
  // updates + 1) that the replays advance from
  cpra_status s = cpra_step(c, t0, nullptr);
  if (s != CPRA_OK || n == 1) return s;
  if (!c->gexec) {
    s = capture_step(c);
    if (s != CPRA_OK) return s;
  }
  for (int64_t k = 1; k < n; ++k) {
    cudaError_t e = cudaGraphLaunch(c->gexec, c->stream);
    if (e != cudaSuccess) return cuda_check(c, e, "step graph launch");
  }
  c->launches += (n - 1) * c->graph_launches;
  c->opt_steps += n - 1;
  c->fwd_valid = false;
  c->have_eval = true;
  return cuda_check(c, cudaGetLastError(), "step graph");
}
cpra_status cpra_forward(cpra_ctx* c, const float* theta_dev, const float* emb_dev, float gamma,
                         float* terms_dev) {
  NvtxRange range("cpra_forward");
  if (!c || !theta_dev || !emb_dev || !terms_dev)
    return c ? fail(c, CPRA_EINVAL, "cpra_forward: NULL pointer") : CPRA_EINVAL;
  if (!std::isfinite(gamma)) return fail(c, CPRA_EINVAL, "cpra_forward: gamma must be finite");
  cudaStream_t st = c->stream;
  cpra_status s = cuda_check(c, cudaMemcpyAsync(c->theta, theta_dev, sizeof(float) * c->nparam,
                                                cudaMemcpyDeviceToDevice, st), "theta");
  if (s == CPRA_OK)
    s = cuda_check(c, cudaMemcpyAsync(c->X0m, emb_dev, sizeof(float) * c->N * c->H0,
                                      cudaMemcpyDeviceToDevice, st), "embeddings");
  if (s != CPRA_OK) return s;
  refresh_shadows(c);
  refresh_emb_shadow(c);
  s = run_forward_and_loss(c, gamma, true);
  if (s != CPRA_OK) return s;
  total_loss_launch(c->terms, c->cfg.problem != CPRA_MAXCUT ? c->lambda_d : nullptr, c->S, gamma,
                    c->cfg.nu, terms_dev, st);
  c->launches += 1;
  c->fwd_valid = true;
  return cuda_check(c, cudaGetLastError(), "forward kernels");
}

cpra_status cpra_backward(cpra_ctx* c, float scale, float* grad_theta_dev, float* grad_emb_dev) {
  NvtxRange range("cpra_backward");
  if (!c || !grad_theta_dev) return c ? fail(c, CPRA_EINVAL, "cpra_backward: NULL pointer") : CPRA_EINVAL;
  if (!c->fwd_valid) return fail(c, CPRA_ESTATE, "cpra_backward: no cpra_forward to differentiate");
  cpra_status s = run_backward(c, grad_emb_dev != nullptr);
  if (s != CPRA_OK) return s;
  scale_copy_launch(c->nparam, scale, c->grad, grad_theta_dev, c->stream);
  c->launches += 1;
  if (grad_emb_dev) {
    scale_copy_launch(c->N * c->H0, scale, c->gX0, grad_emb_dev, c->stream);
    c->launches += 1;
  }
  return cuda_check(c, cudaGetLastError(), "backward kernels");
}

cpra_status cpra_round_eval(cpra_ctx* c, cpra_shot_eval* out, int64_t* pair_hamming_sum,
                            uint32_t* x_bits_out) {
  NvtxRange range("cpra_round_eval");
  if (!c || !out) return c ? fail(c, CPRA_EINVAL, "out is NULL") : CPRA_EINVAL;
  if (!c->have_eval) {
    cpra_status s = run_forward_and_loss(c, gamma_at(c->cfg, 0), false);
    if (s != CPRA_OK) return s;
  }
  cudaStream_t st = c->stream;
  cpra_status s = cuda_check(c, cudaMemcpyAsync(out, c->eval_rec, sizeof(cpra_shot_eval) * c->S,
                                                cudaMemcpyDeviceToHost, st), "eval readback");
  if (s == CPRA_OK && pair_hamming_sum)
    s = cuda_check(c, cudaMemcpyAsync(pair_hamming_sum, c->ham_d, sizeof(int64_t),
                                      cudaMemcpyDeviceToHost, st), "hamming readback");
  if (s == CPRA_OK && x_bits_out)
    s = cuda_check(c, cudaMemcpyAsync(x_bits_out, c->xbits, sizeof(uint32_t) * c->N * c->W,
                                      cudaMemcpyDeviceToHost, st), "bits readback");
  if (s == CPRA_OK) s = cuda_check(c, cudaStreamSynchronize(st), "eval sync");
  return s;
}

cpra_status cpra_set_metrics_log(cpra_ctx* c, const char* path) {
  if (!c) return CPRA_EINVAL;
  if (c->metrics) std::fclose(c->metrics);
  c->metrics = nullptr;
  if (!path) return CPRA_OK;
  c->metrics = std::fopen(path, "a");
  if (!c->metrics) return fail(c, CPRA_EINVAL, std::string("cannot open metrics log ") + path);
  return CPRA_OK;
}

cpra_status cpra_solve(cpra_ctx* c, int64_t steps, int64_t eval_every, cpra_shot_eval* best_out,
                       int64_t* best_step_out) {
  NvtxRange range("cpra_solve");
  if (!c || !best_out || steps < 1) return c ? fail(c, CPRA_EINVAL, "bad solve arguments") : CPRA_EINVAL;
  if (eval_every < 1) eval_every = steps;
  using Clock = std::chrono::steady_clock;
  const Clock::time_point t_begin = Clock::now();
  Clock::time_point t_last = t_begin;
  std::vector<cpra_shot_eval> cur((size_t)c->S);
  std::vector<int64_t> best_step((size_t)c->S, -1);
  for (int s = 0; s < c->S; ++s) {
    best_out[s].objective = -1;
    best_out[s].violations = 0;
    best_out[s].qubo = 0.0;
    best_out[s].value = -1.0;
  }
  for (int64_t t = 0; t < steps;) {
    // steps t .. t_eval in one call (a captured step replayed), then evaluate
    int64_t t_eval = (t == 0) ? 0 : std::min(steps - 1, (t + eval_every - 1) / eval_every * eval_every);
    const int64_t n_steps = t_eval - t + 1;
    cpra_status st = cpra_steps(c, t, n_steps);
    if (st != CPRA_OK) return st;
    t = t_eval + 1;
    {
      int64_t ham = 0;
      st = cpra_round_eval(c, cur.data(), c->metrics ? &ham : nullptr, nullptr);
      if (st != CPRA_OK) return st;
      st = check_err_flag(c);
      if (st != CPRA_OK) return st;
      if (c->metrics) {
        const Clock::time_point now = Clock::now();
        st = write_metrics(c, t_eval, n_steps, std::chrono::duration<double>(now - t_last).count(),
                           std::chrono::duration<double>(now - t_begin).count(), cur.data(), ham);
        if (st != CPRA_OK) return st;
        t_last = Clock::now();
      }
      for (int s = 0; s < c->S; ++s) {
        const bool ok = c->cfg.problem == CPRA_MAXCUT || cur[s].violations == 0;
        // weighted MIS and DBM rank by value (weight, reward), the others by
        // the integer objective; objective -1 marks a shot with none yet
        const bool by_value = c->wmis || c->cfg.problem == CPRA_DBM || c->ew_d != nullptr;
        const bool better = best_out[s].objective < 0 ||
                            (by_value ? cur[s].value > best_out[s].value
                                      : cur[s].objective > best_out[s].objective);
        if (ok && better) {
          best_out[s] = cur[s];
          best_step[s] = t_eval;
        }
      }
      if (es_on(c)) {
        EarlyStopState h;
        st = read_early_stop(c, &h);
        if (st != CPRA_OK) return fail(c, st, "early-stopping state readback");
        if (h.stopped) break;
      }
    }
  }
  if (best_step_out) std::memcpy(best_step_out, best_step.data(), sizeof(int64_t) * c->S);
  return CPRA_OK;
}

size_t cpra_tensor_bytes(const cpra_ctx* c, int32_t which) {
  if (!c) return 0;
  const size_t NH = (size_t)c->N * c->H0 * sizeof(float);
  switch (which) {
    case CPRA_T_THETA: case CPRA_T_THETA_M: case CPRA_T_THETA_V: case CPRA_T_GRAD:
      return (size_t)c->nparam * sizeof(float);
    case CPRA_T_EMB: case CPRA_T_EMB_M: case CPRA_T_EMB_V: case CPRA_T_EMB_GRAD:
      return NH;
    case CPRA_T_P: case CPRA_T_GZ2:
      return (size_t)c->N * c->S * sizeof(float);
    case CPRA_T_STEP:
      return sizeof(int64_t);
    case CPRA_T_TERMS:
      return (3 * (size_t)c->S + 1) * sizeof(float);
    default:
      return 0;
  }
}

static float* flat_ptr(cpra_ctx* c, int32_t which) {
  switch (which) {
    case CPRA_T_THETA: return c->theta;
    case CPRA_T_THETA_M: return c->theta_m;
    case CPRA_T_THETA_V: return c->theta_v;
    case CPRA_T_GRAD: return c->grad;
    case CPRA_T_EMB: return c->X0m;
    case CPRA_T_EMB_M: return c->X0_m;
    case CPRA_T_EMB_V: return c->X0_v;
    case CPRA_T_EMB_GRAD: return c->gX0;
    case CPRA_T_TERMS: return c->terms;
    default: return nullptr;
  }
}

static float bf16_bits_to_float(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

cpra_status cpra_get_tensor(cpra_ctx* c, int32_t which, void* host, size_t nbytes) {
  if (!c || !host) return c ? fail(c, CPRA_EINVAL, "host is NULL") : CPRA_EINVAL;
  const size_t want = cpra_tensor_bytes(c, which);
  if (want == 0 || nbytes != want) return fail(c, CPRA_EINVAL, "bad tensor id or size");
  cudaStream_t st = c->stream;
  cpra_status s = CPRA_OK;
  if (which == CPRA_T_STEP) {
    s = cuda_check(c, cudaStreamSynchronize(st), "sync");
    if (s == CPRA_OK && es_on(c)) {
      EarlyStopState h;
      s = read_early_stop(c, &h);
    }
    std::memcpy(host, &c->opt_steps, sizeof(int64_t));
    return s;
  }
  if (which == CPRA_T_P) {
    s = cuda_check(c, cudaMemcpy2DAsync(host, sizeof(float) * c->S, c->P, sizeof(float) * c->S_pad,
                                        sizeof(float) * c->S, c->N, cudaMemcpyDeviceToHost, st), "P");
  } else if (which == CPRA_T_GZ2) {
    if (c->act_dt == DT_F32) {
      s = cuda_check(c, cudaMemcpy2DAsync(host, sizeof(float) * c->S, c->GZ2, sizeof(float) * c->S_pad,
                                          sizeof(float) * c->S, c->N, cudaMemcpyDeviceToHost, st), "GZ2");
    } else {
      std::vector<uint16_t> tmp((size_t)c->N * c->S);
      s = cuda_check(c, cudaMemcpy2DAsync(tmp.data(), 2 * c->S, c->GZ2, 2 * (size_t)c->S_pad, 2 * c->S,
                                          c->N, cudaMemcpyDeviceToHost, st), "GZ2");
      if (s == CPRA_OK) s = cuda_check(c, cudaStreamSynchronize(st), "sync");
      float* h = static_cast<float*>(host);
      for (size_t k = 0; k < tmp.size(); ++k) h[k] = bf16_bits_to_float(tmp[k]);
      return s;
    }
  } else {
    s = cuda_check(c, cudaMemcpyAsync(host, flat_ptr(c, which), nbytes, cudaMemcpyDeviceToHost, st), "get");
  }
  if (s == CPRA_OK) s = cuda_check(c, cudaStreamSynchronize(st), "sync");
  return s;
}

cpra_status cpra_set_tensor(cpra_ctx* c, int32_t which, const void* host, size_t nbytes) {
  if (!c || !host) return c ? fail(c, CPRA_EINVAL, "host is NULL") : CPRA_EINVAL;
  const size_t want = cpra_tensor_bytes(c, which);
  if (want == 0 || nbytes != want) return fail(c, CPRA_EINVAL, "bad tensor id or size");
  cudaStream_t st = c->stream;
  if (which == CPRA_T_STEP) {
    cpra_status s = cuda_check(c, cudaStreamSynchronize(st), "sync");
    int64_t v;
    std::memcpy(&v, host, sizeof(v));
    if (v < 0) return fail(c, CPRA_EINVAL, "step counter must be >= 0");
    c->opt_steps = v;
    return s;
  }
  if (which == CPRA_T_P || which == CPRA_T_GZ2 || which == CPRA_T_TERMS)
    return fail(c, CPRA_EINVAL, "tensor is read-only");
  cpra_status s = cuda_check(c, cudaMemcpyAsync(flat_ptr(c, which), host, nbytes,
                                                cudaMemcpyHostToDevice, st), "set");
  if (s != CPRA_OK) return s;
  c->fwd_valid = false;
  if (which == CPRA_T_THETA) refresh_shadows(c);
  if (which == CPRA_T_EMB) refresh_emb_shadow(c);
  c->have_eval = false;
  return cuda_check(c, cudaStreamSynchronize(st), "sync");
}

struct StateHeader {
  char magic[8];
  int64_t version, N, H0, H1, S, nparam, opt_steps;
};

cpra_status cpra_get_state(cpra_ctx* c, void* buf, size_t* nbytes) {
  if (!c || !nbytes) return CPRA_EINVAL;
  const size_t tb = (size_t)c->nparam * sizeof(float);
  const size_t eb = (size_t)c->N * c->H0 * sizeof(float);
  const size_t total = sizeof(StateHeader) + sizeof(EarlyStopState) + 3 * tb + 3 * eb;
  if (!buf) { *nbytes = total; return CPRA_OK; }
  if (*nbytes < total) return fail(c, CPRA_EINVAL, "state buffer too small");
  StateHeader h{};
  std::memcpy(h.magic, "CPRAST01", 8);
  h.version = 2; h.N = c->N; h.H0 = c->H0; h.H1 = c->H1; h.S = c->S; h.nparam = c->nparam;
  cpra_status s = cuda_check(c, cudaStreamSynchronize(c->stream), "sync");
  if (s != CPRA_OK) return s;
  EarlyStopState es;
  s = read_early_stop(c, &es);
  if (s != CPRA_OK) return fail(c, s, "early-stopping state readback");
  h.opt_steps = c->opt_steps;
  char* p = static_cast<char*>(buf);
  std::memcpy(p, &h, sizeof(h));
  p += sizeof(h);
  std::memcpy(p, &es, sizeof(es));
  p += sizeof(es);
  const int32_t ids[6] = {CPRA_T_THETA, CPRA_T_THETA_M, CPRA_T_THETA_V,
                          CPRA_T_EMB, CPRA_T_EMB_M, CPRA_T_EMB_V};
  for (int k = 0; k < 6; ++k) {
    const size_t nb = k < 3 ? tb : eb;
    s = cpra_get_tensor(c, ids[k], p, nb);
    if (s != CPRA_OK) return s;
    p += nb;
  }
  *nbytes = total;
  return CPRA_OK;
}

cpra_status cpra_set_state(cpra_ctx* c, const void* buf, size_t nbytes) {
  if (!c || !buf) return CPRA_EINVAL;
  const size_t tb = (size_t)c->nparam * sizeof(float);
  const size_t eb = (size_t)c->N * c->H0 * sizeof(float);
  const size_t total = sizeof(StateHeader) + sizeof(EarlyStopState) + 3 * tb + 3 * eb;
  if (nbytes != total) return fail(c, CPRA_ESTATE, "state blob has the wrong size");
  StateHeader h;
  std::memcpy(&h, buf, sizeof(h));
  if (std::memcmp(h.magic, "CPRAST01", 8) != 0 || h.version != 2 || h.N != c->N ||
      h.H0 != c->H0 || h.H1 != c->H1 || h.S != c->S || h.nparam != c->nparam)
    return fail(c, CPRA_ESTATE, "state blob does not match this context");
  const char* p = static_cast<const char*>(buf) + sizeof(h);
  EarlyStopState es;
  std::memcpy(&es, p, sizeof(es));
  p += sizeof(es);
  cpra_status se = cuda_check(c, cudaMemcpyAsync(c->es, &es, sizeof(es), cudaMemcpyHostToDevice,
                                                 c->stream), "early-stopping state");
  if (se == CPRA_OK) se = cuda_check(c, cudaStreamSynchronize(c->stream), "sync");
  if (se != CPRA_OK) return se;
  const int32_t ids[6] = {CPRA_T_THETA, CPRA_T_THETA_M, CPRA_T_THETA_V,
                          CPRA_T_EMB, CPRA_T_EMB_M, CPRA_T_EMB_V};
  for (int k = 0; k < 6; ++k) {
    const size_t nb = k < 3 ? tb : eb;
    cpra_status s = cpra_set_tensor(c, ids[k], p, nb);
    if (s != CPRA_OK) return s;
    p += nb;
  }
  c->opt_steps = h.opt_steps;
  return CPRA_OK;
}

cpra_status cpra_get_P(cpra_ctx* c, float* host_NxS) {
  if (!c) return CPRA_EINVAL;
  return cpra_get_tensor(c, CPRA_T_P, host_NxS, cpra_tensor_bytes(c, CPRA_T_P));
}

int64_t cpra_param_count(const cpra_ctx* c) { return c ? c->nparam : 0; }
int64_t cpra_launch_count(const cpra_ctx* c) { return c ? c->launches : 0; }

int64_t cpra_early_stop_step(cpra_ctx* c) {
  if (!c || !es_on(c)) return -1;
  EarlyStopState h;
  if (read_early_stop(c, &h) != CPRA_OK) return -1;
  return h.stopped ? (int64_t)h.stop_step : -1;
}

cpra_status cpra_inject_error_flag(cpra_ctx* c, int32_t bits) {
  if (!c) return CPRA_EINVAL;
  if (bits < 1 || bits > 3) return fail(c, CPRA_EINVAL, "cpra_inject_error_flag: bits must be 1..3");
  int flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, c->err_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  flag |= bits;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->err_flag, &flag, sizeof(int), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return cuda_check(c, e, "error-flag injection");
}

void cpra_profile_enable(cpra_ctx* c, int on) {
  if (!c) return;
  if (on && c->prof_ring.empty()) {
    c->prof_ring.resize(4096);
    for (auto& r : c->prof_ring) {
      cudaEventCreate(&r.a);
      cudaEventCreate(&r.b);
    }
  }
  c->prof = on != 0 && !c->prof_ring.empty();
}

int32_t cpra_profile_read(cpra_ctx* c, double* ms_out, int64_t* launches_out, int32_t n_ids) {
  if (!c) return 0;
  cudaStreamSynchronize(c->stream);
  for (size_t k = 0; k < c->prof_used; ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->prof_ring[k].a, c->prof_ring[k].b) == cudaSuccess) {
      c->prof_ms[c->prof_ring[k].id] += ms;
      c->prof_n[c->prof_ring[k].id] += 1;
    }
  }
  c->prof_used = 0;
  const int n = std::min<int>(n_ids, K_COUNT_);
  for (int k = 0; k < n; ++k) {
    if (ms_out) ms_out[k] = c->prof_ms[k];
    if (launches_out) launches_out[k] = c->prof_n[k];
  }
  for (int k = 0; k < K_COUNT_; ++k) {
    c->prof_ms[k] = 0;
    c->prof_n[k] = 0;
  }
  return K_COUNT_;
}

const char* cpra_kernel_name(int32_t id) {
  if (id < 0 || id >= K_COUNT_) return "";
  return kKernelNames[id];
}

const char* cpra_last_error(const cpra_ctx* c) { return c ? c->err.c_str() : g_init_err.c_str(); }

const char* cpra_status_string(cpra_status s) {
  switch (s) {
    case CPRA_OK: return "ok";
    case CPRA_EINVAL: return "invalid argument";
    case CPRA_ENOMEM: return "out of device memory";
    case CPRA_ECUDA: return "CUDA error";
    case CPRA_ENUMERIC: return "non-finite value";
    case CPRA_ETIMEOUT: return "device wait timed out";
    case CPRA_ESTATE: return "state mismatch";
  }
  return "unknown status";
}

void cpra_destroy(cpra_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  for (auto& r : c->prof_ring) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
  }
  drop_graph(c);
  if (c->dbm_mem) cudaFree(c->dbm_mem);
  if (c->ew_mem) cudaFree(c->ew_mem);
  if (c->metrics) std::fclose(c->metrics);
  if (c->own_ws && c->ws) cudaFree(c->ws);
  if (c->init_logits) cudaFree(c->init_logits);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

cpra_status cpra_set_node_weights(cpra_ctx* c, const float* w, int64_t ld, int32_t on_device) {
  if (!c) return CPRA_EINVAL;
  if (!c->w_d) return fail(c, CPRA_EINVAL, "cpra_set_node_weights: not a weighted-MIS context");
  if (!w || ld < c->S) return fail(c, CPRA_EINVAL, "cpra_set_node_weights: NULL or ld < S");
  cudaStream_t st = c->stream;
  c->have_eval = false;
  cpra_status s = cuda_check(c, cudaMemsetAsync(c->w_d, 0, sizeof(float) * c->N * c->S_pad, st),
                             "memset");
  if (s == CPRA_OK)
    s = cuda_check(c, cudaMemcpy2DAsync(c->w_d, sizeof(float) * c->S_pad, w, sizeof(float) * ld,
                                        sizeof(float) * c->S, c->N,
                                        on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                        st),
                   "node weights");
  if (s == CPRA_OK) s = cuda_check(c, cudaStreamSynchronize(st), "sync");
  return s;
}

namespace {
// Whether the CSR is the constraint graph of an N1 x N2 matching: node r*N2 + k
// adjacent exactly to the other pairs of row r and of column k.
bool is_constraint_graph(int N1, int N2, const int* rowptr, const int* col) {
  const int deg = N1 + N2 - 2;
  std::vector<int> want;
  want.reserve(deg);
  for (int r = 0; r < N1; ++r)
    for (int k = 0; k < N2; ++k) {
      const int64_t i = (int64_t)r * N2 + k;
      if (rowptr[i + 1] - rowptr[i] != deg) return false;
      want.clear();
      for (int q = 0; q < N2; ++q)
        if (q != k) want.push_back(r * N2 + q);
      for (int q = 0; q < N1; ++q)
        if (q != r) want.push_back(q * N2 + k);
      std::sort(want.begin(), want.end());
      for (int e = 0; e < deg; ++e)
        if (col[rowptr[i] + e] != want[e]) return false;
    }
  return true;
}
}  // namespace

cpra_status cpra_set_dbm(cpra_ctx* c, int32_t N1, const float* C, const float* M, int64_t ld,
                         const float* lam4, const float* pq) {
  if (!c) return CPRA_EINVAL;
  if (c->cfg.problem != CPRA_DBM) return fail(c, CPRA_EINVAL, "cpra_set_dbm: not a DBM context");
  if (!C || !M || !lam4 || !pq) return fail(c, CPRA_EINVAL, "cpra_set_dbm: NULL array");
  if (ld < c->S) return fail(c, CPRA_EINVAL, "cpra_set_dbm: ld < S");
  if (N1 < 1 || c->N % N1) return fail(c, CPRA_EINVAL, "cpra_set_dbm: N1 must divide N");
  const int S = c->S;
  for (int64_t n = 0; n < c->N; ++n)
    for (int s = 0; s < S; ++s) {
      const float cv = C[n * ld + s], mv = M[n * ld + s];
      if (!std::isfinite(cv)) return fail(c, CPRA_EINVAL, "cpra_set_dbm: non-finite C");
      if (!(mv >= 0.f && mv <= 1.f)) return fail(c, CPRA_EINVAL, "cpra_set_dbm: M outside [0, 1]");
    }
  for (int s = 0; s < S; ++s) {
    for (int k = 0; k < 4; ++k)
      if (!std::isfinite(lam4[4 * s + k])) return fail(c, CPRA_EINVAL, "cpra_set_dbm: non-finite lambda");
    for (int k = 0; k < 2; ++k)
      if (!(pq[2 * s + k] >= 0.f && pq[2 * s + k] <= 1.f))
        return fail(c, CPRA_EINVAL, "cpra_set_dbm: p, q outside [0, 1]");
  }
  const int N2 = (int)(c->N / N1);
  const int64_t ldd = c->S_pad;
  const int lines = N1 + N2;
  const int64_t ldl = std::max(c->H0, c->H1);
  float* lr = nullptr;
  float* lk = nullptr;
  // one allocation: C, M, rowc, colc, line sums, shot coefficients, eval partials
  auto carve_dbm = [&](void* base, DbmDev& d) -> size_t {
    Carver cv(base);
    float* Cd = cv.take<float>((size_t)c->N * ldd);
    float* Md = cv.take<float>((size_t)c->N * ldd);
    float* l4 = cv.take<float>((size_t)4 * S);
    float* pqd = cv.take<float>((size_t)2 * S);
    d.C = Cd; d.M = Md; d.lam4 = l4; d.pq = pqd;
    d.rowc = cv.take<float>((size_t)N1 * ldd);
    d.colc = cv.take<float>((size_t)N2 * ldd);
    d.line = cv.take<float>((size_t)lines * 3 * ldd);
    d.shot = cv.take<float>((size_t)3 * ldd);
    d.ecnt = cv.take<int>((size_t)lines * ldd);
    d.eU = cv.take<double>((size_t)N1 * ldd);
    d.eC = cv.take<double>((size_t)N1 * ldd);
    lr = cv.take<float>((size_t)N1 * ldl);
    lk = cv.take<float>((size_t)N2 * ldl);
    return cv.off + kAlign;
  };
  cudaStream_t st = c->stream;
  c->fwd_valid = false;
  c->have_eval = false;
  if (c->dbm_mem && c->dbm.N1 != N1) {  // new shape: reallocate (the captured step
    cudaStreamSynchronize(st);           // holds the old pointers)
    drop_graph(c);
    cudaFree(c->dbm_mem);
    c->dbm_mem = nullptr;
  }
  if (!c->dbm_mem) {
    DbmDev probe;
    const size_t bytes = carve_dbm(nullptr, probe);
    if (c->cfg.mem_cap_bytes && c->ws_bytes + bytes > c->cfg.mem_cap_bytes)
      return fail(c, CPRA_ENOMEM, "cpra_set_dbm: exceeds mem_cap_bytes");
    if (cudaMalloc(&c->dbm_mem, bytes) != cudaSuccess) {
      cudaGetLastError();
      c->dbm_mem = nullptr;
      return fail(c, CPRA_ENOMEM, "cpra_set_dbm: device allocation failed");
    }
    c->dbm_bytes = (int64_t)bytes;
    DbmDev d;
    d.N1 = N1;
    d.N2 = N2;
    d.ld = ldd;
    carve_dbm(c->dbm_mem, d);
    c->dbm = d;
    c->line_R = lr;
    c->line_K = lk;
    c->ldl = ldl;
    // aggregate through line sums when the graph is this matching's
    // constraint graph (checked on a host copy of the CSR)
    std::vector<int> rp((size_t)c->N + 1), cl((size_t)std::max<int64_t>(c->nnz, 1));
    bool ok = cudaStreamSynchronize(st) == cudaSuccess &&
              cudaMemcpy(rp.data(), c->rowptr, sizeof(int) * rp.size(), cudaMemcpyDeviceToHost) ==
                  cudaSuccess &&
              cudaMemcpy(cl.data(), c->col, sizeof(int) * cl.size(), cudaMemcpyDeviceToHost) ==
                  cudaSuccess;
    if (!ok) cudaGetLastError();
    c->line_agg = ok && is_constraint_graph(N1, N2, rp.data(), cl.data());
    drop_graph(c);  // the captured step (if any) has the gathered aggregations
  }
  cpra_status s = cuda_check(c, cudaMemsetAsync(c->dbm_mem, 0, (size_t)c->dbm_bytes, st), "memset");
  const size_t row = sizeof(float) * (size_t)S;
  if (s == CPRA_OK)
    s = cuda_check(c, cudaMemcpy2DAsync(const_cast<float*>(c->dbm.C), sizeof(float) * ldd, C,
                                        sizeof(float) * ld, row, c->N, cudaMemcpyHostToDevice, st),
                   "DBM rewards");
  if (s == CPRA_OK)
    s = cuda_check(c, cudaMemcpy2DAsync(const_cast<float*>(c->dbm.M), sizeof(float) * ldd, M,
                                        sizeof(float) * ld, row, c->N, cudaMemcpyHostToDevice, st),
                   "DBM fields");
  if (s == CPRA_OK)
    s = cuda_check(c, cudaMemcpyAsync(const_cast<float*>(c->dbm.lam4), lam4, sizeof(float) * 4 * S,
                                      cudaMemcpyHostToDevice, st), "DBM lambdas");
  if (s == CPRA_OK)
    s = cuda_check(c, cudaMemcpyAsync(const_cast<float*>(c->dbm.pq), pq, sizeof(float) * 2 * S,
                                      cudaMemcpyHostToDevice, st), "DBM p, q");
  if (s == CPRA_OK) s = cuda_check(c, cudaStreamSynchronize(st), "sync");
  return s;
}

cpra_status cpra_set_init_logits(cpra_ctx* c, const float* logits, int64_t ld, int32_t on_device) {
  if (!c) return CPRA_EINVAL;
  cudaStream_t st = c->stream;
  c->fwd_valid = false;
  c->have_eval = false;
  drop_graph(c);  // the captured step carries the offset pointer
  if (!logits) {  // back to the plain network
    cpra_status s = cuda_check(c, cudaStreamSynchronize(st), "sync");
    if (c->init_logits) cudaFree(c->init_logits);
    c->init_logits = nullptr;
    return s;
  }
  if (ld < c->S) return fail(c, CPRA_EINVAL, "cpra_set_init_logits: ld < S");
  const size_t act = c->act_dt == DT_BF16 ? 2 : 4;
  const size_t bytes = (size_t)c->N * c->S_pad * act;
  if (!c->init_logits) {
    if (c->cfg.mem_cap_bytes && c->ws_bytes + bytes > c->cfg.mem_cap_bytes)
      return fail(c, CPRA_ENOMEM, "cpra_set_init_logits: exceeds mem_cap_bytes");
    if (cudaMalloc(&c->init_logits, bytes) != cudaSuccess) {
      cudaGetLastError();
      c->init_logits = nullptr;
      return fail(c, CPRA_ENOMEM, "cpra_set_init_logits: device allocation failed");
    }
  }
  // stage as contiguous FP32 [N x S] on the device, then convert into the
  // padded activation-dtype buffer (pad columns 0)
  float* tmp = nullptr;
  if (cudaMalloc(&tmp, sizeof(float) * (size_t)c->N * c->S) != cudaSuccess) {
    cudaGetLastError();
    return fail(c, CPRA_ENOMEM, "cpra_set_init_logits: staging allocation failed");
  }
  cpra_status s = cuda_check(
      c, cudaMemcpy2DAsync(tmp, sizeof(float) * c->S, logits, sizeof(float) * ld,
                           sizeof(float) * c->S, c->N,
                           on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st),
      "init logits");
  if (s == CPRA_OK) s = cuda_check(c, cudaMemsetAsync(c->init_logits, 0, bytes, st), "memset");
  if (s == CPRA_OK) {
    copy_rows_launch(c->N, c->S, tmp, c->init_logits, c->S_pad, c->act_dt, st);
    c->launches += 1;
    s = cuda_check(c, cudaStreamSynchronize(st), "sync");
  }
  cudaFree(tmp);
  return s;
}

// ------------------------------------------------------------ op level
size_t cpra_op_loss_scratch_bytes(int64_t N, int32_t S) {
  (void)N;
  if (S < 1 || S > 1024) return 0;
  return (size_t)kLossMaxGrid * loss_pstride(S) * sizeof(float) +
         kAlign + (2 * (size_t)S + 1) * sizeof(unsigned long long);
}

cpra_status cpra_op_loss(int64_t N, int32_t S, const int32_t* rowptr, const int32_t* col,
                         const float* P, int64_t ldp, const float* lambda, int32_t problem,
                         int32_t alpha, float gamma, float nu, int32_t diversity_kind,
                         int32_t grad_kind, float* G, int64_t ldg, uint32_t* x_bits,
                         float* terms, void* scratch, size_t scratch_bytes, void* cuda_stream) {
  NvtxRange range("cpra_op_loss");
  if (N < 1 || S < 1 || S > 1024 || !rowptr || !col || !P || !G || !terms || !scratch)
    return CPRA_EINVAL;
  if (ldp < S || ldp % 4 || ldg < S || ldg % 4 || ldg > round_up(S, 16)) return CPRA_EINVAL;
  if (problem != CPRA_MIS && problem != CPRA_MAXCUT) return CPRA_EINVAL;
  if (problem == CPRA_MIS && !lambda) return CPRA_EINVAL;
  if (alpha < 2 || alpha % 2 || diversity_kind < 0 || diversity_kind > 1) return CPRA_EINVAL;
  if (grad_kind != 0 && grad_kind != 1) return CPRA_EINVAL;
  if (scratch_bytes < cpra_op_loss_scratch_bytes(N, S)) return CPRA_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  Carver cv(scratch);
  LossArgs a;
  a.N = N; a.S = S; a.ldp = ldp; a.ldg = ldg; a.rowptr = rowptr; a.col = col; a.P = P;
  a.lambda = lambda; a.problem = problem; a.alpha = alpha; a.div_kind = diversity_kind;
  a.grad_kind = grad_kind; a.gamma = gamma; a.nu = nu; a.G = G; a.dg = DT_F32;
  a.xbits = x_bits; a.pstride = loss_pstride(S);
  a.partials = cv.take<float>((size_t)kLossMaxGrid * a.pstride);
  a.do_loss = 1;
  const int grid = loss_launch(a, device_sm_count() * 4, st);
  colsum_finalize(a.partials, grid, a.pstride, 4 * S + 1, terms, nullptr, 0, 0, nullptr, st);
  return cudaGetLastError() == cudaSuccess ? CPRA_OK : CPRA_ECUDA;
}

size_t cpra_op_round_eval_scratch_bytes(int32_t S) {
  if (S < 1 || S > 1024) return 0;
  return (2 * (size_t)S + 1) * sizeof(unsigned long long);
}

cpra_status cpra_op_round_eval(int64_t N, int32_t S, const int32_t* rowptr, const int32_t* col,
                               const float* P, int64_t ldp, const float* lambda, int32_t problem,
                               uint32_t* x_bits, cpra_shot_eval* out, int64_t* pair_hamming,
                               void* counters, size_t counters_bytes, void* cuda_stream) {
  NvtxRange range("cpra_op_round_eval");
  if (N < 1 || S < 1 || S > 1024 || !rowptr || !col || !P || !x_bits || !out || !pair_hamming ||
      !counters)
    return CPRA_EINVAL;
  if (ldp < S || ldp % 4) return CPRA_EINVAL;
  if (problem != CPRA_MIS && problem != CPRA_MAXCUT) return CPRA_EINVAL;
  if (problem == CPRA_MIS && !lambda) return CPRA_EINVAL;
  if (counters_bytes < cpra_op_round_eval_scratch_bytes(S)) return CPRA_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  LossArgs a;
  a.N = N; a.S = S; a.ldp = ldp; a.ldg = round_up(S, 4); a.rowptr = rowptr; a.col = col; a.P = P;
  a.lambda = lambda; a.problem = problem; a.xbits = x_bits;
  a.do_loss = 0;
  auto* cnt = static_cast<unsigned long long*>(counters);
  if (cudaMemsetAsync(cnt, 0, cpra_op_round_eval_scratch_bytes(S), st) != cudaSuccess)
    return CPRA_ECUDA;
  const int sms = device_sm_count();
  loss_launch(a, sms * 4, st);  // rounding bits
  eval_bits_launch(N, S, rowptr, col, x_bits, problem, cnt, sms, st);
  eval_finalize(cnt, S, problem, lambda, out, reinterpret_cast<long long*>(pair_hamming), st);
  return cudaGetLastError() == cudaSuccess ? CPRA_OK : CPRA_ECUDA;
}

int64_t cpra_csr_check(int64_t* first_row, int64_t* first_entry) {
  if (first_row) *first_row = -1;
  if (first_entry) *first_entry = -1;
#ifdef CPRA_CHECKED
  if (cudaDeviceSynchronize() != cudaSuccess) return -2;
  CsrCheck r;
  csr_check_collect_spmm(&r);
  csr_check_collect_eval(&r);
  csr_check_collect_loss<0>(&r);
  csr_check_collect_loss<1>(&r);
  csr_check_collect_loss<2>(&r);
  csr_check_collect_loss<3>(&r);
  csr_check_collect_loss<4>(&r);
  if (first_row && r.first_row != CsrCheck().first_row) *first_row = r.first_row;
  if (first_entry && r.first_entry != CsrCheck().first_entry) *first_entry = r.first_entry;
  return (int64_t)r.count;
#else
  return -1;
#endif
}

}  // extern "C"
