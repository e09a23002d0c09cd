// Host-side launchers of the CPRA kernels (internal interface between the
// C-ABI layer and the kernel translation units).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cpra {

enum DType { DT_F32 = 0, DT_BF16 = 1 };

// Per-step scalars of a training step, computed on the device by
// step_scalars_launch so that a step's launches carry no per-step host
// arguments (the step can be captured once and replayed): the annealing
// weight gamma_t of the linear schedule and the Adam bias corrections for
// the step's update.  t / updates are the step's schedule index and the
// number of updates before it; next_t / next_updates are what the following
// step takes when it reads them from here.
struct StepScalars {
  float gamma, bc1, bc2;
  int pad;
  long long t, updates;
  long long next_t, next_updates;
};
// from_device = 0: the step is (t, updates); 1: it is (next_t, next_updates).
void step_scalars_launch(StepScalars* sc, int from_device, long long t, long long updates,
                         float gamma0, float gamma1, long long T, float beta1, float beta2,
                         cudaStream_t st);

// ---------------------------------------------------------------- SpMM
// Row-gather SpMM over the symmetric CSR (Eq. GCN aggregate step):
//   Y_i = s_i * (add_i + sum_{j in N(i)} X_j)  [* 1[mask_i > 0]]
// with s_i = 1/|N(i)| (0 for isolated i) when `mean`, else 1.  X, add and
// mask share the activation dtype dx; Y has dtype dy.  H % (16/sizeof(X)) == 0
// and all row strides keep 16-byte alignment.  Optionally writes per-block
// column sums of Y (before the dtype conversion) to colsum_partials[grid][H].
struct SpmmArgs {
  int64_t N = 0;
  int H = 0;
  const int* rowptr = nullptr;
  const int* col = nullptr;
  const float* inv_deg = nullptr;
  const void* X = nullptr;
  int64_t ldx = 0;
  void* Y = nullptr;
  int64_t ldy = 0;
  int mean = 1;
  const void* add = nullptr;
  int64_t ldadd = 0;
  const void* mask = nullptr;
  int64_t ldm = 0;
  float* colsum_partials = nullptr;
  int dx = DT_F32;
  int dy = DT_F32;
  int* err_flag = nullptr;  // device word; bit 1 set if a bounded wait gave up
  // Mask given as bits instead of values (with add and colsum, mean = 0): bit
  // (k % 16) of mask_bits[i*ldmb + k/16] is 1[mask_ik > 0] (EPI_RELU_BITS).
  const uint16_t* mask_bits = nullptr;
  int64_t ldmb = 0;
  // Fused embedding update (adam = 1, with add, mean = 0, dy = f32): the row
  // result g_i is the embedding gradient; Adam updates emb/emb_m/emb_v
  // ([N x H] f32, row stride H) and writes the updated row to shadow (dtype
  // dx, row stride lds).  Y may be null (the gradient is then not stored).
  int adam = 0;
  const int* halt = nullptr;  // while *halt != 0 the embedding rows are left as they are
  const StepScalars* sc = nullptr;  // when set, bc1 / bc2 are sc->bc1 / sc->bc2
  float* emb = nullptr;
  float* emb_m = nullptr;
  float* emb_v = nullptr;
  void* shadow = nullptr;
  int64_t lds = 0;
  float lr = 0.f, beta1 = 0.f, beta2 = 0.f, eps = 0.f, wd = 0.f, bc1 = 1.f, bc2 = 1.f;
  int64_t lde = 0;    // row stride of emb / emb_m / emb_v (0: H)
  int64_t ldcs = 0;   // row stride of colsum_partials (0: H)
  int nsl = 1;        // column slices (set by spmm_launch)
  int h_full = 0;     // row width before slicing (set by spmm_launch)
  // The graph is the constraint graph of an N1 x N2 matching (node r*N2 + k
  // adjacent to every other pair of row r and of column k): with line_r /
  // line_k the FP32 line sums of X ([N1 x ldl], [N2 x ldl], dbm_line_sums_launch),
  // the neighbour sum is read from them instead of gathered (rowptr / col unused).
  const float* line_r = nullptr;
  const float* line_k = nullptr;
  int line_n2 = 0;
  int64_t ldl = 0;
};
constexpr int kSliceH = 1024;  // widest row one SpMM launch covers
// Column-slice width of an aggregation: with line sums (three row reads per
// node instead of a gather) the rows are cut to one 16-byte chunk per lane,
// so that the light per-row work runs at full occupancy.
inline int spmm_slice_width(const SpmmArgs& a) {
  return a.line_r ? (a.dx == DT_BF16 ? 256 : 128) : kSliceH;
}
inline int spmm_slices(const SpmmArgs& a) {
  const int w = spmm_slice_width(a);
  return a.H <= w ? 1 : (a.H + w - 1) / w;
}
// Five operand sets are supported (the ones the training step uses):
// rows wider than spmm_slice_width run as column slices of one launch.
// mean aggregation (no add/mask/colsum, dy == dx), add + mask + colsum with
// mean = 0 (dy == dx; the mask as values or as bits), add only with mean = 0
// (dy = f32), and the latter with the fused embedding update (adam = 1).  The grid is the
// number of blocks resident at once on num_sms SMs, at most max_grid.
// Returns the grid size used (the row count of colsum_partials), or -1 for
// an operand set outside these three (nothing is launched).
int spmm_launch(const SpmmArgs& a, int num_sms, int max_grid, cudaStream_t st);

// ---------------------------------------------------------------- loss
// Fused SpMM + relaxed loss + rounding/evaluation (see cpra_op_loss).
// Diverse bipartite matching (Eq. matching-cost-function): x_ij is node
// i*N2 + j; every per-shot array has row stride ld (>= S, a multiple of 4).
struct DbmDev {
  int N1 = 0, N2 = 0;
  int64_t ld = 0;
  const float* C = nullptr;     // N x ld: reward C_ij of shot s's instance
  const float* M = nullptr;     // N x ld: 1 if i and j are in different fields
  const float* lam4 = nullptr;  // S x 4: lambda_1..4 of shot s
  const float* pq = nullptr;    // S x 2: p, q of shot s
  float* rowc = nullptr;        // N1 x ld: lambda_1 1[R_is > 1], R_is = sum_j P_(ij)s
  float* colc = nullptr;        // N2 x ld: lambda_2 1[K_js > 1], K_js = sum_i P_(ij)s
  float* line = nullptr;        // (N1+N2) x 3 x ld: per-line ReLU excess, T and U parts
  float* shot = nullptr;        // 3 x ld: b_s, d_s, pen_s (dl/dx = -C + rowc + colc + b + d M)
  int* ecnt = nullptr;          // (N1+N2) x ld: pairs per line of the rounded shots
  double* eU = nullptr;         // N1 x ld: sum_j M x per row line
  double* eC = nullptr;         // N1 x ld: sum_j C x per row line
};

struct LossArgs {
  int64_t N = 0;
  int S = 0;
  int64_t ldp = 0, ldg = 0;
  const int* rowptr = nullptr;
  const int* col = nullptr;
  const float* P = nullptr;
  const float* lambda = nullptr;
  int problem = 0, alpha = 2, div_kind = 0, grad_kind = 0;
  float gamma = 0.f, nu = 0.f;
  const StepScalars* sc = nullptr;  // when set, gamma is sc->gamma
  const float* w = nullptr;   // weighted MIS (problem 0): node weights N x ldw, cost -sum w P
  int64_t ldw = 0;
  const float* ew = nullptr;    // MaxCut (problem 1): edge weight per CSR entry, or null (unit)
  const float* wdeg = nullptr;  //   and the weighted degree sum_j A_ij per node
  void* G = nullptr;             // dtype dg, N x ldg
  int dg = DT_F32;
  uint32_t* xbits = nullptr;     // N x W, W = ceil(S/32)
  float* partials = nullptr;     // [grid][pstride]: cost S | pen S | ann S | psi | gsum S
  int64_t pstride = 0;
  int do_loss = 1;               // 0: rounding bits only
  int* err_flag = nullptr;       // device word; bit 1 set if a bounded wait gave up
  DbmDev dbm;                    // problem 2 (DBM): instance and per-step line sums
};
int64_t loss_pstride(int S);
constexpr int kLossMaxGrid = 2048;
// Returns the grid size used (row count of partials).
int loss_launch(const LossArgs& a, int max_grid, cudaStream_t st);
// The loss kernels' instances for one problem (0 MIS, 1 MaxCut, 2 DBM,
// 3 weighted MIS, 4 MaxCut with edge weights), each compiled in its own
// object from k_loss_problem.cu; nch = ldg / 4.  loss_launch_bits (in the
// problem-0 object) packs the rounding bits alone, nch = ceil(S / 4).
template <int PROBLEM>
int loss_launch_problem(const LossArgs& a, int nch, int max_grid, int staged_grid, cudaStream_t st);
template <> int loss_launch_problem<0>(const LossArgs&, int, int, int, cudaStream_t);
template <> int loss_launch_problem<1>(const LossArgs&, int, int, int, cudaStream_t);
template <> int loss_launch_problem<2>(const LossArgs&, int, int, int, cudaStream_t);
template <> int loss_launch_problem<3>(const LossArgs&, int, int, int, cudaStream_t);
template <> int loss_launch_problem<4>(const LossArgs&, int, int, int, cudaStream_t);
int loss_launch_bits(const LossArgs& a, int nch, int max_grid, cudaStream_t st);

// Sum partial rows: out[c] = sum_{b < nblocks} part[b*pstride + c], c < ncols,
// in a fixed order; also copies out[copy_from .. copy_from+copy_n) to out2
// when out2 != null and flags non-finite sums in *err_flag (bit 0).
void colsum_finalize(const float* part, int nblocks, int64_t pstride, int ncols,
                     float* out, float* out2, int copy_from, int copy_n,
                     int* err_flag, cudaStream_t st);

// Exact integer evaluation of rounded shots from their bits (k_eval.cu):
// adds to counters obj[S] (MIS set size / MaxCut cut edges), viol[S] (MIS
// edges inside the set) and counters[2S] = sum_i k_i (S - k_i); problem 2
// reads no edges (set sizes and the Hamming sum only).  The counters must be
// zeroed by the caller.  sms: the device's SM count (the grid is one wave of
// resident blocks at most).
//
// With fin (problems 0 and 1 only) the launch also writes the per-shot
// records: the last block to finish (a ticket in counters[2S+1]) reads the
// counters, writes the records as eval_finalize does, and sets counters
// [0, 2S+1] back to zero, so the next launch needs no reset.  The counters
// array then holds 2S+2 words, zero before the first such launch.
struct EvalFinalize {
  const float* lambda = nullptr;   // MIS penalty weights [S]
  const double* wvalue = nullptr;  // shot values (weighted MIS / MaxCut), or null
  void* records = nullptr;         // ShotEvalRec [S]
  long long* ham = nullptr;        // pair-Hamming total, or null
};
void eval_bits_launch(int64_t N, int S, const int* rowptr, const int* col, const uint32_t* bits,
                      int problem, unsigned long long* counters, int sms, cudaStream_t st,
                      const EvalFinalize* fin = nullptr);

// Device image of cpra_shot_eval.
struct ShotEvalRec {
  long long objective;
  long long violations;
  double qubo;
  double value;
};
// Per-shot records from the integer counters: objective, violations and the
// FP64 qubo value; pair-Hamming total copied out.
void eval_finalize(const unsigned long long* counters, int S, int problem,
                   const float* lambda, void* out_records, long long* pair_hamming,
                   cudaStream_t st, const double* wvalue = nullptr);
// Weighted MIS: value[s] = sum_i w_is x_is in FP64 from the rounding bits,
// per-block partial rows (part[blocks][S], blocks <= max_blocks) summed in a
// fixed order.
void weighted_value_launch(int64_t N, int S, const uint32_t* bits, const float* w, int64_t ldw,
                           double* part, int max_blocks, double* value, cudaStream_t st);
// Weighted MaxCut: value[s] = sum of A_ij over the edges j > i with
// x_is != x_js (FP64, fixed order; part holds max_blocks x S partials).
void weighted_cut_launch(int64_t N, int S, const int* rowptr, const int* col, const float* ew,
                         const uint32_t* bits, double* part, int max_blocks, double* value,
                         cudaStream_t st);

// ---------------------------------------------------------------- DBM (k_dbm.cu)
// Line sums of the relaxed matching P (FP32, N x ldp): R, K, T, U in the
// fixed orders j (rows), i (columns), then rows / columns ascending; fills
// d.rowc, d.colc and d.shot for the loss kernel's problem-2 epilogue.
void dbm_sums_launch(const DbmDev& d, int S, const float* P, int64_t ldp, cudaStream_t st);
// Exact evaluation of the rounded matchings (bits N x ceil(S/32)): per shot
// objective = pairs, violations = rows and columns with more than one pair
// plus the failed diversity constraints, value = sum C x and qubo = l(x) in
// FP64; records as in eval_finalize, pair-Hamming total from counters[2S].
// Line sums of an activation block X [N1*N2 x H] (dtype dx, row stride ldx)
// in FP32: R[r*ldl + h] = sum_k X[r*N2 + k][h], K[k*ldl + h] = sum_r X[r*N2 + k][h],
// summed in index order.
void dbm_line_sums_launch(int N1, int N2, int H, const void* X, int64_t ldx, int dx, float* R,
                          float* K, int64_t ldl, cudaStream_t st);
void dbm_eval_launch(const DbmDev& d, int S, const uint32_t* bits,
                     const unsigned long long* counters, void* out_records,
                     long long* pair_hamming, cudaStream_t st);

// ---------------------------------------------------------------- GEMM
enum Epi { EPI_PARTIAL = 0, EPI_BIAS_RELU = 1, EPI_BIAS_SIGMOID = 2, EPI_SPLIT = 3,
           EPI_RELU_BITS = 4, EPI_BIAS = 5 };
// C[m, n] = sum_k A(m, k) B(n, k), FP32 accumulation.
//   A(m, k) = A[m*lda + k] if a_kmajor else A[k*lda + m]; same for B.
// Epilogues:
//   EPI_PARTIAL      out0 (f32) + z*M*ld0 <- C for split z of gridDim.z
//   EPI_BIAS_RELU    out0[m, n] <- max(C + bias[n], 0); with out1 also its mask
//                    as bits (layout of EPI_RELU_BITS, uint16 row stride ld1)
//   EPI_BIAS         out0[m, n] <- C + bias[n] for n < n_valid, else 0
//   EPI_BIAS_SIGMOID out0[m, n] <- 1/(1+exp(-(C + bias[n] [+ addend[m*ld_add + n]])))
//                    for n < n_valid, else 0 (addend, dtype d_add, may be null)
//   EPI_SPLIT        n < split: out0[m, n] <- C; else out1[m, n-split] <- C * row_scale[m]
//   EPI_RELU_BITS    ReLU mask only: bit (n % 16) of the uint16 out0[m*ld0 + n/16] is
//                    1[h > 0] for h = max(C + bias[n], 0) rounded to dtype d0 (so the
//                    mask equals the one read from a stored activation); Nc % 16 == 0
struct GemmArgs {
  int64_t M = 0;
  int Nc = 0;
  int64_t K = 0;
  const void* A = nullptr;
  int64_t lda = 0;
  int da = DT_F32;
  int a_kmajor = 1;
  const void* B = nullptr;
  int64_t ldb = 0;
  int db = DT_F32;
  int b_kmajor = 1;
  // split-TF32 tensor-core path: mid and lo parts of B (B holds the hi part)
  const void* B_mid = nullptr;
  const void* B_lo = nullptr;
  int epi = EPI_PARTIAL;
  const float* bias = nullptr;
  void* out0 = nullptr;
  int64_t ld0 = 0;
  int d0 = DT_F32;
  void* out1 = nullptr;
  int64_t ld1 = 0;
  int d1 = DT_F32;
  int split = 0;
  const float* row_scale = nullptr;
  int n_valid = 0;
  int splits = 1;
  int* err_flag = nullptr;  // device word; bit 1 set if a bounded wait gave up
  const void* addend = nullptr;  // EPI_BIAS_SIGMOID: per-element pre-activation offset
  int64_t ld_add = 0;
  int d_add = DT_F32;
};
void gemm_simt_launch(const GemmArgs& g, cudaStream_t st);
// gemm_simt_launch's instances for one (A, B) DType pair, each compiled in
// its own object; grid = (M tiles, Nc tiles, splits).
template <int DA, int DB> void gemm_simt_launch_typed(const GemmArgs& g, dim3 grid, cudaStream_t st);
template <> void gemm_simt_launch_typed<DT_F32, DT_F32>(const GemmArgs&, dim3, cudaStream_t);
template <> void gemm_simt_launch_typed<DT_F32, DT_BF16>(const GemmArgs&, dim3, cudaStream_t);
template <> void gemm_simt_launch_typed<DT_BF16, DT_F32>(const GemmArgs&, dim3, cudaStream_t);
template <> void gemm_simt_launch_typed<DT_BF16, DT_BF16>(const GemmArgs&, dim3, cudaStream_t);
// out[r*ldo + c] = sum_z part[z*M*ldp + r*ldp + c] for r < M, c < Nc.
void splitk_reduce(const float* part, int splits, int M, int Nc, int64_t ldp,
                   float* out, int64_t ldo, cudaStream_t st);

// ---------------------------------------------------------------- misc
// Adam on n parameters; skipped entirely while *halt != 0 (halt may be null).
// With sc non-null the bias corrections are sc->bc1, sc->bc2.
void adam_launch(int64_t n, float* theta, float* m, float* v, const float* g,
                 float lr, float beta1, float beta2, float eps, float wd,
                 float bc1, float bc2, const int* halt, const StepScalars* sc,
                 cudaStream_t st);

// Early-stopping monitor (Implementation paragraph), one thread: from the
// step's loss terms (cost S | pen S | ann S) forms l = sum_s (cost_s +
// lambda_s pen_s) (lambda null: cost only) and phi = gamma * sum_s ann_s in
// FP64 in the order s = 0..S-1; a step is stale when for both values the
// change from the previous step is > 0 or |change| <= tol; after `patience`
// consecutive stale steps sets `stopped`, stop_step = t and
// updates_at_stop = the Adam updates applied so far.  Does nothing once
// stopped.
struct EarlyStopState {
  double prev_l, prev_phi;
  long long stop_step;        // -1 while running
  long long updates_at_stop;
  int count;                  // consecutive stale steps
  int have_prev;
  int stopped;                // halts the parameter updates
  int pad;
};
// gamma, t and updates are the step's, read from sc.  With ann_below > 0 a
// step whose annealing sum falls below it also stops the run; patience 0
// disables the stale-step rule.
void early_stop_launch(const float* terms, const float* lambda, int S, float tol, int patience,
                       float ann_below, const StepScalars* sc, EarlyStopState* st,
                       cudaStream_t stream);
// ---------------------------------------------------------------- warm start (k_warm.cu)
// Node features [N x F]: 1, deg/8, then N(0,1) from the stream of `seed`.
void ws_features_launch(int64_t N, const int* rowptr, uint64_t seed, int F, float* out,
                        cudaStream_t st);
void inv_degree_launch(int64_t N, const int* rowptr, float* inv, cudaStream_t st);
// Binary cross-entropy of logits Z [N x ldz] against target bits [N x ceil(S/32)]:
// G = (sigmoid(Z) - y) * inv_count (dtype dg, pad columns up to S_pad zeroed);
// per-block loss sums to partial[grid]; returns the grid.
int ws_bce_launch(int64_t N, int S, int S_pad, const float* Z, int64_t ldz, const uint32_t* bits,
                  void* G, int64_t ldg, int dg, float inv_count, float* partial, int max_grid,
                  cudaStream_t st);
// Per-block column sums of X [N x C] (dtype dx) over contiguous row ranges
// into partial[blocks][C]; returns the number of blocks (<= max_blocks).
int rows_colsum_launch(int64_t N, int C, const void* X, int64_t ldx, int dx, float* partial,
                       int max_blocks, cudaStream_t st);
// BF16 copies Ws [rows_pad x cols] and Wt [cols x rows_pad] of FP32 W [rows x cols].
void weight_pair_launch(const float* W, int rows, int cols, int rows_pad, void* Ws, void* Wt,
                        cudaStream_t st);

// dst[i*ld + k] = value for k < S, 0 for S <= k < ld.
void fill_rows_launch(int64_t N, int S, int64_t ld, float value, float* dst, cudaStream_t st);
void copy_rows_launch(int64_t N, int H, const float* src, void* dst, int64_t ldd,
                      int ddst, cudaStream_t st);
// BF16 shadows of the dense weights:
//   W1s [H1 x 2H0] = Wcat1, W1t [2H0 x H1] = Wcat1^T,
//   W2s [S_pad x 2H1] = Wcat2 (pad rows 0), W2t [2H1 x S_pad] = Wcat2^T (pad cols 0).
void weight_shadows_launch(const float* theta, int H0, int H1, int S, int S_pad,
                           void* W1s, void* W1t, void* W2s, void* W2t, cudaStream_t st);
// FP32 form on the tensor cores: the dense weights split exactly into three
// TF32 parts (split3: hi, mid, lo), in the layouts of the BF16 shadows (W1:
// H1 x 2H0 and its transpose; W2: S_pad x 2H1, rows past S zero, and its
// transpose).  W[k] is part k (0 hi, 1 mid, 2 lo); Wt[k] its transpose.
void weight_split_launch(const float* theta, int H0, int H1, int S, int S_pad, float* const* W1,
                         float* const* W1t, float* const* W2, float* const* W2t, cudaStream_t st);
// ORs bits into the device error word (bit 2, value 4: a kernel could not be
// set up and its product was not computed).
void flag_error_launch(int* flag, int bits, cudaStream_t st);
void init_uniform_launch(float* p, int64_t n, float bound, uint64_t seed,
                         uint64_t tag, cudaStream_t st);
void init_normal_launch(float* p, int64_t n, uint64_t seed, uint64_t tag,
                        cudaStream_t st);
void upcast_rows_launch(int64_t N, int S, const void* src, int64_t lds, int dsrc,
                        float* dst, cudaStream_t st);
// out[0..3S] = terms[0..3S] (cost, pen, ann per shot, Psi) and
// out[3S+1] = R = sum_s (cost_s + lambda_s pen_s) + gamma sum_s ann_s + nu Psi
// (lambda NULL: no penalty term), summed in a fixed order in FP64.
void total_loss_launch(const float* terms, const float* lambda, int S, float gamma, float nu,
                       float* out, cudaStream_t st);
// dst[i] = scale * src[i]
void scale_copy_launch(int64_t n, float scale, const float* src, float* dst, cudaStream_t st);

// Failures of the in-kernel CSR checks of the checked build (csr_row /
// csr_col in common.cuh): how many checks failed (a bad row or index counts
// once per lane and launch that reads it), the smallest row with a bad range
// and the smallest CSR position with a bad column index (INT64_MAX if none).
struct CsrCheck {
  unsigned long long count = 0;
  long long first_row = 0x7fffffffffffffffLL;
  long long first_entry = 0x7fffffffffffffffLL;
};
#ifdef CPRA_CHECKED
void csr_check_collect_spmm(CsrCheck* r);
void csr_check_collect_eval(CsrCheck* r);
template <int PROBLEM> void csr_check_collect_loss(CsrCheck* r);
template <> void csr_check_collect_loss<0>(CsrCheck* r);
template <> void csr_check_collect_loss<1>(CsrCheck* r);
template <> void csr_check_collect_loss<2>(CsrCheck* r);
template <> void csr_check_collect_loss<3>(CsrCheck* r);
template <> void csr_check_collect_loss<4>(CsrCheck* r);
#endif

}  // namespace cpra
