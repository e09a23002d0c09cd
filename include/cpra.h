/*
 * cpra.h -- C ABI of the GB300 (sm_103a) implementation of one training step
 * of CPRA, the continuous parallel relaxation annealing solver of Ichikawa &
 * Iwashita, "Continuous Parallel Relaxation for Finding Diverse Solutions in
 * Combinatorial Optimization Problems".
 *
 * One step = GNN forward (Eq. GCN, App. B.1, two layers as in App. C.1)
 *          -> S relaxed QUBO losses with the annealing term and, optionally,
 *             the shot-diversity term (Eq. CPRA-loss-function-GNN-penalty and
 *             Eq. CPRA-loss-function-GNN-variation)
 *          -> hand-written adjoint -> Adam
 *          -> rounding x = 1[P > 0.5] (App. C.2) and integer evaluation of all
 *             S shots (MIS / MaxCut objectives of Table objective-functions).
 *
 * Conventions for every entry point
 *   - Plain C types only.  "host" pointers are ordinary CPU memory; "device"
 *     pointers are CUDA global memory of the current device.
 *   - Host input arrays are read during the call and never retained; the
 *     caller keeps ownership.  Outputs go to caller-allocated buffers.
 *   - No entry point aborts or throws.  Errors are returned as cpra_status;
 *     cpra_last_error() gives a message for context calls.
 *   - Graph input: symmetric CSR, rowptr int64[N+1] with rowptr[0] = 0,
 *     col int32[nnz] with 0 <= col < N, strictly increasing within each row
 *     (no duplicates), no self-loops, and (i,j) present iff (j,i) present.
 *     nnz = 2|E| must be < 2^31.  Isolated nodes are allowed (their mean
 *     aggregation is 0).  Anything else is CPRA_EINVAL.
 *   - Matrices are row-major.  P and the shot-indexed buffers use a row
 *     stride S_pad = round_up(S, 16) elements; pad columns are never read as
 *     data.
 */
#ifndef CPRA_H
#define CPRA_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define CPRA_API __attribute__((visibility("default")))
#else
#define CPRA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CPRA_OK = 0,
  CPRA_EINVAL = 1,   /* bad argument, graph or configuration              */
  CPRA_ENOMEM = 2,   /* device allocation failed or exceeds mem_cap_bytes  */
  CPRA_ECUDA = 3,    /* a CUDA runtime / driver call failed                */
  CPRA_ENUMERIC = 4, /* non-finite loss term detected                      */
  CPRA_ETIMEOUT = 5, /* a bounded device-side wait gave up                 */
  CPRA_ESTATE = 6    /* state blob does not match this context             */
} cpra_status;

enum { CPRA_MIS = 0, CPRA_MAXCUT = 1,                 /* Table objective-functions */
       CPRA_WMIS = 2,    /* weighted MIS: shot s solves the MIS QUBO with node weights
                            w_:s (the task family of the paper's two-stage experiment);
                            weights from cpra_set_node_weights, 1 until set */
       CPRA_DBM = 3 };   /* diverse bipartite matching (Eq. matching-cost-function):
                            node i*N2 + j is the pair variable x_ij; shot s has its
                            own instance (C, M, lambda_1..4, p, q) from cpra_set_dbm */
enum { CPRA_FP32 = 0, CPRA_BF16 = 1 };                /* dense-layer arithmetic   */
enum { CPRA_FP32_TENSOR = 0, CPRA_FP32_CUDA_CORES = 1 };  /* engine of the FP32 form */
enum { CPRA_DIV_STD = 0, CPRA_DIV_VAR = 1 };          /* Psi form                 */

/* Configuration.  cpra_config_default() fills every field. */
typedef struct cpra_config {
  int32_t problem;          /* CPRA_MIS, CPRA_MAXCUT, CPRA_WMIS or CPRA_DBM       */
  int32_t S;                /* shots = columns of P, 1..1024                      */
  int32_t H0;               /* node-embedding width (multiple of 16, <= 4096)    */
  int32_t H1;               /* hidden width (multiple of 16, <= 4096)            */
  int32_t alpha;            /* even exponent of the annealing term, >= 2          */
  int32_t precision;        /* CPRA_FP32: all FP32; CPRA_BF16: dense layers BF16
                               on tensor cores with FP32 accumulation             */
  int32_t recompute;        /* 1: H1 is not kept for the backward (only its ReLU
                               mask, as bits written by the layer-1 GEMM), so the
                               activation blocks [X0|M1], [H1|M2] share memory
                               with the gradient blocks (2 N (H0 + H1) values
                               less, N H1 / 8 bytes more)                      */
  int32_t train_embedding;  /* 1: node embeddings h^0 are trained (default)       */
  int32_t diversity_kind;   /* CPRA_DIV_STD (Eq. ...-variation) or CPRA_DIV_VAR   */
  int32_t keep_emb_grad;    /* 0 (default): cpra_step fuses the embedding Adam
                               step into the last backward aggregation and does
                               not store dR/dh^0; 1: it also stores dR/dh^0
                               (CPRA_T_EMB_GRAD), 512 MB more HBM traffic per
                               10^6 x 128 embedding                             */
  const float* lambda;      /* host [S], penalty lambda_s per shot ((W)MIS);
                               copied at init; may be NULL for MaxCut and DBM (not
                               read: DBM penalties come with cpra_set_dbm)         */
  float nu;                 /* diversity weight (0 disables Psi)                  */
  float gamma0, gamma1;     /* annealing: gamma_t linear from gamma0 to gamma1    */
  int64_t schedule_steps;   /*   over t = 0 .. schedule_steps-1                   */
  float lr, beta1, beta2, eps;
  float weight_decay;       /* 0: Adam; > 0: decoupled AdamW decay                */
  uint64_t seed;            /* parameter / embedding initialisation              */
  uint64_t mem_cap_bytes;   /* 0: none; else init fails with CPRA_ENOMEM when the
                               device workspace would exceed it                    */
  float es_tol;             /* early stopping (Implementation paragraph): a step
                               is stale when both the penalty-form loss
                               sum_s (cost_s + lambda_s pen_s) and the annealing
                               term gamma_t sum_s ann_s rose or changed by at
                               most es_tol (absolute, FP64 sums over s in
                               order); after es_patience consecutive stale
                               steps the step that completes the run stops:
                               it and every later cpra_step leave parameters
                               and Adam state unchanged                      */
  int32_t es_patience;      /* 0: no early stopping                             */
  float es_ann_below;       /* > 0: a step whose annealing term sum_s ann_s is
                               below this value also stops the run (the two-stage
                               experiment's rule); 0: off                       */
  int32_t train_encoder;    /* 1 (default): all parameters train; 0: only the
                               head [B2|W2], b2 trains (the fine-tuning stage of
                               the two-stage schedule); layer 1 and the
                               embeddings keep their values                    */
  int32_t fp32_engine;      /* FP32 form only.  CPRA_FP32_TENSOR (default): the
                               dense layers and input gradients run on the
                               tensor cores with split-TF32 operands (each FP32
                               value exactly as three TF32 parts; six products
                               per pair, FP32 accumulation: FP32 accuracy);
                               shapes the tensor-core kernel does not take, and
                               the weight gradients, stay on CUDA cores.
                               CPRA_FP32_CUDA_CORES: every dense product on
                               CUDA cores.  Ignored by the BF16 form          */
} cpra_config;

/* Result of rounding one shot (App. C.2) and evaluating it exactly. */
typedef struct cpra_shot_eval {
  int64_t objective;   /* (W)MIS: |{i : x_i = 1}|;  MaxCut: number of cut edges;
                          DBM: matched pairs sum_ij x_ij                       */
  int64_t violations;  /* (W)MIS: edges with both ends in the set; MaxCut: 0;
                          DBM: rows and columns with more than one pair plus the
                          diversity constraints (of 2) that fail               */
  double qubo;         /* l(x): -value + lambda_s * violations ((W)MIS);
                          -value (MaxCut); Eq. matching-cost-function (DBM), FP64 */
  double value;        /* objective in the problem's units: set size, total
                          weight sum_i w_is x_is (WMIS, FP64), cut size,
                          reward sum_ij C_ij x_ij (DBM, FP64)                  */
} cpra_shot_eval;

typedef struct cpra_ctx cpra_ctx;

/* Fills *cfg with defaults: MIS, S = 8, H0 = H1 = 16, alpha = 2, FP32,
   recompute 0, train_embedding 1, keep_emb_grad 0, DIV_STD, nu = 0,
   gamma -2 -> 0.1 over 3000 steps, Adam lr 1e-3, betas (0.9, 0.999),
   eps 1e-8, wd 0, seed 1, no early stopping (es_patience 0, es_tol 1e-5,
   es_ann_below 0), train_encoder 1, fp32_engine CPRA_FP32_TENSOR. */
CPRA_API void cpra_config_default(cpra_config* cfg);

/* Number of trainable GNN parameters excluding node embeddings:
   2*H1*H0 + H1 + 2*S*H1 + S (self weight, neighbour weight and bias per
   layer; this reproduces the counts printed in the Experiments section's
   tables, e.g. 5,083,076 for H0 = H1 = 1584, S = 20). */
CPRA_API int64_t cpra_param_count_for(int32_t H0, int32_t H1, int32_t S);

/* Device bytes a context needs for this graph size and configuration
   (0 if the configuration is invalid). */
CPRA_API size_t cpra_workspace_bytes(int64_t N, int64_t nnz, const cpra_config* cfg);

/* Creates a context: validates and uploads the graph (host CSR, see
   conventions), copies cfg and lambda, and initialises theta ~
   U(+-1/sqrt(fan_in)) and h^0 ~ N(0,1) from cfg->seed.
   w: host float[nnz], the edge weight A_ij of each CSR entry, or NULL for
   unit weights.  Weights enter the MaxCut QUBO of Table objective-functions,
   sum_{i<j} A_ij (2 x_i x_j - x_i - x_j): the relaxed cost, its gradient
   2 (A P)_i - sum_j A_ij, and the records (objective = number of cut edges,
   value = cut weight sum of A_ij over cut edges in FP64, qubo = -value;
   cpra_solve ranks shots by value).  The GNN's mean aggregation stays
   unweighted.  They must be finite and symmetric (the two entries of an
   edge equal); with another problem, or otherwise, CPRA_EINVAL.  The
   context keeps a device copy (its own allocation, freed by cpra_destroy).
   dev_workspace: device buffer of >= cpra_workspace_bytes() bytes owned by
   the caller for the context's lifetime, or NULL to let the library
   allocate (and free in cpra_destroy).  cuda_stream: cudaStream_t to order
   all work on, or NULL for a stream owned by the context.  On failure *out
   is NULL. */
CPRA_API cpra_status cpra_init_graph(cpra_ctx** out, int64_t N, const int64_t* rowptr,
                            const int32_t* col, const float* w,
                            const cpra_config* cfg, void* dev_workspace,
                            size_t workspace_bytes, void* cuda_stream);

/* One training step at schedule index t (gamma_t = gamma0 + (gamma1 -
   gamma0) * t / (schedule_steps - 1), clamped).  Runs forward, loss, adjoint,
   Adam (bias-corrected with the context's own step counter, which this call
   increments) and the rounding/evaluation of the P of this step's forward.
   loss_terms_out: host float[3S+1] receiving cost_s (S), pen_s (S), ann_s (S)
   and Psi, or NULL.  Asynchronous on the context stream when NULL; otherwise
   synchronises and returns CPRA_ENUMERIC if a term is not finite. */
CPRA_API cpra_status cpra_step(cpra_ctx* ctx, int64_t t, float* loss_terms_out);

/* Differentiable form of the same computation (for autograd frameworks).
 * cpra_forward copies theta (device float [param_count], flat layout of
 * CPRA_T_THETA) and the node embeddings h^0 (device float [N x H0]) into the
 * context, runs the GNN forward (Eq. GCN twice, App. C.1) and the fused loss
 * at the given gamma (Eq. CPRA-loss-function-GNN-penalty / -variation) and
 * writes terms_dev (device float [3S+2]): cost_s (S), pen_s (S), ann_s (S),
 * Psi, then the total R = sum_s (cost_s + lambda_s pen_s) + gamma sum_s ann_s
 * + nu Psi.  It also evaluates the rounded shots (cpra_round_eval reads it).
 * cpra_backward runs the hand-written adjoint of the last cpra_forward and
 * writes scale * dR/dtheta (device float [param_count]) and, unless
 * grad_emb_dev is NULL, scale * dR/dh^0 (device float [N x H0]).  Neither
 * call touches the Adam state or the step counter.  cpra_backward returns
 * CPRA_ESTATE if no cpra_forward precedes it (cpra_step, cpra_set_tensor and
 * cpra_set_state invalidate the forward).  Both are asynchronous on the
 * context stream. */
CPRA_API cpra_status cpra_forward(cpra_ctx* ctx, const float* theta_dev, const float* emb_dev,
                                  float gamma, float* terms_dev);
CPRA_API cpra_status cpra_backward(cpra_ctx* ctx, float scale, float* grad_theta_dev,
                                   float* grad_emb_dev);

/* n consecutive steps with schedule indices t0 .. t0+n-1, the same as n
   cpra_step calls without loss readback: the first runs directly, the rest
   replay one step captured as a CUDA graph (captured on the first call that
   needs it, with the context stream; per-step values such as gamma_t and
   the Adam bias corrections are computed on the device).  Asynchronous. */
CPRA_API cpra_status cpra_steps(cpra_ctx* ctx, int64_t t0, int64_t n);

/* Copies the evaluation of the most recent cpra_step (or, before any step,
   of a fresh forward pass) to the host.  out: host [S]; pair_hamming_sum:
   host int64 receiving sum_i k_i (S - k_i) = sum_{s<l} d_H(x_s, x_l)
   (Prop. 3.2), or NULL; x_bits_out: host uint32 [N][ceil(S/32)] with bit
   (s mod 32) of word s/32 = x_is, or NULL.  Synchronises. */
CPRA_API cpra_status cpra_round_eval(cpra_ctx* ctx, cpra_shot_eval* out,
                            int64_t* pair_hamming_sum, uint32_t* x_bits_out);

/* Runs `steps` steps starting at schedule index 0 and, every eval_every
   steps and after the last, tracks per shot the best evaluation: MIS the
   largest objective with violations == 0 (objective -1 if none seen),
   weighted MIS the largest value with violations == 0 (value -1 if none),
   MaxCut the largest cut (with edge weights, the largest cut weight).  best_out: host [S]; best_step_out: host [S] step
   index of that evaluation (or -1), may be NULL.  With es_patience > 0 the
   loop ends at the first evaluation after early stopping fired (the
   parameters are frozen from the stopping step on). */
CPRA_API cpra_status cpra_solve(cpra_ctx* ctx, int64_t steps, int64_t eval_every,
                       cpra_shot_eval* best_out, int64_t* best_step_out);

/* Metrics log (JSON Lines): with a path, cpra_solve appends one JSON object
   per evaluation to that file, opened for appending:
     {"t": step index evaluated, "gamma": gamma_t, "steps": steps since the
      previous evaluation, "seconds": their wall time with this evaluation,
      "elapsed": seconds since the cpra_solve call began, "psi": Psi,
      "pair_hamming": sum_i k_i (S - k_i) of the rounded shots,
      "cost" / "pen" / "ann": [S] loss terms of step t,
      "objective" / "violations" / "value": [S] records of step t's rounding}
   -- the quantities the paper's early stopping monitors (Implementation
   paragraph) and the solution quality per evaluation.  Logging costs one
   host copy of 3S+1 floats per evaluation.  path NULL closes the log; the
   context closes it in cpra_destroy.  Errors: CPRA_EINVAL (the file cannot
   be opened; cpra_solve returns it when a write fails). */
CPRA_API cpra_status cpra_set_metrics_log(cpra_ctx* ctx, const char* path);

/* Weighted MIS (problem CPRA_WMIS): node weights w [N x ld] float (ld >= S),
   w_is for node i in shot s, on the host (on_device = 0) or the current
   device (on_device = 1); copied into the context's workspace.
   Synchronises.  Errors: CPRA_EINVAL (not a WMIS context, NULL, ld < S). */
CPRA_API cpra_status cpra_set_node_weights(cpra_ctx* ctx, const float* w, int64_t ld,
                                           int32_t on_device);

/* Diverse bipartite matching instances (problem CPRA_DBM; Eq.
   matching-cost-function, App. problem specification).  The graph given to
   cpra_init_graph has N = N1 * N2 nodes, node i*N2 + j being the pair
   variable x_ij (i < N1 on one side, j < N2 on the other).  Shot s carries
   its own instance: C and M are float [N x ld] (ld >= S, row-major),
   C[(i*N2+j)*ld + s] the reward C_ij of shot s and M[...] its field
   indicator (1: i and j are in different fields, 0: the same field; any
   value in [0, 1] is accepted); lam4 is float [S x 4], the penalties
   (lambda_1, lambda_2, lambda_3, lambda_4) of shot s, and pq float [S x 2]
   its diversity shares (p, q).  All on the host.  The penalty grid (one
   instance repeated, S penalty vectors) and multi-instance CPRA (S
   instances, one penalty vector; App. multi-instance) are both this layout.
   The library copies them into device memory it allocates itself (2 N
   round_up(S,16) floats plus line buffers of about 6 (N1 + N2) round_up(S,16)
   floats, counted against mem_cap_bytes, freed by cpra_destroy).  Required
   before the first step, forward or evaluation of a DBM context; a later call
   with the same N1 replaces the instances in place.  Synchronises.  Errors:
   CPRA_EINVAL (not a DBM context, a NULL array, ld < S, N1 < 1 or not dividing
   N, a non-finite value, p or q or M outside [0, 1]), CPRA_ENOMEM. */
CPRA_API cpra_status cpra_set_dbm(cpra_ctx* ctx, int32_t N1, const float* C, const float* M,
                                  int64_t ld, const float* lam4, const float* pq);

/* Schedule index t of the cpra_step at which early stopping fired, or -1
   (also when es_patience is 0).  Synchronises. */
CPRA_API int64_t cpra_early_stop_step(cpra_ctx* ctx);

/* Warm start: a fixed per-node, per-shot offset L0 added to the head's
   pre-activation, Z2 = [H1|M2] Wcat2^T + b2 + L0, so that P = sigma(Z2)
   starts near sigma(L0) while the GCN output is small; the paper's
   neighbourhood of this idea is its meta-learned initialisation and
   two-stage training (Related work; App. C.4).  logits: float [N x ld]
   (ld >= S), row-major, on the host (on_device = 0) or the current device
   (on_device = 1); the library keeps a copy in the dense layers' dtype
   (bfloat16 in the BF16 form) in device memory it allocates itself
   (N x round_up(S,16) values, counted against mem_cap_bytes, freed by
   cpra_destroy).  NULL removes the offset.  Synchronises.  Errors:
   CPRA_EINVAL (ld < S), CPRA_ENOMEM. */
CPRA_API cpra_status cpra_set_init_logits(cpra_ctx* ctx, const float* logits, int64_t ld,
                                          int32_t on_device);

/* Tensors a context exposes for checkpoints, tests and inspection. */
enum {
  CPRA_T_THETA = 0,     /* float [param_count] flat: Wcat1=[B1|W1] (H1 x 2H0),
                           b1 (H1), Wcat2=[B2|W2] (S x 2H1), b2 (S)          */
  CPRA_T_THETA_M = 1,   /* float [param_count] Adam first moment              */
  CPRA_T_THETA_V = 2,   /* float [param_count] Adam second moment             */
  CPRA_T_EMB = 3,       /* float [N x H0] node embeddings h^0 (FP32 master)   */
  CPRA_T_EMB_M = 4,     /* float [N x H0]                                     */
  CPRA_T_EMB_V = 5,     /* float [N x H0]                                     */
  CPRA_T_GRAD = 6,      /* float [param_count] dR/dtheta of the last step     */
  CPRA_T_EMB_GRAD = 7,  /* float [N x H0] dR/dh^0 of the last cpra_step with
                           keep_emb_grad = 1 (or of the last cpra_backward)  */
  CPRA_T_P = 8,         /* float [N x S] P of the last forward                */
  CPRA_T_GZ2 = 9,       /* float [N x S] dR/dZ2 of the last step (upcast)     */
  CPRA_T_STEP = 10,     /* int64 [1] Adam step counter                        */
  CPRA_T_TERMS = 11,    /* float [3S+1] loss terms of the last step           */
  CPRA_T_COUNT_ = 12
};

/* Size in bytes of tensor `which` (0 if unknown). */
CPRA_API size_t cpra_tensor_bytes(const cpra_ctx* ctx, int32_t which);
/* Copies tensor `which` to / from host memory of exactly nbytes.
   Synchronises.  Setting CPRA_T_THETA or CPRA_T_EMB refreshes the BF16
   shadows used by the dense layers. */
CPRA_API cpra_status cpra_get_tensor(cpra_ctx* ctx, int32_t which, void* host, size_t nbytes);
CPRA_API cpra_status cpra_set_tensor(cpra_ctx* ctx, int32_t which, const void* host, size_t nbytes);

/* Checkpoint: opaque blob with theta, its Adam moments, the embeddings and
   their moments, and the step counter.  With buf == NULL, *nbytes receives
   the size.  cpra_set_state checks the header against the context
   (CPRA_ESTATE on mismatch).  Resuming reproduces an uninterrupted run
   bit for bit. */
CPRA_API cpra_status cpra_get_state(cpra_ctx* ctx, void* buf, size_t* nbytes);
CPRA_API cpra_status cpra_set_state(cpra_ctx* ctx, const void* buf, size_t nbytes);

/* host [N x S] float: P of the last forward. */
CPRA_API cpra_status cpra_get_P(cpra_ctx* ctx, float* host_NxS);

CPRA_API int64_t cpra_param_count(const cpra_ctx* ctx);
/* Kernel launches issued by this context so far. */
CPRA_API int64_t cpra_launch_count(const cpra_ctx* ctx);

/* Per-kernel device timing.  While enabled, each step records CUDA events
   around its kernels on the context stream.  cpra_profile_read synchronises
   and returns, per kernel id (see cpra_kernel_name), the summed device
   milliseconds and the launch count since the last read, then resets them. */
CPRA_API void cpra_profile_enable(cpra_ctx* ctx, int on);
CPRA_API int32_t cpra_profile_read(cpra_ctx* ctx, double* ms_out, int64_t* launches_out,
                          int32_t n_ids);
CPRA_API const char* cpra_kernel_name(int32_t id);

/* Fault-injection hook for tests of the failure paths (no counterpart in the
   paper).  ORs `bits` into the context's device error word on the context
   stream, exactly as a kernel does when one of its bounded waits gives up
   (bit 1, value 2: CPRA_ETIMEOUT) or when a loss term is not finite (bit 0,
   value 1: CPRA_ENUMERIC).  The next call that reads the word -- cpra_step
   with loss_terms_out non-NULL, or cpra_solve at its next evaluation --
   returns that status (CPRA_ETIMEOUT first if both bits are set) and clears
   the word; the context stays usable.  No GPU fault is involved.  Errors:
   CPRA_EINVAL (NULL ctx, bits outside 1..3), CPRA_ECUDA. */
CPRA_API cpra_status cpra_inject_error_flag(cpra_ctx* ctx, int32_t bits);

/* Message of the last error on ctx; with ctx == NULL, the message of the
   last failed cpra_init_graph on the calling thread. */
CPRA_API const char* cpra_last_error(const cpra_ctx* ctx);
CPRA_API const char* cpra_status_string(cpra_status s);
CPRA_API void cpra_destroy(cpra_ctx* ctx);

/* ------------------------------------------------------------------------
 * Op-level entry points on caller-owned DEVICE memory, ordered on
 * `cuda_stream` (NULL = legacy default stream).  They allocate nothing.
 * ---------------------------------------------------------------------- */

/* Fused SpMM + relaxed loss (the step's loss stage).  For every node i and
 * shot s < S, with Q = A P (A the unit-weight adjacency of the CSR):
 *   MIS:    cost_s = -sum_i P_is,  pen_s = 1/2 sum_i P_is Q_is
 *           dR/dP_is = -1 + lambda_s Q_is + ...
 *   MaxCut: cost_s = sum_i P_is Q_is - sum_i deg_i P_is,  pen_s = 0
 *           dR/dP_is = 2 Q_is - deg_i + ...
 *   both:   ann_s = sum_i 1 - (2P_is - 1)^alpha,
 *           ... - 2 alpha gamma (2P_is - 1)^(alpha-1) + nu dPsi/dP_is
 *   Psi = -S sum_i STD_s(P_i.)  (DIV_STD; gradient 0 on rows with VAR = 0)
 *       = -S^2 sum_i VAR_s(P_i.) (DIV_VAR)
 * (Eq. CPRA-loss-function-GNN-penalty / -variation, Table
 * objective-functions.)  Q is never stored.
 *   rowptr, col : device int32 [N+1], [nnz]: rowptr nondecreasing from 0
 *                 to nnz, 0 <= col[e] < N.  These device arrays are not
 *                 checked by the normal build (entries outside these bounds
 *                 make the kernels read outside the arrays); the checked
 *                 build tests them in the kernels (cpra_csr_check).
 *   P           : device float [N x ldp], ldp >= S, ldp % 4 == 0
 *   lambda      : device float [S] (MIS; ignored for MaxCut, may be NULL)
 *   grad_kind   : 0 -> G = dR/dP * P (1 - P)  (= dR/dZ2 under a sigmoid head)
 *                 1 -> G = dR/dP
 *   G           : device float [N x ldg], ldg >= S, ldg % 4 == 0; columns
 *                 S..ldg-1 are written 0
 *   x_bits      : device uint32 [N x ceil(S/32)] rounded P (x = P > 0.5f),
 *                 or NULL
 *   terms       : device float [4S+1]: cost_s, pen_s, ann_s, Psi, then
 *                 sum_i G_is per shot (S)
 *   scratch     : device, >= cpra_op_loss_scratch_bytes(N, S) bytes
 * Results are deterministic (fixed-order reductions). */
CPRA_API size_t cpra_op_loss_scratch_bytes(int64_t N, int32_t S);
CPRA_API cpra_status cpra_op_loss(int64_t N, int32_t S, const int32_t* rowptr,
                         const int32_t* col, const float* P, int64_t ldp,
                         const float* lambda, int32_t problem, int32_t alpha,
                         float gamma, float nu, int32_t diversity_kind,
                         int32_t grad_kind, float* G, int64_t ldg,
                         uint32_t* x_bits, float* terms, void* scratch,
                         size_t scratch_bytes, void* cuda_stream);

/* Rounding + exact integer evaluation of S shots from P (App. C.2):
 * x_is = 1[P_is > 0.5f]; per shot objective / violations / qubo as in
 * cpra_shot_eval (qubo reduced in FP64), and sum_i k_i (S - k_i).
 *   P        : device float [N x ldp]
 *   x_bits   : device uint32 [N x ceil(S/32)] work/output buffer
 *   lambda   : device float [S] (MIS) or NULL
 *   out      : device cpra_shot_eval [S]
 *   pair_hamming : device int64 [1]
 *   counters : device, >= cpra_op_round_eval_scratch_bytes(S) bytes
 * Bit-exact and deterministic (integer reductions). */
CPRA_API size_t cpra_op_round_eval_scratch_bytes(int32_t S);
CPRA_API cpra_status cpra_op_round_eval(int64_t N, int32_t S, const int32_t* rowptr,
                               const int32_t* col, const float* P, int64_t ldp,
                               const float* lambda, int32_t problem,
                               uint32_t* x_bits, cpra_shot_eval* out,
                               int64_t* pair_hamming, void* counters,
                               size_t counters_bytes, void* cuda_stream);

/* Checked build.  libcpra_checked.so is this library compiled with
 * CPRA_CHECKED: every kernel that walks the graph (the aggregations, the fused
 * loss, the integer evaluation, the warm-start network's aggregations) tests
 * each row range it reads against 0 <= rowptr[i] <= rowptr[i+1] <= rowptr[N]
 * and each column index against 0 <= col[e] < N before using it.  A failing
 * row is read as empty and a failing index as node 0, so no access leaves
 * the arrays; the launch completes and its results are undefined.  There is
 * no trap and no device assert: the failures are counted in device words.
 * (The device CSR of a context was validated on the host by
 * cpra_init_graph; the op-level calls and cpra_ws_* take device CSR arrays
 * as given.)
 * cpra_csr_check synchronises the device, returns the number of checks that
 * failed since the previous call (a bad row or index is counted once for
 * every lane and launch that reads it) and clears the words; *first_row
 * receives the smallest row whose range failed and *first_entry the
 * smallest CSR position whose column index failed (-1 for none; either
 * pointer may be NULL).  -2 if the synchronisation reports a CUDA error.
 * The normal build returns -1 and writes -1. */
CPRA_API int64_t cpra_csr_check(int64_t* first_row, int64_t* first_entry);

/* Allocation-free variant of cpra_op_loss.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- code
 * embedded in an application that owns all device memory through its own
 * pool or a fixed budget, and latency-critical paths where an allocation
 * (and the device synchronisation it can imply) is not acceptable.
 * Arguments and results are those of cpra_op_loss without the scratch
 * buffer: the kernel's per-block partial sums live in a fixed device
 * array of about 8.4 MB inside the library, which every GPU that loads the
 * library holds until the process exits.
 *   - S must be <= CPRA_NOALLOC_MAX_S; larger S returns CPRA_EINVAL without
 *     launching anything.  N is not limited.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress); make that first call before any stream
 *     capture.  With CUDA's default lazy module loading that first call is
 *     also when the device reserves the array, so a caller with a fixed
 *     memory budget should make it at start-up, before it commits its own
 *     pool; if the device has no room for the array then, the call returns
 *     CPRA_ENOMEM.
 *   - Every call on a device shares the one array, which keeps the last
 *     call's contents; each call writes every partial row before reading
 *     it, so nothing needs clearing.  Calls that overlap on the GPU
 *     (unordered streams, concurrent host threads) race on the array:
 *     order them on one stream.
 *   - Allocates nothing: no cudaMalloc, cudaFree or allocating library call. */
#define CPRA_NOALLOC_MAX_S 1024
CPRA_API cpra_status cpra_op_loss_noalloc(int64_t N, int32_t S, const int32_t* rowptr,
                                          const int32_t* col, const float* P, int64_t ldp,
                                          const float* lambda, int32_t problem, int32_t alpha,
                                          float gamma, float nu, int32_t diversity_kind,
                                          int32_t grad_kind, float* G, int64_t ldg,
                                          uint32_t* x_bits, float* terms, void* cuda_stream);

/* ------------------------------------------------------------------------
 * Warm-start network.  A three-layer GCN with the layer of Eq. GCN (self
 * weight B, neighbour weight W on the row-mean aggregate, bias; ReLU after
 * layers 1 and 2) maps fixed node features (1, deg/8 and F-2 standard
 * normal draws per node from a seeded counter-based stream) to S logits per
 * node.  It is trained with the mean binary cross-entropy against rounded
 * CPRA solutions x_is, and its logits seed a CPRA run through
 * cpra_set_init_logits.  The paper has no such network; its nearest ideas
 * are the meta-learned initialisation and the two-stage (S' -> S) training
 * it discusses.  Graph arguments are DEVICE pointers: rowptr int32 [N+1],
 * col int32 [nnz] (symmetric CSR, the layout of cpra_init_graph),
 * features float [N x F], target bits uint32 [N x ceil(S/32)] with bit
 * (s mod 32) of word s/32 = x_is (cpra_round_eval's layout), logits float
 * [N x ld].  All calls are ordered on the network's stream.
 * ------------------------------------------------------------------------ */
typedef struct cpra_ws cpra_ws;
typedef struct cpra_ws_config {
  int32_t F;           /* feature width, multiple of 16, >= 16             */
  int32_t H;           /* hidden width, multiple of 16                     */
  int32_t S;           /* logits per node (shots), 1..1024                 */
  int32_t precision;   /* CPRA_FP32 or CPRA_BF16 (dense layers)            */
  float lr, beta1, beta2, eps, weight_decay;   /* Adam / AdamW            */
  uint64_t seed;       /* parameter initialisation                         */
} cpra_ws_config;

/* F = 16, H = 64, S = 32, BF16, Adam lr 1e-3 (0.9, 0.999, 1e-8), wd 0, seed 1. */
CPRA_API void cpra_ws_config_default(cpra_ws_config* cfg);
/* Flat parameter layout: Wcat1 = [B1|W1] (H x 2F), b1 (H), Wcat2 (H x 2H),
   b2 (H), Wcat3 (S x 2H), b3 (S); 0 for an invalid configuration. */
CPRA_API int64_t cpra_ws_param_count(const cpra_ws_config* cfg);
/* Creates a network for graphs of up to max_nodes nodes and max_nnz CSR
   entries (its activations are sized for them and allocated by the
   library).  Parameters: U(+-1/sqrt(fan_in)) from cfg->seed.  Errors:
   CPRA_EINVAL, CPRA_ENOMEM, CPRA_ECUDA. */
CPRA_API cpra_status cpra_ws_create(cpra_ws** out, const cpra_ws_config* cfg, int64_t max_nodes,
                                    int64_t max_nnz, void* cuda_stream);
/* Writes the node features of a graph (see above) to features [N x F]. */
CPRA_API cpra_status cpra_ws_features(cpra_ws* ws, int64_t N, const int32_t* rowptr,
                                      uint64_t graph_seed, float* features);
/* One training step on one graph (or a disjoint union of graphs): forward,
   mean binary cross-entropy over the N x S logits, hand-written adjoint,
   Adam.  loss_out: host float receiving the loss, or NULL (then no
   synchronisation).  Errors: CPRA_EINVAL (N or nnz above the sizes given at
   creation), CPRA_ECUDA, CPRA_ETIMEOUT. */
CPRA_API cpra_status cpra_ws_train_step(cpra_ws* ws, int64_t N, int64_t nnz,
                                        const int32_t* rowptr, const int32_t* col,
                                        const float* features, const uint32_t* target_bits,
                                        float* loss_out);
/* Forward only: logits [N x ld] (ld >= S).  Graphs larger than the sizes
   given at creation are processed in node order through the same buffers
   only if they fit; otherwise CPRA_EINVAL. */
CPRA_API cpra_status cpra_ws_predict(cpra_ws* ws, int64_t N, int64_t nnz, const int32_t* rowptr,
                                     const int32_t* col, const float* features, float* logits,
                                     int64_t ld);
/* Host copies of the flat parameters (float [cpra_ws_param_count]); gradient
   of the last training step with which = 1.  Synchronise. */
CPRA_API cpra_status cpra_ws_get_params(cpra_ws* ws, int32_t which, float* host, size_t count);
CPRA_API cpra_status cpra_ws_set_params(cpra_ws* ws, const float* host, size_t count);
CPRA_API void cpra_ws_destroy(cpra_ws* ws);

#ifdef __cplusplus
}
#endif
#endif /* CPRA_H */
