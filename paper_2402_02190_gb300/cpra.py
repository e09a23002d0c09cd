"""Python binding of the CPRA C ABI (include/cpra.h).

Argument marshalling only: every step of the method runs in the CUDA kernels
of libcpra.so.  PyTorch supplies device memory (the context workspace and
op-level buffers) and the CUDA stream.  There is no CPU fallback: if the
library is missing or no GPU is present, calls raise.

Module-level functions carry the C names (``cpra_init_graph``, ``cpra_step``,
``cpra_round_eval``, ``cpra_solve``, ``cpra_op_loss`` ...).  ``Solver`` is a
small convenience wrapper around one context.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libcpra.so")
# the checked build: in-kernel CSR bound checks, read through cpra_csr_check
LIB_CHECKED_PATH = os.path.join(_HERE, "lib", "libcpra_checked.so")
_LIB_PATHS = {"release": LIB_PATH, "checked": LIB_CHECKED_PATH}

CPRA_OK, CPRA_EINVAL, CPRA_ENOMEM, CPRA_ECUDA, CPRA_ENUMERIC, CPRA_ETIMEOUT, CPRA_ESTATE = range(7)
MIS, MAXCUT, WMIS, DBM = 0, 1, 2, 3
FP32, BF16 = 0, 1
DIV_STD, DIV_VAR = 0, 1
FP32_TENSOR, FP32_CUDA_CORES = 0, 1
(T_THETA, T_THETA_M, T_THETA_V, T_EMB, T_EMB_M, T_EMB_V, T_GRAD, T_EMB_GRAD, T_P, T_GZ2,
 T_STEP, T_TERMS) = range(12)

ABI_FUNCTIONS = (
    "cpra_config_default", "cpra_param_count_for", "cpra_workspace_bytes", "cpra_init_graph",
    "cpra_step", "cpra_round_eval", "cpra_solve", "cpra_tensor_bytes", "cpra_get_tensor",
    "cpra_set_tensor", "cpra_get_state", "cpra_set_state", "cpra_get_P", "cpra_param_count",
    "cpra_launch_count", "cpra_profile_enable", "cpra_profile_read", "cpra_kernel_name",
    "cpra_last_error", "cpra_status_string", "cpra_destroy", "cpra_op_loss_scratch_bytes",
    "cpra_op_loss", "cpra_op_round_eval_scratch_bytes", "cpra_op_round_eval",
    "cpra_op_loss_noalloc", "cpra_forward", "cpra_backward", "cpra_early_stop_step",
    "cpra_set_init_logits", "cpra_steps", "cpra_set_node_weights", "cpra_set_dbm",
    "cpra_inject_error_flag", "cpra_ws_config_default", "cpra_ws_param_count", "cpra_ws_create",
    "cpra_ws_features", "cpra_ws_train_step", "cpra_ws_predict", "cpra_ws_get_params",
    "cpra_ws_set_params", "cpra_ws_destroy", "cpra_csr_check", "cpra_set_metrics_log",
)
NOALLOC_MAX_S = 1024


class CpraError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"cpra status {status}: {msg}")
        self.status = status


class Config(C.Structure):
    _fields_ = [
        ("problem", C.c_int32), ("S", C.c_int32), ("H0", C.c_int32), ("H1", C.c_int32),
        ("alpha", C.c_int32), ("precision", C.c_int32), ("recompute", C.c_int32),
        ("train_embedding", C.c_int32), ("diversity_kind", C.c_int32), ("keep_emb_grad", C.c_int32),
        ("lambda_", C.POINTER(C.c_float)), ("nu", C.c_float), ("gamma0", C.c_float),
        ("gamma1", C.c_float), ("schedule_steps", C.c_int64), ("lr", C.c_float),
        ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
        ("weight_decay", C.c_float), ("seed", C.c_uint64), ("mem_cap_bytes", C.c_uint64),
        ("es_tol", C.c_float), ("es_patience", C.c_int32), ("es_ann_below", C.c_float),
        ("train_encoder", C.c_int32), ("fp32_engine", C.c_int32),
    ]


class WsConfig(C.Structure):
    _fields_ = [
        ("F", C.c_int32), ("H", C.c_int32), ("S", C.c_int32), ("precision", C.c_int32),
        ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
        ("weight_decay", C.c_float), ("seed", C.c_uint64),
    ]


class ShotEval(C.Structure):
    _fields_ = [("objective", C.c_int64), ("violations", C.c_int64), ("qubo", C.c_double),
                ("value", C.c_double)]


SHOT_EVAL_DTYPE = np.dtype([("objective", "<i8"), ("violations", "<i8"), ("qubo", "<f8"),
                            ("value", "<f8")])

_libs = {}
_variant = os.environ.get("CPRA_LIBRARY", "release")


def use_library(variant: str) -> str:
    """Selects the library the module-level calls go to: "release"
    (libcpra.so) or "checked" (libcpra_checked.so).  Returns the previous
    choice.  A context belongs to the library that created it: switch only
    between contexts, never with one open."""
    global _variant
    if variant not in _LIB_PATHS:
        raise ValueError(f"unknown library variant {variant!r}")
    prev, _variant = _variant, variant
    return prev


def lib():
    """Loads the selected library (raises if it has not been built)."""
    if _variant in _libs:
        return _libs[_variant]
    path = _LIB_PATHS[_variant]
    if not os.path.exists(path):
        raise ImportError(
            f"{path} is missing: build it with paper_2402_02190_gb300.build.build()")
    L = C.CDLL(path)
    vp, i32, i64, f32, sz = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_size_t
    P_cfg = C.POINTER(Config)
    sigs = {
        "cpra_config_default": (None, [P_cfg]),
        "cpra_param_count_for": (i64, [i32, i32, i32]),
        "cpra_workspace_bytes": (sz, [i64, i64, P_cfg]),
        "cpra_init_graph": (C.c_int, [C.POINTER(vp), i64, vp, vp, vp, P_cfg, vp, sz, vp]),
        "cpra_step": (C.c_int, [vp, i64, vp]),
        "cpra_forward": (C.c_int, [vp, vp, vp, f32, vp]),
        "cpra_backward": (C.c_int, [vp, f32, vp, vp]),
        "cpra_round_eval": (C.c_int, [vp, vp, vp, vp]),
        "cpra_solve": (C.c_int, [vp, i64, i64, vp, vp]),
        "cpra_tensor_bytes": (sz, [vp, i32]),
        "cpra_get_tensor": (C.c_int, [vp, i32, vp, sz]),
        "cpra_set_tensor": (C.c_int, [vp, i32, vp, sz]),
        "cpra_get_state": (C.c_int, [vp, vp, C.POINTER(sz)]),
        "cpra_set_state": (C.c_int, [vp, vp, sz]),
        "cpra_get_P": (C.c_int, [vp, vp]),
        "cpra_param_count": (i64, [vp]),
        "cpra_launch_count": (i64, [vp]),
        "cpra_early_stop_step": (i64, [vp]),
        "cpra_inject_error_flag": (i32, [vp, i32]),
        "cpra_steps": (i32, [vp, i64, i64]),
        "cpra_set_node_weights": (i32, [vp, vp, i64, i32]),
        "cpra_set_dbm": (i32, [vp, i32, vp, vp, i64, vp, vp]),
        "cpra_set_init_logits": (i32, [vp, vp, i64, i32]),
        "cpra_profile_enable": (None, [vp, C.c_int]),
        "cpra_profile_read": (i32, [vp, vp, vp, i32]),
        "cpra_kernel_name": (C.c_char_p, [i32]),
        "cpra_last_error": (C.c_char_p, [vp]),
        "cpra_status_string": (C.c_char_p, [C.c_int]),
        "cpra_destroy": (None, [vp]),
        "cpra_ws_config_default": (None, [vp]),
        "cpra_ws_param_count": (i64, [vp]),
        "cpra_ws_create": (i32, [vp, vp, i64, i64, vp]),
        "cpra_ws_features": (i32, [vp, i64, vp, C.c_uint64, vp]),
        "cpra_ws_train_step": (i32, [vp, i64, i64, vp, vp, vp, vp, vp]),
        "cpra_ws_predict": (i32, [vp, i64, i64, vp, vp, vp, vp, i64]),
        "cpra_ws_get_params": (i32, [vp, i32, vp, sz]),
        "cpra_ws_set_params": (i32, [vp, vp, sz]),
        "cpra_ws_destroy": (None, [vp]),
        "cpra_op_loss_scratch_bytes": (sz, [i64, i32]),
        "cpra_op_loss": (C.c_int, [i64, i32, vp, vp, vp, i64, vp, i32, i32, f32, f32, i32, i32,
                                   vp, i64, vp, vp, vp, sz, vp]),
        "cpra_op_loss_noalloc": (C.c_int, [i64, i32, vp, vp, vp, i64, vp, i32, i32, f32, f32,
                                           i32, i32, vp, i64, vp, vp, vp]),
        "cpra_csr_check": (i64, [vp, vp]),
        "cpra_set_metrics_log": (i32, [vp, C.c_char_p]),
        "cpra_op_round_eval_scratch_bytes": (sz, [i32]),
        "cpra_op_round_eval": (C.c_int, [i64, i32, vp, vp, vp, i64, vp, i32, vp, vp, vp, vp, sz,
                                         vp]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _libs[_variant] = L
    return L


def cpra_csr_check():
    """(failed checks since the last call, smallest bad row, smallest bad CSR
    position) from the checked build; (-1, -1, -1) from the release build."""
    row, ent = C.c_int64(-1), C.c_int64(-1)
    n = lib().cpra_csr_check(C.byref(row), C.byref(ent))
    return int(n), int(row.value), int(ent.value)


def _check(status: int, ctx=None):
    if status != CPRA_OK:
        L = lib()
        msg = L.cpra_last_error(ctx).decode() if ctx is not None else L.cpra_last_error(None).decode()
        raise CpraError(status, msg or L.cpra_status_string(status).decode())


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _stream_handle(stream):
    if stream is None:
        import torch
        if not torch.cuda.is_available():
            return None
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def cpra_config_default() -> Config:
    cfg = Config()
    lib().cpra_config_default(C.byref(cfg))
    return cfg


def make_config(**kw) -> Config:
    cfg = cpra_config_default()
    for k, v in kw.items():
        if k == "lambda_":
            raise ValueError("pass lambda to cpra_init_graph / Solver")
        setattr(cfg, k, v)
    return cfg


def cpra_param_count_for(H0: int, H1: int, S: int) -> int:
    return int(lib().cpra_param_count_for(H0, H1, S))


def cpra_workspace_bytes(N: int, nnz: int, cfg: Config) -> int:
    return int(lib().cpra_workspace_bytes(N, nnz, C.byref(cfg)))


def cpra_init_graph(rowptr, col, cfg: Config, lam=None, workspace=None, stream=None,
                    weights=None):
    """Returns (ctx handle, workspace tensor or None).  ``workspace`` may be a
    torch uint8 CUDA tensor; with ``workspace='torch'`` one of the right size
    is allocated by PyTorch's caching allocator.  ``weights``: per-CSR-entry
    edge weights A_ij (MaxCut), or None for unit weights."""
    import torch
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    N = len(rowptr) - 1
    lam_arr = None
    if lam is not None:
        lam_arr = np.ascontiguousarray(lam, dtype=np.float32)
        if lam_arr.size != cfg.S:
            raise ValueError("lambda must have S entries")
        cfg.lambda_ = lam_arr.ctypes.data_as(C.POINTER(C.c_float))
    ws_ptr, ws_bytes = None, 0
    if isinstance(workspace, str) and workspace == "torch":
        nb = cpra_workspace_bytes(N, int(rowptr[-1]), cfg)
        if nb == 0:
            raise CpraError(CPRA_EINVAL, "invalid configuration")
        workspace = torch.empty(nb, dtype=torch.uint8, device="cuda")
    if workspace is not None:
        ws_ptr, ws_bytes = C.c_void_p(workspace.data_ptr()), workspace.numel()
    w_arr = None
    if weights is not None:
        w_arr = np.ascontiguousarray(weights, dtype=np.float32)
        if w_arr.size != col.size:
            raise ValueError("weights must have one entry per CSR entry")
    h = C.c_void_p()
    st = lib().cpra_init_graph(C.byref(h), N, _ptr(rowptr), _ptr(col) if col.size else None,
                               _ptr(w_arr) if w_arr is not None and w_arr.size else None,
                               C.byref(cfg), ws_ptr, ws_bytes, _stream_handle(stream))
    cfg.lambda_ = None
    _check(st)
    return h, workspace


def cpra_step(ctx, t: int, want_terms: bool = False):
    if want_terms:
        S = (lib().cpra_tensor_bytes(ctx, T_TERMS) // 4 - 1) // 3
        out = np.empty(3 * S + 1, dtype=np.float32)
        _check(lib().cpra_step(ctx, t, _ptr(out)), ctx)
        return out
    _check(lib().cpra_step(ctx, t, None), ctx)
    return None


def cpra_forward(ctx, theta, emb, gamma: float, terms) -> None:
    """theta, emb, terms: torch CUDA float32 tensors (contiguous)."""
    _check(lib().cpra_forward(ctx, C.c_void_p(theta.data_ptr()), C.c_void_p(emb.data_ptr()),
                              C.c_float(gamma), C.c_void_p(terms.data_ptr())), ctx)


def cpra_backward(ctx, scale: float, grad_theta, grad_emb=None) -> None:
    _check(lib().cpra_backward(ctx, C.c_float(scale), C.c_void_p(grad_theta.data_ptr()),
                               C.c_void_p(grad_emb.data_ptr()) if grad_emb is not None else None),
           ctx)


def _S_of(ctx):
    return (lib().cpra_tensor_bytes(ctx, T_TERMS) // 4 - 1) // 3


def cpra_round_eval(ctx, want_bits: bool = False, N: int | None = None):
    S = _S_of(ctx)
    rec = np.zeros(S, dtype=SHOT_EVAL_DTYPE)
    ham = np.zeros(1, dtype=np.int64)
    bits = None
    if want_bits:
        if N is None:
            N = lib().cpra_tensor_bytes(ctx, T_P) // (4 * S)
        bits = np.zeros((N, (S + 31) // 32), dtype=np.uint32)
    _check(lib().cpra_round_eval(ctx, _ptr(rec), _ptr(ham), _ptr(bits) if bits is not None else None),
           ctx)
    return rec, int(ham[0]), bits


def cpra_solve(ctx, steps: int, eval_every: int):
    S = _S_of(ctx)
    rec = np.zeros(S, dtype=SHOT_EVAL_DTYPE)
    st = np.zeros(S, dtype=np.int64)
    _check(lib().cpra_solve(ctx, steps, eval_every, _ptr(rec), _ptr(st)), ctx)
    return rec, st


_TENSOR_DTYPES = {T_STEP: np.int64}


def cpra_get_tensor(ctx, which: int) -> np.ndarray:
    nb = lib().cpra_tensor_bytes(ctx, which)
    dt = _TENSOR_DTYPES.get(which, np.float32)
    out = np.empty(nb // np.dtype(dt).itemsize, dtype=dt)
    _check(lib().cpra_get_tensor(ctx, which, _ptr(out), nb), ctx)
    return out


def cpra_set_tensor(ctx, which: int, arr) -> None:
    dt = _TENSOR_DTYPES.get(which, np.float32)
    a = np.ascontiguousarray(arr, dtype=dt).ravel()
    _check(lib().cpra_set_tensor(ctx, which, _ptr(a), a.nbytes), ctx)


def cpra_get_state(ctx) -> bytes:
    n = C.c_size_t(0)
    _check(lib().cpra_get_state(ctx, None, C.byref(n)), ctx)
    buf = np.empty(n.value, dtype=np.uint8)
    _check(lib().cpra_get_state(ctx, _ptr(buf), C.byref(n)), ctx)
    return buf.tobytes()


def cpra_set_state(ctx, blob: bytes) -> None:
    buf = np.frombuffer(blob, dtype=np.uint8).copy()
    _check(lib().cpra_set_state(ctx, _ptr(buf), buf.nbytes), ctx)


def cpra_get_P(ctx, N: int, S: int) -> np.ndarray:
    out = np.empty((N, S), dtype=np.float32)
    _check(lib().cpra_get_P(ctx, _ptr(out)), ctx)
    return out


def cpra_param_count(ctx) -> int:
    return int(lib().cpra_param_count(ctx))


def cpra_launch_count(ctx) -> int:
    return int(lib().cpra_launch_count(ctx))


def cpra_set_node_weights(ctx, w) -> None:
    """Weighted MIS node weights: a host array [N, S] or a CUDA tensor [N, S]."""
    if hasattr(w, "is_cuda") and w.is_cuda:
        t = w.float().contiguous()
        _check(lib().cpra_set_node_weights(ctx, C.c_void_p(t.data_ptr()), t.shape[1], 1), ctx)
        return
    a = np.ascontiguousarray(w, dtype=np.float32)
    _check(lib().cpra_set_node_weights(ctx, _ptr(a), a.shape[1], 0), ctx)


def cpra_set_dbm(ctx, N1: int, C_rew, M, lam4, pq) -> None:
    """Matching instances of a DBM context: C_rew, M host arrays [N, S]
    (node i*N2 + j, shot s), lam4 [S, 4] = (lambda_1..4), pq [S, 2] = (p, q)."""
    c = np.ascontiguousarray(C_rew, dtype=np.float32)
    m = np.ascontiguousarray(M, dtype=np.float32)
    l4 = np.ascontiguousarray(lam4, dtype=np.float32)
    pqa = np.ascontiguousarray(pq, dtype=np.float32)
    if c.shape != m.shape or c.ndim != 2 or l4.shape != (c.shape[1], 4) or pqa.shape != (c.shape[1], 2):
        raise ValueError("cpra_set_dbm: C, M [N, S], lam4 [S, 4], pq [S, 2]")
    _check(lib().cpra_set_dbm(ctx, int(N1), _ptr(c), _ptr(m), c.shape[1], _ptr(l4), _ptr(pqa)), ctx)


def cpra_steps(ctx, t0: int, n: int) -> None:
    _check(lib().cpra_steps(ctx, int(t0), int(n)), ctx)


def cpra_inject_error_flag(ctx, bits: int) -> None:
    """Fault injection for tests: sets the context's device error word as a
    kernel whose bounded wait gave up (bits=2) or that produced a non-finite
    loss term (bits=1) would."""
    _check(lib().cpra_inject_error_flag(ctx, int(bits)), ctx)


def cpra_early_stop_step(ctx) -> int:
    return int(lib().cpra_early_stop_step(ctx))


def cpra_set_init_logits(ctx, logits) -> None:
    """logits: None, a host array [N, S] or a CUDA tensor [N, S] (float32)."""
    if logits is None:
        _check(lib().cpra_set_init_logits(ctx, None, 0, 0), ctx)
        return
    if hasattr(logits, "is_cuda") and logits.is_cuda:
        t = logits.float().contiguous()
        _check(lib().cpra_set_init_logits(ctx, C.c_void_p(t.data_ptr()), t.shape[1], 1), ctx)
        return
    a = np.ascontiguousarray(logits, dtype=np.float32)
    _check(lib().cpra_set_init_logits(ctx, _ptr(a), a.shape[1], 0), ctx)


def paper_preset(problem: int, max_steps: int = 50_000) -> dict:
    """Configuration keywords of the paper's experiments (Implementation
    paragraph): AdamW lr 1e-4, weight decay 1e-2; gamma(0) = -20 for MIS and
    -6 for MaxCut rising by 1e-3 per step (a linear schedule over max_steps);
    alpha = 2; early stopping with tolerance 1e-5 and patience 1000."""
    g0 = -6.0 if problem == MAXCUT else -20.0
    return dict(lr=1e-4, weight_decay=1e-2, gamma0=g0, gamma1=g0 + 1e-3 * (max_steps - 1),
                schedule_steps=max_steps, alpha=2, es_tol=1e-5, es_patience=1000)


def cpra_profile_enable(ctx, on: bool = True) -> None:
    lib().cpra_profile_enable(ctx, 1 if on else 0)


def cpra_profile_read(ctx) -> dict:
    ms = np.zeros(64, dtype=np.float64)
    n = np.zeros(64, dtype=np.int64)
    k = lib().cpra_profile_read(ctx, _ptr(ms), _ptr(n), 64)
    return {lib().cpra_kernel_name(i).decode(): (float(ms[i]), int(n[i])) for i in range(k)}


def cpra_destroy(ctx) -> None:
    if ctx:
        lib().cpra_destroy(ctx)


# ------------------------------------------------------------------ op level
def cpra_op_loss_scratch_bytes(N: int, S: int) -> int:
    return int(lib().cpra_op_loss_scratch_bytes(N, S))


def cpra_op_loss(rowptr32, col32, P, lam, problem, alpha, gamma, nu, div_kind, grad_kind,
                 G, x_bits, terms, scratch, stream=None):
    """All array arguments are torch CUDA tensors (lam / x_bits may be None)."""
    N, S = P.shape[0], terms.numel() // 4
    st = lib().cpra_op_loss(
        N, S, C.c_void_p(rowptr32.data_ptr()), C.c_void_p(col32.data_ptr()),
        C.c_void_p(P.data_ptr()), P.stride(0),
        C.c_void_p(lam.data_ptr()) if lam is not None else None, problem, alpha,
        C.c_float(gamma), C.c_float(nu), div_kind, grad_kind, C.c_void_p(G.data_ptr()),
        G.stride(0), C.c_void_p(x_bits.data_ptr()) if x_bits is not None else None,
        C.c_void_p(terms.data_ptr()), C.c_void_p(scratch.data_ptr()), scratch.numel(),
        _stream_handle(stream))
    _check(st)


def cpra_op_loss_noalloc(rowptr32, col32, P, lam, problem, alpha, gamma, nu, div_kind,
                         grad_kind, G, x_bits, terms, stream=None):
    """cpra_op_loss without a scratch argument, for callers that cannot
    allocate device memory (the library keeps a fixed device array for its
    partial sums).  S is limited to NOALLOC_MAX_S; calls must not overlap on
    the GPU."""
    N, S = P.shape[0], terms.numel() // 4
    if S > NOALLOC_MAX_S:
        raise CpraError(CPRA_EINVAL,
                        f"S={S} exceeds the allocation-free limit of {NOALLOC_MAX_S} shots")
    st = lib().cpra_op_loss_noalloc(
        N, S, C.c_void_p(rowptr32.data_ptr()), C.c_void_p(col32.data_ptr()),
        C.c_void_p(P.data_ptr()), P.stride(0),
        C.c_void_p(lam.data_ptr()) if lam is not None else None, problem, alpha,
        C.c_float(gamma), C.c_float(nu), div_kind, grad_kind, C.c_void_p(G.data_ptr()),
        G.stride(0), C.c_void_p(x_bits.data_ptr()) if x_bits is not None else None,
        C.c_void_p(terms.data_ptr()), _stream_handle(stream))
    _check(st)


def cpra_op_round_eval_scratch_bytes(S: int) -> int:
    return int(lib().cpra_op_round_eval_scratch_bytes(S))


def cpra_op_round_eval(rowptr32, col32, P, S, lam, problem, x_bits, out_records, pair_hamming,
                       counters, stream=None):
    N = P.shape[0]
    if out_records.numel() * out_records.element_size() < S * SHOT_EVAL_DTYPE.itemsize:
        raise ValueError("out_records holds fewer than S cpra_shot_eval records")
    st = lib().cpra_op_round_eval(
        N, S, C.c_void_p(rowptr32.data_ptr()), C.c_void_p(col32.data_ptr()),
        C.c_void_p(P.data_ptr()), P.stride(0),
        C.c_void_p(lam.data_ptr()) if lam is not None else None, problem,
        C.c_void_p(x_bits.data_ptr()), C.c_void_p(out_records.data_ptr()),
        C.c_void_p(pair_hamming.data_ptr()), C.c_void_p(counters.data_ptr()), counters.numel(),
        _stream_handle(stream))
    _check(st)


class Solver:
    """One CPRA context on the current CUDA device."""

    def __init__(self, rowptr, col, lam=None, stream=None, weights=None, **cfg_kw):
        import torch
        self.cfg = make_config(**cfg_kw)
        self.N = len(rowptr) - 1
        self.S = self.cfg.S
        # A dedicated torch stream: its handle is what the library orders all
        # work on, so torch events recorded on it time the library's kernels.
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.ctx, self._ws = cpra_init_graph(rowptr, col, self.cfg, lam=lam, workspace="torch",
                                             stream=self.stream, weights=weights)

    def step(self, t: int, want_terms: bool = False):
        return cpra_step(self.ctx, t, want_terms)

    def round_eval(self, want_bits: bool = False):
        return cpra_round_eval(self.ctx, want_bits, self.N)

    def solve(self, steps: int, eval_every: int):
        return cpra_solve(self.ctx, steps, eval_every)

    def set_metrics_log(self, path) -> None:
        """cpra_solve appends one JSON line per evaluation to `path` (None
        closes the log)."""
        _check(lib().cpra_set_metrics_log(
            self.ctx, None if path is None else os.fsencode(path)), self.ctx)

    def set_node_weights(self, w) -> None:
        if hasattr(w, "is_cuda") and w.is_cuda:
            import torch
            self.stream.wait_stream(torch.cuda.current_stream())
        cpra_set_node_weights(self.ctx, w)

    def set_dbm(self, N1: int, C_rew, M, lam4, pq) -> None:
        cpra_set_dbm(self.ctx, N1, C_rew, M, lam4, pq)

    def steps(self, t0: int, n: int) -> None:
        cpra_steps(self.ctx, t0, n)

    def early_stop_step(self) -> int:
        return cpra_early_stop_step(self.ctx)

    def set_init_logits(self, logits) -> None:
        if hasattr(logits, "is_cuda") and logits.is_cuda:
            import torch
            # the copy runs on the solver's stream: order it after the producer
            self.stream.wait_stream(torch.cuda.current_stream())
        cpra_set_init_logits(self.ctx, logits)

    def get(self, which: int) -> np.ndarray:
        return cpra_get_tensor(self.ctx, which)

    def set(self, which: int, arr) -> None:
        cpra_set_tensor(self.ctx, which, arr)

    def P(self) -> np.ndarray:
        return cpra_get_P(self.ctx, self.N, self.S)

    @property
    def param_count(self) -> int:
        return cpra_param_count(self.ctx)

    @property
    def launches(self) -> int:
        return cpra_launch_count(self.ctx)

    def close(self) -> None:
        if self.ctx:
            cpra_destroy(self.ctx)
            self.ctx = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ warm start
def ws_config(**kw) -> WsConfig:
    cfg = WsConfig()
    lib().cpra_ws_config_default(C.byref(cfg))
    for k, v in kw.items():
        if not hasattr(cfg, k):
            raise AttributeError(k)
        setattr(cfg, k, v)
    return cfg


def cpra_ws_param_count(cfg: WsConfig) -> int:
    return int(lib().cpra_ws_param_count(C.byref(cfg)))


class WarmStartNet:
    """The warm-start network of the C ABI (cpra_ws_*).  Graph tensors are
    CUDA tensors: rowptr/col int32, features float32 [N, F], target bits
    uint32 stored as int32 [N, ceil(S/32)]."""

    def __init__(self, max_nodes: int, max_nnz: int, stream=None, **cfg_kw):
        import torch
        self.cfg = ws_config(**cfg_kw)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        h = C.c_void_p()
        st = lib().cpra_ws_create(C.byref(h), C.byref(self.cfg), int(max_nodes), int(max_nnz),
                                  C.c_void_p(self.stream.cuda_stream))
        if st != CPRA_OK:
            raise CpraError(st, f"cpra_ws_create failed ({st})")
        self.ws = h
        self.nparam = cpra_ws_param_count(self.cfg)

    def _wait(self):
        import torch
        self.stream.wait_stream(torch.cuda.current_stream())

    @staticmethod
    def _p(t):
        return C.c_void_p(t.data_ptr())

    def features(self, rowptr, graph_seed: int):
        import torch
        self._wait()
        N = rowptr.numel() - 1
        out = torch.empty((N, self.cfg.F), dtype=torch.float32, device=rowptr.device)
        _check(lib().cpra_ws_features(self.ws, N, self._p(rowptr), C.c_uint64(graph_seed),
                                      self._p(out)))
        out.record_stream(self.stream)
        torch.cuda.current_stream().wait_stream(self.stream)
        return out

    def train_step(self, rowptr, col, features, target_bits, want_loss: bool = True):
        import torch
        self._wait()
        loss = C.c_float(0.0)
        _check(lib().cpra_ws_train_step(self.ws, rowptr.numel() - 1, col.numel(), self._p(rowptr),
                                        self._p(col), self._p(features), self._p(target_bits),
                                        C.byref(loss) if want_loss else None))
        for t in (rowptr, col, features, target_bits):
            t.record_stream(self.stream)
        return float(loss.value) if want_loss else None

    def predict(self, rowptr, col, features):
        import torch
        self._wait()
        N = rowptr.numel() - 1
        S = self.cfg.S
        ld = (S + 3) // 4 * 4
        out = torch.empty((N, ld), dtype=torch.float32, device=rowptr.device)
        _check(lib().cpra_ws_predict(self.ws, N, col.numel(), self._p(rowptr), self._p(col),
                                     self._p(features), self._p(out), ld))
        out.record_stream(self.stream)
        torch.cuda.current_stream().wait_stream(self.stream)
        return out[:, :S]

    def params(self, which: int = 0) -> np.ndarray:
        out = np.empty(self.nparam, dtype=np.float32)
        _check(lib().cpra_ws_get_params(self.ws, which, _ptr(out), out.size))
        return out

    def set_params(self, theta) -> None:
        a = np.ascontiguousarray(theta, dtype=np.float32)
        _check(lib().cpra_ws_set_params(self.ws, _ptr(a), a.size))

    def close(self) -> None:
        if self.ws:
            lib().cpra_ws_destroy(self.ws)
            self.ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

