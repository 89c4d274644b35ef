"""Python binding of libiaskit.so (INV-ASKIT on one GB300, arXiv 1602.01376).

Argument marshalling only: every step of the factorization and the solve runs in
the library's CUDA kernels.  Host arrays are numpy; device arrays are torch CUDA
tensors (used only as device memory).  There is no CPU fallback: if the shared
library cannot be loaded, every call raises.

Function names follow the C ABI in include/iaskit.h.
"""
from __future__ import annotations

import ctypes
import json
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libiaskit.so")

IASKIT_OK = 0
ERRORS = {
    -1: "IASKIT_ERR_ARG",
    -2: "IASKIT_ERR_INPUT",
    -3: "IASKIT_ERR_NOMEM",
    -4: "IASKIT_ERR_SINGULAR",
    -5: "IASKIT_ERR_NOT_FACTORED",
    -6: "IASKIT_ERR_NOT_CONVERGED",
    -7: "IASKIT_ERR_TIMEOUT",
    -8: "IASKIT_ERR_CUDA",
    -9: "IASKIT_ERR_UNSUPPORTED",
}
EXPORTS = [
    "iaskit_factor", "iaskit_factor_device", "iaskit_solve", "iaskit_solve_device",
    "iaskit_apply", "iaskit_apply_device", "iaskit_set_option", "iaskit_get_option",
    "iaskit_set_stream", "iaskit_stats", "iaskit_last_error", "iaskit_free", "iaskit_depth",
    "iaskit_get_perm", "iaskit_get_knn", "iaskit_get_ranks", "iaskit_get_skeleton",
    "iaskit_get_samples", "iaskit_get_P", "iaskit_knn_noalloc", "iaskit_factor_batched",
    "iaskit_factor_batched_device", "iaskit_num_problems", "iaskit_solve_batched",
    "iaskit_solve_batched_device", "iaskit_sampler_train", "iaskit_sampler_set_weights",
    "iaskit_sampler_get_weights", "iaskit_mlp_forward", "iaskit_mlp_train_step", "iaskit_get_learned",
    "iaskit_kernel_block", "iaskit_refactor", "iaskit_predict", "iaskit_predict_device",
    "iaskit_gemm_tile", "iaskit_tune_gemm",
]

MLP_NPARAM = 17793


class IaskitError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


_lib: Optional[ctypes.CDLL] = None

_c_double_p = ctypes.POINTER(ctypes.c_double)
_c_int32_p = ctypes.POINTER(ctypes.c_int32)


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libiaskit.so (build it first with ``paper_1602_01376_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: run paper_1602_01376_gb300.build.build() first")
    lib = ctypes.CDLL(path)
    i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
    sig = {
        "iaskit_factor": ([vp, i64, i32, dbl, dbl, i32, i32, dbl], i32),
        "iaskit_factor_device": ([vp, i64, i32, dbl, dbl, i32, i32, dbl], i32),
        "iaskit_solve": ([vp, i32], i32),
        "iaskit_solve_device": ([vp, i32], i32),
        "iaskit_apply": ([vp, vp, i32], i32),
        "iaskit_apply_device": ([vp, vp, i32], i32),
        "iaskit_set_option": ([ctypes.c_char_p, dbl], i32),
        "iaskit_get_option": ([ctypes.c_char_p, _c_double_p], i32),
        "iaskit_set_stream": ([vp], i32),
        "iaskit_stats": ([ctypes.c_char_p, ctypes.c_size_t], i32),
        "iaskit_last_error": ([], ctypes.c_char_p),
        "iaskit_free": ([], None),
        "iaskit_depth": ([], i32),
        "iaskit_get_perm": ([vp], i32),
        "iaskit_get_knn": ([vp, i32], i32),
        "iaskit_get_ranks": ([vp, i32], i32),
        "iaskit_get_skeleton": ([i32, i32, vp, i32], i32),
        "iaskit_get_samples": ([i32, i32, vp, i32], i32),
        "iaskit_get_P": ([i32, i32, vp, i64], i32),
        "iaskit_knn_noalloc": ([vp, i64, i32, i32, vp, vp], i32),
        "iaskit_factor_batched": ([i32, vp, vp, i32, vp, vp, i32, i32, dbl], i32),
        "iaskit_factor_batched_device": ([i32, vp, vp, i32, vp, vp, i32, i32, dbl], i32),
        "iaskit_num_problems": ([], i32),
        "iaskit_refactor": ([vp, i32], i32),
        "iaskit_predict": ([vp, i64, vp, i32, vp], i32),
        "iaskit_predict_device": ([vp, i64, vp, i32, vp], i32),
        "iaskit_gemm_tile": ([i32, i32, i32, i32], i32),
        "iaskit_tune_gemm": ([i32, i32, i32, i32, i32, i32, i32, _c_double_p], i32),
        "iaskit_solve_batched": ([vp, i32], i32),
        "iaskit_solve_batched_device": ([vp, i32], i32),
        "iaskit_sampler_train": ([vp, i64, i32, dbl, i32, i32, dbl, i32, dbl], i32),
        "iaskit_sampler_set_weights": ([vp, i32], i32),
        "iaskit_sampler_get_weights": ([vp, i32], i32),
        "iaskit_mlp_forward": ([vp, i64, vp], i32),
        "iaskit_mlp_train_step": ([vp, vp, i64, dbl, vp, vp], i32),
        "iaskit_get_learned": ([i32, i32, vp, vp, vp, i32, vp], i32),
        "iaskit_kernel_block": ([vp, i64, i32, dbl, vp, i32, vp, i32, dbl, i32, vp], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    load_tile_table()   # the committed autotuned grouped-GEMM tile shapes, when present
    return lib


def _check(rc: int) -> int:
    if rc < 0:
        raise IaskitError(rc, _lib.iaskit_last_error().decode())
    return rc


def _host_f64(a, order="C") -> np.ndarray:
    return np.require(np.asarray(a, dtype=np.float64), requirements=[order[0], "A", "W"])


def _dev_ptr(t) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float64:
        raise TypeError("expected a CUDA float64 torch tensor")
    return t.data_ptr()


# ------------------------------------------------------------------ public calls
def iaskit_factor(points, h: float, lam: float, leaf_m: int, s_max: int, tol: float) -> None:
    """Factorize lambda I + K~ for host points (N x d float64)."""
    lib = load()
    X = _host_f64(points, "C")
    N, d = X.shape
    _check(lib.iaskit_factor(X.ctypes.data, N, d, h, lam, leaf_m, s_max, tol))


def iaskit_factor_device(points, h: float, lam: float, leaf_m: int, s_max: int, tol: float) -> None:
    """Factorize from a CUDA float64 tensor of shape (N, d), row-major contiguous."""
    lib = load()
    if not points.is_contiguous():
        raise ValueError("points must be contiguous")
    N, d = points.shape
    _check(lib.iaskit_factor_device(_dev_ptr(points), N, d, h, lam, leaf_m, s_max, tol))


def iaskit_factor_batched(points_list, h_list, lam_list, leaf_m: int, s_max: int, tol: float) -> None:
    """Factor independent problems together (host arrays, one (N_q, d) array each)."""
    lib = load()
    Xs = [_host_f64(x, "C") for x in points_list]
    q = len(Xs)
    d = Xs[0].shape[1]
    ptrs = (ctypes.c_void_p * q)(*[x.ctypes.data for x in Xs])
    Ns = np.array([x.shape[0] for x in Xs], dtype=np.int64)
    hs = np.asarray(h_list, dtype=np.float64)
    ls = np.asarray(lam_list, dtype=np.float64)
    _check(lib.iaskit_factor_batched(q, ptrs, Ns.ctypes.data, d, hs.ctypes.data, ls.ctypes.data,
                                     leaf_m, s_max, tol))


def iaskit_factor_batched_device(points, Ns, h_list, lam_list, leaf_m: int, s_max: int,
                                 tol: float) -> None:
    """Factor independent problems from one CUDA float64 tensor (sum N_q, d)."""
    lib = load()
    Nv = np.asarray(Ns, dtype=np.int64)
    hs = np.asarray(h_list, dtype=np.float64)
    ls = np.asarray(lam_list, dtype=np.float64)
    _check(lib.iaskit_factor_batched_device(len(Nv), _dev_ptr(points), Nv.ctypes.data,
                                            points.shape[1], hs.ctypes.data, ls.ctypes.data,
                                            leaf_m, s_max, tol))


def iaskit_num_problems() -> int:
    return _check(load().iaskit_num_problems())


def iaskit_refactor(lam) -> None:
    """Refactor the current factorization for new lambda values (a scalar for a single
    problem, else one value per problem in batch order); tree, kNN lists, skeletons and
    P are kept."""
    lib = load()
    ls = np.ascontiguousarray(np.atleast_1d(np.asarray(lam, dtype=np.float64)))
    _check(lib.iaskit_refactor(ls.ctypes.data, len(ls)))


def iaskit_solve_batched(rhs_list) -> list:
    """Solve every problem of a batch; rhs_list[q] is (N_q,) or (N_q, nrhs)."""
    lib = load()
    arrs = [np.array(np.asarray(u, dtype=np.float64).reshape(len(u), -1), order="F", copy=True)
            for u in rhs_list]
    nrhs = arrs[0].shape[1]
    ptrs = (ctypes.c_void_p * len(arrs))(*[a.ctypes.data for a in arrs])
    _check(lib.iaskit_solve_batched(ptrs, nrhs))
    return [a[:, 0] if np.asarray(u).ndim == 1 else a for a, u in zip(arrs, rhs_list)]


def iaskit_solve_batched_device(rhs, nrhs: int) -> None:
    """In place on one contiguous CUDA float64 tensor holding every problem's
    N_q x nrhs column-major block in turn (sum_q N_q * nrhs elements)."""
    lib = load()
    if not rhs.is_contiguous():
        raise ValueError("rhs must be contiguous")
    _check(lib.iaskit_solve_batched_device(_dev_ptr(rhs), nrhs))


def iaskit_solve(rhs) -> np.ndarray:
    """w = (lambda I + K~)^{-1} u for host u (N,) or (N, nrhs); returns a new array."""
    lib = load()
    u = np.asarray(rhs, dtype=np.float64)
    vec = u.ndim == 1
    U = np.array(u.reshape(u.shape[0], -1), dtype=np.float64, order="F", copy=True)
    _check(lib.iaskit_solve(U.ctypes.data, U.shape[1]))
    return U[:, 0] if vec else U


def iaskit_solve_device(rhs) -> None:
    """In place on a CUDA float64 tensor laid out N x nrhs column-major (i.e. the
    tensor is (nrhs, N) contiguous, or (N,) for one right-hand side)."""
    lib = load()
    if not rhs.is_contiguous():
        raise ValueError("rhs must be contiguous")
    nrhs = 1 if rhs.dim() == 1 else rhs.shape[0]
    _check(lib.iaskit_solve_device(_dev_ptr(rhs), nrhs))


def iaskit_apply(w) -> np.ndarray:
    """u = (lambda I + K~) w by the FP64 hierarchical MatVec (host arrays); with option
    "near_field" = 1, u = (lambda I + K~ + S) w, the kNN-separated operator."""
    lib = load()
    x = np.asarray(w, dtype=np.float64)
    vec = x.ndim == 1
    W = np.array(x.reshape(x.shape[0], -1), dtype=np.float64, order="F", copy=True)
    U = np.empty_like(W, order="F")
    _check(lib.iaskit_apply(W.ctypes.data, U.ctypes.data, W.shape[1]))
    return U[:, 0] if vec else U


def iaskit_apply_device(w, u, nrhs=None) -> None:
    """u = (lambda I + K~) w on CUDA float64 tensors laid out like iaskit_solve_device's
    right-hand sides; nrhs defaults to w.shape[0] for a 2-D tensor, else 1."""
    lib = load()
    if nrhs is None:
        nrhs = 1 if w.dim() == 1 else w.shape[0]
    _check(lib.iaskit_apply_device(_dev_ptr(w), _dev_ptr(u), nrhs))


def iaskit_predict(test_points, w) -> np.ndarray:
    """Exact kernel sums K(test, X) w of the factored problem: test (M, d) host array,
    w (N,) or (N, nrhs) in original point order; returns (M,) or (M, nrhs)."""
    T = _host_f64(test_points)
    if T.ndim != 2:
        raise ValueError("test_points must be (M, d)")
    W = np.asarray(w, dtype=np.float64)
    vec = W.ndim == 1
    W2 = np.asfortranarray(W[:, None] if vec else W)
    out = np.empty((T.shape[0], W2.shape[1]), dtype=np.float64, order="F")
    _check(load().iaskit_predict(T.ctypes.data, T.shape[0], W2.ctypes.data, W2.shape[1], out.ctypes.data))
    return out[:, 0] if vec else out


def iaskit_predict_device(test_points, w, scores, nrhs=None) -> None:
    """iaskit_predict on CUDA float64 tensors: test (M, d) row-major, w laid out like
    iaskit_solve_device's right-hand sides ((nrhs, N) or (N,)), scores (nrhs, M) or (M,)."""
    if nrhs is None:
        nrhs = 1 if w.dim() == 1 else w.shape[0]
    _check(load().iaskit_predict_device(_dev_ptr(test_points), test_points.shape[0], _dev_ptr(w), nrhs,
                                        _dev_ptr(scores)))


GEMM_SHAPES = {"64x64": 0, "256x16": 1, "128x32": 3, "512x8": 4}


def iaskit_gemm_tile(fp64: bool, n_bucket: int, m_bucket: int, shape) -> None:
    """Install (or with shape None clear) the CUDA-core tile shape of one bucket of the
    grouped-GEMM tile table."""
    code = -1 if shape is None else GEMM_SHAPES[shape] if isinstance(shape, str) else int(shape)
    _check(load().iaskit_gemm_tile(int(bool(fp64)), n_bucket, m_bucket, code))


def iaskit_tune_gemm(fp64: bool, M: int, N: int, K: int, count: int, shape, reps: int = 5) -> float:
    """Milliseconds of one grouped CUDA-core GEMM launch of `count` M x N x K problems."""
    ms = ctypes.c_double()
    code = GEMM_SHAPES[shape] if isinstance(shape, str) else int(shape)
    _check(load().iaskit_tune_gemm(int(bool(fp64)), M, N, K, count, code, reps, ctypes.byref(ms)))
    return ms.value


TILE_TABLE = os.path.join(_HERE, "gemm_tiles.json")


def load_tile_table(path: str = TILE_TABLE) -> int:
    """Install the committed autotuned tile table (written by the autotune module);
    returns the number of entries installed (0 without a table)."""
    if not os.path.exists(path):
        return 0
    with open(path) as f:
        table = json.load(f)
    n = 0
    for e in table["entries"]:
        iaskit_gemm_tile(e["fp64"], e["n_bucket"], e["m_bucket"], e["shape"])
        n += 1
    return n


def iaskit_set_option(key: str, value: float) -> None:
    _check(load().iaskit_set_option(key.encode(), float(value)))


def iaskit_get_option(key: str) -> float:
    v = ctypes.c_double()
    _check(load().iaskit_get_option(key.encode(), ctypes.byref(v)))
    return v.value


def iaskit_set_stream(stream) -> None:
    """Accepts a torch.cuda.Stream, an int handle, or None for the default stream."""
    handle = 0 if stream is None else getattr(stream, "cuda_stream", stream)
    _check(load().iaskit_set_stream(ctypes.c_void_p(handle)))


def iaskit_stats() -> dict:
    lib = load()
    n = lib.iaskit_stats(None, 0)
    buf = ctypes.create_string_buffer(n + 16)
    lib.iaskit_stats(buf, len(buf))
    return json.loads(buf.value.decode())


def iaskit_last_error() -> str:
    return load().iaskit_last_error().decode()


def iaskit_free() -> None:
    load().iaskit_free()


def iaskit_depth() -> int:
    return _check(load().iaskit_depth())


def iaskit_get_perm(N: int) -> np.ndarray:
    out = np.empty(N, dtype=np.int32)
    _check(load().iaskit_get_perm(out.ctypes.data))
    return out


def iaskit_get_knn(N: int, kappa: int) -> np.ndarray:
    out = np.empty((N, kappa), dtype=np.int32)
    _check(load().iaskit_get_knn(out.ctypes.data, kappa))
    return out


def iaskit_get_ranks() -> np.ndarray:
    L = iaskit_depth()
    out = np.empty(2 << L, dtype=np.int32)
    _check(load().iaskit_get_ranks(out.ctypes.data, out.size))
    return out


def iaskit_get_skeleton(level: int, index: int, cap: int = 4096) -> np.ndarray:
    out = np.empty(cap, dtype=np.int32)
    s = _check(load().iaskit_get_skeleton(level, index, out.ctypes.data, cap))
    return out[:s].copy()


def iaskit_get_samples(level: int, index: int, cap: int = 1 << 16) -> np.ndarray:
    out = np.empty(cap, dtype=np.int32)
    n = _check(load().iaskit_get_samples(level, index, out.ctypes.data, cap))
    return out[:n].copy()


def iaskit_get_P(level: int, index: int, s: int, cap: int = 1 << 22) -> np.ndarray:
    out = np.empty(cap, dtype=np.float64)
    nc = _check(load().iaskit_get_P(level, index, out.ctypes.data, cap))
    return out[: s * nc].reshape(nc, s).T.copy()


KERNEL_FORMS = {"fp64": 0, "pair": 1, "fp32": 2, "sliced": 3}


def iaskit_kernel_block(points, h: float, rows, cols, diag: float = 0.0, form: str = "fp64") -> np.ndarray:
    """K(x_rows, x_cols) (+ diag where row point == column point) from the library's
    kernel-block kernels: form "fp64", "pair" (FP32 pairs), "fp32" or "sliced" (FP64 with
    the dot products on the tensor cores)."""
    X = np.ascontiguousarray(points, dtype=np.float64)
    r = np.ascontiguousarray(rows, dtype=np.int32)
    c = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.empty((len(c), len(r)), dtype=np.float64)   # column-major nr x nc
    _check(load().iaskit_kernel_block(X.ctypes.data, X.shape[0], X.shape[1], h, r.ctypes.data, len(r),
                                      c.ctypes.data, len(c), diag, KERNEL_FORMS[form], out.ctypes.data))
    return out.T.copy()


def iaskit_knn_noalloc(points, kappa: int, out, stream=None) -> None:
    """kNN lists into a caller-provided device buffer, with no device allocation.

    points: CUDA float64 tensor (N, d), contiguous; out: CUDA int32 tensor (N, kappa),
    contiguous.  For callers that cannot allocate device memory (see iaskit.h).
    """
    import torch
    lib = load()
    if not points.is_contiguous() or not out.is_contiguous():
        raise ValueError("points and out must be contiguous")
    if out.dtype != torch.int32 or not out.is_cuda:
        raise TypeError("out must be a CUDA int32 tensor")
    N, d = points.shape
    handle = 0 if stream is None else getattr(stream, "cuda_stream", stream)
    _check(lib.iaskit_knn_noalloc(_dev_ptr(points), N, d, kappa, out.data_ptr(),
                                  ctypes.c_void_p(handle)))


# ------------------------------------------------------------- learned sampling
def iaskit_sampler_train(points, h: float, leaf_m: int, s_max: int, tol: float, epochs: int,
                         lr: float) -> None:
    """Label the candidates of every node of this host problem and train the MLP."""
    X = _host_f64(points)
    _check(load().iaskit_sampler_train(X.ctypes.data, X.shape[0], X.shape[1], float(h), leaf_m,
                                       s_max, float(tol), epochs, float(lr)))


def iaskit_sampler_set_weights(w) -> None:
    a = np.ascontiguousarray(np.asarray(w, dtype=np.float32).reshape(-1))
    _check(load().iaskit_sampler_set_weights(a.ctypes.data, a.size))


def iaskit_sampler_get_weights() -> np.ndarray:
    out = np.empty(MLP_NPARAM, dtype=np.float32)
    _check(load().iaskit_sampler_get_weights(out.ctypes.data, out.size))
    return out


def iaskit_mlp_forward(feats) -> np.ndarray:
    F = np.ascontiguousarray(np.asarray(feats, dtype=np.float32).reshape(-1, 8))
    out = np.empty(F.shape[0], dtype=np.float32)
    _check(load().iaskit_mlp_forward(F.ctypes.data, F.shape[0], out.ctypes.data))
    return out


def iaskit_mlp_train_step(feats, targets, lr: float):
    """One Adam step; returns (gradient before the step, loss)."""
    F = np.ascontiguousarray(np.asarray(feats, dtype=np.float32).reshape(-1, 8))
    t = np.ascontiguousarray(np.asarray(targets, dtype=np.float32).reshape(-1))
    g = np.empty(MLP_NPARAM, dtype=np.float32)
    loss = np.zeros(1, dtype=np.float32)
    _check(load().iaskit_mlp_train_step(F.ctypes.data, t.ctypes.data, F.shape[0], float(lr),
                                        g.ctypes.data, loss.ctypes.data))
    return g, float(loss[0])


def iaskit_get_learned(level: int, index: int, cap: int = 1 << 16):
    """(candidates, features (n, 8), scores or targets, info[4]) of a kept node."""
    cand = np.empty(cap, dtype=np.int32)
    feat = np.empty((cap, 8), dtype=np.float32)
    val = np.empty(cap, dtype=np.float32)
    info = np.zeros(4, dtype=np.float64)
    n = _check(load().iaskit_get_learned(level, index, cand.ctypes.data, feat.ctypes.data,
                                         val.ctypes.data, cap, info.ctypes.data))
    return cand[:n].astype(np.int64), feat[:n].copy(), val[:n].copy(), info


def mlp_pack(p: dict) -> np.ndarray:
    """Oracle-style parameter dict -> the library's flat FP32 layout."""
    return np.concatenate([np.asarray(p[k], dtype=np.float64).reshape(-1)
                           for k in ("W1", "b1", "W2", "b2", "w3", "b3")]).astype(np.float32)


def mlp_unpack(w) -> dict:
    """The library's flat layout -> a dict of float64 arrays (W1, b1, W2, b2, w3, b3)."""
    w = np.asarray(w, dtype=np.float64)
    return {"W1": w[0:1024].reshape(128, 8), "b1": w[1024:1152], "W2": w[1152:17536].reshape(128, 128),
            "b2": w[17536:17664], "w3": w[17664:17792], "b3": w[17792:17793]}
