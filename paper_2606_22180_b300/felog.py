"""Python binding of ``libfelog.so`` (the C ABI declared in ``include/felog.h``).

Argument marshalling only: every step runs in the library's CUDA kernels.
PyTorch supplies device memory and the current CUDA stream.  There is no CPU
fallback; if the library or a CUDA device is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libfelog.so")

FELOG_OK = 0
FELOG_ERR_TIMEOUT = 6
FELOG_SGNS_HOGWILD, FELOG_SGNS_MINIBATCH, FELOG_SGNS_TILE = 0, 1, 2
FELOG_FP32, FELOG_BF16_SR = 0, 1

# exported symbols (the boundary); tests check each one is present
SYMBOLS = [
    "felog_status_string", "felog_last_cuda_error",
    "felog_validate_csr",
    "felog_compact_workspace_bytes", "felog_compact_active",
    "felog_compact_active_noalloc_max_n", "felog_compact_active_noalloc",
    "felog_walk", "felog_count",
    "felog_noise_workspace_bytes", "felog_noise_table",
    "felog_init_tables",
    "felog_sr_bf16", "felog_train_workspace_bytes", "felog_train",
    "felog_feedback",
    "felog_embed_workspace_bytes", "felog_embed",
    "felog_walk_node2vec",
    "felog_pipeline_workspace_bytes", "felog_embed_pipelined",
    "felog_fabc_max_k", "felog_fabc_workspace_bytes", "felog_fabc_max_bytes", "felog_fabc_select",
    "felog_fabc_encode", "felog_fabc_decode",
    "felog_batch_create", "felog_batch_destroy", "felog_batch_device_bytes", "felog_batch_reset",
    "felog_batch_step", "felog_batch_run", "felog_batch_read", "felog_batch_job_buffers",
    "felog_batch_autotune", "felog_batch_set_tuning", "felog_batch_set_wait_limit", "felog_grid_barrier_check",
    "felog_server_create", "felog_server_destroy", "felog_server_now", "felog_server_job_bytes",
    "felog_server_submit", "felog_server_poll", "felog_server_wait", "felog_server_fetch",
    "felog_server_drain", "felog_server_get_stats",
]


class FelogError(RuntimeError):
    pass


class _Csr(ctypes.Structure):
    _fields_ = [("offsets", ctypes.c_void_p), ("cols", ctypes.c_void_p), ("n", ctypes.c_int32),
                ("nnz", ctypes.c_int64)]


class _WalkParams(ctypes.Structure):
    _fields_ = [("length", ctypes.c_int32), ("walks_per_round", ctypes.c_int32)]


class _TrainParams(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("window", ctypes.c_int32), ("negatives", ctypes.c_int32),
                ("lr0", ctypes.c_float), ("lr_total_tokens", ctypes.c_int64),
                ("mode", ctypes.c_int32), ("minibatch", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("hogwild_rows_per_warp", ctypes.c_int32),
                ("hogwild_form", ctypes.c_int32), ("tile_negatives", ctypes.c_int32),
                ("tile_ctas", ctypes.c_int32), ("stage_flush", ctypes.c_int32)]


class _FeedbackParams(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int32), ("mu", ctypes.c_double), ("ks", ctypes.c_int32),
                ("max_rounds", ctypes.c_int32), ("reactivate", ctypes.c_int32)]


class RoundStats(ctypes.Structure):
    _fields_ = [("round", ctypes.c_int32), ("n_active", ctypes.c_int32), ("n_next", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("tokens", ctypes.c_int64),
                ("walk_steps", ctypes.c_int64), ("loss", ctypes.c_double),
                ("ms_walk", ctypes.c_float), ("ms_noise", ctypes.c_float),
                ("ms_train", ctypes.c_float), ("ms_feedback", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


_lib = None


def load() -> ctypes.CDLL:
    """Load the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise FelogError(f"{LIB_PATH} is missing: build it with python -m paper_2606_22180_b300.build")
    lib = ctypes.CDLL(LIB_PATH)
    P, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
    sz = ctypes.c_size_t
    st = ctypes.c_int
    sig = {
        "felog_status_string": (ctypes.c_char_p, [st]),
        "felog_last_cuda_error": (ctypes.c_char_p, []),
        "felog_validate_csr": (st, [P, P, i32, P, P]),
        "felog_compact_workspace_bytes": (sz, [i32]),
        "felog_compact_active": (st, [P, i32, P, P, P, sz, P]),
        "felog_compact_active_noalloc_max_n": (i32, []),
        "felog_compact_active_noalloc": (st, [P, i32, P, P, P]),
        "felog_walk": (st, [P, P, i32, P, u64, i32, P, P, P]),
        "felog_count": (st, [P, i64, i32, P, P]),
        "felog_walk_node2vec": (st, [P, P, i32, P, f64, f64, u64, i32, P, P, P]),
        "felog_noise_workspace_bytes": (sz, [i32]),
        "felog_noise_table": (st, [P, i32, P, P, P, P, sz, P]),
        "felog_init_tables": (st, [i32, i32, i32, u64, P, P, P]),
        "felog_train_workspace_bytes": (sz, [i64, i32, i32, P]),
        "felog_sr_bf16": (st, [P, P, i64, P, P]),
        "felog_train": (st, [P, i64, i32, i32, P, P, P, P, u64, i32, i64, P, P, P, P, sz, P]),
        "felog_feedback": (st, [P, P, i32, i32, P, u64, i32, P, P, P, P, P]),
        "felog_embed_workspace_bytes": (sz, [i32, P, P]),
        "felog_embed": (st, [P, P, P, P, u64, P, P, P, P, P, sz, P]),
        "felog_pipeline_workspace_bytes": (sz, [i32, P, P, i32, i32]),
        "felog_embed_pipelined": (st, [P, P, P, P, i32, u64, P, P, P, P, P, P, sz, P]),
        "felog_fabc_max_k": (i32, []),
        "felog_fabc_workspace_bytes": (sz, [i64]),
        "felog_fabc_max_bytes": (sz, [i64, i32, i32]),
        "felog_fabc_select": (st, [P, i32, i32, i32, P, P, P, P, sz, P]),
        "felog_fabc_encode": (st, [P, i64, i32, P, i32, P, sz, P, P, sz, P]),
        "felog_fabc_decode": (st, [P, sz, i64, i32, i32, P, P, sz, P]),
        "felog_batch_create": (st, [P, i32, P, P, P, P]),
        "felog_batch_destroy": (st, [P]),
        "felog_batch_device_bytes": (sz, [P]),
        "felog_batch_reset": (st, [P, P]),
        "felog_batch_step": (st, [P, P]),
        "felog_batch_run": (st, [P, i32, P]),
        "felog_batch_read": (st, [P, P, P, P, P]),
        "felog_batch_job_buffers": (st, [P, i32, P]),
        "felog_batch_autotune": (st, [P, ctypes.c_char_p, P, P]),
        "felog_batch_set_tuning": (st, [P, P]),
        "felog_batch_set_wait_limit": (st, [P, f64]),
        "felog_grid_barrier_check": (st, [i32, i32, f64, P, P]),
        "felog_server_create": (st, [P, P]),
        "felog_server_destroy": (st, [P]),
        "felog_server_now": (f64, [P]),
        "felog_server_job_bytes": (sz, [P, i32, i64, i32]),
        "felog_server_submit": (st, [P, P, P, i32, i64, i32, u64, P]),
        "felog_server_poll": (st, [P, u64, P]),
        "felog_server_wait": (st, [P, u64, f64, P]),
        "felog_server_fetch": (st, [P, u64, P]),
        "felog_server_drain": (st, [P, f64]),
        "felog_server_get_stats": (st, [P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, what: str) -> None:
    if status != FELOG_OK:
        lib = load()
        msg = lib.felog_status_string(status).decode()
        cuda = lib.felog_last_cuda_error().decode()
        raise FelogError(f"{what}: {msg}" + (f" ({cuda})" if cuda else ""))


def _require_cuda(*tensors) -> None:
    if not torch.cuda.is_available():
        raise FelogError("no CUDA device: the FeLoG path has no CPU fallback")
    for t in tensors:
        if t is not None and not t.is_cuda:
            raise FelogError("tensors passed to the FeLoG library must live on the GPU")
        if t is not None and not t.is_contiguous():
            raise FelogError("tensors passed to the FeLoG library must be contiguous")


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _workspace(nbytes: int, device) -> torch.Tensor:
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


@dataclasses.dataclass
class DeviceGraph:
    """An undirected CSR resident on the GPU (int32 offsets and cols)."""

    offsets: torch.Tensor
    cols: torch.Tensor

    @property
    def n(self) -> int:
        return int(self.offsets.numel() - 1)

    @property
    def nnz(self) -> int:
        return int(self.cols.numel())

    @classmethod
    def from_host(cls, csr, device="cuda") -> "DeviceGraph":
        off = torch.as_tensor(csr.offsets, dtype=torch.int32).to(device)
        cols = torch.as_tensor(csr.cols, dtype=torch.int32).to(device)
        return cls(off, cols)

    def _c(self) -> _Csr:
        _require_cuda(self.offsets, self.cols)
        return _Csr(self.offsets.data_ptr(), self.cols.data_ptr() if self.nnz else 0, self.n, self.nnz)


def table_dtype(precision: int) -> torch.dtype:
    return torch.float32 if precision == FELOG_FP32 else torch.bfloat16


# ---------------------------------------------------------------------------
# One wrapper per C entry point, with the same name.
# ---------------------------------------------------------------------------

CSR_ENDS, CSR_DECREASING, CSR_COL_RANGE, CSR_ORDER, CSR_SELF_LOOP, CSR_START_RANGE = 1, 2, 4, 8, 16, 32


def felog_validate_csr(g: DeviceGraph, starts: torch.Tensor | None = None,
                       status: torch.Tensor | None = None) -> torch.Tensor:
    """Device-side check of the graph (and of a start list); returns the
    device int32 status word (0: valid, else an OR of the CSR_* bits)."""
    _require_cuda(starts, status)
    lib = load()
    if status is None:
        status = torch.empty(1, dtype=torch.int32, device=g.offsets.device)
    csr = g._c()
    n_starts = 0 if starts is None else starts.numel()
    _check(lib.felog_validate_csr(ctypes.byref(csr), _ptr(starts), n_starts, _ptr(status), _stream()),
           "felog_validate_csr")
    return status


def felog_grid_barrier_check(phantom: int = 0, passes: int = 1, seconds: float = 1.0) -> tuple[int, int]:
    """The persistent batched kernel's grid barrier on its own (see felog.h):
    returns (status, where); status is FELOG_OK or FELOG_ERR_TIMEOUT, and
    where the index of the barrier whose wait ran out (-1 if none).  Other
    statuses raise."""
    if not torch.cuda.is_available():
        raise FelogError("no CUDA device: the FeLoG path has no CPU fallback")
    lib = load()
    where = ctypes.c_int32(-2)
    st = lib.felog_grid_barrier_check(int(phantom), int(passes), float(seconds), ctypes.byref(where), _stream())
    if st not in (FELOG_OK, FELOG_ERR_TIMEOUT):
        _check(st, "felog_grid_barrier_check")
    return int(st), int(where.value)


def felog_compact_active(active: torch.Tensor):
    """Ascending indices of the nonzero flags; returns (starts[n], n_active device int32[1])."""
    _require_cuda(active)
    lib = load()
    n = active.numel()
    starts = torch.empty(max(n, 1), dtype=torch.int32, device=active.device)
    n_active = torch.empty(1, dtype=torch.int32, device=active.device)
    ws = _workspace(lib.felog_compact_workspace_bytes(n), active.device)
    _check(lib.felog_compact_active(_ptr(active), n, _ptr(starts), _ptr(n_active), _ptr(ws),
                                    ws.numel(), _stream()), "felog_compact_active")
    return starts, n_active


def felog_compact_active_noalloc(active: torch.Tensor, starts: torch.Tensor, n_active: torch.Tensor):
    """Compaction without any device allocation by the library (scratch is a
    static device array); the caller supplies starts[n] and n_active[1]."""
    _require_cuda(active, starts, n_active)
    lib = load()
    _check(lib.felog_compact_active_noalloc(_ptr(active), active.numel(), _ptr(starts), _ptr(n_active),
                                            _stream()), "felog_compact_active_noalloc")
    return starts, n_active


def felog_walk(g: DeviceGraph, starts: torch.Tensor, n_starts: int, length: int,
               walks_per_round: int, seed: int, round_: int, counts: torch.Tensor | None = None,
               out: torch.Tensor | None = None) -> torch.Tensor:
    """Uniform truncated walks; returns int32 [n_starts * walks_per_round, length]."""
    _require_cuda(starts, counts, out)
    lib = load()
    if out is None:
        out = torch.empty((n_starts * walks_per_round, length), dtype=torch.int32, device=starts.device)
    wp = _WalkParams(length, walks_per_round)
    csr = g._c()
    _check(lib.felog_walk(ctypes.byref(csr), _ptr(starts), n_starts, ctypes.byref(wp), seed, round_,
                          _ptr(out), _ptr(counts), _stream()), "felog_walk")
    return out


def felog_walk_node2vec(g: DeviceGraph, starts: torch.Tensor, n_starts: int, length: int,
                        walks_per_round: int, p: float, q: float, seed: int, round_: int,
                        counts: torch.Tensor | None = None, out: torch.Tensor | None = None) -> torch.Tensor:
    """node2vec walks (return parameter p, in-out parameter q); int32 [n_starts * wpr, length]."""
    _require_cuda(starts, counts, out)
    lib = load()
    if out is None:
        out = torch.empty((n_starts * walks_per_round, length), dtype=torch.int32, device=starts.device)
    wp = _WalkParams(length, walks_per_round)
    csr = g._c()
    _check(lib.felog_walk_node2vec(ctypes.byref(csr), _ptr(starts), n_starts, ctypes.byref(wp), p, q, seed,
                                   round_, _ptr(out), _ptr(counts), _stream()), "felog_walk_node2vec")
    return out


def felog_count(tokens: torch.Tensor, n: int, counts: torch.Tensor | None = None) -> torch.Tensor:
    _require_cuda(tokens, counts)
    lib = load()
    if counts is None:
        counts = torch.zeros(n, dtype=torch.int32, device=tokens.device)
    _check(lib.felog_count(_ptr(tokens), tokens.numel(), n, _ptr(counts), _stream()), "felog_count")
    return counts


def felog_noise_table(counts: torch.Tensor):
    """Alias table of the unigram^0.75 distribution: (thr uint64 as int64, alias int32, S [1])."""
    _require_cuda(counts)
    lib = load()
    n = counts.numel()
    dev = counts.device
    thr = torch.empty(n, dtype=torch.int64, device=dev)
    alias = torch.empty(n, dtype=torch.int32, device=dev)
    S = torch.empty(1, dtype=torch.int64, device=dev)
    ws = _workspace(lib.felog_noise_workspace_bytes(n), dev)
    _check(lib.felog_noise_table(_ptr(counts), n, _ptr(thr), _ptr(alias), _ptr(S), _ptr(ws),
                                 ws.numel(), _stream()), "felog_noise_table")
    return thr, alias, S


def felog_init_tables(n: int, dim: int, precision: int, seed: int, device="cuda"):
    _require_cuda()
    lib = load()
    dt = table_dtype(precision)
    phi_in = torch.empty((n, dim), dtype=dt, device=device)
    phi_out = torch.empty((n, dim), dtype=dt, device=device)
    _check(lib.felog_init_tables(n, dim, precision, seed, _ptr(phi_in), _ptr(phi_out), _stream()),
           "felog_init_tables")
    return phi_in, phi_out


def train_params(dim=128, window=10, negatives=5, lr0=0.025, lr_total_tokens=1, mode=FELOG_SGNS_HOGWILD,
                 minibatch=4096, precision=FELOG_FP32, hogwild_rows_per_warp=0,
                 hogwild_form=0, tile_negatives=0, tile_ctas=0, stage_flush=0) -> _TrainParams:
    return _TrainParams(dim, window, negatives, lr0, lr_total_tokens, mode, minibatch, precision,
                        hogwild_rows_per_warp, hogwild_form, tile_negatives, tile_ctas, stage_flush)


def feedback_params(enabled=True, mu=0.65, ks=8, max_rounds=10, reactivate=False) -> _FeedbackParams:
    return _FeedbackParams(int(enabled), mu, ks, max_rounds, int(reactivate))


def felog_sr_bf16(x: torch.Tensor, r16: torch.Tensor) -> torch.Tensor:
    """Stochastic rounding of float32 x to bf16 patterns with the 16-bit random
    values r16 (int16 tensor holding uint16 bits, same length); returns the
    patterns as an int16 tensor."""
    _require_cuda(x, r16)
    if x.dtype != torch.float32 or r16.dtype != torch.int16 or x.numel() != r16.numel():
        raise FelogError("felog_sr_bf16: float32 x and int16 r16 of the same length")
    out = torch.empty(x.numel(), dtype=torch.int16, device=x.device)
    _check(load().felog_sr_bf16(_ptr(x), _ptr(r16), x.numel(), _ptr(out), _stream()), "felog_sr_bf16")
    return out


def felog_train(walks: torch.Tensor, n: int, tp: _TrainParams, thr: torch.Tensor, alias: torch.Tensor,
                S: torch.Tensor, seed: int, round_: int, clock_base: int, phi_in: torch.Tensor,
                phi_out: torch.Tensor, loss: torch.Tensor | None = None,
                workspace: torch.Tensor | None = None) -> torch.Tensor:
    """SGNS over walks [n_walks, L]; updates the tables in place; returns loss (device f64 [1])."""
    _require_cuda(walks, thr, alias, S, phi_in, phi_out, loss, workspace)
    lib = load()
    n_walks, L = walks.shape
    if loss is None:
        loss = torch.empty(1, dtype=torch.float64, device=walks.device)
    need = lib.felog_train_workspace_bytes(n_walks, L, n, ctypes.byref(tp))
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, walks.device)
    _check(lib.felog_train(_ptr(walks), n_walks, L, n, ctypes.byref(tp), _ptr(thr), _ptr(alias),
                           _ptr(S), seed, round_, clock_base, _ptr(phi_in), _ptr(phi_out), _ptr(loss),
                           _ptr(workspace), workspace.numel(), _stream()), "felog_train")
    return loss


def felog_fabc_select(counts: torch.Tensor, L: int, k_max: int = 32):
    """FaBC top-k (Eq. 8) from device corpus counts; returns (ids list, F_k)."""
    _require_cuda(counts)
    lib = load()
    ws = _workspace(lib.felog_fabc_workspace_bytes(0), counts.device)
    ids = (ctypes.c_int32 * max(k_max, 1))()
    k = ctypes.c_int32(0)
    F = ctypes.c_double(0.0)
    _check(lib.felog_fabc_select(_ptr(counts), counts.numel(), L, k_max, ids, ctypes.byref(k), ctypes.byref(F),
                                 _ptr(ws), ws.numel(), _stream()), "felog_fabc_select")
    return [ids[i] for i in range(k.value)], F.value


def felog_fabc_encode(walks: torch.Tensor, ids: torch.Tensor, workspace: torch.Tensor | None = None,
                      out: torch.Tensor | None = None, tail: torch.Tensor | None = None):
    """FaBC encoding of walks [n_seq, L] (device int32) with device ids [k];
    returns (device uint8 buffer of capacity max_bytes, device int64 tail count).
    `out` and `tail` may be passed in to be reused."""
    _require_cuda(walks, ids, workspace, out, tail)
    lib = load()
    n_seq, L = walks.shape
    k = ids.numel()
    cap = lib.felog_fabc_max_bytes(n_seq, L, k)
    if out is None:
        out = torch.empty(cap, dtype=torch.uint8, device=walks.device)
    if tail is None:
        tail = torch.empty(1, dtype=torch.int64, device=walks.device)
    need = lib.felog_fabc_workspace_bytes(n_seq)
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, walks.device)
    _check(lib.felog_fabc_encode(_ptr(walks), n_seq, L, _ptr(ids) if k else None, k, _ptr(out), out.numel(),
                                 _ptr(tail), _ptr(workspace), workspace.numel(), _stream()), "felog_fabc_encode")
    return out, tail


def fabc_encoded_bytes(n_seq: int, L: int, k: int, tail: int) -> int:
    return 4 * n_seq * k + n_seq * k * ((L + 7) // 8) + 4 * tail


def fabc_workspace(n_seq: int, device="cuda") -> torch.Tensor:
    """A device workspace for encoding or decoding n_seq sequences, to reuse across calls."""
    return _workspace(load().felog_fabc_workspace_bytes(n_seq), device)


def felog_fabc_decode(buf: torch.Tensor, n_seq: int, L: int, k: int, walks: torch.Tensor | None = None,
                      workspace: torch.Tensor | None = None) -> torch.Tensor:
    """Inverse of felog_fabc_encode; returns device int32 walks [n_seq, L]."""
    _require_cuda(buf, walks, workspace)
    lib = load()
    if walks is None:
        walks = torch.empty((n_seq, L), dtype=torch.int32, device=buf.device)
    need = lib.felog_fabc_workspace_bytes(n_seq)
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, buf.device)
    _check(lib.felog_fabc_decode(_ptr(buf), buf.numel(), n_seq, L, k, _ptr(walks), _ptr(workspace),
                                 workspace.numel(), _stream()), "felog_fabc_decode")
    return walks


def felog_feedback(g: DeviceGraph, phi_in: torch.Tensor, precision: int, fp: _FeedbackParams,
                   seed: int, round_: int, active_in: torch.Tensor, want_psi: bool = True):
    """Psi and the next active set; returns (psi f64 [n] or None, active_out u8 [n], n_next [1])."""
    _require_cuda(phi_in, active_in)
    lib = load()
    n = g.n
    dev = phi_in.device
    active_out = torch.empty(n, dtype=torch.uint8, device=dev)
    psi = torch.empty(n, dtype=torch.float64, device=dev) if want_psi else None
    n_next = torch.empty(1, dtype=torch.int32, device=dev)
    csr = g._c()
    _check(lib.felog_feedback(ctypes.byref(csr), _ptr(phi_in), phi_in.shape[1], precision,
                              ctypes.byref(fp), seed, round_, _ptr(active_in), _ptr(active_out),
                              _ptr(psi), _ptr(n_next), _stream()), "felog_feedback")
    return psi, active_out, n_next


def embed_workspace_bytes(n: int, length: int, walks_per_round: int, tp: _TrainParams) -> int:
    lib = load()
    wp = _WalkParams(length, walks_per_round)
    return int(lib.felog_embed_workspace_bytes(n, ctypes.byref(wp), ctypes.byref(tp)))


def felog_embed(g: DeviceGraph, length: int, walks_per_round: int, tp: _TrainParams,
                fp: _FeedbackParams, seed: int, phi_in: torch.Tensor | None = None,
                phi_out: torch.Tensor | None = None, workspace: torch.Tensor | None = None):
    """Algorithm 1 end to end; returns (phi_in, phi_out, [RoundStats dicts])."""
    _require_cuda(phi_in, phi_out, workspace)
    lib = load()
    dev = g.offsets.device
    dt = table_dtype(tp.precision)
    if phi_in is None:
        phi_in = torch.empty((g.n, tp.dim), dtype=dt, device=dev)
    if phi_out is None:
        phi_out = torch.empty((g.n, tp.dim), dtype=dt, device=dev)
    wp = _WalkParams(length, walks_per_round)
    need = lib.felog_embed_workspace_bytes(g.n, ctypes.byref(wp), ctypes.byref(tp))
    if need == 0:
        raise FelogError("felog_embed: invalid parameters")
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    stats = (RoundStats * max(fp.max_rounds, 1))()
    rounds = ctypes.c_int32(0)
    csr = g._c()
    _check(lib.felog_embed(ctypes.byref(csr), ctypes.byref(wp), ctypes.byref(tp), ctypes.byref(fp),
                           seed, _ptr(phi_in), _ptr(phi_out), stats, ctypes.byref(rounds),
                           _ptr(workspace), workspace.numel(), _stream()), "felog_embed")
    return phi_in, phi_out, [stats[i].as_dict() for i in range(rounds.value)]


class PipelineStats(ctypes.Structure):
    _fields_ = [("wall_ms", ctypes.c_double), ("train_busy_ms", ctypes.c_double),
                ("sample_busy_ms", ctypes.c_double), ("overlap_ms", ctypes.c_double),
                ("rounds", ctypes.c_int32), ("feedback_lag", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


def felog_embed_pipelined(g: DeviceGraph, length: int, walks_per_round: int, tp: _TrainParams,
                          fp: _FeedbackParams, seed: int, feedback_lag: int = 1,
                          phi_in: torch.Tensor | None = None, phi_out: torch.Tensor | None = None,
                          workspace: torch.Tensor | None = None):
    """Algorithm 1 as the round-interleaved pipeline (Section 5.3); returns
    (phi_in, phi_out, [RoundStats dicts], pipeline stats dict)."""
    _require_cuda(phi_in, phi_out, workspace)
    lib = load()
    dev = g.offsets.device
    dt = table_dtype(tp.precision)
    if phi_in is None:
        phi_in = torch.empty((g.n, tp.dim), dtype=dt, device=dev)
    if phi_out is None:
        phi_out = torch.empty((g.n, tp.dim), dtype=dt, device=dev)
    wp = _WalkParams(length, walks_per_round)
    need = lib.felog_pipeline_workspace_bytes(g.n, ctypes.byref(wp), ctypes.byref(tp), fp.max_rounds, feedback_lag)
    if need == 0:
        raise FelogError("felog_embed_pipelined: invalid parameters")
    if workspace is None or workspace.numel() < need:
        workspace = _workspace(need, dev)
    stats = (RoundStats * max(fp.max_rounds, 1))()
    ps = PipelineStats()
    rounds = ctypes.c_int32(0)
    csr = g._c()
    _check(lib.felog_embed_pipelined(ctypes.byref(csr), ctypes.byref(wp), ctypes.byref(tp), ctypes.byref(fp),
                                     feedback_lag, seed, _ptr(phi_in), _ptr(phi_out), stats, ctypes.byref(ps),
                                     ctypes.byref(rounds), _ptr(workspace), workspace.numel(), _stream()),
           "felog_embed_pipelined")
    return phi_in, phi_out, [stats[i].as_dict() for i in range(rounds.value)], ps.as_dict()


# ---------------------------------------------------------------------------
# Batching form
# ---------------------------------------------------------------------------
class _Job(ctypes.Structure):
    _fields_ = [("graph", _Csr), ("seed", ctypes.c_uint64), ("dim", ctypes.c_int32),
                ("phi_in", ctypes.c_void_p), ("phi_out", ctypes.c_void_p)]


class JobStats(ctypes.Structure):
    _fields_ = [("rounds", ctypes.c_int32), ("done", ctypes.c_int32), ("tokens", ctypes.c_int64),
                ("n_live", ctypes.c_int64), ("loss_last", ctypes.c_double)]


class _JobBuffers(ctypes.Structure):
    _fields_ = [("active0", ctypes.c_void_p), ("active1", ctypes.c_void_p), ("starts", ctypes.c_void_p),
                ("walks", ctypes.c_void_p), ("counts", ctypes.c_void_p), ("thr", ctypes.c_void_p),
                ("alias", ctypes.c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("walk_block", ctypes.c_int32), ("sgns_blocks_per_sm", ctypes.c_int32),
                ("feedback_blocks_per_sm", ctypes.c_int32), ("from_cache", ctypes.c_int32),
                ("sgns_form", ctypes.c_int32)]


class Batch:
    """Many embedding jobs trained together (felog_batch_* calls).

    graphs: list of DeviceGraph; dims and seeds per job.  The batch owns its
    per-job work buffers; the tables it trains are allocated here and exposed
    as ``phi_in[j]`` / ``phi_out[j]``.
    """

    def __init__(self, graphs, dims, seeds, length, walks_per_round, tp: _TrainParams,
                 fp: _FeedbackParams):
        _require_cuda(*[g.offsets for g in graphs])
        lib = load()
        self.lib, self.graphs, self.tp, self.fp = lib, list(graphs), tp, fp
        dt = table_dtype(tp.precision)
        dev = graphs[0].offsets.device
        self.phi_in = [torch.empty((g.n, d), dtype=dt, device=dev) for g, d in zip(graphs, dims)]
        self.phi_out = [torch.empty((g.n, d), dtype=dt, device=dev) for g, d in zip(graphs, dims)]
        jobs = (_Job * len(graphs))()
        for j, (g, d, sd) in enumerate(zip(graphs, dims, seeds)):
            jobs[j] = _Job(g._c(), sd, d, self.phi_in[j].data_ptr(), self.phi_out[j].data_ptr())
        self.wp = _WalkParams(length, walks_per_round)
        handle = ctypes.c_void_p(0)
        _check(lib.felog_batch_create(jobs, len(graphs), ctypes.byref(self.wp), ctypes.byref(tp),
                                      ctypes.byref(fp), ctypes.byref(handle)), "felog_batch_create")
        self.handle = handle
        self.n_jobs = len(graphs)

    def close(self):
        if self.handle:
            self.lib.felog_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_bytes(self) -> int:
        return int(self.lib.felog_batch_device_bytes(self.handle))

    def reset(self):
        _check(self.lib.felog_batch_reset(self.handle, _stream()), "felog_batch_reset")

    def step(self):
        _check(self.lib.felog_batch_step(self.handle, _stream()), "felog_batch_step")

    def run(self, use_graph: bool | int = True, persistent: bool = False):
        """All rounds: ordinary launches (use_graph False), one CUDA graph (True),
        or one persistent kernel (persistent=True)."""
        mode = 2 if persistent else int(bool(use_graph))
        _check(self.lib.felog_batch_run(self.handle, mode, _stream()), "felog_batch_run")

    def set_tuning(self, walk_block: int = 256, sgns_blocks_per_sm: int = 2, feedback_blocks_per_sm: int = 16,
                   sgns_form: int = 2):
        """Launch shapes of the batched kernels (see felog_tuning)."""
        t = Tuning(walk_block, sgns_blocks_per_sm, feedback_blocks_per_sm, 0, sgns_form)
        _check(self.lib.felog_batch_set_tuning(self.handle, ctypes.byref(t)), "felog_batch_set_tuning")

    def set_wait_limit(self, seconds: float):
        """Budget of each grid-barrier wait of the persistent form."""
        _check(self.lib.felog_batch_set_wait_limit(self.handle, float(seconds)), "felog_batch_set_wait_limit")

    def autotune(self, cache_path: str | None = None) -> dict:
        t = Tuning()
        _check(self.lib.felog_batch_autotune(self.handle, cache_path.encode() if cache_path else None,
                                             ctypes.byref(t), _stream()), "felog_batch_autotune")
        return {k: getattr(t, k) for k, _ in t._fields_}

    def read(self):
        """Per-job stats (dicts) and per-round |V_a| and loss arrays [rounds, jobs]."""
        import numpy as np

        stats = (JobStats * self.n_jobs)()
        R = max(self.fp.max_rounds, 1)
        na = np.zeros((R, self.n_jobs), np.int32)
        ls = np.zeros((R, self.n_jobs), np.float64)
        _check(self.lib.felog_batch_read(self.handle, stats, na.ctypes.data_as(ctypes.c_void_p),
                                         ls.ctypes.data_as(ctypes.c_void_p), _stream()), "felog_batch_read")
        return [{k: getattr(stats[j], k) for k, _ in JobStats._fields_} for j in range(self.n_jobs)], na, ls

    def job_walks(self, j: int, rows: int) -> torch.Tensor:
        """A copy of job j's walks of the last round (rows = its |V_a| * wpr)."""
        b = _JobBuffers()
        _check(self.lib.felog_batch_job_buffers(self.handle, j, ctypes.byref(b)), "felog_batch_job_buffers")
        return _device_view(b.walks, rows * self.wp.length, torch.int32).view(rows, self.wp.length).clone()

    def job_table(self, j: int):
        """Copies of job j's alias table (thr, alias) and corpus counts of the last round."""
        b = _JobBuffers()
        _check(self.lib.felog_batch_job_buffers(self.handle, j, ctypes.byref(b)), "felog_batch_job_buffers")
        n = self.graphs[j].n
        return (_device_view(b.thr, n, torch.int64).clone(), _device_view(b.alias, n, torch.int32).clone(),
                _device_view(b.counts, n, torch.int32).clone())


class _CudaArray:
    """A library-owned device buffer exposed through __cuda_array_interface__."""

    _TYPESTR = {torch.int32: "<i4", torch.int64: "<i8", torch.uint8: "|u1"}

    def __init__(self, ptr: int, numel: int, dtype):
        self.__cuda_array_interface__ = {"data": (int(ptr), False), "shape": (int(numel),),
                                         "typestr": self._TYPESTR[dtype], "version": 2}


def _device_view(ptr: int, numel: int, dtype) -> torch.Tensor:
    """A tensor aliasing numel elements at a library-owned device address."""
    if numel == 0:
        return torch.empty(0, dtype=dtype, device="cuda")
    torch.cuda.current_stream().synchronize()
    return torch.as_tensor(_CudaArray(ptr, numel, dtype), device="cuda")


# ---------------------------------------------------------------------------
# Serving form
# ---------------------------------------------------------------------------
JOB_QUEUED, JOB_RUNNING, JOB_DONE, JOB_REJECTED, JOB_FAILED = 0, 1, 2, 3, 4


class _ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_resident", ctypes.c_int32),
                ("drain_on_destroy", ctypes.c_int32), ("walk", _WalkParams), ("train", _TrainParams),
                ("feedback", _FeedbackParams)]


class Result(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("rounds", ctypes.c_int32), ("n", ctypes.c_int32),
                ("dim", ctypes.c_int32), ("tokens", ctypes.c_int64), ("n_live", ctypes.c_int64),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("loss_last", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64), ("completed", ctypes.c_int64),
                ("rejected", ctypes.c_int64), ("steps", ctypes.c_int64), ("resident_jobs", ctypes.c_int32),
                ("peak_resident_jobs", ctypes.c_int32), ("queued", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("resident_bytes", ctypes.c_size_t), ("peak_resident_bytes", ctypes.c_size_t),
                ("busy_seconds", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class Server:
    """Continuous-batching embedding server (felog_server_* calls)."""

    def __init__(self, hbm_budget: int, length: int, walks_per_round: int, tp: _TrainParams,
                 fp: _FeedbackParams, max_resident: int = 0, drain_on_destroy: bool = False):
        _require_cuda()
        self.lib = load()
        cfg = _ServerConfig(hbm_budget, max_resident, int(drain_on_destroy),
                            _WalkParams(length, walks_per_round), tp, fp)
        h = ctypes.c_void_p(0)
        _check(self.lib.felog_server_create(ctypes.byref(cfg), ctypes.byref(h)), "felog_server_create")
        self.handle = h
        self.dims = {}

    def now(self) -> float:
        return float(self.lib.felog_server_now(self.handle))

    def job_bytes(self, n: int, nnz: int, dim: int) -> int:
        return int(self.lib.felog_server_job_bytes(self.handle, n, nnz, dim))

    def submit(self, csr, dim: int, seed: int) -> int:
        import numpy as np

        off = np.ascontiguousarray(csr.offsets, dtype=np.int32)
        cols = np.ascontiguousarray(csr.cols, dtype=np.int32)
        rid = ctypes.c_uint64(0)
        _check(self.lib.felog_server_submit(self.handle, off.ctypes.data_as(ctypes.c_void_p),
                                            cols.ctypes.data_as(ctypes.c_void_p), off.shape[0] - 1,
                                            cols.shape[0], dim, seed, ctypes.byref(rid)), "felog_server_submit")
        self.dims[rid.value] = (off.shape[0] - 1, dim)
        return rid.value

    def poll(self, rid: int) -> dict:
        r = Result()
        _check(self.lib.felog_server_poll(self.handle, rid, ctypes.byref(r)), "felog_server_poll")
        return r.as_dict()

    def wait(self, rid: int, timeout: float = 600.0) -> dict:
        r = Result()
        _check(self.lib.felog_server_wait(self.handle, rid, timeout, ctypes.byref(r)), "felog_server_wait")
        return r.as_dict()

    def fetch(self, rid: int):
        import numpy as np

        n, dim = self.dims.pop(rid)
        out = np.empty((n, dim), np.float32)
        _check(self.lib.felog_server_fetch(self.handle, rid, out.ctypes.data_as(ctypes.c_void_p)),
               "felog_server_fetch")
        return out

    def drain(self, timeout: float = 600.0):
        _check(self.lib.felog_server_drain(self.handle, timeout), "felog_server_drain")

    def stats(self) -> dict:
        s = ServerStats()
        _check(self.lib.felog_server_get_stats(self.handle, ctypes.byref(s)), "felog_server_get_stats")
        return s.as_dict()

    def close(self):
        if self.handle:
            st = self.lib.felog_server_destroy(self.handle)
            self.handle = ctypes.c_void_p(0)
            _check(st, "felog_server_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
