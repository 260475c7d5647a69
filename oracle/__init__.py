"""CPU oracle for the FeLoG walk + SGNS hot path (test infrastructure).

Only the test suite, the smoke check and the benchmark's CPU-baseline leg may
import this package.  It wraps ``felog_oracle.c`` (plain C, binary64, no FMA
contraction), which shares no code with the CUDA library.  See the C file for
the paper passage each function follows.

Pins that tie it to the paper and to mathematics rather than to itself live in
``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "felog_oracle.c")
_LIB = os.path.join(_HERE, "_felog_oracle.so")

STREAM_WALK, STREAM_PSI, STREAM_NEG, STREAM_INIT, STREAM_SR = 0, 1, 2, 3, 4


_BASE_SRC = os.path.join(_HERE, "felog_cpu_baseline.c")
_BASE_LIB = os.path.join(_HERE, "_felog_cpu_baseline.so")
_FLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def _stale(lib_path: str, srcs) -> bool:
    return not os.path.exists(lib_path) or any(os.path.getmtime(lib_path) < os.path.getmtime(s) for s in srcs)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (binary64, no contraction, no fast-math),
    and the all-cores timed baseline (the oracle's routines under OpenMP)."""
    if force or _stale(_LIB, [_SRC]):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc"] + _FLAGS + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    if force or _stale(_BASE_LIB, [_SRC, _BASE_SRC]):
        tmp = _BASE_LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc"] + _FLAGS + ["-fopenmp", "-o", tmp, _SRC, _BASE_SRC, "-lm"])
        os.replace(tmp, _BASE_LIB)
    return _LIB


class _TrainParams(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("window", ctypes.c_int32),
                ("negatives", ctypes.c_int32), ("lr0", ctypes.c_double),
                ("lr_total_tokens", ctypes.c_int64)]


class _FeedbackParams(ctypes.Structure):
    _fields_ = [("enabled", ctypes.c_int32), ("mu", ctypes.c_double), ("ks", ctypes.c_int32),
                ("max_rounds", ctypes.c_int32), ("reactivate", ctypes.c_int32)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        sig = {
            "oracle_philox": (None, [u64, P, P]),
            "oracle_walk": (ctypes.c_int, [P, P, i32, P, i32, i32, i32, u64, i32, P]),
            "oracle_counts": (None, [P, i64, i32, P]),
            "oracle_walk_node2vec": (ctypes.c_int, [P, P, i32, P, i32, i32, i32, f64, f64, u64, i32, P]),
            "oracle_noise_table": (ctypes.c_int, [P, i32, P, P, P, P]),
            "oracle_draw_negative": (i32, [P, P, i32, u64, u64, i32, i64, i32, i32, i32]),
            "oracle_init_tables": (None, [i32, i32, u64, P, P]),
            "oracle_sr_bf16": (ctypes.c_uint32, [ctypes.c_uint32, ctypes.c_uint32]),
            "oracle_sr_bf16_keyed": (ctypes.c_uint32, [ctypes.c_uint32, u64, ctypes.c_uint32,
                                                       ctypes.c_uint32, ctypes.c_uint32]),
            "oracle_sr_bf16_row": (None, [P, i64, u64, ctypes.c_uint32, ctypes.c_uint32, P]),
            "oracle_sr_bf16_array": (None, [P, P, i64, P]),
            "oracle_learning_rate": (f64, [f64, i64, i64]),
            "oracle_pair_update": (f64, [P, P, i32, i32, f64, P]),
            "oracle_sgns_serial": (f64, [P, i64, i32, i32, P, P, P, u64, u64, i32, i64, P, P]),
            "oracle_sgns_minibatch": (f64, [P, i64, i32, i32, P, i64, P, P, u64, u64, i32, i64,
                                            P, P, P]),
            "oracle_tile_negatives": (None, [P, P, i32, u64, u64, i32, i64, i32, P]),
            "oracle_sgns_tile": (f64, [P, i64, i32, i32, P, i32, i32, i32, P, P, u64, u64, i32,
                                       i64, P, P, P]),
            "oracle_fabc_select": (i32, [P, i32, i32, i32, P, P]),
            "oracle_fabc_encode": (i64, [P, i64, i32, P, i32, P]),
            "oracle_fabc_decode": (None, [P, i64, i32, i32, P]),
            "oracle_psi_subset": (None, [i64, i32, u64, i32, i32, P]),
            "oracle_psi_node": (f64, [P, P, P, i32, i32, u64, i32, i32]),
            "oracle_feedback": (i64, [P, P, i32, P, i32, P, u64, i32, P, P, P]),
            "oracle_embed": (i32, [P, P, i32, i32, i32, P, P, i32, i64, u64, P, P, P]),
            "oracle_embed_lag": (i32, [P, P, i32, i32, i32, P, P, i32, i64, u64, i32, P, P, P]),
            "oracle_auc_pairs": (f64, [P, i64, P, i64]),
            "oracle_link_scores": (None, [P, i32, P, i64, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_lib, name)
            fn.restype = res
            fn.argtypes = args
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------------------------------------------------------------------
def philox(seed: int, ctr) -> np.ndarray:
    """Philox4x32-10 block for counter (x0, x1, x2, x3) and 64-bit key seed."""
    c = _c(ctr, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().oracle_philox(seed, _p(c), _p(out))
    return out


def walk(offsets, cols, starts, L: int, wpr: int, seed: int, round_: int) -> np.ndarray:
    off, col, st = _c(offsets, np.int32), _c(cols, np.int32), _c(starts, np.int32)
    out = np.empty((wpr * st.shape[0], L), np.int32)
    rc = lib().oracle_walk(_p(off), _p(col), off.shape[0] - 1, _p(st), st.shape[0], L, wpr,
                           seed, round_, _p(out))
    if rc:
        raise ValueError(f"oracle_walk failed ({rc})")
    return out


def walk_node2vec(offsets, cols, starts, L: int, wpr: int, p: float, q: float, seed: int,
                  round_: int) -> np.ndarray:
    """node2vec second-order walks (return parameter p, in-out parameter q)."""
    off, col, st = _c(offsets, np.int32), _c(cols, np.int32), _c(starts, np.int32)
    out = np.empty((wpr * st.shape[0], L), np.int32)
    rc = lib().oracle_walk_node2vec(_p(off), _p(col), off.shape[0] - 1, _p(st), st.shape[0], L, wpr,
                                    p, q, seed, round_, _p(out))
    if rc:
        raise ValueError(f"oracle_walk_node2vec failed ({rc})")
    return out


def counts(walks, n: int) -> np.ndarray:
    w = _c(walks, np.int32)
    out = np.empty(n, np.uint32)
    lib().oracle_counts(_p(w), w.size, n, _p(out))
    return out


def noise_table(cnt):
    """Integer alias table for the unigram^0.75 noise distribution.

    Returns (W, thr, alias, S).
    """
    c = _c(cnt, np.uint32)
    n = c.shape[0]
    W = np.empty(n, np.uint64)
    thr = np.empty(n, np.uint64)
    alias = np.empty(n, np.int32)
    S = ctypes.c_uint64(0)
    rc = lib().oracle_noise_table(_p(c), n, _p(W), _p(thr), _p(alias), ctypes.byref(S))
    if rc:
        raise RuntimeError(f"oracle_noise_table failed ({rc})")
    return W, thr, alias, int(S.value)


def draw_negative(thr, alias, S: int, seed: int, round_: int, walk_idx: int, pos: int, q: int,
                  k: int) -> int:
    return int(lib().oracle_draw_negative(_p(thr), _p(alias), thr.shape[0], S, seed, round_,
                                          walk_idx, pos, q, k))


def init_tables(n: int, d: int, seed: int):
    phi_in = np.empty((n, d), np.float64)
    phi_out = np.empty((n, d), np.float64)
    lib().oracle_init_tables(n, d, seed, _p(phi_in), _p(phi_out))
    return phi_in, phi_out


def sr_bf16(xbits: int, r16: int) -> int:
    """Stochastic rounding of the binary32 pattern xbits to bfloat16 with the
    16 random bits r16; returns the bf16 pattern."""
    return int(lib().oracle_sr_bf16(xbits & 0xffffffff, r16 & 0xffff))


def sr_bf16_keyed(xbits: int, seed: int, element: int, row: int, counter: int) -> int:
    """Stochastic rounding with bits from the rounding stream (stream 4) keyed
    by (element / 4, row, counter)."""
    return int(lib().oracle_sr_bf16_keyed(xbits & 0xffffffff, seed, element, row, counter))


def sr_bf16_array(xbits, r16) -> np.ndarray:
    """Stochastic rounding of binary32 patterns (uint32 array) with the given
    16-bit random values (uint16 array of the same length); returns uint16."""
    x = _c(xbits, np.uint32)
    r = _c(r16, np.uint16)
    assert x.shape == r.shape
    out = np.empty(x.shape[0], np.uint16)
    lib().oracle_sr_bf16_array(_p(x), _p(r), x.shape[0], _p(out))
    return out


def sr_bf16_row(xbits, seed: int, row: int, counter: int) -> np.ndarray:
    """Stochastic rounding of a row of binary32 patterns (uint32 array);
    element i takes its bits from key (i / 4, row, counter).  Returns uint16."""
    x = _c(xbits, np.uint32)
    out = np.empty(x.shape[0], np.uint16)
    lib().oracle_sr_bf16_row(_p(x), x.shape[0], seed, row, counter, _p(out))
    return out


def learning_rate(lr0: float, t: int, T: int) -> float:
    return float(lib().oracle_learning_rate(lr0, t, T))


def pair_update(in_x: np.ndarray, outs: list, eta: float) -> float:
    """Apply one Eq. 2 pair update in place; outs[0] is the center's phi_out row."""
    d = in_x.shape[0]
    ptrs = (ctypes.c_void_p * len(outs))(*[o.ctypes.data for o in outs])
    scratch = np.empty(d, np.float64)
    return float(lib().oracle_pair_update(_p(in_x), ptrs, len(outs), d, eta, _p(scratch)))


def _tp(dim, window, negatives, lr0, T):
    return _TrainParams(dim, window, negatives, lr0, T)


def sgns_serial(walks, n: int, dim: int, window: int, negatives: int, lr0: float, T: int,
                thr, alias, S: int, seed: int, round_: int, clock_base: int,
                phi_in: np.ndarray, phi_out: np.ndarray) -> float:
    w = _c(walks, np.int32)
    assert phi_in.dtype == np.float64 and phi_in.flags.c_contiguous
    assert phi_out.dtype == np.float64 and phi_out.flags.c_contiguous
    tp = _tp(dim, window, negatives, lr0, T)
    return float(lib().oracle_sgns_serial(_p(w), w.shape[0], w.shape[1], n, ctypes.byref(tp),
                                          _p(thr), _p(alias), S, seed, round_, clock_base,
                                          _p(phi_in), _p(phi_out)))


def sgns_minibatch(walks, n: int, dim: int, window: int, negatives: int, lr0: float, T: int,
                   B: int, thr, alias, S: int, seed: int, round_: int, clock_base: int,
                   phi_in: np.ndarray, phi_out: np.ndarray, per_batch: bool = False):
    w = _c(walks, np.int32)
    assert phi_in.dtype == np.float64 and phi_in.flags.c_contiguous
    assert phi_out.dtype == np.float64 and phi_out.flags.c_contiguous
    tp = _tp(dim, window, negatives, lr0, T)
    nb = (w.size + B - 1) // B
    bl = np.zeros(max(nb, 1), np.float64)
    loss = float(lib().oracle_sgns_minibatch(_p(w), w.shape[0], w.shape[1], n, ctypes.byref(tp),
                                             B, _p(thr), _p(alias), S, seed, round_, clock_base,
                                             _p(phi_in), _p(phi_out), _p(bl)))
    return (loss, bl[:nb]) if per_batch else loss


def tile_negatives(thr, alias, n: int, S: int, seed: int, round_: int, t: int, Ns: int) -> np.ndarray:
    out = np.empty(Ns, np.int32)
    lib().oracle_tile_negatives(_p(thr), _p(alias), n, S, seed, round_, t, Ns, _p(out))
    return out


def sgns_tile(walks, n: int, dim: int, window: int, negatives: int, lr0: float, T_total: int,
              tile_centers: int, Ns: int, thr, alias, S: int, seed: int, round_: int,
              clock_base: int, phi_in: np.ndarray, phi_out: np.ndarray, per_tile: bool = False,
              normalize: bool = True):
    """Shared-negatives tile form of Eq. 2, tiles of `tile_centers` centers in
    corpus order, Ns shared negatives per tile of weight negatives / Ns;
    normalize divides a node's summed tile increment by its rows in the tile."""
    w = _c(walks, np.int32)
    assert phi_in.dtype == np.float64 and phi_in.flags.c_contiguous
    assert phi_out.dtype == np.float64 and phi_out.flags.c_contiguous
    tp = _tp(dim, window, negatives, lr0, T_total)
    nt = (w.size + tile_centers - 1) // tile_centers
    tl = np.zeros(max(nt, 1), np.float64)
    loss = float(lib().oracle_sgns_tile(_p(w), w.shape[0], w.shape[1], n, ctypes.byref(tp),
                                        tile_centers, Ns, int(normalize), _p(thr), _p(alias), S,
                                        seed, round_,
                                        clock_base, _p(phi_in), _p(phi_out), _p(tl)))
    return (loss, tl[:nt]) if per_tile else loss


def psi_subset(deg: int, ks: int, seed: int, v: int, round_: int) -> np.ndarray:
    out = np.empty(ks, np.int64)
    lib().oracle_psi_subset(deg, ks, seed, v, round_, _p(out))
    return out


def psi_node(offsets, cols, phi: np.ndarray, ks: int, seed: int, round_: int, v: int) -> float:
    off, col = _c(offsets, np.int32), _c(cols, np.int32)
    ph = _c(phi, np.float64)
    return float(lib().oracle_psi_node(_p(off), _p(col), _p(ph), ph.shape[1], ks, seed, round_, v))


def feedback(offsets, cols, phi: np.ndarray, active_in, enabled: bool, mu: float, ks: int,
             reactivate: bool, seed: int, round_: int):
    """Psi of the evaluated nodes and the next active set (Eq. 4, Eq. 5)."""
    off, col = _c(offsets, np.int32), _c(cols, np.int32)
    ph = _c(phi, np.float64)
    n = off.shape[0] - 1
    a_in = _c(active_in, np.uint8)
    a_out = np.empty(n, np.uint8)
    psi = np.empty(n, np.float64)
    fp = _FeedbackParams(int(enabled), mu, ks, 0, int(reactivate))
    cnt = lib().oracle_feedback(_p(off), _p(col), n, _p(ph), ph.shape[1], ctypes.byref(fp), seed,
                                round_, _p(a_in), _p(a_out), _p(psi))
    return psi, a_out, int(cnt)


def embed(offsets, cols, L: int, wpr: int, dim: int, window: int, negatives: int, lr0: float,
          feedback_enabled: bool, mu: float, ks: int, max_rounds: int, reactivate: bool,
          seed: int, mode: str = "serial", B: int = 4096, T: int = 0, feedback_lag: int = 0):
    """Algorithm 1 end to end; returns (phi_in, phi_out, stats[rounds, 4]).
    mode: "serial", "minibatch" (B positions per batch) or "tile" (tiles of
    128 - 2 window centers with B shared negatives, row averaging).
    feedback_lag = 1: V_a^{r+1} from Psi on the table as round r's training
    starts (the round-interleaved reading of Section 5.3)."""
    off, col = _c(offsets, np.int32), _c(cols, np.int32)
    n = off.shape[0] - 1
    phi_in = np.empty((n, dim), np.float64)
    phi_out = np.empty((n, dim), np.float64)
    stats = np.zeros((max_rounds, 4), np.float64)
    tp = _tp(dim, window, negatives, lr0, T)
    fp = _FeedbackParams(int(feedback_enabled), mu, ks, max_rounds, int(reactivate))
    rounds = lib().oracle_embed_lag(_p(off), _p(col), n, L, wpr, ctypes.byref(tp), ctypes.byref(fp),
                                    {"serial": 0, "minibatch": 1, "tile": 2}[mode], B, seed, int(feedback_lag),
                                    _p(phi_in), _p(phi_out), _p(stats))
    return phi_in, phi_out, stats[:rounds]


def auc_pairs(pos_scores, neg_scores) -> float:
    """AUC by its definition over every (positive, negative) pair."""
    p, q = _c(pos_scores, np.float64), _c(neg_scores, np.float64)
    return float(lib().oracle_auc_pairs(_p(p), p.shape[0], _p(q), q.shape[0]))


def link_scores(phi: np.ndarray, pairs) -> np.ndarray:
    ph = _c(phi, np.float64)
    pr = _c(pairs, np.int32)
    out = np.empty(pr.shape[0], np.float64)
    lib().oracle_link_scores(_p(ph), ph.shape[1], _p(pr), pr.shape[0], _p(out))
    return out


def link_auc(phi: np.ndarray, pos_pairs, neg_pairs) -> float:
    return auc_pairs(link_scores(phi, pos_pairs), link_scores(phi, neg_pairs))


def fabc_select(counts, L: int, k_max: int):
    """FaBC top-k (Section 5.2.2, Eq. 7, Eq. 8): (ids, F_k)."""
    cnt = _c(counts, np.uint32)
    ids = np.zeros(max(k_max, 1), np.int32)
    F = ctypes.c_double(0.0)
    k = lib().oracle_fabc_select(_p(cnt), cnt.size, L, k_max, _p(ids), ctypes.byref(F))
    return ids[:k].copy(), F.value


def fabc_encode(walks, ids) -> np.ndarray:
    """FaBC encoding of walks[N][L] with the selected ids (bytes)."""
    w = _c(walks, np.int32)
    sel = _c(ids, np.int32)
    N, L = w.shape
    k = sel.size
    out = np.zeros(4 * N * k + N * k * ((L + 7) // 8) + 4 * N * L, np.uint8)
    size = lib().oracle_fabc_encode(_p(w), N, L, _p(sel) if k else None, k, _p(out))
    return out[:size].copy()


def fabc_decode(buf, N: int, L: int, k: int) -> np.ndarray:
    b = _c(buf, np.uint8)
    w = np.zeros((N, L), np.int32)
    lib().oracle_fabc_decode(_p(b), N, L, k, _p(w))
    return w


# ---------------------------------------------------------------------------
# the timed CPU baseline: the oracle's routines on every host core
# ---------------------------------------------------------------------------
_base = None


def baseline_lib() -> ctypes.CDLL:
    global _base
    if _base is None:
        build()
        _base = ctypes.CDLL(_BASE_LIB)
        P = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        sig = {
            "baseline_threads": (ctypes.c_int, []),
            "baseline_walk": (ctypes.c_int, [P, P, i32, P, i32, i32, u64, i32, P]),
            "baseline_sgns_hogwild": (f64, [P, i64, i32, i32, P, P, P, u64, u64, i32, i64, P, P]),
            "baseline_psi": (None, [P, P, P, i32, i32, u64, i32, P, i64, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(_base, name)
            fn.restype = res
            fn.argtypes = args
    return _base


def baseline_threads() -> int:
    return int(baseline_lib().baseline_threads())


def baseline_walk(offsets, cols, starts, L: int, seed: int, round_: int) -> np.ndarray:
    """oracle.walk with one walk per start, the starts split over all cores
    (bit-identical to the single call)."""
    off, col, st = _c(offsets, np.int32), _c(cols, np.int32), _c(starts, np.int32)
    out = np.empty((st.shape[0], L), np.int32)
    rc = baseline_lib().baseline_walk(_p(off), _p(col), off.shape[0] - 1, _p(st), st.shape[0], L, seed,
                                      round_, _p(out))
    if rc:
        raise ValueError("start out of range")
    return out


def baseline_sgns_hogwild(walks, n: int, dim: int, window: int, negatives: int, lr0: float, T: int,
                          thr, alias, S: int, seed: int, round_: int, clock_base: int,
                          phi_in: np.ndarray, phi_out: np.ndarray) -> float:
    """Binary64 Hogwild SGNS: chunks of walks through the serial oracle on
    all cores, sharing the tables without locks."""
    w = _c(walks, np.int32)
    tp = _tp(dim, window, negatives, lr0, T)
    return float(baseline_lib().baseline_sgns_hogwild(_p(w), w.shape[0], w.shape[1], n, ctypes.byref(tp),
                                                      _p(thr), _p(alias), S, seed, round_, clock_base,
                                                      _p(phi_in), _p(phi_out)))


def baseline_psi(offsets, cols, phi: np.ndarray, ks: int, seed: int, round_: int, nodes) -> np.ndarray:
    """Psi of the listed nodes on all cores (bit-identical to oracle.psi_node)."""
    off, col, nd = _c(offsets, np.int32), _c(cols, np.int32), _c(nodes, np.int32)
    out = np.empty(nd.shape[0], np.float64)
    baseline_lib().baseline_psi(_p(off), _p(col), _p(phi), phi.shape[1], ks, seed, round_, _p(nd), nd.shape[0],
                                _p(out))
    return out
