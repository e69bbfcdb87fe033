"""Oracle for the ensemble SSA: TEST INFRASTRUCTURE, not part of the product.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The CUDA library never does, and this package
never imports the CUDA library.

``ssa_oracle.cpp`` holds the plain single-threaded FP64 statement of the
method (Gillespie direct method, Sec. 2; mass-action model format, Sec. 3.2;
selective memory with average as combining function, Sec. 3.2.1 / Fig. 3).
This module builds it with g++ (``-O2 -ffp-contract=off``), computes the
integer constants of its fixed-point logarithm with Python integers, and wraps
it with numpy.

Pins (see ``tests/test_oracle_*.py``): Philox4x32-10 against triton's
independent implementation (run by its CPU interpreter); the logarithm
against mpmath and libm;
the sampler against closed forms (birth-death Poisson law, isomerisation
binomial law, expected event count), the exact CTMC transient by matrix
exponential on tiny networks, and the first-step law.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ssa_oracle.cpp")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

SCHEDULE_L = 0     # left-to-right a0 / prefix sums
SCHEDULE_W32 = 1   # 32-lane chunked sums + Kogge-Stone scan
PRECISION_FP64 = 0  # FP64 propensities (exact mode)
PRECISION_FP32 = 1  # binary32 propensities and selection sums, FP64 a0 and time
FLAG_TRUNCATED = 1
FLAG_OVERFLOW = 2
MAX_EVENTS = (1 << 32) - 1  # the event index is a 32-bit Philox counter word


# ---------------------------------------------------------------- constants
def _atanh_ratio_scaled(a: int, b: int, bits: int) -> int:
    """floor-sum approximation of atanh(a/b) * 2**bits (0 < a < b), Python ints.

    Series atanh(z) = sum_k z^(2k+1) / (2k+1); every term is floored, so the
    error is below (number of terms) * 2**-bits."""
    total = 0
    k = 0
    num = a
    den = b
    while True:
        term = (num << bits) // (den * (2 * k + 1))
        if term == 0:
            break
        total += term
        num *= a * a
        den *= b * b
        k += 1
    return total


def _round_shift(v: int, shift: int) -> int:
    """round(v / 2**shift), halves up (no exact halves occur here)."""
    return (v + (1 << (shift - 1))) >> shift


def log_constants():
    """Integer constants of the fixed-point -ln(u) (Tang-style table method).

    F_i = 1 + (2i+1)/1024 for i in 0..511.
      inv[i] = round(2^64 / F_i) = round(2^74 / (1025 + 2i))
      lnf[i] = round(2^64 ln F_i), ln F_i = 2 atanh((2i+1) / (2049 + 2i))
      ln2    = round(2^64 ln 2),   ln 2 = 2 atanh(1/3)
      k3, k5 = round(2^31 / 3), round(2^31 / 5)
    """
    W = 256
    inv = [_round_shift((1 << 75) // (1025 + 2 * i), 1) for i in range(512)]
    lnf = [_round_shift(2 * _atanh_ratio_scaled(2 * i + 1, 2049 + 2 * i, W), W - 64) for i in range(512)]
    ln2 = _round_shift(2 * _atanh_ratio_scaled(1, 3, W), W - 64)
    k3 = _round_shift((1 << 32) // 3, 1)
    k5 = _round_shift((1 << 32) // 5, 1)
    return inv, lnf, ln2, k3, k5


# ---------------------------------------------------------------- build / load
def build(force: bool = False) -> str:
    """Compile the oracle shared library (g++, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["g++", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c++17", "-shared", "-fPIC",
           "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _u64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _i64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _i32p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _f64p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def lib():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = build()
        L = ctypes.CDLL(path)
        vp = ctypes.c_void_p
        i32, i64, u64, f64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        L.oracle_init_log.argtypes = [vp, vp, u64, i64, i64]
        L.oracle_init_log.restype = ctypes.c_int
        L.oracle_philox4x32.argtypes = [vp, vp, vp]
        L.oracle_philox4x32.restype = None
        L.oracle_neg_log_u.argtypes = [u64]
        L.oracle_neg_log_u.restype = f64
        L.oracle_neg_log_u_many.argtypes = [i64, vp, vp]
        L.oracle_neg_log_u_many.restype = None
        L.oracle_uniform_grid.argtypes = [ctypes.c_int, f64, vp]
        L.oracle_uniform_grid.restype = None
        L.oracle_run.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, i64, i64, f64, ctypes.c_int, vp,
                                 u64, u64, i64, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp, vp]
        L.oracle_run.restype = ctypes.c_int
        L.oracle_trace.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, i64, f64, ctypes.c_int, vp, u64,
                                   u64, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]
        L.oracle_trace.restype = ctypes.c_int
        L.oracle_grad.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, i64, i64, f64, ctypes.c_int, vp,
                                  u64, u64, i64, ctypes.c_int, vp, vp, vp]
        L.oracle_grad.restype = ctypes.c_int
        L.oracle_avg_xy.argtypes = [ctypes.c_int, ctypes.c_int, vp, vp, vp, vp, i64, i64, f64, u64, u64, i64,
                                    ctypes.c_int, ctypes.c_int, i64, i64, vp, vp, vp, vp, vp]
        L.oracle_avg_xy.restype = ctypes.c_int
        L.oracle_set_modifiers.argtypes = [ctypes.c_int, vp, vp, vp, vp]
        L.oracle_set_modifiers.restype = ctypes.c_int
        L.oracle_select.argtypes = [ctypes.c_int, vp, ctypes.c_int, f64]
        L.oracle_select.restype = ctypes.c_int
        L.oracle_prefix.argtypes = [ctypes.c_int, vp, ctypes.c_int, vp, vp]
        L.oracle_prefix.restype = None
        L.oracle_fp32_a0.argtypes = [ctypes.c_int, vp, ctypes.c_int]
        L.oracle_fp32_a0.restype = f64
        L.oracle_finalize.argtypes = [i64, ctypes.c_int, ctypes.c_int, vp, vp, vp, vp]
        L.oracle_finalize.restype = None
        inv, lnf, ln2, k3, k5 = log_constants()
        a_inv = np.array(inv, dtype=np.uint64)
        a_lnf = np.array(lnf, dtype=np.uint64)
        rc = L.oracle_init_log(a_inv.ctypes.data, a_lnf.ctypes.data, ln2, k3, k5)
        if rc != 0:
            raise RuntimeError("oracle_init_log failed")
        _lib = L
        return L


# ---------------------------------------------------------------- wrappers
def philox4x32(ctr, key) -> np.ndarray:
    """Philox4x32-10 block for a 4-word counter and 2-word key (uint32)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().oracle_philox4x32(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def neg_log_u(q) -> np.ndarray:
    """-ln(q * 2^-53) for odd q in [1, 2^53) (fixed-point method)."""
    qa = np.ascontiguousarray(np.atleast_1d(q), dtype=np.uint64)
    out = np.empty(qa.shape[0], dtype=np.float64)
    lib().oracle_neg_log_u_many(qa.shape[0], qa.ctypes.data, out.ctypes.data)
    return out


def uniform_grid(n_grid: int, t_end: float) -> np.ndarray:
    g = np.empty(n_grid, dtype=np.float64)
    lib().oracle_uniform_grid(n_grid, float(t_end), g.ctypes.data)
    return g


def _set_modifiers(L, net):
    """Rate modifiers of `net` for the oracle calls this thread makes next."""
    mods = getattr(net, "modifier_arrays", lambda: None)()
    if mods is None:
        L.oracle_set_modifiers(0, None, None, None, None)
        return None
    f, k, lo, hi = (np.ascontiguousarray(a) for a in mods)
    L.oracle_set_modifiers(net.n_reactions, f.ctypes.data, k.ctypes.data, lo.ctypes.data, hi.ctypes.data)
    return (f, k, lo, hi)  # keep the arrays alive for the call


def _model_arrays(net):
    R = np.ascontiguousarray(net.reactants, dtype=np.int32)
    P = np.ascontiguousarray(net.products, dtype=np.int32)
    c = np.ascontiguousarray(net.rates, dtype=np.float64)
    x0 = np.ascontiguousarray(net.x0, dtype=np.int32)
    return R, P, c, x0


class OracleResult:
    def __init__(self, S1, S2, totals, traj_events=None, traj_hash=None, traj_flags=None, S3=None, S4=None):
        self.S1, self.S2 = S1, S2
        self.S3, self.S4 = S3, S4
        self.events, self.truncated, self.overflowed, self.max_x = (int(v) for v in totals)
        self.traj_events, self.traj_hash, self.traj_flags = traj_events, traj_hash, traj_flags


def run(net, n_traj: int, t_end: float, n_grid: int, seed: int, grid=None, traj_begin: int = 0,
        stream: int = 0, max_events: int = MAX_EVENTS, schedule: int = SCHEDULE_L,
        per_traj: bool = False, threads: int = 1, ids=None, precision: int = PRECISION_FP64,
        moments: bool = False) -> OracleResult:
    """Runs trajectory ids [traj_begin, traj_begin + n_traj) (or the explicit
    list ``ids``) and returns the exact int64 grid sums S1 = sum x,
    S2 = sum x^2 (shape [G, S]) plus totals.  ``threads`` > 1 splits the ids
    over Python threads (the C call releases the GIL) and adds the int64
    partial sums, which is exact and order-independent."""
    L = lib()
    R, P, c, x0 = _model_arrays(net)
    S, M = net.n_species, net.n_reactions
    g = uniform_grid(n_grid, t_end) if grid is None else np.ascontiguousarray(grid, dtype=np.float64)
    G = int(g.shape[0])
    if ids is not None:
        spans = [(int(i), int(i) + 1) for i in ids]
    else:
        spans = [(traj_begin, traj_begin + n_traj)]
    n_total = sum(e - b for b, e in spans)

    def work(span_list):
        s1 = np.zeros((G, S), dtype=np.int64)
        s2 = np.zeros((G, S), dtype=np.int64)
        s3 = np.zeros((G, S), dtype=np.float64) if moments else None
        s4 = np.zeros((G, S), dtype=np.float64) if moments else None
        tot = np.zeros(4, dtype=np.int64)
        cnt = sum(e - b for b, e in span_list)
        ev = np.zeros(cnt, dtype=np.int64) if per_traj else None
        hs = np.zeros(cnt, dtype=np.uint64) if per_traj else None
        fl = np.zeros(cnt, dtype=np.int32) if per_traj else None
        off = 0
        for b, e in span_list:
            n = e - b
            keep = _set_modifiers(L, net)  # noqa: F841
            rc = L.oracle_run(S, M, R.ctypes.data, P.ctypes.data, c.ctypes.data, x0.ctypes.data, b, e,
                              float(t_end), G, g.ctypes.data, int(seed), int(stream), int(max_events),
                              int(schedule), int(precision), s1.ctypes.data, s2.ctypes.data,
                              s3.ctypes.data if moments else None, s4.ctypes.data if moments else None,
                              ev[off:].ctypes.data if per_traj else None,
                              hs[off:].ctypes.data if per_traj else None,
                              fl[off:].ctypes.data if per_traj else None, tot.ctypes.data)
            if rc != 0:
                raise ValueError("oracle_run rejected its arguments")
            off += n
        return s1, s2, tot, ev, hs, fl, s3, s4

    if threads <= 1 or n_total < 2:
        parts = [work(spans)]
    else:
        # split ids into `threads` contiguous chunks
        flat = []
        for b, e in spans:
            flat.append((b, e))
        if len(flat) == 1:
            b, e = flat[0]
            bounds = np.linspace(b, e, threads + 1).astype(np.int64)
            chunks = [[(int(bounds[i]), int(bounds[i + 1]))] for i in range(threads) if bounds[i + 1] > bounds[i]]
        else:
            per = (len(flat) + threads - 1) // threads
            chunks = [flat[i:i + per] for i in range(0, len(flat), per)]
        with ThreadPoolExecutor(max_workers=len(chunks)) as ex:
            parts = list(ex.map(work, chunks))
    S1 = np.zeros((G, S), dtype=np.int64)
    S2 = np.zeros((G, S), dtype=np.int64)
    tot = np.zeros(4, dtype=np.int64)
    S3 = sum(p[6] for p in parts) if moments else None
    S4 = sum(p[7] for p in parts) if moments else None
    with np.errstate(over="ignore"):
        for s1, s2, t, *_ in parts:
            S1 = (S1.view(np.uint64) + s1.view(np.uint64)).view(np.int64)
            S2 = (S2.view(np.uint64) + s2.view(np.uint64)).view(np.int64)
            tot[:3] += t[:3]
            tot[3] = max(tot[3], t[3])
    if per_traj:
        ev = np.concatenate([p[3] for p in parts])
        hs = np.concatenate([p[4] for p in parts])
        fl = np.concatenate([p[5] for p in parts])
        return OracleResult(S1, S2, tot, ev, hs, fl, S3, S4)
    return OracleResult(S1, S2, tot, S3=S3, S4=S4)


def trace(net, traj_id: int, t_end: float, n_grid: int, seed: int, grid=None, stream: int = 0,
          max_events: int = MAX_EVENTS, schedule: int = SCHEDULE_L, record_max: int = 100000,
          precision: int = PRECISION_FP64):
    """One trajectory: (event times, reaction indices, per-grid states [G, S], flags)."""
    L = lib()
    R, P, c, x0 = _model_arrays(net)
    g = uniform_grid(n_grid, t_end) if grid is None else np.ascontiguousarray(grid, dtype=np.float64)
    G = int(g.shape[0])
    rt = np.zeros(record_max, dtype=np.float64)
    rj = np.zeros(record_max, dtype=np.int32)
    xs = np.zeros((G, net.n_species), dtype=np.int64)
    ne = np.zeros(1, dtype=np.int64)
    keep = _set_modifiers(L, net)  # noqa: F841
    flags = L.oracle_trace(net.n_species, net.n_reactions, R.ctypes.data, P.ctypes.data, c.ctypes.data,
                           x0.ctypes.data, int(traj_id), float(t_end), G, g.ctypes.data, int(seed), int(stream),
                           int(max_events), int(schedule), int(precision), record_max, rt.ctypes.data,
                           rj.ctypes.data,
                           xs.ctypes.data, ne.ctypes.data)
    n = int(min(ne[0], record_max))
    return rt[:n], rj[:n], xs, int(flags), int(ne[0])


def grad(net, n_traj: int, t_end: float, n_grid: int, seed: int, dL_dmean, mean, grid=None, traj_begin: int = 0,
         stream: int = 0, max_events: int = MAX_EVENTS, schedule: int = SCHEDULE_L, threads: int = 1,
         ids=None):
    """Per-trajectory likelihood-ratio contributions g [n, M] (FP64 mode):
    dL/dc = g.mean(axis=0), its standard error g.std(ddof=1) / sqrt(n)."""
    L = lib()
    R, P, c, x0 = _model_arrays(net)
    S, M = net.n_species, net.n_reactions
    g = uniform_grid(n_grid, t_end) if grid is None else np.ascontiguousarray(grid, dtype=np.float64)
    G = int(g.shape[0])
    w = np.ascontiguousarray(dL_dmean, dtype=np.float64).reshape(G, S)
    mu = np.ascontiguousarray(mean, dtype=np.float64).reshape(G, S)
    spans = [(int(i), int(i) + 1) for i in ids] if ids is not None else [(traj_begin, traj_begin + n_traj)]
    if ids is None and threads > 1 and n_traj > 1:
        bounds = np.linspace(traj_begin, traj_begin + n_traj, threads + 1).astype(np.int64)
        spans = [(int(bounds[i]), int(bounds[i + 1])) for i in range(threads) if bounds[i + 1] > bounds[i]]
    rows = sum(e - b for b, e in spans)
    out = np.zeros((rows, M), dtype=np.float64)
    offs = np.cumsum([0] + [e - b for b, e in spans])

    def work(i):
        b, e = spans[i]
        view = out[offs[i]:offs[i + 1]]
        keep = _set_modifiers(L, net)  # noqa: F841
        rc = L.oracle_grad(S, M, R.ctypes.data, P.ctypes.data, c.ctypes.data, x0.ctypes.data, b, e, float(t_end),
                           G, g.ctypes.data, int(seed), int(stream), int(max_events), int(schedule), w.ctypes.data,
                           mu.ctypes.data, view.ctypes.data)
        if rc != 0:
            raise ValueError("oracle_grad rejected its arguments")
    if threads > 1 and len(spans) > 1:
        with ThreadPoolExecutor(max_workers=min(threads, len(spans))) as ex:
            list(ex.map(work, range(len(spans))))
    else:
        for i in range(len(spans)):
            work(i)
    return out


def avg_xy(net, n_traj: int, t_end: float, seed: int, window: int, traj_begin: int = 0, stream: int = 0,
           max_events: int = MAX_EVENTS, schedule: int = SCHEDULE_W32, precision: int = PRECISION_FP64,
           max_points: int = None):
    """Selective memory along time: (t [P], mean [P, S], mean of x^2 [P, S],
    number of union points U).  Window p averages union points
    [p window, (p + 1) window) of the Avg-Y curve; window 1 returns Avg-Y
    itself (t = the union of event times with 0)."""
    L = lib()
    R, P, c, x0 = _model_arrays(net)
    S, M = net.n_species, net.n_reactions
    cap = int(max_points) if max_points is not None else 0
    npts = np.zeros(1, dtype=np.int64)
    nu = np.zeros(1, dtype=np.int64)
    for attempt in range(2):
        t = np.zeros(max(cap, 1))
        mean = np.zeros((max(cap, 1), S))
        msq = np.zeros((max(cap, 1), S))
        keep = _set_modifiers(L, net)  # noqa: F841
        rc = L.oracle_avg_xy(S, M, R.ctypes.data, P.ctypes.data, c.ctypes.data, x0.ctypes.data, int(traj_begin),
                             int(n_traj), float(t_end), int(seed), int(stream), int(max_events), int(schedule),
                             int(precision), int(window), cap, t.ctypes.data, mean.ctypes.data, msq.ctypes.data,
                             npts.ctypes.data, nu.ctypes.data)
        if rc != 0:
            raise ValueError("oracle_avg_xy rejected its arguments")
        if cap >= npts[0] or max_points is not None:
            break
        cap = int(npts[0])
    n = int(min(npts[0], cap))
    return t[:n], mean[:n], msq[:n], int(nu[0])


def select(a, target: float, schedule: int = SCHEDULE_L) -> int:
    """The reaction index the direct method picks for propensities ``a`` and
    the target r2 * total (-1 when every a_j is zero)."""
    av = np.ascontiguousarray(a, dtype=np.float64)
    return int(lib().oracle_select(av.shape[0], av.ctypes.data, int(schedule), float(target)))


def prefix_sums(a, schedule: int = SCHEDULE_L):
    """(prefix, a0) of propensities ``a`` in the given summation schedule."""
    av = np.ascontiguousarray(a, dtype=np.float64)
    pre = np.empty_like(av)
    a0 = np.zeros(1, dtype=np.float64)
    lib().oracle_prefix(int(av.shape[0]), av.ctypes.data, int(schedule), pre.ctypes.data, a0.ctypes.data)
    return pre, float(a0[0])


def fp32_a0(a32, schedule: int = SCHEDULE_W32) -> float:
    """a0 of the FP32-propensity mode for binary32 propensities ``a32``: one
    compensated binary32 pair (L) or the lanes' pairs combined by the W32
    scan in pair arithmetic (W32), widened to FP64 once."""
    av = np.ascontiguousarray(a32, dtype=np.float32)
    return float(lib().oracle_fp32_a0(int(av.shape[0]), av.ctypes.data, int(schedule)))


def finalize(n_traj: int, S1: np.ndarray, S2: np.ndarray):
    """mean = S1/N, var = (N S2 - S1^2)/(N(N-1)) with an exact int128 numerator."""
    G, S = S1.shape
    s1 = np.ascontiguousarray(S1, dtype=np.int64)
    s2 = np.ascontiguousarray(S2, dtype=np.int64)
    mean = np.empty((G, S), dtype=np.float64)
    var = np.empty((G, S), dtype=np.float64)
    lib().oracle_finalize(int(n_traj), G, S, s1.ctypes.data, s2.ctypes.data, mean.ctypes.data, var.ctypes.data)
    return mean, var
