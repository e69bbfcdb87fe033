"""Python binding of libssa (include/ssa.h): argument marshalling only.

Every step of the simulation and reduction runs in libssa's CUDA kernels.  If
``_build/libssa.so`` is missing or fails to load, every call raises; there is
no CPU path.  PyTorch supplies device memory (outputs, workspace) and the
CUDA stream for device-memory runs.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np

from . import build as _build

# status codes (ssa_status)
SSA_OK, SSA_EINVAL, SSA_ENOMEM, SSA_ECUDA, SSA_EOVERFLOW, SSA_ETRUNCATED, SSA_ETIMEOUT, SSA_EUNSUPPORTED = range(8)
PREC = {"fp64": 0, "fp32": 1}
SCHED = {"auto": 0, "thread": 1, "warp": 2}
REDUCE = {"auto": 0, "shared": 1, "global": 2}
MEM_HOST, MEM_DEVICE = 0, 1
TRAJ_TRUNCATED, TRAJ_OVERFLOW = 1, 2

# Functions declared in include/ssa.h.
EXPORTS = [
    "ssa_status_string", "ssa_last_error", "ssa_run_opts_init", "ssa_model_create", "ssa_model_destroy",
    "ssa_model_info", "ssa_ensemble_workspace_size", "ssa_ensemble_run", "ssa_ensemble_run_noalloc",
    "ssa_batch_create", "ssa_batch_tune", "ssa_batch_launch", "ssa_batch_result", "ssa_batch_network_stats",
    "ssa_batch_destroy", "ssa_batch_run", "ssa_ensemble_grad", "ssa_ensemble_avg_xy",
    "ssa_model_set_rate_modifier", "ssa_release_cached_memory", "ssa_finalize_sums",
]


class SSAError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libssa status {status}: {msg}")
        self.status = status


class RunOpts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32), ("schedule", ctypes.c_int32), ("memory", ctypes.c_int32),
        ("reduce", ctypes.c_int32), ("block_threads", ctypes.c_int32), ("grid_blocks", ctypes.c_int32),
        ("max_events", ctypes.c_int64), ("traj_offset", ctypes.c_uint64), ("stream_id", ctypes.c_uint64),
        ("cuda_stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
        ("traj_events", ctypes.c_void_p), ("traj_hash", ctypes.c_void_p), ("traj_flags", ctypes.c_void_p),
        ("device_totals", ctypes.c_void_p), ("sim_event_begin", ctypes.c_void_p), ("sim_event_end", ctypes.c_void_p),
        ("log_records", ctypes.c_int64),
    ]


class RunStats(ctypes.Structure):
    _fields_ = [("events", ctypes.c_int64), ("truncated", ctypes.c_int64), ("overflowed", ctypes.c_int64),
                ("max_x", ctypes.c_int64), ("kernel_ms", ctypes.c_double), ("schedule", ctypes.c_int32),
                ("handoffs", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads libssa.so (building it first if sources are newer)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not _build.up_to_date():
            _build.build()
        L = ctypes.CDLL(_build.LIB)
        vp, i32, i64, u64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        L.ssa_status_string.argtypes = [ctypes.c_int]
        L.ssa_status_string.restype = ctypes.c_char_p
        L.ssa_last_error.argtypes = []
        L.ssa_last_error.restype = ctypes.c_char_p
        L.ssa_run_opts_init.argtypes = [ctypes.POINTER(RunOpts)]
        L.ssa_run_opts_init.restype = None
        L.ssa_model_create.argtypes = [i32, i32, vp, vp, vp, vp, ctypes.POINTER(vp)]
        L.ssa_model_create.restype = ctypes.c_int
        L.ssa_model_set_rate_modifier.argtypes = [vp, i32, i32, f64, f64, f64]
        L.ssa_model_set_rate_modifier.restype = ctypes.c_int
        L.ssa_model_destroy.argtypes = [vp]
        L.ssa_model_destroy.restype = None
        L.ssa_model_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.ssa_model_info.restype = ctypes.c_int
        L.ssa_ensemble_workspace_size.argtypes = [vp, i64, i32, ctypes.POINTER(RunOpts), ctypes.POINTER(ctypes.c_size_t)]
        L.ssa_ensemble_workspace_size.restype = ctypes.c_int
        L.ssa_ensemble_run.argtypes = [vp, i64, f64, i32, vp, u64, ctypes.POINTER(RunOpts), vp, vp, vp, vp,
                                       ctypes.POINTER(RunStats)]
        L.ssa_ensemble_run.restype = ctypes.c_int
        L.ssa_ensemble_run_noalloc.argtypes = L.ssa_ensemble_run.argtypes
        L.ssa_ensemble_run_noalloc.restype = ctypes.c_int
        L.ssa_batch_create.argtypes = [i32, vp, vp, vp, vp, vp, ctypes.POINTER(RunOpts), ctypes.POINTER(vp)]
        L.ssa_batch_create.restype = ctypes.c_int
        L.ssa_batch_tune.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(f64)]
        L.ssa_batch_tune.restype = ctypes.c_int
        L.ssa_batch_launch.argtypes = [vp, u64, vp, vp, vp, vp, ctypes.POINTER(RunStats)]
        L.ssa_batch_launch.restype = ctypes.c_int
        L.ssa_batch_result.argtypes = [vp, i32, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                       ctypes.POINTER(vp)]
        L.ssa_batch_result.restype = ctypes.c_int
        L.ssa_batch_network_stats.argtypes = [vp, i32, ctypes.POINTER(RunStats)]
        L.ssa_batch_network_stats.restype = ctypes.c_int
        L.ssa_batch_destroy.argtypes = [vp]
        L.ssa_batch_destroy.restype = None
        L.ssa_batch_run.argtypes = [i32, vp, vp, vp, vp, vp, u64, ctypes.POINTER(RunOpts), vp, vp]
        L.ssa_batch_run.restype = ctypes.c_int
        L.ssa_ensemble_grad.argtypes = [vp, i64, f64, i32, vp, u64, ctypes.POINTER(RunOpts), vp, vp, vp, vp]
        L.ssa_ensemble_grad.restype = ctypes.c_int
        L.ssa_ensemble_avg_xy.argtypes = [vp, i64, f64, u64, ctypes.POINTER(RunOpts), i64, i64, vp, vp, vp,
                                          ctypes.POINTER(i64), ctypes.POINTER(i64)]
        L.ssa_ensemble_avg_xy.restype = ctypes.c_int
        L.ssa_finalize_sums.argtypes = [i64, i32, i32, vp, vp, vp, vp]
        L.ssa_finalize_sums.restype = ctypes.c_int
        L.ssa_release_cached_memory.argtypes = []
        L.ssa_release_cached_memory.restype = ctypes.c_int
        _lib = L
        return L


def _check(st: int):
    if st != SSA_OK:
        L = lib()
        raise SSAError(st, L.ssa_last_error().decode(errors="replace") or L.ssa_status_string(st).decode())


class Model:
    """A reaction network copied into libssa (ssa_model_create)."""

    def __init__(self, reactants, products, rates, x0):
        R = np.ascontiguousarray(reactants, dtype=np.int32)
        P = np.ascontiguousarray(products, dtype=np.int32)
        c = np.ascontiguousarray(rates, dtype=np.float64)
        x = np.ascontiguousarray(x0, dtype=np.int32)
        if R.ndim != 2 or P.shape != R.shape or c.shape != (R.shape[0],) or x.shape != (R.shape[1],):
            raise ValueError("reactants/products must be [M, S], rates [M], x0 [S]")
        self.n_reactions, self.n_species = int(R.shape[0]), int(R.shape[1])
        h = ctypes.c_void_p()
        _check(lib().ssa_model_create(self.n_species, self.n_reactions, R.ctypes.data, P.ctypes.data,
                                      c.ctypes.data, x.ctypes.data, ctypes.byref(h)))
        self._h = h

    @classmethod
    def from_network(cls, net) -> "Model":
        m = cls(net.reactants, net.products, net.rates, net.x0)
        for j, sp, slope, lo, hi in getattr(net, "modifiers", []):
            m.set_rate_modifier(j, sp, slope, lo, hi)
        return m

    def set_rate_modifier(self, reaction: int, species: int, slope: float, lo: float = 0.0,
                          hi: float = float("inf")):
        """ssa_model_set_rate_modifier: rate = min(max(c + slope x_species, lo), hi)."""
        _check(lib().ssa_model_set_rate_modifier(self._h, int(reaction), int(species), float(slope), float(lo),
                                                 float(hi)))

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ssa_model_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class EnsembleResult:
    mean: object
    var: object
    sum1: object
    sum2: object
    events: int
    truncated: int
    overflowed: int
    max_x: int
    kernel_ms: float
    traj_events: object = None
    traj_hash: object = None
    traj_flags: object = None
    schedule: int = 0  # SCHED value of the schedule that ran (1 thread, 2 warp)
    handoffs: int = 0  # trajectories passed between warps (thread schedule)


def make_opts(precision="fp64", schedule="auto", reduce="auto", memory=MEM_HOST, max_events=0, traj_offset=0,
              stream_id=0, block_threads=0, grid_blocks=0, cuda_stream=None, workspace=None, workspace_bytes=0,
              device_totals=None, sim_event_begin=None, sim_event_end=None, log_records=0):
    o = RunOpts()
    lib().ssa_run_opts_init(ctypes.byref(o))
    o.precision = PREC[precision]
    o.schedule = SCHED[schedule]
    o.reduce = REDUCE[reduce]
    o.memory = memory
    o.max_events = int(max_events)
    o.traj_offset = int(traj_offset)
    o.stream_id = int(stream_id)
    o.block_threads = int(block_threads)
    o.grid_blocks = int(grid_blocks)
    o.cuda_stream = cuda_stream
    o.workspace = workspace
    o.workspace_bytes = int(workspace_bytes)
    o.device_totals = device_totals
    o.sim_event_begin = sim_event_begin
    o.sim_event_end = sim_event_end
    o.log_records = int(log_records)
    return o


def workspace_bytes(model: Model, n_traj: int, n_grid: int, opts: RunOpts) -> int:
    out = ctypes.c_size_t()
    _check(lib().ssa_ensemble_workspace_size(model.handle, int(n_traj), int(n_grid), ctypes.byref(opts),
                                             ctypes.byref(out)))
    return int(out.value)


def ensemble_run(model: Model, n_traj: int, t_end: float, n_grid: int, seed: int, grid=None, *, device=None,
                 per_traj: bool = False, want_sums: bool = True, stats: bool = True, **opt_kw) -> EnsembleResult:
    """ssa_ensemble_run.  ``device=None`` runs with host buffers (numpy in and
    out, synchronous); a torch device runs with torch-allocated device buffers
    on torch's current stream of that device."""
    L = lib()
    G, S = int(n_grid if grid is None else len(grid)), model.n_species
    st = RunStats()
    if device is None:
        opts = make_opts(memory=MEM_HOST, **opt_kw)
        mean = np.empty((G, S), dtype=np.float64)
        var = np.empty((G, S), dtype=np.float64)
        s1 = np.empty((G, S), dtype=np.int64) if want_sums else None
        s2 = np.empty((G, S), dtype=np.int64) if want_sums else None
        g = None if grid is None else np.ascontiguousarray(grid, dtype=np.float64)
        tev = np.empty(n_traj, dtype=np.int64) if per_traj else None
        ths = np.empty(n_traj, dtype=np.uint64) if per_traj else None
        tfl = np.empty(n_traj, dtype=np.int32) if per_traj else None
        if per_traj:
            opts.traj_events, opts.traj_hash, opts.traj_flags = tev.ctypes.data, ths.ctypes.data, tfl.ctypes.data
        _check(L.ssa_ensemble_run(model.handle, int(n_traj), float(t_end), G,
                                  None if g is None else g.ctypes.data, int(seed), ctypes.byref(opts),
                                  mean.ctypes.data, var.ctypes.data, None if s1 is None else s1.ctypes.data,
                                  None if s2 is None else s2.ctypes.data, ctypes.byref(st) if stats else None))
    else:
        import torch
        dev = torch.device(device)
        stream = torch.cuda.current_stream(dev)
        opts = make_opts(memory=MEM_DEVICE, cuda_stream=stream.cuda_stream, **opt_kw)
        with torch.cuda.device(dev):
            mean = torch.empty((G, S), dtype=torch.float64, device=dev)
            var = torch.empty((G, S), dtype=torch.float64, device=dev)
            s1 = torch.empty((G, S), dtype=torch.int64, device=dev) if want_sums else None
            s2 = torch.empty((G, S), dtype=torch.int64, device=dev) if want_sums else None
            g = None if grid is None else torch.as_tensor(grid, dtype=torch.float64, device=dev).contiguous()
            tev = torch.empty(n_traj, dtype=torch.int64, device=dev) if per_traj else None
            ths = torch.empty(n_traj, dtype=torch.int64, device=dev) if per_traj else None
            tfl = torch.empty(n_traj, dtype=torch.int32, device=dev) if per_traj else None
            if per_traj:
                opts.traj_events, opts.traj_hash, opts.traj_flags = tev.data_ptr(), ths.data_ptr(), tfl.data_ptr()
            if opts.workspace is None:
                nbytes = workspace_bytes(model, n_traj, G, opts)
                ws = torch.empty(nbytes, dtype=torch.uint8, device=dev)
                opts.workspace, opts.workspace_bytes = ws.data_ptr(), nbytes
            _check(L.ssa_ensemble_run(model.handle, int(n_traj), float(t_end), G,
                                      None if g is None else g.data_ptr(), int(seed), ctypes.byref(opts),
                                      mean.data_ptr(), var.data_ptr(), None if s1 is None else s1.data_ptr(),
                                      None if s2 is None else s2.data_ptr(), ctypes.byref(st) if stats else None))
    return EnsembleResult(mean, var, s1, s2, int(st.events), int(st.truncated), int(st.overflowed), int(st.max_x),
                          float(st.kernel_ms), tev, ths, tfl, int(st.schedule), int(st.handoffs))


def ensemble_grad(model: Model, n_traj: int, t_end: float, n_grid: int, seed: int, dL_dmean, mean, grid=None, *,
                  device=None, per_traj: bool = False, traj_events=None, **opt_kw):
    """ssa_ensemble_grad: (dL/drates [M], standard errors [M], per-trajectory
    contributions [M, N] or None).  ``device=None``: numpy in and out;
    a torch device: torch tensors on that device (torch's current stream).
    ``traj_events``: the forward's per-trajectory event counts (int64 [N],
    same memory space), to replay the longest trajectories first."""
    L = lib()
    M = model.n_reactions
    G = int(n_grid if grid is None else len(grid))
    if device is None:
        w = np.ascontiguousarray(dL_dmean, dtype=np.float64)
        mu = np.ascontiguousarray(mean, dtype=np.float64)
        g = None if grid is None else np.ascontiguousarray(grid, dtype=np.float64)
        out = np.empty(M)
        se = np.empty(M)
        traj = np.empty((M, int(n_traj))) if per_traj else None
        opts = make_opts(memory=MEM_HOST, workspace=None if traj is None else traj.ctypes.data,
                         workspace_bytes=0 if traj is None else traj.nbytes, **opt_kw)
        if traj_events is not None:
            tev = np.ascontiguousarray(traj_events, dtype=np.int64)
            assert tev.shape == (int(n_traj),)
            opts.traj_events = tev.ctypes.data
        _check(L.ssa_ensemble_grad(model.handle, int(n_traj), float(t_end), G,
                                   None if g is None else g.ctypes.data, int(seed), ctypes.byref(opts),
                                   w.ctypes.data, mu.ctypes.data, out.ctypes.data, se.ctypes.data))
        return out, se, traj
    import torch
    dev = torch.device(device)
    stream = torch.cuda.current_stream(dev)
    w = torch.as_tensor(dL_dmean, dtype=torch.float64, device=dev).contiguous()
    mu = torch.as_tensor(mean, dtype=torch.float64, device=dev).contiguous()
    g = None if grid is None else torch.as_tensor(grid, dtype=torch.float64, device=dev).contiguous()
    out = torch.empty(M, dtype=torch.float64, device=dev)
    se = torch.empty(M, dtype=torch.float64, device=dev)
    traj = torch.empty((M, int(n_traj)), dtype=torch.float64, device=dev) if per_traj else None
    opts = make_opts(memory=MEM_DEVICE, cuda_stream=stream.cuda_stream,
                     workspace=None if traj is None else traj.data_ptr(),
                     workspace_bytes=0 if traj is None else traj.numel() * 8, **opt_kw)
    if traj_events is not None:
        tev = torch.as_tensor(traj_events, device=dev).to(torch.int64).contiguous()
        assert tev.shape == (int(n_traj),)
        opts.traj_events = tev.data_ptr()
    _check(L.ssa_ensemble_grad(model.handle, int(n_traj), float(t_end), G, None if g is None else g.data_ptr(),
                               int(seed), ctypes.byref(opts), w.data_ptr(), mu.data_ptr(), out.data_ptr(),
                               se.data_ptr()))
    return out, se, traj


def ensemble_avg_xy(model: Model, n_traj: int, t_end: float, seed: int, window: int = 0, *, max_points=None,
                    **opt_kw):
    """ssa_ensemble_avg_xy with host outputs: (t [P], mean [P, S], mean of
    x^2 [P, S], number of union points U).  window 0 means n_traj; window 1
    gives Avg-Y on the union of event times.  Without max_points, room for
    65,536 windows is offered first and the call is repeated only when there
    are more."""
    L = lib()
    S = model.n_species
    P = ctypes.c_int64()
    U = ctypes.c_int64()
    cap = 65536 if max_points is None else int(max_points)
    while True:
        t = np.empty(max(cap, 1))
        mean = np.empty((max(cap, 1), S))
        msq = np.empty((max(cap, 1), S))
        opts = make_opts(memory=MEM_HOST, **opt_kw)
        _check(L.ssa_ensemble_avg_xy(model.handle, int(n_traj), float(t_end), int(seed), ctypes.byref(opts),
                                     int(window), int(cap), t.ctypes.data, mean.ctypes.data, msq.ctypes.data,
                                     ctypes.byref(P), ctypes.byref(U)))
        if max_points is not None or int(P.value) <= cap:
            break
        cap = int(P.value)
    n = min(int(P.value), int(cap))
    return t[:n], mean[:n], msq[:n], int(U.value)


def release_cached_memory() -> None:
    """ssa_release_cached_memory: return the workspaces the library keeps
    between calls to the driver."""
    _check(lib().ssa_release_cached_memory())


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr


class Batch:
    """A batch of networks run together (ssa_batch_create / _tune / _launch).

    ``device=None`` keeps outputs on the host (numpy, synchronous launches); a
    torch device makes launch() return torch tensors on that device, filled on
    torch's current stream."""

    def __init__(self, models, n_traj, t_end, n_grid, grids=None, *, device=None, **opt_kw):
        self.n = len(models)
        self.models = list(models)  # the batch references the models: keep them alive
        self.n_traj = np.ascontiguousarray(n_traj, dtype=np.int64)
        self.t_end = np.ascontiguousarray(t_end, dtype=np.float64)
        self.n_grid = np.ascontiguousarray(n_grid, dtype=np.int32)
        if not (self.n_traj.shape == self.t_end.shape == self.n_grid.shape == (self.n,)):
            raise ValueError("n_traj, t_end and n_grid need one entry per model")
        self.device = device
        if device is not None:
            import torch
            dev = torch.device(device)
            self._stream = torch.cuda.current_stream(dev)
            opt_kw.setdefault("cuda_stream", self._stream.cuda_stream)
            self.opts = make_opts(memory=MEM_DEVICE, **opt_kw)
        else:
            self.opts = make_opts(memory=MEM_HOST, **opt_kw)
        self._grids = None
        gp = None
        if grids is not None:
            self._grids = [None if g is None else np.ascontiguousarray(g, dtype=np.float64) for g in grids]
            gp = _ptr_array([None if g is None else g.ctypes.data for g in self._grids])
        hp = _ptr_array([m.handle.value for m in self.models])
        h = ctypes.c_void_p()
        _check(lib().ssa_batch_create(self.n, hp, self.n_traj.ctypes.data, self.t_end.ctypes.data,
                                      self.n_grid.ctypes.data, gp, ctypes.byref(self.opts), ctypes.byref(h)))
        self._h = h
        self.species = [m.n_species for m in self.models]

    def tune(self):
        """Autotunes the launch shape; returns (block_threads, split, sample_ms)."""
        t, sp, ms = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_double()
        _check(lib().ssa_batch_tune(self._h, ctypes.byref(t), ctypes.byref(sp), ctypes.byref(ms)))
        return int(t.value), bool(sp.value), float(ms.value)

    def launch(self, seed: int, want_sums: bool = False, stats: bool = True):
        """Runs the batch; returns (list of per-network dicts with mean, var
        and, if asked, sum1 / sum2; RunStats or None)."""
        outs = []
        for b in range(self.n):
            shape = (int(self.n_grid[b]), self.species[b])
            if self.device is None:
                o = {"mean": np.empty(shape), "var": np.empty(shape)}
                if want_sums:
                    o["sum1"] = np.empty(shape, dtype=np.int64)
                    o["sum2"] = np.empty(shape, dtype=np.int64)
            else:
                import torch
                o = {"mean": torch.empty(shape, dtype=torch.float64, device=self.device),
                     "var": torch.empty(shape, dtype=torch.float64, device=self.device)}
                if want_sums:
                    o["sum1"] = torch.empty(shape, dtype=torch.int64, device=self.device)
                    o["sum2"] = torch.empty(shape, dtype=torch.int64, device=self.device)
            outs.append(o)

        def ptr(a):
            return a.ctypes.data if isinstance(a, np.ndarray) else a.data_ptr()

        def arr(key):
            if key not in outs[0]:
                return None
            return _ptr_array([ptr(o[key]) for o in outs])

        st = RunStats()
        _check(lib().ssa_batch_launch(self._h, int(seed), arr("mean"), arr("var"), arr("sum1"), arr("sum2"),
                                      ctypes.byref(st) if stats else None))
        return outs, (st if stats else None)

    def network_stats(self, index: int) -> RunStats:
        st = RunStats()
        _check(lib().ssa_batch_network_stats(self._h, int(index), ctypes.byref(st)))
        return st

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().ssa_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
