"""Thin Python binding of libsand's C-ABI (include/sand.h).

Argument marshalling only: every step of a query runs in libsand's CUDA
kernels.  PyTorch provides device memory (tensors, the workspace) and the
current CUDA stream.  There is no CPU fallback: if libsand.so is missing or
cannot load, importing the functions raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsand.so")

SAND_OK, SAND_EINVAL, SAND_ENOMEM, SAND_EFORMAT, SAND_ECUDA, SAND_ETIMEOUT, SAND_ENOMAP, SAND_EUNSUPPORTED = range(8)
_STATUS = {0: "SAND_OK", 1: "SAND_EINVAL", 2: "SAND_ENOMEM", 3: "SAND_EFORMAT", 4: "SAND_ECUDA",
           5: "SAND_ETIMEOUT", 6: "SAND_ENOMAP", 7: "SAND_EUNSUPPORTED"}
PRECISION = {"fp32": 0, "fp32_simt": 1, "fp16": 2, "bf16": 3, "fp8": 4}
TAIL_LINEAR, TAIL_MULT = 0, 1
ACT_SINE, ACT_RELU, ACT_FINER = 0, 1, 2
ENC_NONE, ENC_FOURIER = 0, 1
FLAG_NAN_INPUT, FLAG_TIMEOUT = 1, 2


class SandError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class TmlpDesc(ctypes.Structure):
    _fields_ = [("n_layers", ctypes.c_int32), ("width", ctypes.c_int32), ("in_dim", ctypes.c_int32),
                ("tail_kind", ctypes.c_int32), ("activation", ctypes.c_int32), ("encoder", ctypes.c_int32),
                ("n_freq", ctypes.c_int32), ("omega0", ctypes.c_float)]


class DepthMapDesc(ctypes.Structure):
    _fields_ = [("max_level", ctypes.c_int32), ("n_layers", ctypes.c_int32), ("n_nodes", ctypes.c_int32)]


class QueryOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_depth", ctypes.c_int32), ("full_depth", ctypes.c_int32),
                ("all_tails", ctypes.c_int32), ("d_exit_layers", ctypes.c_void_p), ("d_workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("stage_events", ctypes.c_void_p),
                ("wait_limit_us", ctypes.c_uint32), ("reserved", ctypes.c_int32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_int32), ("precision", ctypes.c_int32), ("mem_budget", ctypes.c_size_t),
                ("max_batch_points", ctypes.c_int64), ("model_precision", ctypes.c_void_p)]


class ServerReport(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_int64), ("batches", ctypes.c_int64), ("points", ctypes.c_int64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("queries_per_s", ctypes.c_double), ("arena_bytes", ctypes.c_size_t), ("span_ms", ctypes.c_double),
                ("batch_ms_sum", ctypes.c_double)]


class TraceOpts(ctypes.Structure):
    _fields_ = [("max_steps", ctypes.c_int32), ("hit_eps", ctypes.c_float), ("poll_every", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


RAY_MISS, RAY_HIT, RAY_STEPS, RAY_NAN = 0, 1, 2, 3


class MapBuildOpts(ctypes.Structure):
    _fields_ = [("samples_per_axis", ctypes.c_int32), ("r", ctypes.c_float), ("far_sign", ctypes.c_int32),
                ("precision", ctypes.c_int32)]


class TrainOpts(ctypes.Structure):
    _fields_ = [("max_points", ctypes.c_int64), ("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float), ("reserved", ctypes.c_int32)]


class QueryStats(ctypes.Structure):
    _fields_ = [("flags", ctypes.c_uint32), ("n_network", ctypes.c_uint32), ("count", ctypes.c_uint32 * 16)]


_lib = None
EXPORTS = ("sand_load_tmlp", "sand_load_tmlp_mem", "sand_load_depth_map", "sand_load_depth_map_mem",
           "sand_workspace_bytes", "sand_query_sdf", "sand_query_sdf_grad", "sand_query_sdf_host",
           "sand_read_stats", "sand_model_desc", "sand_free", "sand_last_error", "sand_server_create",
           "sand_server_submit", "sand_server_wait", "sand_server_stats", "sand_server_destroy",
           "sand_trace_state_bytes", "sand_sphere_trace", "sand_build_depth_map", "sand_query_sdf_dynamic",
           "sand_probe_rate", "sand_query_sdf_noalloc", "sand_trainer_create", "sand_train_step",
           "sand_trainer_params", "sand_trainer_commit", "sand_trainer_status", "sand_trainer_destroy")


def lib() -> ctypes.CDLL:
    """Load libsand.so (built by __graft_entry__.build() / paper_2604_25936_gb300.build)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libsand.so is not built (%s); run `python -c 'import __graft_entry__ as g; g.build()'`"
                          % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    P, I64, I32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    L.sand_load_tmlp.argtypes = [ctypes.c_char_p, I32, ctypes.POINTER(P)]
    L.sand_load_tmlp_mem.argtypes = [ctypes.POINTER(TmlpDesc), P, ctypes.c_size_t, I32, ctypes.POINTER(P)]
    L.sand_load_depth_map.argtypes = [P, ctypes.c_char_p]
    L.sand_load_depth_map_mem.argtypes = [P, ctypes.POINTER(DepthMapDesc), P, P, P]
    L.sand_workspace_bytes.argtypes = [P, I64, I32]
    L.sand_workspace_bytes.restype = ctypes.c_size_t
    L.sand_query_sdf.argtypes = [P, P, I64, P, ctypes.POINTER(QueryOpts), P]
    L.sand_query_sdf_grad.argtypes = [P, P, I64, P, P, ctypes.POINTER(QueryOpts), P]
    L.sand_query_sdf_host.argtypes = [P, P, I64, P, ctypes.POINTER(QueryOpts), P]
    L.sand_read_stats.argtypes = [P, P, ctypes.POINTER(QueryStats), P]
    L.sand_model_desc.argtypes = [P, ctypes.POINTER(TmlpDesc)]
    L.sand_free.argtypes = [P]
    L.sand_last_error.restype = ctypes.c_char_p
    L.sand_server_create.argtypes = [P, I32, ctypes.POINTER(ServerOpts), ctypes.POINTER(P)]
    L.sand_server_submit.argtypes = [P, I32, P, I64, P, ctypes.POINTER(ctypes.c_uint64)]
    L.sand_server_wait.argtypes = [P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]
    L.sand_server_stats.argtypes = [P, ctypes.POINTER(ServerReport)]
    L.sand_server_destroy.argtypes = [P]
    L.sand_trace_state_bytes.argtypes = [I64]
    L.sand_trace_state_bytes.restype = ctypes.c_size_t
    L.sand_sphere_trace.argtypes = [P, P, I32, P, I64, ctypes.POINTER(TraceOpts), ctypes.POINTER(QueryOpts), P, P, P,
                                    P, P]
    L.sand_build_depth_map.argtypes = [P, ctypes.POINTER(DepthMapDesc), P, P, ctypes.POINTER(MapBuildOpts), P, P]
    L.sand_query_sdf_dynamic.argtypes = [P, P, I64, ctypes.c_float, P, P, ctypes.POINTER(QueryOpts), P]
    L.sand_probe_rate.argtypes = [I32, I32, I32, I32, P, P]
    L.sand_query_sdf_noalloc.argtypes = [P, P, I64, P, ctypes.POINTER(QueryOpts), P]
    L.sand_trainer_create.argtypes = [P, ctypes.POINTER(TrainOpts), ctypes.POINTER(P)]
    L.sand_train_step.argtypes = [P, P, P, I64, P, P, I32, P]
    L.sand_trainer_params.argtypes = [P, P, ctypes.c_size_t]
    L.sand_trainer_commit.argtypes = [P]
    L.sand_trainer_status.argtypes = [P, P]
    L.sand_trainer_destroy.argtypes = [P]
    for name in EXPORTS:
        if name not in ("sand_workspace_bytes", "sand_last_error", "sand_trace_state_bytes"):
            getattr(L, name).restype = ctypes.c_int
    _lib = L
    return L


PROBE_FFMA, PROBE_SIN = 0, 1
PROBE_THREADS, PROBE_CHAINS = 256, 8


def probe_rate(kind: int, n_blocks: int, iters: int, sink: torch.Tensor, stream: Optional[torch.cuda.Stream] = None):
    """Launch an issue-rate probe (sand_probe_rate) on sink's device: PROBE_FFMA runs
    2 * PROBE_CHAINS * iters * PROBE_THREADS * n_blocks FLOP, PROBE_SIN
    PROBE_CHAINS * iters * PROBE_THREADS * n_blocks hardware sines.  Time it with events."""
    assert sink.is_cuda and sink.dtype == torch.float32 and sink.numel() >= n_blocks * PROBE_THREADS
    _check(lib().sand_probe_rate(int(kind), sink.device.index, int(n_blocks), int(iters),
                                 ctypes.c_void_p(sink.data_ptr()), _stream_handle(stream)))


def _check(status: int):
    if status != SAND_OK:
        raise SandError(status, lib().sand_last_error().decode(errors="replace"))


def _stream_handle(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _as_points(points: torch.Tensor, device: int) -> torch.Tensor:
    if not isinstance(points, torch.Tensor) or points.dtype != torch.float32 or points.dim() != 2 or points.shape[1] != 3:
        raise ValueError("points must be a float32 tensor of shape [n, 3]")
    if points.device.type != "cuda" or points.device.index != device:
        raise ValueError("points must live on cuda:%d" % device)
    return points.contiguous()


class Model:
    """A T-MLP plus its depth map, resident on one GPU (a libsand sand_model handle)."""

    def __init__(self, handle: ctypes.c_void_p, device: int):
        self._h = handle
        self.device = device
        d = TmlpDesc()
        _check(lib().sand_model_desc(self._h, ctypes.byref(d)))
        self.desc = d
        self._ws = None

    # ---------------------------------------------------------------- loading
    @classmethod
    def from_file(cls, path: str, device: int = 0) -> "Model":
        h = ctypes.c_void_p()
        _check(lib().sand_load_tmlp(path.encode(), device, ctypes.byref(h)))
        return cls(h, device)

    @classmethod
    def from_params(cls, n_layers, width, in_dim, tail_kind, activation, encoder, n_freq, omega0,
                    params: np.ndarray, device: int = 0) -> "Model":
        d = TmlpDesc(n_layers, width, in_dim, tail_kind, activation, encoder, n_freq, omega0)
        p = np.ascontiguousarray(params, dtype=np.float32)
        h = ctypes.c_void_p()
        _check(lib().sand_load_tmlp_mem(ctypes.byref(d), p.ctypes.data_as(ctypes.c_void_p), p.size, device,
                                        ctypes.byref(h)))
        return cls(h, device)

    def load_depth_map(self, path: str) -> None:
        _check(lib().sand_load_depth_map(self._h, path.encode()))

    def set_depth_map(self, max_level: int, n_layers: int, child: np.ndarray, depth: np.ndarray,
                      far: np.ndarray) -> None:
        c = np.ascontiguousarray(child, np.int32)
        d = np.ascontiguousarray(depth, np.uint8)
        f = np.ascontiguousarray(far, np.float32)
        if not (c.size == d.size == f.size):
            raise ValueError("child, depth and far must have one entry per node")
        desc = DepthMapDesc(max_level, n_layers, c.size)
        _check(lib().sand_load_depth_map_mem(self._h, ctypes.byref(desc), c.ctypes.data_as(ctypes.c_void_p),
                                             d.ctypes.data_as(ctypes.c_void_p), f.ctypes.data_as(ctypes.c_void_p)))

    # ---------------------------------------------------------------- queries
    def workspace_bytes(self, n: int, grad: bool = False) -> int:
        return int(lib().sand_workspace_bytes(self._h, int(n), int(grad)))

    def workspace(self, n: int, grad: bool = False) -> torch.Tensor:
        """A torch-allocated device workspace big enough for n points (reused when possible)."""
        need = self.workspace_bytes(n, grad)
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda:%d" % self.device)
        return self._ws

    def _opts(self, precision: str, max_depth: int, full_depth: bool, exit_layers, ws, events=None) -> QueryOpts:
        if precision not in PRECISION:
            raise ValueError("precision must be one of %s" % sorted(PRECISION))
        o = QueryOpts()
        if events is not None:
            if len(events) != 3:
                raise ValueError("events: three torch.cuda.Event(enable_timing=True)")
            for e in events:
                if not e.cuda_event:
                    e.record()  # torch creates the event handle on first record
            arr = (ctypes.c_void_p * 3)(*[e.cuda_event for e in events])
            o.stage_events = ctypes.cast(arr, ctypes.c_void_p)
            o._keep = arr
        o.precision = PRECISION[precision]
        o.max_depth = int(max_depth)
        o.full_depth = int(bool(full_depth))
        o.d_exit_layers = exit_layers.data_ptr() if exit_layers is not None else None
        if ws is not None:
            base = ws.data_ptr()
            off = (-base) % 256
            o.d_workspace = base + off
            o.workspace_bytes = ws.numel() - off
        return o

    def query(self, points: torch.Tensor, precision: str = "fp32", max_depth: int = 0, full_depth: bool = False,
              exit_layers: bool = False, out: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
              stream: Optional[torch.cuda.Stream] = None, events=None, all_tails: bool = False):
        """SDF at every point (SAND inference; full_depth=True runs the plain T-MLP to layer L; with
        all_tails as well, returns [n, L]: y_1 .. y_L of every point).
        events: optional three timing events recorded before the lookup, before and after the T-MLP kernel."""
        pts = _as_points(points, self.device)
        n = pts.shape[0]
        if out is None:
            shape = (n, self.desc.n_layers) if all_tails else (n,)
            out = torch.empty(shape, dtype=torch.float32, device=pts.device)
        el = torch.empty(n, dtype=torch.uint8, device=pts.device) if exit_layers else None
        ws = workspace if workspace is not None else self.workspace(0 if full_depth else n)
        o = self._opts(precision, max_depth, full_depth, el, ws, events)
        o.all_tails = int(bool(all_tails))
        _check(lib().sand_query_sdf(self._h, ctypes.c_void_p(pts.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                    ctypes.byref(o), _stream_handle(stream)))
        return (out, el) if exit_layers else out

    def query_grad(self, points: torch.Tensor, precision: str = "fp32", max_depth: int = 0, full_depth: bool = False,
                   exit_layers: bool = False, workspace: Optional[torch.Tensor] = None,
                   stream: Optional[torch.cuda.Stream] = None):
        """(SDF, dSDF/dx) at every point."""
        pts = _as_points(points, self.device)
        n = pts.shape[0]
        out = torch.empty(n, dtype=torch.float32, device=pts.device)
        grad = torch.empty((n, 3), dtype=torch.float32, device=pts.device)
        el = torch.empty(n, dtype=torch.uint8, device=pts.device) if exit_layers else None
        ws = workspace if workspace is not None else self.workspace(0 if full_depth else n, grad=True)
        o = self._opts(precision, max_depth, full_depth, el, ws)
        _check(lib().sand_query_sdf_grad(self._h, ctypes.c_void_p(pts.data_ptr()), n, ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(grad.data_ptr()), ctypes.byref(o), _stream_handle(stream)))
        return (out, grad, el) if exit_layers else (out, grad)

    def query_host(self, points, out=None, precision: str = "fp32", max_depth: int = 0, full_depth: bool = False,
                   stream: Optional[torch.cuda.Stream] = None):
        """SDF for host-memory points (numpy or CPU tensor, ideally pinned); copies run inside libsand."""
        if isinstance(points, torch.Tensor):
            if points.device.type != "cpu" or points.dtype != torch.float32:
                raise ValueError("host points must be a float32 CPU tensor")
            pts = points.contiguous()
            n = pts.shape[0]
            if out is None:
                out = torch.empty(n, dtype=torch.float32, pin_memory=pts.is_pinned())
            pp, op = pts.data_ptr(), out.data_ptr()
        else:
            pts = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
            n = pts.shape[0]
            if out is None:
                out = np.empty(n, np.float32)
            pp, op = pts.ctypes.data, out.ctypes.data
        o = self._opts(precision, max_depth, full_depth, None, None)
        _check(lib().sand_query_sdf_host(self._h, ctypes.c_void_p(pp), n, ctypes.c_void_p(op), ctypes.byref(o),
                                         _stream_handle(stream)))
        return out

    def sphere_trace(self, origin: torch.Tensor, dirs: torch.Tensor, max_steps: int = 64, hit_eps: float = 1e-4,
                     precision: str = "fp32", max_depth: int = 0, normals: bool = True, poll_every: int = 8,
                     stream: Optional[torch.cuda.Stream] = None):
        """Sphere-trace rays through the SAND SDF.  origin: [3] (shared) or [n, 3]; dirs: [n, 3].
        Returns (t [n], state [n] uint8 RAY_*, steps [n] uint8, grad [n, 3] at hits or None)."""
        d = _as_points(dirs, self.device)
        n = d.shape[0]
        o = origin.to(device=d.device, dtype=torch.float32).contiguous()
        per_ray = o.dim() == 2
        if (per_ray and tuple(o.shape) != (n, 3)) or (not per_ray and o.numel() != 3):
            raise ValueError("origin must be [3] or [n, 3]")
        t = torch.empty(n, dtype=torch.float32, device=d.device)
        state = torch.empty(n, dtype=torch.uint8, device=d.device)
        steps = torch.empty(n, dtype=torch.uint8, device=d.device)
        g = torch.empty((n, 3), dtype=torch.float32, device=d.device) if normals else None
        to = TraceOpts(int(max_steps), float(hit_eps), int(poll_every), 0)
        q = self._opts(precision, max_depth, False, None, None)
        _check(lib().sand_sphere_trace(self._h, ctypes.c_void_p(o.data_ptr()), int(per_ray),
                                       ctypes.c_void_p(d.data_ptr()), n, ctypes.byref(to), ctypes.byref(q),
                                       ctypes.c_void_p(t.data_ptr()), ctypes.c_void_p(state.data_ptr()),
                                       ctypes.c_void_p(steps.data_ptr()),
                                       ctypes.c_void_p(g.data_ptr() if g is not None else 0), _stream_handle(stream)))
        return t, state, steps, g

    def query_dynamic(self, points: torch.Tensor, r: float = 1.5e-4, precision: str = "fp32",
                      stream: Optional[torch.cuda.Stream] = None):
        """Octree-free dynamic exit (Table 6): (y, exit layer uint8) per point, stopping at the first
        layer whose tail |t_i| < r."""
        pts = _as_points(points, self.device)
        n = pts.shape[0]
        out = torch.empty(n, dtype=torch.float32, device=pts.device)
        el = torch.empty(n, dtype=torch.uint8, device=pts.device)
        o = self._opts(precision, 0, False, None, None)
        _check(lib().sand_query_sdf_dynamic(self._h, ctypes.c_void_p(pts.data_ptr()), n, float(r),
                                            ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(el.data_ptr()),
                                            ctypes.byref(o), _stream_handle(stream)))
        return out, el

    def build_depth_map(self, max_level: int, child: np.ndarray, near: np.ndarray, samples_per_axis: int = 4,
                        r: float = 1.5e-4, far_sign: bool = False, precision: str = "fp32",
                        stream: Optional[torch.cuda.Stream] = None) -> np.ndarray:
        """Depths of the octree's leaves from this network (Eq. 5-6), uint8 per node; far leaves 0
        unless far_sign.  `near` flags the leaves whose cells meet the shape."""
        if precision not in PRECISION:
            raise ValueError("precision must be one of %s" % sorted(PRECISION))
        c = np.ascontiguousarray(child, np.int32)
        nr = np.ascontiguousarray(near, np.uint8)
        if c.size != nr.size:
            raise ValueError("child and near must have one entry per node")
        out = np.zeros(c.size, np.uint8)
        desc = DepthMapDesc(int(max_level), int(self.desc.n_layers), c.size)
        o = MapBuildOpts(int(samples_per_axis), float(r), int(bool(far_sign)), PRECISION[precision])
        _check(lib().sand_build_depth_map(self._h, ctypes.byref(desc), c.ctypes.data_as(ctypes.c_void_p),
                                          nr.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o),
                                          out.ctypes.data_as(ctypes.c_void_p), _stream_handle(stream)))
        return out

    def stats(self, workspace: Optional[torch.Tensor] = None, stream: Optional[torch.cuda.Stream] = None) -> dict:
        """Flags and per-exit-layer counts left by the last query on `workspace` (synchronises the stream)."""
        st = QueryStats()
        ws = workspace if workspace is not None else self._ws
        ptr = None
        if ws is not None:
            ptr = ws.data_ptr() + ((-ws.data_ptr()) % 256)
        _check(lib().sand_read_stats(self._h, ctypes.c_void_p(ptr) if ptr else None, ctypes.byref(st),
                                     _stream_handle(stream)))
        return {"flags": int(st.flags), "n_network": int(st.n_network), "count": [int(c) for c in st.count]}

    def free(self) -> None:
        if self._h:
            _check(lib().sand_free(self._h))
            self._h = None

    def __del__(self):
        try:
            if getattr(self, "_h", None) and _lib is not None:
                _lib.sand_free(self._h)
                self._h = None
        except Exception:
            pass


class SandSDF(torch.autograd.Function):
    """y = SAND SDF of points; backward multiplies the upstream gradient by dy/dx
    from libsand's gradient kernel (forward-mode tangents in the same pass)."""

    @staticmethod
    def forward(ctx, points: torch.Tensor, model: Model, precision: str = "fp32", max_depth: int = 0):
        if points.requires_grad:
            y, g = model.query_grad(points.detach(), precision=precision, max_depth=max_depth,
                                    workspace=model.workspace(points.shape[0], True))
            ctx.save_for_backward(g)
        else:
            y = model.query(points, precision=precision, max_depth=max_depth)
            ctx.save_for_backward(None)
        return y

    @staticmethod
    def backward(ctx, grad_out):
        (g,) = ctx.saved_tensors
        return grad_out[:, None] * g, None, None, None


class Server:
    """Continuous-batching server over resident models (sand_server_* in include/sand.h).

    submit() takes host points (numpy float32 [n, 3] or a CPU tensor; pinned memory lets
    the copies overlap) and returns a ticket; wait() returns (sdf, latency_ms).
    """

    def __init__(self, models, precision="fp32", n_streams: int = 3, mem_budget: int = 1 << 30,
                 max_batch_points: int = 1 << 22):
        """precision: one name for every model, or a list with one name per model."""
        self.models = list(models)
        precs = [precision] * len(self.models) if isinstance(precision, str) else list(precision)
        if len(precs) != len(self.models) or any(p not in PRECISION for p in precs):
            raise ValueError("precision must be one of %s (or one per model)" % sorted(PRECISION))
        arr = (ctypes.c_void_p * len(self.models))(*[m._h for m in self.models])
        per = (ctypes.c_int32 * len(self.models))(*[PRECISION[p] for p in precs])
        o = ServerOpts(int(n_streams), PRECISION[precs[0]], int(mem_budget), int(max_batch_points),
                       ctypes.cast(per, ctypes.c_void_p))
        h = ctypes.c_void_p()
        _check(lib().sand_server_create(arr, len(self.models), ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        self._live = {}

    def submit(self, model: int, points, out=None) -> int:
        if isinstance(points, torch.Tensor):
            if points.device.type != "cpu" or points.dtype != torch.float32:
                raise ValueError("host points must be a float32 CPU tensor")
            pts = points.contiguous()
            n = pts.shape[0]
            out = out if out is not None else torch.empty(n, dtype=torch.float32, pin_memory=pts.is_pinned())
            pp, op = pts.data_ptr(), out.data_ptr()
        else:
            pts = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
            n = pts.shape[0]
            out = out if out is not None else np.empty(n, np.float32)
            pp, op = pts.ctypes.data, out.ctypes.data
        t = ctypes.c_uint64()
        _check(lib().sand_server_submit(self._h, int(model), ctypes.c_void_p(pp), n, ctypes.c_void_p(op), ctypes.byref(t)))
        self._live[t.value] = (pts, out)
        return t.value

    def wait(self, ticket: int, timeout: float = 120.0):
        lat = ctypes.c_double()
        st = lib().sand_server_wait(self._h, ctypes.c_uint64(ticket), float(timeout), ctypes.byref(lat))
        _, out = self._live.pop(ticket, (None, None))
        _check(st)
        return out, lat.value

    def stats(self) -> dict:
        r = ServerReport()
        _check(lib().sand_server_stats(self._h, ctypes.byref(r)))
        return {k: getattr(r, k) for k, _ in ServerReport._fields_}

    def close(self):
        if self._h:
            lib().sand_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Trainer:
    """T-MLP training (Sec. 3.3): the loss over every tail (Eq. 4 / Eq. 8) and Adam, on a model's
    float32 master copy (sand_trainer_*).  step() takes device points [n, 3] and targets [n]."""

    def __init__(self, model: Model, max_points: int = 1 << 17, lr: float = 1e-4, beta1: float = 0.9,
                 beta2: float = 0.999, eps: float = 1e-8):
        self.model = model
        o = TrainOpts(int(max_points), float(lr), float(beta1), float(beta2), float(eps), 0)
        h = ctypes.c_void_p()
        _check(lib().sand_trainer_create(model._h, ctypes.byref(o), ctypes.byref(h)))
        self._h = h
        d = model.desc
        L, W, D = d.n_layers, d.width, d.in_dim
        self.n_params = W * D + W + (L - 1) * W * W + (L - 1) * W + L * 2 * W + L * 2

    def step(self, points: torch.Tensor, targets: torch.Tensor, update: bool = True, loss: Optional[torch.Tensor] = None,
             grad: Optional[torch.Tensor] = None, stream: Optional[torch.cuda.Stream] = None):
        """One training step; returns (loss [1], grad [n_params] or None) as device tensors."""
        pts = _as_points(points, self.model.device)
        t = targets.contiguous()
        if t.dtype != torch.float32 or t.numel() != pts.shape[0] or t.device != pts.device:
            raise ValueError("targets: float32 [n] on the points' device")
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=pts.device)
        gp = grad.data_ptr() if grad is not None else None
        _check(lib().sand_train_step(self._h, ctypes.c_void_p(pts.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                     pts.shape[0], ctypes.c_void_p(loss.data_ptr()), ctypes.c_void_p(gp) if gp else None,
                                     int(bool(update)), _stream_handle(stream)))
        return loss, grad

    def params(self) -> np.ndarray:
        out = np.empty(self.n_params, np.float32)
        _check(lib().sand_trainer_params(self._h, out.ctypes.data_as(ctypes.c_void_p), out.size))
        return out

    def commit(self) -> None:
        _check(lib().sand_trainer_commit(self._h))

    def status(self, stream: Optional[torch.cuda.Stream] = None) -> None:
        _check(lib().sand_trainer_status(self._h, _stream_handle(stream)))

    def close(self) -> None:
        if self._h:
            lib().sand_trainer_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
