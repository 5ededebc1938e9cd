"""Thin ctypes binding of the C ABI in ``include/fcofdm.h``.

Argument marshalling only: every step of FC synthesis/analysis runs in the CUDA
library ``_build/libfcofdm.so``. There is no CPU fallback; if the library has
not been built the first call raises ``RuntimeError``.

The functions keep the C names (``fc_plan_create``, ``fc_query``,
``fc_tx_synthesize``, ``fc_rx_analyze``, ``fc_plan_destroy``,
``fc_status_string``). ``Plan`` is a small owner object around them that takes
torch device tensors (complex64, or with ``FC_FLAG_IO_BF16`` bfloat16 tensors holding
interleaved (re, im) pairs, e.g. of shape [streams, length, 2]) and the current torch
CUDA stream.
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfcofdm.so")

FC_OK, FC_ERR_INVALID, FC_ERR_UNSUPPORTED, FC_ERR_NOMEM, FC_ERR_CUDA, FC_ERR_TIMEOUT = range(6)
FC_CONTINUOUS, FC_SYMBOL_SYNC = 0, 1
FC_FLAG_GENERIC_KERNELS = 1
FC_FLAG_REDUCED_RX = 2
FC_FLAG_TENSOR_DFT = 4
FC_FLAG_IO_TIME = 8
FC_FLAG_IO_BF16 = 16
FC_OLA, FC_OLS = 0, 1
FC_TX, FC_RX = 0, 1

EXPORTED = ("fc_plan_create", "fc_geometry_check", "fc_query", "fc_tx_synthesize", "fc_rx_analyze", "fc_plan_destroy",
            "fc_status_string", "fc_last_error", "fc_tx_synthesize_static", "fc_state_create", "fc_state_reset",
            "fc_state_destroy", "fc_tx_synthesize_stream", "fc_rx_analyze_stream", "fc_plan_autotune",
            "fc_plan_choice", "fc_batch_create", "fc_batch_launch", "fc_batch_destroy", "fc_server_create",
            "fc_server_add_carrier", "fc_server_carrier_sizes", "fc_server_run", "fc_server_destroy",
            "fc_server_serve", "fc_server_set_limits", "fc_plan_set_first_wait_limit", "fc_batch_autotune",
            "fc_plan_radices",
            "fc_plan_device_status", "fc_plan_set_choice", "fc_pipeline_create", "fc_pipeline_destroy",
            "fc_tx_synthesize_host", "fc_rx_analyze_host")


class FcGroup(ctypes.Structure):
    _fields_ = [("n_long", ctypes.c_int32), ("n_overlap", ctypes.c_int32), ("lead_pad", ctypes.c_int32),
                ("n_symbols", ctypes.c_int32), ("n_cp", ctypes.POINTER(ctypes.c_int32))]


class FcSubband(ctypes.Structure):
    _fields_ = [("l_short", ctypes.c_int32), ("l_ofdm", ctypes.c_int32), ("n_active", ctypes.c_int32),
                ("centre_bin", ctypes.c_int32), ("group", ctypes.c_int32),
                ("weights", ctypes.POINTER(ctypes.c_double))]


class FcGeometry(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("scheme_tx", ctypes.c_int32), ("scheme_rx", ctypes.c_int32),
                ("n_groups", ctypes.c_int32), ("groups", ctypes.POINTER(FcGroup)),
                ("n_subbands", ctypes.c_int32), ("subbands", ctypes.POINTER(FcSubband)),
                ("flags", ctypes.c_int32)]


class FcSizes(ctypes.Structure):
    _fields_ = [("grid_len", ctypes.c_int64), ("wave_len", ctypes.c_int64), ("nominal_len", ctypes.c_int64),
                ("workspace_per_stream", ctypes.c_int64), ("tx_kernels", ctypes.c_int32),
                ("rx_kernels", ctypes.c_int32), ("slot_len", ctypes.c_int64), ("stream_delay", ctypes.c_int64),
                ("time_tx_len", ctypes.c_int64), ("time_rx_len", ctypes.c_int64), ("tx_in_len", ctypes.c_int64),
                ("rx_out_len", ctypes.c_int64), ("sample_bytes", ctypes.c_int64)]


class FcBatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("state", ctypes.c_void_p), ("direction", ctypes.c_int32),
                ("n_streams", ctypes.c_int32), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t)]


class FcServeRequest(ctypes.Structure):
    _fields_ = [("arrival_s", ctypes.c_double), ("carrier", ctypes.c_int32), ("direction", ctypes.c_int32),
                ("host_in", ctypes.c_void_p), ("host_out", ctypes.c_void_p)]


class FcServeRecord(ctypes.Structure):
    _fields_ = [("latency_s", ctypes.c_double), ("wait_s", ctypes.c_double), ("batch", ctypes.c_int32),
                ("batched", ctypes.c_int32), ("device_start_ms", ctypes.c_float), ("device_end_ms", ctypes.c_float)]


_lib = None
_lock = threading.Lock()


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libfcofdm.so (raises RuntimeError when it is missing)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"FC CUDA library not built: {path} is missing "
                               "(run `python -m paper_2008_00672_gb300.build`)")
        lib = ctypes.CDLL(path)
        vp, i32, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_size_t
        lib.fc_plan_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(FcGeometry), i32]
        lib.fc_plan_create.restype = ctypes.c_int
        lib.fc_geometry_check.argtypes = [ctypes.POINTER(FcGeometry), ctypes.POINTER(FcSizes)]
        lib.fc_geometry_check.restype = ctypes.c_int
        lib.fc_query.argtypes = [vp, ctypes.POINTER(FcSizes)]
        lib.fc_query.restype = ctypes.c_int
        lib.fc_tx_synthesize.argtypes = [vp, i32, vp, vp, vp, sz, vp]
        lib.fc_tx_synthesize.restype = ctypes.c_int
        lib.fc_rx_analyze.argtypes = [vp, i32, vp, vp, vp, sz, vp]
        lib.fc_rx_analyze.restype = ctypes.c_int
        lib.fc_tx_synthesize_static.argtypes = [vp, i32, vp, vp, vp]
        lib.fc_tx_synthesize_static.restype = ctypes.c_int
        lib.fc_state_create.argtypes = [vp, i32, ctypes.POINTER(vp)]
        lib.fc_state_create.restype = ctypes.c_int
        lib.fc_state_reset.argtypes = [vp, vp]
        lib.fc_state_reset.restype = ctypes.c_int
        lib.fc_state_destroy.argtypes = [vp]
        lib.fc_state_destroy.restype = None
        lib.fc_state_bytes.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64)]
        lib.fc_state_bytes.restype = ctypes.c_int
        lib.fc_state_export.argtypes = [vp, vp, ctypes.c_uint64, vp]
        lib.fc_state_export.restype = ctypes.c_int
        lib.fc_state_import.argtypes = [vp, vp, ctypes.c_uint64, vp]
        lib.fc_state_import.restype = ctypes.c_int
        lib.fc_tx_synthesize_stream.argtypes = [vp, vp, vp, vp, vp, sz, vp]
        lib.fc_tx_synthesize_stream.restype = ctypes.c_int
        lib.fc_rx_analyze_stream.argtypes = [vp, vp, vp, vp, vp, sz, vp]
        lib.fc_rx_analyze_stream.restype = ctypes.c_int
        lib.fc_plan_autotune.argtypes = [vp, i32, i32, vp]
        lib.fc_plan_autotune.restype = ctypes.c_int
        lib.fc_plan_set_choice.argtypes = [vp, i32, i32, i32, i32]
        lib.fc_plan_set_choice.restype = ctypes.c_int
        lib.fc_plan_choice.argtypes = [vp, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.fc_plan_choice.restype = ctypes.c_int
        lib.fc_batch_create.argtypes = [ctypes.POINTER(FcBatchItem), i32, i32, i32, ctypes.POINTER(vp)]
        lib.fc_batch_create.restype = ctypes.c_int
        lib.fc_batch_launch.argtypes = [vp, vp]
        lib.fc_batch_launch.restype = ctypes.c_int
        lib.fc_batch_destroy.argtypes = [vp]
        lib.fc_batch_destroy.restype = None
        lib.fc_server_create.argtypes = [i32, i32, ctypes.c_uint64, ctypes.POINTER(vp)]
        lib.fc_server_create.restype = ctypes.c_int
        lib.fc_server_add_carrier.argtypes = [vp, ctypes.POINTER(FcGeometry), ctypes.POINTER(i32)]
        lib.fc_server_add_carrier.restype = ctypes.c_int
        lib.fc_server_carrier_sizes.argtypes = [vp, i32, ctypes.POINTER(FcSizes)]
        lib.fc_server_carrier_sizes.restype = ctypes.c_int
        lib.fc_server_run.argtypes = [vp, ctypes.POINTER(FcServeRequest), i32, ctypes.POINTER(ctypes.c_double)]
        lib.fc_server_run.restype = ctypes.c_int
        lib.fc_plan_radices.argtypes = [vp, i32, ctypes.POINTER(i32), ctypes.POINTER(i32)]
        lib.fc_plan_radices.restype = ctypes.c_int
        lib.fc_batch_autotune.argtypes = [vp, i32, vp]
        lib.fc_batch_autotune.restype = ctypes.c_int
        lib.fc_plan_set_first_wait_limit.argtypes = [vp, ctypes.c_uint32]
        lib.fc_plan_set_first_wait_limit.restype = ctypes.c_int
        lib.fc_server_serve.argtypes = [vp, ctypes.POINTER(FcServeRequest), i32, ctypes.POINTER(FcServeRecord)]
        lib.fc_server_serve.restype = ctypes.c_int
        lib.fc_server_set_limits.argtypes = [vp, ctypes.c_uint64, i32, i32]
        lib.fc_server_set_limits.restype = ctypes.c_int
        lib.fc_server_destroy.argtypes = [vp]
        lib.fc_server_destroy.restype = None
        lib.fc_plan_device_status.argtypes = [vp]
        lib.fc_plan_device_status.restype = ctypes.c_int
        lib.fc_pipeline_create.argtypes = [vp, i32, i32, ctypes.POINTER(vp)]
        lib.fc_pipeline_create.restype = ctypes.c_int
        lib.fc_pipeline_destroy.argtypes = [vp]
        lib.fc_pipeline_destroy.restype = None
        lib.fc_tx_synthesize_host.argtypes = [vp, i32, vp, vp, vp]
        lib.fc_tx_synthesize_host.restype = ctypes.c_int
        lib.fc_rx_analyze_host.argtypes = [vp, i32, vp, vp, vp]
        lib.fc_rx_analyze_host.restype = ctypes.c_int
        lib.fc_plan_destroy.argtypes = [vp]
        lib.fc_plan_destroy.restype = None
        lib.fc_status_string.argtypes = [ctypes.c_int]
        lib.fc_status_string.restype = ctypes.c_char_p
        lib.fc_last_error.argtypes = []
        lib.fc_last_error.restype = ctypes.c_char_p
        _lib = lib
        return lib


class FcError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load_library()
        super().__init__(f"{where}: {lib.fc_status_string(status).decode()} ({lib.fc_last_error().decode()})")
        self.status = status


def _check(status: int, where: str):
    if status != FC_OK:
        raise FcError(status, where)


def _marshal_geometry(geom):
    """Build the C structs from any object with the Geometry attributes; keeps the
    backing arrays alive in the returned tuple."""
    keep = []
    groups = (FcGroup * len(geom.groups))()
    for i, g in enumerate(geom.groups):
        cps = (ctypes.c_int32 * len(g.n_cp))(*[int(v) for v in g.n_cp])
        keep.append(cps)
        groups[i] = FcGroup(int(g.n_long), int(g.n_overlap), int(getattr(g, "lead_pad", -1)), len(g.n_cp), cps)
    subs = (FcSubband * len(geom.subbands))()
    for i, s in enumerate(geom.subbands):
        w = (ctypes.c_double * int(s.l_short))(*[float(v) for v in s.weights])
        keep.append(w)
        subs[i] = FcSubband(int(s.l_short), int(s.l_ofdm), int(s.n_active), int(s.centre_bin), int(s.group), w)
    geo = FcGeometry(int(geom.mode), int(geom.scheme_tx), int(geom.scheme_rx), len(geom.groups), groups,
                     len(geom.subbands), subs, int(getattr(geom, "flags", 0)))
    return geo, (groups, subs, keep)


# --------------------------------------------------------------------------
# C-named functions
# --------------------------------------------------------------------------

def fc_plan_create(geom, device: int = 0) -> ctypes.c_void_p:
    lib = load_library()
    geo, _keep = _marshal_geometry(geom)
    h = ctypes.c_void_p()
    _check(lib.fc_plan_create(ctypes.byref(h), ctypes.byref(geo), int(device)), "fc_plan_create")
    return h


def fc_geometry_check(geom) -> FcSizes:
    """Host-only validation of a geometry; returns the per-stream sizes."""
    lib = load_library()
    geo, _keep = _marshal_geometry(geom)
    out = FcSizes()
    _check(lib.fc_geometry_check(ctypes.byref(geo), ctypes.byref(out)), "fc_geometry_check")
    return out


def fc_query(plan) -> FcSizes:
    out = FcSizes()
    _check(load_library().fc_query(plan, ctypes.byref(out)), "fc_query")
    return out


def fc_tx_synthesize(plan, n_streams: int, grid_in: int, wave_out: int, workspace: int = 0,
                     workspace_bytes: int = 0, stream: int = 0):
    _check(load_library().fc_tx_synthesize(plan, int(n_streams), grid_in, wave_out, workspace or None,
                                           int(workspace_bytes), stream or None), "fc_tx_synthesize")


def fc_rx_analyze(plan, n_streams: int, wave_in: int, grid_out: int, workspace: int = 0,
                  workspace_bytes: int = 0, stream: int = 0):
    _check(load_library().fc_rx_analyze(plan, int(n_streams), wave_in, grid_out, workspace or None,
                                        int(workspace_bytes), stream or None), "fc_rx_analyze")


def fc_tx_synthesize_static(plan, n_streams: int, grid_in: int, wave_out: int, stream: int = 0):
    """TX with the library's built-in device workspace instead of a caller buffer
    (for callers that cannot allocate device memory at run time)."""
    _check(load_library().fc_tx_synthesize_static(plan, int(n_streams), grid_in, wave_out, stream or None),
           "fc_tx_synthesize_static")


def fc_state_create(plan, n_streams: int) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().fc_state_create(plan, int(n_streams), ctypes.byref(h)), "fc_state_create")
    return h


def fc_state_reset(state, stream: int = 0):
    _check(load_library().fc_state_reset(state, stream or None), "fc_state_reset")


def fc_state_destroy(state):
    if state:
        load_library().fc_state_destroy(state)


def fc_state_bytes(state) -> int:
    n = ctypes.c_uint64()
    _check(load_library().fc_state_bytes(state, ctypes.byref(n)), "fc_state_bytes")
    return n.value


def fc_state_export(state, host: int, nbytes: int, stream: int = 0):
    _check(load_library().fc_state_export(state, host or None, int(nbytes), stream or None), "fc_state_export")


def fc_state_import(state, host: int, nbytes: int, stream: int = 0):
    _check(load_library().fc_state_import(state, host or None, int(nbytes), stream or None), "fc_state_import")


def fc_tx_synthesize_stream(plan, state, grid_in: int, slot_out: int, workspace: int = 0, workspace_bytes: int = 0,
                            stream: int = 0):
    _check(load_library().fc_tx_synthesize_stream(plan, state, grid_in, slot_out, workspace or None,
                                                  int(workspace_bytes), stream or None), "fc_tx_synthesize_stream")


def fc_rx_analyze_stream(plan, state, slot_in: int, grid_out: int, workspace: int = 0, workspace_bytes: int = 0,
                         stream: int = 0):
    _check(load_library().fc_rx_analyze_stream(plan, state, slot_in, grid_out, workspace or None,
                                               int(workspace_bytes), stream or None), "fc_rx_analyze_stream")


def fc_plan_autotune(plan, n_streams: int, reps: int = 5, stream: int = 0):
    _check(load_library().fc_plan_autotune(plan, int(n_streams), int(reps), stream or None), "fc_plan_autotune")


def fc_plan_set_choice(plan, n_streams: int, direction: int, chunks_per_stream: int, generic_kernels: int = 0):
    _check(load_library().fc_plan_set_choice(plan, int(n_streams), int(direction), int(chunks_per_stream),
                                             int(generic_kernels)), "fc_plan_set_choice")


def fc_plan_choice(plan, n_streams: int, direction: int):
    """(chunks per stream, generic kernels) an execute call with n_streams will use."""
    k, g = ctypes.c_int32(), ctypes.c_int32()
    _check(load_library().fc_plan_choice(plan, int(n_streams), int(direction), ctypes.byref(k), ctypes.byref(g)),
           "fc_plan_choice")
    return int(k.value), int(g.value)


FC_BATCH_GRAPH, FC_BATCH_PERSISTENT = 1, 2


def fc_batch_create(items, n_lanes: int = 8, use_graph: bool = True, persistent: bool = False) -> ctypes.c_void_p:
    arr = (FcBatchItem * len(items))(*items)
    h = ctypes.c_void_p()
    mode = (FC_BATCH_GRAPH if use_graph else 0) | (FC_BATCH_PERSISTENT if persistent else 0)
    _check(load_library().fc_batch_create(arr, len(items), int(n_lanes), mode, ctypes.byref(h)), "fc_batch_create")
    return h


def fc_batch_launch(batch, stream: int = 0):
    _check(load_library().fc_batch_launch(batch, stream or None), "fc_batch_launch")


def fc_batch_destroy(batch):
    if batch:
        load_library().fc_batch_destroy(batch)


def fc_server_create(device: int = 0, n_lanes: int = 8, hbm_reserve_bytes: int = 0) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().fc_server_create(int(device), int(n_lanes), int(hbm_reserve_bytes), ctypes.byref(h)),
           "fc_server_create")
    return h


def fc_server_add_carrier(server, geom) -> int:
    geo, _keep = _marshal_geometry(geom)
    cid = ctypes.c_int32(-1)
    _check(load_library().fc_server_add_carrier(server, ctypes.byref(geo), ctypes.byref(cid)), "fc_server_add_carrier")
    return int(cid.value)


def fc_server_carrier_sizes(server, carrier: int) -> FcSizes:
    out = FcSizes()
    _check(load_library().fc_server_carrier_sizes(server, int(carrier), ctypes.byref(out)), "fc_server_carrier_sizes")
    return out


def fc_server_run(server, requests) -> list:
    """requests: sequence of FcServeRequest; returns the latencies in seconds."""
    arr = (FcServeRequest * len(requests))(*requests)
    lat = (ctypes.c_double * len(requests))()
    _check(load_library().fc_server_run(server, arr, len(requests), lat), "fc_server_run")
    return list(lat)


def fc_server_serve(server, requests) -> list:
    """requests: sequence of FcServeRequest; returns one FcServeRecord per request."""
    arr = (FcServeRequest * len(requests))(*requests)
    rec = (FcServeRecord * len(requests))()
    _check(load_library().fc_server_serve(server, arr, len(requests), rec), "fc_server_serve")
    return list(rec)


def fc_server_set_limits(server, arena_bytes: int, max_batch: int = 64, max_inflight: int = 2):
    _check(load_library().fc_server_set_limits(server, int(arena_bytes), int(max_batch), int(max_inflight)),
           "fc_server_set_limits")


def fc_server_destroy(server):
    if server:
        load_library().fc_server_destroy(server)


def fc_pipeline_create(plan, chunk_streams: int, depth: int = 3) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().fc_pipeline_create(plan, int(chunk_streams), int(depth), ctypes.byref(h)),
           "fc_pipeline_create")
    return h


def fc_pipeline_destroy(pipeline):
    if pipeline:
        load_library().fc_pipeline_destroy(pipeline)


def fc_tx_synthesize_host(pipeline, n_streams: int, host_grid: int, host_wave: int, stream: int = 0):
    _check(load_library().fc_tx_synthesize_host(pipeline, int(n_streams), host_grid, host_wave, stream or None),
           "fc_tx_synthesize_host")


def fc_rx_analyze_host(pipeline, n_streams: int, host_wave: int, host_grid: int, stream: int = 0):
    _check(load_library().fc_rx_analyze_host(pipeline, int(n_streams), host_wave, host_grid, stream or None),
           "fc_rx_analyze_host")


def fc_plan_destroy(plan):
    if plan:
        load_library().fc_plan_destroy(plan)


def fc_status_string(status: int) -> str:
    return load_library().fc_status_string(int(status)).decode()


# --------------------------------------------------------------------------
# torch convenience owner
# --------------------------------------------------------------------------

class Plan:
    """Owns one fc_plan; execute calls take complex64 CUDA tensors, or bfloat16 CUDA
    tensors of (re, im) pairs when the plan was made with FC_FLAG_IO_BF16."""

    def __init__(self, geom, device: int = 0):
        self.device = int(device)
        self.handle = fc_plan_create(geom, self.device)
        s = fc_query(self.handle)
        self.grid_len = int(s.grid_len)
        self.wave_len = int(s.wave_len)
        self.nominal_len = int(s.nominal_len)
        self.workspace_per_stream = int(s.workspace_per_stream)
        self.tx_kernels = int(s.tx_kernels)
        self.rx_kernels = int(s.rx_kernels)
        self.slot_len = int(s.slot_len)
        self.stream_delay = int(s.stream_delay)
        self.tx_in_len = int(s.tx_in_len)       # grid_len, or the time-domain TX input length
        self.rx_out_len = int(s.rx_out_len)     # grid_len, or the time-domain RX output length
        self.sample_bytes = int(s.sample_bytes)
        self.io_bf16 = self.sample_bytes == 4   # complex-BF16 I/O buffers
        self._ws = None

    def close(self):
        if self.handle:
            fc_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, n_streams: int, reps: int = 5, stream=None):
        """Measure every launch shape for n_streams streams and keep the fastest."""
        fc_plan_autotune(self.handle, n_streams, reps, self._stream_handle(stream))

    def set_choice(self, n_streams: int, direction: int, chunks_per_stream: int, generic_kernels: int = 0):
        fc_plan_set_choice(self.handle, n_streams, direction, chunks_per_stream, generic_kernels)

    def radices(self, n: int) -> list:
        """The generic kernels' radix schedule of the plan's n-point transform."""
        r = (ctypes.c_int32 * 8)()
        k = ctypes.c_int32(0)
        _check(load_library().fc_plan_radices(self.handle, int(n), r, ctypes.byref(k)), "fc_plan_radices")
        return [int(r[i]) for i in range(k.value)]

    def choice(self, n_streams: int, direction: int):
        return fc_plan_choice(self.handle, n_streams, direction)

    def workspace(self, n_streams: int):
        """A device workspace large enough for n_streams (allocated by torch, reused)."""
        import torch
        need = self.workspace_per_stream * int(n_streams)
        if need == 0:
            return None
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=f"cuda:{self.device}")
        return self._ws

    @staticmethod
    def _stream_handle(stream):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        return int(stream.cuda_stream)

    def tx_synthesize(self, grid, wave_out, workspace=None, stream=None):
        n = self._streams(grid, self.tx_in_len, wave_out, self.wave_len, self.io_bf16)
        ws = workspace if workspace is not None else self.workspace(n)
        fc_tx_synthesize(self.handle, n, grid.data_ptr(), wave_out.data_ptr(),
                         ws.data_ptr() if ws is not None else 0,
                         ws.numel() * ws.element_size() if ws is not None else 0, self._stream_handle(stream))
        return wave_out

    def rx_analyze(self, wave, grid_out, workspace=None, stream=None):
        n = self._streams(wave, self.wave_len, grid_out, self.rx_out_len, self.io_bf16)
        ws = workspace if workspace is not None else self.workspace(n)
        fc_rx_analyze(self.handle, n, wave.data_ptr(), grid_out.data_ptr(),
                      ws.data_ptr() if ws is not None else 0,
                      ws.numel() * ws.element_size() if ws is not None else 0, self._stream_handle(stream))
        return grid_out

    @staticmethod
    def _samples(t, bf16: bool, cuda: bool) -> int:
        """Complex samples in t (complex64, or bfloat16 (re, im) pairs)."""
        import torch
        want = torch.bfloat16 if bf16 else torch.complex64
        if t.dtype != want or t.is_cuda != cuda or not t.is_contiguous():
            raise ValueError(f"expected contiguous {'bfloat16 (re, im)' if bf16 else 'complex64'} "
                             f"{'CUDA' if cuda else 'host'} tensors")
        n = t.numel()
        if bf16 and n % 2:
            raise ValueError("a bfloat16 tensor of complex samples has an even number of elements")
        return n // 2 if bf16 else n

    @staticmethod
    def _streams(a, la, b, lb, bf16: bool = False, cuda: bool = True) -> int:
        na, nb = Plan._samples(a, bf16, cuda), Plan._samples(b, bf16, cuda)
        if na % la or nb % lb or na // la != nb // lb:
            raise ValueError("input and output sizes do not match the plan")
        return na // la


class State:
    """Owns one fc_state: per-stream TX tail and RX look-behind for stream calls
    (consecutive slots whose concatenated results equal one frame of the repeated
    geometry)."""

    def __init__(self, plan: Plan, n_streams: int):
        self.plan = plan
        self.n_streams = int(n_streams)
        self.handle = fc_state_create(plan.handle, self.n_streams)

    def close(self):
        if self.handle:
            fc_state_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, stream=None):
        fc_state_reset(self.handle, Plan._stream_handle(stream))

    def export(self, stream=None):
        """Checkpoint: the TX tails and RX look-behinds as host bytes (numpy uint8), after
        the work queued on `stream` has finished."""
        import numpy as np
        buf = np.zeros(fc_state_bytes(self.handle), dtype=np.uint8)
        fc_state_export(self.handle, buf.ctypes.data if buf.size else 0, buf.size, Plan._stream_handle(stream))
        return buf

    def load(self, checkpoint, stream=None):
        """Resume from a checkpoint that export() of a state of the same plan sizes and
        stream count returned."""
        import numpy as np
        buf = np.ascontiguousarray(checkpoint, dtype=np.uint8)
        fc_state_import(self.handle, buf.ctypes.data if buf.size else 0, buf.size, Plan._stream_handle(stream))

    def tx(self, grid, slot_out, workspace=None, stream=None):
        p = self.plan
        n = Plan._streams(grid, p.tx_in_len, slot_out, p.slot_len, p.io_bf16)
        if n != self.n_streams:
            raise ValueError("the state was created for another number of streams")
        ws = workspace if workspace is not None else p.workspace(n)
        fc_tx_synthesize_stream(p.handle, self.handle, grid.data_ptr(), slot_out.data_ptr(),
                                ws.data_ptr() if ws is not None else 0,
                                ws.numel() * ws.element_size() if ws is not None else 0, Plan._stream_handle(stream))
        return slot_out

    def rx(self, slot_in, grid_out, workspace=None, stream=None):
        p = self.plan
        n = Plan._streams(slot_in, p.slot_len, grid_out, p.rx_out_len, p.io_bf16)
        if n != self.n_streams:
            raise ValueError("the state was created for another number of streams")
        ws = workspace if workspace is not None else p.workspace(n)
        fc_rx_analyze_stream(p.handle, self.handle, slot_in.data_ptr(), grid_out.data_ptr(),
                             ws.data_ptr() if ws is not None else 0,
                             ws.numel() * ws.element_size() if ws is not None else 0, Plan._stream_handle(stream))
        return grid_out


class Batch:
    """Owns one fc_batch over (plan, direction, input tensor, output tensor[, state])
    items; launch() runs them all (forked over lanes, replayed as a CUDA graph)."""

    def __init__(self, items, n_lanes: int = 8, use_graph: bool = True, persistent: bool = False):
        self._keep = []
        c_items = []
        for it in items:
            plan, direction, src, dst = it[:4]
            state = it[4] if len(it) > 4 else None
            if state is not None:
                ls, ld = (plan.tx_in_len, plan.slot_len) if direction == FC_TX else (plan.slot_len, plan.rx_out_len)
            else:
                ls, ld = (plan.tx_in_len, plan.wave_len) if direction == FC_TX else (plan.wave_len, plan.rx_out_len)
            n = Plan._streams(src, ls, dst, ld, plan.io_bf16)
            self._keep.append((plan, src, dst, state))
            c_items.append(FcBatchItem(plan.handle.value, state.handle.value if state is not None else None,
                                       int(direction), n, src.data_ptr(), dst.data_ptr(), None, 0))
        self.handle = fc_batch_create(c_items, n_lanes, use_graph, persistent)

    def launch(self, stream=None):
        fc_batch_launch(self.handle, Plan._stream_handle(stream))

    def autotune(self, reps: int = 5, stream=None):
        """Time the whole batch under each candidate launch shape; keep the fastest."""
        _check(load_library().fc_batch_autotune(self.handle, int(reps), Plan._stream_handle(stream)),
               "fc_batch_autotune")

    def close(self):
        if self.handle:
            fc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Owns one fc_server. add_carrier(geom) -> id; run(requests) / serve(requests)
    replay (arrival_s, carrier, direction, host_in, host_out) requests in real time with
    page-locked CPU tensors (continuous batching) and return the latencies (seconds) /
    the per-request records."""

    def __init__(self, device: int = 0, n_lanes: int = 8, hbm_reserve_bytes: int = 0):
        self.handle = fc_server_create(device, n_lanes, hbm_reserve_bytes)
        self.sizes = []

    def add_carrier(self, geom) -> int:
        cid = fc_server_add_carrier(self.handle, geom)
        self.sizes.append(fc_server_carrier_sizes(self.handle, cid))
        return cid

    def set_limits(self, arena_bytes: int, max_batch: int = 64, max_inflight: int = 2):
        fc_server_set_limits(self.handle, arena_bytes, max_batch, max_inflight)

    def run(self, requests):
        """Latencies (seconds) of the requests."""
        return [r.latency_s for r in self.serve(requests)]

    def serve(self, requests):
        """One FcServeRecord per request: latency, wait, batch, whether it ran in the
        batch's persistent launch, the batch's device compute interval."""
        reqs = []
        for t, cid, direction, h_in, h_out in requests:
            z = self.sizes[cid]
            n_in, n_out = (z.tx_in_len, z.slot_len) if direction == FC_TX else (z.slot_len, z.rx_out_len)
            for x, n in ((h_in, n_in), (h_out, n_out)):
                if Plan._samples(x, z.sample_bytes == 4, cuda=False) != n:
                    raise ValueError("expected host tensors of the carrier's sizes")
            reqs.append(FcServeRequest(float(t), int(cid), int(direction), h_in.data_ptr(), h_out.data_ptr()))
        return fc_server_serve(self.handle, reqs)

    def close(self):
        if self.handle:
            fc_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pipeline:
    """Owns one fc_pipeline: host-buffer TX / RX with copies and kernels of chunks of
    streams overlapped. tx(grid, wave) / rx(wave, grid) take contiguous CPU tensors of
    the plan's sample type (complex64, or bfloat16 (re, im) pairs; page-locked for
    overlap) and are asynchronous on `stream`."""

    def __init__(self, plan: Plan, chunk_streams: int, depth: int = 3):
        self.plan = plan
        self.handle = fc_pipeline_create(plan.handle, chunk_streams, depth)

    def _host(self, a, b, la, lb) -> int:
        return Plan._streams(a, la, b, lb, self.plan.io_bf16, cuda=False)

    def tx(self, host_grid, host_wave, stream=None):
        n = self._host(host_grid, host_wave, self.plan.tx_in_len, self.plan.wave_len)
        fc_tx_synthesize_host(self.handle, n, host_grid.data_ptr(), host_wave.data_ptr(), Plan._stream_handle(stream))
        return host_wave

    def rx(self, host_wave, host_grid, stream=None):
        n = self._host(host_wave, host_grid, self.plan.wave_len, self.plan.rx_out_len)
        fc_rx_analyze_host(self.handle, n, host_wave.data_ptr(), host_grid.data_ptr(), Plan._stream_handle(stream))
        return host_grid

    def close(self):
        if self.handle:
            fc_pipeline_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
