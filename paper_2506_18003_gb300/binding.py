"""Thin Python binding of libscd.so (include/scd.h): ctypes declarations plus torch-tensor
marshalling under the same names as the C entry points.

Argument marshalling only: every step of every estimator runs in the library's CUDA
kernels.  There is no CPU fallback; if the library is missing or cannot be loaded the
call raises.  PyTorch supplies device memory and the current stream.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libscd.so")

SCD_OK, SCD_ERR_ARG, SCD_ERR_UNSUPPORTED, SCD_ERR_CUDA, SCD_ERR_WORKSPACE, SCD_ERR_TIMEOUT, SCD_ERR_INTERNAL = range(7)
SCD_FP32, SCD_SPLIT_BF16 = 0, 1
PRECISIONS = {"fp32": SCD_FP32, "split": SCD_SPLIT_BF16, "split_bf16": SCD_SPLIT_BF16}


class ScdOpts(ctypes.Structure):
    _fields_ = [
        ("stream", ctypes.c_void_p),
        ("precision", ctypes.c_int32),
        ("map_power", ctypes.c_int32),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
        ("stage_events", ctypes.POINTER(ctypes.c_void_p)),
        ("n_stage_events", ctypes.c_int32),
        ("schedule", ctypes.c_int32),
        ("y", ctypes.c_void_p),
        ("conjugate", ctypes.c_int32),
        ("normalise", ctypes.c_int32),
    ]


_vp, _i32, _i64, _sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
_opts_p = ctypes.POINTER(ScdOpts)

# name -> (restype, argtypes); every function include/scd.h declares
SIGNATURES = {
    "scd_fam": (_i32, [_vp, _i64, _i32, _i32, _i32, _vp, _vp, _opts_p]),
    "scd_fam_workspace_bytes": (_sz, [_i64, _i32, _i32, _i32, _i32]),
    "scd_ssca": (_i32, [_vp, _i64, _i32, _vp, _vp, _opts_p]),
    "scd_ssca_workspace_bytes": (_sz, [_i64, _i32, _i32]),
    "scd_fam_map": (_i32, [_vp, _i32, _i32, _i32, _vp, _opts_p]),
    "scd_ssca_map": (_i32, [_vp, _i64, _i32, _vp, _opts_p]),
    "scd_fam_alpha_profile": (_i32, [_vp, _i32, _i32, _i32, _vp, _opts_p]),
    "scd_ssca_alpha_profile": (_i32, [_vp, _i64, _i32, _vp, _opts_p]),
    "scd_fam_host": (_i32, [_vp, _i64, _i32, _i32, _i32, _vp, _vp, _opts_p]),
    "scd_fam_host_workspace_bytes": (_sz, [_i64, _i32, _i32, _i32, _i32]),
    "scd_ssca_host": (_i32, [_vp, _i64, _i32, _vp, _vp, _opts_p]),
    "scd_ssca_host_workspace_bytes": (_sz, [_i64, _i32, _i32]),
    "scd_fam_noalloc": (_i32, [_vp, _i64, _i32, _i32, _i32, _vp, _vp, _opts_p]),
    "scd_batch_plan_create": (_i32, [_i32, _i32, ctypes.POINTER(ctypes.c_int64), _i32, _i32, _i32,
                                     ctypes.POINTER(ctypes.c_void_p)]),
    "scd_batch_query": (_i32, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                               ctypes.POINTER(ctypes.c_size_t)]),
    "scd_batch_run": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "scd_batch_plan_destroy": (None, [_vp]),
    "scd_batch_run_host": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "scd_batch_host_wait": (_i32, [_vp]),
    "scd_host_alloc": (_i32, [_sz, ctypes.POINTER(_vp)]),
    "scd_host_free": (_i32, [_vp]),
    "scd_batch_plan_set_output": (_i32, [_vp, _i32]),
    "scd_batch_plan_set_schedule": (_i32, [_vp, _i32]),
    "scd_batch_plan_create_exact": (_i32, [_i32, _i32, ctypes.POINTER(ctypes.c_int64), _i32, _i32, _i32,
                                           ctypes.POINTER(_vp)]),
    "scd_batch_tune": (_i32, [_vp, _vp, _vp, _vp, _vp, _vp, _i32]),
    "scd_stream_plan_create": (_i32, [_i32, _i64, _i64, _i32, _i32, _i32, _i32, ctypes.POINTER(ctypes.c_void_p)]),
    "scd_stream_advance": (_i32, [_vp, _vp, _vp, _i32, _vp]),
    "scd_ssca_tune": (_i32, [_vp, _i64, _i32, _vp, _vp, _opts_p, _i32]),
    "scd_events_create": (_i32, [_i32, ctypes.POINTER(ctypes.c_void_p)]),
    "scd_events_destroy": (_i32, [_i32, ctypes.POINTER(ctypes.c_void_p)]),
    "scd_event_elapsed_ms": (_i32, [_vp, _vp, ctypes.POINTER(ctypes.c_float)]),
    "scd_event_record": (_i32, [_vp, _vp]),
    "scd_check_device": (_i32, [_vp]),
    "scd_launch_count": (ctypes.c_uint64, []),
    "scd_prepare": (_i32, [_i32, _i64, _i32, _i32]),
    "scd_chebyshev_window": (_i32, [_i32, ctypes.c_double, _vp, _vp]),
    "scd_release_cache": (None, []),
    "scd_status_string": (ctypes.c_char_p, [_i32]),
    "scd_last_error": (ctypes.c_char_p, []),
    "scd_version": (_i32, []),
}

_lib = None


def load(path: str | None = None):
    """Loads libscd.so (built in-tree by build.py) and declares its signatures."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libscd.so not found at {p}: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if path is None:
        _lib = lib
    return lib


class ScdError(RuntimeError):
    def __init__(self, status: int, where: str):
        lib = load()
        msg = lib.scd_status_string(status).decode()
        if status == SCD_ERR_CUDA:
            msg += f" ({lib.scd_last_error().decode()})"
        super().__init__(f"{where}: {msg}")
        self.status = status


def check(status: int, where: str) -> None:
    if status != SCD_OK:
        raise ScdError(status, where)


# ----------------------------------------------------------------------------- torch layer
def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need(t, dtype, numel, name):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() < numel:
        raise TypeError(f"{name} must be a contiguous {dtype} tensor of at least {numel} elements")


SCHEDULES = {"auto": 0, "stages": 1, "persistent": 2, "fused": 3}


NORMALISE = {None: 0, "none": 0, "power": 1, "peak": 2}


def make_opts(stream=None, precision="fp32", workspace=None, map_power=1, schedule="auto", y=None,
              conjugate=False, normalise=None) -> ScdOpts:
    o = ScdOpts()
    o.normalise = NORMALISE[normalise] if not isinstance(normalise, int) else normalise
    o.stream = _stream(stream)
    o.schedule = SCHEDULES[schedule]
    o.y = None if y is None else y.data_ptr()
    o.conjugate = 1 if conjugate else 0
    o.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    o.map_power = int(map_power)
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel() * workspace.element_size()
    return o


def _workspace(nbytes, device, workspace):
    torch = _torch()
    if workspace is not None:
        return workspace
    return torch.empty(max(1, nbytes), dtype=torch.uint8, device=device)


def _partner(x, y):
    torch = _torch()
    if y is not None:
        _need(y, torch.complex64, x.numel(), "y")
        if y.numel() != x.numel():
            raise TypeError("y must have as many samples as x")
    return y


def scd_fam(x, Np: int, L: int, P: int, window=None, out=None, precision="fp32", stream=None, workspace=None,
            y=None, conjugate=False, normalise=None):
    """FAM estimate of the complex64 CUDA tensor x; returns complex64 [Np, Np, P].
    y: second signal of a cross estimate; conjugate: the conjugate estimate; normalise:
    None, "power" (consumed samples scaled to mean power 1) or "peak" (peak magnitude 1)."""
    torch = _torch()
    lib = load()
    _need(x, torch.complex64, 1, "x")
    N = x.numel()
    y = _partner(x, y)
    if window is not None:
        _need(window, torch.float32, Np, "window")
    if out is None:
        out = torch.empty((Np, Np, P), dtype=torch.complex64, device=x.device)
    _need(out, torch.complex64, Np * Np * P, "out")
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    ws = _workspace(lib.scd_fam_workspace_bytes(N, Np, L, P, prec), x.device, workspace)
    o = make_opts(stream, prec, ws, y=y, conjugate=conjugate, normalise=normalise)
    check(lib.scd_fam(_ptr(x), N, Np, L, P, _ptr(window), _ptr(out), ctypes.byref(o)), "scd_fam")
    return out


def scd_ssca(x, Np: int, window=None, out=None, precision="fp32", stream=None, workspace=None, schedule="auto",
             y=None, conjugate=False, normalise=None):
    """SSCA estimate of the complex64 CUDA tensor x (N = x.numel()); returns complex64 [Np, N].
    y: second signal of a cross estimate; conjugate: the conjugate estimate; normalise: as
    scd_fam."""
    torch = _torch()
    lib = load()
    _need(x, torch.complex64, 1, "x")
    N = x.numel()
    y = _partner(x, y)
    if window is not None:
        _need(window, torch.float32, Np, "window")
    if out is None:
        out = torch.empty((Np, N), dtype=torch.complex64, device=x.device)
    _need(out, torch.complex64, Np * N, "out")
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    ws = _workspace(lib.scd_ssca_workspace_bytes(N, Np, prec), x.device, workspace)
    o = make_opts(stream, prec, ws, schedule=schedule, y=y, conjugate=conjugate, normalise=normalise)
    check(lib.scd_ssca(_ptr(x), N, Np, _ptr(window), _ptr(out), ctypes.byref(o)), "scd_ssca")
    return out


def scd_fam_map(S, Np: int, L: int, P: int, map=None, power: int = 1, stream=None, conjugate=False):
    """(f, alpha) grid float32 [2 Np, 2 P L] of a FAM estimate S (conjugate: of a conjugate
    estimate)."""
    torch = _torch()
    lib = load()
    _need(S, torch.complex64, Np * Np * P, "S")
    if map is None:
        map = torch.empty((2 * Np, 2 * P * L), dtype=torch.float32, device=S.device)
    _need(map, torch.float32, 4 * Np * P * L, "map")
    o = make_opts(stream, "fp32", None, power, conjugate=conjugate)
    check(lib.scd_fam_map(_ptr(S), Np, L, P, _ptr(map), ctypes.byref(o)), "scd_fam_map")
    return map


def scd_ssca_map(S, N: int, Np: int, map=None, power: int = 1, stream=None):
    """(f, alpha) grid float32 [Np, 2 N] of an SSCA estimate S."""
    torch = _torch()
    lib = load()
    _need(S, torch.complex64, Np * N, "S")
    if map is None:
        map = torch.empty((Np, 2 * N), dtype=torch.float32, device=S.device)
    _need(map, torch.float32, 2 * Np * N, "map")
    o = make_opts(stream, "fp32", None, power)
    check(lib.scd_ssca_map(_ptr(S), N, Np, _ptr(map), ctypes.byref(o)), "scd_ssca_map")
    return map


def scd_fam_alpha_profile(S, Np: int, L: int, P: int, profile=None, power: int = 1, stream=None, conjugate=False):
    """Largest |S|^power over f per alpha column of the FAM map: float32 [2 P L]."""
    torch = _torch()
    lib = load()
    _need(S, torch.complex64, Np * Np * P, "S")
    if profile is None:
        profile = torch.empty(2 * P * L, dtype=torch.float32, device=S.device)
    _need(profile, torch.float32, 2 * P * L, "profile")
    o = make_opts(stream, "fp32", None, power, conjugate=conjugate)
    check(lib.scd_fam_alpha_profile(_ptr(S), Np, L, P, _ptr(profile), ctypes.byref(o)), "scd_fam_alpha_profile")
    return profile


def scd_ssca_alpha_profile(S, N: int, Np: int, profile=None, power: int = 1, stream=None):
    """Largest |S|^power over f per alpha column of the SSCA map: float32 [2 N]."""
    torch = _torch()
    lib = load()
    _need(S, torch.complex64, Np * N, "S")
    if profile is None:
        profile = torch.empty(2 * N, dtype=torch.float32, device=S.device)
    _need(profile, torch.float32, 2 * N, "profile")
    o = make_opts(stream, "fp32", None, power)
    check(lib.scd_ssca_alpha_profile(_ptr(S), N, Np, _ptr(profile), ctypes.byref(o)), "scd_ssca_alpha_profile")
    return profile


def scd_ssca_tune(x, Np: int, window=None, out=None, precision="fp32", stream=None, workspace=None, reps=3):
    """Times scd_ssca's schedules for (N, Np, precision) and keeps the fastest for "auto"."""
    torch = _torch()
    lib = load()
    N = x.numel()
    if out is None:
        out = torch.empty((Np, N), dtype=torch.complex64, device=x.device)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    ws = _workspace(lib.scd_ssca_workspace_bytes(N, Np, prec), x.device, workspace)
    o = make_opts(stream, prec, ws)
    check(lib.scd_ssca_tune(_ptr(x), N, Np, _ptr(window), _ptr(out), ctypes.byref(o), reps), "scd_ssca_tune")
    return out


def scd_chebyshev_window(Np: int, atten_db: float = 100.0, window=None, stream=None, device="cuda"):
    """Dolph-Chebyshev window float32[Np] on the device (the chebwin of Algorithms 1 and 2)."""
    torch = _torch()
    lib = load()
    if window is None:
        window = torch.empty(Np, dtype=torch.float32, device=device)
    _need(window, torch.float32, Np, "window")
    check(lib.scd_chebyshev_window(Np, float(atten_db), _ptr(window), _stream(stream)), "scd_chebyshev_window")
    return window


def scd_check_device(stream=None) -> None:
    """Raises ScdError(SCD_ERR_TIMEOUT) if a bounded device-side wait expired."""
    check(load().scd_check_device(_stream(stream)), "scd_check_device")


def scd_prepare(estimator: str, N: int, Np: int, P: int = 2) -> None:
    lib = load()
    check(lib.scd_prepare({"fam": 0, "ssca": 1}[estimator], N, Np, P), "scd_prepare")


class HostBuffer:
    """Page-locked host memory (scd_host_alloc) of `numel` elements of `dtype`, viewed as the
    CPU tensor `.tensor` (valid until close())."""

    def __init__(self, numel, dtype):
        torch = _torch()
        self.lib = load()
        nbytes = int(numel) * torch.empty((), dtype=dtype).element_size()
        p = ctypes.c_void_p()
        check(self.lib.scd_host_alloc(nbytes, ctypes.byref(p)), "scd_host_alloc")
        self.ptr, self.nbytes = p.value, nbytes
        buf = (ctypes.c_char * nbytes).from_address(self.ptr)
        self.tensor = torch.frombuffer(buf, dtype=torch.uint8).view(dtype)

    def close(self):
        if self.ptr:
            self.tensor = None
            check(self.lib.scd_host_free(ctypes.c_void_p(self.ptr)), "scd_host_free")
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchPlan:
    """A batch of uneven-length signals for one estimator (scd_batch_plan_* of the C ABI).

    estimator: "fam" or "ssca"; lengths: signal lengths; the arenas are torch tensors:
    x_arena complex64[x_offsets[-1]], out_arena complex64[out_offsets[-1]]."""

    def __init__(self, estimator: str, lengths, Np: int, L: int = 1, precision="fp32", exact=False):
        """exact: every sample used (scd_batch_plan_create_exact: FAM P_i = (len_i - Np)//L + 1,
        SSCA N_i = len_i, not rounded down to powers of two)."""
        lib = load()
        self.lib = lib
        self.estimator = estimator
        self.nsig = len(lengths)
        self.Np, self.L = Np, L
        arr = (ctypes.c_int64 * self.nsig)(*[int(v) for v in lengths])
        handle = ctypes.c_void_p()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        create = lib.scd_batch_plan_create_exact if exact else lib.scd_batch_plan_create
        check(create({"fam": 0, "ssca": 1}[estimator], self.nsig, arr, Np, L, prec, ctypes.byref(handle)),
              "scd_batch_plan_create_exact" if exact else "scd_batch_plan_create")
        self.handle = handle
        self._query()

    profile_power = 0

    def set_output(self, mode: str = "estimate", power: int = 1):
        """mode "estimate" (the SCD of every signal) or "profile" (only each signal's alpha
        profile of |S|^power, reduced inside the kernel; the out arena becomes float32)."""
        p = 0 if mode == "estimate" else int(power)
        check(self.lib.scd_batch_plan_set_output(self.handle, p), "scd_batch_plan_set_output")
        self.profile_power = p
        self._query()

    def set_schedule(self, schedule: str = "auto"):
        """"persistent" (one launch), "stages" (one launch per stage and size), "fused" (SSCA,
        FP32: the channeliser, channel-data product and first strip pass in one kernel per size
        class, where its tiles fit) or "auto" (the autotuned choice, else the estimator's
        default)."""
        check(self.lib.scd_batch_plan_set_schedule(self.handle, SCHEDULES[schedule]), "scd_batch_plan_set_schedule")

    def out_dtype(self):
        return _torch().float32 if self.profile_power else _torch().complex64

    def _query(self):
        lib, handle, n = self.lib, self.handle, self.nsig
        xo, oo = (ctypes.c_int64 * (n + 1))(), (ctypes.c_int64 * (n + 1))()
        sz, used = (ctypes.c_int64 * n)(), (ctypes.c_int64 * n)()
        ws = ctypes.c_size_t()
        check(lib.scd_batch_query(handle, xo, oo, sz, used, ctypes.byref(ws)), "scd_batch_query")
        self.x_offsets, self.out_offsets = list(xo), list(oo)
        self.sizes, self.used = list(sz), list(used)
        self.workspace_bytes = ws.value

    def run(self, x_arena, out_arena, workspace, window=None, stream=None):
        torch = _torch()
        _need(x_arena, torch.complex64, self.x_offsets[-1], "x_arena")
        _need(out_arena, self.out_dtype(), self.out_offsets[-1], "out_arena")
        check(self.lib.scd_batch_run(self.handle, _ptr(x_arena), _ptr(window), _ptr(out_arena),
                                     _ptr(workspace), _stream(stream)), "scd_batch_run")

    def run_host(self, x_host, x_arena, out_arena, out_host, workspace, window=None, stream=None):
        """scd_batch_run_host: copies x_host (a CPU tensor, ideally a HostBuffer's; None when
        x_arena already holds the input) into x_arena, runs the plan into out_arena and copies it
        into out_host (a CPU tensor) on the plan's copy stream; returns once enqueued (host_wait)."""
        torch = _torch()
        _need(x_arena, torch.complex64, self.x_offsets[-1], "x_arena")
        _need(out_arena, self.out_dtype(), self.out_offsets[-1], "out_arena")
        for t, n, name in ((x_host, self.x_offsets[-1] * 8, "x_host"),
                           (out_host, self.out_offsets[-1] * out_arena.element_size(), "out_host")):
            if t is None and name == "x_host":
                continue
            if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_contiguous() or \
                    t.numel() * t.element_size() < n:
                raise TypeError(f"{name} must be a contiguous CPU tensor of at least {n} bytes")
        check(self.lib.scd_batch_run_host(self.handle, _ptr(x_host), _ptr(x_arena), _ptr(window), _ptr(out_arena),
                                          _ptr(out_host), _ptr(workspace), _stream(stream)), "scd_batch_run_host")

    def host_wait(self):
        """Blocks until every copy run_host queued on this plan has reached host memory."""
        check(self.lib.scd_batch_host_wait(self.handle), "scd_batch_host_wait")

    def tune(self, x_arena, out_arena, workspace, window=None, stream=None, reps=3):
        """Times the persistent schedule's sizing candidates on these buffers, keeps the fastest
        (scd_batch_tune); the output holds a valid estimate afterwards."""
        check(self.lib.scd_batch_tune(self.handle, _ptr(x_arena), _ptr(window), _ptr(out_arena), _ptr(workspace),
                                      _stream(stream), reps), "scd_batch_tune")

    def output(self, out_arena, i):
        """View of signal i's estimate in the output arena."""
        a, b = self.out_offsets[i], self.out_offsets[i + 1]
        if self.profile_power:
            return out_arena[a:b]
        if self.estimator == "fam":
            return out_arena[a:b].view(self.Np, self.Np, self.sizes[i])
        return out_arena[a:b].view(self.Np, self.sizes[i])

    def close(self):
        if self.handle is not None and self.handle.value:
            self.lib.scd_batch_plan_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class StreamPlan(BatchPlan):
    """Successive windows of one continuous signal (scd_stream_plan_create / scd_stream_advance):
    nwin windows of window_len samples every hop samples per group.  The arenas are torch
    tensors as for BatchPlan; x_offsets[-1] is the arena length (span)."""

    def __init__(self, estimator: str, window_len: int, hop: int, nwin: int, Np: int, L: int = 1,
                 precision="fp32"):
        lib = load()
        self.lib = lib
        self.estimator = estimator
        self.nsig = nwin
        self.Np, self.L = Np, L
        self.window_len, self.hop = window_len, hop
        handle = ctypes.c_void_p()
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        check(lib.scd_stream_plan_create({"fam": 0, "ssca": 1}[estimator], window_len, hop, nwin, Np, L, prec,
                                         ctypes.byref(handle)), "scd_stream_plan_create")
        self.handle = handle
        self._query()

    @property
    def span(self):
        return self.x_offsets[-1]

    def advance(self, x_arena, samples, stream=None):
        """Slides x_arena to the next group; samples: the next nwin*hop stream samples, a
        complex64 tensor on the host (pinned for full speed) or on the device."""
        torch = _torch()
        _need(x_arena, torch.complex64, self.span, "x_arena")
        if samples.dtype != torch.complex64 or not samples.is_contiguous() or samples.numel() < self.nsig * self.hop:
            raise TypeError(f"samples must be a contiguous complex64 tensor of {self.nsig * self.hop} elements")
        check(self.lib.scd_stream_advance(self.handle, _ptr(x_arena), _ptr(samples), 0 if samples.is_cuda else 1,
                                          _stream(stream)), "scd_stream_advance")
