"""Thin ctypes binding of libsprot (C ABI in include/sprot.h).

Only argument marshalling lives here: every step of the estimator runs in the library's CUDA
kernels. Device arrays are torch CUDA tensors (torch provides device memory and streams);
host arrays are numpy arrays used with the SPROT_HOST_PTRS flag. ``load()`` raises if the
library has not been built -- there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsprot.so")

OK, E_INVAL, E_NOMEM, E_CUDA, E_TIMEOUT, E_NOAXIS, E_UNIMPL, E_BUSY = 0, -1, -2, -3, -4, -5, -6, -7
HOST_PTRS = 0x1
SUBCELL_AXIS = 0x2
MAX_K = 8
MAX_BANDS = 96

EXPORTS = [
    "sprot_default_params", "sprot_status_string", "sprot_estimate_rotation",
    "sprot_estimate_rotations_k", "sprot_estimate_rotations_ex", "sprot_axis_vote",
    "sprot_axis_vote_sampled", "sprot_axis_vote_eps", "sprot_refine_axis",
    "sprot_select_peaks", "sprot_estimate_batch", "sprot_autotune_grid", "sprot_server_create",
    "sprot_server_submit", "sprot_server_wait", "sprot_server_destroy",
    "sprot_release_workspaces", "sprot_release_stream_workspace", "sprot_kernel_launch_count", "sprot_probe_smem_atomic_rate",
    "sprot_kernel_timing", "sprot_kernel_timing_read", "sprot_vote_plan", "sprot_vote_plan_sm",
    "sprot_axis_vote_noalloc",
    "sprot_default_knobs", "sprot_autotune_plan", "sprot_autotune_batch", "sprot_tuned_plan",
    "sprot_set_tuned_plan", "sprot_autotune_reset", "sprot_server_request_bytes",
]


class Params(C.Structure):
    _fields_ = [("grid", C.c_int32), ("angle_bins", C.c_int32), ("k", C.c_int32),
                ("nms_deg", C.c_float), ("gate_window", C.c_int32), ("angle_window", C.c_int32),
                ("tau", C.c_double), ("flags", C.c_uint32)]


class Rotation(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("R_init", C.c_double * 9), ("R_vote", C.c_double * 9),
                ("axis", C.c_double * 3), ("theta", C.c_double), ("cell_row", C.c_int32),
                ("cell_col", C.c_int32), ("angle_bin", C.c_int32), ("axis_votes", C.c_uint32),
                ("angle_votes", C.c_uint32), ("n_vote_set", C.c_uint32), ("n_inliers", C.c_uint32),
                ("n_degenerate", C.c_uint32), ("cell_offset", C.c_double * 2)]

    def to_dict(self) -> dict:
        return dict(
            R=np.array(self.R[:]).reshape(3, 3), R_init=np.array(self.R_init[:]).reshape(3, 3),
            R_vote=np.array(self.R_vote[:]).reshape(3, 3), axis=np.array(self.axis[:]),
            theta=float(self.theta), cell=(int(self.cell_row), int(self.cell_col)),
            bin=int(self.angle_bin), axis_votes=int(self.axis_votes),
            angle_votes=int(self.angle_votes), n_vote_set=int(self.n_vote_set),
            n_inliers=int(self.n_inliers), n_degenerate=int(self.n_degenerate),
            cell_offset=(float(self.cell_offset[0]), float(self.cell_offset[1])))


class Debug(C.Structure):
    _fields_ = [("grid", C.c_void_p), ("hist", C.c_void_p), ("bins", C.c_void_p),
                ("vote_set", C.c_void_p)]


class Instance(C.Structure):
    _fields_ = [("P", C.c_void_p), ("Q", C.c_void_p), ("n", C.c_int64), ("params", Params),
                ("out", C.POINTER(Rotation)), ("n_found", C.POINTER(C.c_int32)),
                ("labels", C.c_void_p)]


class Knobs(C.Structure):
    _fields_ = [("vote_rounds", C.c_int32), ("chunk_div", C.c_int32), ("batch_slice", C.c_int32),
                ("batch_div", C.c_int32), ("ms_tuned", C.c_double), ("ms_default", C.c_double)]

    def to_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class ServerCfg(C.Structure):
    _fields_ = [("device_budget_bytes", C.c_size_t), ("max_batch", C.c_int32),
                ("max_queue", C.c_int32), ("device", C.c_int32)]


class Request(C.Structure):
    _fields_ = [("P", C.c_void_p), ("Q", C.c_void_p), ("n", C.c_int64), ("params", Params)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("n_found", C.c_int32), ("rot", Rotation * MAX_K),
                ("t_submit_ms", C.c_double), ("t_admit_ms", C.c_double), ("t_done_ms", C.c_double)]


class SprotError(RuntimeError):
    def __init__(self, status: int, what: str, text: str):
        super().__init__(f"{what}: {text} ({status})")
        self.status = status


_LIB = None


def load(path: str = LIB_PATH):
    """Loads libsprot.so (built by ``paper_2502_06337_gb300.build``) and declares its ABI."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_2502_06337_gb300.build.build() first")
    lib = C.CDLL(path)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    lib.sprot_default_params.argtypes = [C.POINTER(Params)]
    lib.sprot_default_params.restype = None
    lib.sprot_status_string.argtypes = [C.c_int]
    lib.sprot_status_string.restype = C.c_char_p
    lib.sprot_estimate_rotation.argtypes = [vp, vp, i64, C.POINTER(Params), C.POINTER(Rotation), vp, vp]
    lib.sprot_estimate_rotations_k.argtypes = [vp, vp, i64, C.POINTER(Params), C.POINTER(Rotation),
                                               C.POINTER(i32), vp, vp]
    lib.sprot_estimate_rotations_ex.argtypes = [vp, vp, i64, C.POINTER(Params), C.POINTER(Rotation),
                                                C.POINTER(i32), vp, C.POINTER(Debug), vp]
    lib.sprot_axis_vote.argtypes = [vp, vp, i64, i32, vp, vp]
    lib.sprot_axis_vote_sampled.argtypes = [vp, vp, i64, i32, i32, vp, vp]
    lib.sprot_axis_vote_eps.argtypes = [vp, vp, i64, i32, C.c_float, vp, vp]
    lib.sprot_vote_plan.argtypes = [i64, i32, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
    lib.sprot_vote_plan_sm.argtypes = [i64, i32, i32, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
    lib.sprot_axis_vote_noalloc.argtypes = [vp, vp, i64, i32, vp, vp]
    lib.sprot_refine_axis.argtypes = [vp, vp, i64, vp, i32, vp, C.POINTER(C.c_double),
                                      C.POINTER(C.c_double), C.POINTER(i64), vp]
    lib.sprot_select_peaks.argtypes = [vp, i32, i32, C.c_float, vp, vp, vp, vp]
    lib.sprot_estimate_batch.argtypes = [C.POINTER(Instance), i64, vp]
    lib.sprot_autotune_grid.argtypes = [i64]
    lib.sprot_autotune_grid.restype = i32
    lib.sprot_default_knobs.argtypes = [C.POINTER(Knobs)]
    lib.sprot_default_knobs.restype = None
    lib.sprot_autotune_plan.argtypes = [vp, vp, i64, C.POINTER(Params), i32, C.POINTER(Knobs), vp]
    lib.sprot_autotune_batch.argtypes = [C.POINTER(Instance), i64, i32, C.POINTER(Knobs), vp]
    lib.sprot_tuned_plan.argtypes = [i64, i32, i32, C.POINTER(Knobs)]
    lib.sprot_tuned_plan.restype = i32
    lib.sprot_set_tuned_plan.argtypes = [i64, i32, i32, C.POINTER(Knobs)]
    lib.sprot_autotune_reset.argtypes = []
    lib.sprot_autotune_reset.restype = None
    lib.sprot_server_create.argtypes = [C.POINTER(ServerCfg), C.POINTER(vp)]
    lib.sprot_server_request_bytes.argtypes = [C.POINTER(ServerCfg), C.POINTER(Request)]
    lib.sprot_server_request_bytes.restype = C.c_size_t
    lib.sprot_server_submit.argtypes = [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]
    lib.sprot_server_wait.argtypes = [vp, C.c_uint64, i32, C.POINTER(Result)]
    lib.sprot_server_destroy.argtypes = [vp]
    lib.sprot_release_workspaces.argtypes = []
    lib.sprot_release_workspaces.restype = None
    lib.sprot_release_stream_workspace.argtypes = [vp]
    lib.sprot_release_stream_workspace.restype = None
    lib.sprot_kernel_launch_count.argtypes = []
    lib.sprot_kernel_launch_count.restype = C.c_uint64
    lib.sprot_probe_smem_atomic_rate.argtypes = [i32, C.POINTER(C.c_double), vp]
    lib.sprot_kernel_timing.argtypes = [C.c_int]
    lib.sprot_kernel_timing.restype = None
    lib.sprot_kernel_timing_read.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_uint64)]
    lib.sprot_kernel_timing_read.restype = None
    for name in ["sprot_estimate_rotation", "sprot_estimate_rotations_k", "sprot_estimate_rotations_ex",
                 "sprot_axis_vote", "sprot_axis_vote_sampled", "sprot_vote_plan", "sprot_vote_plan_sm", "sprot_axis_vote_noalloc", "sprot_axis_vote_eps", "sprot_refine_axis",
                 "sprot_select_peaks",
                 "sprot_estimate_batch", "sprot_autotune_plan", "sprot_autotune_batch", "sprot_set_tuned_plan",
                 "sprot_server_create", "sprot_server_submit", "sprot_server_wait",
                 "sprot_server_destroy", "sprot_probe_smem_atomic_rate"]:
        getattr(lib, name).restype = C.c_int
    _LIB = lib
    return lib


def status_text(status: int) -> str:
    return load().sprot_status_string(status).decode()


def check(status: int, what: str, allowed=()):
    if status != OK and status not in allowed:
        raise SprotError(status, what, status_text(status))
    return status


def make_params(grid=256, angle_bins=360, k=1, nms_deg=2.0, gate_window=1, angle_window=1,
                tau=0.05, flags=0) -> Params:
    return Params(int(grid), int(angle_bins), int(k), float(nms_deg), int(gate_window),
                  int(angle_window), float(tau), int(flags))


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch

    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _check_points(P, Q):
    import torch

    for X in (P, Q):
        if isinstance(X, np.ndarray):
            assert X.dtype == np.float32 and X.ndim == 2 and X.shape[1] == 3 and X.flags.c_contiguous
        else:
            assert isinstance(X, torch.Tensor) and X.dtype == torch.float32 and X.is_contiguous()
            assert X.dim() == 2 and X.shape[1] == 3
    assert P.shape == Q.shape


def estimate_rotation(P, Q, params: Params, mask=None, stream=None):
    """One rotation (k = 1). P, Q: device tensors, or numpy arrays with HOST_PTRS set in
    params.flags. ``mask``: optional n-byte output (uint8 tensor / array)."""
    _check_points(P, Q)
    lib = load()
    out = Rotation()
    st = lib.sprot_estimate_rotation(_ptr(P), _ptr(Q), P.shape[0], C.byref(params), C.byref(out),
                                     _ptr(mask), _stream(stream))
    check(st, "sprot_estimate_rotation")
    return out.to_dict()


def estimate_rotations(P, Q, params: Params, labels=None, debug: dict | None = None, stream=None,
                       allow_noaxis=False):
    """Up to params.k rotations. ``labels``: optional n int32 output. ``debug``: optional dict
    of device tensors {'grid': G*G u32 (int32 view), 'hist': k*J, 'bins': k*n int16,
    'vote_set': k*n uint8} filled with the intermediates. Returns a list of dicts."""
    _check_points(P, Q)
    lib = load()
    outs = (Rotation * max(1, params.k))()
    nf = C.c_int32(0)
    dbg = None
    if debug is not None:
        dbg = Debug(_ptr(debug.get("grid")), _ptr(debug.get("hist")), _ptr(debug.get("bins")),
                    _ptr(debug.get("vote_set")))
    st = lib.sprot_estimate_rotations_ex(_ptr(P), _ptr(Q), P.shape[0], C.byref(params), outs,
                                         C.byref(nf), _ptr(labels),
                                         C.byref(dbg) if dbg is not None else None, _stream(stream))
    check(st, "sprot_estimate_rotations_ex", allowed=(E_NOAXIS,) if allow_noaxis else ())
    return [outs[a].to_dict() for a in range(nf.value)]


def axis_vote(P, Q, G: int, grid, stream=None):
    """Fills the device tensor ``grid`` (G*G 32-bit) with the accumulator."""
    _check_points(P, Q)
    st = load().sprot_axis_vote(_ptr(P), _ptr(Q), P.shape[0], int(G), _ptr(grid), _stream(stream))
    check(st, "sprot_axis_vote")


def vote_plan(n: int, G: int, batched: bool = False, n_sm: int | None = None):
    """The axis vote's work split for n pairs on a G x G grid: dict(band_row0, slices), for the
    current device, or without a GPU for a device of ``n_sm`` SMs."""
    nb, sl = C.c_int32(0), C.c_int32(0)
    rows = (C.c_int32 * (MAX_BANDS + 1))()
    if n_sm is None:
        check(load().sprot_vote_plan(int(n), int(G), 1 if batched else 0, C.byref(nb), rows, C.byref(sl)),
              "sprot_vote_plan")
    else:
        check(load().sprot_vote_plan_sm(int(n), int(G), 1 if batched else 0, int(n_sm), C.byref(nb), rows,
                                        C.byref(sl)), "sprot_vote_plan_sm")
    return dict(band_row0=list(rows[:nb.value + 1]), slices=sl.value)


def axis_vote_sampled(P, Q, G: int, J: int, grid, stream=None):
    """Fills the device tensor ``grid`` (G*G 32-bit) with Algorithm 1's sampled accumulator
    (J points per circle)."""
    _check_points(P, Q)
    st = load().sprot_axis_vote_sampled(_ptr(P), _ptr(Q), P.shape[0], int(G), int(J), _ptr(grid),
                                        _stream(stream))
    check(st, "sprot_axis_vote_sampled")


def axis_vote_eps(P, Q, G: int, eps: float, grid, stream=None):
    """Fills the device tensor ``grid`` (G*G 32-bit) with the eps-band accumulator of Eq. 9."""
    _check_points(P, Q)
    st = load().sprot_axis_vote_eps(_ptr(P), _ptr(Q), P.shape[0], int(G), float(eps), _ptr(grid),
                                    _stream(stream))
    check(st, "sprot_axis_vote_eps")


def refine_axis(P, Q, labels=None, label: int = 0, hint=None, stream=None):
    """Least-squares axis (Eq. 10) of the pairs with labels == label (all pairs when labels
    is None). Returns dict(axis, lambda_min, count) or None when the axis is not determined."""
    _check_points(P, Q)
    axis = (C.c_double * 3)()
    lam = C.c_double(0.0)
    cnt = C.c_int64(0)
    h = (C.c_double * 3)(*[float(x) for x in hint]) if hint is not None else None
    st = load().sprot_refine_axis(_ptr(P), _ptr(Q), P.shape[0], _ptr(labels), int(label), h, axis,
                                  C.byref(lam), C.byref(cnt), _stream(stream))
    if st == E_NOAXIS:
        return None
    check(st, "sprot_refine_axis")
    return dict(axis=np.array(axis[:]), lambda_min=lam.value, count=cnt.value)


def select_peaks(grid, G: int, k: int, nms_deg: float, cells, counts, n_found, stream=None):
    st = load().sprot_select_peaks(_ptr(grid), int(G), int(k), float(nms_deg), _ptr(cells),
                                   _ptr(counts), _ptr(n_found), _stream(stream))
    check(st, "sprot_select_peaks")


def _struct_dtype(ctype, prefix="", base=0, out=None):
    """numpy dtype fields (name, format, offset) of a ctypes structure, flattened."""
    out = [] if out is None else out
    for name, t in ctype._fields_:
        off = base + getattr(ctype, name).offset
        if isinstance(t, type) and issubclass(t, C.Structure):
            _struct_dtype(t, prefix + name + ".", off, out)
        else:
            fmt = {C.c_int32: "<i4", C.c_uint32: "<u4", C.c_int64: "<i8", C.c_float: "<f4",
                   C.c_double: "<f8"}.get(t, "<u8")  # pointers: 64-bit addresses
            out.append((prefix + name, fmt, off))
    return out


_INSTANCE_FIELDS = None
_ROTATION_DTYPE = None


def _rotation_dtype():
    global _ROTATION_DTYPE
    if _ROTATION_DTYPE is None:
        f = []
        for name, t in Rotation._fields_:
            off = getattr(Rotation, name).offset
            if name in ("R", "R_init", "R_vote"):
                f.append((name, ("<f8", (9,)), off))
            elif name == "axis":
                f.append((name, ("<f8", (3,)), off))
            elif name == "cell_offset":
                f.append((name, ("<f8", (2,)), off))
            else:
                f.append((name, {C.c_double: "<f8", C.c_int32: "<i4", C.c_uint32: "<u4"}[t], off))
        _ROTATION_DTYPE = np.dtype({"names": [x[0] for x in f], "formats": [x[1] for x in f],
                                    "offsets": [x[2] for x in f], "itemsize": C.sizeof(Rotation)})
    return _ROTATION_DTYPE


class BatchResult:
    """Rotations of a batched solve, kept as one array; res[i] is the list of rotation dicts of
    instance i (built on access)."""

    def __init__(self, rot: np.ndarray, n_found: np.ndarray, kmax: int):
        self.rot = rot.reshape(len(n_found), kmax)
        self.n_found = n_found

    def __len__(self):
        return len(self.n_found)

    def _one(self, i):
        out = []
        for a in range(int(self.n_found[i])):
            r = self.rot[i, a]
            out.append(dict(R=r["R"].reshape(3, 3).copy(), R_init=r["R_init"].reshape(3, 3).copy(),
                            R_vote=r["R_vote"].reshape(3, 3).copy(), axis=r["axis"].copy(),
                            theta=float(r["theta"]), cell=(int(r["cell_row"]), int(r["cell_col"])),
                            bin=int(r["angle_bin"]), axis_votes=int(r["axis_votes"]),
                            angle_votes=int(r["angle_votes"]), n_vote_set=int(r["n_vote_set"]),
                            n_inliers=int(r["n_inliers"]), n_degenerate=int(r["n_degenerate"]),
                            cell_offset=(float(r["cell_offset"][0]), float(r["cell_offset"][1]))))
        return out

    def __getitem__(self, i):
        if isinstance(i, slice):
            return [self._one(j) for j in range(*i.indices(len(self)))]
        return self._one(i if i >= 0 else len(self) + i)

    def __iter__(self):
        return (self._one(i) for i in range(len(self)))


_PARAMS_DTYPE = None


def _params_dtype():
    """numpy dtype of one sprot_params, so that a list of Params converts in one pass."""
    global _PARAMS_DTYPE
    if _PARAMS_DTYPE is None:
        f = _struct_dtype(Params)
        _PARAMS_DTYPE = np.dtype({"names": [x[0] for x in f], "formats": [x[1] for x in f],
                                  "offsets": [x[2] for x in f], "itemsize": C.sizeof(Params)})
    return _PARAMS_DTYPE


def _instance_table(problems):
    """The sprot_instance table of a batch as one numpy record array in the layout of
    sprot_instance, with the output arrays it points into: (table, rotations, n_found, kmax).
    A batch of thousands costs a few list passes and no per-field Python work: the Params
    structures are converted from their raw bytes in one step."""
    import torch

    global _INSTANCE_FIELDS
    if _INSTANCE_FIELDS is None:
        _INSTANCE_FIELDS = _struct_dtype(Instance)
    m = len(problems)
    fields = _INSTANCE_FIELDS
    dt = np.dtype({"names": [f[0] for f in fields], "formats": [f[1] for f in fields],
                   "offsets": [f[2] for f in fields], "itemsize": C.sizeof(Instance)})
    Ps = [pb[0] for pb in problems]
    Qs = [pb[1] for pb in problems]
    f32 = torch.float32
    for P, Q in zip(Ps, Qs):
        if not (isinstance(P, torch.Tensor) and isinstance(Q, torch.Tensor) and P.dtype is f32 and
                Q.dtype is f32 and P.dim() == 2 and P.shape[1] == 3 and P.shape == Q.shape and
                P.is_contiguous() and Q.is_contiguous()):
            _check_points(P, Q)  # names the failure
            raise ValueError("P and Q must be contiguous float32 tensors of shape (n, 3)")
    prm = np.frombuffer(b"".join([bytes(pb[2]) for pb in problems]), dtype=_params_dtype())
    kmax = max(1, int(prm["k"].max())) if m else 1
    tab = np.zeros(m, dtype=dt)
    tab["P"] = np.fromiter((P.data_ptr() for P in Ps), np.uint64, m)
    tab["Q"] = np.fromiter((Q.data_ptr() for Q in Qs), np.uint64, m)
    tab["n"] = np.fromiter((P.shape[0] for P in Ps), np.int64, m)
    tab["labels"] = np.fromiter((pb[3].data_ptr() if len(pb) > 3 and pb[3] is not None else 0
                                 for pb in problems), np.uint64, m)
    for name in prm.dtype.names:
        tab["params." + name] = prm[name]
    rot = np.zeros(m * kmax, dtype=_rotation_dtype())
    n_found = np.zeros(m, dtype=np.int32)
    tab["out"] = rot.ctypes.data + np.arange(m, dtype=np.uint64) * np.uint64(kmax * C.sizeof(Rotation))
    tab["n_found"] = n_found.ctypes.data + np.arange(m, dtype=np.uint64) * np.uint64(4)
    return tab, rot, n_found, kmax


def params_array(m: int, **fields) -> np.ndarray:
    """m sprot_params as one numpy record array (the defaults of make_params, then ``fields``,
    each a scalar or a length-m array), for the packed batch calls."""
    arr = np.zeros(m, dtype=_params_dtype())
    base = make_params()
    for name, _ in Params._fields_:
        arr[name] = fields.get(name, getattr(base, name))
    return arr


def _packed_table(P, Q, offsets, params, labels=None):
    """The sprot_instance table of instances stored back to back: instance i is rows
    offsets[i]:offsets[i + 1] of the device tensors P and Q (and of ``labels``, an n-element
    int32 device tensor, if given). ``params``: one Params for every instance, or a record
    array from params_array. Returns (table, rotations, n_found, kmax)."""
    _check_points(P, Q)
    off = np.asarray(offsets, dtype=np.int64)
    m = len(off) - 1
    if m < 1 or off[0] != 0 or off[-1] != P.shape[0] or np.any(np.diff(off) < 1):
        raise ValueError("offsets must rise strictly from 0 to n")
    if isinstance(params, Params):
        prm = np.frombuffer(bytes(params) * m, dtype=_params_dtype())
    else:
        prm = np.asarray(params)
        if prm.dtype != _params_dtype() or prm.shape != (m,):
            raise ValueError("params: a Params or params_array(m, ...)")
    if labels is not None and (labels.dtype != __import__("torch").int32 or labels.numel() != P.shape[0]
                               or not labels.is_contiguous()):
        raise ValueError("labels must be a contiguous int32 tensor of n elements")
    global _INSTANCE_FIELDS
    if _INSTANCE_FIELDS is None:
        _INSTANCE_FIELDS = _struct_dtype(Instance)
    fields = _INSTANCE_FIELDS
    dt = np.dtype({"names": [f[0] for f in fields], "formats": [f[1] for f in fields],
                   "offsets": [f[2] for f in fields], "itemsize": C.sizeof(Instance)})
    kmax = max(1, int(prm["k"].max()))
    tab = np.zeros(m, dtype=dt)
    row = off[:-1].astype(np.uint64)
    tab["P"] = np.uint64(P.data_ptr()) + row * np.uint64(12)
    tab["Q"] = np.uint64(Q.data_ptr()) + row * np.uint64(12)
    tab["n"] = np.diff(off)
    tab["labels"] = 0 if labels is None else np.uint64(labels.data_ptr()) + row * np.uint64(4)
    for name in prm.dtype.names:
        tab["params." + name] = prm[name]
    rot = np.zeros(m * kmax, dtype=_rotation_dtype())
    n_found = np.zeros(m, dtype=np.int32)
    tab["out"] = rot.ctypes.data + np.arange(m, dtype=np.uint64) * np.uint64(kmax * C.sizeof(Rotation))
    tab["n_found"] = n_found.ctypes.data + np.arange(m, dtype=np.uint64) * np.uint64(4)
    return tab, rot, n_found, kmax


def estimate_batch_packed(P, Q, offsets, params, labels=None, stream=None):
    """sprot_estimate_batch over instances stored back to back in P and Q (see _packed_table):
    the batch's table costs a few numpy operations whatever its size. Returns (BatchResult,
    array of the grid sides used)."""
    tab, rot, n_found, kmax = _packed_table(P, Q, offsets, params, labels)
    st = load().sprot_estimate_batch(tab.ctypes.data_as(C.POINTER(Instance)), len(tab), _stream(stream))
    check(st, "sprot_estimate_batch")
    return BatchResult(rot, n_found, kmax), tab["params.grid"].copy()


def autotune_batch_packed(P, Q, offsets, params, reps: int = 3, stream=None) -> dict:
    """autotune_batch for a packed batch."""
    tab, rot, n_found, _ = _packed_table(P, Q, offsets, params)
    k = Knobs()
    st = load().sprot_autotune_batch(tab.ctypes.data_as(C.POINTER(Instance)), len(tab), int(reps),
                                     C.byref(k), _stream(stream))
    del rot, n_found
    check(st, "sprot_autotune_batch")
    return k.to_dict()


def estimate_batch(problems, stream=None):
    """problems: list of (P, Q, Params[, labels]) with device tensors. Returns (BatchResult,
    array of the grid sides used)."""
    tab, rot, n_found, kmax = _instance_table(problems)
    st = load().sprot_estimate_batch(tab.ctypes.data_as(C.POINTER(Instance)), len(problems), _stream(stream))
    check(st, "sprot_estimate_batch")
    return BatchResult(rot, n_found, kmax), tab["params.grid"].copy()


def default_knobs() -> dict:
    k = Knobs()
    load().sprot_default_knobs(C.byref(k))
    return k.to_dict()


def autotune_plan(P, Q, params: Params, reps: int = 3, stream=None) -> dict:
    """Times the candidate plans of the single solve of (P, Q, params) and stores the fastest
    for its class (sprot_autotune_plan). Returns the winner's knobs with both times."""
    _check_points(P, Q)
    k = Knobs()
    st = load().sprot_autotune_plan(_ptr(P), _ptr(Q), P.shape[0], C.byref(params), int(reps), C.byref(k),
                                    _stream(stream))
    check(st, "sprot_autotune_plan")
    return k.to_dict()


def autotune_batch(problems, reps: int = 3, stream=None) -> dict:
    """As autotune_plan for a batch (sprot_autotune_batch); problems as for estimate_batch."""
    # the table points into rot and n_found: they must outlive the call
    tab, rot, n_found, _ = _instance_table(problems)
    k = Knobs()
    st = load().sprot_autotune_batch(tab.ctypes.data_as(C.POINTER(Instance)), len(problems), int(reps),
                                     C.byref(k), _stream(stream))
    del rot, n_found
    check(st, "sprot_autotune_batch")
    return k.to_dict()


def tuned_plan(n: int, G: int = 0, batched: bool = False):
    """(tuned?, knobs) a solve of this class would use on the current device."""
    k = Knobs()
    found = load().sprot_tuned_plan(int(n), int(G), 1 if batched else 0, C.byref(k))
    return bool(found), k.to_dict()


def set_tuned_plan(n: int, knobs: dict, G: int = 0, batched: bool = False):
    """Stores knobs for the class of (n, G) or of a batch with mean n (sprot_set_tuned_plan)."""
    k = Knobs(*[int(knobs[f]) if f not in ("ms_tuned", "ms_default") else float(knobs.get(f, 0.0))
                for f, _ in Knobs._fields_])
    check(load().sprot_set_tuned_plan(int(n), int(G), 1 if batched else 0, C.byref(k)), "sprot_set_tuned_plan")


def autotune_reset():
    load().sprot_autotune_reset()


class Server:
    """Continuous-batching server over host requests (sprot_server_*)."""

    def __init__(self, budget_bytes: int, max_batch: int = 256, max_queue: int = 65536, device: int = 0):
        self.lib = load()
        cfg = ServerCfg(int(budget_bytes), int(max_batch), int(max_queue), int(device))
        self.cfg = cfg
        h = C.c_void_p()
        check(self.lib.sprot_server_create(C.byref(cfg), C.byref(h)), "sprot_server_create")
        self.h = h
        self._keep = {}

    def request_bytes(self, P: np.ndarray, Q: np.ndarray, params: Params) -> int:
        """Bytes the admission counts for this request against the budget."""
        req = Request(_ptr(P), _ptr(Q), P.shape[0], params)
        return int(self.lib.sprot_server_request_bytes(C.byref(self.cfg), C.byref(req)))

    def submit(self, P: np.ndarray, Q: np.ndarray, params: Params) -> int:
        _check_points(P, Q)
        req = Request(_ptr(P), _ptr(Q), P.shape[0], params)
        t = C.c_uint64(0)
        check(self.lib.sprot_server_submit(self.h, C.byref(req), C.byref(t)), "sprot_server_submit")
        self._keep[t.value] = (P, Q)
        return t.value

    def try_submit(self, P, Q, params: Params):
        """Like submit, but returns the status instead of raising on NOMEM/BUSY."""
        req = Request(_ptr(P), _ptr(Q), P.shape[0], params)
        t = C.c_uint64(0)
        st = self.lib.sprot_server_submit(self.h, C.byref(req), C.byref(t))
        if st == OK:
            self._keep[t.value] = (P, Q)
        return st, t.value

    def wait(self, ticket: int, timeout_ms: int = -1):
        res = Result()
        st = self.lib.sprot_server_wait(self.h, C.c_uint64(ticket), int(timeout_ms), C.byref(res))
        if st == E_TIMEOUT:
            return None
        check(st, "sprot_server_wait")
        self._keep.pop(ticket, None)
        return dict(status=int(res.status), rotations=[res.rot[a].to_dict() for a in range(res.n_found)],
                    t_submit_ms=res.t_submit_ms, t_admit_ms=res.t_admit_ms, t_done_ms=res.t_done_ms)

    def close(self):
        if self.h:
            check(self.lib.sprot_server_destroy(self.h), "sprot_server_destroy")
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def launch_count() -> int:
    return int(load().sprot_kernel_launch_count())


def probe_smem_atomic_rate(iters: int = 4096, stream=None) -> float:
    r = C.c_double(0.0)
    check(load().sprot_probe_smem_atomic_rate(int(iters), C.byref(r), _stream(stream)),
          "sprot_probe_smem_atomic_rate")
    return r.value


def kernel_timing(enable: bool):
    load().sprot_kernel_timing(1 if enable else 0)


def kernel_timing_read():
    """(total axis-vote kernel milliseconds, launches) since timing was enabled."""
    ms, n = C.c_double(0.0), C.c_uint64(0)
    load().sprot_kernel_timing_read(C.byref(ms), C.byref(n))
    return ms.value, int(n.value)


def release_workspaces():
    load().sprot_release_workspaces()


def release_stream_workspace(stream=None):
    """Frees the library's workspace of ``stream`` (default: the current torch stream); call
    before the stream is destroyed."""
    load().sprot_release_stream_workspace(_stream(stream))
