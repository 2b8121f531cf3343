"""Python binding of libtnep (ctypes): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: it converts numpy arrays or torch tensors into
pointers and sizes, calls the library and raises TnepError on a non-zero
status.  All computation runs in the CUDA kernels of libtnep.so; there is no
CPU fallback, and importing this module fails loudly if the library has not
been built.
"""

from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtnep.so")

TNEP_OK = 0
TNEP_ERR_INVALID = 1
STATUS_NAMES = {
    0: "TNEP_OK", 1: "TNEP_ERR_INVALID", 2: "TNEP_ERR_OOM", 3: "TNEP_ERR_BOX_TOO_SMALL",
    4: "TNEP_ERR_NEIGHBOR_OVERFLOW", 5: "TNEP_ERR_CUDA", 6: "TNEP_ERR_TIMEOUT",
    7: "TNEP_ERR_UNSUPPORTED", 8: "TNEP_ERR_BUSY", 9: "TNEP_ERR_NO_DEVICE",
}
TNEP_SPECTRUM_IR, TNEP_SPECTRUM_RAMAN_ISO, TNEP_SPECTRUM_RAMAN_ANISO = 0, 1, 2
(TNEP_OPT_FRAMES_PER_BATCH, TNEP_OPT_MAX_NEIGHBORS, TNEP_OPT_BLOCK_ATOMS, TNEP_OPT_LAST_KERNEL_MS,
 TNEP_OPT_CELL_DIV, TNEP_OPT_LAST_KERNEL_LAUNCHES, TNEP_OPT_LAST_NBR_MS,
 TNEP_OPT_KERNEL_LAUNCHES_TOTAL, TNEP_OPT_SKIN, TNEP_OPT_LAST_SKIN_USED,
 TNEP_OPT_POPULATION_FORM, TNEP_OPT_CELL_XDIV, TNEP_OPT_ALLOC_COUNT, TNEP_OPT_WAIT_TRIES,
 TNEP_OPT_PAIR_CACHE) = range(15)

# Every symbol include/tnep.h declares (tests check the library exports them).
EXPORTED = [
    "tnep_create", "tnep_destroy", "tnep_last_error", "tnep_output_dim", "tnep_eval",
    "tnep_eval_batch", "tnep_neighbors", "tnep_eval_population", "tnep_spectrum",
    "tnep_set_option", "tnep_get_option", "tnep_spectrum_noalloc",
    "tnep_server_start", "tnep_submit", "tnep_poll", "tnep_wait", "tnep_server_stats", "tnep_server_stop",
    "tnep_population_create", "tnep_population_eval", "tnep_population_info", "tnep_population_destroy",
    "tnep_snes_create", "tnep_snes_run", "tnep_snes_state", "tnep_snes_info", "tnep_snes_destroy",
    "tnep_snes_normals", "tnep_snes_update",
    "tnep_raman_tensor", "tnep_raman_polarized", "tnep_raman_porto_map",
    "tnep_set_masses", "tnep_add_com_dipole", "tnep_eval_batch_cell",
]
TNEP_NOALLOC_MAX_T = 32768


class TnepError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Request(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("pos", C.c_void_p), ("box", C.c_void_p), ("types", C.c_void_p)]


class ModelDesc(C.Structure):
    _fields_ = [
        ("rank", C.c_int), ("n_max_R", C.c_int), ("n_max_A", C.c_int), ("basis_R", C.c_int),
        ("basis_A", C.c_int), ("l_max", C.c_int), ("use_4body", C.c_int), ("n_hidden", C.c_int),
        ("per_type_nn", C.c_int), ("params", C.POINTER(C.c_float)), ("n_params", C.c_size_t),
        ("q_scaler", C.POINTER(C.c_float)), ("mlp_precision", C.c_int),
    ]


class SnesConfig(C.Structure):
    _fields_ = [("n_pop", C.c_int), ("eta_mu", C.c_double), ("eta_sigma", C.c_double),
                ("lambda1", C.c_double), ("lambda2", C.c_double), ("seed", C.c_ulonglong)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run paper_2312_05233_gb300.build.build() first")
    lib = C.CDLL(LIB_PATH)
    vp, ip, fp, dp = C.c_void_p, C.POINTER(C.c_int), C.c_void_p, C.c_void_p
    sig = {
        "tnep_create": (C.c_int, [C.POINTER(ModelDesc), C.c_int, C.c_int, C.POINTER(C.c_char_p),
                                  C.POINTER(C.c_float), C.c_int, C.POINTER(vp)]),
        "tnep_destroy": (None, [vp]),
        "tnep_last_error": (C.c_char_p, []),
        "tnep_output_dim": (C.c_int, [vp, C.c_int]),
        "tnep_eval": (C.c_int, [vp, C.c_int, C.c_int, fp, fp, vp, dp, vp]),
        "tnep_eval_batch": (C.c_int, [vp, C.c_int, ip, fp, fp, vp, dp, fp, vp]),
        "tnep_neighbors": (C.c_int, [vp, C.c_int, ip, fp, fp, vp, vp, vp, C.c_int, vp, C.c_int, vp]),
        "tnep_eval_population": (C.c_int, [vp, C.c_int, C.c_int, fp, C.c_int, ip, fp, fp, vp, dp, dp, dp, vp]),
        "tnep_spectrum": (C.c_int, [dp, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, dp, dp, dp, vp]),
        "tnep_spectrum_noalloc": (C.c_int, [dp, C.c_int, C.c_int, C.c_double, C.c_int, C.c_int, C.c_int, dp, dp,
                                            dp, vp]),
        "tnep_server_start": (C.c_int, [vp, C.c_size_t, C.c_int, C.c_int, C.c_int, C.POINTER(vp)]),
        "tnep_submit": (C.c_int, [vp, C.POINTER(Request), C.POINTER(C.c_uint64)]),
        "tnep_poll": (C.c_int, [vp, C.c_uint64, dp, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
        "tnep_wait": (C.c_int, [vp, C.c_uint64, dp, C.c_double, C.POINTER(C.c_double)]),
        "tnep_server_stats": (C.c_int, [vp, dp]),
        "tnep_server_stop": (None, [vp]),
        "tnep_population_create": (C.c_int, [vp, C.c_int, C.c_int, fp, C.c_int, ip, fp, fp, vp, dp, C.POINTER(vp)]),
        "tnep_population_eval": (C.c_int, [vp, fp, dp, dp]),
        "tnep_population_info": (C.c_int, [vp, dp]),
        "tnep_population_destroy": (None, [vp]),
        "tnep_snes_create": (C.c_int, [vp, C.c_int, C.POINTER(SnesConfig), dp, dp, C.c_int, ip, fp, fp, vp, dp,
                                       C.POINTER(vp)]),
        "tnep_snes_run": (C.c_int, [vp, C.c_int, dp]),
        "tnep_snes_state": (C.c_int, [vp, dp, dp, C.POINTER(C.c_longlong)]),
        "tnep_snes_info": (C.c_int, [vp, dp]),
        "tnep_snes_destroy": (None, [vp]),
        "tnep_snes_normals": (C.c_int, [C.c_ulonglong, C.c_longlong, C.c_int, C.c_int, dp, vp]),
        "tnep_snes_update": (C.c_int, [C.c_int, C.c_int, dp, dp, dp, dp, C.c_double, C.c_double, vp]),
        "tnep_raman_tensor": (C.c_int, [dp, C.c_int, C.c_double, C.c_int, C.c_int, dp, dp, vp]),
        "tnep_raman_polarized": (C.c_int, [dp, C.c_int, C.c_int, dp, dp, dp, vp]),
        "tnep_raman_porto_map": (C.c_int, [dp, C.c_int, C.c_int, dp, C.c_int, dp, dp, vp]),
        "tnep_set_masses": (C.c_int, [vp, dp]),
        "tnep_add_com_dipole": (C.c_int, [vp, C.c_int, ip, fp, fp, vp, dp, dp, C.c_int, vp]),
        "tnep_eval_batch_cell": (C.c_int, [vp, C.c_int, ip, fp, fp, vp, dp, vp]),
        "tnep_set_option": (C.c_int, [vp, C.c_int, C.c_double]),
        "tnep_get_option": (C.c_int, [vp, C.c_int, C.POINTER(C.c_double)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()


def lib():
    return _lib


def _check(status: int):
    if status != TNEP_OK:
        raise TnepError(status, _lib.tnep_last_error().decode(errors="replace"))


# ------------------------------------------------------------------ marshalling
class _Buf:
    """A contiguous buffer and its pointer; keeps host copies alive."""

    def __init__(self, x, dtype, name, writable=False):
        self.obj = None
        self.ptr = None
        if x is None:
            return
        try:
            import torch
            if isinstance(x, torch.Tensor):
                tdt = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32}[dtype]
                if x.dtype != tdt or not x.is_contiguous():
                    if writable:
                        raise TypeError(f"{name} must be a contiguous {tdt} tensor")
                    x = x.to(tdt).contiguous()
                self.obj = x
                self.ptr = x.data_ptr()
                return
        except ImportError:
            pass
        a = np.asarray(x)
        if writable:
            if a.dtype != dtype or not a.flags.c_contiguous or not a.flags.writeable:
                raise TypeError(f"{name} must be a writable C-contiguous {np.dtype(dtype).name} array")
        else:
            a = np.ascontiguousarray(a, dtype=dtype)
        self.obj = a
        self.ptr = a.ctypes.data if a.size else None


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(getattr(stream, "cuda_stream"))


@dataclass
class Model:
    """A model for tnep_create: hyper-parameters plus flat float32 parameters."""

    rank: int
    params: np.ndarray
    n_max_R: int = 4
    n_max_A: int = 4
    basis_R: int = 8
    basis_A: int = 8
    l_max: int = 4
    use_4body: int = 1
    n_hidden: int = 30
    per_type_nn: int = 1
    q_scaler: np.ndarray | None = None
    mlp_precision: int = 0

    @classmethod
    def from_hyper(cls, hp, params, q_scaler=None, mlp_precision=0):
        return cls(rank=hp.rank, params=params, n_max_R=hp.n_max_R, n_max_A=hp.n_max_A,
                   basis_R=hp.basis_R, basis_A=hp.basis_A, l_max=hp.l_max, use_4body=hp.use_4body,
                   n_hidden=hp.n_hidden, per_type_nn=hp.per_type_nn, q_scaler=q_scaler,
                   mlp_precision=mlp_precision)


class Context:
    """Owns a tnep_ctx handle; the methods are the C entry points."""

    def __init__(self, handle, models, n_types):
        self.handle = handle
        self.models = models
        self.n_types = n_types
        self.dims = [_lib.tnep_output_dim(handle, k) for k in range(len(models))]

    def close(self):
        if self.handle:
            _lib.tnep_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def tnep_create(models, n_types: int, cutoffs=(6.0, 4.0), device: int = 0, type_names=None) -> Context:
    models = list(models)
    descs = (ModelDesc * len(models))()
    keep = []
    for k, m in enumerate(models):
        p = np.ascontiguousarray(m.params, dtype=np.float32)
        s = None if m.q_scaler is None else np.ascontiguousarray(m.q_scaler, dtype=np.float32)
        keep += [p, s]
        d = descs[k]
        d.rank, d.n_max_R, d.n_max_A = m.rank, m.n_max_R, m.n_max_A
        d.basis_R, d.basis_A, d.l_max, d.use_4body = m.basis_R, m.basis_A, m.l_max, m.use_4body
        d.n_hidden, d.per_type_nn, d.mlp_precision = m.n_hidden, m.per_type_nn, m.mlp_precision
        d.params = p.ctypes.data_as(C.POINTER(C.c_float))
        d.n_params = p.size
        d.q_scaler = s.ctypes.data_as(C.POINTER(C.c_float)) if s is not None else None
    cut = (C.c_float * 2)(float(cutoffs[0]), float(cutoffs[1]))
    names = None
    if type_names is not None:
        names = (C.c_char_p * len(type_names))(*[n.encode() for n in type_names])
    h = C.c_void_p()
    _check(_lib.tnep_create(descs, len(models), int(n_types), names, cut, int(device), C.byref(h)))
    return Context(h, models, n_types)


def tnep_set_option(ctx: Context, option: int, value: float):
    _check(_lib.tnep_set_option(ctx.handle, int(option), float(value)))


def tnep_get_option(ctx: Context, option: int) -> float:
    v = C.c_double()
    _check(_lib.tnep_get_option(ctx.handle, int(option), C.byref(v)))
    return v.value


def _alloc_out(like_device, shape, dtype):
    if like_device is not None:
        import torch
        return torch.empty(shape, dtype={np.float64: torch.float64, np.float32: torch.float32}[dtype],
                           device=like_device)
    return np.empty(shape, dtype=dtype)


def _device_of(x):
    try:
        import torch
        if isinstance(x, torch.Tensor) and x.is_cuda:
            return x.device
    except ImportError:
        pass
    return None


def tnep_eval(ctx: Context, pos, box, types, out=None, stream=None):
    """pos [F][N][3], box [F][3] or [3] or None, types [N] -> out [n_models][F][C] blocks.

    Returns a list with one [F][C_m] array (or tensor) per model."""
    shp = tuple(pos.shape)
    F, N = int(shp[0]), int(shp[1])
    if box is not None and np.ndim(np.asarray(box.cpu() if hasattr(box, "cpu") else box)) == 1:
        b = np.asarray(box.cpu() if hasattr(box, "cpu") else box, dtype=np.float32)
        box = np.ascontiguousarray(np.broadcast_to(b, (F, 3)))
    P = _Buf(pos, np.float32, "pos")
    B = _Buf(box, np.float32, "box")
    T = _Buf(types, np.int32, "types")
    tot = sum(ctx.dims)
    if out is None:
        out = _alloc_out(_device_of(pos), (F * tot,), np.float64)
    O = _Buf(out, np.float64, "out", writable=True)
    _check(_lib.tnep_eval(ctx.handle, F, N, P.ptr, B.ptr, T.ptr, O.ptr, _stream_ptr(stream)))
    res, off = [], 0
    for c in ctx.dims:
        res.append(out[off:off + F * c].reshape(F, c))
        off += F * c
    return res


def tnep_eval_batch(ctx: Context, offsets, pos, box, types, per_atom=False, out=None, stream=None):
    """Uneven structures: offsets [S+1] (host), pos [N][3], box [S][3] or None, types [N].

    Returns (list of [S][C_m], list of [N][C_m] per-atom arrays or None)."""
    offs = np.ascontiguousarray(offsets, dtype=np.int32)
    S = len(offs) - 1
    N = int(offs[-1])
    P = _Buf(pos, np.float32, "pos")
    B = _Buf(box, np.float32, "box")
    T = _Buf(types, np.int32, "types")
    tot = sum(ctx.dims)
    dev = _device_of(pos)
    if out is None:
        out = _alloc_out(dev, (S * tot,), np.float64)
    O = _Buf(out, np.float64, "out", writable=True)
    pa = _alloc_out(dev, (N * tot,), np.float32) if per_atom else None
    PA = _Buf(pa, np.float32, "per_atom", writable=True)
    _check(_lib.tnep_eval_batch(ctx.handle, S, offs.ctypes.data_as(C.POINTER(C.c_int)), P.ptr, B.ptr, T.ptr,
                                O.ptr, PA.ptr if per_atom else None, _stream_ptr(stream)))
    res, pres, off, poff = [], [], 0, 0
    for c in ctx.dims:
        res.append(out[off:off + S * c].reshape(S, c))
        off += S * c
        if per_atom:
            pres.append(pa[poff:poff + N * c].reshape(N, c))
            poff += N * c
    return res, (pres if per_atom else None)


def tnep_eval_batch_cell(ctx: Context, offsets, pos, cell, types, stream=None):
    """General periodic cells: cell [S][3][3] (rows = lattice vectors, zeros = open) or None.

    Returns a list of [S][C_m] arrays, one per model."""
    offs = np.ascontiguousarray(offsets, dtype=np.int32)
    S = len(offs) - 1
    P = _Buf(pos, np.float32, "pos")
    H = _Buf(None if cell is None else np.asarray(cell, dtype=np.float32).reshape(S, 9), np.float32, "cell")
    T = _Buf(types, np.int32, "types")
    tot = sum(ctx.dims)
    out = np.zeros(S * tot)
    _check(_lib.tnep_eval_batch_cell(ctx.handle, S, offs.ctypes.data_as(C.POINTER(C.c_int)), P.ptr, H.ptr, T.ptr,
                                     out.ctypes.data, _stream_ptr(stream)))
    res, off = [], 0
    for c in ctx.dims:
        res.append(out[off:off + S * c].reshape(S, c))
        off += S * c
    return res


def tnep_neighbors(ctx: Context, offsets, pos, box, cap_R=256, cap_A=128, stream=None):
    """Returns (counts_R [N], counts_A [N], list_R [N][cap_R], list_A [N][cap_A]) as numpy."""
    offs = np.ascontiguousarray(offsets, dtype=np.int32)
    S = len(offs) - 1
    N = int(offs[-1])
    P = _Buf(pos, np.float32, "pos")
    B = _Buf(box, np.float32, "box")
    cR = np.zeros(N, np.int32)
    cA = np.zeros(N, np.int32)
    lR = np.full((N, cap_R), -1, np.int32)
    lA = np.full((N, cap_A), -1, np.int32)
    _check(_lib.tnep_neighbors(ctx.handle, S, offs.ctypes.data_as(C.POINTER(C.c_int)), P.ptr, B.ptr,
                               cR.ctypes.data, cA.ctypes.data, lR.ctypes.data, cap_R, lA.ctypes.data, cap_A,
                               _stream_ptr(stream)))
    return cR, cA, lR, lA


def tnep_eval_population(ctx: Context, model: int, params, offsets, pos, box, types, target,
                         want_out=False, stream=None):
    """params [P][n_params] (host) -> (rmse [P], predictions [P][S][C] or None)."""
    prm = np.ascontiguousarray(params, dtype=np.float32)
    Pn = prm.shape[0]
    offs = np.ascontiguousarray(offsets, dtype=np.int32)
    S = len(offs) - 1
    c = ctx.dims[model]
    P = _Buf(pos, np.float32, "pos")
    B = _Buf(box, np.float32, "box")
    T = _Buf(types, np.int32, "types")
    TG = _Buf(target, np.float64, "target")
    rmse = np.zeros(Pn, np.float64)
    out = np.zeros((Pn, S, c), np.float64) if want_out else None
    _check(_lib.tnep_eval_population(ctx.handle, int(model), Pn, prm.ctypes.data, S,
                                     offs.ctypes.data_as(C.POINTER(C.c_int)), P.ptr, B.ptr, T.ptr, TG.ptr,
                                     rmse.ctypes.data, out.ctypes.data if want_out else None,
                                     _stream_ptr(stream)))
    return rmse, out


def tnep_spectrum(series, dt_fs: float, kind: int = TNEP_SPECTRUM_IR, max_lag: int = 0, subtract_mean=True,
                  want_acf=False, stream=None):
    """series [T][3 or 9] float64 (host or device) -> (freq_cm1, spec[, acf]) numpy."""
    S = _Buf(series, np.float64, "series")
    Tn, Cn = int(series.shape[0]), int(series.shape[1])
    M = Tn // 2 if max_lag <= 0 else int(max_lag)
    freq = np.zeros(M + 1)
    spec = np.zeros(M + 1)
    acf = np.zeros(M + 1) if want_acf else None
    _check(_lib.tnep_spectrum(S.ptr, Tn, Cn, float(dt_fs), int(kind), int(max_lag), int(bool(subtract_mean)),
                              freq.ctypes.data, spec.ctypes.data, acf.ctypes.data if want_acf else None,
                              _stream_ptr(stream)))
    return (freq, spec, acf) if want_acf else (freq, spec)


def tnep_spectrum_noalloc(series, dt_fs: float, kind: int, freq_out, spec_out, acf_out=None, max_lag: int = 0,
                          subtract_mean=True, stream=None):
    """Device series [T][C] -> fills the device tensors freq_out, spec_out (and acf_out).

    Asynchronous on `stream`; uses the library's static scratch (no allocation).
    The C entry point cannot see buffer lengths, so this wrapper checks them
    before the call: series must be a contiguous 2-D float64 CUDA tensor (no
    converted temporary, which could be freed while the call still reads it),
    and every output a contiguous float64 tensor on the same device with at
    least M + 1 elements, M = max_lag or T // 2."""
    import torch
    if not isinstance(series, torch.Tensor) or series.dim() != 2:
        raise TnepError(TNEP_ERR_INVALID, "series must be a 2-D [T][C] tensor")
    if series.dtype != torch.float64 or not series.is_contiguous():
        raise TypeError("series must be a contiguous torch.float64 tensor")
    Tn, Cn = int(series.shape[0]), int(series.shape[1])
    M = Tn // 2 if max_lag <= 0 else int(max_lag)
    outs = [("freq_out", freq_out), ("spec_out", spec_out)] + ([("acf_out", acf_out)] if acf_out is not None else [])
    for name, t in outs:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if t.numel() < M + 1:
            raise TnepError(TNEP_ERR_INVALID, f"{name} holds {t.numel()} elements, needs M + 1 = {M + 1}")
    if series.device.type != "cuda":
        raise TnepError(TNEP_ERR_INVALID, "series must be a CUDA tensor")
    for name, t in outs:
        if t.device != series.device:
            raise TnepError(TNEP_ERR_INVALID, f"{name} is on {t.device}, series on {series.device}")
    S = _Buf(series, np.float64, "series")
    F = _Buf(freq_out, np.float64, "freq_out", writable=True)
    P = _Buf(spec_out, np.float64, "spec_out", writable=True)
    A = _Buf(acf_out, np.float64, "acf_out", writable=True)
    _check(_lib.tnep_spectrum_noalloc(S.ptr, Tn, Cn, float(dt_fs), int(kind), int(max_lag),
                                      int(bool(subtract_mean)), F.ptr, P.ptr, A.ptr, _stream_ptr(stream)))


TNEP_ERR_BUSY = 8
TNEP_ERR_TIMEOUT = 6


class Server:
    """Owns a tnep_server handle (continuous-batching serving loop)."""

    def __init__(self, handle, ctx):
        self.handle = handle
        self.ctx = ctx
        self.width = sum(ctx.dims)

    def submit(self, pos, types, box=None):
        """Returns a ticket, or None when the request is not admitted (BUSY)."""
        p = np.ascontiguousarray(pos, dtype=np.float32)
        t = np.ascontiguousarray(types, dtype=np.int32)
        b = None if box is None else np.ascontiguousarray(box, dtype=np.float32)
        req = Request(len(t), p.ctypes.data if p.size else None, b.ctypes.data if b is not None else None,
                      t.ctypes.data if t.size else None)
        tk = C.c_uint64()
        st = _lib.tnep_submit(self.handle, C.byref(req), C.byref(tk))
        if st == TNEP_ERR_BUSY:
            return None
        _check(st)
        return tk.value

    def poll(self, ticket):
        """(done, result [width] or None, latency_s)."""
        out = np.zeros(self.width)
        done = C.c_int()
        lat = C.c_double()
        _check(_lib.tnep_poll(self.handle, C.c_uint64(ticket), out.ctypes.data, C.byref(done), C.byref(lat)))
        return (bool(done.value), out if done.value else None, lat.value)

    def wait(self, ticket, timeout_s=60.0):
        """(result [width], latency_s); raises TnepError(TIMEOUT) when not finished in time."""
        out = np.zeros(self.width)
        lat = C.c_double()
        _check(_lib.tnep_wait(self.handle, C.c_uint64(ticket), out.ctypes.data, float(timeout_s), C.byref(lat)))
        return out, lat.value

    def stats(self):
        st = np.zeros(6)
        _check(_lib.tnep_server_stats(self.handle, st.ctypes.data))
        return dict(completed=st[0], batches=st[1], atoms=st[2], bytes_in_use=st[3], inflight=st[4],
                    pending=st[5])

    def stop(self):
        if self.handle:
            _lib.tnep_server_stop(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()


def tnep_server_start(ctx: Context, mem_budget_bytes: int = 8 << 30, max_slots: int = 4096, n_pipelines: int = 3,
                      max_batch_atoms: int = 1 << 19) -> Server:
    h = C.c_void_p()
    _check(_lib.tnep_server_start(ctx.handle, int(mem_budget_bytes), int(max_slots), int(n_pipelines),
                                  int(max_batch_atoms), C.byref(h)))
    return Server(h, ctx)


class Population:
    """Owns a tnep_population handle: resident structures, graph-captured generations."""

    def __init__(self, handle, n_pop, n_structs, width):
        self.handle = handle
        self.n_pop, self.n_structs, self.width = n_pop, n_structs, width

    def eval(self, params, want_out=False):
        prm = np.ascontiguousarray(params, dtype=np.float32)
        assert prm.shape[0] == self.n_pop
        rmse = np.zeros(self.n_pop)
        out = np.zeros((self.n_pop, self.n_structs, self.width)) if want_out else None
        _check(_lib.tnep_population_eval(self.handle, prm.ctypes.data, rmse.ctypes.data,
                                         out.ctypes.data if want_out else None))
        return rmse, out

    def info(self):
        v = np.zeros(14)
        _check(_lib.tnep_population_info(self.handle, v.ctypes.data))
        return dict(block=int(v[0]), pop_major=int(v[1]), factored=int(v[2]), tune_ms=v[3:11].tolist(),
                    last_ms=v[11], atoms=int(v[12]), tensor_core_ms=v[13])

    def close(self):
        if self.handle:
            _lib.tnep_population_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tnep_population_create(ctx: Context, model: int, params, offsets, pos, box, types, target) -> Population:
    prm = np.ascontiguousarray(params, dtype=np.float32)
    offs = np.ascontiguousarray(offsets, dtype=np.int32)
    S = len(offs) - 1
    P = _Buf(pos, np.float32, "pos")
    B = _Buf(box, np.float32, "box")
    T = _Buf(types, np.int32, "types")
    TG = _Buf(target, np.float64, "target")
    h = C.c_void_p()
    _check(_lib.tnep_population_create(ctx.handle, int(model), prm.shape[0], prm.ctypes.data, S,
                                       offs.ctypes.data_as(C.POINTER(C.c_int)), P.ptr, B.ptr, T.ptr, TG.ptr,
                                       C.byref(h)))
    return Population(h, prm.shape[0], S, ctx.dims[model])


class Snes:
    """Owns a tnep_snes handle: the SNES training loop on resident structures."""

    def __init__(self, handle, n_pop, dim):
        self.handle = handle
        self.n_pop, self.dim = n_pop, dim

    def run(self, n_gen):
        """Runs n_gen generations; returns history [n_gen][3] (best loss, its RMSE, mean loss)."""
        hist = np.zeros((max(int(n_gen), 0), 3))
        _check(_lib.tnep_snes_run(self.handle, int(n_gen), hist.ctypes.data if n_gen > 0 else None))
        return hist

    def state(self):
        mu = np.zeros(self.dim)
        sigma = np.zeros(self.dim)
        g = C.c_longlong()
        _check(_lib.tnep_snes_state(self.handle, mu.ctypes.data, sigma.ctypes.data, C.byref(g)))
        return mu, sigma, g.value

    def info(self):
        v = np.zeros(4)
        _check(_lib.tnep_snes_info(self.handle, v.ctypes.data))
        return dict(generation=int(v[0]), dim=int(v[1]), n_pop=int(v[2]), ms_per_generation=v[3])

    def close(self):
        if self.handle:
            _lib.tnep_snes_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tnep_snes_create(ctx: Context, model: int, n_pop, mu0, sigma0, offsets, pos, box, types, target,
                     seed=0, eta_mu=0.0, eta_sigma=0.0, lambda1=0.0, lambda2=0.0) -> Snes:
    mu = np.ascontiguousarray(mu0, dtype=np.float64)
    sg = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma0, dtype=np.float64), mu.shape))
    offs = np.ascontiguousarray(offsets, dtype=np.int32)
    S = len(offs) - 1
    P = _Buf(pos, np.float32, "pos")
    B = _Buf(box, np.float32, "box")
    T = _Buf(types, np.int32, "types")
    TG = _Buf(target, np.float64, "target")
    cfg = SnesConfig(int(n_pop), float(eta_mu), float(eta_sigma), float(lambda1), float(lambda2), int(seed))
    h = C.c_void_p()
    _check(_lib.tnep_snes_create(ctx.handle, int(model), C.byref(cfg), mu.ctypes.data, sg.ctypes.data, S,
                                 offs.ctypes.data_as(C.POINTER(C.c_int)), P.ptr, B.ptr, T.ptr, TG.ptr,
                                 C.byref(h)))
    return Snes(h, int(n_pop), mu.size)


def tnep_snes_normals(seed, generation, n_pop, dim, s, stream=None):
    """Fills the device tensor s [n_pop][dim] (float64) with the generation's normals."""
    S = _Buf(s, np.float64, "s", writable=True)
    _check(_lib.tnep_snes_normals(int(seed), int(generation), int(n_pop), int(dim), S.ptr, _stream_ptr(stream)))


def tnep_snes_update(loss, s, mu, sigma, eta_mu=1.0, eta_sigma=0.0, stream=None):
    """In-place SNES update of the device tensors mu, sigma [dim] from s [P][dim] and loss [P]."""
    L = _Buf(loss, np.float64, "loss")
    S = _Buf(s, np.float64, "s")
    M = _Buf(mu, np.float64, "mu", writable=True)
    G = _Buf(sigma, np.float64, "sigma", writable=True)
    n_pop, dim = int(np.shape(s)[0]) if s is not None else 0, int(np.shape(s)[1]) if s is not None else 0
    _check(_lib.tnep_snes_update(n_pop, dim, L.ptr, S.ptr, M.ptr, G.ptr, float(eta_mu), float(eta_sigma),
                                 _stream_ptr(stream)))


def tnep_raman_tensor(series, dt_fs, max_lag=0, subtract_mean=True, stream=None):
    """Returns (freq_cm1 [M+1], L [M+1][9][9]) as numpy arrays."""
    S = _Buf(series, np.float64, "series")
    T = int(np.shape(series)[0])
    M = int(max_lag) if max_lag and max_lag > 0 else T // 2
    freq = np.zeros(M + 1)
    L = np.zeros((M + 1, 9, 9))
    _check(_lib.tnep_raman_tensor(S.ptr, T, float(dt_fs), M, int(bool(subtract_mean)), freq.ctypes.data,
                                  L.ctypes.data, _stream_ptr(stream)))
    return freq, L


def tnep_raman_polarized(L, n, eps, stream=None):
    """spec [n_orient][M+1] for the rows of n and eps."""
    Lb = _Buf(L, np.float64, "L")
    nb = _Buf(np.atleast_2d(np.asarray(n, dtype=np.float64)), np.float64, "n")
    eb = _Buf(np.atleast_2d(np.asarray(eps, dtype=np.float64)), np.float64, "eps")
    M = int(np.shape(L)[0]) - 1
    O = nb.obj.shape[0]
    if eb.obj.shape[0] != O:
        raise ValueError("n and eps need the same number of rows")
    out = np.zeros((O, M + 1))
    _check(_lib.tnep_raman_polarized(Lb.ptr, M, O, nb.ptr, eb.ptr, out.ctypes.data, _stream_ptr(stream)))
    return out


def tnep_raman_porto_map(L, thetas, axis=2, stream=None):
    """(parallel, crossed) spectra [n_theta][M+1] for crystal rotations theta (rad) about `axis`."""
    Lb = _Buf(L, np.float64, "L")
    th = _Buf(np.atleast_1d(np.asarray(thetas, dtype=np.float64)), np.float64, "thetas")
    M = int(np.shape(L)[0]) - 1
    O = th.obj.shape[0]
    par = np.zeros((O, M + 1))
    crs = np.zeros((O, M + 1))
    _check(_lib.tnep_raman_porto_map(Lb.ptr, M, O, th.ptr, int(axis), par.ctypes.data, crs.ctypes.data,
                                     _stream_ptr(stream)))
    return par, crs


def tnep_set_masses(ctx, masses):
    m = np.ascontiguousarray(masses, dtype=np.float64)
    _check(_lib.tnep_set_masses(ctx.handle, m.ctypes.data))


def tnep_add_com_dipole(ctx, offsets, pos, box, types, charge, mu, col=0, stream=None):
    """mu [S][W] float64 (contiguous, writable; columns col..col+2 hold the
    dipole, e.g. the output of tnep_eval_batch) gets Q r_COM added in place."""
    offs = np.ascontiguousarray(offsets, dtype=np.int32)
    S = len(offs) - 1
    P = _Buf(pos, np.float32, "pos")
    B = _Buf(box, np.float32, "box")
    T = _Buf(types, np.int32, "types")
    Q = _Buf(charge, np.float64, "charge")
    M = _Buf(mu, np.float64, "mu", writable=True)
    _check(_lib.tnep_add_com_dipole(ctx.handle, S, offs.ctypes.data_as(C.POINTER(C.c_int)), P.ptr, B.ptr, T.ptr,
                                    Q.ptr, M.ptr + 8 * int(col), int(np.shape(mu)[1]), _stream_ptr(stream)))
