"""Thin ctypes binding of libshearseg.so (the C ABI in include/shearseg.h).

Argument marshalling only: every function here forwards to the entry point of
the same name, raising ``ShearsegError`` on a negative status.  Pointers are
plain integers (``tensor.data_ptr()`` for device memory, numpy ``ctypes.data``
for host memory); streams are integers (``torch.cuda.current_stream().cuda_stream``)
or None.  There is no fallback: if the library cannot be loaded, every call
raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

SHF_OK = 0
SHF_ERR_ARG = -1
SHF_ERR_SIZE = -2
SHF_ERR_OOM = -3
SHF_ERR_CUDA = -4
SHF_ERR_NONFINITE = -5
SHF_ERR_TIMEOUT = -6
SHF_ERR_STATE = -7
SHF_ERR_IO = -8

SEG_U, SEG_W, SEG_BW, SEG_BV, SEG_S, SEG_LABELS, SEG_GAP, SEG_ENERGY, SEG_ITER, SEG_STV, SEG_V = range(11)

_lock = threading.Lock()
_lib = None


class ShearsegError(RuntimeError):
    def __init__(self, fn: str, code: int, msg: str):
        super().__init__(f"{fn} failed with status {code}: {msg}")
        self.code = code


class seg_params(ctypes.Structure):
    _fields_ = [
        ("gamma", ctypes.c_float),
        ("J", ctypes.c_int),
        ("Lambda", ctypes.POINTER(ctypes.c_float)),
        ("max_iters", ctypes.c_int),
        ("tol", ctypes.c_float),
        ("check_every", ctypes.c_int),
    ]


class tv_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_float), ("lambda_", ctypes.c_float), ("per_label", ctypes.c_int)]


class nl_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_float), ("lambda_", ctypes.c_float), ("patch", ctypes.c_int),
                ("window", ctypes.c_int), ("a", ctypes.c_float), ("neighbours", ctypes.c_int),
                ("solve_steps", ctypes.c_int)]


_VP = ctypes.c_void_p
_I = ctypes.c_int


class seg_plan(ctypes.Structure):
    _fields_ = [("fast", ctypes.c_int), ("wave_mib", ctypes.c_int), ("col_ctas_per_sm", ctypes.c_int),
                ("tile_cols", ctypes.c_int), ("tile_rows", ctypes.c_int), ("groups", ctypes.c_int),
                ("us_per_iter", ctypes.c_float), ("row_kernel", ctypes.c_int), ("col_kernel", ctypes.c_int),
                ("serial", ctypes.c_int), ("sms", ctypes.c_int)]


_PLAN_FIELDS = ("fast", "wave_mib", "col_ctas_per_sm", "tile_cols", "tile_rows", "groups", "us_per_iter",
                "row_kernel", "col_kernel", "serial", "sms")

_SIG = {
    "shf_version": (_I, []),
    "shf_last_error": (ctypes.c_char_p, []),
    "shfilters_build": (_I, [_I, _I, _I, _VP, ctypes.POINTER(_VP)]),
    "shfilters_destroy": (_I, [_VP]),
    "shfilters_info": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "shfilters_copy": (_I, [_VP, _VP, _VP]),
    "shearlet_analyze": (_I, [_VP, _VP, _I, _VP, _VP]),
    "shearlet_synthesize": (_I, [_VP, _VP, _I, _VP, _VP]),
    "shearlet_analyze_noalloc": (_I, [_VP, _VP, _I, _VP, _VP]),
    "seg_admm_init": (_I, [_VP, _VP, _I, ctypes.POINTER(ctypes.c_float), _I, ctypes.POINTER(seg_params), _VP,
                           ctypes.POINTER(_VP)]),
    "seg_admm_reset": (_I, [_VP, _VP, _I]),
    "seg_admm_step": (_I, [_VP, _I]),
    "seg_admm_solve": (_I, [_VP, ctypes.POINTER(_I), ctypes.POINTER(ctypes.c_float)]),
    "seg_admm_get": (_I, [_VP, _I, _VP, _I]),
    "seg_admm_set": (_I, [_VP, _I, _VP, _I]),
    "seg_admm_save": (_I, [_VP, ctypes.c_char_p]),
    "seg_admm_load": (_I, [_VP, ctypes.c_char_p]),
    "seg_admm_kernel_times": (_I, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "seg_admm_kernel_name": (ctypes.c_char_p, [_I]),
    "seg_admm_batch_init": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I),
                                 ctypes.POINTER(_VP), ctypes.POINTER(_VP), _VP, _VP, ctypes.POINTER(_VP)]),
    "seg_admm_batch_step": (_I, [_VP, _I]),
    "seg_admm_batch_image": (_I, [_VP, _I, ctypes.POINTER(_VP)]),
    "seg_admm_batch_sync": (_I, [_VP]),
    "seg_admm_batch_destroy": (_I, [_VP]),
    "seg_admm_unrolled_fwd": (_I, [_VP, _I, _I]),
    "seg_admm_unrolled_bwd": (_I, [_VP, _VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _VP,
                                   _VP]),
    "seg_admm_get_plan": (_I, [_VP, ctypes.POINTER(seg_plan)]),
    "seg_admm_set_plan": (_I, [_VP, ctypes.POINTER(seg_plan)]),
    "seg_admm_tune": (_I, [_VP, _I, ctypes.POINTER(seg_plan)]),
    "seg_admm_batch_tune": (_I, [_VP, _I]),
    "seg_admm_batch_set_lanes": (_I, [_VP, _I]),
    "seg_admm_batch_get_lanes": (_I, [_VP, ctypes.POINTER(_I)]),
    "seg_admm_unrolled_bwd_enqueue": (_I, [_VP, _VP]),
    "seg_admm_unrolled_grads": (_I, [_VP, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float), _VP, _VP]),
    "seg_admm_sync": (_I, [_VP]),
    "seg_admm_destroy": (_I, [_VP]),
    "tv_admm_init": (_I, [_I, _I, _VP, _I, ctypes.POINTER(ctypes.c_float), _I, ctypes.POINTER(tv_params), _VP,
                          ctypes.POINTER(_VP)]),
    "tv_admm_reset": (_I, [_VP, _VP, _I]),
    "tv_admm_step": (_I, [_VP, _I]),
    "tv_admm_get": (_I, [_VP, _I, _VP, _I]),
    "tv_admm_set": (_I, [_VP, _I, _VP, _I]),
    "tv_admm_kernel_times": (_I, [_VP, _I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I)]),
    "tv_admm_kernel_name": (ctypes.c_char_p, [_I]),
    "tv_admm_sync": (_I, [_VP]),
    "tv_admm_destroy": (_I, [_VP]),
    "nl_admm_init": (_I, [_I, _I, _VP, _I, ctypes.POINTER(ctypes.c_float), _I, ctypes.POINTER(nl_params), _VP,
                          ctypes.POINTER(_VP)]),
    "nl_admm_reset": (_I, [_VP, _VP, _I]),
    "nl_admm_graph": (_I, [_VP, _VP, _VP, ctypes.POINTER(_I)]),
    "nl_admm_step": (_I, [_VP, _I]),
    "nl_admm_get": (_I, [_VP, _I, _VP, _I]),
    "nl_admm_set": (_I, [_VP, _I, _VP, _I]),
    "nl_admm_kernel_times": (_I, [_VP, _I, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_I)]),
    "nl_admm_kernel_name": (ctypes.c_char_p, [_I]),
    "nl_admm_sync": (_I, [_VP]),
    "nl_admm_barrier_selftest": (_I, [_VP]),
    "nl_admm_destroy": (_I, [_VP]),
}


def library_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True):
    """Loads libshearseg.so (building it first when missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            if build_if_missing and not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"libshearseg.so not found at {_build.LIB}; run paper_1112_1805_gb300.build")
            L = ctypes.CDLL(_build.LIB)
            for name, (res, args) in _SIG.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _call(name: str, *args) -> None:
    L = lib()
    rc = getattr(L, name)(*args)
    if rc != SHF_OK:
        raise ShearsegError(name, rc, L.shf_last_error().decode(errors="replace"))


def _stream(stream):
    return None if stream is None else ctypes.c_void_p(int(stream))


def shf_version() -> int:
    return int(lib().shf_version())


def shf_last_error() -> str:
    return lib().shf_last_error().decode(errors="replace")


def shfilters_build(H: int, W: int, J: int, stream=None) -> int:
    out = _VP()
    _call("shfilters_build", H, W, J, _stream(stream), ctypes.byref(out))
    return out.value


def shfilters_destroy(bank: int) -> None:
    _call("shfilters_destroy", _VP(bank))


def shfilters_info(bank: int):
    eta, H, W, J = _I(), _I(), _I(), _I()
    _call("shfilters_info", _VP(bank), ctypes.byref(eta), ctypes.byref(H), ctypes.byref(W), ctypes.byref(J))
    return eta.value, H.value, W.value, J.value


def shfilters_copy(bank: int, dst: int, stream=None) -> None:
    _call("shfilters_copy", _VP(bank), _VP(dst), _stream(stream))


def shearlet_analyze(bank: int, u: int, nch: int, coef: int, stream=None) -> None:
    _call("shearlet_analyze", _VP(bank), _VP(u), nch, _VP(coef), _stream(stream))


def shearlet_analyze_noalloc(bank: int, u: int, nch: int, coef: int, stream=None) -> None:
    """shearlet_analyze with its temporaries in the library's fixed 32 MiB
    device array instead of freshly allocated memory (for callers that must
    not allocate); overlapping calls on one GPU race on that array."""
    _call("shearlet_analyze_noalloc", _VP(bank), _VP(u), nch, _VP(coef), _stream(stream))


def shearlet_synthesize(bank: int, coef: int, nch: int, u: int, stream=None) -> None:
    _call("shearlet_synthesize", _VP(bank), _VP(coef), nch, _VP(u), _stream(stream))


def make_params(gamma: float, J: int, Lambda, max_iters: int = 0, tol: float = 0.0, check_every: int = 1):
    """Returns (seg_params, keepalive) -- keep the second item alive while the
    struct is in use (it owns the Lambda array)."""
    vals = [float(x) for x in Lambda]
    if len(vals) != J + 1:
        raise ValueError(f"Lambda needs J + 1 = {J + 1} weights, got {len(vals)}")
    lam = (ctypes.c_float * (J + 1))(*vals)
    p = seg_params(float(gamma), int(J), ctypes.cast(lam, ctypes.POINTER(ctypes.c_float)), int(max_iters),
                   float(tol), int(check_every))
    return p, lam


def seg_admm_init(bank: int, f: int, C: int, codebook, K: int, params, stream=None) -> int:
    """codebook: host sequence of K*C floats (label-major)."""
    cb = (ctypes.c_float * (K * C))(*[float(x) for x in codebook])
    out = _VP()
    _call("seg_admm_init", _VP(bank), _VP(f), C, cb, K, ctypes.byref(params), _stream(stream), ctypes.byref(out))
    return out.value


def seg_admm_reset(state: int, f: int, f_on_host: bool) -> None:
    _call("seg_admm_reset", _VP(state), _VP(f), int(bool(f_on_host)))


def seg_admm_step(state: int, n_iters: int) -> None:
    _call("seg_admm_step", _VP(state), int(n_iters))


def seg_admm_solve(state: int):
    it, res = _I(), ctypes.c_float()
    _call("seg_admm_solve", _VP(state), ctypes.byref(it), ctypes.byref(res))
    return it.value, res.value


def seg_admm_get(state: int, what: int, dst: int, dst_on_host: bool) -> None:
    _call("seg_admm_get", _VP(state), int(what), _VP(dst), int(bool(dst_on_host)))


def seg_admm_set(state: int, what: int, src: int, src_on_host: bool) -> None:
    _call("seg_admm_set", _VP(state), int(what), _VP(src), int(bool(src_on_host)))


def seg_admm_save(state: int, path: str) -> None:
    _call("seg_admm_save", _VP(state), path.encode())


def seg_admm_load(state: int, path: str) -> None:
    _call("seg_admm_load", _VP(state), path.encode())


def seg_admm_kernel_times(state: int):
    """{kernel kind: (milliseconds, launches)} for the most recent iteration."""
    ms = (ctypes.c_float * 8)()
    nl = (_I * 8)()
    nk = _I()
    _call("seg_admm_kernel_times", _VP(state), ms, nl, ctypes.byref(nk))
    return {lib().seg_admm_kernel_name(i).decode(): (float(ms[i]), int(nl[i])) for i in range(nk.value)}


def seg_admm_kernel_name(i: int) -> str:
    return lib().seg_admm_kernel_name(int(i)).decode()


def _plan_dict(p: seg_plan) -> dict:
    return {k: getattr(p, k) for k in _PLAN_FIELDS}


def seg_admm_get_plan(state: int) -> dict:
    p = seg_plan()
    _call("seg_admm_get_plan", state, ctypes.byref(p))
    return _plan_dict(p)


def seg_admm_set_plan(state: int, plan: dict) -> None:
    p = seg_plan()
    for k in _PLAN_FIELDS:
        if k in plan:
            setattr(p, k, plan[k])
    _call("seg_admm_set_plan", state, ctypes.byref(p))


def seg_admm_tune(state: int, iters: int = 5) -> dict:
    p = seg_plan()
    _call("seg_admm_tune", state, iters, ctypes.byref(p))
    return _plan_dict(p)


def seg_admm_batch_tune(batch: int, iters: int = 5) -> None:
    _call("seg_admm_batch_tune", batch, iters)


def seg_admm_batch_set_lanes(batch: int, lanes: int) -> None:
    _call("seg_admm_batch_set_lanes", _VP(batch), int(lanes))


def seg_admm_batch_get_lanes(batch: int) -> int:
    out = _I()
    _call("seg_admm_batch_get_lanes", _VP(batch), ctypes.byref(out))
    return int(out.value)


def seg_admm_sync(state: int) -> None:
    _call("seg_admm_sync", _VP(state))


def seg_admm_destroy(state: int) -> None:
    _call("seg_admm_destroy", _VP(state))


def seg_admm_batch_init(H, W, C, K, f_ptrs, codebooks, params_list, stream=None) -> int:
    """Batch of len(H) images.  f_ptrs: device pointers; codebooks: host sequences
    (K_i*C_i floats each); params_list: seg_params structs (their Lambda arrays
    must stay alive)."""
    n = len(H)
    arr = lambda xs: (_I * n)(*[int(x) for x in xs])  # noqa: E731
    fp = (_VP * n)(*[int(p) for p in f_ptrs])
    cbs = [(ctypes.c_float * len(c))(*[float(x) for x in c]) for c in codebooks]
    cbp = (_VP * n)(*[ctypes.cast(c, _VP) for c in cbs])
    prm = (seg_params * n)(*params_list)
    out = _VP()
    _call("seg_admm_batch_init", n, arr(H), arr(W), arr(C), arr(K), fp, cbp, ctypes.cast(prm, _VP),
          _stream(stream), ctypes.byref(out))
    return out.value


def seg_admm_batch_step(batch: int, n_iters: int) -> None:
    _call("seg_admm_batch_step", _VP(batch), int(n_iters))


def seg_admm_batch_image(batch: int, i: int) -> int:
    out = _VP()
    _call("seg_admm_batch_image", _VP(batch), int(i), ctypes.byref(out))
    return out.value


def seg_admm_batch_sync(batch: int) -> None:
    _call("seg_admm_batch_sync", _VP(batch))


def seg_admm_batch_destroy(batch: int) -> None:
    _call("seg_admm_batch_destroy", _VP(batch))


def seg_admm_unrolled_fwd(state: int, T: int, ckpt_every: int) -> None:
    _call("seg_admm_unrolled_fwd", _VP(state), int(T), int(ckpt_every))


def seg_admm_unrolled_bwd(state: int, dL_dw: int, K: int, C: int, J: int, dL_df: int = 0, dL_ds: int = 0):
    """Returns (dL/dcodebook [K*C], dL/dLambda [J+1]) as Python lists; dL_df and
    dL_ds are optional device pointers that receive the image and data-term
    adjoints."""
    dc = (ctypes.c_float * (K * C))()
    dl = (ctypes.c_float * (J + 1))()
    _call("seg_admm_unrolled_bwd", _VP(state), _VP(dL_dw), dc, dl, _VP(dL_df) if dL_df else None,
          _VP(dL_ds) if dL_ds else None)
    return list(dc), list(dl)


def seg_admm_unrolled_bwd_enqueue(state: int, dL_dw: int) -> None:
    _call("seg_admm_unrolled_bwd_enqueue", _VP(state), _VP(dL_dw))


def seg_admm_unrolled_grads(state: int, K: int, C: int, J: int, dL_df: int = 0, dL_ds: int = 0):
    """(dL/dcodebook as a K*C list, dL/dLambda as a J+1 list) of the enqueued sweep."""
    dc = (ctypes.c_float * (K * C))()
    dl = (ctypes.c_float * (J + 1))()
    _call("seg_admm_unrolled_grads", _VP(state), dc, dl, _VP(dL_df) if dL_df else None,
          _VP(dL_ds) if dL_ds else None)
    return list(dc), list(dl)


# ---------------------------------------------------------------------------
# TV-regularised segmentation (Sec. 4, eq. TVreg)
# ---------------------------------------------------------------------------
def tv_admm_init(H: int, W: int, f: int, C: int, codebook, K: int, gamma: float, lam: float, per_label: bool = False,
                 stream=None) -> int:
    cb = (ctypes.c_float * (K * C))(*[float(x) for x in codebook])
    p = tv_params(float(gamma), float(lam), int(bool(per_label)))
    out = _VP()
    _call("tv_admm_init", int(H), int(W), _VP(f), int(C), cb, int(K), ctypes.byref(p), _stream(stream),
          ctypes.byref(out))
    return out.value


def tv_admm_reset(state: int, f: int, f_on_host: bool) -> None:
    _call("tv_admm_reset", _VP(state), _VP(f), int(bool(f_on_host)))


def tv_admm_step(state: int, n_iters: int) -> None:
    _call("tv_admm_step", _VP(state), int(n_iters))


def tv_admm_get(state: int, what: int, dst: int, dst_on_host: bool) -> None:
    _call("tv_admm_get", _VP(state), int(what), _VP(dst), int(bool(dst_on_host)))


def tv_admm_set(state: int, what: int, src: int, src_on_host: bool) -> None:
    _call("tv_admm_set", _VP(state), int(what), _VP(src), int(bool(src_on_host)))


def tv_admm_kernel_times(state: int, n: int) -> dict:
    """{kernel: mean milliseconds} over n iterations launched one by one."""
    ms = (ctypes.c_float * 8)()
    nk = _I()
    _call("tv_admm_kernel_times", _VP(state), int(n), ms, ctypes.byref(nk))
    return {lib().tv_admm_kernel_name(i).decode(): float(ms[i]) for i in range(nk.value)}


def tv_admm_sync(state: int) -> None:
    _call("tv_admm_sync", _VP(state))


def tv_admm_destroy(state: int) -> None:
    _call("tv_admm_destroy", _VP(state))


# ---------------------------------------------------------------------------
# NL-means-regularised segmentation (Sec. 4)
# ---------------------------------------------------------------------------
def nl_admm_init(H: int, W: int, f: int, C: int, codebook, K: int, gamma: float, lam: float, patch: int = 5,
                 window: int = 15, a: float = 2.0, neighbours: int = 5, solve_steps: int = 0, stream=None) -> int:
    cb = (ctypes.c_float * (K * C))(*[float(x) for x in codebook])
    p = nl_params(float(gamma), float(lam), int(patch), int(window), float(a), int(neighbours), int(solve_steps))
    out = _VP()
    _call("nl_admm_init", int(H), int(W), _VP(f), int(C), cb, int(K), ctypes.byref(p), _stream(stream),
          ctypes.byref(out))
    return out.value


def nl_admm_reset(state: int, f: int, f_on_host: bool) -> None:
    _call("nl_admm_reset", _VP(state), _VP(f), int(bool(f_on_host)))


def nl_admm_graph(state: int, P: int, m: int):
    """(nbr [P, m] int32, deg [P] int32, Chebyshev steps per u-step)."""
    import numpy as np

    nbr = np.empty((P, m), dtype=np.int32)
    deg = np.empty(P, dtype=np.int32)
    steps = _I()
    _call("nl_admm_graph", _VP(state), _VP(nbr.ctypes.data), _VP(deg.ctypes.data), ctypes.byref(steps))
    return nbr, deg, steps.value


def nl_admm_step(state: int, n_iters: int) -> None:
    _call("nl_admm_step", _VP(state), int(n_iters))


def nl_admm_get(state: int, what: int, dst: int, dst_on_host: bool) -> None:
    _call("nl_admm_get", _VP(state), int(what), _VP(dst), int(bool(dst_on_host)))


def nl_admm_set(state: int, what: int, src: int, src_on_host: bool) -> None:
    _call("nl_admm_set", _VP(state), int(what), _VP(src), int(bool(src_on_host)))


def nl_admm_kernel_times(state: int, n: int) -> dict:
    ms = (ctypes.c_float * 8)()
    nk = _I()
    _call("nl_admm_kernel_times", _VP(state), int(n), ms, ctypes.byref(nk))
    return {lib().nl_admm_kernel_name(i).decode(): float(ms[i]) for i in range(nk.value)}


def nl_admm_sync(state: int) -> None:
    _call("nl_admm_sync", _VP(state))


def nl_admm_barrier_selftest(state: int) -> None:
    _call("nl_admm_barrier_selftest", _VP(state))


def nl_admm_destroy(state: int) -> None:
    _call("nl_admm_destroy", _VP(state))
