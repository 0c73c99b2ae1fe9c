"""ctypes wrappers for the FP64 oracle (test infrastructure only).

Every function takes and returns numpy float64 arrays in row-major
[.., H, W] layout.  See ``shearseg_oracle.cpp`` for the arithmetic and the
readings of the paper it implements.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "shearseg_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

__all__ = [
    "build", "lib", "set_threads", "get_threads", "num_filters", "window", "filter_specs",
    "filters", "filters_unsymmetrised", "fft2", "dft2_brute", "analyze", "synthesize",
    "data_term", "soft_shrink", "project_simplex", "admm_iterate", "admm_run", "energy",
    "labels", "thresholds", "zero_state", "unrolled_vjp", "ce_loss", "unrolled_grads",
    "tv_grad", "tv_grad_adj", "tv_solve", "tv_shrink", "tv_zero_state", "tv_admm_iterate", "tv_admm_run",
    "tv_energy", "NL_PARAMS", "nl_distance", "nl_graph", "nl_D", "nl_Dt", "nl_solve", "nl_zero_state",
    "nl_admm_iterate", "nl_admm_run", "nl_energy",
]


def build(force: bool = False) -> str:
    """Compile the oracle shared library with g++ (FP64, -O2, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        # no fused multiply-adds: the NL-means graph compares patch distances
        # that must round the same way on every host
        cmd = ["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.POINTER(ctypes.c_int)
            c_int, c_long, c_double = ctypes.c_int, ctypes.c_long, ctypes.c_double
            sig = {
                "oracle_set_threads": (None, [c_int]),
                "oracle_get_threads": (c_int, []),
                "oracle_num_filters": (c_int, [c_int]),
                "oracle_window": (c_int, [c_int, D, c_long, D]),
                "oracle_filter_specs": (c_int, [c_int, I]),
                "oracle_filters": (c_int, [c_int, c_int, c_int, D]),
                "oracle_filters_unsymmetrised": (c_int, [c_int, c_int, c_int, D]),
                "oracle_fft2": (c_int, [c_int, c_int, D, D, c_int]),
                "oracle_dft2_brute": (c_int, [c_int, c_int, D, D, c_int]),
                "oracle_analyze": (c_int, [c_int, c_int, c_int, D, c_int, D, D]),
                "oracle_synthesize": (c_int, [c_int, c_int, c_int, D, c_int, D, D]),
                "oracle_data_term": (c_int, [c_int, c_int, c_int, D, c_int, D, D]),
                "oracle_soft_shrink": (c_int, [D, c_long, c_double, D]),
                "oracle_project_simplex": (c_int, [D, c_long, c_int, D, c_int]),
                "oracle_admm_iterate": (c_int, [c_int, c_int, c_int, c_int, D, D, c_double, c_int,
                                                D, D, D, D, D, D, c_int]),
                "oracle_energy": (c_int, [c_int, c_int, c_int, c_int, D, D, D, D]),
                "oracle_unrolled_vjp": (c_int, [c_int, c_int, c_int, c_int, D, D, c_double, c_int, D, D, D, D]),
                "oracle_labels": (c_int, [c_int, c_int, c_int, D, I, D]),
                "oracle_tv_grad": (c_int, [c_int, c_int, c_int, D, D]),
                "oracle_tv_grad_adj": (c_int, [c_int, c_int, c_int, D, D]),
                "oracle_tv_solve": (c_int, [c_int, c_int, c_int, D, D]),
                "oracle_tv_shrink": (c_int, [c_int, c_int, c_int, D, c_double, c_int, D]),
                "oracle_tv_admm_iterate": (c_int, [c_int, c_int, c_int, D, c_double, c_double, c_int, c_int,
                                                   D, D, D, D, D, D]),
                "oracle_tv_energy": (c_int, [c_int, c_int, c_int, D, D, c_double, c_int, D]),
                "oracle_nl_distance": (c_double, [c_int, c_int, c_int, D, c_int, c_double, c_int, c_int, c_int,
                                                  c_int]),
                "oracle_nl_graph": (c_int, [c_int, c_int, c_int, D, c_int, c_int, c_double, c_int, I, I]),
                "oracle_nl_D": (c_int, [c_int, c_int, c_int, c_int, I, D, D]),
                "oracle_nl_Dt": (c_int, [c_int, c_int, c_int, c_int, I, D, D]),
                "oracle_nl_solve": (c_int, [c_int, c_int, c_int, c_int, I, D, D]),
                "oracle_nl_admm_iterate": (c_int, [c_int, c_int, c_int, c_int, I, D, c_double, c_double, c_int,
                                                   D, D, D, D, D, D]),
                "oracle_nl_energy": (c_int, [c_int, c_int, c_int, c_int, I, D, D, c_double, D]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _d(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc: int, name: str):
    if rc != 0:
        raise ValueError(f"{name}: invalid arguments (rc={rc})")


def set_threads(n: int) -> None:
    lib().oracle_set_threads(int(n))


def get_threads() -> int:
    return int(lib().oracle_get_threads())


def num_filters(J: int) -> int:
    """eta = 2^(J+2) - 3 filters for J scales (Remark 1: 61 at J = 4)."""
    return int(lib().oracle_num_filters(J))


_WINDOWS = {"v": 0, "b": 1, "psi1": 2, "psi2": 3, "varphi": 4}


def window(name: str, x) -> np.ndarray:
    """The 1-D windows of Sec. 2 (eq. psi1_psi2, v, b, varphi)."""
    x = _f64(x)
    y = np.empty_like(x)
    _check(lib().oracle_window(_WINDOWS[name], _d(x), x.size, _d(y)), "window")
    return y


def filter_specs(J: int) -> np.ndarray:
    """(kind, j, k) per filter in bank order; kind 0 low-pass, 1 h-cone, 2 v-cone, 3 glued."""
    eta = num_filters(J)
    out = np.zeros((eta, 3), dtype=np.int32)
    _check(lib().oracle_filter_specs(J, out.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), "filter_specs")
    return out


def thresholds(J: int, Lambda, gamma: float) -> np.ndarray:
    """gamma * Lambda_{j(f)} per filter: Lambda[0] low-pass, Lambda[j+1] scale j."""
    Lambda = np.asarray(Lambda, dtype=np.float64)
    specs = filter_specs(J)
    return np.array([gamma * (Lambda[0] if kind == 0 else Lambda[j + 1]) for kind, j, _ in specs])


def filters(H: int, W: int, J: int) -> np.ndarray:
    """Full-plane filter bank [eta, H, W] in DFT index order (Sec. 2)."""
    out = np.empty((num_filters(J), H, W))
    _check(lib().oracle_filters(H, W, J, _d(out)), "filters")
    return out


def filters_unsymmetrised(H: int, W: int, J: int) -> np.ndarray:
    out = np.empty((num_filters(J), H, W))
    _check(lib().oracle_filters_unsymmetrised(H, W, J, _d(out)), "filters_unsymmetrised")
    return out


def _cplx_call(fn, x, inverse):
    x = np.ascontiguousarray(x, dtype=np.complex128)
    H, W = x.shape
    inp = np.ascontiguousarray(np.stack([x.real, x.imag], axis=-1))
    out = np.empty_like(inp)
    _check(fn(H, W, _d(inp), _d(out), int(bool(inverse))), "fft2")
    return out[..., 0] + 1j * out[..., 1]


def fft2(x, inverse: bool = False) -> np.ndarray:
    """fft2 (no scaling) or ifft2 (factor 1/(HW)) with the oracle's own FFT."""
    return _cplx_call(lib().oracle_fft2, x, inverse)


def dft2_brute(x, inverse: bool = False) -> np.ndarray:
    """The defining double sum of the 2-D DFT (pin for fft2)."""
    return _cplx_call(lib().oracle_dft2_brute, x, inverse)


def analyze(u, J: int, return_imag: bool = False):
    """S applied to each channel (eq. wichtig): u[..., H, W] -> coef[..., eta, H, W]."""
    u = _f64(u)
    lead = u.shape[:-2]
    H, W = u.shape[-2:]
    nch = int(np.prod(lead)) if lead else 1
    coef = np.empty(lead + (num_filters(J), H, W))
    mi = ctypes.c_double(0.0)
    _check(lib().oracle_analyze(H, W, J, _d(u), nch, _d(coef), ctypes.byref(mi)), "analyze")
    return (coef, mi.value) if return_imag else coef


def synthesize(coef, J: int, return_imag: bool = False):
    """S^T applied per channel: coef[..., eta, H, W] -> u[..., H, W]."""
    coef = _f64(coef)
    lead = coef.shape[:-3]
    H, W = coef.shape[-2:]
    assert coef.shape[-3] == num_filters(J)
    nch = int(np.prod(lead)) if lead else 1
    u = np.empty(lead + (H, W))
    mi = ctypes.c_double(0.0)
    _check(lib().oracle_synthesize(H, W, J, _d(coef), nch, _d(u), ctypes.byref(mi)), "synthesize")
    return (u, mi.value) if return_imag else u


def data_term(f, codebook) -> np.ndarray:
    """eq. computationOfs with p = 2: s[k] = sum_ch (f[ch] - c[k, ch])^2.

    f: [H, W] (gray) or [C, H, W]; codebook: [K] or [K, C]."""
    f = _f64(f)
    if f.ndim == 2:
        f = f[None]
    C, H, W = f.shape
    cb = _f64(codebook).reshape(-1, C)
    K = cb.shape[0]
    s = np.empty((K, H, W))
    _check(lib().oracle_data_term(H, W, C, _d(f), K, _d(cb), _d(s)), "data_term")
    return s


def soft_shrink(x, t: float) -> np.ndarray:
    x = _f64(x)
    y = np.empty_like(x)
    _check(lib().oracle_soft_shrink(_d(x), x.size, float(t), _d(y)), "soft_shrink")
    return y


def project_simplex(g, method: str = "sort") -> np.ndarray:
    """Projection of each row of g[..., K] onto the unit simplex."""
    g = _f64(g)
    K = g.shape[-1]
    x = np.empty_like(g)
    m = {"sort": 0, "repeated": 1}[method]
    _check(lib().oracle_project_simplex(_d(g), g.size // K, K, _d(x), m), "project_simplex")
    return x


def admm_iterate(state: dict, s, J: int, Lambda, gamma: float, T: int, proj: str = "sort",
                 record_residual: bool = False):
    """T ADMM iterations of Sec. 3 in place on ``state`` (keys v, bv, w, bw, u).

    Returns the per-iteration fixed-point residuals when requested."""
    s = _f64(s)
    K, H, W = s.shape
    Lam = _f64(Lambda)
    assert Lam.size == J + 1
    for key in ("v", "bv", "w", "bw", "u"):
        assert state[key].dtype == np.float64 and state[key].flags.c_contiguous
    res = np.zeros(max(T, 1)) if record_residual else None
    rc = lib().oracle_admm_iterate(
        H, W, J, K, _d(s), _d(Lam), float(gamma), int(T),
        _d(state["v"]), _d(state["bv"]), _d(state["w"]), _d(state["bw"]), _d(state["u"]),
        _d(res) if res is not None else None, {"sort": 0, "repeated": 1}[proj])
    _check(rc, "admm_iterate")
    return res[:T] if res is not None else None


def zero_state(K: int, J: int, H: int, W: int) -> dict:
    """Initial state: v = b_v = 0, w = b_w = 0 (the paper leaves it open)."""
    eta = num_filters(J)
    return {
        "v": np.zeros((K, eta, H, W)), "bv": np.zeros((K, eta, H, W)),
        "w": np.zeros((K, H, W)), "bw": np.zeros((K, H, W)), "u": np.zeros((K, H, W)),
    }


def admm_run(f, codebook, J: int, Lambda, gamma: float, T: int, proj: str = "sort") -> dict:
    """Data term + zero initial state + T iterations; returns the state with
    labels, gap and energy of w added."""
    s = data_term(f, codebook)
    K, H, W = s.shape
    st = zero_state(K, J, H, W)
    st["fp_res"] = admm_iterate(st, s, J, Lambda, gamma, T, proj=proj, record_residual=True)
    st["s"] = s
    st["labels"], st["gap"] = labels(st["w"])
    st["energy"] = energy(st["w"], s, J, Lambda)
    return st


def energy(x, s, J: int, Lambda) -> float:
    """<x, s> + sum_f Lambda_{j(f)} ||(S x)_f||_1 (eq. problemSegmentation)."""
    x, s, Lam = _f64(x), _f64(s), _f64(Lambda)
    K, H, W = x.shape
    e = ctypes.c_double(0.0)
    _check(lib().oracle_energy(H, W, J, K, _d(x), _d(s), _d(Lam), ctypes.byref(e)), "energy")
    return e.value


def labels(x):
    """argmax over the label axis (ties: lowest index) and the top-two gap."""
    x = _f64(x)
    K, H, W = x.shape
    lab = np.empty((H, W), dtype=np.int32)
    gap = np.empty((H, W))
    _check(lib().oracle_labels(H, W, K, _d(x), lab.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), _d(gap)),
           "labels")
    return lab, gap


def unrolled_vjp(s, J: int, Lambda, gamma: float, T: int, wbar_T):
    """Reverse mode of T ADMM iterations from the zero state (see the C++
    comment): returns (w_T, sbar, Lambar) for the adjoint wbar_T of w_T."""
    s = _f64(s)
    K, H, W = s.shape
    Lam = _f64(Lambda)
    wb = _f64(wbar_T)
    sbar = np.empty_like(s)
    lb = np.empty(J + 1)
    wT = np.empty_like(s)
    _check(lib().oracle_unrolled_vjp(H, W, J, K, _d(s), _d(Lam), float(gamma), int(T), _d(wb), _d(sbar), _d(lb),
                                     _d(wT)), "unrolled_vjp")
    return wT, sbar, lb


def ce_loss(w, labels, eps: float = 1e-6):
    """Cross entropy of the relaxed labelling against a label map:
    -mean_x log(max(w[label(x)](x), eps)); returns (loss, dL/dw)."""
    w = _f64(w)
    K, H, W = w.shape
    P = H * W
    lab = np.asarray(labels)
    wl = np.take_along_axis(w, lab[None].astype(np.int64), axis=0)[0]
    loss = -np.log(np.maximum(wl, eps)).mean()
    g = np.zeros_like(w)
    gl = np.where(wl > eps, -1.0 / (P * np.maximum(wl, eps)), 0.0)
    np.put_along_axis(g, lab[None].astype(np.int64), gl[None], axis=0)
    return loss, g


def unrolled_grads(f, codebook, J: int, Lambda, gamma: float, T: int, labels, eps: float = 1e-6):
    """Loss and gradients of the unrolled solve: d/dcodebook [K][C], d/dLambda
    [J+1] and d/df [C][H][W], through s[k] = sum_ch (f[ch] - c[k][ch])^2."""
    f = _f64(f)
    if f.ndim == 2:
        f = f[None]
    cb = _f64(codebook).reshape(-1, f.shape[0])
    s = data_term(f, cb)
    st = zero_state(s.shape[0], J, s.shape[1], s.shape[2])
    admm_iterate(st, s, J, Lambda, gamma, T)
    loss, wbar = ce_loss(st["w"], labels, eps)
    wT, sbar, lbar = unrolled_vjp(s, J, Lambda, gamma, T, wbar)
    diff = f[None] - cb[:, :, None, None]                       # [K][C][H][W]
    dcb = (sbar[:, None] * (-2.0) * diff).sum(axis=(2, 3))
    df = (sbar[:, None] * 2.0 * diff).sum(axis=0)
    return {"loss": loss, "w": wT, "codebook": dcb, "Lambda": lbar, "f": df, "sbar": sbar}


# ---------------------------------------------------------------------------
# TV-regularised segmentation (Sec. 4, eq. TVreg): the comparison model.
# Gradients and their duals are [K, 2, H, W] (component 0 along rows).
# ---------------------------------------------------------------------------
def tv_grad(u) -> np.ndarray:
    """Periodic forward differences of each plane: u[K, H, W] -> [K, 2, H, W]."""
    u = _f64(u)
    K, H, W = u.shape
    g = np.empty((K, 2, H, W))
    _check(lib().oracle_tv_grad(H, W, K, _d(u), _d(g)), "tv_grad")
    return g


def tv_grad_adj(p) -> np.ndarray:
    """Adjoint of tv_grad: p[K, 2, H, W] -> [K, H, W]."""
    p = _f64(p)
    K, _, H, W = p.shape
    out = np.empty((K, H, W))
    _check(lib().oracle_tv_grad_adj(H, W, K, _d(p), _d(out)), "tv_grad_adj")
    return out


def tv_solve(rhs) -> np.ndarray:
    """(I + grad^T grad)^-1 rhs per plane (periodic, diagonal in the DFT basis)."""
    rhs = _f64(rhs)
    K, H, W = rhs.shape
    u = np.empty_like(rhs)
    _check(lib().oracle_tv_solve(H, W, K, _d(rhs), _d(u)), "tv_solve")
    return u


def tv_shrink(g, t: float, per_label: bool = False) -> np.ndarray:
    """Vector shrinkage of g[K, 2, H, W] by t over all 2K values of a pixel
    (or over the two values of each label with per_label)."""
    g = _f64(g)
    K, _, H, W = g.shape
    v = np.empty_like(g)
    _check(lib().oracle_tv_shrink(H, W, K, _d(g), float(t), int(per_label), _d(v)), "tv_shrink")
    return v


def tv_zero_state(K: int, H: int, W: int) -> dict:
    return {"v": np.zeros((K, 2, H, W)), "bv": np.zeros((K, 2, H, W)), "w": np.zeros((K, H, W)),
            "bw": np.zeros((K, H, W)), "u": np.zeros((K, H, W))}


def tv_admm_iterate(state: dict, s, lam: float, gamma: float, T: int, per_label: bool = False,
                    record_residual: bool = False):
    """T ADMM iterations of the TV model in place on ``state`` (keys v, bv, w, bw, u)."""
    s = _f64(s)
    K, H, W = s.shape
    for key in ("v", "bv", "w", "bw", "u"):
        assert state[key].dtype == np.float64 and state[key].flags.c_contiguous
    res = np.zeros(max(T, 1)) if record_residual else None
    rc = lib().oracle_tv_admm_iterate(H, W, K, _d(s), float(lam), float(gamma), int(per_label), int(T),
                                      _d(state["v"]), _d(state["bv"]), _d(state["w"]), _d(state["bw"]),
                                      _d(state["u"]), _d(res) if res is not None else None)
    _check(rc, "tv_admm_iterate")
    return res[:T] if res is not None else None


def tv_energy(x, s, lam: float, per_label: bool = False) -> float:
    """<x, s> + lam sum_pixels |(I_q (x) grad) x| (eq. TVreg)."""
    x, s = _f64(x), _f64(s)
    K, H, W = x.shape
    e = ctypes.c_double(0.0)
    _check(lib().oracle_tv_energy(H, W, K, _d(x), _d(s), float(lam), int(per_label), ctypes.byref(e)), "tv_energy")
    return e.value


def tv_admm_run(f, codebook, lam: float, gamma: float, T: int, per_label: bool = False) -> dict:
    """Data term + zero state + T TV-ADMM iterations; adds labels, gap, energy."""
    s = data_term(f, codebook)
    K, H, W = s.shape
    st = tv_zero_state(K, H, W)
    st["fp_res"] = tv_admm_iterate(st, s, lam, gamma, T, per_label, record_residual=True)
    st["s"] = s
    st["labels"], st["gap"] = labels(st["w"])
    st["energy"] = tv_energy(st["w"], s, lam, per_label)
    return st


# ---------------------------------------------------------------------------
# NL-means regulariser (Sec. 4): D from patch similarities of f.  Graphs are
# (nbr [P, m] int32, increasing index, -1 padded; deg [P]); D's coefficients
# and their duals are [K, m, H, W].
# ---------------------------------------------------------------------------
# patch size p, search window varpi, Gaussian a, neighbours per pixel mt (Sec. 4)
NL_PARAMS = {"p": 5, "win": 15, "a": 2.0, "mt": 5}


def _i32(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def nl_distance(f, i, j, p: int = 5, a: float = 2.0) -> float:
    """d_a between pixels i = (row, col) and j of f [C, H, W] (or [H, W])."""
    f = _f64(f)
    if f.ndim == 2:
        f = f[None]
    C, H, W = f.shape
    return float(lib().oracle_nl_distance(H, W, C, _d(f), int(p), float(a), int(i[0]), int(i[1]), int(j[0]),
                                          int(j[1])))


def nl_graph(f, p: int = 5, win: int = 15, a: float = 2.0, mt: int = 5):
    """(nbr [H W, 2 mt], deg [H W]) of the NL-means construction of Sec. 4."""
    f = _f64(f)
    if f.ndim == 2:
        f = f[None]
    C, H, W = f.shape
    nbr = np.empty((H * W, 2 * mt), dtype=np.int32)
    deg = np.empty(H * W, dtype=np.int32)
    _check(lib().oracle_nl_graph(H, W, C, _d(f), int(p), int(win), float(a), int(mt),
                                 nbr.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 deg.ctypes.data_as(ctypes.POINTER(ctypes.c_int))), "nl_graph")
    return nbr, deg


def nl_D(nbr, u) -> np.ndarray:
    u = _f64(u)
    K, H, W = u.shape
    nb, pn = _i32(nbr)
    m = nb.shape[1]
    q = np.empty((K, m, H, W))
    _check(lib().oracle_nl_D(H, W, K, m, pn, _d(u), _d(q)), "nl_D")
    return q


def nl_Dt(nbr, q) -> np.ndarray:
    q = _f64(q)
    K, m, H, W = q.shape
    nb, pn = _i32(nbr)
    u = np.empty((K, H, W))
    _check(lib().oracle_nl_Dt(H, W, K, m, pn, _d(q), _d(u)), "nl_Dt")
    return u


def nl_solve(nbr, rhs) -> np.ndarray:
    """(I + D^T D)^-1 rhs per plane (conjugate gradients to 1e-13)."""
    rhs = _f64(rhs)
    K, H, W = rhs.shape
    nb, pn = _i32(nbr)
    u = np.empty_like(rhs)
    _check(lib().oracle_nl_solve(H, W, K, nb.shape[1], pn, _d(rhs), _d(u)), "nl_solve")
    return u


def nl_zero_state(K: int, m: int, H: int, W: int) -> dict:
    return {"v": np.zeros((K, m, H, W)), "bv": np.zeros((K, m, H, W)), "w": np.zeros((K, H, W)),
            "bw": np.zeros((K, H, W)), "u": np.zeros((K, H, W))}


def nl_admm_iterate(state: dict, s, nbr, lam: float, gamma: float, T: int, record_residual: bool = False):
    s = _f64(s)
    K, H, W = s.shape
    nb, pn = _i32(nbr)
    for key in ("v", "bv", "w", "bw", "u"):
        assert state[key].dtype == np.float64 and state[key].flags.c_contiguous
    res = np.zeros(max(T, 1)) if record_residual else None
    rc = lib().oracle_nl_admm_iterate(H, W, K, nb.shape[1], pn, _d(s), float(lam), float(gamma), int(T),
                                      _d(state["v"]), _d(state["bv"]), _d(state["w"]), _d(state["bw"]),
                                      _d(state["u"]), _d(res) if res is not None else None)
    _check(rc, "nl_admm_iterate")
    return res[:T] if res is not None else None


def nl_energy(x, s, nbr, lam: float) -> float:
    x, s = _f64(x), _f64(s)
    K, H, W = x.shape
    nb, pn = _i32(nbr)
    e = ctypes.c_double(0.0)
    _check(lib().oracle_nl_energy(H, W, K, nb.shape[1], pn, _d(x), _d(s), float(lam), ctypes.byref(e)),
           "nl_energy")
    return e.value


def nl_admm_run(f, codebook, lam: float, gamma: float, T: int, graph=None, **graph_params) -> dict:
    """Graph of f (unless given), data term, zero state, T NL-ADMM iterations;
    adds the graph, labels, gap and energy."""
    prm = dict(NL_PARAMS, **graph_params)
    nbr, deg = graph if graph is not None else nl_graph(f, **prm)
    s = data_term(f, codebook)
    K, H, W = s.shape
    st = nl_zero_state(K, nbr.shape[1], H, W)
    st["fp_res"] = nl_admm_iterate(st, s, nbr, lam, gamma, T, record_residual=True)
    st["s"], st["nbr"], st["deg"] = s, nbr, deg
    st["labels"], st["gap"] = labels(st["w"])
    st["energy"] = nl_energy(st["w"], s, nbr, lam)
    return st
