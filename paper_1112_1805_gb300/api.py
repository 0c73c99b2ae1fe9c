"""PyTorch-facing wrappers over the C ABI: tensors in, tensors out.

PyTorch supplies device memory and the current CUDA stream; every step of the
computation runs in libshearseg.so.  Device tensors must be contiguous
float32 on the current CUDA device.
"""

from __future__ import annotations

import numpy as np
import torch

from . import binding as B


def _cur_stream():
    return torch.cuda.current_stream().cuda_stream


def _dev_f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    return t


class FilterBank:
    """Shearlet filter bank for one (H, W, J) (Sec. 2 of the paper)."""

    def __init__(self, H: int, W: int, J: int):
        self.handle = B.shfilters_build(H, W, J, _cur_stream())
        self.eta, self.H, self.W, self.J = B.shfilters_info(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            B.shfilters_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def spectra(self) -> torch.Tensor:
        """FP32 half-plane spectra [eta, H, W//2+1]."""
        out = torch.empty((self.eta, self.H, self.W // 2 + 1), dtype=torch.float32, device="cuda")
        B.shfilters_copy(self.handle, out.data_ptr(), _cur_stream())
        return out

    def analyze(self, u: torch.Tensor) -> torch.Tensor:
        """S per channel: u [..., H, W] -> [..., eta, H, W] (eq. wichtig)."""
        _dev_f32(u, "u")
        lead = u.shape[:-2]
        nch = int(np.prod(lead)) if len(lead) else 1
        coef = torch.empty(tuple(lead) + (self.eta, self.H, self.W), dtype=torch.float32, device=u.device)
        B.shearlet_analyze(self.handle, u.data_ptr(), nch, coef.data_ptr(), _cur_stream())
        return coef

    def synthesize(self, coef: torch.Tensor) -> torch.Tensor:
        """S^T per channel: [..., eta, H, W] -> [..., H, W]."""
        _dev_f32(coef, "coef")
        lead = coef.shape[:-3]
        nch = int(np.prod(lead)) if len(lead) else 1
        u = torch.empty(tuple(lead) + (self.H, self.W), dtype=torch.float32, device=coef.device)
        B.shearlet_synthesize(self.handle, coef.data_ptr(), nch, u.data_ptr(), _cur_stream())
        return u


class ShearletSegmenter:
    """ADMM state for one image (Sec. 3 of the paper).

    f: [C, H, W] or [H, W] float32 CUDA tensor; codebook: [K, C] (host values);
    Lambda: J+1 weights (low-pass first); gamma > 0."""

    def __init__(self, bank: FilterBank, f: torch.Tensor, codebook, Lambda, gamma: float = 1.0,
                 max_iters: int = 500, tol: float = 0.0, check_every: int = 50, stream=None):
        if f.dim() == 2:
            f = f.unsqueeze(0)
        _dev_f32(f, "f")
        cb = np.asarray(codebook, dtype=np.float64).reshape(-1, f.shape[0])
        self.bank = bank
        self.K, self.C = cb.shape
        self.H, self.W, self.eta = bank.H, bank.W, bank.eta
        self._params, self._keep = B.make_params(gamma, bank.J, Lambda, max_iters, tol, check_every)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())  # f may still be in flight on torch's stream
        self.handle = B.seg_admm_init(bank.handle, f.data_ptr(), self.C, cb.ravel().tolist(), self.K, self._params,
                                      self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None) and getattr(self, "_owned", True):
            B.seg_admm_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int) -> None:
        B.seg_admm_step(self.handle, n)

    def solve(self):
        return B.seg_admm_solve(self.handle)

    def synchronize(self) -> None:
        B.seg_admm_sync(self.handle)

    def reset(self, f) -> None:
        """New image: a CUDA tensor, or a host (ideally pinned) tensor / numpy array."""
        if isinstance(f, torch.Tensor) and f.is_cuda:
            _dev_f32(f, "f")
            self.stream.wait_stream(torch.cuda.current_stream())
            B.seg_admm_reset(self.handle, f.data_ptr(), False)
        else:
            a = f if isinstance(f, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32))
            a = a.contiguous()
            B.seg_admm_reset(self.handle, a.data_ptr(), True)

    def _shape(self, what: int):
        K, H, W = self.K, self.H, self.W
        if what in (B.SEG_U, B.SEG_W, B.SEG_BW, B.SEG_S, B.SEG_STV):
            return (K, H, W), torch.float32
        if what in (B.SEG_BV, B.SEG_V):
            return (K, self.eta, H, W), torch.float32
        if what == B.SEG_LABELS:
            return (H, W), torch.int32
        if what == B.SEG_GAP:
            return (H, W), torch.float32
        raise ValueError(what)

    def get(self, what: int) -> torch.Tensor:
        """A state component as a CUDA tensor (written on the state's stream)."""
        if what == B.SEG_ENERGY:
            buf = np.zeros(1, dtype=np.float64)
            B.seg_admm_get(self.handle, what, buf.ctypes.data, True)
            return torch.tensor(buf[0], dtype=torch.float64)
        if what == B.SEG_ITER:
            buf = np.zeros(1, dtype=np.int32)
            B.seg_admm_get(self.handle, what, buf.ctypes.data, True)
            return torch.tensor(int(buf[0]))
        shape, dt = self._shape(what)
        out = torch.empty(shape, dtype=dt, device="cuda")
        B.seg_admm_get(self.handle, what, out.data_ptr(), False)
        self.synchronize()
        return out

    def get_host(self, what: int, out: torch.Tensor | None = None) -> torch.Tensor:
        """A state component copied into host memory (pinned if `out` is)."""
        shape, dt = self._shape(what)
        if out is None:
            out = torch.empty(shape, dtype=dt, pin_memory=True)
        B.seg_admm_get(self.handle, what, out.data_ptr(), True)
        return out

    def set(self, what: int, src: torch.Tensor) -> None:
        shape, dt = self._shape(what)
        src = src.to(dt).contiguous()
        if tuple(src.shape) != shape:
            raise ValueError(f"expected shape {shape}, got {tuple(src.shape)}")
        if src.is_cuda:
            self.stream.wait_stream(torch.cuda.current_stream())
        B.seg_admm_set(self.handle, what, src.data_ptr(), not src.is_cuda)
        if src.is_cuda:
            self.synchronize()

    def plan(self) -> dict:
        """The work plan (launch shapes) of the iteration."""
        return B.seg_admm_get_plan(self.handle)

    def set_plan(self, plan: dict) -> None:
        self.stream.synchronize()
        B.seg_admm_set_plan(self.handle, plan)

    def tune(self, iters: int = 5) -> dict:
        """Autotunes the work plan on this image (the iterate is restored)."""
        torch.cuda.current_stream().synchronize()
        return B.seg_admm_tune(self.handle, iters)

    def energy(self) -> float:
        return float(self.get(B.SEG_ENERGY))

    def labels(self) -> torch.Tensor:
        return self.get(B.SEG_LABELS)

    def save(self, path: str) -> None:
        B.seg_admm_save(self.handle, path)

    def load(self, path: str) -> None:
        B.seg_admm_load(self.handle, path)


class _BorrowedState(ShearletSegmenter):
    """View of a state owned by a batch (readout and injection only)."""

    def __init__(self, handle, K, C, H, W, eta):  # noqa: D401 - no library call here
        self.handle = handle
        self.K, self.C, self.H, self.W, self.eta = K, C, H, W, eta
        self._owned = False

    def close(self):
        self.handle = None

    def step(self, n: int) -> None:
        raise RuntimeError("iterate a batch with ShearletBatch.step")


class ShearletBatch:
    """Independent images of uneven sizes and label counts solved together: one
    CUDA graph per iteration with one concurrent branch per image, or the
    images chained into `lanes` branches.

    images: list of float32 CUDA tensors [C, H, W] or [H, W]; codebooks: list of
    [K, C] host arrays; Lambdas: list of J+1 weight vectors; gammas: list or
    scalar."""

    def __init__(self, images, codebooks, Lambdas, gammas=1.0, stream=None):
        n = len(images)
        imgs = [(t.unsqueeze(0) if t.dim() == 2 else t) for t in images]
        for t in imgs:
            _dev_f32(t, "image")
        if not isinstance(gammas, (list, tuple)):
            gammas = [gammas] * n
        cbs = [np.asarray(c, dtype=np.float64).reshape(-1, t.shape[0]) for c, t in zip(codebooks, imgs)]
        self._keep = []
        params = []
        for lam, g in zip(Lambdas, gammas):
            lam = list(lam)
            p, keep = B.make_params(g, len(lam) - 1, lam)
            params.append(p)
            self._keep.append(keep)
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        torch.cuda.current_stream().synchronize()  # images are read on the images' own streams
        self.shapes = [(int(t.shape[1]), int(t.shape[2]), int(c.shape[0]), int(t.shape[0]), len(l) - 1)
                       for t, c, l in zip(imgs, cbs, Lambdas)]
        self.handle = B.seg_admm_batch_init([s[0] for s in self.shapes], [s[1] for s in self.shapes],
                                            [s[3] for s in self.shapes], [s[2] for s in self.shapes],
                                            [t.data_ptr() for t in imgs], [c.ravel().tolist() for c in cbs], params,
                                            self.stream.cuda_stream)

    def __len__(self):
        return len(self.shapes)

    def close(self):
        if getattr(self, "handle", None):
            B.seg_admm_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int) -> None:
        B.seg_admm_batch_step(self.handle, n)

    def tune(self, iters: int = 5) -> None:
        """Autotunes one plan per distinct image shape, then the batch's lanes
        and SM share."""
        torch.cuda.current_stream().synchronize()
        B.seg_admm_batch_tune(self.handle, iters)

    @property
    def lanes(self) -> int:
        """Chains of images run side by side (0: every image at once)."""
        return B.seg_admm_batch_get_lanes(self.handle)

    @lanes.setter
    def lanes(self, n: int) -> None:
        B.seg_admm_batch_set_lanes(self.handle, n)

    def synchronize(self) -> None:
        B.seg_admm_batch_sync(self.handle)

    def image(self, i: int) -> ShearletSegmenter:
        H, W, K, C, J = self.shapes[i]
        return _BorrowedState(B.seg_admm_batch_image(self.handle, i), K, C, H, W, 2 ** (J + 2) - 3)


class TVSegmenter:
    """ADMM state of the TV-regularised model of Sec. 4 (eq. TVreg) for one
    image: the same data term, simplex constraint and ADMM as
    ShearletSegmenter with the shearlet transform replaced by the periodic
    forward-difference gradient (labels coupled per pixel, or per label).

    f: [C, H, W] or [H, W] float32 CUDA tensor; codebook: [K, C] host values."""

    def __init__(self, f: torch.Tensor, codebook, lam: float, gamma: float = 1.0, per_label: bool = False,
                 stream=None):
        if f.dim() == 2:
            f = f.unsqueeze(0)
        _dev_f32(f, "f")
        cb = np.asarray(codebook, dtype=np.float64).reshape(-1, f.shape[0])
        self.K, self.C = cb.shape
        self.H, self.W = int(f.shape[1]), int(f.shape[2])
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        self.handle = B.tv_admm_init(self.H, self.W, f.data_ptr(), self.C, cb.ravel().tolist(), self.K, gamma, lam,
                                     per_label, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            B.tv_admm_destroy(self.handle)
        self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n: int) -> None:
        B.tv_admm_step(self.handle, n)

    def synchronize(self) -> None:
        B.tv_admm_sync(self.handle)

    def reset(self, f) -> None:
        if isinstance(f, torch.Tensor) and f.is_cuda:
            _dev_f32(f, "f")
            self.stream.wait_stream(torch.cuda.current_stream())
            B.tv_admm_reset(self.handle, f.data_ptr(), False)
        else:
            a = f if isinstance(f, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32))
            B.tv_admm_reset(self.handle, a.contiguous().data_ptr(), True)

    def _shape(self, what: int):
        K, H, W = self.K, self.H, self.W
        if what in (B.SEG_U, B.SEG_W, B.SEG_BW, B.SEG_S):
            return (K, H, W), torch.float32
        if what in (B.SEG_BV, B.SEG_V):
            return (K, 2, H, W), torch.float32
        if what == B.SEG_LABELS:
            return (H, W), torch.int32
        if what == B.SEG_GAP:
            return (H, W), torch.float32
        raise ValueError(what)

    def get(self, what: int) -> torch.Tensor:
        if what == B.SEG_ENERGY:
            buf = np.zeros(1, dtype=np.float64)
            B.tv_admm_get(self.handle, what, buf.ctypes.data, True)
            return torch.tensor(buf[0], dtype=torch.float64)
        if what == B.SEG_ITER:
            buf = np.zeros(1, dtype=np.int32)
            B.tv_admm_get(self.handle, what, buf.ctypes.data, True)
            return torch.tensor(int(buf[0]))
        shape, dt = self._shape(what)
        out = torch.empty(shape, dtype=dt, device="cuda")
        B.tv_admm_get(self.handle, what, out.data_ptr(), False)
        self.synchronize()
        return out

    def get_host(self, what: int, out: torch.Tensor | None = None) -> torch.Tensor:
        shape, dt = self._shape(what)
        if out is None:
            out = torch.empty(shape, dtype=dt, pin_memory=True)
        B.tv_admm_get(self.handle, what, out.data_ptr(), True)
        return out

    def set(self, what: int, src: torch.Tensor) -> None:
        shape, dt = self._shape(what)
        src = src.to(dt).contiguous()
        if tuple(src.shape) != shape:
            raise ValueError(f"expected shape {shape}, got {tuple(src.shape)}")
        if src.is_cuda:
            self.stream.wait_stream(torch.cuda.current_stream())
        B.tv_admm_set(self.handle, what, src.data_ptr(), not src.is_cuda)

    def energy(self) -> float:
        return float(self.get(B.SEG_ENERGY))

    def labels(self) -> torch.Tensor:
        return self.get(B.SEG_LABELS)

    def kernel_times(self, n: int = 5) -> dict:
        """Mean milliseconds per kernel over n iterations (advances the iterate)."""
        return B.tv_admm_kernel_times(self.handle, n)


class NLSegmenter(TVSegmenter):
    """ADMM state of the NL-means-regularised model of Sec. 4 for one image:
    the neighbour graph of f (patch size p, search window varpi, Gaussian a,
    mt neighbours picked per pixel; the paper's 5, 15, 2, 5), then the ADMM
    with the difference matrix D in place of the gradient.

    f: [C, H, W] or [H, W] float32 CUDA tensor; codebook: [K, C] host values."""

    def __init__(self, f: torch.Tensor, codebook, lam: float, gamma: float = 0.2, patch: int = 5, window: int = 15,
                 a: float = 2.0, neighbours: int = 5, solve_steps: int = 0, stream=None):
        if f.dim() == 2:
            f = f.unsqueeze(0)
        _dev_f32(f, "f")
        cb = np.asarray(codebook, dtype=np.float64).reshape(-1, f.shape[0])
        self.K, self.C = cb.shape
        self.H, self.W = int(f.shape[1]), int(f.shape[2])
        self.m = 2 * neighbours
        self.stream = stream if stream is not None else torch.cuda.Stream()
        self.stream.wait_stream(torch.cuda.current_stream())
        torch.cuda.current_stream().synchronize()
        self.handle = B.nl_admm_init(self.H, self.W, f.data_ptr(), self.C, cb.ravel().tolist(), self.K, gamma, lam,
                                     patch, window, a, neighbours, solve_steps, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "handle", None):
            B.nl_admm_destroy(self.handle)
        self.handle = None

    def step(self, n: int) -> None:
        B.nl_admm_step(self.handle, n)

    def synchronize(self) -> None:
        B.nl_admm_sync(self.handle)

    def reset(self, f) -> None:
        if isinstance(f, torch.Tensor) and f.is_cuda:
            _dev_f32(f, "f")
            self.stream.wait_stream(torch.cuda.current_stream())
            torch.cuda.current_stream().synchronize()
            B.nl_admm_reset(self.handle, f.data_ptr(), False)
        else:
            a = f if isinstance(f, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(f, dtype=np.float32))
            B.nl_admm_reset(self.handle, a.contiguous().data_ptr(), True)

    def graph(self):
        """(nbr [H W, m], deg [H W], Chebyshev steps per u-step) of the state's image."""
        return B.nl_admm_graph(self.handle, self.H * self.W, self.m)

    def _shape(self, what: int):
        if what in (B.SEG_BV, B.SEG_V):
            return (self.K, self.m, self.H, self.W), torch.float32
        return TVSegmenter._shape(self, what)

    def get(self, what: int) -> torch.Tensor:
        if what == B.SEG_ENERGY:
            buf = np.zeros(1, dtype=np.float64)
            B.nl_admm_get(self.handle, what, buf.ctypes.data, True)
            return torch.tensor(buf[0], dtype=torch.float64)
        if what == B.SEG_ITER:
            buf = np.zeros(1, dtype=np.int32)
            B.nl_admm_get(self.handle, what, buf.ctypes.data, True)
            return torch.tensor(int(buf[0]))
        shape, dt = self._shape(what)
        out = torch.empty(shape, dtype=dt, device="cuda")
        B.nl_admm_get(self.handle, what, out.data_ptr(), False)
        self.synchronize()
        return out

    def get_host(self, what: int, out: torch.Tensor | None = None) -> torch.Tensor:
        shape, dt = self._shape(what)
        if out is None:
            out = torch.empty(shape, dtype=dt, pin_memory=True)
        B.nl_admm_get(self.handle, what, out.data_ptr(), True)
        return out

    def set(self, what: int, src: torch.Tensor) -> None:
        shape, dt = self._shape(what)
        src = src.to(dt).contiguous()
        if tuple(src.shape) != shape:
            raise ValueError(f"expected shape {shape}, got {tuple(src.shape)}")
        if src.is_cuda:
            self.stream.wait_stream(torch.cuda.current_stream())
        B.nl_admm_set(self.handle, what, src.data_ptr(), not src.is_cuda)

    def kernel_times(self, n: int = 5) -> dict:
        return B.nl_admm_kernel_times(self.handle, n)


class UnrolledSegmentation(torch.autograd.Function):
    """w_T of T ADMM iterations from the zero state as a differentiable function
    of the image f [C, H, W], the codebook [K, C] and the weights Lambda [J+1]
    (the forward keeps every ckpt_every-th state; the backward recomputes the
    segments and runs the adjoint iterations in libshearseg.so)."""

    @staticmethod
    def forward(ctx, f, codebook, Lambda, bank, gamma, T, ckpt_every):
        f3 = (f.unsqueeze(0) if f.dim() == 2 else f).detach().contiguous()
        cb = codebook.detach().double().cpu().numpy().reshape(-1, f3.shape[0])
        lam = Lambda.detach().double().cpu().tolist()
        seg = ShearletSegmenter(bank, f3, cb, lam, float(gamma))
        B.seg_admm_unrolled_fwd(seg.handle, int(T), int(ckpt_every))
        w = seg.get(B.SEG_W)
        ctx.seg, ctx.fdim, ctx.shape = seg, f.dim(), tuple(f3.shape)
        ctx.K, ctx.C, ctx.J = cb.shape[0], cb.shape[1], len(lam) - 1
        ctx.cb_meta = (codebook.dtype, codebook.device, tuple(codebook.shape))
        ctx.lam_meta = (Lambda.dtype, Lambda.device)
        return w

    @staticmethod
    def backward(ctx, grad_w):
        seg = ctx.seg
        gw = grad_w.detach().to(device="cuda", dtype=torch.float32).contiguous()
        seg.stream.wait_stream(torch.cuda.current_stream())
        fbar = torch.empty(ctx.shape, dtype=torch.float32, device="cuda") if ctx.needs_input_grad[0] else None
        dc, dl = B.seg_admm_unrolled_bwd(seg.handle, gw.data_ptr(), ctx.K, ctx.C, ctx.J,
                                         fbar.data_ptr() if fbar is not None else 0)
        cdt, cdev, cshape = ctx.cb_meta
        ldt, ldev = ctx.lam_meta
        gcb = torch.tensor(dc, dtype=cdt, device=cdev).reshape(cshape)
        glam = torch.tensor(dl, dtype=ldt, device=ldev)
        if fbar is not None and ctx.fdim == 2:
            fbar = fbar[0]
        seg.close()
        return fbar, gcb, glam, None, None, None, None


def unrolled_segmentation(f, codebook, Lambda, bank: FilterBank, gamma: float = 1.0, T: int = 50,
                          ckpt_every: int = 10):
    """Differentiable w_T (see UnrolledSegmentation)."""
    return UnrolledSegmentation.apply(f, codebook, Lambda, bank, gamma, T, ckpt_every)
