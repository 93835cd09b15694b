"""Python face of libcollage: a handle class over the C ABI and a torch.autograd.Function.

PyTorch supplies device memory and streams only; rendering, losses, gradients and Adam all run in
libcollage's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dptr(t: torch.Tensor):
    if not t.is_cuda or not t.is_contiguous() or t.dtype != torch.float32:
        raise ValueError("expected a contiguous float32 CUDA tensor")
    return C.c_void_p(t.data_ptr())


class Collage:
    """One handle: n independent collage problems (n > 1 is the batched form)."""

    def __init__(self, problems, **options):
        if isinstance(problems, dict):
            problems = [problems]
        self.lib = L.load()
        self.opts = L.make_options(**options)
        arrs = [L.ProblemArrays(p) for p in problems]
        structs = (L.collage_problem * len(arrs))(*[a.struct for a in arrs])
        h = C.c_void_p()
        L.check(self.lib.collage_create(structs, len(arrs), C.byref(self.opts), C.byref(h)))
        self.h = h
        self.n_probs = len(arrs)
        self.n_elems = int(sum(len(a.kind) for a in arrs))
        self.n_pts = int(sum(int(a.pt_off[-1]) for a in arrs))

    def close(self):
        if getattr(self, "h", None):
            self.lib.collage_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        L.check(st, self.h)

    # level / info -----------------------------------------------------------------------------
    def set_level(self, level: int):
        self._check(self.lib.collage_set_level(self.h, level))

    def info(self) -> dict:
        i = L.collage_info()
        self._check(self.lib.collage_get_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in L.collage_info._fields_}

    # hot path -----------------------------------------------------------------------------------
    def render(self):
        n = self.info()["total_pixels"]
        bw = torch.empty(n, device="cuda", dtype=torch.float32)
        tau = torch.empty(n, device="cuda", dtype=torch.float32)
        self._check(self.lib.collage_render(self.h, _stream(), _dptr(bw), _dptr(tau)))
        return bw, tau

    def loss_backward(self):
        terms = torch.empty(self.n_probs * 5, device="cuda", dtype=torch.float32)
        grad = torch.empty(self.n_elems * 4, device="cuda", dtype=torch.float32)
        self._check(self.lib.collage_loss_backward(self.h, _stream(), _dptr(terms), _dptr(grad)))
        return terms.view(self.n_probs, 5), grad.view(self.n_elems, 4)

    def step(self, n_iters: int = 1):
        self._check(self.lib.collage_step(self.h, _stream(), n_iters))

    def step_async(self, n_iters: int = 1):
        """Enqueue n_iters iterations without waiting; sync() reports a latched overflow."""
        self._check(self.lib.collage_step_async(self.h, _stream(), n_iters))

    def run_schedule(self):
        self._check(self.lib.collage_run_schedule(self.h, _stream()))

    def step_host(self, n_iters, params_in=None, want_params=True, want_loss=True):
        pin = None if params_in is None else np.ascontiguousarray(params_in, np.float32)
        pout = np.empty(self.n_elems * 4, np.float32) if want_params else None
        lout = np.empty(self.n_probs * 5, np.float32) if want_loss else None
        vp = lambda a: None if a is None else a.ctypes.data_as(C.c_void_p)
        self._check(self.lib.collage_step_host(self.h, _stream(), n_iters, vp(pin), vp(pout), vp(lout)))
        return pout, lout

    def loss(self):
        t = torch.empty(self.n_probs * 5, device="cuda", dtype=torch.float32)
        self._check(self.lib.collage_get_loss(self.h, _stream(), _dptr(t)))
        return t.view(self.n_probs, 5)

    # params / state -----------------------------------------------------------------------------
    def get_params(self) -> torch.Tensor:
        t = torch.empty(self.n_elems * 4, device="cuda", dtype=torch.float32)
        self._check(self.lib.collage_get_params(self.h, _stream(), _dptr(t)))
        return t.view(self.n_elems, 4)

    def set_params(self, params: torch.Tensor):
        p = params.detach().reshape(-1).contiguous().float()
        self._check(self.lib.collage_set_params(self.h, _stream(), _dptr(p)))

    # skeleton-based initialisation ------------------------------------------------------------
    def mat_init(self, want_maps: bool = False):
        """Place the elements along the container's medial axis (collage_mat_init); with want_maps,
        also return the axis mask (int32) and the medial width (float32) of every pixel."""
        axis = width = None
        if want_maps:
            n = self.info()["total_pixels"]
            axis = torch.empty(n, device="cuda", dtype=torch.int32)
            width = torch.empty(n, device="cuda", dtype=torch.float32)
        self._check(self.lib.collage_mat_init(
            self.h, _stream(), None if axis is None else C.c_void_p(axis.data_ptr()),
            None if width is None else _dptr(width)))
        return axis, width

    # outline points (fit_controls) ------------------------------------------------------------
    def get_controls(self) -> torch.Tensor:
        t = torch.empty(self.n_pts * 2, device="cuda", dtype=torch.float32)
        self._check(self.lib.collage_get_controls(self.h, _stream(), _dptr(t)))
        return t.view(self.n_pts, 2)

    def set_controls(self, pts: torch.Tensor):
        p = pts.detach().reshape(-1).contiguous().float()
        if p.numel() != 2 * self.n_pts:
            raise ValueError(f"expected {2 * self.n_pts} floats")
        self._check(self.lib.collage_set_controls(self.h, _stream(), _dptr(p)))

    def control_grad(self) -> torch.Tensor:
        t = torch.empty(self.n_pts * 2, device="cuda", dtype=torch.float32)
        self._check(self.lib.collage_get_control_grad(self.h, _stream(), _dptr(t)))
        return t.view(self.n_pts, 2)

    def get_state(self):
        t = torch.empty(self.n_elems * 12, device="cuda", dtype=torch.float32)
        step, level = C.c_int(), C.c_int()
        self._check(self.lib.collage_get_state(self.h, _stream(), _dptr(t), C.byref(step), C.byref(level)))
        return t, step.value, level.value

    def set_state(self, state: torch.Tensor, step: int, level: int):
        s = state.detach().reshape(-1).contiguous().float()
        self._check(self.lib.collage_set_state(self.h, _stream(), _dptr(s), step, level))

    # inspection ---------------------------------------------------------------------------------
    def bins(self):
        n = C.c_int()
        self._check(self.lib.collage_get_bins(self.h, _stream(), None, None, 0, C.byref(n)))
        t = torch.empty(max(n.value, 1), device="cuda", dtype=torch.int32)
        e = torch.empty(max(n.value, 1), device="cuda", dtype=torch.int32)
        self._check(self.lib.collage_get_bins(self.h, _stream(), C.c_void_p(t.data_ptr()),
                                              C.c_void_p(e.data_ptr()), n.value, C.byref(n)))
        return t[:n.value].cpu().numpy(), e[:n.value].cpu().numpy()

    def stage_times(self, n_iters=10):
        out = (C.c_float * L.N_STAGES)()
        self._check(self.lib.collage_stage_times(self.h, _stream(), n_iters, out))
        return dict(zip(L.STAGES, list(out)))

    def autotune(self):
        best = C.c_float()
        self._check(self.lib.collage_autotune(self.h, _stream(), C.byref(best)))
        return self.info()["tile"], best.value

    def tuning(self) -> dict:
        t = L.collage_tuning()
        self._check(self.lib.collage_get_tuning(self.h, C.byref(t)))
        return {f: getattr(t, f) for f, _ in L.collage_tuning._fields_}

    def set_tuning(self, **choice):
        """Applies a launch configuration (the keys of tuning(); missing ones keep their values)."""
        cur = self.tuning()
        cur.update(choice)
        t = L.collage_tuning(**{f: cur[f] for f, _ in L.collage_tuning._fields_})
        self._check(self.lib.collage_set_tuning(self.h, _stream(), C.byref(t)))

    def metrics(self):
        """[n_probs, 8]: object-in-shape, shape, overlap, object-outside-shape pixel counts, then
        LC, OO, EA and L-nU (Sec. 6 and Sec. 6.1) at the current params."""
        out = np.zeros((self.n_probs, 8), np.float64)
        self._check(self.lib.collage_metrics(self.h, _stream(), out.ctypes.data_as(C.c_void_p)))
        return out

    def sync(self):
        self._check(self.lib.collage_sync(self.h, _stream()))


class CollageLoss(torch.autograd.Function):
    """L(params) of Eq. 8 (summed over the handle's problems) with the library's adjoint."""

    @staticmethod
    def forward(ctx, params: torch.Tensor, col: Collage):
        col.set_params(params)
        terms, grad = col.loss_backward()
        ctx.save_for_backward(grad.clone())
        ctx.shape = params.shape
        return terms[:, 4].sum()

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad.reshape(ctx.shape), None


def collage_loss(params: torch.Tensor, col: Collage) -> torch.Tensor:
    return CollageLoss.apply(params, col)
