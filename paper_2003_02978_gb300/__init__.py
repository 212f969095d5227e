"""GB300-native sparse, albedo-corrected matched filter (Foote et al., IEEE TGRS
2020): Python binding of libmf.so.

Every step of the retrieval runs in the library's CUDA kernels; this module
only marshals arguments (device pointers of torch tensors, the current CUDA
stream).  There is no CPU path: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np
import torch

from ._native import MfDesc, MFError, MfTuning, check, lib

ALBEDO = 1
SPARSE = 2
LITERAL = 4
PENALTY_NO_ALBEDO = 8
PERSISTENT = 16  # one work-queue launch after the statistics pass (fused schedule)
FP32 = 0
BF16SPLIT = 1
DEFAULT_FLAGS = ALBEDO | SPARSE

# the six variants of Table I: (n_iter > 0, flags)
TABLE_I = {
    "reference_rmf": (False, 0),
    "albedo_only_mf": (False, ALBEDO),
    "iter_pos_no_albedo": (True, 0),
    "iter_pos_albedo": (True, ALBEDO),
    "rwl1mf": (True, SPARSE),
    "albedo_rwl1mf": (True, ALBEDO | SPARSE),
}

__all__ = ["Plan", "BatchPlan", "Retrieve", "retrieve_differentiable", "retrieve", "MFError", "ALBEDO", "SPARSE", "LITERAL", "PENALTY_NO_ALBEDO", "PERSISTENT",
           "FP32", "BF16SPLIT", "TABLE_I", "library_path"]


def library_path() -> str:
    from ._native import LIB_PATH
    return LIB_PATH


_KINDS = ("stats", "pixel", "solve", "queue")  # launch kinds of the profile and timeline


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _flags(flags, tuning) -> int:
    """Plan flags, with PERSISTENT when the tuning asks for the work-queue
    schedule (``tuning["persistent"]``, as the autotuner may choose)."""
    return int(flags) | (PERSISTENT if (tuning or {}).get("persistent") else 0)


def _tuning(t) -> MfTuning:
    """mf_tuning from a dict {pixel_rows, stat_rows, use_graph} (0 = default)."""
    return MfTuning(pixel_rows=int(t.get("pixel_rows", 0)), stat_rows=int(t.get("stat_rows", 0)),
                    use_graph=int(t.get("use_graph", 0)))


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass(frozen=True)
class Shape:
    rows: int
    cols: int
    bands_total: int
    band_lo: int
    band_hi: int
    col_group: int
    flags: int
    precision: int


class Plan:
    """A retrieval plan: validated shape plus all device workspace (allocated
    once, on the current CUDA device).  ``retrieve`` allocates nothing."""

    def __init__(self, rows, cols, bands_total, band_lo=0, band_hi=None, col_group=1,
                 flags=DEFAULT_FLAGS, precision=FP32, tuning=None):
        band_hi = bands_total if band_hi is None else band_hi
        flags = _flags(flags, tuning)
        self.shape = Shape(int(rows), int(cols), int(bands_total), int(band_lo), int(band_hi),
                           int(col_group), int(flags), int(precision))
        d = MfDesc(rows=rows, cols=cols, bands_total=bands_total, band_lo=band_lo,
                   band_hi=band_hi, col_group=col_group, layout=0, precision=precision,
                   flags=flags)
        h = ctypes.c_void_p()
        if tuning is None:
            check(lib().mf_plan(ctypes.byref(d), ctypes.byref(h)), "mf_plan")
        else:
            t = _tuning(tuning)
            check(lib().mf_plan_ex(ctypes.byref(d), None, 1, ctypes.byref(t), ctypes.byref(h)),
                  "mf_plan_ex")
        self.tuning = tuning
        self._h = h
        self.B = band_hi - band_lo
        self.P = int(lib().mf_num_partitions(h))

    def close(self):
        if getattr(self, "_h", None):
            lib().mf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check_cube(self, cube):
        s = self.shape
        if not (isinstance(cube, torch.Tensor) and cube.is_cuda and cube.dtype == torch.float32):
            raise TypeError("cube must be a CUDA float32 tensor")
        if tuple(cube.shape) != (s.rows, s.cols, s.bands_total) or not cube.is_contiguous():
            raise ValueError(f"cube must be contiguous {(s.rows, s.cols, s.bands_total)}")

    def retrieve(self, cube, k, lam, eps, n_iter, mask=None, alpha_init=None, out=None,
                 albedo=None, stream=None):
        """Enqueue one retrieval on ``stream`` (default: current stream).
        Returns ``out`` (rows, cols) float32 alpha."""
        s = self.shape
        self._check_cube(cube)
        k = torch.as_tensor(k, dtype=torch.float32, device=cube.device).contiguous()
        if k.numel() != self.B:
            raise ValueError(f"k must have {self.B} entries")
        if mask is not None:
            if mask.dtype != torch.uint8 or tuple(mask.shape) != (s.rows, s.cols) or \
                    not mask.is_cuda or not mask.is_contiguous():
                raise ValueError("mask must be a contiguous CUDA uint8 (rows, cols) tensor")
        if alpha_init is not None:
            alpha_init = alpha_init.to(device=cube.device, dtype=torch.float32).contiguous()
        if out is None:
            out = torch.empty((s.rows, s.cols), dtype=torch.float32, device=cube.device)
        check(lib().mf_retrieve(self._h, _ptr(cube), _ptr(k), float(lam), float(eps),
                                int(n_iter), _ptr(mask), _ptr(alpha_init), _ptr(out),
                                _ptr(albedo), _stream_handle(stream)), "mf_retrieve")
        self._k_keepalive = k
        return out

    def retrieve_host(self, cube, k, lam, eps, n_iter, mask=None, out=None, stream=None):
        """Host-buffer retrieval (numpy arrays or CPU tensors, pinned or not):
        copies in, retrieves, copies alpha back, synchronises."""
        s = self.shape
        cube = torch.as_tensor(cube)
        assert cube.dtype == torch.float32 and cube.is_contiguous() and not cube.is_cuda
        k = torch.as_tensor(np.asarray(k, dtype=np.float32)).contiguous()
        if mask is not None:
            mask = torch.as_tensor(mask).to(torch.uint8).contiguous()
        if out is None:
            out = torch.empty((s.rows, s.cols), dtype=torch.float32)
        check(lib().mf_retrieve_host(self._h, _ptr(cube), _ptr(k), float(lam), float(eps),
                                     int(n_iter), _ptr(mask), _ptr(out), _stream_handle(stream)),
              "mf_retrieve_host")
        return out

    def retrieve_host_async(self, cube, k, lam, eps, n_iter, mask=None, out=None, stream=None):
        """Host-buffer retrieval for a stream of cubes (mf_retrieve_host_async):
        cube, mask and out pinned CPU tensors; returns at once, the copy of
        the next call's cube overlapping this call's retrieval.  ``out`` holds
        alpha once ``stream`` (default: the current stream) is synchronised;
        the tensors must stay alive and unchanged until then."""
        s = self.shape
        assert cube.dtype == torch.float32 and cube.is_contiguous() and cube.is_pinned()
        k = torch.as_tensor(np.asarray(k, dtype=np.float32)).contiguous()
        if mask is not None:
            assert mask.dtype == torch.uint8 and mask.is_contiguous() and mask.is_pinned()
        if out is None:
            out = torch.empty((s.rows, s.cols), dtype=torch.float32).pin_memory()
        assert out.is_pinned()
        self._async_k = k  # kept alive with the call (its copy is staged)
        check(lib().mf_retrieve_host_async(self._h, _ptr(cube), _ptr(k), float(lam), float(eps),
                                           int(n_iter), _ptr(mask), _ptr(out),
                                           _stream_handle(stream)),
              "mf_retrieve_host_async")
        return out

    def ckpt_bytes(self, n_iter, cube_grad=False) -> int:
        return int(lib().mf_ckpt_bytes(self._h, int(n_iter), int(bool(cube_grad))))

    def retrieve_energy(self, cube, k, lam, eps, n_iter, mask=None, out=None, stream=None):
        """Retrieval that also returns the objective of every iterate (the
        energy of Fig. 5): (alpha (rows, cols) float32, energy (P, n_iter + 1)
        float64), both CUDA tensors (mf_retrieve_energy)."""
        s = self.shape
        self._check_cube(cube)
        k = torch.as_tensor(k, dtype=torch.float32, device=cube.device).contiguous()
        if out is None:
            out = torch.empty((s.rows, s.cols), dtype=torch.float32, device=cube.device)
        energy = torch.empty((self.P, int(n_iter) + 1), dtype=torch.float64, device=cube.device)
        check(lib().mf_retrieve_energy(self._h, _ptr(cube), _ptr(k), float(lam), float(eps),
                                       int(n_iter), _ptr(mask), _ptr(out), _ptr(energy),
                                       _stream_handle(stream)),
              "mf_retrieve_energy")
        return out, energy

    def retrieve_train(self, cube, k, lam, eps, n_iter, mask=None, cube_grad=False, out=None,
                       ckpt=None, stream=None):
        """Checkpointed retrieval for the backward pass.  Returns (alpha,
        ckpt), ckpt a uint8 CUDA tensor holding the checkpoint (allocated
        here unless given)."""
        s = self.shape
        self._check_cube(cube)
        k = torch.as_tensor(k, dtype=torch.float32, device=cube.device).contiguous()
        if ckpt is None:
            ckpt = torch.empty(self.ckpt_bytes(n_iter, cube_grad) + 256, dtype=torch.uint8,
                               device=cube.device)
        off = (-ckpt.data_ptr()) % 256
        if out is None:
            out = torch.empty((s.rows, s.cols), dtype=torch.float32, device=cube.device)
        check(lib().mf_retrieve_train(self._h, _ptr(cube), _ptr(k), float(lam), float(eps),
                                      int(n_iter), _ptr(mask), _ptr(out),
                                      ctypes.c_void_p(ckpt.data_ptr() + off),
                                      int(bool(cube_grad)), _stream_handle(stream)),
              "mf_retrieve_train")
        self._train = (k, mask, ckpt, off, bool(cube_grad))
        return out, ckpt

    def backward(self, ckpt, grad_alpha, cube_grad=False, stream=None):
        """Adjoint of the last retrieve_train for grad_alpha (rows, cols):
        (grad_k (B,), grad_lambda (), grad_cube (rows, cols, B) or None)."""
        s = self.shape
        k, mask, ck, off, has_cube = self._train
        assert ck is ckpt, "ckpt must be the one returned by retrieve_train"
        dev = ck.device
        g = grad_alpha.to(device=dev, dtype=torch.float32).contiguous()
        grad_k = torch.empty(self.B, dtype=torch.float32, device=dev)
        grad_l = torch.empty((), dtype=torch.float32, device=dev)
        grad_c = torch.empty((s.rows, s.cols, self.B), dtype=torch.float32, device=dev) \
            if cube_grad else None
        check(lib().mf_retrieve_backward(self._h, ctypes.c_void_p(ck.data_ptr() + off), _ptr(g),
                                         _ptr(grad_k), _ptr(grad_l), _ptr(grad_c),
                                         _stream_handle(stream)), "mf_retrieve_backward")
        return grad_k, grad_l, grad_c

    def status(self) -> np.ndarray:
        st = (ctypes.c_int32 * self.P)()
        lib().mf_plan_status(self._h, st)
        return np.frombuffer(st, dtype=np.int32).copy()

    def background(self, stream=None):
        """(mu0 (P, B), cov0 (P, B, B)) float64 CUDA tensors of the last retrieval."""
        mu = torch.empty((self.P, self.B), dtype=torch.float64, device="cuda")
        cov = torch.empty((self.P, self.B, self.B), dtype=torch.float64, device="cuda")
        check(lib().mf_background(self._h, _ptr(mu), _ptr(cov), _stream_handle(stream)),
              "mf_background")
        return mu, cov

    def profile(self, enable: bool = True):
        check(lib().mf_profile(self._h, int(enable)), "mf_profile")

    def profile_read(self):
        """{'stats'|'pixel'|'solve'|'queue': (ms, launches)} since the last read
        ('queue': the persistent work-queue launch of an MF_PERSISTENT plan)."""
        ms = (ctypes.c_double * 4)()
        n = (ctypes.c_int64 * 4)()
        check(lib().mf_profile_read(self._h, ms, n, 4), "mf_profile_read")
        return {name: (ms[i], n[i]) for i, name in enumerate(_KINDS)}

    def timeline(self, enable: bool = True):
        """Device timeline of each retrieval as it runs (graph replay included)."""
        check(lib().mf_timeline(self._h, int(enable)), "mf_timeline")

    def timeline_read(self, cap: int = 4096):
        """[(kind, start_us, end_us)] of the last retrieval's launches, kind
        'stats' | 'pixel' | 'solve' | 'queue', times after its earliest start (None for a
        launch that ran no CTA); clears the timeline."""
        t0 = (ctypes.c_double * cap)()
        t1 = (ctypes.c_double * cap)()
        kd = (ctypes.c_int32 * cap)()
        n = ctypes.c_int32(0)
        check(lib().mf_timeline_read(self._h, t0, t1, kd, int(cap), ctypes.byref(n)),
              "mf_timeline_read")
        return [(_KINDS[kd[i]], None if t0[i] < 0 else t0[i], None if t1[i] < 0 else t1[i])
                for i in range(n.value)]


class BatchPlan(Plan):
    """A plan over many flightlines stacked along rows (``line_rows[l]`` rows
    each; same cols, band window, flags and precision): one retrieval covers
    every line, each with its own partitions, lambda and iteration count."""

    def __init__(self, line_rows, cols, bands_total, band_lo=0, band_hi=None, col_group=1,
                 flags=DEFAULT_FLAGS, precision=FP32, tuning=None):
        line_rows = [int(r) for r in line_rows]
        band_hi = bands_total if band_hi is None else band_hi
        flags = _flags(flags, tuning)
        rows = sum(line_rows)
        self.shape = Shape(rows, int(cols), int(bands_total), int(band_lo), int(band_hi),
                           int(col_group), int(flags), int(precision))
        d = MfDesc(rows=rows, cols=cols, bands_total=bands_total, band_lo=band_lo,
                   band_hi=band_hi, col_group=col_group, layout=0, precision=precision,
                   flags=flags)
        lr = (ctypes.c_int64 * len(line_rows))(*line_rows)
        h = ctypes.c_void_p()
        t = _tuning(tuning or {})
        check(lib().mf_plan_ex(ctypes.byref(d), lr, len(line_rows), ctypes.byref(t),
                               ctypes.byref(h)), "mf_plan_ex")
        self.tuning = tuning
        self._h = h
        self.line_rows = line_rows
        self.n_lines = int(lib().mf_num_lines(h))
        self.B = band_hi - band_lo
        self.P = int(lib().mf_num_partitions(h))

    def retrieve(self, cube, k, lam, eps, n_iter, mask=None, out=None, stream=None):
        """Enqueue one retrieval of every line.  ``lam`` and ``n_iter`` are
        per-line sequences (or scalars for all lines); returns ``out``
        (total rows, cols) float32 alpha, stacked like the cube."""
        s = self.shape
        self._check_cube(cube)
        k = torch.as_tensor(k, dtype=torch.float32, device=cube.device).contiguous()
        if k.numel() != self.B:
            raise ValueError(f"k must have {self.B} entries")
        lam = np.broadcast_to(np.asarray(lam, dtype=np.float64), (self.n_lines,))
        n_iter = np.broadcast_to(np.asarray(n_iter, dtype=np.int32), (self.n_lines,))
        lam_c = (ctypes.c_double * self.n_lines)(*lam.tolist())
        nit_c = (ctypes.c_int32 * self.n_lines)(*n_iter.tolist())
        if mask is not None:
            if mask.dtype != torch.uint8 or tuple(mask.shape) != (s.rows, s.cols) or \
                    not mask.is_cuda or not mask.is_contiguous():
                raise ValueError("mask must be a contiguous CUDA uint8 (rows, cols) tensor")
        if out is None:
            out = torch.empty((s.rows, s.cols), dtype=torch.float32, device=cube.device)
        check(lib().mf_retrieve_batched(self._h, _ptr(cube), _ptr(k), lam_c, float(eps), nit_c,
                                        _ptr(mask), _ptr(out), _stream_handle(stream)),
              "mf_retrieve_batched")
        self._k_keepalive = k
        return out

    def line_slices(self):
        """Row slice of every line in the stacked cube."""
        out, r0 = [], 0
        for r in self.line_rows:
            out.append(slice(r0, r0 + r))
            r0 += r
        return out


class Retrieve(torch.autograd.Function):
    """alpha = retrieval(cube, k, lam) as a differentiable operation: forward
    through mf_retrieve_train, backward through mf_retrieve_backward (the
    hand-written adjoint).  Gradients for cube (band window), k and lam."""

    @staticmethod
    def forward(ctx, cube, k, lam, plan, eps, n_iter, mask, cube_grad):
        alpha, ckpt = plan.retrieve_train(cube.detach(), k.detach(), float(lam), eps, n_iter,
                                          mask=mask, cube_grad=cube_grad)
        ctx.plan, ctx.ckpt, ctx.cube_grad = plan, ckpt, cube_grad
        ctx.lam_shape = lam.shape if isinstance(lam, torch.Tensor) else None
        return alpha

    @staticmethod
    def backward(ctx, grad_alpha):
        need_cube = ctx.cube_grad and ctx.needs_input_grad[0]
        gk, gl, gc = ctx.plan.backward(ctx.ckpt, grad_alpha, cube_grad=need_cube)
        if gc is not None and gc.shape[-1] != ctx.plan.shape.bands_total:
            full = torch.zeros((*gc.shape[:2], ctx.plan.shape.bands_total), dtype=gc.dtype,
                               device=gc.device)
            full[..., ctx.plan.shape.band_lo:ctx.plan.shape.band_hi] = gc
            gc = full
        if ctx.lam_shape is not None:
            gl = gl.reshape(ctx.lam_shape)
        return gc, gk, gl, None, None, None, None, None


def retrieve_differentiable(cube, k, lam, eps=1e-9, n_iter=10, mask=None, plan=None,
                            cube_grad=True):
    """Differentiable retrieval: gradients flow to cube (if cube_grad), k and
    lam (a tensor) through the library's adjoint."""
    if plan is None:
        rows, cols, bt = cube.shape
        plan = Plan(rows, cols, bt)
    lam_t = lam if isinstance(lam, torch.Tensor) else torch.tensor(float(lam))
    return Retrieve.apply(cube, k, lam_t, plan, eps, n_iter, mask, cube_grad)


_PLANS: dict = {}


def retrieve(cube, k, lam=1e-3, eps=1e-9, n_iter=10, mask=None, alpha_init=None, band_lo=0,
             band_hi=None, col_group=1, flags=DEFAULT_FLAGS, precision=FP32, albedo=False):
    """Albedo-corrected reweighted-l1 matched filter on a CUDA cube
    (rows, cols, bands_total); returns alpha (rows, cols) [and r_i]."""
    rows, cols, bt = cube.shape
    key = (rows, cols, bt, band_lo, band_hi, col_group, flags, precision, cube.device.index)
    plan = _PLANS.get(key)
    if plan is None:
        plan = _PLANS[key] = Plan(rows, cols, bt, band_lo, band_hi, col_group, flags, precision)
    alb = torch.empty((rows, cols), dtype=torch.float32, device=cube.device) if albedo else None
    a = plan.retrieve(cube, k, lam, eps, n_iter, mask=mask, alpha_init=alpha_init, albedo=alb)
    return (a, alb) if albedo else a
