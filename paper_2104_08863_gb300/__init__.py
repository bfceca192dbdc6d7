"""GB300 (sm_103a) pressure-Poisson projection for the staggered channel of Sec. 2.

Python face of ``libpoisson.so``: ``Plan`` owns a plan and its torch-allocated workspace;
``Plan.solve``, ``Plan.project`` and ``Plan.project_adjoint`` call the C ABI on the current
torch stream; ``ProjectionFn`` wraps the projection and its hand-written adjoint in
``torch.autograd.Function``.  All arithmetic runs in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native
from ._native import (PP_FP64, PP_FP32, PP_FP32_REFINED, PT_AUTO, PT_THOMAS, PT_PDD_EXACT, PT_PDD_TRUNCATED,
                      POISSON_CHECK_FINITE, POISSON_TIMING, POISSON_GENERIC_FFT, POISSON_SELFTEST_WAIT,
                      POISSON_BATCH_PERSISTENT, PoissonError, check)

__all__ = ["Plan", "BatchPlan", "autotune", "tune_batch", "fp64_fma_rate", "ProjectionFn", "PoissonError", "POISSON_GENERIC_FFT", "PP_FP64", "PP_FP32", "PP_FP32_REFINED",
           "PT_AUTO", "PT_THOMAS", "PT_PDD_EXACT", "PT_PDD_TRUNCATED", "POISSON_CHECK_FINITE", "POISSON_TIMING",
           "POISSON_SELFTEST_WAIT", "POISSON_BATCH_PERSISTENT"]


def _ptr(t: torch.Tensor) -> int:
    return t.data_ptr()


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Plan:
    """A planned solve on one grid: nx x ny x nz cells, periodic lx, lz, wall-normal faces."""

    def __init__(self, nx: int, ny: int, nz: int, y_faces, lx: float = 2 * np.pi, lz: float = np.pi,
                 precision: int = PP_FP64, tridiag: int = PT_AUTO, pdd_parts: int = 0,
                 fp64_low_modes: int = 4, refine_steps: int = 1, flags: int = 0, device=None):
        L = _native.lib()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.precision = int(precision)
        self.device = torch.device(device if device is not None else "cuda")
        self._faces = np.ascontiguousarray(np.asarray(y_faces, dtype=np.float64))
        if self._faces.size != self.ny + 1:
            raise ValueError("y_faces must have ny + 1 entries")
        desc = _native.PoissonDesc(self.nx, self.ny, self.nz, float(lx), float(lz),
                                   self._faces.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                   self.precision, int(tridiag), int(pdd_parts), int(fp64_low_modes),
                                   int(refine_steps), int(flags))
        h = ctypes.c_void_p()
        check(L.poisson_plan_create(ctypes.byref(desc), ctypes.byref(h)), "poisson_plan_create")
        self._h = h
        nbytes = ctypes.c_size_t()
        check(L.poisson_workspace_size(h, ctypes.byref(nbytes)), "poisson_workspace_size")
        self.workspace_bytes = int(nbytes.value)
        with torch.cuda.device(self.device):
            self._ws = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
            off = (-self._ws.data_ptr()) % 256
            check(L.poisson_set_workspace(h, self._ws.data_ptr() + off, self.workspace_bytes, _stream()),
                  "poisson_set_workspace")

    @property
    def dtype(self):
        return torch.float32 if self.precision == PP_FP32 else torch.float64

    @property
    def cell_shape(self):
        return (self.ny, self.nz, self.nx)

    @property
    def v_shape(self):
        return (self.ny + 1, self.nz, self.nx)

    def _check(self, t: torch.Tensor, shape, name: str):
        if t.dtype != self.dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"{name}: expected contiguous CUDA {self.dtype} {tuple(shape)}, got "
                             f"{t.dtype} {tuple(t.shape)} contiguous={t.is_contiguous()} device={t.device}")

    def solve(self, rhs: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        self._check(rhs, self.cell_shape, "rhs")
        if out is None:
            out = torch.empty_like(rhs)
        self._check(out, self.cell_shape, "out")
        check(_native.lib().poisson_solve(self._h, _ptr(rhs), _ptr(out), _stream(stream)), "poisson_solve")
        return out

    def solve_adjoint(self, g: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """q = S^T g, the transpose of ``solve`` as a linear map (g is not modified unless out is g)."""
        self._check(g, self.cell_shape, "g")
        if out is None:
            out = torch.empty_like(g)
        self._check(out, self.cell_shape, "out")
        check(_native.lib().poisson_solve_adjoint(self._h, _ptr(g), _ptr(out), _stream(stream)),
              "poisson_solve_adjoint")
        return out

    def project(self, u, v, w, dt: float, p_out=None, stream=None):
        """In-place projection of (u, v, w); returns p_out (or None).

        PP_FP32_REFINED plans need a pressure buffer (it carries the FP64 right-hand side during
        the solve): one is allocated when p_out is None, and returned."""
        self._check(u, self.cell_shape, "u")
        self._check(v, self.v_shape, "v")
        self._check(w, self.cell_shape, "w")
        pp = 0
        if p_out is None and self.precision == PP_FP32_REFINED:
            p_out = torch.empty(self.cell_shape, dtype=torch.float64, device=u.device)
        if p_out is not None:
            self._check(p_out, self.cell_shape, "p_out")
            pp = _ptr(p_out)
        check(_native.lib().projection_step(self._h, _ptr(u), _ptr(v), _ptr(w), pp, float(dt), _stream(stream)),
              "projection_step")
        return p_out

    def _stage_buffers(self, u, v, w, scratch):
        self._check(u, self.cell_shape, "u")
        self._check(v, self.v_shape, "v")
        self._check(w, self.cell_shape, "w")
        if scratch is None:
            scratch = (torch.empty_like(u), torch.empty_like(v), torch.empty_like(w))
        for t, shp, name in zip(scratch, (self.cell_shape, self.v_shape, self.cell_shape), ("ub", "vb", "wb")):
            self._check(t, shp, name)
        return scratch

    def predict(self, u, v, w, dt: float, nu: float, fx: float, scratch=None, stream=None):
        """In place: (u, v, w) <- the RK2 momentum predictor u_star (Eqs. 5-6).

        scratch: optional (ub, vb, wb) device tensors of the field shapes for the first stage."""
        ub, vb, wb = self._stage_buffers(u, v, w, scratch)
        check(_native.lib().momentum_predictor(self._h, _ptr(u), _ptr(v), _ptr(w), _ptr(ub), _ptr(vb), _ptr(wb),
                                               float(dt), float(nu), float(fx), _stream(stream)),
              "momentum_predictor")

    def timestep(self, u, v, w, dt: float, nu: float, fx: float, p_out=None, scratch=None, stream=None):
        """In place: one full timestep (RK2 predictor, then the projection); returns p_out (or None)."""
        ub, vb, wb = self._stage_buffers(u, v, w, scratch)
        pp = 0
        if p_out is not None:
            self._check(p_out, self.cell_shape, "p_out")
            pp = _ptr(p_out)
        check(_native.lib().projection_timestep(self._h, _ptr(u), _ptr(v), _ptr(w), _ptr(ub), _ptr(vb), _ptr(wb), pp,
                                                float(dt), float(nu), float(fx), _stream(stream)),
              "projection_timestep")
        return p_out

    def timestep_host(self, u_h, v_h, w_h, dt: float, nu: float, fx: float, staging, scratch, p_h=None,
                      stream=None):
        """End-to-end timestep of HOST (pinned) tensors through the library's host entry point.

        staging: (u_d, v_d, w_d, p_d) device tensors; scratch: (ub, vb, wb) device tensors."""
        u_d, v_d, w_d, p_d = staging
        ub, vb, wb = scratch
        check(_native.lib().projection_timestep_host(
            self._h, _ptr(u_h), _ptr(v_h), _ptr(w_h), _ptr(p_h) if p_h is not None else 0,
            _ptr(u_d), _ptr(v_d), _ptr(w_d), _ptr(p_d) if p_d is not None else 0, _ptr(ub), _ptr(vb), _ptr(wb),
            float(dt), float(nu), float(fx), _stream(stream)), "projection_timestep_host")

    def project_adjoint(self, gu, gv, gw, stream=None):
        """In place: g <- P^T g (the adjoint of the projection's velocity map)."""
        self._check(gu, self.cell_shape, "gu")
        self._check(gv, self.v_shape, "gv")
        self._check(gw, self.cell_shape, "gw")
        check(_native.lib().projection_step_adjoint(self._h, _ptr(gu), _ptr(gv), _ptr(gw), _stream(stream)),
              "projection_step_adjoint")

    def project_host(self, u_h, v_h, w_h, dt: float, staging, p_h=None, stream=None):
        """End-to-end projection of HOST (pinned) tensors through the library's host entry point."""
        u_d, v_d, w_d, p_d = staging
        check(_native.lib().projection_step_host(
            self._h, _ptr(u_h), _ptr(v_h), _ptr(w_h), _ptr(p_h) if p_h is not None else 0,
            _ptr(u_d), _ptr(v_d), _ptr(w_d), _ptr(p_d) if p_d is not None else 0, float(dt), _stream(stream)),
            "projection_step_host")

    def divergence(self, u, v, w, dt: float = 1.0, out=None, stream=None) -> torch.Tensor:
        """f = D(u)/dt (Eq. 7) on the cell centres (poisson_divergence)."""
        self._check(u, self.cell_shape, "u")
        self._check(v, self.v_shape, "v")
        self._check(w, self.cell_shape, "w")
        if out is None:
            out = torch.empty_like(u)
        self._check(out, self.cell_shape, "out")
        check(_native.lib().poisson_divergence(self._h, _ptr(u), _ptr(v), _ptr(w), _ptr(out), float(dt),
                                               _stream(stream)), "poisson_divergence")
        return out

    def set_chain(self, slab_cols: int, streams: int = 1):
        """Run the FP32 z-transform / wall-normal / inverse z-transform passes in kx slabs of
        slab_cols columns (0: whole spectrum) over 1 or 2 streams (poisson_plan_set_chain)."""
        with torch.cuda.device(self.device):
            check(_native.lib().poisson_plan_set_chain(self._h, int(slab_cols), int(streams)), "poisson_plan_set_chain")

    def device_status(self, stream=None) -> int:
        return int(_native.lib().poisson_device_status(self._h, _stream(stream)))

    def stage_times(self, max_entries: int = 64):
        """[(kernel name, ms)] of every launch of the last call (needs flags=POISSON_TIMING)."""
        ms = (ctypes.c_float * max_entries)()
        names = (ctypes.c_char_p * max_entries)()
        n = _native.lib().poisson_stage_times(self._h, ms, names, max_entries)
        if n < 0:
            raise RuntimeError("stage timing unavailable (plan created without POISSON_TIMING)")
        return [(names[i].decode(), float(ms[i])) for i in range(min(n, max_entries))]

    @property
    def last_launch_count(self) -> int:
        return int(_native.lib().poisson_last_launch_count(self._h))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _native._LIB is not None:
            _native._LIB.poisson_plan_destroy(h)
            self._h = None


def fp64_fma_rate(device=None) -> float:
    """FP64 FMA throughput of the device in GFLOP/s (poisson_fp64_fma_rate; diagnostics)."""
    dev = torch.device(device if device is not None else "cuda")
    with torch.cuda.device(dev):
        props = torch.cuda.get_device_properties(dev)
        scratch = torch.empty(8 * 256 * 8 * props.multi_processor_count, dtype=torch.uint8, device=dev)
        out = ctypes.c_double()
        check(_native.lib().poisson_fp64_fma_rate(scratch.data_ptr(), scratch.numel(), _stream(), ctypes.byref(out)),
              "poisson_fp64_fma_rate")
    return float(out.value)


def _desc(nx, ny, nz, faces, lx, lz, precision, tridiag, pdd_parts, fp64_low_modes, refine_steps, flags):
    faces = np.ascontiguousarray(np.asarray(faces, dtype=np.float64))
    d = _native.PoissonDesc(int(nx), int(ny), int(nz), float(lx), float(lz),
                            faces.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(precision), int(tridiag),
                            int(pdd_parts), int(fp64_low_modes), int(refine_steps), int(flags))
    return d, faces


def autotune(nx, ny, nz, y_faces, lx=2 * np.pi, lz=np.pi, precision=PP_FP32, fp64_low_modes=4, refine_steps=1,
             stream=None):
    """Time every PDD partition count and both FFT tilings on the device; returns (parts, flags, ms)."""
    d, _keep = _desc(nx, ny, nz, y_faces, lx, lz, precision, PT_PDD_EXACT, 0, fp64_low_modes, refine_steps, 0)
    parts, flags, ms = ctypes.c_int(), ctypes.c_uint(), ctypes.c_float()
    check(_native.lib().poisson_autotune(ctypes.byref(d), _stream(stream), ctypes.byref(parts), ctypes.byref(flags),
                                         ctypes.byref(ms)), "poisson_autotune")
    return int(parts.value), int(flags.value), float(ms.value)


class BatchPlan:
    """Independent solves of uneven sizes run as one graph launch (poisson_solve_batched): one graph
    branch per instance, or with persistent=True one persistent kernel over a device work queue.

    specs: sequence of dicts with keys nx, ny, nz, y_faces (and optional lx, lz, pdd_parts,
    flags).  With tune=True each distinct grid is autotuned once (partition count, FFT tiling).
    selftest_wait=True makes the persistent launch's bounded waits run out (diagnostics:
    POISSON_SELFTEST_WAIT).
    """

    def __init__(self, specs, precision=PP_FP32, fp64_low_modes=4, refine_steps=1, tune=False, device=None,
                 persistent=False, selftest_wait=False):
        L = _native.lib()
        self.device = torch.device(device if device is not None else "cuda")
        self.precision = int(precision)
        self.specs = [dict(s) for s in specs]
        cache = {}
        descs = (_native.PoissonDesc * len(self.specs))()
        self._keep = []
        self.tuned = []
        for i, s in enumerate(self.specs):
            lx, lz = s.get("lx", 2 * np.pi), s.get("lz", np.pi)
            parts, flags = s.get("pdd_parts", 0), s.get("flags", 0)
            if tune:
                key = (s["nx"], s["ny"], s["nz"], tuple(np.round(np.asarray(s["y_faces"]), 12)))
                if key not in cache:
                    cache[key] = autotune(s["nx"], s["ny"], s["nz"], s["y_faces"], lx, lz, precision, fp64_low_modes,
                                          refine_steps)
                parts, flags, _ = cache[key]
            self.tuned.append((parts, flags))
            tri = PT_THOMAS if parts == 1 else (PT_PDD_EXACT if parts > 1 else PT_AUTO)
            if i == 0:
                flags |= (POISSON_BATCH_PERSISTENT if persistent else 0) | (POISSON_SELFTEST_WAIT if selftest_wait else 0)
            d, faces = _desc(s["nx"], s["ny"], s["nz"], s["y_faces"], lx, lz, precision, tri, parts, fp64_low_modes,
                             refine_steps, flags)
            descs[i] = d
            self._keep.append(faces)
        h = ctypes.c_void_p()
        check(L.poisson_plan_batched(descs, len(self.specs), ctypes.byref(h)), "poisson_plan_batched")
        self._h = h
        nbytes = ctypes.c_size_t()
        check(L.poisson_workspace_size(h, ctypes.byref(nbytes)), "poisson_workspace_size")
        self.workspace_bytes = int(nbytes.value)
        with torch.cuda.device(self.device):
            self._ws = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
            off = (-self._ws.data_ptr()) % 256
            check(L.poisson_set_workspace(h, self._ws.data_ptr() + off, self.workspace_bytes, _stream()),
                  "poisson_set_workspace")

    @property
    def dtype(self):
        return torch.float32 if self.precision == PP_FP32 else torch.float64

    def solve(self, rhs, out=None, stream=None):
        n = len(self.specs)
        if len(rhs) != n:
            raise ValueError(f"expected {n} right-hand sides")
        out = [torch.empty_like(r) for r in rhs] if out is None else out
        for s, r, o in zip(self.specs, rhs, out):
            shape = (s["ny"], s["nz"], s["nx"])
            for t in (r, o):
                if t.dtype != self.dtype or tuple(t.shape) != shape or not t.is_contiguous() or not t.is_cuda:
                    raise ValueError(f"expected contiguous CUDA {self.dtype} {shape}")
        pr = (ctypes.c_void_p * n)(*[r.data_ptr() for r in rhs])
        po = (ctypes.c_void_p * n)(*[o.data_ptr() for o in out])
        check(_native.lib().poisson_solve_batched(self._h, pr, po, _stream(stream)), "poisson_solve_batched")
        return out

    @property
    def last_launch_count(self) -> int:
        return int(_native.lib().poisson_last_launch_count(self._h))

    def device_status(self, stream=None) -> int:
        """Synchronise and read (then clear) the batch's status word (PS_ETIMEOUT after a wait ran out)."""
        return int(_native.lib().poisson_device_status(self._h, _stream(stream)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _native._LIB is not None:
            _native._LIB.poisson_plan_destroy(h)
            self._h = None


def _max_parts(ny):
    best = 1
    for P in range(2, 33):
        if ny % P == 0 and ny // P >= 4:
            best = P
    return best


def _scan_parts(ny, mmax):
    """The smallest power-of-two partition P <= 32 whose blocks (ny / P rows, one of the heights of
    the warp-scan PDD tiles) have at most mmax rows, else 0."""
    for P in (1, 2, 4, 8, 16, 32):
        if ny % P == 0 and ny // P <= mmax and ny // P in (1, 2, 3, 4, 6, 8, 12, 16, 24):
            return P
    return 0


def tune_batch(specs, precision=PP_FP32, fp64_low_modes=4, refine_steps=1, device=None, repeats=3):
    """Batch-level autotuner: time whole batched graph launches on the device for several strategies
    and return (best BatchPlan, {strategy: ms}).  Strategies: one graph branch per instance with the
    plan's partition model, with per-shape autotuning (poisson_autotune: partition count and FFT
    tiling), with Thomas everywhere, with the largest partition count; and the persistent
    work-queue launch with blocks of at most 16 or at most 8 rows."""
    dev = torch.device(device if device is not None else "cuda")
    dtype = torch.float32 if precision == PP_FP32 else torch.float64
    gen = torch.Generator(device=dev)
    gen.manual_seed(0)
    rhs = [torch.randn(s["ny"], s["nz"], s["nx"], dtype=dtype, device=dev, generator=gen) for s in specs]
    outs = [torch.empty_like(r) for r in rhs]
    strategies = {
        "model": [dict(s) for s in specs],
        "thomas": [dict(s, pdd_parts=1) for s in specs],
        "max_parts": [dict(s, pdd_parts=_max_parts(s["ny"])) for s in specs],
        "persistent": [dict(s) for s in specs],
        "persistent_m8": [dict(s, pdd_parts=_scan_parts(s["ny"], 8)) for s in specs],
    }
    times, best, best_ms = {}, None, None
    for name in ("model", "per_shape", "thomas", "max_parts", "persistent", "persistent_m8"):
        if name == "persistent_m8" and (precision != PP_FP32 or any(s["pdd_parts"] == 0 for s in strategies[name])):
            continue
        bp = BatchPlan(specs if name == "per_shape" else strategies[name], precision, fp64_low_modes, refine_steps,
                       tune=(name == "per_shape"), device=dev, persistent=name.startswith("persistent"))
        bp.solve(rhs, out=outs)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(repeats):
            bp.solve(rhs, out=outs)
        e1.record()
        torch.cuda.synchronize(dev)
        ms = e0.elapsed_time(e1) / repeats
        times[name] = ms
        if best_ms is None or ms < best_ms:
            best, best_ms = bp, ms
        else:
            del bp
    best.strategy_times = times
    return best, times


class ProjectionFn(torch.autograd.Function):
    """u = P(u*) (Eqs. 4, 7) with the hand-written adjoint backward P^T (same FFT/PDD kernels)."""

    @staticmethod
    def forward(ctx, u, v, w, plan: Plan, dt: float):
        ctx.plan = plan
        uo, vo, wo = u.detach().clone(), v.detach().clone(), w.detach().clone()
        plan.project(uo, vo, wo, dt)
        return uo, vo, wo

    @staticmethod
    def backward(ctx, gu, gv, gw):
        plan = ctx.plan
        gu = gu.detach().clone().contiguous()
        gv = gv.detach().clone().contiguous()
        gw = gw.detach().clone().contiguous()
        plan.project_adjoint(gu, gv, gw)
        return gu, gv, gw, None, None
