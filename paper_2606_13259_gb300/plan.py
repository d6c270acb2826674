"""PyTorch-facing plan object over the C-ABI (argument marshalling only).

Every computation runs in the CUDA library; this module only checks tensor
shapes, dtypes and devices, passes raw pointers and the current CUDA stream,
and wraps the results.  Tensors must live on the CUDA device of the plan.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import numpy as np
import torch

from . import _lib as L

STORAGE = {"f32": L.DAS_STORE_F32, "f16": L.DAS_STORE_F16, "bf16": L.DAS_STORE_BF16, "e4m3": L.DAS_STORE_E4M3,
           "e5m2": L.DAS_STORE_E5M2}


def _stream(stream: Optional[torch.cuda.Stream]) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _ptr(t: torch.Tensor) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


class Plan:
    """A delay-and-sum plan: grid, receive array, transmits, c, fs, f_demod,
    f-number (paper Sec. 2), resident on the current CUDA device.

    elem_pos: (M, 3) metres; elem_normal: (M, 3) unit vectors or None (+z);
    grid: (nx, ny, nz); origin, spacing: metres; tx_kind: (Q,) of
    DAS_TX_DIVERGING / DAS_TX_PLANE / DAS_TX_NONE; tx_vec: (Q, 3) virtual
    sources (m) or unit propagation directions; w_tx: optional (Q, N) transmit
    weights; iq: complex IQ data (else real RF); storage: "f32", "f16", "bf16".
    """

    def __init__(self, elem_pos, grid: Sequence[int], origin, spacing, tx_kind, tx_vec, *, c: float, fs: float,
                 f_demod: float = 0.0, f_number: float = 1.0, n_samples: int, iq: bool,
                 elem_normal=None, t0_ref=(0.0, 0.0, 0.0), t0_offset: bool = True, w_tx=None,
                 storage: str = "f32", max_batch: int = 1):
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2606_13259_gb300.Plan needs a CUDA device")
        lib = L.lib()
        self._lib = lib
        pos = np.ascontiguousarray(np.asarray(elem_pos, dtype=np.float64).reshape(-1, 3))
        nrm = None if elem_normal is None else np.ascontiguousarray(np.asarray(elem_normal, np.float64).reshape(-1, 3))
        kinds = np.asarray(tx_kind, dtype=np.int32).reshape(-1)
        vecs = np.asarray(tx_vec, dtype=np.float64).reshape(-1, 3)
        nx, ny, nz = (int(v) for v in grid)
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.M, self.Q, self.K = pos.shape[0], kinds.shape[0], int(n_samples)
        self.iq = bool(iq)
        self.max_batch = int(max_batch)
        self.storage = storage
        self.device = torch.device("cuda", torch.cuda.current_device())
        self._c = float(c)

        geom = L.Geometry()
        geom.n_elements = self.M
        geom.positions = pos.ctypes.data_as(C.POINTER(C.c_double))
        geom.normals = nrm.ctypes.data_as(C.POINTER(C.c_double)) if nrm is not None else None
        geom.t0_ref = (C.c_double * 3)(*t0_ref)
        g = L.Grid()
        g.nx, g.ny, g.nz = nx, ny, nz
        g.origin = (C.c_double * 3)(*origin)
        g.spacing = (C.c_double * 3)(*spacing)
        txs = (L.Tx * self.Q)()
        wtx = None if w_tx is None else np.ascontiguousarray(np.asarray(w_tx, np.float32).reshape(self.Q, self.N))
        for q in range(self.Q):
            txs[q].kind = int(kinds[q])
            txs[q].vec = (C.c_double * 3)(*vecs[q])
            txs[q].w_tx = wtx[q].ctypes.data_as(C.POINTER(C.c_float)) if wtx is not None else None
        opt = L.Options()
        opt.n_samples = self.K
        opt.sample_type = L.DAS_SAMPLE_C64 if self.iq else L.DAS_SAMPLE_F32
        opt.storage = STORAGE[storage]
        opt.max_batch = self.max_batch
        opt.t0_offset = int(bool(t0_offset))
        handle = C.c_void_p()
        L.check(lib.das_plan_create(C.byref(handle), C.byref(geom), C.byref(g), txs, self.Q, float(c), float(fs),
                                    float(f_demod), float(f_number), C.byref(opt)))
        self._h = handle

    @classmethod
    def from_scene(cls, scene, storage: str = "f32", max_batch: int = 1, c: Optional[float] = None) -> "Plan":
        """Build from any object with the attributes of a scene description
        (nx, ny, nz, origin, spacing, elem_pos, elem_normal, tx_kind, tx_vec,
        t0_ref, t0_offset, c, fs, f_demod, f_number, K, iq, w_tx)."""
        return cls(scene.elem_pos, (scene.nx, scene.ny, scene.nz), scene.origin, scene.spacing, scene.tx_kind,
                   scene.tx_vec, c=scene.c if c is None else c, fs=scene.fs, f_demod=scene.f_demod,
                   f_number=scene.f_number, n_samples=scene.K, iq=scene.iq, elem_normal=scene.elem_normal,
                   t0_ref=scene.t0_ref, t0_offset=scene.t0_offset, w_tx=scene.w_tx, storage=storage,
                   max_batch=max_batch)

    # ------------------------------------------------------------------ state

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.das_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def c(self) -> float:
        return self._c

    def set_c(self, c: float) -> None:
        L.check(self._lib.das_plan_set_c(self._h, float(c)))
        self._c = float(c)

    def info(self) -> dict:
        i = L.PlanInfo()
        L.check(self._lib.das_plan_info(self._h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in L.PlanInfo._fields_}

    def set_tuning(self, frames_per_thread: int = 0, ctas_per_sm: int = 0, staging: bool = False,
                   load_width: int = 0, tensor_cores: bool = False, tc_chain: int = 0,
                   voxels_per_thread: int = 0, adjoint_rows: int = 0, host_io: int = 0) -> None:
        """Kernel shape of the forward pass; tensor_cores selects the tcgen05
        contraction (IQ data with f16 / bf16 storage), tc_chain the MMA
        sub-items per tensor-memory accumulation chain (0: automatic, 1024
        with 4 or more transmits; -1: one chain per tile), voxels_per_thread
        the float32 IQ kernel with one (the default) or two voxels per thread,
        adjoint_rows the sample rows per CTA of the adjoint (0: automatic),
        host_io how the host calls move data (0 / 1 copies, 2 the kernels
        read and write page-locked host memory directly)."""
        t = L.Tuning(int(frames_per_thread), int(ctas_per_sm), 1 if staging else 0, int(load_width),
                     1 if tensor_cores else 0, int(tc_chain), int(voxels_per_thread), int(adjoint_rows),
                     int(host_io))
        L.check(self._lib.das_plan_set_tuning(self._h, C.byref(t)))
        self._tuning = dict(frames_per_thread=int(frames_per_thread), ctas_per_sm=int(ctas_per_sm),
                            staging=bool(staging), load_width=int(load_width), tensor_cores=bool(tensor_cores),
                            tc_chain=int(tc_chain), voxels_per_thread=int(voxels_per_thread),
                            adjoint_rows=int(adjoint_rows), host_io=int(host_io))

    def tuning(self) -> dict:
        """The tuning last set on this plan (all defaults before any set_tuning)."""
        return dict(getattr(self, "_tuning", {}) or dict(
            frames_per_thread=0, ctas_per_sm=0, staging=False, load_width=0, tensor_cores=False, tc_chain=0,
            voxels_per_thread=0, adjoint_rows=0, host_io=0))

    def check(self, stream=None) -> None:
        """Wait for the stream; raise if a kernel recorded a failure (a bounded wait that expired)."""
        L.check(self._lib.das_plan_check(self._h, _stream(stream)))

    def set_wait_test(self, wait_ns: int = 0, probe: bool = False) -> None:
        """Test hook of the kernels' bounded waits (das_plan_set_wait_test):
        the limit of the pipeline waits in ns (0: the default, 1 s) and whether
        one CTA waits on a barrier nothing arrives on."""
        L.check(self._lib.das_plan_set_wait_test(self._h, int(wait_ns), 1 if probe else 0))

    def enable_timing(self, capacity: int) -> None:
        """Record CUDA events around the DAS kernel of the next `capacity` forward calls."""
        L.check(self._lib.das_plan_enable_timing(self._h, int(capacity)))

    def timing(self) -> tuple:
        """(summed kernel milliseconds, number of timed launches) since the last call."""
        ms, n = C.c_double(), C.c_int()
        L.check(self._lib.das_plan_timing(self._h, C.byref(ms), C.byref(n)))
        return float(ms.value), int(n.value)

    # ------------------------------------------------------------------ checks

    @property
    def data_dtype(self) -> torch.dtype:
        return torch.complex64 if self.iq else torch.float32

    def _check(self, t: torch.Tensor, shape_tail, what: str) -> int:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{what} must be a torch.Tensor")
        if t.device != self.device:
            raise ValueError(f"{what} must be on {self.device}, got {t.device}")
        if t.dtype != self.data_dtype:
            raise TypeError(f"{what} must be {self.data_dtype}, got {t.dtype}")
        if not t.is_contiguous():
            raise ValueError(f"{what} must be contiguous")
        if tuple(t.shape[1:]) != tuple(shape_tail):
            raise ValueError(f"{what} must have shape (B, {', '.join(map(str, shape_tail))}), got {tuple(t.shape)}")
        B = t.shape[0]
        if not 1 <= B <= self.max_batch:
            raise ValueError(f"batch {B} outside 1..{self.max_batch}")
        return B

    def _check_host(self, t: torch.Tensor, shape_tail, what: str) -> int:
        if not isinstance(t, torch.Tensor) or t.device.type != "cpu":
            raise ValueError(f"{what} must be a CPU tensor")
        if t.dtype != self.data_dtype or not t.is_contiguous():
            raise ValueError(f"{what} must be a contiguous {self.data_dtype} tensor")
        if t.dim() < 1 or t.numel() != t.shape[0] * int(np.prod(shape_tail)):
            raise ValueError(f"{what} must have shape (B, {', '.join(map(str, shape_tail))}), got {tuple(t.shape)}")
        B = t.shape[0]
        if not 1 <= B <= self.max_batch:
            raise ValueError(f"batch {B} outside 1..{self.max_batch}")
        return B

    # ------------------------------------------------------------------ compute

    def forward(self, y: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """y (B, Q, M, K) -> image (B, nz, ny, nx) (Eq. 2)."""
        B = self._check(y, (self.Q, self.M, self.K), "y")
        if out is None:
            out = torch.empty((B,) + self.shape, dtype=self.data_dtype, device=self.device)
        else:
            self._check(out, self.shape, "out")
        L.check(self._lib.das_forward(self._h, _ptr(y), _ptr(out), B, _stream(stream)))
        return out

    def forward_host(self, y: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """Host tensors in and out (copies inside the library call).  Buffers from
        host_empty keep the copies at link speed after long kernels."""
        B = self._check_host(y, (self.Q, self.M, self.K), "y")
        if out is None:
            out = host_empty((B,) + self.shape, self.data_dtype)
        elif self._check_host(out, self.shape, "out") != B:
            raise ValueError("out must hold as many frames as y")
        L.check(self._lib.das_forward_host(self._h, _ptr(y), _ptr(out), B, _stream(stream)))
        return out

    def forward_host_many(self, ys: Sequence[torch.Tensor], outs: Optional[Sequence[torch.Tensor]] = None,
                          stream=None) -> list:
        """A sequence of host batches (equal frame counts) through the forward
        pass, with each batch's copies overlapped with its neighbours' forward
        passes.  Returns the host images (new host_empty buffers unless given)."""
        ys = list(ys)
        if not ys:
            raise ValueError("no batches")
        B = self._check_host(ys[0], (self.Q, self.M, self.K), "y")
        if any(self._check_host(y, (self.Q, self.M, self.K), "y") != B for y in ys):
            raise ValueError("every batch must hold the same number of frames")
        if outs is None:
            outs = [host_empty((B,) + self.shape, self.data_dtype) for _ in ys]
        outs = list(outs)
        if len(outs) != len(ys) or len({o.data_ptr() for o in outs}) != len(outs):
            raise ValueError("one distinct output buffer per batch")
        if any(self._check_host(o, self.shape, "out") != B for o in outs):
            raise ValueError("outputs must hold as many frames as the batches")
        n = len(ys)
        yp = (C.c_void_p * n)(*[y.data_ptr() for y in ys])
        xp = (C.c_void_p * n)(*[o.data_ptr() for o in outs])
        L.check(self._lib.das_forward_host_many(self._h, yp, xp, n, B, _stream(stream)))
        return outs

    def adjoint(self, x: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """image (B, nz, ny, nx) -> channel data (B, Q, M, K), the conjugate transpose of forward."""
        B = self._check(x.reshape((x.shape[0],) + self.shape), self.shape, "x")
        if out is None:
            out = torch.empty((B, self.Q, self.M, self.K), dtype=self.data_dtype, device=self.device)
        else:
            self._check(out, (self.Q, self.M, self.K), "out")
        L.check(self._lib.das_adjoint(self._h, _ptr(x), _ptr(out), B, _stream(stream)))
        return out

    def grad_c(self, y: torch.Tensor, gx: torch.Tensor, out: Optional[torch.Tensor] = None,
               stream=None) -> torch.Tensor:
        """Re sum conj(gx) dx/dc as a 0-d float64 tensor on the device."""
        B = self._check(y, (self.Q, self.M, self.K), "y")
        self._check(gx.reshape((gx.shape[0],) + self.shape), self.shape, "gx")
        if gx.shape[0] != B:
            raise ValueError("y and gx batch sizes differ")
        if out is None:
            out = torch.empty((), dtype=torch.float64, device=self.device)
        L.check(self._lib.das_grad_c(self._h, _ptr(y), _ptr(gx), _ptr(out), B, _stream(stream)))
        return out

    def count_active(self, stream=None) -> int:
        n = C.c_longlong()
        L.check(self._lib.das_count_active(self._h, C.byref(n), _stream(stream)))
        return int(n.value)


class _HostBlock:
    """Owner of one das_host_alloc block; numpy keeps it alive through the
    array interface for as long as any view of the memory exists."""

    def __init__(self, nbytes: int):
        self._lib = L.lib()
        ptr = C.c_void_p()
        L.check(self._lib.das_host_alloc(C.c_size_t(nbytes), C.byref(ptr)))
        self.ptr = ptr.value
        self.__array_interface__ = {"data": (self.ptr, False), "shape": (nbytes,), "typestr": "|u1", "version": 3}

    def __del__(self):
        if getattr(self, "ptr", None):
            self._lib.das_host_free(C.c_void_p(self.ptr))
            self.ptr = None


def host_empty(shape, dtype: torch.dtype) -> torch.Tensor:
    """A CPU tensor in page-locked huge-page memory (das_host_alloc), the
    fastest host buffer for Plan.forward_host; freed with its last view."""
    import numpy as np

    shape = tuple(int(s) for s in shape)
    n = 1
    for s in shape:
        n *= s
    nbytes = max(1, n * torch.empty((), dtype=dtype).element_size())
    block = np.asarray(_HostBlock(nbytes))
    return torch.from_numpy(block).view(dtype)[:n].view(shape)


class DASFunction(torch.autograd.Function):
    """x = DAS(y; c) with gradients for y (the adjoint map) and for c (the
    sound-speed derivative, delays recomputed in the backward pass)."""

    @staticmethod
    def forward(ctx, y: torch.Tensor, c: torch.Tensor, plan: Plan):
        plan.set_c(float(c))
        ctx.plan = plan
        ctx.c_value = float(c)
        ctx.c_dtype = c.dtype if isinstance(c, torch.Tensor) else torch.float64
        ctx.c_device = c.device if isinstance(c, torch.Tensor) else torch.device("cpu")
        ctx.save_for_backward(y)
        return plan.forward(y.contiguous())

    @staticmethod
    def backward(ctx, gx: torch.Tensor):
        (y,) = ctx.saved_tensors
        plan: Plan = ctx.plan
        plan.set_c(ctx.c_value)
        gx = gx.contiguous()
        gy = plan.adjoint(gx) if ctx.needs_input_grad[0] else None
        gc = None
        if ctx.needs_input_grad[1]:
            gc = plan.grad_c(y.contiguous(), gx).to(device=ctx.c_device, dtype=ctx.c_dtype)
        return gy, gc, None


def das(y: torch.Tensor, c: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable delay-and-sum: image of y at speed of sound c."""
    return DASFunction.apply(y, c, plan)


class Batch:
    """Several plans and all their frames in one persistent launch replayed
    from a CUDA graph (das_batch_* in the C-ABI)."""

    def __init__(self, plans, frames):
        if len(plans) != len(frames):
            raise ValueError("one frame count per plan")
        self._lib = L.lib()
        self.plans = list(plans)
        self.frames = [int(f) for f in frames]
        arr = (C.c_void_p * len(plans))(*[p._h.value for p in plans])
        fr = (C.c_int * len(plans))(*self.frames)
        h = C.c_void_p()
        L.check(self._lib.das_batch_create(C.byref(h), arr, fr, len(plans)))
        self._h = h

    def close(self) -> None:
        if getattr(self, "_h", None):
            self._lib.das_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_tuning(self, frames_per_thread: int = 0, ctas_per_sm: int = 0, staging: bool = False) -> None:
        t = L.Tuning(int(frames_per_thread), int(ctas_per_sm), 1 if staging else 0, 0, 0, 0, 0, 0, 0)
        L.check(self._lib.das_batch_set_tuning(self._h, C.byref(t)))

    def info(self) -> dict:
        fb, n, k = C.c_int(), C.c_int(), C.c_int()
        L.check(self._lib.das_batch_info(self._h, C.byref(fb), C.byref(n), C.byref(k)))
        return {"frames_per_thread": fb.value, "work_items": n.value, "kernels_per_launch": k.value}

    def forward(self, ys, outs=None, stream=None):
        """ys[i]: (frames[i], Q_i, M_i, K_i) -> images [(frames[i], nz, ny, nx)]."""
        if outs is None:
            outs = [torch.empty((f,) + p.shape, dtype=p.data_dtype, device=p.device)
                    for p, f in zip(self.plans, self.frames)]
        for p, f, y, o in zip(self.plans, self.frames, ys, outs):
            if p._check(y, (p.Q, p.M, p.K), "y") != f or p._check(o, p.shape, "out") != f:
                raise ValueError("batch sizes differ from the frame counts of the batch")
        yp = (C.c_void_p * len(ys))(*[y.data_ptr() for y in ys])
        xp = (C.c_void_p * len(outs))(*[o.data_ptr() for o in outs])
        L.check(self._lib.das_batch_forward(self._h, yp, xp, _stream(stream)))
        return outs
