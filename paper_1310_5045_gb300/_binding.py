"""ctypes binding of ``include/ppf.h`` (argument marshalling only).

Every step of the filter runs in libppf's CUDA kernels; torch only provides
device memory and the CUDA stream.  There is no CPU fallback: if the library
or a GPU is missing, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
import threading

from . import _build

SYSTEMATIC, RPA_GS, RPA_SGS, RPA_LGS, RNA = 0, 1, 2, 3, 4
RPA2_GS, RPA2_SGS, RPA2_LGS = 5, 6, 7  # two-stage proportional allocation
ARNA = 8  # adaptive RNA: exchange ratio from the involved groups, ring redrawn when the object is lost
F32, BF16, F16 = 0, 1, 2
PATH_AUTO, PATH_DIRECT, PATH_BINNED = 0, 1, 2  # likelihood path (ppf_set_likelihood_path)
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, EDEGENERATE, ESTATE = range(7)
SCHEMES = {"systematic": SYSTEMATIC, "rpa_gs": RPA_GS, "rpa_sgs": RPA_SGS, "rpa_lgs": RPA_LGS, "rna": RNA,
           "rpa2_gs": RPA2_GS, "rpa2_sgs": RPA2_SGS, "rpa2_lgs": RPA2_LGS, "arna": ARNA}

EXPORTS = ["ppf_create", "ppf_destroy", "ppf_step", "ppf_step_host", "ppf_resample", "ppf_resample_if",
           "ppf_estimate", "ppf_estimate_async",
           "ppf_get_particles", "ppf_set_particles", "ppf_get_groups", "ppf_set_groups", "ppf_get_ring",
           "ppf_set_ring", "ppf_status_string",
           "ppf_last_error", "ppf_profile_enable", "ppf_profile_read", "ppf_systematic_resample_noalloc",
           "ppf_loglik_grad", "ppf_batch_create", "ppf_batch_destroy", "ppf_batch_step", "ppf_batch_resample",
           "ppf_batch_run", "ppf_batch_estimates", "ppf_batch_get_particles", "ppf_batch_autotune",
           "ppf_batch_set_ess_threshold", "ppf_batch_last_error"]


class PPFError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class _Model(C.Structure):
    _fields_ = [
        ("width", C.c_int32), ("height", C.c_int32), ("patch_radius", C.c_int32), ("frame_dtype", C.c_int32),
        ("psf_sigma", C.c_float), ("amplitude", C.c_float), ("background", C.c_float), ("sigma_xi", C.c_float),
        ("sigma_m", C.c_float), ("sigma_v", C.c_float), ("sigma_I", C.c_float), ("v0_max", C.c_float),
        ("seed", C.c_uint64), ("filter_id", C.c_uint32), ("likelihood", C.c_uint32),
    ]


class _Estimate(C.Structure):
    _fields_ = [
        ("mean", C.c_double * 5), ("log_evidence", C.c_double), ("ess", C.c_double),
        ("max_log_weight", C.c_double), ("frame", C.c_int32), ("status_flags", C.c_int32),
        ("links", C.c_int64), ("moved", C.c_int64), ("max_group", C.c_int64), ("min_group", C.c_int64),
    ]


class _FilterEstimate(C.Structure):
    _fields_ = [("mean", C.c_double * 5), ("log_evidence", C.c_double), ("ess", C.c_double),
                ("max_log_weight", C.c_float), ("degenerate", C.c_int32)]


FILTER_ESTIMATE_DTYPE = [("mean", "<f8", (5,)), ("log_evidence", "<f8"), ("ess", "<f8"),
                         ("max_log_weight", "<f4"), ("degenerate", "<i4")]


class _Profile(C.Structure):
    _fields_ = [
        ("launches", C.c_int64), ("steps", C.c_int64), ("resamples", C.c_int64), ("timed_steps", C.c_int64),
        ("prepare_ms", C.c_double), ("step_ms", C.c_double), ("finalize_ms", C.c_double),
        ("resample_ms", C.c_double), ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64),
    ]


@dataclasses.dataclass
class Model:
    """Single-spot tracking model (Sec. 7.1-7.2); mirrors ``ppf_model``."""
    width: int = 128
    height: int = 128
    patch_radius: int = 4
    psf_sigma: float = 1.5
    amplitude: float = 50.0
    background: float = 10.0
    sigma_xi: float = math.sqrt(10.0)
    sigma_m: float = 0.5
    sigma_v: float = 0.1
    sigma_I: float = 1.0
    v0_max: float = 1.0
    seed: int = 0
    filter_id: int = 0
    frame_dtype: int = F32
    likelihood: int = 0  # 0: eq. 4 at the particle; 1: piecewise constant over pixel cells (pcSIR)

    def c(self) -> _Model:
        return _Model(self.width, self.height, self.patch_radius, self.frame_dtype, self.psf_sigma,
                      self.amplitude, self.background, self.sigma_xi, self.sigma_m, self.sigma_v,
                      self.sigma_I, self.v0_max, self.seed & 0xFFFFFFFFFFFFFFFF, self.filter_id,
                      self.likelihood)


@dataclasses.dataclass
class Estimate:
    mean: tuple
    log_evidence: float
    ess: float
    max_log_weight: float
    frame: int
    status_flags: int
    links: int
    moved: int
    max_group: int
    min_group: int
    status: int = OK

    @staticmethod
    def nbytes() -> int:
        """Size of the buffer ParticleFilter.estimate_async writes."""
        return C.sizeof(_Estimate)

    @staticmethod
    def from_buffer(buf) -> "Estimate":
        """Decode a buffer written by ParticleFilter.estimate_async (after the
        stream has run the copy)."""
        e = _Estimate.from_buffer_copy(bytes(buf.numpy().tobytes()) if hasattr(buf, "numpy") else bytes(buf))
        return Estimate(tuple(e.mean), e.log_evidence, e.ess, e.max_log_weight, e.frame, e.status_flags,
                        e.links, e.moved, e.max_group, e.min_group, OK)


_lib = None
_lock = threading.Lock()


def _debug() -> bool:
    return os.environ.get("PPF_DEBUG", "") == "1"


def lib_path() -> str:
    """libppf.so, or libppf_debug.so (device-side index checks) when PPF_DEBUG=1."""
    return _build.LIB_DEBUG if _debug() else _build.LIB


def load(build_if_missing: bool = True):
    """Load the library (building it in-tree first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if build_if_missing:
            _build.build(debug=_debug())
        if not os.path.exists(path):
            raise RuntimeError(f"{os.path.basename(path)} not built ({path}); run "
                               "paper_1310_5045_gb300._build.build()")
        L = C.CDLL(path)
        P = C.POINTER
        vp, ctxp = C.c_void_p, C.c_void_p
        sig = {
            "ppf_create": (C.c_int, [P(_Model), C.c_int64, C.c_int32, vp, P(ctxp)]),
            "ppf_destroy": (None, [ctxp]),
            "ppf_step": (C.c_int, [ctxp, vp, C.c_int32]),
            "ppf_step_host": (C.c_int, [ctxp, vp, C.c_int32]),
            "ppf_resample": (C.c_int, [ctxp, C.c_int, C.c_float]),
            "ppf_resample_if": (C.c_int, [ctxp, C.c_int, C.c_float, C.c_double]),
            "ppf_estimate": (C.c_int, [ctxp, P(_Estimate)]),
            "ppf_estimate_async": (C.c_int, [ctxp, vp]),
            "ppf_get_particles": (C.c_int, [ctxp, vp, vp, vp]),
            "ppf_set_particles": (C.c_int, [ctxp, vp, vp, vp]),
            "ppf_get_groups": (C.c_int, [ctxp, P(C.c_int32), vp]),
            "ppf_set_groups": (C.c_int, [ctxp, vp]),
            "ppf_get_ring": (C.c_int, [ctxp, vp]),
            "ppf_set_ring": (C.c_int, [ctxp, vp]),
            "ppf_status_string": (C.c_char_p, [C.c_int]),
            "ppf_last_error": (C.c_char_p, [ctxp]),
            "ppf_profile_enable": (C.c_int, [ctxp, C.c_int, C.c_int32]),
            "ppf_profile_read": (C.c_int, [ctxp, P(_Profile)]),
            "ppf_systematic_resample_noalloc": (C.c_int, [vp, C.c_int64, C.c_uint64, C.c_uint32, C.c_int32, vp,
                                                          vp]),
            "ppf_loglik_grad": (C.c_int, [ctxp, vp, C.c_int32, P(C.c_float), P(C.c_double), P(C.c_double), vp,
                                          vp]),
            "ppf_batch_create": (C.c_int, [P(_Model), P(C.c_int64), C.c_int32, vp, P(vp)]),
            "ppf_batch_destroy": (None, [vp]),
            "ppf_batch_step": (C.c_int, [vp, vp, C.c_int32]),
            "ppf_batch_resample": (C.c_int, [vp, C.c_int32]),
            "ppf_batch_run": (C.c_int, [vp, vp, C.c_int32, C.c_int32, C.c_int32, vp]),
            "ppf_batch_estimates": (C.c_int, [vp, vp]),
            "ppf_batch_get_particles": (C.c_int, [vp, vp, vp]),
            "ppf_batch_autotune": (C.c_int, [vp, vp, C.c_int32, P(C.c_int32)]),
            "ppf_batch_set_ess_threshold": (C.c_int, [vp, C.c_double]),
            "ppf_batch_last_error": (C.c_char_p, [vp]),
            "ppf_fp32_peak": (C.c_int, [C.c_int32, C.c_int32, P(C.c_double), P(C.c_double)]),
            "ppf_set_likelihood_path": (C.c_int, [ctxp, C.c_int32]),
            "ppf_get_likelihood_path": (C.c_int, [ctxp, P(C.c_int32)]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def systematic_resample_noalloc(lw, seed: int, filter_id: int, frame: int, out=None, stream=None):
    """``ppf_systematic_resample_noalloc``: ancestors of the CUDA float32 log-weights
    ``lw`` for callers that cannot allocate device memory.  ``out`` (CUDA int32,
    same length) receives them; if omitted it is allocated here by torch, which
    a caller that cannot allocate would pass in instead."""
    import torch
    if not lw.is_cuda or lw.dtype != torch.float32 or not lw.is_contiguous():
        raise ValueError("lw must be a contiguous CUDA float32 tensor")
    if out is None:
        out = torch.empty(lw.numel(), dtype=torch.int32, device=lw.device)
    st = stream if stream is not None else torch.cuda.current_stream()
    rc = load().ppf_systematic_resample_noalloc(C.c_void_p(lw.data_ptr()), lw.numel(), seed & 0xFFFFFFFFFFFFFFFF,
                                                filter_id, frame, C.c_void_p(out.data_ptr()),
                                                C.c_void_p(st.cuda_stream))
    if rc != OK:
        raise PPFError(rc, f"ppf_systematic_resample_noalloc: {status_string(rc)}")
    return out


def fp32_peak(packed: bool = False, repeats: int = 5):
    """``ppf_fp32_peak``: the measured FP32 FMA rate of the current device in
    TFLOP/s (packed: two-lane FMAs) and the fastest launch's duration in ms."""
    tf, ms = C.c_double(), C.c_double()
    rc = load().ppf_fp32_peak(1 if packed else 0, int(repeats), C.byref(tf), C.byref(ms))
    if rc != OK:
        raise PPFError(rc, f"ppf_fp32_peak: {status_string(rc)}")
    return tf.value, ms.value


def status_string(s: int) -> str:
    return load().ppf_status_string(s).decode()


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


class ParticleFilter:
    """One SIR filter of N particles on the current CUDA device (``ppf_ctx``)."""

    def __init__(self, model: Model, n: int, group_size: int = 4096, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("ParticleFilter needs a CUDA GPU: the filter runs only in libppf's kernels")
        self._torch = torch
        self.L = load()
        self.model = model
        self.n = int(n)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._ctx = C.c_void_p()
        st = self.L.ppf_create(C.byref(model.c()), self.n, int(group_size),
                               C.c_void_p(self.stream.cuda_stream), C.byref(self._ctx))
        self._check(st, "ppf_create")
        self.frame = 0

    # ------------------------------------------------------------------ utils
    def _check(self, st: int, what: str):
        if st != OK:
            detail = ""
            if self._ctx:
                detail = self.L.ppf_last_error(self._ctx).decode()
            raise PPFError(st, f"{what}: {status_string(st)} {detail}".strip())

    def close(self):
        if getattr(self, "_ctx", None):
            self.L.ppf_destroy(self._ctx)
            self._ctx = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------- calls
    def step(self, frame, k: int | None = None):
        """``ppf_step``: frame is a CUDA tensor (H, W) of the model's dtype."""
        k = self.frame + 1 if k is None else int(k)
        if not frame.is_cuda or not frame.is_contiguous():
            raise ValueError("frame must be a contiguous CUDA tensor")
        self._check(self.L.ppf_step(self._ctx, C.c_void_p(frame.data_ptr()), k), "ppf_step")
        self.frame = k

    def step_host(self, frame, k: int | None = None):
        """``ppf_step_host``: frame is a host tensor/array (pinned for async copies)."""
        k = self.frame + 1 if k is None else int(k)
        ptr = frame.data_ptr() if hasattr(frame, "data_ptr") else frame.ctypes.data
        self._check(self.L.ppf_step_host(self._ctx, C.c_void_p(ptr), k), "ppf_step_host")
        self.frame = k

    def resample(self, scheme=SYSTEMATIC, exchange_ratio: float = 0.1, ess_threshold: float | None = None):
        """Resampling step of Alg. 1; with ess_threshold, only when the last
        step's N_eff is below it (decided on the device)."""
        if isinstance(scheme, str):
            scheme = SCHEMES[scheme]
        if ess_threshold is None:
            self._check(self.L.ppf_resample(self._ctx, int(scheme), float(exchange_ratio)), "ppf_resample")
        else:
            self._check(self.L.ppf_resample_if(self._ctx, int(scheme), float(exchange_ratio),
                                               float(ess_threshold)), "ppf_resample_if")

    def estimate(self, raise_on_flags: bool = False) -> Estimate:
        e = _Estimate()
        st = self.L.ppf_estimate(self._ctx, C.byref(e))
        if st not in (OK, EDEGENERATE, ETIMEOUT) or (raise_on_flags and st != OK):
            self._check(st, "ppf_estimate")
        return Estimate(tuple(e.mean), e.log_evidence, e.ess, e.max_log_weight, e.frame, e.status_flags,
                        e.links, e.moved, e.max_group, e.min_group, st)

    def estimate_async(self, out=None):
        """Enqueue a copy of the estimate into `out` (a page-locked uint8
        tensor of the estimate's size, made when None) and return it without
        waiting; decode with Estimate.from_buffer once the stream has run."""
        torch = self._torch
        if out is None:
            out = torch.empty(C.sizeof(_Estimate), dtype=torch.uint8, pin_memory=True)
        self._check(self.L.ppf_estimate_async(self._ctx, C.c_void_p(out.data_ptr())), "ppf_estimate_async")
        return out

    def get_particles(self, state=True, anc=False, lw_prev=False):
        torch = self._torch
        dev = torch.device("cuda", torch.cuda.current_device())
        s = torch.empty((6, self.n), dtype=torch.float32, device=dev) if state else None
        a = torch.empty(self.n, dtype=torch.int32, device=dev) if anc else None
        p = torch.empty(self.n, dtype=torch.float32, device=dev) if lw_prev else None
        self._check(self.L.ppf_get_particles(self._ctx, C.c_void_p(_ptr(s)), C.c_void_p(_ptr(a)),
                                             C.c_void_p(_ptr(p))), "ppf_get_particles")
        self.stream.synchronize()
        return s, a, p

    def set_particles(self, state, anc=None, lw_prev=None):
        torch = self._torch
        state = state.to(device="cuda", dtype=torch.float32).contiguous()
        if state.shape != (6, self.n):
            raise ValueError("state must be (6, N)")
        if anc is not None:
            anc = anc.to(device="cuda", dtype=torch.int32).contiguous()
        if lw_prev is not None:
            lw_prev = lw_prev.to(device="cuda", dtype=torch.float32).contiguous()
        self._check(self.L.ppf_set_particles(self._ctx, C.c_void_p(_ptr(state)), C.c_void_p(_ptr(anc)),
                                             C.c_void_p(_ptr(lw_prev))), "ppf_set_particles")
        self.stream.synchronize()

    def groups(self):
        import numpy as np
        g = C.c_int32()
        self._check(self.L.ppf_get_groups(self._ctx, C.byref(g), None), "ppf_get_groups")
        off = np.zeros(g.value + 1, dtype=np.int64)
        self._check(self.L.ppf_get_groups(self._ctx, C.byref(g), C.c_void_p(off.ctypes.data)), "ppf_get_groups")
        return off

    def set_groups(self, offsets):
        """Replace the group layout (G + 1 offsets, as returned by groups())."""
        import numpy as np
        off = np.ascontiguousarray(offsets, dtype=np.int64)
        self._check(self.L.ppf_set_groups(self._ctx, C.c_void_p(off.ctypes.data)), "ppf_set_groups")

    def ring(self):
        """ARNA's ring order: ring[p] sends its migrants to ring[(p + 1) % G]."""
        import numpy as np
        r = np.zeros(len(self.groups()) - 1, dtype=np.int32)
        self._check(self.L.ppf_get_ring(self._ctx, C.c_void_p(r.ctypes.data)), "ppf_get_ring")
        return r

    def set_ring(self, ring):
        """Replace ARNA's ring order (a permutation of the G group indices)."""
        import numpy as np
        r = np.ascontiguousarray(ring, dtype=np.int32)
        self._check(self.L.ppf_set_ring(self._ctx, C.c_void_p(r.ctypes.data)), "ppf_set_ring")

    def set_likelihood_path(self, path: int):
        """``ppf_set_likelihood_path``: PATH_AUTO (chosen per step on the device),
        PATH_DIRECT or PATH_BINNED; both paths give the same results."""
        self._check(self.L.ppf_set_likelihood_path(self._ctx, int(path)), "ppf_set_likelihood_path")

    def last_step_binned(self) -> bool:
        """``ppf_get_likelihood_path``: whether the last step took the binned path."""
        v = C.c_int32()
        self._check(self.L.ppf_get_likelihood_path(self._ctx, C.byref(v)), "ppf_get_likelihood_path")
        return bool(v.value)

    def profile_enable(self, enable: bool = True, capacity: int = 4096):
        self._check(self.L.ppf_profile_enable(self._ctx, 1 if enable else 0, int(capacity)), "ppf_profile_enable")

    def profile_read(self) -> dict:
        p = _Profile()
        self._check(self.L.ppf_profile_read(self._ctx, C.byref(p)), "ppf_profile_read")
        return {name: getattr(p, name) for name, _ in _Profile._fields_}

    def loglik_grad(self, frames, theta=None, return_path=False):
        """``ppf_loglik_grad``: L = sum of the per-frame log-evidences over the
        frames (K, H, W CUDA tensor) and dL/d(sigma_PSF, A, I_bg, sigma_m).
        Returns (L, grad[4]) or, with return_path, also the per-frame ancestors
        (K, N) and patch anchors (K, 2, N) of the stop-gradient path."""
        import numpy as np
        torch = self._torch
        if not frames.is_cuda or not frames.is_contiguous():
            raise ValueError("frames must be a contiguous CUDA tensor")
        K = int(frames.shape[0])
        th = None
        if theta is not None:
            th = (C.c_float * 4)(*[float(v) for v in theta])
        L = C.c_double()
        g = (C.c_double * 4)()
        anc = anchors = None
        if return_path:
            anc = torch.empty((K, self.n), dtype=torch.int32, device=frames.device)
            anchors = torch.empty((K, 2, self.n), dtype=torch.int32, device=frames.device)
        st = self.L.ppf_loglik_grad(self._ctx, C.c_void_p(frames.data_ptr()), K, th, C.byref(L), g,
                                    C.c_void_p(_ptr(anc)), C.c_void_p(_ptr(anchors)))
        if st not in (OK, EDEGENERATE):
            self._check(st, "ppf_loglik_grad")
        self.frame = K
        out = (L.value, np.array(list(g)))
        return out + (anc, anchors) if return_path else out


def log_marginal_likelihood(theta, pf: ParticleFilter, frames):
    """Differentiable log marginal likelihood estimate of a filter over frames,
    as a function of theta = (sigma_PSF, A, I_bg, sigma_m) (torch tensor of 4);
    the gradient comes from ppf_loglik_grad (stop-gradient through resampling)."""
    import torch

    class _LML(torch.autograd.Function):
        @staticmethod
        def forward(ctx, th):
            L, g = pf.loglik_grad(frames, th.detach().cpu().tolist())
            ctx.save_for_backward(torch.as_tensor(g, dtype=th.dtype, device=th.device))
            return th.new_tensor(L)

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            return gout * g

    return _LML.apply(theta)


class BatchFilter:
    """F independent SIR filters with uneven particle counts (``ppf_batch``)."""

    def __init__(self, models, ns, stream=None):
        import numpy as np
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("BatchFilter needs a CUDA GPU")
        self._torch = torch
        self.L = load()
        self.F = len(models)
        self.ns = np.asarray(ns, dtype=np.int64)
        self.offsets = np.concatenate([[0], np.cumsum(self.ns)])
        self.ntot = int(self.offsets[-1])
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        arr = (_Model * self.F)(*[m.c() for m in models])
        nn = (C.c_int64 * self.F)(*[int(v) for v in self.ns])
        self._b = C.c_void_p()
        st = self.L.ppf_batch_create(arr, nn, self.F, C.c_void_p(self.stream.cuda_stream), C.byref(self._b))
        if st != OK:
            raise PPFError(st, f"ppf_batch_create: {status_string(st)}")

    def _check(self, st, what):
        if st != OK:
            raise PPFError(st, f"{what}: {status_string(st)} {self.L.ppf_batch_last_error(self._b).decode()}")

    def close(self):
        if getattr(self, "_b", None):
            self.L.ppf_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, frames, k):
        self._check(self.L.ppf_batch_step(self._b, C.c_void_p(frames.data_ptr()), int(k)), "ppf_batch_step")

    def resample(self, k):
        self._check(self.L.ppf_batch_resample(self._b, int(k)), "ppf_batch_resample")

    def set_ess_threshold(self, fraction: float):
        """Alg. 1's N_eff test per filter: resample filter f only while its
        N_eff < fraction * n_f (inf: every frame, the default)."""
        self._check(self.L.ppf_batch_set_ess_threshold(self._b, float(fraction)), "ppf_batch_set_ess_threshold")

    def run(self, frames, k0=1, use_graph=True, estimates=True):
        """K frames (K, F, H, W) of step + resample; returns (K, F) estimates."""
        import numpy as np
        K = int(frames.shape[0])
        out = np.zeros((K, self.F), dtype=FILTER_ESTIMATE_DTYPE) if estimates else None
        st = self.L.ppf_batch_run(self._b, C.c_void_p(frames.data_ptr()), int(k0), K, 1 if use_graph else 0,
                                  C.c_void_p(out.ctypes.data) if estimates else None)
        self._check(st, "ppf_batch_run")
        return out

    def estimates(self):
        import numpy as np
        out = np.zeros(self.F, dtype=FILTER_ESTIMATE_DTYPE)
        st = self.L.ppf_batch_estimates(self._b, C.c_void_p(out.ctypes.data))
        if st not in (OK, EDEGENERATE):
            self._check(st, "ppf_batch_estimates")
        return out

    def get_particles(self, state=True, anc=False):
        torch = self._torch
        s = torch.empty((6, self.ntot), dtype=torch.float32, device="cuda") if state else None
        a = torch.empty(self.ntot, dtype=torch.int32, device="cuda") if anc else None
        self._check(self.L.ppf_batch_get_particles(self._b, C.c_void_p(_ptr(s)), C.c_void_p(_ptr(a))),
                    "ppf_batch_get_particles")
        return s, a

    def autotune(self, frames, k):
        cfg = (C.c_int32 * 3)()
        self._check(self.L.ppf_batch_autotune(self._b, C.c_void_p(frames.data_ptr()), int(k), cfg),
                    "ppf_batch_autotune")
        return {"unit": cfg[0], "block": cfg[1], "blocks_per_sm": cfg[2]}
