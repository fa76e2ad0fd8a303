"""FP64 CPU oracle of the PPF SIR time step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  It is a ctypes wrapper around
``ppf_oracle.c`` (plain C, FP64), which shares no code with the CUDA library.

Every function cites the passage of the paper it follows in the C source.
"""

from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ppf_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libppf_oracle.so")
_lock = threading.Lock()
_lib = None

SYSTEMATIC, RPA_GS, RPA_SGS, RPA_LGS, RNA = 0, 1, 2, 3, 4
RPA2_GS, RPA2_SGS, RPA2_LGS = 5, 6, 7  # two-stage proportional allocation
ARNA = 8  # adaptive RNA (exchange ratio from the involved groups, ring redrawn when lost)
PURPOSE_INIT, PURPOSE_PROP, PURPOSE_RESAMPLE, PURPOSE_GROUP_RESAMPLE, PURPOSE_RING = 0, 1, 2, 3, 4
OK, EDEGENERATE = 0, 5


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, no fast-math, no contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    hdr = os.path.join(_HERE, "ppf_oracle.h")
    fresh = os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(hdr))
    if fresh and not force:
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-Wall", "-o", tmp, _SRC, "-lm"]
    # OpenMP over particles where the toolchain has it; the results do not
    # depend on it (per-particle loops only, reductions summed serially)
    p = subprocess.run(cmd[:-1] + ["-fopenmp", "-lm"], capture_output=True, text=True)
    if p.returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Model(C.Structure):
    _fields_ = [
        ("width", C.c_int32), ("height", C.c_int32), ("patch_radius", C.c_int32), ("likelihood", C.c_int32),
        ("psf_sigma", C.c_double), ("amplitude", C.c_double), ("background", C.c_double),
        ("sigma_xi", C.c_double), ("sigma_m", C.c_double), ("sigma_v", C.c_double),
        ("sigma_I", C.c_double), ("v0_max", C.c_double),
        ("seed", C.c_uint64), ("filter_id", C.c_uint32), ("pad2_", C.c_uint32),
    ]


@dataclasses.dataclass
class Model:
    """Parameters of the single-spot tracking model (Sec. 7.1-7.2)."""
    width: int = 128
    height: int = 128
    patch_radius: int = 4
    psf_sigma: float = 1.5
    amplitude: float = 50.0
    background: float = 10.0
    sigma_xi: float = float(np.sqrt(10.0))
    sigma_m: float = 0.5
    sigma_v: float = 0.1
    sigma_I: float = 1.0
    v0_max: float = 1.0
    seed: int = 0
    filter_id: int = 0
    likelihood: int = 0  # 0: eq. 4 at the particle; 1: piecewise constant over pixel cells (pcSIR)

    def c(self) -> _Model:
        return _Model(self.width, self.height, self.patch_radius, self.likelihood,
                      self.psf_sigma, self.amplitude, self.background, self.sigma_xi,
                      self.sigma_m, self.sigma_v, self.sigma_I, self.v0_max,
                      self.seed & 0xFFFFFFFFFFFFFFFF, self.filter_id, 0)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = C.CDLL(path)
            P = C.POINTER
            u32p, i32p, i64p, u64p, dp, fp = (P(C.c_uint32), P(C.c_int32), P(C.c_int64),
                                              P(C.c_uint64), P(C.c_double), P(C.c_float))
            mp = P(_Model)
            sig = {
                "orc_set_threads": (C.c_int, [C.c_int]),
                "orc_philox": (None, [u32p, u32p, u32p]),
                "orc_u01": (C.c_double, [C.c_uint32]),
                "orc_u21": (C.c_double, [C.c_uint32]),
                "orc_prop_fields": (None, [u32p, u32p]),
                "orc_normals5": (None, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, dp]),
                "orc_init": (None, [mp, C.c_int64, dp]),
                "orc_propagate": (None, [mp, C.c_int64, C.c_int32, dp, i32p, dp, dp]),
                "orc_loglik": (C.c_double, [mp, dp, C.c_double, C.c_double, C.c_double]),
                "orc_propagate_slots": (None, [mp, C.c_int64, C.c_int32, i64p, dp, dp]),
                "orc_loglik_many": (None, [mp, dp, C.c_int64, dp, dp, dp, dp]),
                "orc_weight": (None, [mp, C.c_int64, dp, dp]),
                "orc_summary": (None, [C.c_int64, dp, dp, dp]),
                "orc_scale_bits": (C.c_int, [C.c_int64]),
                "orc_exp2_frac": (C.c_float, [C.c_float]),
                "orc_quantise": (C.c_uint64, [C.c_float, C.c_float, C.c_int]),
                "orc_tickets_below": (C.c_int64, [C.c_uint64, C.c_int64, C.c_uint64, C.c_uint64]),
                "orc_ticket_offset": (C.c_uint64, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                                   C.c_uint32, C.c_uint64]),
                "orc_systematic": (C.c_int, [C.c_int64, u64p, C.c_int64, C.c_uint64, C.c_int64,
                                             i32p, i64p]),
                "orc_schedule": (C.c_int64, [C.c_int, C.c_int32, i64p, i64p, i32p, i32p, i64p]),
                "orc_balanced_offsets": (None, [C.c_int64, C.c_int32, i64p]),
                "orc_resample": (C.c_int, [mp, C.c_int, C.c_double, C.c_int64, C.c_int32, C.c_int32,
                                           i64p, fp, dp, i32p, dp, i64p, i64p]),
                "orc_arna_ring": (None, [C.c_uint64, C.c_uint32, C.c_uint32, C.c_int32, i32p]),
                "orc_resample_arna": (C.c_int, [mp, C.c_double, C.c_int64, C.c_int32, C.c_int32, i64p, fp, dp,
                                                C.c_int32, i32p, i32p, dp, i64p, i64p]),
                "orc_run": (C.c_int, [mp, C.c_int64, C.c_int32, C.c_int, C.c_double, C.c_double, C.c_int32,
                                      dp, dp, dp]),
                "orc_loglik_partials": (None, [mp, dp, C.c_double, C.c_double, C.c_double, C.c_int32,
                                               C.c_int32, dp]),
                "orc_grad_run": (C.c_int, [mp, C.c_int64, C.c_int32, dp, dp, C.c_int, i32p, i32p, dp, dp]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


# ----------------------------------------------------------------------------
# thin wrappers (arrays in / arrays out); all arithmetic is in ppf_oracle.c
# ----------------------------------------------------------------------------
def set_threads(n: int = 0) -> int:
    """Threads of the per-particle loops (0: leave as is); returns the count
    in use (1 without OpenMP).  Results do not depend on it."""
    return int(lib().orc_set_threads(int(n)))


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox(_p(c, C.c_uint32), _p(k, C.c_uint32), _p(out, C.c_uint32))
    return out


def u01(r: int) -> float:
    return lib().orc_u01(int(r))


def u21(field: int) -> float:
    return lib().orc_u21(int(field))


def prop_fields(words) -> np.ndarray:
    w = np.ascontiguousarray(words, dtype=np.uint32)
    f = np.zeros(6, dtype=np.uint32)
    lib().orc_prop_fields(_p(w, C.c_uint32), _p(f, C.c_uint32))
    return f


def normals5(seed: int, slot: int, frame: int, filter_id: int = 0) -> np.ndarray:
    e = np.zeros(5)
    lib().orc_normals5(seed, slot, frame, filter_id, _p(e, C.c_double))
    return e


def init(m: Model, N: int) -> np.ndarray:
    st = np.zeros(6 * N)
    lib().orc_init(C.byref(m.c()), N, _p(st, C.c_double))
    return st.reshape(6, N)


def propagate(m: Model, frame: int, parent: np.ndarray, anc: np.ndarray, lw_prev: np.ndarray) -> np.ndarray:
    """parent: (6, N) state before the step; anc: (N,) parent of each slot."""
    par = np.ascontiguousarray(parent, dtype=np.float64)
    N = anc.shape[0]
    if par.shape != (6, N):
        raise ValueError("parent must be a (6, N) state array")
    a = np.ascontiguousarray(anc, dtype=np.int32)
    lp = np.ascontiguousarray(lw_prev, dtype=np.float64)
    st = np.zeros(6 * N)
    lib().orc_propagate(C.byref(m.c()), N, frame, _p(par.reshape(-1), C.c_double), _p(a, C.c_int32),
                        _p(lp, C.c_double), _p(st, C.c_double))
    return st.reshape(6, N)


def propagate_slots(m: Model, frame: int, slots: np.ndarray, parents5: np.ndarray) -> np.ndarray:
    """Propagate only the given slots; parents5: (5, n) parent x, y, vx, vy, I0 per slot."""
    sl = np.ascontiguousarray(slots, dtype=np.int64)
    n = sl.shape[0]
    par = np.ascontiguousarray(parents5, dtype=np.float64).reshape(5, n)
    out = np.zeros((5, n))
    lib().orc_propagate_slots(C.byref(m.c()), n, frame, _p(sl, C.c_int64), _p(par.reshape(-1), C.c_double),
                              _p(out.reshape(-1), C.c_double))
    return out


def loglik_many(m: Model, frame: np.ndarray, x, y, I0) -> np.ndarray:
    fr = np.ascontiguousarray(frame, dtype=np.float64)
    xx = np.ascontiguousarray(x, dtype=np.float64)
    yy = np.ascontiguousarray(y, dtype=np.float64)
    ii = np.ascontiguousarray(I0, dtype=np.float64)
    out = np.zeros(xx.shape[0])
    lib().orc_loglik_many(C.byref(m.c()), _p(fr, C.c_double), xx.shape[0], _p(xx, C.c_double),
                          _p(yy, C.c_double), _p(ii, C.c_double), _p(out, C.c_double))
    return out


def loglik(m: Model, frame: np.ndarray, x: float, y: float, I0: float) -> float:
    fr = np.ascontiguousarray(frame, dtype=np.float64)
    return lib().orc_loglik(C.byref(m.c()), _p(fr, C.c_double), x, y, I0)


def weight(m: Model, frame: np.ndarray, st: np.ndarray) -> np.ndarray:
    s = np.ascontiguousarray(st, dtype=np.float64).copy()
    N = s.shape[1]
    fr = np.ascontiguousarray(frame, dtype=np.float64)
    lib().orc_weight(C.byref(m.c()), N, _p(fr, C.c_double), _p(s.reshape(-1), C.c_double))
    return s


def summary(st: np.ndarray, lw_prev: np.ndarray) -> dict:
    s = np.ascontiguousarray(st, dtype=np.float64)
    N = s.shape[1]
    lp = np.ascontiguousarray(lw_prev, dtype=np.float64)
    out = np.zeros(8)
    lib().orc_summary(N, _p(s.reshape(-1), C.c_double), _p(lp, C.c_double), _p(out, C.c_double))
    return {"mean": out[:5].copy(), "log_evidence": out[5], "ess": out[6], "max_lw": out[7]}


def scale_bits(n: int) -> int:
    return lib().orc_scale_bits(n)


def exp2_frac(f: float) -> float:
    return lib().orc_exp2_frac(float(np.float32(f)))


def quantise(lw: np.ndarray, M: float | None = None, s: int | None = None) -> np.ndarray:
    lwf = np.asarray(lw, dtype=np.float32).reshape(-1)
    if M is None:
        M = float(lwf.max())
    if s is None:
        s = scale_bits(lwf.shape[0])
    f = lib().orc_quantise
    return np.array([f(float(v), float(M), s) for v in lwf], dtype=np.uint64)


def tickets_below(c: int, n: int, u: int, Q: int) -> int:
    return lib().orc_tickets_below(c, n, u, Q)


def ticket_offset(seed: int, filter_id: int, frame: int, purpose: int, index: int, Q: int) -> int:
    return lib().orc_ticket_offset(seed, filter_id, frame, purpose, index, Q)


def systematic(q: np.ndarray, u: int, n_tickets: int | None = None, base: int = 0):
    qq = np.ascontiguousarray(q, dtype=np.uint64)
    n = qq.shape[0] if n_tickets is None else n_tickets
    anc = np.zeros(n, dtype=np.int32)
    off = np.zeros(qq.shape[0], dtype=np.int64)
    rc = lib().orc_systematic(qq.shape[0], _p(qq, C.c_uint64), n, u, base,
                              _p(anc, C.c_int32), _p(off, C.c_int64))
    return rc, anc, off


def schedule(scheme: int, count: np.ndarray, target: np.ndarray):
    cnt = np.ascontiguousarray(count, dtype=np.int64)
    tgt = np.ascontiguousarray(target, dtype=np.int64)
    G = cnt.shape[0]
    src = np.zeros(2 * G + 1, dtype=np.int32)
    dst = np.zeros(2 * G + 1, dtype=np.int32)
    c = np.zeros(2 * G + 1, dtype=np.int64)
    L = lib().orc_schedule(scheme, G, _p(cnt, C.c_int64), _p(tgt, C.c_int64),
                           _p(src, C.c_int32), _p(dst, C.c_int32), _p(c, C.c_int64))
    return src[:L].copy(), dst[:L].copy(), c[:L].copy()


def balanced_offsets(N: int, G: int) -> np.ndarray:
    off = np.zeros(G + 1, dtype=np.int64)
    lib().orc_balanced_offsets(N, G, _p(off, C.c_int64))
    return off


def resample(m: Model, scheme: int, N: int, frame: int, goff: np.ndarray, lw: np.ndarray,
             lw_sum: np.ndarray | None = None, alpha: float = 0.1):
    """Returns (rc, anc, lw_reset, goff_out, stats[links, moved, max, min])."""
    g = np.ascontiguousarray(goff, dtype=np.int64)
    G = g.shape[0] - 1
    lwf = np.ascontiguousarray(lw, dtype=np.float32)
    lws = np.ascontiguousarray(lwf.astype(np.float64) if lw_sum is None else lw_sum, dtype=np.float64)
    anc = np.zeros(N, dtype=np.int32)
    lwr = np.zeros(N)
    go = np.zeros(G + 1, dtype=np.int64)
    stats = np.zeros(4, dtype=np.int64)
    rc = lib().orc_resample(C.byref(m.c()), scheme, alpha, N, frame, G, _p(g, C.c_int64),
                            _p(lwf, C.c_float), _p(lws, C.c_double), _p(anc, C.c_int32),
                            _p(lwr, C.c_double), _p(go, C.c_int64), _p(stats, C.c_int64))
    return rc, anc, lwr, go, stats


def arna_ring(seed: int, filter_id: int, frame: int, G: int) -> np.ndarray:
    """The ring order ARNA draws when the object is lost: the groups in
    increasing order of the first Philox word of (seed; g, frame, filter,
    RING), ties by group index."""
    ring = np.zeros(G, dtype=np.int32)
    lib().orc_arna_ring(seed, filter_id, frame, G, _p(ring, C.c_int32))
    return ring


def resample_arna(m: Model, N: int, frame: int, goff: np.ndarray, lw: np.ndarray, lost: bool,
                  ring: np.ndarray, lw_sum: np.ndarray | None = None, alpha: float = 0.5):
    """ARNA resampling of one frame.  Returns (rc, anc, lw_reset, goff_out,
    stats[links, moved, max, min, involved], ring_out)."""
    g = np.ascontiguousarray(goff, dtype=np.int64)
    G = g.shape[0] - 1
    lwf = np.ascontiguousarray(lw, dtype=np.float32)
    lws = np.ascontiguousarray(lwf.astype(np.float64) if lw_sum is None else lw_sum, dtype=np.float64)
    rg = np.array(ring, dtype=np.int32)
    anc = np.zeros(N, dtype=np.int32)
    lwr = np.zeros(N)
    go = np.zeros(G + 1, dtype=np.int64)
    stats = np.zeros(5, dtype=np.int64)
    rc = lib().orc_resample_arna(C.byref(m.c()), alpha, N, frame, G, _p(g, C.c_int64), _p(lwf, C.c_float),
                                 _p(lws, C.c_double), 1 if lost else 0, _p(rg, C.c_int32), _p(anc, C.c_int32),
                                 _p(lwr, C.c_double), _p(go, C.c_int64), _p(stats, C.c_int64))
    return rc, anc, lwr, go, stats, rg


def run(m: Model, N: int, frames: np.ndarray, group_size: int = 4096, scheme: int = SYSTEMATIC,
        alpha: float = 0.1, ess_threshold: float = math.inf):
    """Whole SIR run (Alg. 1), resampling when N_eff < ess_threshold (every
    frame by default); returns (rc, est[K, 8], last weighted state (6, N))."""
    fr = np.ascontiguousarray(frames, dtype=np.float64)
    K = fr.shape[0]
    est = np.zeros((K, 8))
    st = np.zeros(6 * N)
    rc = lib().orc_run(C.byref(m.c()), N, group_size, scheme, alpha, ess_threshold, K,
                       _p(fr.reshape(-1), C.c_double), _p(est.reshape(-1), C.c_double), _p(st, C.c_double))
    return rc, est, st.reshape(6, N)


def loglik_partials(m: Model, frame: np.ndarray, x: float, y: float, I0: float, anchor=None) -> np.ndarray:
    """(l, dl/dsigma, dl/dI0, dl/dbg, dl/dx, dl/dy) of one particle."""
    fr = np.ascontiguousarray(frame, dtype=np.float64)
    out = np.zeros(6)
    ax, ay = (-2**31, -2**31) if anchor is None else anchor
    lib().orc_loglik_partials(C.byref(m.c()), _p(fr, C.c_double), x, y, I0, ax, ay, _p(out, C.c_double))
    return out


def grad_run(m: Model, N: int, frames: np.ndarray, theta, anc=None, anchors=None):
    """Log marginal likelihood estimate over the frames (systematic resampling every
    frame, I0 = A) and its gradient w.r.t. (sigma_PSF, A, I_bg, sigma_m), reverse mode.
    Without anc/anchors the run records them (returned); with them it replays them.
    Returns (rc, L, grad[4], anc (K, N), anchors (K, 2, N))."""
    fr = np.ascontiguousarray(frames, dtype=np.float64)
    K = fr.shape[0]
    th = np.ascontiguousarray(theta, dtype=np.float64)
    replay = anc is not None
    a = np.zeros((K, N), dtype=np.int32) if anc is None else np.ascontiguousarray(anc, dtype=np.int32).copy()
    an = (np.zeros((K, 2, N), dtype=np.int32) if anchors is None else
          np.ascontiguousarray(anchors, dtype=np.int32).copy())
    L = np.zeros(1)
    g = np.zeros(4)
    rc = lib().orc_grad_run(C.byref(m.c()), N, K, _p(fr.reshape(-1), C.c_double), _p(th, C.c_double),
                            1 if replay else 0, _p(a.reshape(-1), C.c_int32), _p(an.reshape(-1), C.c_int32),
                            _p(L, C.c_double), _p(g, C.c_double))
    return rc, float(L[0]), g, a, an
