"""GB300 (sm_103a) mixed-precision Deep-NN SP2 density matrices.

Thin ctypes binding over the C ABI of ``libsp2.so`` (declared in
``include/sp2.h``).  Every step of the method runs in the library's CUDA
kernels; this module only marshals torch tensors (device memory, streams)
into pointers and sizes.  There is no fallback: if the library is missing or
the device is not an sm_103a GPU, calls raise.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import re
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

from ._build import LIB as _LIB_PATH

__all__ = [
    "SP2Error",
    "Stats",
    "init",
    "finalize",
    "set_precision",
    "density_matrix",
    "density_matrix_accelerated",
    "density_matrix_batched",
    "density_matrix_batched_accelerated",
    "fermi_expansion",
    "gershgorin",
    "split",
    "layer",
    "observable",
    "network_forward",
    "network_backward",
    "SP2Network",
    "library_path",
    "PRECISIONS",
]

SP2_MAX_LAYERS = 128
PRECISIONS = {"split": 0, "fp16": 1, "fp32": 2}
_STATUS = {
    0: "SP2_OK",
    1: "SP2_NOT_CONVERGED",
    -1: "SP2_ERR_INVALID_ARG",
    -2: "SP2_ERR_NOT_INITIALIZED",
    -3: "SP2_ERR_DEGENERATE_SPECTRUM",
    -4: "SP2_ERR_NONFINITE",
    -5: "SP2_ERR_CUDA",
    -6: "SP2_ERR_OOM",
    -7: "SP2_ERR_DEVICE_TIMEOUT",
    -8: "SP2_ERR_UNSUPPORTED",
    -9: "SP2_ERR_BAD_ESTIMATE",
}
_STOP = {0: "none", 1: "tol", 2: "iderr<=0", 3: "4.5-rule", 4: "max_iter", 5: "bounds"}


class SP2Error(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class _Config(ctypes.Structure):
    _fields_ = [
        ("device", ctypes.c_int),
        ("stream", ctypes.c_void_p),
        ("precision", ctypes.c_int),
        ("lo_scale_exp", ctypes.c_int),
        ("shift_identity", ctypes.c_int),
        ("eps_bias", ctypes.c_double),
    ]


class _Stats(ctypes.Structure):
    _fields_ = [
        ("iterations", ctypes.c_int),
        ("converged_by", ctypes.c_int),
        ("status_device", ctypes.c_int),
        ("n_occ", ctypes.c_int),
        ("e_min", ctypes.c_double),
        ("e_max", ctypes.c_double),
        ("idemp_err", ctypes.c_double),
        ("trace", ctypes.c_double),
        ("alpha", ctypes.c_double),
        ("time_ms", ctypes.c_double),
        ("flops_alg", ctypes.c_double),
        ("prologue_ms", ctypes.c_double),
        ("launches", ctypes.c_int),
        ("sigma", ctypes.c_int8 * SP2_MAX_LAYERS),
        ("iderr", ctypes.c_double * SP2_MAX_LAYERS),
        ("layer_ms", ctypes.c_float * SP2_MAX_LAYERS),
        ("square_ms", ctypes.c_float * SP2_MAX_LAYERS),
        ("energy", ctypes.c_double),
    ]


@dataclasses.dataclass
class Stats:
    status: int
    iterations: int
    converged_by: str
    e_min: float
    e_max: float
    idemp_err: float
    trace: float
    alpha: float
    time_ms: float
    flops_alg: float
    sigmas: List[int]
    iderr: List[float]
    prologue_ms: float = 0.0
    launches: int = 0
    layer_ms: List[float] = dataclasses.field(default_factory=list)
    square_ms: List[float] = dataclasses.field(default_factory=list)
    energy: float = 0.0

    @property
    def converged(self) -> bool:
        return self.status == 0


_lib = None
_state = {"device": None}

_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_F = ctypes.c_float


def library_path() -> str:
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(
            f"{_LIB_PATH} is not built; run `python -c 'import __graft_entry__ as g; g.build()'` first")
    lib = ctypes.CDLL(_LIB_PATH)
    sig = {
        "sp2_init": (_I, [ctypes.POINTER(_Config)]),
        "sp2_finalize": (_I, []),
        "sp2_set_stream": (_I, [_P]),
        "sp2_set_precision": (_I, [_I]),
        "sp2_last_error": (ctypes.c_char_p, []),
        "sp2_density_matrix": (_I, [_P, _I, _I, _D, _I, _P, ctypes.POINTER(_Stats)]),
        "sp2_density_matrix_accelerated": (_I, [_P, _I, _I, _D, _D, _D, _I, _P, ctypes.POINTER(_Stats)]),
        "sp2_density_matrix_batched": (_I, [_P, _P, _P, _I, _D, _I, _P, _P]),
        "sp2_density_matrix_batched_accelerated": (_I, [_P, _P, _P, _P, _P, _I, _D, _I, _P, _P]),
        "sp2_network_forward": (_I, [_P, _I, _I, _I, _P, _I, _P, _P, _P]),
        "sp2_network_backward": (_I, [_P, _I, _I, _I, _P, _I, _P, _P, _P, _P]),
        "sp2_fermi_expansion": (_I, [_P, _I, _I, _I, _P, _P, _D, _D, _P, _P]),
        "sp2_gershgorin": (_I, [_P, _I, _P]),
        "sp2_split": (_I, [_P, _I, _I, _P, _P]),
        "sp2_layer": (_I, [_P, _I, _I, _F, _F, _F, _P, _P]),
        "sp2_observable": (_I, [_P, _P, _I, _P]),
        "sp2_set_fault": (_I, [ctypes.c_char_p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int, allow=(0,)) -> int:
    if status in allow:
        return status
    msg = _load().sp2_last_error().decode(errors="replace")
    raise SP2Error(status, msg)


def init(device: int = 0, precision: str = "split", lo_scale_exp: int = 11, shift_identity: bool = True,
         eps_bias: float = 0.0) -> None:
    """Initialises the library on ``device`` (idempotent)."""
    lib = _load()
    cfg = _Config(device, None, PRECISIONS[precision], lo_scale_exp, 1 if shift_identity else 0, eps_bias)
    _check(lib.sp2_init(ctypes.byref(cfg)))
    _state["device"] = device
    _state["precision"] = precision


def set_fault(spec: Optional[str]) -> None:
    """Arms injected faults for tests of the error paths: "alloc_fail",
    "nan_input", "timeout", "wait_ms=<n>" (comma-separated; None or "none"
    clears).  See sp2_set_fault in include/sp2.h."""
    _check(_load().sp2_set_fault(None if spec is None else spec.encode()))


def finalize() -> None:
    _check(_load().sp2_finalize())
    _state["device"] = None


def set_precision(precision: str) -> None:
    """Library-wide arithmetic of the squarings: "split", "fp16" or "fp32"."""
    _ensure_init(None)
    _check(_load().sp2_set_precision(PRECISIONS[precision]))
    _state["precision"] = precision


class _precision:
    """A per-call precision: switched in for one call, the library-wide one
    restored afterwards."""

    def __init__(self, precision: Optional[str]):
        self.p = precision

    def __enter__(self):
        if self.p is not None:
            self.old = _state.get("precision", "split")
            _check(_load().sp2_set_precision(PRECISIONS[self.p]))

    def __exit__(self, *exc):
        if self.p is not None:
            _load().sp2_set_precision(PRECISIONS[self.old])
        return False


def _ensure_init(t: Optional[torch.Tensor]) -> None:
    dev = t.device.index if (t is not None and t.device.index is not None) else torch.cuda.current_device()
    if _state["device"] != dev:
        init(dev)
    _check(_load().sp2_set_stream(ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)))


def _dev_f32(t: torch.Tensor, name: str) -> torch.Tensor:
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    return t


def _stats(s: _Stats, status: int) -> Stats:
    n = s.iterations
    return Stats(status=status, iterations=n, converged_by=_STOP.get(s.converged_by, str(s.converged_by)),
                 e_min=s.e_min, e_max=s.e_max, idemp_err=s.idemp_err, trace=s.trace, alpha=s.alpha,
                 time_ms=s.time_ms, flops_alg=s.flops_alg, sigmas=[int(v) for v in s.sigma[:n]],
                 iderr=[float(v) for v in s.iderr[:n]], prologue_ms=s.prologue_ms, launches=s.launches,
                 layer_ms=[float(v) for v in s.layer_ms[:s.launches]],
                 square_ms=[float(v) for v in s.square_ms[:s.launches]], energy=float(s.energy))


def _stats_many(st, B: int) -> List[Stats]:
    """Stats of a batched call, read column-wise through one structured-array
    view of the ctypes records (per-element ctypes access would dominate)."""
    a = np.ctypeslib.as_array(st)
    col = {k: a[k].tolist() for k in ("iterations", "launches", "converged_by", "e_min", "e_max", "idemp_err",
                                       "trace", "alpha", "time_ms", "flops_alg", "prologue_ms", "energy")}
    nmax = max(col["iterations"]) if B else 0
    lmax = max(col["launches"]) if B else 0
    sig = a["sigma"][:, :nmax].tolist()
    ide = a["iderr"][:, :nmax].tolist()
    # per-launch times are shared by the instances of one call: convert once
    la, sa = a["layer_ms"][:, :lmax], a["square_ms"][:, :lmax]
    if B and (la == la[0]).all() and (sa == sa[0]).all():
        lms, sms = [la[0].tolist()] * B, [sa[0].tolist()] * B
    else:
        lms, sms = la.tolist(), sa.tolist()
    out = []
    for i in range(B):
        n, nl, c = col["iterations"][i], col["launches"][i], col["converged_by"][i]
        out.append(Stats(status=1 if c == 4 else 0, iterations=n, converged_by=_STOP.get(c, str(c)),
                         e_min=col["e_min"][i], e_max=col["e_max"][i], idemp_err=col["idemp_err"][i],
                         trace=col["trace"][i], alpha=col["alpha"][i], time_ms=col["time_ms"][i],
                         flops_alg=col["flops_alg"][i], sigmas=sig[i][:n], iderr=ide[i][:n],
                         prologue_ms=col["prologue_ms"][i], launches=nl, layer_ms=lms[i][:nl],
                         square_ms=sms[i][:nl], energy=col["energy"][i]))
    return out


def density_matrix(H: torch.Tensor, n_occ: int, tol: float = 0.0, max_iter: int = 100,
                   out: Optional[torch.Tensor] = None, precision: Optional[str] = None,
                   sync: bool = True) -> Tuple[torch.Tensor, Optional[Stats]]:
    """D = theta(mu I - H), Tr D = n_occ, by Deep-NN SP2 (Alg. 1 + Eq. 15).

    Returns (D, stats).  With ``sync=False`` the call only enqueues and
    stats is None.
    """
    _dev_f32(H, "H")
    if H.dim() != 2 or H.shape[0] != H.shape[1]:
        raise ValueError("H must be square")
    _ensure_init(H)
    lib = _load()
    N = H.shape[0]
    D = out if out is not None else torch.empty_like(H)
    _dev_f32(D, "out")
    st = _Stats()
    with _precision(precision):
        status = lib.sp2_density_matrix(H.data_ptr(), N, int(n_occ), float(tol), int(max_iter), D.data_ptr(),
                                        ctypes.byref(st) if sync else None)
    _check(status, allow=(0, 1))
    return D, (_stats(st, status) if sync else None)


def density_matrix_accelerated(H: torch.Tensor, n_occ: int, homo: float, lumo: float, tol: float = 0.0,
                               max_iter: int = 100, out: Optional[torch.Tensor] = None,
                               precision: Optional[str] = None, sync: bool = True):
    """D = theta(mu I - H) by the accelerated Deep-NN SP2 layers, given
    estimates of the HOMO and LUMO eigenvalues of H (a narrower gap than the
    true one is safe).  ``tol`` bounds the eigenvalue distance from 0 and 1
    (0 selects 1e-9).  Returns (D, stats)."""
    _dev_f32(H, "H")
    if H.dim() != 2 or H.shape[0] != H.shape[1]:
        raise ValueError("H must be square")
    _ensure_init(H)
    lib = _load()
    N = H.shape[0]
    D = out if out is not None else torch.empty_like(H)
    _dev_f32(D, "out")
    st = _Stats()
    with _precision(precision):
        status = lib.sp2_density_matrix_accelerated(H.data_ptr(), N, int(n_occ), float(homo), float(lumo),
                                                    float(tol), int(max_iter), D.data_ptr(),
                                                    ctypes.byref(st) if sync else None)
    _check(status, allow=(0, 1))
    return D, (_stats(st, status) if sync else None)


def _batched(Hs, n_occ, tol, max_iter, outs, sync, homo=None, lumo=None):
    if len(Hs) == 0:
        return [], []
    for i, h in enumerate(Hs):
        _dev_f32(h, f"Hs[{i}]")
    _ensure_init(Hs[0])
    lib = _load()
    B = len(Hs)
    sizes = [h.shape[0] for h in Hs]
    if outs is not None:
        Ds = list(outs)
    else:
        # one allocation for all outputs, returned as views (64-element aligned offsets)
        offs, o = [], 0
        for n in sizes:
            offs.append(o)
            o += (n * n + 63) // 64 * 64
        flat = torch.empty(o, dtype=torch.float32, device=Hs[0].device)
        Ds = [flat[off:off + n * n].view(n, n) for off, n in zip(offs, sizes)]
    hp = (ctypes.c_void_p * B)(*[h.data_ptr() for h in Hs])
    dp = (ctypes.c_void_p * B)(*[d.data_ptr() for d in Ds])
    ns = (ctypes.c_int * B)(*sizes)
    no = (ctypes.c_int * B)(*[int(x) for x in n_occ])
    st = (_Stats * B)()
    if homo is None:
        status = lib.sp2_density_matrix_batched(hp, ns, no, B, float(tol), int(max_iter), dp, st if sync else None)
    else:
        ho = (ctypes.c_double * B)(*[float(x) for x in homo])
        lu = (ctypes.c_double * B)(*[float(x) for x in lumo])
        status = lib.sp2_density_matrix_batched_accelerated(hp, ns, no, ho, lu, B, float(tol), int(max_iter), dp,
                                                            st if sync else None)
    _check(status, allow=(0, 1))
    return Ds, (_stats_many(st, B) if sync else None)


def density_matrix_batched(Hs: Sequence[torch.Tensor], n_occ: Sequence[int], tol: float = 0.0,
                           max_iter: int = 100, outs: Optional[Sequence[torch.Tensor]] = None,
                           sync: bool = True):
    """Many independent SP2 problems of uneven size (grouped launches)."""
    return _batched(Hs, n_occ, tol, max_iter, outs, sync)


def density_matrix_batched_accelerated(Hs: Sequence[torch.Tensor], n_occ: Sequence[int], homo: Sequence[float],
                                       lumo: Sequence[float], tol: float = 0.0, max_iter: int = 100,
                                       outs: Optional[Sequence[torch.Tensor]] = None, sync: bool = True):
    """Batched accelerated layers, one HOMO/LUMO estimate pair per instance."""
    if len(homo) != len(Hs) or len(lumo) != len(Hs):
        raise ValueError("one homo and one lumo estimate per instance")
    return _batched(Hs, n_occ, tol, max_iter, outs, sync, homo, lumo)


def fermi_expansion(H: torch.Tensor, theta, c, window: Optional[Tuple[float, float]] = None,
                    out: Optional[torch.Tensor] = None) -> Tuple[torch.Tensor, torch.Tensor]:
    """Finite-temperature expansion D = I - sum_i c_i X_i with
    X_0 = (H - e_lo I)/(e_hi - e_lo) and X_n = a X^2 + b X + c I per layer
    (theta [L, 3], c [L + 1]).  H is [N, N] or [B, N, N]; window (e_lo, e_hi)
    or None for each instance's Gershgorin bounds.  Returns (D, bounds [B, 2])."""
    _dev_f32(H, "H")
    _ensure_init(H)
    Hb = H if H.dim() == 3 else H.unsqueeze(0)
    B, N = Hb.shape[0], Hb.shape[-1]
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(-1, 3))
    cc = np.ascontiguousarray(np.asarray(c, dtype=np.float64).reshape(-1))
    if cc.shape[0] != th.shape[0] + 1:
        raise ValueError("c needs one more entry than theta has layers")
    D = out if out is not None else torch.empty_like(Hb)
    _dev_f32(D, "out")
    bounds = torch.empty((B, 2), dtype=torch.float64, device=H.device)
    lo, hi = (0.0, 0.0) if window is None else (float(window[0]), float(window[1]))
    _check(_load().sp2_fermi_expansion(Hb.data_ptr(), B, N, th.shape[0], th.ctypes.data, cc.ctypes.data, lo, hi,
                                       D.data_ptr(), bounds.data_ptr()))
    return (D if H.dim() == 3 else D[0]), bounds


def gershgorin(H: torch.Tensor) -> Tuple[float, float]:
    """Gershgorin bounds (e_min, e_max) of H, FP64 on the device."""
    _dev_f32(H, "H")
    _ensure_init(H)
    out = (ctypes.c_double * 2)()
    _check(_load().sp2_gershgorin(H.data_ptr(), H.shape[0], out))
    return float(out[0]), float(out[1])


def split(X: torch.Tensor, lo_scale_exp: int = 11) -> Tuple[torch.Tensor, torch.Tensor]:
    """hi = FP16[X], lo = FP16[2^s (X - hi)] (Eq. 12)."""
    _dev_f32(X, "X")
    _ensure_init(X)
    hi = torch.empty(X.shape, dtype=torch.float16, device=X.device)
    lo = torch.empty_like(hi)
    _check(_load().sp2_split(X.data_ptr(), X.shape[0], int(lo_scale_exp), hi.data_ptr(), lo.data_ptr()))
    return hi, lo


def layer(X: torch.Tensor, a: float, b: float, c: float, precision: Optional[str] = None,
          traces: bool = True):
    """X_out = a X^2 + b X + c I for X of shape [N, N] or [B, N, N] (Eq. 16)."""
    _dev_f32(X, "X")
    _ensure_init(X)
    lib = _load()
    Xb = X if X.dim() == 3 else X.unsqueeze(0)
    B, N = Xb.shape[0], Xb.shape[-1]
    out = torch.empty_like(Xb)
    tr = (ctypes.c_double * (2 * B))()
    with _precision(precision):
        _check(lib.sp2_layer(Xb.data_ptr(), B, N, float(a), float(b), float(c), out.data_ptr(),
                             tr if traces else None))
    out = out if X.dim() == 3 else out[0]
    if not traces:
        return out, None
    return out, [(tr[2 * i], tr[2 * i + 1]) for i in range(B)]


def observable(D: torch.Tensor, A: torch.Tensor) -> float:
    """Tr[D A] (Alg. 1 output observable; A = H gives the band energy)."""
    _dev_f32(D, "D")
    _dev_f32(A, "A")
    _ensure_init(D)
    out = ctypes.c_double()
    _check(_load().sp2_observable(D.data_ptr(), A.data_ptr(), D.shape[0], ctypes.byref(out)))
    return float(out.value)


def _host_coef(coef) -> Tuple[ctypes.Array, int]:
    c = torch.as_tensor(coef, dtype=torch.float32).detach().cpu().contiguous().reshape(-1, 3)
    arr = (ctypes.c_float * c.numel())(*c.reshape(-1).tolist())
    return arr, c.shape[0]


def network_forward(H: torch.Tensor, coef, ckpt_every: int = 1, keep_ckpt: bool = True):
    """X_L of the network X_{n+1} = a_n X_n^2 + b_n X_n + c_n I (Eq. 16), X_0
    the Gershgorin-scaled input layer.  Returns (X_L, ckpt or None, bounds)."""
    _dev_f32(H, "H")
    _ensure_init(H)
    Hb = H if H.dim() == 3 else H.unsqueeze(0)
    B, N = Hb.shape[0], Hb.shape[-1]
    carr, L = _host_coef(coef)
    X = torch.empty_like(Hb)
    ck = None
    if keep_ckpt:
        ck = torch.empty((L // ckpt_every + 1, B, N, N), dtype=torch.float32, device=H.device)
    bounds = torch.empty((B, 2), dtype=torch.float64, device=H.device)
    _check(_load().sp2_network_forward(Hb.data_ptr(), B, N, L, carr, int(ckpt_every), X.data_ptr(),
                                       ck.data_ptr() if ck is not None else None, bounds.data_ptr()))
    return X, ck, bounds


def network_backward(H: torch.Tensor, coef, ckpt_every: int, ckpt: torch.Tensor, G_out: torch.Tensor,
                     want_G_in: bool = True):
    """Adjoint of ``network_forward``: returns (dcoef [L,3] float64 CPU, G_in or None)."""
    _dev_f32(H, "H")
    _dev_f32(G_out, "G_out")
    _ensure_init(H)
    Hb = H if H.dim() == 3 else H.unsqueeze(0)
    B, N = Hb.shape[0], Hb.shape[-1]
    carr, L = _host_coef(coef)
    dcoef = (ctypes.c_double * (3 * L))()
    G_in = torch.empty_like(Hb) if want_G_in else None
    _check(_load().sp2_network_backward(Hb.data_ptr(), B, N, L, carr, int(ckpt_every), ckpt.data_ptr(),
                                        G_out.contiguous().data_ptr(), dcoef,
                                        G_in.data_ptr() if G_in is not None else None))
    d = torch.tensor(list(dcoef), dtype=torch.float64).reshape(L, 3)
    return d, G_in


class SP2Network(torch.autograd.Function):
    """torch.autograd wrapper: forward/backward run in the library kernels,
    with layer checkpoints owned by the autograd context."""

    @staticmethod
    def forward(ctx, H, coef, ckpt_every: int = 1):
        X, ck, _ = network_forward(H, coef, ckpt_every, keep_ckpt=True)
        ctx.save_for_backward(H, coef, ck)
        ctx.ckpt_every = ckpt_every
        return X if H.dim() == 3 else X[0]

    @staticmethod
    def backward(ctx, gX):
        H, coef, ck = ctx.saved_tensors
        g = gX if gX.dim() == 3 else gX.unsqueeze(0)
        dcoef, G_in = network_backward(H, coef.detach(), ctx.ckpt_every, ck, g.contiguous().float(), True)
        return None, dcoef.to(coef.dtype).to(coef.device), None
