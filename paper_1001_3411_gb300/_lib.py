"""ctypes binding of libhop.so (include/hop.h): argument marshalling only.

Every function here takes torch tensors (or numpy arrays for the host
variant of ``hop_run``), checks shapes and dtypes, and passes raw pointers to
the C ABI.  All computation runs in the library's CUDA kernels; if the
library is missing the binding raises instead of computing anything itself.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from .build import LIB

HOP_OK, HOP_EINVAL, HOP_ENOMEM, HOP_ECUDA, HOP_ETABLE, HOP_ETIMEOUT, HOP_EDEGENERATE, HOP_ENOMODEL = range(8)
HOP_ESTATIC = 8
HOP_STATIC_LINK_MAX_N = 1 << 20
HOP_RADIUS_PLAIN, HOP_RADIUS_COUNT, HOP_RADIUS_LEARNED = 0, 1, 2
HOP_BATCH_EAGER = 1
MLP_IN, MLP_HID = 27, 64
MLP_NPARAM = 64 * 27 + 64 + 64 * 64 + 64 + 64 + 1

ERROR_NAMES = {0: "HOP_OK", 1: "HOP_EINVAL", 2: "HOP_ENOMEM", 3: "HOP_ECUDA", 4: "HOP_ETABLE",
               5: "HOP_ETIMEOUT", 6: "HOP_EDEGENERATE", 7: "HOP_ENOMODEL", 8: "HOP_ESTATIC"}

EXPORTS = ["hop_default_params", "hop_create", "hop_destroy", "hop_set_stream", "hop_last_error",
           "hop_set_tuning", "hop_density", "hop_link", "hop_boundaries", "hop_merge", "hop_run",
           "hop_get_stats", "hop_mlp_load", "hop_mlp_get", "hop_mlp_samples", "hop_mlp_forward",
           "hop_mlp_grad", "hop_mlp_train", "hop_link_static", "hop_run_batch", "hop_get_tuning",
           "hop_apply_tuning", "hop_autotune", "hop_halo_stats", "hop_subhalos", "hop_boundaries_reduce",
           "hop_set_norm_count"]


class HopParams(C.Structure):
    _fields_ = [("n_dens", C.c_int32), ("n_hop", C.c_int32), ("n_merge", C.c_int32),
                ("delta_outer", C.c_float), ("delta_saddle", C.c_float), ("delta_peak", C.c_float),
                ("box", C.c_double), ("pos_is_f64", C.c_int32), ("radius_mode", C.c_int32)]


class HopStats(C.Structure):
    _fields_ = [("ms_sort", C.c_double), ("ms_radius", C.c_double), ("ms_knn", C.c_double),
                ("ms_link", C.c_double), ("ms_boundaries", C.c_double), ("ms_merge", C.c_double),
                ("ms_total", C.c_double), ("candidates", C.c_int64), ("searches", C.c_int64),
                ("retries", C.c_int64), ("warps", C.c_int64), ("n_chains", C.c_int64),
                ("n_edges", C.c_int64), ("n_groups", C.c_int64),
                ("knn_queries_per_warp", C.c_int32), ("knn_cells_per_radius", C.c_int32),
                ("launches", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HopTuning(C.Structure):
    _fields_ = [("qpw", C.c_int32), ("cpr", C.c_int32), ("buf_factor", C.c_int32), ("ms", C.c_float)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class HopError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERROR_NAMES.get(code, code)}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None


def load_library(path: str = LIB):
    """Loads libhop.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"libhop.so is not built ({path}); run paper_1001_3411_gb300.build()")
        L = C.CDLL(path)
        vp, i32, i64, f32, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_float, C.c_double
        P = C.POINTER(HopParams)
        sig = {
            "hop_default_params": (None, [P]),
            "hop_create": (C.c_int, [C.POINTER(vp), C.c_int, vp]),
            "hop_destroy": (None, [vp]),
            "hop_set_stream": (C.c_int, [vp, vp]),
            "hop_last_error": (C.c_char_p, [vp]),
            "hop_set_tuning": (C.c_int, [vp, i32, i32]),
            "hop_density": (C.c_int, [vp, vp, i64, P, vp, i32, vp, vp]),
            "hop_link": (C.c_int, [vp, vp, vp, i32, i64, i32, vp, vp]),
            "hop_boundaries": (C.c_int, [vp, vp, vp, vp, i32, i64, i32, f32, vp, vp, i64,
                                         C.POINTER(i64)]),
            "hop_merge": (C.c_int, [vp, vp, vp, i64, vp, vp, i64, f32, f32, f32, vp, C.POINTER(i64)]),
            "hop_run": (C.c_int, [vp, vp, i64, P, vp, vp, C.POINTER(i64), vp, i32, vp]),
            "hop_get_stats": (C.c_int, [vp, C.POINTER(HopStats)]),
            "hop_mlp_load": (C.c_int, [vp, vp, f32]),
            "hop_mlp_get": (C.c_int, [vp, vp]),
            "hop_mlp_samples": (C.c_int, [vp, vp, vp, i64, C.POINTER(i64)]),
            "hop_mlp_forward": (C.c_int, [vp, vp, i64, vp]),
            "hop_mlp_grad": (C.c_int, [vp, vp, vp, i64, C.POINTER(f64), vp]),
            "hop_mlp_train": (C.c_int, [vp, vp, vp, i64, i32, i32, f32, C.c_uint64, C.POINTER(f64)]),
            "hop_link_static": (C.c_int, [vp, vp, i32, i64, i32, vp, vp, vp]),
            "hop_run_batch": (C.c_int, [vp, vp, vp, vp, i32, P, vp, vp, vp, vp, i32, i32]),
            "hop_get_tuning": (C.c_int, [vp, C.POINTER(HopTuning)]),
            "hop_halo_stats": (C.c_int, [vp, vp, i32, vp, vp, i64, i64, f64, vp, vp, vp, vp]),
            "hop_subhalos": (C.c_int, [vp, vp, vp, vp, i32, i64, i32, f32, vp, i32, i64, f64, vp, vp]),
            "hop_apply_tuning": (C.c_int, [vp, C.POINTER(HopTuning)]),
            "hop_boundaries_reduce": (C.c_int, [vp, vp, vp, i64, vp, vp, i64, C.POINTER(i64)]),
            "hop_set_norm_count": (C.c_int, [vp, i64]),
            "hop_autotune": (C.c_int, [vp, vp, vp, vp, i32, P, C.POINTER(HopTuning), i32, i32,
                                       C.POINTER(i32)]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
        return L


def default_params(**kw) -> HopParams:
    p = HopParams()
    load_library().hop_default_params(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(C.c_void_p)
    return C.c_void_p(t.data_ptr())


def _need(t, dtype, shape=None, name="tensor"):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {shape}, got {tuple(t.shape)}")


class Hop:
    """One libhop context on a CUDA device; calls enqueue on torch's current stream."""

    def __init__(self, device: int | None = None):
        import torch
        self.L = load_library()
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            stream = torch.cuda.current_stream().cuda_stream
            self._check(self.L.hop_create(C.byref(h), self.device, C.c_void_p(stream)), None)
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.L.hop_destroy(self.h)
            self.h = None

    __del__ = close

    def _check(self, rc, h=-1):
        if rc != HOP_OK:
            hh = self.h if h == -1 else h
            msg = self.L.hop_last_error(hh).decode() if hh else ""
            raise HopError(rc, msg)

    def _sync_stream(self):
        import torch
        self.L.hop_set_stream(self.h, C.c_void_p(torch.cuda.current_stream(self.device).cuda_stream))

    def set_tuning(self, queries_per_warp: int = 0, cells_per_radius: int = 0):
        self._check(self.L.hop_set_tuning(self.h, queries_per_warp, cells_per_radius))

    # ------------------------------------------------------------ stages
    def hop_density(self, pos, params: HopParams, ld_nbr: int | None = None, want_rk=False):
        import torch
        self._sync_stream()
        dt = torch.float64 if params.pos_is_f64 else torch.float32
        _need(pos, dt, (pos.shape[0], 3), "pos")
        n = pos.shape[0]
        dens = torch.empty(n, dtype=torch.float32, device=pos.device)
        nbr = None
        if ld_nbr:
            nbr = torch.empty((n, ld_nbr), dtype=torch.int32, device=pos.device)
        rk = torch.empty(n, dtype=torch.float32, device=pos.device) if want_rk else None
        self._check(self.L.hop_density(self.h, _ptr(pos), n, C.byref(params), _ptr(nbr),
                                       ld_nbr or 0, _ptr(dens), _ptr(rk)))
        return nbr, dens, rk

    def hop_link(self, dens, nbr, n_hop: int, want_hop=True):
        import torch
        self._sync_stream()
        n, ld = nbr.shape
        _need(dens, torch.float32, (n,), "dens")
        _need(nbr, torch.int32, None, "nbr")
        chain = torch.empty(n, dtype=torch.int32, device=dens.device)
        hop = torch.empty(n, dtype=torch.int32, device=dens.device) if want_hop else None
        self._check(self.L.hop_link(self.h, _ptr(dens), _ptr(nbr), ld, n, n_hop, _ptr(hop), _ptr(chain)))
        return hop, chain

    def hop_boundaries(self, chain, dens, nbr, n_merge: int, delta_outer: float):
        import torch
        self._sync_stream()
        n, ld = nbr.shape
        _need(chain, torch.int32, (n,), "chain")
        _need(dens, torch.float32, (n,), "dens")
        _need(nbr, torch.int32, None, "nbr")
        ne = C.c_int64(0)
        rc = self.L.hop_boundaries(self.h, _ptr(chain), _ptr(dens), _ptr(nbr), ld, n, n_merge,
                                   float(delta_outer), None, None, 0, C.byref(ne))
        if rc not in (HOP_OK, HOP_ETABLE, HOP_EINVAL):
            self._check(rc)
        cap = max(1, ne.value)
        pair = torch.empty(cap, dtype=torch.int64, device=dens.device)
        s = torch.empty(cap, dtype=torch.float64, device=dens.device)
        self._check(self.L.hop_boundaries(self.h, _ptr(chain), _ptr(dens), _ptr(nbr), ld, n, n_merge,
                                          float(delta_outer), _ptr(pair), _ptr(s), cap, C.byref(ne)))
        return pair[: ne.value], s[: ne.value]

    def hop_boundaries_reduce(self, pair, s):
        """Each distinct pair of a gathered boundary list once, with its
        largest sum, in ascending pair order."""
        import torch
        self._sync_stream()
        m = pair.shape[0]
        if m:
            _need(pair, torch.int64, (m,), "pair")
            _need(s, torch.float64, (m,), "s")
        dev = torch.device("cuda", self.device)
        out_p = torch.empty(max(m, 1), dtype=torch.int64, device=dev)
        out_s = torch.empty(max(m, 1), dtype=torch.float64, device=dev)
        ne = C.c_int64(0)
        self._check(self.L.hop_boundaries_reduce(self.h, _ptr(pair) if m else None, _ptr(s) if m else None, m,
                                                 _ptr(out_p), _ptr(out_s), max(m, 1), C.byref(ne)))
        return out_p[: ne.value], out_s[: ne.value]

    def set_norm_count(self, n_norm: int):
        self._check(self.L.hop_set_norm_count(self.h, int(n_norm)))

    def hop_merge(self, chain, dens, pair, s, delta_outer, delta_saddle, delta_peak):
        import torch
        self._sync_stream()
        n = chain.shape[0]
        _need(chain, torch.int32, (n,), "chain")
        _need(dens, torch.float32, (n,), "dens")
        group = torch.empty(n, dtype=torch.int32, device=chain.device)
        ng = C.c_int64(0)
        m = pair.shape[0]
        if m:
            _need(pair, torch.int64, (m,), "pair")
            _need(s, torch.float64, (m,), "s")
        self._check(self.L.hop_merge(self.h, _ptr(chain), _ptr(dens), n, _ptr(pair) if m else None,
                                     _ptr(s) if m else None, m, float(delta_outer), float(delta_saddle),
                                     float(delta_peak), _ptr(group), C.byref(ng)))
        return group, ng.value

    def hop_run(self, pos, params: HopParams, ld_nbr: int | None = None, want_chain=False,
                want_dens=True, out=None):
        """The fused path.  ``pos`` is a CUDA tensor or a host (numpy / CPU
        tensor, pinned or not) array; outputs land where ``out`` says
        (default: same kind of memory as ``pos``)."""
        import torch
        self._sync_stream()
        host = isinstance(pos, np.ndarray) or (isinstance(pos, torch.Tensor) and not pos.is_cuda)
        n = pos.shape[0]
        if out is not None:
            dens, group = out.get("dens"), out["group"]
        elif host:
            pin = isinstance(pos, torch.Tensor) and pos.is_pinned()
            group = torch.empty(n, dtype=torch.int32, pin_memory=pin)
            dens = torch.empty(n, dtype=torch.float32, pin_memory=pin) if want_dens else None
        else:
            group = torch.empty(n, dtype=torch.int32, device=pos.device)
            dens = torch.empty(n, dtype=torch.float32, device=pos.device) if want_dens else None
        dev = torch.device("cuda", self.device)
        nbr = torch.empty((n, ld_nbr), dtype=torch.int32, device=dev) if ld_nbr else None
        chain = torch.empty(n, dtype=torch.int32, device=dev) if want_chain else None
        ng = C.c_int64(0)
        self._check(self.L.hop_run(self.h, _ptr(pos), n, C.byref(params), _ptr(dens), _ptr(group),
                                   C.byref(ng), _ptr(nbr), ld_nbr or 0, _ptr(chain)))
        return dict(dens=dens, group=group, n_groups=ng.value, nbr=nbr, chain=chain)

    def hop_run_batch(self, pos, offsets, boxes, params: HopParams, ld_nbr: int | None = None,
                      want_dens=True, eager=False, out=None):
        """Many periodic subvolumes in one pass.  ``pos`` (N x 3 float32) is a
        CUDA tensor or a host array; ``offsets`` (B + 1) and ``boxes`` (B)
        are host sequences.  Group ids are ranks within each subvolume;
        ``n_groups`` is a numpy array of B counts."""
        import torch
        self._sync_stream()
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        bx = np.ascontiguousarray(np.asarray(boxes, dtype=np.float64))
        B = len(bx)
        if off.shape != (B + 1,):
            raise ValueError("offsets must hold B + 1 entries")
        host = isinstance(pos, np.ndarray) or (isinstance(pos, torch.Tensor) and not pos.is_cuda)
        if isinstance(pos, np.ndarray) and pos.dtype != np.float32:
            raise TypeError("pos must be float32")
        n = pos.shape[0]
        if tuple(pos.shape) != (int(off[-1]), 3):
            raise ValueError(f"pos must have shape ({int(off[-1])}, 3), got {tuple(pos.shape)}")
        if out is not None:
            dens, group = out.get("dens"), out["group"]
        elif host:
            pin = isinstance(pos, torch.Tensor) and pos.is_pinned()
            group = torch.empty(n, dtype=torch.int32, pin_memory=pin)
            dens = torch.empty(n, dtype=torch.float32, pin_memory=pin) if want_dens else None
        else:
            _need(pos, torch.float32, (n, 3), "pos")
            group = torch.empty(n, dtype=torch.int32, device=pos.device)
            dens = torch.empty(n, dtype=torch.float32, device=pos.device) if want_dens else None
        dev = torch.device("cuda", self.device)
        nbr = torch.empty((n, ld_nbr), dtype=torch.int32, device=dev) if ld_nbr else None
        ng = np.zeros(B, dtype=np.int64)
        self._check(self.L.hop_run_batch(self.h, _ptr(pos), _ptr(off), _ptr(bx), B, C.byref(params),
                                         _ptr(dens), _ptr(group), _ptr(ng), _ptr(nbr), ld_nbr or 0,
                                         HOP_BATCH_EAGER if eager else 0))
        return dict(dens=dens, group=group, n_groups=ng, nbr=nbr)

    def hop_halo_stats(self, pos, dens, group, n_groups: int, box: float = 1.0):
        """Per group: count (int64), peak index (int32), centre of mass
        (n_groups x 3 float64), maximum radius (float64), as CUDA tensors."""
        import torch
        self._sync_stream()
        n = pos.shape[0]
        f64 = pos.dtype == torch.float64
        _need(pos, torch.float64 if f64 else torch.float32, (n, 3), "pos")
        _need(dens, torch.float32, (n,), "dens")
        _need(group, torch.int32, (n,), "group")
        dev = pos.device
        G = int(n_groups)
        count = torch.empty(max(G, 1), dtype=torch.int64, device=dev)
        peak = torch.empty(max(G, 1), dtype=torch.int32, device=dev)
        com = torch.empty((max(G, 1), 3), dtype=torch.float64, device=dev)
        rmax = torch.empty(max(G, 1), dtype=torch.float64, device=dev)
        self._check(self.L.hop_halo_stats(self.h, _ptr(pos), 1 if f64 else 0, _ptr(dens), _ptr(group), n, G,
                                          float(box), _ptr(count), _ptr(peak), _ptr(com), _ptr(rmax)))
        return count[:G], peak[:G], com[:G], rmax[:G]

    def hop_subhalos(self, chain, dens, nbr, n_merge: int, delta_outer: float, levels, n_min: int = 1,
                     f_poisson: float = 0.0):
        """ADAPTAHOP subhalos: (sub int32 [L, n] CUDA tensor, n_sub int64
        numpy [L]) for the thresholds in ``levels``."""
        import torch
        self._sync_stream()
        n, ld = nbr.shape
        _need(chain, torch.int32, (n,), "chain")
        _need(dens, torch.float32, (n,), "dens")
        _need(nbr, torch.int32, None, "nbr")
        lv = np.ascontiguousarray(np.atleast_1d(levels), dtype=np.float32)
        sub = torch.empty((len(lv), n), dtype=torch.int32, device=dens.device)
        n_sub = np.zeros(len(lv), dtype=np.int64)
        self._check(self.L.hop_subhalos(self.h, _ptr(chain), _ptr(dens), _ptr(nbr), ld, n, int(n_merge),
                                        float(delta_outer), _ptr(lv), len(lv), int(n_min), float(f_poisson),
                                        _ptr(sub), _ptr(n_sub)))
        return sub, n_sub

    def get_tuning(self) -> dict:
        t = HopTuning()
        self._check(self.L.hop_get_tuning(self.h, C.byref(t)))
        return t.as_dict()

    def apply_tuning(self, qpw: int, cpr: int, buf_factor: int = 0):
        t = HopTuning(qpw, cpr, buf_factor, 0.0)
        self._check(self.L.hop_apply_tuning(self.h, C.byref(t)))

    def hop_autotune(self, pos, offsets, boxes, params: HopParams, candidates, reps: int = 3):
        """Times each (qpw, cpr, buf_factor) candidate on the batched pass and
        applies the fastest; returns (best index, [dict per candidate])."""
        self._sync_stream()
        off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int64))
        bx = np.ascontiguousarray(np.asarray(boxes, dtype=np.float64))
        arr = (HopTuning * len(candidates))(*[HopTuning(q, c, f, 0.0) for q, c, f in candidates])
        best = C.c_int32(-1)
        self._check(self.L.hop_autotune(self.h, _ptr(pos), _ptr(off), _ptr(bx), len(bx), C.byref(params),
                                        arr, len(candidates), reps, C.byref(best)))
        return best.value, [a.as_dict() for a in arr]

    def stats(self) -> dict:
        st = HopStats()
        self._check(self.L.hop_get_stats(self.h, C.byref(st)))
        return st.as_dict()

    # -------------------------------------------------------------- MLP
    def hop_mlp_load(self, params: np.ndarray, log_margin: float = 0.0):
        p = np.ascontiguousarray(params, dtype=np.float32)
        if p.shape != (MLP_NPARAM,):
            raise ValueError(f"expected {MLP_NPARAM} parameters")
        self._sync_stream()
        self._check(self.L.hop_mlp_load(self.h, _ptr(p), float(log_margin)))

    def hop_mlp_get(self) -> np.ndarray:
        p = np.empty(MLP_NPARAM, dtype=np.float32)
        self._check(self.L.hop_mlp_get(self.h, _ptr(p)))
        return p

    def hop_mlp_samples(self):
        import torch
        self._sync_stream()
        nc = C.c_int64(0)
        self._check(self.L.hop_mlp_samples(self.h, None, None, 0, C.byref(nc)))
        dev = torch.device("cuda", self.device)
        feat = torch.empty((nc.value, MLP_IN), dtype=torch.float32, device=dev)
        tgt = torch.empty(nc.value, dtype=torch.float32, device=dev)
        self._check(self.L.hop_mlp_samples(self.h, _ptr(feat), _ptr(tgt), nc.value, C.byref(nc)))
        return feat, tgt

    def hop_mlp_forward(self, feat):
        import torch
        self._sync_stream()
        _need(feat, torch.float32, (feat.shape[0], MLP_IN), "feat")
        out = torch.empty(feat.shape[0], dtype=torch.float32, device=feat.device)
        self._check(self.L.hop_mlp_forward(self.h, _ptr(feat), feat.shape[0], _ptr(out)))
        return out

    def hop_mlp_grad(self, feat, target):
        import torch
        self._sync_stream()
        _need(feat, torch.float32, (feat.shape[0], MLP_IN), "feat")
        _need(target, torch.float32, (feat.shape[0],), "target")
        grad = torch.empty(MLP_NPARAM, dtype=torch.float32, device=feat.device)
        loss = C.c_double(0)
        self._check(self.L.hop_mlp_grad(self.h, _ptr(feat), _ptr(target), feat.shape[0], C.byref(loss),
                                        _ptr(grad)))
        return loss.value, grad

    def hop_mlp_train(self, feat, target, epochs=10, batch=4096, lr=1e-3, seed=0):
        import torch
        self._sync_stream()
        _need(feat, torch.float32, (feat.shape[0], MLP_IN), "feat")
        _need(target, torch.float32, (feat.shape[0],), "target")
        loss = C.c_double(0)
        self._check(self.L.hop_mlp_train(self.h, _ptr(feat), _ptr(target), feat.shape[0], int(epochs),
                                         int(batch), float(lr), int(seed), C.byref(loss)))
        return loss.value
