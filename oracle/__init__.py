"""CPU fp64 oracle for the HOP hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product path (``paper_1001_3411_gb300``)
never imports, links or calls it, and this package imports nothing from the
product.  It wraps ``hop_oracle.c`` (plain C, OpenMP over independent
particles) through ctypes; the library is compiled with gcc on first use.

Functions follow HOP as restated in Parallel HOP (arXiv:1001.3411), Sec. 2:
``knn`` (C1), ``density`` (C2), ``link`` (C3, C4), ``boundaries`` (C5),
``merge`` (C6, C7), ``halo_stats`` (C8, Sec. 3), ``hop`` (C1-C7) and
ADAPTAHOP's subhalos (C9, Sec. 6): ``sym_boundaries`` and ``subhalos``.
Every function is pinned by the ``tests/test_oracle_*.py`` files.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hop_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, EINVAL, ENOMEM, ECYCLE, ECAP = 0, 1, 2, 3, 4


def build(force: bool = False) -> str:
    """Compile the oracle library (gcc -O2 -fopenmp); returns its path.

    ``HOP_ORACLE_LIB`` names another build of ``hop_oracle.c`` to load
    instead: the mutation tests point it at copies compiled with one planted
    mistake each, to show that the pins catch it."""
    override = os.environ.get("HOP_ORACLE_LIB")
    if override:
        return override
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-std=c11", "-D_GNU_SOURCE",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            i64, i32, dbl, vp = C.c_int64, C.c_int32, C.c_double, C.c_void_p
            lib.orc_knn.argtypes = [vp, i64, dbl, i32, vp, i64, vp, vp]
            lib.orc_density.argtypes = [vp, i64, i32, i64, dbl, vp]
            lib.orc_link.argtypes = [vp, vp, i32, i64, i32, vp, vp]
            lib.orc_boundaries.argtypes = [vp, vp, vp, i32, i64, i32, dbl, vp, vp, vp, i64, vp]
            lib.orc_merge.argtypes = [vp, vp, i64, vp, vp, vp, i64, dbl, dbl, dbl, vp, vp]
            lib.orc_halo_stats.argtypes = [vp, vp, vp, i64, i64, dbl, vp, vp, vp, vp]
            lib.orc_sym_boundaries.argtypes = [vp, vp, vp, i32, i64, i32, dbl, vp, vp, vp, i64, vp]
            lib.orc_subhalos.argtypes = [vp, vp, i64, vp, vp, vp, i64, vp, i32, i64, dbl, vp, vp]
            lib.orc_set_threads.argtypes = [C.c_int]
            for f in ("orc_knn", "orc_density", "orc_link", "orc_boundaries", "orc_merge",
                      "orc_halo_stats", "orc_sym_boundaries", "orc_subhalos", "orc_num_threads"):
                getattr(lib, f).restype = C.c_int
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def _check(rc: int, what: str):
    if rc != OK:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def num_threads() -> int:
    return _L().orc_num_threads()


def set_threads(n: int) -> None:
    _L().orc_set_threads(int(n))


def knn(pos, k: int, box: float = 1.0, queries=None):
    """C1: (nbr int32 [nq,k], d2 float64 [nq,k]) for the given query indices
    (all particles when None).  pos is promoted to fp64 exactly."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    n = pos.shape[0]
    q = None if queries is None else np.ascontiguousarray(queries, dtype=np.int64)
    nq = n if q is None else q.shape[0]
    nbr = np.empty((nq, k), dtype=np.int32)
    d2 = np.empty((nq, k), dtype=np.float64)
    _check(_L().orc_knn(_p(pos), n, float(box), int(k), None if q is None else _p(q), nq,
                        _p(nbr), _p(d2)), "knn")
    return nbr, d2


def density(d2, n_total: int, box: float = 1.0):
    """C2: fp64 density contrast from each row of sorted squared distances."""
    d2 = np.ascontiguousarray(d2, dtype=np.float64)
    nq, k = d2.shape
    dens = np.empty(nq, dtype=np.float64)
    _check(_L().orc_density(_p(d2), nq, k, int(n_total), float(box), _p(dens)), "density")
    return dens


def link(dens, nbr, n_hop: int):
    """C3 + C4: (hop, chain) int32 arrays; chain labels are root indices."""
    dens = np.ascontiguousarray(dens, dtype=np.float64)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    n, ld = nbr.shape
    hop = np.empty(n, dtype=np.int32)
    chain = np.empty(n, dtype=np.int32)
    _check(_L().orc_link(_p(dens), _p(nbr), ld, n, int(n_hop), _p(hop), _p(chain)), "link")
    return hop, chain


def _table(fn, what, chain, dens, nbr, n_merge, delta_outer):
    chain = np.ascontiguousarray(chain, dtype=np.int32)
    dens = np.ascontiguousarray(dens, dtype=np.float64)
    nbr = np.ascontiguousarray(nbr, dtype=np.int32)
    n, ld = nbr.shape
    ne = C.c_int64(0)
    _check(fn(_p(chain), _p(dens), _p(nbr), ld, n, int(n_merge), float(delta_outer),
              None, None, None, 0, C.byref(ne)), what)
    cap = max(1, ne.value)
    lo = np.empty(cap, dtype=np.int32)
    hi = np.empty(cap, dtype=np.int32)
    s = np.empty(cap, dtype=np.float64)
    _check(fn(_p(chain), _p(dens), _p(nbr), ld, n, int(n_merge), float(delta_outer),
              _p(lo), _p(hi), _p(s), cap, C.byref(ne)), what)
    e = ne.value
    return lo[:e], hi[:e], s[:e]


def boundaries(chain, dens, nbr, n_merge: int, delta_outer: float):
    """C5: (lo int32 [E], hi int32 [E], s float64 [E]) ordered by (lo, hi);
    s is the maximum summed density (twice the average) per chain pair."""
    return _table(_L().orc_boundaries, "boundaries", chain, dens, nbr, n_merge, delta_outer)


def sym_boundaries(chain, dens, nbr, n_merge: int, delta_outer: float):
    """C9a: the pairs of C5 whose chains link each other in both directions
    (lo, hi, s as in ``boundaries``)."""
    return _table(_L().orc_sym_boundaries, "sym_boundaries", chain, dens, nbr, n_merge, delta_outer)


def subhalos(chain, dens, lo, hi, s, levels, n_min: int = 1, f_poisson: float = 0.0):
    """C9b: (sub int32 [L, n], n_sub int64 [L]) for the thresholds in
    ``levels``: per level, the rank of each particle's subhalo or -1."""
    chain = np.ascontiguousarray(chain, dtype=np.int32)
    dens = np.ascontiguousarray(dens, dtype=np.float64)
    lo = np.ascontiguousarray(lo, dtype=np.int32)
    hi = np.ascontiguousarray(hi, dtype=np.int32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    lv = np.ascontiguousarray(np.atleast_1d(levels), dtype=np.float64)
    n = chain.shape[0]
    sub = np.empty((len(lv), n), dtype=np.int32)
    n_sub = np.zeros(len(lv), dtype=np.int64)
    _check(_L().orc_subhalos(_p(chain), _p(dens), n, _p(lo), _p(hi), _p(s), lo.shape[0], _p(lv),
                             len(lv), int(n_min), float(f_poisson), _p(sub), _p(n_sub)), "subhalos")
    return sub, n_sub


def adaptahop(chain, dens, nbr, n_merge: int, delta_outer: float, levels, n_min: int = 1,
              f_poisson: float = 0.0):
    """C9: symmetric boundaries, then subhalos at every level."""
    lo, hi, s = sym_boundaries(chain, dens, nbr, n_merge, delta_outer)
    return subhalos(chain, dens, lo, hi, s, levels, n_min, f_poisson)


def merge(chain, dens, lo, hi, s, delta_outer: float, delta_saddle: float, delta_peak: float):
    """C6 + C7: (group int32 [n], n_groups)."""
    chain = np.ascontiguousarray(chain, dtype=np.int32)
    dens = np.ascontiguousarray(dens, dtype=np.float64)
    lo = np.ascontiguousarray(lo, dtype=np.int32)
    hi = np.ascontiguousarray(hi, dtype=np.int32)
    s = np.ascontiguousarray(s, dtype=np.float64)
    n = chain.shape[0]
    group = np.empty(n, dtype=np.int32)
    ng = C.c_int64(0)
    _check(_L().orc_merge(_p(chain), _p(dens), n, _p(lo), _p(hi), _p(s), lo.shape[0],
                          float(delta_outer), float(delta_saddle), float(delta_peak),
                          _p(group), C.byref(ng)), "merge")
    return group, ng.value


def halo_stats(pos, dens, group, n_groups: int, box: float = 1.0):
    """C8: per group (count int64, peak int32, com [G, 3] fp64, rmax fp64)."""
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    dens = np.ascontiguousarray(dens, dtype=np.float64)
    group = np.ascontiguousarray(group, dtype=np.int32)
    n = group.shape[0]
    count = np.zeros(n_groups, dtype=np.int64)
    peak = np.zeros(n_groups, dtype=np.int32)
    com = np.zeros((n_groups, 3), dtype=np.float64)
    rmax = np.zeros(n_groups, dtype=np.float64)
    _check(_L().orc_halo_stats(_p(pos), _p(dens), _p(group), n, int(n_groups), float(box), _p(count),
                               _p(peak), _p(com), _p(rmax)), "halo_stats")
    return count, peak, com, rmax


DEFAULTS = dict(n_dens=64, n_hop=16, n_merge=4, delta_outer=80.0, delta_saddle=200.0,
                delta_peak=240.0)


def hop(pos, box: float = 1.0, n_dens: int = 64, n_hop: int = 16, n_merge: int = 4,
        delta_outer: float = 80.0, delta_saddle: float = 200.0, delta_peak: float = 240.0):
    """The whole method on the CPU: returns a dict with nbr, d2, dens, hop,
    chain, lo, hi, s, group, n_groups (all fp64 / int32, original order)."""
    n = len(pos)
    nbr, d2 = knn(pos, n_dens, box)
    dens = density(d2, n, box)
    hp, ch = link(dens, nbr, n_hop)
    lo, hi, s = boundaries(ch, dens, nbr, n_merge, delta_outer)
    group, ng = merge(ch, dens, lo, hi, s, delta_outer, delta_saddle, delta_peak)
    return dict(nbr=nbr, d2=d2, dens=dens, hop=hp, chain=ch, lo=lo, hi=hi, s=s,
                group=group, n_groups=ng)
