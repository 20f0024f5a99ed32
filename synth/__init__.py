"""Seeded synthetic particle sets for the HOP halo finder.

This module only draws inputs.  It holds none of HOP's arithmetic (no
distances, densities, links or merges), so both the CPU oracle tests and the
GPU path can take their inputs from here without sharing method code.

Every random number comes from one counter-based generator: the SplitMix64
output function (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) applied to ``base(seed, stream) + (counter + 1) * gamma``
with gamma = 0x9E3779B97F4A7C15.  A draw is therefore a pure function of
(seed, stream, counter): the same on every machine, thread count and chunking.

Workloads (the paper's ENZO datasets are not available; these stand in for
them, with the particle counts and halo structure of a cosmological box):

* ``plummer_box``   -- Plummer spheres plus a uniform background (fp64).
* ``nfw_box``       -- NFW halos with power-law masses plus uniform background.
* ``nfw_batch``     -- many independent periodic subvolumes of uneven size.
* ``uniform_box``   -- Poisson points, used for the mean-density closed form.
* ``lattice_box``   -- a simple cubic lattice (exact distances, many ties).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

__all__ = [
    "uniform01", "uniform_box", "lattice_box", "plummer_box", "nfw_box",
    "nfw_batch", "workload", "WORKLOADS", "workload_seed",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO53 = 1.0 / 9007199254740992.0


def _mix(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function on uint64 arrays (wrapping arithmetic)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _base(seed: int, stream: int) -> np.uint64:
    s = np.array([(seed * 0x100000001B3 + stream * 0x632BE59BD9B4E019) & 0xFFFFFFFFFFFFFFFF],
                 dtype=np.uint64)
    return _mix(s)[0]


def uniform01(seed: int, stream: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1): draw ``start .. start+count-1`` of stream ``stream``."""
    ctr = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = _base(seed, stream) + ctr * _GAMMA
    return (_mix(z) >> np.uint64(11)).astype(np.float64) * _TWO53


def _wrap_f32(pos: np.ndarray, box: float) -> np.ndarray:
    """Wrap into [0, box) and round to fp32; a value that rounds to box becomes 0."""
    p = np.mod(pos, box).astype(np.float32)
    p[p >= np.float32(box)] = 0.0
    return p


def _wrap_f64(pos: np.ndarray, box: float) -> np.ndarray:
    p = np.mod(pos, box)
    p[p >= box] = 0.0
    return p


def _threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _chunked(n: int, fn, chunk: int = 1 << 22) -> None:
    """Run fn(lo, hi) over [0, n) in chunks on a thread pool (numpy releases the GIL)."""
    spans = [(lo, min(n, lo + chunk)) for lo in range(0, n, chunk)]
    if len(spans) <= 1:
        for lo, hi in spans:
            fn(lo, hi)
        return
    with ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(lambda s: fn(*s), spans))


def _isotropic(seed: int, s_mu: int, s_phi: int, lo: int, hi: int):
    mu = 2.0 * uniform01(seed, s_mu, lo, hi - lo) - 1.0
    phi = 2.0 * math.pi * uniform01(seed, s_phi, lo, hi - lo)
    st = np.sqrt(np.maximum(0.0, 1.0 - mu * mu))
    return st * np.cos(phi), st * np.sin(phi), mu


def uniform_box(n: int, seed: int, box: float = 1.0, dtype=np.float32) -> np.ndarray:
    """n Poisson points in [0, box)^3."""
    out = np.empty((n, 3), dtype=np.float64)
    for a in range(3):
        out[:, a] = uniform01(seed, 100 + a, 0, n) * box
    return _wrap_f32(out, box) if dtype == np.float32 else _wrap_f64(out, box)


def lattice_box(m: int, box: float = 1.0, dtype=np.float32) -> np.ndarray:
    """A simple cubic lattice of m^3 points with spacing box/m (x fastest)."""
    g = np.arange(m, dtype=np.float64) * (box / m)
    z, y, x = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)
    return pos.astype(dtype)


def _centres(seed: int, n: int, box: float, min_sep: float) -> np.ndarray:
    """Uniform centres; with min_sep > 0 a candidate closer than min_sep
    (periodic) to an accepted centre is skipped, in counter order."""
    acc = []
    k = 0
    while len(acc) < n:
        c = np.array([uniform01(seed, 10 + a, k, 1)[0] * box for a in range(3)])
        k += 1
        ok = True
        for d in acc:
            v = np.abs(c - d)
            v = np.minimum(v, box - v)
            if float(np.sqrt((v * v).sum())) < min_sep:
                ok = False
                break
        if ok:
            acc.append(c)
        if k > 100000:
            raise RuntimeError("cannot place centres with this separation")
    return np.array(acc)


def plummer_box(n_spheres: int = 20, n_per: int = 1146, a: float = 0.01,
                n_background: int = 9848, seed: int = 0, box: float = 1.0,
                r_max: float = 0.5, min_sep: float = 0.0,
                dtype=np.float64):
    """Plummer spheres (scale radius a, truncated at r_max) plus uniform background.

    The radius is drawn from the Plummer enclosed-mass fraction
    F(r) = r^3 / (r^2 + a^2)^{3/2} restricted to r <= r_max, i.e.
    r = a (u^{-2/3} - 1)^{-1/2} with u uniform in (0, F(r_max)].
    Returns (pos, centres); halo particles come first, sphere by sphere.
    """
    cen = _centres(seed, n_spheres, box, min_sep)
    nh = n_spheres * n_per
    f_max = r_max ** 3 / (r_max ** 2 + a * a) ** 1.5
    u = (1.0 - uniform01(seed, 20, 0, nh)) * f_max
    r = a / np.sqrt(np.maximum(u ** (-2.0 / 3.0) - 1.0, 1e-300))
    ex, ey, ez = _isotropic(seed, 21, 22, 0, nh)
    hid = np.repeat(np.arange(n_spheres), n_per)
    pos = np.empty((nh + n_background, 3), dtype=np.float64)
    pos[:nh, 0] = cen[hid, 0] + r * ex
    pos[:nh, 1] = cen[hid, 1] + r * ey
    pos[:nh, 2] = cen[hid, 2] + r * ez
    for ax in range(3):
        pos[nh:, ax] = uniform01(seed, 30 + ax, 0, n_background) * box
    pos = _wrap_f64(pos, box) if dtype == np.float64 else _wrap_f32(pos, box)
    return pos, cen


def plummer_pair(n_per: int = 1500, a: float = 0.01, sep: float = 0.04, n_background: int = 3000,
                 seed: int = 0, box: float = 1.0, r_max: float = 0.25, dtype=np.float64) -> np.ndarray:
    """Two Plummer spheres of n_per particles (scale radius a) whose centres
    sit sep apart along x about the box centre, plus a uniform background: a
    halo with one subhalo.  Returns (pos, centres)."""
    cen = np.array([[0.5 * box - 0.5 * sep, 0.5 * box, 0.5 * box],
                    [0.5 * box + 0.5 * sep, 0.5 * box, 0.5 * box]])
    nh = 2 * n_per
    f_max = r_max ** 3 / (r_max ** 2 + a * a) ** 1.5
    u = (1.0 - uniform01(seed, 40, 0, nh)) * f_max
    r = a / np.sqrt(np.maximum(u ** (-2.0 / 3.0) - 1.0, 1e-300))
    ex, ey, ez = _isotropic(seed, 41, 42, 0, nh)
    hid = np.repeat(np.arange(2), n_per)
    pos = np.empty((nh + n_background, 3), dtype=np.float64)
    pos[:nh, 0] = cen[hid, 0] + r * ex
    pos[:nh, 1] = cen[hid, 1] + r * ey
    pos[:nh, 2] = cen[hid, 2] + r * ez
    for ax in range(3):
        pos[nh:, ax] = uniform01(seed, 50 + ax, 0, n_background) * box
    pos = _wrap_f64(pos, box) if dtype == np.float64 else _wrap_f32(pos, box)
    return pos, cen


def chain_graph_case(n: int, n_merge: int, n_chains: int, seed: int, mutual: bool = False):
    """A random chain structure for the merging stages, without positions:
    (chain int32 [n], dens float64 [n] holding float32 values, rows int32
    [n, n_merge]).  n_chains roots, each the densest member of its chain
    (hops climb); densities gamma-distributed around 120; rows hold the
    particle itself first, then random particles (with ``mutual``, n_merge - 1
    random pairings, so that every link has its reverse)."""
    rng = np.random.default_rng(seed)
    dens = np.round(rng.gamma(2.0, 60.0, n), 1).astype(np.float32).astype(np.float64)
    roots = rng.choice(n, n_chains, replace=False)
    chain = roots[rng.integers(0, n_chains, n)].astype(np.int32)
    chain[roots] = roots
    top = np.zeros(n)
    np.maximum.at(top, chain, dens)
    dens[roots] = top[roots] + 1.0
    rows = np.empty((n, n_merge), dtype=np.int32)
    rows[:, 0] = np.arange(n)
    if mutual:
        for t in range(1, n_merge):
            p = rng.permutation(n)
            partner = np.empty(n, dtype=np.int32)
            partner[p[0::2]] = p[1::2]
            partner[p[1::2]] = p[0::2]
            rows[:, t] = partner
    else:
        rows[:, 1:] = rng.integers(0, n, (n, n_merge - 1))
    return chain, dens, rows


def _nfw_mu(x):
    return np.log1p(x) - x / (1.0 + x)


class _NfwInverse:
    """Inverse of the NFW enclosed-mass profile mu(x) = ln(1+x) - x/(1+x) on
    [0, c], by monotone interpolation of a dense fp64 table in log x."""

    def __init__(self, c: float, n: int = 400001):
        x = np.concatenate([[0.0], np.geomspace(1e-7 * c, c, n)])
        self.x = x
        self.mu = _nfw_mu(x)
        self.mu_c = float(self.mu[-1])

    def __call__(self, frac: np.ndarray) -> np.ndarray:
        return np.interp(frac * self.mu_c, self.mu, self.x)


def _powerlaw_masses(seed: int, target: int, m_min: float, m_max: float,
                     alpha: float) -> np.ndarray:
    """Integer halo sizes from dN/dM ~ M^-alpha on [m_min, m_max], drawn in
    counter order until they hold ``target`` particles; the last is trimmed."""
    e = 1.0 - alpha
    lo, hi = m_min ** e, m_max ** e
    mean = (e / (e + 1.0)) * (m_max ** (e + 1) - m_min ** (e + 1)) / (hi - lo) if abs(e + 1) > 1e-12 else m_min
    est = int(target / max(mean, 1.0) * 1.5) + 16
    start = 0
    parts = []
    total = 0
    while total < target:
        u = uniform01(seed, 40, start, est)
        m = np.floor((lo + u * (hi - lo)) ** (1.0 / e)).astype(np.int64)
        m = np.clip(m, int(m_min), int(m_max))
        parts.append(m)
        total += int(m.sum())
        start += est
    m = np.concatenate(parts)
    cs = np.cumsum(m)
    k = int(np.searchsorted(cs, target))  # first index where cs >= target
    m = m[: k + 1].copy()
    m[-1] -= int(cs[k] - target)
    return m[m > 0]


def nfw_box(n: int, seed: int, halo_frac: float = 0.6, conc: float = 10.0,
            m_min: float = 100.0, m_max: float = 1e5, alpha: float = 1.9,
            overdensity: float = 200.0, box: float = 1.0, dtype=np.float32):
    """NFW halos (concentration ``conc``, truncated at R_vir) plus uniform background.

    Halo sizes follow dN/dM ~ M^-alpha; R_vir encloses ``overdensity`` times the
    box's mean particle density, R_vir = box (3 M / (4 pi overdensity n))^{1/3}.
    Radii invert the NFW enclosed mass, r = R_vir x / c with mu(x) = u mu(c).
    Halo particles come first (halo by halo), then the background.
    Returns (pos [n,3], halo_sizes).
    """
    n_halo = int(round(halo_frac * n))
    sizes = _powerlaw_masses(seed, n_halo, m_min, m_max, alpha) if n_halo > 0 else np.zeros(0, np.int64)
    nh_count = len(sizes)
    cen = np.empty((nh_count, 3))
    for ax in range(3):
        cen[:, ax] = uniform01(seed, 50 + ax, 0, nh_count) * box
    rvir = box * np.cbrt(3.0 * sizes / (4.0 * math.pi * overdensity * n))
    inv = _NfwInverse(conc)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    pos = np.empty((n, 3), dtype=dtype)

    def halo_chunk(lo, hi):
        hid = np.searchsorted(starts, np.arange(lo, hi), side="right") - 1
        x = inv(1.0 - uniform01(seed, 60, lo, hi - lo))
        r = rvir[hid] * x / conc
        ex, ey, ez = _isotropic(seed, 61, 62, lo, hi)
        p = np.empty((hi - lo, 3))
        p[:, 0] = cen[hid, 0] + r * ex
        p[:, 1] = cen[hid, 1] + r * ey
        p[:, 2] = cen[hid, 2] + r * ez
        pos[lo:hi] = _wrap_f32(p, box) if dtype == np.float32 else _wrap_f64(p, box)

    def bg_chunk(lo, hi):
        p = np.empty((hi - lo, 3))
        for ax in range(3):
            p[:, ax] = uniform01(seed, 70 + ax, lo, hi - lo) * box
        pos[n_halo + lo: n_halo + hi] = _wrap_f32(p, box) if dtype == np.float32 else _wrap_f64(p, box)

    _chunked(n_halo, halo_chunk)
    _chunked(n - n_halo, bg_chunk)
    return pos, sizes


def nfw_batch(n_sub: int = 64, seed: int = 0, n_lo: int = 4096, n_hi: int = 2097152,
              halo_frac: float = 0.7, **kw):
    """``n_sub`` independent periodic unit subvolumes, sizes log-uniform in
    [n_lo, n_hi], each an ``nfw_box`` with its own seed.  Returns
    (pos [sum N_b, 3] fp32, offsets [n_sub+1] int64)."""
    u = uniform01(seed, 80, 0, n_sub)
    sizes = np.floor(np.exp(math.log(n_lo) + u * (math.log(n_hi) - math.log(n_lo)))).astype(np.int64)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pos = np.empty((int(offsets[-1]), 3), dtype=np.float32)
    for b in range(n_sub):
        p, _ = nfw_box(int(sizes[b]), seed * 1000 + 17 + b, halo_frac=halo_frac, **kw)
        pos[offsets[b]:offsets[b + 1]] = p
    return pos, offsets


def workload_seed(config: int, sub: int = 0) -> int:
    """Seed convention: 0x10013411 + config*1000 + sub."""
    return 0x10013411 + config * 1000 + sub


WORKLOADS = {
    "plummer32k": "32,768 fp64 particles: 20 Plummer spheres (a=0.01, 1,146 each) + 9,848 uniform",
    "nfw256": "256^3 fp32 particles: 60% NFW halos (c=10, M in [100,1e5], dN/dM~M^-1.9) + 40% uniform",
    "nfw512": "512^3 fp32 particles: same NFW + 40% background generator",
    "batch64": "64 periodic subvolumes, N_b log-uniform in [16^3,128^3], NFW + 30% background, fp32",
    "nfw1024": "1024^3 fp32 particles: NFW (M up to 1e6) + 40% background",
}


def workload(name: str, sub: int = 0, scale: int | None = None):
    """Build a named workload.  ``scale`` overrides the particle count of the
    NFW boxes (same generator, fewer particles) for small test cases."""
    if name == "plummer32k":
        pos, _ = plummer_box(seed=workload_seed(1, sub), min_sep=0.1)
        return pos
    if name in ("nfw256", "nfw512", "nfw1024"):
        cfg = {"nfw256": (2, 256 ** 3, 1e5), "nfw512": (3, 512 ** 3, 1e5),
               "nfw1024": (5, 1024 ** 3, 1e6)}[name]
        n = scale if scale is not None else cfg[1]
        pos, _ = nfw_box(n, workload_seed(cfg[0], sub), m_max=cfg[2])
        return pos
    if name == "batch64":
        return nfw_batch(seed=workload_seed(4, sub))
    raise KeyError(name)
