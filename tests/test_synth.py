"""The seeded input generators against the recipe they state: the
SplitMix64 stream against its published first outputs, counter addressing,
the wrap to [0, L), the Plummer and NFW radial profiles, the power-law halo
masses, the halo and background fractions, the uniform background and the
batch's log-uniform sizes (Kolmogorov-Smirnov tests at fixed seeds)."""
import math

import numpy as np
import pytest

scipy_stats = pytest.importorskip("scipy.stats")

import synth


def _ks_ok(sample, cdf, alpha=1e-3):
    return scipy_stats.kstest(sample, cdf).pvalue > alpha


def test_splitmix64_matches_its_published_outputs():
    # SplitMix64 seeded with 0 (Steele, Lea & Flood 2014): the first three
    # outputs of the reference generator
    z = np.arange(1, 4, dtype=np.uint64) * synth._GAMMA
    got = [int(v) for v in synth._mix(z)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_draws_are_addressed_by_counter():
    a = synth.uniform01(7, 3, 0, 1000)
    assert np.array_equal(a[400:], synth.uniform01(7, 3, 400, 600))
    assert np.all((a >= 0.0) & (a < 1.0))
    assert not np.array_equal(a, synth.uniform01(7, 4, 0, 1000))     # streams differ
    assert not np.array_equal(a, synth.uniform01(8, 3, 0, 1000))     # seeds differ
    assert _ks_ok(a, "uniform")


def test_wrap_lands_in_the_box():
    x = np.array([[-1e-9, 1.0, 0.5], [1.0 - 1e-9, 2.25, -0.75]])
    w = synth._wrap_f32(x, 1.0)
    assert w.dtype == np.float32 and np.all((w >= 0.0) & (w < 1.0))
    assert w[0, 0] == 0.0 and w[1, 0] == 0.0        # 1 - 1e-9 and -1e-9 round to 1.0f, which becomes 0
    assert w[0, 1] == 0.0 and w[1, 1] == 0.25 and w[1, 2] == 0.25


def test_plummer_radii_follow_the_truncated_profile():
    a, r_max = 0.01, 0.5
    pos, cen = synth.plummer_box(n_spheres=3, n_per=4000, a=a, n_background=500, seed=3, min_sep=0.3)
    f_max = r_max ** 3 / (r_max ** 2 + a * a) ** 1.5
    for s in range(3):
        d = pos[s * 4000:(s + 1) * 4000] - cen[s]
        d -= np.round(d)
        r = np.sqrt((d * d).sum(axis=1))
        assert r.max() <= r_max
        assert _ks_ok(r, lambda x: np.minimum(x ** 3 / (x * x + a * a) ** 1.5 / f_max, 1.0))
        # isotropic: the direction cosines are uniform on [-1, 1]
        assert _ks_ok(d[:, 2] / r, lambda c: (c + 1.0) / 2.0)
    for i in range(3):
        for j in range(i):
            v = np.abs(cen[i] - cen[j])
            v = np.minimum(v, 1.0 - v)
            assert np.sqrt((v * v).sum()) >= 0.3
    assert _ks_ok(pos[12000:, 0], "uniform")


def test_nfw_inverse_profile():
    c = 10.0
    inv = synth._NfwInverse(c)
    u = np.linspace(0.0, 1.0, 1001)
    x = inv(u)
    assert x[0] == 0.0 and x[-1] == pytest.approx(c)
    np.testing.assert_allclose(synth._nfw_mu(x) / synth._nfw_mu(c), u, atol=1e-7)


def test_power_law_masses():
    alpha, m_min, m_max = 1.9, 100.0, 1e5
    m = synth._powerlaw_masses(5, 10_000_000, m_min, m_max, alpha)
    assert m.sum() == 10_000_000
    body = m[:-1]                                   # the last one is trimmed to the target
    assert body.min() >= m_min and body.max() <= m_max
    e = 1.0 - alpha
    lo, hi = m_min ** e, m_max ** e
    # floor(M) <= k  <=>  M < k + 1 for the continuous draw M
    cdf = lambda k: np.clip(((np.floor(k) + 1.0) ** e - lo) / (hi - lo), 0.0, 1.0)
    assert _ks_ok(body + 0.5, cdf)
    # the mean of the continuous law (less the floor's half particle on
    # average), within four standard errors of the heavy-tailed law
    norm = (alpha - 1.0) / (m_min ** (1.0 - alpha) - m_max ** (1.0 - alpha))
    mean = norm * (m_max ** (2.0 - alpha) - m_min ** (2.0 - alpha)) / (2.0 - alpha)
    second = norm * (m_max ** (3.0 - alpha) - m_min ** (3.0 - alpha)) / (3.0 - alpha)
    se = math.sqrt((second - mean * mean) / len(body))
    assert abs(body.mean() - (mean - 0.5)) < 4.0 * se
    assert 850.0 < mean < 950.0                     # about 900 particles per halo


def test_nfw_box_fractions_profile_and_background():
    n, seed, conc = 1_000_000, 9, 10.0
    pos, sizes = synth.nfw_box(n, seed, conc=conc)
    n_halo = int(round(0.6 * n))
    assert sizes.sum() == n_halo and pos.shape == (n, 3) and pos.dtype == np.float32
    assert np.all((pos >= 0.0) & (pos < 1.0))
    # centres as the generator draws them; radii of the largest halo
    nh = len(sizes)
    cen = np.stack([synth.uniform01(seed, 50 + ax, 0, nh) for ax in range(3)], axis=1)
    h = int(np.argmax(sizes))
    start = int(sizes[:h].sum())
    d = pos[start:start + sizes[h]].astype(np.float64) - cen[h]
    d -= np.round(d)
    r = np.sqrt((d * d).sum(axis=1))
    rvir = math.cbrt(3.0 * sizes[h] / (4.0 * math.pi * 200.0 * n))
    assert r.max() <= rvir * (1 + 1e-5)
    mu_c = synth._nfw_mu(conc)
    assert _ks_ok(r, lambda x: np.minimum(synth._nfw_mu(np.asarray(x) * conc / rvir) / mu_c, 1.0))
    # the background is the last 40 %, uniform on every axis
    for ax in range(3):
        assert _ks_ok(pos[n_halo:, ax].astype(np.float64), "uniform")


def test_batch_sizes_are_log_uniform():
    n_lo, n_hi = 16, 4096
    pos, off = synth.nfw_batch(n_sub=120, seed=3, n_lo=n_lo, n_hi=n_hi)
    sizes = np.diff(off)
    assert off[0] == 0 and pos.shape == (off[-1], 3)
    assert sizes.min() >= n_lo and sizes.max() <= n_hi
    # floor of a log-uniform draw: P(size <= k) = P(draw < k + 1)
    cdf = lambda y: np.clip((np.log(np.floor(y) + 1.0) - math.log(n_lo)) / math.log(n_hi / n_lo), 0.0, 1.0)
    assert _ks_ok(sizes + 0.5, cdf)
    # each subvolume is its own box: 30 % of it uniform background
    b = int(np.argmax(sizes))
    sub = pos[off[b]:off[b + 1]]
    assert _ks_ok(sub[int(round(0.7 * len(sub))):, 1].astype(np.float64), "uniform")


def test_workload_seeds_follow_the_convention():
    assert synth.workload_seed(3) == 0x10013411 + 3000
    assert synth.workload_seed(4, 7) == 0x10013411 + 4007
