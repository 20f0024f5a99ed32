"""Pins of the oracle's halo statistics (C8: mass, centre of mass and
maximum radius of every halo, Parallel HOP Sec. 3) against what geometry
fixes: plain means and distances away from the faces, periodic translation
invariance, symmetric shells, subsets, and the Plummer spheres' own centres."""
import numpy as np
import pytest

import oracle
import synth


def _cluster(n, centre, sigma, seed):
    rng = np.random.default_rng(seed)
    return centre + rng.normal(0.0, sigma, (n, 3))


def _peak(dens, idx):
    # greatest density, then the smaller index
    order = np.lexsort((idx, -dens[idx]))
    return idx[order[0]]


def test_compact_cluster_matches_plain_mean_and_distances():
    pos = _cluster(700, np.array([0.5, 0.45, 0.55]), 0.02, 1)
    dens = np.random.default_rng(2).random(700)
    group = np.zeros(700, dtype=np.int32)
    count, peak, com, rmax = oracle.halo_stats(pos, dens, group, 1)
    assert count[0] == 700
    assert peak[0] == _peak(dens, np.arange(700))
    mean = pos.mean(axis=0)
    np.testing.assert_allclose(com[0], mean, rtol=0, atol=1e-13)
    r = np.sqrt(((pos - mean) ** 2).sum(axis=1))
    assert rmax[0] == pytest.approx(r.max(), rel=1e-12)


@pytest.mark.parametrize("shift", [(0.5, 0.55, 0.45), (-0.49, 0.0, 0.5), (0.03, -0.52, 0.51)])
def test_translation_across_faces_moves_the_centre_only(shift):
    base = _cluster(500, np.array([0.5, 0.5, 0.5]), 0.015, 3)
    dens = np.random.default_rng(4).random(500)
    group = np.zeros(500, dtype=np.int32)
    c0, p0, com0, r0 = oracle.halo_stats(base, dens, group, 1)
    moved = np.mod(base + np.array(shift), 1.0)
    c1, p1, com1, r1 = oracle.halo_stats(moved, dens, group, 1)
    assert c1[0] == c0[0] and p1[0] == p0[0]
    want = np.mod(com0[0] + np.array(shift), 1.0)
    d = (com1[0] - want + 0.5) % 1.0 - 0.5          # compare modulo the box
    assert np.abs(d).max() < 1e-12
    assert r1[0] == pytest.approx(r0[0], rel=1e-10)


def test_symmetric_shell_has_its_centre_and_radius():
    rng = np.random.default_rng(5)
    v = rng.normal(size=(200, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    c = np.array([0.02, 0.98, 0.5])                 # straddles two faces
    rho = 0.03
    pts = np.concatenate([c + rho * v, c - rho * v])
    pos = np.mod(pts, 1.0)
    dens = np.ones(400)
    dens[7] = 2.0                                    # the peak
    count, peak, com, rmax = oracle.halo_stats(pos, dens, np.zeros(400, dtype=np.int32), 1)
    assert peak[0] == 7
    d = (com[0] - c + 0.5) % 1.0 - 0.5
    assert np.abs(d).max() < 1e-14
    assert rmax[0] == pytest.approx(rho, rel=1e-12)


@pytest.mark.parametrize("axis,side", [(0, "low"), (0, "high"), (1, "low"), (1, "high")])
def test_centre_wraps_when_the_peak_is_across_a_face(axis, side):
    """A symmetric shell whose centre lies just inside one face while its
    peak particle sits across it: the centre about the peak falls outside
    [0, 1) before wrapping, and must come back to the shell's centre."""
    rng = np.random.default_rng(8 + axis)
    v = rng.normal(size=(150, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    c = np.array([0.5, 0.5, 0.5])
    c[axis] = 0.998 if side == "low" else 0.002
    rho = 0.006
    pts = np.concatenate([c + rho * v, c - rho * v])
    pos = np.mod(pts, 1.0)
    # the peak: the member farthest across the face from the centre
    k = int(np.argmax(pts[:, axis])) if side == "low" else int(np.argmin(pts[:, axis]))
    assert (pts[k, axis] >= 1.0) if side == "low" else (pts[k, axis] < 0.0)
    dens = np.ones(len(pos))
    dens[k] = 2.0
    count, peak, com, rmax = oracle.halo_stats(pos, dens, np.zeros(len(pos), dtype=np.int32), 1)
    assert peak[0] == k
    assert np.all((com[0] >= 0.0) & (com[0] < 1.0))
    np.testing.assert_allclose(com[0], c, rtol=0, atol=1e-14)
    assert rmax[0] == pytest.approx(rho, rel=1e-12)


def test_each_group_equals_its_subset_alone_and_no_halo_is_skipped():
    rng = np.random.default_rng(6)
    pos = rng.random((3000, 3))
    dens = rng.random(3000)
    group = rng.integers(-1, 7, 3000).astype(np.int32)
    count, peak, com, rmax = oracle.halo_stats(pos, dens, group, 7)
    assert count.sum() == (group >= 0).sum()
    for g in range(7):
        sel = np.flatnonzero(group == g)
        c, p, cm, r = oracle.halo_stats(pos[sel], dens[sel], np.zeros(len(sel), dtype=np.int32), 1)
        assert count[g] == c[0] and peak[g] == sel[p[0]]
        np.testing.assert_allclose(com[g], cm[0], rtol=0, atol=1e-15)
        assert rmax[g] == r[0]


def test_group_id_out_of_range_is_an_error():
    pos = np.random.default_rng(7).random((10, 3))
    with pytest.raises(RuntimeError):
        oracle.halo_stats(pos, np.ones(10), np.full(10, 3, dtype=np.int32), 3)


def test_plummer_halo_centres_sit_on_the_sphere_centres():
    """The 20 isolated Plummer spheres: every halo's centre of mass lies
    within a small fraction of the scale radius of one sphere's centre, and
    its maximum radius within the delta_outer surface (about 2.3 a)."""
    a = 0.01
    pos, cen = synth.plummer_box(seed=synth.workload_seed(1), min_sep=0.1)
    r = oracle.hop(pos)
    assert r["n_groups"] == 20
    count, peak, com, rmax = oracle.halo_stats(pos, r["dens"], r["group"], r["n_groups"])
    for g in range(20):
        d = (cen - com[g] + 0.5) % 1.0 - 0.5
        dist = np.sqrt((d ** 2).sum(axis=1))
        assert dist.min() < 0.2 * a, (g, dist.min())
        assert 600 < count[g] <= 1146 + 50
        assert 1.0 * a < rmax[g] < 4.0 * a
