"""The parity gate itself, on the CPU: the checkers the GPU tests use
(`hop_parity.check_knn_rows`, `check_density`) accept the oracle's own
results and the differences the tolerances allow (equal-distance swaps at
the list's edge, density rounding below 1e-5), and reject each plausible
kernel mistake planted in a copy of those results: a neighbour missing, one
too far, two out of order, a duplicate, an exact tie in the wrong order, a
density off by more than the tolerance, a finite density where the oracle
has an infinite one."""
import numpy as np
import pytest

import oracle
import synth
from hop_parity import check_density, check_knn_rows

K = 16


@pytest.fixture(scope="module")
def cloud():
    pos = synth.uniform_box(3000, 21).astype(np.float64)
    q = np.arange(0, 3000, 37)
    nbr, d2 = oracle.knn(pos, K + 4, 1.0, queries=q)
    return pos, q, nbr, d2


@pytest.fixture(scope="module")
def lattice():
    pos = synth.lattice_box(8).astype(np.float64)          # 512 points, every distance tied
    q = np.arange(0, len(pos), 5)
    nbr, d2 = oracle.knn(pos, 32, 1.0, queries=q)
    return pos, q, nbr, d2


def _rejects(pos, rows, q, k=K):
    with pytest.raises(AssertionError):
        check_knn_rows(pos, rows, q, k)


def test_accepts_the_oracle_lists(cloud, lattice):
    pos, q, nbr, _ = cloud
    check_knn_rows(pos, nbr[:, :K], q, K)
    check_knn_rows(pos, nbr[:, :4], q, K)                  # an Nhop prefix of the list
    pos, q, nbr, _ = lattice
    check_knn_rows(pos, nbr[:, :19], q, 19)


def test_accepts_an_equal_distance_swap_at_the_edge(lattice):
    # a list of 10 = 1 + 6 + 3 ends inside the shell of 12 particles at
    # sqrt(2) spacings; the oracle closes it with the smallest remaining
    # index, and any other particle of that shell may close it as well
    pos, q, nbr, d2 = lattice
    rows = nbr[:, :10].copy()
    assert np.all(d2[:, 9] == d2[:, 10])
    rows[:, 9] = nbr[:, 10]
    check_knn_rows(pos, rows, q, 10)


def test_rejects_a_farther_particle_in_place_of_the_last(cloud):
    pos, q, nbr, d2 = cloud
    assert np.all(d2[:, K] > d2[:, K - 1] * (1 + 1e-5))
    rows = nbr[:, :K].copy()
    rows[3, K - 1] = nbr[3, K]
    _rejects(pos, rows, q)


def test_rejects_a_missing_nearer_neighbour(cloud):
    pos, q, nbr, _ = cloud
    rows = nbr[:, :K].copy()
    rows[5] = np.concatenate([nbr[5, :2], nbr[5, 3:K + 1]])   # entry 2 dropped, the (K+1)-th appended
    _rejects(pos, rows, q)


def test_rejects_two_entries_out_of_order(cloud):
    pos, q, nbr, d2 = cloud
    rows = nbr[:, :K].copy()
    assert d2[7, 5] < d2[7, 6] * (1 - 1e-5)
    rows[7, [5, 6]] = rows[7, [6, 5]]
    _rejects(pos, rows, q)


def test_rejects_a_duplicate(cloud):
    pos, q, nbr, _ = cloud
    rows = nbr[:, :K].copy()
    rows[2, K - 1] = rows[2, K - 2]
    _rejects(pos, rows, q)


def test_rejects_an_exact_tie_in_the_wrong_order(lattice):
    pos, q, nbr, d2 = lattice
    rows = nbr[:, :19].copy()
    assert d2[0, 1] == d2[0, 2] and nbr[0, 1] < nbr[0, 2]
    rows[0, [1, 2]] = rows[0, [2, 1]]
    _rejects(pos, rows, q, 19)


def test_rejects_the_self_entry_left_out(cloud):
    pos, q, nbr, _ = cloud
    rows = nbr[:, 1:K + 1].copy()                          # every list shifted by one
    _rejects(pos, rows, q)


def test_density_tolerance_has_teeth(cloud):
    pos, q, nbr, d2 = cloud
    n = len(pos)
    dens = oracle.density(d2[:, :K], n)
    check_density(dens * (1 + 5e-6), d2[:, :K], n)
    check_density(dens * (1 - 5e-6), d2[:, :K], n)
    bad = dens.copy()
    bad[11] *= 1 + 2e-5
    with pytest.raises(AssertionError):
        check_density(bad, d2[:, :K], n)
    # h from the wrong neighbour (the (K-1)-th): far outside the tolerance
    with pytest.raises(AssertionError):
        check_density(oracle.density(d2[:, :K - 1], n), d2[:, :K], n)


def test_density_infinities_must_match():
    # three coincident particles and k = 3: every entry at distance 0
    pos = np.array([[0.5, 0.5, 0.5]] * 3 + [[0.1, 0.2, 0.3], [0.9, 0.8, 0.7]])
    nbr, d2 = oracle.knn(pos, 3)
    dens = oracle.density(d2, len(pos))
    assert np.isinf(dens[:3]).all() and np.isfinite(dens[3:]).all()
    check_density(dens, d2, len(pos))
    bad = dens.copy()
    bad[0] = 1e30
    with pytest.raises(AssertionError):
        check_density(bad, d2, len(pos))
