"""Mutation tests of the oracle's pins.  Each case plants one plausible
mistake in a copy of ``oracle/hop_oracle.c`` (a dropped term, a wrong sign,
bound or index, a reversed order, a missing condition), compiles the copy
and runs the oracle's pin tests against it (``HOP_ORACLE_LIB``): at least one
pin must fail.  The network oracle ``oracle/mlp.py`` is mutated the same way,
in a copy of the package that the pin run imports instead.  The pins come from the paper and the mathematics (brute
force, closed forms, the worked examples), so a mistake that no pin catches
is a mistake the oracle could carry into every parity test."""
import concurrent.futures as cf
import os
import re
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "hop_oracle.c")
PINS = [os.path.join(ROOT, "tests", f) for f in
        ("test_oracle_pins.py", "test_oracle_halo.py", "test_oracle_subhalo.py")]

SLOW = "(poisson_closed_form or plummer)"

# (name, function the mistake sits in, text, replacement); every occurrence
# of the text inside that function is replaced.
MUTANTS = [
    # C1 knn
    ("min_image wraps at a whole box", "min_image", "dx > 0.5 * box", "dx > box"),
    ("min_image wraps negatives at a whole box", "min_image", "dx < -0.5 * box", "dx < -box"),
    ("d2 drops the z term", "orc_knn", "dx * dx + dy * dy + dz * dz", "dx * dx + dy * dy"),
    ("d2 uses dx twice", "orc_knn", "dy * dy + dz * dz", "dx * dx + dz * dz"),
    ("equal distances ordered by larger index", "knn_before", "ja < jb", "ja > jb"),
    ("insertion never reaches the first slot", "orc_knn", "while (t > 0 &&", "while (t > 1 &&"),
    # (Dropping the index from the list order is no mistake in effect: the
    # brute force visits j in ascending order and inserts stably, so equal
    # distances already come out by index.)
    # C2 density
    ("M4 cubic term sign", "m4_w", "+ 0.75 * q * q * q", "- 0.75 * q * q * q"),
    ("M4 quadratic coefficient", "m4_w", "1.0 - 1.5 * q * q", "1.0 - 1.0 * q * q"),
    ("M4 outer branch coefficient", "m4_w", "0.25 * t * t * t", "0.5 * t * t * t"),
    ("M4 support ends at q = 1.5", "m4_w", "if (q < 2.0)", "if (q < 1.5)"),
    ("smoothing length h = r_k", "orc_density", "double h = 0.5 * sqrt(row[k - 1]);", "double h = sqrt(row[k - 1]);"),
    ("normalised by n - 1", "orc_density", "/ (double)n_total", "/ (double)(n_total - 1)"),
    ("self excluded from the sum", "orc_density", "for (int32_t t = 0; t < k; ++t)", "for (int32_t t = 1; t < k; ++t)"),
    ("kernel normalisation h^2", "orc_density", "(M_PI * h * h * h)", "(M_PI * h * h)"),
    ("kernel normalisation without pi", "orc_density", "(M_PI * h * h * h)", "(h * h * h)"),
    ("kernel argument d^2 / h", "orc_density", "m4_w(sqrt(row[t]) / h)", "m4_w(row[t] / h)"),
    ("smoothing length from the (k-1)-th entry", "orc_density", "sqrt(row[k - 1])", "sqrt(row[k - 2])"),
    # C3, C4 link
    ("hop over Nhop - 1 entries", "orc_link", "t < n_hop; ++t", "t < n_hop - 1; ++t"),
    ("hop skips the particle itself", "orc_link", "int32_t best = row[0];", "int32_t best = row[1];"),
    ("equal densities hop to the larger index", "key_greater", "a < b", "a > b"),
    ("hop to the least dense", "key_greater", "dens[a] > dens[b]", "dens[a] < dens[b]"),
    ("chain label is the first hop", "orc_link", "chain[path[t]] = root;", "chain[path[t]] = hop[path[t]];"),
    # C5 boundaries
    ("neighbour's delta_outer test dropped", "orc_boundaries", " || !(dens[j] >= d_outer)", ""),
    ("particle's delta_outer test dropped", "orc_boundaries", "if (!(dens[i] >= d_outer)) continue;", ""),
    ("boundary value is the smaller density", "orc_boundaries", "raw[w].s = dens[i] + dens[j];",
     "raw[w].s = dens[i] < dens[j] ? dens[i] : dens[j];"),
    ("boundary keeps the smallest sum", "link_cmp", "return a->s > b->s ? -1 : 1;", "return a->s < b->s ? -1 : 1;"),
    ("boundaries over Nmerge - 1 entries", "orc_boundaries", "t < n_merge; ++t", "t < n_merge - 1; ++t"),
    ("boundaries keyed by particles", "orc_boundaries", "int32_t a = chain[i], b = chain[j];",
     "int32_t a = (int32_t)i, b = j;"),
    # C6, C7 merge
    ("proto-halo test strict", "orc_merge", "dens[peak[c]] >= d_peak", "dens[peak[c]] > d_peak"),
    ("proto-halo test on delta_saddle", "orc_merge", "dens[peak[c]] >= d_peak", "dens[peak[c]] >= d_saddle"),
    ("saddle test without the factor 2", "orc_merge", "s[e] >= 2.0 * d_saddle", "s[e] >= d_saddle"),
    ("saddle test strict", "orc_merge", "s[e] >= 2.0 * d_saddle", "s[e] > 2.0 * d_saddle"),
    ("owned sets unite through any boundary", "orc_merge", "if (a == b || (owned[a] && owned[b])) continue;",
     "if (a == b) continue;"),
    ("edges taken in ascending order", "edge_cmp", "return a->s > b->s ? -1 : 1;", "return a->s < b->s ? -1 : 1;"),
    ("equal edges ordered by hi first", "edge_cmp", "if (a->lo != b->lo) return a->lo < b->lo ? -1 : 1;", ""),
    ("chain peak is its first member", "orc_merge",
     "if (peak[c] < 0 || key_greater(dens, (int32_t)i, peak[c])) peak[c] = (int32_t)i;",
     "if (peak[c] < 0) peak[c] = (int32_t)i;"),
    ("delta_outer cut dropped", "orc_merge", "(dens[i] >= d_outer && owned[r])", "(owned[r])"),
    ("groups numbered by ascending peak", "peak_cmp", "return a->d > b->d ? -1 : 1;", "return a->d < b->d ? -1 : 1;"),
    # C8 halo statistics
    ("centre not wrapped below 0", "orc_halo_stats", "if (c < 0.0) c += box;", ""),
    ("centre not wrapped at the box", "orc_halo_stats", "if (c >= box) c -= box;", ""),
    ("offsets without the minimum image", "orc_halo_stats",
     "sum[3 * g + d] += min_image(pos[3 * i + d] - pos[3 * (int64_t)peak[g] + d], box);",
     "sum[3 * g + d] += pos[3 * i + d] - pos[3 * (int64_t)peak[g] + d];"),
    ("radius from the peak", "orc_halo_stats", "min_image(pos[3 * i + d] - com[3 * g + d], box)",
     "min_image(pos[3 * i + d] - pos[3 * (int64_t)peak[g] + d], box)"),
    ("halo peak is its first member", "orc_halo_stats",
     "if (peak[g] < 0 || key_greater(dens, (int32_t)i, peak[g])) peak[g] = (int32_t)i;",
     "if (peak[g] < 0) peak[g] = (int32_t)i;"),
    ("centre divided by count + 1", "orc_halo_stats", "/ (double)count[g]", "/ (double)(count[g] + 1)"),
    # C9 subhalos
    ("symmetric pairs emitted twice", "orc_sym_boundaries", "if (raw[t].a > raw[t].b) continue;", ""),
    ("one-way links kept", "orc_sym_boundaries", "if (l == d || raw[l].a != raw[t].b || raw[l].b != raw[t].a) continue;",
     "if (l < d && raw[l].a == raw[t].b && raw[l].b == raw[t].a) { }"),
    ("symmetric value from one direction", "orc_sym_boundaries",
     "s[u] = raw[t].s > raw[l].s ? raw[t].s : raw[l].s;", "s[u] = raw[t].s;"),
    ("subhalo links cut without the factor 2", "orc_subhalos", "s[e] >= 2.0 * ds", "s[e] >= ds"),
    ("subhalo members below the threshold", "orc_subhalos", "out[i] = dens[i] >= ds ?", "out[i] = dens[i] >= 0.0 ?"),
    ("Poisson noise 1/N", "orc_subhalos", "f_poisson / sqrt(N)", "f_poisson / N"),
    ("n_min ignored", "orc_subhalos", " || cnt[c] < n_min", ""),
]


# the same for oracle/mlp.py (function, text, replacement inside that def)
MLP_MUTANTS = [
    ("forward without the second ReLU", "forward", "h2 = np.maximum(h1 @ w2.T + b2, 0.0)", "h2 = h1 @ w2.T + b2"),
    ("forward without the output bias", "forward", "return h2 @ w3 + b3", "return h2 @ w3"),
    ("loss gradient without the factor 2", "loss_and_grad", "dy = 2.0 * r / m", "dy = r / m"),
    ("W2 gradient transposed", "loss_and_grad", "g_w2 = d2.T @ h1", "g_w2 = h1.T @ d2"),
    ("first-layer mask from the second", "loss_and_grad", "d1 = (d2 @ w2) * (a1 > 0)", "d1 = (d2 @ w2) * (a2 > 0)"),
    ("backprop through W2 untransposed", "loss_and_grad", "d1 = (d2 @ w2)", "d1 = (d2 @ w2.T)"),
    ("bf16 rounds ties up", "bf16_round", "(u + np.uint64(0x7FFF) + lsb)", "(u + np.uint64(0x8000))"),
    ("bf16 truncates", "bf16_round", "(u + np.uint64(0x7FFF) + lsb)", "(u)"),
]


def _function_span(src, name):
    m = re.search(r"^[A-Za-z][^\n;]*\b" + re.escape(name) + r"\([^;{]*\)\s*\{", src, re.M)
    assert m, name
    end = src.index("\n}\n", m.end())
    return m.start(), end


def _mutate(src, fn, old, new):
    a, b = _function_span(src, fn)
    body = src[a:b]
    assert old in body, (fn, old)
    return src[:a] + body.replace(old, new) + src[b:]


def _run(case, tmp):
    name, fn, old, new = case
    d = os.path.join(tmp, re.sub(r"\W+", "_", name))
    os.makedirs(d)
    c = os.path.join(d, "hop_oracle.c")
    open(c, "w").write(_mutate(open(SRC).read(), fn, old, new))
    so = os.path.join(d, "liboracle.so")
    cc = subprocess.run(["gcc", "-O2", "-fopenmp", "-std=c11", "-D_GNU_SOURCE", "-shared", "-fPIC", "-o", so, c, "-lm"],
                        capture_output=True, text=True)
    if cc.returncode != 0:
        return name, "does not compile: " + cc.stderr[-300:]
    env = dict(os.environ, HOP_ORACLE_LIB=so, OMP_NUM_THREADS="2", PYTHONDONTWRITEBYTECODE="1")
    out = ""
    # the quick pins first; the large brute-force cases only if they all pass
    for sel in ("not " + SLOW, SLOW):
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-k", sel, *PINS],
                           capture_output=True, text=True, cwd=ROOT, env=env, timeout=600)
        if r.returncode == 1 and " failed" in r.stdout:
            return name, None
        if r.returncode != 0:
            return name, f"pytest exit {r.returncode}: {r.stdout[-300:]}"
        out = r.stdout
    return name, "every pin passes: " + out[-200:]


def _mutate_py(src, fn, old, new):
    a = src.index("\ndef " + fn + "(")
    b = src.find("\ndef ", a + 1)
    b = len(src) if b < 0 else b
    body = src[a:b]
    assert old in body, (fn, old)
    return src[:a] + body.replace(old, new) + src[b:]


def _run_mlp(case, tmp):
    name, fn, old, new = case
    d = os.path.join(tmp, "py_" + re.sub(r"\W+", "_", name))
    pkg = os.path.join(d, "oracle")
    shutil.copytree(os.path.join(ROOT, "oracle"), pkg, ignore=shutil.ignore_patterns("_build", "__pycache__"))
    src = open(os.path.join(ROOT, "oracle", "mlp.py")).read()
    open(os.path.join(pkg, "mlp.py"), "w").write(_mutate_py(src, fn, old, new))
    # cwd first on sys.path: the copy is imported; ROOT on PYTHONPATH keeps
    # the test helpers importable without putting ROOT ahead of the copy
    env = dict(os.environ, PYTHONPATH=ROOT, PYTHONDONTWRITEBYTECODE="1")
    env.pop("HOP_ORACLE_LIB", None)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", "-k", "mlp or bf16",
                        "-c", os.devnull, "--rootdir", d, PINS[0]], capture_output=True, text=True, cwd=d, env=env,
                       timeout=600)
    if r.returncode == 1 and " failed" in r.stdout:
        return name, None
    return name, f"pytest exit {r.returncode}: {r.stdout[-300:]}"


def test_mutant_table_applies_to_the_oracle_source():
    src = open(SRC).read()
    for name, fn, old, new in MUTANTS:
        assert _mutate(src, fn, old, new) != src, name
    assert len({m[0] for m in MUTANTS}) == len(MUTANTS)
    src = open(os.path.join(ROOT, "oracle", "mlp.py")).read()
    for name, fn, old, new in MLP_MUTANTS:
        assert _mutate_py(src, fn, old, new) != src, name


def test_the_mutated_network_oracle_is_the_one_imported(tmp_path):
    """The copy the network mutants run against really replaces the package:
    a copy whose forward pass is broken fails the hand-computed pin, and an
    unchanged copy passes it."""
    name, why = _run_mlp(("identity", "forward", "return h2 @ w3 + b3", "return h2 @ w3 + b3"), str(tmp_path))
    assert why is not None and "exit 0" in why
    name, why = _run_mlp(MLP_MUTANTS[1], str(tmp_path))
    assert why is None


def test_every_planted_mistake_fails_a_pin(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("needs gcc")
    with cf.ThreadPoolExecutor(max_workers=max(2, min(8, (os.cpu_count() or 2) // 2))) as ex:
        results = list(ex.map(lambda m: _run(m, str(tmp_path)), MUTANTS))
        results += list(ex.map(lambda m: _run_mlp(m, str(tmp_path)), MLP_MUTANTS))
    survivors = [f"{name}: {why}" for name, why in results if why is not None]
    assert not survivors, "mistakes no pin catches:\n" + "\n".join(survivors)
