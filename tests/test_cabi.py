"""The C-ABI library builds for sm_103a, loads without a GPU, and exports
every entry point include/hop.h declares; the binding mirrors the header."""
import ctypes
import os
import re

import paper_1001_3411_gb300 as hopgpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hop.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|void|const char \*)\s*(hop_\w+)\s*\(", src, re.M)))


def test_library_exports_every_declared_symbol():
    hopgpu.build_library()
    lib = ctypes.CDLL(hopgpu.LIB)
    names = _declared()
    assert len(names) >= 18
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(hopgpu.EXPORTS) == names


def test_header_constants_match_binding():
    src = open(os.path.join(ROOT, "include", "hop.h")).read()
    assert "#define HOP_MLP_NPARAM (64 * 27 + 64 + 64 * 64 + 64 + 64 + 1)" in src
    assert hopgpu.MLP_NPARAM == 64 * 27 + 64 + 64 * 64 + 64 + 64 + 1
    for name, val in [("HOP_OK", 0), ("HOP_EINVAL", 1), ("HOP_ETABLE", 4), ("HOP_ETIMEOUT", 5),
                      ("HOP_ENOMODEL", 7), ("HOP_RADIUS_LEARNED", 2)]:
        assert re.search(rf"{name} = {val}\b", src), name


def test_default_params_without_gpu():
    p = hopgpu.default_params()
    assert (p.n_dens, p.n_hop, p.n_merge) == (64, 16, 4)
    assert (p.delta_outer, p.delta_saddle, p.delta_peak) == (80.0, 200.0, 240.0)
    assert p.box == 1.0 and p.radius_mode == hopgpu.HOP_RADIUS_PLAIN
    q = hopgpu.default_params(n_dens=65, n_hop=65, radius_mode=hopgpu.HOP_RADIUS_COUNT)
    assert (q.n_dens, q.n_hop, q.radius_mode) == (65, 65, 1)
