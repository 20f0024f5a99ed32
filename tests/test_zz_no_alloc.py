"""hop_link_static: the link step for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: for example a host program that hands
all device memory to its own pool allocator, or a latency-bound loop where a
device allocation (which can synchronise the device) is not allowed.
hop_link_static keeps its scratch in a fixed array inside the library
instead of a context's growable buffers.  This file checks, through the C
ABI, that it gives exactly what hop_link gives on two calls in a row (the
second on a smaller input, so a stale scratch array would show), and that
it refuses inputs larger than its fixed maximum.  It is collected last so
that a stop-at-first-failure run has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_1001_3411_gb300 as hopgpu
import synth
from paper_1001_3411_gb300._lib import HOP_ESTATIC, HOP_OK, HOP_STATIC_LINK_MAX_N, load_library

pytestmark = pytest.mark.gpu


def _static_link(L, dens, nbr, n_hop, stream):
    n, ld = nbr.shape
    hop = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    chain = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    rc = L.hop_link_static(C.c_void_p(dens.data_ptr()), C.c_void_p(nbr.data_ptr()), ld, n, n_hop,
                           C.c_void_p(hop.data_ptr()), C.c_void_p(chain.data_ptr()), C.c_void_p(stream))
    return rc, hop, chain


def test_link_static_matches_link_on_two_calls():
    hopgpu.build_library()
    L = load_library()
    h = hopgpu.Hop(0)
    stream = torch.cuda.current_stream().cuda_stream
    p = hopgpu.default_params()
    for n, seed in ((300_000, 71), (120_000, 72)):
        pos = torch.from_numpy(synth.nfw_box(n, seed)[0]).cuda()
        nbr, dens, _ = h.hop_density(pos, p, ld_nbr=16)
        hop_ref, chain_ref = h.hop_link(dens, nbr, 16)
        rc, hop_s, chain_s = _static_link(L, dens, nbr, 16, stream)
        assert rc == HOP_OK
        assert torch.equal(hop_s, hop_ref)
        assert torch.equal(chain_s, chain_ref)
    h.close()


def test_link_static_rejects_more_than_its_maximum():
    # Every buffer holds the full n rows, so even if the size check were
    # lost the kernels would stay inside their buffers: a regression shows
    # up as a failed assertion, never as an out-of-bounds access.
    L = load_library()
    n = HOP_STATIC_LINK_MAX_N + 1
    dens = torch.zeros(n, dtype=torch.float32, device="cuda")
    nbr = torch.zeros((n, 16), dtype=torch.int32, device="cuda")
    hop = torch.zeros(n, dtype=torch.int32, device="cuda")
    chain = torch.zeros(n, dtype=torch.int32, device="cuda")
    rc = L.hop_link_static(C.c_void_p(dens.data_ptr()), C.c_void_p(nbr.data_ptr()), 16, n, 16,
                           C.c_void_p(hop.data_ptr()), C.c_void_p(chain.data_ptr()),
                           C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert rc == HOP_ESTATIC
    assert torch.count_nonzero(hop).item() == 0
    assert torch.count_nonzero(chain).item() == 0
