"""hanf_estimate_static, the allocation-free estimator, against hanf_estimate.

Callers that cannot allocate device memory while they run (a serving loop
whose memory was reserved up front, or a process sharing the GPU with an
allocator that owns all of it) can compute N(t) of a register array they
already hold with hanf_estimate_static, whose only scratch is a fixed 8 MiB
array inside the library.  This file sorts last so that, if it fails, a run
stopping at the first failure has already run every other test; it needs no
state from them.
"""
import numpy as np
import pytest

from paper_1011_5599_gb300 import graphs as G

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module")
def H():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1011_5599_gb300 import build as B
    B.build()
    import paper_1011_5599_gb300.hanf as H
    return H


def device_registers(h, R):
    """The context's registers of every run, re-laid as the library's
    node-major rows of R*m bytes, in a CUDA tensor."""
    import torch
    rows = np.stack([h.registers(r) for r in range(R)], axis=1)   # n x R x m
    return torch.from_numpy(np.ascontiguousarray(rows).reshape(h.n, -1)).cuda()


@pytest.mark.parametrize("log2m,R,passes", [(6, 4, 3), (4, 1, 0), (8, 2, 5)])
def test_static_estimate_matches_context_estimate(H, log2m, R, passes):
    import torch
    off, tgt = G.web(1 << 13, seed=21)
    with H.HyperANF(off, tgt, log2m, 0x5EED, runs=R) as h:
        for _ in range(passes):
            h.iterate()
        expected = h.estimate()
        regs = device_registers(h, R)
    for call in range(2):          # two calls in a row share the fixed scratch
        out = torch.full((R,), -1.0, dtype=torch.float64, device="cuda")
        H.estimate_static(regs, regs.shape[0], log2m, R, out)
        torch.cuda.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), expected, rtol=RTOL, atol=0,
                                   err_msg=f"call {call}")


def test_static_estimate_rejects_sizes_beyond_its_scratch(H):
    import torch
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(H.HanfError) as e:
        # 8 runs of 2^27 nodes need far more than the fixed 2^20 doubles; the
        # check happens on the host before any work is enqueued
        H.lib()
        rc = H.lib().hanf_estimate_static(dummy.data_ptr(), 1 << 27, 6, 8, out.data_ptr(), None)
        H.check(rc)
    assert e.value.code == H.HANF_EINVAL
    assert "8 MiB" in str(e.value)
