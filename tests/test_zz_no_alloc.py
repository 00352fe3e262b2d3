"""hanf_estimate_static, the allocation-free estimator, against the oracle.

Callers that cannot allocate device memory while they run (a serving loop
whose memory was reserved up front, or a process sharing the GPU with an
allocator that owns all of it) can compute N = sum_v size(c[v]) of a register
array they already hold with hanf_estimate_static, whose only scratch is a
fixed 8 MiB array inside the library.  The register arrays here are seeded
synthetic inputs; the expected values are the oracle's sums of the same
arrays.  Sizes cover a ragged last 64-node block, more than one first-level
reduction CTA (n > 262,144), several runs per row, a non-default stream and
two calls in a row sharing the fixed scratch.  This file sorts last so that,
if it fails, a run stopping at the first failure has already run every other
test; it needs no state from them.
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


def synthetic_registers(n, R, log2m, seed):
    """n rows of R*m registers: geometric values clamped to 31 (the law of
    HyperLogLog registers), every 9th counter of every run empty so that
    linear counting is taken, and some sparse counters."""
    m = 1 << log2m
    rng = np.random.default_rng(seed)
    c = np.minimum(rng.geometric(0.5, (n, R * m)) - 1, 31).astype(np.uint8)
    c[::9] = 0
    sparse = rng.random((n, R * m)) < 0.9
    sparse[1::2] = False
    c[sparse] = 0
    return c


@pytest.mark.parametrize("n,R,log2m,side_stream", [
    (300_001, 2, 6, False),      # ragged last block, 5 first-level reduction CTAs
    (1_000_003, 1, 6, True),     # 16 first-level CTAs, on a stream of its own
    (8_191, 4, 8, False),
    (64, 8, 4, False),
    (1, 1, 5, True),
])
def test_static_estimate_matches_oracle(H, oracle, n, R, log2m, side_stream):
    import torch
    m = 1 << log2m
    c = synthetic_registers(n, R, log2m, seed=n + R)
    expected = np.array([oracle.sum_sizes_mt(c[:, r * m:(r + 1) * m], threads=8)
                         for r in range(R)])
    regs = torch.from_numpy(c).cuda()
    stream = torch.cuda.Stream() if side_stream else torch.cuda.current_stream()
    for call in range(2):          # two calls in a row share the fixed scratch
        out = torch.full((R,), -1.0, dtype=torch.float64, device="cuda")
        with torch.cuda.stream(stream):
            H.estimate_static(regs, n, log2m, R, out, stream=stream)
        stream.synchronize()
        np.testing.assert_allclose(out.cpu().numpy(), expected, rtol=RTOL, atol=0,
                                   err_msg=f"call {call}")


def test_static_estimate_of_a_context_state(H, oracle):
    """The registers a context reaches after three passes: estimated from the
    caller's copy they give the oracle's N(3) of the same graph."""
    import torch
    off, tgt = G.web(1 << 13, seed=21)
    log2m, R = 6, 4
    with H.HyperANF(off, tgt, log2m, 0x5EED, runs=R) as h:
        for _ in range(3):
            h.iterate()
        rows = np.stack([h.registers(r) for r in range(R)], axis=1)   # n x R x m
    regs = torch.from_numpy(np.ascontiguousarray(rows).reshape(rows.shape[0], -1)).cuda()
    out = torch.zeros(R, dtype=torch.float64, device="cuda")
    H.estimate_static(regs, regs.shape[0], log2m, R, out)
    torch.cuda.synchronize()
    for r in range(R):
        c = oracle.init(off.size - 1, log2m, oracle.run_seed(0x5EED, r))
        for _ in range(3):
            c, _ = oracle.union_pass(off, tgt, c)
        np.testing.assert_allclose(out[r].item(), oracle.sum_sizes(c), rtol=RTOL, atol=0)


def test_static_estimate_register_above_31_gives_nan(H):
    import torch
    c = synthetic_registers(1000, 2, 6, seed=3)
    c[500, 64 + 7] = 32                       # run 1 only
    regs = torch.from_numpy(c).cuda()
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    H.estimate_static(regs, 1000, 6, 2, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.isfinite(got[0]) and np.isnan(got[1])


def test_static_estimate_rejects_bad_arguments(H):
    import torch
    out = torch.zeros(8, dtype=torch.float64, device="cuda")
    dummy = torch.zeros(64, dtype=torch.uint8, device="cuda")
    # 8 runs of 2^27 nodes need far more than the fixed 2^20 doubles; the
    # check happens on the host before any work is enqueued
    rc = H.lib().hanf_estimate_static(dummy.data_ptr(), 1 << 27, 6, 8, out.data_ptr(), None)
    assert rc == H.HANF_EINVAL
    assert b"8 MiB" in H.lib().hanf_last_error()
    # a row pointer off the 16-byte grid is refused on the host as well
    rc = H.lib().hanf_estimate_static(dummy.data_ptr() + 8, 1, 4, 1, out.data_ptr(), None)
    assert rc == H.HANF_EINVAL
    assert b"16-byte" in H.lib().hanf_last_error()
