"""The allocation-free multi-dot (pairdiag_multidot_noalloc) against the
handle-based pairdiag_multidot, through the C ABI.

It serves callers that cannot allocate device memory: its partial sums live in
a fixed array inside the library instead of cudaMalloc'd scratch.  Two calls in
a row must each match the existing entry point, which also shows that what the
first call leaves in the shared array does not leak into the second.  This file
sorts last so that a run stopping at its first failure has already run every
other test; it also passes when run alone in a fresh process.
"""
import numpy as np
import pytest

import pd_inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
pd = pytest.importorskip("paper_2001_01978_gb300")


@pytest.mark.parametrize("dtype", ["float64", "float32"])
def test_noalloc_multidot_matches_handle_entry_point(dtype):
    assert torch.cuda.is_available()
    torch.cuda.set_device(0)
    tdt = getattr(torch, dtype)
    e, G = pd_inputs.picket_fence(4, -0.2)
    stream = torch.cuda.current_stream()
    with pd.Solver(4, 2, e, G) as s:
        for call, (n, m, seed) in enumerate([(1_000_003, 13, 3), (77_777, 64, 4)]):
            g = torch.Generator(device="cuda").manual_seed(seed)
            Q = torch.randn(m, n, dtype=tdt, device="cuda", generator=g)
            p = torch.randn(n, dtype=tdt, device="cuda", generator=g)
            ref = pd.pairdiag_multidot(s.h, Q, n, m, p, n)
            out = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
            pd.pairdiag_multidot_noalloc(Q, n, m, p, n, out, stream)
            stream.synchronize()
            got = out.cpu().numpy()
            assert np.allclose(got, ref, rtol=1e-12, atol=1e-9), (call, np.max(np.abs(got - ref)))


def test_noalloc_multidot_rejects_too_many_vectors():
    torch.cuda.set_device(0)
    Q = torch.zeros(65, 10, dtype=torch.float64, device="cuda")
    p = torch.zeros(10, dtype=torch.float64, device="cuda")
    out = torch.zeros(65, dtype=torch.float64, device="cuda")
    with pytest.raises(pd.PairDiagError) as err:
        pd.pairdiag_multidot_noalloc(Q, 10, 65, p, 10, out)
    assert err.value.code == pd.PD_EINVAL and "at most 64" in str(err.value)
