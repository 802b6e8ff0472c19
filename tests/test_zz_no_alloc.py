"""The allocation-free synthesis entry point (for callers that cannot allocate device memory while
they run, e.g. under a host framework's fixed device-memory budget or in a pipeline where
cudaMalloc would synchronise the device) must give the same result as bie_synthesize.  Two calls
in a row check that the shared scratch array is rewritten correctly; this file is collected last
so a failure here comes after every other test has run."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import __graft_entry__ as g
    g.build()
    from paper_1706_07919_gb300 import binding
    return binding


def _case(Nt, M, P, midx, seed):
    rng = np.random.default_rng(seed)
    T = rng.standard_normal((len(midx), M)) + 1j * rng.standard_normal((len(midx), M))
    S = rng.standard_normal((P, Nt // 2 + 1)) + 1j * rng.standard_normal((P, Nt // 2 + 1))
    return torch.tensor(T, device="cuda"), torch.tensor(S, device="cuda")


@pytest.mark.parametrize("out_dtype,tol", [(0, 1e-12), (1, 1e-5)])
def test_noalloc_matches_synthesize_on_two_calls(B, out_dtype, tol):
    from paper_1706_07919_gb300 import Solver

    sol = Solver(0)
    stream = torch.cuda.current_stream().cuda_stream
    dt = torch.float64 if out_dtype == 0 else torch.float32
    cases = [(256, 37, 2, np.array([0, 1, 5, 64, 127, 128]), 1), (1024, 19, 1, np.arange(1, 513), 2)]
    for Nt, M, P, midx, seed in cases:  # two different calls in a row on the shared scratch
        T, S = _case(Nt, M, P, midx, seed)
        ref = sol.synthesize(T, midx, S, Nt, dt)
        got = torch.empty_like(ref)
        B.bie_synthesize_noalloc(T, midx, S, Nt, got, out_dtype, stream)
        torch.cuda.synchronize()
        err = (got - ref).abs().max().item() / ref.abs().max().item()
        assert err <= tol, (Nt, err)
    sol.close()


def test_noalloc_rejects_oversized_requests(B):
    T = torch.zeros((1, 4), dtype=torch.complex128, device="cuda")
    S = torch.zeros((1, 4097), dtype=torch.complex128, device="cuda")
    out = torch.zeros((1, 4, 8192), dtype=torch.float64, device="cuda")
    with pytest.raises(B.BieError) as e:
        B.bie_synthesize_noalloc(T, np.array([1]), S, 8192, out, 0, None)
    assert e.value.code == B.BIE_ERR_INVALID_ARG and "Nt" in str(e.value)
