"""tpf_solve_fp64_noalloc, the solve for callers that cannot allocate device memory.

Some callers get all of their device memory from their own pool and may not call cudaMalloc or
cudaFree (or have a library do it): their memory accounting would break, and those calls can
synchronise the device or block for an unbounded time.  tpf_solve_fp64_noalloc serves them: the
caller passes K, W, S, V and the iteration counts, and the solve's scratch lives in a fixed array
inside libtpf.so.  This file checks, through the C ABI, that it returns what the allocating FP64
path (tpf_solve with TPF_PREC_FP64) returns, within the FP64 tolerance of the other GPU tests, on
two calls in a row (the second call must not see stale state left in the shared array), and that
an oversized request is refused before any device work.  It is collected last so that a failure
here leaves every other test already run.
"""
import numpy as np
import pytest

from paper_2403_04578_gb300 import inputs as G
from paper_2403_04578_gb300 import tpf

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-9  # max |V - V_ref| in pu, as in tests/test_gpu_parity.py


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_the_allocating_fp64_solve_twice(cuda):
    import torch

    f = G.make_feeder(34, 1)
    K, W = tpf.precompute_host(f.n_bus, f.from_bus, f.to_bus, f.z_pu)
    Kd, Wd = _dev(K), _dev(W)
    ref = tpf.Feeder.from_inputs(f)
    # Two different load sets back to back: the second call runs on the array the first one used.
    for seed, T in ((1, 1440), (2, 700)):
        S = _dev(G.load_tensor(f, T, seed))
        V = torch.empty_like(S)
        it = torch.empty(T, dtype=torch.int32, device=S.device)
        st = tpf.solve_fp64_noalloc(Kd, Wd, S, V, it, tol=1e-10)
        torch.cuda.synchronize()
        assert st == tpf.OK, tpf.strerror(st)
        Vr, itr, _, str_ = ref.solve(S, precision="fp64", tol=1e-10)
        assert str_ == tpf.OK
        assert float((V - Vr).abs().max()) <= TOL_FP64
        assert torch.equal(it, itr)
    ref.close()


def test_noalloc_given_start_and_no_iteration_output(cuda):
    """given_start reads V as V_0: from the converged V every column stops after one sweep; and
    with no iteration-count tensor (a NULL pointer in the C ABI) V still matches the FP64 path."""
    import torch

    f = G.make_feeder(34, 1)
    K, W = tpf.precompute_host(f.n_bus, f.from_bus, f.to_bus, f.z_pu)
    Kd, Wd = _dev(K), _dev(W)
    S = _dev(G.load_tensor(f, 500, 3))
    ref = tpf.Feeder.from_inputs(f)
    Vr, _, _, st = ref.solve(S, precision="fp64", tol=1e-10)
    assert st == tpf.OK
    V = Vr.clone()
    it = torch.empty(S.shape[0], dtype=torch.int32, device=S.device)
    st = tpf.solve_fp64_noalloc(Kd, Wd, S, V, it, tol=1e-10, given_start=True)
    torch.cuda.synchronize()
    assert st == tpf.OK, tpf.strerror(st)
    assert bool((it == 1).all())
    assert float((V - Vr).abs().max()) <= 1e-10  # one more sweep moves V by less than tol
    V2 = torch.empty_like(S)
    st = tpf.solve_fp64_noalloc(Kd, Wd, S, V2, None, tol=1e-10)
    torch.cuda.synchronize()
    assert st == tpf.OK, tpf.strerror(st)
    assert float((V2 - Vr).abs().max()) <= TOL_FP64
    ref.close()


def test_noalloc_refuses_requests_beyond_its_array(cuda):
    import torch

    n = 999
    T = (tpf.NOALLOC_SCRATCH_BYTES // (16 * (n + 1))) + 256  # needs more than the 64 MiB array
    K = torch.zeros((n, n), dtype=torch.complex128, device="cuda")
    W = torch.zeros(n, dtype=torch.complex128, device="cuda")
    S = torch.zeros((1, n), dtype=torch.complex128, device="cuda")  # never read: refused first
    st = tpf.lib().tpf_solve_fp64_noalloc(n, K.data_ptr(), W.data_ptr(), T, S.data_ptr(), S.data_ptr(), None,
                                          1e-10, 100, 0, None)
    assert st == tpf.EINVAL
