"""A device wait that runs out is reported, not hung on.

Every wait of the local-solve kernel on a bulk copy is bounded (about two seconds of
clock cycles); when it gives up, the kernel sets the error slot of the device CG state,
skips the rest of its work and returns with no copy in flight, and the host turns the
slot into LS_ERR_DEVICE_TIMEOUT.  The option `test_stall` makes the kernel issue none of
its copies, so every wait runs out: the solve must fail with that status within a few
seconds, and the CUDA context must stay usable (a handle without the hook then solves
to 1e-10 against the oracle).  The same holds for both block (multi right-hand-side)
local-solve kernels.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2107_09006_gb300 as L  # noqa: E402
import oracle as O  # noqa: E402
from workloads import config_tiny  # noqa: E402


@pytest.mark.parametrize("prec,config", [("f64", 1), ("f64", 2), ("f32", 2), ("f32", 3)])
def test_bounded_wait_reports_timeout_and_context_survives(prec, config):
    """Every local-solve configuration (option local_config) takes the error path; in
    the split configuration both CTAs of a cluster give up and meet at the cluster
    barrier before leaving."""
    P = config_tiny()
    S = L.Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, nev_max=16, test_stall=1, factor_prec=prec,
                 local_config=config)
    t0 = time.time()
    with pytest.raises(L.LSError) as ex:
        S.solve(P.b, rtol=1e-8)
    elapsed = time.time() - t0
    assert ex.value.status == L.LS_ERR_DEVICE_TIMEOUT
    assert elapsed < 60.0, elapsed
    S.close()
    torch.cuda.synchronize()
    S2 = L.Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, nev_max=16)
    x, info = S2.solve(P.b, rtol=1e-10)
    assert info["relres_true"] <= 1e-10
    A = O.schwarz.as_csr(P.m, P.n, P.row_ptr, P.col, P.val)
    xo, _ = O.pcg(A, P.b, O.build_two_level(A, P.part, P.nparts, tau=0.0, nev_max=16).apply, rtol=1e-12)
    assert np.linalg.norm(x.cpu().numpy() - xo) <= 1e-8 * np.linalg.norm(xo)
    S2.close()


@pytest.mark.parametrize("prec,kernel", [("f32", 1), ("f32", 2), ("f64", 0)])
def test_block_path_bounded_wait_reports_timeout(prec, kernel):
    """The same on the multi right-hand-side path: the two tensor-core kernels (FP32
    factors: TF32 mma.sync, and tcgen05 whose copy, MMA and compute roles all give up
    together) and the CUDA-core kernel (FP64 factors)."""
    P = config_tiny()
    B = np.stack([P.b, np.random.default_rng(3).standard_normal(P.m)])
    S = L.Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, nev_max=16, factor_prec=prec, test_stall=1,
                 block_kernel=kernel)
    t0 = time.time()
    with pytest.raises(L.LSError) as ex:
        S.solve(B, rtol=1e-8)
    assert ex.value.status == L.LS_ERR_DEVICE_TIMEOUT
    assert time.time() - t0 < 60.0
    S.close()
    torch.cuda.synchronize()
    S2 = L.Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, nev_max=16, factor_prec=prec,
                  block_kernel=kernel)
    X, _ = S2.solve(B, rtol=1e-10)
    its, rel = S2.batch_stats(2)
    assert (rel <= 1e-10).all()
    S2.close()


def test_bad_hook_value_rejected():
    P = config_tiny()
    with pytest.raises(L.LSError) as ex:
        L.Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, nev_max=16, test_stall=2)
    assert ex.value.status == L.LS_ERR_INVALID
