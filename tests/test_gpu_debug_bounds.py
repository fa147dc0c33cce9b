"""The bounds-checked build gives the product build's answers.

libls_schwarz_dbg.so (-DLS_DEBUG_BOUNDS) checks every gather index, scatter index and
factor copy range in the local-solve, scatter and block local-solve kernels; an index out
of range would be reported as LS_ERR_INVALID instead of being used.  On valid inputs the
checks must change nothing: a child process that loads the checked build
(LS_SCHWARZ_BOUNDS=1) solves the same problems as this process with the product build,
through the single-vector path (FP64 and FP32 factors, the cluster-split FP32 local solve, and the row-tile normal product)
and both tensor-core kernels of the block path, and the iterates agree: to 1e-12 in FP64 and 1e-6 with FP32 factors (the
checks add no arithmetic, but the compiler may contract or order the FP32 sums of the
checked build differently).  A check that fired on a valid index would fail the child's
solve with LS_ERR_INVALID.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU containers
    pytest.skip("needs a GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import paper_2107_09006_gb300 as L
from workloads import config_tiny, make_grid_ls, block_partition
assert L.LIBRARY_PATH.endswith(LIBNAME), L.LIBRARY_PATH
P = config_tiny()
m, n, rp, c, v, b, _ = make_grid_ls(96, 96, 4, 8, 3, 0, nrhs=2)
part = block_partition(96, 96, 32, 32)
out = {}
for prec in ("f64", "f32"):
    S = L.Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, nev_max=16, factor_prec=prec, spmv=2,
                 fixed_iters=6)
    out["tiny-" + prec] = S.solve(P.b, rtol=1e-8)[0].cpu().numpy().tolist()
    S.close()
S = L.Solver(P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts, nev_max=16, factor_prec="f32", spmv=2,
             local_config=3, fixed_iters=6)
out["tiny-split-f32"] = S.solve(P.b, rtol=1e-8)[0].cpu().numpy().tolist()
S.close()
S = L.Solver(m, n, rp, c, v, part, 9, nev_max=16, normal_product=2, normal_kernel=4, fixed_iters=6)
out["tiles-f64"] = S.solve(b[0], rtol=1e-8)[0].cpu().numpy().tolist()
S.close()
for kernel in (1, 2):
    S = L.Solver(m, n, rp, c, v, part, 9, nev_max=16, factor_prec="f32", spmv=2, fixed_iters=3,
                 block_kernel=kernel)
    out["block-%d" % kernel] = S.solve(b, rtol=1e-8)[0].cpu().numpy().tolist()
    S.close()
print(json.dumps(out))
'''


def _run(libname, env):
    code = CHILD.replace("ROOT", repr(ROOT)).replace("LIBNAME", repr(libname))
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    assert p.returncode == 0, p.stderr[-3000:]
    return {k: np.array(v) for k, v in json.loads(p.stdout.strip().splitlines()[-1]).items()}


def test_bounds_checked_build_matches_product_build():
    import importlib.util
    spec = importlib.util.spec_from_file_location("_ls_build_g", os.path.join(ROOT, "paper_2107_09006_gb300",
                                                                              "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(debug_bounds=True)
    env = {k: v for k, v in os.environ.items() if k != "LS_SCHWARZ_BOUNDS"}
    prod = _run("libls_schwarz.so", env)
    dbg = _run("libls_schwarz_dbg.so", dict(env, LS_SCHWARZ_BOUNDS="1"))
    for k in prod:
        assert np.all(np.isfinite(dbg[k])), k
        tol = 1e-12 if k.endswith("f64") else 1e-6
        assert np.linalg.norm(dbg[k] - prod[k]) <= tol * np.linalg.norm(prod[k]), k
