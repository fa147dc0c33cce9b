"""CPU-side checks of the C ABI library: it loads, exports every symbol the header
declares, and its host-only index-set builder matches the oracle bit-exactly.
No GPU compute is called here."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2107_09006_gb300 as L
    return L


def test_every_declared_symbol_is_exported(lib):
    hdr = open(os.path.join(ROOT, "include", "ls_schwarz.h")).read()
    declared = set(re.findall(r"^\s*(?:const\s+char\*|void|ls_status)\s+(ls_\w+)\s*\(", hdr, re.M))
    assert declared, "no declarations parsed"
    import ctypes
    so = ctypes.CDLL(lib.LIBRARY_PATH)
    for name in declared:
        assert hasattr(so, name), name
    assert declared == set(lib.EXPORTED)


def test_default_options(lib):
    o = lib.ls_default_options()
    assert (o.nev_max, o.delta_rel, o.s_rel, o.maxit, o.coarse, o.use_graph) == (16, 1e-10, 1e-8, 1000, 1, 1)
    assert (o.variant, o.solver, o.restart, o.spmv, o.test_stall, o.block_kernel) == (0, 0, 100, 0, 0, 0)


@pytest.mark.parametrize("which", ["tiny", "ragged", "example"])
def test_host_index_sets_match_oracle(lib, which):
    import oracle as O
    from workloads import config_tiny, make_grid_ls, block_partition, paper_example, csr_from_dense
    if which == "tiny":
        P = config_tiny()
        m, n, rp, c, v, part, N = P.m, P.n, P.row_ptr, P.col, P.val, P.part, P.nparts
    elif which == "ragged":
        m, n, rp, c, v, _, _ = make_grid_ls(37, 29, 3, 6, 2, 4)
        part = block_partition(37, 29, 10, 7)
        N = int(part.max()) + 1
    else:
        A, part = paper_example()
        rp, c, v = csr_from_dense(A)
        m, n, N = 5, 4, 2
    om_off, om, nI, xi_off, xi = lib.ls_build_index_sets(m, n, rp, c, N, part)
    S = O.index_sets(O.schwarz.as_csr(m, n, rp, c, v), part, N)
    for i in range(N):
        assert np.array_equal(om[om_off[i]:om_off[i + 1]], S.Om[i])
        assert np.array_equal(xi[xi_off[i]:xi_off[i + 1]], S.Xi[i])
        assert nI[i] == len(S.OI[i])


def test_host_index_sets_reject_bad_input(lib):
    from workloads import config_tiny
    P = config_tiny()
    bad = P.col.copy()
    bad[0], bad[1] = bad[1], bad[0]
    with pytest.raises(lib.LSError) as e:
        lib.ls_build_index_sets(P.m, P.n, P.row_ptr, bad, P.nparts, P.part)
    assert e.value.status == lib.LS_ERR_INVALID
    with pytest.raises(lib.LSError):
        lib.ls_build_index_sets(P.m, P.n, P.row_ptr, P.col, P.nparts, np.full(P.n, -1, np.int32))


@pytest.mark.parametrize("struct", ["ls_options", "ls_info"])
def test_struct_layout_matches_header(lib, struct, tmp_path):
    """The ctypes mirrors of the header's structs have the C compiler's layout: size and
    the offset of every field (a field added to one side only would shift the rest)."""
    import ctypes
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cls = getattr(lib, struct)
    lines = [f'printf("%zu\\n", sizeof({struct}));']
    lines += [f'printf("%zu\\n", offsetof({struct}, {name}));' for name, _ in cls._fields_]
    src = tmp_path / "layout.c"
    src.write_text("#include <stddef.h>\n#include <stdio.h>\n#include \"ls_schwarz.h\"\nint main(void) {\n  "
                   + "\n  ".join(lines) + "\n  return 0;\n}\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    want = [ctypes.sizeof(cls)] + [getattr(cls, name).offset for name, _ in cls._fields_]
    assert got == want


def test_enum_values_match_header(lib, tmp_path):
    """Every status, precision and query constant of the binding has the value the C
    compiler gives the header's enumerator of the same name."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    hdr = open(os.path.join(ROOT, "include", "ls_schwarz.h")).read()
    names = sorted(set(re.findall(r"^\s*(LS_(?:OK|ERR_\w+|PREC_\w+|Q_\w+))\s*=", hdr, re.M)))
    assert len(names) >= 20
    src = tmp_path / "enums.c"
    src.write_text("#include <stdio.h>\n#include \"ls_schwarz.h\"\nint main(void) {\n"
                   + "".join(f'  printf("%d\\n", (int){n});\n' for n in names) + "  return 0;\n}\n")
    exe = tmp_path / "enums"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()]
    assert got == [getattr(lib, n) for n in names]


def test_noalloc_binding_rejects_bad_arguments(lib):
    """The allocation-free product's binding refuses, before any C call, what the C side
    would launch kernels on blindly: non-tensors, wrong dtypes, wrong lengths, and
    tensors that are not on the current CUDA device."""
    torch = pytest.importorskip("torch")
    m, n, nnz = 7, 4, 10
    good = dict(row_ptr=torch.zeros(m + 1, dtype=torch.int64), col=torch.zeros(nnz, dtype=torch.int32),
                val=torch.zeros(nnz, dtype=torch.float64), col_ptr=torch.zeros(n + 1, dtype=torch.int64),
                row=torch.zeros(nnz, dtype=torch.int32), cval=torch.zeros(nnz, dtype=torch.float64),
                p=torch.zeros(n, dtype=torch.float64), w=torch.zeros(n, dtype=torch.float64))
    order = ("row_ptr", "col", "val", "col_ptr", "row", "cval", "p", "w")

    def check(require_cuda=False, **over):
        a = dict(good, **over)
        lib._check_noalloc_args(m, n, nnz, *(a[k] for k in order), require_cuda=require_cuda)

    check()  # the host-side shape and dtype checks pass on well-formed arguments
    bad = {"row_ptr": torch.zeros(m + 1, dtype=torch.int32), "col": torch.zeros(nnz, dtype=torch.int64),
           "val": torch.zeros(nnz, dtype=torch.float32), "cval": torch.zeros(nnz + 1, dtype=torch.float64),
           "row": torch.zeros(nnz - 1, dtype=torch.int32), "col_ptr": torch.zeros(n, dtype=torch.int64),
           "p": torch.zeros(n + 1, dtype=torch.float64), "w": np.zeros(n)}
    for k, v in bad.items():
        with pytest.raises(ValueError, match=k):
            check(**{k: v})
    with pytest.raises(ValueError, match="row_ptr"):
        check(row_ptr=torch.zeros(2 * (m + 1), dtype=torch.int64)[::2])  # strided view
    with pytest.raises(ValueError, match="CUDA device"):
        check(require_cuda=True)  # host tensors
    with pytest.raises(ValueError):
        lib.ls_normal_product_noalloc(m, n, *(good[k] for k in order[:6]), nnz, good["p"], good["w"])


def test_bounds_checked_build_exports_the_same_symbols(lib):
    """The bounds-checked variant (-DLS_DEBUG_BOUNDS, libls_schwarz_dbg.so) builds and
    exports exactly the product library's symbols (its GPU behaviour is tested in
    test_gpu_debug_bounds.py)."""
    import ctypes
    import importlib.util
    spec = importlib.util.spec_from_file_location("_ls_build_t", os.path.join(ROOT, "paper_2107_09006_gb300",
                                                                              "_build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    path = mod.build(debug_bounds=True)
    assert os.path.basename(path) == "libls_schwarz_dbg.so"
    so = ctypes.CDLL(path)
    for name in lib.EXPORTED:
        assert hasattr(so, name), name
