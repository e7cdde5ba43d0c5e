"""The C-ABI library loads and exports every entry point include/pamc.h
declares, and rejects malformed instances on the host before any CUDA call
(no GPU needed)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2606_25203_gb300 as pg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            src = open(os.path.join(inc, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(pamc_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return pg.load(torch_allocator=False)


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for nm in names:
        assert hasattr(lib, nm), nm


def _create(lib, rp, col, w):
    h = ctypes.c_void_p()
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int32)
    rc = lib.pamc_create_csr(len(rp) - 1, rp.ctypes.data_as(ctypes.c_void_p),
                             col.ctypes.data_as(ctypes.c_void_p), w.ctypes.data_as(ctypes.c_void_p),
                             0, None, ctypes.byref(h))
    return rc, h


def test_host_validation_errors(lib):
    # asymmetric weight
    assert _create(lib, [0, 1, 2], [1, 0], [1, 2])[0] == 2
    # missing reverse edge
    assert _create(lib, [0, 1, 1], [1], [1])[0] == 2
    # self loop
    assert _create(lib, [0, 1], [0], [1])[0] == 3
    # weight out of range
    assert _create(lib, [0, 1, 2], [1, 0], [200, 200])[0] == 4
    # field range beyond the widest lanes
    # (a vertex with 299 couplings of 127: 37,973 > 32,767, the widest lanes)
    n = 300
    ei = np.zeros(n - 1, dtype=np.int64)
    ej = np.arange(1, n)
    import workloads as W
    star = W.csr_from_edges(n, ei, ej, np.full(n - 1, 127, dtype=np.int64), "star")
    assert _create(lib, star.row_ptr, star.col, star.w)[0] == 4
    # bad row_ptr
    assert _create(lib, [1, 1], [], [])[0] == 1
    assert _create(lib, [0, 2, 1], [1, 0], [1, 1])[0] == 1
    # column out of range
    assert _create(lib, [0, 1, 2], [5, 0], [1, 1])[0] == 1
    buf = ctypes.create_string_buffer(256)
    lib.pamc_last_error(None, buf, 256)
    assert b"column" in buf.value


def test_null_arguments(lib):
    assert lib.pamc_create_csr(4, None, None, None, 0, None, None) == 1
    assert lib.pamc_init(None, None) == 1
    assert lib.pamc_step(None, 1) == 1
    assert lib.pamc_launch_count(None) == 0


def test_params_layout_matches_header(tmp_path):
    """The Python mirror of pamc_params has the C layout (size and every
    field offset), checked against a program compiled from include/pamc.h."""
    fields = [f[0] for f in pg.Params._fields_]
    prog = ["#include <stddef.h>", "#include <stdio.h>", '#include "pamc.h"', "int main(void) {",
            '  printf("%zu\\n", sizeof(pamc_params));']
    prog += [f'  printf("%zu\\n", offsetof(pamc_params, {f}));' for f in fields]
    prog += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(prog) + "\n")
    exe = tmp_path / "layout"
    import subprocess
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    out = [int(x) for x in subprocess.check_output([str(exe)]).split()]
    assert out[0] == ctypes.sizeof(pg.Params)
    for f, off in zip(fields, out[1:]):
        assert getattr(pg.Params, f).offset == off, f


def test_binding_checks_array_lengths():
    """The binding refuses arrays shorter than what the library would read
    (n + 1 row pointers, row_ptr[n] couplings, an n x n matrix) before any
    pointer reaches it."""
    with pytest.raises(ValueError, match="n \\+ 1"):
        pg.pamc_create_csr(3, [0, 1, 2], [1, 0], [1, 1])
    with pytest.raises(ValueError, match="row_ptr\\[n\\]"):
        pg.pamc_create_csr(2, [0, 1, 2], [1], [1, 1])
    with pytest.raises(ValueError, match="n x n"):
        pg.pamc_create_dense(3, np.zeros((3, 2), dtype=np.int8))


def test_binding_checks_sizes_against_the_handle():
    """Buffers sized from a caller's n or R that differ from the handle's are
    refused before the library writes into them (a registered stand-in
    handle; only the refusals run, so no device call is made)."""
    h = ctypes.c_void_p(0x1234)
    pg._dims[h.value] = [10, None]
    try:
        pg._dims_check(h, n=10, R=7)          # R unknown before init: only n is checked
        pg._set_R(h, 4)                        # what pamc_init / pamc_run record
        assert pg._dims[h.value] == [10, 4]
        pg._dims_check(h, n=10, R=4)
        with pytest.raises(ValueError, match="n = 11"):
            pg.pamc_best(h, 11)
        with pytest.raises(ValueError, match="R = 5"):
            pg.pamc_state(h, 5, 10)
        with pytest.raises(ValueError, match="n = 9"):
            pg.pamc_fields(h, 4, 9)
        with pytest.raises(ValueError, match="n = 12"):
            pg.pamc_hamming(h, 12)
        with pytest.raises(ValueError, match="R = 3"):
            pg.pamc_lineage(h, 3)
        with pytest.raises(ValueError, match="R x n"):
            pg.pamc_set_population(h, np.ones((4, 9), dtype=np.int8))
    finally:
        pg._dims.pop(h.value, None)


def test_binding_noalloc_limits_match_header():
    src = open(os.path.join(ROOT, "include", "pamc.h")).read()
    for name, val in (("N", pg.NOALLOC_MAX_N), ("NNZ", pg.NOALLOC_MAX_NNZ),
                      ("SWEEPS", pg.NOALLOC_MAX_SWEEPS), ("R", pg.NOALLOC_MAX_R)):
        m = re.search(rf"#define PAMC_NOALLOC_MAX_{name} (\d+)", src)
        assert m and int(m.group(1)) == val, name
