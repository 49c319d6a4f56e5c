"""The C-ABI library without a GPU: it loads, exports every function that
include/lbm_capi.h declares, was compiled with the textbook D3Q19 table (the
same table as the oracle, which is written separately), and every address its
launches form stays inside its buffers (checked by walking all threads on the
CPU with the kernels' own index helpers)."""
import os
import re

import numpy as np
import pytest

import oracle
from oracle_pins import load_golden_table
from paper_1112_0850_gb300 import build, capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm_capi.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return capi.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_\w+)\s*\(", text)))


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("lbm_create", "lbm_init_equilibrium", "lbm_step", "lbm_macros", "lbm_reduce",
                     "lbm_adjoint_seed", "lbm_adjoint_step", "lbm_adjoint_init_grad", "lbm_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
        assert name in capi.PROTOTYPES, name


def test_compiled_table_matches_textbook_and_oracle(lib, golden_dir):
    from paper_1112_0850_gb300.lattice import lattice_table
    e, w, opp = lattice_table()
    ge, gw = load_golden_table(os.path.join(golden_dir, "d3q19_lattice.txt"))
    assert [tuple(r) for r in e.tolist()] == ge
    assert all(w[i] == float(gw[i]) for i in range(19))
    oe, ow, oopp = oracle.lattice()
    assert np.array_equal(e, oe) and np.array_equal(w, ow) and np.array_equal(opp, oopp)


SIZES = [(1, 1, 1), (1, 3, 2), (3, 1, 1), (2, 2, 2), (5, 4, 3), (8, 6, 5), (31, 3, 2), (32, 2, 2), (33, 7, 5),
         (64, 3, 3), (65, 2, 3), (100, 5, 2), (256, 2, 2), (257, 3, 2), (300, 2, 1), (513, 1, 2)]


@pytest.mark.parametrize("align", ["default", "128"])
@pytest.mark.parametrize("fmt", [0, 1, 2, 3, 4, 5])
@pytest.mark.parametrize("size", SIZES, ids=lambda s: "x".join(map(str, s)))
def test_launch_indices_in_bounds(lib, size, fmt, align):
    nx, ny, nz = size
    row_align = 0 if align == "default" else 128  # default: rows padded to pairs only
    assert lib.lbm_check_launch_indices(nx, ny, nz, fmt, row_align) == 0


def test_launch_index_check_rejects_bad_sizes(lib):
    assert lib.lbm_check_launch_indices(0, 4, 4, 1, 0) == -1
    assert lib.lbm_check_launch_indices(4, 4, 70000, 1, 0) == -1
    assert lib.lbm_check_launch_indices(4, 4, 4, 9, 0) == -1
    assert lib.lbm_check_launch_indices(4, 4, 4, 1, 4) == -1  # narrower than a pair of floats
    assert lib.lbm_check_launch_indices(4, 4, 4, 1, 24) == -1  # not a power of two


def test_status_strings(lib):
    assert capi.status_string(0) == "LBM_OK"
    assert capi.status_string(5) == "LBM_ERR_DIVERGED"
