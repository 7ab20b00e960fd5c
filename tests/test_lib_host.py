"""CPU checks of the C library: it loads and exports every entry point the
header declares, and its host-side structure (J2 numbering, operator
patterns, P2 / R2 transfers, Vanka block sets) equals the oracle's on small
2D and 3D problems.  No GPU is touched (fsi_setup_host_only)."""
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import assemble as oasm
from oracle import fsasm, mesh, transfer
from paper_1909_13201_gb300 import binding
from paper_1909_13201_gb300 import inputs as I

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "fsi.h")


@pytest.fixture(scope="module")
def lib():
    return binding.load_library(build_if_missing=True)


def test_library_exports_every_declared_symbol(lib):
    text = open(HEADER).read()
    declared = set(re.findall(r"^\s*(?:fsi_status|void|const char \*)\s*(fsi_\w+)\s*\(", text, re.M))
    assert {"fsi_setup_hierarchy", "fsi_setup_smoothers", "fsi_solve", "fsi_solve_batched",
            "fsi_adjoint"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(binding.EXPORTED)


CASES = [
    ("c0", lambda: I.make_config(0)),
    ("bulge32", lambda: I.make_channel_2d(32, 3, 3, 77, bulge=True)),
    ("band-thin", lambda: I.make_channel_2d(16, 3, 2, 5, band_width=0.1)),
    ("valve3d", lambda: I.make_valve_3d(8, 2, 1, 9)),
]


@pytest.mark.parametrize("name,mk", CASES)
def test_host_structure_matches_oracle(lib, name, mk):
    p = mk()
    s = binding.FSISolver(p, host_only=True)
    levs = mesh.build_levels(p)
    for l, lev in enumerate(levs):
        f, c, nd = s.dof_map(l)
        np.testing.assert_array_equal(f, lev.dof_field)
        np.testing.assert_array_equal(c, lev.dof_comp)
        np.testing.assert_array_equal(nd, lev.dof_node)
        sz = s.sizes(l)
        np.testing.assert_array_equal(sz["offsets"], lev.group_offsets)
        # operator pattern: covers every oracle nonzero, nothing in fixed rows/columns
        ptr, col = s.pattern(l)
        Pat = sp.csr_matrix((np.ones(col.size), col, ptr), shape=(lev.n_dofs, lev.n_dofs))
        A = oasm.assemble(p, lev)
        A.eliminate_zeros()
        Ac = A.tocoo()
        assert np.all(Pat[Ac.row, Ac.col] == 1)
        Pc = Pat.tocoo()
        off = Pc.row != Pc.col
        assert not lev.fixed[Pc.row[off]].any() and not lev.fixed[Pc.col[off]].any()
        if l >= 1:
            P = transfer.prolongation(lev, levs[l - 1])
            R = transfer.restriction(P, lev, levs[l - 1])
            for which, M in ((0, P), (1, R)):
                ptr, col, val = s.transfer(l, which)
                L = sp.csr_matrix((val, col, ptr), shape=M.shape)
                assert abs(L - M).max() == 0.0, (name, l, which)
            bp, idx = s.blocks(l)
            ob = fsasm.block_index_sets(lev, p.patch)
            assert len(ob) == bp.size - 1
            for j, o in enumerate(ob):
                np.testing.assert_array_equal(idx[bp[j]:bp[j + 1]], o)


def test_host_only_rejects_device_calls(lib):
    p = I.make_config(0)
    s = binding.FSISolver(p, host_only=True)
    with pytest.raises(binding.FSIError) as e:
        s.setup_smoothers()
    assert e.value.status == binding.FSI_ERR_STATE


def test_bad_arguments_return_status(lib):
    p = I.make_channel_2d(12, 3, 1, 1)      # 12 not divisible by 2^(3-1)? it is; use 10
    p.n_fine = 10
    p.material = np.zeros(100, np.uint8)
    p.advection = np.zeros((2, 21 * 21))
    with pytest.raises(binding.FSIError) as e:
        binding.FSISolver(p, host_only=True)
    assert e.value.status == binding.FSI_ERR_ARG
    assert "divisible" in str(e.value)


SWEEP_CASES = [
    ("b1", lambda: I.make_channel_2d(16, 3, 1, 3), 1),
    ("b2-bulge", lambda: I.make_channel_2d(16, 3, 2, 3, bulge=True), 2),
    ("b3", lambda: I.make_channel_2d(24, 3, 3, 5), 3),
    ("b4-bulge", lambda: I.make_channel_2d(32, 3, 4, 7, bulge=True), 4),
    ("valve3d-b1", lambda: I.make_valve_3d(4, 2, 1, 9), 1),
    ("valve3d-b2", lambda: I.make_valve_3d(4, 2, 2, 9), 2),
]


@pytest.mark.parametrize("name,mk,b", SWEEP_CASES)
def test_sweep_passes_match_oracle(lib, name, mk, b):
    """The library's pass of every field-split block (kind and colour of its
    pressure group, the order of the locally multiplicative sweep) equals the
    oracle's on every level, 2D and 3D, b = 1..4."""
    p = mk()
    s = binding.FSISolver(p, host_only=True, patch=b)
    levs = mesh.build_levels(p)
    for l in range(1, len(levs)):
        lev = levs[l]
        tagged = fsasm.blocks_tagged(lev, b)
        col = fsasm.group_colours(lev, b)
        nc = fsasm.colour_period(b) ** lev.dim
        ref = np.array([kind * nc + col[g] for g, kind, _ in tagged], np.int32)
        got = s.block_passes(l)
        np.testing.assert_array_equal(got, ref, err_msg=f"{name} level {l}")
        ptr, idx = s.blocks(l)
        assert len(ptr) - 1 == len(tagged)
