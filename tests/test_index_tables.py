"""The kernels' index tables, checked on the host without a GPU (wf_check_tables): for every
lattice shape, source count and traversal tile height the library can use, the neighbour tables
are symmetric and in range, the traversal order visits every (source, line) pair exactly once, and
the bulk-fed kernels' units cover every (source group, line) pair once. The same checks run inside
the library whenever it builds a table; planted corruptions show that they catch errors."""

import pytest

import paper_0910_0992_gb300 as wf


def _divisors(L):
    return [b for b in range(1, L + 1) if L % b == 0 and b <= 12]


@pytest.mark.parametrize("L", [2, 4, 6, 8, 10, 12, 16, 24])
def test_tables_valid_for_every_layout(L):
    for T in (2, 3, 7, 16, 24, 33, 48, 64, 96, 100, 128, 129, 160, 200, 256):
        if L >= 16 and T not in (16, 64, 128, 256):
            continue  # the large lattices at a few line lengths keep the test quick
        for nrhs in (1, 3, 12):
            for rows in [0] + _divisors(L):
                assert wf.wf_check_tables(L, T, nrhs, rows) == wf.WF_OK, (L, T, nrhs, rows)


@pytest.mark.parametrize("plant", [1, 2, 3])
def test_checks_catch_planted_corruption(plant):
    for L, T, nrhs in ((4, 16, 3), (6, 48, 2), (8, 128, 12)):
        assert wf.wf_check_tables(L, T, nrhs, 0, plant) == wf.WF_ECUDA, (plant, L, T)


def test_invalid_arguments():
    assert wf.wf_check_tables(6, 16, 2, 4) == wf.WF_EINVAL   # 4 rows do not tile L = 6
    assert wf.wf_check_tables(4, 16, 0, 0) == wf.WF_EINVAL   # no sources
    assert wf.wf_check_tables(5, 16, 1, 0) == wf.WF_EINVAL   # odd L
    assert wf.wf_check_tables(4, 16, wf.WF_MAX_SOLVE_RHS + 1, 0) == wf.WF_EINVAL
    assert wf.wf_check_tables(4, 257, 1, 0) == wf.WF_EINVAL  # longer than 32 lanes x 8 sites
