"""The batched-GEMM configuration space (host logic only, no GPU): both
kernel families are present, descriptions are unique, every size in
[2, 32]^3 can run at least one configuration of each family, and the
validity rules the kernels rely on hold (a register tile never exceeds the
matrix, sizes out of range have no valid configuration)."""
import itertools
import re

from paper_1910_08498_gb300 import _lib as L


def _space():
    return [L.fr_gemm_describe_config(i) for i in range(L.fr_gemm_num_configs())]


def test_two_families_with_unique_descriptions():
    d = _space()
    assert len(d) == len(set(d)) == 144
    assert sum("bulk" in x for x in d) == 72


def test_every_size_has_a_configuration_of_each_family():
    d = _space()
    bulk = [i for i, x in enumerate(d) if "bulk" in x]
    coop = [i for i, x in enumerate(d) if "bulk" not in x]
    sizes = range(2, 33)
    for m, n, k in itertools.product(sizes, sizes, (2, 3, 16, 31, 32)):
        assert any(L.fr_gemm_config_valid(i, m, n, k) for i in bulk), (m, n, k)
        assert any(L.fr_gemm_config_valid(i, m, n, k) for i in coop), (m, n, k)


def test_register_tiles_fit_the_matrix_and_sizes_out_of_range_are_rejected():
    d = _space()
    for i, x in enumerate(d):
        mt = re.match(r"bgemm bulk ty=(\d) tx=(\d)", x)
        if mt:
            ty, tx = int(mt.group(1)), int(mt.group(2))
            if ty > 2:
                assert not L.fr_gemm_config_valid(i, 2, 8, 8)
            if tx > 2:
                assert not L.fr_gemm_config_valid(i, 8, 2, 8)
        for bad in [(1, 8, 8), (8, 33, 8), (8, 8, 0), (40, 40, 40)]:
            assert not L.fr_gemm_config_valid(i, *bad)
