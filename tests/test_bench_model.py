"""The bench's operation model of the cluster moves (host logic, no GPU).

icm_ops counts, per ICM pair visited, 3N (overlap, count, step 2a); per moved
pair, one Philox call (98), the rank search, the flip of both copies and the
energy update (3N + N_b); and the growth either per scan of the bit-parallel
flood fill (one word per 16 pairs and site, z + 2 operations) or, for
union-find, per moved pair (2N + N_b: label reset, one union per bond, one
root lookup per site).
"""
import pytest

bench = pytest.importorskip("bench")


def test_icm_ops_terms():
    N, Nb, z = 512, 1536, 6
    assert bench.icm_ops(N, Nb, z, 17, pairs=1, moves=0, scans=0) == 3 * N
    assert bench.icm_ops(N, Nb, z, 17, pairs=0, moves=1, scans=0) == 98 + 3 * N + Nb
    # 17 pairs need two 32-bit words per site (16 pairs per word)
    assert bench.icm_ops(N, Nb, z, 17, pairs=0, moves=0, scans=1) == 2 * N * (z + 2)
    assert bench.icm_ops(N, Nb, z, 16, pairs=0, moves=0, scans=1) == N * (z + 2)


def test_icm_ops_union_find_ignores_scans():
    N, Nb, z = 16384, 32768, 4
    flood = bench.icm_ops(N, Nb, z, 25, pairs=0, moves=10, scans=7)
    uf = bench.icm_ops(N, Nb, z, 25, pairs=0, moves=10, scans=7, union_find=True)
    assert flood == 10 * (98 + 3 * N + Nb) + 7 * 2 * N * (z + 2)
    assert uf == 10 * (98 + 3 * N + Nb) + 10 * (2 * N + Nb)
    assert bench.icm_ops(N, Nb, z, 25, 0, 10, 0, True) == uf


def test_workloads_name_their_sizes():
    for name, wl in bench.WORKLOADS.items():
        assert f"L={wl['L']}" in wl["desc"] or f"C_{wl['L']}" in wl["desc"], name
        assert f"{wl['n_inst']} instance" in wl["desc"] or f"10^{len(str(wl['n_inst'])) - 1} instances" in wl["desc"], name
