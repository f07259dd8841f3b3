"""Seeded input generator: Philox4x32-10 known-answer vectors and workload recipes."""
import math

import numpy as np

import tnx_inputs as I

# Known-answer vectors published with the Random123 library for Philox4x32 with
# 10 rounds (counter words, key words) -> output words.
KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


def test_philox_kat():
    for ctr, key, want in KAT:
        got = I.philox4x32_10(*[[c] for c in ctr], *key)
        assert tuple(int(g[0]) for g in got) == want


def test_normals_moments_and_determinism():
    x = I.normal_at(3, 0, np.arange(200000))
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1) < 0.01
    assert np.array_equal(x[1000:2000], I.normal_at(3, 0, np.arange(1000, 2000)))
    assert not np.array_equal(x[:100], I.normal_at(4, 0, np.arange(100)))


def test_heisenberg_sectors():
    s = I.heisenberg_virtual_sectors(512, 20)
    assert [d for _, d in s] == [1, 1, 1, 1, 2, 7, 18, 37, 61, 82, 90, 82, 61, 37, 18, 7, 2, 1, 1, 1, 1]
    assert [q[0] for q, _ in s] == list(range(-20, 21, 2))
    s = I.heisenberg_virtual_sectors(2048, 40)
    assert len(s) == 41 and sum(d for _, d in s) == 2048


def test_hubbard_sectors():
    for chi, n in [(64, 41), (512, 113), (1024, 145), (4096, 221)]:
        s = I.hubbard_virtual_sectors(chi)
        assert len(s) == n and sum(d for _, d in s) == chi and min(d for _, d in s) >= 1


def test_batched_chis_log_uniform():
    c = I.batched_hubbard_chis(256)
    assert len(c) == 256 and min(c) >= 64 and max(c) <= 1024
    m = np.mean([math.log2(x) for x in c])
    assert 7.6 < m < 8.4


def test_symmetrised_heff_is_hermitian_with_and_without_sector_scaling():
    """The symmetrised environments make the two-site H_eff Hermitian (a Lanczos solve assumes it):
    x.(H y) = y.(H x) to rounding, also when the sectors are scaled over three decades."""
    from oracle import heff as oheff
    for wl in (I.heisenberg_workload(96, 9), I.heisenberg_workload(96, 9, sector_scale=True),
               I.hubbard_workload(64)):
        net, T = oheff.make_heff(wl, symmetric=True)
        ap = oheff.flat_apply(net, T["psi"])
        n = T["psi"].flat().size
        rng = np.random.default_rng(5)
        x, y = rng.standard_normal(n), rng.standard_normal(n)
        hx, hy = ap(x), ap(y)
        asym = abs(x @ hy - y @ hx) / (np.linalg.norm(hx) * np.linalg.norm(y))
        assert asym <= 1e-13, (wl.name, asym)
