"""Oracle pins: symmetries, bonds, block enumeration (paper Sec. 6)."""
import itertools
import os

import numpy as np
import pytest

from oracle.symtensor import (IN, OUT, U1, ZN, Bond, BlockTensor, Symmetry, combine_bonds,
                              enumerate_blocks)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_pins.txt")


def golden(prefix):
    out = []
    for line in open(GOLDEN):
        if line.startswith(prefix + " "):
            out.append(line[len(prefix) + 1:].strip())
    return out


def test_paper_four_blocks():
    """Sec. 6.3: the printed symmetric tensor has exactly these 4 blocks, in this order."""
    u1 = (Symmetry(U1),)
    a = Bond.make(IN, [((1,), 1), ((-1,), 1)], u1)
    c = Bond.make(OUT, [((2,), 1), ((0,), 2), ((-2,), 1)], u1)
    T = BlockTensor([a, a, c])
    want = []
    for g in golden("blocks"):
        idx, q, shp = [x.strip() for x in g.split(":")]
        want.append((tuple(int(x) for x in q.split()), tuple(int(x) for x in shp.split())))
    got = [(q, T.block_shape(q)) for q in T.keys()]
    assert got == want
    assert T.nelem() == 6


def test_paper_bond_combine():
    u1 = (Symmetry(U1),)
    b1 = Bond.make(IN, [((0,), 1), ((1,), 1)], u1)
    b2 = Bond.make(IN, [((2,), 1), ((3,), 1)], u1)
    b12 = combine_bonds(b1, b2)
    want = [tuple(int(x) for x in s.split(":")) for s in golden("combine")[0].split()]
    assert [(q[0], d) for q, d in b12.sectors] == want
    assert b12.dim == 4


def test_paper_u1_z2_bond():
    syms = (Symmetry(U1), Symmetry(ZN, 2))
    b = Bond.make(IN, [((2, 0), 3), ((4, 1), 5)], syms)
    assert b.dim == 8
    assert [q for q, _ in b.sectors] == [(2, 0), (4, 1)]


def test_z3_rules():
    z3 = Symmetry(ZN, 3)
    for q1 in range(3):
        for q2 in range(3):
            assert z3.combine(q1, q2) == (q1 + q2) % 3
        assert z3.reverse(q1) == (-q1) % 3
    u1 = Symmetry(U1)
    assert u1.combine(3, -5) == -2 and u1.reverse(4) == -4


def _rand_bonds(rng, nsym_kinds, rank):
    syms = tuple(nsym_kinds)
    bonds = []
    for _ in range(rank):
        nsec = int(rng.integers(1, 4))
        secs = []
        for _ in range(nsec):
            q = tuple(int(rng.integers(-2, 3)) if s.kind == U1 else int(rng.integers(0, s.n)) for s in syms)
            secs.append((q, int(rng.integers(1, 3))))
        bonds.append(Bond.make(int(rng.choice([IN, OUT])), secs, syms))
    return bonds


@pytest.mark.parametrize("kinds", [(Symmetry(U1),), (Symmetry(U1), Symmetry(U1)), (Symmetry(ZN, 3),),
                                   (Symmetry(U1), Symmetry(ZN, 2))])
def test_enumeration_brute_force(kinds):
    """Zero-flux blocks == every sector tuple whose IN-charges minus OUT-charges vanish."""
    rng = np.random.default_rng(7)
    for rank in (1, 2, 3, 4):
        for _ in range(5):
            bonds = _rand_bonds(rng, kinds, rank)
            want = []
            for t in itertools.product(*[range(b.nsec) for b in bonds]):
                tot = [0] * len(kinds)
                for b, k in zip(bonds, t):
                    for i, s in enumerate(kinds):
                        tot[i] += b.dir * b.sectors[k][0][i]
                ok = all((x == 0) if s.kind == U1 else (x % s.n == 0) for x, s in zip(tot, kinds))
                if ok:
                    want.append(t)
            assert enumerate_blocks(bonds) == sorted(want)


def test_scalar_add_is_error():
    u1 = (Symmetry(U1),)
    a = Bond.make(IN, [((1,), 1), ((-1,), 1)], u1)
    T = BlockTensor([a, a.redirect()])
    with pytest.raises(ValueError):
        T.add_scalar(1.0)


def test_convert_dense_symmetric():
    """Sec. 6.5: dense -> symmetric copies allowed entries, refuses violating ones unless forced."""
    u1 = (Symmetry(U1),)
    a = Bond.make(IN, [((1,), 1), ((-1,), 2)], u1)
    b = Bond.make(OUT, [((1,), 2), ((-1,), 1)], u1)
    rng = np.random.default_rng(0)
    T = BlockTensor([a, b])
    for q in T.keys():
        T.blocks[q] = rng.standard_normal(T.block_shape(q))
    D = T.densify()
    T2 = BlockTensor.from_dense([a, b], D)
    assert np.array_equal(T2.densify(), D)
    D[0, 2] = 1.0   # (q=+1, q=-1) violates the flux
    with pytest.raises(ValueError):
        BlockTensor.from_dense([a, b], D)
    T3 = BlockTensor.from_dense([a, b], D, force=True)
    assert T3.densify()[0, 2] == 0.0
