"""Oracle pins: pairwise block-sparse contraction and fused tables (paper Sec. 7)."""
import itertools

import numpy as np
import pytest

from oracle.brute import brute_network
from oracle.contract import BondMismatch, contract_pair, fused_tables, pair_flops
from oracle.symtensor import IN, OUT, U1, ZN, Bond, BlockTensor, Symmetry


def rand_tensor(rng, bonds):
    T = BlockTensor(bonds)
    for q in T.keys():
        T.blocks[q] = rng.standard_normal(T.block_shape(q))
    return T


def rand_bond(rng, syms, dir):
    nsec = int(rng.integers(1, 4))
    secs = []
    seen = set()
    for _ in range(nsec):
        q = tuple(int(rng.integers(-2, 3)) if s.kind == U1 else int(rng.integers(0, s.n)) for s in syms)
        if q in seen:
            continue
        seen.add(q)
        secs.append((q, int(rng.integers(1, 3))))
    return Bond.make(dir, secs, syms)


def random_pair(rng, syms, ra, rb, nk):
    """A (rank ra) and B (rank rb) sharing nk bonds (B's copy redirected)."""
    shared = [rand_bond(rng, syms, int(rng.choice([IN, OUT]))) for _ in range(nk)]
    fa = [rand_bond(rng, syms, int(rng.choice([IN, OUT]))) for _ in range(ra - nk)]
    fb = [rand_bond(rng, syms, int(rng.choice([IN, OUT]))) for _ in range(rb - nk)]
    la = list(range(ra))
    rng.shuffle(la)
    lb = list(range(rb))
    rng.shuffle(lb)
    A_b = [None] * ra
    B_b = [None] * rb
    pairs = []
    for i in range(nk):
        A_b[la[i]] = shared[i]
        B_b[lb[i]] = shared[i].redirect()
        pairs.append((la[i], lb[i]))
    for i in range(ra - nk):
        A_b[la[nk + i]] = fa[i]
    for i in range(rb - nk):
        B_b[lb[nk + i]] = fb[i]
    return rand_tensor(rng, A_b), rand_tensor(rng, B_b), pairs


SYMS = [(Symmetry(U1),), (Symmetry(U1), Symmetry(U1)), (Symmetry(ZN, 3),)]


@pytest.mark.parametrize("syms", SYMS)
def test_contract_vs_brute_force(syms):
    """Block-pair contraction == explicit loops over every index of the densified tensors."""
    rng = np.random.default_rng(11)
    for trial in range(6):
        ra, rb = int(rng.integers(2, 4)), int(rng.integers(2, 4))
        nk = int(rng.integers(1, min(ra, rb) + 1))
        A, B, pairs = random_pair(rng, syms, ra, rb, nk)
        C = contract_pair(A, B, pairs)
        la = [f"a{i}" for i in range(ra)]
        lb = [f"b{j}" for j in range(rb)]
        for i, j in pairs:
            lb[j] = la[i]
        dims = {}
        for l, b in zip(la, A.bonds):
            dims[l] = b.dim
        for l, b in zip(lb, B.bonds):
            dims[l] = b.dim
        tout = [l for l in la if l not in lb] + [l for l in lb if l not in la]
        ref = brute_network({"A": la, "B": lb}, tout, {"A": A.densify(), "B": B.densify()}, dims)
        np.testing.assert_allclose(C.densify(), ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("syms", SYMS)
def test_charge_conservation(syms):
    """Entries of the densified output outside its zero-flux blocks are exactly zero."""
    rng = np.random.default_rng(12)
    for _ in range(6):
        A, B, pairs = random_pair(rng, syms, 3, 3, 1)
        C = contract_pair(A, B, pairs)
        D = C.densify()
        allowed = np.zeros(D.shape, dtype=bool)
        for q in BlockTensor(C.bonds).keys():
            sl = tuple(slice(b.offsets()[k], b.offsets()[k] + b.sectors[k][1]) for b, k in zip(C.bonds, q))
            allowed[sl] = True
        assert np.all(D[~allowed] == 0.0)
        assert set(C.blocks) <= set(BlockTensor(C.bonds).keys())


def brute_tables(A, B, pairs):
    """Independent table construction: enumerate every matched block pair and
    accumulate per (group charge) the distinct rows / K tuples / columns."""
    pairs = sorted(pairs)
    ka = [p[0] for p in pairs]
    kb = [p[1] for p in pairs]
    fa = [i for i in range(A.rank) if i not in ka]
    fb = [j for j in range(B.rank) if j not in kb]
    groups = {}
    for qa in A.keys():
        for qb in B.keys():
            kta = tuple(qa[i] for i in ka)
            ktb = tuple(qb[j] for j in kb)
            if kta != ktb:
                continue
            g = [0] * len(A.bonds[0].syms)
            for i in ka:
                q = A.bonds[i].sectors[qa[i]][0]
                for c in range(len(g)):
                    g[c] += A.bonds[i].dir * q[c]
            g = tuple(x if s.kind == U1 else x % s.n for x, s in zip(g, A.bonds[0].syms))
            G = groups.setdefault(g, (set(), set(), set()))
            G[0].add(tuple(qa[i] for i in fa))
            G[1].add(kta)
            G[2].add(tuple(qb[j] for j in fb))
    out = []
    for g in sorted(groups):
        rows, ks, cols = groups[g]
        M = sum(int(np.prod([A.bonds[i].sectors[k][1] for i, k in zip(fa, r)])) for r in rows)
        K = sum(int(np.prod([A.bonds[i].sectors[k][1] for i, k in zip(ka, t)])) for t in ks)
        N = sum(int(np.prod([B.bonds[j].sectors[k][1] for j, k in zip(fb, c)])) for c in cols)
        out.append((g, M, K, N))
    return out


@pytest.mark.parametrize("syms", SYMS)
def test_tables_vs_pair_enumeration(syms):
    rng = np.random.default_rng(13)
    for _ in range(8):
        A, B, pairs = random_pair(rng, syms, int(rng.integers(2, 5)), int(rng.integers(2, 5)), 1)
        t = fused_tables(A, B, pairs)
        bt = brute_tables(A, B, pairs)
        assert [tuple(x) for x in t["charges"].tolist()] == [g for g, *_ in bt]
        assert t["MKN"].tolist() == [[M, K, N] for _, M, K, N in bt]
        # every used block lands inside its group's extent, without overlap
        tot = 0
        for (g, r, k), q in zip(t["amap"].tolist(), A.keys()):
            if g >= 0:
                M, K, _ = t["MKN"][g]
                assert 0 <= r < M and 0 <= k < K
                tot += int(np.prod(A.block_shape(q)))
        assert tot == sum(M * K for M, K, _ in t["MKN"].tolist())
        assert pair_flops(A, B, pairs) == sum(2 * M * K * N for M, K, N in t["MKN"].tolist())


def test_bond_checks():
    u1 = (Symmetry(U1),)
    a = Bond.make(IN, [((1,), 1), ((-1,), 1)], u1)
    b = Bond.make(IN, [((1,), 1), ((-1,), 2)], u1)
    rng = np.random.default_rng(0)
    A = rand_tensor(rng, [a, a.redirect()])
    with pytest.raises(BondMismatch):     # both IN
        contract_pair(A, rand_tensor(rng, [a, a.redirect()]), [(0, 0)])
    with pytest.raises(BondMismatch):     # degeneracy differs
        contract_pair(A, rand_tensor(rng, [b.redirect(), a]), [(1, 0)])


def test_paper_symmetric_two_site_hamiltonian():
    """Sec. 6.5: H = s+s- + s-s+ + szsz built from charged aux bonds equals the dense one."""
    u1 = (Symmetry(U1),)
    bi = Bond.make(IN, [((1,), 1), ((-1,), 1)], u1)
    bo = Bond.make(OUT, [((1,), 1), ((-1,), 1)], u1)
    bqo = Bond.make(OUT, [((2,), 1)], u1)
    bqi = Bond.make(IN, [((2,), 1)], u1)
    Sp = BlockTensor([bi, bo, bqo])
    Sp.blocks[(0, 1, 0)][...] = 1.0
    Sm = BlockTensor([bqi, bi, bo])
    Sm.blocks[(0, 1, 0)][...] = 1.0
    Sz = BlockTensor([bi, bo])
    Sz.blocks[(0, 0)][...] = 1.0
    Sz.blocks[(1, 1)][...] = -1.0
    # Sp1(i1,j1,q) Sm2(q,i2,j2) -> (i1,j1,i2,j2) -> permute (i1,i2,j1,j2)
    t1 = contract_pair(Sp, Sm, [(2, 0)]).permute([0, 2, 1, 3])
    # Sm1(q,i1,j1) Sp2(i2,j2,q) -> (i1,j1,i2,j2)
    t2 = contract_pair(Sm, Sp, [(0, 2)]).permute([0, 2, 1, 3])
    t3 = contract_pair(Sz, Sz, []).permute([0, 2, 1, 3])
    H2 = t1.add(t2).add(t3)
    sp = np.array([[0.0, 1.0], [0.0, 0.0]])
    sm = sp.T
    sz = np.diag([1.0, -1.0])
    Hd = (np.kron(sp, sm) + np.kron(sm, sp) + np.kron(sz, sz)).reshape(2, 2, 2, 2)
    assert np.array_equal(H2.densify(), Hd)
    Hsym = BlockTensor.from_dense([bi, bi, bo, bo], Hd)
    assert np.array_equal(Hsym.densify(), H2.densify())
