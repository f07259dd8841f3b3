"""Oracle: pairwise block-sparse contraction and fused charge-sector tables.

Sec. 7 ("Tensor contraction") of arXiv 2401.01921: tensors are contracted by
summing over the indices with common labels; before contracting, the
dimensions are checked and, for symmetric tensors, the bond direction, the
quantum numbers and the dimension of every symmetry block.  Only stored
(zero-flux) blocks take part, so a pair of blocks contributes exactly when
their sectors agree on every contracted leg.

``contract_pair`` is that definition written out: a loop over every pair of
stored blocks, ``np.tensordot`` over the contracted legs for each matching
pair, summed into the output block (free legs of A in A's order, then free
legs of B in B's order).

``fused_tables`` restates the grouping of Sec. 6.2.2 (combine the legs of one
side into one bond, sectors with equal total charge grouped) for a pairwise
contraction: the contracted legs (in A's leg order) are fused into one bond
per total charge g, the free legs of A and of B likewise, and every matched
block pair then lives inside one dense product C_g = A_g B_g.  The convention
(also followed by the CUDA planner and compared bit-exactly):

* a K tuple (sector indices of the contracted legs, in A's leg order) is
  valid if it occurs in a block of A and in a block of B; its group charge g
  is the flux of those legs as seen from A;
* groups are the distinct g of valid K tuples, ascending lexicographically on
  the charge vector (signed integers; Z_n normalised to [0, n));
* inside a group, valid K tuples, rows (free-A tuples of blocks of A whose K
  tuple is valid) and columns (free-B tuples likewise) are ordered
  lexicographically on their sector indices; offsets are prefix sums of the
  products of their degeneracies;
* groups with no row or no column are dropped;
* the output of the contraction stores the blocks (row tuple, column tuple)
  of every group, in block-index order.

Parity: pinned against brute-force dense contraction of random tensors,
against charge conservation (output blocks outside the allowed sectors are
exactly zero after densify), against order independence, and the tables
against a brute-force pairwise enumeration (tests/test_oracle_contract.py).
"""
from __future__ import annotations

import numpy as np

from .symtensor import BlockTensor, Bond, combine_charges, zero_charge, IN, OUT, REGULAR


class BondMismatch(ValueError):
    pass


def check_contractible(ba: Bond, bb: Bond):
    """Sec. 7: contracted bonds must agree in dimension; symmetric ones must have
    opposite directions and equal sectors (charges and degeneracies)."""
    if ba.dim != bb.dim:
        raise BondMismatch("dimension mismatch")
    if ba.syms != bb.syms:
        raise BondMismatch("symmetry mismatch")
    if len(ba.syms) > 0:
        if ba.dir == REGULAR or bb.dir == REGULAR or ba.dir != -bb.dir:
            raise BondMismatch("direction mismatch")
        if ba.sectors != bb.sectors:
            raise BondMismatch("sector mismatch")
    elif ba.sectors != bb.sectors:
        raise BondMismatch("dimension mismatch")


def split_legs(rank_a: int, rank_b: int, pairs):
    """pairs: list of (leg of A, leg of B) to contract, in A's leg order."""
    pairs = sorted(pairs)
    ka = [p[0] for p in pairs]
    kb = [p[1] for p in pairs]
    fa = [i for i in range(rank_a) if i not in ka]
    fb = [i for i in range(rank_b) if i not in kb]
    return ka, kb, fa, fb


def contract_pair(A: BlockTensor, B: BlockTensor, pairs, out_blocks=None) -> BlockTensor:
    """Block-pair definition of the contraction (Sec. 7).

    out_blocks: the output block set (Qn tuples); defaults to the fused-table
    set.  Blocks that receive no contribution are zero.
    """
    ka, kb, fa, fb = split_legs(A.rank, B.rank, pairs)
    for i, j in zip(ka, kb):
        check_contractible(A.bonds[i], B.bonds[j])
    out_bonds = [A.bonds[i] for i in fa] + [B.bonds[j] for j in fb]
    if out_blocks is None:
        out_blocks = fused_tables(A, B, pairs)["out_blocks"]
    out = {}
    for q in out_blocks:
        out[q] = np.zeros(tuple(b.sectors[k][1] for b, k in zip(out_bonds, q)))
    by_k = _index_by_k(B, kb)
    for qa in A.keys():
        for qb in by_k.get(tuple(qa[i] for i in ka), ()):
            if all(qa[i] == qb[j] for i, j in zip(ka, kb)):
                key = tuple(qa[i] for i in fa) + tuple(qb[j] for j in fb)
                prod = np.tensordot(A.blocks[qa], B.blocks[qb], axes=(ka, kb))
                if key not in out:
                    raise AssertionError("matched pair outside the output block set")
                out[key] = out[key] + prod
    return BlockTensor(out_bonds, out)


def _index_by_k(B: BlockTensor, kb):
    """B's blocks listed by their sector tuple on the contracted legs (a lookup
    only: every listed pair is still checked leg by leg)."""
    idx: dict[tuple, list] = {}
    for qb in B.keys():
        idx.setdefault(tuple(qb[j] for j in kb), []).append(qb)
    return idx


def _lex_sorted(tuples):
    return sorted(set(tuples))


def fused_tables(A: BlockTensor, B: BlockTensor, pairs) -> dict:
    """Fused charge-sector tables of one pairwise contraction (convention above)."""
    ka, kb, fa, fb = split_legs(A.rank, B.rank, pairs)
    syms = A.bonds[0].syms if A.rank else (B.bonds[0].syms if B.rank else ())
    akeys = A.keys()
    bkeys = B.keys()
    kt_a = {q: tuple(q[i] for i in ka) for q in akeys}
    kt_b = {q: tuple(q[j] for j in kb) for q in bkeys}
    valid_k = set(kt_a.values()) & set(kt_b.values())

    def kcharge(kt):
        g = zero_charge(syms)
        for i, k in zip(ka, kt):
            g = combine_charges(syms, g, A.bonds[i].signed(k))
        return g

    def tdim(bonds, legs, t):
        d = 1
        for leg, k in zip(legs, t):
            d *= bonds[leg].sectors[k][1]
        return d

    group_of_k = {kt: kcharge(kt) for kt in valid_k}
    rows = {}
    for q in akeys:
        if kt_a[q] in valid_k:
            rows[tuple(q[i] for i in fa)] = group_of_k[kt_a[q]]
    cols = {}
    for q in bkeys:
        if kt_b[q] in valid_k:
            cols[tuple(q[j] for j in fb)] = group_of_k[kt_b[q]]
    charges = sorted(set(group_of_k.values()))
    charges = [g for g in charges if any(v == g for v in rows.values()) and any(v == g for v in cols.values())]
    gid = {g: i for i, g in enumerate(charges)}
    koff, roff, coff = {}, {}, {}
    MKN = []
    out_blocks = []
    for g in charges:
        K = 0
        for kt in _lex_sorted(k for k in valid_k if group_of_k[k] == g):
            koff[kt] = K
            K += tdim(A.bonds, ka, kt)
        M = 0
        rlist = _lex_sorted(r for r, v in rows.items() if v == g)
        for r in rlist:
            roff[r] = M
            M += tdim(A.bonds, fa, r)
        N = 0
        clist = _lex_sorted(c for c, v in cols.items() if v == g)
        for c in clist:
            coff[c] = N
            N += tdim(B.bonds, fb, c)
        MKN.append((M, K, N))
        for r in rlist:
            for c in clist:
                out_blocks.append(r + c)
    amap = []
    for q in akeys:
        kt = kt_a[q]
        r = tuple(q[i] for i in fa)
        if kt in valid_k and group_of_k[kt] in gid and r in rows:
            amap.append((gid[group_of_k[kt]], roff[r], koff[kt]))
        else:
            amap.append((-1, -1, -1))
    bmap = []
    for q in bkeys:
        kt = kt_b[q]
        c = tuple(q[j] for j in fb)
        if kt in valid_k and group_of_k[kt] in gid and c in cols:
            bmap.append((gid[group_of_k[kt]], koff[kt], coff[c]))
        else:
            bmap.append((-1, -1, -1))
    return {
        "charges": np.array(charges, dtype=np.int64).reshape(len(charges), len(syms)),
        "MKN": np.array(MKN, dtype=np.int64).reshape(len(charges), 3),
        "amap": np.array(amap, dtype=np.int64).reshape(len(akeys), 3),
        "bmap": np.array(bmap, dtype=np.int64).reshape(len(bkeys), 3),
        "out_blocks": sorted(out_blocks),
    }


def pair_flops(A: BlockTensor, B: BlockTensor, pairs) -> int:
    """Useful flops of one pairwise contraction: 2*m*k*n summed over matched block pairs."""
    ka, kb, fa, fb = split_legs(A.rank, B.rank, pairs)
    tot = 0
    by_k = _index_by_k(B, kb)
    for qa in A.keys():
        for qb in by_k.get(tuple(qa[i] for i in ka), ()):
            if all(qa[i] == qb[j] for i, j in zip(ka, kb)):
                sa = A.block_shape(qa)
                sb = B.block_shape(qb)
                m = int(np.prod([sa[i] for i in fa]))
                k = int(np.prod([sa[i] for i in ka]))
                n = int(np.prod([sb[j] for j in fb]))
                tot += 2 * m * k * n
    return tot
