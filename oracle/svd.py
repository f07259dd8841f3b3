"""Oracle: singular value decomposition of a block-sparse tensor, with truncation.

Test infrastructure (only tests/, the smoke check and the benchmark's CPU
baseline use it).  Follows Sec. 9.1 ("Mapping from tensor to matrix") and
Sec. 9.2 ("Singular value decomposition") of arXiv 2401.01921:

* the first ``rowrank`` legs are the row legs, the rest the column legs; for a
  symmetric tensor the matrix splits into one dense block per total charge g
  of the row legs (its rows: every row-leg sector tuple with flux g, in
  lexicographic order, each spanning the product of its degeneracies; its
  columns: likewise for the column legs, whose flux balances g);
* every block gets a full SVD (numpy.linalg.svd, the library routine);
* truncation (Svd_truncate): the singular values of all blocks are sorted
  together and only the largest ``keepdim`` are kept; values smaller than
  ``err`` are dropped (the values are not normalised first); ``min_blockdim``
  gives, per block of S, a number of its largest values that are kept even
  if the other rules would drop them; ``return_err`` = 1 returns the largest
  dropped value, 2 all dropped values;
* U keeps the row legs and gains a new leg (OUT) whose sectors are the kept
  charges g (ascending) with the kept counts; V-dagger gains the matching IN
  leg followed by the column legs; S is diagonal between the two.

Readings where the section is silent (listed in the design notes): forced
values count towards keepdim, and the remaining places go to the largest
remaining values (this reproduces the printed min_blockdim example); equal
singular values are ranked by block order, then by position in the block;
a block whose kept count is zero disappears from the new leg.

Pins (tests/test_oracle_svd.py): the printed singular values of the rank-3
example of Sec. 9.1 (6 x 4 matrix of arange(24)); the printed per-block values
of the symmetric example and the printed outcome of keepdim = 4 with and
without min_blockdim; reconstruction and orthogonality.
"""
from __future__ import annotations

import itertools

import numpy as np

from .symtensor import IN, OUT, Bond, BlockTensor, combine_charges, zero_charge


def _flux_of(bonds, qidx, syms):
    f = zero_charge(syms)
    for b, k in zip(bonds, qidx):
        f = combine_charges(syms, f, b.signed(k))
    return f


def matrix_blocks(T: BlockTensor, rowrank: int):
    """Splits T into dense blocks M_g (Sec. 9.1).  Returns a list, ascending in g, of
    (g, row tuples [(tuple, row offset, rows)], column tuples [(tuple, col offset, cols)], M_g)."""
    rb, cb = T.bonds[:rowrank], T.bonds[rowrank:]
    syms = T.bonds[0].syms if T.bonds else ()
    rows, cols = {}, {}
    for q in T.keys():
        rq, cq = q[:rowrank], q[rowrank:]
        g = _flux_of(rb, rq, syms)
        rows.setdefault(g, set()).add(rq)
        cols.setdefault(g, set()).add(cq)
    out = []
    for g in sorted(rows):
        rl, cl, r0, c0 = [], [], 0, 0
        for t in sorted(rows[g]):
            m = int(np.prod([b.sectors[k][1] for b, k in zip(rb, t)])) if rb else 1
            rl.append((t, r0, m))
            r0 += m
        for t in sorted(cols[g]):
            n = int(np.prod([b.sectors[k][1] for b, k in zip(cb, t)])) if cb else 1
            cl.append((t, c0, n))
            c0 += n
        M = np.zeros((r0, c0))
        for t, ro, m in rl:
            for u, co, n in cl:
                blk = T.blocks.get(t + u)
                if blk is not None:
                    M[ro:ro + m, co:co + n] = blk.reshape(m, n)
        out.append((g, rl, cl, M))
    return out


def kept_counts(svals, keepdim=None, err=0.0, min_blockdim=None):
    """Number of values kept per block (svals: per block, descending) under the
    Sec. 9.2 rules; and the dropped values, descending."""
    nb = len(svals)
    forced = [0] * nb
    if min_blockdim is not None:
        if len(min_blockdim) != nb:
            raise ValueError("min_blockdim needs one entry per block of S")
        forced = [min(int(m), len(s)) for m, s in zip(min_blockdim, svals)]
    keep = list(forced)
    budget = None if keepdim is None else max(int(keepdim) - sum(forced), 0)
    rest = []
    for b, s in enumerate(svals):
        for i in range(forced[b], len(s)):
            rest.append((-float(s[i]), b, i))
    rest.sort()
    taken = 0
    for negv, b, i in rest:
        v = -negv
        if v < err:
            break
        if budget is not None and taken >= budget:
            break
        # values of a block are taken largest first, so position i is the next one of block b
        keep[b] += 1
        taken += 1
    dropped = sorted((float(s[i]) for b, s in enumerate(svals) for i in range(keep[b], len(s))), reverse=True)
    return keep, dropped


def svd_truncate(T: BlockTensor, rowrank: int, keepdim=None, err: float = 0.0, min_blockdim=None,
                 return_err: int = 0):
    """Returns (S values per kept block, U, S, Vdag[, err]) as BlockTensors (Sec. 9.2)."""
    syms = T.bonds[0].syms if T.bonds else ()
    blocks = matrix_blocks(T, rowrank)
    dec = []
    for g, rl, cl, M in blocks:
        u, s, vh = np.linalg.svd(M, full_matrices=False)
        dec.append((g, rl, cl, u, s, vh))
    keep, dropped = kept_counts([d[4] for d in dec], keepdim, err, min_blockdim)
    secs = [(d[0], k) for d, k in zip(dec, keep) if k > 0]
    c_out = Bond(OUT, tuple(secs), syms)
    c_in = Bond(IN, tuple(secs), syms)
    rb, cb = T.bonds[:rowrank], T.bonds[rowrank:]
    Ub, Sb, Vb = {}, {}, {}
    svals = []
    ci = 0
    for (g, rl, cl, u, s, vh), k in zip(dec, keep):
        if k == 0:
            continue
        for t, r0, m in rl:
            shp = tuple(b.sectors[x][1] for b, x in zip(rb, t)) + (k,)
            Ub[t + (ci,)] = u[r0:r0 + m, :k].reshape(shp).copy()
        for t, c0, n in cl:
            shp = (k,) + tuple(b.sectors[x][1] for b, x in zip(cb, t))
            Vb[(ci,) + t] = vh[:k, c0:c0 + n].reshape(shp).copy()
        Sb[(ci, ci)] = np.diag(s[:k])
        svals.append(s[:k].copy())
        ci += 1
    U = BlockTensor(list(rb) + [c_out], Ub)
    S = BlockTensor([c_in, c_out], Sb)
    V = BlockTensor([c_in] + list(cb), Vb)
    if return_err == 1:
        return svals, U, S, V, (dropped[0] if dropped else 0.0)
    if return_err == 2:
        return svals, U, S, V, np.array(dropped)
    return svals, U, S, V


def reconstruct(U: BlockTensor, S: BlockTensor, V: BlockTensor, bonds) -> BlockTensor:
    """U * S * Vdag back on the original legs (every zero-flux block of `bonds`)."""
    rowrank = U.rank - 1
    out = BlockTensor(bonds)
    for q in out.keys():
        rq, cq = q[:rowrank], q[rowrank:]
        acc = np.zeros(out.block_shape(q))
        m = int(np.prod(acc.shape[:rowrank])) if rowrank else 1
        n = int(np.prod(acc.shape[rowrank:])) if len(acc.shape) > rowrank else 1
        acc2 = acc.reshape(m, n)
        for (ci, cj), s in S.blocks.items():
            u = U.blocks.get(rq + (ci,))
            v = V.blocks.get((cj,) + cq)
            if u is not None and v is not None:
                acc2 += u.reshape(m, -1) @ s @ v.reshape(-1, n)
        out.blocks[q] = acc2.reshape(acc.shape)
    return out
