"""Oracle: symmetries, bonds and block-sparse tensors (test infrastructure).

Follows Sec. 6 of arXiv 2401.01921 ("UniTensor with Symmetries"):

* 6.1: a U(1) charge combines by integer addition and reverses by negation; a
  Z_n charge combines as (Q1+Q2) mod n and reverses as -Q mod n.  Several
  symmetries combine component-wise.
* 6.2: a bond carries a direction (IN / OUT), an ordered list of sectors
  (charge vector, degeneracy) and its symmetries.  Combining bonds forms all
  pairwise charge sums, grouped into one sector per distinct charge (6.2.2;
  the printed combined bond is sorted ascending).
* 6.3 / Fig. "qnblock": only zero-flux blocks are stored.  The flux of an
  element is the combination of the charges on IN legs and the reversed
  charges on OUT legs; a block is the set of elements sharing one sector per
  leg ("Qn index").  Blocks are numbered in lexicographic order of their Qn
  indices (the printed BLOCK [#0..#3] example), and each block is a dense
  row-major array over the tensor's own leg order.
* 6.5: converting dense -> symmetric copies the allowed entries and fails if
  an entry outside the allowed blocks is non-zero, unless forced.

Parity: pinned by the printed 4-block example, the printed bond combine, the
printed U(1)xZ2 bond, the Z3 rules and by brute-force enumeration over all
sector tuples (tests/test_oracle_symtensor.py).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass

import numpy as np

U1 = 0
ZN = 1
IN = 1
OUT = -1
REGULAR = 0


@dataclass(frozen=True)
class Symmetry:
    kind: int   # U1 or ZN
    n: int = 0  # modulus for ZN

    def combine(self, a: int, b: int) -> int:
        """Sec. 6.1 combine rule."""
        if self.kind == U1:
            return a + b
        return (a + b) % self.n

    def reverse(self, a: int) -> int:
        """Sec. 6.1 reverse rule."""
        if self.kind == U1:
            return -a
        return (-a) % self.n

    def normal(self, a: int) -> int:
        return a if self.kind == U1 else a % self.n


@dataclass(frozen=True)
class Bond:
    """A bond: direction, sectors [(charge tuple, degeneracy)], symmetries (Sec. 6.2)."""
    dir: int
    sectors: tuple
    syms: tuple

    @staticmethod
    def make(dir: int, sectors, syms=()):
        syms = tuple(syms)
        secs = tuple((tuple(int(s.normal(q)) for s, q in zip(syms, qn)), int(d)) for qn, d in sectors)
        return Bond(dir, secs, syms)

    @property
    def dim(self) -> int:
        return sum(d for _, d in self.sectors)

    @property
    def nsec(self) -> int:
        return len(self.sectors)

    def offsets(self) -> list[int]:
        """Dense index where each sector starts (sectors keep creation order)."""
        out, o = [], 0
        for _, d in self.sectors:
            out.append(o)
            o += d
        return out

    def signed(self, k: int) -> tuple:
        """Charge of sector k as it enters the flux: as is on IN, reversed on OUT."""
        q = self.sectors[k][0]
        if self.dir == OUT:
            return tuple(s.reverse(x) for s, x in zip(self.syms, q))
        return q

    def redirect(self) -> "Bond":
        return Bond(-self.dir, self.sectors, self.syms)


def combine_charges(syms, a: tuple, b: tuple) -> tuple:
    return tuple(s.combine(x, y) for s, x, y in zip(syms, a, b))


def zero_charge(syms) -> tuple:
    return tuple(0 for _ in syms)


def combine_bonds(b1: Bond, b2: Bond) -> Bond:
    """Sec. 6.2.2: all pairwise sums, grouped per distinct charge, ascending order."""
    if b1.dir != b2.dir or b1.syms != b2.syms:
        raise ValueError("only bonds with equal direction and symmetries combine")
    acc: dict[tuple, int] = {}
    for q1, d1 in b1.sectors:
        for q2, d2 in b2.sectors:
            q = combine_charges(b1.syms, q1, q2)
            acc[q] = acc.get(q, 0) + d1 * d2
    return Bond(b1.dir, tuple(sorted(acc.items())), b1.syms)


def flux(bonds, qidx) -> tuple:
    syms = bonds[0].syms
    f = zero_charge(syms)
    for b, k in zip(bonds, qidx):
        f = combine_charges(syms, f, b.signed(k))
    return f


def enumerate_blocks(bonds) -> list[tuple]:
    """Zero-flux Qn-index tuples in lexicographic order (Sec. 6.3, block index)."""
    if len(bonds) == 0:
        return [()]
    syms = bonds[0].syms
    z = zero_charge(syms)
    out = []
    for qidx in itertools.product(*[range(b.nsec) for b in bonds]):
        if flux(bonds, qidx) == z:
            out.append(tuple(qidx))
    return out


class BlockTensor:
    """Block-sparse FP64 tensor: bonds + {Qn-index tuple: dense block} (Sec. 6.3)."""

    def __init__(self, bonds, blocks: dict | None = None):
        self.bonds = tuple(bonds)
        if blocks is None:
            blocks = {}
            for q in enumerate_blocks(self.bonds):
                blocks[q] = np.zeros(self.block_shape(q))
        self.blocks = blocks

    @property
    def rank(self) -> int:
        return len(self.bonds)

    def block_shape(self, qidx) -> tuple:
        return tuple(b.sectors[k][1] for b, k in zip(self.bonds, qidx))

    def keys(self) -> list[tuple]:
        return sorted(self.blocks.keys())

    def nelem(self) -> int:
        return sum(int(np.prod(self.block_shape(q))) for q in self.blocks)

    def layout(self):
        """Canonical flat layout: blocks in block-index order, each row-major."""
        out, off = [], 0
        for q in self.keys():
            shp = self.block_shape(q)
            out.append((q, shp, off))
            off += int(np.prod(shp))
        return out

    def flat(self) -> np.ndarray:
        parts = [self.blocks[q].reshape(-1) for q in self.keys()]
        return np.concatenate(parts) if parts else np.zeros(0)

    def dense_coords(self, qidx):
        """Dense (full-bond) coordinates of every element of block qidx, row-major."""
        grids = []
        for b, k in zip(self.bonds, qidx):
            o = b.offsets()[k]
            grids.append(np.arange(o, o + b.sectors[k][1]))
        if not grids:
            return []
        mesh = np.meshgrid(*grids, indexing="ij")
        return [m.reshape(-1) for m in mesh]

    def densify(self) -> np.ndarray:
        """Dense array with zeros outside the stored blocks (Sec. 6.5, symmetric -> dense)."""
        D = np.zeros(tuple(b.dim for b in self.bonds))
        for q, blk in self.blocks.items():
            sl = tuple(slice(b.offsets()[k], b.offsets()[k] + b.sectors[k][1]) for b, k in zip(self.bonds, q))
            D[sl] = blk
        return D

    @staticmethod
    def from_dense(bonds, D: np.ndarray, force: bool = False) -> "BlockTensor":
        """Sec. 6.5 dense -> symmetric; error on a non-zero symmetry-violating entry unless forced."""
        T = BlockTensor(bonds)
        mask = np.zeros(D.shape, dtype=bool)
        for q in T.keys():
            sl = tuple(slice(b.offsets()[k], b.offsets()[k] + b.sectors[k][1]) for b, k in zip(T.bonds, q))
            T.blocks[q] = np.array(D[sl], dtype=np.float64)
            mask[sl] = True
        if not force and np.any(D[~mask] != 0):
            raise ValueError("dense tensor has non-zero entries outside the allowed blocks")
        return T

    def permute(self, perm) -> "BlockTensor":
        """Leg permutation: new leg i is old leg perm[i]."""
        bonds = [self.bonds[p] for p in perm]
        blocks = {tuple(q[p] for p in perm): np.transpose(b, perm).copy() for q, b in self.blocks.items()}
        return BlockTensor(bonds, blocks)

    def copy(self) -> "BlockTensor":
        return BlockTensor(self.bonds, {q: b.copy() for q, b in self.blocks.items()})

    def add(self, other: "BlockTensor") -> "BlockTensor":
        """Element-wise sum of two tensors with equal bonds (union of stored blocks)."""
        if self.bonds != other.bonds:
            raise ValueError("bond mismatch")
        out = self.copy()
        for q, b in other.blocks.items():
            out.blocks[q] = out.blocks[q] + b if q in out.blocks else b.copy()
        return out

    def add_scalar(self, x: float):
        """Sec. 6.3: adding a scalar would break the block structure: always an error."""
        raise ValueError("cannot add a scalar to a block-sparse tensor")


def fill_from_function(T: BlockTensor, value_at) -> BlockTensor:
    """Fill every stored block by evaluating value_at(list of dense coordinate arrays)."""
    for q in T.keys():
        coords = T.dense_coords(q)
        T.blocks[q] = np.asarray(value_at(coords), dtype=np.float64).reshape(T.block_shape(q))
    return T
