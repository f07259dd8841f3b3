"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no part of the contraction method: it produces numbers and
workload recipes only.

* ``philox4x32_10``: the counter-based generator Philox4x32-10 of Salmon,
  Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3"
  (SC'11), written from its published definition (two 32x32->64 multiplies per
  round, Weyl-sequence key schedule, 10 rounds).
* ``normal_at`` / ``uniform_at``: values addressed by (seed, stream id, index),
  so that a tensor element is defined by its DENSE coordinate and not by any
  block layout.  Each side (oracle or library) fills its own blocks by asking
  for the values at the dense coordinates of its block elements.
* Workload recipes: sector lists of the virtual bonds (binomial-shaped U(1)
  Heisenberg sectors, Gaussian-shaped U(1)xU(1) Hubbard sectors), the local
  bases, and the dense MPO tensors W[wL, s_out, s_in, wR] of the spin-1/2
  Heisenberg chain (D=5) and the Jordan-Wigner spinful Hubbard chain (D=6),
  with the charge carried by each MPO channel.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint32 arrays (counter words c0..c3, key k0,k1).

    One round: (hi0,lo0) = M0*c0, (hi1,lo1) = M1*c2;
    new = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); then the key is bumped by
    the Weyl constants.  Returns four uint32 arrays.
    """
    c0 = np.asarray(c0, dtype=np.uint32).copy()
    c1 = np.asarray(c1, dtype=np.uint32).copy()
    c2 = np.asarray(c2, dtype=np.uint32).copy()
    c3 = np.asarray(c3, dtype=np.uint32).copy()
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for _ in range(10):
            p0 = c0.astype(np.uint64) * _M0
            p1 = c2.astype(np.uint64) * _M1
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            k0 = np.uint32(k0 + _W0)
            k1 = np.uint32(k1 + _W1)
    return c0, c1, c2, c3


def _words(seed: int, stream: int, idx):
    idx = np.asarray(idx, dtype=np.int64).astype(np.uint64)
    lo = (idx & _MASK32).astype(np.uint32)
    hi = (idx >> np.uint64(32)).astype(np.uint32)
    s = np.full(lo.shape, np.uint32(stream & 0xFFFFFFFF), dtype=np.uint32)
    z = np.zeros(lo.shape, dtype=np.uint32)
    return philox4x32_10(lo, hi, s, z, seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def _u53(a, b):
    """53-bit uniform in (0, 1] from two 32-bit words."""
    m = (a.astype(np.uint64) >> np.uint64(5)) * np.uint64(1 << 26) + (b.astype(np.uint64) >> np.uint64(6))
    return (m.astype(np.float64) + 1.0) * (1.0 / 9007199254740992.0)


def uniform_at(seed: int, stream: int, idx) -> np.ndarray:
    """U(0,1] value for each index (float64)."""
    x0, x1, _, _ = _words(seed, stream, idx)
    return _u53(x0, x1)


def normal_at(seed: int, stream: int, idx) -> np.ndarray:
    """N(0,1) value for each index: Box-Muller (cosine branch) on two 53-bit uniforms."""
    x0, x1, x2, x3 = _words(seed, stream, idx)
    u1 = _u53(x0, x1)
    u2 = _u53(x2, x3)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


# ----------------------------------------------------------------------------
# Sector recipes
# ----------------------------------------------------------------------------

def largest_remainder(weights, total: int) -> list[int]:
    """Integer degeneracies proportional to ``weights`` summing to ``total``, each >= 1.

    floor of the quota (at least 1); if the sum is short, +1 to the largest
    fractional remainders (ties: lower index); if it is over, -1 from the
    entries above 1 with the smallest remainders (ties: higher index).
    """
    w = np.asarray(weights, dtype=np.float64)
    if total < len(w):
        raise ValueError("total below the number of sectors")
    quota = total * w / w.sum()
    deg = np.maximum(1, np.floor(quota)).astype(np.int64)
    rem = quota - np.floor(quota)
    diff = int(total - deg.sum())
    if diff > 0:
        order = sorted(range(len(w)), key=lambda i: (-rem[i], i))
        for i in order[:diff]:
            deg[i] += 1
    elif diff < 0:
        order = sorted([i for i in range(len(w)) if deg[i] > 1], key=lambda i: (rem[i], -i))
        k = 0
        while diff < 0:
            i = order[k % len(order)]
            if deg[i] > 1:
                deg[i] -= 1
                diff += 1
            k += 1
    return [int(x) for x in deg]


def heisenberg_virtual_sectors(chi: int, n: int) -> list[tuple[tuple[int], int]]:
    """U(1) sectors (2Sz units) of a virtual bond of total dimension ``chi``.

    Charges q = 2k - n, k = 0..n, degeneracy ~ chi * C(n,k)/2^n (largest remainder).
    """
    w = [math.comb(n, k) for k in range(n + 1)]
    deg = largest_remainder(w, chi)
    return [((2 * k - n,), deg[k]) for k in range(n + 1)]


def hubbard_virtual_sectors(chi: int, shift_n: int = 0) -> list[tuple[tuple[int, int], int]]:
    """U(1)xU(1) sectors (N, 2Sz) of a virtual bond of total dimension ``chi``.

    K = max(2, round(log2 chi) - 2); (dN, 2Sz) with |dN|, |2Sz| <= K and
    dN = 2Sz (mod 2), lexicographic ascending; degeneracy ~ exp(-(dN^2+2Sz^2)/(2 (K/2)^2)).
    ``shift_n`` offsets the particle number (right bond of a two-site block: +2).
    """
    K = max(2, int(round(math.log2(chi))) - 2)
    secs = [(dn, sz) for dn in range(-K, K + 1) for sz in range(-K, K + 1) if (dn - sz) % 2 == 0]
    w = [math.exp(-(dn * dn + sz * sz) / (2.0 * (K / 2.0) ** 2)) for dn, sz in secs]
    deg = largest_remainder(w, chi)
    return [((dn + shift_n, sz), d) for (dn, sz), d in zip(secs, deg)]


# ----------------------------------------------------------------------------
# Local operators and MPOs.  W[wL, s_out, s_in, wR] = (operator in channel wL->wR)[s_out, s_in]
# ----------------------------------------------------------------------------

SPIN_PHYS = [((1,), 1), ((-1,), 1)]          # |up>, |dn> in 2Sz units
HUBBARD_PHYS = [((0, 0), 1), ((1, 1), 1), ((1, -1), 1), ((2, 0), 1)]  # |0>,|up>,|dn>,|updn>


@dataclass
class MPO:
    """Dense MPO tensor plus how its channels sit in the charged MPO bond."""
    W: np.ndarray                       # [D, d, d, D]
    channel_charge: list[tuple]         # charge carried by each channel
    bond_sectors: list[tuple[tuple, int]] = field(default_factory=list)  # grouped sectors
    channel_pos: list[int] = field(default_factory=list)  # dense position of channel c in the grouped bond
    left_row: int = 0                   # boundary: row selected on the left edge
    right_col: int = 0                  # boundary: column selected on the right edge

    def W_grouped(self) -> np.ndarray:
        """W with its MPO legs reordered into the grouped-bond dense order."""
        D = self.W.shape[0]
        P = np.zeros((D, D))
        for c, p in enumerate(self.channel_pos):
            P[p, c] = 1.0
        return np.einsum("pa,asbt,qt->psbq", P, self.W, P)


def _group_channels(charges):
    secs = []
    for q in charges:
        if q not in secs:
            secs.append(q)
    pos = []
    counts = {q: 0 for q in secs}
    degs = {q: charges.count(q) for q in secs}
    start = {}
    off = 0
    for q in secs:
        start[q] = off
        off += degs[q]
    for q in charges:
        pos.append(start[q] + counts[q])
        counts[q] += 1
    return [(q, degs[q]) for q in secs], pos


def heisenberg_mpo(J: float = 1.0) -> MPO:
    """Lower-triangular D=5 MPO of H = J sum S_i . S_{i+1} (S = sigma/2).

    W[0,0]=I, W[1,0]=S+, W[2,0]=S-, W[3,0]=Sz, W[4,1]=J/2 S-, W[4,2]=J/2 S+,
    W[4,3]=J Sz, W[4,4]=I; the left edge takes row 4, the right edge column 0.
    Channel charges follow from zero flux with wL IN, s_out IN, s_in OUT, wR OUT:
    q(wL) = q(wR) + q(s_in) - q(s_out).
    """
    I = np.eye(2)
    Sp = np.array([[0.0, 1.0], [0.0, 0.0]])
    Sm = Sp.T.copy()
    Sz = np.diag([0.5, -0.5])
    W = np.zeros((5, 2, 2, 5))
    W[0, :, :, 0] = I
    W[1, :, :, 0] = Sp
    W[2, :, :, 0] = Sm
    W[3, :, :, 0] = Sz
    W[4, :, :, 1] = 0.5 * J * Sm
    W[4, :, :, 2] = 0.5 * J * Sp
    W[4, :, :, 3] = J * Sz
    W[4, :, :, 4] = I
    charges = [(0,), (-2,), (2,), (0,), (0,)]
    secs, pos = _group_channels(charges)
    # order the grouped bond as {0:3, +2:1, -2:1}
    want = [(0,), (2,), (-2,)]
    secs = [(q, dict(secs)[q]) for q in want]
    start = {}
    off = 0
    for q, d in secs:
        start[q] = off
        off += d
    used = {q: 0 for q in want}
    pos = []
    for q in charges:
        pos.append(start[q] + used[q])
        used[q] += 1
    return MPO(W=W, channel_charge=charges, bond_sectors=secs, channel_pos=pos, left_row=4, right_col=0)


def xx_mpo() -> MPO:
    """Lower-triangular D=4 MPO of the XX chain H = sum (Sx Sx + Sy Sy) (the paper's DMRG
    benchmark model, M_D = 4): W[0,0]=I, W[1,0]=S+, W[2,0]=S-, W[3,1]=S-/2, W[3,2]=S+/2,
    W[3,3]=I; the left edge takes row 3, the right edge column 0.  Grouped MPO bond
    {0:2, +2:1, -2:1} (2Sz units), channel charges as in ``heisenberg_mpo``."""
    I = np.eye(2)
    Sp = np.array([[0.0, 1.0], [0.0, 0.0]])
    Sm = Sp.T.copy()
    W = np.zeros((4, 2, 2, 4))
    W[0, :, :, 0] = I
    W[1, :, :, 0] = Sp
    W[2, :, :, 0] = Sm
    W[3, :, :, 1] = 0.5 * Sm
    W[3, :, :, 2] = 0.5 * Sp
    W[3, :, :, 3] = I
    charges = [(0,), (-2,), (2,), (0,)]
    want = [(0,), (2,), (-2,)]
    degs = {q: charges.count(q) for q in want}
    secs = [(q, degs[q]) for q in want]
    start, off = {}, 0
    for q, d in secs:
        start[q] = off
        off += d
    used = {q: 0 for q in want}
    pos = []
    for q in charges:
        pos.append(start[q] + used[q])
        used[q] += 1
    return MPO(W=W, channel_charge=charges, bond_sectors=secs, channel_pos=pos, left_row=3, right_col=0)


def hubbard_local_ops():
    """Local fermion operators on |0>,|up>,|dn>,|updn> with |updn> = c+_up c+_dn |0>."""
    cup_dag = np.zeros((4, 4))
    cup_dag[1, 0] = 1.0
    cup_dag[3, 2] = 1.0
    cdn_dag = np.zeros((4, 4))
    cdn_dag[2, 0] = 1.0
    cdn_dag[3, 1] = -1.0
    F = np.diag([1.0, -1.0, -1.0, 1.0])
    return cup_dag, cdn_dag, F


def hubbard_mpo(t: float = 1.0, U: float = 4.0) -> MPO:
    """Lower-triangular D=6 Jordan-Wigner MPO of the spinful Hubbard chain.

    H = -t sum_sigma (c+_i c_{i+1} + h.c.) + U sum n_up n_dn, modes ordered
    (site, up, dn).  With c+_i c_j = (C+ F)_i (x) C_j and c+_j c_i = (F C)_i (x) C+_j:
    W[0,0]=I, W[1,0]=Cup, W[2,0]=Cup+, W[3,0]=Cdn, W[4,0]=Cdn+, W[5,0]=U n_up n_dn,
    W[5,1]=-t Cup+ F, W[5,2]=-t F Cup, W[5,3]=-t Cdn+ F, W[5,4]=-t F Cdn, W[5,5]=I.
    """
    cup_dag, cdn_dag, F = hubbard_local_ops()
    cup = cup_dag.T.copy()
    cdn = cdn_dag.T.copy()
    I = np.eye(4)
    nud = np.diag([0.0, 0.0, 0.0, 1.0])
    W = np.zeros((6, 4, 4, 6))
    W[0, :, :, 0] = I
    W[1, :, :, 0] = cup
    W[2, :, :, 0] = cup_dag
    W[3, :, :, 0] = cdn
    W[4, :, :, 0] = cdn_dag
    W[5, :, :, 0] = U * nud
    W[5, :, :, 1] = -t * (cup_dag @ F)
    W[5, :, :, 2] = -t * (F @ cup)
    W[5, :, :, 3] = -t * (cdn_dag @ F)
    W[5, :, :, 4] = -t * (F @ cdn)
    W[5, :, :, 5] = I
    charges = [(0, 0), (1, 1), (-1, -1), (1, -1), (-1, 1), (0, 0)]
    secs, pos = _group_channels(charges)
    return MPO(W=W, channel_charge=charges, bond_sectors=secs, channel_pos=pos, left_row=5, right_col=0)


def channel_bar_heisenberg(D: int = 5) -> list[int]:
    """Channel map w -> w-bar that swaps S+ and S- channels (1 <-> 2), in channel order."""
    return [0, 2, 1, 3, 4][:D]


# ----------------------------------------------------------------------------
# Workload descriptions (sizes of the synthetic cases)
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    kind: str                 # "heisenberg" | "hubbard" | "dense"
    chi: int
    left_sectors: list        # [(charge tuple, deg)]
    right_sectors: list
    phys_sectors: list
    mpo: MPO
    seeds: dict
    sector_scale: bool = False   # per first-leg-sector 10^U(-3,0) scaling
    nsym: int = 1


def heisenberg_workload(chi: int, n: int, name: str | None = None, sector_scale: bool = False) -> Workload:
    secs = heisenberg_virtual_sectors(chi, n)
    return Workload(name=name or f"heisenberg_u1_chi{chi}", kind="heisenberg", chi=chi,
                    left_sectors=secs, right_sectors=secs, phys_sectors=SPIN_PHYS,
                    mpo=heisenberg_mpo(), seeds={"L": 1, "R": 2, "psi": 3, "scale": 4},
                    sector_scale=sector_scale, nsym=1)


def hubbard_workload(chi: int, seed_base: int = 1000, name: str | None = None) -> Workload:
    return Workload(name=name or f"hubbard_u1u1_chi{chi}", kind="hubbard", chi=chi,
                    left_sectors=hubbard_virtual_sectors(chi, 0),
                    right_sectors=hubbard_virtual_sectors(chi, 2),
                    phys_sectors=HUBBARD_PHYS, mpo=hubbard_mpo(),
                    seeds={"L": seed_base, "R": seed_base + 1, "psi": seed_base + 2, "scale": seed_base + 3},
                    sector_scale=False, nsym=2)


def dense_workload(chi: int = 32) -> Workload:
    """The dense (no symmetry) chi=32, d=2, D=5 Heisenberg case: one sector per bond."""
    return Workload(name=f"dense_chi{chi}", kind="dense", chi=chi,
                    left_sectors=[((), chi)], right_sectors=[((), chi)], phys_sectors=[((), 2)],
                    mpo=heisenberg_mpo(), seeds={"L": 1, "R": 2, "psi": 3, "scale": 4}, nsym=0)


def batched_hubbard_chis(count: int = 256, seed: int = 6, lo: float = 6.0, hi: float = 10.0) -> list[int]:
    """chi = round(2^U(lo,hi)) per instance (log-uniform in [64, 1024] by default)."""
    u = uniform_at(seed, 0, np.arange(count))
    return [int(round(2.0 ** (lo + (hi - lo) * x))) for x in u]


# ----------------------------------------------------------------------------
# The two-site H_eff network (Fig. "Hpsi_fig"): legs, directions, values
# ----------------------------------------------------------------------------

IN, OUT, REGULAR = 1, -1, 0

HEFF_SPEC = (
    "L: a, w0, ap\n"
    "psi: a, s1, s2, b\n"
    "W1: w0, s1p, s1, w1\n"
    "W2: w1, s2p, s2, w2\n"
    "R: b, w2, bp\n"
    "TOUT: ap, s1p, s2p, bp\n"
    "ORDER:\n"
)

HEFF_NAMES = ["L", "psi", "W1", "W2", "R"]
STREAM = {"L": 1, "R": 2, "psi": 3, "W1": 4, "W2": 4}


def heff_bonds(wl: Workload) -> dict:
    """name -> list of (direction, sectors) per leg, in the blueprint leg order.

    psi[a IN, s1 IN, s2 IN, b OUT]; L[a OUT, w OUT, a' IN]; W[wL IN, s' IN, s OUT, wR OUT];
    R[b IN, w IN, b' OUT]; dense workloads use REGULAR bonds with one sector.
    """
    if wl.kind == "dense":
        D = wl.mpo.W.shape[0]
        d = wl.mpo.W.shape[1]
        v = [(REGULAR, [((), wl.chi)])]
        m = [(REGULAR, [((), D)])]
        p = [(REGULAR, [((), d)])]
        return {"L": v + m + v, "psi": v + p + p + v, "W1": m + p + p + m, "W2": m + p + p + m, "R": v + m + v}
    Ls, Rs, P, M = wl.left_sectors, wl.right_sectors, wl.phys_sectors, wl.mpo.bond_sectors
    return {
        "L": [(OUT, Ls), (OUT, M), (IN, Ls)],
        "psi": [(IN, Ls), (IN, P), (IN, P), (OUT, Rs)],
        "W1": [(IN, M), (IN, P), (OUT, P), (OUT, M)],
        "W2": [(IN, M), (IN, P), (OUT, P), (OUT, M)],
        "R": [(IN, Rs), (IN, M), (OUT, Rs)],
    }


def _sector_of(sectors, idx):
    starts = np.cumsum([0] + [d for _, d in sectors])
    return np.searchsorted(starts, idx, side="right") - 1


def heff_value_fn(wl: Workload, name: str, symmetric: bool = False):
    """Value of tensor ``name`` at dense coordinates (list of int arrays, one per leg).

    L, R, psi: N(0,1) from (seed, stream, row-major dense index); with
    ``symmetric``, L[a,w,a'] <- (L[a,w,a'] + L[a',wbar,a]) / 2 and the same for R,
    where wbar swaps the S+ / S- channels (Heisenberg) or the c / c+ channels
    (Hubbard).  With ``wl.sector_scale``, every element of psi is multiplied by
    10^(-3 u) with u ~ U(0,1] drawn per sector of its first leg, and every element
    of L and R by 10^(-3 (u + u') / 2), u and u' drawn for the sectors of the two
    virtual legs (first and last, which carry the same sectors): the same range,
    and the symmetrised environments stay symmetric, so H_eff stays Hermitian.
    W: the MPO.
    """
    bonds = heff_bonds(wl)[name]
    dims = [sum(d for _, d in secs) for _, secs in bonds]
    if name in ("W1", "W2"):
        Wg = wl.mpo.W_grouped()
        return lambda c: Wg[c[0], c[1], c[2], c[3]]
    seed = wl.seeds[{"L": "L", "R": "R", "psi": "psi"}[name]]
    stream = STREAM[name]

    def flat(c):
        f = np.zeros_like(c[0], dtype=np.int64)
        for x, dm in zip(c, dims):
            f = f * dm + x
        return f

    bar = None
    if name in ("L", "R") and symmetric:
        D = wl.mpo.W.shape[0]
        if wl.kind == "hubbard":
            chbar = [0, 2, 1, 4, 3, 5]
        else:
            chbar = channel_bar_heisenberg(D)
        pos = wl.mpo.channel_pos
        inv = [0] * D
        for ch, p in enumerate(pos):
            inv[p] = ch
        bar = np.array([pos[chbar[inv[p]]] for p in range(D)], dtype=np.int64)

    def fn(c):
        c = [np.asarray(x, dtype=np.int64) for x in c]
        v = normal_at(seed, stream, flat(c))
        if bar is not None:
            v = 0.5 * (v + normal_at(seed, stream, flat([c[2], bar[c[1]], c[0]])))
        if wl.sector_scale:
            secs = bonds[0][1]
            u = uniform_at(wl.seeds["scale"], stream, _sector_of(secs, c[0]))
            if name in ("L", "R"):
                u2 = uniform_at(wl.seeds["scale"], stream, _sector_of(bonds[2][1], c[2]))
                u = 0.5 * (u + u2)
            v = v * np.power(10.0, -3.0 * u)
        return v

    return fn


# ----------------------------------------------------------------------------
# The left environment update of a DMRG sweep (Sec. 11): inputs at bond dimension chi
# ----------------------------------------------------------------------------

ENV_LEFT_SPEC = (
    "L: a, w, ap\n"
    "A: a, s, b\n"
    "W: w, sp, s, wp\n"
    "Ad: ap, sp, bp\n"
    "TOUT: b, wp, bp\n"
)
ENV_NAMES = ["L", "A", "W"]          # Ad is the Dagger of A (Sec. 6.4), made by each side itself
ENV_SEEDS = {"L": (21, 1), "A": (22, 5)}


def env_bonds(chi: int, n: int) -> dict:
    """Legs of L[a OUT, w OUT, a' IN], A[a IN, s IN, b OUT] and W (the Heisenberg MPO):
    a carries the binomial sector list of n (even 2Sz charges), b that of n + 1 (odd
    charges), both summing to chi, so every block of A has s = +-1 between them."""
    a = heisenberg_virtual_sectors(chi, n)
    b = heisenberg_virtual_sectors(chi, n + 1)
    M = heisenberg_mpo().bond_sectors
    return {"L": [(OUT, a), (OUT, M), (IN, a)],
            "A": [(IN, a), (IN, SPIN_PHYS), (OUT, b)],
            "W": [(IN, M), (IN, SPIN_PHYS), (OUT, SPIN_PHYS), (OUT, M)]}


def env_value_fn(name: str, legs: dict):
    """N(0,1) for L and A from (seed, stream, row-major dense index); W: the grouped MPO."""
    if name == "W":
        Wg = heisenberg_mpo().W_grouped()
        return lambda c: Wg[c[0], c[1], c[2], c[3]]
    seed, stream = ENV_SEEDS[name]
    dims = [sum(d for _, d in secs) for _, secs in legs[name]]

    def fn(c):
        f = np.zeros_like(np.asarray(c[0]), dtype=np.int64)
        for x, dm in zip(c, dims):
            f = f * dm + np.asarray(x, dtype=np.int64)
        return normal_at(seed, stream, f)

    return fn
