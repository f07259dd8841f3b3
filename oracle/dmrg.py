"""Oracle: environment updates and the two-site DMRG sweep (test infrastructure).

Follows Sec. 11 of arXiv 2401.01921 (the DMRG benchmark around Fig.
"Hpsi_fig"): the ground state of a chain is an MPS of tensors A_i updated two
at a time; each update contracts the effective Hamiltonian (left environment
L, two MPO tensors, right environment R) with the two-site wavefunction,
takes the lowest eigenvector by Lanczos (Sec. 9.3), splits it by a truncated
SVD (Sec. 9.2) and grows the environment by one site.  The paper defers the
sweep itself to the library's user guide, so the steps are the textbook
two-site DMRG (White 1992; Schollwoeck 2011, Sec. 6):

* MPS tensor A_i[a IN, s IN, b OUT]; L[a OUT, w OUT, a' IN]; R[b IN, w IN,
  b' OUT]; MPO W[wL IN, s' IN, s OUT, wR OUT] (the H_eff conventions); the
  conjugate A^dagger is A with every bond reversed (real tensors, Sec. 6.4
  Dagger);
* left update  L_{i}[b, w', b'] = sum L_{i-1}[a, w, a'] A[a, s, b] W[w, s', s, w'] A^dagger[a', s', b'];
  right update R_{i}[a, w, a'] = sum A[a, s, b] W[w, s', s, w'] R_{i+1}[b, w', b'] A^dagger[a', s', b'];
* boundaries: L_0 selects the MPO's left row, R_{N+1} its right column, on
  one-dimensional bonds of charge 0 (left) and of the target charge (right);
* a sweep runs the bond (i, i+1) from left to right, keeping U as A_i
  (left-canonical) and S V^dagger as A_{i+1}, then from right to left keeping
  V^dagger as A_{i+1} and U S as A_i.

Pins (tests/test_oracle_dmrg.py): growing exact environments k -> k+1 from
identity isometries reproduces the (k+1)-site environments of
``brute.exact_environments``; the XX chain's DMRG energy equals the free-
fermion closed form; the Heisenberg chain's equals dense diagonalisation.
"""
from __future__ import annotations

import numpy as np

import tnx_inputs as inputs

from .heff import flat_apply
from .lanczos import lanczos
from .network import Network
from .svd import svd_truncate
from .symtensor import IN, OUT, Bond, BlockTensor, Symmetry, U1

ENV_LEFT_SPEC = "L: a, w, ap\nA: a, s, b\nW: w, sp, s, wp\nAd: ap, sp, bp\nTOUT: b, wp, bp\n"
ENV_RIGHT_SPEC = "A: a, s, b\nW: w, sp, s, wp\nR: b, wp, bp\nAd: ap, sp, bp\nTOUT: a, w, ap\n"
TWO_SITE_SPEC = "A1: a, s1, m\nA2: m, s2, b\nTOUT: a, s1, s2, b\n"
ABSORB_LEFT_SPEC = "S: c, m\nV: m, s, b\nTOUT: c, s, b\n"     # S V^dagger
ABSORB_RIGHT_SPEC = "U: a, s, m\nS: m, c\nTOUT: a, s, c\n"    # U S


def dagger(A: BlockTensor) -> BlockTensor:
    """Sec. 6.4 Dagger for real tensors: every bond redirected, the same blocks."""
    return BlockTensor([b.redirect() for b in A.bonds], {q: v.copy() for q, v in A.blocks.items()})


def _contract(spec: str, tensors: dict) -> BlockTensor:
    net = Network(spec)
    for n, t in tensors.items():
        net.put(n, t)
    net.set_order(True)
    return net.launch()


def env_left(L: BlockTensor, A: BlockTensor, W: BlockTensor) -> BlockTensor:
    return _contract(ENV_LEFT_SPEC, {"L": L, "A": A, "W": W, "Ad": dagger(A)})


def env_right(R: BlockTensor, A: BlockTensor, W: BlockTensor) -> BlockTensor:
    return _contract(ENV_RIGHT_SPEC, {"A": A, "W": W, "R": R, "Ad": dagger(A)})


def mpo_tensor(mpo, syms) -> BlockTensor:
    M = mpo.bond_sectors
    P = inputs.SPIN_PHYS if mpo.W.shape[1] == 2 else inputs.HUBBARD_PHYS
    bonds = [Bond.make(IN, M, syms), Bond.make(IN, P, syms), Bond.make(OUT, P, syms), Bond.make(OUT, M, syms)]
    return BlockTensor.from_dense(bonds, mpo.W_grouped())


def boundaries(mpo, syms, target):
    """L_0 and R_{N+1}: one-dimensional virtual bonds, the MPO edge row / column."""
    zero = tuple(0 for _ in syms)
    M = mpo.bond_sectors
    D = mpo.W.shape[0]
    l = np.zeros((1, D, 1))
    l[0, mpo.channel_pos[mpo.left_row], 0] = 1.0
    r = np.zeros((1, D, 1))
    r[0, mpo.channel_pos[mpo.right_col], 0] = 1.0
    L0 = BlockTensor.from_dense([Bond.make(OUT, [(zero, 1)], syms), Bond.make(OUT, M, syms),
                                 Bond.make(IN, [(zero, 1)], syms)], l)
    R0 = BlockTensor.from_dense([Bond.make(IN, [(target, 1)], syms), Bond.make(IN, M, syms),
                                 Bond.make(OUT, [(target, 1)], syms)], r)
    return L0, R0


def product_state(states, phys, syms):
    """MPS of a product state: site i in local state states[i] (an index into phys)."""
    zero = tuple(0 for _ in syms)
    q = zero
    mps = []
    for s in states:
        qs = phys[s][0]
        q2 = tuple(a + b for a, b in zip(q, qs))
        A = BlockTensor([Bond.make(IN, [(q, 1)], syms), Bond.make(IN, phys, syms), Bond.make(OUT, [(q2, 1)], syms)])
        A.blocks[(0, s, 0)] = np.ones((1, 1, 1))
        mps.append(A)
        q = q2
    return mps, q


def two_site_update(L, R, W, A1, A2, maxdim, cutoff, lanczos_steps, left_to_right):
    prod = _contract(TWO_SITE_SPEC, {"A1": A1, "A2": A2})
    psi = BlockTensor(prod.bonds)             # every zero-flux block of the two-site bonds
    for q, v in prod.blocks.items():
        psi.blocks[q] = v
    net = Network(inputs.HEFF_SPEC)
    for n, t in (("L", L), ("psi", psi), ("W1", W), ("W2", W), ("R", R)):
        net.put(n, t)
    net.set_order(True)
    op = flat_apply(net, psi)
    lam, x, *_ = lanczos(op, psi.flat(), lanczos_steps)
    lay = psi.layout()
    blocks = {q: x[off:off + int(np.prod(shp))].reshape(shp).copy() for q, shp, off in lay}
    psi = BlockTensor(psi.bonds, blocks)
    svals, U, S, V, terr = svd_truncate(psi, 2, keepdim=maxdim, err=cutoff, return_err=1)
    if left_to_right:
        return lam, U, _contract(ABSORB_LEFT_SPEC, {"S": S, "V": V}), terr
    return lam, _contract(ABSORB_RIGHT_SPEC, {"U": U, "S": S}), V, terr


def dmrg(mpo, nsites: int, maxdim: int, sweeps: int, states=None, cutoff: float = 0.0, lanczos_steps: int = 20):
    """Two-site DMRG; returns (energy after each half sweep, final MPS)."""
    syms = (Symmetry(U1),) * (len(mpo.channel_charge[0]))
    phys = inputs.SPIN_PHYS if mpo.W.shape[1] == 2 else inputs.HUBBARD_PHYS
    if states is None:
        states = [i % 2 for i in range(nsites)]
    mps, target = product_state(states, phys, syms)
    W = mpo_tensor(mpo, syms)
    L0, RN = boundaries(mpo, syms, target)
    Ls = [L0] + [None] * nsites            # Ls[i]: sites 1..i absorbed (Ls[0] = L_0)
    Rs = [None] * (nsites + 1) + [RN]      # Rs[i]: sites i..N absorbed, 1-based (Rs[N+1] = R_{N+1})
    for i in range(nsites, 2, -1):
        Rs[i] = env_right(Rs[i + 1], mps[i - 1], W)
    energies = []
    for sweep in range(sweeps):
        for i in range(1, nsites):                    # bond (i, i+1), 1-based
            lam, A1, A2, _ = two_site_update(Ls[i - 1], Rs[i + 2], W, mps[i - 1], mps[i], maxdim, cutoff,
                                             lanczos_steps, True)
            mps[i - 1], mps[i] = A1, A2
            Ls[i] = env_left(Ls[i - 1], A1, W)
        energies.append(lam)
        for i in range(nsites - 1, 0, -1):
            lam, A1, A2, _ = two_site_update(Ls[i - 1], Rs[i + 2], W, mps[i - 1], mps[i], maxdim, cutoff,
                                             lanczos_steps, False)
            mps[i - 1], mps[i] = A1, A2
            Rs[i + 1] = env_right(Rs[i + 2], A2, W)
        energies.append(lam)
    return energies, mps


def xx_ground_energy(nsites: int) -> float:
    """Open XX chain sum_j (Sx Sx + Sy Sy): Jordan-Wigner free fermions with hopping 1/2,
    single-particle energies cos(pi k / (N + 1)); the ground state fills the negative ones."""
    e = np.cos(np.pi * np.arange(1, nsites + 1) / (nsites + 1))
    return float(e[e < 0].sum())
