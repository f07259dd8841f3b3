"""Oracle: the two-site H_eff*psi network of Fig. "Hpsi_fig" on block-sparse tensors.

psi'[a',s1',s2',b'] = sum L[a,w0,a'] psi[a,s1,s2,b] W[w0,s1',s1,w1] W[w1,s2',s2,w2] R[b,w2,b']
(Sec. 11, Fig. "Hpsi_fig": the effective Hamiltonian of the two-site DMRG
update applied to the two-site wavefunction).  The tensors are built from the
seeded workload description (bonds and dense-coordinate values) and contracted
by ``network.Network`` in the optimal order (or an explicit one).
"""
from __future__ import annotations

import numpy as np

import tnx_inputs as inputs

from .network import Network
from .symtensor import Bond, BlockTensor, Symmetry, U1, fill_from_function


def syms_for(wl) -> tuple:
    return tuple(Symmetry(U1) for _ in range(wl.nsym))


def make_tensor(wl, name: str, symmetric: bool = False, bonds_override=None) -> BlockTensor:
    syms = syms_for(wl)
    spec = bonds_override if bonds_override is not None else inputs.heff_bonds(wl)[name]
    bonds = [Bond.make(d, secs, syms) for d, secs in spec]
    T = BlockTensor(bonds)
    return fill_from_function(T, inputs.heff_value_fn(wl, name, symmetric=symmetric))


def make_heff(wl, symmetric: bool = False, order: str | None = None):
    """Returns (network with all five tensors put, psi)."""
    net = Network(inputs.HEFF_SPEC)
    tensors = {n: make_tensor(wl, n, symmetric=symmetric) for n in inputs.HEFF_NAMES}
    for n in inputs.HEFF_NAMES:
        net.put(n, tensors[n])
    if order:
        net.set_order(False, order)
    else:
        net.set_order(True)
    return net, tensors


def apply(net: Network, psi: BlockTensor, record=None) -> BlockTensor:
    net.put("psi", psi)
    return net.launch(record=record)


def flops(net: Network) -> int:
    rec = []
    net.launch(record=rec)
    return sum(r["flops"] for r in rec)


def flat_apply(net: Network, template: BlockTensor):
    """H_eff as a map on the canonical flat layout of psi (for Lanczos)."""
    lay = template.layout()

    def unflat(x):
        blocks = {}
        for q, shp, off in lay:
            blocks[q] = x[off:off + int(np.prod(shp))].reshape(shp).copy()
        return BlockTensor(template.bonds, blocks)

    def op(x):
        out = apply(net, unflat(x))
        # same bonds and block set as psi (the output keeps psi's legs)
        full = BlockTensor(template.bonds)
        for q in full.keys():
            if q in out.blocks:
                full.blocks[q] = out.blocks[q]
        return full.flat()

    return op
