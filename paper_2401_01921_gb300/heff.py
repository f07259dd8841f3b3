"""Build a network of block-sparse tensors from bond specifications and values.

Generic helper over the binding: each tensor is given as its legs
[(direction, [(charge tuple, degeneracy), ...]), ...] and a function that
returns its values at dense coordinates; blocks are filled from that function
and uploaded.  Used by the tests and the bench to build the two-site H_eff
network of the DMRG update (Fig. "Hpsi_fig" of arXiv 2401.01921).
"""
from __future__ import annotations

from . import U1, Bond, Context, Network, Tensor


def make_bonds(ctx: Context, legs, nsym: int):
    syms = [U1] * nsym
    return [Bond(ctx, d, secs, syms if nsym else ()) for d, secs in legs]


def build_network(ctx: Context, spec: str, tensors: dict, nsym: int, order: str | None = None, prec="f64"):
    """tensors: name -> (legs, value_at).  Returns (network, {name: Tensor}, {name: [Bond]})."""
    net = Network(ctx, spec)
    T, B = {}, {}
    for name, (legs, value_at) in tensors.items():
        B[name] = make_bonds(ctx, legs, nsym)
        T[name] = Tensor(ctx, B[name]).fill(value_at)
        net.put(name, T[name])
    if order == "sparse":
        net.set_order("sparse")
    elif order:
        net.set_order(False, order)
    else:
        net.set_order(True)
    net.set_precision(prec)
    return net, T, B
