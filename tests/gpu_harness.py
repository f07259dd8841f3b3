"""Shared helpers of the GPU parity tests: build the same seeded H_eff network on the
library and on the oracle, and compare results block by block."""
import numpy as np

import tnx_inputs as I
from oracle import heff as oheff
from oracle.symtensor import BlockTensor


def lib_heff(ctx, wl, symmetric=False, order=None, prec="f64"):
    from paper_2401_01921_gb300.heff import build_network
    bonds = I.heff_bonds(wl)
    tensors = {n: (bonds[n], I.heff_value_fn(wl, n, symmetric=symmetric)) for n in I.HEFF_NAMES}
    return build_network(ctx, I.HEFF_SPEC, tensors, wl.nsym, order=order, prec=prec)


def oracle_heff(wl, symmetric=False, order=None):
    return oheff.make_heff(wl, symmetric=symmetric, order=order)


def rel_fro(lib_blocks: dict, ref: BlockTensor) -> float:
    """||lib - ref||_F / ||ref||_F over every stored block (missing blocks = 0)."""
    num = 0.0
    den = 0.0
    keys = set(lib_blocks) | set(ref.blocks)
    for k in keys:
        a = lib_blocks.get(k)
        b = ref.blocks.get(k)
        if b is None:
            num += float(np.sum(a * a))
            continue
        den += float(np.sum(b * b))
        d = b - (a if a is not None else 0.0)
        num += float(np.sum(d * d))
    return np.sqrt(num / den) if den > 0 else np.sqrt(num)


def max_block_rel(lib_blocks: dict, ref: BlockTensor) -> float:
    """Largest ||lib_b - ref_b||_F / ||ref_b||_F over the stored blocks b with ref_b != 0."""
    worst = 0.0
    for k, b in ref.blocks.items():
        n2 = float(np.sum(b * b))
        if n2 == 0.0:
            continue
        a = lib_blocks.get(k)
        d = b - (a if a is not None else 0.0)
        worst = max(worst, np.sqrt(float(np.sum(d * d)) / n2))
    return worst
