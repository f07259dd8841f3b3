"""GPU parity of the paper's higher-rank networks (Sec. 8.1 CTM, Sec. 8.4 PEPS)
against the CPU oracle, through the C-ABI, with the library's own order search.

- The 9-tensor corner-transfer-matrix network (four corners, four edges, the
  site tensor) and the 11-tensor PEPS expectation-value network (six
  boundary-MPS tensors, two PEPS tensors and their conjugates, the operator),
  with random U(1)-symmetric tensors: the scalar they contract to equals the
  oracle's to 1e-12 relative, for the dense-cost search (Sec. 8.3) and the
  block-sparse-cost search, and for the CTM also in the paper's printed ORDER.
- The PEPS network of all-ones tensors of dimension 2 (the printed listing)
  gives 2^24 exactly.
"""
import numpy as np
import pytest

from oracle.network import Network as ONet, parse_spec
from oracle.symtensor import IN, OUT, Bond as OB, BlockTensor, Symmetry, U1

pytestmark = pytest.mark.gpu

SYM = (Symmetry(U1),)

CTM = """c0: t0-c0, t3-c0
c1: t1-c1, t0-c1
c2: t2-c2, t1-c2
c3: t3-c3, t2-c3
t0: t0-c1, w-t0, t0-c0
t1: t1-c2, w-t1, t1-c1
t2: t2-c3, w-t2, t2-c2
t3: t3-c0, w-t3, t3-c3
w: w-t0, w-t1, w-t2, w-t3
TOUT:
ORDER: ((((((((c0,t0),c1),t3),w),t1),c3),t2),c2)
"""

PEPS = """#network file peps_exp_val.net
b0:  b0-b5,  b0-b1,   b0-t0,  b0-t0*
b1:  b0-b1,  b1-b2,   b1-t0,  b1-t0*
b2:  b1-b2,  b2-b3,   b2-t0,  b2-t0*
b3:  b2-b3,  b3-b4,   b3-t1,  b3-t1*
b4:  b3-b4,  b4-b5,   b4-t1,  b4-t1*
b5:  b4-b5,  b0-b5,   b5-t1,  b5-t1*
t0:  op-t0,  t0-t1,   b0-t0,  b1-t0,  b2-t0
t0*: op-t0*, t0*-t1*, b0-t0*, b1-t0*, b2-t0*
t1:  op-t1,  t0-t1,   b3-t1,  b4-t1,  b5-t1
t1*: op-t1*, t0*-t1*, b3-t1*, b4-t1*, b5-t1*
op:  op-t0,  op-t0*,  op-t1,  op-t1*
TOUT:
ORDER:
"""


@pytest.fixture(scope="module")
def ctx():
    import paper_2401_01921_gb300 as tnx
    from paper_2401_01921_gb300 import build
    build.build()
    return tnx.Context(0)


def random_symmetric_network(spec, seed, big_labels=(), big=(2, 4), small=(1, 2)):
    """One random U(1) bond per label (charges -1, 0, +1), OUT on its first tensor and IN on its
    second; every tensor filled with N(0,1) entries in its zero-flux blocks."""
    names, labels, tout, order = parse_spec(spec)
    rng = np.random.default_rng(seed)
    secs = {}
    for n in names:
        for l in labels[n]:
            if l not in secs:
                lo, hi = big if any(l.startswith(p) for p in big_labels) else small
                secs[l] = [((q,), int(rng.integers(lo, hi + 1))) for q in (-1, 0, 1)]
    seen = set()
    tensors = {}
    for n in names:
        bonds = []
        for l in labels[n]:
            d = IN if l in seen else OUT
            seen.add(l)
            bonds.append(OB.make(d, secs[l], SYM))
        T = BlockTensor(bonds)
        for q in T.keys():
            T.blocks[q] = rng.standard_normal(T.block_shape(q))
        tensors[n] = T
    return names, labels, tensors


def contract_lib(ctx, spec, names, tensors, optimal, order=None):
    import paper_2401_01921_gb300 as tnx
    from test_gpu_linalg import to_lib
    net = tnx.Network(ctx, spec)
    keep = []
    for n in names:
        t = to_lib(ctx, tensors[n])
        keep.append(t)
        net.put(n, t)
    if optimal == "explicit":
        net.set_order(False, order)
    else:
        net.set_order(optimal)
    out = net.launch([])
    return float(out.download()[0]), net.get_order()


def contract_oracle(spec, names, tensors):
    net = ONet(spec)
    for n in names:
        net.put(n, tensors[n])
    net.set_order(True)
    out = net.launch()
    return float(out.blocks[()].reshape(-1)[0]) if () in out.blocks else 0.0


@pytest.mark.parametrize("seed", [1, 2])
def test_ctm_network_matches_the_oracle(ctx, seed):
    names, labels, tensors = random_symmetric_network(CTM, seed, big_labels=("t0-c", "t1-c", "t2-c", "t3-c"))
    ref = contract_oracle(CTM, names, tensors)
    assert ref != 0.0
    for mode in (True, "sparse", "explicit"):
        got, order = contract_lib(ctx, CTM, names, tensors, mode, "((((((((c0,t0),c1),t3),w),t1),c3),t2),c2)")
        assert abs(got - ref) <= 1e-12 * abs(ref), (mode, order, got, ref)


@pytest.mark.parametrize("seed", [3, 4])
def test_peps_network_matches_the_oracle(ctx, seed):
    names, labels, tensors = random_symmetric_network(PEPS, seed, big_labels=("b",))
    ref = contract_oracle(PEPS, names, tensors)
    assert ref != 0.0
    for mode in (True, "sparse"):
        got, order = contract_lib(ctx, PEPS, names, tensors, mode)
        assert abs(got - ref) <= 1e-12 * abs(ref), (mode, order, got, ref)


def test_peps_network_of_ones_gives_two_to_the_24(ctx):
    import paper_2401_01921_gb300 as tnx
    names, labels, tout, order = parse_spec(PEPS)
    net = tnx.Network(ctx, PEPS)
    keep = []
    for n in names:
        bonds = [tnx.Bond(ctx, tnx.BD_REG, [((), 2)]) for _ in labels[n]]
        t = tnx.Tensor(ctx, bonds)
        t.upload(np.ones(t.nelem))
        keep.append(t)
        net.put(n, t)
    net.set_order(True)
    assert float(net.launch([]).download()[0]) == 2.0 ** 24
