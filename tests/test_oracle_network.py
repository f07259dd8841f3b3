"""Oracle pins: Network text format, ORDER, optimal order search (paper Sec. 8, Sec. 7)."""
import itertools
import os

import numpy as np
import pytest

import tnx_inputs as I
from oracle import heff
from oracle.brute import brute_network
from oracle.network import (Network, NetworkError, all_trees, optimal_order, parse_order, parse_spec,
                            tree_cost, tree_str)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_pins.txt")


def golden(prefix):
    return [l[len(prefix) + 1:].rstrip("\n") for l in open(GOLDEN) if l.startswith(prefix + " ")]


MMM = "M1: i, j\nM2: j, k\nM3: k, l\nTOUT: i, l\nORDER: ((M1,M2),M3)\n"

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


def test_parse_paper_network():
    names, labels, tout, order = parse_spec(MMM)
    assert names == ["M1", "M2", "M3"]
    lines = [f"[x] {n} : {' '.join(labels[n])}" for n in names]
    assert lines == [g for g in golden("network") if g.startswith("[x]")]
    assert tout == ["i", "l"]
    want_order = [g for g in golden("network") if g.startswith("ORDER")][0].split(":")[1].strip()
    assert tree_str(parse_order(order, names)) == want_order


def test_set_get_order_roundtrip():
    net = Network(MMM)
    net.set_order(False, "(M2,(M1,M3))")
    assert net.get_order() == golden("order")[0]


def test_ctm_network_parses():
    names, labels, tout, order = parse_spec(CTM)
    assert len(names) == 9 and tout == []
    assert tree_str(parse_order(order, names)) == "((((((((c0,t0),c1),t3),w),t1),c3),t2),c2)"


@pytest.mark.parametrize("bad", [
    "A: i, j\nB: j, k\nTOUT: i\n",                 # open label k missing from TOUT
    "A: i, j\nB: j, k\nC: j, m\nTOUT: i, k, m\n",  # label on three tensors
    "A: i, i\nTOUT:\n",                            # trace on one tensor
    "A: i, j\nB: j, k\nTOUT: i, k\nORDER: (A,C)\n",  # unknown name in ORDER
    "A: i, j\nB: j, k\nTOUT: i, k\nORDER: (A,B\n",   # unbalanced
])
def test_bad_specs_rejected(bad):
    with pytest.raises(NetworkError):
        n, l, t, o = parse_spec(bad)
        if o:
            parse_order(o, n)


def test_optimal_equals_exhaustive():
    """DP with cost capping returns the minimum summed cost over every binary tree."""
    rng = np.random.default_rng(5)
    for trial in range(20):
        n = int(rng.integers(3, 6))
        names = [f"T{i}" for i in range(n)]
        labels = {x: [] for x in names}
        dims = {}
        lab = 0
        for i in range(n):
            for j in range(i + 1, n):
                if rng.random() < 0.6 or j == i + 1:
                    l = f"e{lab}"
                    lab += 1
                    labels[names[i]].append(l)
                    labels[names[j]].append(l)
                    dims[l] = int(rng.integers(2, 9))
            if rng.random() < 0.5:
                l = f"o{lab}"
                lab += 1
                labels[names[i]].append(l)
                dims[l] = int(rng.integers(2, 9))
        tree, cost = optimal_order(names, labels, dims)
        best = min(tree_cost(t, labels, dims)[0] for t in all_trees(names))
        assert cost == best == tree_cost(tree, labels, dims)[0]


def test_heff_optimal_order_and_flops():
    """The chi=512 U(1) case: optimal tree and block-sparse flop count."""
    wl = I.heisenberg_workload(512, 20)
    net, _ = heff.make_heff(wl)
    rec = []
    net.launch(record=rec)
    assert net.get_order() == "(L,(((psi,R),W2),W1))"
    fl = [r["flops"] for r in rec]
    fused = sum(sum(2 * M * K * N for M, K, N in r["tables"]["MKN"].tolist()) for r in rec)
    # the fused products also multiply the few zero-flux blocks an intermediate
    # does not store; useful flops count matched block pairs only
    assert sum(fl) <= fused and (fused - sum(fl)) < 1e-6 * sum(fl)
    assert abs(sum(fl) - 1.897e8) / 1.897e8 < 1e-3


def test_heff_vs_brute_force_and_order_independence():
    """Tiny U(1) H_eff: every one of the 105 binary trees gives the brute-force result."""
    wl = I.heisenberg_workload(4, 3)
    net, T = heff.make_heff(wl, order="((((L,psi),W1),W2),R)")
    ref_bs = net.launch()
    dense = {n: T[n].densify() for n in I.HEFF_NAMES}
    dims = net.dims()
    ref = brute_network(net.labels, net.tout, dense, dims)
    assert np.abs(ref_bs.densify() - ref).max() <= 1e-13 * np.abs(ref).max()
    trees = list(all_trees(list(I.HEFF_NAMES)))
    assert len(trees) == 105
    for t in trees:
        net.set_order(False, tree_str(t))
        out = net.launch().densify()
        assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max()


def test_put_with_label_permutation():
    wl = I.heisenberg_workload(6, 3)
    net, T = heff.make_heff(wl)
    out1 = net.launch().densify()
    Rp = T["R"].permute([2, 0, 1])   # legs now (bp, b, w2)
    net.put("R", Rp, ["bp", "b", "w2"])
    out2 = net.launch().densify()
    assert np.array_equal(out1, out2)


def test_launch_requires_all_put():
    net = Network(MMM)
    with pytest.raises(NetworkError):
        net.launch()


# ------------------------------------------------ block-sparse order search
from oracle.contract import pair_flops  # noqa: E402
from oracle.network import sparse_optimal_order, sparse_pair_cost, sparse_tree_cost  # noqa: E402
from oracle.symtensor import U1, ZN, Symmetry  # noqa: E402
from test_oracle_contract import random_pair  # noqa: E402

SPARSE_SYMS = [(Symmetry(U1),), (Symmetry(U1), Symmetry(U1)), (Symmetry(ZN, 3),)]


@pytest.mark.parametrize("syms", SPARSE_SYMS)
def test_sparse_pair_cost_counts_matched_block_pairs(syms):
    """Operands holding every zero-flux block: the charge-count formula equals the
    2mkn sum over the block pairs the contraction code actually matches."""
    rng = np.random.default_rng(23)
    for trial in range(12):
        ra, rb = int(rng.integers(1, 5)), int(rng.integers(1, 5))
        nk = int(rng.integers(0, min(ra, rb) + 1))
        A, B, pairs = random_pair(rng, syms, ra, rb, nk)
        left = {f"a{i}": b for i, b in enumerate(A.bonds)}
        right = {f"b{j}": b for j, b in enumerate(B.bonds)}
        for i, j in pairs:
            right[f"a{i}"] = right.pop(f"b{j}")
        assert sparse_pair_cost(left, right) == pair_flops(A, B, pairs)


def test_sparse_tree_cost_bounds_and_near_optimal():
    """Intermediates may lack some zero-flux blocks, so for every one of the 105
    trees the sector count bounds the flops the contraction records from above;
    the tree it selects records within 2% of the cheapest tree found by trying all."""
    net, _ = heff.make_heff(I.heisenberg_workload(16, 6))
    bonds = {n: list(net.tensors[n].bonds) for n in net.names}
    recorded = {}
    for t in all_trees(list(net.names)):
        net.set_order(False, tree_str(t))
        rec = []
        net.launch(record=rec)
        recorded[tree_str(t)] = sum(r["flops"] for r in rec)
        assert recorded[tree_str(t)] <= sparse_tree_cost(t, net.labels, bonds)
    tree, cost = sparse_optimal_order(net.names, net.labels, bonds)
    assert recorded[tree_str(tree)] <= 1.02 * min(recorded.values())


def test_sparse_order_beats_dense_order_on_heff():
    """chi=512 U(1) H_eff: the sector-counted search contracts the two MPO tensors
    first; by the flops actually recorded that order is cheaper than the dense optimum."""
    wl = I.heisenberg_workload(512, 20)
    net, _ = heff.make_heff(wl)
    bonds = {n: list(net.tensors[n].bonds) for n in net.names}
    tree, cost = sparse_optimal_order(net.names, net.labels, bonds)
    assert tree_str(tree) == "(L,((psi,R),(W1,W2)))"
    flops = {}
    for order in ["(L,((psi,R),(W1,W2)))", "(L,(((psi,R),W2),W1))"]:
        net.set_order(False, order)
        rec = []
        net.launch(record=rec)
        flops[order] = sum(r["flops"] for r in rec)
    assert flops["(L,((psi,R),(W1,W2)))"] < flops["(L,(((psi,R),W2),W1))"]
    assert flops["(L,((psi,R),(W1,W2)))"] <= cost


# Sec. 8.4 listing "code:peps_network": the 11-tensor PEPS expectation value (comment line and
# names with '*' as printed).
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


def test_peps_network_of_ones_counts_its_edges():
    """All-ones tensors of dimension 2 (the listing "code:peps_contraction"): the scalar is
    2^(number of distinct labels), every label being summed over exactly once."""
    from oracle.symtensor import BlockTensor, Bond
    names, labels, tout, order = parse_spec(PEPS)
    assert len(names) == 11 and tout == []
    edges = {l for n in names for l in labels[n]}
    assert len(edges) == 24
    net = Network(PEPS)
    for n in names:
        bonds = [Bond.make(0, [((), 2)]) for _ in labels[n]]
        net.put(n, BlockTensor(bonds, {tuple(0 for _ in bonds): np.ones((2,) * len(bonds))}))
    net.set_order(True)
    out = net.launch()
    assert float(out.blocks[()].reshape(-1)[0]) == 2.0 ** 24
