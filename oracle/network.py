"""Oracle: Network blueprint, PutUniTensor, ORDER and the optimal-order search.

Sec. 8 ("Network") of arXiv 2401.01921:

* 8.1: a network is a text blueprint: one line per tensor ``NAME: l1, l2, ...``
  with dummy labels, ``TOUT: ...`` listing the open labels in output order
  (``;`` may separate row and column labels; an empty TOUT means a scalar),
  and ``ORDER: ...`` a parenthesised binary contraction tree over the names.
  Labels appearing twice are summed over.  An empty ORDER contracts the
  tensors in order of appearance.
* 8.2: PutUniTensor maps the legs of an actual tensor, listed by its own
  labels, onto the dummy labels of the blueprint; Launch contracts and the
  output takes the TOUT order.
* 8.3: setOrder(optimal=True) computes the optimal order from the loaded
  dimensions; getOrder prints the tree, e.g. ``(M2,(M1,M3))``.

Sec. 7: the optimal order is found by the dynamic programming algorithm with
the cost-capping strategy of Pfeifer, Haegeman and Verstraete (PRE 90, 033315,
2014).  Here the cost of a pairwise contraction is the number of
multiply-adds of the dense contraction: the product of the dimensions of all
distinct legs of the two operands.  The DP minimises the summed cost over
binary trees; the cap mu starts at the largest single-tensor size and grows
by a factor 2 (or to the smallest rejected cost, if larger) until a full tree
fits under it.  Ties keep the first split in the enumeration (subsets S1 of S
that contain the lowest member of S, in increasing bitmask order).

Block-sparse search (an addition, for zero-flux block operands): the same
search over trees with each pairwise cost counted over charge sectors
(``sparse_pair_cost``), taken over all binary trees exhaustively.

Parity: the order string round-trip and the printed network are pinned by the
paper's examples; the optimal cost is pinned by exhaustive enumeration of all
binary trees on small networks; the chosen tree among equal-cost ones is a
convention (unpinned), and the contraction result is checked to be
independent of the order (tests/test_oracle_network.py).  The sector count is
pinned by enumerating every block pair of full random tensors and by the
flops recorded when such tensors are actually contracted.
"""
from __future__ import annotations

import math
import re

from .contract import contract_pair
from .symtensor import BlockTensor, combine_charges, zero_charge


class NetworkError(ValueError):
    pass


def parse_spec(text: str):
    """Returns (names, labels per name, tout labels, order string or '')."""
    names, labels, tout, order = [], {}, None, ""
    lines = text.replace(";", ",").split("\n") if isinstance(text, str) else list(text)
    for raw in lines:
        line = raw.strip()
        if not line or line.startswith("#"):      # comment lines, as in the Sec. 8.4 network file
            continue
        if ":" not in line:
            raise NetworkError(f"line without ':' : {line!r}")
        key, rest = line.split(":", 1)
        key = key.strip()
        rest = rest.strip()
        if key == "TOUT":
            tout = [x.strip() for x in rest.split(",") if x.strip()]
        elif key == "ORDER":
            order = rest.replace(" ", "")
        else:
            if key in labels or not re.fullmatch(r"[A-Za-z0-9_\-\.'*]+", key):
                raise NetworkError(f"bad or duplicate tensor name {key!r}")
            labs = [x.strip() for x in rest.split(",") if x.strip()]
            if len(set(labs)) != len(labs):
                raise NetworkError("a label appears twice on one tensor")
            names.append(key)
            labels[key] = labs
    if tout is None:
        raise NetworkError("missing TOUT")
    count = {}
    for n in names:
        for l in labels[n]:
            count[l] = count.get(l, 0) + 1
    if any(c > 2 for c in count.values()):
        raise NetworkError("a label appears on more than two tensors")
    open_labels = [l for l, c in count.items() if c == 1]
    if sorted(open_labels) != sorted(tout):
        raise NetworkError("TOUT must list exactly the open labels")
    return names, labels, tout, order


def parse_order(order: str, names):
    """Parse '((A,B),C)' into nested tuples of names; validates coverage."""
    pos = 0

    def node():
        nonlocal pos
        if pos < len(order) and order[pos] == "(":
            pos += 1
            left = node()
            if pos >= len(order) or order[pos] != ",":
                raise NetworkError("expected ','")
            pos += 1
            right = node()
            if pos >= len(order) or order[pos] != ")":
                raise NetworkError("expected ')'")
            pos += 1
            return (left, right)
        m = re.match(r"[A-Za-z0-9_\-\.'*]+", order[pos:])
        if not m:
            raise NetworkError("expected a tensor name")
        pos += m.end()
        return m.group(0)

    tree = node()
    if pos != len(order):
        raise NetworkError("trailing characters in ORDER")
    leaves = []

    def walk(t):
        if isinstance(t, tuple):
            walk(t[0])
            walk(t[1])
        else:
            leaves.append(t)

    walk(tree)
    if sorted(leaves) != sorted(names) or len(set(leaves)) != len(leaves):
        raise NetworkError("ORDER must name every tensor exactly once")
    return tree


def default_tree(names):
    t = names[0]
    for n in names[1:]:
        t = (t, n)
    return t


def tree_str(t) -> str:
    if isinstance(t, tuple):
        return "(" + tree_str(t[0]) + "," + tree_str(t[1]) + ")"
    return t


def optimal_order(names, labels, dims):
    """DP over subsets with cost capping (Sec. 7; Pfeifer et al. 2014).

    dims: label -> dimension.  Returns (tree, cost).
    """
    n = len(names)
    if n == 1:
        return names[0], 0
    leg_sets = [set(labels[x]) for x in names]
    full = (1 << n) - 1

    def open_legs(mask):
        cnt = {}
        for i in range(n):
            if mask >> i & 1:
                for l in leg_sets[i]:
                    cnt[l] = cnt.get(l, 0) + 1
        # a leg is open for the subset unless both of its ends lie inside it
        return {l for l, c in cnt.items() if c == 1}

    legs = {m: open_legs(m) for m in range(1, full + 1)}

    def pair_cost(m1, m2):
        c = 1
        for l in legs[m1] | legs[m2]:
            c *= dims[l]
        return c

    mu = max(math.prod(dims[l] for l in leg_sets[i]) if leg_sets[i] else 1 for i in range(n))
    while True:
        best = {1 << i: (0, names[i]) for i in range(n)}
        rejected = math.inf
        for size in range(2, n + 1):
            for mask in range(1, full + 1):
                if bin(mask).count("1") != size:
                    continue
                low = mask & (-mask)
                rest = mask ^ low
                cand = None
                sub = rest
                # enumerate S1 = low | s for s subset of rest, s != rest, increasing
                subs = []
                s = 0
                while True:
                    subs.append(s)
                    if s == rest:
                        break
                    s = (s - rest) & rest
                for s in subs:
                    m1 = low | s
                    m2 = mask ^ m1
                    if m2 == 0 or m1 not in best or m2 not in best:
                        continue
                    c = best[m1][0] + best[m2][0] + pair_cost(m1, m2)
                    if c > mu:
                        rejected = min(rejected, c)
                        continue
                    if cand is None or c < cand[0]:
                        cand = (c, (best[m1][1], best[m2][1]))
                if cand is not None:
                    best[mask] = cand
        if full in best:
            return best[full][1], best[full][0]
        mu = max(mu * 2, rejected)


def all_trees(items):
    """Every binary tree over the items (for brute-force pins on small networks)."""
    if len(items) == 1:
        yield items[0]
        return
    first, rest = items[0], items[1:]
    n = len(rest)
    for m in range(0, 1 << n):
        left = [first] + [rest[i] for i in range(n) if m >> i & 1]
        right = [rest[i] for i in range(n) if not m >> i & 1]
        if not right:
            continue
        for tl in all_trees(left):
            for tr in all_trees(right):
                yield (tl, tr)


def tree_cost(tree, labels, dims):
    """Summed pairwise dense cost of a tree; returns (cost, open label set)."""
    if not isinstance(tree, tuple):
        return 0, set(labels[tree])
    c1, l1 = tree_cost(tree[0], labels, dims)
    c2, l2 = tree_cost(tree[1], labels, dims)
    c = 1
    for l in l1 | l2:
        c *= dims[l]
    return c1 + c2 + c, l1 ^ l2


class Network:
    """Blueprint + put tensors + order (Sec. 8)."""

    def __init__(self, spec: str):
        self.names, self.labels, self.tout, order = parse_spec(spec)
        self.tree = parse_order(order, self.names) if order else default_tree(self.names)
        self.optimal = False
        self.tensors: dict[str, BlockTensor] = {}

    def put(self, name: str, T: BlockTensor, labels=None):
        """PutUniTensor (Sec. 8.2): labels[i] is the blueprint label of leg i of T
        (None: T's legs already follow the blueprint line).  The tensor is held
        in blueprint leg order."""
        if name not in self.labels:
            raise NetworkError(f"unknown tensor {name}")
        want = self.labels[name]
        if labels is None:
            labels = list(want)
        if len(labels) != T.rank or sorted(labels) != sorted(want):
            raise NetworkError("labels must be a permutation of the blueprint labels")
        perm = [list(labels).index(l) for l in want]
        self.tensors[name] = T if perm == list(range(T.rank)) else T.permute(perm)

    def set_order(self, optimal: bool, order: str | None = None):
        self.optimal = optimal
        if not optimal:
            if not order:
                raise NetworkError("an explicit order is required with optimal=False")
            self.tree = parse_order(order.replace(" ", ""), self.names)

    def get_order(self) -> str:
        return tree_str(self.tree)

    def dims(self):
        d = {}
        for n in self.names:
            T = self.tensors[n]
            for l, b in zip(self.labels[n], T.bonds):
                d[l] = b.dim
        return d

    def launch(self, record=None) -> BlockTensor:
        """Contract along the tree; output legs in TOUT order (Sec. 8.2)."""
        for n in self.names:
            if n not in self.tensors:
                raise NetworkError(f"tensor {n} not put")
        if self.optimal:
            self.tree, _ = optimal_order(self.names, self.labels, self.dims())

        def run(t):
            if not isinstance(t, tuple):
                return self.tensors[t], list(self.labels[t])
            A, la = run(t[0])
            B, lb = run(t[1])
            pairs = [(la.index(l), lb.index(l)) for l in la if l in lb]
            if record is not None:
                from .contract import fused_tables, pair_flops
                record.append({"A": A, "B": B, "pairs": pairs,
                               "tables": fused_tables(A, B, pairs), "flops": pair_flops(A, B, pairs)})
            C = contract_pair(A, B, pairs)
            ka = [p[0] for p in sorted(pairs)]
            kb = [p[1] for p in sorted(pairs)]
            lc = [l for i, l in enumerate(la) if i not in ka] + [l for j, l in enumerate(lb) if j not in kb]
            return C, lc

        C, lc = run(self.tree)
        perm = [lc.index(l) for l in self.tout]
        return C.permute(perm)


def full_output(C: BlockTensor) -> BlockTensor:
    """The same tensor with every zero-flux block of its bonds stored (zeros where absent)."""
    F = BlockTensor(C.bonds)
    for q, b in C.blocks.items():
        F.blocks[q] = b.copy()
    return F


# ------------------------------------------------ block-sparse order search
# An addition to the paper's dense search (for operands stored as zero-flux
# blocks): the cost of a pairwise contraction is counted over charge sectors.
# Every intermediate is taken to hold all zero-flux blocks of its open legs;
# a contraction costs 2 m k n flops for each combination of sectors of the
# left free legs (m index combinations), the contracted legs (k) and the right
# free legs (n) under which both operands have zero flux.

def _leg_bonds(tree, labels, bonds):
    """Open labels of a subtree with the bond each label has inside it."""
    if not isinstance(tree, tuple):
        return dict(zip(labels[tree], bonds[tree]))
    left = _leg_bonds(tree[0], labels, bonds)
    right = _leg_bonds(tree[1], labels, bonds)
    out = {l: b for l, b in left.items() if l not in right}
    out.update({l: b for l, b in right.items() if l not in left})
    return out


def charge_counts(bond_list, syms):
    """Number of index combinations of the given legs per total signed charge."""
    counts = {zero_charge(syms): 1}
    for b in bond_list:
        nxt = {}
        for q, c in counts.items():
            for k, (_, d) in enumerate(b.sectors):
                q2 = combine_charges(syms, q, b.signed(k))
                nxt[q2] = nxt.get(q2, 0) + c * d
        counts = nxt
    return counts


def sparse_pair_cost(left: dict, right: dict) -> int:
    """Flops of contracting two operands holding every zero-flux block of their
    legs; left/right: label -> bond (with the direction it has in that operand)."""
    shared = [l for l in left if l in right]
    fa = [left[l] for l in left if l not in right]
    fb = [right[l] for l in right if l not in left]
    kb = [left[l] for l in shared]
    if not (fa or fb or kb):
        return 0
    syms = (fa or fb or kb)[0].syms
    ca, ck, cb = charge_counts(fa, syms), charge_counts(kb, syms), charge_counts(fb, syms)
    cost = 0
    for g, nk in ck.items():
        # left operand: free charge + g = 0; right operand sees -g on the shared legs
        need_a = tuple(s.reverse(x) for s, x in zip(syms, g))
        cost += 2 * ca.get(need_a, 0) * nk * cb.get(g, 0)
    return cost


def sparse_tree_cost(tree, labels, bonds) -> int:
    """Summed block-sparse cost of a tree; bonds: name -> bonds in label order."""
    if not isinstance(tree, tuple):
        return 0
    return (sparse_tree_cost(tree[0], labels, bonds) + sparse_tree_cost(tree[1], labels, bonds)
            + sparse_pair_cost(_leg_bonds(tree[0], labels, bonds), _leg_bonds(tree[1], labels, bonds)))


def sparse_optimal_order(names, labels, bonds):
    """Minimum block-sparse cost over every binary tree (exhaustive; small networks).
    Returns (tree, cost); the first tree met wins ties."""
    best = None
    for t in all_trees(list(names)):
        c = sparse_tree_cost(t, labels, bonds)
        if best is None or c < best[1]:
            best = (t, c)
    return best
