"""GPU parity of the reduced / split-precision products against the FP64 oracle.

Split BF16 / FP16 (Ozaki-style slices on tcgen05, exact FP32 chunks, int64
recombination): relative Frobenius error <= 1e-10 on every workload, and
bit-exact on integer inputs whose slices carry them exactly.  FP32: the error
is reported, bounded loosely (1e-5).  TF32 (one pass on the tensor cores):
every output entry within the rounding bound of its products, from the
oracle's contraction of the absolute values.
"""
import numpy as np
import pytest

import tnx_inputs as I

from gpu_harness import lib_heff, max_block_rel, oracle_heff, rel_fro

pytestmark = pytest.mark.gpu

TOL_SPLIT = 1e-10

WORKLOADS = {
    "u1_chi40_ragged": lambda: I.heisenberg_workload(40, 9),
    "u1_chi512": lambda: I.heisenberg_workload(512, 20),
    "u1_chi2048_scaled": lambda: I.heisenberg_workload(2048, 40, sector_scale=True),
    "dense_chi32": lambda: I.dense_workload(32),
    "hubbard_chi128": lambda: I.hubbard_workload(128),
}


@pytest.fixture(scope="module")
def ctx():
    import paper_2401_01921_gb300 as tnx
    from paper_2401_01921_gb300 import build
    build.build()
    return tnx.Context(0)


_REF = {}


def reference(name):
    if name not in _REF:
        onet, _ = oracle_heff(WORKLOADS[name]())
        _REF[name] = onet.launch()
    return _REF[name]


@pytest.mark.parametrize("prec", ["split_bf16", "split_f16"])
@pytest.mark.parametrize("name", list(WORKLOADS))
def test_split_parity(ctx, name, prec):
    wl = WORKLOADS[name]()
    net, T, B = lib_heff(ctx, wl, prec=prec)
    out = net.launch(B["psi"])
    err = rel_fro(out.block_dict(), reference(name))
    print(f"{name} {prec}: rel err {err:.3e}")
    assert err <= TOL_SPLIT, err


@pytest.mark.parametrize("name", ["u1_chi40_ragged", "u1_chi512", "hubbard_chi128"])
def test_output_relayout_folded_into_the_split_epilogue(ctx, name):
    """Under split precision the last product's epilogue stores the output itself (no output-relayout
    launch), in the benched order as in the dense one; FP64 keeps the relayout.  Results stay equal
    to the oracle's within the split bound."""
    wl = WORKLOADS[name]()
    for order in (None, "sparse"):
        for prec, folded in (("split_bf16", True), ("f64", False)):
            net, T, B = lib_heff(ctx, wl, prec=prec, order=order)
            out = net.launch(B["psi"])
            ctx.profile(True)
            net.launch_into(out)
            prof = ctx.profile_read()
            ctx.profile(False)
            assert (prof["final"][1] == 0) == folded, (name, order, prec, prof["final"])
            onet, _ = oracle_heff(wl, order=net.get_order())
            err = rel_fro(out.block_dict(), onet.launch())
            assert err <= (TOL_SPLIT if folded else 1e-12), (name, order, prec, err)


def test_f32_error_reported(ctx):
    wl = WORKLOADS["u1_chi512"]()
    net, T, B = lib_heff(ctx, wl, prec="f32")
    err = rel_fro(net.launch(B["psi"]).block_dict(), reference("u1_chi512"))
    print(f"u1_chi512 f32: rel err {err:.3e}")
    assert 1e-12 < err < 1e-5


def abs_network(wl, order=None):
    """The oracle's H_eff with every tensor replaced by its entrywise absolute value:
    sum |L||psi||W||W||R|, the scale of the rounding error of each output entry."""
    from oracle.symtensor import BlockTensor
    onet, OT = oracle_heff(wl, order=order)
    for n, t in OT.items():
        onet.put(n, BlockTensor(t.bonds, {q: np.abs(b) for q, b in t.blocks.items()}))
    return onet.launch()


@pytest.mark.parametrize("name", ["u1_chi40_ragged", "u1_chi512", "hubbard_chi128"])
def test_tf32_within_rounding_bound(ctx, name):
    """TF32 products round each operand to 11 significant bits (relative 2^-12 each) and sum in FP32
    per K chunk; with two tensor-core products on the path (psi*R-like and L*Y-like steps; the MPO
    products stay FP64) every entry's error is below 2^-9 * (sum of |terms|), and it is a real TF32
    error (far above FP32's)."""
    wl = WORKLOADS[name]()
    net, T, B = lib_heff(ctx, wl, prec="tf32")
    order = net.get_order()
    got = net.launch(B["psi"]).block_dict()
    onet, _ = oracle_heff(wl, order=order)
    ref = onet.launch()
    scale = abs_network(wl, order=order)
    worst = 0.0
    for q, b in ref.blocks.items():
        d = np.abs(got.get(q, 0.0) - b)
        worst = max(worst, float(np.max(d / np.maximum(scale.blocks[q], 1e-300))))
    err = rel_fro(got, ref)
    print(f"{name} tf32: rel err {err:.3e}, worst |err| / sum|terms| {worst:.3e}")
    assert worst <= 2.0 ** -9, worst
    assert 1e-6 < err < 2e-3, err


@pytest.mark.parametrize("chi,n", [(40, 9), (512, 20)])
@pytest.mark.parametrize("prec", ["split_bf16", "split_f16"])
def test_split_exact_on_integers(ctx, prec, chi, n):
    """Integer entries in [-3, 3]: every slice is exact, so the split products equal the FP64 ones bit for bit
    (chi=512 has charge groups with K up to 434, summed exactly in one FP32 level chunk)."""
    import paper_2401_01921_gb300 as tnx
    from paper_2401_01921_gb300.heff import build_network
    wl = I.heisenberg_workload(chi, n)
    bonds = I.heff_bonds(wl)

    def ints(name):
        base = I.heff_value_fn(wl, name)
        if name in ("W1", "W2"):
            return lambda c: np.round(2 * base(c))        # MPO entries 0, +-1/2, 1 -> 0, +-1, 2
        return lambda c: np.clip(np.round(base(c) * 1.5), -3, 3)

    res = {}
    for p in ("f64", prec):
        tensors = {n: (bonds[n], ints(n)) for n in I.HEFF_NAMES}
        net, T, B = build_network(ctx, I.HEFF_SPEC, tensors, wl.nsym, prec=p)
        res[p] = net.launch(B["psi"]).download()
    assert np.abs(res["f64"]).max() > 100
    assert np.array_equal(res["f64"], res[prec])


@pytest.mark.parametrize("K", [100, 200, 300, 700, 2000])
@pytest.mark.parametrize("prec", ["split_bf16", "split_f16"])
def test_split_level_sums_at_large_values(ctx, prec, K):
    """C = A B with every entry of row i of A equal to x_i and every entry of column j of B to y_j, where
    |x_i| and |y_j| are m = v 2^-40 times powers of two and v = 63 (2^35 + 2^28 + 2^21): each entry is its own
    row (column) maximum, so its balanced 7-bit digits are (63, 63, 63, 0, 0, 0), every digit product of a
    level adds with the same sign, and no dropped level holds a nonzero term.  The level sums of a 640-long
    chunk reach 3 * 640 * 63^2 = 7.6e6, above the 2^22 that the one-add integer conversion covers, and the
    product is exact: C_ij = K x_i y_j, exact in FP64 (51 significant bits).  K spans one chunk with every
    level bound by 2^22 (100), fewer such levels (200, 300), and several chunks (700, 2000)."""
    import paper_2401_01921_gb300 as tnx
    from paper_2401_01921_gb300.heff import build_network
    M, N = 200, 100
    m = 63.0 * (2.0 ** 35 + 2.0 ** 28 + 2.0 ** 21) * 2.0 ** -40
    x = np.array([(1.0 if i % 3 else -1.0) * m * 2.0 ** (i % 7 - 3) for i in range(M)])
    y = np.array([(-1.0 if j % 4 == 1 else 1.0) * m * 2.0 ** (j % 5 - 2) for j in range(N)])
    reg = lambda n: (tnx.BD_REG, [((), n)])
    tensors = {"A": ([reg(M), reg(K)], lambda c: x[c[0]]), "B": ([reg(K), reg(N)], lambda c: y[c[1]])}
    exact = float(K) * np.outer(x, y)
    for p in ("f64", prec):
        net, T, B = build_network(ctx, "A: i, k\nB: k, j\nTOUT: i, j\nORDER:\n", tensors, 0, prec=p)
        got = net.launch([B["A"][0], B["B"][1]]).download().reshape(M, N)
        assert np.array_equal(got, exact), (p, float(np.abs(got - exact).max()))


def test_split_lanczos(ctx):
    wl = I.heisenberg_workload(512, 20)
    import paper_2401_01921_gb300 as tnx
    lam = {}
    for p in ("f64", "split_bf16"):
        net, T, B = lib_heff(ctx, wl, symmetric=True, prec=p)
        lam[p], _ = tnx.lanczos(net, "psi", T["psi"], 20)
    assert abs(lam["f64"] - lam["split_bf16"]) <= 1e-10 * abs(lam["f64"])


# Per precision: bound on the relative Frobenius error over all stored elements, and on the largest
# relative error of a single block (the 10^U(-3,0) sector scaling makes some blocks 1000x smaller than
# others that share a row of A or a column of B; the K balancing of the split products keeps their bits).
SWEEP_BOUNDS = {"f64": (1e-12, 1e-12), "split_bf16": (TOL_SPLIT, TOL_SPLIT), "split_f16": (TOL_SPLIT, TOL_SPLIT),
                "f32": (1e-5, 1e-3), "tf32": (2e-3, 2e-2)}


def test_precision_sweep_chi2048(ctx):
    """The C3 sweep: chi=2048 U(1) apply with per-sector 10^U(-3,0) scaling, every precision the
    library offers against the FP64 oracle (errors printed; global and worst-block bounds above)."""
    ref = reference("u1_chi2048_scaled")
    for prec, (tol, tol_blk) in SWEEP_BOUNDS.items():
        net, T, B = lib_heff(ctx, WORKLOADS["u1_chi2048_scaled"](), prec=prec)
        got = net.launch(B["psi"]).block_dict()
        err = rel_fro(got, ref)
        blk = max_block_rel(got, ref)
        print(f"u1_chi2048_scaled {prec}: rel err {err:.3e}, worst block {blk:.3e}")
        assert err <= tol, (prec, err)
        assert blk <= tol_blk, (prec, blk)
