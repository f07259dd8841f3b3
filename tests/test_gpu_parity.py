"""GPU parity: the sm_103a library (through the C-ABI) against the CPU oracle.

Integer tables must match bit-exactly; FP64 results to relative Frobenius
error <= 1e-12 (the accumulation order differs; the oracle sums in numpy).
"""
import math
import re

import numpy as np
import pytest

import tnx_inputs as I
from oracle.brute import exact_environments, heisenberg_dense
from oracle.lanczos import lanczos as oracle_lanczos
from oracle.symtensor import BlockTensor

from gpu_harness import lib_heff, oracle_heff, rel_fro

pytestmark = pytest.mark.gpu

TOL_F64 = 1e-12

WORKLOADS = {
    "u1_chi16": lambda: I.heisenberg_workload(16, 6),
    "u1_chi40_ragged": lambda: I.heisenberg_workload(40, 9),
    "u1_chi512": lambda: I.heisenberg_workload(512, 20),
    "dense_chi32": lambda: I.dense_workload(32),
    "hubbard_chi64": lambda: I.hubbard_workload(64),
    "hubbard_chi128": lambda: I.hubbard_workload(128),
}


@pytest.fixture(scope="module")
def ctx():
    import paper_2401_01921_gb300 as tnx
    from paper_2401_01921_gb300 import build
    build.build()
    c = tnx.Context(0)
    yield c


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_tables_bit_exact(ctx, name):
    wl = WORKLOADS[name]()
    net, T, B = lib_heff(ctx, wl)
    onet, _ = oracle_heff(wl)
    rec = []
    onet.launch(record=rec)
    assert net.get_order() == onet.get_order()
    assert net.nsteps() == len(rec)
    for s, r in enumerate(rec):
        t = net.step_tables(s)
        o = r["tables"]
        assert np.array_equal(t["charges"], o["charges"].astype(np.int32)), f"step {s} charges"
        assert np.array_equal(t["MKN"], o["MKN"]), f"step {s} MKN"
        assert np.array_equal(t["amap"], o["amap"]), f"step {s} amap"
        assert np.array_equal(t["bmap"], o["bmap"]), f"step {s} bmap"
    assert net.flops() == sum(r["flops"] for r in rec)


@pytest.mark.parametrize("name", list(WORKLOADS))
def test_apply_parity_f64(ctx, name):
    wl = WORKLOADS[name]()
    net, T, B = lib_heff(ctx, wl)
    out = net.launch(B["psi"])
    onet, _ = oracle_heff(wl)
    ref = onet.launch()
    err = rel_fro(out.block_dict(), ref)
    assert err <= TOL_F64, err


def test_apply_parity_f64_chi2048_sector_scaled(ctx):
    """chi = 2048, 41 sectors, per-sector 10^U(-3,0) scaling: full-size parity."""
    wl = I.heisenberg_workload(2048, 40, sector_scale=True)
    net, T, B = lib_heff(ctx, wl)
    out = net.launch(B["psi"])
    onet, _ = oracle_heff(wl)
    ref = onet.launch()
    assert rel_fro(out.block_dict(), ref) <= TOL_F64


@pytest.mark.parametrize("prec", ["f64", "split_bf16"])
def test_relayout_bands(ctx, capfd, monkeypatch, prec):
    """Blocks sharing the rows of a narrow matrix are planned as bands for the
    fused MPO step: its packed operand (destination rows of <= 16 columns) and
    the last step's operand read from its output (source rows of <= 64
    columns).  Ragged sector sizes give ragged tiles; the apply must still match
    the oracle."""
    monkeypatch.setenv("TNX_DEBUG_PLAN", "1")
    wl = I.heisenberg_workload(512, 20)
    order = "(L,((psi,R),(W1,W2)))"
    net, T, B = lib_heff(ctx, wl, order=order, prec=prec)
    out = net.launch(B["psi"])
    err = capfd.readouterr().err
    bands = [int(m) for m in re.findall(r"(\d+) band tiles", err)]
    assert sum(1 for b in bands if b > 0) >= 2, err
    onet, _ = oracle_heff(wl, order=order)
    ref = onet.launch()
    tol = TOL_F64 if prec == "f64" else 1e-10   # split precision: the bound of the split-GEMM tests
    assert rel_fro(out.block_dict(), ref) <= tol


@pytest.mark.parametrize("order, mode", [("(L,((psi,R),(W1,W2)))", "scattered into the next operand"),
                                         ("((((L,psi),W1),W2),R)", "written to C")])
def test_fused_skinny_steps(ctx, capfd, monkeypatch, order, mode):
    """MPO steps (every charge group K <= 16) run as one gather-product-scatter
    kernel: in the block-sparse optimal order the output goes straight into the
    last step's operand; in the chain order the W1 step's output is read by a
    fused step again and is written to C.  Both must match the oracle.  (Steps
    whose sectors are so small that the tiles stay nearly empty run unfused.)"""
    monkeypatch.setenv("TNX_DEBUG_PLAN", "1")
    wl = I.heisenberg_workload(512, 20)
    net, T, B = lib_heff(ctx, wl, order=order)
    out = net.launch(B["psi"])
    err = capfd.readouterr().err
    assert "fused skinny" in err and mode in err, err
    onet, _ = oracle_heff(wl, order=order)
    assert rel_fro(out.block_dict(), onet.launch()) <= TOL_F64


def test_launch_into_reuses_plan_and_tracks_new_data(ctx):
    import paper_2401_01921_gb300 as tnx
    wl = I.heisenberg_workload(40, 9)
    net, T, B = lib_heff(ctx, wl)
    out = tnx.Tensor(ctx, B["psi"])
    net.launch_into(out)
    first = out.download()
    T["psi"].scale(-2.0)
    net.launch_into(out)
    assert np.allclose(out.download(), -2.0 * first, rtol=1e-14, atol=0)


def test_explicit_orders_agree(ctx):
    wl = I.heisenberg_workload(16, 6)
    onet, _ = oracle_heff(wl)
    ref = onet.launch()
    for order in ["((((L,psi),W1),W2),R)", "(L,(((psi,R),W2),W1))", "((L,W1),((psi,W2),R))", "(((L,psi),(W1,W2)),R)"]:
        net, T, B = lib_heff(ctx, wl, order=order)
        assert net.get_order() == order
        assert rel_fro(net.launch(B["psi"]).block_dict(), ref) <= TOL_F64


def test_lanczos_parity_dense(ctx):
    """20-step Lanczos on the symmetrised dense chi=32 H_eff: library vs oracle."""
    import paper_2401_01921_gb300 as tnx
    wl = I.dense_workload(32)
    net, T, B = lib_heff(ctx, wl, symmetric=True)
    evec = tnx.Tensor(ctx, B["psi"])
    lam, k = tnx.lanczos(net, "psi", T["psi"], 20, evec)
    onet, OT = oracle_heff(wl, symmetric=True)
    from oracle import heff as oheff
    op = oheff.flat_apply(onet, OT["psi"])
    olam, ox, *_ , ok = oracle_lanczos(op, OT["psi"].flat(), 20)
    assert k == ok == 20
    assert abs(lam - olam) <= 1e-10 * abs(olam)
    assert np.linalg.norm(evec.download() - ox) <= 1e-8


def test_lanczos_parity_u1_chi512(ctx):
    import paper_2401_01921_gb300 as tnx
    wl = I.heisenberg_workload(512, 20)
    net, T, B = lib_heff(ctx, wl, symmetric=True)
    lam, k = tnx.lanczos(net, "psi", T["psi"], 20)
    onet, OT = oracle_heff(wl, symmetric=True)
    from oracle import heff as oheff
    olam, *_ = oracle_lanczos(oheff.flat_apply(onet, OT["psi"]), OT["psi"].flat(), 20)
    assert abs(lam - olam) <= 1e-10 * abs(olam)


@pytest.mark.parametrize("k,energy", [(1, -(3 + 2 * math.sqrt(3)) / 4), (2, None), (3, None)])
def test_lanczos_exact_environment_ground_energy(ctx, k, energy):
    """H_eff with exact environments of 2k+2 sites: Lanczos gives the ED ground energy."""
    import paper_2401_01921_gb300 as tnx
    from paper_2401_01921_gb300.heff import build_network
    mpo = I.heisenberg_mpo()
    env = exact_environments(mpo, k, k, lambda s: (sum(1 if x == 0 else -1 for x in s),))
    Ls, Rs, P, M = env["left_sectors"], env["right_sectors"], I.SPIN_PHYS, mpo.bond_sectors
    Wg = mpo.W_grouped()
    tensors = {
        "L": ([(I.OUT, Ls), (I.OUT, M), (I.IN, Ls)], lambda c: env["L"][c[0], c[1], c[2]]),
        "psi": ([(I.IN, Ls), (I.IN, P), (I.IN, P), (I.OUT, Rs)],
                lambda c: I.normal_at(9, 0, ((c[0] * 2 + c[1]) * 2 + c[2]) * 4096 + c[3])),
        "W1": ([(I.IN, M), (I.IN, P), (I.OUT, P), (I.OUT, M)], lambda c: Wg[c[0], c[1], c[2], c[3]]),
        "W2": ([(I.IN, M), (I.IN, P), (I.OUT, P), (I.OUT, M)], lambda c: Wg[c[0], c[1], c[2], c[3]]),
        "R": ([(I.IN, Rs), (I.IN, M), (I.OUT, Rs)], lambda c: env["R"][c[0], c[1], c[2]]),
    }
    net, T, B = build_network(ctx, I.HEFF_SPEC, tensors, 1)
    n = T["psi"].nelem
    lam, _ = tnx.lanczos(net, "psi", T["psi"], min(n, 80))
    e0 = energy if energy is not None else np.linalg.eigvalsh(heisenberg_dense(2 * k + 2))[0]
    assert abs(lam - e0) < 1e-10


# --------------------------------------------------------------- edge cases
def _u1_bond(ctx, d, secs):
    import paper_2401_01921_gb300 as tnx
    return tnx.Bond(ctx, d, [((q,), g) for q, g in secs], [tnx.U1])


def test_paper_four_blocks_on_device(ctx):
    import paper_2401_01921_gb300 as tnx
    a = _u1_bond(ctx, tnx.BD_IN, [(1, 1), (-1, 1)])
    c = _u1_bond(ctx, tnx.BD_OUT, [(2, 1), (0, 2), (-2, 1)])
    t = tnx.Tensor(ctx, [a, a, c])
    qn, sh, off = t.blocks()
    assert qn.tolist() == [[0, 0, 0], [0, 1, 1], [1, 0, 1], [1, 1, 2]]
    assert sh.tolist() == [[1, 1, 1], [1, 1, 2], [1, 1, 2], [1, 1, 1]]
    assert off.tolist() == [0, 1, 3, 5]


def test_error_codes(ctx):
    import paper_2401_01921_gb300 as tnx
    a = _u1_bond(ctx, tnx.BD_IN, [(1, 1), (-1, 1)])
    b = _u1_bond(ctx, tnx.BD_OUT, [(1, 1), (-1, 1)])
    t = tnx.Tensor(ctx, [a, b])
    with pytest.raises(tnx.TnxError) as e:
        t.add_scalar(1.0)
    assert e.value.name == "TNX_ERR_SYMMETRY"
    with pytest.raises(tnx.TnxError) as e:
        t.put_block([0, 1], np.ones(1))
    assert e.value.name == "TNX_ERR_NO_BLOCK"
    # contracting two IN legs is refused
    net = tnx.Network(ctx, "A: i, j\nB: j, k\nTOUT: i, k\n")
    net.put("A", t)                          # A's j is OUT
    net.put("B", tnx.Tensor(ctx, [b, a]))    # B's j is OUT too
    with pytest.raises(tnx.TnxError) as e:
        net.launch([a, a])
    assert e.value.name == "TNX_ERR_BOND_MISMATCH"
    with pytest.raises(tnx.TnxError) as e:
        tnx.Network(ctx, "A: i, j\nB: j, k\nTOUT: i\n")
    assert e.value.name == "TNX_ERR_NETWORK"
    net2 = tnx.Network(ctx, "A: i, j\nB: j, k\nTOUT: i, k\n")
    with pytest.raises(tnx.TnxError) as e:
        net2.launch([a, b])
    assert e.value.name == "TNX_ERR_NETWORK"


def _rand_tensor(ctx, bonds, seed):
    import paper_2401_01921_gb300 as tnx
    t = tnx.Tensor(ctx, bonds)
    rng = np.random.default_rng(seed)
    t.upload(rng.standard_normal(t.nelem))
    return t


def _oracle_tensor(lib_t, syms):
    from oracle.symtensor import Bond as OB
    ob = [OB.make(b.dir, b.sectors, syms) for b in lib_t.bonds]
    T = BlockTensor(ob, {})
    for k, v in lib_t.block_dict().items():
        T.blocks[k] = v.copy()
    return T


def test_scalar_output_outer_product_and_permuted_put(ctx):
    import paper_2401_01921_gb300 as tnx
    from oracle.network import Network as ONet
    from oracle.symtensor import Symmetry, U1
    syms = (Symmetry(U1),)
    i = _u1_bond(ctx, tnx.BD_IN, [(0, 2), (1, 3), (-1, 1)])
    o = _u1_bond(ctx, tnx.BD_OUT, [(0, 2), (1, 3), (-1, 1)])
    A = _rand_tensor(ctx, [i, o], 1)
    Bt = _rand_tensor(ctx, [i, o], 2)
    # full contraction to a scalar
    net = tnx.Network(ctx, "A: x, y\nB: y, x\nTOUT:\n")
    net.put("A", A)
    net.put("B", Bt)
    s = net.launch([])
    on = ONet("A: x, y\nB: y, x\nTOUT:\n")
    on.put("A", _oracle_tensor(A, syms))
    on.put("B", _oracle_tensor(Bt, syms))
    ref = on.launch()
    assert abs(s.download()[0] - ref.blocks[()].reshape(-1)[0]) <= 1e-13 * abs(ref.blocks[()]).max()
    # outer product (no shared label)
    net = tnx.Network(ctx, "A: a, b\nB: c, d\nTOUT: a, b, c, d\n")
    net.put("A", A)
    net.put("B", Bt)
    out = net.launch([i, o, i, o])
    on = ONet("A: a, b\nB: c, d\nTOUT: a, b, c, d\n")
    on.put("A", _oracle_tensor(A, syms))
    on.put("B", _oracle_tensor(Bt, syms))
    assert rel_fro(out.block_dict(), on.launch()) <= TOL_F64
    # put with a leg permutation: B's legs given as (y, x)
    net = tnx.Network(ctx, "A: x, y\nB: y, z\nTOUT: x, z\n")
    net.put("A", A)
    Bp = _rand_tensor(ctx, [o, i], 3)       # legs (z OUT, y IN): realises B's (y, z) permuted
    net.put("B", Bp, ["z", "y"])
    out = net.launch([i, o])
    on = ONet("A: x, y\nB: y, z\nTOUT: x, z\n")
    on.put("A", _oracle_tensor(A, syms))
    on.put("B", _oracle_tensor(Bp, syms), ["z", "y"])
    assert rel_fro(out.block_dict(), on.launch()) <= TOL_F64


def test_zn_symmetry_contraction(ctx):
    import paper_2401_01921_gb300 as tnx
    from oracle.network import Network as ONet
    from oracle.symtensor import Symmetry, ZN
    syms = (Symmetry(ZN, 3),)
    mk = lambda d: tnx.Bond(ctx, d, [((0,), 2), ((1,), 3), ((2,), 1)], [(tnx.ZN, 3)])
    A = _rand_tensor(ctx, [mk(tnx.BD_IN), mk(tnx.BD_IN), mk(tnx.BD_OUT)], 4)
    Bt = _rand_tensor(ctx, [mk(tnx.BD_IN), mk(tnx.BD_OUT), mk(tnx.BD_OUT)], 5)
    spec = "A: a, b, c\nB: c, d, e\nTOUT: a, b, d, e\n"
    net = tnx.Network(ctx, spec)
    net.put("A", A)
    net.put("B", Bt)
    out = net.launch([A.bonds[0], A.bonds[1], Bt.bonds[1], Bt.bonds[2]])
    on = ONet(spec)
    on.put("A", _oracle_tensor(A, syms))
    on.put("B", _oracle_tensor(Bt, syms))
    assert rel_fro(out.block_dict(), on.launch()) <= TOL_F64


def test_tensor_without_blocks(ctx):
    """Bonds whose charges can never balance: no stored block; contraction gives zeros."""
    import paper_2401_01921_gb300 as tnx
    i = _u1_bond(ctx, tnx.BD_IN, [(1, 2)])
    o = _u1_bond(ctx, tnx.BD_OUT, [(3, 2)])
    A = tnx.Tensor(ctx, [i, o])
    assert A.nblocks == 0 and A.nelem == 0
    ii = _u1_bond(ctx, tnx.BD_IN, [(3, 2)])
    Bt = _rand_tensor(ctx, [ii, o], 6)
    net = tnx.Network(ctx, "A: x, y\nB: y, z\nTOUT: x, z\n")
    net.put("A", A)
    net.put("B", Bt)
    out = net.launch([i, o])
    assert out.nblocks == 0


def test_graph_and_profiler_leave_no_stale_cuda_error(ctx):
    """Profiled, graph-captured launches and Lanczos solves: figures come back and torch keeps working."""
    import torch
    import paper_2401_01921_gb300 as tnx
    wl = I.heisenberg_workload(40, 9)
    net, T, B = lib_heff(ctx, wl, symmetric=True)
    out = tnx.Tensor(ctx, B["psi"])
    ctx.profile(True)
    net.launch_into(out)
    net.launch_into(out)
    lam, k = tnx.lanczos(net, "psi", T["psi"], 8)
    prof = ctx.profile_read()
    ctx.profile(False)
    assert prof["gemm"][1] > 0 and prof["gemm"][0] > 0
    assert prof["vector"][1] > 0
    x = torch.zeros(1024, device="cuda")
    x.add_(1.0)
    torch.cuda.synchronize()
    assert float(x.sum()) == 1024.0


@pytest.mark.parametrize("name", ["u1_chi16", "u1_chi512", "dense_chi32", "hubbard_chi64"])
def test_sparse_order_search(ctx, name):
    """Block-sparse-cost search: the library's tree has the oracle's minimum sector
    count over all 105 trees, and its result matches the oracle in that order."""
    from oracle.network import parse_order, sparse_optimal_order, sparse_tree_cost
    wl = WORKLOADS[name]()
    net, T, B = lib_heff(ctx, wl, order="sparse")
    got = net.get_order()
    onet, _ = oracle_heff(wl)
    bonds = {n: list(onet.tensors[n].bonds) for n in onet.names}
    _, best = sparse_optimal_order(onet.names, onet.labels, bonds)
    assert sparse_tree_cost(parse_order(got, onet.names), onet.labels, bonds) == best
    if name == "u1_chi512":
        assert got == "(L,((psi,R),(W1,W2)))"
    onet.set_order(False, got)
    assert rel_fro(net.launch(B["psi"]).block_dict(), onet.launch()) <= TOL_F64


def test_launch_counter_counts_graph_replays(ctx):
    """Applies replayed from a CUDA graph count their kernels on every replay, and
    the capture itself counts nothing."""
    import paper_2401_01921_gb300 as tnx
    wl = I.heisenberg_workload(40, 9)
    net, T, B = lib_heff(ctx, wl, prec="split_bf16")
    out = tnx.Tensor(ctx, B["psi"])
    net.launch_into(out)   # plan + capture + first replay
    ctx.sync()
    n0 = tnx.kernel_launches()
    net.launch_into(out)
    ctx.sync()
    n1 = tnx.kernel_launches()
    net.launch_into(out)
    net.launch_into(out)
    ctx.sync()
    n2 = tnx.kernel_launches()
    per_apply = n1 - n0
    assert per_apply >= 2 * net.nsteps()   # at least a relayout and a product per step
    assert n2 - n1 == 2 * per_apply
