"""GPU parity of Dagger, the DMRG environment updates and the block-sparse SVD
(paper Sec. 6.4, Sec. 9.2, Sec. 11) against the CPU oracle, through the C-ABI.

Singular values are unique and compared directly (relative 1e-12 of the
largest); singular vectors are not (signs, rotations inside degenerate
values), so the tests compare the truncated products U S V^dagger with the
oracle's and check that U and V^dagger have orthonormal columns / rows.
"""
import itertools

import numpy as np
import pytest

import tnx_inputs as I
from oracle import dmrg as odmrg
from oracle.brute import exact_environments
from oracle.svd import matrix_blocks, reconstruct, svd_truncate
from oracle.symtensor import IN, OUT, Bond as OB, BlockTensor, Symmetry, U1

from gpu_harness import rel_fro

pytestmark = pytest.mark.gpu

SYM = (Symmetry(U1),)


@pytest.fixture(scope="module")
def ctx():
    import paper_2401_01921_gb300 as tnx
    from paper_2401_01921_gb300 import build
    build.build()
    return tnx.Context(0)


def to_lib(ctx, T: BlockTensor):
    import paper_2401_01921_gb300 as tnx
    bonds = []
    for b in T.bonds:
        syms = [tnx.U1 if s.kind == U1 else (tnx.ZN, s.n) for s in b.syms]
        bonds.append(tnx.Bond(ctx, b.dir, list(b.sectors), syms))
    t = tnx.Tensor(ctx, bonds)
    if t.nelem:
        t.upload(T.flat())
    return t


def to_oracle(t, syms=SYM) -> BlockTensor:
    bonds = [OB.make(b.dir, b.sectors, syms if b.nsym else ()) for b in t.bonds]
    return BlockTensor(bonds, {k: v.copy() for k, v in t.block_dict().items()})


# ------------------------------------------------------------------ dagger / environments
def test_dagger_reverses_bonds_and_keeps_data(ctx):
    a = OB.make(IN, [((1,), 2), ((-1,), 1)], SYM)
    b = OB.make(OUT, [((0,), 3), ((2,), 1)], SYM)
    T = BlockTensor([a, a, b])
    rng = np.random.default_rng(0)
    for q in T.keys():
        T.blocks[q] = rng.standard_normal(T.block_shape(q))
    t = to_lib(ctx, T)
    d = t.dagger()
    assert [x.dir for x in d.bonds] == [OUT, OUT, IN]
    assert np.array_equal(d.download(), t.download())


def _env_net(ctx, spec, tensors, out_bonds, prec="f64"):
    import paper_2401_01921_gb300 as tnx
    net = tnx.Network(ctx, spec)
    for n, t in tensors.items():
        net.put(n, t)
    net.set_order(True)
    net.set_precision(prec)
    return net.launch(out_bonds)


def _random_mps_tensor(a_secs, b_secs, seed):
    T = BlockTensor([OB.make(IN, a_secs, SYM), OB.make(IN, I.SPIN_PHYS, SYM), OB.make(OUT, b_secs, SYM)])
    rng = np.random.default_rng(seed)
    for q in T.keys():
        T.blocks[q] = rng.standard_normal(T.block_shape(q))
    return T


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("split_bf16", 1e-10)])
@pytest.mark.parametrize("chi", [16, 64, 256])
def test_environment_updates_match_the_oracle(ctx, chi, prec, tol):
    """L.A.W.A^dagger and A.W.R.A^dagger with random A and environments (Heisenberg MPO),
    native FP64 and split BF16 products."""
    mpo = I.heisenberg_mpo()
    secs = I.heisenberg_virtual_sectors(chi, 8)
    secs2 = I.heisenberg_virtual_sectors(chi + chi // 2, 9)
    W = odmrg.mpo_tensor(mpo, SYM)
    A = _random_mps_tensor(secs, secs2, 1)
    M = mpo.bond_sectors
    rng = np.random.default_rng(2)
    L = BlockTensor([OB.make(OUT, secs, SYM), OB.make(OUT, M, SYM), OB.make(IN, secs, SYM)])
    for q in L.keys():
        L.blocks[q] = rng.standard_normal(L.block_shape(q))
    R = BlockTensor([OB.make(IN, secs2, SYM), OB.make(IN, M, SYM), OB.make(OUT, secs2, SYM)])
    for q in R.keys():
        R.blocks[q] = rng.standard_normal(R.block_shape(q))
    tA, tW, tL, tR = to_lib(ctx, A), to_lib(ctx, W), to_lib(ctx, L), to_lib(ctx, R)
    tAd = tA.dagger()
    outL = _env_net(ctx, odmrg.ENV_LEFT_SPEC, {"L": tL, "A": tA, "W": tW, "Ad": tAd},
                    [tA.bonds[2], tW.bonds[3], tAd.bonds[2]], prec)
    errL = rel_fro(outL.block_dict(), odmrg.env_left(L, A, W))
    outR = _env_net(ctx, odmrg.ENV_RIGHT_SPEC, {"A": tA, "W": tW, "R": tR, "Ad": tAd},
                    [tA.bonds[0], tW.bonds[0], tAd.bonds[0]], prec)
    errR = rel_fro(outR.block_dict(), odmrg.env_right(R, A, W))
    print(f"environment updates chi={chi} {prec}: left {errL:.3e}, right {errR:.3e}")
    assert errL <= tol and errR <= tol, (errL, errR)


def test_exact_environment_grows_by_one_site_on_the_device(ctx):
    """The (k+1)-site environment from the k-site one and an identity isometry, exactly."""
    mpo = I.heisenberg_mpo()
    k = 4
    charge = lambda s: (sum(1 if x == 0 else -1 for x in s),)
    e0 = exact_environments(mpo, k, 0, charge)
    e1 = exact_environments(mpo, k + 1, 0, charge)
    states0 = list(itertools.product(range(2), repeat=k))
    q0 = [charge(s) for s in states0]
    ord0 = sorted(range(len(states0)), key=lambda i: (q0[i], i))
    states1 = list(itertools.product(range(2), repeat=k + 1))
    q1 = [charge(s) for s in states1]
    ord1 = sorted(range(len(states1)), key=lambda i: (q1[i], i))
    pos1 = np.empty(len(ord1), dtype=int)
    pos1[np.array(ord1)] = np.arange(len(ord1))
    Ad = np.zeros((2 ** k, 2, 2 ** (k + 1)))
    for p, i in enumerate(ord0):
        for s in range(2):
            Ad[p, s, pos1[i * 2 + s]] = 1.0
    M = mpo.bond_sectors
    L = BlockTensor.from_dense([OB.make(OUT, e0["left_sectors"], SYM), OB.make(OUT, M, SYM),
                                OB.make(IN, e0["left_sectors"], SYM)], e0["L"])
    A = BlockTensor.from_dense([OB.make(IN, e0["left_sectors"], SYM), OB.make(IN, I.SPIN_PHYS, SYM),
                                OB.make(OUT, e1["left_sectors"], SYM)], Ad)
    W = odmrg.mpo_tensor(mpo, SYM)
    tA = to_lib(ctx, A)
    out = _env_net(ctx, odmrg.ENV_LEFT_SPEC, {"L": to_lib(ctx, L), "A": tA, "W": to_lib(ctx, W), "Ad": tA.dagger()},
                   [tA.bonds[2], to_lib(ctx, W).bonds[3], tA.dagger().bonds[2]])
    assert np.array_equal(to_oracle(out).densify(), e1["L"])


# ------------------------------------------------------------------------- SVD
def _check_svd(ctx, T, rowrank, keepdim=0, err=0.0, min_blockdim=None, absorb=0):
    import paper_2401_01921_gb300 as tnx
    t = to_lib(ctx, T)
    U, S, V, terr, dw = tnx.svd_truncate(t, rowrank, keepdim, err, min_blockdim, absorb)
    osv, oU, oS, oV, oerr = svd_truncate(T, rowrank, keepdim if keepdim > 0 else None, err, min_blockdim,
                                         return_err=2)
    smax = max(float(s[0]) for s in osv)
    # singular values, block by block (the new leg's sectors are the kept charges)
    assert U.bonds[-1].sectors == list(oU.bonds[-1].sectors)
    if absorb == 0:
        got = [np.diag(b) for _, b in sorted(S.block_dict().items())]
        assert [len(g) for g in got] == [len(s) for s in osv]
        for g, s in zip(got, osv):
            assert np.max(np.abs(g - s)) <= 1e-12 * smax, (g, s)
    assert abs(terr - (oerr[0] if len(oerr) else 0.0)) <= 1e-12 * smax
    assert abs(dw - float(np.sum(oerr ** 2))) <= 1e-12 * smax ** 2
    # the truncated product equals the oracle's
    uS = to_oracle(U)
    vS = to_oracle(V)
    if absorb == 0:
        prod = reconstruct(uS, to_oracle(S), vS, T.bonds)
    else:
        eye = BlockTensor([vS.bonds[0], uS.bonds[-1]],
                          {(i, i): np.eye(d) for i, (_, d) in enumerate(vS.bonds[0].sectors)})
        prod = reconstruct(uS, eye, vS, T.bonds)
    ref = reconstruct(oU, oS, oV, T.bonds)
    assert rel_fro(prod.blocks, ref) <= 1e-12
    # orthonormality of the unscaled factor(s), over values well above rounding
    if absorb != 2:
        for g, rl, cl, Mg in matrix_blocks(uS, rowrank):
            assert np.allclose(Mg.T @ Mg, np.eye(Mg.shape[1]), atol=1e-12)
    if absorb != 1:
        for g, rl, cl, Mg in matrix_blocks(vS, 1):
            assert np.allclose(Mg @ Mg.T, np.eye(Mg.shape[0]), atol=1e-12)
    return osv


def test_svd_dense_example_of_the_paper(ctx):
    """Sec. 9.1 / 9.2: the 6 x 4 matrix of arange(24); printed S = 65.6235, 4.18988 (+ noise)."""
    M = np.arange(24, dtype=np.float64).reshape(2, 2, 6).transpose(2, 0, 1)
    bonds = [OB.make(0, [((), 6)]), OB.make(0, [((), 2)]), OB.make(0, [((), 2)])]
    T = BlockTensor(bonds, {(0, 0, 0): M.copy()})
    import paper_2401_01921_gb300 as tnx
    t = to_lib(ctx, T)
    U, S, V, terr, dw = tnx.svd_truncate(t, 1, 3, 1e-10)
    s = np.diag(list(S.block_dict().values())[0])
    assert np.allclose(s, [65.6235, 4.18988], rtol=5e-6)
    assert terr < 1e-12 * 65.6
    _check_svd(ctx, T, 1, keepdim=2)


def _symmetric_example(values, seed=4):
    a = OB.make(IN, [((1,), 2), ((-1,), 2)], SYM)
    c = OB.make(OUT, [((2,), 2), ((0,), 4), ((-2,), 2)], SYM)
    T = BlockTensor([a, a, c])
    rng = np.random.default_rng(seed)
    for (g, rl, cl, Mg), s in zip(matrix_blocks(T, 2), values):
        m, n = Mg.shape
        q1, _ = np.linalg.qr(rng.standard_normal((m, m)))
        q2, _ = np.linalg.qr(rng.standard_normal((n, n)))
        Mg = q1[:, :len(s)] @ np.diag(s) @ q2[:, :len(s)].T
        for t, r0, mm in rl:
            for u, c0, nn in cl:
                T.blocks[t + u] = Mg[r0:r0 + mm, c0:c0 + nn].reshape(T.block_shape(t + u))
    return T


PRINTED = [[1.46508, 0.533174], [2.30323, 1.78985, 1.59579, 1.13015], [1.43749, 0.755563]]


def test_svd_symmetric_example_keepdim_and_min_blockdim(ctx):
    T = _symmetric_example(PRINTED)
    osv = _check_svd(ctx, T, 2, keepdim=4, err=1e-10)
    assert [len(s) for s in osv] == [1, 3]
    osv = _check_svd(ctx, T, 2, keepdim=4, err=1e-10, min_blockdim=[1, 1, 1])
    assert [len(s) for s in osv] == [1, 2, 1]


def _random_two_site(chi, seed, d_sectors=I.SPIN_PHYS):
    secs = I.heisenberg_virtual_sectors(chi, 8)
    T = BlockTensor([OB.make(IN, secs, SYM), OB.make(IN, d_sectors, SYM), OB.make(IN, d_sectors, SYM),
                     OB.make(OUT, secs, SYM)])
    rng = np.random.default_rng(seed)
    for q in T.keys():
        T.blocks[q] = rng.standard_normal(T.block_shape(q))
    return T


@pytest.mark.parametrize("chi,keepdim,absorb", [(16, 0, 0), (40, 24, 0), (64, 48, 1), (64, 48, 2), (160, 100, 0)])
def test_svd_two_site_wavefunction_matches_the_oracle(ctx, chi, keepdim, absorb):
    """The DMRG split: psi[a, s1, s2, b] with rowrank 2 (tall, wide and square blocks)."""
    _check_svd(ctx, _random_two_site(chi, chi), 2, keepdim=keepdim, absorb=absorb)


def test_svd_wide_and_tall_orientations(ctx):
    """rowrank 1 and 3 of the same tensor: blocks wider than tall and taller than wide."""
    T = _random_two_site(24, 7)
    _check_svd(ctx, T, 1)
    _check_svd(ctx, T, 3, keepdim=10)


def test_svd_err_threshold_and_nothing_kept(ctx):
    import paper_2401_01921_gb300 as tnx
    T = _symmetric_example(PRINTED)
    osv = _check_svd(ctx, T, 2, err=1.5)
    assert np.allclose(sorted(float(x) for s in osv for x in s), [1.59579, 1.78985, 2.30323], rtol=1e-12)
    with pytest.raises(tnx.TnxError) as e:
        tnx.svd_truncate(to_lib(ctx, T), 2, 0, 10.0)
    assert e.value.name == "TNX_ERR_ARG"


@pytest.mark.parametrize("m,n", [(90, 60), (250, 200), (320, 300), (600, 400), (400, 600)])
def test_svd_graded_dense_block(ctx, m, n):
    """One dense block whose singular values fall from 1 to 1e-20 (below rounding, as in a DMRG
    wavefunction), tall and wide, up to 400 vectors of length 600; all values kept, so the
    vectors of the values below rounding must come out orthonormal too."""
    rng = np.random.default_rng(m * 1000 + n)
    k = min(m, n)
    s = 10.0 ** (-20.0 * np.arange(k) / k)
    q1, _ = np.linalg.qr(rng.standard_normal((m, k)))
    q2, _ = np.linalg.qr(rng.standard_normal((n, k)))
    M = (q1 * s) @ q2.T
    T = BlockTensor([OB.make(0, [((), m)]), OB.make(0, [((), n)])], {(0, 0): M})
    _check_svd(ctx, T, 1)
