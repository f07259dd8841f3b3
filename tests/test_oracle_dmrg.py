"""Oracle pins: environment updates and the two-site DMRG sweep (paper Sec. 11).

- Growing the exact k-site environments of ``brute.exact_environments`` by one
  site with identity isometries (A maps (k-site state, new site) to the
  (k+1)-site product state) must give the (k+1)-site environments exactly,
  on the left and on the right.
- The XX chain's DMRG energy equals the free-fermion closed form (the paper's
  DMRG benchmark model); the Heisenberg chain's equals dense diagonalisation.
- The Lanczos stopping rule ends an exhausted Krylov space even when every
  alpha is zero (the XX chain's first update from a Neel state).
"""
import itertools

import numpy as np
import pytest

import tnx_inputs as I
from oracle import dmrg
from oracle.brute import exact_environments, heisenberg_dense
from oracle.lanczos import lanczos
from oracle.symtensor import IN, OUT, Bond, BlockTensor, Symmetry, U1

SYM = (Symmetry(U1),)


def _charge(s):
    return (sum(1 if x == 0 else -1 for x in s),)


def _sorted_basis(k, reverse):
    states = list(itertools.product(range(2), repeat=k))
    qs = [_charge(s) for s in states]
    if reverse:
        qs = [tuple(-x for x in q) for q in qs]
    order = sorted(range(len(states)), key=lambda i: (qs[i], i))
    pos = np.empty(len(order), dtype=int)
    pos[np.array(order)] = np.arange(len(order))
    return states, order, pos


@pytest.mark.parametrize("mpo_fn", [I.heisenberg_mpo, I.xx_mpo])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_left_environment_grows_by_one_site_exactly(mpo_fn, k):
    mpo = mpo_fn()
    W = dmrg.mpo_tensor(mpo, SYM)
    e0 = exact_environments(mpo, k, 0, _charge)
    e1 = exact_environments(mpo, k + 1, 0, _charge)
    M = mpo.bond_sectors
    Lk = BlockTensor.from_dense([Bond.make(OUT, e0["left_sectors"], SYM), Bond.make(OUT, M, SYM),
                                 Bond.make(IN, e0["left_sectors"], SYM)], e0["L"])
    st0, ord0, _ = _sorted_basis(k, False)
    st1, _, pos1 = _sorted_basis(k + 1, False)
    A = np.zeros((2 ** k, 2, 2 ** (k + 1)))
    for p, i in enumerate(ord0):
        for s in range(2):
            A[p, s, pos1[i * 2 + s]] = 1.0
    At = BlockTensor.from_dense([Bond.make(IN, e0["left_sectors"], SYM), Bond.make(IN, I.SPIN_PHYS, SYM),
                                 Bond.make(OUT, e1["left_sectors"], SYM)], A)
    got = dmrg.env_left(Lk, At, W).densify()
    assert np.array_equal(got, e1["L"])


@pytest.mark.parametrize("mpo_fn", [I.heisenberg_mpo, I.xx_mpo])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_right_environment_grows_by_one_site_exactly(mpo_fn, k):
    mpo = mpo_fn()
    W = dmrg.mpo_tensor(mpo, SYM)
    e0 = exact_environments(mpo, 0, k, _charge)
    e1 = exact_environments(mpo, 0, k + 1, _charge)
    M = mpo.bond_sectors
    Rk = BlockTensor.from_dense([Bond.make(IN, e0["right_sectors"], SYM), Bond.make(IN, M, SYM),
                                 Bond.make(OUT, e0["right_sectors"], SYM)], e0["R"])
    st0, ord0, _ = _sorted_basis(k, True)
    st1, _, pos1 = _sorted_basis(k + 1, True)
    A = np.zeros((2 ** (k + 1), 2, 2 ** k))
    for p, i in enumerate(ord0):
        for s in range(2):
            A[pos1[s * 2 ** k + i], s, p] = 1.0
    At = BlockTensor.from_dense([Bond.make(IN, e1["right_sectors"], SYM), Bond.make(IN, I.SPIN_PHYS, SYM),
                                 Bond.make(OUT, e0["right_sectors"], SYM)], A)
    got = dmrg.env_right(Rk, At, W).densify()
    assert np.array_equal(got, e1["R"])


def test_dagger_reverses_every_bond_and_keeps_the_blocks():
    a = Bond.make(IN, [((1,), 2), ((-1,), 1)], SYM)
    b = Bond.make(OUT, [((0,), 3), ((2,), 1)], SYM)
    T = BlockTensor([a, a, b])
    rng = np.random.default_rng(0)
    for q in T.keys():
        T.blocks[q] = rng.standard_normal(T.block_shape(q))
    D = dmrg.dagger(T)
    assert [x.dir for x in D.bonds] == [OUT, OUT, IN]
    assert D.keys() == T.keys()
    for q in T.keys():
        assert np.array_equal(D.blocks[q], T.blocks[q])


def test_lanczos_stops_when_every_alpha_is_zero():
    H = 0.5 * np.array([[0.0, 1.0], [1.0, 0.0]])
    lam, x, alpha, beta, k = lanczos(lambda v: H @ v, np.array([1.0, 0.0]), 10)
    assert alpha == [0.0, 0.0] and k == 2
    assert lam == pytest.approx(-0.5, abs=1e-15)


def test_xx_energy_is_the_free_fermion_closed_form():
    e, mps = dmrg.dmrg(I.xx_mpo(), 10, 32, 4)
    assert abs(e[-1] - dmrg.xx_ground_energy(10)) < 1e-10
    assert max(A.bonds[2].dim for A in mps) <= 32


def test_heisenberg_energy_equals_dense_diagonalisation():
    e, mps = dmrg.dmrg(I.heisenberg_mpo(), 8, 16, 2)
    assert abs(e[-1] - np.linalg.eigvalsh(heisenberg_dense(8))[0]) < 1e-11


def test_truncated_dmrg_is_variational():
    """A small bond dimension gives an energy above the exact one and below the product state's."""
    e, mps = dmrg.dmrg(I.xx_mpo(), 12, 4, 2)
    exact = dmrg.xx_ground_energy(12)
    assert exact < e[-1] < 0.0
    assert max(A.bonds[2].dim for A in mps) <= 4
