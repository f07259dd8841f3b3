"""Oracle pins: Lanczos, tridiagonal bisection, exact-diagonalisation energies."""
import math

import numpy as np
import pytest

import tnx_inputs as I
from oracle import heff
from oracle.brute import exact_environments, heisenberg_dense
from oracle.lanczos import lanczos, lowest_eig_bisect, tridiag_eigvec
from oracle.network import Network
from oracle.symtensor import Bond, BlockTensor, Symmetry, U1


def test_bisection_vs_eigvalsh():
    rng = np.random.default_rng(1)
    for k in (1, 2, 5, 17, 30):
        a = rng.standard_normal(k)
        b = np.concatenate([[0.0], rng.standard_normal(k - 1)])
        T = np.diag(a) + np.diag(b[1:], 1) + np.diag(b[1:], -1)
        ev = np.linalg.eigvalsh(T)
        lam = lowest_eig_bisect(list(a), list(b))
        # Sturm counts are backward stable: error within a small multiple of k*eps*||T||
        assert abs(lam - ev[0]) <= 2 * k * np.finfo(float).eps * max(1.0, abs(ev).max())
        y = tridiag_eigvec(list(a), list(b), lam)
        assert np.linalg.norm(T @ y - lam * y) < 1e-10


def test_lanczos_random_matrix():
    rng = np.random.default_rng(2)
    n = 60
    X = rng.standard_normal((n, n))
    H = X + X.T
    lam, x, *_ = lanczos(lambda v: H @ v, rng.standard_normal(n), n)
    ev, V = np.linalg.eigh(H)
    assert abs(lam - ev[0]) < 1e-10 * abs(ev).max()
    assert np.linalg.norm(H @ x - lam * x) < 1e-8


def test_lanczos_stops_on_invariant_subspace():
    H = np.diag(np.arange(1.0, 11.0))
    v0 = np.zeros(10)
    v0[[0, 3]] = 1.0
    lam, x, alpha, beta, k = lanczos(lambda v: H @ v, v0, 10)
    assert k == 2 and abs(lam - 1.0) < 1e-14


def heff_exact(k_left, k_right):
    """H_eff of the open Heisenberg chain with exact environments (N = k_left + k_right + 2)."""
    mpo = I.heisenberg_mpo()
    env = exact_environments(mpo, k_left, k_right, lambda s: (sum(1 if x == 0 else -1 for x in s),))
    u1 = (Symmetry(U1),)
    Ls, Rs, P, M = env["left_sectors"], env["right_sectors"], I.SPIN_PHYS, mpo.bond_sectors
    IN, OUT = I.IN, I.OUT
    bL = [Bond.make(OUT, Ls, u1), Bond.make(OUT, M, u1), Bond.make(IN, Ls, u1)]
    bR = [Bond.make(IN, Rs, u1), Bond.make(IN, M, u1), Bond.make(OUT, Rs, u1)]
    bW = [Bond.make(IN, M, u1), Bond.make(IN, P, u1), Bond.make(OUT, P, u1), Bond.make(OUT, M, u1)]
    bpsi = [Bond.make(IN, Ls, u1), Bond.make(IN, P, u1), Bond.make(IN, P, u1), Bond.make(OUT, Rs, u1)]
    net = Network(I.HEFF_SPEC)
    net.put("L", BlockTensor.from_dense(bL, env["L"]))
    net.put("R", BlockTensor.from_dense(bR, env["R"]))
    Wg = mpo.W_grouped()
    net.put("W1", BlockTensor.from_dense(bW, Wg))
    net.put("W2", BlockTensor.from_dense(bW, Wg))
    psi = BlockTensor(bpsi)
    rng = np.random.default_rng(3)
    for q in psi.keys():
        psi.blocks[q] = rng.standard_normal(psi.block_shape(q))
    net.put("psi", psi)
    net.set_order(True)
    return net, psi


@pytest.mark.parametrize("k,closed", [(0, -0.75), (1, -(3 + 2 * math.sqrt(3)) / 4)])
def test_heff_ground_energy_closed_form(k, closed):
    """N = 2 and N = 4 open Heisenberg chains: E0 = -3/4 and -(3 + 2 sqrt 3)/4."""
    net, psi = heff_exact(k, k)
    op = heff.flat_apply(net, psi)
    n = psi.nelem()
    lam, x, *_ = lanczos(op, psi.flat(), n)
    assert abs(lam - closed) < 1e-12
    assert abs(np.linalg.eigvalsh(heisenberg_dense(2 * k + 2))[0] - closed) < 1e-12


@pytest.mark.parametrize("k", [2, 3])
def test_heff_ground_energy_ed(k):
    """N = 6, 8: Lanczos on H_eff with exact environments == dense ED ground energy."""
    net, psi = heff_exact(k, k)
    op = heff.flat_apply(net, psi)
    lam, *_ = lanczos(op, psi.flat(), min(psi.nelem(), 80))
    e0 = np.linalg.eigvalsh(heisenberg_dense(2 * k + 2))[0]
    assert abs(lam - e0) < 1e-10


def test_lanczos_symmetrised_dense_heff():
    """Symmetrised dense chi=8 H_eff: the operator is symmetric and Lanczos finds eigh's lowest."""
    wl = I.dense_workload(8)
    net, T = heff.make_heff(wl, symmetric=True)
    op = heff.flat_apply(net, T["psi"])
    n = T["psi"].nelem()
    H = np.stack([op(e) for e in np.eye(n)], axis=1)
    assert np.abs(H - H.T).max() < 1e-12 * np.abs(H).max()
    ev = np.linalg.eigvalsh(H)
    lam, x, *_ = lanczos(op, T["psi"].flat(), n)
    assert abs(lam - ev[0]) < 1e-10 * abs(ev).max()


def test_lanczos_symmetrised_u1_heff_is_symmetric():
    wl = I.heisenberg_workload(6, 3)
    net, T = heff.make_heff(wl, symmetric=True)
    op = heff.flat_apply(net, T["psi"])
    n = T["psi"].nelem()
    H = np.stack([op(e) for e in np.eye(n)], axis=1)
    assert np.abs(H - H.T).max() < 1e-12 * np.abs(H).max()
