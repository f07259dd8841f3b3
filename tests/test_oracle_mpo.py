"""Oracle pins: MPOs and dense Hamiltonians against brute force and closed forms."""
import math

import numpy as np
import pytest

import tnx_inputs as I
from oracle.brute import (fermion_modes, heisenberg_dense, hubbard_dense, hubbard_site_basis_perm,
                          mpo_chain_dense)


def test_heisenberg_closed_forms():
    assert abs(np.linalg.eigvalsh(heisenberg_dense(2))[0] + 0.75) < 1e-14
    assert abs(np.linalg.eigvalsh(heisenberg_dense(4))[0] + (3 + 2 * math.sqrt(3)) / 4) < 1e-13


@pytest.mark.parametrize("N", [2, 3, 4])
def test_heisenberg_mpo_chain(N):
    m = I.heisenberg_mpo()
    H = mpo_chain_dense(m.W, m.left_row, m.right_col, N)
    assert np.abs(H - heisenberg_dense(N)).max() < 1e-14


def test_heisenberg_mpo_zero_flux():
    """Every non-zero W[wL, s', s, wR] has q(wL) + q(s') - q(s) - q(wR) = 0."""
    m = I.heisenberg_mpo()
    qs = [1, -1]
    for wl, sp, s, wr in zip(*np.nonzero(m.W)):
        assert m.channel_charge[wl][0] + qs[sp] - qs[s] - m.channel_charge[wr][0] == 0


def test_fermion_anticommutation():
    c = fermion_modes(4)
    for i in range(4):
        for j in range(4):
            ac = c[i] @ c[j].T + c[j].T @ c[i]
            assert np.array_equal(ac, np.eye(16) * (i == j))
            assert not np.any(c[i] @ c[j] + c[j] @ c[i])


def test_hubbard_two_site_closed_form():
    """Two sites at half filling: E0 = (U - sqrt(U^2 + 16 t^2)) / 2."""
    H = hubbard_dense(2, 1.0, 4.0)
    c = fermion_modes(4)
    Ntot = sum(x.T @ x for x in c)
    P = np.diag(Ntot) == 2
    e = np.linalg.eigvalsh(H[np.ix_(P, P)])[0]
    assert abs(e - (4 - math.sqrt(16 + 16)) / 2) < 1e-12


@pytest.mark.parametrize("N", [2, 3, 4, 5])
def test_hubbard_mpo_chain(N):
    m = I.hubbard_mpo()
    H = mpo_chain_dense(m.W, m.left_row, m.right_col, N)
    perm = hubbard_site_basis_perm(N)
    Hd = hubbard_dense(N)
    assert np.abs(H - Hd[np.ix_(perm, perm)]).max() < 1e-13


def test_hubbard_mpo_zero_flux():
    m = I.hubbard_mpo()
    qs = [q for q, _ in I.HUBBARD_PHYS]
    for wl, sp, s, wr in zip(*np.nonzero(m.W)):
        for c in range(2):
            assert m.channel_charge[wl][c] + qs[sp][c] - qs[s][c] - m.channel_charge[wr][c] == 0


def test_mpo_transpose_symmetry():
    """W[w0, s, s', w1] == W[wbar0, s', s, wbar1]: makes the symmetrised H_eff symmetric."""
    m = I.heisenberg_mpo()
    bar = I.channel_bar_heisenberg()
    Wt = m.W.transpose(0, 2, 1, 3)[np.ix_(bar, range(2), range(2), bar)]
    assert np.array_equal(Wt, m.W)
    h = I.hubbard_mpo()
    bar = [0, 2, 1, 4, 3, 5]
    Wt = h.W.transpose(0, 2, 1, 3)[np.ix_(bar, range(4), range(4), bar)]
    assert np.array_equal(Wt, h.W)
