"""Oracle pins: dense brute force, dense Hamiltonians, exact environments.

Used only to pin the other oracle modules against the mathematics.

* ``brute_network``: the network contraction of Sec. 8 written as its
  definition, one explicit loop over every assignment of every label
  (pure Python, tiny sizes only).
* ``heisenberg_dense``: H = J sum_i S_i . S_{i+1} built from Kronecker
  products of the spin-1/2 operators (open chain).
* ``hubbard_dense``: the spinful Hubbard chain built from Jordan-Wigner
  fermion operators on 2N modes ordered (site, up, dn).
* ``mpo_chain_dense``: the operator encoded by N copies of an MPO with its
  boundary row / column (the recursion O_w' = sum_w O_w (x) W[w, :, :, w']).
* ``exact_environments``: left / right environments of an open chain built
  from the full product basis of k sites (identity isometries), so that the
  two-site H_eff of the Fig. "Hpsi_fig" contraction is the full Hamiltonian
  of 2k+2 sites restricted to total charge zero.

Parity: ``heisenberg_dense`` is pinned by the closed forms E0(N=2) = -3/4 and
E0(N=4) = -(3 + 2 sqrt 3)/4; ``hubbard_dense`` by the anticommutation
relations of its mode operators and the two-site closed form; the MPO chain
against both (tests/test_oracle_mpo.py).
"""
from __future__ import annotations

import itertools

import numpy as np


def brute_network(spec_labels: dict, tout: list, dense: dict, dims: dict) -> np.ndarray:
    """out[tout] = sum over all other labels of the product of all tensors."""
    labels = sorted(dims)
    closed = [l for l in labels if l not in tout]
    out = np.zeros(tuple(dims[l] for l in tout))
    names = list(spec_labels)
    for oidx in itertools.product(*[range(dims[l]) for l in tout]):
        val = dict(zip(tout, oidx))
        acc = 0.0
        for cidx in itertools.product(*[range(dims[l]) for l in closed]):
            val.update(zip(closed, cidx))
            p = 1.0
            for n in names:
                p *= dense[n][tuple(val[l] for l in spec_labels[n])]
                if p == 0.0:
                    break
            acc += p
        out[oidx] = acc
    return out


def spin_ops():
    Sp = np.array([[0.0, 1.0], [0.0, 0.0]])
    Sm = Sp.T.copy()
    Sz = np.diag([0.5, -0.5])
    return Sp, Sm, Sz


def _site_op(op, i, N, d):
    mats = [np.eye(d)] * N
    mats = list(mats)
    mats[i] = op
    out = mats[0]
    for m in mats[1:]:
        out = np.kron(out, m)
    return out


def heisenberg_dense(N: int, J: float = 1.0) -> np.ndarray:
    Sp, Sm, Sz = spin_ops()
    H = np.zeros((2 ** N, 2 ** N))
    for i in range(N - 1):
        H += J * 0.5 * (_site_op(Sp, i, N, 2) @ _site_op(Sm, i + 1, N, 2)
                        + _site_op(Sm, i, N, 2) @ _site_op(Sp, i + 1, N, 2))
        H += J * _site_op(Sz, i, N, 2) @ _site_op(Sz, i + 1, N, 2)
    return H


def fermion_modes(nmodes: int):
    """Annihilators c_m on 2^nmodes (Jordan-Wigner, mode 0 leftmost)."""
    a = np.array([[0.0, 1.0], [0.0, 0.0]])   # |0><1| on one mode (basis |0>,|1>)
    Z = np.diag([1.0, -1.0])
    cs = []
    for m in range(nmodes):
        mats = [Z] * m + [a] + [np.eye(2)] * (nmodes - m - 1)
        out = mats[0]
        for x in mats[1:]:
            out = np.kron(out, x)
        cs.append(out)
    return cs


def hubbard_dense(N: int, t: float = 1.0, U: float = 4.0) -> np.ndarray:
    """Hubbard chain on 2N modes; local basis per site (n_up, n_dn) = mode bits."""
    c = fermion_modes(2 * N)
    dim = 2 ** (2 * N)
    H = np.zeros((dim, dim))
    for i in range(N - 1):
        for s in range(2):
            a, b = c[2 * i + s], c[2 * (i + 1) + s]
            H += -t * (a.T @ b + b.T @ a)
    for i in range(N):
        nu = c[2 * i].T @ c[2 * i]
        nd = c[2 * i + 1].T @ c[2 * i + 1]
        H += U * nu @ nd
    return H


def hubbard_site_basis_perm(N: int) -> np.ndarray:
    """Map from the MPO product basis (per site |0>,|up>,|dn>,|updn>) to the mode basis.

    Mode basis bits per site are (n_up, n_dn) with index n_up*2 + n_dn in the
    Kronecker order of fermion_modes; |updn> = c+_up c+_dn |0> matches the
    mode-ordered product c+_{up} c+_{dn} with up before dn.
    """
    local = {0: (0, 0), 1: (1, 0), 2: (0, 1), 3: (1, 1)}
    perm = np.zeros(4 ** N, dtype=np.int64)
    for idx in range(4 ** N):
        digits = []
        x = idx
        for _ in range(N):
            digits.append(x % 4)
            x //= 4
        digits = digits[::-1]
        m = 0
        for dgt in digits:
            nu, nd = local[dgt]
            m = m * 4 + nu * 2 + nd
        perm[idx] = m
    return perm


def mpo_chain_dense(W: np.ndarray, left_row: int, right_col: int, N: int) -> np.ndarray:
    D, d = W.shape[0], W.shape[1]
    O = [np.zeros((1, 1)) for _ in range(D)]
    O[left_row] = np.ones((1, 1))
    for _ in range(N):
        new = [np.zeros((O[0].shape[0] * d, O[0].shape[1] * d)) for _ in range(D)]
        for w in range(D):
            if not O[w].any():
                continue
            for w2 in range(D):
                if W[w, :, :, w2].any():
                    new[w2] += np.kron(O[w], W[w, :, :, w2])
        O = new
    return O[right_col]


def exact_environments(mpo, k_left: int, k_right: int, charge_of_state):
    """Dense L[a, w, a'] and R[b, w, b'] from the full product bases.

    charge_of_state(list of site indices) -> charge tuple of a product state.
    Returns dict with L, R (w in grouped MPO bond order, a/b ordered by sector),
    the left and right bond sector lists [(charge, deg)].
    The right bond carries the reversed charge of the right-block state, so
    zero-flux psi[a, s1, s2, b] spans total charge zero.
    """
    W = mpo.W
    D, d = W.shape[0], W.shape[1]
    # left operators: O_w' = sum_w O_w (x) W[w, :, :, w']
    OL = [np.zeros((1, 1)) for _ in range(D)]
    OL[mpo.left_row] = np.ones((1, 1))
    for _ in range(k_left):
        new = [np.zeros((OL[0].shape[0] * d,) * 2) for _ in range(D)]
        for w in range(D):
            for w2 in range(D):
                if W[w, :, :, w2].any() and OL[w].any():
                    new[w2] += np.kron(OL[w], W[w, :, :, w2])
        OL = new
    # right operators: O_w = sum_w' W[w, :, :, w'] (x) O_w'
    OR = [np.zeros((1, 1)) for _ in range(D)]
    OR[mpo.right_col] = np.ones((1, 1))
    for _ in range(k_right):
        new = [np.zeros((OR[0].shape[0] * d,) * 2) for _ in range(D)]
        for w in range(D):
            for w2 in range(D):
                if W[w, :, :, w2].any() and OR[w2].any():
                    new[w] += np.kron(W[w, :, :, w2], OR[w2])
        OR = new

    def basis(k, reverse):
        states = list(itertools.product(range(d), repeat=k))
        qs = [charge_of_state(list(s)) for s in states]
        if reverse:
            qs = [tuple(-x for x in q) for q in qs]
        order = sorted(range(len(states)), key=lambda i: (qs[i], i))
        secs = []
        for i in order:
            if secs and secs[-1][0] == qs[i]:
                secs[-1] = (qs[i], secs[-1][1] + 1)
            else:
                secs.append((qs[i], 1))
        return np.array(order), secs

    pl, secl = basis(k_left, False)
    pr, secr = basis(k_right, True)
    pos = mpo.channel_pos
    chiL, chiR = len(pl), len(pr)
    L = np.zeros((chiL, D, chiL))
    R = np.zeros((chiR, D, chiR))
    for w in range(D):
        M = OL[w][np.ix_(pl, pl)]          # M[a', a] in sorted basis
        L[:, pos[w], :] = M.T                # L[a, w, a'] = O_w[a', a]
        M = OR[w][np.ix_(pr, pr)]
        R[:, pos[w], :] = M.T                # R[b, w, b'] = O_w[b', b]
    return {"L": L, "R": R, "left_sectors": secl, "right_sectors": secr}
