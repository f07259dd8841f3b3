"""The partial reorthogonalisation rule of the library's Lanczos solve, replayed in numpy on the
oracle's operator (CPU).

The paper defers its Lanczos details to the user guide (Sec. 9.3); the oracle reorthogonalises fully.
The library keeps its basis orthogonal by Simon's rule (Math. Comp. 42, 1984): each step updates
estimates w_{j+1,k} of <v_{j+1}, v_k> from the three-term recurrence plus a rounding term of
sign(.) eps1 |T| (eps1 = sqrt(n) eps / 2, |T| the largest row sum of T so far), sets
w_{j+1,j} = eps1 |T| / beta_{j+1}, and takes one classical Gram-Schmidt pass against all earlier
vectors when an estimate exceeds 1e-10, and again at the next step (after a pass the estimates
restart at eps1).  Replayed here on the oracle's symmetric H_eff (chi = 64, n = 1576, 80 steps,
a space small enough that orthogonality is lost again and again), the rule must take passes, keep
every |<v_j, v_k>| within ten times its threshold, and give the Ritz value of the oracle's fully
reorthogonalised solve.
"""
import numpy as np

import tnx_inputs as I
from oracle import heff as oheff
from oracle.lanczos import lanczos as oracle_lanczos, lowest_eig_bisect

EPS = 2.220446049250313e-16


def partial_reorth_lanczos(apply, v0, nsteps, tau=1e-10, stop_rel=1e-14):
    """Returns (lowest Ritz value, steps, Gram-Schmidt passes, largest |<v_j, v_k>|, j > k)."""
    n = v0.size
    eps1 = np.sqrt(n) * 0.5 * EPS
    V = [v0 / np.linalg.norm(v0)]
    alpha, beta = [], [0.0]
    om = np.zeros(nsteps + 2)        # row j of the estimates, k = 0..j
    om_prev = np.zeros(nsteps + 2)   # row j-1
    om[0] = 1.0
    forced, passes, worst = False, 0, 0.0
    for j in range(nsteps):
        w = apply(V[j])
        a = float(V[j] @ w)
        alpha.append(a)
        u = w - a * V[j]
        if j > 0:
            u = u - beta[j] * V[j - 1]
        bn = float(np.linalg.norm(u))
        tnorm = max(abs(alpha[i]) + beta[i] + (beta[i + 1] if i < j else 0.0) for i in range(j + 1))
        tnorm = max(tnorm, abs(a) + beta[j] + bn)
        e = np.empty(j + 1)
        for k in range(j):
            t = beta[k + 1] * om[k + 1] + (alpha[k] - a) * om[k] - beta[j] * om_prev[k]
            if k > 0:
                t += beta[k] * om[k - 1]
            e[k] = (t + np.copysign(eps1 * tnorm, t)) / bn
        e[j] = eps1 * tnorm / bn
        take = forced or not (np.max(np.abs(e)) <= tau)
        forced = take and not forced
        if take:
            passes += 1
            c = np.array([vk @ u for vk in V])
            for ck, vk in zip(c, V):
                u = u - ck * vk
            bn = float(np.linalg.norm(u))
        om_prev[:j + 1] = om[:j + 1]
        om[:j + 1] = eps1 if take else e
        om[j + 1] = 1.0
        scale = max(max(abs(x) for x in alpha), max(beta))
        if j == nsteps - 1 or bn < stop_rel * scale:
            break
        beta.append(bn)
        V.append(u / bn)
        worst = max(worst, max(abs(float(V[-1] @ vk)) for vk in V[:-1]))
    k = len(alpha)
    return lowest_eig_bisect(alpha, beta[:k]), k, passes, worst


def test_partial_reorthogonalisation_keeps_the_basis_and_the_ritz_value():
    wl = I.heisenberg_workload(64, 20)
    onet, T = oheff.make_heff(wl, symmetric=True)
    op = oheff.flat_apply(onet, T["psi"])
    v0 = T["psi"].flat()
    assert v0.size == 1576
    lam, k, passes, worst = partial_reorth_lanczos(op, v0, 80)
    olam, _, _, _, ok = oracle_lanczos(op, v0, 80)
    print(f"steps {k} (oracle {ok}), passes {passes}, worst |<v_j,v_k>| {worst:.2e}, "
          f"rel {abs(lam - olam) / abs(olam):.2e}")
    assert passes >= 1
    assert worst <= 1e-9, worst
    assert abs(lam - olam) <= 1e-12 * abs(olam)


def test_no_pass_while_the_estimates_stay_small():
    """Twenty steps on the chi = 40 operator: the estimates stay below the threshold and the rule takes
    no pass, so the solve is the plain three-term recurrence; its basis is still orthogonal to 1e-12."""
    wl = I.heisenberg_workload(40, 9)
    onet, T = oheff.make_heff(wl, symmetric=True)
    op = oheff.flat_apply(onet, T["psi"])
    lam, k, passes, worst = partial_reorth_lanczos(op, T["psi"].flat(), 20)
    olam, *_ = oracle_lanczos(op, T["psi"].flat(), 20)
    assert passes == 0, passes
    assert worst <= 1e-12, worst
    assert abs(lam - olam) <= 1e-12 * abs(olam)
