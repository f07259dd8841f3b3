"""Serving loop: requests admitted as slots and memory free up, overlapping on the device.

Each result must be the same alone and in the mix: every request is first run
alone (one at a time, synchronous entry points), then all are submitted at
once to the server and run concurrently; eigenvalues must agree to 1e-12
relative and apply outputs bit for bit (the same kernels on the same data).
A tight memory budget forces evictions, which must not change any result."""
import numpy as np
import pytest

import tnx_inputs as I

from gpu_harness import lib_heff

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2401_01921_gb300 as tnx
    from paper_2401_01921_gb300 import build
    build.build()
    return tnx.Context(0)


def pool(ctx, prec):
    wls = [I.heisenberg_workload(64, 8), I.heisenberg_workload(128, 10), I.hubbard_workload(64, seed_base=2000),
           I.heisenberg_workload(96, 9, sector_scale=True), I.hubbard_workload(128, seed_base=3000)]
    return [lib_heff(ctx, wl, symmetric=True, prec=prec) for wl in wls]


def run_alone(ctx, nets, reqs):
    import paper_2401_01921_gb300 as tnx
    alone = []
    for i, kind, nsteps in reqs:
        net, T, B = nets[i]
        if kind == tnx.REQ_LANCZOS:
            alone.append(tnx.lanczos(net, "psi", T["psi"], nsteps)[0])
        else:
            out = tnx.Tensor(ctx, B["psi"])
            net.launch_into(out)
            alone.append(out.download())
    ctx.sync()
    return alone


def run_mix(ctx, nets, reqs, budget, slots=4):
    """Every request submitted at once; returns (results or error names, stats)."""
    import paper_2401_01921_gb300 as tnx
    srv = tnx.Server(ctx, max_slots=slots, hbm_budget_bytes=budget)
    outs, ids = [], []
    for i, kind, nsteps in reqs:
        net, T, B = nets[i]
        out = tnx.Tensor(ctx, B["psi"]) if kind == tnx.REQ_APPLY else None
        outs.append(out)
        ids.append(srv.submit(net, "psi", T["psi"], kind, nsteps, out))
    res = []
    for (i, kind, nsteps), rid, out in zip(reqs, ids, outs):
        try:
            ev, mv, lat = srv.wait(rid, 60000)
        except tnx.TnxError as e:
            res.append(e.name)
            continue
        assert lat > 0
        if kind == tnx.REQ_LANCZOS:
            assert mv == nsteps
            res.append(ev)
        else:
            res.append(out.download())
    st = srv.stats()
    srv.close()
    return res, st


def requests(nets):
    import paper_2401_01921_gb300 as tnx
    reqs = []
    for i in range(len(nets)):
        reqs.append((i, tnx.REQ_LANCZOS, 12))
        reqs.append((i, tnx.REQ_APPLY, 0))
    return reqs


def check_equal(reqs, res, alone):
    import paper_2401_01921_gb300 as tnx
    for (i, kind, nsteps), got, ref in zip(reqs, res, alone):
        if kind == tnx.REQ_LANCZOS:
            assert abs(got - ref) <= 1e-12 * abs(ref), (got, ref)
        else:
            assert np.array_equal(got, ref)


@pytest.mark.parametrize("prec", ["f64", "split_bf16"])
def test_alone_equals_in_mix(ctx, prec):
    nets = pool(ctx, prec)
    reqs = requests(nets)
    alone = run_alone(ctx, nets, reqs)
    res, st = run_mix(ctx, nets, reqs, 150 * 10**9)
    check_equal(reqs, res, alone)
    assert st["completed"] == len(reqs) and st["evictions"] == 0


@pytest.mark.parametrize("prec", ["f64", "split_bf16"])
def test_tight_budget_admits_by_size_and_never_exceeds_it(ctx, prec):
    """Budget = the largest single network's bytes: every request fits alone but not all together,
    so admission waits and evicts; the peak of the counted resident bytes stays within the budget,
    and every result is still the one computed alone."""
    nets = pool(ctx, prec)
    reqs = requests(nets)
    alone = run_alone(ctx, nets, reqs)
    held = [net.resident() for net, T, B in nets]
    for b, pb in held:
        assert 0 < pb <= b          # the sizing pass agrees with the built plan (which it is part of)
    budget = max(b for b, pb in held)
    assert budget < sum(b for b, pb in held)
    res, st = run_mix(ctx, nets, reqs, budget)
    check_equal(reqs, res, alone)
    assert st["completed"] == len(reqs)
    assert st["evictions"] > 0
    assert st["peak_bytes"] <= budget, (st, budget)


def test_request_larger_than_the_budget_is_refused(ctx):
    nets = pool(ctx, "f64")
    reqs = requests(nets)
    run_alone(ctx, nets, reqs)
    smallest = min(net.resident()[0] for net, T, B in nets)
    res, st = run_mix(ctx, nets, reqs, smallest - 1)
    assert res == ["TNX_ERR_OOM"] * len(reqs)
    assert st["peak_bytes"] == 0


def test_plan_sizing_pass_matches_the_built_plan(ctx):
    """tnx_network_resident sizes a plan without building it; building it then holds exactly that."""
    import paper_2401_01921_gb300 as tnx
    for prec in ("f64", "split_bf16"):
        net, T, B = lib_heff(ctx, I.heisenberg_workload(256, 14), symmetric=True, prec=prec)
        b0, pb = net.resident()
        assert b0 == 0 and pb > 0
        out = tnx.Tensor(ctx, B["psi"])
        net.launch_into(out)
        b1, pb1 = net.resident()
        assert b1 == pb == pb1
