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


@pytest.mark.parametrize("prec", ["f64", "split_bf16"])
@pytest.mark.parametrize("budget", [150 * 10**9, 10**6])
def test_alone_equals_in_mix(ctx, prec, budget):
    import paper_2401_01921_gb300 as tnx
    nets = pool(ctx, prec)
    reqs = []
    for i, (net, T, B) in enumerate(nets):
        reqs.append((i, tnx.REQ_LANCZOS, 12))
        reqs.append((i, tnx.REQ_APPLY, 0))
    # alone
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
    # in the mix: everything submitted at once
    srv = tnx.Server(ctx, max_slots=4, hbm_budget_bytes=budget)
    outs, ids = [], []
    for i, kind, nsteps in reqs:
        net, T, B = nets[i]
        out = tnx.Tensor(ctx, B["psi"]) if kind == tnx.REQ_APPLY else None
        outs.append(out)
        ids.append(srv.submit(net, "psi", T["psi"], kind, nsteps, out))
    for (i, kind, nsteps), rid, out, ref in zip(reqs, ids, outs, alone):
        ev, mv, lat = srv.wait(rid, 60000)
        assert lat > 0
        if kind == tnx.REQ_LANCZOS:
            assert mv == nsteps
            assert abs(ev - ref) <= 1e-12 * abs(ref), (ev, ref)
        else:
            assert np.array_equal(out.download(), ref)
    st = srv.stats()
    assert st["completed"] == len(reqs)
    if budget < 10**8:
        assert st["evictions"] > 0
    srv.close()
