"""Batched launches: many independent H_eff networks in one grouped launch per step.

Each instance of the batch must give exactly what its own launch gives (the
same kernels on the same data), and match the oracle."""
import numpy as np
import pytest

import tnx_inputs as I

from gpu_harness import lib_heff, oracle_heff, rel_fro

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2401_01921_gb300 as tnx
    from paper_2401_01921_gb300 import build
    build.build()
    return tnx.Context(0)


def instances():
    chis = I.batched_hubbard_chis(6, lo=6.0, hi=7.0)
    return [I.hubbard_workload(c, seed_base=1000 + 4 * i) for i, c in enumerate(chis)]


@pytest.mark.parametrize("prec", ["f64", "split_bf16", "tf32"])
def test_batch_equals_individual_launches(ctx, prec):
    import paper_2401_01921_gb300 as tnx
    wls = instances()
    built = [lib_heff(ctx, wl, prec=prec, order="(L,(((psi,R),W2),W1))") for wl in wls]
    single = []
    for net, T, B in built:
        single.append(net.launch(B["psi"]).download())
    outs = [tnx.Tensor(ctx, B["psi"]) for _, _, B in built]
    batch = tnx.Batch(ctx, [n for n, _, _ in built])
    assert batch.flops() == sum(n.flops() for n, _, _ in built)
    batch.launch_into(outs)
    for o, ref in zip(outs, single):
        assert np.array_equal(o.download(), ref)
    choice = batch.autotune(outs)
    assert choice in (0, 152, 304, 456)
    batch.launch_into(outs)
    for o, ref in zip(outs, single):
        assert np.array_equal(o.download(), ref)
    # and against the oracle
    for (net, T, B), o, wl in zip(built, outs, wls):
        onet, _ = oracle_heff(wl, order="(L,(((psi,R),W2),W1))")
        err = rel_fro(o.block_dict(), onet.launch())
        assert err <= {"f64": 1e-12, "split_bf16": 1e-10, "tf32": 2e-3}[prec], err
