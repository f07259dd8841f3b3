"""The allocation-free entry point tnx_match_tables_noalloc, called through the C-ABI.

It serves callers that cannot allocate device memory where they need the
fused charge-sector tables of a contraction (their memory is owned by another
framework or sized up front).  Its working memory is a fixed device array
inside the library.  This test checks, on two calls in a row (the second one
reusing the array the first one left behind), that it returns exactly the
tables the allocating path reports through tnx_network_step_tables.  Integer
tables: the comparison is exact.

The file is named to run last, so a run that stops at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import tnx_inputs as I

pytestmark = pytest.mark.gpu


def _u(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _l(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _first_step_operands(T):
    """Step 0 of the order (L,(((psi,R),W2),W1)) is psi . R over b: A = psi, B = R."""
    psi, R = T["psi"], T["R"]
    qa, _, _ = psi.blocks()
    qb, _, _ = R.blocks()
    bond_b = psi.bonds[3]     # psi's b (OUT) meets R's b (IN)
    kposA, fposA = [3], [0, 1, 2]
    kposB, fposB = [0], [1, 2]
    legs = [bond_b] + [psi.bonds[i] for i in fposA] + [R.bonds[i] for i in fposB]
    nsec = np.array([len(b.sectors) for b in legs], dtype=np.int32)
    degs = np.array([d for b in legs for _, d in b.sectors], dtype=np.int64)
    kq = np.array([bond_b.dir * q for qn, _ in bond_b.sectors for q in qn], dtype=np.int32)
    return qa, qb, nsec, degs, kq, kposA, fposA, kposB, fposB, bond_b.nsym


def _call(tnx, torch, stream, T):
    qa, qb, nsec, degs, kq, kposA, fposA, kposB, fposB, nsym = _first_step_operands(T)
    dqa = torch.from_numpy(np.ascontiguousarray(qa, dtype=np.int32)).cuda()
    dqb = torch.from_numpy(np.ascontiguousarray(qb, dtype=np.int32)).cuda()
    gmax = 4096
    ng = torch.zeros(1, dtype=torch.int32, device="cuda")
    ch = torch.zeros(gmax * nsym, dtype=torch.int32, device="cuda")
    mkn = torch.zeros(gmax * 3, dtype=torch.int64, device="cuda")
    am = torch.zeros(len(qa) * 3, dtype=torch.int64, device="cuda")
    bm = torch.zeros(len(qb) * 3, dtype=torch.int64, device="cuda")
    zn = np.zeros(max(nsym, 1), dtype=np.int32)
    ka, fa = np.array(kposA, dtype=np.int32), np.array(fposA, dtype=np.int32)
    kb, fb = np.array(kposB, dtype=np.int32), np.array(fposB, dtype=np.int32)
    err = C.create_string_buffer(512)
    torch.cuda.synchronize()
    f = tnx.lib().tnx_match_tables_noalloc
    f.restype = C.c_int
    code = f(C.c_void_p(stream.cuda_stream), nsym, _u(zn), len(kposA), len(fposA), len(fposB), _u(nsec), _l(degs),
             _u(kq), C.c_int64(len(qa)), qa.shape[1], C.c_void_p(dqa.data_ptr()), _u(ka), _u(fa),
             C.c_int64(len(qb)), qb.shape[1], C.c_void_p(dqb.data_ptr()), _u(kb), _u(fb), gmax,
             C.c_void_p(ng.data_ptr()), C.c_void_p(ch.data_ptr()), C.c_void_p(mkn.data_ptr()),
             C.c_void_p(am.data_ptr()), C.c_void_p(bm.data_ptr()), err, C.c_size_t(512))
    assert code == 0, err.value.decode()
    G = int(ng.item())
    return {"charges": ch[:G * nsym].cpu().numpy().reshape(G, nsym), "MKN": mkn[:G * 3].cpu().numpy().reshape(G, 3),
            "amap": am.cpu().numpy().reshape(-1, 3), "bmap": bm.cpu().numpy().reshape(-1, 3)}


def test_no_alloc_tables_match_the_allocating_path_twice():
    import torch

    import paper_2401_01921_gb300 as tnx
    from paper_2401_01921_gb300 import build
    from paper_2401_01921_gb300.heff import build_network
    build.build()
    ctx = tnx.Context(0)
    stream = torch.cuda.Stream()
    order = "(L,(((psi,R),W2),W1))"
    for wl in (I.heisenberg_workload(512, 20), I.hubbard_workload(256)):
        bonds = I.heff_bonds(wl)
        tensors = {n: (bonds[n], I.heff_value_fn(wl, n)) for n in I.HEFF_NAMES}
        net, T, B = build_network(ctx, I.HEFF_SPEC, tensors, wl.nsym, order=order)
        want = net.step_tables(0)
        got = _call(tnx, torch, stream, T)
        for key in ("charges", "MKN", "amap", "bmap"):
            assert np.array_equal(got[key], want[key]), key
