"""The allocation-free entry point tnx_match_tables_noalloc, called through the C-ABI.

It serves callers that cannot allocate device memory where they need the
fused charge-sector tables of a contraction (their memory is owned by another
framework or sized up front).  Its working memory is a fixed device array
inside the library.  The GPU test checks, on two calls in a row (the second
one reusing the array the first one left behind), that it returns exactly the
tables the allocating path reports through tnx_network_step_tables and the
oracle's tables of the same step.  Integer tables: the comparison is exact.
The refusals (too little scratch, too many groups, positions that are not a
permutation of the legs, a charge space that would overflow, a sector index
out of range) are checked too; all but the last two GPU cases return before
any device work, so they run on the CPU.

The file is named to run last, so a run that stops at the first failure has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

import tnx_inputs as I

TNX_ERR_ARG = -1
TNX_ERR_UNSUPPORTED = -9
ORDER = "(L,(((psi,R),W2),W1))"


def _u(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _l(a):
    return a.ctypes.data_as(C.POINTER(C.c_int64))


def _lib():
    import paper_2401_01921_gb300 as tnx
    from paper_2401_01921_gb300 import build
    build.build()
    f = tnx.lib().tnx_match_tables_noalloc
    f.restype = C.c_int
    return f


def _raw(f, stream, nsym, zn, nsec, degs, kq, nk, nfa, nfb, nA, rA, qA, kposA, fposA, nB, rB, qB, kposB, fposB, gmax,
         outs=(None, None, None, None, None)):
    """Calls the entry point; qA / qB and the outputs are device pointers (ints) or None."""
    err = C.create_string_buffer(512)
    i32 = lambda a: np.ascontiguousarray(a, dtype=np.int32)
    zn, nsec, kq = i32(zn), i32(nsec), i32(kq)
    degs = np.ascontiguousarray(degs, dtype=np.int64)
    ka, fa, kb, fb = i32(kposA), i32(fposA), i32(kposB), i32(fposB)
    ng, ch, mkn, am, bm = [C.c_void_p(x) for x in outs]
    code = f(C.c_void_p(stream), nsym, _u(zn), nk, nfa, nfb, _u(nsec), _l(degs), _u(kq), C.c_int64(nA), rA,
             C.c_void_p(qA), _u(ka), _u(fa), C.c_int64(nB), rB, C.c_void_p(qB), _u(kb), _u(fb), gmax,
             ng, ch, mkn, am, bm, err, C.c_size_t(512))
    return code, err.value.decode()


def _dummy_outs():
    # host addresses that are never dereferenced: every case using them is refused before device work
    buf = np.zeros(64, dtype=np.int64)
    p = buf.ctypes.data
    return buf, (p, p, p, p, p)


def test_no_alloc_refuses_more_than_its_scratch_without_a_gpu():
    f = _lib()
    keep, outs = _dummy_outs()
    n = 1 << 21                       # one K leg of 2^21 sectors: 32 MiB of tuple-space tables
    code, msg = _raw(f, 0, 1, [0], [n], np.ones(n), np.arange(n), 1, 0, 0, 0, 1, None, [0], [], 0, 1, None, [0], [],
                     16, outs)
    assert code == TNX_ERR_UNSUPPORTED, msg
    assert "bytes of scratch" in msg and str(16 << 20) in msg, msg


def test_no_alloc_refuses_a_charge_space_that_would_overflow():
    f = _lib()
    keep, outs = _dummy_outs()
    big = 1 << 20                     # three U(1) charges, each spanning 2^20 + 1 values: 2^60 charge tuples
    kq = [0, 0, 0, big, big, big]
    code, msg = _raw(f, 0, 3, [0, 0, 0], [2], [1, 1], kq, 1, 0, 0, 0, 1, None, [0], [], 0, 1, None, [0], [], 16, outs)
    assert code == TNX_ERR_UNSUPPORTED, msg
    assert "charge space" in msg, msg


@pytest.mark.parametrize("kposA,fposA,rA", [([0], [0], 2), ([0], [2], 2), ([1], [], 2), ([0], [1, 2], 2)])
def test_no_alloc_refuses_positions_that_are_not_a_permutation(kposA, fposA, rA):
    f = _lib()
    keep, outs = _dummy_outs()
    nfa = len(fposA)
    code, msg = _raw(f, 0, 1, [0], [2] * (1 + nfa), [1] * (2 * (1 + nfa)), [1, -1], 1, nfa, 0, 0, rA, None, kposA,
                     fposA, 0, 1, None, [0], [], 16, outs)
    assert code == TNX_ERR_ARG, msg


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


def _call(f, torch, stream, T, gmax=4096, corrupt=False):
    qa, qb, nsec, degs, kq, kposA, fposA, kposB, fposB, nsym = _first_step_operands(T)
    qa = np.ascontiguousarray(qa, dtype=np.int32)
    if corrupt:
        qa = qa.copy()
        qa[len(qa) // 2, 1] = nsec[2]          # one past the last sector of psi's s1 leg
    dqa = torch.from_numpy(qa).cuda()
    dqb = torch.from_numpy(np.ascontiguousarray(qb, dtype=np.int32)).cuda()
    ng = torch.zeros(1, dtype=torch.int32, device="cuda")
    ch = torch.zeros(gmax * nsym, dtype=torch.int32, device="cuda")
    mkn = torch.zeros(gmax * 3, dtype=torch.int64, device="cuda")
    am = torch.full((len(qa) * 3,), -7, dtype=torch.int64, device="cuda")
    bm = torch.zeros(len(qb) * 3, dtype=torch.int64, device="cuda")
    zn = np.zeros(max(nsym, 1), dtype=np.int32)
    torch.cuda.synchronize()
    code, msg = _raw(f, stream.cuda_stream, nsym, zn, nsec, degs, kq, len(kposA), len(fposA), len(fposB), len(qa),
                     qa.shape[1], dqa.data_ptr(), kposA, fposA, len(qb), qb.shape[1], dqb.data_ptr(), kposB, fposB,
                     gmax, (ng.data_ptr(), ch.data_ptr(), mkn.data_ptr(), am.data_ptr(), bm.data_ptr()))
    if code != 0:
        return code, msg, {"amap": am.cpu().numpy().reshape(-1, 3)}
    G = int(ng.item())
    return code, msg, {"charges": ch[:G * nsym].cpu().numpy().reshape(G, nsym),
                       "MKN": mkn[:G * 3].cpu().numpy().reshape(G, 3),
                       "amap": am.cpu().numpy().reshape(-1, 3), "bmap": bm.cpu().numpy().reshape(-1, 3)}


@pytest.mark.gpu
def test_no_alloc_tables_match_the_allocating_path_and_the_oracle_twice():
    import torch

    import paper_2401_01921_gb300 as tnx
    from oracle import heff as oheff
    from paper_2401_01921_gb300.heff import build_network
    f = _lib()
    ctx = tnx.Context(0)
    stream = torch.cuda.Stream()
    for wl in (I.heisenberg_workload(512, 20), I.hubbard_workload(256)):
        bonds = I.heff_bonds(wl)
        tensors = {n: (bonds[n], I.heff_value_fn(wl, n)) for n in I.HEFF_NAMES}
        net, T, B = build_network(ctx, I.HEFF_SPEC, tensors, wl.nsym, order=ORDER)
        want = net.step_tables(0)
        onet, _ = oheff.make_heff(wl, order=ORDER)
        rec = []
        onet.launch(record=rec)
        oracle = rec[0]["tables"]
        for _ in range(2):
            code, msg, got = _call(f, torch, stream, T)
            assert code == 0, msg
            for key in ("charges", "MKN", "amap", "bmap"):
                assert np.array_equal(got[key], want[key]), key
                ref = oracle[key].astype(np.int32) if key == "charges" else oracle[key]
                assert np.array_equal(got[key], ref), key


@pytest.mark.gpu
def test_no_alloc_reports_too_many_groups_and_bad_sector_indices():
    import torch

    import paper_2401_01921_gb300 as tnx
    from paper_2401_01921_gb300.heff import build_network
    f = _lib()
    ctx = tnx.Context(0)
    stream = torch.cuda.Stream()
    wl = I.heisenberg_workload(64, 8)
    bonds = I.heff_bonds(wl)
    tensors = {n: (bonds[n], I.heff_value_fn(wl, n)) for n in I.HEFF_NAMES}
    net, T, B = build_network(ctx, I.HEFF_SPEC, tensors, wl.nsym, order=ORDER)
    code, msg, _ = _call(f, torch, stream, T, gmax=1)
    assert code == TNX_ERR_UNSUPPORTED and "exceed gmax = 1" in msg, msg
    code, msg, got = _call(f, torch, stream, T, corrupt=True)
    assert code == TNX_ERR_ARG and "sector index" in msg, msg
    assert np.all(got["amap"] == -7)            # nothing written
    code, msg, got = _call(f, torch, stream, T)   # the array is fine for the next call
    assert code == 0, msg
    assert np.array_equal(got["amap"], net.step_tables(0)["amap"])
