"""Python binding of the tnx C-ABI (include/tnx.h): argument marshalling only.

Every computation runs in libtnx.so (sm_103a CUDA kernels).  There is no CPU
fallback: importing this package without the built library raises.  PyTorch
is used for device memory (the allocator callback) and streams.

``lib()`` returns the loaded library, whose functions carry the C names
(``lib().tnx_bond_create`` ...); the small classes below only wrap handles and
convert arrays.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtnx.so")

TNX_OK = 0
ERRORS = {
    -1: "TNX_ERR_ARG", -2: "TNX_ERR_BOND_MISMATCH", -3: "TNX_ERR_SYMMETRY", -4: "TNX_ERR_NO_BLOCK",
    -5: "TNX_ERR_NETWORK", -6: "TNX_ERR_OOM", -7: "TNX_ERR_TIMEOUT", -8: "TNX_ERR_CUDA", -9: "TNX_ERR_UNSUPPORTED",
}
U1, ZN = 0, 1
BD_IN, BD_OUT, BD_REG = 1, -1, 0
PREC_F64, PREC_SPLIT_BF16, PREC_SPLIT_F16, PREC_F32, PREC_TF32 = 0, 1, 2, 3, 4
PREC_NAMES = {"f64": 0, "split_bf16": 1, "split_f16": 2, "f32": 3, "tf32": 4}


class TnxError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


def _load() -> C.CDLL:
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libtnx.so is not built ({LIB_PATH}); run paper_2401_01921_gb300.build.build()")
    return C.CDLL(LIB_PATH)


_lib = None
ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)
_p = C.c_void_p
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)
_SIGS = {
    "tnx_last_error": (C.c_char_p, [_p]),
    "tnx_version": (C.c_char_p, []),
    "tnx_ctx_create": (C.c_int, [C.c_int, _p, ALLOC_FN, FREE_FN, _p, C.POINTER(_p)]),
    "tnx_ctx_destroy": (C.c_int, [_p]),
    "tnx_sync": (C.c_int, [_p]),
    "tnx_bond_create": (C.c_int, [_p, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_int, _i32p, _i64p,
                                  C.POINTER(_p)]),
    "tnx_bond_dim": (C.c_int, [_p, _i64p]),
    "tnx_bond_combine": (C.c_int, [_p, _p, C.POINTER(_p)]),
    "tnx_bond_sectors": (C.c_int, [_p, C.POINTER(C.c_int), _i32p, _i64p]),
    "tnx_bond_destroy": (C.c_int, [_p]),
    "tnx_bond_info": (C.c_int, [_p, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "tnx_tensor_bond": (C.c_int, [_p, C.c_int, C.POINTER(_p)]),
    "tnx_tensor_create": (C.c_int, [_p, C.c_int, C.POINTER(_p), C.POINTER(_p)]),
    "tnx_tensor_destroy": (C.c_int, [_p]),
    "tnx_tensor_rank": (C.c_int, [_p, C.POINTER(C.c_int)]),
    "tnx_tensor_nblocks": (C.c_int, [_p, _i64p]),
    "tnx_tensor_block_info": (C.c_int, [_p, C.c_int64, _i32p, _i64p, _i64p]),
    "tnx_tensor_blocks": (C.c_int, [_p, _i32p, _i64p, _i64p]),
    "tnx_tensor_data": (C.c_int, [_p, C.POINTER(_p), _i64p]),
    "tnx_tensor_put_block": (C.c_int, [_p, _i32p, C.POINTER(C.c_double), C.c_int64]),
    "tnx_tensor_get_block": (C.c_int, [_p, _i32p, C.POINTER(C.c_double), C.c_int64]),
    "tnx_tensor_upload": (C.c_int, [_p, C.POINTER(C.c_double), C.c_int64]),
    "tnx_tensor_download": (C.c_int, [_p, C.POINTER(C.c_double), C.c_int64]),
    "tnx_tensor_scale": (C.c_int, [_p, C.c_double]),
    "tnx_tensor_add_scalar": (C.c_int, [_p, C.c_double]),
    "tnx_tensor_norm": (C.c_int, [_p, C.POINTER(C.c_double)]),
    "tnx_tensor_dagger": (C.c_int, [_p, C.POINTER(_p)]),
    "tnx_svd_truncate": (C.c_int, [_p, C.c_int, C.c_int64, C.c_double, _i64p, C.c_int, C.c_int, C.POINTER(_p),
                                   C.POINTER(_p), C.POINTER(_p), C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "tnx_network_create": (C.c_int, [_p, C.c_char_p, C.POINTER(_p)]),
    "tnx_network_destroy": (C.c_int, [_p]),
    "tnx_network_put": (C.c_int, [_p, C.c_char_p, _p, C.c_int, C.POINTER(C.c_char_p)]),
    "tnx_network_set_order": (C.c_int, [_p, C.c_int, C.c_char_p]),
    "tnx_network_get_order": (C.c_int, [_p, C.c_char_p, C.c_size_t]),
    "tnx_network_set_precision": (C.c_int, [_p, C.c_int]),
    "tnx_network_launch": (C.c_int, [_p, C.POINTER(_p)]),
    "tnx_network_launch_into": (C.c_int, [_p, _p]),
    "tnx_network_flops": (C.c_int, [_p, C.POINTER(C.c_double)]),
    "tnx_network_nsteps": (C.c_int, [_p, C.POINTER(C.c_int)]),
    "tnx_network_resident": (C.c_int, [_p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "tnx_network_step_sizes": (C.c_int, [_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int), _i64p, _i64p]),
    "tnx_network_step_tables": (C.c_int, [_p, C.c_int, _i32p, _i64p, _i64p, _i64p]),
    "tnx_lanczos": (C.c_int, [_p, C.c_char_p, _p, C.c_int, C.POINTER(C.c_double), _p, C.POINTER(C.c_int)]),
    "tnx_dmrg_create": (C.c_int, [_p, C.c_int, _p, C.c_int, C.c_int, _i32p, C.POINTER(_p)]),
    "tnx_dmrg_destroy": (C.c_int, [_p]),
    "tnx_dmrg_sweep": (C.c_int, [_p, C.c_int64, C.c_double, C.c_int, C.c_int, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), _i64p, C.POINTER(C.c_double)]),
    "tnx_dmrg_tensor": (C.c_int, [_p, C.c_int, C.POINTER(_p)]),
    "tnx_batch_create": (C.c_int, [_p, C.c_int, C.POINTER(_p), C.POINTER(_p)]),
    "tnx_batch_destroy": (C.c_int, [_p]),
    "tnx_batch_launch_into": (C.c_int, [_p, C.POINTER(_p)]),
    "tnx_batch_flops": (C.c_int, [_p, C.POINTER(C.c_double)]),
    "tnx_batch_autotune": (C.c_int, [_p, C.POINTER(_p), C.POINTER(C.c_int)]),
    "tnx_server_create": (C.c_int, [_p, C.c_int, C.c_size_t, C.POINTER(_p)]),
    "tnx_server_destroy": (C.c_int, [_p]),
    "tnx_server_submit": (C.c_int, [_p, _p, C.c_char_p, _p, C.c_int, C.c_int, _p, _i64p]),
    "tnx_server_wait": (C.c_int, [_p, C.c_int64, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int),
                                  C.POINTER(C.c_double)]),
    "tnx_server_stats": (C.c_int, [_p, _i64p, _i64p, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "tnx_profile_enable": (C.c_int, [_p, C.c_int]),
    "tnx_profile_read": (C.c_int, [_p, C.POINTER(C.c_double), _i64p, C.POINTER(C.c_double)]),
    "tnx_kernel_launches": (C.c_int, [_i64p]),
    "tnx_profile_classes": (C.c_int, [C.c_void_p, C.c_uint32]),
}
KERNEL_CLASSES = ["match", "relayout", "gemm", "slice", "vector", "final", "skinny"]


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        L = _load()
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _check(ctx_handle, code: int):
    if code != TNX_OK:
        msg = lib().tnx_last_error(ctx_handle) if ctx_handle else b""
        raise TnxError(code, (msg or b"").decode())


# ---------------------------------------------------------------- objects
class Context:
    """tnx_ctx over a CUDA device; device memory from PyTorch's caching allocator."""

    def __init__(self, device: int = 0, stream=None, torch_alloc: bool = True):
        import torch
        self._torch = torch
        self.device = device
        self._keep: dict[int, object] = {}
        if stream is None:
            # a stream of its own: CUDA graphs cannot be captured on the legacy default stream
            stream = torch.cuda.Stream(device)
        self.stream = stream
        sp = C.c_void_p(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        if torch_alloc:
            dev = torch.device("cuda", device)

            def _alloc(n, user):
                try:
                    with torch.cuda.stream(self.stream):
                        t = torch.empty(int(n), dtype=torch.uint8, device=dev)
                except RuntimeError:
                    return None
                p = t.data_ptr()
                self._keep[p] = t
                return p

            def _free(p, n, user):
                self._keep.pop(p, None)

            self._alloc_cb = ALLOC_FN(_alloc)
            self._free_cb = FREE_FN(_free)
        else:
            self._alloc_cb = ALLOC_FN()
            self._free_cb = FREE_FN()
        h = C.c_void_p()
        code = lib().tnx_ctx_create(device, sp, self._alloc_cb, self._free_cb, None, C.byref(h))
        if code != TNX_OK:
            raise TnxError(code, "tnx_ctx_create failed")
        self.h = h

    def check(self, code):
        _check(self.h, code)

    def sync(self):
        self.check(lib().tnx_sync(self.h))

    def close(self):
        if self.h:
            lib().tnx_ctx_destroy(self.h)
            self.h = None

    def profile(self, enable: bool, classes=None, last_apply_only: bool = False):
        """tnx_profile_enable / tnx_profile_classes: CUDA-event timing of every kernel
        class, or only of the named ones (e.g. classes=["gemm"]); last_apply_only:
        Lanczos solves time only the apply of their last step."""
        if classes is None and not last_apply_only:
            self.check(lib().tnx_profile_enable(self.h, 1 if enable else 0))
        else:
            names = KERNEL_CLASSES if classes is None else classes
            mask = sum(1 << KERNEL_CLASSES.index(c) for c in names) if enable else 0
            if mask and last_apply_only:
                mask |= 0x80000000
            self.check(lib().tnx_profile_classes(self.h, mask))

    def profile_read(self) -> dict:
        """{class: (milliseconds, launches, algorithmic work)} since profile(True)."""
        n = len(KERNEL_CLASSES)
        ms = (C.c_double * n)()
        cnt = (C.c_int64 * n)()
        work = (C.c_double * n)()
        self.check(lib().tnx_profile_read(self.h, ms, cnt, work))
        return {k: (ms[i], cnt[i], work[i]) for i, k in enumerate(KERNEL_CLASSES)}


def kernel_launches() -> int:
    """tnx_kernel_launches: CUDA kernels launched by the library in this process."""
    n = C.c_int64()
    lib().tnx_kernel_launches(C.byref(n))
    return n.value


class Bond:
    """tnx_bond: direction, sectors [(charge tuple, degeneracy)], symmetries [U1 | (ZN, n)]."""

    def __init__(self, ctx: Context, dir: int, sectors, syms=()):
        self.ctx = ctx
        syms = list(syms)
        kinds = np.array([U1 if s == U1 else ZN for s in syms] or [0], dtype=np.int32)
        zn = np.array([0 if s == U1 else s[1] for s in syms] or [0], dtype=np.int32)
        nsym = len(syms)
        q = np.array([c for qn, _ in sectors for c in qn] or [0], dtype=np.int32)
        d = np.array([dg for _, dg in sectors], dtype=np.int64)
        h = C.c_void_p()
        ctx.check(lib().tnx_bond_create(ctx.h, dir, nsym, _ptr(kinds, C.c_int), _ptr(zn, C.c_int), len(sectors),
                                        _ptr(q, C.c_int32), _ptr(d, C.c_int64), C.byref(h)))
        self.h = h
        self.dir = dir
        self.sectors = [(tuple(int(c) for c in qn), int(dg)) for qn, dg in sectors]
        self.nsym = nsym

    @classmethod
    def from_handle(cls, ctx: Context, h) -> "Bond":
        """Wraps a bond handle the library created (the wrapper destroys it)."""
        b = cls.__new__(cls)
        b.ctx = ctx
        b.h = h
        d, ns = C.c_int(), C.c_int()
        ctx.check(lib().tnx_bond_info(h, C.byref(d), C.byref(ns), None, None))
        kinds = np.zeros(max(ns.value, 1), dtype=np.int32)
        zn = np.zeros(max(ns.value, 1), dtype=np.int32)
        ctx.check(lib().tnx_bond_info(h, None, None, _ptr(kinds, C.c_int), _ptr(zn, C.c_int)))
        nsec = C.c_int()
        ctx.check(lib().tnx_bond_sectors(h, C.byref(nsec), None, None))
        q = np.zeros(max(nsec.value * ns.value, 1), dtype=np.int32)
        dg = np.zeros(nsec.value, dtype=np.int64)
        ctx.check(lib().tnx_bond_sectors(h, C.byref(nsec), _ptr(q, C.c_int32), _ptr(dg, C.c_int64)))
        b.dir = d.value
        b.nsym = ns.value
        b.sectors = [(tuple(int(x) for x in q[i * ns.value:(i + 1) * ns.value]), int(dg[i])) for i in range(nsec.value)]
        return b

    @property
    def dim(self) -> int:
        return sum(d for _, d in self.sectors)

    def offsets(self):
        return np.concatenate([[0], np.cumsum([d for _, d in self.sectors])])

    def __del__(self):
        try:
            if self.h:
                lib().tnx_bond_destroy(self.h)
        except Exception:
            pass


class Tensor:
    """tnx_tensor: block-sparse FP64 tensor in device memory."""

    def __init__(self, ctx: Context, bonds, handle=None):
        self.ctx = ctx
        self.bonds = list(bonds)
        if handle is None:
            arr = (C.c_void_p * max(1, len(bonds)))(*[b.h for b in bonds])
            h = C.c_void_p()
            ctx.check(lib().tnx_tensor_create(ctx.h, len(bonds), arr, C.byref(h)))
            handle = h
        self.h = handle
        self.rank = len(bonds)
        n = C.c_int64()
        ctx.check(lib().tnx_tensor_nblocks(self.h, C.byref(n)))
        self.nblocks = n.value
        p = C.c_void_p()
        ne = C.c_int64()
        ctx.check(lib().tnx_tensor_data(self.h, C.byref(p), C.byref(ne)))
        self.data_ptr = p.value
        self.nelem = ne.value

    @classmethod
    def from_handle(cls, ctx: Context, h) -> "Tensor":
        """Wraps a tensor handle the library created (its bonds are read back)."""
        r = C.c_int()
        ctx.check(lib().tnx_tensor_rank(h, C.byref(r)))
        bonds = []
        for leg in range(r.value):
            bh = C.c_void_p()
            ctx.check(lib().tnx_tensor_bond(h, leg, C.byref(bh)))
            bonds.append(Bond.from_handle(ctx, bh))
        return cls(ctx, bonds, handle=h)

    def dagger(self) -> "Tensor":
        """tnx_tensor_dagger: every bond redirected, the same blocks (Sec. 6.4)."""
        h = C.c_void_p()
        self.ctx.check(lib().tnx_tensor_dagger(self.h, C.byref(h)))
        return Tensor.from_handle(self.ctx, h)

    def blocks(self):
        """(qn [nblk, rank] int32, shape [nblk, rank] int64, offset [nblk] int64)."""
        r = max(self.rank, 1)
        qn = np.zeros((self.nblocks, r), dtype=np.int32)
        sh = np.zeros((self.nblocks, r), dtype=np.int64)
        off = np.zeros(self.nblocks, dtype=np.int64)
        self.ctx.check(lib().tnx_tensor_blocks(self.h, _ptr(qn, C.c_int32), _ptr(sh, C.c_int64), _ptr(off, C.c_int64)))
        return qn[:, :self.rank], sh[:, :self.rank], off

    def upload(self, x: np.ndarray):
        x = np.ascontiguousarray(x, dtype=np.float64)
        self.ctx.check(lib().tnx_tensor_upload(self.h, _ptr(x, C.c_double), x.size))

    def download(self) -> np.ndarray:
        x = np.zeros(self.nelem, dtype=np.float64)
        self.ctx.check(lib().tnx_tensor_download(self.h, _ptr(x, C.c_double), x.size))
        return x

    def put_block(self, qn, data):
        q = np.ascontiguousarray(qn, dtype=np.int32)
        d = np.ascontiguousarray(data, dtype=np.float64)
        self.ctx.check(lib().tnx_tensor_put_block(self.h, _ptr(q, C.c_int32), _ptr(d, C.c_double), d.size))

    def get_block(self, qn, shape):
        q = np.ascontiguousarray(qn, dtype=np.int32)
        d = np.zeros(int(np.prod(shape)), dtype=np.float64)
        self.ctx.check(lib().tnx_tensor_get_block(self.h, _ptr(q, C.c_int32), _ptr(d, C.c_double), d.size))
        return d.reshape(shape)

    def scale(self, a: float):
        self.ctx.check(lib().tnx_tensor_scale(self.h, a))

    def add_scalar(self, a: float):
        self.ctx.check(lib().tnx_tensor_add_scalar(self.h, a))

    def norm(self) -> float:
        x = C.c_double()
        self.ctx.check(lib().tnx_tensor_norm(self.h, C.byref(x)))
        return x.value

    def dense_coords(self):
        """Dense (full-bond) coordinates of every stored element, in buffer order."""
        qn, sh, off = self.blocks()
        if self.rank == 0 or self.nelem == 0:
            return []
        sizes = np.prod(sh, axis=1)
        blk = np.repeat(np.arange(self.nblocks), sizes)
        local = np.arange(self.nelem, dtype=np.int64) - off[blk]
        coords = [None] * self.rank
        for l in range(self.rank - 1, -1, -1):
            ext = sh[blk, l]
            start = np.asarray(self.bonds[l].offsets())[qn[blk, l]]
            coords[l] = start + local % ext
            local = local // ext
        return coords

    def fill(self, value_at):
        """Fill every block from value_at(list of dense-coordinate arrays) and upload."""
        if self.rank == 0:
            self.upload(np.asarray(value_at([]), dtype=np.float64).reshape(1))
            return self
        if self.nelem == 0:
            return self
        self.upload(np.asarray(value_at(self.dense_coords()), dtype=np.float64).reshape(-1))
        return self

    def block_dict(self, flat=None):
        """{qn tuple: ndarray block} from a download (or the given flat array)."""
        x = self.download() if flat is None else flat
        qn, sh, off = self.blocks()
        out = {}
        for b in range(self.nblocks):
            n = int(np.prod(sh[b])) if self.rank else 1
            out[tuple(int(v) for v in qn[b])] = x[off[b]:off[b] + n].reshape(tuple(sh[b]))
        return out

    def __del__(self):
        try:
            if self.h:
                lib().tnx_tensor_destroy(self.h)
        except Exception:
            pass


class Network:
    """tnx_network: Network blueprint + put tensors + order + precision."""

    def __init__(self, ctx: Context, spec: str):
        self.ctx = ctx
        h = C.c_void_p()
        ctx.check(lib().tnx_network_create(ctx.h, spec.encode(), C.byref(h)))
        self.h = h
        self._refs = {}

    def put(self, name: str, t: Tensor, labels=None):
        if labels is None:
            ctx_code = lib().tnx_network_put(self.h, name.encode(), t.h, 0, None)
        else:
            arr = (C.c_char_p * len(labels))(*[l.encode() for l in labels])
            ctx_code = lib().tnx_network_put(self.h, name.encode(), t.h, len(labels), arr)
        self.ctx.check(ctx_code)
        self._refs[name] = t

    def set_order(self, optimal, order: str | None = None):
        """optimal: False (explicit `order`), True (dense-cost search) or "sparse"
        (block-sparse-cost search)."""
        mode = 2 if optimal == "sparse" else (1 if optimal else 0)
        self.ctx.check(lib().tnx_network_set_order(self.h, mode, order.encode() if order else None))

    def get_order(self) -> str:
        buf = C.create_string_buffer(4096)
        self.ctx.check(lib().tnx_network_get_order(self.h, buf, 4096))
        return buf.value.decode()

    def set_precision(self, prec):
        if isinstance(prec, str):
            prec = PREC_NAMES[prec]
        self.ctx.check(lib().tnx_network_set_precision(self.h, prec))

    def launch(self, out_bonds) -> Tensor:
        h = C.c_void_p()
        self.ctx.check(lib().tnx_network_launch(self.h, C.byref(h)))
        return Tensor(self.ctx, out_bonds, handle=h)

    def launch_into(self, out: Tensor):
        self.ctx.check(lib().tnx_network_launch_into(self.h, out.h))

    def flops(self) -> float:
        x = C.c_double()
        self.ctx.check(lib().tnx_network_flops(self.h, C.byref(x)))
        return x.value

    def resident(self) -> tuple:
        """(bytes held now, bytes its plan needs) - tnx_network_resident."""
        b, pb = C.c_size_t(), C.c_size_t()
        self.ctx.check(lib().tnx_network_resident(self.h, C.byref(b), C.byref(pb)))
        return b.value, pb.value

    def nsteps(self) -> int:
        x = C.c_int()
        self.ctx.check(lib().tnx_network_nsteps(self.h, C.byref(x)))
        return x.value

    def step_tables(self, step: int) -> dict:
        G, ns = C.c_int(), C.c_int()
        nA, nB = C.c_int64(), C.c_int64()
        self.ctx.check(lib().tnx_network_step_sizes(self.h, step, C.byref(G), C.byref(ns), C.byref(nA), C.byref(nB)))
        ch = np.zeros(max(1, G.value * ns.value), dtype=np.int32)
        mkn = np.zeros(max(1, G.value * 3), dtype=np.int64)
        am = np.zeros(max(1, nA.value * 3), dtype=np.int64)
        bm = np.zeros(max(1, nB.value * 3), dtype=np.int64)
        self.ctx.check(lib().tnx_network_step_tables(self.h, step, _ptr(ch, C.c_int32), _ptr(mkn, C.c_int64),
                                                     _ptr(am, C.c_int64), _ptr(bm, C.c_int64)))
        return {"charges": ch[:G.value * ns.value].reshape(G.value, ns.value),
                "MKN": mkn[:G.value * 3].reshape(G.value, 3),
                "amap": am[:nA.value * 3].reshape(nA.value, 3),
                "bmap": bm[:nB.value * 3].reshape(nB.value, 3)}

    def __del__(self):
        try:
            if self.h:
                lib().tnx_network_destroy(self.h)
        except Exception:
            pass


class Batch:
    """tnx_batch: many networks launched together (one launch per kernel class and step)."""

    def __init__(self, ctx: Context, nets):
        self.ctx = ctx
        self.nets = list(nets)
        arr = (C.c_void_p * len(self.nets))(*[n.h for n in self.nets])
        h = C.c_void_p()
        ctx.check(lib().tnx_batch_create(ctx.h, len(self.nets), arr, C.byref(h)))
        self.h = h

    def _outs(self, outs):
        return (C.c_void_p * len(outs))(*[o.h for o in outs])

    def launch_into(self, outs):
        self.ctx.check(lib().tnx_batch_launch_into(self.h, self._outs(outs)))

    def autotune(self, outs) -> int:
        c = C.c_int()
        self.ctx.check(lib().tnx_batch_autotune(self.h, self._outs(outs), C.byref(c)))
        return c.value

    def flops(self) -> float:
        x = C.c_double()
        self.ctx.check(lib().tnx_batch_flops(self.h, C.byref(x)))
        return x.value

    def __del__(self):
        try:
            if self.h:
                lib().tnx_batch_destroy(self.h)
        except Exception:
            pass


REQ_APPLY, REQ_LANCZOS = 0, 1


class Server:
    """tnx_server: continuous-batching request loop over resident networks."""

    def __init__(self, ctx: Context, max_slots: int = 8, hbm_budget_bytes: int = 150 * 10**9):
        self.ctx = ctx
        h = C.c_void_p()
        ctx.check(lib().tnx_server_create(ctx.h, max_slots, hbm_budget_bytes, C.byref(h)))
        self.h = h

    def submit(self, net: Network, slot: str, vec: Tensor, kind: int, nsteps: int = 0, out: Tensor | None = None) -> int:
        i = C.c_int64()
        self.ctx.check(lib().tnx_server_submit(self.h, net.h, slot.encode(), vec.h, kind, nsteps,
                                               out.h if out is not None else None, C.byref(i)))
        return i.value

    def wait(self, rid: int, timeout_ms: int = -1):
        """(eigenvalue, matvecs, latency ms) of request rid."""
        ev, mv, lat = C.c_double(), C.c_int(), C.c_double()
        self.ctx.check(lib().tnx_server_wait(self.h, rid, timeout_ms, C.byref(ev), C.byref(mv), C.byref(lat)))
        return ev.value, mv.value, lat.value

    def stats(self) -> dict:
        c, e = C.c_int64(), C.c_int64()
        u, pk = C.c_size_t(), C.c_size_t()
        self.ctx.check(lib().tnx_server_stats(self.h, C.byref(c), C.byref(e), C.byref(u), C.byref(pk)))
        return {"completed": c.value, "evictions": e.value, "used_bytes": u.value, "peak_bytes": pk.value}

    def close(self):
        if self.h:
            lib().tnx_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Dmrg:
    """tnx_dmrg: two-site DMRG sweeps of a chain with a uniform MPO (Sec. 11)."""

    def __init__(self, ctx: Context, nsites: int, W: Tensor, left_w: int, right_w: int, states):
        self.ctx = ctx
        st = np.ascontiguousarray(states, dtype=np.int32)
        h = C.c_void_p()
        ctx.check(lib().tnx_dmrg_create(ctx.h, nsites, W.h, left_w, right_w, _ptr(st, C.c_int32), C.byref(h)))
        self.h = h
        self.nsites = nsites

    def sweep(self, maxdim: int, cutoff: float = 0.0, lanczos_steps: int = 20, prec="f64") -> dict:
        e, te = C.c_double(), C.c_double()
        mb = C.c_int64()
        ph = (C.c_double * 4)()
        p = PREC_NAMES[prec] if isinstance(prec, str) else int(prec)
        self.ctx.check(lib().tnx_dmrg_sweep(self.h, maxdim, cutoff, lanczos_steps, p, C.byref(e), C.byref(te),
                                            C.byref(mb), ph))
        return {"energy": e.value, "max_trunc_err": te.value, "max_bond": mb.value,
                "ms": {"lanczos": ph[0], "svd": ph[1], "env": ph[2], "sweep": ph[3]}}

    def tensor(self, site: int) -> Tensor:
        h = C.c_void_p()
        self.ctx.check(lib().tnx_dmrg_tensor(self.h, site, C.byref(h)))
        return Tensor.from_handle(self.ctx, h)

    def close(self):
        if self.h:
            lib().tnx_dmrg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def svd_truncate(t: Tensor, rowrank: int, keepdim: int = 0, err: float = 0.0, min_blockdim=None, absorb: int = 0):
    """tnx_svd_truncate (Sec. 9.2).  Returns (U, S or None, Vdag, largest dropped value, dropped weight)."""
    mb = None if min_blockdim is None else np.ascontiguousarray(min_blockdim, dtype=np.int64)
    U, S, V = C.c_void_p(), C.c_void_p(), C.c_void_p()
    te, dw = C.c_double(), C.c_double()
    t.ctx.check(lib().tnx_svd_truncate(t.h, rowrank, keepdim, err, None if mb is None else _ptr(mb, C.c_int64),
                                       0 if mb is None else len(mb), absorb, C.byref(U),
                                       C.byref(S) if absorb == 0 else None, C.byref(V), C.byref(te), C.byref(dw)))
    Sout = Tensor.from_handle(t.ctx, S) if absorb == 0 else None
    return Tensor.from_handle(t.ctx, U), Sout, Tensor.from_handle(t.ctx, V), te.value, dw.value


def lanczos(net: Network, slot: str, v0: Tensor, nsteps: int, evec: Tensor | None = None):
    """tnx_lanczos: returns (lowest eigenvalue, number of matvecs)."""
    ev = C.c_double()
    nm = C.c_int()
    net.ctx.check(lib().tnx_lanczos(net.h, slot.encode(), v0.h, nsteps, C.byref(ev),
                                    evec.h if evec is not None else None, C.byref(nm)))
    return ev.value, nm.value
