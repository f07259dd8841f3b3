"""The C-ABI library builds for sm_103a, loads, and exports every function include/tnx.h declares.

No compute call is made (no GPU needed)."""
import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(os.path.dirname(HERE), "include", "tnx.h")


def declared_functions():
    text = open(HEADER).read()
    return re.findall(r"^(?:tnx_status|const char\*)\s+(tnx_\w+)\(", text, flags=re.M)


def test_header_declares_the_boundary():
    names = set(declared_functions())
    for n in ["tnx_ctx_create", "tnx_bond_create", "tnx_tensor_create", "tnx_network_create", "tnx_network_put",
              "tnx_network_set_order", "tnx_network_get_order", "tnx_network_launch", "tnx_lanczos",
              "tnx_network_step_tables", "tnx_sync", "tnx_last_error"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2401_01921_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    import paper_2401_01921_gb300 as tnx
    assert tnx.lib().tnx_version() == b"tnx 1.0"
