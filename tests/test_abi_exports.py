"""The C ABI library loads without a GPU and exports every function include/ipcheck.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    text = open(os.path.join(ROOT, "include", "ipcheck.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_ ]*?[\s\*]+([A-Za-z_][A-Za-z0-9_]*)\s*\(", text, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


@pytest.fixture(scope="module")
def libipc():
    from paper_2405_04463_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("load_db_shares", "submit_queries", "fetch_match_bits", "ipc_ring_gemm", "ipc_compare",
                     "ipc_or_finalize", "ipc_prep_query", "ipc_split_limbs", "ipc_encode_share"):
        assert required in names


def test_every_declared_symbol_is_exported(libipc):
    missing = [n for n in declared_functions() if not hasattr(libipc, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol(libipc):
    import paper_2405_04463_gb300 as ipc
    assert set(declared_functions()) <= set(ipc._SIGS)


def test_error_paths_need_no_gpu(libipc):
    import paper_2405_04463_gb300 as ipc
    # argument checks reject before touching the device
    with pytest.raises(ipc.IpcError) as e:
        ipc.ipc_split_limbs(0, 0, 0, 0, stream=0)
    assert e.value.rc == ipc.IPC_EINVAL
    g = ipc.ipc_geom(16, 200, 4, -15, 40)   # R > 31
    with pytest.raises(ipc.IpcError):
        ipc.ipc_prep_query(8, 1, g, 0, 8, 8, 128, stream=0)
    with pytest.raises(ipc.IpcError):
        ipc.ipc_ring_gemm("i8mma", [16, 16], [16, 16], 10, 16, 16, 4, 128, 100, 16, 0, 0, 0, 16, 16, 0, stream=0)
    assert "l must be" in ipc.ipc_last_error()


def test_fused_setting_is_validated_without_gpu(libipc):
    """ipc_config.fused reaches the library at its declared place in the struct: a fused context
    on a path without the fused kernel, or with public masks or a lifting variant, is refused by
    the argument checks, before any device call."""
    import paper_2405_04463_gb300 as ipc
    g = ipc.ipc_geom(16, 200, 4, -15, 31)
    for kw in (dict(path="i8mma"), dict(path="i32"), dict(path="tc", plain_mask=True), dict(path="tc", lift="const")):
        with pytest.raises(ipc.IpcError) as e:
            ipc.ipc_create(ipc.make_config(g, fused=True, **kw))
        assert e.value.rc == ipc.IPC_EINVAL and "fused" in str(e.value), kw
