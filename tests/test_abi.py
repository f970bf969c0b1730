"""The C ABI without a GPU: the library loads, exports every function the
public header declares, and rejects bad arguments on the host before any
CUDA call."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER_DIR = os.path.join(ROOT, "include")


def declared_functions():
    names = []
    for fn in sorted(os.listdir(HEADER_DIR)):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(HEADER_DIR, fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(syev3_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1806_06698_gb300 import build as b

    b.build()
    from paper_1806_06698_gb300 import syev3

    return syev3.library()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("syev3_batched", "syev3_batched_ex", "syev3_abi_version"):
        assert required in names, names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"libsyev3.so does not export {name}"


def test_abi_version(lib):
    assert lib.syev3_abi_version() == 2


def test_host_side_argument_checks(lib):
    from paper_1806_06698_gb300 import syev3

    vp = ctypes.c_void_p
    dummy = vp(4096)
    # n < 0, bad dtype, NULL input or output: EINVAL before any CUDA call
    assert lib.syev3_batched(dummy, -1, dummy, dummy, 0, None) == syev3.SYEV3_EINVAL
    assert lib.syev3_batched(dummy, 4, dummy, dummy, 7, None) == syev3.SYEV3_EINVAL
    assert lib.syev3_batched(None, 4, dummy, dummy, 0, None) == syev3.SYEV3_EINVAL
    assert lib.syev3_batched(dummy, 4, None, dummy, 0, None) == syev3.SYEV3_EINVAL
    # misaligned for the element type
    assert lib.syev3_batched(vp(4097), 4, dummy, None, 0, None) == syev3.SYEV3_EINVAL
    # overlapping input and output
    assert lib.syev3_batched(vp(4096), 4, vp(4096 + 8), None, 0, None) == syev3.SYEV3_EINVAL
    # n == 0 is a no-op
    assert lib.syev3_batched(None, 0, None, None, 0, None) == syev3.SYEV3_OK
    assert lib.syev3_status_string(syev3.SYEV3_EINVAL).startswith(b"SYEV3_EINVAL")


def test_method_entry_point_argument_checks(lib):
    from paper_1806_06698_gb300 import syev3

    vp = ctypes.c_void_p
    dummy = vp(4096)
    ok = syev3._Method(syev3.ZF_NEWTON, syev3.DEFLATION_EISPACK)
    call = lib.syev3_batched_method
    # FP64 only; a method must be given and name known variants
    assert call(dummy, 4, vp(8192), None, syev3.SYEV3_F32, ctypes.byref(ok), None, None) == syev3.SYEV3_EINVAL
    assert call(dummy, 4, vp(8192), None, syev3.SYEV3_F64, None, None, None) == syev3.SYEV3_EINVAL
    bad_zf = syev3._Method(3, syev3.DEFLATION_SIMPLIFIED)
    bad_defl = syev3._Method(syev3.ZF_PRODUCTION, 2)
    assert call(dummy, 4, vp(8192), None, syev3.SYEV3_F64, ctypes.byref(bad_zf), None, None) == syev3.SYEV3_EINVAL
    assert call(dummy, 4, vp(8192), None, syev3.SYEV3_F64, ctypes.byref(bad_defl), None, None) == syev3.SYEV3_EINVAL
    # the forward checks apply as for syev3_batched; n == 0 is a no-op
    assert call(dummy, -1, vp(8192), None, syev3.SYEV3_F64, ctypes.byref(ok), None, None) == syev3.SYEV3_EINVAL
    assert call(None, 0, None, None, syev3.SYEV3_F64, ctypes.byref(ok), None, None) == syev3.SYEV3_OK
    assert len(syev3.METHOD_STATS) == 8


def test_workspace_entry_point_argument_checks(lib):
    from paper_1806_06698_gb300 import syev3

    vp = ctypes.c_void_p
    # the workspace is needed by the compensated form only
    assert lib.syev3_workspace_bytes(1000, syev3.SYEV3_F64) == 0
    assert lib.syev3_workspace_bytes(1000, syev3.SYEV3_F32) == 0
    need = lib.syev3_workspace_bytes(1000, syev3.SYEV3_F32_COMPENSATED)
    assert need >= 1000 * 48
    assert lib.syev3_workspace_bytes(0, syev3.SYEV3_F32_COMPENSATED) == 0
    call = lib.syev3_batched_ws
    A, lam = vp(1 << 20), vp(2 << 20)
    # missing, too small or misaligned workspace: EINVAL before any CUDA call
    assert call(A, 1000, lam, None, syev3.SYEV3_F32_COMPENSATED, None, None, 0, None) == syev3.SYEV3_EINVAL
    assert call(A, 1000, lam, None, syev3.SYEV3_F32_COMPENSATED, None, vp(4 << 20), need - 1,
                None) == syev3.SYEV3_EINVAL
    assert call(A, 1000, lam, None, syev3.SYEV3_F32_COMPENSATED, None, vp((4 << 20) + 16), need,
                None) == syev3.SYEV3_EINVAL
    # overlapping the input
    assert call(A, 1000, lam, None, syev3.SYEV3_F32_COMPENSATED, None, A, need, None) == syev3.SYEV3_EINVAL
    # n == 0 is a no-op
    assert call(None, 0, None, None, syev3.SYEV3_F32_COMPENSATED, None, None, 0, None) == syev3.SYEV3_OK


def test_selftest_arith_argument_checks(lib):
    from paper_1806_06698_gb300 import syev3

    vp = ctypes.c_void_p
    call = lib.syev3_selftest_arith
    # every operation the header names (the reciprocal and root helpers and
    # the two integer-pipe conversions) takes n == 0 as a no-op
    for op in (syev3.ARITH_RCP64, syev3.ARITH_RCP32, syev3.ARITH_SQRT32, syev3.ARITH_RSQRT32, syev3.ARITH_F2D,
               syev3.ARITH_D2F):
        assert call(op, None, None, 0, None) == syev3.SYEV3_OK, op
    # an unknown operation or n < 0: EINVAL before any CUDA call
    assert call(syev3.ARITH_D2F + 1, vp(4096), vp(8192), 4, None) == syev3.SYEV3_EINVAL
    assert call(-1, vp(4096), vp(8192), 4, None) == syev3.SYEV3_EINVAL
    assert call(syev3.ARITH_F2D, vp(4096), vp(8192), -1, None) == syev3.SYEV3_EINVAL
    # the conversions read and write different element sizes: a double side
    # misaligned for 8 bytes, or output overlapping input, is rejected
    assert call(syev3.ARITH_F2D, vp(4096), vp(8196), 4, None) == syev3.SYEV3_EINVAL
    assert call(syev3.ARITH_D2F, vp(4100), vp(8192), 4, None) == syev3.SYEV3_EINVAL
    assert call(syev3.ARITH_F2D, vp(4096), vp(4104), 4, None) == syev3.SYEV3_EINVAL
