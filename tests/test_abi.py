"""The C ABI library loads and exports every function include/*.h declares;
host-side argument checks that need no GPU."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

from paper_2604_21128_gb300 import build as qbuild
from paper_2604_21128_gb300 import qla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b([a-z_][a-z0-9_]*)\s*\(", text):
            name = m.group(1)
            start = text.rfind("\n", 0, m.start()) + 1
            line = text[start:m.start()]
            if name in ("sizeof", "defined") or line.strip().startswith("#"):
                continue
            if re.search(r"(qla_status|size_t|void|long long|const char \*|int)\s*\**\s*$", line):
                names.append(name)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    qbuild.build()
    return qla.load()


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ("qla_init_grid", "qla_set_medium", "qla_set_packet", "qla_step",
                     "qla_energy", "qla_fields"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(lib, name), name
    so = qbuild.LIB
    out = os.popen("nm -D --defined-only %s" % so).read()
    for name in names:
        assert re.search(r"\bT %s\b" % name, out), name


def test_workspace_bytes_host_only(lib):
    assert qla.qla_workspace_bytes(0, 5, qla.QLA_FP64, 0) == 0
    assert qla.qla_workspace_bytes(5, 5, 7, 0) == 0
    b64 = qla.qla_workspace_bytes(256, 256, qla.QLA_FP64, 0)
    b32te = qla.qla_workspace_bytes(256, 256, qla.QLA_FP32, qla.QLA_TE_ONLY)
    assert b64 > 2 * 6 * 256 * 256 * 8 and b32te < b64
    # the state ping-pong buffers dominate at scale: 8192^2 FP32 E_z mode
    big = qla.qla_workspace_bytes(8192, 8192, qla.QLA_FP32, qla.QLA_TE_ONLY)
    assert 2 * 3 * 8192 * 8192 * 4 < big < 10 * 8192 * 8192 * 8


def test_double_single_workspace_host_only(lib):
    ds = qla.QLA_DOUBLE_SINGLE
    plain = qla.qla_workspace_bytes(256, 64, qla.QLA_FP64, qla.QLA_TE_ONLY)
    with_ds = qla.qla_workspace_bytes(256, 64, qla.QLA_FP64, qla.QLA_TE_ONLY | ds)
    assert with_ds > plain   # plus one 96-byte double-single record per site
    for nx, ny, prec, flags in [(256, 64, qla.QLA_FP32, ds), (32, 64, qla.QLA_FP64, ds),
                                (65, 64, qla.QLA_FP64, ds), (256, 4, qla.QLA_FP64, ds),
                                (256, 64, qla.QLA_FP64, ds | qla.QLA_POTENTIAL_LITERAL),
                                (256, 64, qla.QLA_FP64, ds | qla.QLA_ANISOTROPIC)]:
        assert qla.qla_workspace_bytes(nx, ny, prec, flags) == 0, (nx, ny, prec, flags)


def test_lattices_past_the_32_bit_offsets_are_refused_host_only(lib):
    """The marching kernels address planes x ny x pitch elements with 32-bit
    offsets: 32768 x 27000 fits with three live planes, not with six."""
    nx, ny = 32768, 27000
    assert 3 * ny * nx <= 2 ** 32 < 6 * ny * nx
    ds = qla.QLA_DOUBLE_SINGLE
    assert qla.qla_workspace_bytes(nx, ny, qla.QLA_FP64, qla.QLA_TE_ONLY | ds) > 0
    assert qla.qla_workspace_bytes(nx, ny, qla.QLA_FP64, ds) == 0
    # plain contexts stay valid (lattices the marching kernel declines step
    # on the tile kernel, whose offsets are 64-bit)
    assert qla.qla_workspace_bytes(nx, ny, qla.QLA_FP32, 0) > 0
    lib_ = qla.load()
    one = lambda v: np.array([v], dtype=np.int32)
    nxa, nya = one(nx), one(ny)
    wb = lambda flags: int(lib_.qla_batch_workspace_bytes(
        1, ctypes.c_void_p(nxa.ctypes.data), ctypes.c_void_p(nya.ctypes.data), qla.QLA_FP32, flags))
    assert wb(qla.QLA_TE_ONLY) > 0
    assert wb(0) == 0


def test_lattices_past_the_32_bit_record_ids_are_refused_host_only(lib):
    """Per-site record indices are 32-bit (4096 shared slots, then one own
    record per site), so nx * ny + 4096 must stay below 2^32."""
    assert 65536 * 65535 + 4096 < 2 ** 32 <= 65536 * 65536 + 4096
    assert qla.qla_workspace_bytes(65536, 65535, qla.QLA_FP32, qla.QLA_TE_ONLY) > 0
    assert qla.qla_workspace_bytes(65536, 65536, qla.QLA_FP32, qla.QLA_TE_ONLY) == 0
    assert qla.qla_workspace_bytes(131072, 32768, qla.QLA_FP32, qla.QLA_TE_ONLY) == 0
    with pytest.raises(qla.QLAError) as e:
        qla.qla_init_grid(65536, 65536, 1.0, qla.QLA_FP32, qla.QLA_TE_ONLY, 0, 0, 0)
    assert e.value.status == 1


@pytest.mark.parametrize("args", [
    (0, 4, 1.0, 0, 0), (4, 0, 1.0, 0, 0), (4, 4, 0.0, 0, 0), (4, 4, float("nan"), 0, 0),
    (4, 4, 1.0, 2, 0), (4, 4, 1.0, 0, 64), (4, 4, 1.0, 0, 2 | 4)])
def test_init_rejects_bad_arguments_before_any_device_call(lib, args):
    nx, ny, d, prec, flags = args
    with pytest.raises(qla.QLAError) as e:
        qla.qla_init_grid(nx, ny, d, prec, flags, 0, 0, 0)
    assert e.value.status == 1


def test_march_plan_of_a_null_context_host_only(lib):
    assert lib.qla_march_plan(None, None, None, None) == 1   # QLA_EINVAL


def test_plateau_unit_workspace_host_only(lib):
    """FP32 E_z and double-single E_z contexts hold a plateau unit list;
    its size grows with the lattice, not with the tuning."""
    te = qla.QLA_TE_ONLY
    a = qla.qla_workspace_bytes(1024, 512, qla.QLA_FP32, te)
    b = qla.qla_workspace_bytes(1024, 1024, qla.QLA_FP32, te)
    assert b > a > 0
    ds = qla.QLA_DOUBLE_SINGLE
    assert qla.qla_workspace_bytes(1024, 512, qla.QLA_FP64, te | ds) > \
        qla.qla_workspace_bytes(1024, 512, qla.QLA_FP64, te)


def test_status_strings(lib):
    lib.qla_status_string.restype = ctypes.c_char_p
    assert lib.qla_status_string(0) == b"QLA_OK"
    assert lib.qla_status_string(5) == b"QLA_ETIMEOUT"


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2604_21128_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.*"), recursive=True):
        if path.endswith((".py", ".cu", ".h", ".cuh")):
            text = open(path).read()
            assert "import oracle" not in text and "from oracle" not in text, path
            assert "qla_oracle" not in text and "orc_" not in text, path
