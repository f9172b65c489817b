"""qla_energy_noalloc: the energy entry point for callers that cannot
allocate device memory (their device memory belongs to another allocator,
or they must not call into the CUDA allocator at all).  It keeps its partial
sums in a fixed array inside the library; this checks it through the C ABI
against qla_energy, on two calls in a row with different inputs, and that a
lattice larger than that array allows is refused.

Collected last so a failure here does not hide any other test's result."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2604_21128_gb300 import build as qbuild
from paper_2604_21128_gb300 import inputs, qla

pytestmark = pytest.mark.gpu

SITES_MAX = 16384 * 16384


def _lib():
    qbuild.build()
    lib = qla.load()
    lib.qla_energy_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_longlong, ctypes.c_longlong,
                                       ctypes.c_void_p, ctypes.c_void_p]
    lib.qla_energy_noalloc.restype = ctypes.c_int
    return lib


def test_energy_noalloc_matches_qla_energy_on_two_calls():
    import torch
    lib = _lib()
    stream = torch.cuda.current_stream()
    cases = [(200, 136, "fp64", False, 11), (256, 190, "fp32", True, 12)]
    results = []
    for nx, ny, prec, te, seed in cases:
        q = inputs.random_state(nx, ny, seed=seed, planes=3 if te else 6)
        live = [2, 3, 4] if te else list(range(6))
        with qla.Grid(nx, ny, 1.0, prec, te_only=te) as g:
            g.set_medium(np.ones((ny, nx)))
            g.set_state(q)
            e_ref = g.energy()
        dt = torch.float64 if prec == "fp64" else torch.float32
        planes = torch.tensor(q[live], dtype=dt, device="cuda").contiguous()
        out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        st = lib.qla_energy_noalloc(ctypes.c_void_p(planes.data_ptr()),
                                    qla.QLA_FP64 if prec == "fp64" else qla.QLA_FP32,
                                    len(live), nx, ny, nx, nx * ny,
                                    ctypes.c_void_p(stream.cuda_stream),
                                    ctypes.c_void_p(out.data_ptr()))
        assert st == 0
        torch.cuda.synchronize()
        e = out.item()
        assert abs(e / e_ref - 1) <= 1e-12, (prec, e, e_ref)
        # and against the oracle's energy (Eq. A13) of the same state, at the
        # precision the planes were stored in
        stored = planes.double().cpu().numpy()
        full = np.zeros((6, ny, nx))
        full[live] = stored
        assert abs(e / oracle.energy(full) - 1) <= 1e-12, (prec, e)
        results.append(e)
    assert results[0] != results[1]


def test_energy_noalloc_rejects_lattices_beyond_its_scratch():
    import torch
    lib = _lib()
    dummy = torch.zeros(1, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    nx, ny = 16384, 16385
    assert nx * ny > SITES_MAX
    st = lib.qla_energy_noalloc(ctypes.c_void_p(dummy.data_ptr()), qla.QLA_FP32, 1, nx, ny,
                                nx, nx * ny, None, ctypes.c_void_p(out.data_ptr()))
    assert st == 1  # QLA_EINVAL, nothing launched
