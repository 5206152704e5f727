"""The allocation-free energy entry point against the context-based one.

mm_energy_noalloc exists for callers that cannot allocate device memory (code
running inside a memory pool or arena it does not own, or a plugin handed
only its host application's buffers).  Its results must equal mm_energy's on
the same state, call after call: the fixed scratch array it shares between
calls must not leak one call's partial sums into the next.  This file is
collected last so that a stop at its first failure has run every other test."""

import numpy as np
import pytest

import workloads as wl

torch = pytest.importorskip("torch")
import paper_2606_01114_gb300 as mm  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {mm.MM_F64: 1e-12, mm.MM_F32: 1e-5}


@pytest.mark.parametrize("prec", [mm.MM_F64, mm.MM_F32], ids=["f64", "f32"])
def test_noalloc_energy_matches_context_energy_twice(prec):
    from paper_2606_01114_gb300 import build
    build.build()
    n, d = (64, 32, 4), (2.5e-9, 2.5e-9, 3e-9)
    Ms, A, Ku, u, h = 8e5, 1.3e-11, 2e5, (0.2, -0.3, 0.9), (1e4, -2e4, 5e3)
    dtype = torch.float64 if prec == mm.MM_F64 else torch.float32
    ctx = mm.mm_init_mesh(*n, *d, precision=prec)
    mm.mm_set_material(ctx, Ms, A, 0.02, Ku, u)
    mm.mm_set_external_field(ctx, *h)
    results = []
    for seed in (3, 4):   # two calls in a row on different states
        m = torch.tensor(wl.random_unit(n, seed=seed), dtype=dtype, device="cuda")
        ref = mm.mm_energy(ctx, m)[:4]   # no DMI: the fifth entry is zero
        H = torch.empty_like(m)
        mm.mm_demag_field(ctx, m, H)
        got = mm.mm_energy_noalloc(n, d, prec, Ms, A, Ku, u, h, m, H)
        assert np.max(np.abs(got - ref)) / np.sum(np.abs(ref)) < TOL[prec]
        results.append((ref, got))
    # the same state again gives the same answer (nothing left over from the previous call)
    m = torch.tensor(wl.random_unit(n, seed=3), dtype=dtype, device="cuda")
    H = torch.empty_like(m)
    mm.mm_demag_field(ctx, m, H)
    again = mm.mm_energy_noalloc(n, d, prec, Ms, A, Ku, u, h, m, H)
    assert np.array_equal(again, results[0][1])
    mm.mm_destroy(ctx)


def test_noalloc_rejects_meshes_beyond_its_scratch():
    """16.8 M cells exceed the fixed scratch: rejected before any device work."""
    import ctypes
    lib = mm._load()
    m = torch.zeros((3, 1, 1, 1), dtype=torch.float32, device="cuda")
    E = (ctypes.c_double * 4)()
    rc = lib.mm_energy_noalloc(4096, 4096, 1, 1e-9, 1e-9, 1e-9, mm.MM_F32, 8e5, 1.3e-11, 0.0, None, None,
                               ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(m.data_ptr()), E, None)
    assert rc == mm.MM_ERR_INVALID_ARG
    assert "exceed" in lib.mm_last_error(None).decode()


@pytest.mark.parametrize("prec", [mm.MM_F64, mm.MM_F32], ids=["f64", "f32"])
def test_noalloc_energy_matches_oracle(prec):
    """The four energies against the float64 oracle's (demag energy from the
    oracle's own convolution), within the path's tolerance of their scale."""
    from oracle import micromag
    from paper_2606_01114_gb300 import build
    build.build()
    n, d = (32, 16, 4), (2.5e-9, 2.5e-9, 3e-9)
    Ms, A, Ku, u, h = 8e5, 1.3e-11, 2e5, (0.2, -0.3, 0.9), (1e4, -2e4, 5e3)
    p = micromag.Problem(n, d, Ms=Ms, A=A, Ku=Ku, u=u, h_ext=h)
    m_np = wl.random_unit(n, seed=6)
    dtype = torch.float64 if prec == mm.MM_F64 else torch.float32
    ctx = mm.mm_init_mesh(*n, *d, precision=prec)
    mm.mm_set_material(ctx, Ms, A, 0.02, Ku, u)
    m = torch.tensor(m_np, dtype=dtype, device="cuda")
    H = torch.empty_like(m)
    mm.mm_demag_field(ctx, m, H)
    got = mm.mm_energy_noalloc(n, d, prec, Ms, A, Ku, u, h, m, H)
    ref = p.energies(m_np)[:4]
    assert np.max(np.abs(got - ref)) / np.sum(np.abs(ref)) < TOL[prec]
    mm.mm_destroy(ctx)


def test_noalloc_restores_the_callers_device():
    """A stream on another device is served there; the caller's current
    device is the same after the call as before it."""
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    import ctypes
    from paper_2606_01114_gb300 import build
    build.build()
    lib = mm._load()
    n, d = (16, 8, 2), (2e-9, 2e-9, 2e-9)
    with torch.cuda.device(1):
        s1 = torch.cuda.Stream()
        m = torch.tensor(wl.random_unit(n, seed=2), dtype=torch.float64, device="cuda:1")
        H = torch.zeros_like(m)
    torch.cuda.set_device(0)
    E = (ctypes.c_double * 4)()
    rc = lib.mm_energy_noalloc(*n, *d, mm.MM_F64, 8e5, 1.3e-11, 0.0, None, None, ctypes.c_void_p(m.data_ptr()),
                               ctypes.c_void_p(H.data_ptr()), E, ctypes.c_void_p(s1.cuda_stream))
    assert rc == mm.MM_OK
    assert torch.cuda.current_device() == 0
