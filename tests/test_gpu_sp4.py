"""Meshes whose sizes are not powers of two (direct-DFT and Bluestein passes) through the C
ABI against the oracle, and an SP4-shaped problem (the paper's validation
geometry): a 100 x 25 x 1 permalloy film of 5 x 5 x 3 nm cells, minimised
from m = (1, 0.25, 0.1) and then driven by the field
(-24.6, 4.3, 0) mT / mu0.  The published SP4 curves are not available, so
the run is checked against the oracle (minimum, then RK4 steps) and the
float32 path against the float64 one over 1 ns of RKF45."""

import numpy as np
import pytest

import workloads as wl
from oracle import micromag

torch = pytest.importorskip("torch")
import paper_2606_01114_gb300 as mm  # noqa: E402

pytestmark = pytest.mark.gpu
MU0 = 4e-7 * np.pi
TOL = {mm.MM_F64: 1e-12, mm.MM_F32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_01114_gb300 import build
    build.build()


def dev(a, prec):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64 if prec == mm.MM_F64 else torch.float32,
                        device="cuda")


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# padded lengths up to 64 take the direct DFT, longer ones the Bluestein passes
# (100 x 50: Px = 200, Py = 100; 350 x 70: Px = 700 with M = 2048; 36 x 200:
# Py = 400)
MESHES = [((100, 25, 1), (5e-9, 5e-9, 3e-9)), ((12, 10, 2), (2e-9, 3e-9, 2.5e-9)), ((7, 5, 4), (3e-9, 2e-9, 2e-9)),
          ((33, 1, 1), (2e-9, 2e-9, 2e-9)), ((1, 18, 2), (2e-9, 2e-9, 2e-9)), ((100, 50, 2), (5e-9, 5e-9, 3e-9)),
          ((350, 70, 1), (2e-9, 2e-9, 2e-9)), ((36, 200, 4), (3e-9, 2e-9, 2e-9))]


@pytest.mark.parametrize("prec", [mm.MM_F64, mm.MM_F32], ids=["f64", "f32"])
@pytest.mark.parametrize("n,d", MESHES, ids=[f"{m[0][0]}x{m[0][1]}x{m[0][2]}" for m in MESHES])
def test_fields_on_meshes_of_any_size(n, d, prec):
    Ms = wl.smooth_field(n, 4e5, 9e5, sigma_cells=2.0, seed=2)
    p = micromag.Problem(n, d, Ms_cell=Ms, Ku=1e5, u=(0, 1, 0), h_ext=(1e4, 0, -5e3))
    ctx = mm.mm_init_mesh(*n, *d, precision=prec)
    mm.mm_set_material(ctx, 8e5, 1.3e-11, 0.02, 1e5, (0, 1, 0))
    mm.mm_set_external_field(ctx, 1e4, 0, -5e3)
    mm.mm_set_material_fields(ctx, dev(Ms, prec))
    m = wl.random_unit(n, seed=3)
    md = dev(m, prec)
    H = torch.empty_like(md)
    mm.mm_demag_field(ctx, md, H)
    assert rel(H.double().cpu().numpy(), p.demag_fft(m)) < TOL[prec]
    mm.mm_effective_field(ctx, md, H)
    assert rel(H.double().cpu().numpy(), p.h_eff(m)) < TOL[prec]
    mm.mm_destroy(ctx)


SP4 = dict(n=(100, 25, 1), d=(5e-9, 5e-9, 3e-9), Ms=8e5, A=1.3e-11, alpha=0.02,
           field1=(-24.6e-3 / MU0, 4.3e-3 / MU0, 0.0))


def sp4_ctx(prec, h=(0, 0, 0)):
    ctx = mm.mm_init_mesh(*SP4["n"], *SP4["d"], precision=prec)
    mm.mm_set_material(ctx, SP4["Ms"], SP4["A"], SP4["alpha"], 0.0, (0, 0, 1))
    mm.mm_set_external_field(ctx, *h)
    return ctx


def sp4_start():
    return wl.uniform(SP4["n"], (1.0, 0.25, 0.1))


def test_sp4_minimum_then_rk4_match_oracle_fp64():
    p = micromag.Problem(SP4["n"], SP4["d"], Ms=SP4["Ms"], A=SP4["A"], alpha=SP4["alpha"])
    ctx = sp4_ctx(mm.MM_F64)
    md = dev(sp4_start(), mm.MM_F64)
    mm.mm_minimize_bb(ctx, md, 1e-6, 20000)
    m_ref, _ = micromag.minimize_bb(p, sp4_start(), 1e-6, 20000)
    m_gpu = md.cpu().numpy()
    assert p.energies(m_gpu).sum() == pytest.approx(p.energies(m_ref).sum(), rel=1e-8, abs=0)
    assert np.mean(m_gpu[0]) == pytest.approx(np.mean(m_ref[0]), abs=1e-4)   # the S-state
    # switching field 1, 200 RK4 steps of 0.1 ps from the GPU's minimum on both sides
    p1 = micromag.Problem(SP4["n"], SP4["d"], Ms=SP4["Ms"], A=SP4["A"], alpha=SP4["alpha"], h_ext=SP4["field1"])
    mm.mm_set_external_field(ctx, *SP4["field1"])
    m = m_gpu.copy()
    for _ in range(200):
        mm.mm_llg_step(ctx, md, 0.0, 1e-13, mm.MM_RK4)
        m = p1.rk4_step(m, 1e-13)
    assert rel(md.cpu().numpy(), m) < 1e-10
    mm.mm_destroy(ctx)


def test_sp4_field1_one_ns_fp32_tracks_fp64():
    traces = {}
    for prec in (mm.MM_F64, mm.MM_F32):
        ctx = sp4_ctx(prec)
        md = dev(sp4_start(), prec)
        mm.mm_minimize_bb(ctx, md, 1e-4 if prec == mm.MM_F32 else 1e-6, 20000)
        mm.mm_set_external_field(ctx, *SP4["field1"])
        t, dt, out = 0.0, 1e-14, []
        for target in np.arange(1, 101) * 1e-11:       # <m> every 10 ps up to 1 ns
            while t < target * (1 - 1e-12):
                t, dt, _ = mm.mm_llg_step(ctx, md, t, min(dt, target - t), mm.MM_RKF45, 1e-6)
            out.append(md.double().mean(dim=(1, 2, 3)).cpu().numpy())
        traces[prec] = np.array(out)
        mm.mm_destroy(ctx)
    d = np.abs(traces[mm.MM_F32] - traces[mm.MM_F64]).max()
    print("SP4 field 1: <m> at 1 ns", traces[mm.MM_F64][-1], "max |<m>_f32 - <m>_f64|", d)
    assert traces[mm.MM_F64][-1][0] < 0          # the film has switched: <m_x> < 0 at 1 ns
    assert d < 2e-2


def test_bluestein_pass_time_on_a_350_cell_film():
    """The Bluestein passes on a 350 x 350 x 4 film (Px = Py = 700, M =
    2048): demag against the oracle at the FP32 tolerance, and the time per
    evaluation (printed)."""
    n, d = (350, 350, 4), (2e-9, 2e-9, 2e-9)
    p = micromag.Problem(n, d)
    m = wl.random_unit(n, seed=21)
    ctx = mm.mm_init_mesh(*n, *d, precision=mm.MM_F32)
    mm.mm_set_material(ctx, 8e5, 1.3e-11, 0.02, 0.0)
    md = dev(m, mm.MM_F32)
    H = torch.empty_like(md)
    mm.mm_demag_field(ctx, md, H)
    assert rel(H.double().cpu().numpy(), p.demag_fft(m)) < 1e-5
    for _ in range(3):
        mm.mm_demag_field(ctx, md, H)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(20):
        mm.mm_demag_field(ctx, md, H)
    b.record()
    torch.cuda.synchronize()
    print(f"350 x 350 x 4 FP32 demag: {a.elapsed_time(b) / 20:.3f} ms per evaluation")
    mm.mm_destroy(ctx)
