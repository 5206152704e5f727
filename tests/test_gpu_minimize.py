"""The Barzilai-Borwein minimiser through the C ABI against the oracle's:
the first 25 iterates in float64 (per-cell Ms, anisotropy, Zeeman), the
converged energy and step count, float32 against float64, vacuum cells, and
the NOT_CONVERGED report at max_iter."""

import numpy as np
import pytest

import workloads as wl
from oracle import micromag

torch = pytest.importorskip("torch")
import paper_2606_01114_gb300 as mm  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_01114_gb300 import build
    build.build()


N, D = (16, 8, 2), (3e-9, 3e-9, 3e-9)
MAT = dict(Ms=8e5, A=1.3e-11, alpha=1.0, Ku=2e5, u=(1.0, 0.0, 0.0), h_ext=(0.0, 2e4, 0.0))


def setup(prec, Ms_cell=None):
    ctx = mm.mm_init_mesh(*N, *D, precision=prec)
    mm.mm_set_material(ctx, MAT["Ms"], MAT["A"], MAT["alpha"], MAT["Ku"], MAT["u"])
    mm.mm_set_external_field(ctx, *MAT["h_ext"])
    dt = torch.float64 if prec == mm.MM_F64 else torch.float32
    if Ms_cell is not None:
        mm.mm_set_material_fields(ctx, torch.tensor(Ms_cell, dtype=dt, device="cuda"))
    p = micromag.Problem(N, D, Ms_cell=Ms_cell, **{k: v for k, v in MAT.items() if not (k == "Ms" and Ms_cell is not None)})
    return ctx, p, dt


def run_gpu(ctx, m0, dt, tol, max_iter):
    m = torch.tensor(m0, dtype=dt, device="cuda")
    try:
        k = mm.mm_minimize_bb(ctx, m, tol, max_iter)
        ok = True
    except mm.MMError as e:
        assert e.code == mm.MM_ERR_NOT_CONVERGED
        k, ok = max_iter, False
    return m.double().cpu().numpy(), k, ok


def test_first_iterates_match_oracle_fp64():
    Ms = wl.smooth_field(N, 4e5, 9e5, sigma_cells=2.0, seed=1)
    ctx, p, dt = setup(mm.MM_F64, Ms)
    m0 = wl.smooth_unit(N, sigma_cells=3.0, seed=4)
    for iters in (1, 2, 25):
        m_gpu, k, ok = run_gpu(ctx, m0, dt, 0.0, iters)
        assert not ok and k == iters
        m_ref, k_ref = micromag.minimize_bb(p, m0, 0.0, iters)
        assert k_ref == iters
        err = np.linalg.norm(m_gpu - m_ref) / np.linalg.norm(m_ref)
        assert err < 1e-11, (iters, err)
    mm.mm_destroy(ctx)


def test_converged_energy_and_steps_match_oracle_fp64():
    ctx, p, dt = setup(mm.MM_F64)
    m0 = wl.random_unit(N, seed=5)
    m_gpu, k, ok = run_gpu(ctx, m0, dt, 1e-7, 20000)
    assert ok
    m_ref, k_ref = micromag.minimize_bb(p, m0, 1e-7, 20000)
    assert p.max_torque(m_gpu) <= 1e-7 * (1 + 1e-9)
    assert p.energies(m_gpu).sum() == pytest.approx(p.energies(m_ref).sum(), rel=1e-9, abs=0)
    # BB is not monotone: rounding steers the path, so the step count is only bounded
    assert k <= 2 * k_ref + 20
    assert k < 2000
    mm.mm_destroy(ctx)


def test_fp32_reaches_fp64_minimum():
    m0 = wl.smooth_unit(N, sigma_cells=3.0, seed=6)
    E = {}
    for prec in (mm.MM_F64, mm.MM_F32):
        ctx, p, dt = setup(prec)
        m_gpu, k, ok = run_gpu(ctx, m0, dt, 1e-3 if prec == mm.MM_F32 else 1e-7, 20000)
        assert ok
        E[prec] = p.energies(m_gpu).sum()
        mm.mm_destroy(ctx)
    assert E[mm.MM_F32] == pytest.approx(E[mm.MM_F64], rel=1e-5, abs=0)


def test_vacuum_cells_stay_and_max_iter_reports():
    Ms = wl.smooth_field(N, 4e5, 9e5, sigma_cells=2.0, seed=7)
    Ms[:, :, :3] = 0.0                        # vacuum strip
    ctx, p, dt = setup(mm.MM_F64, Ms)
    m0 = wl.random_unit(N, seed=8)
    m0[:, Ms == 0] = 0.0
    m_gpu, k, ok = run_gpu(ctx, m0, dt, 1e-7, 20000)
    assert ok
    assert np.all(m_gpu[:, Ms == 0] == 0.0)
    m_ref, _ = micromag.minimize_bb(p, m0, 1e-7, 20000)
    assert p.energies(m_gpu).sum() == pytest.approx(p.energies(m_ref).sum(), rel=1e-9, abs=0)
    m_short, k, ok = run_gpu(ctx, m0, dt, 1e-7, 7)
    assert not ok and k == 7
    mm.mm_destroy(ctx)
