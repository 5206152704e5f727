"""DMI (Eq. 3) through the C ABI against the oracle: effective field,
energies and torque with per-cell Ms and vacuum (interfacial and bulk, both
precisions), 30 RK4 steps in float64 with DMI, the minimiser's converged
energy, and the adjoint's refusal of D != 0."""

import numpy as np
import pytest

import workloads as wl
from oracle import micromag

torch = pytest.importorskip("torch")
import paper_2606_01114_gb300 as mm  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {mm.MM_F64: 1e-12, mm.MM_F32: 1e-5}
KINDS = {"interfacial": mm.MM_DMI_INTERFACIAL, "bulk": mm.MM_DMI_BULK}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_01114_gb300 import build
    build.build()


def dev(a, prec):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64 if prec == mm.MM_F64 else torch.float32,
                        device="cuda")


def rel_l2(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def make(n, d, prec, kind, D, Ms=None, **mat):
    p = micromag.Problem(n, d, Ms_cell=Ms, D=D, dmi=kind, **mat)
    ctx = mm.mm_init_mesh(*n, *d, precision=prec)
    mm.mm_set_material(ctx, 8e5, mat.get("A", 1.3e-11), mat.get("alpha", 0.02), mat.get("Ku", 0.0),
                       mat.get("u", (0, 0, 1)))
    mm.mm_set_external_field(ctx, *mat.get("h_ext", (0, 0, 0)))
    if Ms is not None:
        mm.mm_set_material_fields(ctx, dev(Ms, prec))
    mm.mm_set_dmi(ctx, D, KINDS[kind])
    return p, ctx


@pytest.mark.parametrize("prec", [mm.MM_F64, mm.MM_F32], ids=["f64", "f32"])
@pytest.mark.parametrize("kind", ["interfacial", "bulk"])
def test_field_energy_torque(prec, kind):
    n, d = (16, 8, 4), (2e-9, 2.5e-9, 3e-9)
    Ms = wl.smooth_field(n, 4e5, 9e5, sigma_cells=2.0, seed=3)
    Ms[1, 2, 3] = 0.0
    Ms[3, 7, 15] = 0.0
    p, ctx = make(n, d, prec, kind, 3e-3, Ms, Ku=3e5, u=(0.3, -0.2, 0.9), h_ext=(1e4, -2e4, 3e4))
    m = wl.random_unit(n, seed=4)
    md = dev(m, prec)
    H = torch.empty_like(md)
    mm.mm_effective_field(ctx, md, H)
    assert rel_l2(H.double().cpu().numpy(), p.h_eff(m)) < TOL[prec]
    E, Eo = mm.mm_energy(ctx, md), p.energies(m)
    assert Eo[4] != 0.0
    assert np.max(np.abs(E - Eo)) / np.sum(np.abs(Eo)) < TOL[prec]
    assert mm.mm_max_torque(ctx, md) == pytest.approx(p.max_torque(m), rel=10 * TOL[prec], abs=0)
    mm.mm_destroy(ctx)


@pytest.mark.parametrize("kind", ["interfacial", "bulk"])
def test_rk4_steps_fp64(kind):
    n, d = (16, 16, 2), (2.5e-9, 2.5e-9, 2.5e-9)
    p, ctx = make(n, d, mm.MM_F64, kind, 4e-3, alpha=0.1)
    m = wl.random_unit(n, seed=6)
    md = dev(m, mm.MM_F64)
    dt = 5e-14
    for step in range(30):
        t, h = 0.0, dt
        mm.mm_llg_step(ctx, md, t, h, mm.MM_RK4)
        m = p.rk4_step(m, dt)
    assert rel_l2(md.cpu().numpy(), m) < 1e-11
    mm.mm_destroy(ctx)


def test_minimiser_with_dmi_fp64():
    n, d = (16, 16, 1), (3e-9, 3e-9, 3e-9)
    p, ctx = make(n, d, mm.MM_F64, "interfacial", 3e-3, Ku=5e5, u=(0, 0, 1), alpha=1.0)
    m0 = wl.smooth_unit(n, sigma_cells=3.0, seed=7)
    md = dev(m0, mm.MM_F64)
    k = mm.mm_minimize_bb(ctx, md, 1e-7, 20000)
    m_ref, k_ref = micromag.minimize_bb(p, m0, 1e-7, 20000)
    assert p.energies(md.cpu().numpy()).sum() == pytest.approx(p.energies(m_ref).sum(), rel=1e-9, abs=0)
    # BB is not monotone: rounding steers the path, so the step count is only bounded
    assert k <= 2 * k_ref + 20
    mm.mm_destroy(ctx)


def test_adjoint_rejects_dmi():
    n, d = (8, 8, 1), (3e-9, 3e-9, 3e-9)
    p, ctx = make(n, d, mm.MM_F64, "bulk", 1e-3)
    m = dev(wl.random_unit(n, seed=1), mm.MM_F64)
    lam = torch.zeros_like(m)
    gMs = torch.zeros(ctx.shape1, dtype=torch.float64, device="cuda")
    with pytest.raises(mm.MMError) as e:
        mm.mm_rk4_step_vjp(ctx, m, 1e-13, lam, gMs)
    assert e.value.code == mm.MM_ERR_INVALID_ARG
    with pytest.raises(mm.MMError):
        mm.mm_set_dmi(ctx, 1e-3, 7)
    mm.mm_destroy(ctx)
