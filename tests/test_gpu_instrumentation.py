"""Entry points that serve measurement rather than the method itself:

* mm_kspace_product, the tensor product on an unpruned R2C spectrum, so a
  library FFT (cuFFT through torch.fft) can be timed on the same Newell
  kernel: the cuFFT-based field it gives equals mm_demag_field and the
  oracle's float64 convolution;
* mm_llg_step_host, one step with the state in host memory (the end-to-end
  path the bench times): bit-identical to mm_llg_step on a device copy;
* mm_alu_peak, the measured FMA roofs: positive, ordered as GB300's pipes
  are (FP32 above FP64), and repeatable;
* mm_enable_kernel_timing_mask: only the masked classes carry device time,
  every class's launches are still counted, and a bit above the classes is
  rejected."""

import numpy as np
import pytest

import workloads as wl
from oracle import micromag

torch = pytest.importorskip("torch")
import paper_2606_01114_gb300 as mm  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {mm.MM_F64: 1e-12, mm.MM_F32: 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_01114_gb300 import build
    build.build()


def cufft_demag(ctx, m, Ms):
    """H = -N * (Ms m) with torch.fft (cuFFT) on the padded grid and the
    library's k-space product in between."""
    nx, ny, nz = ctx.n
    P = (2 * nz if nz > 1 else 1, 2 * ny if ny > 1 else 1, 2 * nx if nx > 1 else 1)
    Mp = torch.zeros((3,) + P, dtype=m.dtype, device=m.device)
    Mp[:, :nz, :ny, :nx] = m * Ms
    spec = torch.fft.rfftn(Mp, dim=(1, 2, 3)).contiguous()
    mm.mm_kspace_product(ctx, spec)
    return torch.fft.irfftn(spec, s=P, dim=(1, 2, 3))[:, :nz, :ny, :nx]


@pytest.mark.parametrize("prec", [mm.MM_F64, mm.MM_F32], ids=["f64", "f32"])
@pytest.mark.parametrize("n,d", [((16, 8, 4), (2e-9, 2.5e-9, 3e-9)), ((64, 32, 1), (2e-9, 2e-9, 1e-9)),
                                 ((1, 8, 8), (1e-9, 2e-9, 2e-9)), ((20, 12, 2), (2e-9, 2e-9, 2e-9))])
def test_cufft_path_with_kspace_product_matches_demag(n, d, prec):
    p = micromag.Problem(n, d)
    m = wl.random_unit(n, seed=5)
    dtype = torch.float64 if prec == mm.MM_F64 else torch.float32
    ctx = mm.mm_init_mesh(*n, *d, precision=prec)
    mm.mm_set_material(ctx, 8e5, 1.3e-11, 0.02, 0.0)
    md = torch.tensor(m, dtype=dtype, device="cuda")
    H = torch.empty_like(md)
    mm.mm_demag_field(ctx, md, H)
    Hc = cufft_demag(ctx, md, 8e5)
    ref = p.demag_fft(m)
    got_c = Hc.double().cpu().numpy()
    assert np.linalg.norm(got_c - ref) / np.linalg.norm(ref) < TOL[prec]
    assert float(torch.linalg.vector_norm(Hc.double() - H.double()) / torch.linalg.vector_norm(H.double())) < TOL[prec]
    mm.mm_destroy(ctx)


def test_kspace_product_rejects_a_wrong_layout():
    ctx = mm.mm_init_mesh(8, 8, 2, 1e-9, 1e-9, 1e-9, precision=mm.MM_F32)
    for shape in ((3, 4, 16, 8), (3, 2, 16, 9), (2, 4, 16, 9)):     # the right one is (3, 4, 16, 9)
        bad = torch.zeros(shape, dtype=torch.complex64, device="cuda")
        with pytest.raises(ValueError):
            mm.mm_kspace_product(ctx, bad)
    with pytest.raises(ValueError):
        mm.mm_kspace_product(ctx, torch.zeros((3, 4, 16, 9), dtype=torch.complex128, device="cuda"))
    mm.mm_destroy(ctx)


@pytest.mark.parametrize("prec", [mm.MM_F64, mm.MM_F32], ids=["f64", "f32"])
def test_llg_step_host_equals_device_step(prec):
    n, d = (32, 16, 4), (2.5e-9, 2.5e-9, 3e-9)
    m = wl.random_unit(n, seed=8)
    np_dtype = np.float64 if prec == mm.MM_F64 else np.float32
    ctx = mm.mm_init_mesh(*n, *d, precision=prec)
    mm.mm_set_material(ctx, 8e5, 1.3e-11, 0.1, 1e5)
    md = torch.tensor(m.astype(np_dtype), device="cuda")
    mh = torch.from_numpy(m.astype(np_dtype).copy()).pin_memory()
    t_d, dt_d = 0.0, 1e-14
    t_h, dt_h = 0.0, 1e-14
    for _ in range(3):
        t_d, dt_d, e_d = mm.mm_llg_step(ctx, md, t_d, dt_d, mm.MM_RKF45, 1e-5)
        t_h, dt_h, e_h = mm.mm_llg_step_host(ctx, mh, t_h, dt_h, mm.MM_RKF45, 1e-5)
        assert (t_h, dt_h, e_h) == (t_d, dt_d, e_d)
        assert torch.equal(md.cpu(), mh)
    plain = np.ascontiguousarray(m.astype(np_dtype))        # pageable numpy memory works as well
    mm.mm_llg_step_host(ctx, plain, 0.0, 1e-13, mm.MM_RK4)
    md = torch.tensor(m.astype(np_dtype), device="cuda")
    mm.mm_llg_step(ctx, md, 0.0, 1e-13, mm.MM_RK4)
    assert np.array_equal(plain, md.cpu().numpy())
    mm.mm_destroy(ctx)


def test_alu_peaks_are_measured():
    f64 = mm.mm_alu_peak(mm.MM_ROOF_FP64)
    f32 = mm.mm_alu_peak(mm.MM_ROOF_FP32)
    f32x2 = mm.mm_alu_peak(mm.MM_ROOF_FP32X2)
    print(f"FMA roofs: FP64 {f64 / 1e12:.2f}, FP32 {f32 / 1e12:.1f}, FP32x2 {f32x2 / 1e12:.1f} TFLOP/s")
    assert 0.1e12 < f64 < 10e12
    assert f32 > 5 * f64
    assert f32x2 > 0.5 * f32
    again = mm.mm_alu_peak(mm.MM_ROOF_FP64)
    assert abs(again - f64) < 0.2 * f64
    with pytest.raises(mm.MMError):
        mm.mm_alu_peak(7)


def test_kernel_timing_mask_times_only_the_masked_class():
    n, d = (64, 32, 4), (2e-9, 2e-9, 2e-9)
    ctx = mm.mm_init_mesh(*n, *d, precision=mm.MM_F32)
    mm.mm_set_material(ctx, 8e5, 1.3e-11, 0.5, 0.0)
    m = torch.tensor(wl.random_unit(n, seed=3), dtype=torch.float32, device="cuda")
    zc, st = mm.KERNEL_NAMES.index("zconv"), mm.KERNEL_NAMES.index("stage")
    mm.mm_enable_kernel_timing_mask(ctx, 1 << zc)
    t, dt, _ = mm.mm_llg_step(ctx, m, 0.0, 1e-14, mm.MM_RKF45, 1e-5)
    z_ms, z_n = mm.mm_kernel_time(ctx, zc)
    s_ms, s_n = mm.mm_kernel_time(ctx, st)
    assert z_n >= 6 and z_ms > 0.0
    assert s_n == z_n and s_ms == 0.0
    # all classes: the stage now carries device time too
    mm.mm_enable_kernel_timing(ctx, True)
    mm.mm_llg_step(ctx, m, t, dt, mm.MM_RKF45, 1e-5)
    assert mm.mm_kernel_time(ctx, st)[0] > 0.0
    # off: nothing counted
    mm.mm_enable_kernel_timing_mask(ctx, 0)
    mm.mm_llg_step(ctx, m, t, dt, mm.MM_RKF45, 1e-5)
    assert mm.mm_kernel_time(ctx, zc) == (0.0, 0)
    with pytest.raises(mm.MMError) as e:
        mm.mm_enable_kernel_timing_mask(ctx, 1 << mm.MM_K_COUNT)
    assert e.value.code == mm.MM_ERR_INVALID_ARG
    mm.mm_destroy(ctx)
