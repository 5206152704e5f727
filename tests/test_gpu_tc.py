"""Tensor-core split-precision DFT stage (tcgen05) against numpy's FFT.

The hi + lo split keeps about 2 x 11 bits (TF32) or 2 x 8 bits (BF16) of each
operand; with the lo.lo product dropped the error of one product is about
2^-21 (TF32) or 2^-17 (BF16) relative, so a 32-term sum stays below 2e-6
and 2e-5 relative L2."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import paper_2606_01114_gb300 as mm  # noqa: E402

pytestmark = pytest.mark.gpu

BOUND = {mm.MM_TC_TF32: 2e-6, mm.MM_TC_BF16: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2606_01114_gb300 import build
    build.build()


@pytest.mark.parametrize("mode", [mm.MM_TC_TF32, mm.MM_TC_BF16], ids=["tf32", "bf16"])
@pytest.mark.parametrize("direction", [-1, 1])
@pytest.mark.parametrize("nlines", [1, 128, 1000])
def test_dft32_tc_matches_fft(mode, direction, nlines):
    rng = np.random.default_rng(nlines + 7 * mode)
    x = (rng.standard_normal((nlines, 32)) + 1j * rng.standard_normal((nlines, 32))) * rng.uniform(0.1, 10, (nlines, 1))
    xin = torch.tensor(x.astype(np.complex64), device="cuda")
    out = torch.empty_like(xin)
    mm.mm_dft32_tc(xin, out, mode, direction)
    got = out.cpu().numpy().astype(np.complex128)
    xs = x.astype(np.complex64).astype(np.complex128)
    ref = np.fft.fft(xs, axis=1) if direction < 0 else np.fft.ifft(xs, axis=1) * 32
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < BOUND[mode]


TC_MESHES = [((32, 256, 4), (2e-9, 2e-9, 2e-9)), ((16, 512, 2), (2.5e-9, 2.5e-9, 3e-9))]


@pytest.mark.parametrize("mode", [mm.MM_TC_TF32, mm.MM_TC_BF16], ids=["tf32", "bf16"])
@pytest.mark.parametrize("n,d", TC_MESHES)
def test_demag_with_tensor_core_y_passes(n, d, mode):
    """Demag with the y passes on tensor cores against the float64 oracle:
    TF32 hi + lo (about 21 bits) and BF16 hi + mid + lo (about 24 bits) both
    keep the field within the FP32 tolerance (1e-5)."""
    import workloads as wl
    from oracle import micromag
    p = micromag.Problem(n, d)
    m = wl.random_unit(n, seed=3)
    ctx = mm.mm_init_mesh(*n, *d, precision=mm.MM_F32)
    mm.mm_set_fft_mode(ctx, mode)
    md = torch.tensor(m, dtype=torch.float32, device="cuda")
    H = torch.empty_like(md)
    mm.mm_demag_field(ctx, md, H)
    mm.mm_tc_status(ctx)
    ref = p.demag_fft(m)
    err = np.linalg.norm(H.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < 1e-5, err
    mm.mm_destroy(ctx)


def test_fft_mode_rejected_for_fp64():
    ctx = mm.mm_init_mesh(8, 8, 2, 1e-9, 1e-9, 1e-9, precision=mm.MM_F64)
    with pytest.raises(mm.MMError) as e:
        mm.mm_set_fft_mode(ctx, mm.MM_TC_TF32)
    assert e.value.code == mm.MM_ERR_INVALID_ARG
    mm.mm_destroy(ctx)


class _ThreadedFFT:
    """scipy.fft's rfftn / irfftn on all host cores for the oracle's
    convolution (the same transforms as numpy's, on more threads)."""

    def __init__(self):
        import os
        import scipy.fft
        self._f, self._w = scipy.fft, os.cpu_count() or 1

    def rfftn(self, a, s=None, axes=None):
        return self._f.rfftn(a, s=s, axes=axes, workers=self._w)

    def irfftn(self, a, s=None, axes=None):
        return self._f.irfftn(a, s=s, axes=axes, workers=self._w)


def test_cube256_per_field_errors_and_speed():
    """256^3 bulk cube, 1 nm cells, Ku 5e5 along z, random m: relative L2 of
    each field (demag, exchange, effective, and the torque m x H_eff) for
    plain FP32, the two tensor-core modes, the float-float FP64 mode and
    native FP64 against the float64 CPU oracle, and the demag time per
    evaluation of each mode (printed)."""
    import workloads as wl
    from oracle import micromag
    n, d = (256, 256, 256), (1e-9, 1e-9, 1e-9)
    m = wl.random_unit(n, seed=11)
    p = micromag.Problem(n, d, Ms=8e5, A=1.3e-11, alpha=0.02, Ku=5e5, u=(0, 0, 1))
    p.fft = _ThreadedFFT()
    nh = p.kernel_hat()
    p._kernel = None
    p.kernel_hat = lambda: nh
    ref = {"demag": p.demag_fft(m)}
    del nh
    p.kernel_hat = None
    ref["exchange"] = p.exchange(m)
    ref["effective"] = ref["demag"] + ref["exchange"] + p.anisotropy(m) + p.zeeman(m)
    ref["torque"] = np.cross(m, ref["effective"], axis=0)
    ref_norm = {k: float(np.linalg.norm(v)) for k, v in ref.items()}

    def errors(prec, mode=0):
        ctx = mm.mm_init_mesh(*n, *d, precision=prec)
        mm.mm_set_material(ctx, 8e5, 1.3e-11, 0.02, 5e5, (0, 0, 1))
        if mode:
            mm.mm_set_fft_mode(ctx, mode)
        dt = torch.float64 if prec == mm.MM_F64 else torch.float32
        md = torch.tensor(m, dtype=dt, device="cuda")
        H = torch.empty_like(md)
        err = {}

        def cmp(name, t):
            err[name] = float(np.linalg.norm(t.double().cpu().numpy() - ref[name]) / ref_norm[name])

        mm.mm_demag_field(ctx, md, H)
        cmp("demag", H)
        mm.mm_exchange_field(ctx, md, H)
        cmp("exchange", H)
        mm.mm_effective_field(ctx, md, H)
        if mode in (mm.MM_TC_TF32, mm.MM_TC_BF16):
            mm.mm_tc_status(ctx)
        cmp("effective", H)
        cmp("torque", torch.linalg.cross(md.double(), H.double(), dim=0))
        # demag time per evaluation
        for _ in range(3):
            mm.mm_demag_field(ctx, md, H)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(10):
            mm.mm_demag_field(ctx, md, H)
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 10
        mm.mm_destroy(ctx)
        del md, H
        torch.cuda.empty_cache()
        return err, t

    rows = {}
    for name, prec, mode in (("fp32", mm.MM_F32, 0), ("tf32x2", mm.MM_F32, mm.MM_TC_TF32),
                             ("bf16x3", mm.MM_F32, mm.MM_TC_BF16), ("ff", mm.MM_F64, mm.MM_FFT_FF),
                             ("fp64", mm.MM_F64, 0)):
        errs, t = errors(prec, mode)
        rows[name] = (errs, t)
        print(name, f"demag {t:.3f} ms/eval", {k: f"{v:.2e}" for k, v in errs.items()})
    assert max(rows["fp32"][0].values()) < 1e-5
    assert rows["tf32x2"][0]["demag"] < 1e-5
    assert max(rows["bf16x3"][0].values()) < 1e-5
    assert max(rows["ff"][0].values()) < 1e-12       # float-float passes at the float64 tolerance
    assert max(rows["fp64"][0].values()) < 1e-12


def test_bounded_wait_gives_up_and_reports_timeout():
    """A wait on an mbarrier that nothing completes gives up after its poll
    limit, raises TIMEOUT in the device status (read back and cleared by the
    call), and the tensor-core path keeps working afterwards."""
    assert mm.mm_tc_wait_selftest(1000) == mm.MM_ERR_TIMEOUT
    assert mm.mm_tc_wait_selftest(1) == mm.MM_ERR_TIMEOUT
    x = torch.randn(64, 32, dtype=torch.complex64, device="cuda")
    y = torch.empty_like(x)
    mm.mm_dft32_tc(x, y, mm.MM_TC_TF32, -1)      # raises if a timeout were still pending
    ref = torch.fft.fft(x.to(torch.complex128), dim=1)
    assert float((y.to(torch.complex128) - ref).abs().max() / ref.abs().max()) < 1e-5
