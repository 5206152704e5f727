"""Host logic of bench.py that the roofline line depends on (CPU only):
reading an ncu raw-page CSV into profiles/traffic.json (units, the y pass
direction, the first launch of each pass, the average over the RKF45 stage
launches, the source-hash stamp), invalidating stored traffic when a kernel
family's sources change, and the algorithmic byte model."""

import csv
import json
import os
import shutil

import pytest

import bench

CSRC = os.path.join(bench.ROOT, "paper_2606_01114_gb300", "csrc")


@pytest.fixture
def tree(tmp_path, monkeypatch):
    """A copy of the hashed sources under a temporary root, with an empty
    profiles/ folder; bench.ROOT points there for the test."""
    dst = tmp_path / "paper_2606_01114_gb300" / "csrc"
    dst.mkdir(parents=True)
    for files in bench.KERNEL_SOURCES.values():
        for fn in files:
            shutil.copy(os.path.join(CSRC, fn), dst / fn)
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    return tmp_path


def write_csv(path, rows):
    head = ["ID", "Kernel Name", "dram__bytes_read.sum", "dram__bytes_write.sum"]
    units = ["", "", "Mbyte", "Kbyte"]
    with open(path, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(head)
        w.writerow(units)
        for i, (name, rd, wr) in enumerate(rows):
            w.writerow([str(i), name, f"{rd:,.3f}", f"{wr:,.3f}"])


ROWS = [
    ("void k_xfwd_reg<32, 16>(const float *)", 50.0, 40000.0),
    ("void k_cols_reg<32, 32, (int)-1, 1, 0>(const float2 *)", 100.0, 150000.0),
    ("void k_zconv_reg<32>(float2 *)", 300.0, 150000.0),
    ("void k_cols_reg<32, 32, 1, 0, 1>(const float2 *)", 200.0, 70000.0),
    ("void unnamed>::k_xinv_tma(const float2 *, float *)", 100.0, 20000.0),   # no template arguments
    ("void k_cols_reg<32, 32, (int)-1, 1, 0>(const float2 *)", 999.0, 999.0),   # later launch: ignored
] + [(f"void k_stage4<1, {s}>(Params<float>)", 200.0 + 10.0 * s, 60000.0) for s in range(6)]


def test_ingest_reads_units_direction_first_launch_and_stage_average(tree):
    p = tree / "raw.csv"
    write_csv(p, ROWS)
    assert bench.ingest_ncu(str(p), "f32", "film512 test") == 0
    t = json.load(open(tree / "profiles" / "traffic.json"))
    mb, kb = 1e6, 1e3
    assert t["xfwd/f32"]["bytes_per_launch"] == int(50 * mb + 40000 * kb)
    # y forward is the DIR = -1 instance, its first launch; y inverse the DIR = +1 one
    assert t["yfwd/f32"]["read"] == int(100 * mb) and t["yfwd/f32"]["write"] == int(150000 * kb)
    assert t["yinv/f32"]["read"] == int(200 * mb) and t["yinv/f32"]["write"] == int(70000 * kb)
    assert t["zconv/f32"]["bytes_per_launch"] == int(300 * mb + 150000 * kb)
    assert t["xinv/f32"]["read"] == int(100 * mb)
    # the stage entry averages the six captured stage launches: reads 200 + 10 s, s = 0..5
    assert t["stage/f32"]["read"] == int(225 * mb)
    assert t["stage/f32"]["write"] == int(60000 * kb)
    assert "average of 6" in t["stage/f32"]["kernel"]
    for k in ("xfwd", "yfwd", "zconv", "yinv", "xinv", "stage"):
        assert t[f"{k}/f32"]["source_sha"] == bench.source_hash(k)
        assert bench.ncu_traffic(k, "f32") == t[f"{k}/f32"]["bytes_per_launch"]


def test_stored_traffic_goes_stale_when_a_family_source_changes(tree):
    p = tree / "raw.csv"
    write_csv(p, ROWS)
    bench.ingest_ncu(str(p), "f32", "film512 test")
    assert bench.ncu_traffic("zconv", "f32") is not None
    assert bench.ncu_traffic("stage", "f32") is not None
    with open(tree / "paper_2606_01114_gb300" / "csrc" / "mm_demag.cu", "a") as f:
        f.write("\n// edited\n")
    assert bench.ncu_traffic("zconv", "f32") is None          # demag family changed
    assert bench.ncu_traffic("stage", "f32") is not None      # stage family did not
    assert bench.ncu_traffic("zconv", "f64") is None          # never captured


def test_ingest_keeps_entries_of_kernels_absent_from_the_capture(tree):
    p = tree / "raw.csv"
    write_csv(p, ROWS)
    bench.ingest_ncu(str(p), "f32", "film512 test")
    write_csv(p, [(f"void k_stage4<1, {s}>(Params<float>)", 100.0, 1000.0) for s in range(6)])
    bench.ingest_ncu(str(p), "f32", "film512 test")
    t = json.load(open(tree / "profiles" / "traffic.json"))
    assert t["stage/f32"]["read"] == int(100e6)
    assert t["zconv/f32"]["read"] == int(300e6)


def test_algorithmic_bytes_of_the_film512_passes():
    """512 x 512 x 16, FP32: Hx = 513 kept x frequencies, Py = 1024, Pz = 32."""
    n, s = (512, 512, 16), 4
    N = 512 * 512 * 16
    small = 3 * 16 * 512 * 513 * 8          # complex spectrum after the x pass
    big = 3 * 16 * 1024 * 513 * 8           # after the y pass
    octant = 6 * 17 * 513 * 513 * 4         # real Newell octant
    assert bench.algorithmic_bytes("xfwd", n, s) == 3 * N * 4 + small
    assert bench.algorithmic_bytes("xinv", n, s) == bench.algorithmic_bytes("xfwd", n, s)
    assert bench.algorithmic_bytes("yfwd", n, s) == small + big == bench.algorithmic_bytes("yinv", n, s)
    assert bench.algorithmic_bytes("zconv", n, s) == 2 * big + octant == 510_812_568
    assert bench.algorithmic_bytes("stage", n, s) == pytest.approx(42 * 3 * N * 4 / 6)
    # one field evaluation: about 1.42 GB in FP32, twice that in FP64
    demag = sum(bench.algorithmic_bytes(k, n, s) for k in ("xfwd", "yfwd", "zconv", "yinv", "xinv"))
    assert 1.40e9 < demag < 1.44e9
    assert sum(bench.algorithmic_bytes(k, n, 8) for k in ("xfwd", "yfwd", "zconv", "yinv", "xinv")) == 2 * demag
