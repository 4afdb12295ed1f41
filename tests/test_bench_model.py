"""Host logic of the benchmark (CPU only): the byte models behind the roofline fractions,
the peak lookup and the profiled-traffic lookup."""
import json
import os

import pytest

import bench
import workloads


@pytest.mark.parametrize("name,mb", [("film_small", 0.611856), ("film_large", 371.644536),
                                     ("block", 1466.709528)])
def test_five_pass_model_matches_the_stated_byte_counts(name, mb):
    """Bytes per step of a design that streams every intermediate spectrum through HBM:
    the figures the hot-path measurement plan states for these workloads."""
    f = getattr(workloads, name)().films[0]
    assert bench.five_pass_bytes(f) / 1e6 == pytest.approx(mb, rel=1e-9)


def test_fused_bytes_of_film_large():
    """x pass: read S and m, write S and m; fused y-z pass: read S and T, write S."""
    f = workloads.film_large().films[0]
    b = bench.algorithmic_bytes(None, f)
    S = 3 * 4 * 1025 * 256 * 8                   # [3][nz][Kx][ny] complex FP32
    T = 1025 * 22 * 257 * 4                      # [Kx][22 direct-z slots][Ky] FP32
    N = 1024 * 256 * 4
    assert b["x_fast"] == 2 * S + 24 * N
    assert b["yz_fast"] == 2 * S + T
    assert b["per_cell"] == pytest.approx((4 * S + T + 24 * N) / N)


def test_split_path_bytes_of_the_block():
    """256x256x64 block (split path): x pass as above; y FFT either way: ny rows in, Py rows
    out (or back); z pass: read and write the Py rows and read the 6-component octant."""
    f = workloads.block().films[0]
    b = bench.algorithmic_bytes(None, f)
    N = 256 * 256 * 64
    Kx, Ky, Kz = 257, 257, 65
    A1, A2 = Kx * 256 * 64, Kx * 512 * 64
    assert b["x_fast"] == 2 * 24 * A1 + 24 * N
    assert b["y_fast"] == 24 * A1 + 24 * A2
    assert b["z_fast"] == 48 * A2 + Kx * Ky * Kz * 6 * 4
    assert b["per_cell"] * N / 1e6 == pytest.approx(1416.37788, rel=1e-9)
    # the split path moves the five-pass bytes less one extra read of m
    assert bench.five_pass_bytes(f) - b["per_cell"] * N == pytest.approx(12 * N)


def test_kernel_rooflines():
    f = workloads.block().films[0]
    byt = bench.algorithmic_bytes(None, f)
    r = bench.kernel_rooflines({"y_fast": (2.2, 40), "other": (1.0, 1)}, byt, 6000.0, "measured",
                               "no_such_workload")
    assert set(r) == {"y_fast"}
    y = r["y_fast"]
    assert y["avg_launch_us"] == pytest.approx(55.0)
    assert y["achieved"] == pytest.approx(byt["y_fast"] / 55e-6 / 1e9, abs=0.05)
    assert y["frac"] == pytest.approx(y["achieved"] / 6000.0, abs=1e-4)
    assert y["traffic"] is None


def test_peak_lookup(tmp_path, monkeypatch):
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.measured_peaks() == (6800.0, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6783.5}))
    assert bench.measured_peaks() == (6783.5, "measured")


def test_recorded_traffic_follows_the_kernel_sources():
    """profiles/traffic.json is used only while the kernel sources hash to the profiled ones."""
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as fh:
        rec = json.load(fh)
    got = bench.recorded_traffic("x_fast", "film_large")
    if rec["source_hash"] == bench.kernel_source_hash():
        assert got == rec["kernels"]["film_large"]["x_fast"]
    else:
        assert got is None


def test_all_cores_oracle_replicas():
    """Spawned single-threaded oracle replicas over a common window: every replica reports,
    and the aggregate is the sum of their rates."""
    r = bench.cpu_baseline_all_cores("film_small", 1.0, 2)
    assert r["cores"] == r["replicas"] == 2
    assert r["kind"] == "oracle" and r["unit"] == bench.UNIT
    assert r["value"] > 0
