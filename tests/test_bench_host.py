"""Host-side logic of the benchmark that needs no GPU: the stored DRAM traffic of
the ncu capture is reported only while the CUDA sources it was taken on are
unchanged."""
import bench


def _record(path, build, dram=2658735104):
    path.write_text(
        "# DRAM traffic of one solve step\n"
        "# command: ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum ...\n"
        f"kernel_build: {build}\n"
        f"dram_bytes_per_step: {dram}\n"
        "min_bytes_per_step: 1155468240\n")
    return str(path)


def test_traffic_reported_for_the_sources_it_was_captured_on(tmp_path):
    p = _record(tmp_path / "t.txt", bench._kernel_build_id(), 123456789)
    assert bench.stored_traffic(p) == 123456789.0


def test_traffic_withheld_once_the_sources_change(tmp_path):
    other = "0" * 16 if bench._kernel_build_id() != "0" * 16 else "1" * 16
    assert bench.stored_traffic(_record(tmp_path / "t.txt", other)) is None


def test_traffic_withheld_when_missing_or_malformed(tmp_path):
    assert bench.stored_traffic(str(tmp_path / "absent.txt")) is None
    bad = tmp_path / "bad.txt"
    bad.write_text(f"kernel_build: {bench._kernel_build_id()}\ndram_bytes_per_step: n/a\n")
    assert bench.stored_traffic(str(bad)) is None
    bad.write_text(f"kernel_build: {bench._kernel_build_id()}\n")
    assert bench.stored_traffic(str(bad)) is None


def test_build_id_tracks_the_cuda_sources():
    a = bench._kernel_build_id()
    assert len(a) == 16 and a == bench._kernel_build_id()


def test_pure_python_size_rule_matches_the_library(gfc_lib):
    """The oracle legs take (M, N) from bench.padded_size so they never load the
    product library; it must agree with the library's SMOOTH policy."""
    from paper_1902_00176_gb300 import gfc

    for H, W in [(801, 1200), (64, 96), (1024, 1536), (256, 256), (2, 2), (13, 7), (2000, 2000), (2040, 2048),
                 (127, 1999), (600, 333), (300, 1000), (40, 129), (40, 128), (9, 2051)]:
        assert bench.padded_size(H, W) == gfc.padded_size(H, W), (H, W)
    assert tuple(gfc.row_lengths()) == bench.ROW_LENGTHS


def test_gpus_flag_relaunches_under_torchrun_outside_a_job():
    cmd = bench.torchrun_command(4, ["--gpus", "4", "--steps", "5"], {}, python="py")
    assert cmd[:3] == ["py", "-m", "torch.distributed.run"]
    assert "--nproc-per-node=4" in cmd and "127.0.0.1" in cmd
    assert cmd[-4:] == ["--gpus", "4", "--steps", "5"]
    assert cmd[-5].endswith("bench.py")


def test_gpus_flag_inside_a_job():
    assert bench.torchrun_command(1, [], {}) is None
    assert bench.torchrun_command(2, [], {"WORLD_SIZE": "2"}) is None
    import pytest

    with pytest.raises(ValueError):
        bench.torchrun_command(8, [], {"WORLD_SIZE": "2"})


def test_oracle_error_leg_on_cpu():
    """The oracle-error leg compares recorded fields with the oracle (a field equal to
    the oracle's own result has zero error; a perturbed one does not)."""
    import numpy as np

    import oracle.gfc_oracle as O

    rng = np.random.default_rng(0)
    gx, gy = rng.uniform(-0.1, 0.1, (2, 12, 9))
    M, N = bench.padded_size(12, 9)
    ref = O.solve_from_gradient(gx, gy, M, N, 4)
    smp = []
    bench._sample(smp, "a", "grad", ref.copy(), M, N, gx=gx, gy=gy)
    bench._sample(smp, "b", "grad", ref + 1e-3, M, N, gx=gx, gy=gy)
    e = bench.oracle_errors(smp)
    assert e["a"]["rel_l2"] < 1e-14 and e["a"]["fields"] == 1
    assert abs(e["b"]["max_abs"] - 1e-3) < 1e-9


def test_split_flag_parsing():
    assert bench.parse_split("0:50:2:0") == (0, 50, 2, 0)
    assert bench.parse_split("1:0:1:1") == (1, 0, 1, 1)
    for bad in ("0:50:2", "2:0:1:0", "0:-1:1:0", "0:1:1:2", "a:b:c:d"):
        try:
            bench.parse_split(bad)
        except ValueError:
            continue
        raise AssertionError(bad)


def test_issue_roofline_from_a_record(tmp_path):
    p = tmp_path / "i.txt"
    counts = {k: 1.0e6 for k in bench.ISSUE_KEYS}
    p.write_text(f"kernel_build: {bench._kernel_build_id()}\n" + "".join(f"{k}: {v}\n" for k, v in counts.items()))
    rec = bench.stored_record(str(p), bench.ISSUE_KEYS)
    r = bench.issue_roofline(rec, fields=100, ms_step=0.5, clocks={"sm_mhz": 2000.0})
    # 3e8 warp instructions in 0.5 ms = 0.6 T/s against 152 x 4 x 2 GHz = 1.216 T/s
    assert abs(r["achieved"] - 0.6) < 1e-12 and abs(r["peak"] - 1.216) < 1e-12
    assert abs(r["fp32"]["peak"] - 152 * 128 * 2e9 / 1e12) < 1e-9
    assert bench.issue_roofline(None, 100, 0.5, None) is None
    p.write_text("kernel_build: 0000\n" + "".join(f"{k}: 1\n" for k in bench.ISSUE_KEYS))
    assert bench.stored_record(str(p), bench.ISSUE_KEYS) is None
