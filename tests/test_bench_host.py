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
