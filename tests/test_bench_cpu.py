"""Host-side pieces of the benchmark that fix its roofline numbers (no GPU).

The wavelet roofline counts every level's input read and output write once:
level j of a d-dimensional transform moves 8 B per cell of its 2^{-dj}-sized
input.  The sums are written out here term by term, independently of the
closed form the benchmark uses."""
import pytest

import bench


@pytest.mark.parametrize("dim,levels", [(2, 5), (3, 4), (2, 1), (3, 1), (2, 3)])
def test_dwt_bytes_per_cell_is_the_level_sum(dim, levels):
    expect = sum(8.0 / (2 ** dim) ** j for j in range(levels))
    assert bench.dwt_bytes_per_cell(dim, levels) == pytest.approx(expect, rel=1e-15)


def test_dwt_bytes_match_the_workload_figures():
    # 10.66 B per pixel for the 2D db4 5-level transform, 9.14 B per voxel for the 3D 4-level one
    assert bench.dwt_bytes_per_cell(2, 5) == pytest.approx(10.65625)
    assert bench.dwt_bytes_per_cell(3, 4) == pytest.approx(9.140625)


def test_profile_traffic_is_read_only_for_its_own_source(tmp_path, monkeypatch):
    # a summary whose source hash differs from the current kernel source gives no traffic figure
    spec = dict(bench.WORKLOADS["tree3d"])
    profile = tmp_path / "stale.txt"
    profile.write_text("source_sha256_16: 0000000000000000\ndram_bytes_per_launch: 1.0e8\n")
    monkeypatch.setitem(bench.WORKLOADS, "stale", dict(spec, profile=str(profile)))
    traffic, digest = bench.kernel_traffic("stale")
    assert traffic is None and len(digest) == 16
    profile.write_text(f"source_sha256_16: {digest}\ndram_bytes_per_launch: 1.0e8\n")
    assert bench.kernel_traffic("stale")[0] == pytest.approx(1.0e8)
