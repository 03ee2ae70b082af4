"""Host-side helpers of bench.py (no GPU): the algorithmic byte and operation counts behind the
reported rooflines, the RMSE gate, the split of an epoch's timings, and the rule that a committed
DRAM-traffic record is used only while the kernel source it was taken on is unchanged."""
import json
from types import SimpleNamespace

import pytest

import bench
import synth


def test_sgd_bytes_per_rating_of_the_paper_model():
    # per rating 4 (user slot) + 1 (rating) + K/8 (mask) + 8F (u_i read and write) + 8 (b_i read and
    # write), plus one byte per explicit neighbour rating
    w = SimpleNamespace(F=64, K=64, M=10, N=20)
    stats = {"nnz": 1000, "explicit_neighbours": 6500}
    assert bench.sgd_bytes_per_epoch(stats, w) == 1000 * (4 + 1 + 8 + 512 + 8) + 6500
    # compulsory: the rating stream and one read and one write of every parameter (FP32)
    params = 4 * (10 * 64 + 20 * 64 + 10 + 20 + 2 * 20 * 64)
    assert bench.sgd_min_bytes_per_epoch(stats, w) == 1000 * (4 + 1 + 8) + 6500 + 2 * params


def test_signature_bytes_match_the_netflix_shape_figure():
    w = synth.MID                      # L = 16 x 12 bits: 3 hash words, padded to 3
    nnz = 98_578_120
    b = bench.sig_bytes(w, nnz)
    assert b == 5 * nnz + 8 * (w.N + 1) + 8 * 3 * w.M + 4 * 16 * w.N + 8 * 64 * 3 * w.N
    assert abs(b / 1e6 - 533.0) < 0.5     # the 533 MB quoted beside the signature roofline


def test_integer_peak_and_signature_ops():
    assert bench.INT32_PEAK_TOPS == pytest.approx(152 * 128 * 2.07e9 / 1e12)
    # Eq. 3 as defined: L x bits signed adds per rating
    assert synth.MID.L * synth.MID.bits == 192 and synth.LARGE.L * synth.LARGE.bits == 512


def test_rmse_gate():
    ok = bench.rmse_parity(0.5871, 0.5870, "s")
    assert ok["pass"] and ok["rel"] == pytest.approx(0.0001 / 0.5870)
    bad = bench.rmse_parity(0.60, 0.5870, "s")
    assert not bad["pass"] and bad["bar"] == 2e-3


def test_epoch_split_first_and_later():
    first, later = bench.epoch_split([5.0, 2.0, 2.0, 6.0, 2.0, 4.0], 3)
    assert first == pytest.approx(5.5) and later == pytest.approx(2.0)
    assert bench.epoch_split([3.0, 4.0], 1)[1] is None


def test_traffic_record_only_for_the_source_it_was_taken_on(tmp_path, monkeypatch):
    prof = tmp_path / "profiles"
    prof.mkdir()
    rec = {"sgd_epoch": {"wl": {"kernel_source_sha1": "abc", "dram_bytes_per_epoch": 7}}}
    (prof / "dram_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.profile_entry("sgd_epoch", "wl", "abc")["dram_bytes_per_epoch"] == 7
    assert bench.profile_entry("sgd_epoch", "wl", "changed") is None
    assert bench.profile_entry("sgd_epoch", "other", "abc") is None


def test_committed_traffic_record_matches_the_current_kernel_sources():
    """The committed record names the source hash it was taken on; the bench reports it as traffic
    only while the hash matches (this test fails when a kernel source changes without a new capture)."""
    with open(bench.os.path.join(bench.ROOT, "profiles", "dram_traffic.json")) as f:
        rec = json.load(f)
    assert rec["sgd_epoch"]["mid-480kx17770-100M"]["kernel_source_sha1"] == bench.kernel_hash()
    assert rec["signatures"]["mid-480kx17770-100M"]["kernel_source_sha1"] == \
        bench.kernel_hash(("simlsh.cu", "common.cuh"))
