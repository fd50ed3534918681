"""bench.py's reading of the committed ncu summary of the resident cell
kernels: the file parses, carries every figure the bench line uses, and its
traffic is reported only while the kernel sources are the ones it was
captured from (sha256 prefix of cell_run.cu, common.cuh and classes.cuh)."""
import hashlib
import os

import pytest

pytest.importorskip("torch")
import bench  # noqa: E402

KEYS = ("sources_sha256_16", "dram_bytes_per_interval", "dram_bytes_read_per_interval",
        "dram_bytes_write_per_interval", "warp_instructions_per_interval", "fp32_pipe_frac")


def test_profile_summary_parses_and_matches_its_sources():
    traffic, rec = bench.profile_traffic()
    assert rec is not None
    for k in KEYS:
        assert k in rec, k
    h = hashlib.sha256()
    for f in ("cell_run.cu", "common.cuh", "classes.cuh"):
        h.update(open(os.path.join(bench.ROOT, "paper_2303_07819_gb300", "csrc", f), "rb").read())
    if h.hexdigest()[:16] == rec["sources_sha256_16"]:
        assert traffic == float(rec["dram_bytes_per_interval"])
    else:
        assert traffic is None
    assert 0.0 < float(rec["fp32_pipe_frac"]) < 1.0
    rd, wr, tot = (float(rec[k]) for k in ("dram_bytes_read_per_interval", "dram_bytes_write_per_interval",
                                           "dram_bytes_per_interval"))
    assert rd + wr == tot
    # resident kernels: a floe's state crosses DRAM about once per interval,
    # far below the 56 B per floe-step of the per-step formulation
    floes, n0 = 1982044, 100
    assert tot < 0.05 * floes * n0 * bench.BYTES_PER_FLOE_STEP
