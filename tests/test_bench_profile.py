"""bench.py's reading of the committed ncu summary of the cell-step kernels:
the file parses, carries every figure the bench line uses, and its traffic
is reported only while the kernel sources are the ones it was captured
from (sha256 prefix of cell_step.cu, common.cuh and classes.cuh)."""
import hashlib
import os

import pytest

pytest.importorskip("torch")
import bench  # noqa: E402

KEYS = ("sources_sha256_16", "dram_bytes_read_per_fine_step", "dram_bytes_write_per_fine_step",
        "warp_instructions_per_fine_step", "warp_instructions_list_step", "warp_instructions_rebuild_step",
        "fp32_pipe_frac")


def test_profile_summary_parses_and_matches_its_sources():
    traffic, rec = bench.profile_traffic()
    assert rec is not None
    for k in KEYS:
        assert k in rec, k
    h = hashlib.sha256()
    for f in ("cell_step.cu", "common.cuh", "classes.cuh"):
        h.update(open(os.path.join(bench.ROOT, "paper_2303_07819_gb300", "csrc", f), "rb").read())
    if h.hexdigest()[:16] == rec["sources_sha256_16"]:
        assert traffic == float(rec["dram_bytes_read_per_fine_step"]) + float(rec["dram_bytes_write_per_fine_step"])
    else:
        assert traffic is None
    assert 0.0 < float(rec["fp32_pipe_frac"]) < 1.0
    wl, wr, wf = (float(rec[k]) for k in ("warp_instructions_list_step", "warp_instructions_rebuild_step",
                                          "warp_instructions_per_fine_step"))
    # a gradual-update period: 9 list steps and one rebuild, plus the packed
    # cells' share, which is below a list step's
    assert 0.9 * wl + 0.1 * wr <= wf <= 0.9 * wl + 0.1 * wr + wl
