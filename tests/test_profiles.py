"""The committed ncu summary behind the bench's roofline: its format, and that
it was captured on the kernel source as it stands (the bench reads its
executed flops and DRAM bytes only when the source digest matches)."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_flux_summary_is_of_the_current_source_and_parses():
    kname = "k_flux + k_flux_hard<Euler,M=2>"
    prof = bench.profiled(6_795_002, kname)
    assert prof is not None, "profiles/k_flux_batched_m2.txt is stale or of another kernel: recapture it"
    assert 200.0 < prof["executed_flops_per_cell_update"] < 646.3      # below the oracle's algorithmic count
    # DRAM bytes per launch scaled to the batch: near the 96 B per cell-update of the algorithm
    assert 0.5 < prof["traffic"] / (96.0 * 6_795_002) < 1.5


def test_every_summary_names_its_command_and_source():
    d = os.path.join(ROOT, "profiles")
    for f in sorted(os.listdir(d)):
        text = open(os.path.join(d, f)).read()
        assert "ncu" in text and "--clock-control none" in text, f
        if "source_digest:" in text:
            digest = text.split("source_digest:")[1].split()[0]
            assert digest == bench.source_digest(), f
