"""Host logic of the launch autotuner (no GPU)."""
import numpy as np

from paper_2602_21911_gb300 import autotune, grprec
from paper_2602_21911_gb300 import inputs as I


def test_candidates_cover_every_form_for_short_domains():
    p = dict(n_cells=np.array([4, 100, 512]), system=1, M=2, bc=np.ones(3))
    forms = {c[0] for c in autotune.candidates(p)}
    assert forms == {grprec.GRP_LAUNCH_FLAT, grprec.GRP_LAUNCH_SPLIT, grprec.GRP_LAUNCH_FUSED}
    for mode, threads, cells, k in autotune.candidates(p):
        assert threads in (128, 256) and 64 <= cells <= 1 << 20 and 1 <= k <= 1024


def test_one_long_domain_runs_flat_only():
    p = dict(n_cells=np.array([1 << 20]), system=1, M=2, bc=np.ones(1))
    assert autotune.candidates(p) == [(grprec.GRP_LAUNCH_FLAT, 256, 2048, 1)]


def test_signature_depends_on_the_cell_counts():
    a = dict(n_cells=np.array([4, 100, 512]), system=1, M=2, bc=np.ones(3))
    b = dict(a, n_cells=np.array([4, 100, 511]))
    assert autotune.signature(a) == autotune.signature(dict(a))
    assert autotune.signature(a) != autotune.signature(b)
