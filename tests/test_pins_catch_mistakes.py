"""A sample of the planted-mistake check (no GPU): six of the mistakes
listed in oracle/mutants.py, one from each part of the stage, are each
planted in a scratch copy of the oracle, and every CPU pin runs against the
copy; each must be caught.  The full list runs with
``python oracle/mutants.py``."""
import os
import sys
from concurrent.futures import ThreadPoolExecutor

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, os.path.join(ROOT, "oracle"))
import mutants  # noqa: E402

SAMPLE = ("R_imp_swap", "bc_mirror", "sens_curl2d", "csf_smooth_w", "dt_no_abs", "pr_X_is_Y")


def test_a_sample_of_planted_mistakes_is_caught():
    src = open(os.path.join(ROOT, "oracle", "oracle.c")).read()
    table = dict(mutants.MUTANTS)
    tests = mutants.pins()
    assert not any("catch_mistakes" in t for t in tests)
    with ThreadPoolExecutor(len(SAMPLE)) as ex:
        results = list(ex.map(lambda n: mutants.run_one(src, n, table[n], tests), SAMPLE))
    missed = [name for name, caught, _ in results if not caught]
    assert missed == [], missed
