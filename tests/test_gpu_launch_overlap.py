"""Programmatic dependent launch changes no result bit.

Every kernel launched through wd_launch may be dispatched while its predecessor still
runs and waits for it (griddepcontrol.wait) before touching memory.  A kernel that read or
wrote too early would race with its predecessor; the same calls made with serialised
launches (WD_PDL=0) must therefore give the same bytes.  The case (operator chains in all
five formats, a BLAS chain, host- and graph-driven solves, a graph-mode batch, the serving
queue and the two-slab decomposed operator) runs in two fresh processes, one per setting.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(tmp_path, pdl):
    path = tmp_path / f"pdl{pdl}.npz"
    env = dict(os.environ, WD_PDL=pdl)
    r = subprocess.run([sys.executable, "-m", "tests._launch_overlap_case", str(path)], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    return np.load(path)


def test_launch_overlap_changes_no_bit(tmp_path):
    on, off = _run(tmp_path, "1"), _run(tmp_path, "0")
    assert set(on.files) == set(off.files) and len(on.files) > 20
    for k in sorted(on.files):
        assert np.array_equal(on[k], off[k]), k
