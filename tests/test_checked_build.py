"""The checked build (-DICM_CHECKED): every data-dependent index of the fused
kernel (neighbour positions, coupling rows, threshold entries, partial-energy
slots, mask words, seed sites, PT positions and runs, histogram bins) is
tested against its bound, and an index out of range is recorded in a device
check word instead of being used.  This stands in for a memory checker: on
+-J cases of every lattice kind, diluted, wide-CTA and thread-block-cluster
batches (whose kernel guards its neighbour positions, seed sites and
histogram bins too) and a Gaussian batch, the check words stay zero and the
chain still equals the oracle's."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_finds_no_out_of_range_index():
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_run.py")], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out["rc"] == 0
    assert out["check"][0] == 0, out["check"]         # count, site code, index, bound of the first
    assert out["rc_cluster"] == 0
    assert out["check_cluster"][0] == 0, out["check_cluster"]
    assert out["mismatch"] == []
