"""The committed ncu summaries and the bench's reading of them (host logic).

* every summary gives the command that made it, running committed files;
* the fused-kernel summaries were taken from one build (one source digest);
* bench.recorded_counter returns a summary's counters exactly when the digest
  matches the kernel sources, and None otherwise.
"""
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PROFILES = sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md")))
FUSED = {os.path.basename(p)[len("fused_kernel_"):-3]: p for p in PROFILES
         if os.path.basename(p).startswith("fused_kernel_")}


def _digest(path):
    m = re.search(r"kernel_source_digest: (\w+)", open(path).read())
    return m.group(1) if m else None


def test_summaries_exist_and_name_their_commands():
    assert PROFILES, "no ncu summaries committed"
    for p in PROFILES:
        text = open(p).read()
        cmds = re.findall(r"`(ncu [^`]+)`", text)
        assert cmds, f"{p}: no ncu command"
        for c in cmds:
            assert "--clock-control none" in c, f"{p}: ncu without --clock-control none"
            assert "python bench.py" in c, f"{p}: capture does not run the committed bench"
        assert "_work" not in text


def test_fused_summaries_share_one_build():
    digests = {w: _digest(p) for w, p in FUSED.items()}
    assert {"3d_gauss_L8", "chimera_pmj_C8"} <= set(digests)
    assert all(digests.values()), digests
    assert len(set(digests.values())) == 1, digests


def test_recorded_counter_follows_the_digest(monkeypatch):
    bench = pytest.importorskip("bench")
    for w, p in FUSED.items():
        text = open(p).read()
        ipu = float(re.search(r"instructions_per_update: ([0-9.]+)", text).group(1))
        monkeypatch.setattr(bench, "kernel_source_digest", lambda d=_digest(p): d)
        assert bench.recorded_counter(w, "instructions_per_update") == ipu
        m = re.search(r"traffic_bytes_per_launch: ([0-9.]+)", text)
        if m:
            assert bench.recorded_traffic(w) == float(m.group(1))
        monkeypatch.setattr(bench, "kernel_source_digest", lambda: "0" * 16)
        assert bench.recorded_counter(w, "instructions_per_update") is None
