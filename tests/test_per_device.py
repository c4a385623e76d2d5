"""Per-device launch state (CPU): a kernel attribute, an occupancy or an SM
count cached for one device must not be reused for another. The table the
library keeps them in (csrc/per_device.h) is compiled here into a small
host program that fills entries for fake device ordinals."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2605_02224_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "per_device.h"
using mknn::PerDevice;
struct State { bool attr; int occ_for[33]; };
int main() {
  PerDevice<State> t;
  int calls = 0;
  // device 0: first use sets the attribute and caches occupancy 5 for kcap 16
  auto fill = [&](int dev, int occ) {
    return t.with(dev, -1, [&](State& s) {
      if (!s.attr) { s.attr = true; ++calls; }
      if (!s.occ_for[16]) s.occ_for[16] = occ;
      return s.occ_for[16];
    });
  };
  int a = fill(0, 5);
  int b = fill(1, 3);       // another device: its own entry, its own attribute call
  int c = fill(0, 9);       // device 0 again: cached value, no new attribute call
  int d = fill(64, 7);      // out of range: rejected
  int e = fill(-1, 7);
  std::printf("%d %d %d %d %d %d\n", a, b, c, d, e, calls);
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_per_device_entries_are_separate(tmp_path):
    src = tmp_path / "t.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "t"
    subprocess.run(["g++", "-std=c++17", "-O1", f"-I{CSRC}", str(src), "-o", str(exe),
                    "-lpthread"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert out == ["5", "3", "5", "-1", "-1", "2"]


def test_no_process_wide_launch_state_left():
    """The launch code keeps no process-wide kernel attribute or occupancy
    cache: every such cache is a PerDevice table."""
    for name in ("knn_plain.cu", "batch.cu"):
        with open(os.path.join(CSRC, name)) as f:
            text = f.read()
        assert "std::once_flag" not in text and "call_once" not in text, name
        assert "static int occ" not in text and "static bool attr" not in text, name
        assert "static int sms" not in text, name
