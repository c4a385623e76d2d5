"""Box trees over long successor lists (CPU): the host builder of
csrc/hub_index.cpp is compiled here into a small host program, run on
synthetic tables, and its trees are checked against their definition:

- a tree for exactly the lists of at least min_row entries, and none at all
  when the longest list is shorter than min_longest;
- a tree's entries are its list's entries (same ranks, each with its site's
  coordinates), in chunks of 32, the last chunk padded with rank 2^31 - 1;
- a level-0 node is the exact bounding box and smallest / largest rank of
  its chunk's real entries, a level-l node those of its 32 children, and the
  top level has at most 32 nodes.

The one-warp kernel's walk prunes with these boxes; the GPU tests check
that its rows equal the scan's."""
from __future__ import annotations

import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2605_02224_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>
#include "hub_index.h"

template <class T>
std::vector<T> load(const char* path, size_t count) {
  std::vector<T> v(count);
  FILE* f = std::fopen(path, "rb");
  if (!f || std::fread(v.data(), sizeof(T), count, f) != count) std::exit(2);
  std::fclose(f);
  return v;
}

template <class T>
void save(const char* path, const std::vector<T>& v) {
  FILE* f = std::fopen(path, "wb");
  if (!f) std::exit(3);
  if (!v.empty()) std::fwrite(v.data(), sizeof(T), v.size(), f);
  std::fclose(f);
}

int main(int argc, char** argv) {
  // dir n E min_row min_longest
  if (argc != 6) return 1;
  const std::string dir = argv[1];
  const long long n = std::atoll(argv[2]), E = std::atoll(argv[3]);
  const auto xyz = load<float>((dir + "/xyz").c_str(), 3 * n);
  const auto rowp = load<long long>((dir + "/rowp").c_str(), n + 1);
  const auto succ = load<int>((dir + "/succ").c_str(), E);
  std::vector<int64_t> rp(rowp.begin(), rowp.end());
  mknn::HubIndex H;
  mknn::build_hub_index(n, xyz.data(), rp.data(), succ.data(), std::atoll(argv[4]),
                        std::atoll(argv[5]), &H);
  save((dir + "/hub_of").c_str(), H.hub_of);
  save((dir + "/desc").c_str(), H.desc);
  save((dir + "/ent").c_str(), H.ent);
  save((dir + "/node").c_str(), H.node);
  std::printf("%lld\n", (long long)H.hubs());
  return 0;
}
"""


def _table(seed: int):
    """60,000 random sites; list 0 holds every later site (59,999 entries: a
    tree of three levels), list 1 every third site up to 40,000, lists 2..8
    a few thousand random later sites (two levels), list 9 about 700 (one
    level), the rest up to 40 random ones."""
    rng = np.random.default_rng(seed)
    n = 60_000
    xyz = rng.random((n, 3), dtype=np.float32)
    xyz[: n // 2, 2] *= np.float32(1e-3)            # half the sites on a thin slab
    rows = [np.arange(1, n), np.arange(2, 40_000, 3)]
    for i in range(2, 10):
        rows.append(np.unique(rng.integers(i + 1, n, 3000 + 700 * i if i < 9 else 700)))
    for i in range(10, n):
        cnt = int(rng.integers(0, 41)) if i < n - 1 else 0
        rows.append(np.unique(rng.integers(i + 1, n, cnt)) if cnt and i + 1 < n else
                    np.zeros(0, np.int64))
    rowp = np.zeros(n + 1, np.int64)
    rowp[1:] = np.cumsum([len(r) for r in rows])
    succ = np.concatenate(rows).astype(np.int32)
    return xyz, rowp, succ


def _build(tmp_path, xyz, rowp, succ, min_row, min_longest):
    src = tmp_path / "t.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "t"
    subprocess.run(["g++", "-std=c++17", "-O2", f"-I{CSRC}", str(src),
                    os.path.join(CSRC, "hub_index.cpp"), "-o", str(exe)], check=True)
    d = tmp_path / "io"
    d.mkdir(exist_ok=True)
    xyz.astype(np.float32).tofile(d / "xyz")
    rowp.astype(np.int64).tofile(d / "rowp")
    succ.astype(np.int32).tofile(d / "succ")
    out = subprocess.run([str(exe), str(d), str(len(rowp) - 1), str(len(succ)), str(min_row),
                          str(min_longest)], check=True, capture_output=True, text=True)
    hubs = int(out.stdout.strip())
    return (hubs, np.fromfile(d / "hub_of", np.int32), np.fromfile(d / "desc", np.int32),
            np.fromfile(d / "ent", np.float32).reshape(-1, 4),
            np.fromfile(d / "node", np.float32).reshape(-1, 8))


def _levels(length: int):
    """(offset, count) of each level of a tree over `length` entries."""
    out, c, o = [], (length + 31) // 32, 0
    while True:
        out.append((o, c))
        if c <= 32:
            return out
        o += c
        c = (c + 31) // 32


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_trees_match_their_definition(tmp_path):
    xyz, rowp, succ = _table(5)
    L = np.diff(rowp)
    hubs, hub_of, desc, ent, node = _build(tmp_path, xyz, rowp, succ, 256, 4096)
    long_rows = np.flatnonzero(L >= 256)
    assert hubs == len(long_rows) == 10
    assert np.array_equal(np.flatnonzero(hub_of >= 0), long_rows)
    assert np.array_equal(hub_of[long_rows], np.arange(hubs))
    desc = desc.reshape(-1, 4)
    seen_levels = set()
    for h, i in enumerate(long_rows):
        first, length, node0, levels = (int(x) for x in desc[h])
        row = succ[rowp[i]:rowp[i + 1]]
        assert length == len(row)
        lv = _levels(length)
        assert levels == len(lv) and lv[-1][1] <= 32
        seen_levels.add(levels)
        chunks = (length + 31) // 32
        e = ent[first:first + 32 * chunks]
        ranks = e[:, 3].view(np.int32)
        real, pad = ranks[:length], ranks[length:]
        assert np.all(pad == 2**31 - 1)
        assert np.array_equal(np.sort(real), row)            # the list's entries, reordered
        assert np.array_equal(e[:length, :3], xyz[real])      # each with its site
        # level 0: the exact box and rank range of each chunk's real entries
        for c in range(chunks):
            sl = slice(32 * c, min(length, 32 * c + 32))
            b = node[node0 + c]
            assert np.array_equal(b[:3], e[sl, :3].min(0)) and np.array_equal(b[4:7], e[sl, :3].max(0))
            assert b[3:4].view(np.int32)[0] == real[sl].min()
            assert b[7:8].view(np.int32)[0] == real[sl].max()
        # level l: the union of its 32 children
        for l in range(1, levels):
            off, cnt = lv[l]
            coff, ccnt = lv[l - 1]
            for j in range(cnt):
                ch = node[node0 + coff + 32 * j: node0 + coff + min(ccnt, 32 * j + 32)]
                b = node[node0 + off + j]
                assert np.array_equal(b[:3], ch[:, :3].min(0))
                assert np.array_equal(b[4:7], ch[:, 4:7].max(0))
                assert b[3:4].view(np.int32)[0] == ch[:, 3].view(np.int32).min()
                assert b[7:8].view(np.int32)[0] == ch[:, 7].view(np.int32).max()
    assert seen_levels == {1, 2, 3}
    # Morton order keeps chunks compact: the chunks' boxes of list 0 are far
    # smaller than the list's own box (the walk's pruning depends on it)
    first, length, node0, _ = desc[0]
    boxes = node[node0:node0 + (length + 31) // 32]
    vol = np.prod(boxes[:, 4:7] - boxes[:, :3], axis=1)
    full = np.prod(xyz[1:].max(0) - xyz[1:].min(0))
    assert np.median(vol) < 1e-3 * full


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_no_trees_below_the_longest_list_threshold(tmp_path):
    xyz, rowp, succ = _table(6)
    L = np.diff(rowp)
    hubs, hub_of, desc, ent, node = _build(tmp_path, xyz, rowp, succ, 256, int(L.max()) + 1)
    assert hubs == 0 and hub_of.size == 0 and desc.size == 0 and ent.size == 0
    # the cloud-level threshold met exactly: every long list gets its tree
    hubs, hub_of, *_ = _build(tmp_path, xyz, rowp, succ, 256, int(L.max()))
    assert hubs == int((L >= 256).sum())
