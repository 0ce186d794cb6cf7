"""Host logic of the server without a GPU: the arena allocator and the FIFO
continuous-batching scheduler (the header-only C++ in csrc/tdse_sched.h),
compiled here with g++ into a small command interpreter and driven with
seeded random scenarios.  The allocator is compared with an independent
first-fit model written from its definition (lowest-offset free range that
fits; freed ranges merge with free neighbours); the scheduler is checked
against its contract (FIFO admission, budget and slot limits, min(k, left)
steps per batch, every request finishing, memory returned on release).  The
group cut of the batch engine's pipelined copy-in / propagate / copy-out
(io_groups) is compared with a model written from its definition."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1308_1856_gb300", "csrc")

DRIVER = r"""
#include <iostream>
#include <string>
#include <vector>
#include "tdse_sched.h"
using namespace tdse_sched;
int main() {
  std::string cmd;
  size_t size, align; int slots;
  std::cin >> size >> align >> slots;
  Arena a(size, align);
  Scheduler s(size, slots, align);
  std::vector<int> ps; std::vector<long> pk; std::vector<long long> pid;
  while (std::cin >> cmd) {
    if (cmd == "A") { size_t b; std::cin >> b; size_t o = a.alloc(b);
      std::cout << (o == Arena::npos ? -1LL : (long long)o) << "\n"; }
    else if (cmd == "F") { size_t o; std::cin >> o; std::cout << (a.release(o) ? 1 : 0) << "\n"; }
    else if (cmd == "S") { std::cout << a.in_use() << " " << a.largest_free() << " " << a.free_ranges() << "\n"; }
    else if (cmd == "sub") { size_t b; long k; std::cin >> b >> k; std::cout << s.submit(b, k) << "\n"; }
    else if (cmd == "adm") { auto v = s.admit(); std::cout << v.size();
      for (auto &x : v) std::cout << " " << x.id << " " << x.slot << " " << x.offset; std::cout << "\n"; }
    else if (cmd == "plan") { long k; std::cin >> k; s.plan(k, ps, pk, pid); std::cout << ps.size();
      for (size_t i = 0; i < ps.size(); ++i) std::cout << " " << pid[i] << " " << ps[i] << " " << pk[i];
      std::cout << "\n"; }
    else if (cmd == "adv") { auto f = s.advance(pid, pk); std::cout << f.size();
      for (auto x : f) std::cout << " " << x; std::cout << "\n"; }
    else if (cmd == "poll") { auto f = s.poll(); std::cout << f.size();
      for (auto x : f) std::cout << " " << x; std::cout << "\n"; }
    else if (cmd == "pollrel") { auto f = s.poll(); std::cout << f.size();
      for (auto x : f) { std::cout << " " << x; s.release(x); } std::cout << "\n"; }
    else if (cmd == "rel") { long long id; std::cin >> id; std::cout << s.release(id) << "\n"; }
    else if (cmd == "cut") { int n, g; double r; size_t qu; std::cin >> n >> g >> r >> qu;
      std::vector<size_t> off(n + 1); for (auto &x : off) std::cin >> x;
      auto f = io_groups(off, g, r, qu); std::cout << f.size();
      for (auto x : f) std::cout << " " << x; std::cout << "\n"; }
    else if (cmd == "q") { std::cout << s.queued() << " " << s.running() << " " << s.resident() << " "
      << s.arena().in_use() << " " << s.finished_total() << "\n"; }
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    d = tmp_path_factory.mktemp("sched")
    src = d / "driver.cpp"
    src.write_text(DRIVER)
    exe = d / "driver"
    subprocess.run([gxx, "-std=c++17", "-O1", "-Wall", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    return str(exe)


class Session:
    """Runs a batch of commands through the driver and returns its output lines."""

    def __init__(self, exe, size, align, slots):
        self.exe, self.head = exe, f"{size} {align} {slots}\n"

    def run(self, cmds):
        out = subprocess.run([self.exe], input=self.head + "\n".join(cmds) + "\n", text=True,
                             capture_output=True, check=True).stdout
        return out.strip().split("\n") if out.strip() else []


class FirstFit:
    """First fit from its definition: a sorted list of free (offset, length)."""

    def __init__(self, size, align):
        self.align = align
        self.size = size - size % align
        self.free = [(0, self.size)] if self.size else []
        self.live = {}

    def alloc(self, b):
        need = -(-max(b, 1) // self.align) * self.align
        for k, (o, n) in enumerate(self.free):
            if n >= need:
                self.free[k:k + 1] = [(o + need, n - need)] if n > need else []
                self.live[o] = need
                return o
        return -1

    def release(self, o):
        if o not in self.live:
            return 0
        n = self.live.pop(o)
        self.free.append((o, n))
        self.free.sort()
        merged = []
        for fo, fn in self.free:
            if merged and merged[-1][0] + merged[-1][1] == fo:
                merged[-1] = (merged[-1][0], merged[-1][1] + fn)
            else:
                merged.append((fo, fn))
        self.free = merged
        return 1

    def stats(self):
        return (sum(self.live.values()), max((n for _, n in self.free), default=0), len(self.free))


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_arena_matches_first_fit_model(driver, seed):
    rng = np.random.default_rng(seed)
    size, align = 1 << 20, 256
    model = FirstFit(size, align)
    cmds, expect, live = [], [], []
    for _ in range(600):
        if live and rng.random() < 0.45:
            o = live.pop(int(rng.integers(len(live))))
            cmds.append(f"F {o}")
            expect.append(str(model.release(o)))
        else:
            b = int(rng.integers(1, 60000))
            o = model.alloc(b)
            if o >= 0:
                live.append(o)
            cmds.append(f"A {b}")
            expect.append(str(o))
        if rng.random() < 0.1:
            cmds.append("S")
            expect.append("%d %d %d" % model.stats())
    # releasing an unknown offset fails; freeing everything restores one range
    cmds.append("F 12345")
    expect.append("0")
    for o in live:
        cmds.append(f"F {o}")
        expect.append("1")
    cmds.append("S")
    expect.append(f"0 {size} 1")
    got = Session(driver, size, align, 4).run(cmds)
    assert got == expect


def test_arena_live_ranges_never_overlap(driver):
    rng = np.random.default_rng(7)
    cmds, sizes = [], []
    for _ in range(200):
        b = int(rng.integers(1, 5000))
        cmds.append(f"A {b}")
        sizes.append(b)
    got = [int(x) for x in Session(driver, 1 << 20, 256, 4).run(cmds)]
    spans = sorted((o, o + -(-b // 256) * 256) for o, b in zip(got, sizes) if o >= 0)
    assert all(o % 256 == 0 for o, _ in spans)
    assert all(a[1] <= b[0] for a, b in zip(spans, spans[1:]))
    assert spans[-1][1] <= 1 << 20


def _parse_ints(line):
    return [int(x) for x in line.split()]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_scheduler_contract(driver, seed):
    """Random submissions, step batches, polls and releases: admission is FIFO,
    the budget and slot limits hold, each batch gives min(k, left) steps, and
    every request finishes with exactly its steps."""
    rng = np.random.default_rng(100 + seed)
    size, align, slots = 4 << 20, 256, 6
    sess = Session(driver, size, align, slots)
    cmds = []
    reqs = []
    for _ in range(40):
        b = int(rng.integers(50_000, 1_500_000))
        k = int(rng.integers(1, 700))
        reqs.append((b, k))
        cmds.append(f"sub {b} {k}")
    cmds.append(f"sub {size + 1} 5")       # can never fit
    cmds.append("sub 1000 0")              # no steps
    for _ in range(400):
        cmds += ["adm", "plan 100", "adv", "pollrel", "q"]
    out = sess.run(cmds)
    ids = [int(x) for x in out[:40]]
    assert ids == list(range(1, 41))
    assert out[40] == "-1" and out[41] == "-1"
    # replay the loop; finished requests are released as soon as they are polled
    admitted, done = [], {i: 0 for i in ids}
    pos = 42
    finished = set()
    for _ in range(400):
        adm = _parse_ints(out[pos]); plan = _parse_ints(out[pos + 1]); adv = _parse_ints(out[pos + 2])
        poll = _parse_ints(out[pos + 3]); q = _parse_ints(out[pos + 4])
        pos += 5
        for t in range(adm[0]):
            rid, slot, off = adm[1 + 3 * t: 4 + 3 * t]
            admitted.append(rid)
            assert 0 <= slot < slots and off % align == 0
        for t in range(plan[0]):
            rid, slot, k = plan[1 + 3 * t: 4 + 3 * t]
            left = reqs[rid - 1][1] - done[rid]
            assert k == min(100, left) and k > 0
            done[rid] += k
        for rid in adv[1:]:
            assert done[rid] == reqs[rid - 1][1]
            finished.add(rid)
        assert set(poll[1:]) <= finished
        queued, running, resident, in_use, fin_total = q
        assert resident <= slots and in_use <= size
        assert fin_total == len(finished)
    assert admitted == sorted(admitted)          # FIFO
    assert admitted == ids and finished == set(ids)
    assert all(done[i] == reqs[i - 1][1] for i in ids)
    assert q == [0, 0, 0, 0, 40]


def test_scheduler_releases_and_head_of_line(driver):
    """A large request at the head of the queue blocks smaller ones behind it
    until memory is released; releasing finished requests lets everything
    through, and the arena is empty at the end."""
    size = 1 << 20
    sess = Session(driver, size, 256, 8)
    cmds = ["sub 600000 50", "sub 600000 50", "sub 1000 50", "adm", "q",
            "plan 100", "adv", "poll", "rel 1", "adm", "q", "plan 100", "adv", "poll",
            "rel 2", "rel 3", "q", "rel 99"]
    out = sess.run(cmds)
    assert out[:3] == ["1", "2", "3"]
    assert _parse_ints(out[3])[:2] == [1, 1]               # only request 1 fits
    assert _parse_ints(out[4])[:3] == [2, 1, 1]            # 2 and 3 wait behind the head
    assert _parse_ints(out[5]) == [1, 1, 0, 50]
    assert _parse_ints(out[6]) == [1, 1]
    assert _parse_ints(out[7]) == [1, 1]
    assert out[8] == "0"                                   # request 1 held slot 0
    adm = _parse_ints(out[9])
    assert adm[0] == 2 and adm[1] == 2 and adm[4] == 3     # 2 then 3, FIFO
    assert _parse_ints(out[13]) == [2, 2, 3]
    q = _parse_ints(out[16])
    assert q[:4] == [0, 0, 0, 0]
    assert out[17] == "-2"


def _cut(driver, sizes, groups, r, quantum=0):
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    cmd = f"cut {len(sizes)} {groups} {r!r} {quantum} " + " ".join(map(str, off))
    line = Session(driver, 1024, 256, 1).run([cmd])[0]
    v = _parse_ints(line)
    assert v[0] == len(v) - 1
    return v[1:]


def _cut_model(sizes, groups, r, quantum=0):
    """The cut from its definition.  Weights r^min(g, G-1-g), r clamped to
    [1, 64].  Without a quantum, each cut at the instance boundary nearest
    its target point (the lower one on a tie) among those that leave every
    group an instance.  With a quantum q (and at least q per group): the
    first G//2 groups, forward, and the groups after the middle one,
    backward, each get at most the whole number of waves nearest their
    target (at least one), i.e. the farthest feasible boundary within it."""
    n = len(sizes)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(float)
    G = max(1, min(groups, n))
    r = min(max(r, 1.0), 64.0)
    w = [r ** min(g, G - 1 - g) for g in range(G)]
    target = [0.0] + [off[n] * sum(w[:g]) / sum(w) for g in range(1, G)]
    first = [0] * G + [n]
    if quantum == 0 or off[n] < quantum * G:
        for g in range(1, G):
            lo, hi = first[g - 1] + 1, n - (G - g)
            first[g] = min(range(lo, hi + 1), key=lambda i: (abs(off[i] - target[g]), i))
        return first
    h = G // 2
    for g in range(1, h + 1):
        lo, hi = first[g - 1] + 1, n - (G - g)
        start = off[first[g - 1]]
        t = start + max(1.0, np.floor((target[g] - start) / quantum + 0.5)) * quantum
        ok = [i for i in range(lo, hi + 1) if off[i] <= t]
        first[g] = max(ok) if ok else lo
    for g in range(G - 1, h, -1):
        lo, hi = first[h] + (g - h), first[g + 1] - 1
        end = off[first[g + 1]]
        t = end - max(1.0, np.floor((end - target[g]) / quantum + 0.5)) * quantum
        ok = [i for i in range(lo, hi + 1) if off[i] >= t]
        first[g] = min(ok) if ok else hi
    return first


def test_io_groups_taper(driver):
    """Equal groups at r = 1; the benchmark's FP64 taper (1, 7, 7, 1)/16 at
    r = 7; r clamped to [1, 64]; more groups than instances, and fewer than one."""
    assert _cut(driver, [5] * 12, 4, 1.0) == [0, 3, 6, 9, 12]
    assert _cut(driver, [1] * 16, 4, 7.0) == [0, 1, 8, 15, 16]
    assert _cut(driver, [1] * 130, 4, 1000.0) == [0, 1, 65, 129, 130]
    assert _cut(driver, [1] * 12, 4, 0.5) == [0, 3, 6, 9, 12]
    assert _cut(driver, [1] * 12, 4, -3.0) == [0, 3, 6, 9, 12]
    assert _cut(driver, [4, 9, 2], 7, 3.0) == [0, 1, 2, 3]
    assert _cut(driver, [4, 9, 2], 0, 3.0) == [0, 3]
    assert _cut(driver, [1] * 6, 5, 2.0) == [0, 1, 2, 4, 5, 6]


def test_io_groups_whole_waves(driver):
    """With a wave of 10 units: the edge groups and the first middle group
    get whole waves and the other middle group the fraction; a total below
    one wave per group falls back to the nearest boundaries."""
    assert _cut(driver, [1] * 100, 4, 7.0, 10) == [0, 10, 50, 90, 100]
    assert _cut(driver, [1] * 105, 4, 7.0, 10) == [0, 10, 50, 95, 105]
    assert _cut(driver, [3] * 35, 4, 7.0, 10) == [0, 3, 16, 32, 35]      # at most k waves each
    assert _cut(driver, [1] * 30, 4, 7.0, 10) == _cut(driver, [1] * 30, 4, 7.0)
    assert _cut(driver, [1] * 40, 2, 5.0, 10) == [0, 20, 40]            # two groups: halves
    assert _cut(driver, [1] * 40, 3, 5.0, 10) == [0, 10, 30, 40]
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_io_groups_matches_model(driver, seed):
    """Random instance sizes, group counts and ratios: contiguous non-empty
    groups covering every instance, each cut where the model puts it."""
    rng = np.random.default_rng(seed)
    for _ in range(40):
        n = int(rng.integers(1, 40))
        sizes = rng.integers(1, 100000, size=n).tolist()
        groups = int(rng.integers(1, 10))
        r = float(rng.uniform(0.5, 80.0))
        quantum = int(rng.choice([0, 1000, 50000, 200000]))
        got = _cut(driver, sizes, groups, r, quantum)
        assert got == _cut_model(sizes, groups, r, quantum), (sizes, groups, r, quantum)
        assert got[0] == 0 and got[-1] == n and all(a < b for a, b in zip(got, got[1:]))
