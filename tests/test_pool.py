"""The serving loop's request-scratch allocator (csrc/pool.h, host-only C++) on the CPU.

A small driver compiled with g++ replays random allocate/release sequences; every answer must equal a
first-fit model written here (sizes rounded up to 256 bytes, lowest-offset hole that fits, freed
neighbours merged).  Also checked: live blocks never overlap and stay inside the range, the used count
is the sum of the live blocks, and releasing everything leaves one hole covering the range.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
DRIVER = r"""
#include <cstdio>
#include <cstring>
#include "pool.h"
int main() {
    fh::Pool p;
    unsigned long long bytes;
    if (scanf("%llu", &bytes) != 1) return 2;
    p.init(nullptr, bytes);
    char op[8];
    unsigned long long a, b;
    while (scanf("%7s", op) == 1) {
        if (!strcmp(op, "A")) {
            if (scanf("%llu", &a) != 1) return 2;
            uint64_t off = 0;
            bool ok = p.alloc(a, &off);
            printf("%d %llu %llu\n", ok ? 1 : 0, ok ? (unsigned long long)off : 0ull, (unsigned long long)p.used);
        } else {
            if (scanf("%llu %llu", &a, &b) != 2) return 2;
            p.release(a, b);
            printf("R %llu %zu\n", (unsigned long long)p.used, p.free_.size());
        }
    }
    printf("F");
    for (auto& kv : p.free_) printf(" %llu:%llu", (unsigned long long)kv.first, (unsigned long long)kv.second);
    printf("\n");
    return 0;
}
"""


class FirstFit:
    def __init__(self, n):
        self.free = [[0, n]] if n else []
        self.used = 0

    def alloc(self, n):
        n = (n + 255) // 256 * 256
        for i, (o, s) in enumerate(self.free):
            if s >= n:
                if s == n:
                    self.free.pop(i)
                else:
                    self.free[i] = [o + n, s - n]
                self.used += n
                return o
        return None

    def release(self, o, n):
        n = (n + 255) // 256 * 256
        self.used -= n
        self.free.append([o, n])
        self.free.sort()
        merged = []
        for o2, s2 in self.free:
            if merged and merged[-1][0] + merged[-1][1] == o2:
                merged[-1][1] += s2
            else:
                merged.append([o2, s2])
        self.free = merged


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no g++")
    d = tmp_path_factory.mktemp("pool")
    src = d / "pool_driver.cpp"
    src.write_text(DRIVER)
    exe = d / "pool_driver"
    subprocess.check_call([gxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "paper_2507_03836_gb300", "csrc"),
                           str(src), "-o", str(exe)])
    return str(exe)


@pytest.mark.parametrize("seed", range(6))
def test_first_fit_against_model(driver, seed):
    rs = np.random.default_rng(seed)
    total = int(rs.integers(1, 64)) * 4096 + int(rs.integers(0, 4)) * 256
    model = FirstFit(total)
    live = {}
    ops, expect = [], []
    for _ in range(400):
        if live and rs.random() < 0.45:
            k = list(live)[int(rs.integers(0, len(live)))]
            o, n = live.pop(k)
            model.release(o, n)
            ops.append("R %d %d" % (o, n))
            expect.append(("R", model.used, len(model.free)))
        else:
            n = int(rs.integers(1, total // 4 + 2))
            o = model.alloc(n)
            ops.append("A %d" % n)
            if o is None:
                expect.append((0, 0, model.used))
            else:
                live[len(ops)] = (o, n)
                expect.append((1, o, model.used))
    for o, n in list(live.values()):  # release everything at the end
        model.release(o, n)
        ops.append("R %d %d" % (o, n))
        expect.append(("R", model.used, len(model.free)))
    out = subprocess.run([driver], input="%d\n%s\n" % (total, "\n".join(ops)), capture_output=True, text=True,
                         check=True).stdout.split("\n")
    for line, want in zip(out, expect):
        f = line.split()
        got = ("R", int(f[1]), int(f[2])) if f[0] == "R" else (int(f[0]), int(f[1]), int(f[2]))
        assert got == want, (line, want)
    assert model.used == 0 and model.free == [[0, total]]
    assert out[len(expect)] == "F 0:%d" % total


def test_live_blocks_are_disjoint(driver):
    rs = np.random.default_rng(99)
    total = 1 << 20
    ops, sizes = [], []
    for _ in range(300):
        n = int(rs.integers(1, 20000))
        ops.append("A %d" % n)
        sizes.append((n + 255) // 256 * 256)
    out = subprocess.run([driver], input="%d\n%s\n" % (total, "\n".join(ops)), capture_output=True, text=True,
                         check=True).stdout.split("\n")
    blocks, used = [], 0
    for line, s in zip(out, sizes):
        ok, off, u = (int(x) for x in line.split())
        if ok:
            blocks.append((off, off + s))
            used += s
        assert u == used
    blocks.sort()
    assert all(a[1] <= b[0] for a, b in zip(blocks, blocks[1:])) and blocks[-1][1] <= total
