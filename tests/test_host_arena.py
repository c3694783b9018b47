"""Host logic of the pool: the arena allocator (csrc/lbm_arena.h) under a seeded random sequence
of allocations and releases, checked against a model that tracks every 256-byte block: live
allocations never overlap and stay inside the arena, the free byte count is the arena minus the
live bytes, every allocation is first-fit (the lowest free run long enough), a request that
fits nowhere is refused exactly when no free run is long enough, the free list holds exactly
the maximal free runs (fully coalesced), and releasing everything leaves one run.  No GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

PROGRAM = r"""
#include <stdint.h>
#include <stdio.h>
#include <vector>
#include "lbm_arena.h"

static uint64_t x = 0x9E3779B97F4A7C15ull;
static uint64_t rnd() { x ^= x << 13; x ^= x >> 7; x ^= x << 17; return x; }  // xorshift64

int main() {
    const size_t B = 256, NB = 4096;  // 4096 blocks of 256 bytes
    lbm::Arena a;
    a.init(nullptr, NB * B);
    std::vector<int> owner(NB, -1);   // model: which live allocation holds each block
    struct Live { size_t off, n; };
    std::vector<Live> live;
    for (int step = 0; step < 200000; ++step) {
        const bool do_alloc = live.empty() || rnd() % 100 < 55;
        if (do_alloc) {
            const size_t nb = 1 + (rnd() % 4 == 0 ? rnd() % 600 : rnd() % 40);
            // model first fit: the lowest start of a free run of >= nb blocks
            long want = -1;
            for (size_t i = 0, run = 0; i < NB; ++i) {
                run = owner[i] < 0 ? run + 1 : 0;
                if (run == nb) { want = long(i + 1 - nb); break; }
            }
            size_t off = 0;
            const bool ok = a.alloc(nb * B, &off);
            if (ok != (want >= 0)) { printf("step %d: alloc %zu blocks ok=%d model=%ld\n", step, nb, ok, want); return 1; }
            if (!ok) continue;
            if (off % B || off / B != size_t(want)) { printf("step %d: off %zu, first fit at %ld\n", step, off / B, want); return 1; }
            for (size_t i = off / B; i < off / B + nb; ++i) {
                if (i >= NB || owner[i] >= 0) { printf("step %d: overlap or out of range\n", step); return 1; }
                owner[i] = int(live.size());
            }
            live.push_back({off, nb * B});
        } else {
            const size_t k = rnd() % live.size();
            const Live l = live[k];
            a.release(l.off, l.n);
            for (size_t i = l.off / B; i < (l.off + l.n) / B; ++i) owner[i] = -1;
            live[k] = live.back();
            live.pop_back();
            for (size_t j = 0; j < live.size(); ++j)
                for (size_t i = live[j].off / B; i < (live[j].off + live[j].n) / B; ++i) owner[i] = int(j);
        }
        // the free list is exactly the maximal free runs of the model
        size_t used = 0;
        for (auto &l : live) used += l.n;
        if (a.free_bytes() != NB * B - used) { printf("step %d: free bytes\n", step); return 1; }
        auto it = a.free_.begin();
        for (size_t i = 0; i < NB;) {
            if (owner[i] >= 0) { ++i; continue; }
            size_t j = i;
            while (j < NB && owner[j] < 0) ++j;
            if (it == a.free_.end() || it->first != i * B || it->second != (j - i) * B) {
                printf("step %d: free run [%zu, %zu) not in the list as one entry\n", step, i, j);
                return 1;
            }
            ++it;
            i = j;
        }
        if (it != a.free_.end()) { printf("step %d: extra free-list entry\n", step); return 1; }
    }
    for (auto &l : live) a.release(l.off, l.n);
    if (a.free_.size() != 1 || a.free_.begin()->first != 0 || a.free_.begin()->second != NB * B) {
        printf("not one run after releasing everything\n");
        return 1;
    }
    printf("ok\n");
    return 0;
}
"""


def test_arena_first_fit_and_coalescing(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not found")
    src = tmp_path / "arena.cpp"
    src.write_text(PROGRAM)
    exe = tmp_path / "arena"
    r = subprocess.run([gxx, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_2002_02503_gb300", "csrc"),
                        str(src), "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
