"""The server's device-memory bookkeeping (csrc/pool.h, host C++ only),
compiled on its own with g++ and driven through random allocate/free
sequences against a brute-force byte map."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <cstdio>
#include <cstdlib>
#include <vector>
#include "pool.h"
int main() {
    const uint64_t cap = 1 << 16, align = 64;
    huff::RegionAllocator a(cap, align);
    std::vector<int> owner(cap, -1);               // brute-force map: byte -> live block id
    struct B { uint64_t off, bytes; bool live; };
    std::vector<B> blocks;
    srand(12345);
    for (int step = 0; step < 200000; step++) {
        bool do_alloc = blocks.empty() || rand() % 3 != 0;
        if (do_alloc) {
            uint64_t bytes = 1 + rand() % 3000;
            uint64_t off;
            bool ok = a.alloc(bytes, &off);
            uint64_t need = (bytes + align - 1) / align * align;
            // brute force: is there an aligned free run of `need` bytes at a lower offset?
            uint64_t first = cap;
            for (uint64_t o = 0; o + need <= cap; o += align) {
                bool fr = true;
                for (uint64_t k = o; k < o + need; k += align) if (owner[k] != -1) { fr = false; break; }
                if (fr) { first = o; break; }
            }
            if (ok != (first != cap)) { printf("alloc success mismatch at %d\n", step); return 1; }
            if (ok) {
                if (off != first) { printf("not first fit at %d: %llu vs %llu\n", step, (unsigned long long)off, (unsigned long long)first); return 1; }
                if (off % align) return 2;
                for (uint64_t k = off; k < off + need; k++) { if (owner[k] != -1) return 3; owner[k] = (int)blocks.size(); }
                blocks.push_back({off, bytes, true});
            }
        } else {
            size_t i = rand() % blocks.size();
            if (!blocks[i].live) continue;
            uint64_t need = (blocks[i].bytes + align - 1) / align * align;
            a.release(blocks[i].off, blocks[i].bytes);
            for (uint64_t k = blocks[i].off; k < blocks[i].off + need; k++) owner[k] = -1;
            blocks[i].live = false;
        }
        uint64_t used = 0;
        for (auto &b : blocks) if (b.live) used += (b.bytes + align - 1) / align * align;
        if (used != a.used()) { printf("used mismatch\n"); return 4; }
        if (a.peak() < a.used() || a.peak() > cap) return 5;
    }
    for (auto &b : blocks) if (b.live) a.release(b.off, b.bytes);
    if (a.used() != 0 || a.free_blocks() != 1 || a.largest_free() != cap) { printf("not coalesced\n"); return 6; }
    printf("ok\n");
    return 0;
}
"""


def test_region_allocator_against_brute_force():
    gxx = shutil.which("g++")
    if not gxx:
        pytest.skip("no g++")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "t.cpp")
        exe = os.path.join(d, "t")
        open(src, "w").write(PROGRAM)
        subprocess.run([gxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2010_10039_gb300", "csrc"),
                        src, "-o", exe], check=True)
        r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
        assert r.returncode == 0, r.stdout + r.stderr
        assert r.stdout.strip() == "ok"
