"""The serving loop's first-fit allocator of state-pool ranges
(csrc/range_alloc.h), compiled on its own with the host C++ compiler and
driven through random admit / retire sequences against a slot-by-slot model
of the pool: every range it returns is free and is the lowest-addressed free
run that fits, it refuses only when no free run fits, and its free list stays
equal to the model's free runs (coalesced, nothing lost or leaked)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1003_3896_gb300", "csrc")

SRC = r"""
#include <cstdio>
#include <cstdint>
#include <vector>
#include <utility>
#include "range_alloc.h"

static uint64_t s_rng = 0x9E3779B97F4A7C15ull;
static uint64_t rnd() { s_rng ^= s_rng << 13; s_rng ^= s_rng >> 7; s_rng ^= s_rng << 17; return s_rng; }

static long long bad = 0;
#define CHECK(c, ...) do { if (!(c)) { if (bad < 10) { std::printf(__VA_ARGS__); std::printf("\n"); } ++bad; } } while (0)

// free runs of the model, in address order
static std::vector<std::pair<int64_t, int64_t>> runs(const std::vector<char> &used)
{
    std::vector<std::pair<int64_t, int64_t>> r;
    const int64_t cap = (int64_t)used.size();
    for (int64_t i = 0; i < cap;) {
        if (used[i]) { ++i; continue; }
        int64_t j = i;
        while (j < cap && !used[j]) ++j;
        r.push_back({i, j - i});
        i = j;
    }
    return r;
}

int main()
{
    long long allocs = 0, refusals = 0, releases = 0;
    for (int trial = 0; trial < 300; ++trial) {
        const int64_t cap = 1 + (int64_t)(rnd() % 4000);
        nb::RangeAlloc ra(cap);
        std::vector<char> used(cap, 0);
        std::vector<std::pair<int64_t, int64_t>> live;
        for (int op = 0; op < 400; ++op) {
            if (live.empty() || rnd() % 100 < 55) {
                // jobs of very uneven size, as in the serving trace
                const int64_t n = 1 + (int64_t)(rnd() % (rnd() % 4 == 0 ? cap : 1 + cap / 16));
                const auto fr = runs(used);
                int64_t want = -1;
                for (auto &f : fr)
                    if (f.second >= n) { want = f.first; break; }
                const int64_t off = ra.alloc(n);
                CHECK(off == want, "alloc(%lld) gave %lld, first fit %lld", (long long)n,
                      (long long)off, (long long)want);
                if (off >= 0) {
                    for (int64_t i = off; i < off + n; ++i) {
                        CHECK(!used[i], "slot %lld handed out twice", (long long)i);
                        used[i] = 1;
                    }
                    live.push_back({off, n});
                    ++allocs;
                } else {
                    ++refusals;
                }
            } else {
                const size_t k = rnd() % live.size();
                const auto r = live[k];
                live[k] = live.back();
                live.pop_back();
                ra.release(r.first, r.second);
                for (int64_t i = r.first; i < r.first + r.second; ++i) used[i] = 0;
                ++releases;
            }
            // the allocator's free list is exactly the model's free runs
            const auto fr = runs(used);
            CHECK(ra.free_.size() == fr.size(), "free list has %zu runs, model %zu",
                  ra.free_.size(), fr.size());
            size_t q = 0;
            for (auto &e : ra.free_) {
                if (q < fr.size())
                    CHECK(e.first == fr[q].first && e.second == fr[q].second,
                          "free run [%lld, +%lld) vs model [%lld, +%lld)", (long long)e.first,
                          (long long)e.second, (long long)fr[q].first, (long long)fr[q].second);
                ++q;
            }
        }
        // retire everything: one free run of the whole pool again
        for (auto &r : live) ra.release(r.first, r.second);
        CHECK(ra.free_.size() == 1 && ra.free_.begin()->first == 0 &&
              ra.free_.begin()->second == cap, "pool not whole after retiring all jobs");
    }
    nb::RangeAlloc empty(0);
    CHECK(empty.alloc(1) == -1, "empty pool handed out a range");
    std::printf("allocs %lld refusals %lld releases %lld failures %lld\n", allocs, refusals,
                releases, bad);
    return bad ? 1 : 0;
}
"""


def test_first_fit_against_a_model_of_the_pool(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "range_alloc_check.cpp"
    src.write_text(SRC)
    exe = tmp_path / "range_alloc_check"
    subprocess.run([cxx, "-std=c++17", "-O2", "-I", CSRC, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures 0" in r.stdout
    fields = dict(zip(r.stdout.split()[0::2], r.stdout.split()[1::2]))
    assert int(fields["allocs"]) > 0 and int(fields["refusals"]) > 0 and int(fields["releases"]) > 0
