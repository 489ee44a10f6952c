"""The stream-K work decomposition of the pair kernels (Decomp, make_decomp),
checked on the CPU against the library's own host code: a small host program
links libnbsym.so and exercises nb::make_decomp, Decomp::U and Decomp::owner,
with no GPU.

What must hold for every launch the planner can make:
* the blocks' unit runs [U(g), U(g+1)) are non-empty and tile [0, W) exactly,
  and owner(u) names the block whose run holds u;
* the 32-bit division path (taken when (W + 1)(G + 1) < 2^32) gives the same
  U and owner as the 64-bit one;
* no i-block's units are spread over more owner blocks than the decomposition's
  partial-slot count, which must not exceed the pool's slot capacity (unless
  the grid is one block): a violation would write past the slot planes.
Checked exhaustively for W, G <= 300, at the 32-bit boundary, and over
thousands of random ensembles and launch shapes, up to 2^19 - 1 clusters.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1003_3896_gb300")

SRC = r"""
#include <cstdio>
#include <cstdint>
#include <vector>
#include "nb_internal.cuh"

using namespace nb;

static uint64_t s_rng = 0x243F6A8885A308D3ull;
static uint64_t rnd() { s_rng ^= s_rng << 13; s_rng ^= s_rng >> 7; s_rng ^= s_rng << 17; return s_rng; }
static int64_t rnd_in(int64_t lo, int64_t hi) { return lo + (int64_t)(rnd() % (uint64_t)(hi - lo + 1)); }

static long long bad = 0;
#define CHECK(c, ...) do { if (!(c)) { if (bad < 10) { std::printf(__VA_ARGS__); std::printf("\n"); } ++bad; } } while (0)

// runs tile [0, W), each non-empty, owner consistent; narrow equals wide
static void check_runs(const Decomp &d, bool all_units)
{
    Decomp w = d;
    w.narrow = 0;
    CHECK(d.U(0) == 0 && d.U(d.G) == d.W, "U ends W=%lld G=%lld", (long long)d.W, (long long)d.G);
    const int64_t gstep = d.G > 4096 ? d.G / 4096 : 1;
    for (int64_t g = 0; g < d.G; g += gstep) {
        CHECK(d.U(g + 1) > d.U(g), "empty run g=%lld", (long long)g);
        CHECK(d.U(g) == w.U(g), "narrow U g=%lld", (long long)g);
    }
    auto one = [&](int64_t u) {
        const int64_t g = d.owner(u);
        CHECK(g >= 0 && g < d.G && d.U(g) <= u && u < d.U(g + 1),
              "owner u=%lld g=%lld W=%lld G=%lld", (long long)u, (long long)g, (long long)d.W,
              (long long)d.G);
        CHECK(g == w.owner(u), "narrow owner u=%lld", (long long)u);
    };
    if (all_units) {
        for (int64_t u = 0; u < d.W; ++u) one(u);
    } else {
        for (int k = 0; k < 20000; ++k) one(rnd_in(0, d.W - 1));
        for (int64_t u = 0; u < 64 && u < d.W; ++u) { one(u); one(d.W - 1 - u); }
    }
}

int main()
{
    long long cases = 0;
    // exhaustive small grids: every G for every W
    for (int64_t W = 1; W <= 300; ++W)
        for (int64_t G = 1; G <= W; ++G) {
            const Decomp d = make_decomp(W, 1, TILE, G, 1 << 20, TILE, 0);
            CHECK(d.G == G, "grid changed W=%lld G=%lld", (long long)W, (long long)G);
            check_runs(d, true);
            ++cases;
        }
    // around the 32-bit boundary of the narrow path
    for (int64_t W : {(1ll << 22) - 3, (1ll << 22) - 2, (1ll << 22) - 1, (1ll << 22), 65535ll,
                      65536ll, 65537ll, 3000000ll})
        for (int64_t G : {1ll, 2ll, 1023ll, 1024ll, 1025ll, 65535ll, 65536ll, 9120ll}) {
            if (G > W) continue;
            const Decomp d = make_decomp(W, 1, TILE, G, 1 << 20, TILE, 0);
            check_runs(d, false);
            ++cases;
        }
    // random ensembles and launch shapes, as the planner builds them
    long long narrow_seen = 0, wide_seen = 0, shrunk = 0;
    for (int trial = 0; trial < 4002; ++trial) {
        // two trials at the ensemble-size limit's scale: 65536 and 2^19 - 1
        // clusters of 1-100 bodies; the rest 1 or up to 600 clusters
        const int K = trial >= 4000 ? (trial == 4000 ? 65536 : (1 << 19) - 1)
                                    : (trial % 3 == 0 ? 1 : (int)rnd_in(1, 600));
        const int Is[4] = {1, 2, 4, 8};
        const int I = Is[rnd() % 4];
        const int ipb = TILE * I;
        const int jts[3] = {128, 64, 32};
        const int rows = (int)(rnd() % 5 == 0);
        const int jt = rows ? TILE : jts[rnd() % 3];
        std::vector<int64_t> nk(K), uoff(K + 1, 0);
        int64_t max_ntiles = 1;
        for (int k = 0; k < K; ++k) {
            nk[k] = K == 1 ? rnd_in(1, 1600000) : rnd_in(1, K > 600 ? 100 : 9000);
            const int64_t nt = (nk[k] + TILE - 1) / TILE;
            if (nt > max_ntiles) max_ntiles = nt;
        }
        Decomp probe;
        probe.jt = jt;
        probe.rows = rows;
        for (int k = 0; k < K; ++k) {
            const int64_t nt = (nk[k] + TILE - 1) / TILE;
            const int64_t ib = (nk[k] + ipb - 1) / ipb;
            uoff[k + 1] = uoff[k] + ib * probe.units_per_iblock(nt);
        }
        const int64_t W = uoff[K];
        const int64_t slot_cap = rnd() % 4 == 0 ? rnd_in(2, 8) : 64;
        const int64_t G = rnd_in(1, 152 * 6 * 8);
        const Decomp d = make_decomp(W, max_ntiles, ipb, G, slot_cap, jt, rows);
        CHECK(d.G >= 1 && d.G <= d.W, "grid out of range");
        CHECK(d.slots <= slot_cap || d.G == 1, "slots %lld > cap %lld", (long long)d.slots,
              (long long)slot_cap);
        if (d.G < (G < W ? G : W)) ++shrunk;
        if (d.narrow) ++narrow_seen; else ++wide_seen;
        check_runs(d, d.W <= 20000);
        // every i-block of every cluster: owner blocks of its unit span
        for (int k = 0; k < K; ++k) {
            const int64_t nt = d.units_per_iblock((nk[k] + TILE - 1) / TILE);
            const int64_t ib = (nk[k] + ipb - 1) / ipb;
            for (int64_t b = 0; b < ib; ++b) {
                const int64_t u0 = uoff[k] + b * nt;
                const int64_t first = d.owner(u0);
                const int64_t count = d.owner(u0 + nt - 1) - first + 1;
                CHECK(count >= 1 && count <= d.slots, "i-block k=%d b=%lld spans %lld blocks > slots %lld",
                      k, (long long)b, (long long)count, (long long)d.slots);
            }
        }
        ++cases;
    }
    std::printf("cases %lld narrow %lld wide %lld shrunk %lld failures %lld\n", cases, narrow_seen,
                wide_seen, shrunk, bad);
    return bad ? 1 : 0;
}
"""


def test_decomposition_tiles_units_and_bounds_slots(tmp_path):
    from paper_1003_3896_gb300 import build
    lib = build.build()
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = tmp_path / "decomp_check.cu"
    src.write_text(SRC)
    exe = tmp_path / "decomp_check"
    subprocess.run([nvcc, *build.ARCH, "-O2", "-std=c++17", "-I", os.path.join(PKG, "csrc"),
                    str(src), "-o", str(exe), "-L", os.path.dirname(lib), "-lnbsym",
                    "-Xlinker", "-rpath=" + os.path.dirname(lib)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "failures 0" in r.stdout
    # both division paths and the grid-shrinking loop were exercised
    fields = dict(zip(r.stdout.split()[0::2], r.stdout.split()[1::2]))
    assert int(fields["narrow"]) > 0 and int(fields["wide"]) > 0 and int(fields["shrunk"]) > 0
