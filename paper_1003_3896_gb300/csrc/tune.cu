// tune.cu -- autotuner of the pair kernels' launch shape.
//
// The shape of one pair-force launch is (I, jt, b): I bodies per thread,
// which sets the width TILE * I of the i-block a work unit covers; jt, the
// j bodies of a unit (TILE, TILE / 2 or TILE / 4), which sets how many units
// a small cluster has; and b blocks per SM, which sets the grid G = b * SMs
// (at most the unit count) and so how finely the units are cut into
// per-block runs: up to the occupancy limit one resident wave, above it
// several waves of shorter runs.  The best shape depends on the arithmetic
// (registers per thread), on N (small clusters need more, smaller units to
// fill 152 SMs) and on the cluster mix of a batch, so it is measured rather
// than modelled: every variant the library has compiled is timed on the
// loaded state with CUDA events and the fastest is kept.
//
// Choices are remembered process-wide per workload shape (SM count,
// precision, cluster count, bodies, widest cluster in tiles), so every
// context or serving group of that shape starts from the tuned plan, and can
// be saved to / loaded from a text file so a tuned shape replays across runs.
// A shape changes where the j-sums are split between partial slots, so
// results of two shapes can differ at the rounding level (within the
// precision's tolerance); with one shape they are bit-reproducible.
#include <cstdio>
#include <initializer_list>
#include <map>
#include <mutex>
#include <tuple>

#include "engine.h"

namespace nb {

namespace {

using Key = std::tuple<int, int, int32_t, int64_t, int64_t>;
std::mutex g_mu;
std::map<Key, PairShape> g_table;

Key key_of(const TuneKey &k) { return Key(k.sms, k.precision, k.K, k.n, k.max_ntiles); }

bool shape_valid(int precision, const PairShape &s)
{
    return s.I > 0 && s.blocks_per_sm > 0 && s.jt >= 32 && s.jt <= TILE && TILE % s.jt == 0 &&
           pair_variant_exists(mode_of(precision), s.I);
}

}  // namespace

TuneKey tune_key(const Pool &P, const ClusterSet &C, int precision)
{
    TuneKey k;
    k.sms = P.num_sms;
    k.precision = precision;
    k.K = C.K;
    k.n = C.n;
    k.max_ntiles = C.max_ntiles;
    return k;
}

bool tune_lookup(const TuneKey &k, PairShape *out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_table.find(key_of(k));
    if (it == g_table.end()) return false;
    *out = it->second;
    return true;
}

void tune_store(const TuneKey &k, const PairShape &s)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_table[key_of(k)] = s;
}

void tune_clear()
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_table.clear();
}

int64_t tune_entries()
{
    std::lock_guard<std::mutex> lk(g_mu);
    return (int64_t)g_table.size();
}

int tune_save(const char *path)
{
    std::lock_guard<std::mutex> lk(g_mu);
    FILE *f = std::fopen(path, "w");
    if (!f) return set_error(NB_EINVAL, "cannot open %s for writing", path);
    std::fprintf(f, "nbsym-tune 2\n");
    for (const auto &e : g_table) {
        const Key &k = e.first;
        std::fprintf(f, "%d %d %d %lld %lld %d %d %d\n", std::get<0>(k), std::get<1>(k),
                     (int)std::get<2>(k), (long long)std::get<3>(k), (long long)std::get<4>(k),
                     e.second.I, e.second.jt, e.second.blocks_per_sm);
    }
    const bool ok = std::fclose(f) == 0;
    return ok ? NB_OK : set_error(NB_EINVAL, "writing %s failed", path);
}

int tune_load(const char *path, int64_t *loaded)
{
    FILE *f = std::fopen(path, "r");
    if (!f) return set_error(NB_EINVAL, "cannot open %s", path);
    int version = 0;
    if (std::fscanf(f, "nbsym-tune %d", &version) != 1 || version != 2) {
        std::fclose(f);
        return set_error(NB_EINVAL, "%s is not a tuning file of version 2", path);
    }
    int64_t count = 0;
    int sms, prec, K, I, jt, b;
    long long n, mt;
    std::map<Key, PairShape> add;
    for (;;) {
        const int r =
            std::fscanf(f, "%d %d %d %lld %lld %d %d %d", &sms, &prec, &K, &n, &mt, &I, &jt, &b);
        if (r == EOF) break;
        if (r != 8 || sms <= 0 || prec < NB_FP64 || prec > NB_DS_NEAR || K <= 0 || n <= 0 ||
            mt <= 0) {
            std::fclose(f);
            return set_error(NB_EINVAL, "%s: malformed entry %lld", path, (long long)count + 1);
        }
        PairShape s{I, b, jt};
        if (!shape_valid(prec, s)) {
            std::fclose(f);
            return set_error(NB_EINVAL, "%s: entry %lld names a shape this build lacks", path,
                             (long long)count + 1);
        }
        add[Key(sms, prec, K, n, mt)] = s;
        ++count;
    }
    std::fclose(f);
    std::lock_guard<std::mutex> lk(g_mu);
    for (const auto &e : add) g_table[e.first] = e.second;
    if (loaded) *loaded = count;
    return NB_OK;
}

// Mean time of one force evaluation with the given plan as a step runs it
// (*ms: the pair launch, with the mixed mode's near-pair pass beside it on
// the side stream), over reps evaluations after one untimed one, and of one
// kick that consumes its partial slots (*kick_ms).  Shapes are chosen by the
// sum: a grid of more blocks may win in the pair kernel and lose it again in
// the kick (more partial slots per i-block to sum), and a single resident
// wave has no slack for the near-pair pass's share of the SMs.  The kick
// reads and writes positions and velocities in the pool's staging buffer
// instead of the state and leaves the float planes alone, so the state is
// not touched.
static int time_plan(const Pool &P, const ClusterSet &C, const Plan &pl, const Phys &ph,
                     cudaStream_t st, int reps, cudaEvent_t e0, cudaEvent_t e1, double *ms,
                     double *kick_ms)
{
    int rc = enq_force(P, C, pl, ph, st, nullptr, nullptr, nullptr);
    if (rc) return rc;
    NB_TRY(cudaEventRecord(e0, st));
    for (int r = 0; r < reps && rc == NB_OK; ++r)
        rc = enq_force(P, C, pl, ph, st, nullptr, nullptr, nullptr);
    if (rc) return rc;
    NB_TRY(cudaEventRecord(e1, st));
    NB_TRY(cudaEventSynchronize(e1));
    float t = 0.f;
    NB_TRY(cudaEventElapsedTime(&t, e0, e1));
    *ms = t / reps;
    DevState so = view(P, C, pl);
    so.x = P.stage;
    so.y = P.stage + P.cap;
    so.z = P.stage + 2 * P.cap;
    so.vx = P.stage + 3 * P.cap;
    so.vy = P.stage + 4 * P.cap;
    so.vz = P.stage + 5 * P.cap;
    NB_TRY(launch_kick_drift(so, pl.pl.d, 1.0, 1.0, 1, 0, ph.ext, st));
    NB_TRY(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r)
        NB_TRY(launch_kick_drift(so, pl.pl.d, 1.0, 1.0, 1, 0, ph.ext, st));
    NB_TRY(cudaEventRecord(e1, st));
    NB_TRY(cudaEventSynchronize(e1));
    NB_TRY(cudaEventElapsedTime(&t, e0, e1));
    *kick_ms = t / reps;
    return NB_OK;
}

int tune_pair(const Pool &P, ClusterSet &C, int precision, const Phys &ph, cudaStream_t st,
              int reps, TuneReport &rep, Plan &out)
{
    if (reps < 1) reps = 1;
    const int mode = plan_mode(C, precision);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    NB_TRY(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return set_error(NB_ECUDA, "cudaEventCreate failed");
    }
    int rc = NB_OK;
    rep = TuneReport();
    rep.precision = precision;
    PairShape best{0, 0, 0};
    double best_ms = 0, best_cost = 0;   // evaluation time and cost of the best shape
    int64_t best_gw = 0;
    std::vector<int64_t> seen;   // (I, grid, jt) already timed
    do {
        // the shape the planner would pick without a tuned entry
        Plan def;
        rc = plan_make(P, C, precision, st, def, nullptr, /*use_table=*/false);
        if (rc) break;
        double def_kick = 0;
        rc = time_plan(P, C, def, ph, st, reps, e0, e1, &rep.default_ms, &def_kick);
        rep.default_cost_ms = rep.default_ms + def_kick;
        if (rc) break;
        const int Is[] = {1, 2, 4, 8};
        for (int I : Is) {
            if (!pair_variant_exists(mode, I)) continue;
            const int occ = pair_occupancy(mode, I);
            // finer j-ranges only pay when full-width units are scarce
            int64_t w_full = 0;
            for (int32_t k = 0; k < C.K; ++k)
                w_full += ((C.nk[k] + TILE * I - 1) / (TILE * I)) * ((C.nk[k] + TILE - 1) / TILE);
            const bool scarce = w_full < 2 * (int64_t)P.num_sms * occ;
            // grids of 1 to MAX_WAVES resident waves, and single waves a
            // little below the occupancy limit.  With the near-pair pass
            // beside the pair kernel only grids of DEFAULT_WAVES or more
            // waves: the side stream's blocks, resident first, leave a grid
            // of one or two waves unevenly placed over the SMs (some get
            // three of its blocks, some one), and such a kernel runs at the
            // pace of its most loaded SM (a one-wave grid of the 512-cluster
            // ensemble took 2.23 ms timed alone and 3.37 ms in the step
            // graph); later waves go to whichever SM frees a slot.
            const bool beside = mode == PM_DS_NEAR;
            int bs[8], nb = 0;
            for (int w : {MAX_WAVES, DEFAULT_WAVES, 2})
                if (!beside || w >= DEFAULT_WAVES) bs[nb++] = w * occ;
            for (int b = occ; !beside && b >= 1 && b > occ - 4; --b) bs[nb++] = b;
            for (int jt = TILE; rc == NB_OK && jt >= (scarce ? 32 : TILE); jt /= 2)
            for (int q = 0; q < nb; ++q) {
                const int b = bs[q];
                const PairShape s{I, b, jt};
                Plan pl;
                rc = plan_make(P, C, precision, st, pl, &s, false);
                if (rc) break;
                const int64_t tag = (pl.pl.d.G * 16 + I) * 256 + jt;
                bool dup = false;
                for (int64_t v : seen) dup = dup || v == tag;
                if (dup) continue;
                seen.push_back(tag);
                double ms = 0, kick = 0;
                rc = time_plan(P, C, pl, ph, st, reps, e0, e1, &ms, &kick);
                if (rc) break;
                ++rep.candidates;
                // cost: one force evaluation and one kick; within 0.2% the
                // shape with fewer blocks x i-block width (fewer partial
                // slots) wins
                const double cost = ms + kick;
                const double tie = 1.002;
                const int64_t gw = pl.pl.d.G * I;
                if (best.I == 0 || cost * (gw > best_gw ? tie : 1.0) <
                                       best_cost * (gw < best_gw ? tie : 1.0)) {
                    best = s;
                    best_ms = ms;
                    best_cost = cost;
                    best_gw = gw;
                    rep.grid = pl.pl.d.G;
                }
            }
            if (rc) break;
        }
        if (rc) break;
        if (best.I == 0) {
            rc = set_error(NB_ECUDA, "no pair-kernel shape could be timed");
            break;
        }
        rep.shape = best;
        rep.pair_ms = best_ms;
        rep.cost_ms = best_cost;
        tune_store(tune_key(P, C, precision), best);
        rc = plan_make(P, C, precision, st, out, &best, false);
    } while (0);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}

}  // namespace nb
