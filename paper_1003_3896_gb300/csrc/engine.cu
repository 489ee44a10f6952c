// engine.cu -- state pool, cluster-set tables, launch plans and the enqueue
// functions shared by the context API and the serving loop.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "engine.h"

namespace nb {

namespace {
thread_local std::string g_err;
}

int set_error(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

const char *last_error() { return g_err.c_str(); }

// ---- pool --------------------------------------------------------------------

int64_t part_elems_for(const Pool &P, int64_t n)
{
    const int64_t giw = (int64_t)P.num_sms * MAX_WAVES * 3072;
    const int64_t slots_n = giw + 2 * n, cap_n = MAX_PART_SLOTS * n;
    return 3 * (slots_n < cap_n ? slots_n : cap_n);
}

int pool_create(Pool &P, int device, int64_t cap, bool own_part)
{
    P.device = device;
    P.cap = cap;
    if (cudaDeviceGetAttribute(&P.num_sms, cudaDevAttrMultiProcessorCount, device) !=
        cudaSuccess)
        return set_error(NB_ECUDA, "cudaDeviceGetAttribute failed");
    DevState &s = P.s;
    s.cap = cap;
    // partial sums: a set of n bodies needs about G * ipb / n + 2 slots per
    // body, where G * ipb <= SMs * MAX_WAVES * (resident blocks * i-block
    // width) and the last factor is at most 3072 for every compiled variant
    // (8 x 256, 6 x 512, 3 x 1024).  The planes are laid out per set (stride
    // n, linear body index), so 3 (giw + 2 cap) doubles give a set of n
    // bodies (giw + 2 cap) / n slots: a small set in a large pool (a serving
    // group) gets as many as a context of its own size.  make_decomp
    // shrinks a grid that would need more than a set has.  Sets that run
    // concurrently in one pool (the serving loop's groups) cannot share this
    // storage: such a pool has none, and each set reserves its own.
    s.part_elems = own_part ? part_elems_for(P, cap) : 0;
    s.part_slots = 0;
    s.pstride = 0;
    s.red_len = 0;
    bool ok = true;
    auto A = [&](void **q, size_t bytes) {
        if (ok && cudaMalloc(q, bytes) != cudaSuccess) {
            *q = nullptr;
            ok = false;
        }
    };
    const size_t c8 = (size_t)cap * 8, c4 = (size_t)cap * 4;
    A((void **)&s.x, c8); A((void **)&s.y, c8); A((void **)&s.z, c8);
    A((void **)&s.vx, c8); A((void **)&s.vy, c8); A((void **)&s.vz, c8); A((void **)&s.m, c8);
    A((void **)&s.xh, c4); A((void **)&s.yh, c4); A((void **)&s.zh, c4); A((void **)&s.mf, c4);
    A((void **)&s.xl, c4); A((void **)&s.yl, c4); A((void **)&s.zl, c4);
    A((void **)&s.jd, 2 * (size_t)cap * sizeof(float4));
    A((void **)&s.jl, 2 * (size_t)cap * sizeof(float4));
    if (s.part_elems > 0) A((void **)&s.part, (size_t)s.part_elems * 8);
    A((void **)&s.corr, 3 * c8);
    A((void **)&P.stage, 7 * c8);
    if (!ok) {
        cudaGetLastError();
        pool_destroy(P);
        return set_error(NB_ENOMEM, "device allocation failed for %lld bodies",
                         (long long)cap);
    }
    return NB_OK;
}

void pool_destroy(Pool &P)
{
    DevState &s = P.s;
    void *ptrs[] = {s.x,  s.y,  s.z,  s.vx, s.vy, s.vz, s.m,    s.xh,    s.yh,
                    s.zh, s.mf, s.xl, s.yl, s.zl, s.jd, s.jl, s.part, s.corr, P.stage};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    s = DevState();
    P.stage = nullptr;
    P.cap = 0;
}

// ---- cluster sets ------------------------------------------------------------

namespace {
inline size_t al(size_t b) { return (b + 255) / 256 * 256; }
}

int set_create(ClusterSet &C, int32_t kcap, int64_t body_cap, int priority)
{
    C.kcap = kcap;
    C.scap = (body_cap + SEG_BODIES - 1) / SEG_BODIES + kcap;
    const size_t k8 = (size_t)kcap * 8, k81 = (size_t)(kcap + 1) * 8;
    const size_t bytes = al(k8) * 2 + al(k81) * 3 + al((size_t)kcap * 4) * 2 + al(k8) * 2 +
                         al((size_t)C.scap * 4) + al((size_t)C.scap * 8) * 2 +
                         al((size_t)(kcap + 1) * 4) + al((size_t)kcap * sizeof(Frame)) +
                         al((size_t)kcap * DIAG_STRIDE * 8) + al(k8);
    if (cudaMalloc(&C.dmem, bytes) != cudaSuccess) {
        cudaGetLastError();
        C.dmem = nullptr;
        return set_error(NB_ENOMEM, "cluster tables: device allocation failed");
    }
    // reduction partials (one row of 16 doubles per segment), the near-pair
    // cell table and body copies, and the non-finite flag
    C.body_cap = body_cap;
    C.ng_hcap = near_table_size(body_cap);
    bool ok = true;
    auto A = [&](void **q, size_t b) {
        if (ok && cudaMalloc(q, b) != cudaSuccess) {
            *q = nullptr;
            ok = false;
        }
    };
    A((void **)&C.red, (size_t)C.scap * 16 * 8);
    A((void **)&C.ng_bucket, (size_t)body_cap * 4);
    A((void **)&C.ng_entry, (size_t)body_cap * 4);
    A((void **)&C.ng_rank, (size_t)body_cap * 4);
    A((void **)&C.ng_total, sizeof(int));
    A((void **)&C.flag, sizeof(int));
    A((void **)&C.cid, (size_t)body_cap * 4);
    A((void **)&C.ng_spos, (size_t)body_cap * 16);
    A((void **)&C.ng_slo, (size_t)body_cap * 16);
    A((void **)&C.ng_slot, (size_t)C.ng_hcap * sizeof(NgSlot));
    if (!ok) {
        cudaGetLastError();
        set_destroy(C);
        return set_error(NB_ENOMEM, "cluster tables: device allocation failed");
    }
    if (cudaStreamCreateWithPriority(&C.side, cudaStreamNonBlocking, priority) != cudaSuccess ||
        cudaEventCreateWithFlags(&C.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&C.join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        set_destroy(C);
        return set_error(NB_ECUDA, "cluster tables: stream or event creation failed");
    }
    cudaMemset(C.dmem, 0, bytes);
    return NB_OK;
}

int set_reserve_part(ClusterSet &C, int64_t elems, cudaStream_t st)
{
    if (C.part && C.part_elems >= elems) return NB_OK;
    const int64_t want = C.part ? (elems > C.part_elems * 3 / 2 ? elems : C.part_elems * 3 / 2)
                                : elems;
    if (C.part) {
        NB_TRY(cudaFreeAsync(C.part, st));
        C.part = nullptr;
        C.part_elems = 0;
    }
    void *q = nullptr;
    if (cudaMallocAsync(&q, (size_t)want * 8, st) != cudaSuccess) {
        cudaGetLastError();
        return set_error(NB_ENOMEM, "partial-sum storage: %lld bytes not available",
                         (long long)want * 8);
    }
    C.part = static_cast<double *>(q);
    C.part_elems = want;
    return NB_OK;
}

void set_destroy(ClusterSet &C)
{
    void *ptrs[] = {C.dmem,    C.red,   C.ng_bucket, C.ng_entry, C.ng_total, C.flag,
                    C.cid,     C.ng_spos, C.ng_slo,  C.ng_slot,  C.ng_rank};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (C.part) cudaFree(C.part);
    if (C.fork) cudaEventDestroy(C.fork);
    if (C.join) cudaEventDestroy(C.join);
    if (C.side) cudaStreamDestroy(C.side);
    C = ClusterSet();
}

int set_define(ClusterSet &C, int32_t K, const int64_t *boff, const int64_t *nk,
               const double *eps, const double *dts)
{
    if (K < 1 || K > C.kcap) return set_error(NB_EINVAL, "cluster count %d outside [1, %d]", K, C.kcap);
    C.K = K;
    C.boff.assign(boff, boff + K);
    C.nk.assign(nk, nk + K);
    C.eps.assign(K, 0.0);
    C.dts.assign(K, 1.0);
    C.noff.assign(K + 1, 0);
    for (int32_t k = 0; k < K; ++k) {
        if (nk[k] < 1) return set_error(NB_EINVAL, "cluster %d has no bodies", k);
        C.eps[k] = eps ? eps[k] : 0.0;
        if (dts) C.dts[k] = dts[k];
        C.noff[k + 1] = C.noff[k] + nk[k];
    }
    C.n = C.noff[K];
    // widest cluster in j-tiles (independent of the i-block width; part of
    // the tuned-shape key, so known before the layout)
    C.max_ntiles = 0;
    for (int32_t k = 0; k < K; ++k) {
        const int64_t nt = (C.nk[k] + TILE - 1) / TILE;
        if (nt > C.max_ntiles) C.max_ntiles = nt;
    }
    C.eps2d.resize(K);
    C.eps2f.resize(K);
    for (int32_t k = 0; k < K; ++k) {
        C.eps2d[k] = C.eps[k] * C.eps[k];
        C.eps2f[k] = (float)C.eps2d[k];
    }
    C.ipb = 0;   // layout pending
    return NB_OK;
}

int set_layout(ClusterSet &C, int ipb, cudaStream_t st, int jt)
{
    if (jt < 32 || jt > TILE || TILE % jt != 0)
        return set_error(NB_EINVAL, "j-range width %d must divide %d and be >= 32", jt, TILE);
    const int64_t per_tile = TILE / jt;
    const int32_t K = C.K;
    C.ipb = ipb;
    C.ntiles.resize(K);
    C.uoff.assign(K + 1, 0);
    C.uoff_pot.assign(K + 1, 0);
    C.max_ntiles = 0;
    C.seg_off.assign(K + 1, 0);
    C.seg_k.clear();
    C.seg_lo.clear();
    C.seg_hi.clear();
    for (int32_t k = 0; k < K; ++k) {
        const int64_t nt = (C.nk[k] + TILE - 1) / TILE;
        C.ntiles[k] = (int32_t)nt;
        if (nt > C.max_ntiles) C.max_ntiles = nt;
        C.uoff[k + 1] = C.uoff[k] + ((C.nk[k] + ipb - 1) / ipb) * nt * per_tile;
        C.uoff_pot[k + 1] = C.uoff_pot[k] + nt * nt;
        for (int64_t lo = C.noff[k]; lo < C.noff[k + 1]; lo += SEG_BODIES) {
            C.seg_k.push_back(k);
            C.seg_lo.push_back(lo);
            C.seg_hi.push_back(lo + SEG_BODIES < C.noff[k + 1] ? lo + SEG_BODIES : C.noff[k + 1]);
        }
        C.seg_off[k + 1] = (int32_t)C.seg_k.size();
    }
    const int64_t S = (int64_t)C.seg_k.size();
    if (S > C.scap) return set_error(NB_EINVAL, "too many reduction segments");
    // device layout (must match set_create's size computation)
    const size_t k8 = (size_t)C.kcap * 8, k81 = (size_t)(C.kcap + 1) * 8;
    char *p = C.dmem;
    auto take = [&](size_t bytes) {
        char *q = p;
        p += al(bytes);
        return q;
    };
    int64_t *d_boff = (int64_t *)take(k8);
    int64_t *d_nk = (int64_t *)take(k8);
    int64_t *d_noff = (int64_t *)take(k81);
    int64_t *d_uoff = (int64_t *)take(k81);
    int64_t *d_uoffp = (int64_t *)take(k81);
    int32_t *d_ntiles = (int32_t *)take((size_t)C.kcap * 4);
    float *d_eps2f = (float *)take((size_t)C.kcap * 4);
    double *d_eps2d = (double *)take(k8);
    double *d_dts = (double *)take(k8);
    int32_t *d_segk = (int32_t *)take((size_t)C.scap * 4);
    int64_t *d_seglo = (int64_t *)take((size_t)C.scap * 8);
    int64_t *d_seghi = (int64_t *)take((size_t)C.scap * 8);
    int32_t *d_segoff = (int32_t *)take((size_t)(C.kcap + 1) * 4);
    C.frame = (Frame *)take((size_t)C.kcap * sizeof(Frame));
    C.diag = (double *)take((size_t)C.kcap * DIAG_STRIDE * 8);
    double *d_mu = (double *)take(k8);
    if ((int32_t)C.mu.size() != K) C.mu.assign(K, 0.0);
    auto up = [&](void *dst, const void *src, size_t bytes) {
        return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st)
                     : cudaSuccess;
    };
    NB_TRY(up(d_boff, C.boff.data(), K * 8));
    NB_TRY(up(d_nk, C.nk.data(), K * 8));
    NB_TRY(up(d_noff, C.noff.data(), (K + 1) * 8));
    NB_TRY(up(d_uoff, C.uoff.data(), (K + 1) * 8));
    NB_TRY(up(d_uoffp, C.uoff_pot.data(), (K + 1) * 8));
    NB_TRY(up(d_ntiles, C.ntiles.data(), K * 4));
    NB_TRY(up(d_eps2f, C.eps2f.data(), K * 4));
    NB_TRY(up(d_eps2d, C.eps2d.data(), K * 8));
    NB_TRY(up(d_dts, C.dts.data(), K * 8));
    NB_TRY(up(d_mu, C.mu.data(), K * 8));
    NB_TRY(up(d_segk, C.seg_k.data(), S * 4));
    NB_TRY(up(d_seglo, C.seg_lo.data(), S * 8));
    NB_TRY(up(d_seghi, C.seg_hi.data(), S * 8));
    NB_TRY(up(d_segoff, C.seg_off.data(), (K + 1) * 4));
    Clusters &c = C.cl;
    c.K = K;
    c.boff = d_boff;
    c.nk = d_nk;
    c.noff = d_noff;
    c.uoff = d_uoff;
    c.ntiles = d_ntiles;
    c.eps2f = d_eps2f;
    c.eps2d = d_eps2d;
    c.dts = d_dts;
    c.mu = d_mu;
    c.frame = C.frame;
    c.S = (int32_t)S;
    c.seg_k = d_segk;
    c.seg_lo = d_seglo;
    c.seg_hi = d_seghi;
    c.seg_off = d_segoff;
    c.cid = C.cid;
    if (K > 1) NB_TRY(launch_cluster_map(c, C.cid, C.n, st));
    // pageable copies are staged before returning; make the tables visible
    // to kernels launched on other streams too
    NB_TRY(cudaStreamSynchronize(st));
    C.cl_pot = c;
    C.cl_pot.uoff = d_uoffp;
    return NB_OK;
}

// ---- plans -------------------------------------------------------------------

bool sp_family(int mode) { return mode == PM_DS_NEAR || mode == PM_DS_FULL || mode == PM_FP32; }

int mode_of(int precision)
{
    switch (precision) {
    case NB_FP64: return PM_FP64;
    case NB_FP32: return PM_FP32;
    case NB_DS_FULL: return PM_DS_FULL;
    case NB_DD: return PM_DD;
    default: return PM_DS_NEAR;
    }
}

bool float_planes(int precision) { return precision != NB_FP64; }

// Launch order of the pair kernel's blocks over set C: largest estimated work
// first, so that the blocks handed out last, which set the kernel's tail
// when the grid runs in waves, are the cheap ones (longest-processing-time
// first).  A unit's work is its j count (the cluster's last j-tile clipped
// to its bodies rounded up to 32) times the packed i-pairs its i-block
// evaluates per warp (sp: the pairs holding bodies; the float-float kernel
// evaluates all of them), each warp's pairs plus half a pair for its share
// of the j-stream loads; each segment (a run of one i-block's units) adds
// the cost of 16 j of a full i-block for its set-up and write-out.  Only the
// order depends on these estimates: any order gives the same sums.
void block_order(ClusterSet &C, const Decomp &d, int I, bool partial)
{
    const int64_t G = d.G;
    const double full = (TILE / 32) * (I / 2 + 0.5);
    std::vector<double> cost((size_t)G, 0.0);
    for (int64_t g = 0; g < G; ++g) {
        int64_t u = d.U(g);
        const int64_t uend = d.U(g + 1);
        double c = 0.0;
        while (u < uend) {
            const int32_t k = (int32_t)(std::upper_bound(C.uoff.begin(),
                                                         C.uoff.begin() + C.K + 1, u) -
                                        C.uoff.begin()) - 1;
            const int64_t nt = d.units_per_iblock(C.ntiles[k]);
            const int64_t lu = u - C.uoff[k];
            const int64_t rb = lu / nt, t0 = lu - rb * nt;
            const int64_t t1 = std::min(nt, t0 + (uend - u));
            const int64_t n = C.nk[k], ib0 = rb * d.ipb;
            double act = full;
            if (partial) {
                act = 0.0;
                for (int w = 0; w < TILE / 32; ++w) {
                    const int64_t lw = ib0 + 32 * w;
                    int64_t kmax = n > lw ? (n - lw + TILE - 1) / TILE : 0;
                    if (kmax > I) kmax = I;
                    if (kmax > 0) act += (kmax + 1) / 2 + 0.5;
                }
            }
            const int64_t jend = (n + 31) / 32 * 32;
            const int64_t j0 = t0 * d.jt, j1 = std::min(t1 * d.jt, jend);
            if (j1 > j0) c += act * (double)(j1 - j0);
            c += 16.0 * full;
            u += t1 - t0;
        }
        cost[(size_t)g] = c;
    }
    std::vector<int64_t> idx((size_t)G);
    for (int64_t g = 0; g < G; ++g) idx[(size_t)g] = g;
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int64_t a, int64_t b) { return cost[(size_t)a] > cost[(size_t)b]; });
    C.bperm.resize((size_t)G);
    for (int64_t q = 0; q < G; ++q) C.bperm[(size_t)q] = (uint16_t)idx[(size_t)q];
    C.bperm_G = G;
    C.bperm_W = d.W;
    C.bperm_jt = d.jt;
    C.bperm_ipb = d.ipb;
}

int plan_make(const Pool &P, ClusterSet &C, int precision, cudaStream_t st, Plan &out,
              const PairShape *force, bool use_table, int waves)
{
    Plan pl;
    pl.precision = precision;
    pl.pl.mode = plan_mode(C, precision);
    const int64_t mean = C.n / (C.K > 0 ? C.K : 1);
    int I, bps = 0, jt = 0;
    PairShape tuned;
    if (force) {
        I = force->I;
        bps = force->blocks_per_sm;
        jt = force->jt;
    } else if (use_table && tune_lookup(tune_key(P, C, precision), &tuned) &&
               pair_variant_exists(pl.pl.mode, tuned.I)) {
        I = tuned.I;
        bps = tuned.blocks_per_sm;
        jt = tuned.jt;
    } else if (pl.pl.mode == PM_FP64) {
        I = 1;
    } else if (pl.pl.mode == PM_DD) {
        I = 2;   // measured fastest at N = 262144
    } else if (pl.pl.mode == PM_DS_FULL) {
        I = mean < 16384 ? 2 : 4;
    } else {
        // float pairs (mixed and pure float): 8 bodies per thread measured
        // fastest at N = 65536 and N = 262144 and on the 512-cluster
        // ensemble (mean N 2519); small clusters keep 2 so the i-blocks
        // stay narrow enough to give every resident block a unit
        I = mean < 2048 ? 2 : 8;
    }
    if (!pair_variant_exists(pl.pl.mode, I))
        return set_error(NB_EINVAL, "no pair kernel with %d bodies per thread for this precision",
                         I);
    pl.pl.I = I;
    int occ = pair_occupancy(pl.pl.mode, I);
    if (occ < 1) occ = 1;
    if (waves > 0) bps = (waves < MAX_WAVES ? waves : MAX_WAVES) * occ;
    pl.pl.blocks_per_sm = bps > 0 ? (bps < MAX_WAVES * occ ? bps : MAX_WAVES * occ)
                                  : DEFAULT_WAVES * occ;
    const int64_t want = (int64_t)P.num_sms * pl.pl.blocks_per_sm;
    const int64_t resident = (int64_t)P.num_sms * occ;
    if (jt == 0) {
        // full-width j-tiles, halved while the units are too few to give
        // every resident block one (small clusters)
        int64_t w_full = 0;
        for (int32_t k = 0; k < C.K; ++k)
            w_full += ((C.nk[k] + TILE * I - 1) / (TILE * I)) * ((C.nk[k] + TILE - 1) / TILE);
        jt = TILE;
        while (jt > 32 && w_full * (TILE / jt) < resident) jt /= 2;
    }
    int rc = set_layout(C, TILE * I, st, jt);
    if (rc) return rc;
    pl.pl.um = true;
    for (int32_t k = 0; k < C.K && pl.pl.um; ++k) pl.pl.um = C.mu[k] > 0;
    const int64_t W = C.uoff[C.K];
    int64_t G = want < W ? want : W;   // at least one unit per block
    const int64_t slot_cap = part_slot_cap(P, C);
    pl.pl.d = make_decomp(W, C.max_ntiles, TILE * I, G, slot_cap, jt);
    pl.pl.d.fpart = sp_family(pl.pl.mode) ? 1 : 0;
    // several clusters by value: launch the blocks largest-work first.  Not
    // with the near-pair pass beside the pair kernel: its kernels get SMs as
    // the pair kernel's blocks drain, and on the 512-cluster ensemble the
    // tighter tail left them less room (pair kernel 2.5% faster, step 2%
    // slower); in the other modes it made the step 0.5-2.6% faster
    C.bperm_G = -1;
    if (pl.pl.mode != PM_FP64 && pl.pl.mode != PM_DS_NEAR && C.K > 1 && C.K <= PARAM_CLUSTERS &&
        pl.pl.d.G <= PERM_CAP && !pl.pl.d.rows)
        block_order(C, pl.pl.d, I, sp_family(pl.pl.mode));
    for (int32_t k = 0; k < C.K; ++k)
        if (C.eps2d[k] == 0.0) pl.pl.d.mask_self = 1;
    int occ_pot = pair_occupancy(PM_FP64, 1);
    if (occ_pot < 1) occ_pot = 1;
    const int64_t Wp = C.uoff_pot[C.K];
    int64_t Gp = (int64_t)P.num_sms * occ_pot;
    if (Wp / 2 < Gp) Gp = Wp / 2 > 0 ? Wp / 2 : 1;
    pl.pot = make_decomp(Wp, C.max_ntiles, TILE, Gp, slot_cap);
    out = pl;
    return NB_OK;
}

int plan_mode(const ClusterSet &C, int precision)
{
    const int m = mode_of(precision);
    if (m != PM_DS_NEAR || precision == NB_DS_NEAR) return m;
    double pairs = 0;
    for (int32_t k = 0; k < C.K; ++k) pairs += (double)C.nk[k] * (double)C.nk[k];
    return pairs <= DS_FULL_MAX_PAIRS ? PM_DS_FULL : PM_DS_NEAR;
}

DevState view(const Pool &P, const ClusterSet &C, const Plan &pl)
{
    DevState s = view(P, C, (int)pl.precision);
    if (pl.pl.mode != PM_DS_NEAR) s.corr = nullptr;
    return s;
}

int64_t part_slot_cap(const Pool &P, const ClusterSet &C)
{
    const int64_t elems = C.part ? C.part_elems : P.s.part_elems;
    const int64_t per = C.n > 0 ? elems / (3 * C.n) : MAX_PART_SLOTS;
    return per < MAX_PART_SLOTS ? per : MAX_PART_SLOTS;
}

DevState view(const Pool &P, const ClusterSet &C, int precision)
{
    DevState s = P.s;
    s.cl = C.cl;
    s.n = C.n;
    if (C.part) {
        s.part = C.part;
        s.part_elems = C.part_elems;
    }
    s.pstride = C.n > 0 ? C.n : 1;
    s.part_slots = part_slot_cap(P, C);
    s.diag = C.diag;
    s.red = C.red;
    s.red_len = C.scap * 16;
    s.ng_bucket = C.ng_bucket;
    s.ng_entry = C.ng_entry;
    s.ng_total = C.ng_total;
    s.ng_hcap = C.ng_hcap;
    s.ng_spos = C.ng_spos;
    s.ng_slo = C.ng_slo;
    s.ng_slot = C.ng_slot;
    s.ng_rank = C.ng_rank;
    s.flag = C.flag;
    if (precision != NB_DS && precision != NB_DS_NEAR) s.corr = nullptr;
    return s;
}

// ---- enqueue -----------------------------------------------------------------

namespace {
void count(int64_t *k, int64_t v)
{
    if (k) *k += v;
}
constexpr int64_t NEAR_KERNELS = 5;   // launch_near_correct (memsets not counted)
}  // namespace

int enq_split(const Pool &P, const ClusterSet &C, const Plan &pl, const Phys &ph,
              cudaStream_t st, int64_t *kernels)
{
    if (!float_planes(pl.precision)) return NB_OK;
    const DevState s = view(P, C, pl);
    const bool near = pl.pl.mode == PM_DS_NEAR;
    NB_TRY(launch_frame(s, ph.near_frac, near, st));
    NB_TRY(launch_split(s, st));
    count(kernels, near ? 5 : 3);
    return NB_OK;
}

int enq_force(const Pool &P, const ClusterSet &C, const Plan &pl, const Phys &ph,
              cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1, int64_t *kernels)
{
    const DevState s = view(P, C, pl);
    // inside a stream capture an event record must be an external node to
    // time anything; outside it is a plain record
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    NB_TRY(cudaStreamIsCapturing(st, &cs));
    const unsigned evf =
        cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (ev0) NB_TRY(cudaEventRecordWithFlags(ev0, st, evf));
    HostTab ht;
    ht.K = C.K;
    ht.uoff = C.uoff.data();
    ht.boff = C.boff.data();
    ht.noff = C.noff.data();
    ht.nk = C.nk.data();
    ht.ntiles = C.ntiles.data();
    ht.eps2f = C.eps2f.data();
    ht.mu = C.mu.data();
    const Decomp &d = pl.pl.d;
    if (C.bperm_G == d.G && C.bperm_W == d.W && C.bperm_jt == d.jt && C.bperm_ipb == d.ipb &&
        !d.rows) {
        ht.perm = C.bperm.data();
        ht.nperm = (int32_t)C.bperm.size();
    }
    // the near-pair pass (mixed mode) forks onto the set's side stream and
    // runs beside the pair kernel: both read only the float planes, and they
    // write different buffers (corr, part), so the overlap cannot change a
    // result; the join orders it before whatever follows on st
    const bool near = pl.pl.mode == PM_DS_NEAR;
    if (near) {
        NB_TRY(cudaEventRecord(C.fork, st));
        NB_TRY(cudaStreamWaitEvent(C.side, C.fork, 0));
        NB_TRY(launch_near_correct(s, ph.G, pl.pl.um, C.side));
        NB_TRY(cudaEventRecord(C.join, C.side));
        count(kernels, NEAR_KERNELS);
    }
    NB_TRY(launch_pair(s, pl.pl, ht, ph.G, st));
    if (ev1) NB_TRY(cudaEventRecordWithFlags(ev1, st, evf));
    count(kernels, 1);
    if (near) NB_TRY(cudaStreamWaitEvent(st, C.join, 0));
    return NB_OK;
}

int enq_step(const Pool &P, const ClusterSet &C, const Plan &pl, const Phys &ph, int order,
             double h, cudaStream_t st, const std::vector<cudaEvent_t> *evs, int64_t *kernels)
{
    const bool sp = float_planes(pl.precision);
    const DevState s = view(P, C, pl);
    double wk[7];
    int K;
    if (order == 2) {
        K = 1;
        wk[0] = 1.0;
    } else {
        K = 7;
        const double w0 = 1.0 - 2.0 * (SI6_W1 + SI6_W2 + SI6_W3);
        const double seq[7] = {SI6_W3, SI6_W2, SI6_W1, w0, SI6_W1, SI6_W2, SI6_W3};
        for (int k = 0; k < 7; ++k) wk[k] = seq[k];
    }
    if (sp) {
        const bool near = pl.pl.mode == PM_DS_NEAR;
        NB_TRY(launch_frame(s, ph.near_frac, near, st));
        count(kernels, near ? 4 : 2);
    }
    // drift of the first leapfrog's half step (and the split it feeds, mass
    // words included: the later splits of the step rewrite coordinates only)
    NB_TRY(launch_kick_drift(s, pl.pl.d, 0.0, 0.5 * wk[0] * h, 0, sp ? 2 : 0, ph.ext, st));
    count(kernels, 1);
    for (int k = 0; k < K; ++k) {
        // adjacent half drifts of consecutive leapfrogs merge
        const double hd = 0.5 * (wk[k] + (k + 1 < K ? wk[k + 1] : 0.0)) * h;
        const bool last = (k + 1 == K);
        cudaEvent_t e0 = evs ? (*evs)[2 * k] : nullptr, e1 = evs ? (*evs)[2 * k + 1] : nullptr;
        int rc = enq_force(P, C, pl, ph, st, e0, e1, kernels);
        if (rc) return rc;
        NB_TRY(launch_kick_drift(s, pl.pl.d, wk[k] * h, hd, 1, (sp && !last) ? 1 : 0, ph.ext,
                                 st));
        count(kernels, 1);
    }
    return NB_OK;
}

int enq_accel_out(const Pool &P, const ClusterSet &C, const Plan &pl, const Phys &ph,
                  double *out, cudaStream_t st, int64_t *kernels)
{
    const DevState s = view(P, C, pl);
    NB_TRY(launch_accel_out(s, pl.pl.d, ph.ext, out, st));
    count(kernels, 1);
    return NB_OK;
}

int enq_energy(const Pool &P, const ClusterSet &C, const Plan &pl, const Phys &ph,
               cudaStream_t st, int64_t *kernels)
{
    DevState s = view(P, C, pl);
    s.cl = C.cl_pot;
    NB_TRY(launch_potential(s, pl.pot, st));
    NB_TRY(launch_energy_reduce(s, pl.pot, ph.ext, ph.G, st));
    count(kernels, 3);
    return NB_OK;
}

int enq_torque(const Pool &P, const ClusterSet &C, const Phys &ph, cudaStream_t st,
               int64_t *kernels)
{
    const DevState s = view(P, C, NB_FP64);
    NB_TRY(launch_torque(s, ph.ext, st));
    count(kernels, 2);
    return NB_OK;
}

}  // namespace nb
