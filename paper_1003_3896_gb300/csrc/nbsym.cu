// nbsym.cu -- the context API of include/nbsym.h on top of the engine.
//
// A context owns a state pool, one cluster set (one cluster for nb_create,
// K fixed-size clusters for nb_create_batch), the launch plan of its current
// precision, and one CUDA graph per (order, dt) holding a whole integration
// step, replayed nsteps times by nb_step.
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "engine.h"

using namespace nb;

namespace {

struct StepGraph {
    int order = 0;
    double dt = 0;
    int prof = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<cudaEvent_t> ev;   // (start, stop) per pair launch when prof
    int64_t kernels = 0;
};

bool finite_pos(double v) { return std::isfinite(v) && v > 0; }

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace

struct nb_ctx {
    nb_params p{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    Pool pool;
    ClusterSet set;
    Plan plan;
    Phys phys;
    bool batch = false;
    std::vector<int64_t> sizes;    // batch cluster sizes
    std::vector<double> eps_k, dts_k;
    std::vector<double> mu_k;      // common mass per cluster (0: masses differ)
    int64_t n = 0;                 // bodies loaded (0: none)
    bool planned = false;
    bool split_stale = true;
    std::vector<StepGraph> graphs;
    bool prof_on = false;
    nb_prof_t prof{};
    cudaEvent_t pe0 = nullptr, pe1 = nullptr;
};

namespace {

int check_params(const nb_params *p)
{
    if (!p) return set_error(NB_EINVAL, "params is NULL");
    if (!finite_pos(p->G)) return set_error(NB_EINVAL, "G must be finite and > 0");
    if (!std::isfinite(p->eps) || p->eps < 0)
        return set_error(NB_EINVAL, "eps must be finite and >= 0");
    if (p->precision < NB_FP64 || p->precision > NB_DS_NEAR)
        return set_error(NB_EINVAL, "precision must be NB_FP64, NB_DS, NB_FP32, NB_DS_FULL, "
                                    "NB_DD or NB_DS_NEAR");
    if (p->ext_on) {
        if (!std::isfinite(p->Md) || p->Md < 0 || !std::isfinite(p->Mb) || p->Mb < 0 ||
            !std::isfinite(p->ad) || p->ad < 0 || !finite_pos(p->bd) || !finite_pos(p->ab))
            return set_error(NB_EINVAL, "external field needs Md, Mb, ad >= 0 and bd, ab > 0");
    }
    if (!std::isfinite(p->near_frac)) return set_error(NB_EINVAL, "near_frac must be finite");
    if (!std::isfinite(p->Mbh) || p->Mbh < 0 || !std::isfinite(p->eps_bh) || p->eps_bh < 0)
        return set_error(NB_EINVAL, "Mbh and eps_bh must be finite and >= 0");
    return NB_OK;
}

Phys phys_of(const nb_params &p)
{
    Phys ph;
    ph.G = p.G;
    ph.near_frac = p.near_frac > 0 ? p.near_frac : 0.4;
    ph.ext.on = p.ext_on;
    ph.ext.G = p.G;
    ph.ext.Md = p.Md;
    ph.ext.ad = p.ad;
    ph.ext.bd = p.bd;
    ph.ext.Mb = p.Mb;
    ph.ext.ab = p.ab;
    ph.ext.Mbh = p.Mbh;
    ph.ext.eps2bh = p.eps_bh * p.eps_bh;
    return ph;
}

void free_graphs(nb_ctx *c)
{
    for (auto &g : c->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        for (auto e : g.ev) cudaEventDestroy(e);
    }
    c->graphs.clear();
}

// (Re)define the cluster set for n bodies and lay it out for the current
// precision; cached step graphs are dropped.
int replan(nb_ctx *c, int64_t n)
{
    std::vector<int64_t> boff, nk;
    if (c->batch) {
        int64_t off = 0;
        for (int64_t s : c->sizes) {
            boff.push_back(off);
            nk.push_back(s);
            off += s;
        }
    } else {
        boff.push_back(0);
        nk.push_back(n);
        c->eps_k.assign(1, c->p.eps);
        if (c->dts_k.size() != 1) c->dts_k.assign(1, 1.0);
    }
    int rc = set_define(c->set, (int32_t)nk.size(), boff.data(), nk.data(), c->eps_k.data(),
                        c->dts_k.data());
    if (rc) return rc;
    if (c->mu_k.size() == nk.size())
        c->set.mu = c->mu_k;
    else
        c->set.mu.assign(nk.size(), 0.0);
    rc = plan_make(c->pool, c->set, c->p.precision, c->stream, c->plan);
    if (rc) return rc;
    free_graphs(c);
    c->planned = true;
    c->split_stale = true;
    return NB_OK;
}

int refresh_split(nb_ctx *c)
{
    if (!c->split_stale) return NB_OK;
    int64_t k = 0;
    int rc = enq_split(c->pool, c->set, c->plan, c->phys, c->stream, &k);
    if (rc) return rc;
    if (c->prof_on) c->prof.kernel_launches += k;
    c->split_stale = false;
    return NB_OK;
}

int get_graph(nb_ctx *c, int order, double h, StepGraph **out)
{
    const int prof = c->prof_on ? 1 : 0;
    for (auto &g : c->graphs)
        if (g.order == order && g.dt == h && g.prof == prof) {
            *out = &g;
            return NB_OK;
        }
    StepGraph g;
    g.order = order;
    g.dt = h;
    g.prof = prof;
    if (prof) {
        g.ev.resize(2 * (order == 2 ? 1 : 7));
        for (auto &e : g.ev) NB_TRY(cudaEventCreate(&e));
    }
    NB_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enq_step(c->pool, c->set, c->plan, c->phys, order, h, c->stream,
                      prof ? &g.ev : nullptr, &g.kernels);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (rc != NB_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        for (auto ev : g.ev) cudaEventDestroy(ev);
        if (rc != NB_OK) return rc;
        return set_error(NB_ECUDA, "stream capture failed: %s", cudaGetErrorString(e));
    }
    g.graph = graph;
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        for (auto ev : g.ev) cudaEventDestroy(ev);
        return set_error(NB_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    if (c->graphs.size() >= 8) {
        auto &old = c->graphs.front();
        cudaGraphExecDestroy(old.exec);
        cudaGraphDestroy(old.graph);
        for (auto ev : old.ev) cudaEventDestroy(ev);
        c->graphs.erase(c->graphs.begin());
    }
    c->graphs.push_back(g);
    *out = &c->graphs.back();
    return NB_OK;
}

int check_flag(nb_ctx *c, const char *what)
{
    int h = 0;
    NB_TRY(cudaMemcpyAsync(&h, c->set.flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    NB_TRY(cudaStreamSynchronize(c->stream));
    if (h) return set_error(NB_ENONFINITE, "%s: non-finite values (coincident bodies with eps = 0?)", what);
    return NB_OK;
}

int create_common(const nb_params *p, int64_t cap, const int64_t *sizes, int64_t K,
                  nb_ctx **out)
{
    if (!out) return set_error(NB_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check_params(p);
    if (rc) return rc;
    if (cap < 1 || cap > ((int64_t)1 << 26))
        return set_error(NB_EINVAL, "capacity must be in [1, 2^26]");
    int ndev = 0;
    NB_TRY(cudaGetDeviceCount(&ndev));
    if (p->device < 0 || p->device >= ndev)
        return set_error(NB_EINVAL, "no CUDA device %d", p->device);
    DeviceGuard dg(p->device);
    nb_ctx *c = new (std::nothrow) nb_ctx();
    if (!c) return set_error(NB_ENOMEM, "host allocation failed");
    c->p = *p;
    c->phys = phys_of(*p);
    if (p->stream) {
        c->stream = (cudaStream_t)p->stream;
    } else if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return set_error(NB_ECUDA, "cudaStreamCreate failed");
    } else {
        c->own_stream = true;
    }
    rc = pool_create(c->pool, p->device, cap);
    if (!rc) rc = set_create(c->set, (int32_t)K, cap);
    if (!rc && (cudaEventCreate(&c->pe0) != cudaSuccess || cudaEventCreate(&c->pe1) != cudaSuccess))
        rc = set_error(NB_ECUDA, "cudaEventCreate failed");
    if (!rc && sizes) {
        c->batch = true;
        c->sizes.assign(sizes, sizes + K);
        c->eps_k.assign(K, p->eps);
        c->dts_k.assign(K, 1.0);
    }
    if (rc) {
        nb_destroy(c);
        return rc;
    }
    *out = c;
    return NB_OK;
}

}  // namespace

namespace nb {
// The parameter checks of nb_create, shared with the no-allocation entry point.
int check_nb_params(const nb_params *p) { return check_params(p); }
}  // namespace nb

extern "C" {

int nb_abi_version(void) { return NB_ABI_VERSION; }

int nb_stage_weights(int order, double *w)
{
    if (!w) return set_error(NB_EINVAL, "w is NULL");
    if (order == 2) {
        w[0] = 1.0;
        return 1;
    }
    if (order != 6) return set_error(NB_EINVAL, "order must be 2 or 6");
    const double w0 = 1.0 - 2.0 * (SI6_W1 + SI6_W2 + SI6_W3);
    const double seq[7] = {SI6_W3, SI6_W2, SI6_W1, w0, SI6_W1, SI6_W2, SI6_W3};
    for (int k = 0; k < 7; ++k) w[k] = seq[k];
    return 7;
}

const char *nb_last_error(void) { return last_error(); }

void nb_params_default(nb_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->G = 1.0;
    p->eps = 0.0;
    p->precision = NB_DS;
    p->ext_on = 0;
    p->Md = 100.0;
    p->ad = 6.5;
    p->bd = 0.26;
    p->Mb = 15.0;
    p->ab = 0.7;
    p->device = 0;
    p->stream = nullptr;
    p->near_frac = 0.0;
}

int nb_create(const nb_params *p, int64_t n_capacity, nb_ctx **out)
{
    return create_common(p, n_capacity, nullptr, 1, out);
}

int nb_create_batch(const nb_params *p, int64_t n_clusters, const int64_t *sizes,
                    nb_ctx **out)
{
    if (!out) return set_error(NB_EINVAL, "out is NULL");
    *out = nullptr;
    if (!sizes || n_clusters < 1 || n_clusters > (1 << 19))
        return set_error(NB_EINVAL, "need 1 <= n_clusters <= 2^19 and a sizes array");
    int64_t tot = 0;
    for (int64_t k = 0; k < n_clusters; ++k) {
        if (sizes[k] < 1) return set_error(NB_EINVAL, "cluster %lld has no bodies", (long long)k);
        tot += sizes[k];
    }
    return create_common(p, tot, sizes, n_clusters, out);
}

void nb_destroy(nb_ctx *c)
{
    if (!c) return;
    DeviceGuard dg(c->p.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_graphs(c);
    set_destroy(c->set);
    pool_destroy(c->pool);
    if (c->pe0) cudaEventDestroy(c->pe0);
    if (c->pe1) cudaEventDestroy(c->pe1);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

static int load_common(nb_ctx *c, int64_t n, const double *pos, const double *vel,
                       const double *mass, cudaMemcpyKind kind)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    if (!pos || !vel || !mass) return set_error(NB_EINVAL, "pos, vel and mass must be non-NULL");
    if (n < 1 || n > c->pool.cap)
        return set_error(NB_EINVAL, "n=%lld outside [1, capacity=%lld]", (long long)n,
                         (long long)c->pool.cap);
    if (c->batch && n != c->pool.cap)
        return set_error(NB_EINVAL, "a batch context loads exactly the sum of its cluster sizes (%lld)",
                         (long long)c->pool.cap);
    DeviceGuard dg(c->p.device);
    if (!c->planned || n != c->n) {
        int rc = replan(c, n);
        if (rc) return rc;
    }
    c->n = n;
    const double *dp = pos, *dv = vel, *dm = mass;
    if (kind == cudaMemcpyHostToDevice) {
        double *sp = c->pool.stage, *sv = sp + 3 * c->pool.cap, *sm = sp + 6 * c->pool.cap;
        NB_TRY(cudaMemcpyAsync(sp, pos, (size_t)(3 * n) * sizeof(double), kind, c->stream));
        NB_TRY(cudaMemcpyAsync(sv, vel, (size_t)(3 * n) * sizeof(double), kind, c->stream));
        NB_TRY(cudaMemcpyAsync(sm, mass, (size_t)n * sizeof(double), kind, c->stream));
        dp = sp;
        dv = sv;
        dm = sm;
    }
    NB_TRY(launch_unpack(view(c->pool, c->set, c->p.precision), dp, dv, dm, c->stream));
    // clusters whose bodies all have one mass get the pair kernels' uniform-
    // mass form; the plan follows the masses
    NB_TRY(launch_mass_range(view(c->pool, c->set, c->p.precision), c->stream));
    const int32_t K = c->set.K;
    std::vector<double> range((size_t)K * DIAG_STRIDE);
    NB_TRY(cudaMemcpyAsync(range.data(), c->set.diag, range.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
    NB_TRY(cudaStreamSynchronize(c->stream));
    std::vector<double> mu((size_t)K);
    for (int32_t k = 0; k < K; ++k) {
        const double lo = range[(size_t)k * DIAG_STRIDE], hi = range[(size_t)k * DIAG_STRIDE + 1];
        mu[k] = lo == hi && lo > 0 && std::isfinite(lo) ? lo : 0.0;
    }
    if (mu != c->mu_k) {
        c->mu_k = mu;
        int rc = replan(c, n);
        if (rc) return rc;
    }
    c->split_stale = true;
    return NB_OK;
}

int nb_load(nb_ctx *c, int64_t n, const double *pos, const double *vel, const double *mass)
{
    return load_common(c, n, pos, vel, mass, cudaMemcpyHostToDevice);
}

int nb_load_device(nb_ctx *c, int64_t n, const double *pos, const double *vel,
                   const double *mass)
{
    return load_common(c, n, pos, vel, mass, cudaMemcpyDeviceToDevice);
}

int nb_set_cluster_params(nb_ctx *c, const double *eps, const double *dt_scale)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    const int64_t K = c->batch ? (int64_t)c->sizes.size() : 1;
    for (int64_t k = 0; k < K; ++k) {
        if (eps && (!std::isfinite(eps[k]) || eps[k] < 0))
            return set_error(NB_EINVAL, "eps[%lld] must be finite and >= 0", (long long)k);
        if (dt_scale && !finite_pos(dt_scale[k]))
            return set_error(NB_EINVAL, "dt_scale[%lld] must be finite and > 0", (long long)k);
    }
    if (eps) {
        c->eps_k.assign(eps, eps + K);
        if (!c->batch) c->p.eps = eps[0];
    }
    if (dt_scale) c->dts_k.assign(dt_scale, dt_scale + K);
    if (c->n > 0) {
        DeviceGuard dg(c->p.device);
        return replan(c, c->n);
    }
    return NB_OK;
}

static int accel_common(nb_ctx *c, double *out, bool host)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    if (!out) return set_error(NB_EINVAL, "acc_out is NULL");
    if (c->n == 0) return set_error(NB_ESTATE, "nb_accel before nb_load");
    DeviceGuard dg(c->p.device);
    int rc = refresh_split(c);
    if (rc) return rc;
    int64_t k = 0;
    if (c->prof_on) NB_TRY(cudaEventRecord(c->pe0, c->stream));
    rc = enq_force(c->pool, c->set, c->plan, c->phys, c->stream, nullptr,
                   c->prof_on ? c->pe1 : nullptr, &k);
    if (rc) return rc;
    NB_TRY(cudaMemsetAsync(c->set.flag, 0, sizeof(int), c->stream));
    double *dst = host ? c->pool.stage : out;
    rc = enq_accel_out(c->pool, c->set, c->plan, c->phys, dst, c->stream, &k);
    if (rc) return rc;
    if (host)
        NB_TRY(cudaMemcpyAsync(out, dst, (size_t)(3 * c->n) * sizeof(double),
                               cudaMemcpyDeviceToHost, c->stream));
    rc = check_flag(c, "nb_accel");
    if (c->prof_on) {
        float ms = 0;
        NB_TRY(cudaEventElapsedTime(&ms, c->pe0, c->pe1));
        c->prof.pair_launches += 1;
        c->prof.pair_ms += ms;
        for (int64_t q = 0; q < c->set.K; ++q) c->prof.interactions += c->set.nk[q] * c->set.nk[q];
        c->prof.kernel_launches += k;
    }
    return rc;
}

int nb_accel(nb_ctx *c, double *acc_out) { return accel_common(c, acc_out, true); }

int nb_accel_device(nb_ctx *c, double *d_acc_out) { return accel_common(c, d_acc_out, false); }

int nb_accel_range(nb_ctx *c, int64_t i0, int64_t i1, double *acc_out)
{
    if (!c || !acc_out) return set_error(NB_EINVAL, "NULL argument");
    if (c->n == 0) return set_error(NB_ESTATE, "nb_accel_range before nb_load");
    if (c->set.K != 1) return set_error(NB_EINVAL, "nb_accel_range takes one cluster");
    if (i0 < 0 || i1 > c->n || i0 >= i1)
        return set_error(NB_EINVAL, "range [%lld, %lld) outside [0, %lld)", (long long)i0,
                         (long long)i1, (long long)c->n);
    DeviceGuard dg(c->p.device);
    int rc = refresh_split(c);
    if (rc) return rc;
    // whole i-block rows of the range, one block per run of rows: each row's
    // j sum is done in order by one block, as in any other range launch
    const Plan &pl = c->plan;
    PairLaunch rl = pl.pl;
    const int ipb = TILE * rl.I;
    const int64_t b0 = i0 / ipb, b1 = (i1 + ipb - 1) / ipb, W = b1 - b0;
    int64_t G = (int64_t)c->pool.num_sms * rl.blocks_per_sm;
    if (G > W) G = W;
    rl.d = make_decomp(W, c->set.max_ntiles, ipb, G, part_slot_cap(c->pool, c->set), TILE, 1);
    rl.d.b0 = b0;
    rl.d.mask_self = pl.pl.d.mask_self;
    rl.d.fpart = pl.pl.d.fpart;
    const DevState s = view(c->pool, c->set, pl);
    const int64_t uoff[2] = {0, W};
    HostTab ht;
    ht.K = 1;
    ht.uoff = uoff;
    ht.boff = c->set.boff.data();
    ht.nk = c->set.nk.data();
    ht.ntiles = c->set.ntiles.data();
    ht.eps2f = c->set.eps2f.data();
    ht.mu = c->set.mu.data();
    NB_TRY(launch_pair(s, rl, ht, c->phys.G, c->stream));
    if (rl.mode == PM_DS_NEAR) NB_TRY(launch_near_correct(s, c->phys.G, rl.um, c->stream));
    NB_TRY(cudaMemsetAsync(c->set.flag, 0, sizeof(int), c->stream));
    double *out = c->pool.stage;   // 3 (i1 - i0) <= 7 cap doubles
    NB_TRY(launch_accel_out_range(s, rl.d, c->phys.ext, out, i0, i1, c->stream));
    NB_TRY(cudaMemcpyAsync(acc_out, out, sizeof(double) * 3 * (size_t)(i1 - i0),
                           cudaMemcpyDeviceToHost, c->stream));
    return check_flag(c, "nb_accel_range");
}

int nb_substep_range(nb_ctx *c, int64_t i0, int64_t i1, double kick, double drift)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    if (c->n == 0) return set_error(NB_ESTATE, "nb_substep_range before nb_load");
    if (c->set.K != 1) return set_error(NB_EINVAL, "nb_substep_range takes one cluster");
    if (i0 < 0 || i1 > c->n || i0 >= i1)
        return set_error(NB_EINVAL, "range [%lld, %lld) outside [0, %lld)", (long long)i0,
                         (long long)i1, (long long)c->n);
    if (!std::isfinite(kick) || !std::isfinite(drift))
        return set_error(NB_EINVAL, "kick and drift must be finite");
    DeviceGuard dg(c->p.device);
    const Plan &pl = c->plan;
    PairLaunch rl = pl.pl;
    const int ipb = TILE * rl.I;
    const int64_t b0 = i0 / ipb, b1 = (i1 + ipb - 1) / ipb, W = b1 - b0;
    int64_t G = (int64_t)c->pool.num_sms * rl.blocks_per_sm;
    if (G > W) G = W;
    rl.d = make_decomp(W, c->set.max_ntiles, ipb, G, part_slot_cap(c->pool, c->set), TILE, 1);
    rl.d.b0 = b0;
    rl.d.mask_self = pl.pl.d.mask_self;
    rl.d.fpart = pl.pl.d.fpart;
    const DevState s = view(c->pool, c->set, pl);
    if (kick != 0.0) {
        // the force evaluation of nb_accel_range (whole i-block rows, each
        // summed in order by one block), consumed by the kick of the range
        int rc = refresh_split(c);
        if (rc) return rc;
        const int64_t uoff[2] = {0, W};
        HostTab ht;
        ht.K = 1;
        ht.uoff = uoff;
        ht.boff = c->set.boff.data();
        ht.nk = c->set.nk.data();
        ht.ntiles = c->set.ntiles.data();
        ht.eps2f = c->set.eps2f.data();
        ht.mu = c->set.mu.data();
        NB_TRY(launch_pair(s, rl, ht, c->phys.G, c->stream));
        if (rl.mode == PM_DS_NEAR) NB_TRY(launch_near_correct(s, c->phys.G, rl.um, c->stream));
    }
    NB_TRY(launch_kick_drift_range(s, rl.d, kick, drift, kick != 0.0 ? 1 : 0, 0, c->phys.ext,
                                   i0, i1, c->stream));
    NB_TRY(cudaStreamSynchronize(c->stream));
    c->split_stale = true;
    return NB_OK;
}

static int set_state_common(nb_ctx *c, const double *pos, const double *vel, bool host)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    if (c->n == 0) return set_error(NB_ESTATE, "nb_set_state before nb_load");
    if (!pos && !vel) return NB_OK;
    DeviceGuard dg(c->p.device);
    const int64_t n = c->n;
    const double *dp = pos, *dv = vel;
    if (host) {
        double *sp = c->pool.stage, *sv = c->pool.stage + 3 * c->pool.cap;
        if (pos)
            NB_TRY(cudaMemcpyAsync(sp, pos, (size_t)(3 * n) * sizeof(double),
                                   cudaMemcpyHostToDevice, c->stream));
        if (vel)
            NB_TRY(cudaMemcpyAsync(sv, vel, (size_t)(3 * n) * sizeof(double),
                                   cudaMemcpyHostToDevice, c->stream));
        dp = pos ? sp : nullptr;
        dv = vel ? sv : nullptr;
    }
    NB_TRY(launch_set_state(view(c->pool, c->set, c->p.precision), dp, dv, c->stream));
    NB_TRY(cudaStreamSynchronize(c->stream));
    c->split_stale = true;
    return NB_OK;
}

int nb_set_state(nb_ctx *c, const double *pos, const double *vel)
{
    return set_state_common(c, pos, vel, true);
}

int nb_set_state_device(nb_ctx *c, const double *d_pos, const double *d_vel)
{
    return set_state_common(c, d_pos, d_vel, false);
}

int nb_step(nb_ctx *c, int order, double dt, int64_t nsteps)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    if (order != 2 && order != 6) return set_error(NB_EINVAL, "order must be 2 or 6");
    if (!finite_pos(dt)) return set_error(NB_EINVAL, "dt must be finite and > 0");
    if (nsteps < 0) return set_error(NB_EINVAL, "nsteps must be >= 0");
    if (c->n == 0) return set_error(NB_ESTATE, "nb_step before nb_load");
    if (nsteps == 0) return NB_OK;
    DeviceGuard dg(c->p.device);
    StepGraph *g = nullptr;
    int rc = get_graph(c, order, dt, &g);
    if (rc) return rc;
    int64_t pairs = 0;
    for (int64_t q = 0; q < c->set.K; ++q) pairs += c->set.nk[q] * c->set.nk[q];
    for (int64_t k = 0; k < nsteps; ++k) {
        NB_TRY(cudaGraphLaunch(g->exec, c->stream));
        if (c->prof_on) {
            NB_TRY(cudaStreamSynchronize(c->stream));
            for (size_t q = 0; q + 1 < g->ev.size(); q += 2) {
                float ms = 0;
                NB_TRY(cudaEventElapsedTime(&ms, g->ev[q], g->ev[q + 1]));
                c->prof.pair_ms += ms;
                c->prof.pair_launches += 1;
                c->prof.interactions += pairs;
            }
            c->prof.kernel_launches += g->kernels;
        }
    }
    NB_TRY(cudaStreamSynchronize(c->stream));
    c->split_stale = true;
    return NB_OK;
}

static int energy_common(nb_ctx *c, std::vector<double> &d)
{
    if (c->n == 0) return set_error(NB_ESTATE, "nb_energy before nb_load");
    DeviceGuard dg(c->p.device);
    NB_TRY(cudaMemsetAsync(c->set.flag, 0, sizeof(int), c->stream));
    int64_t k = 0;
    int rc = enq_energy(c->pool, c->set, c->plan, c->phys, c->stream, &k);
    if (rc) return rc;
    d.resize((size_t)c->set.K * DIAG_STRIDE);
    NB_TRY(cudaMemcpyAsync(d.data(), c->set.diag, d.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
    if (c->prof_on) c->prof.kernel_launches += k;
    return check_flag(c, "nb_energy");
}

static void to_energy(const double *d, nb_energy_t *o)
{
    o->K = d[0];
    o->W = d[1];
    o->W_ext = d[2];
    o->E = d[3];
    for (int q = 0; q < 3; ++q) {
        o->P[q] = d[4 + q];
        o->L[q] = d[7 + q];
    }
}

int nb_energy(nb_ctx *c, nb_energy_t *out)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    if (!out) return set_error(NB_EINVAL, "out is NULL");
    std::vector<double> d;
    int rc = energy_common(c, d);
    double tot[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t k = 0; k < c->set.K && !d.empty(); ++k)
        for (int q = 0; q < 10; ++q) tot[q] += d[k * DIAG_STRIDE + q];
    to_energy(tot, out);
    return rc;
}

int nb_energy_clusters(nb_ctx *c, nb_energy_t *out)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    if (!out) return set_error(NB_EINVAL, "out is NULL");
    std::vector<double> d;
    int rc = energy_common(c, d);
    for (int64_t k = 0; k < c->set.K && !d.empty(); ++k) to_energy(&d[k * DIAG_STRIDE], &out[k]);
    return rc;
}

int nb_torque(nb_ctx *c, double *out)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    if (!out) return set_error(NB_EINVAL, "out is NULL");
    if (c->n == 0) return set_error(NB_ESTATE, "nb_torque before nb_load");
    out[0] = out[1] = out[2] = 0.0;
    if (!c->p.ext_on) return NB_OK;
    DeviceGuard dg(c->p.device);
    int rc = enq_torque(c->pool, c->set, c->phys, c->stream, nullptr);
    if (rc) return rc;
    std::vector<double> d((size_t)c->set.K * DIAG_STRIDE);
    NB_TRY(cudaMemcpyAsync(d.data(), c->set.diag, d.size() * sizeof(double),
                           cudaMemcpyDeviceToHost, c->stream));
    NB_TRY(cudaStreamSynchronize(c->stream));
    for (int64_t k = 0; k < c->set.K; ++k)
        for (int q = 0; q < 3; ++q) out[q] += d[k * DIAG_STRIDE + 10 + q];
    return NB_OK;
}

static int state_common(nb_ctx *c, double *pos, double *vel, bool host)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    if (c->n == 0) return set_error(NB_ESTATE, "nb_get_state before nb_load");
    if (!pos && !vel) return NB_OK;
    DeviceGuard dg(c->p.device);
    const int64_t n = c->n;
    double *dp = pos, *dv = vel;
    if (host) {
        dp = pos ? c->pool.stage : nullptr;
        dv = vel ? c->pool.stage + 3 * c->pool.cap : nullptr;
    }
    NB_TRY(launch_pack(view(c->pool, c->set, c->p.precision), dp, dv, c->stream));
    if (host) {
        if (pos)
            NB_TRY(cudaMemcpyAsync(pos, dp, (size_t)(3 * n) * sizeof(double),
                                   cudaMemcpyDeviceToHost, c->stream));
        if (vel)
            NB_TRY(cudaMemcpyAsync(vel, dv, (size_t)(3 * n) * sizeof(double),
                                   cudaMemcpyDeviceToHost, c->stream));
    }
    NB_TRY(cudaStreamSynchronize(c->stream));
    return NB_OK;
}

int nb_get_state(nb_ctx *c, double *pos, double *vel) { return state_common(c, pos, vel, true); }

int nb_get_state_device(nb_ctx *c, double *pos, double *vel)
{
    return state_common(c, pos, vel, false);
}

int64_t nb_size(const nb_ctx *c)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    return c->n;
}

int64_t nb_clusters(const nb_ctx *c)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    return c->batch ? (int64_t)c->sizes.size() : 1;
}

int nb_set_precision(nb_ctx *c, int precision)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    if (precision < NB_FP64 || precision > NB_DS_NEAR)
        return set_error(NB_EINVAL, "bad precision");
    DeviceGuard dg(c->p.device);
    c->p.precision = precision;
    if (c->n > 0) return replan(c, c->n);
    return NB_OK;
}

int nb_accel_symmetric(nb_ctx *c, double *acc_out, double *pair_ms)
{
    if (!c || !acc_out) return set_error(NB_EINVAL, "NULL argument");
    if (c->n == 0) return set_error(NB_ESTATE, "nb_accel_symmetric before nb_load");
    if (c->set.K != 1) return set_error(NB_EINVAL, "nb_accel_symmetric takes one cluster");
    DeviceGuard dg(c->p.device);
    const int64_t n = c->n;
    float *acc = nullptr;
    double *out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = NB_OK;
    do {
        if (cudaMalloc(&acc, sizeof(float) * 3 * (size_t)n) != cudaSuccess ||
            cudaMalloc(&out, sizeof(double) * 3 * (size_t)n) != cudaSuccess) {
            cudaGetLastError();
            rc = set_error(NB_ENOMEM, "device allocation failed");
            break;
        }
        if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
            rc = set_error(NB_ECUDA, "event creation failed");
            break;
        }
        // float planes about a fresh frame (the context's own split, if any,
        // is recomputed before its next float-plane use)
        const DevState s = view(c->pool, c->set, NB_FP32);
        if (launch_frame(s, c->phys.near_frac, false, c->stream) != cudaSuccess ||
            launch_split(s, c->stream) != cudaSuccess) {
            rc = set_error(NB_ECUDA, "frame/split launch failed");
            break;
        }
        c->split_stale = true;
        rc = sym_accel(c->pool, c->set, c->phys, acc, out, c->stream, e0, e1);
        if (rc) break;
        if (cudaMemcpyAsync(acc_out, out, sizeof(double) * 3 * (size_t)n, cudaMemcpyDeviceToHost,
                            c->stream) != cudaSuccess ||
            cudaStreamSynchronize(c->stream) != cudaSuccess) {
            rc = set_error(NB_ECUDA, "copy-out failed: %s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (pair_ms) *pair_ms = ms;
    } while (0);
    if (acc) cudaFree(acc);
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return rc;
}

int nb_tune(nb_ctx *c, int reps, nb_tune_t *out)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    if (reps < 1 || reps > 1000) return set_error(NB_EINVAL, "reps must be in [1, 1000]");
    if (c->n == 0) return set_error(NB_ESTATE, "nb_tune before nb_load");
    DeviceGuard dg(c->p.device);
    int rc = refresh_split(c);
    if (rc) return rc;
    TuneReport rep;
    Plan pl;
    rc = tune_pair(c->pool, c->set, c->p.precision, c->phys, c->stream, reps, rep, pl);
    if (rc) return rc;
    c->plan = pl;
    free_graphs(c);
    if (out) {
        out->precision = rep.precision;
        out->bodies_per_thread = rep.shape.I;
        out->blocks_per_sm = rep.shape.blocks_per_sm;
        out->j_tile = rep.shape.jt;
        out->candidates = rep.candidates;
        out->grid = rep.grid;
        out->pair_ms = rep.pair_ms;
        out->default_ms = rep.default_ms;
        out->cost_ms = rep.cost_ms;
        out->default_cost_ms = rep.default_cost_ms;
    }
    return NB_OK;
}

int nb_pair_shape(nb_ctx *c, int *bodies_per_thread, int *blocks_per_sm, int *j_tile,
                  int64_t *grid)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    if (c->n == 0 || !c->planned) return set_error(NB_ESTATE, "nothing loaded");
    if (bodies_per_thread) *bodies_per_thread = c->plan.pl.I;
    if (blocks_per_sm) *blocks_per_sm = c->plan.pl.blocks_per_sm;
    if (j_tile) *j_tile = c->plan.pl.d.jt;
    if (grid) *grid = c->plan.pl.d.G;
    return NB_OK;
}

int nb_tune_save(const char *path)
{
    if (!path) return set_error(NB_EINVAL, "path is NULL");
    return tune_save(path);
}

int64_t nb_tune_load(const char *path)
{
    if (!path) return set_error(NB_EINVAL, "path is NULL");
    int64_t n = 0;
    const int rc = tune_load(path, &n);
    return rc ? rc : n;
}

int64_t nb_tune_entries(void) { return tune_entries(); }

void nb_tune_clear(void) { tune_clear(); }

int nb_prof_enable(nb_ctx *c, int on)
{
    if (!c) return set_error(NB_EINVAL, "ctx is NULL");
    c->prof_on = on != 0;
    if (c->prof_on) std::memset(&c->prof, 0, sizeof c->prof);
    return NB_OK;
}

int nb_prof_read(nb_ctx *c, nb_prof_t *out)
{
    if (!c || !out) return set_error(NB_EINVAL, "NULL argument");
    *out = c->prof;
    return NB_OK;
}

}  // extern "C"
