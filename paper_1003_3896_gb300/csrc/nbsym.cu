// nbsym.cu -- host runtime behind the C ABI of include/nbsym.h.
//
// A context owns the device state of one particle system, its stream, the
// launch configuration of each kernel, and one CUDA graph per (order, dt)
// holding a whole integration step, replayed nsteps times by nb_step.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "nb_internal.cuh"
#include "../../include/nbsym.h"

using namespace nb;

namespace {

thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define NB_CUDA(call)                                                                     \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(NB_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
    } while (0)

// Sixth-order SI6A weights (Kinoshita, Yoshida & Nakai 1991, Table 1 first
// column = Yoshida's 1990 solution A); w0 = 1 - 2 (w1 + w2 + w3).
constexpr double SI6_W1 = -1.17767998417887;
constexpr double SI6_W2 = 0.235573213359357;
constexpr double SI6_W3 = 0.784513610477560;

struct StepGraph {
    int order = 0;
    double dt = 0;
    int precision = -1;
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
    DevState s;
    double *stage = nullptr;     // (7 cap) host-transfer staging on the device
    int num_sms = 0;
    bool loaded = false;
    bool split_stale = true;
    PairLaunch pl{};
    Decomp pot{};
    std::vector<StepGraph> graphs;
    bool prof_on = false;
    nb_prof_t prof{};
    cudaEvent_t pe0 = nullptr, pe1 = nullptr;   // direct-launch profiling events
};

namespace {

bool sp_mode(int precision) { return precision != NB_FP64; }

int pair_mode_of(int precision)
{
    switch (precision) {
    case NB_FP64: return PM_FP64;
    case NB_FP32: return PM_FP32;
    case NB_DS_FULL: return PM_DS_FULL;
    default: return PM_DS_NEAR;
    }
}

// Launch configuration of the pair kernel for n bodies: bodies per thread
// from the problem size, grid = resident blocks on every SM (persistent),
// capped so each block gets at least two units and the slot buffer suffices.
PairLaunch choose_pair(const nb_ctx *c, int mode, int64_t n)
{
    PairLaunch pl;
    pl.mode = mode;
    if (mode == PM_FP64)
        pl.I = 1;
    else
        // measured at N = 65536: mixed is fastest at 4 bodies per thread, pure
        // float (no near-pair test, fewer live registers) at 8
        pl.I = n < 16384 ? 2 : (mode == PM_FP32 ? 8 : 4);
    if (const char *env = getenv("NBSYM_PAIR_I")) {
        // tuning override: bodies per thread of the pair kernel
        const int I = atoi(env);
        if (pair_variant_exists(mode, I)) pl.I = I;
    }
    pl.blocks_per_sm = pair_occupancy(mode, pl.I);
    if (pl.blocks_per_sm < 1) pl.blocks_per_sm = 1;
    int64_t G = (int64_t)c->num_sms * pl.blocks_per_sm;
    Decomp d = make_decomp(n, TILE * pl.I, G);
    if (d.W / 2 < G) d = make_decomp(n, TILE * pl.I, d.W / 2 > 0 ? d.W / 2 : 1);
    while (d.max_slots() > c->s.part_slots && d.G > 1)
        d = make_decomp(n, TILE * pl.I, d.G - d.G / 8 - 1);
    pl.d = d;
    return pl;
}

Decomp choose_pot(const nb_ctx *c, int64_t n)
{
    int occ = pair_occupancy(PM_FP64, 1);
    if (occ < 1) occ = 1;
    Decomp d = make_decomp(n, TILE, (int64_t)c->num_sms * occ);
    if (d.W / 2 < d.G) d = make_decomp(n, TILE, d.W / 2 > 0 ? d.W / 2 : 1);
    while (d.max_slots() > c->s.part_slots && d.G > 1)
        d = make_decomp(n, TILE, d.G - d.G / 8 - 1);
    return d;
}

ExtField ext_of(const nb_params &p)
{
    ExtField e;
    e.on = p.ext_on;
    e.G = p.G;
    e.Md = p.Md;
    e.ad = p.ad;
    e.bd = p.bd;
    e.Mb = p.Mb;
    e.ab = p.ab;
    return e;
}

double near_frac_of(const nb_params &p) { return p.near_frac > 0 ? p.near_frac : 0.4; }

void free_graphs(nb_ctx *c)
{
    for (auto &g : c->graphs) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        if (g.graph) cudaGraphDestroy(g.graph);
        for (auto e : g.ev) cudaEventDestroy(e);
    }
    c->graphs.clear();
}

void free_state(nb_ctx *c)
{
    DevState &s = c->s;
    double *d64[] = {s.x, s.y, s.z, s.vx, s.vy, s.vz, s.m, s.part, s.red, s.diag, c->stage};
    for (double *q : d64)
        if (q) cudaFree(q);
    float *d32[] = {s.xh, s.yh, s.zh, s.mf, s.xl, s.yl, s.zl};
    for (float *q : d32)
        if (q) cudaFree(q);
    if (s.jd) cudaFree(s.jd);
    if (s.jl) cudaFree(s.jl);
    if (s.corr) cudaFree(s.corr);
    if (s.ng_key) cudaFree(s.ng_key);
    int *di[] = {s.ng_bucket, s.ng_entry, s.ng_count, s.ng_start, s.ng_bsum};
    for (int *q : di)
        if (q) cudaFree(q);
    if (s.frame) cudaFree(s.frame);
    if (s.flag) cudaFree(s.flag);
    s = DevState();
    c->stage = nullptr;
}

int check_params(const nb_params *p)
{
    if (!p) return fail(NB_EINVAL, "params is NULL");
    if (!finite_pos(p->G)) return fail(NB_EINVAL, "G must be finite and > 0");
    if (!std::isfinite(p->eps) || p->eps < 0) return fail(NB_EINVAL, "eps must be finite and >= 0");
    if (p->precision < NB_FP64 || p->precision > NB_DS_FULL)
        return fail(NB_EINVAL, "precision must be NB_FP64, NB_DS, NB_FP32 or NB_DS_FULL");
    if (p->ext_on) {
        if (!std::isfinite(p->Md) || p->Md < 0 || !std::isfinite(p->Mb) || p->Mb < 0 ||
            !std::isfinite(p->ad) || p->ad < 0 || !finite_pos(p->bd) || !finite_pos(p->ab))
            return fail(NB_EINVAL, "external field needs Md, Mb, ad >= 0 and bd, ab > 0");
    }
    if (!std::isfinite(p->near_frac)) return fail(NB_EINVAL, "near_frac must be finite");
    return NB_OK;
}

// Enqueue the float frame and split when the float planes are stale.
int refresh_split(nb_ctx *c)
{
    if (!sp_mode(c->p.precision) || !c->split_stale) return NB_OK;
    NB_CUDA(launch_frame(c->s, near_frac_of(c->p), c->p.eps, c->stream));
    NB_CUDA(launch_split(c->s, c->stream));
    c->split_stale = false;
    return NB_OK;
}

// The state as the consumers of the pair partial sums see it: the near-pair
// correction plane is added only in the mixed (NB_DS) mode.
DevState view(const nb_ctx *c)
{
    DevState s = c->s;
    if (c->p.precision != NB_DS) s.corr = nullptr;
    return s;
}

// Kernels enqueued by launch_near_correct (two memsets are not counted).
constexpr int64_t NEAR_KERNELS = 7;

int near_correct(nb_ctx *c)
{
    if (c->p.precision != NB_DS) return NB_OK;
    NB_CUDA(launch_near_correct(c->s, c->p.eps, c->p.G, c->stream));
    return NB_OK;
}

int launch_pair_timed(nb_ctx *c)
{
    if (c->prof_on) NB_CUDA(cudaEventRecord(c->pe0, c->stream));
    NB_CUDA(launch_pair(c->s, c->pl, c->p.G, c->p.eps, c->stream));
    if (c->prof_on) {
        NB_CUDA(cudaEventRecord(c->pe1, c->stream));
        NB_CUDA(cudaEventSynchronize(c->pe1));
        float ms = 0;
        NB_CUDA(cudaEventElapsedTime(&ms, c->pe0, c->pe1));
        c->prof.pair_launches += 1;
        c->prof.pair_ms += ms;
        c->prof.interactions += c->s.n * c->s.n;
        c->prof.kernel_launches += 1;
    }
    return NB_OK;
}

// Enqueue one whole step (the body of the captured graph).
int enqueue_step(nb_ctx *c, int order, double h, StepGraph *g)
{
    const bool sp = sp_mode(c->p.precision);
    const ExtField ext = ext_of(c->p);
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
    int64_t kernels = 0;
    if (sp) {
        NB_CUDA(launch_frame(c->s, near_frac_of(c->p), c->p.eps, c->stream));
        kernels += 2;
    }
    const DevState sv = view(c);
    // drift of the first leapfrog's half step (and the split it feeds)
    NB_CUDA(launch_kick_drift(sv, c->pl.d, 0.0, 0.5 * wk[0] * h, 0, sp ? 1 : 0, ext, c->p.G,
                              c->stream));
    kernels += 1;
    for (int k = 0; k < K; ++k) {
        // adjacent half drifts of consecutive leapfrogs merge
        const double hd = 0.5 * (wk[k] + (k + 1 < K ? wk[k + 1] : 0.0)) * h;
        const bool last = (k + 1 == K);
        if (g && g->prof)
            NB_CUDA(cudaEventRecordWithFlags(g->ev[2 * k], c->stream, cudaEventRecordExternal));
        NB_CUDA(launch_pair(c->s, c->pl, c->p.G, c->p.eps, c->stream));
        if (g && g->prof)
            NB_CUDA(cudaEventRecordWithFlags(g->ev[2 * k + 1], c->stream,
                                             cudaEventRecordExternal));
        int rc = near_correct(c);
        if (rc) return rc;
        if (c->p.precision == NB_DS) kernels += NEAR_KERNELS;
        NB_CUDA(launch_kick_drift(sv, c->pl.d, wk[k] * h, hd, 1, (sp && !last) ? 1 : 0, ext,
                                  c->p.G, c->stream));
        kernels += 2;
    }
    if (g) g->kernels = kernels;
    return NB_OK;
}

int get_graph(nb_ctx *c, int order, double h, StepGraph **out)
{
    const int prof = c->prof_on ? 1 : 0;
    for (auto &g : c->graphs)
        if (g.order == order && g.dt == h && g.precision == c->p.precision && g.prof == prof) {
            *out = &g;
            return NB_OK;
        }
    StepGraph g;
    g.order = order;
    g.dt = h;
    g.precision = c->p.precision;
    g.prof = prof;
    if (prof) {
        const int K = order == 2 ? 1 : 7;
        g.ev.resize(2 * K);
        for (auto &e : g.ev) NB_CUDA(cudaEventCreate(&e));
    }
    NB_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue_step(c, order, h, &g);
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
    if (rc != NB_OK || e != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        for (auto ev : g.ev) cudaEventDestroy(ev);
        if (rc != NB_OK) return rc;
        return fail(NB_ECUDA, "stream capture failed: %s", cudaGetErrorString(e));
    }
    g.graph = graph;
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(graph);
        for (auto ev : g.ev) cudaEventDestroy(ev);
        return fail(NB_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    }
    // keep the cache small: one graph per (order, dt, precision, prof)
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

int configure(nb_ctx *c)
{
    if (c->s.n <= 0) return NB_OK;
    c->pl = choose_pair(c, pair_mode_of(c->p.precision), c->s.n);
    c->pot = choose_pot(c, c->s.n);
    free_graphs(c);
    return NB_OK;
}

int check_flag(nb_ctx *c, const char *what)
{
    int h = 0;
    NB_CUDA(cudaMemcpyAsync(&h, c->s.flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    NB_CUDA(cudaStreamSynchronize(c->stream));
    if (h) return fail(NB_ENONFINITE, "%s: non-finite values (coincident bodies with eps = 0?)", what);
    return NB_OK;
}

}  // namespace

extern "C" {

int nb_abi_version(void) { return NB_ABI_VERSION; }

const char *nb_last_error(void) { return g_err.c_str(); }

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
    if (!out) return fail(NB_EINVAL, "out is NULL");
    *out = nullptr;
    int rc = check_params(p);
    if (rc) return rc;
    if (n_capacity < 1 || n_capacity > ((int64_t)1 << 26))
        return fail(NB_EINVAL, "n_capacity must be in [1, 2^26]");
    int ndev = 0;
    NB_CUDA(cudaGetDeviceCount(&ndev));
    if (p->device < 0 || p->device >= ndev) return fail(NB_EINVAL, "no CUDA device %d", p->device);
    DeviceGuard dg(p->device);
    nb_ctx *c = new (std::nothrow) nb_ctx();
    if (!c) return fail(NB_ENOMEM, "host allocation failed");
    c->p = *p;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, p->device);
    if (e != cudaSuccess) {
        delete c;
        return fail(NB_ECUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    }
    c->num_sms = prop.multiProcessorCount;
    if (p->stream) {
        c->stream = (cudaStream_t)p->stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            delete c;
            return fail(NB_ECUDA, "cudaStreamCreate: %s", cudaGetErrorString(e));
        }
        c->own_stream = true;
    }
    DevState &s = c->s;
    s.cap = n_capacity;
    // slot planes: enough for the finest decomposition any mode picks
    const int64_t iblocks_min = (n_capacity + 4 * TILE - 1) / (4 * TILE);
    const int64_t gmax = (int64_t)c->num_sms * 16;
    int64_t slots = (gmax + iblocks_min - 1) / iblocks_min + 2;
    if (slots > 64) slots = 64;
    if (slots < 4) slots = 4;
    s.part_slots = slots;
    s.red_len = 16 * reduce_blocks();
    bool ok = true;
    auto A64 = [&](double **q, int64_t cnt) {
        if (ok && cudaMalloc(q, (size_t)cnt * sizeof(double)) != cudaSuccess) ok = false;
    };
    auto A32 = [&](float **q, int64_t cnt) {
        if (ok && cudaMalloc(q, (size_t)cnt * sizeof(float)) != cudaSuccess) ok = false;
    };
    A64(&s.x, s.cap); A64(&s.y, s.cap); A64(&s.z, s.cap);
    A64(&s.vx, s.cap); A64(&s.vy, s.cap); A64(&s.vz, s.cap); A64(&s.m, s.cap);
    A32(&s.xh, s.cap); A32(&s.yh, s.cap); A32(&s.zh, s.cap); A32(&s.mf, s.cap);
    A32(&s.xl, s.cap); A32(&s.yl, s.cap); A32(&s.zl, s.cap);
    A64(&s.part, s.part_slots * 3 * s.cap);
    A64(&s.red, s.red_len);
    A64(&s.diag, 16);
    A64(&c->stage, 7 * s.cap);
    if (ok && cudaMalloc(&s.jd, (size_t)(2 * s.cap) * sizeof(float4)) != cudaSuccess) ok = false;
    if (ok && cudaMalloc(&s.jl, (size_t)(2 * s.cap) * sizeof(float4)) != cudaSuccess) ok = false;
    // near-pair correction: correction planes and the hash grid
    s.ng_hcap = near_table_size(s.cap);
    A64(&s.corr, 3 * s.cap);
    auto AI = [&](int **q, int64_t cnt) {
        if (ok && cudaMalloc(q, (size_t)cnt * sizeof(int)) != cudaSuccess) ok = false;
    };
    AI(&s.ng_bucket, s.cap);
    AI(&s.ng_entry, s.cap);
    AI(&s.ng_count, s.ng_hcap);
    AI(&s.ng_start, s.ng_hcap + 1);
    AI(&s.ng_bsum, s.ng_hcap / 1024 + 1);
    if (ok && cudaMalloc(&s.ng_key, (size_t)s.cap * sizeof(uint64_t)) != cudaSuccess) ok = false;
    if (ok && cudaMalloc(&s.frame, sizeof(Frame)) != cudaSuccess) ok = false;
    if (ok && cudaMalloc(&s.flag, sizeof(int)) != cudaSuccess) ok = false;
    if (ok && cudaEventCreate(&c->pe0) != cudaSuccess) ok = false;
    if (ok && cudaEventCreate(&c->pe1) != cudaSuccess) ok = false;
    if (!ok) {
        cudaGetLastError();
        nb_destroy(c);
        return fail(NB_ENOMEM, "device allocation failed for capacity %lld",
                    (long long)n_capacity);
    }
    *out = c;
    return NB_OK;
}

void nb_destroy(nb_ctx *c)
{
    if (!c) return;
    DeviceGuard dg(c->p.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    free_graphs(c);
    free_state(c);
    if (c->pe0) cudaEventDestroy(c->pe0);
    if (c->pe1) cudaEventDestroy(c->pe1);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

static int load_common(nb_ctx *c, int64_t n, const double *pos, const double *vel,
                       const double *mass, cudaMemcpyKind kind)
{
    if (!c) return fail(NB_EINVAL, "ctx is NULL");
    if (!pos || !vel || !mass) return fail(NB_EINVAL, "pos, vel and mass must be non-NULL");
    if (n < 1 || n > c->s.cap) return fail(NB_EINVAL, "n=%lld outside [1, capacity=%lld]",
                                            (long long)n, (long long)c->s.cap);
    DeviceGuard dg(c->p.device);
    const bool reconf = (c->s.n != n);
    c->s.n = n;
    const double *dp = pos, *dv = vel, *dm = mass;
    if (kind == cudaMemcpyHostToDevice) {
        double *sp = c->stage, *sv = c->stage + 3 * c->s.cap, *sm = c->stage + 6 * c->s.cap;
        NB_CUDA(cudaMemcpyAsync(sp, pos, (size_t)(3 * n) * sizeof(double), kind, c->stream));
        NB_CUDA(cudaMemcpyAsync(sv, vel, (size_t)(3 * n) * sizeof(double), kind, c->stream));
        NB_CUDA(cudaMemcpyAsync(sm, mass, (size_t)n * sizeof(double), kind, c->stream));
        dp = sp;
        dv = sv;
        dm = sm;
    }
    NB_CUDA(launch_unpack(c->s, dp, dv, dm, c->stream));
    NB_CUDA(cudaStreamSynchronize(c->stream));
    c->loaded = true;
    c->split_stale = true;
    if (reconf) return configure(c);
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

static int accel_common(nb_ctx *c, double *out, bool host)
{
    if (!c) return fail(NB_EINVAL, "ctx is NULL");
    if (!out) return fail(NB_EINVAL, "acc_out is NULL");
    if (!c->loaded) return fail(NB_ESTATE, "nb_accel before nb_load");
    DeviceGuard dg(c->p.device);
    int rc = refresh_split(c);
    if (rc) return rc;
    rc = launch_pair_timed(c);
    if (rc) return rc;
    rc = near_correct(c);
    if (rc) return rc;
    if (c->prof_on && c->p.precision == NB_DS) c->prof.kernel_launches += NEAR_KERNELS + 1;
    NB_CUDA(cudaMemsetAsync(c->s.flag, 0, sizeof(int), c->stream));
    double *dst = host ? c->stage : out;
    NB_CUDA(launch_accel_out(view(c), c->pl.d, ext_of(c->p), c->p.G, dst, c->stream));
    if (host)
        NB_CUDA(cudaMemcpyAsync(out, dst, (size_t)(3 * c->s.n) * sizeof(double),
                                cudaMemcpyDeviceToHost, c->stream));
    return check_flag(c, "nb_accel");
}

int nb_accel(nb_ctx *c, double *acc_out) { return accel_common(c, acc_out, true); }

int nb_accel_device(nb_ctx *c, double *d_acc_out) { return accel_common(c, d_acc_out, false); }

int nb_step(nb_ctx *c, int order, double dt, int64_t nsteps)
{
    if (!c) return fail(NB_EINVAL, "ctx is NULL");
    if (order != 2 && order != 6) return fail(NB_EINVAL, "order must be 2 or 6");
    if (!finite_pos(dt)) return fail(NB_EINVAL, "dt must be finite and > 0");
    if (nsteps < 0) return fail(NB_EINVAL, "nsteps must be >= 0");
    if (!c->loaded) return fail(NB_ESTATE, "nb_step before nb_load");
    if (nsteps == 0) return NB_OK;
    DeviceGuard dg(c->p.device);
    StepGraph *g = nullptr;
    int rc = get_graph(c, order, dt, &g);
    if (rc) return rc;
    for (int64_t k = 0; k < nsteps; ++k) {
        NB_CUDA(cudaGraphLaunch(g->exec, c->stream));
        if (c->prof_on) {
            NB_CUDA(cudaStreamSynchronize(c->stream));
            for (size_t q = 0; q + 1 < g->ev.size(); q += 2) {
                float ms = 0;
                NB_CUDA(cudaEventElapsedTime(&ms, g->ev[q], g->ev[q + 1]));
                c->prof.pair_ms += ms;
                c->prof.pair_launches += 1;
                c->prof.interactions += c->s.n * c->s.n;
            }
            c->prof.kernel_launches += g->kernels;
        }
    }
    NB_CUDA(cudaStreamSynchronize(c->stream));
    c->split_stale = true;
    return NB_OK;
}

int nb_energy(nb_ctx *c, nb_energy_t *out)
{
    if (!c) return fail(NB_EINVAL, "ctx is NULL");
    if (!out) return fail(NB_EINVAL, "out is NULL");
    if (!c->loaded) return fail(NB_ESTATE, "nb_energy before nb_load");
    DeviceGuard dg(c->p.device);
    NB_CUDA(cudaMemsetAsync(c->s.flag, 0, sizeof(int), c->stream));
    NB_CUDA(launch_potential(c->s, c->pot, c->p.eps, c->stream));
    NB_CUDA(launch_energy_reduce(c->s, c->pot, ext_of(c->p), c->p.G, c->stream));
    double d[10];
    NB_CUDA(cudaMemcpyAsync(d, c->s.diag, sizeof d, cudaMemcpyDeviceToHost, c->stream));
    int rc = check_flag(c, "nb_energy");
    if (c->prof_on) c->prof.kernel_launches += 3;
    out->K = d[0];
    out->W = d[1];
    out->W_ext = d[2];
    out->E = d[3];
    for (int k = 0; k < 3; ++k) {
        out->P[k] = d[4 + k];
        out->L[k] = d[7 + k];
    }
    return rc;
}

int nb_torque(nb_ctx *c, double *out)
{
    if (!c) return fail(NB_EINVAL, "ctx is NULL");
    if (!out) return fail(NB_EINVAL, "out is NULL");
    if (!c->loaded) return fail(NB_ESTATE, "nb_torque before nb_load");
    DeviceGuard dg(c->p.device);
    if (!c->p.ext_on) {
        out[0] = out[1] = out[2] = 0.0;
        return NB_OK;
    }
    NB_CUDA(launch_torque(c->s, ext_of(c->p), c->stream));
    NB_CUDA(cudaMemcpyAsync(out, c->s.diag + 10, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                            c->stream));
    NB_CUDA(cudaStreamSynchronize(c->stream));
    return NB_OK;
}

static int state_common(nb_ctx *c, double *pos, double *vel, bool host)
{
    if (!c) return fail(NB_EINVAL, "ctx is NULL");
    if (!c->loaded) return fail(NB_ESTATE, "nb_get_state before nb_load");
    if (!pos && !vel) return NB_OK;
    DeviceGuard dg(c->p.device);
    const int64_t n = c->s.n;
    double *dp = pos, *dv = vel;
    if (host) {
        dp = pos ? c->stage : nullptr;
        dv = vel ? c->stage + 3 * c->s.cap : nullptr;
    }
    NB_CUDA(launch_pack(c->s, dp, dv, c->stream));
    if (host) {
        if (pos)
            NB_CUDA(cudaMemcpyAsync(pos, dp, (size_t)(3 * n) * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream));
        if (vel)
            NB_CUDA(cudaMemcpyAsync(vel, dv, (size_t)(3 * n) * sizeof(double),
                                    cudaMemcpyDeviceToHost, c->stream));
    }
    NB_CUDA(cudaStreamSynchronize(c->stream));
    return NB_OK;
}

int nb_get_state(nb_ctx *c, double *pos, double *vel) { return state_common(c, pos, vel, true); }

int nb_get_state_device(nb_ctx *c, double *pos, double *vel)
{
    return state_common(c, pos, vel, false);
}

int64_t nb_size(const nb_ctx *c)
{
    if (!c) return NB_EINVAL;
    return c->loaded ? c->s.n : 0;
}

int nb_set_precision(nb_ctx *c, int precision)
{
    if (!c) return fail(NB_EINVAL, "ctx is NULL");
    if (precision < NB_FP64 || precision > NB_DS_FULL) return fail(NB_EINVAL, "bad precision");
    DeviceGuard dg(c->p.device);
    c->p.precision = precision;
    c->split_stale = true;
    return configure(c);
}

int nb_prof_enable(nb_ctx *c, int on)
{
    if (!c) return fail(NB_EINVAL, "ctx is NULL");
    c->prof_on = on != 0;
    if (c->prof_on) std::memset(&c->prof, 0, sizeof c->prof);
    return NB_OK;
}

int nb_prof_read(nb_ctx *c, nb_prof_t *out)
{
    if (!c || !out) return fail(NB_EINVAL, "NULL argument");
    *out = c->prof;
    return NB_OK;
}

}  // extern "C"
