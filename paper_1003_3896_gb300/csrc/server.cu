// server.cu -- the serving loop: integration jobs of different size, order
// and precision share one GPU by continuous batching.
//
// A scheduler thread owns the device.  Submitted jobs wait in a FIFO queue;
// a job is admitted when a resident-job slot is free and a contiguous range
// of the state pool (sized from the HBM budget) can hold its bodies.  Its
// initial conditions are then uploaded into that range.  Resident jobs are
// grouped by (precision, order, size class); each group is one cluster set of the engine
// (one cluster per job, with the job's softening and step length), advanced
// one step at a time by one pair-kernel launch per force evaluation on the
// group's own stream, so the groups' work overlaps on the device.  Between two
// steps of a group, finished jobs leave it (their state is copied back and
// their pool range freed) and newly admitted jobs join it.  A job whose state
// is not finite when it finishes is failed alone.  A group moves all its jobs
// in lockstep, so jobs below SMALL_JOB bodies are grouped apart from larger
// ones: a small job then waits at each step for other small jobs only, not
// for a step of a 131072-body job (on the bounded serving trace this lowered
// the median latency by 7-11% at the same throughput).  The small jobs'
// groups enqueue on streams of the device's greatest priority, the others on
// its least: when both have kernels ready, the block scheduler hands SMs to
// the small jobs' blocks first, which approximates shortest job first on the
// device (bounded trace: median latency 6.3-6.6 -> 3.5-3.7 s, p99 and
// throughput unchanged or slightly better).
//
// Up to two steps of a group are in flight: the next one is enqueued while
// the current one runs whenever no member finishes at the current one and no
// job waits to join or leave, so the group's stream does not idle while the
// scheduler notices a finished step.  (Steps are enqueued kernel by kernel:
// a step graph per group, captured again at each membership change, made the
// served trace slower, since its jobs join and leave at every few steps.)
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "engine.h"
#include "range_alloc.h"

using namespace nb;

namespace {

using Clock = std::chrono::steady_clock;

struct Job {
    int64_t id = 0;
    nb_job_desc d{};
    std::vector<double> pos, vel, mass;   // initial conditions, then the result
    double mu = 0;                        // the common mass of its bodies (0: they differ)
    int state = NB_JOB_QUEUED;
    int64_t steps_done = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int64_t off = -1;                     // pool range start while resident
    int group = -1;
    bool cancel = false;
    std::string error;
};

// One of a group's two step buffers: its pair-launch timing events, its
// completion event and what it stepped.
struct StepSlot {
    cudaEvent_t done = nullptr;
    std::vector<cudaEvent_t> ev;          // (start, stop) of each pair launch of the step
    std::vector<int64_t> stepping;        // members of the step in flight
    int64_t step_pairs = 0;               // interactions of that step
};

struct Group {
    int precision = 0, order = 2;
    cudaStream_t stream = nullptr;
    ClusterSet set;
    Plan plan;
    std::vector<int64_t> members;         // job ids in the current set
    bool dirty = true;                    // membership changed since the last layout
    StepSlot slot[2];
    int head = 0;                         // oldest step in flight
    int nflight = 0;                      // steps in flight (0, 1 or 2)
};

constexpr size_t PAIR_IV_CAP = (size_t)1 << 20;

// Jobs with fewer bodies than this form their own groups.
constexpr int64_t SMALL_JOB = 16384;
constexpr int NGROUPS = 12;               // (FP64, NB_DS, NB_DD) x (order 2, 6) x (small, large)

// Bytes of device memory the pool and the group scratch use per body slot:
// state, float planes, j-stream, near-pair correction, staging, near-pair
// scratch; plus the groups' partial sums, 2 x 24 bytes per body of a group
// beyond a fixed part of at most 3 x 8 x SMs x 6 x 3072 bytes per group.
constexpr double BYTES_PER_BODY = 7 * 8 + 7 * 4 + 64 + 2 * 3 * 8 + 3 * 8 + 7 * 8 + 5 * (16 + 16);

}  // namespace

struct nb_server {
    nb_server_params p{};
    Phys phys;
    Pool pool;
    RangeAlloc ranges;
    int64_t cap = 0;
    Group groups[NGROUPS];
    ClusterSet io;                        // one-cluster set for uploads and downloads
    cudaStream_t io_stream = nullptr;
    std::mutex mu;
    std::condition_variable cv;
    std::map<int64_t, std::unique_ptr<Job>> jobs;
    std::deque<int64_t> queue;
    int64_t next_id = 1;
    int resident = 0;
    bool stop = false;
    std::thread thr;
    Clock::time_point t0;
    nb_server_stats_t stats{};
    std::string fatal;
    // device-time intervals [start, end) of the pair launches, ms after the
    // reference event, by arithmetic (the first PAIR_IV_CAP of each)
    cudaEvent_t ref = nullptr;
    std::vector<std::pair<float, float>> iv[3];
};

namespace {

double now_s(const nb_server *s)
{
    return std::chrono::duration<double>(Clock::now() - s->t0).count();
}

// Group of a job: its arithmetic (FP64 jobs run float-float when the server
// was created with fp64_via_dd), its order and its size class.
int group_index(const nb_server *s, int precision, int order, int64_t n)
{
    if (precision == NB_FP64 && s->p.fp64_via_dd) precision = NB_DD;
    const int a = precision == NB_FP64 ? 0 : (precision == NB_DS ? 1 : 2);
    return 4 * a + 2 * (order == 6 ? 1 : 0) + (n < SMALL_JOB ? 0 : 1);
}

// Copy a job's interleaved host arrays into its pool range (io stream).
int upload(nb_server *s, Job &j)
{
    const int64_t n = j.d.n;
    const int64_t off = j.off;
    const int64_t nk = n;
    const double e = j.d.eps, one = 1.0;
    int rc = set_define(s->io, 1, &off, &nk, &e, &one);
    if (!rc) rc = set_layout(s->io, TILE, s->io_stream);
    if (rc) return rc;
    double *sp = s->pool.stage + 7 * off, *sv = sp + 3 * n, *sm = sp + 6 * n;
    NB_TRY(cudaMemcpyAsync(sp, j.pos.data(), 3 * n * 8, cudaMemcpyHostToDevice, s->io_stream));
    NB_TRY(cudaMemcpyAsync(sv, j.vel.data(), 3 * n * 8, cudaMemcpyHostToDevice, s->io_stream));
    NB_TRY(cudaMemcpyAsync(sm, j.mass.data(), n * 8, cudaMemcpyHostToDevice, s->io_stream));
    NB_TRY(launch_unpack(view(s->pool, s->io, NB_FP64), sp, sv, sm, s->io_stream));
    NB_TRY(cudaStreamSynchronize(s->io_stream));
    return NB_OK;
}

int download(nb_server *s, Job &j)
{
    const int64_t n = j.d.n;
    const int64_t off = j.off, nk = n;
    const double e = j.d.eps, one = 1.0;
    int rc = set_define(s->io, 1, &off, &nk, &e, &one);
    if (!rc) rc = set_layout(s->io, TILE, s->io_stream);
    if (rc) return rc;
    double *sp = s->pool.stage + 7 * off, *sv = sp + 3 * n;
    NB_TRY(launch_pack(view(s->pool, s->io, NB_FP64), sp, sv, s->io_stream));
    NB_TRY(cudaMemcpyAsync(j.pos.data(), sp, 3 * n * 8, cudaMemcpyDeviceToHost, s->io_stream));
    NB_TRY(cudaMemcpyAsync(j.vel.data(), sv, 3 * n * 8, cudaMemcpyDeviceToHost, s->io_stream));
    NB_TRY(cudaStreamSynchronize(s->io_stream));
    return NB_OK;
}

void finish(nb_server *s, Job &j, int state, const char *err)
{
    if (j.off >= 0) {
        s->ranges.release(j.off, j.d.n);
        j.off = -1;
        --s->resident;
    }
    j.state = state;
    j.t_done = now_s(s);
    if (err) j.error = err;
    if (state == NB_JOB_DONE) ++s->stats.completed;
    if (state == NB_JOB_FAILED) ++s->stats.failed;
    if (state == NB_JOB_CANCELLED) ++s->stats.cancelled;
    --s->stats.running;
}

// Admit queued jobs in arrival order while a slot and a pool range are free.
// Called with the lock held; uploads run with it held too (short).
void admit(nb_server *s)
{
    while (!s->queue.empty() && s->resident < s->p.max_jobs) {
        Job &j = *s->jobs[s->queue.front()];
        if (j.cancel) {
            s->queue.pop_front();
            j.state = NB_JOB_CANCELLED;
            j.t_done = now_s(s);
            ++s->stats.cancelled;
            --s->stats.queued;
            continue;
        }
        const int64_t off = s->ranges.alloc(j.d.n);
        if (off < 0) break;   // strict FIFO: the head waits for room
        s->queue.pop_front();
        j.off = off;
        ++s->resident;
        --s->stats.queued;
        ++s->stats.running;
        ++s->stats.admitted;
        j.t_admit = now_s(s);
        const int rc = upload(s, j);
        if (rc) {
            finish(s, j, NB_JOB_FAILED, last_error());
            continue;
        }
        j.state = NB_JOB_RUNNING;
        j.group = group_index(s, j.d.precision, j.d.order, j.d.n);
        Group &g = s->groups[j.group];
        g.members.push_back(j.id);
        g.dirty = true;
    }
}

// The oldest step in flight of group g has completed: count it; when no
// other step is in flight, retire finished or cancelled jobs.
void complete_step(nb_server *s, Group &g)
{
    StepSlot &sl = g.slot[g.head];
    g.head ^= 1;
    --g.nflight;
    s->stats.interactions += (double)sl.step_pairs;
    // device time of the step's pair launches, by arithmetic
    const int a = g.precision == NB_FP64 ? 0 : (g.precision == NB_DS ? 1 : 2);
    for (int q = 0; q < (g.order == 6 ? 7 : 1); ++q) {
        float ms = 0.f, t0 = 0.f, t1 = 0.f;
        if (cudaEventElapsedTime(&ms, sl.ev[2 * q], sl.ev[2 * q + 1]) == cudaSuccess)
            s->stats.pair_ms[a] += ms;
        if (s->iv[a].size() < PAIR_IV_CAP &&
            cudaEventElapsedTime(&t0, s->ref, sl.ev[2 * q]) == cudaSuccess &&
            cudaEventElapsedTime(&t1, s->ref, sl.ev[2 * q + 1]) == cudaSuccess)
            s->iv[a].emplace_back(t0, t1);
    }
    s->stats.pair_interactions[a] += (double)sl.step_pairs;
    for (int64_t id : sl.stepping) {
        Job &j = *s->jobs[id];
        ++j.steps_done;
    }
    // a second step was enqueued only if nobody finishes at this one; a
    // cancelled job leaves once nothing of its group is in flight
    if (g.nflight > 0) return;
    std::vector<int64_t> keep;
    for (int64_t id : g.members) {
        Job &j = *s->jobs[id];
        if (j.cancel) {
            finish(s, j, NB_JOB_CANCELLED, nullptr);
            g.dirty = true;
            continue;
        }
        if (j.steps_done >= j.d.nsteps) {
            int rc = download(s, j);
            bool finite = rc == NB_OK;
            for (size_t q = 0; finite && q < j.pos.size(); ++q)
                finite = std::isfinite(j.pos[q]) && std::isfinite(j.vel[q]);
            if (rc)
                finish(s, j, NB_JOB_FAILED, last_error());
            else if (!finite)
                finish(s, j, NB_JOB_FAILED, "state became non-finite");
            else
                finish(s, j, NB_JOB_DONE, nullptr);
            g.dirty = true;
            continue;
        }
        keep.push_back(id);
    }
    g.members.swap(keep);
}

// Whether the step after the one in flight may be enqueued now: the layout
// is current, nobody waits to join, and no member finishes or is cancelled
// at the step in flight.
bool can_enqueue_ahead(const nb_server *s, const Group &g)
{
    if (g.nflight != 1 || g.dirty) return false;
    for (int64_t id : g.members) {
        const Job &j = *s->jobs.at(id);
        if (j.cancel || j.steps_done + 1 >= j.d.nsteps) return false;
    }
    return true;
}

// Enqueue the next step of group g (lock held: the tables are rebuilt from
// the job records when the membership changed, which happens only with no
// step of the group in flight).
int launch_step(nb_server *s, Group &g)
{
    if (g.members.empty()) return NB_OK;
    if (g.dirty) {
        std::vector<int64_t> boff, nk;
        std::vector<double> eps, dts, mu;
        for (int64_t id : g.members) {
            const Job &j = *s->jobs[id];
            boff.push_back(j.off);
            nk.push_back(j.d.n);
            eps.push_back(j.d.eps);
            dts.push_back(j.d.dt);
            mu.push_back(j.mu);
        }
        int rc = set_define(g.set, (int32_t)nk.size(), boff.data(), nk.data(), eps.data(),
                            dts.data());
        g.set.mu = mu;
        // the group's own partial sums: groups step concurrently
        if (!rc) rc = set_reserve_part(g.set, part_elems_for(s->pool, g.set.n), g.stream);
        // the large jobs' groups: the most waves, so their blocks are short
        // and free SM slots for the small jobs' kernels sooner
        const bool large = ((&g - s->groups) & 1) != 0;
        if (!rc)
            rc = plan_make(s->pool, g.set, g.precision, g.stream, g.plan, nullptr, true,
                           large ? MAX_WAVES : 0);
        if (rc) return rc;
        g.dirty = false;
    }
    StepSlot &sl = g.slot[(g.head + g.nflight) & 1];
    int64_t k = 0;
    const int rc = enq_step(s->pool, g.set, g.plan, s->phys, g.order, 1.0, g.stream, &sl.ev, &k);
    if (rc) return rc;
    NB_TRY(cudaEventRecord(sl.done, g.stream));
    ++g.nflight;
    sl.stepping = g.members;
    sl.step_pairs = 0;
    for (int64_t q = 0; q < g.set.K; ++q)
        sl.step_pairs += g.set.nk[q] * g.set.nk[q] * (g.order == 6 ? 7 : 1);
    s->stats.kernel_launches += k;
    return NB_OK;
}

void fail_all(nb_server *s, const char *why)
{
    for (auto &g : s->groups) {
        for (int64_t id : g.members) finish(s, *s->jobs[id], NB_JOB_FAILED, why);
        g.members.clear();
        g.nflight = 0;
        g.dirty = true;
    }
}

void run(nb_server *s)
{
    cudaSetDevice(s->p.device);
    std::unique_lock<std::mutex> lk(s->mu);
    while (!s->stop) {
        admit(s);
        bool busy = false;
        for (auto &g : s->groups) {
            bool failed = false;
            while (g.nflight > 0) {
                const cudaError_t q = cudaEventQuery(g.slot[g.head].done);
                if (q == cudaErrorNotReady) break;
                if (q != cudaSuccess) {
                    s->fatal = cudaGetErrorString(q);
                    fail_all(s, s->fatal.c_str());
                    failed = true;
                    break;
                }
                complete_step(s, g);
                if (g.nflight == 0) admit(s);
            }
            if (failed) continue;
            if (!g.members.empty() && (g.nflight == 0 || can_enqueue_ahead(s, g))) {
                const int rc = launch_step(s, g);
                if (rc) {
                    s->fatal = last_error();
                    fail_all(s, s->fatal.c_str());
                    continue;
                }
            }
            if (g.nflight > 0) busy = true;
        }
        s->cv.notify_all();
        if (busy) {
            // a step is running: poll again shortly without holding the lock
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(50));
            lk.lock();
        } else {
            s->cv.wait_for(lk, std::chrono::milliseconds(2));
        }
    }
}

bool valid_desc(const nb_server *s, const nb_job_desc *d)
{
    return d && d->n >= 1 && d->n <= s->cap && (d->order == 2 || d->order == 6) &&
           (d->precision == NB_FP64 || d->precision == NB_DS || d->precision == NB_DD) &&
           std::isfinite(d->dt) && d->dt > 0 && d->nsteps >= 1 && std::isfinite(d->eps) &&
           d->eps >= 0;
}

}  // namespace

extern "C" {

void nb_server_params_default(nb_server_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof *p);
    p->device = 0;
    p->hbm_budget_bytes = 4.0e9;
    p->max_jobs = 64;
    p->G = 1.0;
    p->Md = 100.0;
    p->ad = 6.5;
    p->bd = 0.26;
    p->Mb = 15.0;
    p->ab = 0.7;
    p->fp64_via_dd = 1;
}

int nb_server_create(const nb_server_params *p, nb_server **out)
{
    if (!out) return set_error(NB_EINVAL, "out is NULL");
    *out = nullptr;
    if (!p || !(p->hbm_budget_bytes > 0) || p->max_jobs < 1 || p->max_jobs > (1 << 16) ||
        !(p->G > 0) || (p->ext_on && !(p->bd > 0 && p->ab > 0)) || !(p->Mbh >= 0) ||
        !std::isfinite(p->Mbh) || !(p->eps_bh >= 0) || !std::isfinite(p->eps_bh))
        return set_error(NB_EINVAL, "bad server parameters");
    int ndev = 0;
    NB_TRY(cudaGetDeviceCount(&ndev));
    if (p->device < 0 || p->device >= ndev) return set_error(NB_EINVAL, "no CUDA device %d", p->device);
    NB_TRY(cudaSetDevice(p->device));
    nb_server *s = new (std::nothrow) nb_server();
    if (!s) return set_error(NB_ENOMEM, "host allocation failed");
    s->p = *p;
    s->phys.G = p->G;
    s->phys.near_frac = p->near_frac > 0 ? p->near_frac : 0.4;
    s->phys.ext.on = p->ext_on;
    s->phys.ext.G = p->G;
    s->phys.ext.Md = p->Md;
    s->phys.ext.ad = p->ad;
    s->phys.ext.bd = p->bd;
    s->phys.ext.Mb = p->Mb;
    s->phys.ext.ab = p->ab;
    s->phys.ext.Mbh = p->Mbh;
    s->phys.ext.eps2bh = p->eps_bh * p->eps_bh;
    int64_t cap = (int64_t)(p->hbm_budget_bytes / BYTES_PER_BODY);
    if (cap > ((int64_t)1 << 26)) cap = (int64_t)1 << 26;
    if (cap < 1) {
        delete s;
        return set_error(NB_EINVAL, "HBM budget too small for one body");
    }
    s->cap = cap;
    int rc = pool_create(s->pool, p->device, cap, /*own_part=*/false);
    int least = 0, greatest = 0;
    if (!rc && cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess)
        rc = set_error(NB_ECUDA, "stream priority query failed");
    for (int g = 0; g < NGROUPS && !rc; ++g) {
        Group &gr = s->groups[g];
        gr.precision = g < 4 ? NB_FP64 : (g < 8 ? NB_DS : NB_DD);
        gr.order = (g & 2) ? 6 : 2;
        const int prio = (g & 1) ? least : greatest;   // the small jobs' groups first
        rc = set_create(gr.set, p->max_jobs, cap, prio);
        if (!rc && cudaStreamCreateWithPriority(&gr.stream, cudaStreamNonBlocking, prio) != cudaSuccess)
            rc = set_error(NB_ECUDA, "stream creation failed");
        for (StepSlot &sl : gr.slot) {
            if (!rc && cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess)
                rc = set_error(NB_ECUDA, "event creation failed");
            sl.ev.assign(14, nullptr);   // 7 force evaluations per step at most
            for (auto &e : sl.ev)
                if (!rc && cudaEventCreate(&e) != cudaSuccess)
                    rc = set_error(NB_ECUDA, "event creation failed");
        }
    }
    if (!rc) rc = set_create(s->io, 1, cap);
    // uploads and downloads are synchronised by the scheduler thread, which
    // feeds no group while it waits: their pack / unpack kernels go first
    if (!rc && cudaStreamCreateWithPriority(&s->io_stream, cudaStreamNonBlocking, greatest) != cudaSuccess)
        rc = set_error(NB_ECUDA, "stream creation failed");
    if (!rc && (cudaEventCreate(&s->ref) != cudaSuccess ||
                cudaEventRecord(s->ref, s->io_stream) != cudaSuccess ||
                cudaEventSynchronize(s->ref) != cudaSuccess))
        rc = set_error(NB_ECUDA, "reference event failed");
    if (rc) {
        nb_server_destroy(s);
        return rc;
    }
    s->ranges = RangeAlloc(cap);
    s->t0 = Clock::now();
    s->thr = std::thread(run, s);
    *out = s;
    return NB_OK;
}

void nb_server_destroy(nb_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv.notify_all();
    if (s->thr.joinable()) s->thr.join();
    cudaSetDevice(s->p.device);
    for (auto &g : s->groups) {
        if (g.stream) cudaStreamSynchronize(g.stream);
        set_destroy(g.set);
        for (StepSlot &sl : g.slot) {
            if (sl.done) cudaEventDestroy(sl.done);
            for (auto e : sl.ev)
                if (e) cudaEventDestroy(e);
        }
        if (g.stream) cudaStreamDestroy(g.stream);
    }
    set_destroy(s->io);
    if (s->io_stream) cudaStreamDestroy(s->io_stream);
    if (s->ref) cudaEventDestroy(s->ref);
    pool_destroy(s->pool);
    delete s;
}

int nb_server_submit(nb_server *s, const nb_job_desc *d, const double *pos, const double *vel,
                     const double *mass, int64_t *job_id)
{
    if (!s || !job_id || !pos || !vel || !mass) return set_error(NB_EINVAL, "NULL argument");
    if (!valid_desc(s, d))
        return set_error(NB_EINVAL, "bad job: need 1 <= n <= %lld, order 2 or 6, a known "
                                    "precision, dt > 0, nsteps >= 1, eps >= 0",
                         (long long)s->cap);
    auto j = std::make_unique<Job>();
    j->d = *d;
    j->pos.assign(pos, pos + 3 * d->n);
    j->vel.assign(vel, vel + 3 * d->n);
    j->mass.assign(mass, mass + d->n);
    j->mu = mass[0] > 0 && std::isfinite(mass[0]) ? mass[0] : 0.0;
    for (int64_t q = 1; q < d->n && j->mu > 0; ++q)
        if (mass[q] != j->mu) j->mu = 0.0;
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->fatal.empty()) return set_error(NB_ECUDA, "server stopped: %s", s->fatal.c_str());
    j->id = s->next_id++;
    j->t_submit = now_s(s);
    *job_id = j->id;
    s->queue.push_back(j->id);
    s->jobs[j->id] = std::move(j);
    ++s->stats.submitted;
    ++s->stats.queued;
    s->cv.notify_all();
    return NB_OK;
}

static void fill_status(const Job &j, nb_job_status *st)
{
    st->state = j.state;
    st->steps_done = j.steps_done;
    st->t_submit = j.t_submit;
    st->t_admit = j.t_admit;
    st->t_done = j.t_done;
}

int nb_server_poll(nb_server *s, int64_t job_id, nb_job_status *st)
{
    if (!s || !st) return set_error(NB_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error(NB_EINVAL, "unknown job %lld", (long long)job_id);
    fill_status(*it->second, st);
    return NB_OK;
}

int nb_server_wait(nb_server *s, int64_t job_id, double timeout_s, nb_job_status *st)
{
    if (!s || !st) return set_error(NB_EINVAL, "NULL argument");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error(NB_EINVAL, "unknown job %lld", (long long)job_id);
    const Job &j = *it->second;
    const auto until = Clock::now() + std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0);
    while (j.state == NB_JOB_QUEUED || j.state == NB_JOB_RUNNING) {
        if (s->cv.wait_until(lk, until) == std::cv_status::timeout &&
            (j.state == NB_JOB_QUEUED || j.state == NB_JOB_RUNNING)) {
            fill_status(j, st);
            return set_error(NB_ETIMEOUT, "job %lld not finished", (long long)job_id);
        }
    }
    fill_status(j, st);
    return NB_OK;
}

int nb_server_result(nb_server *s, int64_t job_id, double *pos, double *vel)
{
    if (!s) return set_error(NB_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error(NB_EINVAL, "unknown job %lld", (long long)job_id);
    Job &j = *it->second;
    if (j.state == NB_JOB_FAILED)
        return set_error(NB_ENONFINITE, "job %lld failed: %s", (long long)job_id, j.error.c_str());
    if (j.state != NB_JOB_DONE) return set_error(NB_ESTATE, "job %lld has no result", (long long)job_id);
    if (pos) std::memcpy(pos, j.pos.data(), j.pos.size() * 8);
    if (vel) std::memcpy(vel, j.vel.data(), j.vel.size() * 8);
    return NB_OK;
}

int nb_server_cancel(nb_server *s, int64_t job_id)
{
    if (!s) return set_error(NB_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error(NB_EINVAL, "unknown job %lld", (long long)job_id);
    Job &j = *it->second;
    if (j.state == NB_JOB_QUEUED || j.state == NB_JOB_RUNNING) j.cancel = true;
    s->cv.notify_all();
    return NB_OK;
}

int nb_server_forget(nb_server *s, int64_t job_id)
{
    if (!s) return set_error(NB_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->jobs.find(job_id);
    if (it == s->jobs.end()) return set_error(NB_EINVAL, "unknown job %lld", (long long)job_id);
    const int st = it->second->state;
    if (st == NB_JOB_QUEUED || st == NB_JOB_RUNNING)
        return set_error(NB_ESTATE, "job %lld is not finished", (long long)job_id);
    s->jobs.erase(it);
    return NB_OK;
}

// Total length of the union of intervals (sorted copy, merged in one sweep).
static double union_ms(std::vector<std::pair<float, float>> v)
{
    std::sort(v.begin(), v.end());
    double tot = 0.0, a = 0.0, b = -1.0;
    bool open = false;
    for (const auto &x : v) {
        if (!open || x.first > b) {
            if (open) tot += b - a;
            a = x.first;
            b = x.second;
            open = true;
        } else if (x.second > b) {
            b = x.second;
        }
    }
    if (open) tot += b - a;
    return tot;
}

int nb_server_stats(nb_server *s, nb_server_stats_t *out)
{
    if (!s || !out) return set_error(NB_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    out->capacity_bodies = s->cap;
    out->clock_s = now_s(s);
    std::vector<std::pair<float, float>> all;
    for (int a = 0; a < 3; ++a) {
        out->pair_busy_ms[a] = union_ms(s->iv[a]);
        all.insert(all.end(), s->iv[a].begin(), s->iv[a].end());
    }
    out->pair_busy_ms_any = union_ms(std::move(all));
    return NB_OK;
}

}  // extern "C"
