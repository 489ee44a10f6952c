// engine.h -- host-side engine behind the C ABI: a device state pool, the
// tables of a cluster set living in it, launch plans, and the functions that
// enqueue force evaluations, integration steps and diagnostics.  Used by the
// context API (nbsym.cu) and the serving loop (server.cu).
#pragma once

#include <string>
#include <vector>

#include "nb_internal.cuh"
#include "../../include/nbsym.h"

namespace nb {

// Thread-local error message shared by every entry point.
int set_error(int code, const char *fmt, ...);
const char *last_error();

// Validation of nb_params (nb_create's rules): NB_OK, or NB_EINVAL with the
// message set.
int check_nb_params(const nb_params *p);

#define NB_TRY(call)                                                                       \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return ::nb::set_error(NB_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

// Device arrays for up to cap bodies (pool slots); DevState::cl and n are
// filled per cluster set by view().
struct Pool {
    int device = 0;
    int num_sms = 0;
    int64_t cap = 0;
    DevState s;
    double *stage = nullptr;   // (7 cap) staging for interleaved host transfers
};
// own_part: allocate the partial-sum storage of a single cluster set (a
// context); a pool shared by concurrent sets (the serving loop's groups)
// leaves it out, and each set reserves its own (set_reserve_part).
int pool_create(Pool &P, int device, int64_t cap, bool own_part = true);
// Partial-sum doubles a set of n bodies may need: 3 min(giw + 2 n,
// MAX_PART_SLOTS n), giw the widest grid's i-rows (SMs x MAX_WAVES x 3072).
int64_t part_elems_for(const Pool &P, int64_t n);
void pool_destroy(Pool &P);

// Tables of one cluster set in a pool (host copy + device copy).
struct ClusterSet {
    int32_t K = 0, kcap = 0;
    int64_t scap = 0;
    int64_t n = 0;             // bodies, noff[K]
    int64_t max_ntiles = 0;
    int ipb = 0;               // i-block width the pair units are counted with
    std::vector<int64_t> boff, nk, noff, uoff, uoff_pot, seg_lo, seg_hi;
    std::vector<int32_t> ntiles, seg_k, seg_off;
    std::vector<float> eps2f;
    std::vector<double> eps, eps2d, dts;
    std::vector<double> mu;    // common mass per cluster (0: masses differ); set by
                               // the loader before planning, uploaded by set_layout
    char *dmem = nullptr;      // device copy of the tables
    double *red = nullptr;     // reduction partials [scap][16]
    // per-set scratch, so sets in one pool can run concurrently on different
    // streams: near-pair hash grid over the set's linear bodies and the flag
    int64_t body_cap = 0, ng_hcap = 0;
    int *ng_bucket = nullptr, *ng_rank = nullptr, *ng_entry = nullptr, *ng_total = nullptr,
        *flag = nullptr;
    int32_t *cid = nullptr;    // linear body -> cluster map
    float4 *ng_spos = nullptr, *ng_slo = nullptr;
    NgSlot *ng_slot = nullptr;
    Frame *frame = nullptr;    // [kcap]
    double *diag = nullptr;    // [kcap][DIAG_STRIDE]
    Clusters cl, cl_pot;       // device views (pair units / potential units)
    // side stream and fork / join events: the near-pair pass runs beside the
    // pair kernel (it reads only the float planes, and writes only corr)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // the set's own partial-sum storage (NULL: the pool's); sets that run
    // concurrently in one pool must each have their own
    double *part = nullptr;
    int64_t part_elems = 0;
    // launch order of the pair kernel's blocks for the decomposition of the
    // last plan made (grid bperm_G over bperm_W units of width bperm_jt,
    // i-blocks of bperm_ipb bodies; bperm_G = -1: none)
    std::vector<uint16_t> bperm;
    int64_t bperm_G = -1, bperm_W = -1;
    int bperm_jt = 0, bperm_ipb = 0;
};
// priority: of the set's side stream (the near-pair pass), as for the stream
// its steps are enqueued on (0: the default).
int set_create(ClusterSet &C, int32_t kcap, int64_t body_cap, int priority = 0);
// Launch order of the pair kernel's blocks for decomposition d over C's
// clusters (host only; fills C.bperm, a permutation of [0, d.G), and its key):
// largest estimated work first.  I: bodies per thread; partial: the kernel
// evaluates only the packed i-pairs that hold bodies.
void block_order(ClusterSet &C, const Decomp &d, int I, bool partial);
// Give the set its own partial-sum storage of at least elems doubles, grown
// (stream-ordered allocation on st) when smaller; none of the set's work may
// be in flight.
int set_reserve_part(ClusterSet &C, int64_t elems, cudaStream_t st);
void set_destroy(ClusterSet &C);
// Clusters k = 0..K-1 at pool slots [boff[k], boff[k] + nk[k]), softening
// eps[k] and step scale dts[k] (NULL: 1).  Host only; set_layout uploads.
int set_define(ClusterSet &C, int32_t K, const int64_t *boff, const int64_t *nk,
               const double *eps, const double *dts);
// Count pair units for i-blocks of ipb bodies and j-ranges of jt bodies (a
// divisor of TILE), build reduction segments and upload every table
// (stream-ordered).
int set_layout(ClusterSet &C, int ipb, cudaStream_t st, int jt = TILE);

struct Plan {
    int precision = -1;
    PairLaunch pl{};
    Decomp pot{};
};
// Launch shape of the pair kernel: I bodies per thread (i-block width
// TILE * I), jt j bodies per unit (TILE, TILE / 2 or TILE / 4) and
// blocks_per_sm, the grid per SM (grid = blocks_per_sm * SMs, at most the
// unit count).  Up to the occupancy limit the grid is resident at once;
// above it the grid runs in waves (at most MAX_WAVES), the hardware handing
// each further block to whichever SM frees a slot.  Resident blocks of one SM
// do not progress at one rate (the warp scheduler favours the oldest), so a
// single resident wave of equal unit runs ends with SMs holding one slow
// block; waves even that out, while every block's units and partial slot
// stay fixed by its index (results stay bit-reproducible).
constexpr int MAX_WAVES = 6;
constexpr int DEFAULT_WAVES = 4;
struct PairShape {
    int I = 0;
    int blocks_per_sm = 0;
    int jt = 0;   // 0: chosen by the planner
};
// Choose the pair kernel variant and decompositions for a cluster set and
// lay the set out for it.  The shape is `force` when given, else the tuned
// entry for the set's shape (when use_table), else the built-in heuristic.
// waves > 0: that many waves of resident blocks whatever the shape's own
// grid (the bodies per thread still come from force, the table or the
// heuristic).
int plan_make(const Pool &P, ClusterSet &C, int precision, cudaStream_t st, Plan &out,
              const PairShape *force = nullptr, bool use_table = true, int waves = 0);

// ---- autotuner (tune.cu) -----------------------------------------------------
struct TuneKey {
    int sms = 0, precision = 0;
    int32_t K = 0;
    int64_t n = 0, max_ntiles = 0;
};
struct TuneReport {
    int precision = 0;
    PairShape shape;
    int64_t grid = 0;
    int candidates = 0;
    double pair_ms = 0, default_ms = 0;
    double cost_ms = 0, default_cost_ms = 0;
};
TuneKey tune_key(const Pool &P, const ClusterSet &C, int precision);
bool tune_lookup(const TuneKey &k, PairShape *out);
void tune_store(const TuneKey &k, const PairShape &s);
void tune_clear();
int64_t tune_entries();
int tune_save(const char *path);
int tune_load(const char *path, int64_t *loaded);
struct Phys;
// Time every compiled shape of the precision's pair kernel on the set's
// current state (reps force evaluations, near-pair pass included, and reps
// kicks each; the state is untouched), remember the shape with the least
// evaluation + kick time for the set's shape and return the plan built with
// it.  Needs the float planes current.
int tune_pair(const Pool &P, ClusterSet &C, int precision, const Phys &ph, cudaStream_t st,
              int reps, TuneReport &rep, Plan &out);

struct Phys {
    double G = 1.0;
    double near_frac = 0.4;
    ExtField ext{};
};

// Kernel-facing state of a cluster set: the pool arrays with the set's tables
// (near-pair correction attached when the precision is NB_DS, or, given a
// plan, when the plan runs the near-pair pass).
DevState view(const Pool &P, const ClusterSet &C, int precision);
DevState view(const Pool &P, const ClusterSet &C, const Plan &pl);
// Pair-kernel family of a plan: the precision's, except that NB_DS on a set
// of at most DS_FULL_MAX_PAIRS pairs forms the double-single difference on
// every pair (no near-pair pass).
int plan_mode(const ClusterSet &C, int precision);
// Partial slots per body the set has in its storage (its own, else the
// pool's) for its current bodies.
int64_t part_slot_cap(const Pool &P, const ClusterSet &C);
int mode_of(int precision);
bool float_planes(int precision);

// Enqueue-only operations (no synchronisation).  *kernels, when given, is
// increased by the number of kernels enqueued.
int enq_split(const Pool &P, const ClusterSet &C, const Plan &pl, const Phys &ph,
              cudaStream_t st, int64_t *kernels);
// Pair forces (+ near-pair correction in the mixed mode) into partial slots;
// ev0/ev1 (optional) bracket the pair kernel with external event records.
int enq_force(const Pool &P, const ClusterSet &C, const Plan &pl, const Phys &ph,
              cudaStream_t st, cudaEvent_t ev0, cudaEvent_t ev1, int64_t *kernels);
// One step of length dt (times each cluster's scale) of order 2 or 6.
// evs (optional) has 2 events per force evaluation for the pair kernels.
int enq_step(const Pool &P, const ClusterSet &C, const Plan &pl, const Phys &ph, int order,
             double dt, cudaStream_t st, const std::vector<cudaEvent_t> *evs, int64_t *kernels);
int enq_accel_out(const Pool &P, const ClusterSet &C, const Plan &pl, const Phys &ph,
                  double *out, cudaStream_t st, int64_t *kernels);
// Energy / momentum per cluster into C.diag.
int enq_energy(const Pool &P, const ClusterSet &C, const Plan &pl, const Phys &ph,
               cudaStream_t st, int64_t *kernels);
int enq_torque(const Pool &P, const ClusterSet &C, const Phys &ph, cudaStream_t st,
               int64_t *kernels);

// N(N-1)/2 variant (sym.cu): accelerations of a one-cluster set with each
// unordered pair evaluated once, float arithmetic, float-atomic sums in acc
// (device, 3 n floats); interleaved double rows to out (device).  e0/e1
// bracket the pair kernel.  Needs the float planes current.
int sym_accel(const Pool &P, const ClusterSet &C, const Phys &ph, float *acc, double *out,
              cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1);

// SI6A weights (Kinoshita, Yoshida & Nakai 1991, Table 1 first column =
// Yoshida's 1990 solution A); w0 = 1 - 2 (w1 + w2 + w3).
constexpr double SI6_W1 = -1.17767998417887;
constexpr double SI6_W2 = 0.235573213359357;
constexpr double SI6_W3 = 0.784513610477560;

}  // namespace nb
