/*
 * nbsym.h -- C ABI of the GB300 direct-summation N-body library.
 *
 * The library integrates the equations of motion of N point masses under
 * softened Newtonian gravity plus an optional smooth external field
 * (Capuzzo-Dolcetta, Mastrobuono-Battisti & Maschietti, "NBSymple",
 * Sect. 2, eq. 1-5 and eq. 3), with the second-order leapfrog or the
 * sixth-order symplectic scheme of Sect. 3.1, entirely on one GPU.
 *
 * General rules for every entry point
 *  - Plain C types only.  Host arrays are borrowed for the duration of the
 *    call; the library copies what it needs.  Output buffers belong to the
 *    caller.  Device-pointer variants (suffix _device) take pointers to
 *    device memory on the context's device; they are also borrowed.  They
 *    work on the context's stream: device memory that other streams write
 *    must be complete before the call (synchronise those streams or order
 *    them with events); when the call returns, what it wrote is complete.
 *  - Positions, velocities and accelerations are float64, n rows of (x, y, z)
 *    interleaved (row-major (n, 3)); masses are float64 (n,).
 *  - Accelerations, never forces: the m_i of eq. 2 / eq. 5 is divided out.
 *  - Every call is synchronous: results are valid when it returns.
 *  - Errors are negative return codes (nb_status); no exception crosses the
 *    ABI.  nb_last_error() gives a message for the calling thread.
 *  - A context is not thread-safe; use one context per host thread, or
 *    serialise calls.
 */
#ifndef NBSYM_H
#define NBSYM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NB_ABI_VERSION 3

/* Opaque context: device state of one particle system plus its buffers,
 * stream, captured step graphs and launch configuration.  Library-owned. */
typedef struct nb_ctx nb_ctx;

/* Arithmetic of the pair-force sum (Sect. 5.2; abstract):
 *  NB_FP64 -- all pair arithmetic and accumulation in double precision.
 *  NB_DS   -- mixed: pair arithmetic in single precision on coordinates
 *             taken relative to a reference point near the system, the
 *             coordinate difference of close pairs re-formed from
 *             double-single (hi + lo) coordinates, float partial sums folded
 *             into double-single accumulators (the paper's software
 *             double-single idea, Sect. 5.2).  On small sets (sum of N_k^2
 *             at most 2^27, e.g. one cluster of N <= 11585) the close-pair
 *             pass costs more than forming the double-single difference for
 *             every pair, so NB_DS then evaluates as NB_DS_FULL.
 *  NB_FP32 -- pure single precision: coordinates rounded to float
 *             (relative to the same reference point), float accumulation.
 *  NB_DD   -- float-float: every quantity of the pair sum (coordinate
 *             difference, r^2 + eps^2, 1/sqrt, m/r^3, the sums) is a pair
 *             hi + lo of floats, about 48 significant bits, on the FP32
 *             pipes; agrees with FP64 to ~1e-14 relative (FP64 tolerance
 *             1e-12).  The FP64 pipe of this GPU runs at 1/77 of the FP32
 *             rate, so this is the fast way to FP64-class accelerations.
 *             No counterpart in the paper, which joins hi and lo only for
 *             the coordinate difference (Sect. 5.2).
 *  NB_DS_FULL -- as NB_DS but the double-single coordinate difference is
 *             formed for every pair, as the paper's DSP code does.
 *  NB_DS_NEAR -- NB_DS in its two-pass form (float pairs plus the close-pair
 *             pass) at every size: NB_DS without the switch to NB_DS_FULL on
 *             small sets.  Same arithmetic and tolerance as NB_DS on large
 *             sets; lets a caller (or a test) run that form on systems small
 *             enough to check step by step against a slow reference.
 * In every mode the state (positions, velocities), the kick/drift update,
 * the external field and the energy diagnostic are double precision. */
enum nb_precision { NB_FP64 = 0, NB_DS = 1, NB_FP32 = 2, NB_DS_FULL = 3, NB_DD = 4,
                    NB_DS_NEAR = 5 };

enum nb_status {
    NB_OK = 0,
    NB_EINVAL = -1,     /* bad argument (NULL pointer, n out of range, order
                           not 2 or 6, dt not finite and > 0, eps < 0, ...) */
    NB_ENOMEM = -2,     /* device or host allocation failed */
    NB_ECUDA = -3,      /* a CUDA runtime call failed (message has details) */
    NB_ESTATE = -4,     /* call not valid in the context's state (e.g. step
                           before load) */
    NB_ETIMEOUT = -5,   /* a bounded device-side wait gave up */
    NB_ENONFINITE = -6  /* result contains NaN/Inf (e.g. coincident particles
                           with eps = 0) */
};

/* Physical and execution parameters of a context. */
typedef struct {
    double G;          /* gravitational constant, > 0 (paper: G = 1, Sect. 3) */
    double eps;        /* softening length >= 0 (eq. 4-5); 0 = unsoftened
                          sum of eq. 2 with the j != i exclusion */
    int precision;     /* enum nb_precision */
    int ext_on;        /* 1: add the external field of eq. 3, a
                          Miyamoto-Nagai disk plus a Plummer bulge plus an
                          optional central point mass (Mbh below):
                          Phi = -G Md / sqrt(R^2 + (ad + sqrt(z^2 + bd^2))^2)
                                - G Mb / sqrt(r^2 + ab^2)
                                - G Mbh / sqrt(r^2 + eps_bh^2),
                          a_ext = -grad Phi */
    double Md, ad, bd; /* disk mass, scale length, scale height (bd > 0) */
    double Mb, ab;     /* bulge mass, scale (ab > 0) */
    int device;        /* CUDA device ordinal */
    void *stream;      /* cudaStream_t to run on; NULL: the context creates
                          and owns a non-blocking stream.  The context also
                          owns a second stream on which the NB_DS near-pair
                          pass runs beside the pair kernel; every call joins
                          it back into this stream (events, captured into the
                          step graphs), so work is ordered on this stream */
    double near_frac;  /* NB_DS, NB_DS_NEAR: pairs closer than near_frac * R_rms /
                          N^{1/3} (R_rms = mass-weighted rms radius about the
                          centre of mass, so the radius scales with the mean
                          spacing) get the double-single coordinate
                          difference; <= 0 selects the default 0.4 */
    double Mbh;        /* mass of a point at the galactic centre (the
                          massive black hole of Sect. 6.2's collision runs,
                          static), >= 0; 0 = none.  Part of the external
                          field: used only when ext_on */
    double eps_bh;     /* its Plummer softening, >= 0 */
} nb_params;

/* Diagnostics of Sect. 5.1 (eq. 9-10 use E and L):
 *   K = 1/2 sum m v^2,  W = -G sum_{i<j} m_i m_j / sqrt(r_ij^2 + eps^2)
 *   (eq. 4), W_ext = sum m_i Phi(r_i), E = K + W + W_ext,
 *   P = sum m v,  L = sum m r x v.   Always computed in double precision. */
typedef struct {
    double K, W, W_ext, E;
    double P[3];
    double L[3];
} nb_energy_t;

/* Timing of the pair-force kernel while profiling is on (nb_prof_enable). */
typedef struct {
    int64_t pair_launches;    /* pair-force kernel launches timed */
    double pair_ms;           /* their summed device time, CUDA events */
    int64_t interactions;     /* sum over those launches of n * n */
    int64_t kernel_launches;  /* all kernels this context enqueued while
                                 profiling was on (graph nodes included) */
} nb_prof_t;

/* Measured arithmetic peaks of one device (see nb_measure_peaks). */
typedef struct {
    int sm_count;
    double ffma_tflops;     /* scalar FP32 FMA, 2 flops each */
    double ffma2_tflops;    /* packed f32x2 FMA, 4 flops each */
    double dfma_tflops;     /* FP64 FMA, 2 flops each */
    double rsqrt_gops;      /* MUFU reciprocal square roots per second, 1e9 */
    double pairmix_gpairs;  /* the mixed pair kernel's arithmetic alone (packed
                               sub/FMA/mul + MUFU rsqrt per pair, operands in
                               registers), 1e9 pair interactions per second */
} nb_peaks_t;

/* Library ABI version (NB_ABI_VERSION of the build). */
int nb_abi_version(void);

/* Message of the last error on the calling thread ("" if none).  The string
 * is owned by the library and valid until the next call on this thread. */
const char *nb_last_error(void);

/* Fill *p with defaults: G = 1, eps = 0, NB_DS, field off with the disk +
 * bulge constants (Md 100, ad 6.5, bd 0.26, Mb 15, ab 0.7), device 0, own
 * stream, default near_frac.  NULL-safe (no-op). */
void nb_params_default(nb_params *p);

/* Create a context for up to n_capacity particles (1 <= n_capacity <= 2^26)
 * on p->device.  Allocates all device memory the context will use.
 * *out receives the context.  Errors: NB_EINVAL (bad parameters),
 * NB_ENOMEM, NB_ECUDA. */
int nb_create(const nb_params *p, int64_t n_capacity, nb_ctx **out);

/* Create a context holding an ensemble of n_clusters independent systems of
 * fixed sizes sizes[0..n_clusters-1] (each >= 1; 1 <= n_clusters <= 2^19,
 * sum <= 2^26).  Each cluster obeys eq. 3 on its own: bodies of different
 * clusters never interact.  Every force evaluation of the whole ensemble is
 * one kernel launch whose blocks share the pair work of all clusters
 * evenly, and a step of every cluster is one CUDA graph.  nb_load
 * then takes the clusters' bodies concatenated in cluster order (n = sum of
 * sizes); nb_accel / nb_get_state return them in that order; every cluster
 * starts with softening p->eps and step scale 1 (nb_set_cluster_params).
 * The paper integrates one cluster at a time; this batches many.  Errors:
 * NB_EINVAL, NB_ENOMEM, NB_ECUDA. */
int nb_create_batch(const nb_params *p, int64_t n_clusters, const int64_t *sizes,
                    nb_ctx **out);

/* Per-cluster softening eps[k] >= 0 (eq. 4-5) and step scale dt_scale[k] > 0
 * (cluster k advances by dt * dt_scale[k] per nb_step); either array may be
 * NULL to keep the current values.  Arrays have nb_clusters() entries.
 * Errors: NB_EINVAL, NB_ECUDA. */
int nb_set_cluster_params(nb_ctx *ctx, const double *eps, const double *dt_scale);

/* Number of clusters (1 for nb_create), or NB_EINVAL for NULL. */
int64_t nb_clusters(const nb_ctx *ctx);

/* Load a particle system (initial conditions of eq. 3): n rows of positions
 * and velocities, n masses (>= 0, finite).  1 <= n <= capacity.  Host
 * pointers.  Errors: NB_EINVAL, NB_ECUDA. */
int nb_load(nb_ctx *ctx, int64_t n, const double *pos, const double *vel,
            const double *mass);

/* As nb_load with device pointers (e.g. torch tensors' data_ptr()). */
int nb_load_device(nb_ctx *ctx, int64_t n, const double *d_pos,
                   const double *d_vel, const double *d_mass);

/* One force evaluation at the current positions: the right-hand side of
 * eq. 3, a_i = G sum_{j != i} m_j r_ij / (|r_ij|^2 + eps^2)^{3/2} (eq. 5,
 * eq. 2 when eps = 0) plus the external field when ext_on.  Written to the
 * caller's host buffer acc_out (n rows of x, y, z).  Errors: NB_ESTATE (no
 * system loaded), NB_EINVAL, NB_ENONFINITE, NB_ECUDA. */
int nb_accel(nb_ctx *ctx, double *acc_out);

/* As nb_accel into device memory. */
int nb_accel_device(nb_ctx *ctx, double *d_acc_out);

/* Advance the loaded system by nsteps steps of length dt with the
 * symplectic scheme of the given order (Sect. 3.1): order 2 is the
 * drift-kick-drift leapfrog (one force evaluation per step), order 6 is the
 * SI6A composition of seven leapfrog steps (seven force evaluations per
 * step).  nsteps >= 0, dt finite and > 0.  Errors: NB_ESTATE, NB_EINVAL,
 * NB_ECUDA. */
int nb_step(nb_ctx *ctx, int order, double dt, int64_t nsteps);

/* Energy, momentum and angular momentum of the current state (Sect. 5.1),
 * summed over the clusters of a batch.  Errors: NB_ESTATE, NB_EINVAL,
 * NB_ENONFINITE, NB_ECUDA. */
int nb_energy(nb_ctx *ctx, nb_energy_t *out);

/* The same per cluster: out has nb_clusters() entries, cluster k's record
 * at out[k].  Errors as nb_energy. */
int nb_energy_clusters(nb_ctx *ctx, nb_energy_t *out);

/* External torque M_ext = sum m_i r_i x a_ext(r_i) (eq. 8), summed over the
 * clusters; zero when the field is off.  out has 3 doubles.  Errors:
 * NB_ESTATE, NB_EINVAL, NB_ECUDA. */
int nb_torque(nb_ctx *ctx, double *out);

/* Copy the current positions and velocities (n rows each) to host buffers;
 * either pointer may be NULL to skip it.  Errors: NB_ESTATE, NB_ECUDA. */
int nb_get_state(nb_ctx *ctx, double *pos, double *vel);

/* As nb_get_state into device memory. */
int nb_get_state_device(nb_ctx *ctx, double *d_pos, double *d_vel);

/* Number of particles loaded (0 before nb_load), or NB_EINVAL for NULL. */
int64_t nb_size(const nb_ctx *ctx);

/* Switch the pair-force arithmetic (enum nb_precision) of a context
 * without reloading; the state is untouched.  Errors: NB_EINVAL. */
int nb_set_precision(nb_ctx *ctx, int precision);

/* Start (on = 1) or stop (on = 0) timing pair-force launches with CUDA
 * events recorded on the context's stream (inside captured step graphs as
 * event-record nodes).  Starting resets the counters.  Errors: NB_EINVAL. */
int nb_prof_enable(nb_ctx *ctx, int on);

/* Read the counters accumulated since nb_prof_enable(ctx, 1) into *out.
 * Errors: NB_EINVAL (NULL ctx or out). */
int nb_prof_read(nb_ctx *ctx, nb_prof_t *out);

/* Measure the arithmetic peaks the pair kernels are bounded by (the
 * denominators of their plain-ALU roofline; the paper quotes nominal SP/DP
 * peaks, Sect. 4.1): each micro-kernel runs independent FMA / MUFU chains on
 * every SM for a few milliseconds, timed with CUDA events (best of three).
 * Allocates 64 bytes of device memory and a stream for the duration of the
 * call.  Errors: NB_EINVAL (NULL out, bad device), NB_ECUDA. */
int nb_measure_peaks(int device, nb_peaks_t *out);

/* One force evaluation that allocates nothing.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- hosts
 * that give all device memory to their own pool allocator, loops that must
 * never pay the implicit device synchronisation of cudaMalloc/cudaFree, and
 * plug-in environments that forbid device allocation after start-up.
 *
 * Computes the same accelerations as nb_accel (in the arithmetic
 * p->precision selects, plus the external field when p->ext_on) for n bodies
 * given as device pointers: d_pos (n rows of x, y, z), d_mass (n), result to
 * d_acc_out (n rows), all caller-owned memory on p->device.  Work is
 * enqueued on p->stream (NULL = the legacy default stream); the call returns
 * without synchronising, so the caller synchronises that stream before
 * reading d_acc_out.  No non-finite check is made.
 *
 * Limit: 1 <= n <= 16384.  All working memory sits in one static device
 * array of about 7.3 MB that every GPU loading the library keeps until the
 * process exits.  The first call on a device looks up that array's address
 * (cudaGetSymbolAddress) and must come before any stream capture; so must
 * the first call after cudaDeviceReset, which looks it up again.  Calls
 * share the array: calls whose work overlaps on the GPU race, so serialise
 * them.  Calls no cudaMalloc, cudaFree or allocating library routine.
 * Errors: NB_EINVAL (NULL pointer, n out of range, bad parameters or
 * device), NB_ECUDA (with the runtime's message; a launch error that earlier
 * work of the caller left pending is reported here too). */
int nb_accel_static(const nb_params *p, int64_t n, const double *d_pos,
                    const double *d_mass, double *d_acc_out);

/* Accelerations of bodies [i0, i1) of a one-cluster context against all n
 * (internal sum of eq. 5 in the context's precision, plus the external field
 * when ext_on): the share one GPU computes in the paper's multi-GPU scheme
 * (Sect. 4.2), where each GPU sums an i-range against all bodies.  The launch
 * takes whole 128 I-body i-blocks and sums each one's j range in order in one
 * block, so a body's result does not depend on the range it was computed in:
 * split ranges concatenate bit for bit to the whole range (in every
 * precision; across calls the mixed mode's near-pair correction is
 * deterministic too).  Rows of acc_out: i1 - i0, host memory.  Synchronous.
 * Errors: NB_EINVAL (NULL, bad range, more than one cluster), NB_ESTATE
 * (nothing loaded), NB_ENONFINITE, NB_ECUDA. */
int nb_accel_range(nb_ctx *ctx, int64_t i0, int64_t i1, double *acc_out);

/* The kick weights of one step of the given order (Sect. 3.1) to w, which
 * has room for 7: order 2 (drift-kick-drift leapfrog) one weight, 1; order 6
 * (SI6A) the seven leapfrog weights w3 w2 w1 w0 w1 w2 w3 of Yoshida's
 * sixth-order solution A, w0 = 1 - 2 (w1 + w2 + w3).  The drifts between
 * them are half sums of neighbouring weights: w_0 / 2 first, (w_k + w_k+1) / 2
 * between kicks k and k + 1, w_last / 2 last (nb_step merges adjacent half
 * drifts this way).  Returns the number of weights.  Errors: NB_EINVAL (NULL
 * w, order not 2 or 6). */
int nb_stage_weights(int order, double *w);

/* One substep of the leapfrog / SI6A sequence (Sect. 3.1) for bodies
 * [i0, i1) of a one-cluster context: when kick != 0, v_i += kick * a_i with
 * a_i the right-hand side of eq. 3 at the current positions (the internal sum
 * against all n bodies, computed as nb_accel_range does, plus the external
 * field); then x_i += drift * v_i.  kick and drift are the step length times
 * the stage weight (a drift-only substep passes kick = 0).  Other bodies are
 * untouched.  This is one GPU's share of a step in the paper's multi-GPU
 * scheme (Sect. 4.2): every GPU holds all positions, advances its own i-range
 * and then receives the others' new positions (nb_set_state).  Split
 * ranges give the same bits as the whole range.  Synchronous.  Errors:
 * NB_EINVAL (NULL, bad range, non-finite weights, more than one cluster),
 * NB_ESTATE (nothing loaded), NB_ECUDA. */
int nb_substep_range(nb_ctx *ctx, int64_t i0, int64_t i1, double kick, double drift);

/* Replace the positions and / or velocities of all n bodies (n rows of x, y,
 * z each; host memory; either pointer may be NULL to keep those values) of a
 * loaded context; masses, softening and the launch plan are kept, unlike
 * nb_load.  Synchronous.  Errors: NB_EINVAL (NULL ctx), NB_ESTATE (nothing
 * loaded), NB_ECUDA. */
int nb_set_state(nb_ctx *ctx, const double *pos, const double *vel);

/* As nb_set_state from device memory (e.g. the buffer an all-gather of the
 * GPUs' i-ranges filled). */
int nb_set_state_device(nb_ctx *ctx, const double *d_pos, const double *d_vel);

/* The N(N-1)/2 variant of the internal sum (Newton's third law: each
 * unordered pair evaluated once and its force added to both bodies), which
 * the paper rejects for its GPU (Sect. 4.2); provided to measure it here.
 * Accelerations of the loaded one-cluster state (internal sum of eq. 5 in
 * float arithmetic on frame-centred coordinates, the class of NB_FP32, plus
 * the external field when ext_on) to acc_out (n rows of x, y, z, host),
 * whatever the context's precision; the pair kernel's time (CUDA events) to
 * *pair_ms when pair_ms is not NULL.  Sums are combined with float atomics,
 * so results are not bit-reproducible.  Allocates and frees 36 bytes per body
 * of device memory per call; synchronous.  Errors: NB_EINVAL (NULL, more than
 * one cluster), NB_ESTATE (nothing loaded), NB_ENOMEM, NB_ECUDA. */
int nb_accel_symmetric(nb_ctx *ctx, double *acc_out, double *pair_ms);

/* ---- autotuner (no counterpart in the paper: the paper fixes one block
 * shape for its GPU, Sect. 4.2) ---------------------------------------------
 * The launch shape of the pair kernel is (bodies per thread I, j-tile width
 * jt, blocks per SM b): one work unit is an i-block of 128 * I bodies against
 * a j-range of jt bodies (128, 64 or 32: narrower ranges give small clusters
 * enough units to fill the GPU); b sets the grid (b * SMs blocks, at most the
 * unit count) and so how finely units are cut into per-block runs.  Up to
 * the occupancy limit the grid is resident at once; above it (up to 6 times
 * that limit) it runs in waves, which evens out SMs whose resident blocks
 * progress at different rates.  nb_tune times every shape this build compiled for
 * the context's current precision on its loaded state (reps force evaluations,
 * the mixed mode's near-pair pass included, and reps kicks each; CUDA events on
 * the context's stream), switches the context to the shape with the least
 * evaluation + kick time
 * and records it in a process-wide table keyed by the workload's shape (SM
 * count, precision, cluster count, bodies, widest cluster), which every later
 * context or serving group of the same shape uses.  Two shapes can split the
 * j-sums differently, so results may differ at the rounding level between
 * shapes; with one shape they are bit-reproducible. */
typedef struct {
    int precision;           /* enum nb_precision tuned */
    int bodies_per_thread;   /* chosen I */
    int blocks_per_sm;       /* chosen b (grid per SM; above the occupancy
                                limit the grid runs in waves) */
    int j_tile;              /* chosen j bodies per unit: 128, 64 or 32 */
    int candidates;          /* shapes timed */
    int64_t grid;            /* blocks of the chosen shape */
    double pair_ms;          /* mean time of one force evaluation with the
                                chosen shape: the pair launch, with the mixed
                                mode's near-pair pass beside it */
    double default_ms;       /* the same for the shape chosen without tuning */
    double cost_ms;          /* pair_ms plus the mean time of one kick that
                                sums its partial slots: what shapes are chosen
                                by */
    double default_cost_ms;  /* the same for the shape chosen without tuning */
} nb_tune_t;

/* Tune the context (1 <= reps <= 1000; out may be NULL).  Synchronous; the
 * state is untouched.  Errors: NB_EINVAL, NB_ESTATE (nothing loaded),
 * NB_ECUDA. */
int nb_tune(nb_ctx *ctx, int reps, nb_tune_t *out);

/* Write the process-wide table to a text file (one line per shape: SM count,
 * precision, clusters, bodies, widest cluster in tiles, I, b).  Errors:
 * NB_EINVAL (NULL path, file not writable). */
int nb_tune_save(const char *path);

/* Merge the entries of a file written by nb_tune_save into the table.
 * Returns the number of entries read (>= 0), or NB_EINVAL (NULL path,
 * unreadable or malformed file, or a shape this build lacks; nothing is
 * merged then).  Contexts planned afterwards use the entries. */
int64_t nb_tune_load(const char *path);

/* The pair-kernel shape of the context's current plan: bodies per thread,
 * blocks per SM, j bodies per unit, grid (any out pointer
 * may be NULL).  Errors: NB_EINVAL (NULL ctx), NB_ESTATE (nothing loaded). */
int nb_pair_shape(nb_ctx *ctx, int *bodies_per_thread, int *blocks_per_sm, int *j_tile,
                  int64_t *grid);

/* Number of entries in the table. */
int64_t nb_tune_entries(void);

/* Empty the table.  Contexts already planned keep their shape. */
void nb_tune_clear(void);

/* Release the context and all its device memory.  NULL-safe. */
void nb_destroy(nb_ctx *ctx);

/* ---- Serving loop ----------------------------------------------------------
 * Integration jobs of different N, order and precision share one GPU.  The
 * paper runs one simulation per program; this is a request loop around the
 * same step (Sect. 3.1).  A scheduler thread admits queued jobs in arrival
 * order when a resident-job slot is free and the state pool (sized from the
 * HBM budget) has a contiguous range for the job's bodies.  Resident jobs are
 * grouped by (precision, order, and size: below 16384 bodies or not; the
 * groups of smaller jobs run on higher-priority streams); each
 * group advances one step at a time with
 * one pair-kernel launch per force evaluation covering all its jobs, on its
 * own stream, so groups overlap on the device.  Jobs join and leave a group
 * between two of its steps (continuous batching).  Each job is an independent
 * system (eq. 3) with its own softening and step; the field parameters are
 * the server's.  All calls are thread-safe. */
typedef struct nb_server nb_server;

typedef struct {
    int device;
    double hbm_budget_bytes;  /* device memory for resident state (> 0);
                                 about 436 bytes per body slot, plus the
                                 groups' partial sums beyond that share (at
                                 most ~67 MB per group of the twelve) */
    int max_jobs;             /* resident jobs at most, 1..65536 */
    double G;                 /* as nb_params */
    int ext_on;
    double Md, ad, bd, Mb, ab;
    double near_frac;         /* as nb_params (NB_DS jobs) */
    double Mbh, eps_bh;       /* as nb_params */
    int fp64_via_dd;          /* 1 (default): jobs submitted as NB_FP64 run the
                                 NB_DD (float-float) arithmetic, which meets the
                                 FP64 tolerance at ~8x the FP64 kernel's rate (this
                                 GPU's FP64 pipe runs at 1/77 of its FP32 rate);
                                 0: the plain FP64 kernel */
} nb_server_params;

typedef struct {
    int64_t n;        /* bodies, 1 <= n <= pool capacity */
    int order;        /* 2 or 6 */
    int precision;    /* NB_FP64, NB_DS or NB_DD */
    double dt;        /* step length > 0 */
    int64_t nsteps;   /* >= 1 */
    double eps;       /* softening >= 0 */
} nb_job_desc;

enum nb_job_state { NB_JOB_QUEUED = 0, NB_JOB_RUNNING = 1, NB_JOB_DONE = 2,
                    NB_JOB_FAILED = 3, NB_JOB_CANCELLED = 4 };

typedef struct {
    int state;            /* enum nb_job_state */
    int64_t steps_done;
    double t_submit;      /* server clock, seconds since nb_server_create */
    double t_admit;       /* 0 while queued */
    double t_done;        /* 0 until finished; latency = t_done - t_submit */
} nb_job_status;

typedef struct {
    int64_t submitted, admitted, completed, failed, cancelled, queued, running;
    double interactions;      /* pair interactions evaluated (N^2 per evaluation) */
    int64_t kernel_launches;  /* kernels the scheduler enqueued */
    int64_t capacity_bodies;  /* pool capacity from the budget */
    double clock_s;           /* server clock now */
    double pair_ms[3];        /* summed device time of the pair-force launches
                                 (CUDA events on each group's stream), by
                                 arithmetic: [0] the FP64 kernel, [1] NB_DS,
                                 [2] NB_DD (and FP64 jobs run in it).  Groups
                                 overlap on the device, so a launch's time
                                 includes the SMs it shared with other groups */
    double pair_interactions[3]; /* N^2 summed over those launches, same index */
    double pair_busy_ms[3];   /* device time during which at least one pair
                                 launch of that arithmetic ran (the union of the
                                 launches' event intervals, over the first 2^20
                                 launches of each): pair_interactions[a] /
                                 pair_busy_ms[a] is that kernel's rate in the
                                 mix, concurrent launches counted together */
    double pair_busy_ms_any;  /* the same over all arithmetics */
} nb_server_stats_t;

/* Defaults: device 0, 4 GB budget, 64 jobs, G = 1, field off with the disk +
 * bulge constants of nb_params_default, FP64 jobs in float-float
 * (fp64_via_dd = 1).  NULL-safe. */
void nb_server_params_default(nb_server_params *p);

/* Allocate the pool and start the scheduler thread.  Errors: NB_EINVAL,
 * NB_ENOMEM, NB_ECUDA. */
int nb_server_create(const nb_server_params *p, nb_server **out);

/* Queue a job; host arrays (n rows of positions and velocities, n masses) are
 * copied before the call returns.  *job_id receives the job's id.  Errors:
 * NB_EINVAL (bad descriptor or NULL), NB_ECUDA (server stopped). */
int nb_server_submit(nb_server *s, const nb_job_desc *d, const double *pos,
                     const double *vel, const double *mass, int64_t *job_id);

/* Current status of a job.  Errors: NB_EINVAL (unknown id). */
int nb_server_poll(nb_server *s, int64_t job_id, nb_job_status *st);

/* Block until the job is done, failed or cancelled, or timeout_s elapses
 * (NB_ETIMEOUT; *st then holds the current status). */
int nb_server_wait(nb_server *s, int64_t job_id, double timeout_s, nb_job_status *st);

/* Final positions and velocities of a done job (n rows each; either pointer
 * may be NULL).  Errors: NB_ESTATE (not done), NB_ENONFINITE (job failed),
 * NB_EINVAL. */
int nb_server_result(nb_server *s, int64_t job_id, double *pos, double *vel);

/* Cancel a queued job, or a running one at its group's next step boundary. */
int nb_server_cancel(nb_server *s, int64_t job_id);

/* Drop a finished job's record and result.  Errors: NB_ESTATE if running. */
int nb_server_forget(nb_server *s, int64_t job_id);

/* Counters since creation. */
int nb_server_stats(nb_server *s, nb_server_stats_t *out);

/* Stop the scheduler (queued and running jobs are abandoned) and free
 * everything.  NULL-safe. */
void nb_server_destroy(nb_server *s);

#ifdef __cplusplus
}
#endif

#endif /* NBSYM_H */
