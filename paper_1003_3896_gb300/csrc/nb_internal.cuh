// nb_internal.cuh -- device layout, work decomposition and launcher
// declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nb {

// Tile width of the pair kernels: a unit of pair work is TILE j bodies
// against one i-block of TILE * I bodies.
constexpr int TILE = 128;

// Position of padding j slots: far enough that its mass-0 contribution is an
// exact 0, small enough that its squared distance stays finite in float.
constexpr float FAR_F = 1.0e18f;
constexpr double FAR_D = 1.0e150;

// Reference frame of one cluster's single-precision coordinates (Sect. 5.2's
// "delicate evaluation of coordinate difference"): positions are stored as
// float hi = fl(x - c) and lo = fl((x - c) - hi).
struct Frame {
    double cx, cy, cz;   // reference point (mass-weighted centre)
    double r2rms;        // mass-weighted mean |x - c|^2
    float th2;           // near-pair threshold on r^2 + eps^2
    float dth;           // near-pair radius d_th (th2 = d_th^2 + eps^2)
};

// A set of K independent clusters living in one state pool.  Cluster k owns
// pool slots [boff[k], boff[k] + nk[k]); bodies are also numbered linearly,
// cluster after cluster, through the prefix sums noff.  A single system is
// K = 1; a batched ensemble or a serving batch is K > 1.  Device pointers.
struct Clusters {
    int32_t K = 0;
    const int64_t *boff = nullptr;   // [K]   first pool slot of cluster k
    const int64_t *nk = nullptr;     // [K]   bodies of cluster k
    const int64_t *noff = nullptr;   // [K+1] prefix sums of nk (linear body index)
    const int64_t *uoff = nullptr;   // [K+1] prefix sums of pair units
    const int32_t *ntiles = nullptr; // [K]   j tiles of cluster k = ceil(nk / TILE)
    const float *eps2f = nullptr;    // [K]   eps^2 (float)
    const double *eps2d = nullptr;   // [K]   eps^2 (double)
    const double *dts = nullptr;     // [K]   step-length scale of cluster k
    Frame *frame = nullptr;          // [K]
    // reduction segments: each covers a run of one cluster's linear bodies
    int32_t S = 0;
    const int32_t *seg_k = nullptr;  // [S]
    const int64_t *seg_lo = nullptr; // [S]   linear body range [lo, hi)
    const int64_t *seg_hi = nullptr;
    const int32_t *seg_off = nullptr;// [K+1] segments of cluster k: [seg_off[k], seg_off[k+1])
    const int32_t *cid = nullptr;    // [noff[K]] cluster of each linear body (K > 1)
    const double *mu = nullptr;      // [K]   the common mass of cluster k's bodies, 0 if
                                     //       they differ
};

// Cluster of linear body t: one load from the precomputed map (K = 1: 0).
__device__ __forceinline__ int32_t cluster_of(const Clusters &c, int64_t t)
{
    return c.K == 1 ? 0 : c.cid[t];
}

// largest k in [0, K) with off[k] <= t (off[0] = 0 <= t < off[K])
__host__ __device__ __forceinline__ int32_t find_cluster(const int64_t *off, int32_t K, int64_t t)
{
    int32_t lo = 0, hi = K;
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (off[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// Slot of the near-pair cell table: cell key (all ones: empty) and the
// cell's range [start, end) in the cell-ordered body copies.
struct __align__(16) NgSlot {
    unsigned long long key;
    int start, end;
};

// Device state pool.  FP64 structure-of-arrays planes are the state; float
// planes are derived copies for the single-precision paths.  All indexed by
// pool slot.
struct DevState {
    int64_t cap = 0;       // pool slots
    int64_t n = 0;         // bodies in the current cluster set (noff[K])
    Clusters cl;
    double *x = nullptr, *y = nullptr, *z = nullptr;
    double *vx = nullptr, *vy = nullptr, *vz = nullptr, *m = nullptr;
    float *xh = nullptr, *yh = nullptr, *zh = nullptr, *mf = nullptr;
    float *xl = nullptr, *yl = nullptr, *zl = nullptr;
    // j-stream copies, two float4 per body, each coordinate duplicated so a
    // packed f32x2 operand serves two i bodies: jd = (xh, xh, yh, yh),
    // (zh, zh, m, m); jl = (xl, xl, yl, yl), (zl, zl, ml, ml) with ml the
    // float rounding residue of the mass.
    float4 *jd = nullptr, *jl = nullptr;
    // partial sums of the pair decomposition, [slot][3][pstride] indexed by
    // the linear body index of the current set (pstride = its body count), so
    // a set of n bodies has part_elems / (3 n) slots whatever the pool's size
    double *part = nullptr;
    int64_t part_elems = 0;     // doubles allocated
    int64_t pstride = 0;        // slot-plane stride: bodies of the current set
    int64_t part_slots = 0;     // slots per body available to the current set
    // near-pair correction of the mixed mode (nullptr corr: not applied)
    double *corr = nullptr;     // [3][cap]
    // per linear body: table slot of its cell, arrival rank in the cell, and
    // (per cell-ordered position) the body index before ordering
    int *ng_bucket = nullptr, *ng_rank = nullptr, *ng_entry = nullptr;
    // cell-ordered copies (hi x, y, z, m) and (lo x, y, z, linear index)
    float4 *ng_spos = nullptr, *ng_slo = nullptr;
    NgSlot *ng_slot = nullptr;                       // cell table [H]
    int *ng_total = nullptr;                         // bodies placed in the grid
    int64_t ng_hcap = 0;                             // slots allocated
    double *red = nullptr;      // reduction partials [segment][16]
    int64_t red_len = 0;
    double *diag = nullptr;     // [K][16] reduction results (energy, torque)
    int *flag = nullptr;        // non-finite flag
};

// Stream-K-style decomposition of the pair work of a cluster set.  A unit is
// (cluster k, i-block b, j-range t of jt bodies); units are numbered cluster
// by cluster, u = uoff[k] + b * units_per_iblock(ntiles[k]) + t, W units in
// all.  Block g of the grid (resident at once, or run in waves when G exceeds
// the resident blocks) owns the contiguous units [U(g), U(g+1)),
// U(g) = floor(g W / G); every unit is jt x TILE*I pairs, so blocks get equal
// work whatever the cluster sizes.  Each (cluster, i-block, block g) segment
// writes its own partial slot g - gfirst; consumers add an i-block's slots in
// slot order, so results do not depend on timing.
struct Decomp {
    int32_t ipb = TILE;   // bodies per i-block = TILE * I
    // j bodies per unit: TILE or a divisor of it down to 32 (finer units give
    // small clusters enough of them to fill the GPU)
    int32_t jt = TILE;
    // rows: a unit is a whole i-block row (all its j, summed in order by one
    // block), so every body's sum is the same whatever other rows share the
    // launch; b0: first i-block of the launch (i-range launches)
    int32_t rows = 0;
    int64_t b0 = 0;
    int64_t W = 0;        // total units
    int64_t G = 1;        // blocks (grid size), 1 <= G <= W
    int64_t slots = 1;    // max partial slots any i-block needs
    // 1 when some cluster has eps = 0: the j == i term is then masked in every
    // cluster (for eps > 0 it is exactly zero anyway), which keeps the
    // decision a launch-wide constant
    int32_t mask_self = 0;
    // 1: the partial sums are float pairs (hi, lo), the single-precision pair
    // kernels' double-single sums already scaled by G m, which consumers add
    // in float-float arithmetic on the FP32 pipes; 0: doubles (FP64 and
    // float-float kernels, potential sums)
    int32_t fpart = 0;

    // 1 when (W + 1) (G + 1) < 2^32: U and owner then divide in 32 bits (a
    // 64-bit division costs tens of instructions, on the kick's hot path)
    int32_t narrow = 0;
    __host__ __device__ int64_t U(int64_t g) const
    {
        if (narrow) return (int64_t)(((uint32_t)g * (uint32_t)W) / (uint32_t)G);
        return (g * W) / G;
    }
    // largest g with U(g) <= u
    __host__ __device__ int64_t owner(int64_t u) const
    {
        if (narrow)
            return (int64_t)(((uint32_t)(u + 1) * (uint32_t)G + (uint32_t)W - 1u) / (uint32_t)W) - 1;
        return ((u + 1) * G + W - 1) / W - 1;
    }
    // units per i-block of a cluster of ntiles TILE-wide j-tiles
    __host__ __device__ int64_t units_per_iblock(int64_t ntiles) const
    {
        return rows ? 1 : ntiles * (TILE / jt);
    }
};

// Partial slots of the i-block holding linear body t of cluster k, and the
// first owner block (the slot of block g is g - first).
__device__ __forceinline__ void iblock_slots(const Decomp &d, const Clusters &c, int32_t k,
                                             int64_t li, int64_t &first, int64_t &count)
{
    const int64_t b = (li >> (__ffs(d.ipb) - 1)) - d.b0;   // ipb = TILE * I, a power of two
    const int64_t nt = d.units_per_iblock(c.ntiles[k]);
    const int64_t u0 = c.uoff[k] + b * nt;
    first = d.owner(u0);
    count = d.owner(u0 + nt - 1) - first + 1;
}

struct ExtField {
    int on;
    double G, Md, ad, bd, Mb, ab;
    double Mbh, eps2bh;   // central point mass (0: none) and its softening^2
};

// ---- launchers (pair.cu) ---------------------------------------------------
// mode: 0 = mixed (float pairs, double-single sums; near pairs corrected by
// near.cu), 1 = mixed with double-single difference on every pair,
// 2 = pure float, 3 = double, 4 = float-float (every operation on hi + lo
// pairs of floats, FP64-class accuracy on the FP32 pipes).
enum PairMode { PM_DS_NEAR = 0, PM_DS_FULL = 1, PM_FP32 = 2, PM_FP64 = 3, PM_DD = 4 };
// The single-precision family (pair_sp_kernel): its partial sums are float
// pairs (Decomp::fpart).
bool sp_family(int mode);

struct PairLaunch {
    int mode;
    int I;           // i-bodies per thread
    int blocks_per_sm;
    Decomp d;
    // every cluster has equal masses (mu[k] > 0): the pair kernels leave m
    // out of the pair term and scale the sums by mu[k]
    bool um = false;
};

// Host copy of the per-cluster values the pair kernels need per segment.  Up
// to PARAM_CLUSTERS clusters travel by value as a kernel parameter, where the
// compiler knows them to be uniform across the block (loop bounds and
// addresses then live in uniform registers); larger sets read the device
// tables of Clusters.
constexpr int PARAM_CLUSTERS = 512;

// Up to this many pairs per evaluation the mixed mode forms the double-single
// difference on every pair (PM_DS_FULL) instead of running the near-pair
// pass, whose fixed launch cost exceeds that extra arithmetic on small sets.
constexpr double DS_FULL_MAX_PAIRS = 134217728.0;   // 2^27
struct HostTab {
    int32_t K = 0;
    const int64_t *uoff = nullptr, *boff = nullptr, *nk = nullptr;
    const int64_t *noff = nullptr;   // first linear body of each cluster (NULL: 0)
    const int32_t *ntiles = nullptr;
    const float *eps2f = nullptr;
    const double *mu = nullptr;
    // launch order of the blocks (NULL: their index order): launch position
    // q runs block perm[q] of the decomposition, nperm = its grid
    const uint16_t *perm = nullptr;
    int32_t nperm = 0;
};

// Grids up to this many blocks launched by value with more than one cluster
// carry a launch order in the parameter table (uint16 entries; the table of
// PARAM_CLUSTERS clusters plus this stays inside the 32 KB parameter space).
constexpr int PERM_CAP = 4096;

// Partial slots per body at most, whatever the storage would allow.
constexpr int64_t MAX_PART_SLOTS = 128;

// Resident blocks per SM of a pair-kernel variant (occupancy query).
int pair_occupancy(int mode, int I);
bool pair_variant_exists(int mode, int I);
// Decomposition of the pair work of clusters with host-side sizes nk and
// tiles, given units per cluster (host arrays), i-block width, target grid.
Decomp make_decomp(int64_t W, int64_t max_ntiles, int ipb, int64_t G, int64_t slot_cap,
                   int jt = TILE, int rows = 0);
cudaError_t launch_pair(const DevState &s, const PairLaunch &pl, const HostTab &ht, double G,
                        cudaStream_t st);
// Potential sums phi_i = sum_{j != i} m_j / sqrt(r^2 + eps^2) (FP64) into
// slot planes of s.part (component 0); decomposition with ipb = TILE.
cudaError_t launch_potential(const DevState &s, const Decomp &d, cudaStream_t st);

// ---- near-pair correction (near.cu) ----------------------------------------
// Cell-table slots used for n bodies (four per body of every cluster).
int64_t near_table_size(int64_t n);
// corr_i = G sum over pairs closer than the cluster's near radius of the
// double-single minus the float contribution (written to s.corr).
// um: the pair kernel left the (uniform) mass out of the pair term; the
// correction does the same and scales by cl.mu[k].
cudaError_t launch_near_correct(const DevState &s, double G, bool um, cudaStream_t st);

// ---- launchers (integrate.cu) ----------------------------------------------
// Fill the body -> cluster map cid[0, n) of a cluster set.
cudaError_t launch_cluster_map(const Clusters &c, int32_t *cid, int64_t n, cudaStream_t st);
// Interleaved (linear body, 3) arrays <-> pool planes.
cudaError_t launch_unpack(const DevState &s, const double *pos, const double *vel,
                          const double *mass, cudaStream_t st);
cudaError_t launch_pack(const DevState &s, double *pos, double *vel, cudaStream_t st);
// Positions and / or velocities (NULL: kept) into the pool planes.
cudaError_t launch_set_state(const DevState &s, const double *pos, const double *vel,
                             cudaStream_t st);
// Frame origin and rms radius of every cluster; with near, also the
// near-pair radius of the mixed mode's correction pass (2 or 4 kernels).
cudaError_t launch_frame(const DevState &s, double near_frac, bool near, cudaStream_t st);
// Smallest and largest mass of every cluster into diag[k][0], diag[k][1].
cudaError_t launch_mass_range(const DevState &s, cudaStream_t st);
cudaError_t launch_split(const DevState &s, cudaStream_t st);
// One fused substep: optional kick v += wk dt_k (a_int + a_ext) from the
// partial slots of decomposition d, then drift x += wd dt_k v, then refresh
// the float planes: do_split 0 no, 1 coordinates only, 2 coordinates and the
// j-stream mass words (needed once after any load; masses never change).
cudaError_t launch_kick_drift(const DevState &s, const Decomp &d, double wk, double wd,
                              int do_kick, int do_split, const ExtField &ext, cudaStream_t st);
// The same for linear bodies [t0, t1) only.
cudaError_t launch_kick_drift_range(const DevState &s, const Decomp &d, double wk, double wd,
                                    int do_kick, int do_split, const ExtField &ext, int64_t t0,
                                    int64_t t1, cudaStream_t st);
cudaError_t launch_accel_out(const DevState &s, const Decomp &d, const ExtField &ext,
                             double *out_aos, cudaStream_t st);
// The same for linear bodies [t0, t1) only, row t - t0 of out_aos.
cudaError_t launch_accel_out_range(const DevState &s, const Decomp &d, const ExtField &ext,
                                   double *out_aos, int64_t t0, int64_t t1, cudaStream_t st);
cudaError_t launch_energy_reduce(const DevState &s, const Decomp &d, const ExtField &ext,
                                 double G, cudaStream_t st);
cudaError_t launch_torque(const DevState &s, const ExtField &ext, cudaStream_t st);

constexpr int SEG_BODIES = 512;    // bodies per reduction segment (one block each)
constexpr int DIAG_STRIDE = 16;    // doubles per cluster in diag

}  // namespace nb
