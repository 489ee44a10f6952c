// nb_internal.cuh -- device layout, work decomposition and launcher
// declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nb {

// Tile width of the pair kernels: one j per thread per plane when a tile is
// staged in shared memory, and the i-block is TILE * I particles wide.
constexpr int TILE = 128;

// Position of padding j slots: far enough that its mass-0 contribution is an
// exact 0 and it never passes the near-pair test, small enough that its
// squared distance stays finite in float.
constexpr float FAR_F = 1.0e18f;
constexpr double FAR_D = 1.0e150;

// Reference frame of the single-precision coordinates (Sect. 4.2's
// "delicate evaluation of coordinate difference"): positions are stored as
// float hi = fl(x - c) and lo = fl((x - c) - hi).  th2 is the squared
// near-pair radius plus eps^2, compared with the float r^2 + eps^2.
struct Frame {
    double cx, cy, cz;   // reference point (mass-weighted centre)
    double r2rms;        // mass-weighted mean |x - c|^2
    float th2;           // near-pair threshold on r^2 + eps^2
    float dth;           // near-pair radius d_th (th2 = d_th^2 + eps^2)
};

// Device state of one particle system.  FP64 structure-of-arrays planes are
// the state; float planes are derived copies for the single-precision paths.
struct DevState {
    int64_t n = 0, cap = 0;
    double *x = nullptr, *y = nullptr, *z = nullptr;
    double *vx = nullptr, *vy = nullptr, *vz = nullptr, *m = nullptr;
    float *xh = nullptr, *yh = nullptr, *zh = nullptr, *mf = nullptr;
    float *xl = nullptr, *yl = nullptr, *zl = nullptr;
    // j-stream copies, two float4 per body, each coordinate duplicated so a
    // packed f32x2 operand serves two i bodies: jd = (xh, xh, yh, yh),
    // (zh, zh, m, m); jl = (xl, xl, yl, yl), (zl, zl, 0, 0).
    float4 *jd = nullptr, *jl = nullptr;
    double *part = nullptr;     // partial sums [slot][3][cap]
    int64_t part_slots = 0;
    // near-pair correction of the mixed mode (nullptr corr: not applied)
    double *corr = nullptr;     // [3][cap]
    uint64_t *ng_key = nullptr; // cell key per body
    int *ng_bucket = nullptr, *ng_entry = nullptr;   // per body
    int *ng_count = nullptr, *ng_start = nullptr;    // per bucket (start: H + 1)
    int *ng_bsum = nullptr;                          // scan block totals
    int64_t ng_hcap = 0;                             // buckets allocated
    double *red = nullptr;      // block partials of reductions
    int64_t red_len = 0;
    double *aos = nullptr;      // (cap, 3) staging for interleaved I/O
    Frame *frame = nullptr;
    double *diag = nullptr;     // [16] reduction results (energy, torque)
    int *flag = nullptr;        // non-finite flag
};

// Persistent ("stream-K") decomposition of the N x N pair work.  Unit u is
// (i-block b, j-tile t) with u = b * ntiles + t; persistent block g owns the
// contiguous units [U(g), U(g+1)), U(g) = floor(g W / G).  Each (b, g)
// segment writes its own partial slot k = g - gfirst(b); consumers add the
// slots of an i-block in slot order, so results do not depend on timing.
struct Decomp {
    int64_t n;
    int32_t ipb;      // particles per i-block = TILE * I
    int32_t ntiles;   // ceil(n / TILE)
    int64_t iblocks;  // ceil(n / ipb)
    int64_t W;        // iblocks * ntiles
    int64_t G;        // persistent blocks (grid size), 1 <= G <= W

    __host__ __device__ int64_t U(int64_t g) const { return (g * W) / G; }
    // largest g with U(g) <= u
    __host__ __device__ int64_t owner(int64_t u) const {
        return ((u + 1) * G + W - 1) / W - 1;
    }
    __host__ __device__ int64_t gfirst(int64_t b) const { return owner(b * ntiles); }
    __host__ __device__ int64_t nslots(int64_t b) const {
        return owner(b * ntiles + ntiles - 1) - gfirst(b) + 1;
    }
    __host__ __device__ int64_t max_slots() const {
        return (G + iblocks - 1) / iblocks + 1;
    }
};

Decomp make_decomp(int64_t n, int ipb, int64_t G);

struct ExtField {
    int on;
    double G, Md, ad, bd, Mb, ab;
};

// ---- launchers (pair.cu) ---------------------------------------------------
// mode: 0 = mixed with near-pair double-single fix-up, 1 = mixed with
// double-single difference on every pair, 2 = pure float, 3 = double.
enum PairMode { PM_DS_NEAR = 0, PM_DS_FULL = 1, PM_FP32 = 2, PM_FP64 = 3 };

struct PairLaunch {
    int mode;
    int I;           // i-particles per thread
    int blocks_per_sm;
    Decomp d;
};

// Resident blocks per SM of a pair-kernel variant (occupancy query).
int pair_occupancy(int mode, int I);
bool pair_variant_exists(int mode, int I);
cudaError_t launch_pair(const DevState &s, const PairLaunch &pl, double G, double eps,
                        cudaStream_t st);
// Potential sum phi_i = sum_{j != i} m_j / sqrt(r^2 + eps^2) (FP64) into
// slot planes of s.part (component 0).
cudaError_t launch_potential(const DevState &s, const Decomp &d, double eps, cudaStream_t st);

// ---- near-pair correction (near.cu) ----------------------------------------
// Hash-table buckets used for n bodies (power of two >= 2n).
int64_t near_table_size(int64_t n);
// corr_i = G sum over pairs closer than the frame's near radius of the
// double-single minus the float contribution (written to s.corr).
cudaError_t launch_near_correct(const DevState &s, double eps, double G, cudaStream_t st);

// ---- launchers (integrate.cu) ----------------------------------------------
cudaError_t launch_unpack(const DevState &s, const double *pos, const double *vel,
                          const double *mass, cudaStream_t st);
cudaError_t launch_pack(const DevState &s, double *pos, double *vel, cudaStream_t st);
cudaError_t launch_frame(const DevState &s, double near_frac, double eps, cudaStream_t st);
cudaError_t launch_split(const DevState &s, cudaStream_t st);
// One fused substep: optional kick v += hk (a_int + a_ext) from the partial
// slots of decomposition d, then drift x += hd v, then (optionally) refresh
// the float planes.
cudaError_t launch_kick_drift(const DevState &s, const Decomp &d, double hk, double hd,
                              int do_kick, int do_split, const ExtField &ext, double G,
                              cudaStream_t st);
cudaError_t launch_accel_out(const DevState &s, const Decomp &d, const ExtField &ext,
                             double G, double *out_aos, cudaStream_t st);
cudaError_t launch_energy_reduce(const DevState &s, const Decomp &d, const ExtField &ext,
                                 double G, cudaStream_t st);
cudaError_t launch_torque(const DevState &s, const ExtField &ext, cudaStream_t st);

int reduce_blocks();   // number of block partials the reductions use

}  // namespace nb
