// near.cu -- near-pair correction of the mixed-precision pair sum (NB_DS).
//
// The mixed pair kernel evaluates every pair in float on coordinates taken
// relative to the cluster's frame origin c (hi = fl(x - c)).  For pairs
// closer than the near radius d_th the rounding of hi dominates the error of
// the coordinate difference (Sect. 5.2's "delicate evaluation of coordinate
// difference"), so this pass finds them with a spatial grid and adds, per
// body i,
//     corr_i = G sum_{j near i, j != i} [ f(d_ij^ds) - f(d_ij^float) ]
// where d^ds = (hi_j - hi_i) + (lo_j - lo_i) is the double-single difference
// and f(d^float) is recomputed with exactly the operations of the pair
// kernel, so it cancels that kernel's float contribution to within the
// rounding of its running sum.  Cells carry the cluster index, so bodies of
// different clusters never pair.
//
// Grid: cubic cells of side h = CELL_SCALE d_th.  Since h > 2 d_th, the
// d_th-ball around a body reaches, along each axis, only its own cell and the
// neighbour on the side of the cell half the body sits in, so each body looks
// at 2 x 2 x 2 cells.  The 10% margin in CELL_SCALE absorbs the float rounding
// of x / h for every cell coordinate the key can hold.  Occupied cells live
// in an open-addressing table (linear probing, at most one cell per four
// slots, so that probes for the many empty neighbour cells end fast) whose
// slot records carry the cell's range in a cell-ordered copy of
// the bodies, so a probe costs one 16-byte load and never walks another
// cell's bodies.  Each cluster k owns the slots [4 noff[k], 4 noff[k+1]):
// its bodies' probes stay in a region proportional to its size (cache
// locality for ensembles of small clusters), and probing wraps inside it.  Near pairs are rare (a few tenths per body in a Plummer
// sphere), so the pass is dominated by these probes.
//
// Deterministic: within a cell the bodies are ordered by linear index, and
// every body visits its 8 cells in a fixed order, so the FP64 correction sums
// do not depend on timing (which slot a cell lands in may vary; the sums do
// not depend on it).
#include "nb_internal.cuh"

namespace nb {

__device__ __forceinline__ float near_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

constexpr int CELL_BITS = 15;                 // per coordinate
constexpr int CELL_OFF = 1 << (CELL_BITS - 1);
constexpr int CELL_MAX = CELL_OFF - 2;        // |cell| <= CELL_MAX, neighbours <= CELL_OFF - 1
constexpr float CELL_SCALE = 2.2f;            // h / d_th
constexpr unsigned long long NG_EMPTY = ~0ull;

__device__ __forceinline__ uint64_t cell_key(int32_t k, int cx, int cy, int cz)
{
    return ((uint64_t)(uint32_t)k << (3 * CELL_BITS)) |
           ((uint64_t)(cx + CELL_OFF) << (2 * CELL_BITS)) |
           ((uint64_t)(cy + CELL_OFF) << CELL_BITS) | (uint64_t)(cz + CELL_OFF);
}

// Region of cluster k's cells in the slot table.
constexpr int SLOTS_PER_BODY = 4;

struct Region {
    int64_t base;   // first slot
    uint32_t size;  // slots (SLOTS_PER_BODY n_k)
};

__device__ __forceinline__ Region region_of(const Clusters &c, int32_t k)
{
    Region r;
    r.base = SLOTS_PER_BODY * c.noff[k];
    r.size = (uint32_t)(SLOTS_PER_BODY * c.nk[k]);
    return r;
}

// Multiplicative (Fibonacci) hash of the key (the middle bits of
// key * 2^64/phi), reduced to the region by a multiply-shift.
__device__ __forceinline__ int64_t slot_of(uint64_t key, const Region &r)
{
    const uint32_t h = (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 32);
    return r.base + (int64_t)(((uint64_t)h * r.size) >> 32);
}

// Next slot of the linear probe, wrapping inside the region.
__device__ __forceinline__ int64_t next_slot(int64_t b, const Region &r)
{
    return b + 1 == r.base + r.size ? r.base : b + 1;
}

// Cell coordinate of v (clamped to the key's range) and the side, -1 or +1,
// of the neighbour its d_th-interval can reach.
__device__ __forceinline__ int cell_coord(float v, float inv_h, int &side)
{
    const float q = v * inv_h;
    const float f = floorf(q);
    side = q - f < 0.5f ? -1 : 1;
    return (int)fminf(fmaxf(f, -(float)CELL_MAX), (float)CELL_MAX);
}

// Per body: the cell key, insertion of the cell into the slot table and the
// body's rank among its cell's arrivals.
__global__ void near_cell_kernel(DevState s)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    const int32_t k = cluster_of(s.cl, t);
    const int64_t i = s.cl.boff[k] + t - s.cl.noff[k];
    const float dth = s.cl.frame[k].dth;
    if (!(dth > 0.f)) {   // no pair can pass the test r^2 + eps^2 < eps^2
        s.ng_bucket[t] = -1;
        return;
    }
    const float ih = 1.0f / (CELL_SCALE * dth);
    int sx, sy, sz;
    const int cx = cell_coord(s.xh[i], ih, sx), cy = cell_coord(s.yh[i], ih, sy),
              cz = cell_coord(s.zh[i], ih, sz);
    const uint64_t key = cell_key(k, cx, cy, cz);
    // the region has more slots than the cluster has bodies, so a free or
    // matching slot always exists; the bound only caps the loop
    const Region rg = region_of(s.cl, k);
    int64_t b = slot_of(key, rg);
    for (uint32_t p = 0; p < rg.size; ++p) {
        const unsigned long long prev = atomicCAS(&s.ng_slot[b].key, NG_EMPTY, key);
        if (prev == NG_EMPTY || prev == key) break;
        b = next_slot(b, rg);
    }
    s.ng_bucket[t] = (int)b;
    s.ng_rank[t] = atomicAdd(&s.ng_count[b], 1);
}

// Exclusive scan of ng_count[0, H) into ng_start: per-block scan of 1024
// entries, then a single block scans the block totals, then a fix-up pass.
constexpr int SCAN_T = 256, SCAN_E = 4, SCAN_B = SCAN_T * SCAN_E;

__global__ void scan_block_kernel(const int *__restrict__ in, int *__restrict__ out,
                                  int *__restrict__ bsum, int64_t H)
{
    __shared__ int sh[SCAN_T];
    const int64_t base = blockIdx.x * (int64_t)SCAN_B + threadIdx.x * SCAN_E;
    int v[SCAN_E], run = 0;
#pragma unroll
    for (int k = 0; k < SCAN_E; ++k) {
        v[k] = base + k < H ? in[base + k] : 0;
        run += v[k];
    }
    sh[threadIdx.x] = run;
    __syncthreads();
    for (int w = 1; w < SCAN_T; w <<= 1) {
        const int t = threadIdx.x >= w ? sh[threadIdx.x - w] : 0;
        __syncthreads();
        sh[threadIdx.x] += t;
        __syncthreads();
    }
    int acc = sh[threadIdx.x] - run;
#pragma unroll
    for (int k = 0; k < SCAN_E; ++k) {
        if (base + k < H) out[base + k] = acc;
        acc += v[k];
    }
    if (threadIdx.x == SCAN_T - 1) bsum[blockIdx.x] = sh[SCAN_T - 1];
}

// Exclusive scan of the nb block totals in one pass of one block: each of
// TOP_T threads sums its own run of ceil(nb / TOP_T) totals, the runs' sums
// are scanned with warp shuffles, and each thread writes its run's prefixes.
constexpr int TOP_T = 1024;

__global__ void __launch_bounds__(TOP_T) scan_top_kernel(int *bsum, int nb)
{
    __shared__ int wsum[TOP_T / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int per = (nb + TOP_T - 1) / TOP_T;
    const int lo = t * per, hi = lo + per < nb ? lo + per : nb;
    int local = 0;
    for (int i = lo; i < hi; ++i) local += bsum[i];
    int x = local;   // inclusive scan over the warp
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (w == 0) {
        int v = wsum[lane];
        for (int d = 1; d < 32; d <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, v, d);
            if (lane >= d) v += y;
        }
        wsum[lane] = v;
    }
    __syncthreads();
    int run = x - local + (w > 0 ? wsum[w - 1] : 0);
    for (int i = lo; i < hi; ++i) {
        const int v = bsum[i];
        bsum[i] = run;
        run += v;
    }
}

// Adds the block offsets; out[H] = the number of bodies in the grid (fewer
// than n when a cluster has no near radius, e.g. a single body).
__global__ void scan_add_kernel(int *out, const int *bsum, const int *count, int64_t H)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < H) out[i] += bsum[i / SCAN_B];
    if (i == H - 1) out[H] = out[i] + count[i];
}

// Bodies into their cell's range, in arrival order.
__global__ void near_scatter_kernel(DevState s)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    const int b = s.ng_bucket[t];
    if (b < 0) return;
    s.ng_entry[s.ng_start[b] + s.ng_rank[t]] = (int)t;
}

// Final place of each body in its cell = number of cell members with a
// smaller linear index; writes the cell-ordered copies of its float planes
// (lo.w = t) and, from the cell's first body, the slot's range.  Bodies
// outside the grid get their (zero) correction here.
__global__ void near_rank_kernel(DevState s)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    const int b = s.ng_bucket[t];
    const int32_t k = cluster_of(s.cl, t);
    const int64_t i = s.cl.boff[k] + t - s.cl.noff[k];
    if (b < 0) {   // not in the grid (no near radius): no correction
        s.corr[i] = 0.0;
        s.corr[s.cap + i] = 0.0;
        s.corr[2 * s.cap + i] = 0.0;
        return;
    }
    const int lo = s.ng_start[b], hi = s.ng_start[b + 1];
    int r = 0;
    for (int e = lo; e < hi; ++e) r += s.ng_entry[e] < (int)t ? 1 : 0;
    s.ng_spos[lo + r] = make_float4(s.xh[i], s.yh[i], s.zh[i], s.mf[i]);
    s.ng_slo[lo + r] = make_float4(s.xl[i], s.yl[i], s.zl[i], __int_as_float((int)t));
    if (r == 0) {
        s.ng_slot[b].start = lo;
        s.ng_slot[b].end = hi;
    }
}

// One thread per body in cell order (entry e of the cell-ordered copies), so
// that the threads of a warp share cells, probes and member lists: probe its
// 8 cells (first loads issued together), then visit their bodies in cell
// order.  The cell and side are recomputed from the copy's float position
// with the cell kernel's arithmetic.  Bodies outside the grid got a zero
// correction from near_rank_kernel.  UM: the pair kernel left the common
// mass out of the pair term (multiplying its sums by it afterwards); the
// correction repeats exactly that and scales by the cluster's mass.
template <bool UM>
__global__ void __launch_bounds__(256) near_correct_kernel(DevState s, double G)
{
    const int64_t e0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e0 >= s.ng_start[SLOTS_PER_BODY * s.n]) return;   // bodies in the grid
    const float4 P = s.ng_spos[e0];
    const float4 Lo = s.ng_slo[e0];
    const int t = __float_as_int(Lo.w);
    const int32_t k = cluster_of(s.cl, t);
    double ax = 0.0, ay = 0.0, az = 0.0;
    {
        const float ih = 1.0f / (CELL_SCALE * s.cl.frame[k].dth);
        int sx, sy, sz;
        const int cx = cell_coord(P.x, ih, sx), cy = cell_coord(P.y, ih, sy),
                  cz = cell_coord(P.z, ih, sz);
        const Region rg = region_of(s.cl, k);
        uint64_t key[8];
        int64_t slot[8];
        NgSlot v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            key[q] = cell_key(k, cx + (q & 1 ? sx : 0), cy + (q & 2 ? sy : 0),
                              cz + (q & 4 ? sz : 0));
            slot[q] = slot_of(key[q], rg);
            v[q] = s.ng_slot[slot[q]];
        }
        const float eps2 = s.cl.eps2f[k];
        const float th2 = s.cl.frame[k].th2;
        const float xi = P.x, yi = P.y, zi = P.z;
        const float lxi = Lo.x, lyi = Lo.y, lzi = Lo.z;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            NgSlot c = v[q];
            int64_t b = slot[q];
            for (uint32_t p = 1; p < rg.size && c.key != key[q] && c.key != NG_EMPTY; ++p) {
                b = next_slot(b, rg);
                c = s.ng_slot[b];
            }
            if (c.key != key[q]) continue;   // empty cell
            for (int e = c.start; e < c.end; ++e) {
                const float4 Pj = s.ng_spos[e];
                const float4 Lj = s.ng_slo[e];
                if (__float_as_int(Lj.w) == t) continue;
                // the pair kernel's float contribution, operation for operation
                const float mj = Pj.w;
                const float ddx = __fadd_rn(Pj.x, -xi);
                const float ddy = __fadd_rn(Pj.y, -yi);
                const float ddz = __fadd_rn(Pj.z, -zi);
                float r2 = __fmaf_rn(ddx, ddx, eps2);
                r2 = __fmaf_rn(ddy, ddy, r2);
                r2 = __fmaf_rn(ddz, ddz, r2);
                if (!(r2 < th2)) continue;
                const float ri = near_rsqrt(r2);
                const float sf = UM ? __fmul_rn(ri, __fmul_rn(ri, ri))
                                    : __fmul_rn(__fmul_rn(mj, ri), __fmul_rn(ri, ri));
                // the same pair with the double-single coordinate difference
                const float ex = __fadd_rn(ddx, __fsub_rn(Lj.x, lxi));
                const float ey = __fadd_rn(ddy, __fsub_rn(Lj.y, lyi));
                const float ez = __fadd_rn(ddz, __fsub_rn(Lj.z, lzi));
                float e2 = __fmaf_rn(ex, ex, eps2);
                e2 = __fmaf_rn(ey, ey, e2);
                e2 = __fmaf_rn(ez, ez, e2);
                const float re = near_rsqrt(e2);
                const float se = UM ? __fmul_rn(re, __fmul_rn(re, re))
                                    : __fmul_rn(__fmul_rn(mj, re), __fmul_rn(re, re));
                ax += (double)__fmul_rn(ex, se) - (double)__fmul_rn(ddx, sf);
                ay += (double)__fmul_rn(ey, se) - (double)__fmul_rn(ddy, sf);
                az += (double)__fmul_rn(ez, se) - (double)__fmul_rn(ddz, sf);
            }
        }
    }
    const int64_t i = s.cl.boff[k] + t - s.cl.noff[k];
    const double Gm = UM ? G * s.cl.mu[k] : G;
    s.corr[i] = Gm * ax;
    s.corr[s.cap + i] = Gm * ay;
    s.corr[2 * s.cap + i] = Gm * az;
}

int64_t near_table_size(int64_t n)
{
    return SLOTS_PER_BODY * n;
}

cudaError_t launch_near_correct(const DevState &s, double G, bool um, cudaStream_t st)
{
    const int64_t H = near_table_size(s.n);
    if (H > s.ng_hcap) return cudaErrorInvalidValue;
    const unsigned nbn = (unsigned)((s.n + 255) / 256);
    const unsigned nbh = (unsigned)((H + 255) / 256);
    const int nscan = (int)((H + SCAN_B - 1) / SCAN_B);
    cudaError_t e = cudaMemsetAsync(s.ng_slot, 0xff, (size_t)H * sizeof(NgSlot), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(s.ng_count, 0, (size_t)H * sizeof(int), st);
    if (e != cudaSuccess) return e;
    near_cell_kernel<<<nbn, 256, 0, st>>>(s);
    scan_block_kernel<<<nscan, SCAN_T, 0, st>>>(s.ng_count, s.ng_start, s.ng_bsum, H);
    scan_top_kernel<<<1, TOP_T, 0, st>>>(s.ng_bsum, nscan);
    scan_add_kernel<<<nbh, 256, 0, st>>>(s.ng_start, s.ng_bsum, s.ng_count, H);
    near_scatter_kernel<<<nbn, 256, 0, st>>>(s);
    near_rank_kernel<<<nbn, 256, 0, st>>>(s);
    if (um)
        near_correct_kernel<true><<<nbn, 256, 0, st>>>(s, G);
    else
        near_correct_kernel<false><<<nbn, 256, 0, st>>>(s, G);
    return cudaGetLastError();
}

}  // namespace nb
