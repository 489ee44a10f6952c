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
// Pass: clear the table (one memset), insert cells and count arrivals, let
// each cell's first arrival claim its range of the cell-ordered copies (one
// atomic add on a running total), scatter, order each cell by body index and
// write the copies, correct.
//
// Deterministic: within a cell the bodies are ordered by linear index, and
// every body visits its 8 cells in a fixed order, so the FP64 correction sums
// do not depend on timing (which slot a cell lands in, and where its range
// lands, may vary; the sums do not depend on either).
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
    if (t == 0) *s.ng_total = 0;   // read only by the claim pass, which follows
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
    // the slot's end counts arrivals from -1 (the empty record) until the
    // claim pass turns it into the range end
    s.ng_rank[t] = atomicAdd(&s.ng_slot[b].end, 1) + 1;
}

// After all insertions: the first arrival of each cell claims the cell's
// range of the cell-ordered copies.  A block sums its claims (warp-shuffle
// scan, then across the warps) and takes one range of the running total with
// a single atomic add; a claim per atomic on one address would serialise.
// Ranges land in the order the blocks claim them; only their contents,
// ordered by body index, enter the sums.  The slot keeps [start, end).
constexpr int CLAIM_T = 256;

__global__ void __launch_bounds__(CLAIM_T) near_claim_kernel(DevState s)
{
    __shared__ int wsum[CLAIM_T / 32];
    __shared__ int base;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int b = -1, cnt = 0;
    if (t < s.n) {
        b = s.ng_bucket[t];
        if (b >= 0 && s.ng_rank[t] == 0)
            cnt = s.ng_slot[b].end + 1;   // arrivals counted from -1
        else
            b = -1;
    }
    int x = cnt;   // inclusive scan over the warp
    for (int d = 1; d < 32; d <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int q = 0; q < CLAIM_T / 32; ++q) {
            const int v = wsum[q];
            wsum[q] = run;
            run += v;
        }
        base = run > 0 ? atomicAdd(s.ng_total, run) : 0;
    }
    __syncthreads();
    if (b >= 0) {
        const int st = base + wsum[w] + x - cnt;
        s.ng_slot[b].start = st;
        s.ng_slot[b].end = st + cnt;
    }
}

// Bodies into their cell's range, in arrival order.
__global__ void near_scatter_kernel(DevState s)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    const int b = s.ng_bucket[t];
    if (b < 0) return;
    s.ng_entry[s.ng_slot[b].start + s.ng_rank[t]] = (int)t;
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
    const int lo = s.ng_slot[b].start, hi = s.ng_slot[b].end;
    int r = 0;
    for (int e = lo; e < hi; ++e) r += s.ng_entry[e] < (int)t ? 1 : 0;
    s.ng_spos[lo + r] = make_float4(s.xh[i], s.yh[i], s.zh[i], s.mf[i]);
    s.ng_slo[lo + r] = make_float4(s.xl[i], s.yl[i], s.zl[i], __int_as_float((int)t));
}

// One thread per body in cell order (entry e of the cell-ordered copies), so
// that the threads of a warp share cells, probes and member lists: probe its
// 8 cells (first loads issued together), then visit their bodies in cell
// order.  The cell and side are recomputed from the copy's float position
// with the cell kernel's arithmetic.  Bodies outside the grid got a zero
// correction from near_rank_kernel.  UM: the pair kernel left the common
// mass out of the pair term (multiplying its sums by it afterwards); the
// correction repeats exactly that and scales by the cluster's mass.
constexpr int NC_T = 256;   // threads per block of the correction

template <bool UM>
__global__ void __launch_bounds__(NC_T) near_correct_kernel(DevState s, double G)
{
    // per thread: the ranges of its 8 probed cells (empty: start = end), so
    // that one flat loop walks all its candidates; a loop per cell would
    // run as long as the warp's longest member list for every cell
    __shared__ int2 rng[8][NC_T];
    const int tid = threadIdx.x;
    const int64_t e0 = blockIdx.x * (int64_t)blockDim.x + tid;
    if (e0 >= *s.ng_total) return;   // bodies in the grid
    const float4 P = s.ng_spos[e0];
    const float4 Lo = s.ng_slo[e0];
    const int t = __float_as_int(Lo.w);
    const int32_t k = cluster_of(s.cl, t);
    double ax = 0.0, ay = 0.0, az = 0.0;
    int total = 0;
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
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            NgSlot c = v[q];
            int64_t b = slot[q];
            for (uint32_t p = 1; p < rg.size && c.key != key[q] && c.key != NG_EMPTY; ++p) {
                b = next_slot(b, rg);
                c = s.ng_slot[b];
            }
            const bool hit = c.key == key[q];
            rng[q][tid] = hit ? make_int2(c.start, c.end) : make_int2(0, 0);
            total += hit ? c.end - c.start : 0;
        }
    }
    const float eps2 = s.cl.eps2f[k];
    const float th2 = s.cl.frame[k].th2;
    const float xi = P.x, yi = P.y, zi = P.z;
    const float lxi = Lo.x, lyi = Lo.y, lzi = Lo.z;
    // candidates in cell order 0..7, each cell's members in body order,
    // NBT at a time: their indices are resolved first, so their position
    // loads are in flight together; only the few candidates inside the near
    // radius load their lo words (one candidate in twenty on a Plummer
    // sphere).  The body itself is the candidate at its own cell-ordered
    // position e0.
    constexpr int NBT = 4;
    int q = 0;
    int2 r = rng[0][tid];
    int e = r.x;
    for (int it = 0; it < total; it += NBT) {
        int ee[NBT];
#pragma unroll
        for (int b = 0; b < NBT; ++b) {
            ee[b] = -1;
            if (it + b < total) {
                while (e >= r.y) {
                    r = rng[++q][tid];
                    e = r.x;
                }
                ee[b] = e++;
            }
        }
        float4 Pb[NBT];
#pragma unroll
        for (int b = 0; b < NBT; ++b)
            Pb[b] = s.ng_spos[ee[b] >= 0 ? ee[b] : e0];
#pragma unroll
        for (int b = 0; b < NBT; ++b) {
            if (ee[b] < 0) break;
            const float4 Pj = Pb[b];
            // the pair kernel's float contribution, operation for operation
            const float mj = Pj.w;
            const float ddx = __fadd_rn(Pj.x, -xi);
            const float ddy = __fadd_rn(Pj.y, -yi);
            const float ddz = __fadd_rn(Pj.z, -zi);
            float r2 = __fmaf_rn(ddx, ddx, eps2);
            r2 = __fmaf_rn(ddy, ddy, r2);
            r2 = __fmaf_rn(ddz, ddz, r2);
            if (ee[b] == (int)e0 || !(r2 < th2)) continue;
            const float4 Lj = s.ng_slo[ee[b]];
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
    // empty records: key all ones, start = end = -1
    cudaError_t e = cudaMemsetAsync(s.ng_slot, 0xff, (size_t)H * sizeof(NgSlot), st);
    if (e != cudaSuccess) return e;
    near_cell_kernel<<<nbn, 256, 0, st>>>(s);
    near_claim_kernel<<<nbn, CLAIM_T, 0, st>>>(s);
    near_scatter_kernel<<<nbn, 256, 0, st>>>(s);
    near_rank_kernel<<<nbn, 256, 0, st>>>(s);
    if (um)
        near_correct_kernel<true><<<(unsigned)((s.n + NC_T - 1) / NC_T), NC_T, 0, st>>>(s, G);
    else
        near_correct_kernel<false><<<(unsigned)((s.n + NC_T - 1) / NC_T), NC_T, 0, st>>>(s, G);
    return cudaGetLastError();
}

}  // namespace nb
