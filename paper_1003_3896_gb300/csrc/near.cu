// near.cu -- near-pair correction of the mixed-precision pair sum (NB_DS).
//
// The mixed pair kernel evaluates every pair in float on coordinates taken
// relative to the cluster's frame origin c (hi = fl(x - c)).  For pairs
// closer than the near radius d_th the rounding of hi dominates the error of
// the coordinate difference (Sect. 4.2's "delicate evaluation of coordinate
// difference"), so this pass finds them with a spatial hash grid of cell size
// d_th and adds, per body i,
//     corr_i = G sum_{j near i, j != i} [ f(d_ij^ds) - f(d_ij^float) ]
// where d^ds = (hi_j - hi_i) + (lo_j - lo_i) is the double-single difference
// and f(d^float) is recomputed with exactly the operations of the pair
// kernel, so it cancels that kernel's float contribution to within the
// rounding of its running sum.  Cells carry the cluster index, so bodies of
// different clusters never pair.
//
// Deterministic: bodies are counting-sorted into hash buckets, each bucket is
// then sorted by linear body index, and every body visits its 27 neighbour
// cells in a fixed lane order with a fixed shuffle-tree sum, so the FP64
// correction sums do not depend on timing.
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

__device__ __forceinline__ int cell_coord(float v, float inv_h)
{
    float c = floorf(v * inv_h);
    c = fminf(fmaxf(c, -(float)(CELL_OFF - 2)), (float)(CELL_OFF - 2));
    return (int)c;
}

__device__ __forceinline__ uint64_t cell_key(int32_t k, int cx, int cy, int cz)
{
    return ((uint64_t)(uint32_t)k << (3 * CELL_BITS)) |
           ((uint64_t)(cx + CELL_OFF) << (2 * CELL_BITS)) |
           ((uint64_t)(cy + CELL_OFF) << CELL_BITS) | (uint64_t)(cz + CELL_OFF);
}

__device__ __forceinline__ uint32_t cell_bucket(int32_t k, int cx, int cy, int cz,
                                                uint32_t mask)
{
    const uint32_t h = ((uint32_t)cx * 73856093u) ^ ((uint32_t)cy * 19349663u) ^
                       ((uint32_t)cz * 83492791u) ^ ((uint32_t)k * 2654435761u);
    return h & mask;
}

// Inverse cell size: cells 0.1% wider than the near radius, so two bodies
// whose float separation is below d_th never land two cells apart after the
// rounding of x / h.
__device__ __forceinline__ float inv_cell(const Frame &f)
{
    return f.dth > 0.f ? 1.0f / (1.001f * f.dth) : 0.f;
}

__global__ void near_cell_kernel(DevState s, uint32_t mask)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    const int32_t k = cluster_of(s.cl, t);
    const int64_t i = s.cl.boff[k] + t - s.cl.noff[k];
    const float ih = inv_cell(s.cl.frame[k]);
    const int cx = cell_coord(s.xh[i], ih), cy = cell_coord(s.yh[i], ih),
              cz = cell_coord(s.zh[i], ih);
    s.ng_key[t] = cell_key(k, cx, cy, cz);
    const uint32_t b = cell_bucket(k, cx, cy, cz, mask);
    s.ng_bucket[t] = (int)b;
    atomicAdd(&s.ng_count[b], 1);
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

__global__ void scan_top_kernel(int *bsum, int nb)
{
    __shared__ int sh[SCAN_T];
    int carry = 0;
    for (int c0 = 0; c0 < nb; c0 += SCAN_T) {
        const int idx = c0 + threadIdx.x;
        const int v = idx < nb ? bsum[idx] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int w = 1; w < SCAN_T; w <<= 1) {
            const int t = threadIdx.x >= w ? sh[threadIdx.x - w] : 0;
            __syncthreads();
            sh[threadIdx.x] += t;
            __syncthreads();
        }
        if (idx < nb) bsum[idx] = carry + sh[threadIdx.x] - v;
        const int tot = sh[SCAN_T - 1];
        __syncthreads();
        carry += tot;
    }
}

__global__ void scan_add_kernel(int *out, const int *bsum, int64_t H, int64_t n)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < H) out[i] += bsum[i / SCAN_B];
    if (i == 0) out[H] = (int)n;
}

__global__ void near_scatter_kernel(DevState s)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    const int b = s.ng_bucket[t];
    const int pos = s.ng_start[b] + atomicAdd(&s.ng_count[b], 1);
    s.ng_entry[pos] = (int)t;
}

// Bodies of each bucket in ascending linear index (buckets hold ~1 body).
__global__ void near_sort_kernel(DevState s, int64_t H)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= H) return;
    const int lo = s.ng_start[b], hi = s.ng_start[b + 1];
    for (int a = lo + 1; a < hi; ++a) {
        const int v = s.ng_entry[a];
        int k = a - 1;
        while (k >= lo && s.ng_entry[k] > v) {
            s.ng_entry[k + 1] = s.ng_entry[k];
            --k;
        }
        s.ng_entry[k + 1] = v;
    }
}

// One warp per body t; lane l < 27 visits neighbour cell (l % 3 - 1,
// l / 3 % 3 - 1, l / 9 - 1); the lane sums are combined by a fixed shuffle tree.
__global__ void near_correct_kernel(DevState s, uint32_t mask, double G)
{
    const int64_t t = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= s.n) return;   // whole warps exit together
    const int32_t k = cluster_of(s.cl, t);
    const int64_t base = s.cl.boff[k] - s.cl.noff[k];
    const int64_t i = base + t;
    const Frame f = s.cl.frame[k];
    const float eps2 = s.cl.eps2f[k];
    const float th2 = f.th2;
    const float ih = inv_cell(f);
    const float xi = s.xh[i], yi = s.yh[i], zi = s.zh[i];
    const float lxi = s.xl[i], lyi = s.yl[i], lzi = s.zl[i];
    const int cx = cell_coord(xi, ih), cy = cell_coord(yi, ih), cz = cell_coord(zi, ih);
    double ax = 0.0, ay = 0.0, az = 0.0;
    if (lane < 27) {
        const int dx = lane % 3 - 1, dy = lane / 3 % 3 - 1, dz = lane / 9 - 1;
        const uint64_t key = cell_key(k, cx + dx, cy + dy, cz + dz);
        const uint32_t b = cell_bucket(k, cx + dx, cy + dy, cz + dz, mask);
        const int lo = s.ng_start[b], hi = s.ng_start[b + 1];
        for (int e = lo; e < hi; ++e) {
            const int tj = s.ng_entry[e];
            if (tj == t || s.ng_key[tj] != key) continue;
            const int64_t j = base + tj;
            // the pair kernel's float contribution, operation for operation
            const float mj = s.mf[j];
            const float ddx = __fadd_rn(s.xh[j], -xi);
            const float ddy = __fadd_rn(s.yh[j], -yi);
            const float ddz = __fadd_rn(s.zh[j], -zi);
            float r2 = __fmaf_rn(ddx, ddx, eps2);
            r2 = __fmaf_rn(ddy, ddy, r2);
            r2 = __fmaf_rn(ddz, ddz, r2);
            if (!(r2 < th2)) continue;
            const float ri = near_rsqrt(r2);
            const float sf = __fmul_rn(__fmul_rn(mj, ri), __fmul_rn(ri, ri));
            // the same pair with the double-single coordinate difference
            const float ex = __fadd_rn(ddx, __fsub_rn(s.xl[j], lxi));
            const float ey = __fadd_rn(ddy, __fsub_rn(s.yl[j], lyi));
            const float ez = __fadd_rn(ddz, __fsub_rn(s.zl[j], lzi));
            float e2 = __fmaf_rn(ex, ex, eps2);
            e2 = __fmaf_rn(ey, ey, e2);
            e2 = __fmaf_rn(ez, ez, e2);
            const float re = near_rsqrt(e2);
            const float se = __fmul_rn(__fmul_rn(mj, re), __fmul_rn(re, re));
            ax += (double)__fmul_rn(ex, se) - (double)__fmul_rn(ddx, sf);
            ay += (double)__fmul_rn(ey, se) - (double)__fmul_rn(ddy, sf);
            az += (double)__fmul_rn(ez, se) - (double)__fmul_rn(ddz, sf);
        }
    }
    for (int w = 16; w > 0; w >>= 1) {
        ax += __shfl_down_sync(0xffffffffu, ax, w);
        ay += __shfl_down_sync(0xffffffffu, ay, w);
        az += __shfl_down_sync(0xffffffffu, az, w);
    }
    if (lane == 0) {
        s.corr[i] = G * ax;
        s.corr[s.cap + i] = G * ay;
        s.corr[2 * s.cap + i] = G * az;
    }
}

int64_t near_table_size(int64_t n)
{
    int64_t H = 1024;
    while (H < 2 * n) H <<= 1;
    return H;
}

cudaError_t launch_near_correct(const DevState &s, double G, cudaStream_t st)
{
    const int64_t H = near_table_size(s.n);
    if (H > s.ng_hcap) return cudaErrorInvalidValue;
    const uint32_t mask = (uint32_t)(H - 1);
    const unsigned nbn = (unsigned)((s.n + 255) / 256);
    const unsigned nbh = (unsigned)((H + 255) / 256);
    const int nscan = (int)((H + SCAN_B - 1) / SCAN_B);
    cudaError_t e = cudaMemsetAsync(s.ng_count, 0, (size_t)H * sizeof(int), st);
    if (e != cudaSuccess) return e;
    near_cell_kernel<<<nbn, 256, 0, st>>>(s, mask);
    scan_block_kernel<<<nscan, SCAN_T, 0, st>>>(s.ng_count, s.ng_start, s.ng_bsum, H);
    scan_top_kernel<<<1, SCAN_T, 0, st>>>(s.ng_bsum, nscan);
    scan_add_kernel<<<nbh, 256, 0, st>>>(s.ng_start, s.ng_bsum, H, s.n);
    e = cudaMemsetAsync(s.ng_count, 0, (size_t)H * sizeof(int), st);
    if (e != cudaSuccess) return e;
    near_scatter_kernel<<<nbn, 256, 0, st>>>(s);
    near_sort_kernel<<<nbh, 256, 0, st>>>(s, H);
    near_correct_kernel<<<(unsigned)((s.n * 32 + 255) / 256), 256, 0, st>>>(s, mask, G);
    return cudaGetLastError();
}

}  // namespace nb
