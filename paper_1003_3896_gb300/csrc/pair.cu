// pair.cu -- all-pairs softened gravity (eq. 5; eq. 2 when eps = 0) on sm_103a.
//
// Every kernel here walks the same persistent decomposition (Decomp): a grid
// of G blocks, one contiguous run of (i-block, j-tile) units per block.  A
// j-tile of TILE bodies is staged in shared memory and broadcast to all
// threads; each thread owns I i-bodies and accumulates their sums in
// registers (the tiling of Sect. 3.2 after Nyland et al., with one thread
// per body generalised to I bodies per thread and the j range split across
// blocks so every SM gets the same amount of work).  Every pair of the N x N
// array is evaluated, as in the paper (Sect. 3.2), not N(N-1)/2.
//
// Single-precision family (one template, three modes):
//   PM_DS_NEAR  float pair arithmetic on coordinates relative to the frame
//               origin; pairs whose float r^2 falls below frame->th2 are
//               recomputed with the double-single coordinate difference
//               (hi_j - hi_i) + (lo_j - lo_i) and their float contribution
//               replaced; per-tile float sums are folded into double-single
//               accumulators (Sect. 4.2's software double precision).
//   PM_DS_FULL  the double-single coordinate difference on every pair.
//   PM_FP32     float coordinates and float accumulation throughout (per-tile
//               float sums added in float).
// Arithmetic is written with explicit round-to-nearest intrinsics so the
// near-pair fix-up can reproduce the main loop's float contribution bit for
// bit.  Two j bodies share each packed f32x2 instruction; rsqrt runs on the
// MUFU pipe (rsqrt.approx).
#include "nb_internal.cuh"

namespace nb {

Decomp make_decomp(int64_t n, int ipb, int64_t G)
{
    Decomp d;
    d.n = n;
    d.ipb = ipb;
    d.ntiles = (int32_t)((n + TILE - 1) / TILE);
    d.iblocks = (n + ipb - 1) / ipb;
    d.W = d.iblocks * (int64_t)d.ntiles;
    if (G > d.W) G = d.W;
    if (G < 1) G = 1;
    d.G = G;
    return d;
}

__device__ __forceinline__ float rsqrt_mufu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Add float t to the double-single number (hi, lo): Knuth's two-sum of hi and
// t, error folded into lo, then Dekker's fast two-sum to renormalise.
__device__ __forceinline__ void ds_add(float &hi, float &lo, float t)
{
    const float s = __fadd_rn(hi, t);
    const float bp = __fsub_rn(s, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(t, bp));
    const float l = __fadd_rn(lo, e);
    const float h = __fadd_rn(s, l);
    lo = __fsub_rn(l, __fsub_rn(h, s));
    hi = h;
}

template <int I>
struct IBodies {
    int idx[I];
    float2 nx[I], ny[I], nz[I];      // (-x, -x): hi coordinates, negated, packed twice
    float2 nlx[I], nly[I], nlz[I];   // lo coordinates, negated (full double-single mode)
};

// Near-pair fix-up for the 8 j bodies [jj, jj + 8) of the staged tile: for
// each pair whose float r^2 + eps^2 is below th2, subtract the float
// contribution the main loop added (recomputed identically) and add the one
// formed from the double-single coordinate difference.
template <int I>
__device__ __forceinline__ void near_fixup(const float *sx, const float *sy, const float *sz,
                                        const float *sm, int jj, int jglob, int n,
                                        const IBodies<I> &bi, const float *__restrict__ xl,
                                        const float *__restrict__ yl,
                                        const float *__restrict__ zl, float eps2, float th2,
                                        float2 (&ax)[I], float2 (&ay)[I], float2 (&az)[I])
{
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
        const int j = jglob + jj + q;
        const float xj = sx[jj + q], yj = sy[jj + q], zj = sz[jj + q], mj = sm[jj + q];
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const float dx = __fadd_rn(xj, bi.nx[k].x);
            const float dy = __fadd_rn(yj, bi.ny[k].x);
            const float dz = __fadd_rn(zj, bi.nz[k].x);
            float r2 = __fmaf_rn(dx, dx, eps2);
            r2 = __fmaf_rn(dy, dy, r2);
            r2 = __fmaf_rn(dz, dz, r2);
            if (r2 < th2 && j != bi.idx[k]) {
                const float ri = rsqrt_mufu(r2);
                const float s = __fmul_rn(__fmul_rn(mj, ri), __fmul_rn(ri, ri));
                // i past the end of the system mirrors body n-1 (its result is
                // discarded); read its lo coordinates from a valid slot
                const int ic = bi.idx[k] < n ? bi.idx[k] : n - 1;
                const float ex = __fadd_rn(dx, __fsub_rn(xl[j], xl[ic]));
                const float ey = __fadd_rn(dy, __fsub_rn(yl[j], yl[ic]));
                const float ez = __fadd_rn(dz, __fsub_rn(zl[j], zl[ic]));
                float e2 = __fmaf_rn(ex, ex, eps2);
                e2 = __fmaf_rn(ey, ey, e2);
                e2 = __fmaf_rn(ez, ez, e2);
                const float re = rsqrt_mufu(e2);
                const float se = __fmul_rn(__fmul_rn(mj, re), __fmul_rn(re, re));
                const float cx = __fsub_rn(__fmul_rn(ex, se), __fmul_rn(dx, s));
                const float cy = __fsub_rn(__fmul_rn(ey, se), __fmul_rn(dy, s));
                const float cz = __fsub_rn(__fmul_rn(ez, se), __fmul_rn(dz, s));
                if (q & 1) {
                    ax[k].y = __fadd_rn(ax[k].y, cx);
                    ay[k].y = __fadd_rn(ay[k].y, cy);
                    az[k].y = __fadd_rn(az[k].y, cz);
                } else {
                    ax[k].x = __fadd_rn(ax[k].x, cx);
                    ay[k].x = __fadd_rn(ay[k].x, cy);
                    az[k].x = __fadd_rn(az[k].x, cz);
                }
            }
        }
    }
}

// One staged tile: TILE j bodies against the thread's I i bodies, two j per
// packed instruction.  MASK zeroes the j == i term (eps = 0 diagonal tiles).
template <int I, int MODE, bool MASK>
__device__ __forceinline__ void tile_pass(const float *sx, const float *sy, const float *sz,
                                          const float *sm, const float *slx, const float *sly,
                                          const float *slz, int jglob, int n, const IBodies<I> &bi,
                                          const float *__restrict__ xl,
                                          const float *__restrict__ yl,
                                          const float *__restrict__ zl, float eps2, float th2,
                                          float2 (&ax)[I], float2 (&ay)[I], float2 (&az)[I])
{
    const float2 e2 = make_float2(eps2, eps2);
#pragma unroll 1
    for (int jj = 0; jj < TILE; jj += 8) {
        bool near = false;
#pragma unroll
        for (int q = 0; q < 8; q += 2) {
            const float2 xj = *reinterpret_cast<const float2 *>(sx + jj + q);
            const float2 yj = *reinterpret_cast<const float2 *>(sy + jj + q);
            const float2 zj = *reinterpret_cast<const float2 *>(sz + jj + q);
            const float2 mj = *reinterpret_cast<const float2 *>(sm + jj + q);
            float2 lxj, lyj, lzj;
            if (MODE == PM_DS_FULL) {
                lxj = *reinterpret_cast<const float2 *>(slx + jj + q);
                lyj = *reinterpret_cast<const float2 *>(sly + jj + q);
                lzj = *reinterpret_cast<const float2 *>(slz + jj + q);
            }
#pragma unroll
            for (int k = 0; k < I; ++k) {
                float2 dx = __fadd2_rn(xj, bi.nx[k]);
                float2 dy = __fadd2_rn(yj, bi.ny[k]);
                float2 dz = __fadd2_rn(zj, bi.nz[k]);
                if (MODE == PM_DS_FULL) {
                    dx = __fadd2_rn(dx, __fadd2_rn(lxj, bi.nlx[k]));
                    dy = __fadd2_rn(dy, __fadd2_rn(lyj, bi.nly[k]));
                    dz = __fadd2_rn(dz, __fadd2_rn(lzj, bi.nlz[k]));
                }
                float2 r2 = __ffma2_rn(dx, dx, e2);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dz, dz, r2);
                if (MODE == PM_DS_NEAR) near |= (fminf(r2.x, r2.y) < th2);
                const float2 ri = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
                float2 s = __fmul2_rn(__fmul2_rn(mj, ri), __fmul2_rn(ri, ri));
                if (MASK) {
                    if (jglob + jj + q == bi.idx[k]) s.x = 0.f;
                    if (jglob + jj + q + 1 == bi.idx[k]) s.y = 0.f;
                }
                ax[k] = __ffma2_rn(dx, s, ax[k]);
                ay[k] = __ffma2_rn(dy, s, ay[k]);
                az[k] = __ffma2_rn(dz, s, az[k]);
            }
        }
        if (MODE == PM_DS_NEAR) {
            if (__any_sync(0xffffffffu, near))
                near_fixup<I>(sx, sy, sz, sm, jj, jglob, n, bi, xl, yl, zl, eps2, th2, ax, ay, az);
        }
    }
}

template <int I, int MODE>
__global__ void __launch_bounds__(TILE) pair_sp_kernel(
    const float *__restrict__ xh, const float *__restrict__ yh, const float *__restrict__ zh,
    const float *__restrict__ mf, const float *__restrict__ xl, const float *__restrict__ yl,
    const float *__restrict__ zl, const Frame *__restrict__ frame, Decomp d, float eps2,
    int mask_self, double G, double *__restrict__ part, int64_t cap)
{
    constexpr bool FULL = (MODE == PM_DS_FULL);
    constexpr bool DSACC = (MODE != PM_FP32);
    __shared__ __align__(16) float sx[TILE], sy[TILE], sz[TILE], sm[TILE];
    __shared__ __align__(16) float slx[FULL ? TILE : 2], sly[FULL ? TILE : 2],
        slz[FULL ? TILE : 2];

    const int tid = threadIdx.x;
    const int n = (int)d.n;
    const int64_t g = blockIdx.x;
    int64_t u = d.U(g);
    const int64_t uend = d.U(g + 1);
    const float th2 = (MODE == PM_DS_NEAR) ? frame->th2 : 0.f;

    while (u < uend) {
        const int64_t b = u / d.ntiles;
        const int t0 = (int)(u - b * d.ntiles);
        const int t1 = (int)((int64_t)t0 + (uend - u) < d.ntiles ? t0 + (uend - u) : d.ntiles);
        const int64_t slot = g - d.gfirst(b);
        const int ib0 = (int)(b * d.ipb);

        IBodies<I> bi;
        float hx[I], hy[I], hz[I], lx[I], ly[I], lz[I];
        float2 ax[I], ay[I], az[I];
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = ib0 + tid + k * TILE;
            const int ic = i < n ? i : n - 1;
            bi.idx[k] = i;
            const float x = xh[ic], y = yh[ic], z = zh[ic];
            bi.nx[k] = make_float2(-x, -x);
            bi.ny[k] = make_float2(-y, -y);
            bi.nz[k] = make_float2(-z, -z);
            if (FULL) {
                const float a = xl[ic], c = yl[ic], e = zl[ic];
                bi.nlx[k] = make_float2(-a, -a);
                bi.nly[k] = make_float2(-c, -c);
                bi.nlz[k] = make_float2(-e, -e);
            }
            hx[k] = hy[k] = hz[k] = lx[k] = ly[k] = lz[k] = 0.f;
            ax[k] = ay[k] = az[k] = make_float2(0.f, 0.f);
        }

        for (int t = t0; t < t1; ++t) {
            const int jglob = t * TILE;
            const int j = jglob + tid;
            __syncthreads();
            if (j < n) {
                sx[tid] = xh[j];
                sy[tid] = yh[j];
                sz[tid] = zh[j];
                sm[tid] = mf[j];
                if (FULL) {
                    slx[tid] = xl[j];
                    sly[tid] = yl[j];
                    slz[tid] = zl[j];
                }
            } else {
                sx[tid] = FAR_F;
                sy[tid] = FAR_F;
                sz[tid] = FAR_F;
                sm[tid] = 0.f;
                if (FULL) slx[tid] = sly[tid] = slz[tid] = 0.f;
            }
            __syncthreads();
            const bool diag = mask_self && jglob < ib0 + d.ipb && jglob + TILE > ib0;
            if (diag)
                tile_pass<I, MODE, true>(sx, sy, sz, sm, slx, sly, slz, jglob, n, bi, xl, yl, zl,
                                         eps2, th2, ax, ay, az);
            else
                tile_pass<I, MODE, false>(sx, sy, sz, sm, slx, sly, slz, jglob, n, bi, xl, yl, zl,
                                          eps2, th2, ax, ay, az);
#pragma unroll
            for (int k = 0; k < I; ++k) {
                const float tx = __fadd_rn(ax[k].x, ax[k].y);
                const float ty = __fadd_rn(ay[k].x, ay[k].y);
                const float tz = __fadd_rn(az[k].x, az[k].y);
                if (DSACC) {
                    ds_add(hx[k], lx[k], tx);
                    ds_add(hy[k], ly[k], ty);
                    ds_add(hz[k], lz[k], tz);
                } else {
                    // pure float: tile sums added in float (two-level summation)
                    hx[k] = __fadd_rn(hx[k], tx);
                    hy[k] = __fadd_rn(hy[k], ty);
                    hz[k] = __fadd_rn(hz[k], tz);
                }
                ax[k] = ay[k] = az[k] = make_float2(0.f, 0.f);
            }
        }

#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = bi.idx[k];
            if (i < n) {
                const double rx = (double)hx[k] + (double)lx[k];
                const double ry = (double)hy[k] + (double)ly[k];
                const double rz = (double)hz[k] + (double)lz[k];
                double *p = part + (slot * 3) * cap + i;
                p[0] = G * rx;
                p[cap] = G * ry;
                p[2 * cap] = G * rz;
            }
        }
        u += t1 - t0;
    }
}

// Double-precision pair kernel: the plain FP64 baseline (Sect. 3.2's DP mode
// with structures of four doubles), same tiling and decomposition.
template <int I, bool POT>
__global__ void __launch_bounds__(TILE) pair_fp64_kernel(
    const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
    const double *__restrict__ m, Decomp d, double eps2, int mask_self, double G,
    double *__restrict__ part, int64_t cap)
{
    __shared__ double sx[TILE], sy[TILE], sz[TILE], sm[TILE];
    const int tid = threadIdx.x;
    const int n = (int)d.n;
    const int64_t g = blockIdx.x;
    int64_t u = d.U(g);
    const int64_t uend = d.U(g + 1);

    while (u < uend) {
        const int64_t b = u / d.ntiles;
        const int t0 = (int)(u - b * d.ntiles);
        const int t1 = (int)((int64_t)t0 + (uend - u) < d.ntiles ? t0 + (uend - u) : d.ntiles);
        const int64_t slot = g - d.gfirst(b);
        const int ib0 = (int)(b * d.ipb);
        int idx[I];
        double xi[I], yi[I], zi[I], ax[I], ay[I], az[I];
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = ib0 + tid + k * TILE;
            const int ic = i < n ? i : n - 1;
            idx[k] = i;
            xi[k] = x[ic];
            yi[k] = y[ic];
            zi[k] = z[ic];
            ax[k] = ay[k] = az[k] = 0.0;
        }
        for (int t = t0; t < t1; ++t) {
            const int jglob = t * TILE;
            const int j = jglob + tid;
            __syncthreads();
            if (j < n) {
                sx[tid] = x[j];
                sy[tid] = y[j];
                sz[tid] = z[j];
                sm[tid] = m[j];
            } else {
                sx[tid] = sy[tid] = sz[tid] = FAR_D;
                sm[tid] = 0.0;
            }
            __syncthreads();
            const bool diag = (POT || mask_self) && jglob < ib0 + d.ipb && jglob + TILE > ib0;
#pragma unroll 2
            for (int jj = 0; jj < TILE; ++jj) {
                const double xj = sx[jj], yj = sy[jj], zj = sz[jj], mj = sm[jj];
#pragma unroll
                for (int k = 0; k < I; ++k) {
                    const double dx = xj - xi[k], dy = yj - yi[k], dz = zj - zi[k];
                    double r2 = fma(dx, dx, eps2);
                    r2 = fma(dy, dy, r2);
                    r2 = fma(dz, dz, r2);
                    const double ri = rsqrt(r2);
                    if (POT) {
                        double w = mj * ri;
                        if (diag && jglob + jj == idx[k]) w = 0.0;
                        ax[k] += w;
                    } else {
                        double s = (mj * ri) * (ri * ri);
                        if (diag && jglob + jj == idx[k]) s = 0.0;
                        ax[k] = fma(dx, s, ax[k]);
                        ay[k] = fma(dy, s, ay[k]);
                        az[k] = fma(dz, s, az[k]);
                    }
                }
            }
        }
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = idx[k];
            if (i < n) {
                double *p = part + (slot * 3) * cap + i;
                if (POT) {
                    p[0] = ax[k];
                } else {
                    p[0] = G * ax[k];
                    p[cap] = G * ay[k];
                    p[2 * cap] = G * az[k];
                }
            }
        }
        u += t1 - t0;
    }
}

// ---- variant table -----------------------------------------------------------

typedef void (*sp_kernel_t)(const float *, const float *, const float *, const float *,
                            const float *, const float *, const float *, const Frame *,
                            Decomp, float, int, double, double *, int64_t);
typedef void (*dp_kernel_t)(const double *, const double *, const double *, const double *,
                            Decomp, double, int, double, double *, int64_t);

static sp_kernel_t sp_variant(int mode, int I)
{
#define NB_SP(M, II) \
    if (mode == M && I == II) return pair_sp_kernel<II, M>;
    NB_SP(PM_DS_NEAR, 1) NB_SP(PM_DS_NEAR, 2) NB_SP(PM_DS_NEAR, 4)
    NB_SP(PM_DS_FULL, 1) NB_SP(PM_DS_FULL, 2) NB_SP(PM_DS_FULL, 4)
    NB_SP(PM_FP32, 1) NB_SP(PM_FP32, 2) NB_SP(PM_FP32, 4)
#undef NB_SP
    return nullptr;
}

static dp_kernel_t dp_variant(int I)
{
    if (I == 1) return pair_fp64_kernel<1, false>;
    if (I == 2) return pair_fp64_kernel<2, false>;
    return nullptr;
}

bool pair_variant_exists(int mode, int I)
{
    if (mode == PM_FP64) return dp_variant(I) != nullptr;
    return sp_variant(mode, I) != nullptr;
}

int pair_occupancy(int mode, int I)
{
    int nb = 0;
    cudaError_t e;
    if (mode == PM_FP64)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dp_variant(I), TILE, 0);
    else
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sp_variant(mode, I), TILE, 0);
    if (e != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_pair(const DevState &s, const PairLaunch &pl, double G, double eps,
                        cudaStream_t st)
{
    const int mask_self = eps == 0.0 ? 1 : 0;
    const dim3 grid((unsigned)pl.d.G), block(TILE);
    if (pl.mode == PM_FP64) {
        dp_kernel_t k = dp_variant(pl.I);
        if (!k) return cudaErrorInvalidValue;
        k<<<grid, block, 0, st>>>(s.x, s.y, s.z, s.m, pl.d, eps * eps, mask_self, G, s.part,
                                  s.cap);
    } else {
        sp_kernel_t k = sp_variant(pl.mode, pl.I);
        if (!k) return cudaErrorInvalidValue;
        k<<<grid, block, 0, st>>>(s.xh, s.yh, s.zh, s.mf, s.xl, s.yl, s.zl, s.frame, pl.d,
                                  (float)(eps * eps), mask_self, G, s.part, s.cap);
    }
    return cudaGetLastError();
}

cudaError_t launch_potential(const DevState &s, const Decomp &d, double eps, cudaStream_t st)
{
    pair_fp64_kernel<1, true><<<(unsigned)d.G, TILE, 0, st>>>(s.x, s.y, s.z, s.m, d, eps * eps,
                                                               1, 1.0, s.part, s.cap);
    return cudaGetLastError();
}

}  // namespace nb
