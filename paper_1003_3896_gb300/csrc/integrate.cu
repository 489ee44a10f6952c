// integrate.cu -- O(N) kernels over a set of clusters: state layout
// conversion, the per-cluster float frame and split, the fused kick(+external
// field)/drift substep of the symplectic schemes (Sect. 3.1), and
// deterministic per-cluster reductions for the diagnostics of Sect. 5.1.
// All state arithmetic is double precision (Sect. 4.2: the time advance is
// the round-off sensitive part).
//
// Per-body kernels run over linear body indices t (cluster after cluster);
// the set's body -> cluster map gives t's cluster k, and its pool slot is
// boff[k] + t - noff[k].
// Reductions run per segment (a run of one cluster's bodies), then one block
// per cluster adds its segments in a fixed tree order.
#include "nb_internal.cuh"
#include "split.cuh"

namespace nb {

constexpr int RT = 256;   // threads per reduction block
constexpr int OT = 256;   // threads per block of the per-body kernels, at most

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Threads per block of a per-body kernel over n bodies: OT, or fewer (a
// multiple of 32) when n is small, so the blocks spread over at least ~300
// SMs' worth of slots; these kernels carry FP64 arithmetic and dependent
// loads, and a small system on a few SMs waits on one SM's FP64 pipe.
static inline int ot_for(int64_t n)
{
    int t = 32;
    while (t < OT && (int64_t)t * 304 < n) t *= 2;
    return t;
}

struct BodyRef {
    int32_t k;     // cluster
    int64_t li;    // index inside the cluster
    int64_t gi;    // pool slot
};

__device__ __forceinline__ BodyRef body_at(const Clusters &c, int64_t t)
{
    BodyRef r;
    r.k = cluster_of(c, t);
    r.li = t - c.noff[r.k];
    r.gi = c.boff[r.k] + r.li;
    return r;
}

// Acceleration of the smooth field of eq. 3, a = -grad Phi, for the
// Miyamoto-Nagai disk plus Plummer bulge potential
//   Phi = -G Md / sqrt(R^2 + (ad + sqrt(z^2 + bd^2))^2) - G Mb / sqrt(r^2 + ab^2).
// Written with three reciprocal square roots and no division: the FP64 pipe
// of this part runs at a small fraction of the FP32 rate, and a double
// division or square root costs several times an rsqrt.
__device__ __forceinline__ void field_accel(const ExtField &e, double x, double y, double z,
                                            double &ax, double &ay, double &az)
{
    // the inverse square-root powers refined in double from float estimates
    // (split.cuh: the FP64 pipe carries the kick here)
    const double R2 = x * x + y * y;
    const double s2 = z * z + e.bd * e.bd;
    const double rs = rsqrt_pow<true>(s2);       // 1 / sqrt(z^2 + bd^2)
    const double q = e.ad + s2 * rs;             // ad + sqrt(z^2 + bd^2)
    const double kd = e.G * e.Md * rsqrt_pow<false>(R2 + q * q);
    const double kb = e.G * e.Mb * rsqrt_pow<false>(R2 + z * z + e.ab * e.ab);
    double kh = 0.0;   // softened central point mass
    if (e.Mbh > 0) kh = e.G * e.Mbh * rsqrt_pow<false>(R2 + z * z + e.eps2bh);
    ax = -(kd + kb + kh) * x;
    ay = -(kd + kb + kh) * y;
    az = -(kd * q * rs + kb + kh) * z;
}

__device__ __forceinline__ double field_phi(const ExtField &e, double x, double y, double z)
{
    const double R2 = x * x + y * y;
    const double q = e.ad + sqrt(z * z + e.bd * e.bd);
    const double ph = e.Mbh > 0 ? e.G * e.Mbh * rsqrt(R2 + z * z + e.eps2bh) : 0.0;
    return -e.G * e.Md * rsqrt(R2 + q * q) - e.G * e.Mb * rsqrt(R2 + z * z + e.ab * e.ab) - ph;
}

// Tree reduction of NV doubles over a block of RT threads; fixed order.
template <int NV>
__device__ void block_sum(double (&v)[NV], double *sh)
{
    const int t = threadIdx.x;
    __syncthreads();
    for (int k = 0; k < NV; ++k) sh[k * RT + t] = v[k];
    __syncthreads();
    for (int w = RT / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int k = 0; k < NV; ++k) sh[k * RT + t] += sh[k * RT + t + w];
        __syncthreads();
    }
    for (int k = 0; k < NV; ++k) v[k] = sh[k * RT];
}

// Sum of the NV segment partials of cluster blockIdx.x (fixed order).
template <int NV>
__device__ void cluster_sum(const DevState &s, double (&v)[NV], double *sh)
{
    const int k = blockIdx.x;
    for (int q = 0; q < NV; ++q) v[q] = 0.0;
    for (int sg = s.cl.seg_off[k] + threadIdx.x; sg < s.cl.seg_off[k + 1]; sg += RT)
        for (int q = 0; q < NV; ++q) v[q] += s.red[(int64_t)sg * 16 + q];
    block_sum<NV>(v, sh);
}

// ---- layout ------------------------------------------------------------------

__global__ void unpack_kernel(DevState s, const double *__restrict__ pos,
                              const double *__restrict__ vel, const double *__restrict__ mass)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    const int64_t i = body_at(s.cl, t).gi;
    s.x[i] = pos[3 * t];
    s.y[i] = pos[3 * t + 1];
    s.z[i] = pos[3 * t + 2];
    s.vx[i] = vel[3 * t];
    s.vy[i] = vel[3 * t + 1];
    s.vz[i] = vel[3 * t + 2];
    s.m[i] = mass[t];
    s.mf[i] = __double2float_rn(mass[t]);   // masses never change after load
}

// Positions and / or velocities (NULL: kept) of a loaded state.
__global__ void set_state_kernel(DevState s, const double *__restrict__ pos,
                                 const double *__restrict__ vel)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    const int64_t i = body_at(s.cl, t).gi;
    if (pos) {
        s.x[i] = pos[3 * t];
        s.y[i] = pos[3 * t + 1];
        s.z[i] = pos[3 * t + 2];
    }
    if (vel) {
        s.vx[i] = vel[3 * t];
        s.vy[i] = vel[3 * t + 1];
        s.vz[i] = vel[3 * t + 2];
    }
}

__global__ void pack_kernel(DevState s, double *__restrict__ pos, double *__restrict__ vel)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    const int64_t i = body_at(s.cl, t).gi;
    if (pos) {
        pos[3 * t] = s.x[i];
        pos[3 * t + 1] = s.y[i];
        pos[3 * t + 2] = s.z[i];
    }
    if (vel) {
        vel[3 * t] = s.vx[i];
        vel[3 * t + 1] = s.vy[i];
        vel[3 * t + 2] = s.vz[i];
    }
}

// cid[t] = cluster of linear body t (binary search once per layout).
__global__ void cluster_map_kernel(Clusters c, int32_t *cid, int64_t n)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t < n) cid[t] = find_cluster(c.noff, c.K, t);
}

cudaError_t launch_cluster_map(const Clusters &c, int32_t *cid, int64_t n, cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    cluster_map_kernel<<<blocks_for(n, ot_for(n)), ot_for(n), 0, st>>>(c, cid, n);
    return cudaGetLastError();
}

cudaError_t launch_unpack(const DevState &s, const double *pos, const double *vel,
                          const double *mass, cudaStream_t st)
{
    unpack_kernel<<<blocks_for(s.n, ot_for(s.n)), ot_for(s.n), 0, st>>>(s, pos, vel, mass);
    return cudaGetLastError();
}

cudaError_t launch_set_state(const DevState &s, const double *pos, const double *vel,
                             cudaStream_t st)
{
    set_state_kernel<<<blocks_for(s.n, ot_for(s.n)), ot_for(s.n), 0, st>>>(s, pos, vel);
    return cudaGetLastError();
}

cudaError_t launch_pack(const DevState &s, double *pos, double *vel, cudaStream_t st)
{
    pack_kernel<<<blocks_for(s.n, ot_for(s.n)), ot_for(s.n), 0, st>>>(s, pos, vel);
    return cudaGetLastError();
}

// ---- frame and split ---------------------------------------------------------

__global__ void frame_partial_kernel(DevState s)
{
    __shared__ double sh[5 * RT];
    const int sg = blockIdx.x;
    const int32_t k = s.cl.seg_k[sg];
    const int64_t base = s.cl.boff[k] - s.cl.noff[k];
    double v[5] = {0, 0, 0, 0, 0};
    for (int64_t t = s.cl.seg_lo[sg] + threadIdx.x; t < s.cl.seg_hi[sg]; t += RT) {
        const int64_t i = base + t;
        const double m = s.m[i], x = s.x[i], y = s.y[i], z = s.z[i];
        v[0] += m;
        v[1] += m * x;
        v[2] += m * y;
        v[3] += m * z;
        v[4] += m * (x * x + y * y + z * z);
    }
    block_sum<5>(v, sh);
    if (threadIdx.x == 0)
        for (int q = 0; q < 5; ++q) s.red[(int64_t)sg * 16 + q] = v[q];
}

__global__ void frame_final_kernel(DevState s, double near_frac)
{
    __shared__ double sh[5 * RT];
    double v[5];
    cluster_sum<5>(s, v, sh);
    if (threadIdx.x == 0) {
        const int k = blockIdx.x;
        Frame f;
        const double M = v[0];
        const double iM = M > 0 ? 1.0 / M : 0.0;   // one division, four products
        f.cx = v[1] * iM;
        f.cy = v[2] * iM;
        f.cz = v[3] * iM;
        const double r2 = M > 0 ? v[4] * iM - (f.cx * f.cx + f.cy * f.cy + f.cz * f.cz) : 0.0;
        f.r2rms = r2 > 0 ? r2 : 0.0;
        // no near-pair radius yet (set by frame_scale_kernel when the plan
        // runs the near-pair pass)
        f.th2 = (float)s.cl.eps2d[k];
        f.dth = 0.f;
        s.cl.frame[k] = f;
    }
}

// Smallest and largest mass per segment, then per cluster (into diag[k][0..1]).
__global__ void mass_range_partial_kernel(DevState s)
{
    __shared__ double lo_sh[RT], hi_sh[RT];
    const int sg = blockIdx.x;
    const int32_t k = s.cl.seg_k[sg];
    const int64_t base = s.cl.boff[k] - s.cl.noff[k];
    double lo = INFINITY, hi = -INFINITY;
    for (int64_t t = s.cl.seg_lo[sg] + threadIdx.x; t < s.cl.seg_hi[sg]; t += RT) {
        const double m = s.m[base + t];
        lo = fmin(lo, m);
        hi = fmax(hi, m);
    }
    lo_sh[threadIdx.x] = lo;
    hi_sh[threadIdx.x] = hi;
    __syncthreads();
    for (int w = RT / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            lo_sh[threadIdx.x] = fmin(lo_sh[threadIdx.x], lo_sh[threadIdx.x + w]);
            hi_sh[threadIdx.x] = fmax(hi_sh[threadIdx.x], hi_sh[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        s.red[(int64_t)sg * 16] = lo_sh[0];
        s.red[(int64_t)sg * 16 + 1] = hi_sh[0];
    }
}

__global__ void mass_range_final_kernel(DevState s)
{
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= s.cl.K) return;
    double lo = INFINITY, hi = -INFINITY;
    for (int sg = s.cl.seg_off[k]; sg < s.cl.seg_off[k + 1]; ++sg) {
        lo = fmin(lo, s.red[(int64_t)sg * 16]);
        hi = fmax(hi, s.red[(int64_t)sg * 16 + 1]);
    }
    s.diag[(int64_t)k * DIAG_STRIDE] = lo;
    s.diag[(int64_t)k * DIAG_STRIDE + 1] = hi;
}

cudaError_t launch_mass_range(const DevState &s, cudaStream_t st)
{
    mass_range_partial_kernel<<<s.cl.S, RT, 0, st>>>(s);
    mass_range_final_kernel<<<(s.cl.K + 127) / 128, 128, 0, st>>>(s);
    return cudaGetLastError();
}

// Harmonic moment about the frame origin: sum m / |x - c| (per segment),
// with a floor of 1e-3 R_rms on the distance.
__global__ void frame_harmonic_kernel(DevState s)
{
    __shared__ double sh[2 * RT];
    const int sg = blockIdx.x;
    const int32_t k = s.cl.seg_k[sg];
    const int64_t base = s.cl.boff[k] - s.cl.noff[k];
    const Frame f = s.cl.frame[k];
    const double floor2 = 1e-6 * f.r2rms + 1e-300;
    double v[2] = {0, 0};
    for (int64_t t = s.cl.seg_lo[sg] + threadIdx.x; t < s.cl.seg_hi[sg]; t += RT) {
        const int64_t i = base + t;
        const double dx = s.x[i] - f.cx, dy = s.y[i] - f.cy, dz = s.z[i] - f.cz;
        v[0] += s.m[i] * rsqrt(dx * dx + dy * dy + dz * dz + floor2);
        v[1] += s.m[i];
    }
    block_sum<2>(v, sh);
    if (threadIdx.x == 0)
        for (int q = 0; q < 2; ++q) s.red[(int64_t)sg * 16 + q] = v[q];
}

// Near-pair radius d_th = near_frac * S / N^{1/3}: a mean-spacing scale like
// the paper's softening rule (Sect. 2), so the expected number of near
// neighbours per body does not grow with N.  S = min(R_rms, 3 R_h) with the
// harmonic radius R_h = M / sum(m / |x - c|): for centrally concentrated
// clusters (Plummer: R_rms = 2.6 R_h; uniform sphere: 1.2 R_h) S is the rms
// radius, but once escapers or a disrupted halo inflate R_rms, S follows the
// bound core instead, so the core does not crowd into a few cells.
__global__ void frame_scale_kernel(DevState s, double near_frac)
{
    __shared__ double sh[2 * RT];
    double v[2];
    cluster_sum<2>(s, v, sh);
    if (threadIdx.x == 0) {
        const int k = blockIdx.x;
        Frame f = s.cl.frame[k];
        double scale2 = f.r2rms;
        if (v[0] > 0) {
            const double rh = v[1] / v[0];
            if (9.0 * rh * rh < scale2) scale2 = 9.0 * rh * rh;
        }
        const double nk = (double)s.cl.nk[k];
        const double spacing2 = scale2 / cbrt(nk * nk);
        f.th2 = (float)(near_frac * near_frac * spacing2 + s.cl.eps2d[k]);
        f.dth = (float)(near_frac * sqrt(spacing2));
        s.cl.frame[k] = f;
    }
}

cudaError_t launch_frame(const DevState &s, double near_frac, bool near, cudaStream_t st)
{
    frame_partial_kernel<<<s.cl.S, RT, 0, st>>>(s);
    frame_final_kernel<<<s.cl.K, RT, 0, st>>>(s, near_frac);
    if (near) {
        frame_harmonic_kernel<<<s.cl.S, RT, 0, st>>>(s);
        frame_scale_kernel<<<s.cl.K, RT, 0, st>>>(s, near_frac);
    }
    return cudaGetLastError();
}

// hi = fl32(x - c), lo = fl32((x - c) - hi): the double-single representation
// of Sect. 5.2, taken relative to the cluster's frame origin.
// MASS: also write the mass words of the j-stream copies (m and its float
// rounding residue); the kick's per-substep splits leave them as the step's
// first split wrote them (masses never change).
template <bool MASS>
__device__ __forceinline__ void split_one(const DevState &s, const Frame &f, int64_t i,
                                          double x, double y, double z)
{
    float hx, hy, hz, lx, ly, lz;
    split_ds(x - f.cx, hx, lx);
    split_ds(y - f.cy, hy, ly);
    split_ds(z - f.cz, hz, lz);
    s.xh[i] = hx;
    s.yh[i] = hy;
    s.zh[i] = hz;
    s.xl[i] = lx;
    s.yl[i] = ly;
    s.zl[i] = lz;
    s.jd[2 * i] = make_float4(hx, hx, hy, hy);
    s.jl[2 * i] = make_float4(lx, lx, ly, ly);
    if (MASS) {
        const float m = s.mf[i];
        const float ml = __double2float_rn(s.m[i] - (double)m);   // mass lo part (float-float)
        s.jd[2 * i + 1] = make_float4(hz, hz, m, m);
        s.jl[2 * i + 1] = make_float4(lz, lz, ml, ml);
    } else {
        *reinterpret_cast<float2 *>(&s.jd[2 * i + 1]) = make_float2(hz, hz);
        *reinterpret_cast<float2 *>(&s.jl[2 * i + 1]) = make_float2(lz, lz);
    }
}

__global__ void split_kernel(DevState s)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= s.n) return;
    const BodyRef r = body_at(s.cl, t);
    const int64_t i = r.gi;
    s.mf[i] = __double2float_rn(s.m[i]);
    split_one<true>(s, s.cl.frame[r.k], i, s.x[i], s.y[i], s.z[i]);
}

cudaError_t launch_split(const DevState &s, cudaStream_t st)
{
    split_kernel<<<blocks_for(s.n, ot_for(s.n)), ot_for(s.n), 0, st>>>(s);
    return cudaGetLastError();
}

// ---- substep -----------------------------------------------------------------

// SB: slots loaded together (a grid run in waves gives an i-block tens of
// slots; an ensemble of small clusters a few, where a narrower batch keeps
// registers, and so resident warps, for the memory latency)
// Add the float pair (p, e) to the float-float number (h, l): Knuth's
// two-sum of the high parts, the error and the low parts folded in, then
// Dekker's fast two-sum to renormalise.
__device__ __forceinline__ void ff_add(float &h, float &l, float p, float e)
{
    const float s = __fadd_rn(h, p);
    const float bp = __fsub_rn(s, h);
    const float err = __fadd_rn(__fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(p, bp)),
                                __fadd_rn(l, e));
    h = __fadd_rn(s, err);
    l = __fsub_rn(err, __fsub_rn(h, s));
}

// Float-pair partial sums (Decomp::fpart): added in slot order in
// float-float arithmetic, SB loads at a time, then widened to double from
// their bits (the conversion instruction runs on the FP64 pipe, 1/77 of the
// FP32 rate here).
template <int SB>
__device__ __forceinline__ void sum_slots_ff(const DevState &s, int64_t count, int64_t t,
                                             double &ax, double &ay, double &az)
{
    const float2 *part2 = reinterpret_cast<const float2 *>(s.part);
    float hx = 0.f, lx = 0.f, hy = 0.f, ly = 0.f, hz = 0.f, lz = 0.f;
    for (int64_t k0 = 0; k0 < count; k0 += SB) {
        float2 bx[SB], by[SB], bz[SB];
#pragma unroll
        for (int q = 0; q < SB; ++q) {
            bx[q] = by[q] = bz[q] = make_float2(0.f, 0.f);
            if (k0 + q < count) {
                const float2 *p = part2 + ((k0 + q) * 3) * s.pstride + t;
                bx[q] = p[0];
                by[q] = p[s.pstride];
                bz[q] = p[2 * s.pstride];
            }
        }
#pragma unroll
        for (int q = 0; q < SB; ++q)
            if (k0 + q < count) {
                ff_add(hx, lx, bx[q].x, bx[q].y);
                ff_add(hy, ly, by[q].x, by[q].y);
                ff_add(hz, lz, bz[q].x, bz[q].y);
            }
    }
    ax = widen(hx) + widen(lx);
    ay = widen(hy) + widen(ly);
    az = widen(hz) + widen(lz);
}

template <int SB, bool FP>
__device__ __forceinline__ void sum_slots(const DevState &s, const Decomp &d, const BodyRef &r,
                                          int64_t t, double &ax, double &ay, double &az)
{
    int64_t first, count;
    iblock_slots(d, s.cl, r.k, r.li, first, count);
    (void)first;
    if (FP) {
        sum_slots_ff<SB>(s, count, t, ax, ay, az);
        if (s.corr) {
            ax += s.corr[r.gi];
            ay += s.corr[s.cap + r.gi];
            az += s.corr[2 * s.cap + r.gi];
        }
        return;
    }
    ax = ay = az = 0.0;
    // slots in order, SB at a time so the loads are in flight together
    for (int64_t k0 = 0; k0 < count; k0 += SB) {
        double bx[SB], by[SB], bz[SB];
#pragma unroll
        for (int q = 0; q < SB; ++q) {
            bx[q] = by[q] = bz[q] = 0.0;
            if (k0 + q < count) {
                const double *p = s.part + ((k0 + q) * 3) * s.pstride + t;
                bx[q] = p[0];
                by[q] = p[s.pstride];
                bz[q] = p[2 * s.pstride];
            }
        }
#pragma unroll
        for (int q = 0; q < SB; ++q)
            if (k0 + q < count) {
                ax += bx[q];
                ay += by[q];
                az += bz[q];
            }
    }
    if (s.corr) {
        ax += s.corr[r.gi];
        ay += s.corr[s.cap + r.gi];
        az += s.corr[2 * s.cap + r.gi];
    }
}

// EXT: the external field is on (a separate variant keeps its registers out
// of the field-free kick).
template <bool EXT, int SB, bool FP>
__global__ void kick_drift_kernel(DevState s, Decomp d, double wk, double wd, int do_kick,
                                  int do_split, ExtField ext, int64_t t0, int64_t t1)
{
    const int64_t t = t0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= t1) return;
    const BodyRef r = body_at(s.cl, t);
    const int64_t i = r.gi;
    const double dt = s.cl.dts[r.k];
    double x = s.x[i], y = s.y[i], z = s.z[i];
    double vx = s.vx[i], vy = s.vy[i], vz = s.vz[i];
    if (do_kick) {
        double ax, ay, az;
        sum_slots<SB, FP>(s, d, r, t, ax, ay, az);
        if (EXT) {
            double ex, ey, ez;
            field_accel(ext, x, y, z, ex, ey, ez);
            ax += ex;
            ay += ey;
            az += ez;
        }
        const double hk = wk * dt;
        vx += hk * ax;
        vy += hk * ay;
        vz += hk * az;
        s.vx[i] = vx;
        s.vy[i] = vy;
        s.vz[i] = vz;
    }
    const double hd = wd * dt;
    x += hd * vx;
    y += hd * vy;
    z += hd * vz;
    s.x[i] = x;
    s.y[i] = y;
    s.z[i] = z;
    if (do_split == 2)
        split_one<true>(s, s.cl.frame[r.k], i, x, y, z);
    else if (do_split)
        split_one<false>(s, s.cl.frame[r.k], i, x, y, z);
}

cudaError_t launch_kick_drift(const DevState &s, const Decomp &d, double wk, double wd,
                              int do_kick, int do_split, const ExtField &ext, cudaStream_t st)
{
    return launch_kick_drift_range(s, d, wk, wd, do_kick, do_split, ext, 0, s.n, st);
}

cudaError_t launch_kick_drift_range(const DevState &s, const Decomp &d, double wk, double wd,
                                    int do_kick, int do_split, const ExtField &ext, int64_t t0,
                                    int64_t t1, cudaStream_t st)
{
    if (t1 <= t0) return cudaSuccess;
    // blocks of at most 128 threads: with ~100 registers a thread, 128-thread
    // blocks pack 20 warps on an SM against 16 for 256 (the kick waits on
    // memory; the ensemble's kick ran 8% faster)
    const int64_t m = t1 - t0;
    const int t = ot_for(m) < 128 ? ot_for(m) : 128;
    const unsigned nb = blocks_for(m, t);
    const bool narrow = d.slots <= 4;   // every i-block has at most 4 slots
#define NB_KD(E, B, F) kick_drift_kernel<E, B, F><<<nb, t, 0, st>>>(s, d, wk, wd, do_kick, do_split, ext, t0, t1)
    if (d.fpart) {
        if (ext.on) {
            if (narrow) NB_KD(true, 4, true); else NB_KD(true, 8, true);
        } else {
            if (narrow) NB_KD(false, 4, true); else NB_KD(false, 8, true);
        }
    } else {
        if (ext.on) {
            if (narrow) NB_KD(true, 4, false); else NB_KD(true, 8, false);
        } else {
            if (narrow) NB_KD(false, 4, false); else NB_KD(false, 8, false);
        }
    }
#undef NB_KD
    return cudaGetLastError();
}

template <bool FP>
__global__ void accel_out_kernel(DevState s, Decomp d, ExtField ext, double *__restrict__ out,
                                 int64_t t0, int64_t t1)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t t = t0 + q;
    if (t >= t1) return;
    const BodyRef r = body_at(s.cl, t);
    double ax, ay, az;
    sum_slots<8, FP>(s, d, r, t, ax, ay, az);
    if (ext.on) {
        double ex, ey, ez;
        field_accel(ext, s.x[r.gi], s.y[r.gi], s.z[r.gi], ex, ey, ez);
        ax += ex;
        ay += ey;
        az += ez;
    }
    out[3 * q] = ax;
    out[3 * q + 1] = ay;
    out[3 * q + 2] = az;
    if (!isfinite(ax) || !isfinite(ay) || !isfinite(az)) atomicOr(s.flag, 1);
}

cudaError_t launch_accel_out(const DevState &s, const Decomp &d, const ExtField &ext,
                             double *out_aos, cudaStream_t st)
{
    return launch_accel_out_range(s, d, ext, out_aos, 0, s.n, st);
}

cudaError_t launch_accel_out_range(const DevState &s, const Decomp &d, const ExtField &ext,
                                   double *out_aos, int64_t t0, int64_t t1, cudaStream_t st)
{
    const int t = ot_for(t1 - t0);
    if (d.fpart)
        accel_out_kernel<true><<<blocks_for(t1 - t0, t), t, 0, st>>>(s, d, ext, out_aos, t0, t1);
    else
        accel_out_kernel<false><<<blocks_for(t1 - t0, t), t, 0, st>>>(s, d, ext, out_aos, t0, t1);
    return cudaGetLastError();
}

// ---- diagnostics -------------------------------------------------------------

// Per segment: K, sum m_i phi_i, W_ext, P, L, non-finite count (10 values).
// d is the potential kernel's decomposition (s.cl.uoff must be its units).
__global__ void energy_partial_kernel(DevState s, Decomp d, ExtField ext)
{
    __shared__ double sh[10 * RT];
    const int sg = blockIdx.x;
    const int32_t k = s.cl.seg_k[sg];
    double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t t = s.cl.seg_lo[sg] + threadIdx.x; t < s.cl.seg_hi[sg]; t += RT) {
        BodyRef r;
        r.k = k;
        r.li = t - s.cl.noff[k];
        r.gi = s.cl.boff[k] + r.li;
        const int64_t i = r.gi;
        const double m = s.m[i], x = s.x[i], y = s.y[i], z = s.z[i];
        const double vx = s.vx[i], vy = s.vy[i], vz = s.vz[i];
        int64_t first, count;
        iblock_slots(d, s.cl, k, r.li, first, count);
        double phi = 0.0;
        for (int64_t q0 = 0; q0 < count; q0 += 8) {
            double bp[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                bp[q] = q0 + q < count ? s.part[((q0 + q) * 3) * s.pstride + t] : 0.0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (q0 + q < count) phi += bp[q];
        }
        v[0] += 0.5 * m * (vx * vx + vy * vy + vz * vz);
        v[1] += m * phi;
        if (ext.on) v[2] += m * field_phi(ext, x, y, z);
        v[3] += m * vx;
        v[4] += m * vy;
        v[5] += m * vz;
        v[6] += m * (y * vz - z * vy);
        v[7] += m * (z * vx - x * vz);
        v[8] += m * (x * vy - y * vx);
        if (!isfinite(phi) || !isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(vx) ||
            !isfinite(vy) || !isfinite(vz))
            v[9] += 1.0;
    }
    block_sum<10>(v, sh);
    if (threadIdx.x == 0)
        for (int q = 0; q < 10; ++q) s.red[(int64_t)sg * 16 + q] = v[q];
}

__global__ void energy_final_kernel(DevState s, double G)
{
    __shared__ double sh[10 * RT];
    double v[10];
    cluster_sum<10>(s, v, sh);
    if (threadIdx.x == 0) {
        double *o = s.diag + (int64_t)blockIdx.x * DIAG_STRIDE;
        const double W = -0.5 * G * v[1];
        o[0] = v[0];
        o[1] = W;
        o[2] = v[2];
        o[3] = v[0] + W + v[2];
        for (int q = 0; q < 6; ++q) o[4 + q] = v[3 + q];
        if (v[9] != 0.0 || !isfinite(o[3])) atomicOr(s.flag, 1);
    }
}

cudaError_t launch_energy_reduce(const DevState &s, const Decomp &d, const ExtField &ext,
                                 double G, cudaStream_t st)
{
    energy_partial_kernel<<<s.cl.S, RT, 0, st>>>(s, d, ext);
    energy_final_kernel<<<s.cl.K, RT, 0, st>>>(s, G);
    return cudaGetLastError();
}

// External torque of eq. 8: sum m_i r_i x a_ext(r_i), per cluster.
__global__ void torque_partial_kernel(DevState s, ExtField ext)
{
    __shared__ double sh[3 * RT];
    const int sg = blockIdx.x;
    const int32_t k = s.cl.seg_k[sg];
    const int64_t base = s.cl.boff[k] - s.cl.noff[k];
    double v[3] = {0, 0, 0};
    for (int64_t t = s.cl.seg_lo[sg] + threadIdx.x; t < s.cl.seg_hi[sg]; t += RT) {
        const int64_t i = base + t;
        const double m = s.m[i], x = s.x[i], y = s.y[i], z = s.z[i];
        double ax, ay, az;
        field_accel(ext, x, y, z, ax, ay, az);
        v[0] += m * (y * az - z * ay);
        v[1] += m * (z * ax - x * az);
        v[2] += m * (x * ay - y * ax);
    }
    block_sum<3>(v, sh);
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) s.red[(int64_t)sg * 16 + q] = v[q];
}

__global__ void torque_final_kernel(DevState s)
{
    __shared__ double sh[3 * RT];
    double v[3];
    cluster_sum<3>(s, v, sh);
    if (threadIdx.x == 0)
        for (int q = 0; q < 3; ++q) s.diag[(int64_t)blockIdx.x * DIAG_STRIDE + 10 + q] = v[q];
}

cudaError_t launch_torque(const DevState &s, const ExtField &ext, cudaStream_t st)
{
    torque_partial_kernel<<<s.cl.S, RT, 0, st>>>(s, ext);
    torque_final_kernel<<<s.cl.K, RT, 0, st>>>(s);
    return cudaGetLastError();
}

}  // namespace nb
