// integrate.cu -- O(N) kernels: state layout conversion, the float frame and
// split, the fused kick(+external field)/drift substep of the symplectic
// schemes (Sect. 3.1), and deterministic reductions for the diagnostics of
// Sect. 4.1.  All state arithmetic is double precision (Sect. 3.2: the time
// advance is the round-off sensitive part).
#include "nb_internal.cuh"

namespace nb {

constexpr int RB = 256;        // reduction blocks (fixed: results independent of timing)
constexpr int RT = 256;        // threads per reduction block
constexpr int OT = 256;        // threads per block of the per-particle kernels

int reduce_blocks() { return RB; }

static inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

// Acceleration of the smooth field of eq. 3, a = -grad Phi, for the
// Miyamoto-Nagai disk plus Plummer bulge potential
//   Phi = -G Md / sqrt(R^2 + (ad + sqrt(z^2 + bd^2))^2) - G Mb / sqrt(r^2 + ab^2).
// Written with three reciprocal square roots and no division: the FP64 pipe
// of this part runs at a small fraction of the FP32 rate, and a double
// division or square root costs several times an rsqrt.
__device__ __forceinline__ void field_accel(const ExtField &e, double x, double y, double z,
                                            double &ax, double &ay, double &az)
{
    const double R2 = x * x + y * y;
    const double s2 = z * z + e.bd * e.bd;
    const double rs = rsqrt(s2);                 // 1 / sqrt(z^2 + bd^2)
    const double q = e.ad + s2 * rs;             // ad + sqrt(z^2 + bd^2)
    const double rD = rsqrt(R2 + q * q);
    const double kd = e.G * e.Md * (rD * rD * rD);
    const double rB = rsqrt(R2 + z * z + e.ab * e.ab);
    const double kb = e.G * e.Mb * (rB * rB * rB);
    ax = -(kd + kb) * x;
    ay = -(kd + kb) * y;
    az = -(kd * q * rs + kb) * z;
}

__device__ __forceinline__ double field_phi(const ExtField &e, double x, double y, double z)
{
    const double R2 = x * x + y * y;
    const double q = e.ad + sqrt(z * z + e.bd * e.bd);
    return -e.G * e.Md * rsqrt(R2 + q * q) - e.G * e.Mb * rsqrt(R2 + z * z + e.ab * e.ab);
}

// Tree reduction of NV doubles over a block of RT threads; fixed order.
template <int NV>
__device__ void block_sum(double (&v)[NV], double *sh)
{
    const int t = threadIdx.x;
    for (int k = 0; k < NV; ++k) sh[k * RT + t] = v[k];
    __syncthreads();
    for (int w = RT / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int k = 0; k < NV; ++k) sh[k * RT + t] += sh[k * RT + t + w];
        __syncthreads();
    }
    for (int k = 0; k < NV; ++k) v[k] = sh[k * RT];
}

// ---- layout ------------------------------------------------------------------

__global__ void unpack_kernel(DevState s, const double *__restrict__ pos,
                              const double *__restrict__ vel, const double *__restrict__ mass)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    s.x[i] = pos[3 * i];
    s.y[i] = pos[3 * i + 1];
    s.z[i] = pos[3 * i + 2];
    s.vx[i] = vel[3 * i];
    s.vy[i] = vel[3 * i + 1];
    s.vz[i] = vel[3 * i + 2];
    s.m[i] = mass[i];
    s.mf[i] = __double2float_rn(mass[i]);   // masses never change after load
}

__global__ void pack_kernel(DevState s, double *__restrict__ pos, double *__restrict__ vel)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    if (pos) {
        pos[3 * i] = s.x[i];
        pos[3 * i + 1] = s.y[i];
        pos[3 * i + 2] = s.z[i];
    }
    if (vel) {
        vel[3 * i] = s.vx[i];
        vel[3 * i + 1] = s.vy[i];
        vel[3 * i + 2] = s.vz[i];
    }
}

cudaError_t launch_unpack(const DevState &s, const double *pos, const double *vel,
                          const double *mass, cudaStream_t st)
{
    unpack_kernel<<<blocks_for(s.n, OT), OT, 0, st>>>(s, pos, vel, mass);
    return cudaGetLastError();
}

cudaError_t launch_pack(const DevState &s, double *pos, double *vel, cudaStream_t st)
{
    pack_kernel<<<blocks_for(s.n, OT), OT, 0, st>>>(s, pos, vel);
    return cudaGetLastError();
}

// ---- frame and split ---------------------------------------------------------

__global__ void frame_partial_kernel(DevState s)
{
    __shared__ double sh[5 * RT];
    double v[5] = {0, 0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < s.n; i += (int64_t)RB * RT) {
        const double m = s.m[i], x = s.x[i], y = s.y[i], z = s.z[i];
        v[0] += m;
        v[1] += m * x;
        v[2] += m * y;
        v[3] += m * z;
        v[4] += m * (x * x + y * y + z * z);
    }
    block_sum<5>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 5; ++k) s.red[blockIdx.x * 5 + k] = v[k];
}

__global__ void frame_final_kernel(DevState s, double near_frac, double eps)
{
    __shared__ double sh[5 * RT];
    double v[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < RB; b += RT)
        for (int k = 0; k < 5; ++k) v[k] += s.red[b * 5 + k];
    block_sum<5>(v, sh);
    if (threadIdx.x == 0) {
        Frame f;
        const double M = v[0];
        f.cx = M > 0 ? v[1] / M : 0.0;
        f.cy = M > 0 ? v[2] / M : 0.0;
        f.cz = M > 0 ? v[3] / M : 0.0;
        double r2 = M > 0 ? v[4] / M - (f.cx * f.cx + f.cy * f.cy + f.cz * f.cz) : 0.0;
        f.r2rms = r2 > 0 ? r2 : 0.0;
        // near-pair radius: near_frac times the rms radius over N^{1/3}, a
        // mean-spacing scale like the paper's softening rule (Sect. 2), so
        // the expected number of near neighbours per body is independent of N
        const double spacing2 = f.r2rms / cbrt((double)s.n * (double)s.n);
        f.th2 = (float)(near_frac * near_frac * spacing2 + eps * eps);
        f.dth = (float)(near_frac * sqrt(spacing2));
        *s.frame = f;
    }
}

cudaError_t launch_frame(const DevState &s, double near_frac, double eps, cudaStream_t st)
{
    frame_partial_kernel<<<RB, RT, 0, st>>>(s);
    frame_final_kernel<<<1, RT, 0, st>>>(s, near_frac, eps);
    return cudaGetLastError();
}

// hi = fl32(x - c), lo = fl32((x - c) - hi): the double-single representation
// of Sect. 4.2, taken relative to the frame origin.
__device__ __forceinline__ void split_one(const DevState &s, const Frame &f, int64_t i,
                                          double x, double y, double z)
{
    const double rx = x - f.cx, ry = y - f.cy, rz = z - f.cz;
    const float hx = __double2float_rn(rx), hy = __double2float_rn(ry),
                hz = __double2float_rn(rz);
    s.xh[i] = hx;
    s.yh[i] = hy;
    s.zh[i] = hz;
    const float lx = __double2float_rn(rx - (double)hx);
    const float ly = __double2float_rn(ry - (double)hy);
    const float lz = __double2float_rn(rz - (double)hz);
    s.xl[i] = lx;
    s.yl[i] = ly;
    s.zl[i] = lz;
    const float m = s.mf[i];
    s.jd[2 * i] = make_float4(hx, hx, hy, hy);
    s.jd[2 * i + 1] = make_float4(hz, hz, m, m);
    s.jl[2 * i] = make_float4(lx, lx, ly, ly);
    s.jl[2 * i + 1] = make_float4(lz, lz, 0.f, 0.f);
}

__global__ void split_kernel(DevState s)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    const Frame f = *s.frame;
    s.mf[i] = __double2float_rn(s.m[i]);
    split_one(s, f, i, s.x[i], s.y[i], s.z[i]);
}

cudaError_t launch_split(const DevState &s, cudaStream_t st)
{
    split_kernel<<<blocks_for(s.n, OT), OT, 0, st>>>(s);
    return cudaGetLastError();
}

// ---- substep -----------------------------------------------------------------

__device__ __forceinline__ void sum_slots(const DevState &s, const Decomp &d, int64_t i,
                                          double &ax, double &ay, double &az)
{
    const int64_t b = i / d.ipb;
    const int64_t ns = d.nslots(b);
    ax = ay = az = 0.0;
    for (int64_t k = 0; k < ns; ++k) {
        const double *p = s.part + (k * 3) * s.cap + i;
        ax += p[0];
        ay += p[s.cap];
        az += p[2 * s.cap];
    }
    if (s.corr) {
        ax += s.corr[i];
        ay += s.corr[s.cap + i];
        az += s.corr[2 * s.cap + i];
    }
}

__global__ void kick_drift_kernel(DevState s, Decomp d, double hk, double hd, int do_kick,
                                  int do_split, ExtField ext)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    double x = s.x[i], y = s.y[i], z = s.z[i];
    double vx = s.vx[i], vy = s.vy[i], vz = s.vz[i];
    if (do_kick) {
        double ax, ay, az;
        sum_slots(s, d, i, ax, ay, az);
        if (ext.on) {
            double ex, ey, ez;
            field_accel(ext, x, y, z, ex, ey, ez);
            ax += ex;
            ay += ey;
            az += ez;
        }
        vx += hk * ax;
        vy += hk * ay;
        vz += hk * az;
        s.vx[i] = vx;
        s.vy[i] = vy;
        s.vz[i] = vz;
    }
    x += hd * vx;
    y += hd * vy;
    z += hd * vz;
    s.x[i] = x;
    s.y[i] = y;
    s.z[i] = z;
    if (do_split) split_one(s, *s.frame, i, x, y, z);
}

cudaError_t launch_kick_drift(const DevState &s, const Decomp &d, double hk, double hd,
                              int do_kick, int do_split, const ExtField &ext, double G,
                              cudaStream_t st)
{
    (void)G;
    kick_drift_kernel<<<blocks_for(s.n, OT), OT, 0, st>>>(s, d, hk, hd, do_kick, do_split, ext);
    return cudaGetLastError();
}

__global__ void accel_out_kernel(DevState s, Decomp d, ExtField ext, double *__restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    double ax, ay, az;
    sum_slots(s, d, i, ax, ay, az);
    if (ext.on) {
        double ex, ey, ez;
        field_accel(ext, s.x[i], s.y[i], s.z[i], ex, ey, ez);
        ax += ex;
        ay += ey;
        az += ez;
    }
    out[3 * i] = ax;
    out[3 * i + 1] = ay;
    out[3 * i + 2] = az;
    if (!isfinite(ax) || !isfinite(ay) || !isfinite(az)) atomicOr(s.flag, 1);
}

cudaError_t launch_accel_out(const DevState &s, const Decomp &d, const ExtField &ext,
                             double G, double *out_aos, cudaStream_t st)
{
    (void)G;
    accel_out_kernel<<<blocks_for(s.n, OT), OT, 0, st>>>(s, d, ext, out_aos);
    return cudaGetLastError();
}

// ---- diagnostics -------------------------------------------------------------

// Per block: K, sum m_i phi_i, W_ext, P, L (10 values).
__global__ void energy_partial_kernel(DevState s, Decomp d, ExtField ext)
{
    __shared__ double sh[10 * RT];
    double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < s.n; i += (int64_t)RB * RT) {
        const double m = s.m[i], x = s.x[i], y = s.y[i], z = s.z[i];
        const double vx = s.vx[i], vy = s.vy[i], vz = s.vz[i];
        const int64_t ns = d.nslots(i / d.ipb);
        double phi = 0.0;
        for (int64_t k = 0; k < ns; ++k) phi += s.part[(k * 3) * s.cap + i];
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
        for (int k = 0; k < 10; ++k) s.red[blockIdx.x * 10 + k] = v[k];
}

__global__ void energy_final_kernel(DevState s, double G)
{
    __shared__ double sh[10 * RT];
    double v[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < RB; b += RT)
        for (int k = 0; k < 10; ++k) v[k] += s.red[b * 10 + k];
    block_sum<10>(v, sh);
    if (threadIdx.x == 0) {
        const double W = -0.5 * G * v[1];
        s.diag[0] = v[0];
        s.diag[1] = W;
        s.diag[2] = v[2];
        s.diag[3] = v[0] + W + v[2];
        for (int k = 0; k < 6; ++k) s.diag[4 + k] = v[3 + k];
        if (v[9] != 0.0 || !isfinite(s.diag[3])) atomicOr(s.flag, 1);
    }
}

cudaError_t launch_energy_reduce(const DevState &s, const Decomp &d, const ExtField &ext,
                                 double G, cudaStream_t st)
{
    energy_partial_kernel<<<RB, RT, 0, st>>>(s, d, ext);
    energy_final_kernel<<<1, RT, 0, st>>>(s, G);
    return cudaGetLastError();
}

// External torque of eq. 8: sum m_i r_i x a_ext(r_i).
__global__ void torque_partial_kernel(DevState s, ExtField ext)
{
    __shared__ double sh[3 * RT];
    double v[3] = {0, 0, 0};
    for (int64_t i = blockIdx.x * (int64_t)RT + threadIdx.x; i < s.n; i += (int64_t)RB * RT) {
        const double m = s.m[i], x = s.x[i], y = s.y[i], z = s.z[i];
        double ax, ay, az;
        field_accel(ext, x, y, z, ax, ay, az);
        v[0] += m * (y * az - z * ay);
        v[1] += m * (z * ax - x * az);
        v[2] += m * (x * ay - y * ax);
    }
    block_sum<3>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) s.red[blockIdx.x * 3 + k] = v[k];
}

__global__ void torque_final_kernel(DevState s)
{
    __shared__ double sh[3 * RT];
    double v[3] = {0, 0, 0};
    for (int b = threadIdx.x; b < RB; b += RT)
        for (int k = 0; k < 3; ++k) v[k] += s.red[b * 3 + k];
    block_sum<3>(v, sh);
    if (threadIdx.x == 0)
        for (int k = 0; k < 3; ++k) s.diag[10 + k] = v[k];
}

cudaError_t launch_torque(const DevState &s, const ExtField &ext, cudaStream_t st)
{
    torque_partial_kernel<<<RB, RT, 0, st>>>(s, ext);
    torque_final_kernel<<<1, RT, 0, st>>>(s);
    return cudaGetLastError();
}

}  // namespace nb
