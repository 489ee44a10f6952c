// sym.cu -- the N(N-1)/2 variant of the pair sum (Newton's third law): each
// unordered pair is evaluated once and its force added to both bodies.  The
// paper rejects it for its GPU (Sect. 4.2); here it is built to measure it on
// this one, in the pure-float class of NB_FP32 (float pair arithmetic on
// frame-centred coordinates).
//
// Work: tile pairs (I, J), I <= J, of 64 x 64 bodies over the upper triangle,
// split into equal contiguous runs, one per resident block.  A block of 128
// threads is a 16 x 8 grid; thread (a, b) keeps bodies I*64 + 4a .. 4a + 3 and
// J*64 + 8b .. 8b + 7 in registers and evaluates their 32 pairs, so a pair
// costs 16 FMA-pipe operations for two interactions (differences, r^2, r^-3,
// the two mass factors, both accumulations) against 12 for one in the full
// kernel.  A block keeps its i sums in registers while its run of tile
// pairs stays in one row I; the j side of each tile pair (and the i side at a
// row change) is summed over the threads in a fixed order through shared
// memory and then added to the global sums with float atomics, whose order is
// not fixed, so results are not bit-reproducible (they stay within the float
// tolerance).  Diagonal tile pairs keep only j > i.
#include "engine.h"

namespace nb {
namespace {

constexpr int ST = 64;            // bodies per tile side
constexpr int SA = 16, SB = 8;    // thread grid
constexpr int PI = ST / SA;       // i bodies per thread (4)
constexpr int PJ = ST / SB;       // j bodies per thread (8)

__device__ __forceinline__ float sym_rsqrt(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Tile pair q of the upper triangle of nt tiles, row-major: (I, J), I <= J.
__device__ __forceinline__ void tile_pair(int64_t q, int64_t nt, int64_t &I, int64_t &J)
{
    // rows have nt, nt - 1, ... entries; the row start of row I is
    // I * nt - I (I - 1) / 2.  Solve by a float estimate, then fix up.
    const double b = 2.0 * nt + 1.0;
    int64_t r = (int64_t)((b - sqrt(b * b - 8.0 * (double)q)) / 2.0);
    if (r < 0) r = 0;
    if (r > nt - 1) r = nt - 1;
    auto start = [nt](int64_t i) { return i * nt - i * (i - 1) / 2; };
    while (r > 0 && start(r) > q) --r;
    while (r + 1 < nt && start(r + 1) <= q) ++r;
    I = r;
    J = r + (q - start(r));
}

__global__ void __launch_bounds__(SA * SB) pair_sym_kernel(
    const float *__restrict__ xh, const float *__restrict__ yh, const float *__restrict__ zh,
    const float *__restrict__ mf, int64_t base, int n, float eps2, int64_t W, int64_t G,
    float *__restrict__ acc)
{
    // per-thread partials of the current tile pair's j side (and, at a row
    // change, of the i side), summed in a fixed order
    __shared__ float part[3][SA][ST];
    const int tid = threadIdx.x;
    const int a = tid % SA, b = tid / SA;
    const int64_t nt = (n + ST - 1) / ST;
    const int64_t g = blockIdx.x;
    const int64_t q0 = g * W / G, q1 = (g + 1) * W / G;
    float xi[PI], yi[PI], zi[PI], mi[PI], axi[PI], ayi[PI], azi[PI];
    int64_t I = -1;
    // i sums of row I: partials over b into part (rows b), then global adds
    auto flush_i = [&](int64_t row) {
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PI; ++u) {
            part[0][b][a * PI + u] = axi[u];
            part[1][b][a * PI + u] = ayi[u];
            part[2][b][a * PI + u] = azi[u];
        }
        __syncthreads();
        for (int k = tid; k < 3 * ST; k += SA * SB) {
            const int c = k / ST, t = k % ST;
            float v = 0.f;
            for (int r = 0; r < SB; ++r) v += part[c][r][t];
            const int64_t i = row * ST + t;
            if (i < n) atomicAdd(&acc[(int64_t)c * n + i], v);
        }
    };
    for (int64_t q = q0; q < q1; ++q) {
        int64_t Iq, J;
        tile_pair(q, nt, Iq, J);
        if (Iq != I) {
            if (I >= 0) flush_i(I);
            I = Iq;
#pragma unroll
            for (int u = 0; u < PI; ++u) {
                const int64_t i = I * ST + a * PI + u;
                const bool in = i < n;
                xi[u] = in ? xh[base + i] : FAR_F;
                yi[u] = in ? yh[base + i] : FAR_F;
                zi[u] = in ? zh[base + i] : FAR_F;
                mi[u] = in ? mf[base + i] : 0.f;
                axi[u] = ayi[u] = azi[u] = 0.f;
            }
        }
        float xj[PJ], yj[PJ], zj[PJ], mj[PJ], axj[PJ], ayj[PJ], azj[PJ];
#pragma unroll
        for (int v = 0; v < PJ; ++v) {
            const int64_t j = J * ST + b * PJ + v;
            const bool in = j < n;
            // a far padding j must not coincide with a far padding i
            xj[v] = in ? xh[base + j] : -FAR_F;
            yj[v] = in ? yh[base + j] : -FAR_F;
            zj[v] = in ? zh[base + j] : -FAR_F;
            mj[v] = in ? mf[base + j] : 0.f;
            axj[v] = ayj[v] = azj[v] = 0.f;
        }
        const bool diag = I == J;
#pragma unroll
        for (int u = 0; u < PI; ++u) {
#pragma unroll
            for (int v = 0; v < PJ; ++v) {
                const float dx = __fadd_rn(xj[v], -xi[u]);
                const float dy = __fadd_rn(yj[v], -yi[u]);
                const float dz = __fadd_rn(zj[v], -zi[u]);
                float r2 = __fmaf_rn(dx, dx, eps2);
                r2 = __fmaf_rn(dy, dy, r2);
                r2 = __fmaf_rn(dz, dz, r2);
                const float ri = sym_rsqrt(r2);
                float ri3 = __fmul_rn(__fmul_rn(ri, ri), ri);
                if (diag && b * PJ + v <= a * PI + u) ri3 = 0.f;   // j > i only
                const float si_ = __fmul_rn(mj[v], ri3), sj_ = __fmul_rn(mi[u], ri3);
                axi[u] = __fmaf_rn(dx, si_, axi[u]);
                ayi[u] = __fmaf_rn(dy, si_, ayi[u]);
                azi[u] = __fmaf_rn(dz, si_, azi[u]);
                axj[v] = __fmaf_rn(-dx, sj_, axj[v]);
                ayj[v] = __fmaf_rn(-dy, sj_, ayj[v]);
                azj[v] = __fmaf_rn(-dz, sj_, azj[v]);
            }
        }
        // j sums of this tile pair: partials over a, fixed-order sum
        __syncthreads();
#pragma unroll
        for (int v = 0; v < PJ; ++v) {
            part[0][a][b * PJ + v] = axj[v];
            part[1][a][b * PJ + v] = ayj[v];
            part[2][a][b * PJ + v] = azj[v];
        }
        __syncthreads();
        for (int k = tid; k < 3 * ST; k += SA * SB) {
            const int c = k / ST, t = k % ST;
            float v = 0.f;
#pragma unroll
            for (int r = 0; r < SA; ++r) v += part[c][r][t];
            const int64_t j = J * ST + t;
            if (j < n) atomicAdd(&acc[(int64_t)c * n + j], v);
        }
    }
    if (I >= 0) flush_i(I);
}

// out[3 t + c] = G acc[c][t] (+ the external field), interleaved rows.
__global__ void sym_out_kernel(DevState s, const float *__restrict__ acc, int n, double G,
                               ExtField ext, double *__restrict__ out)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t i = s.cl.boff[0] + t;
    double ax = G * (double)acc[t], ay = G * (double)acc[n + t], az = G * (double)acc[2 * n + t];
    if (ext.on) {
        // same closed form as the kick (a_ext = -grad Phi); see integrate.cu
        const double x = s.x[i], y = s.y[i], z = s.z[i];
        const double R2 = x * x + y * y;
        const double s2 = z * z + ext.bd * ext.bd;
        const double rs = rsqrt(s2);
        const double qd = ext.ad + s2 * rs;
        const double rD = rsqrt(R2 + qd * qd);
        const double kd = ext.G * ext.Md * (rD * rD * rD);
        const double rB = rsqrt(R2 + z * z + ext.ab * ext.ab);
        const double kb = ext.G * ext.Mb * (rB * rB * rB);
        double kh = 0.0;
        if (ext.Mbh > 0) {
            const double rH = rsqrt(R2 + z * z + ext.eps2bh);
            kh = ext.G * ext.Mbh * (rH * rH * rH);
        }
        ax -= (kd + kb + kh) * x;
        ay -= (kd + kb + kh) * y;
        az -= (kd * qd * rs + kb + kh) * z;
    }
    out[3 * t] = ax;
    out[3 * t + 1] = ay;
    out[3 * t + 2] = az;
}

}  // namespace

int sym_accel(const Pool &P, const ClusterSet &C, const Phys &ph, float *acc, double *out,
              cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1)
{
    if (C.K != 1) return set_error(NB_EINVAL, "the N(N-1)/2 variant takes one cluster");
    const DevState s = view(P, C, NB_FP32);
    const int n = (int)C.nk[0];
    const int64_t nt = (n + ST - 1) / ST;
    const int64_t W = nt * (nt + 1) / 2;
    int blocks = 0;
    NB_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, pair_sym_kernel, SA * SB, 0));
    int64_t G = (int64_t)P.num_sms * (blocks > 0 ? blocks : 1);
    if (G > W) G = W;
    NB_TRY(cudaMemsetAsync(acc, 0, sizeof(float) * 3 * (size_t)n, st));
    NB_TRY(cudaEventRecord(e0, st));
    pair_sym_kernel<<<(unsigned)G, SA * SB, 0, st>>>(s.xh, s.yh, s.zh, s.mf, C.boff[0], n,
                                                    C.eps2f[0], W, G, acc);
    NB_TRY(cudaGetLastError());
    NB_TRY(cudaEventRecord(e1, st));
    sym_out_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, acc, n, ph.G, ph.ext, out);
    NB_TRY(cudaGetLastError());
    return NB_OK;
}

}  // namespace nb
