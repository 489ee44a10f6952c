// pair.cu -- all-pairs softened gravity (eq. 5; eq. 2 when eps = 0) on sm_103a.
//
// Every kernel here walks the same decomposition (Decomp) of the pair work of
// a set of independent clusters: a grid of G blocks (one resident wave or
// several), one contiguous run of (cluster, i-block, j-tile) units per block,
// so every block gets the same amount of work whatever the cluster sizes are
// (one cluster, or an ensemble of uneven clusters in one launch).  Each thread
// owns I i-bodies and keeps their sums in registers; every pair of each
// cluster's N x N array is evaluated, as in the paper (Sect. 4.2), not
// N(N-1)/2.  Clusters of equal masses leave m out of the pair term (scaled in
// afterwards), and in partly filled i-blocks a warp evaluates only the packed
// i-pairs that hold bodies.
//
// Single-precision family (one template, three modes):
//   PM_DS_NEAR  float pair arithmetic on coordinates relative to the cluster's
//               frame origin, float partial sums over 512 j folded into double-single
//               accumulators (Sect. 5.2's software double precision); pairs
//               closer than the near radius are re-formed from the
//               double-single coordinate difference (hi_j - hi_i) +
//               (lo_j - lo_i) by the separate correction pass of near.cu.
//   PM_DS_FULL  the double-single coordinate difference on every pair.
//   PM_FP32     float coordinates and float accumulation throughout (the
//               512-j partial sums added in float).
//
// Data movement: no block-wide barrier.  Each warp streams its j bodies in
// chunks of 32 through a warp-private shared-memory buffer: lane l loads body
// (chunk + l) one chunk ahead into registers, stores it, and after
// __syncwarp every lane reads the chunk back as broadcasts.  j bodies are
// stored pre-duplicated, (x, x, y, y) (z, z, m, m), so one packed f32x2
// instruction serves two i bodies of the same thread with no register moves.
// rsqrt runs on the MUFU pipe (rsqrt.approx).  Arithmetic uses explicit
// round-to-nearest intrinsics so the near-pair correction reproduces this
// loop's float contribution bit for bit.
#include <cstring>

#include "nb_internal.cuh"
#include "split.cuh"

namespace nb {

Decomp make_decomp(int64_t W, int64_t max_ntiles, int ipb, int64_t G, int64_t slot_cap, int jt,
                   int rows)
{
    Decomp d;
    d.ipb = ipb;
    d.jt = jt;
    d.rows = rows;
    const int64_t max_units = d.units_per_iblock(max_ntiles);
    d.W = W > 0 ? W : 1;
    if (G > d.W) G = d.W;
    if (G < 1) G = 1;
    for (;;) {
        d.G = G;
        d.slots = (max_units * G + d.W - 1) / d.W + 1;
        if (d.slots <= slot_cap || G == 1) break;
        G = G - G / 8 - 1;
        if (G < 1) G = 1;
    }
    d.narrow = (double)(d.W + 1) * (double)(d.G + 1) < 4294967296.0 ? 1 : 0;
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

// One contiguous run of units of block g inside one cluster's i-block.
struct Segment {
    int32_t k;        // cluster
    int64_t base;     // first pool slot of the cluster
    int64_t lbase;    // its first linear body index (partial sums are stored by it)
    int32_t nk;       // bodies of the cluster
    int32_t b;        // i-block
    int32_t t0, t1;   // units [t0, t1) of the i-block
    int32_t J0, J1;   // their j range
    int64_t slot;     // partial slot of this block for the i-block
};

// Per-cluster values by value (kernel parameter): uniform across the block.
// The widest table also carries the blocks' launch order (nperm = 0: index
// order).
template <int KC>
struct ParamTab {
    int32_t K;
    int32_t nperm;
    uint16_t perm[KC >= PARAM_CLUSTERS ? PERM_CAP : 1];
    int64_t uoff[KC + 1];
    int64_t boff[KC];
    int64_t noff[KC];
    double mu[KC];
    int32_t nk[KC];
    int32_t ntiles[KC];
    float eps2f[KC];
};

// Block of the decomposition this launch position runs.  Launch position q
// runs block perm[q] when the table carries an order (the host sorts the
// blocks by estimated work, largest first, so the blocks launched last, which
// set the kernel's tail, are the cheap ones); every block keeps its units and
// partial slot, so the results do not depend on the order.
template <int KC>
__device__ __forceinline__ int64_t block_of(const ParamTab<KC> &t)
{
    if (KC >= PARAM_CLUSTERS && t.nperm > 0) return t.perm[blockIdx.x];
    return blockIdx.x;
}

// largest k in [0, K) with off[k] <= t
template <typename T>
__device__ __forceinline__ int32_t find_in(const T *off, int32_t K, int64_t t)
{
    int32_t lo = 0, hi = K;
    while (hi - lo > 1) {
        const int32_t mid = (lo + hi) >> 1;
        if (off[mid] <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// End of a unit's j range, clipped to the cluster's bodies rounded up to 32
// (a whole warp chunk): the last j-tile of a cluster stops there instead of
// running 128 wide over padding that adds exactly zero.
__device__ __forceinline__ int32_t clip_j(int32_t J1, int32_t nk)
{
    const int32_t jend = (nk + 31) & ~31;
    return J1 < jend ? J1 : jend;
}

template <int KC>
__device__ __forceinline__ Segment segment_at(const Decomp &d, const ParamTab<KC> &t, int64_t g,
                                              int64_t u, int64_t uend)
{
    Segment s;
    s.k = KC == 1 ? 0 : find_in(t.uoff, t.K, u);
    const int64_t u0 = t.uoff[s.k];
    const int32_t nt = (int32_t)d.units_per_iblock(t.ntiles[s.k]);
    const int64_t lu = u - u0;
    const int64_t rb = lu / nt;
    s.b = (int32_t)(d.b0 + rb);
    s.t0 = (int32_t)(lu - rb * nt);
    const int64_t left = uend - u;
    s.t1 = (int64_t)s.t0 + left < nt ? (int32_t)(s.t0 + left) : nt;
    s.J0 = d.rows ? 0 : s.t0 * d.jt;
    s.J1 = d.rows ? t.ntiles[s.k] * TILE : s.t1 * d.jt;
    s.base = t.boff[s.k];
    s.lbase = t.noff[s.k];
    s.nk = t.nk[s.k];
    s.J1 = clip_j(s.J1, s.nk);
    s.slot = g - d.owner(u0 + rb * nt);
    return s;
}

__device__ __forceinline__ Segment segment_at(const Decomp &d, const Clusters &c, int64_t g,
                                              int64_t u, int64_t uend)
{
    Segment s;
    s.k = find_cluster(c.uoff, c.K, u);
    const int64_t u0 = c.uoff[s.k];
    const int32_t nt = (int32_t)d.units_per_iblock(c.ntiles[s.k]);
    const int64_t lu = u - u0;
    const int64_t rb = lu / nt;
    s.b = (int32_t)(d.b0 + rb);
    s.t0 = (int32_t)(lu - rb * nt);
    const int64_t left = uend - u;
    s.t1 = (int64_t)s.t0 + left < nt ? (int32_t)(s.t0 + left) : nt;
    s.J0 = d.rows ? 0 : s.t0 * d.jt;
    s.J1 = d.rows ? c.ntiles[s.k] * TILE : s.t1 * d.jt;
    s.base = c.boff[s.k];
    s.lbase = c.noff[s.k];
    s.nk = (int32_t)c.nk[s.k];
    s.J1 = clip_j(s.J1, s.nk);
    s.slot = g - d.owner(u0 + rb * nt);
    return s;
}

constexpr int CH = 32;            // j bodies per warp chunk
constexpr int WARPS = TILE / 32;  // warps per block
constexpr int FOLD = 4 * TILE;    // j bodies per float partial sum before the fold

// Thread-private i bodies, two per packed register pair: pair p holds bodies
// k = 2p (.x) and k = 2p + 1 (.y), local body k = ib0 + tid + k * TILE.
template <int P>
struct IPairs {
    float2 nx[P], ny[P], nz[P];     // negated hi coordinates
    float2 nlx[P], nly[P], nlz[P];  // negated lo coordinates (full double-single mode)
    float2 ax[P], ay[P], az[P];     // float sums of the current FOLD j bodies
};

// One chunk of CH j bodies (local indices j0 ...) against the thread's 2P i
// bodies (local indices ibase + k * TILE).  MASK zeroes the j == i term
// (eps = 0, diagonal chunks).  UM (all masses of the cluster equal): the pair
// term is d / r^3 without m_j, one multiply fewer; the caller scales by m.
// At P = 4 the chunk stays a loop of two groups of 16 j: fully unrolled, the
// kernel's code outgrows the instruction cache and runs 30% slower, while
// groups of 8 j left 1% on the table.  PA: the
// packed pairs evaluated, the first PA of P (a partly filled i-block leaves
// the others as padding for every lane of the warp; a variant per count keeps
// each loop fully unrolled, where a runtime bound inside it cost more than the
// padding).
template <int P, int MODE, bool MASK, bool UM, int PA = P>
__device__ __forceinline__ void chunk_pass(const float4 (*cb)[4], int j0, int ibase,
                                           IPairs<P> &ip, float eps2)
{
    const float2 e2 = make_float2(eps2, eps2);
    constexpr int GS = 16;                      // j bodies per unrolled group
    constexpr int GU = P >= 4 ? 1 : CH / GS;
#pragma unroll GU
    for (int g = 0; g < CH / GS; ++g) {
#pragma unroll
        for (int q = 0; q < GS; ++q) {
            const int jj = g * GS + q;
            const float4 A = cb[jj][0];
            const float4 B = cb[jj][1];
            const float2 xx = make_float2(A.x, A.y), yy = make_float2(A.z, A.w);
            const float2 zz = make_float2(B.x, B.y), mm = make_float2(B.z, B.w);
            float2 lxx, lyy, lzz;
            if (MODE == PM_DS_FULL) {
                const float4 C = cb[jj][2];
                const float4 D = cb[jj][3];
                lxx = make_float2(C.x, C.y);
                lyy = make_float2(C.z, C.w);
                lzz = make_float2(D.x, D.y);
            }
#pragma unroll
            for (int p = 0; p < PA; ++p) {
                float2 dx = __fadd2_rn(xx, ip.nx[p]);
                float2 dy = __fadd2_rn(yy, ip.ny[p]);
                float2 dz = __fadd2_rn(zz, ip.nz[p]);
                if (MODE == PM_DS_FULL) {
                    dx = __fadd2_rn(dx, __fadd2_rn(lxx, ip.nlx[p]));
                    dy = __fadd2_rn(dy, __fadd2_rn(lyy, ip.nly[p]));
                    dz = __fadd2_rn(dz, __fadd2_rn(lzz, ip.nlz[p]));
                }
                float2 r2 = __ffma2_rn(dx, dx, e2);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dz, dz, r2);
                const float2 ri = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
                float2 s = UM ? __fmul2_rn(ri, __fmul2_rn(ri, ri))
                              : __fmul2_rn(__fmul2_rn(mm, ri), __fmul2_rn(ri, ri));
                if (MASK) {
                    const int j = j0 + jj;
                    if (j == ibase + 2 * p * TILE) s.x = 0.f;
                    if (j == ibase + (2 * p + 1) * TILE) s.y = 0.f;
                }
                ip.ax[p] = __ffma2_rn(dx, s, ip.ax[p]);
                ip.ay[p] = __ffma2_rn(dy, s, ip.ay[p]);
                ip.az[p] = __ffma2_rn(dz, s, ip.az[p]);
            }
        }
    }
}

// Resident blocks per SM the register allocation is bounded for: 2P bodies per
// thread trade registers against shared-memory broadcasts per pair.  The
// every-pair double-single mode holds three more packed coordinates per i-pair
// and a second j-stream word per body, so it gets a looser cap (6 blocks at
// P = 1, 3 at P = 2); under the caps of the other modes it spilled (12 bytes
// per thread at P = 1, up to 1.4 KB at P = 2), and 4 blocks at P = 2 still
// spilled 16 bytes.
__host__ __device__ constexpr int sp_min_blocks(int P, int MODE)
{
    return MODE == PM_DS_FULL ? (P == 1 ? 6 : (P == 2 ? 3 : 2))
                              : (P == 1 ? 8 : (P == 2 ? 6 : 3));
}

// KC > 0: the cluster values come from the by-value table tab (K <= KC);
// KC == 0: from the device tables of c.
template <int KC>
using TabOf = ParamTab<KC == 0 ? 1 : KC>;

template <int P, int MODE, int KC, bool UM>
__global__ void __launch_bounds__(TILE, sp_min_blocks(P, MODE)) pair_sp_kernel(
    const float4 *__restrict__ jd, const float4 *__restrict__ jl,
    const float *__restrict__ xh, const float *__restrict__ yh, const float *__restrict__ zh,
    const float *__restrict__ xl, const float *__restrict__ yl, const float *__restrict__ zl,
    Clusters c, const __grid_constant__ TabOf<KC> tab, Decomp d, double G,
    double *__restrict__ part, int64_t ps)
{
    constexpr int I = 2 * P;
    constexpr bool FULL = (MODE == PM_DS_FULL);
    constexpr bool DSACC = (MODE != PM_FP32);
    constexpr int NV = FULL ? 4 : 2;
    __shared__ __align__(16) float4 cbuf[WARPS][CH][4];
    __shared__ float acc_sh[6 * I][TILE];   // per-thread running sums: hi x,y,z then lo x,y,z

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int w = tid >> 5;
    const float4(*cb)[4] = cbuf[w];
    const int64_t g = block_of(tab);
    int64_t u = d.U(g);
    const int64_t uend = d.U(g + 1);
    const float4 far4 = make_float4(FAR_F, FAR_F, FAR_F, FAR_F);
    const float4 farm = make_float4(FAR_F, FAR_F, 0.f, 0.f);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    while (u < uend) {
        const Segment sg = KC > 0 ? segment_at(d, tab, g, u, uend) : segment_at(d, c, g, u, uend);
        const int n = sg.nk;
        const int64_t base = sg.base;
        const float eps2 = KC > 0 ? tab.eps2f[sg.k] : c.eps2f[sg.k];
        const bool mask_self = d.mask_self != 0;
        const int ib0 = sg.b * d.ipb;
        const int ibase = ib0 + tid;
        const float4 *jdk = jd + 2 * base;
        const float4 *jlk = jl + 2 * base;

        IPairs<P> ip;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int ia = ibase + 2 * p * TILE, ib = ia + TILE;
            const int64_t ca = base + (ia < n ? ia : n - 1), cb2 = base + (ib < n ? ib : n - 1);
            ip.nx[p] = make_float2(-xh[ca], -xh[cb2]);
            ip.ny[p] = make_float2(-yh[ca], -yh[cb2]);
            ip.nz[p] = make_float2(-zh[ca], -zh[cb2]);
            if (FULL) {
                ip.nlx[p] = make_float2(-xl[ca], -xl[cb2]);
                ip.nly[p] = make_float2(-yl[ca], -yl[cb2]);
                ip.nlz[p] = make_float2(-zl[ca], -zl[cb2]);
            }
            ip.ax[p] = ip.ay[p] = ip.az[p] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int r = 0; r < 6 * I; ++r) acc_sh[r][tid] = 0.f;

        const int J0 = sg.J0, J1 = sg.J1;
        // packed pairs of this warp holding at least one body of the cluster
        // (warp-uniform): its lanes' bodies are ib0 + 32 w + lane + k TILE
        const int lw = ib0 + 32 * w;
        int kmax = n > lw ? (n - lw + TILE - 1) / TILE : 0;
        if (kmax > I) kmax = I;
        const int pact = (kmax + 1) / 2;
        float4 pf[4];
        {
            const int j = J0 + lane;
            pf[0] = j < n ? jdk[2 * j] : far4;
            pf[1] = j < n ? jdk[2 * j + 1] : farm;
            if (FULL) {
                pf[2] = j < n ? jlk[2 * j] : zero4;
                pf[3] = j < n ? jlk[2 * j + 1] : zero4;
            }
        }
        for (int jc = J0; jc < J1; jc += CH) {
#pragma unroll
            for (int v = 0; v < NV; ++v) cbuf[w][lane][v] = pf[v];
            __syncwarp();
            if (jc + CH < J1) {
                const int j = jc + CH + lane;
                pf[0] = j < n ? jdk[2 * j] : far4;
                pf[1] = j < n ? jdk[2 * j + 1] : farm;
                if (FULL) {
                    pf[2] = j < n ? jlk[2 * j] : zero4;
                    pf[3] = j < n ? jlk[2 * j + 1] : zero4;
                }
            }
            const bool diag = mask_self && jc < ib0 + d.ipb && jc + CH > ib0;
            if (pact >= P) {
                if (diag)
                    chunk_pass<P, MODE, true, UM>(cb, jc, ibase, ip, eps2);
                else
                    chunk_pass<P, MODE, false, UM>(cb, jc, ibase, ip, eps2);
            } else if (P > 1 && pact == (P > 1 ? P - 1 : 1)) {
                if (diag)
                    chunk_pass<P, MODE, true, UM, (P > 1 ? P - 1 : 1)>(cb, jc, ibase, ip, eps2);
                else
                    chunk_pass<P, MODE, false, UM, (P > 1 ? P - 1 : 1)>(cb, jc, ibase, ip, eps2);
            } else if (P > 2 && pact == (P > 2 ? P - 2 : 1)) {
                if (diag)
                    chunk_pass<P, MODE, true, UM, (P > 2 ? P - 2 : 1)>(cb, jc, ibase, ip, eps2);
                else
                    chunk_pass<P, MODE, false, UM, (P > 2 ? P - 2 : 1)>(cb, jc, ibase, ip, eps2);
            } else if (P > 3 && pact == 1) {
                if (diag)
                    chunk_pass<P, MODE, true, UM, 1>(cb, jc, ibase, ip, eps2);
                else
                    chunk_pass<P, MODE, false, UM, 1>(cb, jc, ibase, ip, eps2);
            }
            __syncwarp();
            if (((jc + CH - J0) & (FOLD - 1)) == 0 || jc + CH >= J1) {
                // every FOLD j and at the segment's end: fold the float
                // partial sums into the running sums
#pragma unroll
                for (int p = 0; p < P; ++p) {
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int kk = 2 * p + h;
                        const float t[3] = {h ? ip.ax[p].y : ip.ax[p].x,
                                            h ? ip.ay[p].y : ip.ay[p].x,
                                            h ? ip.az[p].y : ip.az[p].x};
#pragma unroll
                        for (int cc = 0; cc < 3; ++cc) {
                            float hi = acc_sh[cc * I + kk][tid];
                            if (DSACC) {
                                float lo = acc_sh[(3 + cc) * I + kk][tid];
                                ds_add(hi, lo, t[cc]);
                                acc_sh[(3 + cc) * I + kk][tid] = lo;
                            } else {
                                hi = __fadd_rn(hi, t[cc]);
                            }
                            acc_sh[cc * I + kk][tid] = hi;
                        }
                    }
                    ip.ax[p] = ip.ay[p] = ip.az[p] = make_float2(0.f, 0.f);
                }
            }
        }

        // partial sums as float pairs: the double-single sum times G m (m the
        // cluster's common mass in the uniform-mass form), a float-float
        // product (FMA-exact h gh plus the cross terms), normalised
        const double Gm = UM ? G * (KC > 0 ? tab.mu[sg.k] : c.mu[sg.k]) : G;
        const float gh = __double2float_rn(Gm), gl = __double2float_rn(Gm - (double)gh);
        float2 *part2 = reinterpret_cast<float2 *>(part);
#pragma unroll
        for (int kk = 0; kk < I; ++kk) {
            const int i = ibase + kk * TILE;
            if (i < n) {
                float2 *o = part2 + (sg.slot * 3) * ps + sg.lbase + i;
#pragma unroll
                for (int cc = 0; cc < 3; ++cc) {
                    const float h = acc_sh[cc * I + kk][tid], l = acc_sh[(3 + cc) * I + kk][tid];
                    const float pr = __fmul_rn(h, gh);
                    float e = __fmaf_rn(h, gh, -pr);
                    e = __fmaf_rn(h, gl, __fmaf_rn(l, gh, e));
                    const float s = __fadd_rn(pr, e);
                    o[cc * ps] = make_float2(s, __fsub_rn(e, __fsub_rn(s, pr)));
                }
            }
        }
        u += sg.t1 - sg.t0;
    }
}

// ---- float-float pair kernel (PM_DD) -------------------------------------------
// FP64-class accuracy on the FP32 pipes: every quantity of the pair sum is an
// unevaluated sum hi + lo of two floats (about 48 significant bits), built from
// Knuth's two-sum, Dekker's fast two-sum and FMA-exact products, packed over two
// i bodies per f32x2 instruction.  Coordinates are the double-single split of
// x - c (the paper's 14-digit format, Sect. 5.2); the coordinate difference,
// r^2 + eps^2, (r^2 + eps^2)^(-3/2) (a float rsqrt estimate y0 corrected by
// the series of (1 - v)^(-3/2) in the residual v = 1 - (r^2 + eps^2) y0^2),
// m / r^3 and the sums are all float-float.  Against a plain FP64
// sum it agrees to ~1e-14 relative (the 48-bit coordinates alone account for
// that), so it stands in for the FP64 pipe, which on this GPU runs at 1/77 of
// the FP32 rate.  The sums of r^2 + eps^2, whose terms are all non-negative,
// order their operands with max / min (ALU pipe) and use Dekker's three-
// operation sum; signed sums keep Knuth's six (ordering them by magnitude
// costs more issue slots than it saves).  UM (all masses of the cluster
// equal): 1 / r^3 without m, the caller scales by m.

__device__ __forceinline__ float2 f2neg(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __fadd2_rn(a, f2neg(b)); }

// s + e = a + b exactly (Knuth).
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = __fadd2_rn(a, b);
    const float2 bb = f2sub(s, a);
    e = __fadd2_rn(f2sub(a, f2sub(s, bb)), f2sub(b, bb));
}

// s + e = a + b exactly when |a| >= |b| (Dekker).
__device__ __forceinline__ void fast_two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = __fadd2_rn(a, b);
    e = f2sub(b, f2sub(s, a));
}

// s + e = a + b exactly for a, b >= 0: the larger operand first (max / min
// run on the ALU pipe, which this kernel leaves idle), then Dekker's fast
// two-sum, three FMA-pipe operations instead of Knuth's six.
__device__ __forceinline__ void pos_two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    const float2 hi = make_float2(fmaxf(a.x, b.x), fmaxf(a.y, b.y));
    const float2 lo = make_float2(fminf(a.x, b.x), fminf(a.y, b.y));
    s = __fadd2_rn(a, b);
    e = f2sub(lo, f2sub(s, hi));
}

// (ah + al) - (bh + bl), normalised.
__device__ __forceinline__ void ff_diff(float2 ah, float2 al, float2 bh, float2 bl, float2 &dh,
                                        float2 &dl)
{
    float2 s, e;
    two_sum2(ah, f2neg(bh), s, e);
    e = __fadd2_rn(e, f2sub(al, bl));
    fast_two_sum2(s, e, dh, dl);
}

// h^2 + (2 h l) as an unnormalised pair (p, e): p = fl(h^2), e its error plus
// the cross term.
__device__ __forceinline__ void ff_sq(float2 h, float2 l, float2 &p, float2 &e)
{
    p = __fmul2_rn(h, h);
    e = __ffma2_rn(h, h, f2neg(p));
    e = __ffma2_rn(__fadd2_rn(h, h), l, e);
}

// (ah + al)(bh + bl) without the al bl term, unnormalised.
__device__ __forceinline__ void ff_mul(float2 ah, float2 al, float2 bh, float2 bl, float2 &p,
                                       float2 &e)
{
    p = __fmul2_rn(ah, bh);
    e = __ffma2_rn(ah, bh, f2neg(p));
    e = __ffma2_rn(ah, bl, e);
    e = __ffma2_rn(al, bh, e);
}

template <int P>
struct FFI {
    float2 xh[P], yh[P], zh[P], xl[P], yl[P], zl[P];         // i coordinates
    float2 axh[P], axl[P], ayh[P], ayl[P], azh[P], azl[P];   // running sums
};

template <int P, bool MASK, bool UM>
__device__ __forceinline__ void chunk_pass_ff(const float4 (*cb)[4], int j0, int ibase,
                                              FFI<P> &q, float2 e2h, float2 e2l)
{
    const float2 one = make_float2(1.f, 1.f);
    const float2 c32 = make_float2(1.5f, 1.5f), c158 = make_float2(1.875f, 1.875f);
#pragma unroll 2
    for (int jj = 0; jj < CH; ++jj) {
        const float4 A = cb[jj][0], B = cb[jj][1], Cl = cb[jj][2], D = cb[jj][3];
        const float2 xjh = make_float2(A.x, A.y), yjh = make_float2(A.z, A.w);
        const float2 zjh = make_float2(B.x, B.y), mjh = make_float2(B.z, B.w);
        const float2 xjl = make_float2(Cl.x, Cl.y), yjl = make_float2(Cl.z, Cl.w);
        const float2 zjl = make_float2(D.x, D.y), mjl = make_float2(D.z, D.w);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            float2 dxh, dxl, dyh, dyl, dzh, dzl;
            ff_diff(xjh, xjl, q.xh[p], q.xl[p], dxh, dxl);
            ff_diff(yjh, yjl, q.yh[p], q.yl[p], dyh, dyl);
            ff_diff(zjh, zjl, q.zh[p], q.zl[p], dzh, dzl);
            // r^2 + eps^2
            float2 px, ex, py, ey, pz, ez;
            ff_sq(dxh, dxl, px, ex);
            ff_sq(dyh, dyl, py, ey);
            ff_sq(dzh, dzl, pz, ez);
            float2 s1, t1, s2, t2, s3, t3;   // all terms >= 0
            pos_two_sum2(px, py, s1, t1);
            pos_two_sum2(s1, pz, s2, t2);
            pos_two_sum2(s2, e2h, s3, t3);
            // R = r^2 + eps^2 as the unnormalised pair (s3, err), |err| <= 2^-21 s3
            const float2 err = __fadd2_rn(__fadd2_rn(__fadd2_rn(ex, ey), __fadd2_rn(ez, e2l)),
                                          __fadd2_rn(__fadd2_rn(t1, t2), t3));
            // s = R^(-3/2) from the float estimate y0 of 1 / sqrt(s3): with
            // R y0^2 = 1 - v, R^(-3/2) = y0^3 (1 - v)^(-3/2) = y0^3 (1 + 3/2 v
            // + 15/8 v^2 + O(v^3)), |v| ~ 2^-22.  v is formed from the exact
            // square y0^2 = q + qe (one FMA each term: 1 - s3 q cancels
            // exactly to ~2^-22 before it rounds), y0^3 = c + ce exactly to
            // float-float, and the series factor goes into the low word.
            const float2 y0 = make_float2(rsqrt_mufu(s3.x), rsqrt_mufu(s3.y));
            const float2 qh = __fmul2_rn(y0, y0);
            const float2 qe = __ffma2_rn(y0, y0, f2neg(qh));
            float2 v = __ffma2_rn(f2neg(s3), qh, one);
            v = __ffma2_rn(f2neg(s3), qe, v);
            v = __ffma2_rn(f2neg(err), qh, v);
            const float2 c3 = __fmul2_rn(qh, y0);
            float2 ce = __ffma2_rn(qh, y0, f2neg(c3));
            ce = __ffma2_rn(qe, y0, ce);
            const float2 kv = __fmul2_rn(__ffma2_rn(v, c158, c32), v);
            float2 sh, sl;
            if (UM) {
                sh = c3;
                sl = __ffma2_rn(c3, kv, ce);
            } else {
                ff_mul(mjh, mjl, c3, __ffma2_rn(c3, kv, ce), sh, sl);
            }
            if (MASK) {
                const int j = j0 + jj;
                if (j == ibase + 2 * p * TILE) sh.x = sl.x = 0.f;
                if (j == ibase + (2 * p + 1) * TILE) sh.y = sl.y = 0.f;
            }
            // a += s d
            float2 fh, fl, t, te;
            ff_mul(sh, sl, dxh, dxl, fh, fl);
            two_sum2(q.axh[p], fh, t, te);
            q.axh[p] = t;
            q.axl[p] = __fadd2_rn(q.axl[p], __fadd2_rn(te, fl));
            ff_mul(sh, sl, dyh, dyl, fh, fl);
            two_sum2(q.ayh[p], fh, t, te);
            q.ayh[p] = t;
            q.ayl[p] = __fadd2_rn(q.ayl[p], __fadd2_rn(te, fl));
            ff_mul(sh, sl, dzh, dzl, fh, fl);
            two_sum2(q.azh[p], fh, t, te);
            q.azh[p] = t;
            q.azl[p] = __fadd2_rn(q.azl[p], __fadd2_rn(te, fl));
        }
    }
}

template <int P, int KC, bool UM>
__global__ void __launch_bounds__(TILE) pair_ff_kernel(
    const float4 *__restrict__ jd, const float4 *__restrict__ jl,
    const float *__restrict__ xh, const float *__restrict__ yh, const float *__restrict__ zh,
    const float *__restrict__ xl, const float *__restrict__ yl, const float *__restrict__ zl,
    Clusters c, const __grid_constant__ TabOf<KC> tab, Decomp d, double G,
    double *__restrict__ part, int64_t ps)
{
    constexpr int I = 2 * P;
    __shared__ __align__(16) float4 cbuf[WARPS][CH][4];
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int w = tid >> 5;
    const float4(*cb)[4] = cbuf[w];
    const int64_t g = block_of(tab);
    int64_t u = d.U(g);
    const int64_t uend = d.U(g + 1);
    const float4 far4 = make_float4(FAR_F, FAR_F, FAR_F, FAR_F);
    const float4 farm = make_float4(FAR_F, FAR_F, 0.f, 0.f);
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);

    while (u < uend) {
        const Segment sg = KC > 0 ? segment_at(d, tab, g, u, uend) : segment_at(d, c, g, u, uend);
        const int n = sg.nk;
        const int64_t base = sg.base;
        const float e2hf = KC > 0 ? tab.eps2f[sg.k] : c.eps2f[sg.k];
        const float e2lf = __double2float_rn(c.eps2d[sg.k] - (double)e2hf);
        const float2 e2h = make_float2(e2hf, e2hf), e2l = make_float2(e2lf, e2lf);
        const bool mask_self = d.mask_self != 0;
        const int ib0 = sg.b * d.ipb;
        const int ibase = ib0 + tid;
        const float4 *jdk = jd + 2 * base;
        const float4 *jlk = jl + 2 * base;

        FFI<P> q;
        // chunk sums are float-float; they are added into FP64 running sums
        // after every chunk of CH j bodies, so the float lo word never
        // accumulates more than CH roundings
        double dax[I], day[I], daz[I];
#pragma unroll
        for (int k = 0; k < I; ++k) dax[k] = day[k] = daz[k] = 0.0;
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const int ia = ibase + 2 * p * TILE, ib = ia + TILE;
            const int64_t ca = base + (ia < n ? ia : n - 1), cb2 = base + (ib < n ? ib : n - 1);
            q.xh[p] = make_float2(xh[ca], xh[cb2]);
            q.yh[p] = make_float2(yh[ca], yh[cb2]);
            q.zh[p] = make_float2(zh[ca], zh[cb2]);
            q.xl[p] = make_float2(xl[ca], xl[cb2]);
            q.yl[p] = make_float2(yl[ca], yl[cb2]);
            q.zl[p] = make_float2(zl[ca], zl[cb2]);
            q.axh[p] = q.axl[p] = q.ayh[p] = q.ayl[p] = q.azh[p] = q.azl[p] = make_float2(0.f, 0.f);
        }
        const int J0 = sg.J0, J1 = sg.J1;
        float4 pf[4];
        {
            const int j = J0 + lane;
            pf[0] = j < n ? jdk[2 * j] : far4;
            pf[1] = j < n ? jdk[2 * j + 1] : farm;
            pf[2] = j < n ? jlk[2 * j] : zero4;
            pf[3] = j < n ? jlk[2 * j + 1] : zero4;
        }
        for (int jc = J0; jc < J1; jc += CH) {
#pragma unroll
            for (int v = 0; v < 4; ++v) cbuf[w][lane][v] = pf[v];
            __syncwarp();
            if (jc + CH < J1) {
                const int j = jc + CH + lane;
                pf[0] = j < n ? jdk[2 * j] : far4;
                pf[1] = j < n ? jdk[2 * j + 1] : farm;
                pf[2] = j < n ? jlk[2 * j] : zero4;
                pf[3] = j < n ? jlk[2 * j + 1] : zero4;
            }
            const bool diag = mask_self && jc < ib0 + d.ipb && jc + CH > ib0;
            if (diag)
                chunk_pass_ff<P, true, UM>(cb, jc, ibase, q, e2h, e2l);
            else
                chunk_pass_ff<P, false, UM>(cb, jc, ibase, q, e2h, e2l);
            __syncwarp();
#pragma unroll
            for (int p = 0; p < P; ++p) {
                dax[2 * p] += (double)q.axh[p].x + (double)q.axl[p].x;
                dax[2 * p + 1] += (double)q.axh[p].y + (double)q.axl[p].y;
                day[2 * p] += (double)q.ayh[p].x + (double)q.ayl[p].x;
                day[2 * p + 1] += (double)q.ayh[p].y + (double)q.ayl[p].y;
                daz[2 * p] += (double)q.azh[p].x + (double)q.azl[p].x;
                daz[2 * p + 1] += (double)q.azh[p].y + (double)q.azl[p].y;
                q.axh[p] = q.axl[p] = q.ayh[p] = q.ayl[p] = q.azh[p] = q.azl[p] =
                    make_float2(0.f, 0.f);
            }
        }
        const double Gm = UM ? G * (KC > 0 ? tab.mu[sg.k] : c.mu[sg.k]) : G;
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = ibase + k * TILE;
            if (i < n) {
                double *o = part + (sg.slot * 3) * ps + sg.lbase + i;
                o[0] = Gm * dax[k];
                o[ps] = Gm * day[k];
                o[2 * ps] = Gm * daz[k];
            }
        }
        u += sg.t1 - sg.t0;
    }
}

// Double-precision pair kernel: the plain FP64 baseline (Sect. 4.2's DP mode
// with structures of four doubles).  The block's j-range is staged through
// shared memory up to TILE bodies at a time and broadcast to the threads'
// i bodies.  With POT it sums the softened potential m_j / sqrt(r^2 + eps^2)
// of eq. 4 instead (j = i always excluded), for the energy diagnostic.  UM
// (all masses of the cluster equal): the pair term is d / r^3 without m_j,
// one multiply fewer on the FP64 pipe; the sums are scaled by G m.
template <int I, bool POT, bool UM = false>
__global__ void __launch_bounds__(TILE) pair_fp64_kernel(
    const double *__restrict__ x, const double *__restrict__ y, const double *__restrict__ z,
    const double *__restrict__ m, Clusters c, Decomp d, double G, double *__restrict__ part,
    int64_t ps)
{
    __shared__ double sx[TILE], sy[TILE], sz[TILE], sm[TILE];
    const int tid = threadIdx.x;
    const int64_t g = blockIdx.x;
    int64_t u = d.U(g);
    const int64_t uend = d.U(g + 1);

    while (u < uend) {
        const Segment sg = segment_at(d, c, g, u, uend);
        const int n = sg.nk;
        const int64_t base = sg.base;
        const double eps2 = c.eps2d[sg.k];
        const bool mask_self = POT || d.mask_self != 0;
        const int ib0 = sg.b * d.ipb;
        int idx[I];
        double xi[I], yi[I], zi[I], ax[I], ay[I], az[I];
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = ib0 + tid + k * TILE;
            const int64_t ic = base + (i < n ? i : n - 1);
            idx[k] = i;
            xi[k] = x[ic];
            yi[k] = y[ic];
            zi[k] = z[ic];
            ax[k] = ay[k] = az[k] = 0.0;
        }
        const int J0 = sg.J0, J1 = sg.J1;
        for (int jglob = J0; jglob < J1; jglob += TILE) {
            const int w = J1 - jglob < TILE ? J1 - jglob : TILE;   // j bodies staged
            const int j = jglob + tid;
            __syncthreads();
            if (tid < w) {
                if (j < n) {
                    sx[tid] = x[base + j];
                    sy[tid] = y[base + j];
                    sz[tid] = z[base + j];
                    sm[tid] = m[base + j];
                } else {
                    sx[tid] = sy[tid] = sz[tid] = FAR_D;
                    sm[tid] = 0.0;
                }
            }
            __syncthreads();
            const bool diag = mask_self && jglob < ib0 + d.ipb && jglob + w > ib0;
#pragma unroll 2
            for (int jj = 0; jj < w; ++jj) {
                const double xj = sx[jj], yj = sy[jj], zj = sz[jj], mj = sm[jj];
#pragma unroll
                for (int k = 0; k < I; ++k) {
                    const double dx = xj - xi[k], dy = yj - yi[k], dz = zj - zi[k];
                    double r2 = fma(dx, dx, eps2);
                    r2 = fma(dy, dy, r2);
                    r2 = fma(dz, dz, r2);
                    if (POT) {
                        double wgt = mj * rsqrt_pow<true>(r2);
                        if (diag && jglob + jj == idx[k]) wgt = 0.0;
                        ax[k] += wgt;
                    } else {
                        double s = UM ? rsqrt_pow<false>(r2) : mj * rsqrt_pow<false>(r2);
                        if (diag && jglob + jj == idx[k]) s = 0.0;
                        ax[k] = fma(dx, s, ax[k]);
                        ay[k] = fma(dy, s, ay[k]);
                        az[k] = fma(dz, s, az[k]);
                    }
                }
            }
        }
        const double Gm = UM ? G * c.mu[sg.k] : G;   // UM: the cluster's common mass
#pragma unroll
        for (int k = 0; k < I; ++k) {
            const int i = idx[k];
            if (i < n) {
                double *p = part + (sg.slot * 3) * ps + sg.lbase + i;
                if (POT) {
                    p[0] = ax[k];
                } else {
                    p[0] = Gm * ax[k];
                    p[ps] = Gm * ay[k];
                    p[2 * ps] = Gm * az[k];
                }
            }
        }
        u += sg.t1 - sg.t0;
    }
}

// ---- variant table -----------------------------------------------------------

template <int KC>
using sp_kernel_t = void (*)(const float4 *, const float4 *, const float *, const float *,
                             const float *, const float *, const float *, const float *,
                             Clusters, TabOf<KC>, Decomp, double, double *, int64_t);
typedef void (*dp_kernel_t)(const double *, const double *, const double *, const double *,
                            Clusters, Decomp, double, double *, int64_t);

// I (bodies per thread) = 2P for the single-precision family.
template <int KC>
static sp_kernel_t<KC> sp_variant(int mode, int I, bool um = false)
{
#define NB_SP(M, II)                                                      \
    if (mode == M && I == II)                                             \
        return um ? pair_sp_kernel<II / 2, M, KC, true> : pair_sp_kernel<II / 2, M, KC, false>;
    NB_SP(PM_DS_NEAR, 2) NB_SP(PM_DS_NEAR, 4) NB_SP(PM_DS_NEAR, 8)
    NB_SP(PM_DS_FULL, 2) NB_SP(PM_DS_FULL, 4)
    NB_SP(PM_FP32, 2) NB_SP(PM_FP32, 4) NB_SP(PM_FP32, 8)
#undef NB_SP
    if (mode == PM_DD && I == 2)
        return um ? pair_ff_kernel<1, KC, true> : pair_ff_kernel<1, KC, false>;
    if (mode == PM_DD && I == 4)
        return um ? pair_ff_kernel<2, KC, true> : pair_ff_kernel<2, KC, false>;
    return nullptr;
}

// The parameter-table width used for a set of K clusters.
static int kc_for(int32_t K) { return K == 1 ? 1 : (K <= PARAM_CLUSTERS ? PARAM_CLUSTERS : 0); }

template <int KC>
static cudaError_t launch_sp(const DevState &s, const PairLaunch &pl, const HostTab &ht,
                             double G, cudaStream_t st)
{
    sp_kernel_t<KC> k = sp_variant<KC>(pl.mode, pl.I, pl.um);
    if (!k) return cudaErrorInvalidValue;
    TabOf<KC> t;
    std::memset(&t, 0, sizeof t);
    if (KC > 0) {
        if (ht.K > KC) return cudaErrorInvalidValue;
        t.K = ht.K;
        if (KC >= PARAM_CLUSTERS && ht.perm && ht.nperm == pl.d.G && ht.nperm <= PERM_CAP) {
            t.nperm = ht.nperm;
            std::memcpy(t.perm, ht.perm, (size_t)ht.nperm * sizeof(uint16_t));
        }
        for (int32_t q = 0; q < ht.K; ++q) {
            t.uoff[q] = ht.uoff[q];
            t.boff[q] = ht.boff[q];
            t.noff[q] = ht.noff ? ht.noff[q] : 0;
            t.nk[q] = (int32_t)ht.nk[q];
            t.ntiles[q] = ht.ntiles[q];
            t.eps2f[q] = ht.eps2f[q];
            t.mu[q] = ht.mu ? ht.mu[q] : 0.0;
        }
        t.uoff[ht.K] = ht.uoff[ht.K];
    }
    k<<<(unsigned)pl.d.G, TILE, 0, st>>>(s.jd, s.jl, s.xh, s.yh, s.zh, s.xl, s.yl, s.zl, s.cl, t,
                                         pl.d, G, s.part, s.pstride);
    return cudaGetLastError();
}

static dp_kernel_t dp_variant(int I, bool um = false)
{
    if (I == 1) return um ? pair_fp64_kernel<1, false, true> : pair_fp64_kernel<1, false>;
    if (I == 2) return um ? pair_fp64_kernel<2, false, true> : pair_fp64_kernel<2, false>;
    return nullptr;
}

bool pair_variant_exists(int mode, int I)
{
    if (mode == PM_FP64) return dp_variant(I) != nullptr;
    return sp_variant<1>(mode, I) != nullptr;
}

int pair_occupancy(int mode, int I)
{
    int nb = 0;
    cudaError_t e;
    if (mode == PM_FP64) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, dp_variant(I), TILE, 0);
    } else {
        // the narrowest over the parameter-table widths
        int a = 0, b = 0, c = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, sp_variant<1>(mode, I), TILE, 0);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &b, sp_variant<PARAM_CLUSTERS>(mode, I), TILE, 0);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, sp_variant<0>(mode, I), TILE, 0);
        nb = a < b ? a : b;
        nb = nb < c ? nb : c;
    }
    if (e != cudaSuccess) return 0;
    return nb;
}

cudaError_t launch_pair(const DevState &s, const PairLaunch &pl, const HostTab &ht, double G,
                        cudaStream_t st)
{
    if (pl.mode == PM_FP64) {
        dp_kernel_t k = dp_variant(pl.I, pl.um);
        if (!k) return cudaErrorInvalidValue;
        k<<<(unsigned)pl.d.G, TILE, 0, st>>>(s.x, s.y, s.z, s.m, s.cl, pl.d, G, s.part,
                                             s.pstride);
        return cudaGetLastError();
    }
    switch (kc_for(ht.K)) {
    case 1: return launch_sp<1>(s, pl, ht, G, st);
    case PARAM_CLUSTERS: return launch_sp<PARAM_CLUSTERS>(s, pl, ht, G, st);
    default: return launch_sp<0>(s, pl, ht, G, st);
    }
}

cudaError_t launch_potential(const DevState &s, const Decomp &d, cudaStream_t st)
{
    pair_fp64_kernel<1, true><<<(unsigned)d.G, TILE, 0, st>>>(s.x, s.y, s.z, s.m, s.cl, d, 1.0,
                                                               s.part, s.pstride);
    return cudaGetLastError();
}

}  // namespace nb
