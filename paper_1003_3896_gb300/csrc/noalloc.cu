// noalloc.cu -- nb_accel_static: one force evaluation that allocates nothing.
//
// For callers that cannot call cudaMalloc: hosts that hand all device memory
// to their own pool allocator (an extra cudaMalloc fails or fragments it),
// loops that must never pay the implicit device synchronisation of
// cudaMalloc/cudaFree, and plug-in environments whose policy forbids device
// allocation after start-up.  Every piece of working memory the evaluation
// needs (double and float planes, the packed j-stream, the cluster tables and
// reference frame, reduction partials, the pair kernels' partial-sum slots
// and the near-pair grid) lives in one file-scope __device__ array of fixed
// size, NA_BYTES below, sized for at most NA_MAX_N bodies.  Every GPU that
// loads this library holds that array until the process exits.
//
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in object), so the first call on each device, with that
// device current, looks the address up with cudaGetSymbolAddress and caches
// it beside the device's current context.  That first call should therefore
// come before any stream capture.  A call that finds another context current
// (the primary context was torn down by cudaDeviceReset and created anew)
// looks the address up again, so it too should come before any capture.
//
// Every call shares the one array and leaves its contents behind; each call
// writes every scratch element it later reads (its tables are rebuilt on the
// device, the non-finite flag is cleared), so nothing leaks from one call into
// the next.  Calls whose work overlaps on the GPU (different streams, or
// several host threads) race on the array: serialise them.
#include <cuda.h>   // CUcontext (types only; the driver call is found at run time)

#include <mutex>

#include "nb_internal.cuh"
#include "../../include/nbsym.h"
#include "engine.h"

namespace nb {
namespace {

constexpr int64_t NA_MAX_N = 16384;   // bodies per call, at most
constexpr int64_t NA_SLOTS = 8;       // partial-sum slots per body
constexpr int64_t NA_SEGS = (NA_MAX_N + SEG_BODIES - 1) / SEG_BODIES;
constexpr int64_t NA_H = 65536;       // near_table_size(NA_MAX_N)

constexpr int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }
constexpr int64_t OFF_D = 0;                                                // x y z m
constexpr int64_t OFF_F = OFF_D + align256(4 * NA_MAX_N * 8);               // 7 float planes
constexpr int64_t OFF_J = OFF_F + align256(7 * NA_MAX_N * 4);               // jd, jl
constexpr int64_t OFF_P = OFF_J + align256(4 * NA_MAX_N * 16);              // partial slots
constexpr int64_t OFF_C = OFF_P + align256(NA_SLOTS * 3 * NA_MAX_N * 8);    // near-pair correction
constexpr int64_t OFF_I = OFF_C + align256(3 * NA_MAX_N * 8);               // bucket, rank, entry
constexpr int64_t OFF_Q = OFF_I + align256(3 * NA_MAX_N * 4);               // spos slo
constexpr int64_t OFF_S = OFF_Q + align256(2 * NA_MAX_N * 16);              // cell table
constexpr int64_t OFF_H = OFF_S + align256(NA_H * (int64_t)sizeof(NgSlot));  // grid total
constexpr int64_t OFF_T = OFF_H + align256(4);                               // tables
// tables of the single cluster: boff nk noff[2] uoff[2] eps2d dts (int64/double),
// seg_lo[S] seg_hi[S], then ntiles eps2f seg_k[S] seg_off[2] flag (32-bit)
constexpr int64_t T64 = 8 + 2 * NA_SEGS;
constexpr int64_t T32 = 5 + NA_SEGS;
constexpr int64_t OFF_R = OFF_T + align256(T64 * 8 + T32 * 4);              // reductions
constexpr int64_t OFF_G = OFF_R + align256(NA_SEGS * 16 * 8);               // frame, diag
constexpr int64_t NA_BYTES = OFF_G + align256(sizeof(Frame) + DIAG_STRIDE * 8);

static __device__ __align__(256) unsigned char na_scratch[NA_BYTES];

constexpr int MAX_DEV = 64;
std::mutex g_mu;
unsigned char *g_base[MAX_DEV] = {};
CUcontext g_ctx[MAX_DEV] = {};

typedef CUresult (*ctx_get_current_t)(CUcontext *);

// The driver's cuCtxGetCurrent, found once through the runtime (no link-time
// dependency on the driver library).
ctx_get_current_t ctx_get_current()
{
    static ctx_get_current_t fn = nullptr;
    static bool looked = false;
    if (!looked) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<ctx_get_current_t>(f);
        looked = true;
    }
    return fn;
}

// Device address of na_scratch on the current device: looked up once per
// device and context, with that device current.  Sets the error message.
int scratch_base(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= MAX_DEV)
        return set_error(NB_EINVAL, "nb_accel_static: device %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    const ctx_get_current_t get = ctx_get_current();
    CUcontext ctx = nullptr;
    if (!get || get(&ctx) != CUDA_SUCCESS || !ctx)
        return set_error(NB_ECUDA, "nb_accel_static: no current CUDA context on device %d", dev);
    if (!g_base[dev] || g_ctx[dev] != ctx) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, na_scratch);
        if (e != cudaSuccess || !p)
            return set_error(NB_ECUDA, "nb_accel_static: cudaGetSymbolAddress failed: %s",
                             cudaGetErrorString(e));
        g_base[dev] = static_cast<unsigned char *>(p);
        g_ctx[dev] = ctx;
    }
    *out = g_base[dev];
    return NB_OK;
}

struct TablePtrs {
    int64_t *boff, *nk, *noff, *uoff, *seg_lo, *seg_hi;
    double *eps2d, *dts;
    int32_t *ntiles, *seg_k, *seg_off;
    float *eps2f;
    int *flag;
};

// Tables of one cluster of n bodies at pool slot 0, written on the device.
__global__ void na_tables_kernel(TablePtrs t, int64_t n, double eps, int ipb)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int64_t nt = (n + TILE - 1) / TILE;
    t.boff[0] = 0;
    t.nk[0] = n;
    t.noff[0] = 0;
    t.noff[1] = n;
    t.uoff[0] = 0;
    t.uoff[1] = ((n + ipb - 1) / ipb) * nt;
    t.ntiles[0] = (int32_t)nt;
    t.eps2d[0] = eps * eps;
    t.eps2f[0] = (float)(eps * eps);
    t.dts[0] = 1.0;
    int32_t S = 0;
    for (int64_t lo = 0; lo < n; lo += SEG_BODIES, ++S) {
        t.seg_k[S] = 0;
        t.seg_lo[S] = lo;
        t.seg_hi[S] = lo + SEG_BODIES < n ? lo + SEG_BODIES : n;
    }
    t.seg_off[0] = 0;
    t.seg_off[1] = S;
    *t.flag = 0;
}

__global__ void na_unpack_kernel(DevState s, const double *__restrict__ pos,
                                 const double *__restrict__ mass)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= s.n) return;
    s.x[i] = pos[3 * i];
    s.y[i] = pos[3 * i + 1];
    s.z[i] = pos[3 * i + 2];
    s.m[i] = mass[i];
    s.mf[i] = __double2float_rn(mass[i]);
}

}  // namespace
}  // namespace nb

using namespace nb;

extern "C" int nb_accel_static(const nb_params *p, int64_t n, const double *d_pos,
                               const double *d_mass, double *d_acc_out)
{
    if (!p || !d_pos || !d_mass || !d_acc_out)
        return set_error(NB_EINVAL, "nb_accel_static: NULL argument");
    if (n < 1 || n > NA_MAX_N)
        return set_error(NB_EINVAL, "nb_accel_static: n must be in [1, %d]", (int)NA_MAX_N);
    const int prc = check_nb_params(p);
    if (prc) return prc;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess)
        return set_error(NB_ECUDA, "nb_accel_static: no usable CUDA device");
    if (p->device != prev && cudaSetDevice(p->device) != cudaSuccess)
        return set_error(NB_EINVAL, "nb_accel_static: bad device %d", p->device);
    int rc = NB_OK;
    // a failed runtime call: its message is recorded (cudaGetLastError also
    // returns an error that earlier work of the caller left pending)
    auto fail = [](const char *what, cudaError_t e) {
        return set_error(NB_ECUDA, "nb_accel_static: %s failed: %s", what, cudaGetErrorString(e));
    };
    do {
        unsigned char *b = nullptr;
        rc = scratch_base(p->device, &b);
        if (rc) break;
        if (near_table_size(NA_MAX_N) != NA_H) {
            rc = set_error(NB_ECUDA, "nb_accel_static: near-pair table size mismatch");
            break;
        }
        cudaStream_t st = (cudaStream_t)p->stream;
        const int64_t N = NA_MAX_N;
        DevState s;
        s.n = n;
        s.cap = N;
        double *d = reinterpret_cast<double *>(b + OFF_D);
        s.x = d;
        s.y = d + N;
        s.z = d + 2 * N;
        s.m = d + 3 * N;
        float *f = reinterpret_cast<float *>(b + OFF_F);
        s.xh = f;
        s.yh = f + N;
        s.zh = f + 2 * N;
        s.mf = f + 3 * N;
        s.xl = f + 4 * N;
        s.yl = f + 5 * N;
        s.zl = f + 6 * N;
        s.jd = reinterpret_cast<float4 *>(b + OFF_J);
        s.jl = s.jd + 2 * N;
        s.part = reinterpret_cast<double *>(b + OFF_P);
        s.part_elems = NA_SLOTS * 3 * NA_MAX_N;
        s.pstride = n;                   // n <= NA_MAX_N: at least NA_SLOTS slots
        s.part_slots = NA_SLOTS;
        s.corr = reinterpret_cast<double *>(b + OFF_C);
        s.ng_bucket = reinterpret_cast<int *>(b + OFF_I);
        s.ng_rank = s.ng_bucket + N;
        s.ng_entry = s.ng_bucket + 2 * N;
        s.ng_spos = reinterpret_cast<float4 *>(b + OFF_Q);
        s.ng_slo = s.ng_spos + N;
        s.ng_slot = reinterpret_cast<NgSlot *>(b + OFF_S);
        s.ng_total = reinterpret_cast<int *>(b + OFF_H);
        s.ng_hcap = NA_H;
        TablePtrs t;
        int64_t *t64 = reinterpret_cast<int64_t *>(b + OFF_T);
        t.boff = t64;
        t.nk = t64 + 1;
        t.noff = t64 + 2;
        t.uoff = t64 + 4;
        t.eps2d = reinterpret_cast<double *>(t64 + 6);
        t.dts = reinterpret_cast<double *>(t64 + 7);
        t.seg_lo = t64 + 8;
        t.seg_hi = t64 + 8 + NA_SEGS;
        int32_t *t32 = reinterpret_cast<int32_t *>(t64 + T64);
        t.ntiles = t32;
        t.eps2f = reinterpret_cast<float *>(t32 + 1);
        t.seg_off = t32 + 2;
        t.flag = t32 + 4;
        t.seg_k = t32 + 5;
        s.flag = t.flag;
        s.red = reinterpret_cast<double *>(b + OFF_R);
        s.red_len = NA_SEGS * 16;
        Frame *frame = reinterpret_cast<Frame *>(b + OFF_G);
        s.diag = reinterpret_cast<double *>(b + OFF_G + sizeof(Frame));

        int sms = 0;
        cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
        if (e != cudaSuccess) {
            rc = fail("cudaDeviceGetAttribute", e);
            break;
        }
        PairLaunch pl;
        pl.mode = p->precision == NB_FP64 ? PM_FP64
                  : p->precision == NB_FP32 ? PM_FP32
                  : p->precision == NB_DS_FULL ? PM_DS_FULL
                  : p->precision == NB_DD ? PM_DD
                  : p->precision == NB_DS_NEAR ? PM_DS_NEAR
                  : (double)n * (double)n <= DS_FULL_MAX_PAIRS ? PM_DS_FULL : PM_DS_NEAR;
        pl.I = pl.mode == PM_FP64 ? 1 : 2;
        const int ipb = TILE * pl.I;
        pl.blocks_per_sm = pair_occupancy(pl.mode, pl.I);
        if (pl.blocks_per_sm < 1) pl.blocks_per_sm = 1;
        const int64_t nt = (n + TILE - 1) / TILE;
        const int64_t W = ((n + ipb - 1) / ipb) * nt;
        int64_t G = (int64_t)sms * pl.blocks_per_sm;
        if (W / 2 < G) G = W / 2 > 0 ? W / 2 : 1;
        pl.d = make_decomp(W, nt, ipb, G, NA_SLOTS);
        pl.d.mask_self = p->eps == 0.0 ? 1 : 0;
        pl.d.fpart = sp_family(pl.mode) ? 1 : 0;

        Clusters &c = s.cl;
        c.K = 1;
        c.boff = t.boff;
        c.nk = t.nk;
        c.noff = t.noff;
        c.uoff = t.uoff;
        c.ntiles = t.ntiles;
        c.eps2f = t.eps2f;
        c.eps2d = t.eps2d;
        c.dts = t.dts;
        c.frame = frame;
        c.S = (int32_t)((n + SEG_BODIES - 1) / SEG_BODIES);
        c.seg_k = t.seg_k;
        c.seg_lo = t.seg_lo;
        c.seg_hi = t.seg_hi;
        c.seg_off = t.seg_off;

        ExtField ext;
        ext.on = p->ext_on;
        ext.G = p->G;
        ext.Md = p->Md;
        ext.ad = p->ad;
        ext.bd = p->bd;
        ext.Mb = p->Mb;
        ext.ab = p->ab;
        ext.Mbh = p->Mbh;
        ext.eps2bh = p->eps_bh * p->eps_bh;

        na_tables_kernel<<<1, 32, 0, st>>>(t, n, p->eps, ipb);
        na_unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, d_pos, d_mass);
        if ((e = cudaGetLastError()) != cudaSuccess) {
            rc = fail("table / unpack launch", e);
            break;
        }
        if (pl.mode != PM_FP64) {
            const double nf = p->near_frac > 0 ? p->near_frac : 0.4;
            if ((e = launch_frame(s, nf, pl.mode == PM_DS_NEAR, st)) != cudaSuccess ||
                (e = launch_split(s, st)) != cudaSuccess) {
                rc = fail("frame / split launch", e);
                break;
            }
        }
        const int64_t h_uoff[2] = {0, W}, h_boff[1] = {0}, h_nk[1] = {n};
        const int32_t h_nt[1] = {(int32_t)nt};
        const float h_e2[1] = {(float)(p->eps * p->eps)};
        HostTab ht;
        ht.K = 1;
        ht.uoff = h_uoff;
        ht.boff = h_boff;
        ht.nk = h_nk;
        ht.ntiles = h_nt;
        ht.eps2f = h_e2;
        if ((e = launch_pair(s, pl, ht, p->G, st)) != cudaSuccess) {
            rc = fail("pair kernel launch", e);
            break;
        }
        // the mixed mode re-forms near pairs from the double-single difference
        if (pl.mode == PM_DS_NEAR) {
            if ((e = launch_near_correct(s, p->G, false, st)) != cudaSuccess) {
                rc = fail("near-pair pass launch", e);
                break;
            }
        } else {
            s.corr = nullptr;
        }
        if ((e = launch_accel_out(s, pl.d, ext, d_acc_out, st)) != cudaSuccess)
            rc = fail("output launch", e);
    } while (0);
    if (prev != p->device) cudaSetDevice(prev);
    return rc;
}
