// noalloc.cu -- nb_accel_static: one force evaluation that allocates nothing.
//
// For callers that cannot call cudaMalloc: hosts that hand all device memory
// to their own pool allocator (an extra cudaMalloc fails or fragments it),
// loops that must never pay the implicit device synchronisation of
// cudaMalloc/cudaFree, and plug-in environments whose policy forbids device
// allocation after start-up.  Every piece of working memory the evaluation
// needs (double and float planes, the packed j-stream, the reference frame,
// reduction partials and the pair kernels' partial-sum slots) lives in one
// file-scope __device__ array of fixed size, NA_BYTES below, sized for at most
// NA_MAX_N bodies.  Every GPU that loads this library holds that array until
// the process exits.
//
// Host code cannot use the array's name as a device address (on the host it
// names a stand-in object), so the first call on each device, with that
// device current, looks the address up with cudaGetSymbolAddress and caches
// it.  That first call should therefore come before any stream capture.
//
// Every call shares the one array and leaves its contents behind; each call
// writes every scratch element it later reads (and clears the non-finite
// flag it uses), so nothing leaks from one call into the next.  Calls whose
// work overlaps on the GPU (different streams, or several host threads) race
// on the array: serialise them.
#include <mutex>

#include "nb_internal.cuh"
#include "../../include/nbsym.h"

namespace nb {
namespace {

constexpr int64_t NA_MAX_N = 16384;   // bodies per call, at most
constexpr int64_t NA_SLOTS = 8;       // partial-sum slots per body
constexpr int64_t NA_RED = 16 * 256;  // reduction partials (16 x reduce_blocks())

constexpr int64_t align256(int64_t b) { return (b + 255) / 256 * 256; }
constexpr int64_t OFF_D = 0;                                                // x y z m
constexpr int64_t OFF_F = OFF_D + align256(4 * NA_MAX_N * 8);               // 7 float planes
constexpr int64_t OFF_J = OFF_F + align256(7 * NA_MAX_N * 4);               // jd, jl
constexpr int64_t OFF_P = OFF_J + align256(4 * NA_MAX_N * 16);              // partial slots
constexpr int64_t OFF_R = OFF_P + align256(NA_SLOTS * 3 * NA_MAX_N * 8);    // reductions
constexpr int64_t OFF_G = OFF_R + align256(NA_RED * 8);                     // diag, frame, flag
constexpr int64_t NA_H = 32768;                                             // near_table_size(NA_MAX_N)
constexpr int64_t OFF_C = OFF_G + align256(16 * 8 + sizeof(Frame) + 16);    // near-pair correction
constexpr int64_t OFF_K = OFF_C + align256(3 * NA_MAX_N * 8);               // cell keys
constexpr int64_t OFF_I = OFF_K + align256(NA_MAX_N * 8);                   // bucket, entry
constexpr int64_t OFF_H = OFF_I + align256(2 * NA_MAX_N * 4);               // count, start, bsum
constexpr int64_t NA_BYTES = OFF_H + align256((2 * NA_H + 1 + NA_H / 1024 + 1) * 4);

static __device__ __align__(256) unsigned char na_scratch[NA_BYTES];

constexpr int MAX_DEV = 64;
std::mutex g_mu;
unsigned char *g_base[MAX_DEV] = {};

// Device address of na_scratch on the current device (looked up once).
int scratch_base(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= MAX_DEV) return NB_EINVAL;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_base[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, na_scratch) != cudaSuccess || !p) return NB_ECUDA;
        g_base[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_base[dev];
    return NB_OK;
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
    if (!p || !d_pos || !d_mass || !d_acc_out) return NB_EINVAL;
    if (n < 1 || n > NA_MAX_N) return NB_EINVAL;
    if (!(p->G > 0) || !(p->eps >= 0) || p->precision < NB_FP64 || p->precision > NB_DS_FULL)
        return NB_EINVAL;
    if (p->ext_on && !(p->bd > 0 && p->ab > 0)) return NB_EINVAL;
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) return NB_ECUDA;
    if (p->device != prev && cudaSetDevice(p->device) != cudaSuccess) return NB_EINVAL;
    int rc = NB_OK;
    do {
        unsigned char *b = nullptr;
        rc = scratch_base(p->device, &b);
        if (rc) break;
        cudaStream_t st = (cudaStream_t)p->stream;
        DevState s;
        s.n = n;
        s.cap = NA_MAX_N;
        double *d = reinterpret_cast<double *>(b + OFF_D);
        s.x = d;
        s.y = d + NA_MAX_N;
        s.z = d + 2 * NA_MAX_N;
        s.m = d + 3 * NA_MAX_N;
        float *f = reinterpret_cast<float *>(b + OFF_F);
        s.xh = f;
        s.yh = f + NA_MAX_N;
        s.zh = f + 2 * NA_MAX_N;
        s.mf = f + 3 * NA_MAX_N;
        s.xl = f + 4 * NA_MAX_N;
        s.yl = f + 5 * NA_MAX_N;
        s.zl = f + 6 * NA_MAX_N;
        s.jd = reinterpret_cast<float4 *>(b + OFF_J);
        s.jl = s.jd + 2 * NA_MAX_N;
        s.part = reinterpret_cast<double *>(b + OFF_P);
        s.part_slots = NA_SLOTS;
        s.red = reinterpret_cast<double *>(b + OFF_R);
        s.red_len = NA_RED;
        s.diag = reinterpret_cast<double *>(b + OFF_G);
        s.frame = reinterpret_cast<Frame *>(b + OFF_G + 16 * 8);
        s.flag = reinterpret_cast<int *>(b + OFF_G + 16 * 8 + sizeof(Frame));
        s.corr = reinterpret_cast<double *>(b + OFF_C);
        s.ng_key = reinterpret_cast<uint64_t *>(b + OFF_K);
        s.ng_bucket = reinterpret_cast<int *>(b + OFF_I);
        s.ng_entry = s.ng_bucket + NA_MAX_N;
        s.ng_count = reinterpret_cast<int *>(b + OFF_H);
        s.ng_start = s.ng_count + NA_H;
        s.ng_bsum = s.ng_start + NA_H + 1;
        s.ng_hcap = NA_H;
        if (near_table_size(NA_MAX_N) != NA_H) {
            rc = NB_ECUDA;
            break;
        }

        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device) !=
            cudaSuccess) {
            rc = NB_ECUDA;
            break;
        }
        PairLaunch pl;
        pl.mode = p->precision == NB_FP64 ? PM_FP64
                  : p->precision == NB_FP32 ? PM_FP32
                  : p->precision == NB_DS_FULL ? PM_DS_FULL : PM_DS_NEAR;
        pl.I = pl.mode == PM_FP64 ? 1 : 2;
        pl.blocks_per_sm = pair_occupancy(pl.mode, pl.I);
        if (pl.blocks_per_sm < 1) pl.blocks_per_sm = 1;
        Decomp dc = make_decomp(n, TILE * pl.I, (int64_t)sms * pl.blocks_per_sm);
        if (dc.W / 2 < dc.G) dc = make_decomp(n, TILE * pl.I, dc.W / 2 > 0 ? dc.W / 2 : 1);
        while (dc.max_slots() > NA_SLOTS && dc.G > 1)
            dc = make_decomp(n, TILE * pl.I, dc.G - dc.G / 8 - 1);
        pl.d = dc;

        ExtField ext;
        ext.on = p->ext_on;
        ext.G = p->G;
        ext.Md = p->Md;
        ext.ad = p->ad;
        ext.bd = p->bd;
        ext.Mb = p->Mb;
        ext.ab = p->ab;

        na_unpack_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(s, d_pos, d_mass);
        if (cudaGetLastError() != cudaSuccess) { rc = NB_ECUDA; break; }
        if (pl.mode != PM_FP64) {
            const double nf = p->near_frac > 0 ? p->near_frac : 0.4;
            if (launch_frame(s, nf, p->eps, st) != cudaSuccess ||
                launch_split(s, st) != cudaSuccess) {
                rc = NB_ECUDA;
                break;
            }
        }
        if (cudaMemsetAsync(s.flag, 0, sizeof(int), st) != cudaSuccess ||
            launch_pair(s, pl, p->G, p->eps, st) != cudaSuccess) {
            rc = NB_ECUDA;
            break;
        }
        // the mixed mode re-forms near pairs from the double-single difference
        if (pl.mode == PM_DS_NEAR) {
            if (launch_near_correct(s, p->eps, p->G, st) != cudaSuccess) {
                rc = NB_ECUDA;
                break;
            }
        } else {
            s.corr = nullptr;
        }
        if (launch_accel_out(s, pl.d, ext, p->G, d_acc_out, st) != cudaSuccess)
            rc = NB_ECUDA;
    } while (0);
    if (prev != p->device) cudaSetDevice(prev);
    return rc;
}
