// onmf_project_static: the projection of onmf_project for callers that
// cannot allocate device memory. A real-time audio callback cannot wait for
// cudaMalloc (it may synchronize the whole device and may fail at run time),
// and hosts that hand the library a fixed memory arena forbid allocations on
// their own. This entry point keeps its scratch (the derived images of W, the
// column sums and the per-tile loss slots) in one fixed device array below;
// the caller passes inputs and outputs.
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "onmf.h"
#include "onmf_cluster.cuh"
#include "onmf_kernels.cuh"
#include "onmf_launch.h"

namespace {

// Scratch shared by every call on a device; it lives as long as the library
// stays loaded. Each call overwrites what it uses, so two calls that run at
// the same time on the GPU (e.g. on two streams) race on it.
static __device__ __align__(256) unsigned char g_static_scratch[ONMF_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_addr[kMaxDevices] = {};
bool g_configured[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Device address of the scratch array for the current device, looked up
// once per device (with that device current) and cached.
onmf_status scratch_address(void **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return ONMF_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return ONMF_ECUDA;
        }
        g_addr[dev] = p;
    }
    if (!g_configured[dev]) {
        if (onmf::configure_kernels() != cudaSuccess) return ONMF_ECUDA;
        g_configured[dev] = true;
    }
    *out = g_addr[dev];
    return ONMF_OK;
}

}  // namespace

// The kernels' error bits are the ones the header promises to err_out.
static_assert(onmf::ERR_INPUT == ONMF_DEVERR_INPUT && onmf::ERR_NUMERIC == ONMF_DEVERR_NUMERIC &&
                  onmf::ERR_TIMEOUT == ONMF_DEVERR_TIMEOUT && onmf::ERR_CONFIG == ONMF_DEVERR_CONFIG,
              "device error bits");

extern "C" onmf_status onmf_project_static(const float *W, int32_t F, int32_t K, const float *V,
                                           int64_t ldv, int64_t n, float *H_out, int64_t ldh,
                                           double eps, double h_exponent, int32_t n_inner,
                                           int32_t precision, double *obj_sum, int32_t *err_out,
                                           void *stream) {
    using namespace onmf;
    if (!W || F < 1 || K < 1 || n < 0 || (n > 0 && !V) || ldv < F || (H_out && ldh < K) ||
        n_inner < 0 || !(eps >= 0.0) || !(h_exponent > 0.0) ||
        (precision != ONMF_FP32 && precision != ONMF_MIXED) || K > 256 || F > 8192)
        return ONMF_EINVAL;
    if (precision == ONMF_MIXED && F > 1024) return ONMF_EINVAL;
    const Shape sh = make_shape(F, K);
    // the same h-solve as onmf_project
    const int prec = select_prec(precision == ONMF_MIXED, sh, ONMF_HSOLVE_AUTO);
    ClusterTiles ct;
    if (prec == PREC_CL) {
        ct = cluster_tiles(sh, n > 0 ? n : 1);
        if (ct.C == 0) return ONMF_EINVAL;
    }
    const int tile = prec == PREC_TC ? kTcTile : kTile;
    const long long ntiles = prec == PREC_CL ? ct.slots : (n + tile - 1) / tile;  // loss slots
    // scratch layout: [W image][row-major bf16 W][column sums][per-tile loss]
    const size_t img = prec == PREC_FP32 ? (size_t)F * K * 4
                       : prec == PREC_CL ? 0
                                         : (size_t)sh.Kp * sh.WLD * 2;
    const size_t rows = (prec == PREC_TC || prec == PREC_CL) ? (size_t)F * sh.Kp * 2 : 0;
    const size_t off_rows = align256(img);
    const size_t off_sw = off_rows + align256(rows);
    const size_t off_loss = off_sw + align256((size_t)K * 4);
    const size_t need = off_loss + (size_t)(ntiles > 0 ? ntiles : 1) * 8;
    if (need > ONMF_STATIC_SCRATCH_BYTES - 256) return ONMF_EINVAL;
    size_t smem = prec == PREC_CL ? ct.smem : tile_smem_bytes(sh, prec);
    if (prec == PREC_TC && smem < 116 * 1024) smem = 116 * 1024;  // one CTA per SM (TMEM)
    if (smem > max_dynamic_smem()) return ONMF_EINVAL;
    void *base = nullptr;
    onmf_status st = scratch_address(&base);
    if (st != ONMF_OK) return st;
    unsigned char *b = static_cast<unsigned char *>(base);
    cudaStream_t q = reinterpret_cast<cudaStream_t>(stream);
    float *Wrm = prec == PREC_FP32 ? reinterpret_cast<float *>(b) : nullptr;
    __nv_bfloat16 *Wimg =
        (prec == PREC_MIXED || prec == PREC_TC) ? reinterpret_cast<__nv_bfloat16 *>(b) : nullptr;
    __nv_bfloat16 *Wrow = rows ? reinterpret_cast<__nv_bfloat16 *>(b + off_rows) : nullptr;
    float *swpart = reinterpret_cast<float *>(b + off_sw);
    double *loss = reinterpret_cast<double *>(b + off_loss);
    // the padding of the bf16 image must read as zero whatever an earlier
    // call of another shape left there
    if (Wimg && cudaMemsetAsync(Wimg, 0, img, q) != cudaSuccess) return ONMF_ECUDA;
    if (Wrow && cudaMemsetAsync(Wrow, 0, rows, q) != cudaSuccess) return ONMF_ECUDA;
    // the kernels OR their error bits into the caller's word when there is
    // one, else into the last 256 bytes of the scratch (then nobody reads them)
    int *err = err_out ? reinterpret_cast<int *>(err_out)
                       : reinterpret_cast<int *>(b + ONMF_STATIC_SCRATCH_BYTES - 256);
    if (cudaMemsetAsync(err, 0, sizeof(int), q) != cudaSuccess) return ONMF_ECUDA;
    if (launch_prepare(sh, W, Wrm, Wimg, swpart, q, Wrow) != cudaSuccess) return ONMF_ECUDA;
    if (n == 0) {
        if (obj_sum && cudaMemsetAsync(obj_sum, 0, sizeof(double), q) != cudaSuccess)
            return ONMF_ECUDA;
        return ONMF_OK;
    }
    TileArgs a;
    memset(&a, 0, sizeof a);
    a.s = sh;
    a.eps = (float)eps;
    a.gamma = (float)h_exponent;
    a.n_in = n_inner;
    a.V = V;
    a.ldv = ldv;
    a.n = n;
    a.H_out = H_out;
    a.ldh = ldh;
    a.final_pass = obj_sum ? 1 : 0;
    a.Wcm = W;
    a.Wrm = Wrm;
    a.Wimg = Wimg;
    a.Wrow = Wrow;
    a.swpart = swpart;
    a.loss_part = obj_sum ? loss : nullptr;
    a.err = err;
    if (prec == PREC_CL) {
        if (launch_tiles_cluster(a, ct.C, ct.grid, smem, q) != cudaSuccess) return ONMF_ECUDA;
    } else {
        int dev = 0, nsm = 1;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        const int grid = (int)(ntiles < 2LL * nsm ? ntiles : 2LL * nsm);
        if (launch_tiles(a, prec, grid, smem, q) != cudaSuccess) return ONMF_ECUDA;
    }
    if (obj_sum && launch_sum(loss, ntiles, obj_sum, 0, q) != cudaSuccess) return ONMF_ECUDA;
    return ONMF_OK;
}
