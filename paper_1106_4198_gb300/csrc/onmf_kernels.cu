// libonmf kernels: host-side launchers, the FP32 instantiation of the step
// kernels (onmf_step.cuh), and the small helper kernels (derived images of
// W, ordered sums, the batch W step and rescales).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

#include "onmf.h"
#include "onmf_cluster.cuh"
#include "onmf_device.cuh"
#include "onmf_kernels.cuh"
#include "onmf_launch.h"
#include "onmf_serve.cuh"
#include "onmf_step.cuh"

namespace onmf {

// Guards the per-device caches of launch queries below.
static std::mutex g_cache_mu;

// Derived images of a dictionary W (column-major F x K): the row-major copy,
// the bf16 W^T image and the column sums. One warp per column.
__global__ void __launch_bounds__(kThreads) prepare_kernel(Shape s, const float *Wcm, float *Wrm,
                                                           __nv_bfloat16 *Wimg,
                                                           __nv_bfloat16 *Wrow, float *swpart) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int nw = gridDim.x * kWarps;
    for (int k = gw; k < s.K; k += nw) {
        float sum = 0.f;
        for (int f = lane; f < s.F; f += 32) {
            const float w = Wcm[f + (long long)k * s.F];
            sum += w;
            if (Wrm) Wrm[(long long)f * s.K + k] = w;
            if (Wimg) Wimg[(long long)k * s.WLD + f] = __float2bfloat16_rn(w);
            if (Wrow) Wrow[(long long)f * s.Kp + k] = __float2bfloat16_rn(w);
        }
        sum = warp_sum(sum);
        if (lane == 0) swpart[k] = sum;
    }
}

__global__ void __launch_bounds__(kThreads) sum_kernel(const double *x, long long n, double *out,
                                                       int accumulate) {
    __shared__ double red[kThreads];
    double r = block_sum_ordered(x, n, red);
    if (threadIdx.x == 0) *out = accumulate ? *out + r : r;
}

// --------------------------------------------------------------- batch

// W <- W o sqrt((P H^T)/(Q H^T)) from the chunk partials (fixed order).
__global__ void __launch_bounds__(kThreads) batch_wstep_kernel(Shape s, const float *part,
                                                               int nchunks, float *W) {
    const long long n = (long long)s.F * s.K;
    for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kThreads) {
        const int k = (int)(i / s.F), f = (int)(i - (long long)k * s.F);
        float ph = 0.f, qh = 0.f;
        for (int c = 0; c < nchunks; ++c) {
            ph += part[(((long long)c * 2 + 0) * s.Fp16 + f) * s.Kh + k];
            qh += part[(((long long)c * 2 + 1) * s.Fp16 + f) * s.Kh + k];
        }
        if (qh > 0.f) W[i] = W[i] * sqrtf(__fdiv_rn(ph, qh));
    }
}

// Column sums of W; W_:k /= s_k and scale[k] = s_k (1 where not rescaled).
__global__ void __launch_bounds__(kThreads) batch_normalize_kernel(Shape s, int normalize, float *W,
                                                                   float *scale, int *err) {
    const int lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kWarps + (threadIdx.x >> 5);
    const int nw = gridDim.x * kWarps;
    for (int k = gw; k < s.K; k += nw) {
        float *col = W + (long long)k * s.F;
        float sum = 0.f;
        for (int f = lane; f < s.F; f += 32) sum += col[f];
        sum = warp_sum(sum);
        const bool sc = normalize && sum > 0.f;
        const float inv = sc ? __frcp_rn(sum) : 1.f;
        bool bad = false;
        for (int f = lane; f < s.F; f += 32) {
            float w = col[f] * inv;
            bad |= !isfinite(w);
            col[f] = w;
        }
        if (bad) flag_error(err, ERR_NUMERIC);
        if (lane == 0) scale[k] = sc ? sum : 1.f;
    }
}

__global__ void __launch_bounds__(kThreads) batch_scale_h_kernel(int K, long long N, float *H,
                                                                 const float *scale) {
    const long long n = (long long)K * N;
    for (long long i = blockIdx.x * (long long)kThreads + threadIdx.x; i < n;
         i += (long long)gridDim.x * kThreads) {
        H[i] *= scale[i % K];
    }
}

// Batch start point: H_kn = sum_f (eps + V_fn) / sum W for every k.
__global__ void __launch_bounds__(kThreads) batch_h0_kernel(Shape s, const float *V, long long ldv,
                                                            long long N, float eps,
                                                            const float *swpart, float *H) {
    const int lane = threadIdx.x & 31;
    __shared__ float s_sw;
    if (threadIdx.x < 32) {
        float a = 0.f;
        for (int k = lane; k < s.K; k += 32) a += swpart[k];
        a = warp_sum(a);
        if (lane == 0) s_sw = a;
    }
    __syncthreads();
    const float sw = s_sw;
    const long long gw = blockIdx.x * (long long)kWarps + (threadIdx.x >> 5);
    const long long nw = (long long)gridDim.x * kWarps;
    for (long long n = gw; n < N; n += nw) {
        float a = 0.f;
        for (int f = lane; f < s.F; f += 32) a += eps + V[n * ldv + f];
        a = warp_sum(a);
        for (int k = lane; k < s.K; k += 32) H[n * s.K + k] = a / sw;
    }
}

// ===================================================================== host

static int64_t g_launches = 0;

int64_t kernel_launches() { return __atomic_load_n(&g_launches, __ATOMIC_RELAXED); }
static void count_launch(int n = 1) { __atomic_fetch_add(&g_launches, n, __ATOMIC_RELAXED); }

static size_t hsolve_smem(const Shape &s, int prec) {
    if (prec == PREC_TC) return tc_layout(s).total;
    return prec == PREC_MIXED ? mixed_layout(s).total : hsolve_fp32_smem_bytes(s);
}

bool tc_shape_supported(const Shape &s) { return tc_supported(s); }

size_t online_smem_bytes(const Shape &s, int prec) {
    size_t p1 = hsolve_smem(s, prec);
    size_t p2 = stats_smem_bytes(prec);
    if (prec == PREC_MIXED && p2 < kStatsSmemBytes) p2 = kStatsSmemBytes;  // tcgen05 statistics
    return p1 > p2 ? p1 : p2;
}

size_t tile_smem_bytes(const Shape &s, int prec) { return hsolve_smem(s, prec); }

size_t batch_stats_smem_bytes(int prec) { return stats_smem_bytes(prec); }

// Mixed-precision kernels are instantiated per k-slab count in
// onmf_mixed_lo.cu (1..4) and onmf_mixed_hi.cu (5..8).
const void *mixed_online_lo(int prec, int ks);
const void *mixed_online_hi(int prec, int ks);
const void *mixed_tile_lo(int prec, int ks);
const void *mixed_tile_hi(int prec, int ks);
const void *mixed_serve_lo(int ks);
const void *mixed_serve_hi(int ks);
// The penalized mma variants (1..8), in onmf_mixed_pen.cu.
const void *mixed_online_pen(int ks);
const void *mixed_tile_pen(int ks);

// Cluster h-solve kernels, instantiated per k16-slab count in
// onmf_cluster_lo.cu (1..8) and onmf_cluster_hi.cu (9..16).
const void *cluster_online_lo(int ks);
const void *cluster_online_hi(int ks);
const void *cluster_tile_lo(int ks);
const void *cluster_tile_hi(int ks);

static const void *cluster_online_fn(int ks) {
    return ks <= 8 ? cluster_online_lo(ks) : cluster_online_hi(ks);
}
static const void *cluster_tile_fn(int ks) {
    return ks <= 8 ? cluster_tile_lo(ks) : cluster_tile_hi(ks);
}

size_t cluster_smem_bytes(const Shape &s, int C, bool online) {
    const size_t h = cl_layout(s, C).total;
    const size_t st = online ? stats_smem_bytes(PREC_MIXED) : 0;
    return h > st ? h : st;
}

static cudaLaunchConfig_t cluster_config(int C, int grid, size_t smem, cudaStream_t stream,
                                         cudaLaunchAttribute *at, bool cooperative) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    at[1].id = cudaLaunchAttributeCooperative;
    at[1].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = cooperative ? 2 : 1;
    return cfg;
}

int cluster_max_active(const Shape &s, int C, bool online) {
    // cached per (device, k16 slabs, C, online, shared memory): the answer is
    // an occupancy query that depends on nothing else
    static std::map<std::tuple<int, int, int, int, size_t>, int> cache;
    int dev = 0;
    cudaGetDevice(&dev);
    const size_t smem = cluster_smem_bytes(s, C, online);
    const auto key = std::make_tuple(dev, s.Kp / 16, C, online ? 1 : 0, smem);
    {
        std::lock_guard<std::mutex> lock(g_cache_mu);
        auto it = cache.find(key);
        if (it != cache.end()) return it->second;
    }
    const void *fn = online ? cluster_online_fn(s.Kp / 16) : cluster_tile_fn(s.Kp / 16);
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = cluster_config(C, C * 1024, smem, 0, at, false);
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    std::lock_guard<std::mutex> lock(g_cache_mu);
    cache[key] = n;
    return n;
}

// Cluster size for `frames` frames per launch round: the smallest C whose
// 32-frame tiles give at least 3/4 of the SMs a CTA, else the largest C
// that fits (0 if none does).
int cluster_choose(const Shape &s, long long frames, int num_sms, size_t smem_limit, bool online) {
    const long long tiles = (frames + kClTile - 1) / kClTile;
    int best = 0;
    for (int C = 1; C <= kClMaxC; C *= 2) {
        if (!cl_supported(s, C) || cluster_smem_bytes(s, C, online) > smem_limit) continue;
        best = C;
        if (tiles * C >= (long long)num_sms * 3 / 4) break;
    }
    return best;
}

// The h-solve kernel for a shape and an onmf_hsolve choice, or -1 if the
// shape does not allow that choice. K > 128 needs the cluster h-solve (the
// whole bf16 W^T no longer fits one CTA's shared memory). Under AUTO the
// environment variable ONMF_HSOLVE=mma|tc|cluster selects a variant where
// the shape allows it.
int select_prec(bool mixed, const Shape &s, int hsolve) {
    if (!mixed) return PREC_FP32;
    const bool big = s.Kp > 128;
    switch (hsolve) {
    case ONMF_HSOLVE_MMA: return big ? -1 : PREC_MIXED;
    case ONMF_HSOLVE_TC: return (!big && tc_supported(s)) ? PREC_TC : -1;
    case ONMF_HSOLVE_CLUSTER: return PREC_CL;
    case ONMF_HSOLVE_AUTO: break;
    default: return -1;
    }
    const char *env = getenv("ONMF_HSOLVE");
    if (env && strcmp(env, "tc") == 0 && !big && tc_supported(s)) return PREC_TC;
    if (env && strcmp(env, "mma") == 0 && !big) return PREC_MIXED;
    if (env && strcmp(env, "cluster") == 0) return PREC_CL;
    return big ? PREC_CL : PREC_MIXED;
}

ClusterTiles cluster_tiles(const Shape &s, long long n) {
    ClusterTiles r;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    r.C = cluster_choose(s, n, nsm, max_dynamic_smem(), false);
    if (r.C == 0) return r;
    const long long tiles = (n + kClTile - 1) / kClTile;
    const long long act = std::max(1, cluster_max_active(s, r.C, false));
    r.grid = (int)(std::min(tiles, 2 * act) * r.C);
    r.smem = cluster_smem_bytes(s, r.C, false);
    r.slots = tiles * r.C;
    return r;
}

// Serving kernels: FP32 (one variant) or mixed, one per k16-slab count.
const void *serve_fn(int prec, int ks) {
    if (prec == PREC_FP32) return (const void *)serve_hsolve_kernel<PREC_FP32, 0>;
    return ks <= 4 ? mixed_serve_lo(ks) : mixed_serve_hi(ks);
}

// Serving phases 2 and 3 (not specialized by dictionary size).
const void *serve_stats_fn(int prec) {
    return prec == PREC_FP32 ? (const void *)serve_stats_kernel<PREC_FP32>
                             : (const void *)serve_stats_kernel<PREC_MIXED>;
}
const void *serve_gather_fn() { return (const void *)serve_gather_kernel<kGatherU>; }
const void *serve_rescale_fn(int prec) {
    return prec == PREC_FP32 ? (const void *)serve_rescale_kernel<PREC_FP32>
                             : (const void *)serve_rescale_kernel<PREC_MIXED>;
}

// pen: the penalized variant (the mma path only; FP32 takes penalties in its
// one instantiation)
static const void *online_fn(int prec, int ks, bool pen = false) {
    if (prec == PREC_FP32) return (const void *)online_kernel<PREC_FP32, 0>;
    if (pen && prec == PREC_MIXED) return mixed_online_pen(ks);
    return ks <= 4 ? mixed_online_lo(prec, ks) : mixed_online_hi(prec, ks);
}
static const void *tile_fn(int prec, int ks, bool pen = false) {
    if (prec == PREC_FP32) return (const void *)tile_kernel<PREC_FP32, 0>;
    if (pen && prec == PREC_MIXED) return mixed_tile_pen(ks);
    return ks <= 4 ? mixed_tile_lo(prec, ks) : mixed_tile_hi(prec, ks);
}
static const void *bstats_fn(int prec) {
    return prec != PREC_FP32 ? (const void *)batch_stats_kernel<PREC_MIXED>
                              : (const void *)batch_stats_kernel<PREC_FP32>;
}

// Allow each kernel the largest dynamic shared memory the device grants a
// block (the opt-in limit minus the kernel's static shared memory).
cudaError_t configure_kernels() {
    int dev = 0, optin = 0;
    cudaError_t e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) !=
        cudaSuccess)
        return e;
    std::vector<const void *> fns = {online_fn(0, 0), tile_fn(0, 0), bstats_fn(0), bstats_fn(1),
                                     serve_fn(PREC_FP32, 0)};
    for (int p = PREC_MIXED; p <= PREC_TC; ++p)
        for (int ks = 1; ks <= 8; ++ks) {
            fns.push_back(online_fn(p, ks));
            fns.push_back(tile_fn(p, ks));
        }
    for (int ks = 1; ks <= 8; ++ks) {
        fns.push_back(serve_fn(PREC_MIXED, ks));
        fns.push_back(online_fn(PREC_MIXED, ks, true));
        fns.push_back(tile_fn(PREC_MIXED, ks, true));
    }
    for (int p = PREC_FP32; p <= PREC_MIXED; ++p) fns.push_back(serve_stats_fn(p));
    fns.push_back(serve_any_fn());
    for (int ks = 1; ks <= 16; ++ks) {
        fns.push_back(cluster_online_fn(ks));
        fns.push_back(cluster_tile_fn(ks));
    }
    for (const void *fn : fns) {
        cudaFuncAttributes at;
        if ((e = cudaFuncGetAttributes(&at, fn)) != cudaSuccess) return e;
        const int dyn = optin - (int)at.sharedSizeBytes;
        if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn)) !=
            cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

// The kernels' static shared memory does not change once the library is
// loaded, so the answer is computed once per device (about 80 attribute
// queries) and cached.
static size_t max_dynamic_smem_uncached() {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes at;
    size_t worst = 0;
    std::vector<const void *> fns = {online_fn(0, 0), tile_fn(0, 0)};
    for (int p = PREC_MIXED; p <= PREC_TC; ++p)
        for (int ks = 1; ks <= 8; ++ks) {
            fns.push_back(online_fn(p, ks));
            fns.push_back(tile_fn(p, ks));
        }
    for (int ks = 1; ks <= 8; ++ks) {
        fns.push_back(online_fn(PREC_MIXED, ks, true));
        fns.push_back(tile_fn(PREC_MIXED, ks, true));
    }
    for (int ks = 1; ks <= 16; ++ks) {
        fns.push_back(cluster_online_fn(ks));
        fns.push_back(cluster_tile_fn(ks));
    }
    for (const void *fn : fns)
        if (cudaFuncGetAttributes(&at, fn) == cudaSuccess && at.sharedSizeBytes > worst)
            worst = at.sharedSizeBytes;
    return (size_t)optin > worst ? optin - worst : 0;
}

size_t max_dynamic_smem() {
    constexpr int kDevs = 64;
    static size_t cached[kDevs];
    static bool have[kDevs];
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs)
        return max_dynamic_smem_uncached();
    std::lock_guard<std::mutex> lock(g_cache_mu);
    if (!have[dev]) {
        cached[dev] = max_dynamic_smem_uncached();
        have[dev] = true;
    }
    return cached[dev];
}

cudaError_t max_coresident_blocks(int prec, int ks, size_t smem, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, online_fn(prec, ks),
                                                         kThreads, smem);
}

cudaError_t launch_online(const StepArgs &a, int prec, int grid, size_t smem,
                          cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(a.bar, 0, 16 + 4 * kMaxRanges, stream);
    if (e != cudaSuccess) return e;
    StepArgs copy = a;
    void *args[] = {&copy};
    const bool pen = a.hpen > 0.f || a.wpen > 0.f;
    e = cudaLaunchCooperativeKernel(online_fn(prec, a.s.Kp / 16, pen), dim3(grid),
                                    dim3(kThreads), args, smem, stream);
    if (e == cudaSuccess) count_launch();
    return e;
}

// The online step on clusters of C CTAs, always as a cooperative launch: its
// grid barriers need every CTA resident at once, which only a cooperative
// launch guarantees (a plain launch sized by the occupancy query can still
// find SMs taken, e.g. by the frame-pull kernel that runs beside it, and
// its barrier would then run out after 2 s instead of failing at launch).
// A runtime that refuses the cooperative attribute together with a cluster
// dimension gets an error here, not a weaker launch.
cudaError_t launch_online_cluster(const StepArgs &a, int C, int grid, size_t smem,
                                  cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    StepArgs copy = a;
    int c = C;
    void *args[] = {&copy, &c};
    const void *fn = cluster_online_fn(a.s.Kp / 16);
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = cluster_config(C, grid, smem, stream, at, true);
    e = cudaLaunchKernelExC(&cfg, fn, args);
    if (e == cudaSuccess) count_launch();
    return e;
}

cudaError_t launch_tiles_cluster(const TileArgs &a, int C, int grid, size_t smem,
                                 cudaStream_t stream) {
    TileArgs copy = a;
    int c = C;
    void *args[] = {&copy, &c};
    cudaLaunchAttribute at[2];
    cudaLaunchConfig_t cfg = cluster_config(C, grid, smem, stream, at, false);
    cudaError_t e = cudaLaunchKernelExC(&cfg, cluster_tile_fn(a.s.Kp / 16), args);
    if (e == cudaSuccess) count_launch();
    return e;
}

cudaError_t launch_tiles(const TileArgs &a, int prec, int grid, size_t smem, cudaStream_t stream) {
    TileArgs copy = a;
    void *args[] = {&copy};
    cudaError_t e = cudaLaunchKernel(tile_fn(prec, a.s.Kp / 16, a.hpen > 0.f), dim3(grid),
                                     dim3(kThreads), args, smem, stream);
    if (e == cudaSuccess) count_launch();
    return e;
}

cudaError_t launch_prepare(const Shape &s, const float *Wcm, float *Wrm, __nv_bfloat16 *Wimg,
                           float *swpart, cudaStream_t stream, __nv_bfloat16 *Wrow) {
    const int grid = (s.K + kWarps - 1) / kWarps;
    prepare_kernel<<<grid, kThreads, 0, stream>>>(s, Wcm, Wrm, Wimg, Wrow, swpart);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_sum(const double *x, long long n, double *out, int accumulate,
                       cudaStream_t stream) {
    sum_kernel<<<1, kThreads, 0, stream>>>(x, n, out, accumulate);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_stats(const Shape &s, int prec, const void *Pg, const void *Qg,
                               const void *Hg, long long betap, long long N, int nchunks,
                               float *part, int grid, cudaStream_t stream) {
    const size_t smem = stats_smem_bytes(prec);
    void *args[8];
    Shape sc = s;
    const void *p = Pg, *q = Qg, *h = Hg;
    long long bp = betap, n = N;
    int nc = nchunks;
    float *pt = part;
    args[0] = &sc;
    args[1] = &p;
    args[2] = &q;
    args[3] = &h;
    args[4] = &bp;
    args[5] = &n;
    args[6] = &nc;
    args[7] = &pt;
    cudaError_t e = cudaLaunchKernel(bstats_fn(prec), dim3(grid), dim3(kThreads), args, smem, stream);
    if (e == cudaSuccess) count_launch();
    return e;
}

cudaError_t launch_batch_wstep(const Shape &s, const float *part, int nchunks, float *W,
                               cudaStream_t stream) {
    const long long n = (long long)s.F * s.K;
    const int grid = (int)min(4096LL, (n + kThreads - 1) / kThreads);
    batch_wstep_kernel<<<grid, kThreads, 0, stream>>>(s, part, nchunks, W);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_normalize(const Shape &s, int normalize, float *W, float *scale, int *err,
                                   cudaStream_t stream) {
    const int grid = (s.K + kWarps - 1) / kWarps;
    batch_normalize_kernel<<<grid, kThreads, 0, stream>>>(s, normalize, W, scale, err);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_scale_h(int K, long long N, float *H, const float *scale,
                                 cudaStream_t stream) {
    const long long n = (long long)K * N;
    const int grid = (int)min(8192LL, (n + kThreads - 1) / kThreads);
    batch_scale_h_kernel<<<grid, kThreads, 0, stream>>>(K, N, H, scale);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_batch_h0(const Shape &s, const float *V, long long ldv, long long N, float eps,
                            const float *swpart, float *H, cudaStream_t stream) {
    const int grid = (int)min(4096LL, (N + kWarps - 1) / kWarps);
    batch_h0_kernel<<<grid, kThreads, 0, stream>>>(s, V, ldv, N, eps, swpart, H);
    count_launch();
    return cudaGetLastError();
}

// Row gather / scatter for passes over a finite data set in a given order:
// dst row r <- src row idx[first + r] (gather), dst row idx[first + r] <- src
// row r (scatter); idx NULL means rows first + r. One warp per row.
__global__ void __launch_bounds__(kThreads) gather_rows_kernel(float *dst, long long ld_dst,
                                                              const float *src, long long ld_src,
                                                              const long long *idx, long long first,
                                                              long long n, int width) {
    const int lane = threadIdx.x & 31;
    for (long long r = blockIdx.x * (long long)kWarps + (threadIdx.x >> 5); r < n;
         r += (long long)gridDim.x * kWarps) {
        const long long sr = idx ? idx[first + r] : first + r;
        for (int c = lane; c < width; c += 32) dst[r * ld_dst + c] = src[sr * ld_src + c];
    }
}

__global__ void __launch_bounds__(kThreads) scatter_rows_kernel(float *dst, long long ld_dst,
                                                               const float *src, long long ld_src,
                                                               const long long *idx,
                                                               long long first, long long n,
                                                               int width) {
    const int lane = threadIdx.x & 31;
    for (long long r = blockIdx.x * (long long)kWarps + (threadIdx.x >> 5); r < n;
         r += (long long)gridDim.x * kWarps) {
        const long long dr = idx ? idx[first + r] : first + r;
        for (int c = lane; c < width; c += 32) dst[dr * ld_dst + c] = src[r * ld_src + c];
    }
}

__global__ void __launch_bounds__(kThreads) index_rows_kernel(long long *dst, const long long *idx,
                                                             long long first, long long n) {
    for (long long r = blockIdx.x * (long long)kThreads + threadIdx.x; r < n;
         r += (long long)gridDim.x * kThreads)
        dst[r] = idx ? idx[first + r] : first + r;
}

// Frames from mapped pinned host memory into a device ring slot, pulled by
// the SMs (the step kernel leaves some free) instead of a copy engine: rows
// of F floats, source leading dimension lds, destination dense. float4 with
// four loads in flight per thread when both ends allow it.
__global__ void __launch_bounds__(kThreads) pull_rows_kernel(float *__restrict__ dst, int F,
                                                            const float *__restrict__ src,
                                                            long long lds, long long n,
                                                            int vec) {
    const long long T = (long long)gridDim.x * kThreads;
    const long long t0 = blockIdx.x * (long long)kThreads + threadIdx.x;
    if (vec) {
        const long long nv = n * F / 4;
        const float4 *s4 = reinterpret_cast<const float4 *>(src);
        float4 *d4 = reinterpret_cast<float4 *>(dst);
        for (long long i = t0; i < nv; i += 4 * T) {
            float4 r[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i + u * T < nv) r[u] = s4[i + u * T];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (i + u * T < nv) d4[i + u * T] = r[u];
        }
    } else {
        const int lane = threadIdx.x & 31;
        for (long long r = t0 >> 5; r < n; r += T >> 5)
            for (int c = lane; c < F; c += 32) dst[r * F + c] = src[r * lds + c];
    }
}

cudaError_t launch_pull_rows(float *dst, int F, const float *src, long long lds, long long n,
                             cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    const int vec = lds == F && ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0 &&
                    ((long long)n * F) % 4 == 0;
    pull_rows_kernel<<<kPullCtas, kThreads, 0, stream>>>(dst, F, src, lds, n, vec);
    count_launch();
    return cudaGetLastError();
}

static int rows_grid(long long n) {
    const long long g = (n + kWarps - 1) / kWarps;
    return (int)(g < 4096 ? (g > 0 ? g : 1) : 4096);
}

cudaError_t launch_gather_rows(float *dst, long long ld_dst, const float *src, long long ld_src,
                               const long long *idx, long long first, long long n, int width,
                               cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    gather_rows_kernel<<<rows_grid(n), kThreads, 0, stream>>>(dst, ld_dst, src, ld_src, idx, first,
                                                              n, width);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_scatter_rows(float *dst, long long ld_dst, const float *src, long long ld_src,
                                const long long *idx, long long first, long long n, int width,
                                cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    scatter_rows_kernel<<<rows_grid(n), kThreads, 0, stream>>>(dst, ld_dst, src, ld_src, idx,
                                                               first, n, width);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_index_rows(long long *dst, const long long *idx, long long first, long long n,
                              cudaStream_t stream) {
    if (n <= 0) return cudaSuccess;
    const long long g = (n + kThreads - 1) / kThreads;
    index_rows_kernel<<<(int)(g < 1024 ? g : 1024), kThreads, 0, stream>>>(dst, idx, first, n);
    count_launch();
    return cudaGetLastError();
}

// Fault-path self-test: runs one of the library's bounded waits on a
// condition that can never hold, so the wait must run out, flag ERR_TIMEOUT
// and leave the kernel with the context intact.
//   which 0: grid barrier expecting one CTA more than the grid has;
//   which 1: mbarrier phase that nothing arrives on;
//   which 2: as 1, while the CTA holds tensor memory, which it frees before
//            returning (the exit path of the tcgen05 h-solve kernels).
__global__ void __launch_bounds__(kThreads) wait_selftest_kernel(int which, unsigned *counter,
                                                                 int *err,
                                                                 unsigned long long *elapsed) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tslot;
    cta_err_init(err);
    const uint64_t t0 = global_ns();
    if (which == 0) {
        unsigned epoch = 0;
        grid_sync(counter, gridDim.x + 1, epoch, err);
    } else {
        if (threadIdx.x == 0) {
            mbar_init(&bar, 1);
            fence_mbar_init();
        }
        if (which == 2 && threadIdx.x < 32) tmem_alloc(&tslot, 32);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (threadIdx.x == 0) mbar_wait_bounded(&bar, 0, err);
        tc_fence_before();
        __syncthreads();
        if (which == 2 && threadIdx.x < 32) tmem_dealloc(tslot, 32);
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) *elapsed = global_ns() - t0;
}

cudaError_t launch_wait_selftest(int which, unsigned *counter, int *err,
                                 unsigned long long *elapsed, cudaStream_t stream) {
    void *args[] = {&which, &counter, &err, &elapsed};
    cudaError_t e = which == 0 ? cudaLaunchCooperativeKernel((const void *)wait_selftest_kernel,
                                                             dim3(2), dim3(kThreads), args, 0,
                                                             stream)
                               : cudaLaunchKernel((const void *)wait_selftest_kernel, dim3(2),
                                                  dim3(kThreads), args, 0, stream);
    if (e == cudaSuccess) count_launch();
    return e;
}

}  // namespace onmf
