// C ABI of libonmf (include/onmf.h): state management, the minibatch
// staging of Algorithm 1's frame stream, host/device pointer handling and
// the batch cycle driver. Every step of the arithmetic runs in the kernels of
// onmf_kernels.cu; this file only allocates, copies and launches.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "onmf.h"
#include "onmf_cluster.cuh"
#include "onmf_device.cuh"
#include "onmf_kernels.cuh"
#include "onmf_launch.h"

using namespace onmf;

namespace {

thread_local char g_msg[512] = "";

// NVTX range around a library call (shows in Nsight timelines; no cost
// without a tool attached).
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range &) = delete;
    Range &operator=(const Range &) = delete;
};

void set_msg(const char *what, cudaError_t e) {
    snprintf(g_msg, sizeof g_msg, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                   \
    do {                                           \
        cudaError_t e_ = (call);                   \
        if (e_ != cudaSuccess) {                   \
            set_msg(#call, e_);                    \
            return e_ == cudaErrorMemoryAllocation ? ONMF_ENOMEM : ONMF_ECUDA; \
        }                                          \
    } while (0)

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

onmf_status status_from_err(int bits) {
    if (bits & ERR_CONFIG) return ONMF_ECUDA;
    if (bits & ERR_TIMEOUT) return ONMF_ETIMEOUT;
    if (bits & (ERR_INPUT | ERR_NUMERIC)) return ONMF_ENUMERIC;
    return ONMF_OK;
}

double rho_of(const onmf_config &c, long long nb) {
    if (c.n_ref <= 0) return 1.0;
    return std::pow(c.r, (double)nb / (double)c.n_ref);
}

struct Segment {
    int off, n;      // columns of the staging buffer
    float *dst;      // caller's H_out for these frames
    long long ldh;
};

int g_configured = 0;

// Mixed precision runs the mma.sync h-solve unless ONMF_HSOLVE=tc selects the
// tcgen05 one (where the shape allows it: F >= 128 with at most 32 rows past
// the last 128-row tile, K <= 128). At 16-frame tiles a tcgen05 MMA costs a
// fixed ~55 cycles (N <= 64), which leaves the two within ~10% of each other
// on the online minibatch; the faster one is picked per shape by measurement.
// The tcgen05 kernels allocate all 512 TMEM columns per CTA; asking for more
// than half of an SM's shared memory keeps them at one CTA per SM, so an
// allocation never waits on a co-resident CTA (which, inside a cooperative
// launch, could be waiting at a grid barrier).
size_t tc_min_smem(int prec, size_t smem) {
    const size_t one_per_sm = 116 * 1024;
    return (prec == PREC_TC && smem < one_per_sm) ? one_per_sm : smem;
}

int pick_prec(int precision, const Shape &sh, int hsolve = ONMF_HSOLVE_AUTO) {
    return select_prec(precision == ONMF_MIXED, sh, hsolve);
}

onmf_status ensure_configured() {
    if (!g_configured) {
        CK(configure_kernels());
        g_configured = 1;
    }
    return ONMF_OK;
}

}  // namespace

struct onmf_state {
    onmf_config cfg;
    Shape s;
    cudaStream_t stream;
    int prec;
    int C = 0;  // CTAs per cluster (cluster h-solve)
    // state
    float *Wcm = nullptr, *Wrm = nullptr, *Wn = nullptr, *swpart = nullptr;
    __nv_bfloat16 *Wimg = nullptr, *Wrow = nullptr;
    double *A = nullptr, *B = nullptr, *loss_sum = nullptr;
    // scratch
    void *Pg = nullptr, *Qg = nullptr, *Hg = nullptr;
    float *part = nullptr;  // frame-range partial sums of the tcgen05 statistics
    long long *stamps = nullptr;  // phase-timing builds only
    int betap = 0;
    double *loss_part = nullptr, *tmp_sum = nullptr;
    unsigned *bar = nullptr;
    int *err_d = nullptr;
    int *err_h = nullptr;  // pinned mirror of err_d
    // staging of a partial minibatch
    float *staging = nullptr, *Hstage = nullptr;
    int staged = 0;
    std::vector<Segment> segs;
    // host-input ring: copies on copy_stream overlap the step kernels
    float *vring[2] = {nullptr, nullptr};
    float *hring[2] = {nullptr, nullptr};
    cudaEvent_t ring_ev[2] = {nullptr, nullptr};    // slot consumed by the step kernels
    cudaEvent_t ring_full[2] = {nullptr, nullptr};  // slot filled by the copy
    cudaStream_t copy_stream = nullptr;
    long long ring_frames = 0;
    // warm restarts: gathered frames and h of a pass, staged start points
    float *gV = nullptr, *gH = nullptr, *Hin_stage = nullptr;
    long long *stage_idx = nullptr;
    long long gcap = 0;
    bool warm_staged = false;  // the staged frames came from a warm push
    float *warm_H = nullptr;   // their h rows live in this array (ld warm_ldh)
    long long warm_ldh = 0;
    double *obj_h = nullptr;  // pinned
    long long t = 0;
    int sticky = ONMF_OK;
    int grid = 1, tile_grid = 1;
    size_t smem = 0, tile_smem = 0;
    int num_sms = 1;
};

static onmf_status check_sticky(onmf_state *s) {
    if (s->sticky != ONMF_OK) return ONMF_ESTATE;
    int bits = __atomic_load_n(s->err_h, __ATOMIC_ACQUIRE);
    if (bits) {
        s->sticky = status_from_err(bits);
        return (onmf_status)s->sticky;
    }
    return ONMF_OK;
}

static onmf_status mirror_err(onmf_state *s) {
    CK(cudaMemcpyAsync(s->err_h, s->err_d, sizeof(int), cudaMemcpyDeviceToHost, s->stream));
    return ONMF_OK;
}

static onmf_status sync_and_check(onmf_state *s) {
    CK(cudaStreamSynchronize(s->stream));
    int bits = *s->err_h;
    if (bits && s->sticky == ONMF_OK) s->sticky = status_from_err(bits);
    return s->sticky == ONMF_OK ? ONMF_OK : (onmf_status)s->sticky;
}

static onmf_status prepare_images(onmf_state *s) {
    CK(launch_prepare(s->s, s->Wcm, s->prec == PREC_FP32 ? s->Wrm : nullptr, s->Wimg, s->swpart,
                      s->stream, s->Wrow));
    return ONMF_OK;
}

extern "C" {

void onmf_config_default(onmf_config *c, int32_t F, int32_t K) {
    if (!c) return;
    memset(c, 0, sizeof *c);
    c->F = F;
    c->K = K;
    c->beta = 1000;
    c->n_inner = 10;
    c->eps = 1e-12;
    c->r = 1.0;
    c->n_ref = 0;
    c->h_exponent = 0.5;
    c->normalize = 1;
    c->rho_on_new = 0;
    c->precision = ONMF_FP32;
    c->h_penalty = 0.0;
    c->h_penalty_a = 1.0;
    c->w_penalty = 0.0;
}

const char *onmf_status_string(onmf_status st) {
    switch (st) {
    case ONMF_OK: return "ONMF_OK";
    case ONMF_EINVAL: return "ONMF_EINVAL: invalid argument";
    case ONMF_ENOMEM: return "ONMF_ENOMEM: out of memory";
    case ONMF_EBUDGET: return "ONMF_EBUDGET: memory budget exceeded";
    case ONMF_ECUDA: return "ONMF_ECUDA: CUDA runtime error";
    case ONMF_ENUMERIC: return "ONMF_ENUMERIC: invalid input value or non-finite result";
    case ONMF_ETIMEOUT: return "ONMF_ETIMEOUT: device wait timed out";
    case ONMF_ESTATE: return "ONMF_ESTATE: state holds a sticky error";
    case ONMF_EAGAIN: return "ONMF_EAGAIN: not ready";
    }
    return "unknown onmf status";
}

const char *onmf_last_error_message(void) { return g_msg; }

int64_t onmf_kernel_launches(void) { return kernel_launches(); }

int32_t onmf_abi_version(void) { return ONMF_ABI_VERSION; }

onmf_status onmf_selftest_wait(int32_t which, void *stream, int64_t *elapsed_ns) {
    if (which < 0 || which > 2) return ONMF_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    unsigned *counter = nullptr;
    int *err = nullptr;
    unsigned long long *el = nullptr;
    onmf_status rc = ONMF_OK;
    int bits = 0;
    unsigned long long el_h = 0;
    cudaError_t e = cudaMalloc((void **)&counter, 256);
    if (e == cudaSuccess) {
        err = (int *)((char *)counter + 64);
        el = (unsigned long long *)((char *)counter + 128);
        e = cudaMemsetAsync(counter, 0, 256, st);
    }
    if (e == cudaSuccess) e = launch_wait_selftest(which, counter, err, el, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bits, err, sizeof bits, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&el_h, el, sizeof el_h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        set_msg("wait self-test", e);
        rc = e == cudaErrorMemoryAllocation ? ONMF_ENOMEM : ONMF_ECUDA;
    } else {
        rc = status_from_err(bits);
        if (elapsed_ns) *elapsed_ns = (int64_t)el_h;
    }
    if (counter) cudaFree(counter);
    return rc;
}

void onmf_destroy(onmf_state *s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    if (s->copy_stream) cudaStreamSynchronize(s->copy_stream);
    void *dev[] = {s->Wcm, s->Wrm, s->Wn, s->swpart, s->Wimg, s->Wrow, s->A, s->B, s->loss_sum, s->Pg,
                   s->Qg, s->Hg, s->part, s->stamps, s->loss_part, s->tmp_sum, s->bar, s->err_d, s->staging,
                   s->Hstage, s->vring[0], s->vring[1], s->hring[0], s->hring[1],
                   s->gV,     s->gH,       s->Hin_stage, s->stage_idx};
    for (void *p : dev)
        if (p) cudaFree(p);
    if (s->err_h) cudaFreeHost(s->err_h);
    if (s->obj_h) cudaFreeHost(s->obj_h);
    for (int i = 0; i < 2; ++i) {
        if (s->ring_ev[i]) cudaEventDestroy(s->ring_ev[i]);
        if (s->ring_full[i]) cudaEventDestroy(s->ring_full[i]);
    }
    if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
    delete s;
}

onmf_status onmf_init(const onmf_config *cfg, const float *W0, int32_t W0_on_device,
                      void *stream, onmf_state **out) {
    (void)W0_on_device;
    if (!cfg || !W0 || !out) return ONMF_EINVAL;
    *out = nullptr;
    const onmf_config &c = *cfg;
    if (c.F < 1 || c.F > 8192 || c.K < 1 || c.K > 256 || c.beta < 1 || c.beta > (1 << 20) ||
        c.n_inner < 0 || c.n_inner > 100000 || !(c.eps >= 0.0) || !std::isfinite(c.eps) ||
        !(c.r >= 0.0 && c.r <= 1.0) || !(c.h_exponent > 0.0) || c.hsolve < 0 || c.hsolve > 3 ||
        (c.precision != ONMF_FP32 && c.precision != ONMF_MIXED) || c.accumulate < 0 ||
        c.accumulate > 2 || c.stats_ranges < 0 || c.stats_ranges > kMaxRanges ||
        !(c.h_penalty >= 0.0) || !std::isfinite(c.h_penalty) ||
        !(c.h_penalty_a > 0.0) || !std::isfinite(c.h_penalty_a) || !(c.w_penalty >= 0.0) ||
        !std::isfinite(c.w_penalty))
        return ONMF_EINVAL;

    if (c.precision == ONMF_MIXED && c.F > 1024) {
        snprintf(g_msg, sizeof g_msg, "mixed precision supports F <= 1024");
        return ONMF_EINVAL;
    }
    // the kernel choice and what it takes are host checks, before any device work
    const int prec = pick_prec(c.precision, make_shape(c.F, c.K), c.hsolve);
    if (prec < 0) {
        snprintf(g_msg, sizeof g_msg, "h-solve %d does not support F=%d K=%d", c.hsolve, c.F, c.K);
        return ONMF_EINVAL;
    }
    if ((c.h_penalty > 0.0 || c.w_penalty > 0.0) && prec != PREC_FP32 && prec != PREC_MIXED &&
        prec != PREC_CL) {
        snprintf(g_msg, sizeof g_msg, "penalties run on the FP32, mma and cluster paths");
        return ONMF_EINVAL;
    }
    onmf_status st = ensure_configured();
    if (st != ONMF_OK) return st;
    onmf_state *s = new onmf_state();
    s->cfg = c;
    s->s = make_shape(c.F, c.K);
    s->stream = reinterpret_cast<cudaStream_t>(stream);
    s->prec = prec;
    const Shape &sh = s->s;
    const size_t FK = (size_t)c.F * c.K;
    s->betap = (c.beta + 15) / 16 * 16;
    const size_t elem = s->prec == PREC_FP32 ? 4 : 2;
    const int ntiles = (c.beta + kTile - 1) / kTile;
    // loss slots: one per 8-frame tile, or one per (32-frame tile, cluster CTA)
    const int nslots = std::max(ntiles, (c.beta + kClTile - 1) / kClTile * kClMaxC);
    auto fail = [&](onmf_status e) {
        onmf_destroy(s);
        return e;
    };
#define AL(ptr, bytes)                                                         \
    do {                                                                       \
        cudaError_t e_ = cudaMalloc((void **)&(ptr), (bytes));                 \
        if (e_ != cudaSuccess) {                                               \
            set_msg("cudaMalloc", e_);                                         \
            return fail(ONMF_ENOMEM);                                          \
        }                                                                      \
    } while (0)
    AL(s->Wcm, FK * 4);
    AL(s->Wn, FK * 4);
    AL(s->swpart, (size_t)c.K * 4);
    AL(s->A, FK * 8);
    AL(s->B, FK * 8);
    AL(s->loss_sum, 8);
    AL(s->tmp_sum, 8);
    if (s->prec == PREC_FP32) {
        AL(s->Wrm, FK * 4);
        AL(s->Hg, (size_t)s->betap * sh.Kh * 4);
    } else {
        if (s->prec != PREC_CL) AL(s->Wimg, (size_t)sh.Kp * sh.WLD * 2);
        // the mma h-solve writes H in 128-row core blocks (the tcgen05
        // statistics' A operand), the others k rows of betap frames
        AL(s->Hg, (size_t)(s->prec == PREC_MIXED ? 128 : sh.Kh) * s->betap * 2);
        if (s->prec == PREC_TC || s->prec == PREC_CL) AL(s->Wrow, (size_t)sh.F * sh.Kp * 2);
    }
    // P and Q: on the mma path one interleaved core-matrix buffer in Pg,
    // 2 KB per (64-frequency tile, 8-frame group)
    const size_t pq_bytes = s->prec == PREC_MIXED
                                ? (size_t)((sh.Fp16 + 63) / 64) * (s->betap / 8) * 2048
                                : (size_t)s->betap * sh.Fp16 * elem;
    AL(s->Pg, pq_bytes);
    AL(s->Qg, (size_t)s->betap * sh.Fp16 * elem);
    AL(s->loss_part, (size_t)nslots * 8);
    AL(s->bar, 16 + 4 * kMaxRanges);
    AL(s->err_d, 16);
    AL(s->staging, (size_t)c.beta * c.F * 4);
    AL(s->Hstage, (size_t)c.beta * c.K * 4);
#undef AL
    if (cudaHostAlloc((void **)&s->err_h, 16, cudaHostAllocDefault) != cudaSuccess ||
        cudaHostAlloc((void **)&s->obj_h, 16, cudaHostAllocDefault) != cudaSuccess)
        return fail(ONMF_ENOMEM);
    *s->err_h = 0;
    cudaStream_t q = s->stream;
    cudaError_t e = cudaSuccess;
    if (s->Wimg && e == cudaSuccess) e = cudaMemsetAsync(s->Wimg, 0, (size_t)sh.Kp * sh.WLD * 2, q);
    if (s->Wrow && e == cudaSuccess) e = cudaMemsetAsync(s->Wrow, 0, (size_t)sh.F * sh.Kp * 2, q);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(s->Hg, 0,
                            (size_t)(s->prec == PREC_MIXED ? 128 : sh.Kh) * s->betap * elem, q);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->Pg, 0, pq_bytes, q);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->Qg, 0, (size_t)s->betap * sh.Fp16 * elem, q);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->A, 0, FK * 8, q);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->B, 0, FK * 8, q);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->loss_sum, 0, 8, q);
    if (e == cudaSuccess) e = cudaMemsetAsync(s->err_d, 0, 16, q);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s->Wcm, W0, FK * 4, cudaMemcpyDefault, q);
    if (e != cudaSuccess) {
        set_msg("init copies", e);
        return fail(ONMF_ECUDA);
    }
    if ((st = prepare_images(s)) != ONMF_OK) return fail(st);
    // launch geometry
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&s->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (s->prec == PREC_CL) {
        s->C = cluster_choose(sh, c.beta, s->num_sms, max_dynamic_smem(), true);
        if (s->C == 0) {
            snprintf(g_msg, sizeof g_msg, "no cluster layout fits F=%d K=%d", c.F, c.K);
            return fail(ONMF_EINVAL);
        }
        s->smem = cluster_smem_bytes(sh, s->C, true);
    } else {
        s->smem = tc_min_smem(s->prec, online_smem_bytes(sh, s->prec));
    }
    s->tile_smem = tc_min_smem(s->prec, tile_smem_bytes(sh, s->prec));
    if (s->smem > max_dynamic_smem()) {
        snprintf(g_msg, sizeof g_msg, "shared memory need %zu exceeds the device limit", s->smem);
        return fail(ONMF_EINVAL);
    }
    const int units = (sh.Fp16 / 16) * (sh.Kh / 32);
    if (s->prec == PREC_CL) {
        // whole clusters, all co-resident: enough for the tiles and the units
        const int act = cluster_max_active(sh, s->C, true);
        if (act < 1) {
            snprintf(g_msg, sizeof g_msg, "no co-resident cluster of %d CTAs", s->C);
            return fail(ONMF_ECUDA);
        }
        const int tiles = (c.beta + kClTile - 1) / kClTile;
        const int want = std::max(tiles, (std::max(units, c.K) + s->C - 1) / s->C);
        s->grid = std::min(want, act) * s->C;
    } else {
        int per_sm = 0;
        if ((e = max_coresident_blocks(s->prec, sh.Kp / 16, s->smem, &per_sm)) != cudaSuccess ||
            per_sm < 1) {
            set_msg("occupancy", e);
            return fail(ONMF_ECUDA);
        }
        const int tiles = s->prec == PREC_TC ? (c.beta + kTcTile - 1) / kTcTile : ntiles;
        int want = std::max(std::max(tiles, units), (c.K + kWarps - 1) / kWarps);
        s->grid = std::min(want, per_sm * s->num_sms);
    }
    s->tile_grid = s->num_sms;
#ifdef ONMF_PHASE_STAMPS
    {
        const size_t sb = (size_t)kStampMb * kStampCtas * kStampPts * 8;
        if ((e = cudaMalloc((void **)&s->stamps, sb)) != cudaSuccess ||
            (e = cudaMemsetAsync(s->stamps, 0, sb, q)) != cudaSuccess) {
            set_msg("cudaMalloc", e);
            return fail(ONMF_ENOMEM);
        }
    }
#endif
    if (s->prec == PREC_MIXED) {
        // partial sums of the frame ranges of a full minibatch (a partial
        // one has no more ranges)
        const StatsSplit sp = stats_split(c.beta, s->grid, (sh.Fp16 + 63) / 64, c.stats_ranges);
        if ((e = cudaMalloc((void **)&s->part, (size_t)sp.S * 2 * c.K * sh.Fp16 * 4)) !=
            cudaSuccess) {
            set_msg("cudaMalloc", e);
            return fail(ONMF_ENOMEM);
        }
    }
    // sanity: all of W0 finite and >= 0 (checked on the host copy)
    std::vector<float> w(FK);
    if (cudaMemcpyAsync(w.data(), s->Wcm, FK * 4, cudaMemcpyDeviceToHost, q) != cudaSuccess ||
        cudaStreamSynchronize(q) != cudaSuccess)
        return fail(ONMF_ECUDA);
    for (float v : w)
        if (!(v >= 0.f) || std::isinf(v)) return fail(ONMF_EINVAL);
    *out = s;
    return ONMF_OK;
}

}  // extern "C"

// Run nmb minibatches (all of beta frames except the last, nb_last) read
// from device memory V (ldv), writing h to device H (ldh) when non-NULL.
static onmf_status run_minibatches(onmf_state *s, const float *V, long long ldv, int nmb,
                                   int nb_last, float *H, long long ldh,
                                   const float *H_in = nullptr, long long ldh_in = 0) {
    Range range_("online step launch");
    if (nmb <= 0) return ONMF_OK;
    const onmf_config &c = s->cfg;
    StepArgs a;
    a.s = s->s;
    a.eps = (float)c.eps;
    a.gamma = (float)c.h_exponent;
    a.n_in = c.n_inner;
    a.normalize = c.normalize;
    a.rho_on_new = c.rho_on_new;
    a.acc = c.accumulate;
    a.stats_ranges = c.stats_ranges;
    a.hpen = (float)c.h_penalty;
    a.hpen_a = (float)c.h_penalty_a;
    a.wpen = (float)c.w_penalty;
    a.V = V;
    a.ldv = ldv;
    a.nmb = nmb;
    a.beta = c.beta;
    a.nb_last = nb_last;
    a.rho_full = rho_of(c, c.beta);
    a.rho_last = rho_of(c, nb_last);
    a.H_out = H;
    a.ldh = ldh;
    a.H_in = H_in;
    a.ldh_in = ldh_in;
    a.Wcm = s->Wcm;
    a.Wrm = s->Wrm;
    a.Wimg = s->Wimg;
    a.Wrow = s->Wrow;
    a.Wn = s->Wn;
    a.A = s->A;
    a.B = s->B;
    a.loss_sum = s->loss_sum;
    a.swpart = s->swpart;
    a.Pg = s->Pg;
    a.Qg = s->Qg;
    a.Hg = s->Hg;
    a.part = s->part;
    a.betap = s->betap;
    a.loss_part = s->loss_part;
    a.bar = s->bar;
    a.err = s->err_d;
    a.stamps = s->stamps;
    if (s->prec == PREC_CL)
        CK(launch_online_cluster(a, s->C, s->grid, s->smem, s->stream));
    else
        CK(launch_online(a, s->prec, s->grid, s->smem, s->stream));
    s->t += (long long)(nmb - 1) * c.beta + nb_last;
    return mirror_err(s);
}

// Process the staging buffer as one minibatch of `staged` frames and hand
// the h of its frames to the recorded destinations.
static onmf_status run_staged(onmf_state *s) {
    const int n = s->staged;
    if (n == 0) return ONMF_OK;
    if (s->warm_staged) {
        // warm restarts: start points in Hin_stage, solved in place, then back
        // to the caller's rows named by stage_idx
        const int K = s->cfg.K;
        onmf_status st = run_minibatches(s, s->staging, s->cfg.F, 1, n, s->Hin_stage, K,
                                         s->Hin_stage, K);
        if (st != ONMF_OK) return st;
        CK(launch_scatter_rows(s->warm_H, s->warm_ldh, s->Hin_stage, K, s->stage_idx, 0, n, K,
                               s->stream));
        s->staged = 0;
        s->warm_staged = false;
        return ONMF_OK;
    }
    bool want_h = !s->segs.empty();
    onmf_status st = run_minibatches(s, s->staging, s->cfg.F, 1, n, want_h ? s->Hstage : nullptr,
                                     s->cfg.K);
    if (st != ONMF_OK) return st;
    for (const Segment &g : s->segs) {
        CK(cudaMemcpy2DAsync(g.dst, g.ldh * 4, s->Hstage + (size_t)g.off * s->cfg.K,
                             (size_t)s->cfg.K * 4, (size_t)s->cfg.K * 4, g.n, cudaMemcpyDefault,
                             s->stream));
    }
    s->segs.clear();
    s->staged = 0;
    return ONMF_OK;
}

// Frames already on the device (V) with optional H destination (host or device).
static onmf_status push_device(onmf_state *s, const float *V, long long ldv, long long n,
                               float *H, long long ldh) {
    const onmf_config &c = s->cfg;
    const bool hdev = H && is_device_ptr(H);
    long long i = 0;
    auto stage = [&](long long from, int count) -> onmf_status {
        CK(cudaMemcpy2DAsync(s->staging + (size_t)s->staged * c.F, (size_t)c.F * 4,
                             V + from * ldv, (size_t)ldv * 4, (size_t)c.F * 4, count,
                             cudaMemcpyDeviceToDevice, s->stream));
        if (H) s->segs.push_back(Segment{s->staged, count, H + from * ldh, ldh});
        s->staged += count;
        return ONMF_OK;
    };
    onmf_status st;
    if (s->staged > 0) {
        int take = (int)std::min<long long>(c.beta - s->staged, n);
        if ((st = stage(0, take)) != ONMF_OK) return st;
        i = take;
        if (s->staged == c.beta && (st = run_staged(s)) != ONMF_OK) return st;
    }
    long long nfull = (n - i) / c.beta;
    while (nfull > 0) {
        // bound a single launch to ~2^20 frames so one call never monopolizes the GPU
        int chunk = (int)std::min<long long>(nfull, std::max(1, (1 << 20) / c.beta));
        if (H && !hdev) {
            // device H for the chunk, then copy to the caller's host memory
            float *Hd = nullptr;
            size_t bytes = (size_t)chunk * c.beta * c.K * 4;
            CK(cudaMallocAsync((void **)&Hd, bytes, s->stream));
            st = run_minibatches(s, V + i * ldv, ldv, chunk, c.beta, Hd, c.K);
            if (st == ONMF_OK) {
                cudaError_t e = cudaMemcpy2DAsync(H + i * ldh, ldh * 4, Hd, (size_t)c.K * 4,
                                                  (size_t)c.K * 4, (size_t)chunk * c.beta,
                                                  cudaMemcpyDeviceToHost, s->stream);
                if (e != cudaSuccess) {
                    set_msg("H copy", e);
                    st = ONMF_ECUDA;
                }
            }
            cudaFreeAsync(Hd, s->stream);
            if (st != ONMF_OK) return st;
        } else {
            st = run_minibatches(s, V + i * ldv, ldv, chunk, c.beta, H ? H + i * ldh : nullptr, ldh);
            if (st != ONMF_OK) return st;
        }
        i += (long long)chunk * c.beta;
        nfull -= chunk;
    }
    if (i < n) {
        if ((st = stage(i, (int)(n - i))) != ONMF_OK) return st;
    }
    return ONMF_OK;
}

extern "C" {

onmf_status onmf_push_frames(onmf_state *s, const float *V, int64_t ldv, int64_t n, float *H_out,
                             int64_t ldh) {
    Range range_("onmf_push_frames");
    if (!s) return ONMF_EINVAL;
    onmf_status st = check_sticky(s);
    if (st != ONMF_OK) return st;
    if (n < 0 || (n > 0 && !V) || ldv < s->cfg.F || (H_out && ldh < s->cfg.K)) return ONMF_EINVAL;
    if (n == 0) return ONMF_OK;
    if (s->staged > 0 && s->warm_staged) {
        snprintf(g_msg, sizeof g_msg, "frames of a warm-restart pass are staged: flush first");
        return ONMF_ESTATE;
    }
    if (is_device_ptr(V)) return push_device(s, V, ldv, n, H_out, ldh);
    // host frames: copy through a double-buffered device ring, chunk by chunk,
    // on a copy stream so the copy of chunk i+1 overlaps the steps of chunk i
    const onmf_config &c = s->cfg;
    if (!s->vring[0]) {
        // slots of ~64k frames: small enough that the copy of a push's first
        // slot (the one part not hidden behind compute) stays short
        s->ring_frames = (long long)std::max(1, (1 << 16) / c.beta) * c.beta;
        CK(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking));
        for (int b = 0; b < 2; ++b) {
            CK(cudaMalloc((void **)&s->vring[b], (size_t)s->ring_frames * c.F * 4));
            CK(cudaEventCreateWithFlags(&s->ring_ev[b], cudaEventDisableTiming));
            CK(cudaEventCreateWithFlags(&s->ring_full[b], cudaEventDisableTiming));
            CK(cudaEventRecord(s->ring_ev[b], s->stream));
        }
    }
    // slot sizes ramp up within a push (8 minibatches, then x4 up to a full
    // slot): the first copy, the one nothing hides, stays short, and each
    // later copy is shorter than the step kernels of the slot before it
    // pinned host memory mapped into the device's address space is pulled by
    // a few CTAs on the SMs the step kernel leaves free; other host memory
    // goes through the copy engine
    const float *Vmap = nullptr;
    {
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, V) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer)
            Vmap = reinterpret_cast<const float *>(pa.devicePointer);
        else
            cudaGetLastError();
    }
    long long i = 0, cap = std::min(s->ring_frames, 8LL * c.beta);
    int b = 0;
    while (i < n) {
        long long m = std::min(cap, n - i);
        cap = std::min(s->ring_frames, 4 * cap);
        CK(cudaStreamWaitEvent(s->copy_stream, s->ring_ev[b], 0));  // slot consumed
        if (Vmap)
            CK(launch_pull_rows(s->vring[b], c.F, Vmap + i * ldv, ldv, m, s->copy_stream));
        else if (ldv == c.F)
            CK(cudaMemcpyAsync(s->vring[b], V + i * ldv, (size_t)m * c.F * 4,
                               cudaMemcpyHostToDevice, s->copy_stream));
        else
            CK(cudaMemcpy2DAsync(s->vring[b], (size_t)c.F * 4, V + i * ldv, (size_t)ldv * 4,
                                 (size_t)c.F * 4, m, cudaMemcpyHostToDevice, s->copy_stream));
        CK(cudaEventRecord(s->ring_full[b], s->copy_stream));
        CK(cudaStreamWaitEvent(s->stream, s->ring_full[b], 0));  // slot filled
        st = push_device(s, s->vring[b], c.F, m, H_out ? H_out + i * ldh : nullptr, ldh);
        if (st != ONMF_OK) return st;
        CK(cudaEventRecord(s->ring_ev[b], s->stream));
        i += m;
        b ^= 1;
    }
    return ONMF_OK;
}

onmf_status onmf_push_frames_warm(onmf_state *s, const float *V, int64_t ldv, int64_t n,
                                  const int64_t *order, float *H, int64_t ldh) {
    Range range_("onmf_push_frames_warm");
    if (!s) return ONMF_EINVAL;
    onmf_status st = check_sticky(s);
    if (st != ONMF_OK) return st;
    const onmf_config &c = s->cfg;
    if (n < 0 || ldv < c.F || ldh < c.K || (n > 0 && (!V || !H))) return ONMF_EINVAL;
    if (n == 0) return ONMF_OK;
    if (!is_device_ptr(V) || !is_device_ptr(H) || (order && !is_device_ptr(order))) {
        snprintf(g_msg, sizeof g_msg, "warm restarts take device V, H and order");
        return ONMF_EINVAL;
    }
    if (s->staged > 0 && (!s->warm_staged || s->warm_H != H || s->warm_ldh != ldh)) {
        snprintf(g_msg, sizeof g_msg, "other frames are staged: flush first");
        return ONMF_ESTATE;
    }
    cudaStream_t q = s->stream;
    const long long *idx = reinterpret_cast<const long long *>(order);
    if (!s->Hin_stage) {
        s->gcap = (long long)std::max(1, (1 << 18) / c.beta) * c.beta;
        CK(cudaMalloc((void **)&s->Hin_stage, (size_t)c.beta * c.K * 4));
        CK(cudaMalloc((void **)&s->stage_idx, (size_t)c.beta * 8));
        CK(cudaMalloc((void **)&s->gV, (size_t)s->gcap * c.F * 4));
        CK(cudaMalloc((void **)&s->gH, (size_t)s->gcap * c.K * 4));
    }
    s->warm_H = H;
    s->warm_ldh = ldh;
    // frames [i, i + m) of the pass -> staging rows [staged, staged + m)
    auto stage = [&](long long i, long long m) -> onmf_status {
        CK(launch_gather_rows(s->staging + (size_t)s->staged * c.F, c.F, V, ldv, idx, i, m, c.F, q));
        CK(launch_gather_rows(s->Hin_stage + (size_t)s->staged * c.K, c.K, H, ldh, idx, i, m, c.K, q));
        CK(launch_index_rows(s->stage_idx + s->staged, idx, i, m, q));
        s->staged += (int)m;
        s->warm_staged = true;
        return ONMF_OK;
    };
    long long i = 0;
    if (s->staged > 0) {
        const long long take = std::min<long long>(c.beta - s->staged, n);
        if ((st = stage(0, take)) != ONMF_OK) return st;
        i = take;
        if (s->staged == c.beta && (st = run_staged(s)) != ONMF_OK) return st;
    }
    long long nfull = (n - i) / c.beta;
    while (nfull > 0) {
        const long long chunk = std::min<long long>(nfull, s->gcap / c.beta);
        const long long m = chunk * c.beta;
        CK(launch_gather_rows(s->gV, c.F, V, ldv, idx, i, m, c.F, q));
        CK(launch_gather_rows(s->gH, c.K, H, ldh, idx, i, m, c.K, q));
        st = run_minibatches(s, s->gV, c.F, (int)chunk, c.beta, s->gH, c.K, s->gH, c.K);
        if (st != ONMF_OK) return st;
        CK(launch_scatter_rows(H, ldh, s->gH, c.K, idx, i, m, c.K, q));
        i += m;
        nfull -= chunk;
    }
    if (i < n && (st = stage(i, n - i)) != ONMF_OK) return st;
    return ONMF_OK;
}

onmf_status onmf_flush(onmf_state *s) {
    Range range_("onmf_flush");
    if (!s) return ONMF_EINVAL;
    onmf_status st = check_sticky(s);
    if (st != ONMF_OK) return st;
    return run_staged(s);
}

onmf_status onmf_synchronize(onmf_state *s) {
    if (!s) return ONMF_EINVAL;
    return sync_and_check(s);
}

onmf_status onmf_get_W(onmf_state *s, float *W_out, int32_t on_device) {
    (void)on_device;
    if (!s || !W_out) return ONMF_EINVAL;
    onmf_status st = sync_and_check(s);
    if (st != ONMF_OK && st != ONMF_ENUMERIC) return st;
    CK(cudaMemcpy(W_out, s->Wcm, (size_t)s->cfg.F * s->cfg.K * 4, cudaMemcpyDefault));
    return st;
}

onmf_status onmf_get_stats(onmf_state *s, double *A, double *B, int64_t *t, double *loss_sum) {
    if (!s) return ONMF_EINVAL;
    if (s->cfg.accumulate != ONMF_ACC_FP64 && ((A && is_device_ptr(A)) || (B && is_device_ptr(B))))
        return ONMF_EINVAL;  // the conversion to doubles runs on the host
    onmf_status st = sync_and_check(s);
    const size_t FK = (size_t)s->cfg.F * s->cfg.K;
    if (A) CK(cudaMemcpy(A, s->A, FK * 8, cudaMemcpyDefault));
    if (B) CK(cudaMemcpy(B, s->B, FK * 8, cudaMemcpyDefault));
    if (s->cfg.accumulate != ONMF_ACC_FP64) {
        // float pairs (hi, lo) in the same 8 bytes -> hi + lo as a double
        for (double *X : {A, B}) {
            if (!X) continue;
            for (size_t i = 0; i < FK; ++i) {
                float v[2];
                memcpy(v, X + i, 8);
                X[i] = (double)v[0] + (double)v[1];
            }
        }
    }
    if (loss_sum) CK(cudaMemcpy(loss_sum, s->loss_sum, 8, cudaMemcpyDefault));
    if (t) *t = s->t;
    return st;
}

onmf_status onmf_set_state(onmf_state *s, const float *W, const double *A, const double *B,
                           int64_t t, double loss_sum) {
    if (!s || !W || !A || !B || t < 0) return ONMF_EINVAL;
    if (is_device_ptr(W) || is_device_ptr(A) || is_device_ptr(B)) return ONMF_EINVAL;
    CK(cudaStreamSynchronize(s->stream));
    const size_t FK = (size_t)s->cfg.F * s->cfg.K;
    for (size_t i = 0; i < FK; ++i)
        if (!(W[i] >= 0.f) || std::isinf(W[i]) || !(A[i] >= 0.0) || !(B[i] >= 0.0))
            return ONMF_EINVAL;
    CK(cudaMemcpy(s->Wcm, W, FK * 4, cudaMemcpyDefault));
    if (s->cfg.accumulate == ONMF_ACC_FP64) {
        CK(cudaMemcpy(s->A, A, FK * 8, cudaMemcpyDefault));
        CK(cudaMemcpy(s->B, B, FK * 8, cudaMemcpyDefault));
    } else {
        // doubles -> (hi, lo) float pairs (lo = 0 for plain FP32)
        std::vector<float> pair(2 * FK);
        for (int which = 0; which < 2; ++which) {
            const double *X = which ? B : A;
            for (size_t i = 0; i < FK; ++i) {
                const float hi = (float)X[i];
                pair[2 * i] = hi;
                pair[2 * i + 1] =
                    s->cfg.accumulate == ONMF_ACC_FP32_COMP ? (float)(X[i] - (double)hi) : 0.f;
            }
            CK(cudaMemcpy(which ? s->B : s->A, pair.data(), FK * 8, cudaMemcpyHostToDevice));
        }
    }
    CK(cudaMemcpy(s->loss_sum, &loss_sum, 8, cudaMemcpyHostToDevice));
    CK(cudaMemset(s->err_d, 0, 16));
    *s->err_h = 0;
    s->sticky = ONMF_OK;
    s->staged = 0;
    s->segs.clear();
    s->t = t;
    onmf_status st = prepare_images(s);
    if (st != ONMF_OK) return st;
    return sync_and_check(s);
}

onmf_status onmf_project(onmf_state *s, const float *V, int64_t ldv, int64_t n, float *H_out,
                         int64_t ldh, int32_t n_inner, double *obj_sum) {
    Range range_("onmf_project");
    if (!s) return ONMF_EINVAL;
    onmf_status st = check_sticky(s);
    if (st != ONMF_OK) return st;
    const onmf_config &c = s->cfg;
    if (n < 0 || (n > 0 && !V) || ldv < c.F || (H_out && ldh < c.K)) return ONMF_EINVAL;
    if (obj_sum) *obj_sum = 0.0;
    if (n == 0) return ONMF_OK;
    const int nin = n_inner < 0 ? c.n_inner : n_inner;
    const bool vdev = is_device_ptr(V);
    const bool hdev = !H_out || is_device_ptr(H_out);
    const float *Vd = V;
    float *Vtmp = nullptr, *Htmp = nullptr;
    double *lp = nullptr;
    const int tile = s->prec == PREC_TC ? kTcTile : kTile;
    long long ntiles = (n + tile - 1) / tile;  // loss slots
    ClusterTiles ct;
    if (s->prec == PREC_CL) {
        ct = cluster_tiles(s->s, n);
        if (ct.C == 0) return ONMF_EINVAL;
        ntiles = ct.slots;
    }
    cudaStream_t q = s->stream;
    if (!vdev) {
        CK(cudaMallocAsync((void **)&Vtmp, (size_t)n * c.F * 4, q));
        CK(cudaMemcpy2DAsync(Vtmp, (size_t)c.F * 4, V, (size_t)ldv * 4, (size_t)c.F * 4, n,
                             cudaMemcpyHostToDevice, q));
        Vd = Vtmp;
    }
    float *Hd = H_out;
    long long ldhd = ldh;
    if (H_out && !hdev) {
        CK(cudaMallocAsync((void **)&Htmp, (size_t)n * c.K * 4, q));
        Hd = Htmp;
        ldhd = c.K;
    }
    if (obj_sum) CK(cudaMallocAsync((void **)&lp, (size_t)ntiles * 8, q));
    TileArgs a;
    memset(&a, 0, sizeof a);
    a.hpen = (float)c.h_penalty;  // a penalized model projects with its penalty
    a.hpen_a = (float)c.h_penalty_a;
    a.s = s->s;
    a.eps = (float)c.eps;
    a.gamma = (float)c.h_exponent;
    a.n_in = nin;
    a.V = Vd;
    a.ldv = vdev ? ldv : c.F;
    a.n = n;
    a.H_out = Hd;
    a.ldh = ldhd;
    a.final_pass = obj_sum ? 1 : 0;
    a.Wcm = s->Wcm;
    a.Wrm = s->Wrm;
    a.Wimg = s->Wimg;
    a.Wrow = s->Wrow;
    a.swpart = s->swpart;
    a.loss_part = lp;
    a.err = s->err_d;
    if (s->prec == PREC_CL) {
        CK(launch_tiles_cluster(a, ct.C, ct.grid, ct.smem, q));
    } else {
        const int grid = (int)std::min<long long>(ntiles, (long long)s->tile_grid * 2);
        CK(launch_tiles(a, s->prec, grid, s->tile_smem, q));
    }
    if (Htmp)
        CK(cudaMemcpy2DAsync(H_out, ldh * 4, Htmp, (size_t)c.K * 4, (size_t)c.K * 4, n,
                             cudaMemcpyDeviceToHost, q));
    if (obj_sum) {
        CK(launch_sum(lp, ntiles, s->tmp_sum, 0, q));
        CK(cudaMemcpyAsync(s->obj_h, s->tmp_sum, 8, cudaMemcpyDeviceToHost, q));
    }
    if (Vtmp) cudaFreeAsync(Vtmp, q);
    if (Htmp) cudaFreeAsync(Htmp, q);
    if (lp) cudaFreeAsync(lp, q);
    if ((st = mirror_err(s)) != ONMF_OK) return st;
    if (obj_sum || Htmp) {
        st = sync_and_check(s);
        if (obj_sum) *obj_sum = *s->obj_h;
        return st;
    }
    return ONMF_OK;
}

onmf_status nmf_batch_init_H(const float *V, int64_t ldv, const float *W, float *H, int32_t F,
                             int32_t K, int64_t N, double eps, void *stream) {
    if (!V || !W || !H || F < 1 || K < 1 || K > 256 || N < 0 || ldv < F) return ONMF_EINVAL;
    onmf_status st = ensure_configured();
    if (st != ONMF_OK) return st;
    if (N == 0) return ONMF_OK;
    cudaStream_t q = reinterpret_cast<cudaStream_t>(stream);
    Shape sh = make_shape(F, K);
    float *sw = nullptr;
    CK(cudaMallocAsync((void **)&sw, (size_t)K * 4, q));
    CK(launch_prepare(sh, W, nullptr, nullptr, sw, q));
    CK(launch_batch_h0(sh, V, ldv, N, (float)eps, sw, H, q));
    cudaFreeAsync(sw, q);
    return ONMF_OK;
}

}  // extern "C"

// Device scratch of batch IS-NMF cycles for one shape, sized for at most
// N_max frames and allocated once (nmf_batch_plan_create), so that the
// cycles themselves (nmf_batch_plan_step) allocate nothing.
struct nmf_batch_plan {
    int F = 0, K = 0, precision = 0, prec = 0, dev = 0, nsm = 1;
    long long Nmax = 0;
    Shape sh{};
    size_t elem = 4;
    long long betap_max = 0, slots_max = 0;
    static constexpr int kMaxChunks = 16;  // frame ranges of the statistics
    static constexpr int kObjCap = 256;    // objectives held on the device at once
    float *Wrm = nullptr, *swp = nullptr, *part = nullptr, *scale = nullptr;
    __nv_bfloat16 *Wimg = nullptr, *Wrow = nullptr;
    void *Pg = nullptr, *Qg = nullptr, *Hg = nullptr;
    double *lp = nullptr, *obj_d = nullptr;
    int *err = nullptr;
    std::vector<void *> owned;
    // stream-ordered plan (the one-shot nmf_batch_step): buffers come from
    // and go back to the stream's memory pool, in stream order
    bool ordered = false;
    cudaStream_t q = nullptr;
};

static void batch_plan_free(nmf_batch_plan *p) {
    if (!p) return;
    if (p->ordered) {
        for (void *x : p->owned) cudaFreeAsync(x, p->q);
    } else {
        int cur = 0;
        cudaGetDevice(&cur);
        cudaSetDevice(p->dev);
        cudaDeviceSynchronize();  // no kernel of the plan may still run
        for (void *x : p->owned) cudaFree(x);
        cudaSetDevice(cur);
    }
    delete p;
}

static onmf_status batch_plan_make(int32_t F, int32_t K, int64_t N_max, int32_t precision,
                                   bool ordered, cudaStream_t q, nmf_batch_plan **out);

extern "C" {

onmf_status nmf_batch_plan_create(int32_t F, int32_t K, int64_t N_max, int32_t precision,
                                  nmf_batch_plan **out) {
    return batch_plan_make(F, K, N_max, precision, false, nullptr, out);
}

}  // extern "C"

static onmf_status batch_plan_make(int32_t F, int32_t K, int64_t N_max, int32_t precision,
                                   bool ordered, cudaStream_t q, nmf_batch_plan **out) {
    if (!out) return ONMF_EINVAL;
    *out = nullptr;
    if (F < 1 || F > 8192 || K < 1 || K > 256 || N_max < 1 ||
        (precision != ONMF_FP32 && precision != ONMF_MIXED))
        return ONMF_EINVAL;
    if (precision == ONMF_MIXED && F > 1024) return ONMF_EINVAL;
    onmf_status st = ensure_configured();
    if (st != ONMF_OK) return st;
    nmf_batch_plan *p = new (std::nothrow) nmf_batch_plan;
    if (!p) return ONMF_ENOMEM;
    p->F = F;
    p->K = K;
    p->Nmax = N_max;
    p->ordered = ordered;
    p->q = q;
    p->precision = precision;
    p->sh = make_shape(F, K);
    p->prec = pick_prec(precision, p->sh);
    cudaGetDevice(&p->dev);
    cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->dev);
    p->elem = p->prec == PREC_FP32 ? 4 : 2;
    p->betap_max = (N_max + 15) / 16 * 16;
    // loss slots of every h-solve at any N <= N_max: one per 8 frames (mma,
    // FP32), per 16 (tcgen05), or C <= 8 per 32 (cluster), plus a margin for
    // the cluster size chosen at small N
    p->slots_max = (N_max + 3) / 4 + 8LL * kClMaxC + 64;
    const Shape &sh = p->sh;
    auto al = [&](void **x, size_t bytes) -> bool {
        if ((ordered ? cudaMallocAsync(x, bytes, q) : cudaMalloc(x, bytes)) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        p->owned.push_back(*x);
        return true;
    };
    bool ok = al((void **)&p->swp, (size_t)K * 4) && al((void **)&p->scale, (size_t)K * 4) &&
              al((void **)&p->part, (size_t)nmf_batch_plan::kMaxChunks * 2 * sh.Fp16 * sh.Kh * 4) &&
              al(&p->Pg, (size_t)p->betap_max * sh.Fp16 * p->elem) &&
              al(&p->Qg, (size_t)p->betap_max * sh.Fp16 * p->elem) &&
              al(&p->Hg, (size_t)p->betap_max * sh.Kh * p->elem) &&
              al((void **)&p->lp, (size_t)p->slots_max * 8) &&
              al((void **)&p->obj_d, (size_t)nmf_batch_plan::kObjCap * 8) &&
              al((void **)&p->err, 16);
    if (ok && p->prec == PREC_FP32) ok = al((void **)&p->Wrm, (size_t)F * K * 4);
    if (ok && p->prec != PREC_FP32 && p->prec != PREC_CL)
        ok = al((void **)&p->Wimg, (size_t)sh.Kp * sh.WLD * 2);
    if (ok && (p->prec == PREC_TC || p->prec == PREC_CL))
        ok = al((void **)&p->Wrow, (size_t)F * sh.Kp * 2);
    if (!ok) {
        batch_plan_free(p);
        snprintf(g_msg, sizeof g_msg, "batch plan allocation failed");
        return ONMF_ENOMEM;
    }
    // padding of the images and of H stays zero for the plan's life (the
    // kernels write only the live rows)
    cudaError_t e = cudaSuccess;
    if (p->Wimg) e = cudaMemsetAsync(p->Wimg, 0, (size_t)sh.Kp * sh.WLD * 2, q);
    if (p->Wrow && e == cudaSuccess) e = cudaMemsetAsync(p->Wrow, 0, (size_t)F * sh.Kp * 2, q);
    if (e == cudaSuccess) e = cudaMemsetAsync(p->Hg, 0, (size_t)p->betap_max * sh.Kh * p->elem, q);
    if (e == cudaSuccess && !ordered) e = cudaStreamSynchronize(q);
    if (e != cudaSuccess) {
        set_msg("batch plan init", e);
        batch_plan_free(p);
        return ONMF_ECUDA;
    }
    *out = p;
    return ONMF_OK;
}

extern "C" {

void nmf_batch_plan_destroy(nmf_batch_plan *p) { batch_plan_free(p); }

onmf_status nmf_batch_plan_step(nmf_batch_plan *p, const float *V, int64_t ldv, float *W, float *H,
                                int64_t N, double eps, double h_exponent, int32_t n_iter,
                                int32_t normalize, double *obj_out, void *stream) {
    Range range_("nmf_batch_plan_step");
    if (!p || !V || !W || !H || N < 1 || N > p->Nmax || ldv < p->F || n_iter < 0 ||
        !(eps >= 0.0) || !(h_exponent > 0.0))
        return ONMF_EINVAL;
    if (n_iter == 0) return ONMF_OK;
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != p->dev) return ONMF_EINVAL;
    cudaStream_t q = reinterpret_cast<cudaStream_t>(stream);
    const Shape &sh = p->sh;
    const int prec = p->prec, K = p->K, nsm = p->nsm;
    const long long betap = (N + 15) / 16 * 16;
    const int tile = prec == PREC_TC ? kTcTile : kTile;
    long long ntiles = (N + tile - 1) / tile;  // loss slots
    ClusterTiles ct;
    if (prec == PREC_CL) {
        ct = cluster_tiles(sh, N);
        if (ct.C == 0) return ONMF_EINVAL;
        ntiles = ct.slots;
    }
    if (ntiles > p->slots_max) return ONMF_EINVAL;
    const int units = (sh.Fp16 / 16) * (sh.Kh / 32);
    // frame ranges per output tile of the statistics: the count (<= 16, at
    // least 256 frames a range) whose units fill whole rounds of one CTA per
    // SM best; ties go to fewer ranges
    int nchunks = 1;
    {
        double best = -1.0;
        for (int c = 1; c <= nmf_batch_plan::kMaxChunks && (c == 1 || (long long)c * 256 <= N);
             ++c) {
            const long long U = (long long)units * c, rounds = (U + nsm - 1) / nsm;
            const double eff = (double)U / (double)(rounds * nsm);
            if (eff > best + 1e-9) {
                best = eff;
                nchunks = c;
            }
        }
    }
    cudaError_t e = cudaMemsetAsync(p->err, 0, 16, q);
    const size_t tsm = tc_min_smem(prec, tile_smem_bytes(sh, prec));
    const int tgrid = (int)std::min<long long>(ntiles, 2LL * nsm);
    auto run_tiles = [&](const TileArgs &x) {
        return prec == PREC_CL ? launch_tiles_cluster(x, ct.C, ct.grid, ct.smem, q)
                               : launch_tiles(x, prec, tgrid, tsm, q);
    };
    TileArgs a;
    memset(&a, 0, sizeof a);
    a.s = sh;
    a.eps = (float)eps;
    a.gamma = (float)h_exponent;
    a.V = V;
    a.ldv = ldv;
    a.n = N;
    a.Wcm = W;
    a.Wrm = p->Wrm;
    a.Wimg = p->Wimg;
    a.Wrow = p->Wrow;
    a.swpart = p->swp;
    a.err = p->err;
    a.betap = betap;
    constexpr int cap = nmf_batch_plan::kObjCap;
    std::vector<double> objs;
    if (obj_out) objs.resize((size_t)n_iter);
    // objective slot of the iterate after cycle i, and the copy-out of full
    // blocks of kObjCap objectives (the device holds one block at a time)
    auto obj_slot = [&](int i) { return p->obj_d + (i % cap); };
    auto flush_block = [&](int last) -> cudaError_t {
        const int first = last / cap * cap;
        return cudaMemcpyAsync(objs.data() + first, p->obj_d, (size_t)(last - first + 1) * 8,
                               cudaMemcpyDeviceToHost, q);
    };
    for (int it = 0; it < n_iter && e == cudaSuccess; ++it) {
        // one pass over the frames: the H step (its first X gives the
        // objective of the previous iterate), then X from the updated H and
        // the P, Q, H rows of the W step
        e = launch_prepare(sh, W, p->Wrm, p->Wimg, p->swp, q, p->Wrow);
        TileArgs h = a;
        h.n_in = 1;
        h.H_in = H;
        h.ldh_in = K;
        h.H_out = H;
        h.ldh = K;
        h.loss_first = (it > 0 && obj_out) ? 1 : 0;
        h.final_pass = 1;
        h.loss_part = h.loss_first ? p->lp : nullptr;
        h.Pg = p->Pg;
        h.Qg = p->Qg;
        h.Hg = p->Hg;
        if (e == cudaSuccess) e = run_tiles(h);
        if (e == cudaSuccess && h.loss_first) {
            e = launch_sum(p->lp, ntiles, obj_slot(it - 1), 0, q);
            if (e == cudaSuccess && (it - 1) % cap == cap - 1) e = flush_block(it - 1);
        }
        if (e == cudaSuccess)
            e = launch_batch_stats(sh, prec, p->Pg, p->Qg, p->Hg, betap, N, nchunks, p->part,
                                   std::min(units * nchunks, prec == PREC_FP32 ? 2 * nsm : nsm),
                                   q);
        if (e == cudaSuccess) e = launch_batch_wstep(sh, p->part, nchunks, W, q);
        if (e == cudaSuccess) e = launch_batch_normalize(sh, normalize, W, p->scale, p->err, q);
        if (e == cudaSuccess) e = launch_batch_scale_h(K, N, H, p->scale, q);
    }
    if (e == cudaSuccess && obj_out) {
        // objective of the final iterate
        e = launch_prepare(sh, W, p->Wrm, p->Wimg, p->swp, q, p->Wrow);
        TileArgs o = a;
        o.n_in = 0;
        o.H_in = H;
        o.ldh_in = K;
        o.final_pass = 1;
        o.loss_part = p->lp;
        if (e == cudaSuccess) e = run_tiles(o);
        if (e == cudaSuccess) e = launch_sum(p->lp, ntiles, obj_slot(n_iter - 1), 0, q);
        if (e == cudaSuccess) e = flush_block(n_iter - 1);
    }
    int errh = 0;
    if (e == cudaSuccess && obj_out) {
        e = cudaMemcpyAsync(&errh, p->err, 4, cudaMemcpyDeviceToHost, q);
        if (e == cudaSuccess) e = cudaStreamSynchronize(q);
        for (int i = 0; i < n_iter; ++i) obj_out[i] = objs[(size_t)i] / (double)N;
    }
    if (e != cudaSuccess) {
        set_msg("nmf_batch_plan_step", e);
        return ONMF_ECUDA;
    }
    return errh ? status_from_err(errh) : ONMF_OK;
}

onmf_status nmf_batch_step(const float *V, int64_t ldv, float *W, float *H, int32_t F, int32_t K,
                           int64_t N, double eps, double h_exponent, int32_t n_iter,
                           int32_t normalize, int32_t precision, double *obj_out, void *stream) {
    Range range_("nmf_batch_step");
    if (!V || !W || !H || F < 1 || F > 8192 || K < 1 || K > 256 || N < 1 || ldv < F ||
        n_iter < 0 || !(eps >= 0.0) || !(h_exponent > 0.0) ||
        (precision != ONMF_FP32 && precision != ONMF_MIXED))
        return ONMF_EINVAL;
    if (precision == ONMF_MIXED && F > 1024) return ONMF_EINVAL;
    if (n_iter == 0) {
        onmf_status st = ensure_configured();
        return st;
    }
    // a plan whose buffers come from the stream's pool and return to it in
    // stream order: the call stays asynchronous unless obj_out is given
    cudaStream_t q = reinterpret_cast<cudaStream_t>(stream);
    nmf_batch_plan *p = nullptr;
    onmf_status st = batch_plan_make(F, K, N, precision, true, q, &p);
    if (st != ONMF_OK) return st;
    st = nmf_batch_plan_step(p, V, ldv, W, H, N, eps, h_exponent, n_iter, normalize, obj_out,
                             stream);
    batch_plan_free(p);
    return st;
}

#ifdef ONMF_PHASE_STAMPS
// Phase-timing builds only (not part of the ABI in include/onmf.h): copies
// the clock64 stamps of the state's last launch (kStampMb x kStampCtas x
// kStampPts long longs, see onmf_kernels.cuh) to host memory and clears
// them; *grid receives the CTAs of the online launch. Synchronizes.
onmf_status onmf_phase_stamps(onmf_state *s, long long *host, int64_t n, int32_t *grid) {
    if (!s || !host || !s->stamps) return ONMF_EINVAL;
    const size_t sb = (size_t)kStampMb * kStampCtas * kStampPts * 8;
    if ((size_t)n * 8 < sb) return ONMF_EINVAL;
    if (cudaStreamSynchronize(s->stream) != cudaSuccess ||
        cudaMemcpy(host, s->stamps, sb, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemset(s->stamps, 0, sb) != cudaSuccess)
        return ONMF_ECUDA;
    if (grid) *grid = s->grid;
    return ONMF_OK;
}
#endif

}  // extern "C"
