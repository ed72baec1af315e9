// The per-tile h-solve of Algorithm 1 (arXiv:1106.4198, Section 2.3):
// for kTile frames at a time and W fixed, run n_in majorization-minimization
// steps  x = eps + W h,  p = y/x^2,  q = 1/x,  h <- h * ((W^T p)/(W^T q))^gamma
// from the fresh-restart point h0 = sum_f y_f / sum_{f,k} W_fk (or from a
// given H for the batch H step), then one more x = eps + W h for the
// statistics and the loss. Two implementations share the interface:
//   hsolve_tile_fp32   FP32 SIMT (the plain form),
//   hsolve_tile_mixed  BF16 tensor cores (mma.sync m16n8k16, FP32 accumulate)
//                      with W^T resident in shared memory (bulk-copied) and
//                      the frame tile staged by a bulk copy; the ratios y/x^2
//                      and 1/x stay FP32 and are rounded to BF16 only as the
//                      operand of the W^T product.
#pragma once

#include "onmf_device.cuh"
#include "onmf_kernels.cuh"

namespace onmf {

// Everything one tile needs besides the shape and W.
struct TileJob {
    const float *Vt;  // first frame of the tile
    long long ldv;
    int nvalid;        // frames of the tile that exist (1..kTile)
    long long j0;      // index of the tile's first frame in Pg/Qg/Hg/H_out/H_in
    const float *H_in; // warm start (K x frames, ld ldh_in) or NULL
    long long ldh_in;
    float *H_out;      // K x frames (ldh) or NULL
    long long ldh;
    int n_in;
    int loss_first;  // loss of the first X only (a final pass then adds none)
    int final_pass;
    double *loss_slot;  // receives the tile's loss (or NULL)
    void *Pg, *Qg, *Hg;
    long long betap;
    // mixed path only: the tile's frames are already on their way into
    // shared memory (issued by the previous tile of this CTA), and the
    // frames of the CTA's next tile to issue once this one no longer needs
    // the buffer (NULL: none)
    int v_staged = 0;
    const float *Vnext = nullptr;
    int nvalid_next = 0;
    // FP32 path: the h penalty lambda * log(a + sum_k h_k) (lambda = 0: none)
    float hpen = 0.f, hpen_a = 1.f;
    // mixed path: write P, Q and H in the core-matrix layout of the tcgen05
    // statistics (stats_tc.cuh) instead of frame rows
    int pq_core = 0;
    // phase-timing builds: clock64 slots of this tile's steps, or NULL (0-2
    // staging, 3-12 after each inner iteration, 13 final ratios, 14 outputs,
    // 15 after step A of the tenth iteration; 18-21 the steps of the frame
    // staging when it runs in the barrier window)
    long long *hst = nullptr;
    // mma path: frames already staged and converted (mixed_stage_frames)
    int v_ready = 0;
};

#ifdef ONMF_PHASE_STAMPS
#define ONMF_HSTAMP(t, i)                                      \
    do {                                                       \
        if ((t).hst && threadIdx.x == 0) (t).hst[(i)] = clock64(); \
    } while (0)
#else
#define ONMF_HSTAMP(t, i) \
    do {                  \
    } while (0)
#endif

// Whether a tile's frames go to shared memory by one bulk copy: contiguous
// rows (ld = F), a 16-byte aligned start and a multiple of 16 bytes.
__host__ __device__ inline bool tile_bulk(const float *Vt, long long ldv, int F, int nvalid) {
    const size_t bytes = (size_t)nvalid * F * 4;
    return ldv == F && (reinterpret_cast<uintptr_t>(Vt) & 15) == 0 && bytes % 16 == 0;
}

// Compile-time tags, so that a hot loop is instantiated once per value of a
// run-time switch that is uniform over the CTA (the exponent mode, whether
// the loss is wanted) instead of carrying the rarely taken path (powf, logf)
// as predicated code in every iteration.
template <int V> struct IntTag {
    static constexpr int value = V;
};

// Exponent mode of the h update: 0 for gamma = 1/2, 1 for gamma = 1, 2 else.
__host__ __device__ inline int gamma_mode(float gamma) {
    return gamma == 0.5f ? 0 : (gamma == 1.0f ? 1 : 2);
}

// h * r^gamma for the exponent mode GM.
template <int GM>
__device__ __forceinline__ float scale_pow(float h, float r, float gamma) {
    if (GM == 0) return h * sqrtf(r);
    if (GM == 1) return h * r;
    return h * powf(r, gamma);
}

// Run f(IntTag<mode>{}) for the exponent mode of gamma.
template <class Fn>
__device__ __forceinline__ void with_gamma_mode(float gamma, Fn &&f) {
    const int gm = gamma_mode(gamma);
    if (gm == 0)
        f(IntTag<0>{});
    else if (gm == 1)
        f(IntTag<1>{});
    else
        f(IntTag<2>{});
}

__device__ __forceinline__ bool bad_value(float v) { return !(v >= 0.f) || isinf(v); }

// Sum of the K column sums of the normalized W (the denominator of h0), by
// warp 1: thread 0 may be busy issuing a bulk copy (and its proxy fence)
// just before, and the two round trips to L2 then overlap.
__device__ __forceinline__ float sum_w(const float *swpart, int K, float *s_tmp) {
    if (threadIdx.x >= 32 && threadIdx.x < 64) {
        const int l = threadIdx.x - 32;
        float a = 0.f;
        for (int k = l; k < K; k += 32) a += swpart[k];
        a = warp_sum(a);
        if (l == 0) *s_tmp = a;
    }
    __syncthreads();
    float r = *s_tmp;
    return r;
}

// ------------------------------------------------------------------ FP32

// Shared memory of the FP32 h-solve, in floats.
__host__ __device__ inline size_t hsolve_fp32_smem_bytes(const Shape &s) {
    size_t fl = 3ull * s.F * kTile + (size_t)s.Kh * kTile + (size_t)kWarps * 128 * 16 + 64;
    return fl * sizeof(float);
}

static __device__ void hsolve_tile_fp32(const Shape &s, float eps, float gamma, const float *Wcm,
                                 const float *Wrm, float sw, const TileJob &t,
                                 unsigned char *smem, int *err) {
    const int F = s.F, K = s.K, Kh = s.Kh;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float *y_s = reinterpret_cast<float *>(smem);  // [F][8]
    float *p_s = y_s + (size_t)F * kTile;          // [F][8]
    float *q_s = p_s + (size_t)F * kTile;          // [F][8]
    float *h_s = q_s + (size_t)F * kTile;          // [Kh][8]
    float *red = h_s + (size_t)Kh * kTile;         // [8][128][16]
    float *misc = red + kWarps * 128 * 16;         // sy[8], lw[8], hsum[8]
    float *sy = misc, *lw = misc + 8;

    // frame tile -> y = eps + v (y = 1 in frames past the end of the data)
    for (int i = tid; i < kTile * F; i += kThreads) {
        int j = i / F, f = i - j * F;
        float y = 1.f;
        if (j < t.nvalid) {
            float v = __ldg(t.Vt + (long long)j * t.ldv + f);
            if (bad_value(v)) flag_error(err, ERR_INPUT);
            y = eps + v;
        }
        y_s[f * kTile + j] = y;
    }
    __syncthreads();
    if (t.H_in) {
        for (int i = tid; i < Kh * kTile; i += kThreads) {
            int k = i / kTile, j = i % kTile;
            h_s[i] = (k < K && j < t.nvalid) ? t.H_in[(t.j0 + j) * t.ldh_in + k] : 0.f;
        }
    } else {
        // h0 = sum_f y_f / sum W for every k (fresh restart)
        float a = 0.f;
        for (int f = lane; f < F; f += 32) a += y_s[f * kTile + warp];
        a = warp_sum(a);
        if (lane == 0) sy[warp] = a;
        __syncthreads();
        for (int i = tid; i < Kh * kTile; i += kThreads) {
            int k = i / kTile, j = i % kTile;
            h_s[i] = (k < K) ? sy[j] / sw : 0.f;
        }
    }
    __syncthreads();

    float lacc = 0.f;
    const int mainF = (F / kThreads) * kThreads;
    for (int it = 0;; ++it) {
        const bool last = (it == t.n_in);
        if (last && !t.final_pass) break;
        const bool want_loss =
            t.loss_slot && ((last && t.final_pass && !t.loss_first) || (it == 0 && t.loss_first));
        auto finish_row_t = [&](auto loss_tag, int f, const float (&acc)[kTile]) {
            constexpr bool LOSS = decltype(loss_tag)::value != 0;
            float4 ya = *reinterpret_cast<const float4 *>(y_s + f * kTile);
            float4 yb = *reinterpret_cast<const float4 *>(y_s + f * kTile + 4);
            float ys[kTile] = {ya.x, ya.y, ya.z, ya.w, yb.x, yb.y, yb.z, yb.w};
            float pv[kTile], qv[kTile];
#pragma unroll
            for (int j = 0; j < kTile; ++j) {
                float x = eps + acc[j];
                float q = __frcp_rn(x);
                qv[j] = q;
                pv[j] = ys[j] * q * q;
                if (LOSS && j < t.nvalid) {
                    float r = ys[j] * q;
                    lacc += (r - 1.f) - logf(r);
                }
            }
            *reinterpret_cast<float4 *>(p_s + f * kTile) = make_float4(pv[0], pv[1], pv[2], pv[3]);
            *reinterpret_cast<float4 *>(p_s + f * kTile + 4) = make_float4(pv[4], pv[5], pv[6], pv[7]);
            *reinterpret_cast<float4 *>(q_s + f * kTile) = make_float4(qv[0], qv[1], qv[2], qv[3]);
            *reinterpret_cast<float4 *>(q_s + f * kTile + 4) = make_float4(qv[4], qv[5], qv[6], qv[7]);
        };
        // the loss is a separate instantiation (no logf where it is not needed)
        auto finish_row = [&](int f, const float (&acc)[kTile]) {
            if (want_loss)
                finish_row_t(IntTag<1>{}, f, acc);
            else
                finish_row_t(IntTag<0>{}, f, acc);
        };
        // x = eps + W h: rows [0, mainF) one per thread, the rest split over k by warps
        for (int f = tid; f < mainF; f += kThreads) {
            float acc[kTile];
#pragma unroll
            for (int j = 0; j < kTile; ++j) acc[j] = 0.f;
            const float *wc = Wcm + f;
#pragma unroll 4
            for (int k = 0; k < K; ++k) {
                float w = wc[(long long)k * F];
                float4 ha = *reinterpret_cast<const float4 *>(h_s + k * kTile);
                float4 hb = *reinterpret_cast<const float4 *>(h_s + k * kTile + 4);
                acc[0] = fmaf(w, ha.x, acc[0]);
                acc[1] = fmaf(w, ha.y, acc[1]);
                acc[2] = fmaf(w, ha.z, acc[2]);
                acc[3] = fmaf(w, ha.w, acc[3]);
                acc[4] = fmaf(w, hb.x, acc[4]);
                acc[5] = fmaf(w, hb.y, acc[5]);
                acc[6] = fmaf(w, hb.z, acc[6]);
                acc[7] = fmaf(w, hb.w, acc[7]);
            }
            finish_row(f, acc);
        }
        for (int f = mainF + warp; f < F; f += kWarps) {
            float acc[kTile];
#pragma unroll
            for (int j = 0; j < kTile; ++j) acc[j] = 0.f;
            for (int k = lane; k < K; k += 32) {
                float w = Wcm[f + (long long)k * F];
#pragma unroll
                for (int j = 0; j < kTile; ++j) acc[j] = fmaf(w, h_s[k * kTile + j], acc[j]);
            }
#pragma unroll
            for (int j = 0; j < kTile; ++j) acc[j] = warp_sum(acc[j]);
            if (lane == 0) finish_row(f, acc);
        }
        __syncthreads();
        if (last) break;

        // the h penalty's tangent needs each frame's sum_k h_k before this
        // step (warp j: frame j); read after the barrier below
        float *hsum = misc + 16;
        if (t.hpen > 0.f && warp < kTile) {
            float a = 0.f;
            for (int k = lane; k < K; k += 32) a += h_s[k * kTile + warp];
            a = warp_sum(a);
            if (lane == 0) hsum[warp] = a;
        }
        // W^T p and W^T q: lanes take k, warps take contiguous row ranges
        const int fper = (F + kWarps - 1) / kWarps;
        const int f_lo = warp * fper, f_hi = min(F, f_lo + fper);
        for (int k0 = 0; k0 < K; k0 += 128) {
            float nm[4][kTile], dn[4][kTile];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < kTile; ++j) nm[i][j] = dn[i][j] = 0.f;
            for (int f = f_lo; f < f_hi; ++f) {
                float4 pa = *reinterpret_cast<const float4 *>(p_s + f * kTile);
                float4 pb = *reinterpret_cast<const float4 *>(p_s + f * kTile + 4);
                float4 qa = *reinterpret_cast<const float4 *>(q_s + f * kTile);
                float4 qb = *reinterpret_cast<const float4 *>(q_s + f * kTile + 4);
                float pv[kTile] = {pa.x, pa.y, pa.z, pa.w, pb.x, pb.y, pb.z, pb.w};
                float qv[kTile] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    int k = k0 + lane + 32 * i;
                    float w = (k < K) ? Wrm[(long long)f * K + k] : 0.f;
#pragma unroll
                    for (int j = 0; j < kTile; ++j) {
                        nm[i][j] = fmaf(w, pv[j], nm[i][j]);
                        dn[i][j] = fmaf(w, qv[j], dn[i][j]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                float *r = red + ((size_t)warp * 128 + lane + 32 * i) * 16;
#pragma unroll
                for (int j = 0; j < kTile; j += 4) {
                    *reinterpret_cast<float4 *>(r + j) =
                        make_float4(nm[i][j], nm[i][j + 1], nm[i][j + 2], nm[i][j + 3]);
                    *reinterpret_cast<float4 *>(r + 8 + j) =
                        make_float4(dn[i][j], dn[i][j + 1], dn[i][j + 2], dn[i][j + 3]);
                }
            }
            __syncthreads();
            with_gamma_mode(gamma, [&](auto gm) {
                constexpr int GM = decltype(gm)::value;
                for (int e = tid; e < 128 * kTile; e += kThreads) {
                    int kk = e / kTile, j = e % kTile, k = k0 + kk;
                    if (k < K) {
                        float num = 0.f, den = 0.f;
#pragma unroll
                        for (int w = 0; w < kWarps; ++w) {
                            num += red[((size_t)w * 128 + kk) * 16 + j];
                            den += red[((size_t)w * 128 + kk) * 16 + 8 + j];
                        }
                        float h = h_s[k * kTile + j];
                        // lambda psi'(s~) joins the denominator (Section 2.2, "Extensions")
                        if (t.hpen > 0.f) den += __fdiv_rn(t.hpen, t.hpen_a + hsum[j]);
                        if (den > 0.f) h = scale_pow<GM>(h, __fdiv_rn(num, den), gamma);
                        h_s[k * kTile + j] = h;
                    }
                }
            });
            __syncthreads();
        }
    }

    // outputs
    if (t.final_pass) {
        float *Pg = reinterpret_cast<float *>(t.Pg);
        float *Qg = reinterpret_cast<float *>(t.Qg);
        float *Hg = reinterpret_cast<float *>(t.Hg);
        const int Fp = s.Fp16;
        if (Pg) {
            for (int i = tid; i < kTile * Fp; i += kThreads) {
                int j = i / Fp, f = i - j * Fp;
                bool ok = j < t.nvalid && f < F;
                long long o = (t.j0 + j) * Fp + f;
                Pg[o] = ok ? p_s[f * kTile + j] : 0.f;
                Qg[o] = ok ? q_s[f * kTile + j] : 0.f;
            }
            for (int i = tid; i < kTile * Kh; i += kThreads) {
                int j = i / Kh, k = i - j * Kh;
                Hg[(t.j0 + j) * Kh + k] = (j < t.nvalid) ? h_s[k * kTile + j] : 0.f;
            }
        }
    }
    if (t.H_out) {
        for (int i = tid; i < t.nvalid * K; i += kThreads) {
            int j = i / K, k = i - j * K;
            t.H_out[(t.j0 + j) * t.ldh + k] = h_s[k * kTile + j];
        }
    }
    if (t.loss_slot) {
        float l = warp_sum(lacc);
        if (lane == 0) lw[warp] = l;
        __syncthreads();
        if (tid == 0) {
            double d = 0.0;
            for (int w = 0; w < kWarps; ++w) d += (double)lw[w];
            *t.loss_slot = d;
        }
    }
    __syncthreads();
}

// ----------------------------------------------------------------- MIXED

constexpr int kMtMax = 5;    // m16 row tiles of x = eps + W h per warp per pass

struct MixedLayout {
    size_t w, pq, h, yraw, yt, misc, total;  // byte offsets
    int HLD;
};

__host__ __device__ inline MixedLayout mixed_layout(const Shape &s) {
    MixedLayout L;
    L.HLD = s.Kp + 8;
    size_t o = 0;
    L.w = o;
    o += (size_t)s.Kp * s.WLD * 2;
    o = (o + 127) / 128 * 128;
    L.pq = o;
    o += (size_t)16 * s.WLD * 2;
    o = (o + 127) / 128 * 128;
    L.h = o;
    o += (size_t)kTile * L.HLD * 2;
    o = (o + 127) / 128 * 128;
    L.yraw = o;
    o += (size_t)kTile * s.F * 4;
    o = (o + 127) / 128 * 128;
    L.yt = o;
    o += (size_t)s.Fp16 * kTile * 4;
    o = (o + 127) / 128 * 128;
    L.misc = o;
    // frame sums [8], loss per warp [8], the penalty's per-warp h sums
    // [2][8][8] from float 32, the staging's per-warp frame sums [8][8] from
    // float 160
    o += 1024;
    L.total = o;
    return L;
}

// Issue the bulk copy of W^T (bf16 image) into shared memory; the h-solve
// waits for it (mbarrier `bar`) after issuing its own frame-tile copy.
// issue_wimg_nosync: the same without the CTA barrier before it, for a caller
// whose threads are already past their last use of that shared memory.
__device__ __forceinline__ void issue_wimg_nosync(const Shape &s, const __nv_bfloat16 *Wimg,
                                                  unsigned char *smem, uint64_t *bar) {
    const MixedLayout L = mixed_layout(s);
    const unsigned bytes = (unsigned)((size_t)s.Kp * s.WLD * 2);
    if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.global;\n" ::: "memory");
        fence_proxy_async_shared();
        mbar_arrive_expect_tx(bar, bytes);
        bulk_g2s(smem + L.w, Wimg, bytes, bar);
    }
}

__device__ __forceinline__ void issue_wimg(const Shape &s, const __nv_bfloat16 *Wimg,
                                           unsigned char *smem, uint64_t *bar) {
    __syncthreads();
    issue_wimg_nosync(s, Wimg, smem, bar);
}

// The frames of a tile of the mma h-solve into shared memory (bulk copy
// when contiguous and aligned, possibly issued already: TileJob::v_staged),
// then each frame's sum_f y_f (the start point's numerator), the input check
// and the f-major copy y = eps + v. It needs V alone, so the online step runs
// it for a CTA's next tile while the CTA waits at a grid barrier, or inside
// its statistics unit while warp 0 issues the MMAs (TileJob::v_ready then
// skips it in the h-solve).
//
// stage_frames_core is the staging proper, run by warps 1-7 alone (named
// barrier 1): the frame sums come from one fixed partition of those 224
// threads wherever the staging runs, so every caller forms the same bits.
// The caller keeps the bulk-copy parity (it flips it in every thread).
constexpr int kStageThreads = kThreads - 32;

__device__ __forceinline__ void stage_bar() {
    asm volatile("bar.sync 1, %0;" ::"n"(kStageThreads) : "memory");
}

#ifdef ONMF_PHASE_STAMPS
#define ONMF_SSTAMP(t, i)                                       \
    do {                                                        \
        if ((t).hst && threadIdx.x == 32) (t).hst[(i)] = clock64(); \
    } while (0)
#else
#define ONMF_SSTAMP(t, i) \
    do {                  \
    } while (0)
#endif

static __device__ __forceinline__ void stage_frames_core(const Shape &s, float eps, const TileJob &t,
                                         unsigned char *smem, uint64_t *vbar, unsigned vparity,
                                         int *err) {
    const int F = s.F, Fp = s.Fp16;
    const MixedLayout L = mixed_layout(s);
    const int u = threadIdx.x - 32, lane = threadIdx.x & 31, w = (threadIdx.x >> 5) - 1;
    float *y_raw = reinterpret_cast<float *>(smem + L.yraw);
    float *yT = reinterpret_cast<float *>(smem + L.yt);
    float *sy = reinterpret_cast<float *>(smem + L.misc);
    ONMF_SSTAMP(t, 18);
    // ---- frame tile -> shared memory (bulk copy when contiguous and aligned;
    //      possibly issued already)
    if (tile_bulk(t.Vt, t.ldv, F, t.nvalid)) {
        if (u == 0 && !t.v_staged) {
            fence_proxy_async_shared();
            mbar_arrive_expect_tx(vbar, (unsigned)((size_t)t.nvalid * F * 4));
            bulk_g2s(y_raw, t.Vt, (unsigned)((size_t)t.nvalid * F * 4), vbar);
        }
        mbar_wait_bounded(vbar, vparity, err);
    } else {
        for (int i = u; i < t.nvalid * F; i += kStageThreads) {
            int j = i / F, f = i - j * F;
            y_raw[i] = __ldg(t.Vt + (long long)j * t.ldv + f);
        }
        stage_bar();
    }
    ONMF_SSTAMP(t, 19);
    // f-major copy y = eps + v, input check and frame sums in one pass:
    // thread u always has frame j = u & 7 (entry f * 8 + j of yT), so it adds
    // its own entries of frame j; the threads of each frame then combine
    // theirs (lanes j, j+8, j+16, j+24, then the seven warps in order)
    {
        constexpr int U = 6;  // independent loads in flight per thread
        constexpr int FS = kStageThreads / 8;  // frequencies per pass
        const int j = u & 7;
        const bool jv = j < t.nvalid;
        const float *src = y_raw + j * F;
        float a = 0.f;
        // input check on the bits: with -0 taken as +0, a frame value is
        // valid (finite, not negative, not NaN) iff its bits are below those
        // of +inf, so the largest bits seen decide (one max per entry)
        unsigned mx = 0u;
        for (int f0 = u >> 3; f0 < Fp; f0 += FS * U) {
            float v[U];
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int f = f0 + FS * q;
                v[q] = (jv && f < F) ? src[f] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < U; ++q) {
                const int f = f0 + FS * q;
                if (f < Fp) {
                    const bool in = jv && f < F;
                    const unsigned b = __float_as_uint(v[q]);
                    mx = max(mx, b == 0x80000000u ? 0u : b);
                    const float y = eps + v[q];
                    if (in) a += y;
                    yT[f * 8 + j] = in ? y : 1.f;
                }
            }
        }
        if (mx >= 0x7f800000u) flag_error(err, ERR_INPUT);
        a += __shfl_xor_sync(0xffffffffu, a, 8);
        a += __shfl_xor_sync(0xffffffffu, a, 16);
        if (lane < 8) sy[160 + w * 8 + lane] = a;
        stage_bar();
        ONMF_SSTAMP(t, 20);
        if (u < 8) {
            float sum = 0.f;
            for (int q = 0; q < kStageThreads / 32; ++q) sum += sy[160 + q * 8 + u];
            // placeholder frames (j >= nvalid): y = 1 at every f
            sy[u] = (u < t.nvalid) ? sum : (float)F;
        }
    }
    ONMF_SSTAMP(t, 21);
}

// The staging by the whole CTA (warp 0 idles): every thread flips the
// parity of the frame copy.
static __device__ void mixed_stage_frames(const Shape &s, float eps, const TileJob &t,
                                          unsigned char *smem, uint64_t *vbar,
                                          unsigned &vparity, int *err) {
    __syncthreads();  // the previous user of the frame buffers is done
    if (threadIdx.x >= 32) stage_frames_core(s, eps, t, smem, vbar, vparity, err);
    if (tile_bulk(t.Vt, t.ldv, s.F, t.nvalid)) vparity ^= 1u;
    __syncthreads();
}

// Pending bulk copy of W^T that a tile must wait for before its first use.
struct WStage {
    uint64_t *bar;
    unsigned *parity;
    bool pending;
};

// The tensor-core h-solve of one tile (KS = Kp/16 k16 steps; KS = 0 takes
// the count from the shape at run time, one instantiation for every
// dictionary size, as the one-launch serving kernel uses). W^T is in
// shared memory as bf16 (row k = column k of W). Per iteration:
//   step A  x = eps + W h: each warp owns m16 row tiles (interleaved
//           accumulator chains over the KS k-steps), then p = y/x^2 and
//           q = 1/x in FP32, rounded to bf16 and stored transposed with
//           stmatrix as the 16 x Fp operand [P | Q]^T;
//   step B  [W^T p | W^T q]: warp w < KS owns k in [16w, 16w+16) and all of
//           F (4 interleaved chains per n-tile); the accumulator fragment
//           holds (W^T p)_k and (W^T q)_k of the same (frame, k), so the h
//           update happens in registers (FP32 master h).
template <int KS, bool PEN = false>
static __device__ void hsolve_tile_mixed(const Shape &s, float eps, float gamma, float sw,
                                  const TileJob &t, unsigned char *smem, WStage &ws,
                                  uint64_t *vbar, unsigned &vparity, int *err) {
    const int F = s.F, K = s.K, WLD = s.WLD, Fp = s.Fp16;
    const MixedLayout L = mixed_layout(s);
    const int HLD = L.HLD;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, tq = lane & 3;
    const int mi = lane >> 3, r8 = lane & 7;
    __nv_bfloat16 *W_s = reinterpret_cast<__nv_bfloat16 *>(smem + L.w);
    __nv_bfloat16 *PQ_s = reinterpret_cast<__nv_bfloat16 *>(smem + L.pq);
    __nv_bfloat16 *H_s = reinterpret_cast<__nv_bfloat16 *>(smem + L.h);
    float *y_raw = reinterpret_cast<float *>(smem + L.yraw);  // [8][F] raw v (bulk target)
    float *yT = reinterpret_cast<float *>(smem + L.yt);       // [Fp][8] y = eps + v
    float *misc = reinterpret_cast<float *>(smem + L.misc);
    float *sy = misc, *lw = misc + 8;
    // PEN: per-warp sums over the warp's k of each frame's h, double-buffered
    // by iteration parity ([2][kWarps][kTile]); the h penalty's tangent needs
    // sum_k h_k of the h before each update (Section 2.2, "Extensions")
    float *hpart = misc + 32;
    const int FT = Fp / 16;
    const int NKS = KS > 0 ? KS : s.Kp / 16;  // k16 steps


    ONMF_HSTAMP(t, 0);
    if (!t.v_ready) mixed_stage_frames(s, eps, t, smem, vbar, vparity, err);
    ONMF_HSTAMP(t, 1);
    // the raw frames are no longer needed: the next tile's go into the buffer
    if (t.Vnext && tid == 0) {
        const unsigned nb = (unsigned)((size_t)t.nvalid_next * F * 4);
        fence_proxy_async_shared();
        mbar_arrive_expect_tx(vbar, nb);
        bulk_g2s(y_raw, t.Vnext, nb, vbar);
    }

    // ---- h in registers: warp w < KS owns k = 16w + {2tq, 2tq+1, 8+2tq, 9+2tq}, frame g
    float hr[4] = {0.f, 0.f, 0.f, 0.f};
    const bool hown = warp < NKS;
    // PEN: this warp's share of frame g's sum_k h_k (the four lanes of frame
    // g add their entries; the tq = 0 lane writes)
    auto put_hsum = [&](int buf) {
        float v = (hr[0] + hr[1]) + (hr[2] + hr[3]);
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        if (tq == 0) hpart[(buf * kWarps + warp) * kTile + g] = v;
    };
    if (hown) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int k = 16 * warp + 2 * tq + (e & 1) + 8 * (e >> 1);
            float h = 0.f;
            if (k < K) {
                if (t.H_in)
                    h = (g < t.nvalid) ? t.H_in[(t.j0 + g) * t.ldh_in + k] : 0.f;
                else
                    h = sy[g] / sw;
            }
            hr[e] = h;
        }
        *reinterpret_cast<uint32_t *>(H_s + g * HLD + 16 * warp + 2 * tq) = pack_bf16(hr[0], hr[1]);
        *reinterpret_cast<uint32_t *>(H_s + g * HLD + 16 * warp + 8 + 2 * tq) =
            pack_bf16(hr[2], hr[3]);
        if constexpr (PEN) put_hsum(0);
    }
    // W^T is first read by step A: its bulk copy (issued before the frame
    // tile) overlaps the frame sums and the start point above
    if (ws.pending) {
        mbar_wait_bounded(ws.bar, *ws.parity, err);
        *ws.parity ^= 1u;
        ws.pending = false;
    }
    __syncthreads();
    ONMF_HSTAMP(t, 2);

    // the loss sum_{valid f, j} r - 1 - log r (r = y/x: d_IS of Section 2,
    // summed over frames as in Eq. 1): the r - 1 (lr1) and the base-2 logs
    // (ll2, the hardware's approximate log2, absolute error about 2^-22 near
    // r = 1 and a few ulp elsewhere; zero, infinite and NaN r give the same
    // +inf or NaN loss as an exact log) are added per thread and combined
    // once, log r = log2 r * log 2
    float lacc = 0.f, lr1 = 0.f, ll2 = 0.f;
    // whether this thread's two frames (2 tq, 2 tq + 1) are real frames, in
    // registers for the loss (the tile descriptor may live in local memory)
    const bool fv0 = 2 * tq < t.nvalid, fv1 = 2 * tq + 1 < t.nvalid;
    for (int it = 0;; ++it) {
        const bool last = (it == t.n_in);
        if (last && !t.final_pass) break;
        const bool want_loss =
            t.loss_slot && ((last && t.final_pass && !t.loss_first) || (it == 0 && t.loss_first));
        // ---- step A: x = eps + W h (groups of kMtMax m16 tiles per warp;
        //      every ldmatrix of a k-step is issued before its MMAs)
        for (int mg = warp; mg < FT; mg += kWarps * kMtMax) {
            float d[kMtMax][4];
#pragma unroll
            for (int i = 0; i < kMtMax; ++i)
#pragma unroll
                for (int e = 0; e < 4; ++e) d[i][e] = eps;
            const __nv_bfloat16 *wa = W_s + (r8 + 8 * (mi >> 1)) * WLD + 8 * (mi & 1) + 16 * mg;
#pragma unroll
            for (int ks = 0; ks < NKS; ++ks) {
                const uint32_t b0 =
                    *reinterpret_cast<const uint32_t *>(H_s + g * HLD + 16 * ks + 2 * tq);
                const uint32_t b1 =
                    *reinterpret_cast<const uint32_t *>(H_s + g * HLD + 16 * ks + 8 + 2 * tq);
                uint32_t a[kMtMax][4];
#pragma unroll
                for (int i = 0; i < kMtMax; ++i)
                    if (mg + kWarps * i < FT)
                        ldmatrix_x4_trans(a[i], wa + 16 * ks * WLD + 16 * kWarps * i);
#pragma unroll
                for (int i = 0; i < kMtMax; ++i)
                    if (mg + kWarps * i < FT) mma_bf16_16816(d[i], a[i], b0, b1);
            }
            // p = y/x^2, q = 1/x (FP32), bf16, stored transposed: PQ_s[j][f],
            // PQ_s[8+j][f]; the loss is a separate instantiation (no logf in
            // the iterations that do not need it)
            auto ratios = [&](auto loss_tag) {
                constexpr bool LOSS = decltype(loss_tag)::value != 0;
#pragma unroll
                for (int i = 0; i < kMtMax; ++i) {
                    const int mt = mg + kWarps * i;
                    if (mt < FT) {
                        const int f0 = 16 * mt;
                        const float2 ya = *reinterpret_cast<const float2 *>(yT + (f0 + g) * 8 + 2 * tq);
                        const float2 yb =
                            *reinterpret_cast<const float2 *>(yT + (f0 + g + 8) * 8 + 2 * tq);
                        const float yv[4] = {ya.x, ya.y, yb.x, yb.y};
                        float pv[4], qv[4];
#pragma unroll
                        for (int e = 0; e < 4; ++e) {
                            const int f = f0 + g + 8 * (e >> 1);
                            const float q = rcp_approx(d[i][e]);
                            const float p = yv[e] * q * q;
                            const bool ok = f < F;
                            pv[e] = ok ? p : 0.f;
                            qv[e] = ok ? q : 0.f;
                            if (LOSS && ok && ((e & 1) ? fv1 : fv0)) {
                                const float r = yv[e] * q;
                                lr1 += r - 1.f;
                                ll2 += __log2f(r);
                            }
                        }
                        stmatrix_x4_trans(PQ_s + (r8 + 8 * (mi >> 1)) * WLD + f0 + 8 * (mi & 1),
                                          pack_bf16(pv[0], pv[1]), pack_bf16(pv[2], pv[3]),
                                          pack_bf16(qv[0], qv[1]), pack_bf16(qv[2], qv[3]));
                    }
                }
            };
            if (want_loss)
                ratios(IntTag<1>{});
            else
                ratios(IntTag<0>{});
        }
        __syncthreads();
        if (last) {
            ONMF_HSTAMP(t, 13);
            break;
        }
        if (it == 9) ONMF_HSTAMP(t, 15);

        // ---- step B: [W^T p | W^T q] and the h update
        if (hown) {
            float c0[4][4], c1[4][4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int e = 0; e < 4; ++e) c0[u][e] = c1[u][e] = 0.f;
            const __nv_bfloat16 *arow = PQ_s + (r8 + 8 * (mi & 1)) * WLD + 8 * (mi >> 1);
            const __nv_bfloat16 *brow = W_s + (16 * warp + r8 + 8 * (mi >> 1)) * WLD + 8 * (mi & 1);
            // a single k16 step left over by the groups of four (F = 16n + 1,
            // e.g. 513: the step of f = 512 alone) goes first, into the first
            // accumulator pair, rather than as a ninth group of its own at the end
            const int FTg = (FT & 3) == 1 ? FT - 1 : FT;
            if (FTg != FT) {
                uint32_t a[4], b[4];
                ldmatrix_x4(a, arow + 16 * FTg);
                ldmatrix_x4(b, brow + 16 * FTg);
                mma_bf16_16816(c0[0], a, b[0], b[1]);
                mma_bf16_16816(c1[0], a, b[2], b[3]);
            }
            for (int fs = 0; fs < FTg; fs += 4) {
                uint32_t a[4][4], b[4][4];
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (fs + u < FTg) {
                        ldmatrix_x4(a[u], arow + 16 * (fs + u));
                        ldmatrix_x4(b[u], brow + 16 * (fs + u));
                    }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (fs + u < FTg) {
                        mma_bf16_16816(c0[u], a[u], b[u][0], b[u][1]);
                        mma_bf16_16816(c1[u], a[u], b[u][2], b[u][3]);
                    }
            }
            float n0[4], n1[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                n0[e] = (c0[0][e] + c0[1][e]) + (c0[2][e] + c0[3][e]);
                n1[e] = (c1[0][e] + c1[1][e]) + (c1[2][e] + c1[3][e]);
            }
            // n[0..1] = (W^T p)[k, k+1] of frame g, n[2..3] = (W^T q)[k, k+1]
            const float num[4] = {n0[0], n0[1], n1[0], n1[1]};
            float den[4] = {n0[2], n0[3], n1[2], n1[3]};
            if constexpr (PEN) {
                // lambda psi'(s~) joins the denominator, s~ = sum_k h_k of frame g
                float hs = 0.f;
                for (int w = 0; w < NKS; ++w) hs += hpart[((it & 1) * kWarps + w) * kTile + g];
                const float pen = t.hpen > 0.f ? __fdiv_rn(t.hpen, t.hpen_a + hs) : 0.f;
#pragma unroll
                for (int e = 0; e < 4; ++e) den[e] += pen;
            }
            with_gamma_mode(gamma, [&](auto gm) {
                constexpr int GM = decltype(gm)::value;
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (den[e] > 0.f) hr[e] = scale_pow<GM>(hr[e], __fdividef(num[e], den[e]), gamma);
            });
            *reinterpret_cast<uint32_t *>(H_s + g * HLD + 16 * warp + 2 * tq) =
                pack_bf16(hr[0], hr[1]);
            *reinterpret_cast<uint32_t *>(H_s + g * HLD + 16 * warp + 8 + 2 * tq) =
                pack_bf16(hr[2], hr[3]);
            if constexpr (PEN) put_hsum((it + 1) & 1);
        }
        __syncthreads();
        if (it < 10) ONMF_HSTAMP(t, 3 + it);
    }

    // ---- outputs
    if (t.final_pass && t.Pg && t.pq_core) {
        // core-matrix layout (8 frames x 16 bytes per core): the frames of
        // this tile are frame group gi; 64-frequency tile ft of P and Q is one
        // 2 KB block [P f 0-7 | ... | P f 56-63 | Q f 0-7 | ... | Q f 56-63],
        // row j = frame; H is one 2 KB block per group, row k = 8 frames of h_k
        unsigned char *PQc = reinterpret_cast<unsigned char *>(t.Pg);
        unsigned char *Hc = reinterpret_cast<unsigned char *>(t.Hg);
        const long long G = t.betap / 8, gi = t.j0 / 8;
        const int cpr = Fp / 8;  // 16-byte chunks per row = core matrices per P or Q
        // eight lanes per core matrix (lane & 7 = frame j): a warp writes four
        // whole 128-byte core matrices, 512 contiguous bytes within a block
        const int j = tid & 7;
        for (int cc = tid >> 3; cc < 2 * cpr; cc += kThreads / 8) {
            const int which = cc >= cpr ? 1 : 0, c = cc - which * cpr;
            uint4 v = make_uint4(0, 0, 0, 0);
            if (j < t.nvalid)
                v = *reinterpret_cast<const uint4 *>(PQ_s + (which * 8 + j) * WLD + 8 * c);
            *reinterpret_cast<uint4 *>(PQc + ((long long)(c >> 3) * G + gi) * 2048 +
                                       (which * 8 + (c & 7)) * 128 + j * 16) = v;
        }
        for (int k = tid; k < NKS * 16; k += kThreads) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = 2 * e;
                const float a = (j < t.nvalid) ? __bfloat162float(H_s[j * HLD + k]) : 0.f;
                const float b = (j + 1 < t.nvalid) ? __bfloat162float(H_s[(j + 1) * HLD + k]) : 0.f;
                w[e] = pack_bf16(a, b);
            }
            *reinterpret_cast<uint4 *>(Hc + gi * 2048 + (long long)k * 16) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    } else if (t.final_pass && t.Pg) {
        __nv_bfloat16 *Pg = reinterpret_cast<__nv_bfloat16 *>(t.Pg);
        __nv_bfloat16 *Qg = reinterpret_cast<__nv_bfloat16 *>(t.Qg);
        __nv_bfloat16 *Hg = reinterpret_cast<__nv_bfloat16 *>(t.Hg);
        const int cpr = Fp / 8;  // 16-byte chunks per row
        // warp per (p|q, frame) row, lanes over the chunks (no index division)
        for (int row = warp; row < 2 * kTile; row += kWarps) {
            const int which = row >> 3, j = row & 7;
            __nv_bfloat16 *dst = (which ? Qg : Pg) + (t.j0 + j) * Fp;
            for (int c = lane; c < cpr; c += 32) {
                uint4 v = make_uint4(0, 0, 0, 0);
                if (j < t.nvalid) v = *reinterpret_cast<const uint4 *>(PQ_s + row * WLD + 8 * c);
                *reinterpret_cast<uint4 *>(dst + 8 * c) = v;
            }
        }
        for (int k = tid; k < NKS * 16; k += kThreads) {
            uint32_t w[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int j = 2 * e;
                __nv_bfloat16 a = (j < t.nvalid) ? H_s[j * HLD + k] : __float2bfloat16_rn(0.f);
                __nv_bfloat16 b = (j + 1 < t.nvalid) ? H_s[(j + 1) * HLD + k] : __float2bfloat16_rn(0.f);
                __nv_bfloat162 pr;
                pr.x = a;
                pr.y = b;
                w[e] = *reinterpret_cast<uint32_t *>(&pr);
            }
            *reinterpret_cast<uint4 *>(Hg + (long long)k * t.betap + t.j0) =
                make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
    ONMF_HSTAMP(t, 14);
    if (t.H_out && hown && g < t.nvalid) {
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int k = 16 * warp + 2 * tq + (e & 1) + 8 * (e >> 1);
            if (k < K) t.H_out[(t.j0 + g) * t.ldh + k] = hr[e];
        }
    }
    if (t.loss_slot) {
        lacc += lr1 - ll2 * 0.6931471805599453f;
        float l = warp_sum(lacc);
        if (lane == 0) lw[warp] = l;
        __syncthreads();
        if (tid == 0) {  // FP32 like the terms (no FP64 on the critical path)
            float sum = 0.f;
            for (int w = 0; w < kWarps; ++w) sum += lw[w];
            *t.loss_slot = (double)sum;
        }
    }
    __syncthreads();
}

}  // namespace onmf
