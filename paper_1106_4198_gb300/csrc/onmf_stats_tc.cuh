// Statistics and dictionary step of Algorithm 1 (arXiv:1106.4198, Section
// 2.3, Eq. aux_fun) for the mixed-precision online step, on the tcgen05
// tensor cores:
//
//   phase 2   a_fk = W_fk^2 sum_j P_jf H_kj,  b_fk = sum_j Q_jf H_kj  as one
//             contraction per work unit (64 frequencies x one range of frames):
//             D[k, n] = sum_j H[k, j] [P | Q][j, n], M = 128 dictionary rows
//             (K <= 128, rows past K are zero), N = 128 (64 frequencies of P,
//             64 of Q), 16 frames per instruction. An instruction of this
//             shape costs about 200 clocks at any N up to 256 (measured on a
//             GB300), so N is taken wide; operands bulk-copied into
//             shared memory in core-matrix form (two stages, the copy of one
//             chunk overlapping the MMAs of the other), the FP32 accumulator
//             in tensor memory, read back with tcgen05.ld and written as one
//             partial sum per frame range;
//   phase 3   one CTA per dictionary column: the partial sums of the frame
//             ranges added in a fixed order, A <- rho A + a, B <- rho B + b,
//             W' = sqrt(A/B), the column sum s_k, W = W'/s_k, A /= s_k,
//             B *= s_k and the bf16 image row of W, all on values held in
//             registers (one pass over the column).
//
// Global layouts (written by hsolve_tile_mixed with TileJob::pq_core):
//   PQc  per (64-frequency tile t, 8-frame group g) a 2 KB block at
//        (t * G + g) * 2048: sixteen core matrices [P f0-7 | ... | P f56-63 |
//        Q f0-7 | ... | Q f56-63] of 8 rows (frames) x 16 bytes (8 bf16
//        frequencies); frequencies past Fp16 stay zero;
//   Hc   per group g a 2 KB block at g * 2048: 128 rows (k) x 16 bytes
//        (8 bf16 frames); rows k >= K stay zero;
//   part [split s][P or Q][k][Fp16] float partial sums (k < K).
// In shared memory a chunk's groups sit back to back in the same form, so the
// descriptors are: A (H, K-major) leading byte offset 2048 between 8-frame
// cores, stride byte offset 128 between 8-row cores; B ([P|Q], MN-major)
// leading byte offset 2048 between 8-frame cores, stride byte offset 128
// between 8-frequency cores.
//
// Included by onmf_step.cuh after the arithmetic of A and B (DF, ACC_*) and
// before the persistent online kernel that calls these functions.
#pragma once

#include "onmf_device.cuh"
#include "onmf_hsolve.cuh"
#include "onmf_kernels.cuh"
#include "onmf_tc.cuh"

namespace onmf {

constexpr int kStatsStageGroups = 16;                  // 8-frame groups per stage
constexpr size_t kStatsStageBytes = (size_t)kStatsStageGroups * (2048 + 2048);
constexpr size_t kStatsSmemBytes = 2 * kStatsStageBytes;  // two stages
constexpr uint32_t kStatsTmemCols = 128;

// mbarriers of the statistics and their phase parities: two stages, each
// with a bulk-copy barrier (ld) and an MMA-commit barrier (mma), tracked by
// the issuing thread 0, and one barrier per unit that every thread waits on
// (done).
struct StatsBars {
    uint64_t *ld[2], *mma[2], *done;
    unsigned pl[2], pm[2], pd;
};

// Frames of the CTA's next h-solve tile that warps 1-7 stage while a
// statistics unit's thread 0 waits for its range and issues the MMAs (their
// bulk copy already issued; the caller flips the copy's parity afterwards).
struct StageJob {
    const float *Vt;  // first frame of the tile; NULL: nothing to stage
    long long ldv;
    int nvalid;
    long long *hst;  // phase-timing stamps of the staging, or NULL
    float eps;
    uint64_t *vbar;
    unsigned vparity;
};

// One work unit of phase 2: 64-frequency tile t, frame range s (groups
// [s*gps, ...)), in chunks of at most kStatsStageGroups groups through two
// shared-memory stages: the bulk copy of chunk c+1 runs while the MMAs of
// chunk c do. tcol: the CTA's tensor-memory columns (128).
static __device__ void stats_unit_tc(int t, int s, int gps, int ng, long long G,
                                     const unsigned char *PQc, const unsigned char *Hc,
                                     float *part, int K, int Fp, unsigned char *smem,
                                     uint32_t tcol, StatsBars &sb, unsigned *rcnt, int *err,
                                     long long *ust, const Shape &sh, const StageJob job) {
    // ust: 8 clock64 slots of this unit (phase-timing builds), else NULL
#ifdef ONMF_PHASE_STAMPS
#define ONMF_USTAMP(i)                                     \
    do {                                                   \
        if (ust && threadIdx.x == 0) ust[(i)] = clock64(); \
    } while (0)
#else
#define ONMF_USTAMP(i) \
    do {               \
    } while (0)
#endif
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g0 = s * gps, g1 = min(ng, g0 + gps);
    const int nch = (g1 - g0 + kStatsStageGroups - 1) / kStatsStageGroups;
    auto H_of = [&](int st) { return smem + st * kStatsStageBytes; };
    auto PQ_of = [&](int st) { return smem + st * kStatsStageBytes + kStatsStageGroups * 2048; };
    __syncthreads();  // the previous user of this shared memory is done
    if (tid == 0) {
        // wait until every h-solve tile (8-frame group) of the range has
        // published its rows (bounded like every wait here)
        bool ok = true;
        {
            const unsigned need = (unsigned)(g1 - g0);
            const uint64_t t0 = global_ns();
            unsigned spins = 0;
            while (ld_acquire_gpu(rcnt + s) < need) {
                if ((++spins & 255u) == 0 && global_ns() - t0 > kWaitLimitNs) {
                    flag_error(err, ERR_TIMEOUT);
                    ok = false;
                    break;
                }
            }
        }
        ONMF_USTAMP(0);
#ifdef ONMF_PHASE_STAMPS
        if (ust) ust[-1] = (long long)global_ns();  // clock64 and ns at both ends
#endif
        auto issue = [&](int c) {
            const int st = c & 1;
            const int a = g0 + c * kStatsStageGroups, n = min(kStatsStageGroups, g1 - a);
            fence_proxy_async_shared();
            mbar_arrive_expect_tx(sb.ld[st], (unsigned)n * 4096u);
            bulk_g2s(H_of(st), Hc + (long long)a * 2048, (unsigned)n * 2048u, sb.ld[st]);
            bulk_g2s(PQ_of(st), PQc + ((long long)t * G + a) * 2048, (unsigned)n * 2048u,
                     sb.ld[st]);
        };
        if (ok) issue(0);
        if (ok && nch > 1) issue(1);
        const uint32_t id = tc_idesc(128, 128);
        for (int c = 0; c < nch && ok; ++c) {
            const int st = c & 1;
            const int a = g0 + c * kStatsStageGroups, n = min(kStatsStageGroups, g1 - a);
            if (n & 1) {  // the last 16-frame step has one group: the other reads zero
                uint4 *hz = reinterpret_cast<uint4 *>(H_of(st) + (size_t)n * 2048);
                uint4 *pz = reinterpret_cast<uint4 *>(PQ_of(st) + (size_t)n * 2048);
                for (int i = 0; i < 2048 / 16; ++i) {
                    hz[i] = make_uint4(0, 0, 0, 0);
                    pz[i] = make_uint4(0, 0, 0, 0);
                }
                fence_proxy_async_shared();
            }
            ok = mbar_wait_bounded(sb.ld[st], sb.pl[st], err);
            sb.pl[st] ^= 1u;
            if (c == 0) ONMF_USTAMP(1);
            if (!ok) break;
            tc_fence_after();
            for (int ks = 0; ks < (n + 1) / 2; ++ks)
                tc_mma_smem_a(tcol, tc_desc(H_of(st) + (size_t)ks * 4096, 2048, 128),
                              tc_desc(PQ_of(st) + (size_t)ks * 4096, 2048, 128), id,
                              (c > 0 || ks > 0) ? 1u : 0u);
            if (c + 2 < nch) {
                // the stage is refilled once its MMAs have read it
                tc_commit(sb.mma[st]);
                ok = mbar_wait_bounded(sb.mma[st], sb.pm[st], err);
                sb.pm[st] ^= 1u;
                if (ok) issue(c + 2);
            }
        }
        ONMF_USTAMP(2);
        tc_commit(sb.done);  // arrives once every MMA above is done
    } else if (job.Vt && tid >= 32) {
        // the frame buffers lie past the stages and the accumulator tile
        TileJob tn;
        tn.Vt = job.Vt;
        tn.ldv = job.ldv;
        tn.nvalid = job.nvalid;
        tn.v_staged = 1;
        tn.hst = job.hst;
        stage_frames_core(sh, job.eps, tn, smem, job.vbar, job.vparity, err);
    }
    const bool ok = mbar_wait_bounded(sb.done, sb.pd, err);
    sb.pd ^= 1u;
    ONMF_USTAMP(3);
    tc_fence_after();
    // accumulators: warp w reads lanes 32 (w % 4) .. (k) and the 64 columns of
    // P (w < 4) or Q (w >= 4) into a shared-memory tile [P|Q][k][64 (+4 pad)]
    // (both stages are free once the MMAs are done), so that the partial
    // sums leave in whole rows; the tile's frequencies past Fp are not stored
    constexpr int kRow = 68;  // floats per row: 16-byte chunks of 8 rows hit 8 bank groups
    float *T = reinterpret_cast<float *>(smem);
    const int q = warp & 3, which = warp >> 2;
    const int k = 32 * q + lane;
    const int nf = min(64, Fp - 64 * t);  // a multiple of 16
    const uint32_t ta = tcol + ((uint32_t)(32 * q) << 16) + 64u * which;
    float *trow = T + ((size_t)which * 128 + k) * kRow;
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
        uint32_t r0[8], r1[8];
        tmem_ld8_async(ta + c0, r0);
        tmem_ld8_async(ta + c0 + 8, r1);
        tmem_wait_ld(r0);
        tmem_wait_ld(r1);
        float4 *d4 = reinterpret_cast<float4 *>(trow + c0);
        d4[0] = make_float4(__uint_as_float(r0[0]), __uint_as_float(r0[1]),
                            __uint_as_float(r0[2]), __uint_as_float(r0[3]));
        d4[1] = make_float4(__uint_as_float(r0[4]), __uint_as_float(r0[5]),
                            __uint_as_float(r0[6]), __uint_as_float(r0[7]));
        d4[2] = make_float4(__uint_as_float(r1[0]), __uint_as_float(r1[1]),
                            __uint_as_float(r1[2]), __uint_as_float(r1[3]));
        d4[3] = make_float4(__uint_as_float(r1[4]), __uint_as_float(r1[5]),
                            __uint_as_float(r1[6]), __uint_as_float(r1[7]));
    }
    __syncthreads();
    ONMF_USTAMP(4);
    if (ok) {
        // half a warp per row (16 float4 = 64 frequencies), rows (which, k)
        const int c4 = lane & 15;
        if (4 * c4 < nf)
            for (int row = 2 * warp + (lane >> 4); row < 2 * K; row += 2 * kWarps) {
                const int w2 = row >= K ? 1 : 0, k2 = row - w2 * K;
                const float4 v =
                    *reinterpret_cast<const float4 *>(T + ((size_t)w2 * 128 + k2) * kRow + 4 * c4);
                *reinterpret_cast<float4 *>(part + (((long long)s * 2 + w2) * K + k2) * Fp + 64 * t +
                                            4 * c4) = v;
            }
    }
    ONMF_USTAMP(5);
    tc_fence_before();
    __syncthreads();  // every read of the accumulator precedes the next MMA
    ONMF_USTAMP(6);
#ifdef ONMF_PHASE_STAMPS
    if (ust && threadIdx.x == 0) ust[7] = (long long)global_ns();
#endif
#undef ONMF_USTAMP
}

// ---- phase 3: one dictionary column per CTA (strided), every value of the
// column in registers (F <= kColRows).
constexpr int kColPer = 4;                    // frequencies per thread
constexpr int kColRows = kColPer * kThreads;  // 1024 >= F on the mixed path

// A <- rho A + a (or A + rho a with rho_on_new) for one entry in the state's
// arithmetic; `raw` is the stored 8 bytes (a double, a float, or a float
// pair) and is replaced by the new stored form; returns the new value as a
// float, the operand of W' = sqrt(A/B). rhof = (float)rho, converted once by
// the caller. The arithmetic is a template parameter: the FP32 modes then
// hold no FP64 instruction at all (the FP64 rate of this GPU is a small
// fraction of its FP32 rate, so even per-thread conversions and divisions in
// double show up in the column pass, and so do FP64 instructions of an
// untaken mode that the compiler predicates instead of branching around).
template <int ACCM>
__device__ __forceinline__ float ab_accumulate(double rho, float rhof, int rho_on_new, float inc,
                                               double &raw) {
    if constexpr (ACCM == ACC_FP64) {
        const double v = rho_on_new ? fma(rho, (double)inc, raw) : fma(rho, raw, (double)inc);
        raw = v;
        return (float)v;
    }
    DF x;
    memcpy(&x, &raw, 8);
    if constexpr (ACCM == ACC_FP32) {
        const float v = rho_on_new ? __fmaf_rn(rhof, inc, x.hi) : __fmaf_rn(rhof, x.hi, inc);
        x = {v, 0.f};
    } else {
        x = rho_on_new ? df_add_mul(x, rhof, inc) : df_mul_add(x, rhof, inc);
    }
    memcpy(&raw, &x, 8);
    return x.hi;
}

// The rescale of one stored entry: A / s (div) or B * s; FP64 sums use the
// double reciprocal invd = 1/s and the double sd = s; the compensated pairs
// multiply by the reciprocal pair (ih, il) of s.
template <int ACCM>
__device__ __forceinline__ double ab_rescale(double raw, float sum, double invd,
                                             double sd, float ih, float il, bool div) {
    if constexpr (ACCM == ACC_FP64) return div ? raw * invd : raw * sd;
    DF x;
    memcpy(&x, &raw, 8);
    if constexpr (ACCM == ACC_FP32)
        x = {div ? __fdiv_rn(x.hi, sum) : __fmul_rn(x.hi, sum), 0.f};
    else
        x = div ? df_mul_pair(x, ih, il) : df_mul_add(x, sum, 0.f);
    double r;
    memcpy(&r, &x, 8);
    return r;
}

// W, A, B of one column, in registers (thread tid: rows tid + u * kThreads).
struct ColVals {
    float w[kColPer];
    double A[kColPer], B[kColPer];
};

// Load W, A, B of column k. They depend on no other CTA's work of this
// minibatch, so a CTA loads its first column between its arrival at the grid
// barrier before phase 3 and its wait there.
__device__ __forceinline__ void col_load(const StepArgs &a, int k, ColVals &v) {
    const int F = a.s.F;
#pragma unroll
    for (int u = 0; u < kColPer; ++u) {
        const int f = threadIdx.x + u * kThreads;
        if (f < F && k < a.s.K) {
            const long long i = f + (long long)k * F;
            v.w[u] = a.Wcm[i];
            v.A[u] = a.A[i];
            v.B[u] = a.B[i];
        } else {
            v.w[u] = 0.f;
            v.A[u] = v.B[u] = 0.0;
        }
    }
}

// WPEN: the dictionary penalty mu * sum W, W' = sqrt(A/(B + mu)).
// pre: W, A, B of the CTA's first column (k = first), loaded by col_load.
// ACCM: the arithmetic of A and B (ACC_*), fixed at compile time.
template <bool WPEN, int ACCM>
static __device__ void column_step(const StepArgs &a, int S, double rho, float *red8, int first,
                                   int stride, const ColVals &pre, long long *cst = nullptr) {
    // cst: 5 clock64 slots of the first column (phase-timing builds), else NULL
#ifdef ONMF_PHASE_STAMPS
#define ONMF_CSTAMP(i)                                                  \
    do {                                                                \
        if (cst && k == first && threadIdx.x == 0) cst[(i)] = clock64(); \
    } while (0)
#else
#define ONMF_CSTAMP(i) \
    do {               \
    } while (0)
#endif
    const Shape &s = a.s;
    const int F = s.F, K = s.K, Fp = s.Fp16;
    const int tid = threadIdx.x;
    const float rhof = (float)rho;
    const long long step = (long long)K * Fp;  // floats between P (or Q) partials of two ranges
    for (int k = first; k < K; k += stride) {
        ColVals v;
        ONMF_CSTAMP(0);
        if (k == first)
            v = pre;
        else
            col_load(a, k, v);
        // the frame ranges' partial sums, added in range order (eight ranges'
        // loads in flight at a time; a missing range adds +0)
        float ph[kColPer], qh[kColPer];
#pragma unroll
        for (int u = 0; u < kColPer; ++u) ph[u] = qh[u] = 0.f;
        const float *pp = a.part + (long long)k * Fp + tid;
        for (int r0 = 0; r0 < S; r0 += 8) {
            float pv[8][kColPer], qv[8][kColPer];
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int u = 0; u < kColPer; ++u) {
                    const int f = tid + u * kThreads;
                    const bool ok = r0 + j < S && f < F;
                    const float *q = pp + (2LL * (r0 + j)) * step + u * kThreads;
                    pv[j][u] = ok ? __ldcg(q) : 0.f;
                    qv[j][u] = ok ? __ldcg(q + step) : 0.f;
                }
#pragma unroll
            for (int j = 0; j < 8; ++j)
#pragma unroll
                for (int u = 0; u < kColPer; ++u) {
                    ph[u] += pv[j][u];
                    qh[u] += qv[j][u];
                }
        }
        ONMF_CSTAMP(1);
        float wn[kColPer];
        float part_sum = 0.f;
#pragma unroll
        for (int u = 0; u < kColPer; ++u) {
            const int f = tid + u * kThreads;
            wn[u] = 0.f;
            if (f < F) {
                const float w = v.w[u];
                const float An =
                    ab_accumulate<ACCM>(rho, rhof, a.rho_on_new, ph[u] * w * w, v.A[u]);
                const float Bn = ab_accumulate<ACCM>(rho, rhof, a.rho_on_new, qh[u], v.B[u]);
                const float Bd = WPEN ? Bn + a.wpen : Bn;
                wn[u] = (Bd > 0.f) ? sqrtf(__fdiv_rn(An, Bd)) : w;
                part_sum += wn[u];
            }
        }
        ONMF_CSTAMP(2);
        const float sum = block_sum_f(part_sum, red8);
        ONMF_CSTAMP(3);
        const bool sc = a.normalize && sum > 0.f;
        const float inv = sc ? __frcp_rn(sum) : 1.f;
        const float invl = sc ? __fmul_rn(__fmaf_rn(-inv, sum, 1.f), inv) : 0.f;
        // the double forms of 1/s and s only where A, B are doubles; one
        // thread divides (a double division per thread costs a visible part
        // of the pass at this GPU's FP64 rate) and shares the quotient
        const bool d64 = sc && ACCM == ACC_FP64;
        double invd = 1.0;
        if (d64) {
            __shared__ double s_invd;
            if (tid == 0) s_invd = 1.0 / (double)sum;
            __syncthreads();
            invd = s_invd;
        }
        const double sd = d64 ? (double)sum : 1.0;
        bool bad = false;
#pragma unroll
        for (int u = 0; u < kColPer; ++u) {
            const int f = tid + u * kThreads;
            if (f < F) {
                const long long i = f + (long long)k * F;
                const float wv = wn[u] * inv;
                bad |= !isfinite(wv);
                a.Wcm[i] = wv;
                a.A[i] = sc ? ab_rescale<ACCM>(v.A[u], sum, invd, sd, inv, invl, true) : v.A[u];
                a.B[i] = sc ? ab_rescale<ACCM>(v.B[u], sum, invd, sd, inv, invl, false) : v.B[u];
                a.Wimg[(long long)k * s.WLD + f] = __float2bfloat16_rn(wv);
            }
        }
        if (bad) flag_error(a.err, ERR_NUMERIC);
        if (tid == 0) a.swpart[k] = sc ? sum * inv : sum;
        ONMF_CSTAMP(4);
    }
#undef ONMF_CSTAMP
}

}  // namespace onmf
