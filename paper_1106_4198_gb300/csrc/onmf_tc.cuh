// tcgen05 (5th-generation tensor core) form of the h-solve of Algorithm 1
// (arXiv:1106.4198, Section 2.3): 16 frames per CTA, W held in tensor memory
// (TMEM) as the A operand of both products so that the inner loop reads only
// the small h and [p|q] operands from shared memory.
//
//   step A   X = W H        M = 128 frequency rows per tile, N = 16 frames,
//                           K = 16 dictionary columns per instruction
//   step B   [Nm|Dn] = W^T [P|Q]   M = 128 dictionary columns (K <= 128),
//                           N = 32 (16 frames of p, 16 of q), K = 16 rows of F
//
// One thread issues the MMAs (tcgen05.mma, cta_group::1, kind::f16, bf16
// operands, FP32 accumulators in TMEM) and commits them to an mbarrier; all
// 8 warps read the accumulators back with tcgen05.ld (warp w sees TMEM lanes
// 32*(w%4)..+31) for the FP32 ratios and the h update. Rows of F beyond the
// last full 128-row tile (F = 2^n + 1 leaves one) are handled on the CUDA
// cores. Layouts (no swizzle, 8 x 16-byte core matrices; leading byte offset
// = stride between core matrices along K, stride byte offset = along M/N):
//   H   (B of step A, MN-major)  core (k/8, n/8) at (k/8)*256 + (n/8)*128
//   P|Q (B of step B, MN-major)  core (f/8, n/8) at (f/8)*512 + (n/8)*128,
//                                n = frame (p) or 16 + frame (q)
//   W   (A of step A from shared memory, K-major) core (m/8, k/8) at
//                                (m/8)*(256*KS) + (k/8)*128
//   TMEM: [0, 64) accumulators; [64, 64 + Ftc/2) W^T (lane = k, column pairs
//   along f); then W tiles for step A (lane = f - 128 t, pairs along k).
#pragma once

#include "onmf_device.cuh"
#include "onmf_hsolve.cuh"
#include "onmf_kernels.cuh"

namespace onmf {

constexpr int kTcMaxTail = 32;     // rows of F handled on CUDA cores
constexpr uint32_t kTmemCols = 512;

struct TcLayout {
    int Ftc, ntail, nmt, KS, tiles_tm;  // tensor-core rows, tail rows, M tiles, k16 steps
    uint32_t col_D, col_WT, col_WA;     // TMEM columns
    size_t h, pq, wa, yraw, yt, tw, tx, misc, total;  // shared-memory byte offsets
};

__host__ __device__ inline TcLayout tc_layout(const Shape &s) {
    TcLayout L;
    L.Ftc = s.F / 128 * 128;
    L.ntail = s.F - L.Ftc;
    L.nmt = L.Ftc / 128;
    L.KS = s.Kp / 16;
    L.col_D = 0;
    L.col_WT = 64;
    L.col_WA = 64 + L.Ftc / 2;
    const int free_cols = (int)kTmemCols - 64 - L.Ftc / 2;
    int fit = free_cols > 0 ? free_cols / (8 * L.KS) : 0;
    L.tiles_tm = fit < L.nmt ? fit : L.nmt;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = (o + bytes + 127) / 128 * 128;
        return at;
    };
    L.h = take((size_t)L.KS * 512);
    L.pq = take((size_t)(L.Ftc / 16) * 1024);
    L.wa = take((size_t)(L.nmt - L.tiles_tm) * 16 * 256 * L.KS);
    L.yraw = take((size_t)kTcTile * s.F * 4);
    L.yt = L.yraw;  // (no f-major copy: reads go to the frame-major tile)
    L.tw = take((size_t)(L.ntail > 0 ? L.ntail : 1) * 128 * 4);        // tail rows of W (fp32)
    L.tx = take((size_t)(L.ntail > 0 ? L.ntail : 1) * (4 * 16 + 32) * 4);  // partials, p, q
    L.misc = take(512);
    L.total = o;
    return L;
}

// Shapes the tensor-core h-solve serves (the mma.sync one covers the rest).
__host__ __device__ inline bool tc_supported(const Shape &s) {
    const TcLayout L = tc_layout(s);
    return L.nmt >= 1 && L.nmt <= 4 && L.ntail <= kTcMaxTail && s.K <= 128 &&
           L.col_WA + (uint32_t)(L.tiles_tm * 8 * L.KS) <= kTmemCols;
}

// --------------------------------------------------------- tcgen05 wrappers

__device__ __forceinline__ void tmem_alloc(uint32_t *slot_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(slot_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// Shared-memory matrix descriptor, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(const void *smem_ptr, uint32_t lbo, uint32_t sbo) {
    const uint32_t a = smem_u32(smem_ptr);
    uint64_t d = (uint64_t)((a >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor: bf16 x bf16 -> f32, A K-major, B MN-major.
__host__ __device__ constexpr uint32_t tc_idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 16) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_mma_tmem_a(uint32_t d_tmem, uint32_t a_tmem, uint64_t b_desc,
                                              uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_mma_smem_a(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                              uint32_t idesc, uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// TMEM load without the wait; the registers are valid only after tmem_wait_ld.
__device__ __forceinline__ void tmem_ld8_async(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                   "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr));
}

// Wait for every outstanding TMEM load of this thread; taking r as in-out
// operands keeps the compiler from using them before the wait.
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&r)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;\n"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]),
                   "+r"(r[6]), "+r"(r[7]));
}

__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t (&r)[8]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};\n" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]));
}

__device__ __forceinline__ void tmem_st_wait() {
    asm volatile("tcgen05.wait::st.sync.aligned;\n" ::: "memory");
}

// Make generic shared-memory and TMEM writes visible to the tensor core
// and order them with the MMAs issued after the barrier.
__device__ __forceinline__ void tc_sync() {
    fence_proxy_async_shared();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

// ------------------------------------------------------------ W staging

// Load the current W (bf16 images in global memory) into TMEM and the
// shared-memory A tiles. Wimg: row k = column k of W (ld WLD); Wrow: row f =
// row f of W (ld Kp). Tail rows of W go to shared memory as FP32.
static __device__ void stage_w_tc(const Shape &s, const TcLayout &L, const __nv_bfloat16 *Wimg,
                           const __nv_bfloat16 *Wrow, const float *Wcm, uint32_t tbase,
                           unsigned char *smem) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = warp & 3, half = warp >> 2;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    // W^T into TMEM: lane k, columns col_WT + 8*st + c = pair (f = 16*st + 2c, +1)
    {
        const int k = 32 * q + lane;
        const int nst = L.Ftc / 16;
        const int s0 = half * (nst / 2), s1 = half ? nst : nst / 2;
        for (int st0 = s0; st0 < s1; st0 += 4) {
            uint32_t r[4][8];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int st = st0 + u;
                if (k < s.Kp && st < s1) {
                    const uint4 *src =
                        reinterpret_cast<const uint4 *>(Wimg + (long long)k * s.WLD + 16 * st);
                    const uint4 a = __ldcg(src), b = __ldcg(src + 1);
                    r[u][0] = a.x; r[u][1] = a.y; r[u][2] = a.z; r[u][3] = a.w;
                    r[u][4] = b.x; r[u][5] = b.y; r[u][6] = b.z; r[u][7] = b.w;
                } else {
#pragma unroll
                    for (int c = 0; c < 8; ++c) r[u][c] = 0u;
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (st0 + u < s1) tmem_st8(tbase + lane_base + L.col_WT + 8 * (st0 + u), r[u]);
        }
    }
    // W tiles of step A: TMEM for t < tiles_tm, shared memory (K-major cores) otherwise
    for (int t = half; t < L.nmt; t += 2) {
        const int f = 128 * t + 32 * q + lane;
        const uint4 *src = reinterpret_cast<const uint4 *>(Wrow + (long long)f * s.Kp);
        if (t < L.tiles_tm) {
            for (int st = 0; st < L.KS; ++st) {
                const uint4 a = __ldcg(src + 2 * st), b = __ldcg(src + 2 * st + 1);
                uint32_t r[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
                tmem_st8(tbase + lane_base + L.col_WA + 8 * (t * L.KS + st), r);
            }
        } else {
            unsigned char *wa = smem + L.wa + (size_t)(t - L.tiles_tm) * 16 * 256 * L.KS;
            const int m = f - 128 * t;
            for (int kc = 0; kc < 2 * L.KS; ++kc) {
                const uint4 v = __ldcg(src + kc);
                *reinterpret_cast<uint4 *>(wa + (m / 8) * (256 * L.KS) + kc * 128 + (m % 8) * 16) = v;
            }
        }
    }
    // tail rows (FP32) for the CUDA-core part
    float *tw = reinterpret_cast<float *>(smem + L.tw);
    for (int i = tid; i < L.ntail * 128; i += kThreads) {
        const int r = i / 128, k = i % 128;
        tw[i] = k < s.K ? Wcm[(L.Ftc + r) + (long long)k * s.F] : 0.f;
    }
    tmem_st_wait();
}

// -------------------------------------------------------------- h-solve

template <int KS>
__device__ void hsolve_tile_tc(const Shape &s, float eps, float gamma, float sw, const TileJob &t,
                               unsigned char *smem, uint32_t tbase, uint64_t *mbarA,
                               uint64_t *mbarB, unsigned &parA, unsigned &parB, uint64_t *vbar,
                               unsigned &vparity, int *err) {
    const TcLayout L = tc_layout(s);
    const int F = s.F, K = s.K, Fp = s.Fp16;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int q = warp & 3, half = warp >> 2;
    const uint32_t lane_base = (uint32_t)(32 * q) << 16;
    unsigned char *H_s = smem + L.h;
    unsigned char *PQ_s = smem + L.pq;
    float *y_raw = reinterpret_cast<float *>(smem + L.yraw);  // [16][F]
    float *tw = reinterpret_cast<float *>(smem + L.tw);       // [ntail][128]
    float *txp = reinterpret_cast<float *>(smem + L.tx);      // [ntail][4][16] partials
    float *tpq = txp + (size_t)(L.ntail > 0 ? L.ntail : 1) * 64;  // [ntail][32] p, q
    float *misc = reinterpret_cast<float *>(smem + L.misc);
    float *sy = misc;        // [16]
    float *lw = misc + 16;   // [8]
    const int k = 32 * q + lane;  // dictionary column owned in the h update
    const int jb = 8 * half;      // first of this thread's 8 frames

    // ---- frame tile -> shared memory
    {
        const size_t bytes = (size_t)t.nvalid * F * 4;
        const bool bulk = (t.ldv == F) && ((reinterpret_cast<uintptr_t>(t.Vt) & 15) == 0) &&
                          (bytes % 16 == 0);
        __syncthreads();
        if (bulk) {
            if (tid == 0) {
                fence_proxy_async_shared();
                mbar_arrive_expect_tx(vbar, (unsigned)bytes);
                bulk_g2s(y_raw, t.Vt, (unsigned)bytes, vbar);
            }
            mbar_wait_bounded(vbar, vparity, err);
            vparity ^= 1u;
        } else {
            for (int i = tid; i < t.nvalid * F; i += kThreads) {
                const int j = i / F, f = i - j * F;
                y_raw[i] = __ldg(t.Vt + (long long)j * t.ldv + f);
            }
        }
        __syncthreads();
    }
    {
        for (int j = warp; j < kTcTile; j += kWarps) {
            float a = 0.f;
            if (j < t.nvalid) {
                for (int f = lane; f < F; f += 32) {
                    const float v = y_raw[j * F + f];
                    if (bad_value(v)) flag_error(err, ERR_INPUT);
                    a += eps + v;
                }
            } else {
                a = (float)F;
            }
            a = warp_sum(a);
            if (lane == 0) sy[j] = a;
        }
    }
    __syncthreads();

    // ---- h in registers: thread owns column k, frames jb..jb+7
    float hr[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int j = jb + e;
        float h = 0.f;
        if (k < K) {
            if (t.H_in)
                h = j < t.nvalid ? t.H_in[(t.j0 + j) * t.ldh_in + k] : 0.f;
            else
                h = sy[j] / sw;
        }
        hr[e] = h;
    }
    auto write_h = [&]() {
        if (k < 16 * KS) {
            uint4 v;
            v.x = pack_bf16(hr[0], hr[1]);
            v.y = pack_bf16(hr[2], hr[3]);
            v.z = pack_bf16(hr[4], hr[5]);
            v.w = pack_bf16(hr[6], hr[7]);
            *reinterpret_cast<uint4 *>(H_s + (k / 8) * 256 + half * 128 + (k % 8) * 16) = v;
        }
    };
    // partial sums over this thread's k of the tail rows' x
    auto tail_partials = [&]() {
        for (int r = 0; r < L.ntail; ++r) {
            const float w = tw[r * 128 + k];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float v = warp_sum(w * hr[e]);
                if (lane == 0) txp[(r * 4 + q) * 16 + jb + e] = v;
            }
        }
    };
    write_h();
    tail_partials();
    tc_sync();

    float lacc = 0.f;
    const uint32_t idA = tc_idesc(128, 16), idB = tc_idesc(128, 32);
    for (int it = 0;; ++it) {
        const bool last = (it == t.n_in);
        if (last && !t.final_pass) break;
        const bool want_loss =
            t.loss_slot && ((last && t.final_pass && !t.loss_first) || (it == 0 && t.loss_first));
        // ---- step A on the tensor core: X = W H
        if (tid == 0) {
            for (int mt = 0; mt < L.nmt; ++mt) {
#pragma unroll
                for (int st = 0; st < KS; ++st) {
                    const uint64_t bdesc = tc_desc(H_s + st * 512, 256, 128);
                    const uint32_t dcol = tbase + L.col_D + 16 * mt;
                    if (mt < L.tiles_tm) {
                        tc_mma_tmem_a(dcol, tbase + L.col_WA + 8 * (mt * KS + st), bdesc, idA,
                                      st > 0);
                    } else {
                        const unsigned char *wa =
                            smem + L.wa + (size_t)(mt - L.tiles_tm) * 16 * 256 * KS;
                        tc_mma_smem_a(dcol, tc_desc(wa + st * 256, 128, 256 * KS), bdesc, idA,
                                      st > 0);
                    }
                }
            }
            tc_commit(mbarA);
        }
        // tail rows on the CUDA cores while the MMAs run
        for (int i = tid; i < L.ntail * kTcTile; i += kThreads) {
            const int r = i / kTcTile, j = i % kTcTile;
            const float x = eps + ((txp[(r * 4 + 0) * 16 + j] + txp[(r * 4 + 1) * 16 + j]) +
                                   (txp[(r * 4 + 2) * 16 + j] + txp[(r * 4 + 3) * 16 + j]));
            const float y = j < t.nvalid ? eps + y_raw[j * F + L.Ftc + r] : 1.f;
            const float qv = rcp_approx(x);
            tpq[r * 32 + j] = y * qv * qv;
            tpq[r * 32 + 16 + j] = qv;
            if (want_loss && j < t.nvalid) {
                const float rr = y * qv;
                lacc += (rr - 1.f) - logf(rr);
            }
        }
        mbar_wait_bounded(mbarA, parA, err);
        parA ^= 1u;
        tc_fence_after();
        // ---- p = y/x^2, q = 1/x from the accumulators; P|Q operand of step B
        uint32_t xr[4][8];
#pragma unroll
        for (int mt = 0; mt < 4; ++mt)
            if (mt < L.nmt) tmem_ld8_async(tbase + lane_base + L.col_D + 16 * mt + jb, xr[mt]);
#pragma unroll
        for (int mt = 0; mt < 4; ++mt)
            if (mt < L.nmt) tmem_wait_ld(xr[mt]);
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            if (mt >= L.nmt) continue;
            const int f = 128 * mt + 32 * q + lane;
            float x[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) x[e] = __uint_as_float(xr[mt][e]);
            // frame-major reads: consecutive lanes take consecutive f (no bank conflicts)
            float yv[8];
#pragma unroll
            for (int e = 0; e < 8; ++e)
                yv[e] = (jb + e < t.nvalid) ? eps + y_raw[(jb + e) * F + f] : 1.f;
            float pv[8], qv[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const float xe = eps + x[e];
                qv[e] = rcp_approx(xe);
                pv[e] = yv[e] * qv[e] * qv[e];
            }
            if (want_loss) {  // kept out of the loop above (no predicated logf)
#pragma unroll
                for (int e = 0; e < 8; ++e)
                    if (jb + e < t.nvalid) {
                        const float rr = yv[e] * qv[e];
                        lacc += (rr - 1.f) - logf(rr);
                    }
            }
            if (last) {
                if (t.final_pass && t.Pg) {
                    __nv_bfloat16 *Pg = reinterpret_cast<__nv_bfloat16 *>(t.Pg);
                    __nv_bfloat16 *Qg = reinterpret_cast<__nv_bfloat16 *>(t.Qg);
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const bool ok = jb + e < t.nvalid;
                        const long long o = (t.j0 + jb + e) * Fp + f;
                        Pg[o] = __float2bfloat16_rn(ok ? pv[e] : 0.f);
                        Qg[o] = __float2bfloat16_rn(ok ? qv[e] : 0.f);
                    }
                }
            } else {
                uint4 P4, Q4;
                P4.x = pack_bf16(pv[0], pv[1]);
                P4.y = pack_bf16(pv[2], pv[3]);
                P4.z = pack_bf16(pv[4], pv[5]);
                P4.w = pack_bf16(pv[6], pv[7]);
                Q4.x = pack_bf16(qv[0], qv[1]);
                Q4.y = pack_bf16(qv[2], qv[3]);
                Q4.z = pack_bf16(qv[4], qv[5]);
                Q4.w = pack_bf16(qv[6], qv[7]);
                unsigned char *row = PQ_s + (f / 8) * 512 + (f % 8) * 16;
                *reinterpret_cast<uint4 *>(row + half * 128) = P4;
                *reinterpret_cast<uint4 *>(row + (2 + half) * 128) = Q4;
            }
        }
        if (last) {
            // tail rows of P, Q for the statistics
            if (t.final_pass && t.Pg) {
                __nv_bfloat16 *Pg = reinterpret_cast<__nv_bfloat16 *>(t.Pg);
                __nv_bfloat16 *Qg = reinterpret_cast<__nv_bfloat16 *>(t.Qg);
                for (int i = tid; i < L.ntail * kTcTile; i += kThreads) {
                    const int r = i / kTcTile, j = i % kTcTile;
                    const bool ok = j < t.nvalid;
                    const long long o = (t.j0 + j) * Fp + L.Ftc + r;
                    Pg[o] = __float2bfloat16_rn(ok ? tpq[r * 32 + j] : 0.f);
                    Qg[o] = __float2bfloat16_rn(ok ? tpq[r * 32 + 16 + j] : 0.f);
                }
            }
            break;
        }
        tc_sync();
        // ---- step B on the tensor core: [W^T p | W^T q]
        if (tid == 0) {
            const int nst = L.Ftc / 16;
            for (int st = 0; st < nst; ++st)
                tc_mma_tmem_a(tbase + L.col_D, tbase + L.col_WT + 8 * st,
                              tc_desc(PQ_s + st * 1024, 512, 128), idB, st > 0);
            tc_commit(mbarB);
        }
        mbar_wait_bounded(mbarB, parB, err);
        parB ^= 1u;
        tc_fence_after();
        // ---- h update: thread (k, frames jb..jb+7)
        {
            uint32_t nr[8], dr[8];
            tmem_ld8_async(tbase + lane_base + L.col_D + jb, nr);
            tmem_ld8_async(tbase + lane_base + L.col_D + 16 + jb, dr);
            tmem_wait_ld(nr);
            tmem_wait_ld(dr);
            float nm[8], dn[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                nm[e] = __uint_as_float(nr[e]);
                dn[e] = __uint_as_float(dr[e]);
            }
            for (int r = 0; r < L.ntail; ++r) {
                const float w = tw[r * 128 + k];
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    nm[e] = fmaf(w, tpq[r * 32 + jb + e], nm[e]);
                    dn[e] = fmaf(w, tpq[r * 32 + 16 + jb + e], dn[e]);
                }
            }
            if (k < K) {
                with_gamma_mode(gamma, [&](auto gm) {
                    constexpr int GM = decltype(gm)::value;
#pragma unroll
                    for (int e = 0; e < 8; ++e)
                        if (dn[e] > 0.f) hr[e] = scale_pow<GM>(hr[e], __fdividef(nm[e], dn[e]), gamma);
                });
            }
            __syncthreads();  // every thread has read the tail p, q of this iteration
            write_h();
            tail_partials();
        }
        tc_sync();
    }

    // ---- outputs
    if (t.final_pass && t.Hg && k < 16 * KS) {
        __nv_bfloat16 *Hg = reinterpret_cast<__nv_bfloat16 *>(t.Hg);
        uint4 v;
        float hv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) hv[e] = jb + e < t.nvalid ? hr[e] : 0.f;
        v.x = pack_bf16(hv[0], hv[1]);
        v.y = pack_bf16(hv[2], hv[3]);
        v.z = pack_bf16(hv[4], hv[5]);
        v.w = pack_bf16(hv[6], hv[7]);
        *reinterpret_cast<uint4 *>(Hg + (long long)k * t.betap + t.j0 + jb) = v;
    }
    if (t.H_out && k < K) {
#pragma unroll
        for (int e = 0; e < 8; ++e)
            if (jb + e < t.nvalid) t.H_out[(t.j0 + jb + e) * t.ldh + k] = hr[e];
    }
    if (t.loss_slot) {
        const float l = warp_sum(lacc);
        if (lane == 0) lw[warp] = l;
        __syncthreads();
        if (tid == 0) {
            double dsum = 0.0;
            for (int w = 0; w < kWarps; ++w) dsum += (double)lw[w];
            *t.loss_slot = dsum;
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
}

}  // namespace onmf
