// Templated step kernels of libonmf: the persistent online step (Algorithm 1
// of arXiv:1106.4198, one launch = many minibatches), the tile kernel used by
// projection and the batch H step, and the split-N statistics of the batch
// W step. Included by the translation units that instantiate them.
//
// One online minibatch of the persistent kernel (the launch is cooperative,
// so all CTAs are co-resident and every grid-wide wait is bounded):
//   1. h-solve of every 8-frame tile (frames are independent given W); each
//      tile leaves its final P = Y/X^2, Q = 1/X and H rows in L2-resident
//      scratch and its d_IS sum in a per-tile slot;
//   2. statistics a = (P H^T) o W^2, b = Q H^T;
//   3. A <- rho A + a, B <- rho B + b, W' = sqrt(A/B), the L1 rescale of every
//      column (W = W'/s, A /= s, B *= s), the derived images of W, and the
//      running loss.
// Mixed precision: each h-solve tile releases its frame range (a release
// increment of the range's counter) instead of a grid barrier; the
// statistics are tcgen05 MMAs per (64-frequency tile, frame range) unit that
// wait only for their range and leave FP32 partial sums; one arrive/wait
// grid barrier (the next minibatch's frames are staged and the column's
// W, A, B loaded while it is open), then one pass per dictionary column does
// all of step 3 with the partial sums reduced in a fixed order; a grid
// barrier before the next minibatch. FP32: a grid barrier after step 1,
// step 2 on (16 rows x 32 columns) output tiles with A, B and W' updated in
// their epilogue, a grid barrier, step 3 one CTA per column, a grid barrier.
#pragma once

#include "onmf_device.cuh"
#include "onmf_hsolve.cuh"
#include "onmf_kernels.cuh"
#include "onmf_tc.cuh"

namespace onmf {

// ---------------------------------------------------------------- phase 2

constexpr int kChunk = 1024;  // frames per shared-memory chunk (mixed stats)
constexpr int kPS = 24;       // row stride (bf16) of the P/Q chunk rows
constexpr int kHS = kChunk + 8;

__host__ __device__ inline size_t stats_smem_bytes(int prec) {
    if (prec != PREC_FP32)
        return (size_t)2 * kChunk * kPS * 2 + (size_t)32 * kHS * 2 + 2 * 16 * 32 * 4;
    return (size_t)kWarps * 16 * 32 * 2 * 4 + 2 * 16 * 32 * 4;
}

// Accumulate sum_j P[j][f] H[j][k] and sum_j Q[j][f] H[j][k] over frames
// [jb, je) for the output tile rows 16*mt.. and columns 32*ks.. into
// acc[2][16][32] (shared memory). Warp w: P (w < 4) or Q, and a quarter of
// the frames of each chunk; it loads each P/Q fragment once and applies it to
// all four n8 tiles of k. The four quarters are added in order at the end.
static __device__ void stats_unit_mixed(const Shape &s, int mt, int ks, const __nv_bfloat16 *Pg,
                                 const __nv_bfloat16 *Qg, const __nv_bfloat16 *Hg,
                                 long long betap, long long jb, long long je, unsigned char *smem,
                                 float *acc) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, tq = lane & 3, mi = lane >> 3, r8 = lane & 7;
    __nv_bfloat16 *P_s = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *Q_s = P_s + kChunk * kPS;
    __nv_bfloat16 *H_s = Q_s + kChunk * kPS;
    const int quarter = warp & 3, which = warp >> 2;
    const int Fp = s.Fp16;
    const int f0 = 16 * mt, k0 = 32 * ks;
    float c[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int e = 0; e < 4; ++e) c[u][e] = 0.f;
    const __nv_bfloat16 *X_s = which ? Q_s : P_s;
    for (long long cb = jb; cb < je; cb += kChunk) {
        const int nf = (int)min((long long)kChunk, je - cb);
        const int nfr = (nf + 15) / 16 * 16;  // rows touched by the k16 steps
        // P and Q rows (16 values = two 16-byte chunks per frame), no index division
        for (int i = tid; i < nfr * 2; i += kThreads) {
            const int jj = i >> 1, half = i & 1;
            const bool ok = jj < nf;
            const long long o = (cb + jj) * Fp + f0 + 8 * half;
            cp_async16(P_s + jj * kPS + 8 * half, ok ? Pg + o : Pg, ok ? 16 : 0);
            cp_async16(Q_s + jj * kPS + 8 * half, ok ? Qg + o : Qg, ok ? 16 : 0);
        }
        // H rows k0..k0+31: warp per row, lanes over 8-frame chunks
        const int nch = nfr / 8;
        for (int kk = warp; kk < 32; kk += kWarps)
            for (int ch = lane; ch < nch; ch += 32) {
                const int jj = 8 * ch;
                const bool ok = jj < nf;
                const __nv_bfloat16 *src = ok ? Hg + (long long)(k0 + kk) * betap + cb + jj : Hg;
                cp_async16(H_s + kk * kHS + jj, src, ok ? 16 : 0);
            }
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        const int nks = nfr / 16;
        const int kb = quarter * nks / 4, ke = (quarter + 1) * nks / 4;
        const __nv_bfloat16 *xrow = X_s + (r8 + 8 * (mi >> 1)) * kPS + 8 * (mi & 1);
        const __nv_bfloat16 *hrow = H_s + (r8 + 8 * (mi >> 1)) * kHS + 8 * (mi & 1);
        for (int ksi = kb; ksi < ke; ++ksi) {
            uint32_t a[4], b0[4], b1[4];
            ldmatrix_x4_trans(a, xrow + 16 * ksi * kPS);
            ldmatrix_x4(b0, hrow + 16 * ksi);             // k rows 0..15
            ldmatrix_x4(b1, hrow + 16 * kHS + 16 * ksi);  // k rows 16..31
            mma_bf16_16816(c[0], a, b0[0], b0[1]);
            mma_bf16_16816(c[1], a, b0[2], b0[3]);
            mma_bf16_16816(c[2], a, b1[0], b1[1]);
            mma_bf16_16816(c[3], a, b1[2], b1[3]);
        }
        __syncthreads();
    }
    // quarters -> acc, in quarter order (the chunk buffers are free now)
    float *red = reinterpret_cast<float *>(smem);  // [8 warps][16][32]
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int ff = g + 8 * (e >> 1), kk = 8 * u + 2 * tq + (e & 1);
            red[(warp * 16 + ff) * 32 + kk] = c[u][e];
        }
    __syncthreads();
    for (int e = tid; e < 2 * 512; e += kThreads) {
        const int w4 = e >> 9, rem = e & 511;  // P (0) or Q (1), then (ff, kk)
        const float *r = red + (w4 * 4) * 512 + rem;
        acc[w4 * 512 + rem] = ((r[0] + r[512]) + r[1024]) + r[1536];
    }
    __syncthreads();
}

static __device__ void stats_unit_fp32(const Shape &s, int mt, int ks, const float *Pg, const float *Qg,
                                const float *Hg, long long jb, long long je, unsigned char *smem,
                                float *acc) {
    const int tid = threadIdx.x, lane = tid & 31, grp = tid >> 5;
    float *red = reinterpret_cast<float *>(smem);  // [8][16][32][2]
    const int fb = lane >> 3, kb = lane & 7;
    const int Fp = s.Fp16, Kh = s.Kh;
    const int f0 = 16 * mt + 4 * fb, k0 = 32 * ks + 4 * kb;
    float cp[4][4], cq[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) cp[a][b] = cq[a][b] = 0.f;
    const long long len = je - jb;
    const long long per = (len + kWarps - 1) / kWarps;
    const long long j1 = jb + grp * per, j2 = min(je, j1 + per);
#pragma unroll 4
    for (long long j = j1; j < j2; ++j) {
        const float4 p = __ldcg(reinterpret_cast<const float4 *>(Pg + j * Fp + f0));
        const float4 q = __ldcg(reinterpret_cast<const float4 *>(Qg + j * Fp + f0));
        const float4 h = __ldcg(reinterpret_cast<const float4 *>(Hg + j * Kh + k0));
        const float pv[4] = {p.x, p.y, p.z, p.w}, qv[4] = {q.x, q.y, q.z, q.w};
        const float hv[4] = {h.x, h.y, h.z, h.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                cp[a][b] = fmaf(pv[a], hv[b], cp[a][b]);
                cq[a][b] = fmaf(qv[a], hv[b], cq[a][b]);
            }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            float *r = red + (((size_t)grp * 16 + 4 * fb + a) * 32 + 4 * kb + b) * 2;
            r[0] = cp[a][b];
            r[1] = cq[a][b];
        }
    __syncthreads();
    for (int e = tid; e < 512; e += kThreads) {
        const int ff = e >> 5, kk = e & 31;
        float sp = 0.f, sq = 0.f;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            sp += red[(((size_t)w * 16 + ff) * 32 + kk) * 2];
            sq += red[(((size_t)w * 16 + ff) * 32 + kk) * 2 + 1];
        }
        acc[ff * 32 + kk] = sp;
        acc[(16 + ff) * 32 + kk] = sq;
    }
    __syncthreads();
}

// The same sums over a long frame range (the batch W step): chunks of
// kChunkP frames in two shared-memory stages, the copy of chunk c+1 in
// flight while chunk c is multiplied. Same warp roles as stats_unit_mixed.
constexpr int kChunkP = 448;
constexpr int kHSP = kChunkP + 8;
constexpr size_t kStageP = (size_t)2 * kChunkP * kPS * 2 + (size_t)32 * kHSP * 2;
static_assert(2 * kStageP <= (size_t)2 * kChunk * kPS * 2 + (size_t)32 * kHS * 2,
              "two pipelined stages fit where one chunk of stats_unit_mixed goes");

static __device__ void stats_unit_mixed_pipe(const Shape &s, int mt, int ks,
                                             const __nv_bfloat16 *Pg, const __nv_bfloat16 *Qg,
                                             const __nv_bfloat16 *Hg, long long betap,
                                             long long jb, long long je, unsigned char *smem,
                                             float *acc) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, tq = lane & 3, mi = lane >> 3, r8 = lane & 7;
    const int quarter = warp & 3, which = warp >> 2;
    const int Fp = s.Fp16;
    const int f0 = 16 * mt, k0 = 32 * ks;
    auto P_of = [&](int st) { return reinterpret_cast<__nv_bfloat16 *>(smem + st * kStageP); };
    auto Q_of = [&](int st) { return P_of(st) + kChunkP * kPS; };
    auto H_of = [&](int st) { return P_of(st) + 2 * kChunkP * kPS; };
    auto issue = [&](long long cb, int st) {
        const int nf = (int)min((long long)kChunkP, je - cb);
        const int nfr = (nf + 15) / 16 * 16;
        __nv_bfloat16 *P_s = P_of(st), *Q_s = Q_of(st), *H_s = H_of(st);
        for (int i = tid; i < nfr * 2; i += kThreads) {
            const int jj = i >> 1, half = i & 1;
            const bool ok = jj < nf;
            const long long o = (cb + jj) * Fp + f0 + 8 * half;
            cp_async16(P_s + jj * kPS + 8 * half, ok ? Pg + o : Pg, ok ? 16 : 0);
            cp_async16(Q_s + jj * kPS + 8 * half, ok ? Qg + o : Qg, ok ? 16 : 0);
        }
        const int nch = nfr / 8;
        for (int kk = warp; kk < 32; kk += kWarps)
            for (int ch = lane; ch < nch; ch += 32) {
                const int jj = 8 * ch;
                const bool ok = jj < nf;
                const __nv_bfloat16 *src = ok ? Hg + (long long)(k0 + kk) * betap + cb + jj : Hg;
                cp_async16(H_s + kk * kHSP + jj, src, ok ? 16 : 0);
            }
        cp_async_commit();
    };
    float c[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int e = 0; e < 4; ++e) c[u][e] = 0.f;
    const long long nchunk = (je - jb + kChunkP - 1) / kChunkP;
    if (nchunk > 0) issue(jb, 0);
    for (long long ci = 0; ci < nchunk; ++ci) {
        const long long cb = jb + ci * kChunkP;
        const int st = (int)(ci & 1);
        if (ci + 1 < nchunk) {
            issue(cb + kChunkP, st ^ 1);
            cp_async_wait_group1();
        } else {
            cp_async_wait_all();
        }
        __syncthreads();
        const int nf = (int)min((long long)kChunkP, je - cb);
        const int nks = (nf + 15) / 16;
        const int kb = quarter * nks / 4, ke = (quarter + 1) * nks / 4;
        const __nv_bfloat16 *X_s = which ? Q_of(st) : P_of(st);
        const __nv_bfloat16 *xrow = X_s + (r8 + 8 * (mi >> 1)) * kPS + 8 * (mi & 1);
        const __nv_bfloat16 *hrow = H_of(st) + (r8 + 8 * (mi >> 1)) * kHSP + 8 * (mi & 1);
        for (int ksi = kb; ksi < ke; ++ksi) {
            uint32_t a[4], b0[4], b1[4];
            ldmatrix_x4_trans(a, xrow + 16 * ksi * kPS);
            ldmatrix_x4(b0, hrow + 16 * ksi);
            ldmatrix_x4(b1, hrow + 16 * kHSP + 16 * ksi);
            mma_bf16_16816(c[0], a, b0[0], b0[1]);
            mma_bf16_16816(c[1], a, b0[2], b0[3]);
            mma_bf16_16816(c[2], a, b1[0], b1[1]);
            mma_bf16_16816(c[3], a, b1[2], b1[3]);
        }
        __syncthreads();
    }
    float *red = reinterpret_cast<float *>(smem);  // [8 warps][16][32]
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int ff = g + 8 * (e >> 1), kk = 8 * u + 2 * tq + (e & 1);
            red[(warp * 16 + ff) * 32 + kk] = c[u][e];
        }
    __syncthreads();
    for (int e = tid; e < 2 * 512; e += kThreads) {
        const int w4 = e >> 9, rem = e & 511;
        const float *r = red + (w4 * 4) * 512 + rem;
        acc[w4 * 512 + rem] = ((r[0] + r[512]) + r[1024]) + r[1536];
    }
    __syncthreads();
}

template <int PREC>
__device__ __forceinline__ void stats_unit(const Shape &s, int mt, int ks, const void *Pg,
                                           const void *Qg, const void *Hg, long long betap,
                                           long long jb, long long je, unsigned char *smem,
                                           float *acc) {
    if (PREC != PREC_FP32)
        stats_unit_mixed(s, mt, ks, reinterpret_cast<const __nv_bfloat16 *>(Pg),
                         reinterpret_cast<const __nv_bfloat16 *>(Qg),
                         reinterpret_cast<const __nv_bfloat16 *>(Hg), betap, jb, je, smem, acc);
    else
        stats_unit_fp32(s, mt, ks, reinterpret_cast<const float *>(Pg),
                        reinterpret_cast<const float *>(Qg), reinterpret_cast<const float *>(Hg),
                        jb, je, smem, acc);
}

// ---- arithmetic of the running statistics A and B. Every entry is 8
// bytes: a double (ACC_FP64), a float (ACC_FP32, second half zero) or a
// float pair (hi, lo) with hi = fl(hi + lo) (ACC_FP32C), kept by
// error-free transformations: TwoSum (Knuth, TAOCP vol. 2, 4.2.2), the exact
// error of a product by one FMA, and FastTwoSum (Dekker 1971) to
// renormalize. The explicit _rn intrinsics keep the compiler from fusing
// or reassociating these steps.
enum { ACC_FP64 = 0, ACC_FP32 = 1, ACC_FP32C = 2 };

struct DF {
    float hi, lo;
};

__device__ __forceinline__ DF two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}

__device__ __forceinline__ DF fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

// x * c + d
__device__ __forceinline__ DF df_mul_add(DF x, float c, float d) {
    const float p = __fmul_rn(x.hi, c);
    const float pe = __fmaf_rn(x.hi, c, -p);
    const DF t = two_sum(p, d);
    return fast_two_sum(t.hi, __fadd_rn(__fmaf_rn(x.lo, c, pe), t.lo));
}

// x + c * d
__device__ __forceinline__ DF df_add_mul(DF x, float c, float d) {
    const float p = __fmul_rn(c, d);
    const float pe = __fmaf_rn(c, d, -p);
    const DF t = two_sum(x.hi, p);
    return fast_two_sum(t.hi, __fadd_rn(__fadd_rn(x.lo, pe), t.lo));
}

// x / c (the remainder of the leading quotient is exact by one FMA)
__device__ __forceinline__ DF df_div(DF x, float c) {
    const float q = __fdiv_rn(x.hi, c);
    const float r = __fmaf_rn(-q, c, x.hi);
    return fast_two_sum(q, __fdiv_rn(__fadd_rn(r, x.lo), c));
}

// x * (ih + il), ih + il a float pair (a reciprocal: ih = 1/c rounded, il =
// (1 - ih c) ih its first correction); no division per entry
__device__ __forceinline__ DF df_mul_pair(DF x, float ih, float il) {
    const float p = __fmul_rn(x.hi, ih);
    const float pe = __fmaf_rn(x.hi, ih, -p);
    return fast_two_sum(p, __fmaf_rn(x.hi, il, __fmaf_rn(x.lo, ih, pe)));
}

__device__ __forceinline__ DF df_load(const double *p) {
    const float2 v = *reinterpret_cast<const float2 *>(p);
    return {v.x, v.y};
}

__device__ __forceinline__ void df_store(double *p, DF x) {
    *reinterpret_cast<float2 *>(p) = make_float2(x.hi, x.lo);
}

// A <- rho A + a, B <- rho B + b, W' = sqrt(A/B) for the tile's entries
// (Algorithm 1; the past-scaling reading of rho unless rho_on_new), in the
// arithmetic `accm` of A and B. The increments a, b are FP32 in every mode.
// WPEN: the dictionary penalty mu * sum W (FP32 path), W' = sqrt(A/(B + mu)).
template <bool WPEN = false>
static __device__ void epilogue_unit(const Shape &s, const float *Wcm, double *A, double *B,
                                     float *Wn, double rho, int rho_on_new, int accm, int mt,
                                     int ks, const float *acc, float wpen = 0.f) {
    const int F = s.F, K = s.K;
    const float rhof = (float)rho;
    for (int e = threadIdx.x; e < 512; e += kThreads) {
        const int kk = e >> 4, ff = e & 15;
        const int f = 16 * mt + ff, k = 32 * ks + kk;
        if (f >= F || k >= K) continue;
        const long long i = f + (long long)k * F;
        const float w = Wcm[i];
        const float af = acc[ff * 32 + kk] * w * w;
        const float bf = acc[(16 + ff) * 32 + kk];
        float An, Bn;  // the new A and B rounded to FP32, for W'
        if (accm == ACC_FP64) {
            const double av = (double)af, bv = (double)bf;
            const double A0 = A[i], B0 = B[i];
            double Ad, Bd;
            if (rho_on_new) {
                Ad = fma(rho, av, A0);
                Bd = fma(rho, bv, B0);
            } else {
                Ad = fma(rho, A0, av);
                Bd = fma(rho, B0, bv);
            }
            A[i] = Ad;
            B[i] = Bd;
            An = (float)Ad;
            Bn = (float)Bd;
        } else if (accm == ACC_FP32) {
            const float A0 = df_load(A + i).hi, B0 = df_load(B + i).hi;
            An = rho_on_new ? __fmaf_rn(rhof, af, A0) : __fmaf_rn(rhof, A0, af);
            Bn = rho_on_new ? __fmaf_rn(rhof, bf, B0) : __fmaf_rn(rhof, B0, bf);
            df_store(A + i, {An, 0.f});
            df_store(B + i, {Bn, 0.f});
        } else {
            const DF A0 = df_load(A + i), B0 = df_load(B + i);
            const DF Ad = rho_on_new ? df_add_mul(A0, rhof, af) : df_mul_add(A0, rhof, af);
            const DF Bd = rho_on_new ? df_add_mul(B0, rhof, bf) : df_mul_add(B0, rhof, bf);
            df_store(A + i, Ad);
            df_store(B + i, Bd);
            An = Ad.hi;
            Bn = Bd.hi;
        }
        const float Bd = WPEN ? Bn + wpen : Bn;
        Wn[i] = (Bd > 0.f) ? sqrtf(__fdiv_rn(An, Bd)) : w;
    }
}

template <int PREC, bool PEN = false>
static __device__ __forceinline__ void online_epilogue(const StepArgs &a, int mt, int ks,
                                                       double rho, const float *acc) {
    if constexpr (PREC == PREC_FP32 || PEN)
        epilogue_unit<true>(a.s, a.Wcm, a.A, a.B, a.Wn, rho, a.rho_on_new, a.acc, mt, ks, acc,
                            a.wpen);
    else
        epilogue_unit(a.s, a.Wcm, a.A, a.B, a.Wn, rho, a.rho_on_new, a.acc, mt, ks, acc);
}

// Fixed-order sum of one float per thread over the CTA.
__device__ __forceinline__ float block_sum_f(float v, float *red8) {
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red8[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = 0.f;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) r += red8[w];
    __syncthreads();
    return r;
}

// One CTA per column: s_k = sum_f W'_fk, then the L1 rescale of Algorithm 1
// and the derived images of W. Each thread keeps its rows in registers
// (up to 4 * kThreads rows per pass).
template <int PREC>
static __device__ void normalize_columns(const Shape &s, int normalize, const float *__restrict__ Wn,
                                  float *__restrict__ Wcm, float *__restrict__ Wrm,
                                  __nv_bfloat16 *__restrict__ Wimg,
                                  __nv_bfloat16 *__restrict__ Wrow, double *__restrict__ A,
                                  double *__restrict__ B, int accm, float *__restrict__ swpart,
                                  int *err, float *red8, int first, int stride) {
    const int F = s.F, K = s.K;
    const int tid = threadIdx.x;
    for (int k = first; k < K; k += stride) {
        const float *col = Wn + (long long)k * F;
        float part = 0.f;
        for (int f = tid; f < F; f += kThreads) part += col[f];
        const float sum = block_sum_f(part, red8);
        const bool sc = normalize && sum > 0.f;
        const float inv = sc ? __frcp_rn(sum) : 1.f;
        const double invd = sc ? 1.0 / (double)sum : 1.0;
        const double sd = sc ? (double)sum : 1.0;
        bool bad = false;
        for (int f0 = 0; f0 < F; f0 += 4 * kThreads) {
            float w[4];
            double av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int f = f0 + tid + u * kThreads;
                if (f < F) {
                    const long long i = f + (long long)k * F;
                    w[u] = col[f];
                    if (A) {
                        av[u] = A[i];
                        bv[u] = B[i];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int f = f0 + tid + u * kThreads;
                if (f < F) {
                    const long long i = f + (long long)k * F;
                    const float wv = w[u] * inv;
                    bad |= !isfinite(wv);
                    Wcm[i] = wv;
                    if (A && sc) {
                        if (accm == ACC_FP64) {
                            A[i] = av[u] * invd;
                            B[i] = bv[u] * sd;
                        } else {
                            // the same 8 bytes as a float pair
                            DF a2, b2;
                            memcpy(&a2, &av[u], 8);
                            memcpy(&b2, &bv[u], 8);
                            if (accm == ACC_FP32) {
                                a2 = {__fdiv_rn(a2.hi, sum), 0.f};
                                b2 = {__fmul_rn(b2.hi, sum), 0.f};
                            } else {
                                a2 = df_div(a2, sum);
                                b2 = df_mul_add(b2, sum, 0.f);
                            }
                            df_store(A + i, a2);
                            df_store(B + i, b2);
                        }
                    }
                    if (PREC == PREC_FP32) {
                        Wrm[(long long)f * K + k] = wv;
                    } else {
                        if (PREC != PREC_CL)
                            Wimg[(long long)k * s.WLD + f] = __float2bfloat16_rn(wv);
                        if (PREC == PREC_TC || PREC == PREC_CL)
                            Wrow[(long long)f * s.Kp + k] = __float2bfloat16_rn(wv);
                    }
                }
            }
        }
        if (bad) flag_error(err, ERR_NUMERIC);
        if (tid == 0) swpart[k] = sc ? sum * inv : sum;
    }
}

// Deterministic sum of n doubles by one CTA (fixed chunking and tree).
static __device__ double block_sum_ordered(const double *x, long long n, double *red) {
    const int tid = threadIdx.x;
    const long long per = (n + kThreads - 1) / kThreads;
    double a = 0.0;
    const long long lo = tid * per, hi = min(n, lo + per);
    for (long long i = lo; i < hi; ++i) a += x[i];
    red[tid] = a;
    __syncthreads();
    for (int st = kThreads / 2; st > 0; st >>= 1) {
        if (tid < st) red[tid] += red[tid + st];
        __syncthreads();
    }
    double r = red[0];
    __syncthreads();
    return r;
}

template <int PREC, int KS, bool PEN = false>
__device__ __forceinline__ void hsolve_tile(const Shape &s, float eps, float gamma,
                                            const float *Wcm, const float *Wrm, float sw,
                                            const TileJob &t, unsigned char *smem, WStage &ws,
                                            uint64_t *vbar, unsigned &vpar, int *err) {
    if constexpr (PREC == PREC_MIXED)
        hsolve_tile_mixed<KS, PEN>(s, eps, gamma, sw, t, smem, ws, vbar, vpar, err);
    else
        hsolve_tile_fp32(s, eps, gamma, Wcm, Wrm, sw, t, smem, err);
}

}  // namespace onmf

#include "onmf_stats_tc.cuh"

namespace onmf {

// ----------------------------------------------------- persistent online step

// PEN: the penalized variant of the mma path (Section 2.2, "Extensions");
// the FP32 path takes the penalties in its one instantiation.
template <int PREC, int KS, bool PEN = false>
__global__ void __launch_bounds__(kThreads, 1) online_kernel(StepArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[9];
    __shared__ float s_tmp;
    __shared__ float s_red8[kWarps];
    __shared__ double s_red[kThreads];
    __shared__ uint32_t s_tslot;
    cta_err_init(a.err);
    if (threadIdx.x == 0) {
        for (int i = 0; i < 9; ++i) mbar_init(&mbar[i], 1);
        fence_mbar_init();
    }
    // tensor memory: the tcgen05 h-solve's W and accumulators, or the
    // accumulator of the tcgen05 statistics (mma h-solve)
    if (PREC == PREC_TC && threadIdx.x < 32) tmem_alloc(&s_tslot, kTmemCols);
    if (PREC == PREC_MIXED && threadIdx.x < 32) tmem_alloc(&s_tslot, kStatsTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = (PREC == PREC_TC || PREC == PREC_MIXED) ? s_tslot : 0u;
    unsigned wpar = 0, vpar = 0, epoch = 0, parA = 0, parB = 0;
    StatsBars sb{{&mbar[4], &mbar[5]}, {&mbar[6], &mbar[7]}, &mbar[8], {0u, 0u}, {0u, 0u}, 0u};
    constexpr int TILE = PREC == PREC_TC ? kTcTile : kTile;
    const unsigned G = gridDim.x;
    const Shape &s = a.s;
    const int FT = s.Fp16 / 16, KT = s.Kh / 32;
    const int nunits = FT * KT;
    float *acc = reinterpret_cast<float *>(smem + stats_smem_bytes(PREC) - 2 * 16 * 32 * 4);
    // mma path: the frames of this CTA's first tile of the next minibatch
    // are bulk-copied into shared memory during the current one (right after
    // the CTA's h-solve when that buffer lies outside the statistics' shared
    // memory, else after the statistics) and staged and converted while the
    // CTA waits at the barrier before the column pass
    bool v_prefetched = false, v_ready = false;
    const bool early_v = PREC == PREC_MIXED && mixed_layout(a.s).yraw >= kStatsSmemBytes;
    // the CTA's first tile of minibatch mb (false: none, or not one bulk copy)
    auto first_tile = [&](int mb, TileJob &tn) -> bool {
        const int nbn = (mb == a.nmb - 1) ? a.nb_last : a.beta;
        const int tn0 = (int)blockIdx.x;
        if (tn0 * TILE >= nbn) return false;
        tn.Vt = a.V + ((long long)mb * a.beta + (long long)tn0 * TILE) * a.ldv;
        tn.ldv = a.ldv;
        tn.nvalid = min(TILE, nbn - tn0 * TILE);
        tn.v_staged = 1;
        return tile_bulk(tn.Vt, a.ldv, a.s.F, tn.nvalid);
    };
    auto prefetch = [&](int mb) {
        TileJob tn;
        if (!first_tile(mb, tn)) return;
        if (threadIdx.x == 0) {
            const unsigned bytes = (unsigned)((size_t)tn.nvalid * a.s.F * 4);
            fence_proxy_async_shared();
            mbar_arrive_expect_tx(&mbar[1], bytes);
            bulk_g2s(smem + mixed_layout(a.s).yraw, tn.Vt, bytes, &mbar[1]);
        }
        v_prefetched = true;
    };
    for (int m = 0; m < a.nmb; ++m) {
        const bool lastmb = (m == a.nmb - 1);
        const int nb = lastmb ? a.nb_last : a.beta;
        const double rho = lastmb ? a.rho_last : a.rho_full;
        const float *Vm = a.V + (long long)m * a.beta * a.ldv;
        float *Hm = a.H_out ? a.H_out + (long long)m * a.beta * a.ldh : nullptr;
        const float *Him = a.H_in ? a.H_in + (long long)m * a.beta * a.ldh_in : nullptr;
        const int ntiles = ceil_div(nb, TILE);
        ONMF_STAMP(a.stamps, m, 0);
        // mma path: frame ranges of the statistics; a tile's range counter
        // counts its h-solve done (phase 2 waits per range, not for the grid)
        const int FT64 = (s.Fp16 + 63) / 64;
        const StatsSplit sp = stats_split(nb, (int)G, FT64, a.stats_ranges);
        unsigned *rcnt = a.bar + 4;
        // ---- phase 1: h-solve of every tile
        if ((int)blockIdx.x < ntiles) {
            WStage ws{&mbar[0], &wpar, false};
            float sw;
            if (PREC == PREC_MIXED) {
                // the loads of the column sums (warp 1) go out before the
                // W^T image copy (thread 0), with no CTA barrier between
                // (the grid barrier that ended the last minibatch, or the
                // kernel's start, leaves the CTA synchronized and the image's
                // shared memory unused), so that they do not queue behind
                // the image copies of every CTA; added as sum_w adds them
                float swr[4] = {0.f, 0.f, 0.f, 0.f};  // K <= 128 on this path
                if ((threadIdx.x >> 5) == 1)
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int k = (int)(threadIdx.x & 31) + 32 * i;
                        if (k < s.K) swr[i] = a.swpart[k];
                    }
                issue_wimg_nosync(s, a.Wimg, smem, &mbar[0]);
                ws.pending = true;
                if ((threadIdx.x >> 5) == 1) {
                    float v = 0.f;
#pragma unroll
                    for (int i = 0; i < 4; ++i) v += swr[i];
                    v = warp_sum(v);
                    if ((threadIdx.x & 31) == 0) s_tmp = v;
                }
                __syncthreads();
                sw = s_tmp;
            } else {
                sw = sum_w(a.swpart, s.K, &s_tmp);
            }
            if (PREC == PREC_TC) stage_w_tc(s, tc_layout(s), a.Wimg, a.Wrow, a.Wcm, tbase, smem);
            for (int tile = blockIdx.x; tile < ntiles; tile += G) {
                TileJob t;
                t.Vt = Vm + (long long)tile * TILE * a.ldv;
                t.ldv = a.ldv;
                t.nvalid = min(TILE, nb - tile * TILE);
                t.j0 = (long long)tile * TILE;
                t.H_in = Him;
                t.ldh_in = a.ldh_in;
                t.H_out = Hm;
                t.ldh = a.ldh;
                t.n_in = a.n_in;
                if constexpr (PREC == PREC_FP32 || PEN) {
                    t.hpen = a.hpen;
                    t.hpen_a = a.hpen_a;
                }
                t.loss_first = 0;
                t.final_pass = 1;
                t.pq_core = PREC == PREC_MIXED ? 1 : 0;
                t.loss_slot = a.loss_part + tile;
                t.Pg = a.Pg;
                t.Qg = a.Qg;
                t.Hg = a.Hg;
                t.betap = a.betap;
                t.v_ready = (PREC == PREC_MIXED && tile == (int)blockIdx.x && v_ready) ? 1 : 0;
                v_ready = false;
#ifdef ONMF_PHASE_STAMPS
                t.hst = (a.stamps && tile == (int)blockIdx.x && m < kStampMb)
                            ? a.stamps + ((long long)m * G + blockIdx.x) * kStampPts + 16
                            : nullptr;
#endif
                v_prefetched = false;
                if (tile == (int)blockIdx.x) ONMF_STAMP(a.stamps, m, 38);
                if constexpr (PREC == PREC_TC)
                    hsolve_tile_tc<KS>(s, a.eps, a.gamma, sw, t, smem, tbase, &mbar[2], &mbar[3],
                                       parA, parB, &mbar[1], vpar, a.err);
                else
                    hsolve_tile<PREC, KS, PEN>(s, a.eps, a.gamma, a.Wcm, a.Wrm, sw, t, smem, ws,
                                          &mbar[1], vpar, a.err);
                if (tile == (int)blockIdx.x) ONMF_STAMP(a.stamps, m, 39);
                if constexpr (PREC == PREC_MIXED) {
                    // the tile's P, Q, H rows are written (the h-solve ends
                    // with a CTA barrier): publish them to its frame range,
                    // for the bulk copies (async proxy) of phase 2
                    if (threadIdx.x == 0) {
                        asm volatile("fence.proxy.async.global;\n" ::: "memory");
                        red_release_gpu_add(rcnt + tile / sp.gps, 1u);
                    }
                }
            }
        }
        if (early_v && !lastmb) prefetch(m + 1);
        ONMF_STAMP(a.stamps, m, 1);
        if (PREC != PREC_MIXED && !grid_sync(a.bar, G, epoch, a.err)) break;
        ONMF_STAMP(a.stamps, m, 2);
        if constexpr (PREC == PREC_MIXED) {
            // ---- phase 2: [P H^T | Q H^T] partial sums on the tensor cores,
            // each unit as soon as the h-solves of its frame range are done
            const int ng = (nb + 7) / 8;
            // the next tile's frames, on their way since the h-solve ended,
            // are staged by warps 1-7 during the CTA's first unit (the
            // window before the column pass then has nothing left to do)
            StageJob job{nullptr, 0, 0, nullptr, a.eps, &mbar[1], vpar};
            const bool stage_in_unit = early_v && v_prefetched && (int)blockIdx.x < FT64 * sp.S;
            if (stage_in_unit) {
                const int nbn = (m + 1 == a.nmb - 1) ? a.nb_last : a.beta;  // as first_tile
                job.Vt = a.V + ((long long)(m + 1) * a.beta + (long long)blockIdx.x * TILE) * a.ldv;
                job.ldv = a.ldv;
                job.nvalid = min(TILE, nbn - (int)blockIdx.x * TILE);
#ifdef ONMF_PHASE_STAMPS
                if (a.stamps && m < kStampMb)  // points 34-37 of this minibatch
                    job.hst = a.stamps + ((long long)m * G + blockIdx.x) * kStampPts + 16;
#endif
            }
            for (int u = blockIdx.x; u < FT64 * sp.S; u += G) {
                stats_unit_tc(u % FT64, u / FT64, sp.gps, ng, a.betap / 8,
                              reinterpret_cast<const unsigned char *>(a.Pg),
                              reinterpret_cast<const unsigned char *>(a.Hg), a.part, s.K, s.Fp16,
                              smem, tbase, sb, rcnt, a.err,
                              a.stamps ? a.stamps + ((long long)m * G + blockIdx.x) * kStampPts + 8
                                       : nullptr,
                              s, job);
                job.Vt = nullptr;
            }
            if (stage_in_unit) {
                if (tile_bulk(a.V + ((long long)(m + 1) * a.beta + (long long)blockIdx.x * TILE) * a.ldv,
                              a.ldv, s.F, job.nvalid))
                    vpar ^= 1u;
                v_prefetched = false;
                v_ready = true;
            }
            ONMF_STAMP(a.stamps, m, 3);
            // the frames of this CTA's first tile of the next minibatch (if
            // not on their way yet: phase 3 uses no dynamic shared memory);
            // then, while the other CTAs finish phase 2, W, A, B of the CTA's
            // column load and those frames are staged and converted
            if (!lastmb && !early_v) prefetch(m + 1);
            grid_arrive(a.bar, epoch);
            ColVals pre;
            col_load(a, blockIdx.x, pre);
            ONMF_STAMP(a.stamps, m, 32);
            if (v_prefetched) {
                TileJob tn;
                first_tile(m + 1, tn);
#ifdef ONMF_PHASE_STAMPS
                if (a.stamps && m < kStampMb)  // points 34-37 of this minibatch
                    tn.hst = a.stamps + ((long long)m * G + blockIdx.x) * kStampPts + 16;
#endif
                mixed_stage_frames(s, a.eps, tn, smem, &mbar[1], vpar, a.err);
                v_prefetched = false;
                v_ready = true;
            }
            ONMF_STAMP(a.stamps, m, 33);
            if (!grid_wait(a.bar, G, epoch, a.err)) break;
            ONMF_STAMP(a.stamps, m, 4);
            // ---- phase 3: partial sums, A, B, W' = sqrt(A/B), rescale, image
            {
                long long *cst = a.stamps && m < kStampMb
                                     ? a.stamps + ((long long)m * G + blockIdx.x) * kStampPts + 40
                                     : nullptr;
                if (a.acc == ACC_FP64)
                    column_step<PEN, ACC_FP64>(a, sp.S, rho, s_red8, blockIdx.x, gridDim.x, pre, cst);
                else if (a.acc == ACC_FP32)
                    column_step<PEN, ACC_FP32>(a, sp.S, rho, s_red8, blockIdx.x, gridDim.x, pre, cst);
                else
                    column_step<PEN, ACC_FP32C>(a, sp.S, rho, s_red8, blockIdx.x, gridDim.x, pre,
                                                cst);
            }
            // the range counters start from zero in the next minibatch (every
            // reader of them passed the barrier above; the next barrier
            // orders these stores before the next increments)
            if (blockIdx.x == 0)
                for (int i = threadIdx.x; i < sp.S; i += kThreads) rcnt[i] = 0u;
        } else {
            // ---- phase 2: statistics and W' = sqrt(A/B)
            for (int u = blockIdx.x; u < nunits; u += G) {
                const int mt = u % FT, ks = u / FT;
                stats_unit<PREC>(s, mt, ks, a.Pg, a.Qg, a.Hg, a.betap, 0, nb, smem, acc);
                online_epilogue<PREC, PEN>(a, mt, ks, rho, acc);
                __syncthreads();
            }
            if (!grid_sync(a.bar, G, epoch, a.err)) break;
            // ---- phase 3: column sums, rescale, images, loss
            normalize_columns<PREC>(s, a.normalize, a.Wn, a.Wcm, a.Wrm, a.Wimg, a.Wrow, a.A,
                                    a.B, a.acc, a.swpart, a.err, s_red8, blockIdx.x, gridDim.x);
        }
        if (blockIdx.x == G - 1) {
            double l = block_sum_ordered(a.loss_part, ntiles, s_red);
            if (threadIdx.x == 0) *a.loss_sum += l;
        }
        if (PREC != PREC_FP32) asm volatile("fence.proxy.async.global;\n" ::: "memory");
        ONMF_STAMP(a.stamps, m, 5);
        if (!lastmb && !grid_sync(a.bar, G, epoch, a.err)) break;
        ONMF_STAMP(a.stamps, m, 6);
    }
    // leaving early (a flagged error): a prefetched frame tile still in
    // flight lands before the shared memory goes away
    if (PREC == PREC_MIXED && v_prefetched) mbar_wait_bounded(&mbar[1], vpar, a.err);
    if (PREC == PREC_TC || PREC == PREC_MIXED) {
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x < 32) tmem_dealloc(tbase, PREC == PREC_TC ? kTmemCols : kStatsTmemCols);
    }
}

// ----------------------------------------------- projection / batch tiles

template <int PREC, int KS, bool PEN = false>
__global__ void __launch_bounds__(kThreads, 1) tile_kernel(TileArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[4];
    __shared__ float s_tmp;
    __shared__ uint32_t s_tslot;
    constexpr int TILE = PREC == PREC_TC ? kTcTile : kTile;
    const long long ntiles = (a.n + TILE - 1) / TILE;
    if ((long long)blockIdx.x >= ntiles) return;
    if (threadIdx.x == 0) {
        for (int i = 0; i < 4; ++i) mbar_init(&mbar[i], 1);
        fence_mbar_init();
    }
    if (PREC == PREC_TC && threadIdx.x < 32) tmem_alloc(&s_tslot, kTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = PREC == PREC_TC ? s_tslot : 0u;
    unsigned wpar = 0, vpar = 0, parA = 0, parB = 0;
    const float sw = sum_w(a.swpart, a.s.K, &s_tmp);
    WStage ws{&mbar[0], &wpar, false};
    if (PREC == PREC_MIXED) {
        issue_wimg(a.s, a.Wimg, smem, &mbar[0]);
        ws.pending = true;
    }
    if (PREC == PREC_TC) stage_w_tc(a.s, tc_layout(a.s), a.Wimg, a.Wrow, a.Wcm, tbase, smem);
    bool staged = false;  // this tile's frames were issued by the previous one
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        TileJob t;
        t.Vt = a.V + tile * TILE * a.ldv;
        t.ldv = a.ldv;
        t.nvalid = (int)min((long long)TILE, a.n - tile * TILE);
        t.j0 = tile * TILE;
        t.H_in = a.H_in;
        t.ldh_in = a.ldh_in;
        t.H_out = a.H_out;
        t.ldh = a.ldh;
        t.n_in = a.n_in;
        t.loss_first = a.loss_first;
        t.final_pass = a.final_pass;
        t.loss_slot = a.loss_part ? a.loss_part + tile : nullptr;
        if constexpr (PREC == PREC_FP32 || PEN) {
            t.hpen = a.hpen;
            t.hpen_a = a.hpen_a;
        }
        t.Pg = a.Pg;
        t.Qg = a.Qg;
        t.Hg = a.Hg;
        t.betap = a.betap;
        if constexpr (PREC == PREC_MIXED) {
            // the mma h-solve copies the next tile's frames while it computes
            const long long next = tile + gridDim.x;
            t.v_staged = staged;
            if (next < ntiles) {
                const float *vn = a.V + next * TILE * a.ldv;
                const int nn = (int)min((long long)TILE, a.n - next * TILE);
                if (tile_bulk(vn, a.ldv, a.s.F, nn)) {
                    t.Vnext = vn;
                    t.nvalid_next = nn;
                }
            }
            staged = t.Vnext != nullptr;
        }
        if constexpr (PREC == PREC_TC)
            hsolve_tile_tc<KS>(a.s, a.eps, a.gamma, sw, t, smem, tbase, &mbar[2], &mbar[3], parA,
                               parB, &mbar[1], vpar, a.err);
        else
            hsolve_tile<PREC, KS, PEN>(a.s, a.eps, a.gamma, a.Wcm, a.Wrm, sw, t, smem, ws, &mbar[1],
                                  vpar, a.err);
    }
    if (PREC == PREC_TC) {
        tc_fence_before();
        __syncthreads();
        if (threadIdx.x < 32) tmem_dealloc(tbase, kTmemCols);
    }
}

// Split-N statistics: partial sums over frame chunk `c` of P H^T and Q H^T
// for every (16 x 32) output tile -> part[c][2][Fp16][Kh].
template <int PREC>
__global__ void __launch_bounds__(kThreads, 1)
    batch_stats_kernel(Shape s, const void *Pg, const void *Qg, const void *Hg, long long betap,
                       long long N, int nchunks, float *part) {
    extern __shared__ __align__(128) unsigned char smem[];
    float *acc = reinterpret_cast<float *>(smem + stats_smem_bytes(PREC) - 2 * 16 * 32 * 4);
    const int FT = s.Fp16 / 16, KT = s.Kh / 32;
    const long long per = ((N + nchunks - 1) / nchunks + 15) / 16 * 16;
    const long long units = (long long)FT * KT * nchunks;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const int c = (int)(u / (FT * KT));
        const int r = (int)(u - (long long)c * FT * KT);
        const int mt = r % FT, ks = r / FT;
        const long long jb = c * per, je = min(N, jb + per);
        if (jb < je) {
            if constexpr (PREC != PREC_FP32)
                stats_unit_mixed_pipe(s, mt, ks, reinterpret_cast<const __nv_bfloat16 *>(Pg),
                                      reinterpret_cast<const __nv_bfloat16 *>(Qg),
                                      reinterpret_cast<const __nv_bfloat16 *>(Hg), betap, jb, je,
                                      smem, acc);
            else
                stats_unit<PREC>(s, mt, ks, Pg, Qg, Hg, betap, jb, je, smem, acc);
        } else {
            for (int e = threadIdx.x; e < 1024; e += kThreads) acc[e] = 0.f;
            __syncthreads();
        }
        for (int e = threadIdx.x; e < 1024; e += kThreads) {
            const int which = e >> 9, ff = (e >> 5) & 15, kk = e & 31;
            part[(((long long)c * 2 + which) * s.Fp16 + 16 * mt + ff) * s.Kh + 32 * ks + kk] =
                acc[e];
        }
        __syncthreads();
    }
}

}  // namespace onmf
