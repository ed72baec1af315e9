// libonmf kernels: the persistent online step (Algorithm 1 of
// arXiv:1106.4198, one launch = many minibatches), projection, and the batch
// multiplicative-update cycle (Section 2.1).
//
// One online minibatch is three grid-wide phases separated by bounded grid
// barriers (the launch is cooperative, so all CTAs are co-resident):
//   1. h-solve of every frame tile (frames are independent given W); each
//      tile leaves its final P = Y/X^2, Q = 1/X and H rows in L2-resident
//      scratch and its d_IS sum in a per-tile slot;
//   2. statistics a = (P H^T) o W^2, b = Q H^T on (16 rows x 32 columns)
//      output tiles, then A <- rho A + a, B <- rho B + b and
//      W' = sqrt(A/B) for the tile's entries;
//   3. one warp per dictionary column: s_k = sum_f W'_fk by warp shuffles,
//      W = W'/s, A /= s, B *= s, the derived W images, the loss sum.
#include <cstdio>

#include "onmf_device.cuh"
#include "onmf_hsolve.cuh"
#include "onmf_kernels.cuh"
#include "onmf_launch.h"

namespace onmf {

// ---------------------------------------------------------------- phase 2

constexpr int kChunk = 256;  // frames per shared-memory chunk (mixed stats)
constexpr int kPS = 24;      // row stride (bf16) of the P/Q chunk rows
constexpr int kHS = kChunk + 8;

__host__ __device__ inline size_t stats_smem_bytes(int prec) {
    if (prec == PREC_MIXED)
        return (size_t)2 * kChunk * kPS * 2 + (size_t)32 * kHS * 2 + 2 * 16 * 32 * 4;
    return (size_t)kWarps * 16 * 32 * 2 * 4 + 2 * 16 * 32 * 4;
}

// Accumulate sum_j P[j][f] H[j][k] and sum_j Q[j][f] H[j][k] over frames
// [jb, je) for the output tile rows 16*mt.. and columns 32*ks.. into
// acc[2][16][32] (shared memory).
__device__ void stats_unit_mixed(const Shape &s, int mt, int ks, const __nv_bfloat16 *Pg,
                                 const __nv_bfloat16 *Qg, const __nv_bfloat16 *Hg,
                                 long long betap, long long jb, long long je, unsigned char *smem,
                                 float *acc) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int g = lane >> 2, tq = lane & 3, mi = lane >> 3, r8 = lane & 7;
    __nv_bfloat16 *P_s = reinterpret_cast<__nv_bfloat16 *>(smem);
    __nv_bfloat16 *Q_s = P_s + kChunk * kPS;
    __nv_bfloat16 *H_s = Q_s + kChunk * kPS;
    const int nt = warp & 3, which = warp >> 2;
    const int Fp = s.Fp16;
    const int f0 = 16 * mt, k0 = 32 * ks;
    float c0[4] = {0.f, 0.f, 0.f, 0.f}, c1[4] = {0.f, 0.f, 0.f, 0.f};
    const __nv_bfloat16 *X_s = which ? Q_s : P_s;
    for (long long c = jb; c < je; c += kChunk) {
        const int nf = (int)min((long long)kChunk, je - c);
        for (int i = tid; i < kChunk * 4; i += kThreads) {
            const int w = i / (kChunk * 2), rem = i - w * kChunk * 2;
            const int jj = rem >> 1, half = rem & 1;
            const __nv_bfloat16 *base = w ? Qg : Pg;
            const bool ok = jj < nf;
            const __nv_bfloat16 *src = ok ? base + (c + jj) * Fp + f0 + 8 * half : base;
            __nv_bfloat16 *dst = (w ? Q_s : P_s) + jj * kPS + 8 * half;
            cp_async16(dst, src, ok ? 16 : 0);
        }
        for (int i = tid; i < 32 * (kChunk / 8); i += kThreads) {
            const int kk = i / (kChunk / 8), ch = i - kk * (kChunk / 8);
            const int jj = 8 * ch;
            const bool ok = jj < nf;
            const __nv_bfloat16 *src = ok ? Hg + (long long)(k0 + kk) * betap + c + jj : Hg;
            cp_async16(H_s + kk * kHS + jj, src, ok ? 16 : 0);
        }
        cp_async_commit();
        cp_async_wait_all();
        __syncthreads();
        const int nks = (nf + 15) / 16;
        const __nv_bfloat16 *hrow = H_s + (8 * nt + g) * kHS + 2 * tq;
        int ksi = 0;
        for (; ksi + 1 < nks; ksi += 2) {
            uint32_t a[4], b[4];
            ldmatrix_x4_trans(a, X_s + (16 * ksi + r8 + 8 * (mi >> 1)) * kPS + 8 * (mi & 1));
            ldmatrix_x4_trans(b, X_s + (16 * (ksi + 1) + r8 + 8 * (mi >> 1)) * kPS + 8 * (mi & 1));
            mma_bf16_16816(c0, a, *reinterpret_cast<const uint32_t *>(hrow + 16 * ksi),
                           *reinterpret_cast<const uint32_t *>(hrow + 16 * ksi + 8));
            mma_bf16_16816(c1, b, *reinterpret_cast<const uint32_t *>(hrow + 16 * (ksi + 1)),
                           *reinterpret_cast<const uint32_t *>(hrow + 16 * (ksi + 1) + 8));
        }
        if (ksi < nks) {
            uint32_t a[4];
            ldmatrix_x4_trans(a, X_s + (16 * ksi + r8 + 8 * (mi >> 1)) * kPS + 8 * (mi & 1));
            mma_bf16_16816(c0, a, *reinterpret_cast<const uint32_t *>(hrow + 16 * ksi),
                           *reinterpret_cast<const uint32_t *>(hrow + 16 * ksi + 8));
        }
        __syncthreads();
    }
#pragma unroll
    for (int e = 0; e < 4; ++e) {
        const int ff = g + 8 * (e >> 1), kk = 8 * nt + 2 * tq + (e & 1);
        acc[(which * 16 + ff) * 32 + kk] = c0[e] + c1[e];
    }
    __syncthreads();
}

__device__ void stats_unit_fp32(const Shape &s, int mt, int ks, const float *Pg, const float *Qg,
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
#pragma unroll 2
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

template <int PREC>
__device__ __forceinline__ void stats_unit(const Shape &s, int mt, int ks, const void *Pg,
                                           const void *Qg, const void *Hg, long long betap,
                                           long long jb, long long je, unsigned char *smem,
                                           float *acc) {
    if (PREC == PREC_MIXED)
        stats_unit_mixed(s, mt, ks, reinterpret_cast<const __nv_bfloat16 *>(Pg),
                         reinterpret_cast<const __nv_bfloat16 *>(Qg),
                         reinterpret_cast<const __nv_bfloat16 *>(Hg), betap, jb, je, smem, acc);
    else
        stats_unit_fp32(s, mt, ks, reinterpret_cast<const float *>(Pg),
                        reinterpret_cast<const float *>(Qg), reinterpret_cast<const float *>(Hg),
                        jb, je, smem, acc);
}

// A <- rho A + a, B <- rho B + b, W' = sqrt(A/B) for the tile's entries
// (Algorithm 1; the past-scaling reading of rho unless rho_on_new).
__device__ void online_epilogue(const StepArgs &a, int mt, int ks, double rho, const float *acc) {
    const int F = a.s.F, K = a.s.K;
    for (int e = threadIdx.x; e < 512; e += kThreads) {
        const int kk = e >> 4, ff = e & 15;
        const int f = 16 * mt + ff, k = 32 * ks + kk;
        if (f >= F || k >= K) continue;
        const long long i = f + (long long)k * F;
        const float w = a.Wcm[i];
        const double av = (double)(acc[ff * 32 + kk] * w * w);
        const double bv = (double)acc[(16 + ff) * 32 + kk];
        double An, Bn;
        if (a.rho_on_new) {
            An = a.A[i] + rho * av;
            Bn = a.B[i] + rho * bv;
        } else {
            An = rho * a.A[i] + av;
            Bn = rho * a.B[i] + bv;
        }
        a.A[i] = An;
        a.B[i] = Bn;
        a.Wn[i] = (Bn > 0.0) ? sqrtf(__fdiv_rn((float)An, (float)Bn)) : w;
    }
}

// One warp per column: s_k = sum_f W'_fk (warp shuffles), then the L1
// rescale of Algorithm 1 and the derived images of W.
template <int PREC>
__device__ void normalize_columns(const Shape &s, int normalize, const float *Wn, float *Wcm,
                                  float *Wrm, __nv_bfloat16 *Wimg, double *A, double *B,
                                  float *swpart, int *err, int first_warp, int nwarps) {
    const int F = s.F, K = s.K;
    const int lane = threadIdx.x & 31;
    for (int k = first_warp; k < K; k += nwarps) {
        const float *col = Wn + (long long)k * F;
        float sum = 0.f;
        for (int f = lane; f < F; f += 32) sum += col[f];
        sum = warp_sum(sum);
        const bool sc = normalize && sum > 0.f;
        const float inv = sc ? __frcp_rn(sum) : 1.f;
        const double invd = sc ? 1.0 / (double)sum : 1.0;
        const double sd = sc ? (double)sum : 1.0;
        bool bad = false;
        for (int f = lane; f < F; f += 32) {
            const long long i = f + (long long)k * F;
            const float w = col[f] * inv;
            bad |= !isfinite(w);
            Wcm[i] = w;
            if (A) {
                A[i] *= invd;
                B[i] *= sd;
            }
            if (PREC == PREC_FP32)
                Wrm[(long long)f * K + k] = w;
            else
                Wimg[(long long)k * s.WLD + f] = __float2bfloat16_rn(w);
        }
        if (bad) flag_error(err, ERR_NUMERIC);
        if (lane == 0) swpart[k] = sc ? sum * inv : sum;
    }
}

// Deterministic sum of n doubles by one CTA (fixed chunking and tree).
__device__ double block_sum_ordered(const double *x, long long n, double *red) {
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

// ----------------------------------------------------- persistent online step

template <int PREC>
__global__ void __launch_bounds__(kThreads, 1) online_kernel(StepArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ float s_tmp;
    __shared__ double s_red[kThreads];
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned wpar = 0, vpar = 0, epoch = 0;
    const unsigned G = gridDim.x;
    const Shape &s = a.s;
    const int FT = s.Fp16 / 16, KS = s.Kh / 32;
    const int nunits = FT * KS;
    float *acc = reinterpret_cast<float *>(smem + stats_smem_bytes(PREC) - 2 * 16 * 32 * 4);
    for (int m = 0; m < a.nmb; ++m) {
        const bool lastmb = (m == a.nmb - 1);
        const int nb = lastmb ? a.nb_last : a.beta;
        const double rho = lastmb ? a.rho_last : a.rho_full;
        const float *Vm = a.V + (long long)m * a.beta * a.ldv;
        float *Hm = a.H_out ? a.H_out + (long long)m * a.beta * a.ldh : nullptr;
        const int ntiles = ceil_div(nb, kTile);
        // ---- phase 1: h-solve of every tile
        if ((int)blockIdx.x < ntiles) {
            const float sw = sum_w(a.swpart, s.K, &s_tmp);
            if (PREC == PREC_MIXED) stage_wimg(s, a.Wimg, smem, &mbar[0], wpar, a.err);
            for (int tile = blockIdx.x; tile < ntiles; tile += G) {
                TileJob t;
                t.Vt = Vm + (long long)tile * kTile * a.ldv;
                t.ldv = a.ldv;
                t.nvalid = min(kTile, nb - tile * kTile);
                t.j0 = (long long)tile * kTile;
                t.H_in = nullptr;
                t.ldh_in = 0;
                t.H_out = Hm;
                t.ldh = a.ldh;
                t.n_in = a.n_in;
                t.loss_first = 0;
                t.final_pass = 1;
                t.loss_slot = a.loss_part + tile;
                t.Pg = a.Pg;
                t.Qg = a.Qg;
                t.Hg = a.Hg;
                t.betap = a.betap;
                if (PREC == PREC_MIXED)
                    hsolve_tile_mixed(s, a.eps, a.gamma, sw, t, smem, &mbar[1], vpar, a.err);
                else
                    hsolve_tile_fp32(s, a.eps, a.gamma, a.Wcm, a.Wrm, sw, t, smem, a.err);
            }
        }
        if (!grid_sync(a.bar, G, epoch, a.err)) return;
        // ---- phase 2: statistics and W' = sqrt(A/B)
        for (int u = blockIdx.x; u < nunits; u += G) {
            const int mt = u % FT, ks = u / FT;
            stats_unit<PREC>(s, mt, ks, a.Pg, a.Qg, a.Hg, a.betap, 0, nb, smem, acc);
            online_epilogue(a, mt, ks, rho, acc);
            __syncthreads();
        }
        if (!grid_sync(a.bar, G, epoch, a.err)) return;
        // ---- phase 3: column sums, rescale, images, loss
        normalize_columns<PREC>(s, a.normalize, a.Wn, a.Wcm, a.Wrm, a.Wimg, a.A, a.B, a.swpart,
                                a.err, blockIdx.x * kWarps + (threadIdx.x >> 5), G * kWarps);
        if (blockIdx.x == 0) {
            double l = block_sum_ordered(a.loss_part, ntiles, s_red);
            if (threadIdx.x == 0) *a.loss_sum += l;
        }
        if (PREC == PREC_MIXED) asm volatile("fence.proxy.async.global;\n" ::: "memory");
        if (!lastmb && !grid_sync(a.bar, G, epoch, a.err)) return;
    }
}

// ----------------------------------------------- projection / batch tiles

template <int PREC>
__global__ void __launch_bounds__(kThreads, 1) tile_kernel(TileArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ float s_tmp;
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned wpar = 0, vpar = 0;
    const long long ntiles = (a.n + kTile - 1) / kTile;
    if ((long long)blockIdx.x >= ntiles) return;
    const float sw = sum_w(a.swpart, a.s.K, &s_tmp);
    if (PREC == PREC_MIXED) stage_wimg(a.s, a.Wimg, smem, &mbar[0], wpar, a.err);
    for (long long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        TileJob t;
        t.Vt = a.V + tile * kTile * a.ldv;
        t.ldv = a.ldv;
        t.nvalid = (int)min((long long)kTile, a.n - tile * kTile);
        t.j0 = tile * kTile;
        t.H_in = a.H_in;
        t.ldh_in = a.ldh_in;
        t.H_out = a.H_out;
        t.ldh = a.ldh;
        t.n_in = a.n_in;
        t.loss_first = a.loss_first;
        t.final_pass = a.final_pass;
        t.loss_slot = a.loss_part ? a.loss_part + tile : nullptr;
        t.Pg = a.Pg;
        t.Qg = a.Qg;
        t.Hg = a.Hg;
        t.betap = a.betap;
        if (PREC == PREC_MIXED)
            hsolve_tile_mixed(a.s, a.eps, a.gamma, sw, t, smem, &mbar[1], vpar, a.err);
        else
            hsolve_tile_fp32(a.s, a.eps, a.gamma, a.Wcm, a.Wrm, sw, t, smem, a.err);
    }
}

// Derived images of a dictionary W (column-major F x K): the row-major copy,
// the bf16 W^T image and the column sums. One warp per column.
__global__ void __launch_bounds__(kThreads) prepare_kernel(Shape s, const float *Wcm, float *Wrm,
                                                           __nv_bfloat16 *Wimg, float *swpart) {
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

// Split-N statistics: partial sums over frame chunk `c` of P H^T and Q H^T
// for every (16 x 32) output tile -> part[c][2][Fp16][Kh].
template <int PREC>
__global__ void __launch_bounds__(kThreads, 1)
    batch_stats_kernel(Shape s, const void *Pg, const void *Qg, const void *Hg, long long betap,
                       long long N, int nchunks, float *part) {
    extern __shared__ __align__(128) unsigned char smem[];
    float *acc = reinterpret_cast<float *>(smem + stats_smem_bytes(PREC) - 2 * 16 * 32 * 4);
    const int FT = s.Fp16 / 16, KS = s.Kh / 32;
    const long long per = ((N + nchunks - 1) / nchunks + 15) / 16 * 16;
    const long long units = (long long)FT * KS * nchunks;
    for (long long u = blockIdx.x; u < units; u += gridDim.x) {
        const int c = (int)(u / (FT * KS));
        const int r = (int)(u - (long long)c * FT * KS);
        const int mt = r % FT, ks = r / FT;
        const long long jb = c * per, je = min(N, jb + per);
        if (jb < je) {
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

size_t online_smem_bytes(const Shape &s, int prec) {
    size_t p1 = prec == PREC_MIXED ? mixed_layout(s).total : hsolve_fp32_smem_bytes(s);
    size_t p2 = stats_smem_bytes(prec);
    return p1 > p2 ? p1 : p2;
}

size_t tile_smem_bytes(const Shape &s, int prec) {
    return prec == PREC_MIXED ? mixed_layout(s).total : hsolve_fp32_smem_bytes(s);
}

size_t batch_stats_smem_bytes(int prec) { return stats_smem_bytes(prec); }

static const void *online_fn(int prec) {
    return prec == PREC_MIXED ? (const void *)online_kernel<PREC_MIXED>
                              : (const void *)online_kernel<PREC_FP32>;
}
static const void *tile_fn(int prec) {
    return prec == PREC_MIXED ? (const void *)tile_kernel<PREC_MIXED>
                              : (const void *)tile_kernel<PREC_FP32>;
}
static const void *bstats_fn(int prec) {
    return prec == PREC_MIXED ? (const void *)batch_stats_kernel<PREC_MIXED>
                              : (const void *)batch_stats_kernel<PREC_FP32>;
}

cudaError_t configure_kernels() {
    cudaError_t e;
    for (int p = 0; p < 2; ++p) {
        if ((e = cudaFuncSetAttribute(online_fn(p), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      227 * 1024)) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(tile_fn(p), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      227 * 1024)) != cudaSuccess)
            return e;
        if ((e = cudaFuncSetAttribute(bstats_fn(p), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      227 * 1024)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

cudaError_t max_coresident_blocks(int prec, size_t smem, int *blocks_per_sm) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, online_fn(prec), kThreads,
                                                         smem);
}

cudaError_t launch_online(const StepArgs &a, int prec, int grid, size_t smem,
                          cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(a.bar, 0, sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    StepArgs copy = a;
    void *args[] = {&copy};
    e = cudaLaunchCooperativeKernel(online_fn(prec), dim3(grid), dim3(kThreads), args, smem, stream);
    if (e == cudaSuccess) count_launch();
    return e;
}

cudaError_t launch_tiles(const TileArgs &a, int prec, int grid, size_t smem, cudaStream_t stream) {
    TileArgs copy = a;
    void *args[] = {&copy};
    cudaError_t e = cudaLaunchKernel(tile_fn(prec), dim3(grid), dim3(kThreads), args, smem, stream);
    if (e == cudaSuccess) count_launch();
    return e;
}

cudaError_t launch_prepare(const Shape &s, const float *Wcm, float *Wrm, __nv_bfloat16 *Wimg,
                           float *swpart, cudaStream_t stream) {
    const int grid = (s.K + kWarps - 1) / kWarps;
    prepare_kernel<<<grid, kThreads, 0, stream>>>(s, Wcm, Wrm, Wimg, swpart);
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

}  // namespace onmf
