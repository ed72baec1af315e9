// Kernels built on the cluster h-solve (onmf_cluster.cuh): the persistent
// online step (Algorithm 1: h-solve of every tile, statistics, W step and
// rescale per minibatch, as online_kernel in onmf_step.cuh) and the tile
// kernel of the projection and of the batch H step. The launch carries a
// cluster dimension of C CTAs; the online step is also cooperative.
#pragma once

#include "onmf_cluster.cuh"
#include "onmf_step.cuh"

namespace onmf {

template <int KS>
__global__ void __launch_bounds__(kThreads, 1) online_cluster_kernel(StepArgs a, int C) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ float s_tmp;
    __shared__ float s_red8[kWarps];
    __shared__ double s_red[kThreads];
    __shared__ int s_vote[2][kClMaxC];
    const Shape &s = a.s;
    const ClLayout L = cl_layout(s, C);
    const int rank = (int)cluster_ctarank();
    const int cid = blockIdx.x / C, ncl = gridDim.x / C;
    const unsigned G = gridDim.x;
    const int FT = s.Fp16 / 16, KT = s.Kh / 32;
    const int nunits = FT * KT;
    float *acc = reinterpret_cast<float *>(smem + stats_smem_bytes(PREC_MIXED) - 2 * 16 * 32 * 4);
    unsigned epoch = 0;
    int vp = 0, seq = 0;
    cta_err_init(a.err);
    // the launch must carry clusters of exactly C CTAs, or the remote
    // addresses below would name CTAs that do not exist
    if (cluster_nctarank() != (unsigned)C || gridDim.x % C != 0) {
        if (threadIdx.x == 0) flag_error(a.err, ERR_CONFIG);
        return;
    }
    cluster_sync();  // every CTA of the cluster runs before any remote access
    for (int m = 0; m < a.nmb; ++m) {
        const bool lastmb = (m == a.nmb - 1);
        const int nb = lastmb ? a.nb_last : a.beta;
        const double rho = lastmb ? a.rho_last : a.rho_full;
        const float *Vm = a.V + (long long)m * a.beta * a.ldv;
        float *Hm = a.H_out ? a.H_out + (long long)m * a.beta * a.ldh : nullptr;
        const float *Him = a.H_in ? a.H_in + (long long)m * a.beta * a.ldh_in : nullptr;
        const int ntiles = ceil_div(nb, kClTile);
        // ---- phase 1: h-solve of every 32-frame tile, one cluster per tile
        if (cid < ntiles) {
            const float sw = sum_w(a.swpart, s.K, &s_tmp);
            cl_stage_w(s, L, rank, a.Wrow, smem);
            for (int tile = cid; tile < ntiles; tile += ncl) {
                TileJob t;
                t.Vt = Vm + (long long)tile * kClTile * a.ldv;
                t.ldv = a.ldv;
                t.nvalid = min(kClTile, nb - tile * kClTile);
                t.j0 = (long long)tile * kClTile;
                t.H_in = Him;
                t.ldh_in = a.ldh_in;
                t.H_out = Hm;
                t.ldh = a.ldh;
                t.n_in = a.n_in;
                t.hpen = a.hpen;
                t.hpen_a = a.hpen_a;
                t.loss_first = 0;
                t.final_pass = 1;
                t.loss_slot = a.loss_part + (long long)tile * C + rank;
                t.Pg = a.Pg;
                t.Qg = a.Qg;
                t.Hg = a.Hg;
                t.betap = a.betap;
                hsolve_tile_cluster<KS>(s, L, rank, a.eps, a.gamma, sw, t, smem, seq++, a.err);
            }
        }
        if (!cl_grid_sync(a.bar, G, epoch, a.err, s_vote, vp, C, rank)) break;
        // ---- phase 2: statistics and W' = sqrt(A/B)
        for (int u = blockIdx.x; u < nunits; u += G) {
            const int mt = u % FT, ks = u / FT;
            stats_unit<PREC_MIXED>(s, mt, ks, a.Pg, a.Qg, a.Hg, a.betap, 0, nb, smem, acc);
            // the dictionary penalty's form: W' = sqrt(A/(B + mu)); mu = 0
            // adds +0 to B, the same bits as the plain form
            online_epilogue<PREC_MIXED, true>(a, mt, ks, rho, acc);
            __syncthreads();
        }
        if (!cl_grid_sync(a.bar, G, epoch, a.err, s_vote, vp, C, rank)) break;
        // ---- phase 3: column sums, rescale, bf16 rows of W, loss
        normalize_columns<PREC_CL>(s, a.normalize, a.Wn, a.Wcm, a.Wrm, a.Wimg, a.Wrow, a.A, a.B,
                                   a.acc, a.swpart, a.err, s_red8, blockIdx.x, gridDim.x);
        if (blockIdx.x == G - 1) {
            const double l = block_sum_ordered(a.loss_part, (long long)ntiles * C, s_red);
            if (threadIdx.x == 0) *a.loss_sum += l;
        }
        if (!lastmb && !cl_grid_sync(a.bar, G, epoch, a.err, s_vote, vp, C, rank)) break;
    }
    cluster_sync();  // no CTA leaves while a peer may still address its shared memory
}

template <int KS>
__global__ void __launch_bounds__(kThreads, 1) tile_cluster_kernel(TileArgs a, int C) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ float s_tmp;
    const ClLayout L = cl_layout(a.s, C);
    const int rank = (int)cluster_ctarank();
    const long long cid = blockIdx.x / C, ncl = gridDim.x / C;
    const long long ntiles = (a.n + kClTile - 1) / kClTile;
    int seq = 0;
    if (cluster_nctarank() != (unsigned)C || gridDim.x % C != 0) {
        if (threadIdx.x == 0) flag_error(a.err, ERR_CONFIG);
        return;
    }
    cluster_sync();
    if (cid < ntiles) {
        const float sw = sum_w(a.swpart, a.s.K, &s_tmp);
        cl_stage_w(a.s, L, rank, a.Wrow, smem);
        for (long long tile = cid; tile < ntiles; tile += ncl) {
            TileJob t;
            t.Vt = a.V + tile * kClTile * a.ldv;
            t.ldv = a.ldv;
            t.nvalid = (int)min((long long)kClTile, a.n - tile * kClTile);
            t.j0 = tile * kClTile;
            t.H_in = a.H_in;
            t.ldh_in = a.ldh_in;
            t.H_out = a.H_out;
            t.ldh = a.ldh;
            t.n_in = a.n_in;
            t.hpen = a.hpen;
            t.hpen_a = a.hpen_a;
            t.loss_first = a.loss_first;
            t.final_pass = a.final_pass;
            t.loss_slot = a.loss_part ? a.loss_part + tile * C + rank : nullptr;
            t.Pg = a.Pg;
            t.Qg = a.Qg;
            t.Hg = a.Hg;
            t.betap = a.betap;
            hsolve_tile_cluster<KS>(a.s, L, rank, a.eps, a.gamma, sw, t, smem, seq++, a.err);
        }
    }
    cluster_sync();
}

}  // namespace onmf
