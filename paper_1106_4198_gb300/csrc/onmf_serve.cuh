// Device side of serving (see onmf_serve.cu): one CTA runs the whole
// Algorithm 1 step (arXiv:1106.4198) of one chunk of one stream at CTA
// scope: the h-solve of its 8-frame tiles, statistics and A/B/W' on
// (16 x 32) tiles, and the column rescale, with the same tile functions as
// the persistent single-stream kernel and a fixed order of operations, so a
// chunk's result does not depend on the batch it runs in.
#pragma once

#include "onmf_step.cuh"

namespace onmf {

struct ServeItem {
    Shape s;
    int n;  // frames of the chunk (its minibatch size)
    int n_in;
    float eps, gamma;
    int normalize, rho_on_new;
    double rho;
    const float *V;  // F x n, ld F
    float *H_out;    // K x n, ld K (device) or null
    float *Wcm, *Wrm, *Wn, *swpart;
    __nv_bfloat16 *Wimg;
    double *A, *B, *loss_sum;
    void *Pg, *Qg, *Hg;
    int betap;
    double *loss_part;
    double *chunk_loss;
    int *err;
};

template <int PREC, int KS>
static __device__ __forceinline__ void run_item_(const ServeItem *__restrict__ ip, unsigned char *smem, uint64_t *mbar,
                                unsigned &wpar, unsigned &vpar, float *s_tmp, float *s_red8,
                                double *s_red, float *acc) {
    // fields are read from the work list (global memory) where they are used,
    // rather than copied into registers for the whole item
    const ServeItem &it = *ip;
    const Shape s = it.s;
    const int ntiles = ceil_div(it.n, kTile);
    const float sw = sum_w(it.swpart, s.K, s_tmp);
    WStage ws{&mbar[0], &wpar, false};
    if (PREC == PREC_MIXED) {
        issue_wimg(s, it.Wimg, smem, &mbar[0]);
        ws.pending = true;
    }
    for (int tile = 0; tile < ntiles; ++tile) {
        TileJob t;
        t.Vt = it.V + (long long)tile * kTile * s.F;
        t.ldv = s.F;
        t.nvalid = min(kTile, it.n - tile * kTile);
        t.j0 = (long long)tile * kTile;
        t.H_in = nullptr;
        t.ldh_in = 0;
        t.H_out = it.H_out;
        t.ldh = s.K;
        t.n_in = it.n_in;
        t.loss_first = 0;
        t.final_pass = 1;
        t.loss_slot = it.loss_part + tile;
        t.Pg = it.Pg;
        t.Qg = it.Qg;
        t.Hg = it.Hg;
        t.betap = it.betap;
        hsolve_tile<PREC, KS>(s, it.eps, it.gamma, it.Wcm, it.Wrm, sw, t, smem, ws, &mbar[1], vpar,
                              it.err);
    }
    __threadfence();
    __syncthreads();
    const int FT = s.Fp16 / 16, KT = s.Kh / 32;
    for (int u = 0; u < FT * KT; ++u) {
        const int mt = u % FT, ks = u / FT;
        stats_unit<PREC>(s, mt, ks, it.Pg, it.Qg, it.Hg, it.betap, 0, it.n, smem, acc);
        epilogue_unit(s, it.Wcm, it.A, it.B, it.Wn, it.rho, it.rho_on_new, mt, ks, acc);
        __syncthreads();
    }
    __threadfence();
    __syncthreads();
    normalize_columns<PREC>(s, it.normalize, it.Wn, it.Wcm, it.Wrm, it.Wimg, nullptr, it.A, it.B,
                            it.swpart, it.err, s_red8, 0, 1);
    const double l = block_sum_ordered(it.loss_part, ntiles, s_red);
    if (threadIdx.x == 0) {
        *it.chunk_loss = l;
        *it.loss_sum += l;
    }
    if (PREC != PREC_FP32) asm volatile("fence.proxy.async.global;\n" ::: "memory");
    __threadfence();
    __syncthreads();
}

// One launch per dictionary size: every item of the launch has Kp = 16*KS
// (KS = 0 on the FP32 path, which is not specialized).
template <int PREC, int KS>
__global__ void __launch_bounds__(kThreads, 1) serve_kernel(const ServeItem *items, int nitems) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ float s_tmp;
    __shared__ float s_red8[kWarps];
    __shared__ double s_red[kThreads];
    if (threadIdx.x == 0) {
        mbar_init(&mbar[0], 1);
        mbar_init(&mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned wpar = 0, vpar = 0;
    float *acc = reinterpret_cast<float *>(smem + stats_smem_bytes(PREC) - 2 * 16 * 32 * 4);
    for (int i = blockIdx.x; i < nitems; i += gridDim.x)
        run_item_<PREC, KS>(items + i, smem, mbar, wpar, vpar, &s_tmp, s_red8, s_red, acc);
}

}  // namespace onmf
