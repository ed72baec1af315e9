// Device side of serving (see onmf_serve.cu): the Algorithm 1 step
// (arXiv:1106.4198) of a batch of chunks of different streams, one
// minibatch per chunk, in three phases after a copy of the frames (below).
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
    const float *V;     // F x n, ld F, in the batch's device frame buffer
    const float *Vsrc;  // the same frames in mapped pinned host memory
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

// Serving runs a batch of chunks (one minibatch each, of streams with
// different dictionaries and lengths) as three launches, so the work of
// even a single chunk spreads over the GPU: the h-solve of every (chunk,
// 8-frame tile) pair, the statistics of every (chunk, 16x32 output tile)
// pair, and the rescale of every (chunk, column) pair; the kernel boundaries
// separate the phases. The tile, statistics and rescale functions are those
// of the persistent single-stream kernel, so a chunk's result does not
// depend on the batch it runs in. off[i] is the first work pair of item i
// and off[n] one past the last; a launch covers items range[0] <=
// i < range[1], read from device memory so that one captured launch serves
// every batch; pairs are taken in grid-stride order.

// Item owning work pair p: the largest i with off[i] <= p.
__device__ __forceinline__ int serve_item_of(const int *off, int n, int p) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (off[mid] <= p)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Phase 0: the frames of every chunk from the pinned host buffer it was
// submitted into (mapped into the device's address space) to its slice of
// the batch's device frame buffer. Work pairs are (chunk, block of
// kGatherF4 float4, U per thread, loads before stores); both ends are
// 16-byte aligned and padded to a whole float4, so the copy is in float4
// throughout.
constexpr int kGatherU = 4, kGatherF4 = kGatherU * kThreads;

template <int U>
__global__ void __launch_bounds__(kThreads) serve_gather_kernel(const ServeItem *items,
                                                                const int *off,
                                                                const int *range) {
    const int i0 = range[0], nitems = range[1] - i0;
    items += i0;
    off += i0;
    const int base = off[0], total = off[nitems] - base;
    for (int p = blockIdx.x; p < total; p += gridDim.x) {
        const int i = serve_item_of(off, nitems, base + p);
        const ServeItem &it = items[i];
        const long long nv = ((long long)it.n * it.s.F + 3) >> 2;
        const long long v0 = (long long)(base + p - off[i]) * kGatherF4 + threadIdx.x;
        const float4 *src = reinterpret_cast<const float4 *>(it.Vsrc);
        float4 *dst = reinterpret_cast<float4 *>(const_cast<float *>(it.V));
        float4 r[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long v = v0 + u * kThreads;
            if (v < nv) r[u] = src[v];
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const long long v = v0 + u * kThreads;
            if (v < nv) dst[v] = r[u];
        }
    }
}

// Phase 1: h-solve of (chunk, tile) pairs; every item of the launch has
// Kp = 16*KS (KS = 0 on the FP32 path, which is not specialized).
template <int PREC, int KS>
__global__ void __launch_bounds__(kThreads, 1) serve_hsolve_kernel(const ServeItem *items,
                                                                  const int *off, const int *range) {
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
    WStage ws{&mbar[0], &wpar, false};
    int staged = -1;  // item whose W^T image is in shared memory
    const int i0 = range[0], nitems = range[1] - i0;
    items += i0;
    off += i0;
    const int base = off[0], total = off[nitems] - base;
    for (int p = blockIdx.x; p < total; p += gridDim.x) {
        const int i = serve_item_of(off, nitems, base + p);
        const ServeItem &it = items[i];
        const Shape s = it.s;
        const int tile = base + p - off[i];
        const float sw = sum_w(it.swpart, s.K, &s_tmp);
        if (PREC == PREC_MIXED && i != staged) {
            issue_wimg(s, it.Wimg, smem, &mbar[0]);
            ws.pending = true;
            staged = i;
        }
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
}

// Phase 1 of the mixed path over chunks of every dictionary size in ONE
// launch: the mma h-solve with the k16-slab count read from each chunk's
// shape at run time (the same operations in the same order as the per-size
// instantiations serve_hsolve_kernel<PREC_MIXED, KS>), so a batch that mixes
// dictionary sizes needs no launch per size.
template <int PREC>
__global__ void __launch_bounds__(kThreads, 1) serve_hsolve_any_kernel(const ServeItem *items,
                                                                      const int *off,
                                                                      const int *range) {
    static_assert(PREC == PREC_MIXED, "the FP32 h-solve is not specialized by size");
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
    WStage ws{&mbar[0], &wpar, false};
    int staged = -1;  // item whose W^T image is in shared memory
    const int i0 = range[0], nitems = range[1] - i0;
    items += i0;
    off += i0;
    const int base = off[0], total = off[nitems] - base;
    for (int p = blockIdx.x; p < total; p += gridDim.x) {
        const int i = serve_item_of(off, nitems, base + p);
        const ServeItem &it = items[i];
        const Shape s = it.s;
        const int tile = base + p - off[i];
        const float sw = sum_w(it.swpart, s.K, &s_tmp);
        if (i != staged) {
            issue_wimg(s, it.Wimg, smem, &mbar[0]);
            ws.pending = true;
            staged = i;
        }
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
        hsolve_tile<PREC_MIXED, 0>(s, it.eps, it.gamma, it.Wcm, it.Wrm, sw, t, smem, ws, &mbar[1],
                                   vpar, it.err);
    }
}

// Phase 2: statistics, A, B and W' = sqrt(A/B) of (chunk, output tile) pairs.
template <int PREC>
__global__ void __launch_bounds__(kThreads, 1) serve_stats_kernel(const ServeItem *items,
                                                                 const int *off, const int *range) {
    extern __shared__ __align__(128) unsigned char smem[];
    float *acc = reinterpret_cast<float *>(smem + stats_smem_bytes(PREC) - 2 * 16 * 32 * 4);
    const int i0 = range[0], nitems = range[1] - i0;
    items += i0;
    off += i0;
    const int base = off[0], total = off[nitems] - base;
    for (int p = blockIdx.x; p < total; p += gridDim.x) {
        const int i = serve_item_of(off, nitems, base + p);
        const ServeItem &it = items[i];
        const Shape s = it.s;
        const int FT = s.Fp16 / 16, u = base + p - off[i];
        const int mt = u % FT, ks = u / FT;
        stats_unit<PREC>(s, mt, ks, it.Pg, it.Qg, it.Hg, it.betap, 0, it.n, smem, acc);
        epilogue_unit(s, it.Wcm, it.A, it.B, it.Wn, it.rho, it.rho_on_new, ACC_FP64, mt, ks, acc);
        __syncthreads();
    }
}

// Phase 3: the rescale of (chunk, column) pairs; pair K of an item (one
// past its last column) adds the chunk's loss.
template <int PREC>
__global__ void __launch_bounds__(kThreads) serve_rescale_kernel(const ServeItem *items,
                                                                const int *off,
                                                                const int *range) {
    __shared__ float s_red8[kWarps];
    __shared__ double s_red[kThreads];
    const int i0 = range[0], nitems = range[1] - i0;
    items += i0;
    off += i0;
    const int base = off[0], total = off[nitems] - base;
    for (int p = blockIdx.x; p < total; p += gridDim.x) {
        const int i = serve_item_of(off, nitems, base + p);
        const ServeItem &it = items[i];
        const Shape s = it.s;
        const int k = base + p - off[i];
        if (k < s.K) {
            normalize_columns<PREC>(s, it.normalize, it.Wn, it.Wcm, it.Wrm, it.Wimg, nullptr,
                                    it.A, it.B, ACC_FP64, it.swpart, it.err, s_red8, k, s.K);
        } else {
            const double l = block_sum_ordered(it.loss_part, ceil_div(it.n, kTile), s_red);
            if (threadIdx.x == 0) {
                *it.chunk_loss = l;
                *it.loss_sum += l;
            }
        }
        __syncthreads();
    }
    if (PREC != PREC_FP32) asm volatile("fence.proxy.async.global;\n" ::: "memory");
}

}  // namespace onmf
