// Measurement probe (not part of libonmf): the cost of one tcgen05.mma
// (cta_group::1, kind::f16, bf16 x bf16 -> f32, M = 128, K = 16) as a
// function of N, with A in shared memory or in tensor memory and one or four
// accumulators. One CTA, one issuing thread; clock64 around `iters` MMAs
// issued back to back and around their completion (one commit). Operands
// are zeros (the cost does not depend on the values). Then the throughput of
// the warp-level mma.sync m16n8k16 (bf16 -> f32) from registers: W warps per
// SM, each with C independent accumulator chains. Prints one JSON line per
// configuration. Built and run by `python bench.py --probe-tcgen05`.
#include <cstdio>

#include "onmf_tc.cuh"

using namespace onmf;

__global__ void __launch_bounds__(128, 1) probe(int N, int tmemA, int nacc, int iters,
                                                 long long *out, int *err) {
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t slot;
    for (int i = threadIdx.x; i < 16384 / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_mbar_init();
    }
    if (threadIdx.x < 32) tmem_alloc(&slot, 512);
    fence_proxy_async_shared();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tb = slot;
    {  // A in tensor memory: columns 448..455 of the warp's 32 lanes, zero
        uint32_t z[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        tmem_st8(tb + ((uint32_t)(32 * (threadIdx.x >> 5)) << 16) + 448, z);
        tmem_st_wait();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {
        const uint32_t id = tc_idesc(128, N);
        const uint64_t adesc = tc_desc(smem, 128, 256);                   // K-major, 128 x 16
        const uint64_t bdesc = tc_desc(smem + 4096, (N / 8) * 128, 128);  // MN-major, 16 x N
        const long long t0 = clock64();
        for (int i = 0; i < iters; ++i) {
            const uint32_t d = tb + (uint32_t)((i % nacc) * N);
            if (tmemA)
                tc_mma_tmem_a(d, tb + 448, bdesc, id, 1u);
            else
                tc_mma_smem_a(d, adesc, bdesc, id, 1u);
        }
        const long long t1 = clock64();
        tc_commit(&bar);
        mbar_wait_bounded(&bar, 0, err);
        const long long t2 = clock64();
        out[0] = t1 - t0;
        out[1] = t2 - t0;
    }
    tc_fence_before();
    __syncthreads();
    if (threadIdx.x < 32) tmem_dealloc(tb, 512);
}

// mma.sync throughput: every warp runs `iters` rounds of C independent
// m16n8k16 products (operands in registers); clock64 of warp 0.
template <int C>
__global__ void mma_sync_probe(int iters, long long *out, float *sink) {
    uint32_t a[4] = {threadIdx.x, threadIdx.x + 1, threadIdx.x + 2, threadIdx.x + 3};
    float d[C][4];
#pragma unroll
    for (int c = 0; c < C; ++c)
#pragma unroll
        for (int e = 0; e < 4; ++e) d[c][e] = 0.f;
    __syncthreads();
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < C; ++c) mma_bf16_16816(d[c], a, a[0] ^ (uint32_t)c, a[1]);
    __syncthreads();
    const long long t1 = clock64();
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < C; ++c) s += d[c][0] + d[c][1] + d[c][2] + d[c][3];
    sink[blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the products
    if (threadIdx.x == 0) out[0] = t1 - t0;
}

template <int C>
static int run_mma_sync(int warps, long long *d_out, float *d_sink) {
    const int iters = 4096;
    mma_sync_probe<C><<<1, 32 * warps>>>(iters, d_out, d_sink);
    if (cudaDeviceSynchronize() != cudaSuccess) return 1;
    long long h = 0;
    cudaMemcpy(&h, d_out, 8, cudaMemcpyDeviceToHost);
    const double n = (double)warps * C * iters;
    printf("{\"mma_sync\": \"m16n8k16 bf16\", \"warps\": %d, \"chains\": %d, "
           "\"clk_per_mma_per_sm\": %.2f, \"mac_per_clk\": %.0f}\n",
           warps, C, (double)h / n, n * 16 * 8 * 16 / (double)h);
    return 0;
}

int main() {
    long long *d_out = nullptr;
    int *d_err = nullptr;
    if (cudaMalloc(&d_out, 16) != cudaSuccess || cudaMalloc(&d_err, 4) != cudaSuccess) return 1;
    cudaMemset(d_err, 0, 4);
    cudaFuncSetAttribute(probe, cudaFuncAttributeMaxDynamicSharedMemorySize, 16384);
    const int Ns[] = {16, 32, 64, 128, 256};
    const int iters = 256;
    for (int N : Ns)
        for (int tmemA = 0; tmemA < 2; ++tmemA)
            for (int nacc : {1, 4}) {
                if (nacc * N > 448) continue;  // accumulators below the A columns
                probe<<<1, 128, 16384>>>(N, tmemA, nacc, iters, d_out, d_err);
                const cudaError_t e = cudaDeviceSynchronize();
                long long h[2] = {0, 0};
                int herr = 0;
                cudaMemcpy(h, d_out, 16, cudaMemcpyDeviceToHost);
                cudaMemcpy(&herr, d_err, 4, cudaMemcpyDeviceToHost);
                if (e != cudaSuccess || herr) {
                    printf("{\"error\": \"cuda %d, device flags %d\"}\n", (int)e, herr);
                    return 1;
                }
                printf("{\"M\": 128, \"N\": %d, \"K\": 16, \"A\": \"%s\", \"accumulators\": %d, "
                       "\"issue_clk_per_mma\": %.1f, \"total_clk_per_mma\": %.1f, "
                       "\"mac_per_clk\": %.0f}\n",
                       N, tmemA ? "tmem" : "smem", nacc, (double)h[0] / iters,
                       (double)h[1] / iters, 128.0 * N * 16 * iters / (double)h[1]);
            }
    float *d_sink = nullptr;
    if (cudaMalloc(&d_sink, 16 * 32 * 4) != cudaSuccess) return 1;
    if (run_mma_sync<1>(1, d_out, d_sink) || run_mma_sync<4>(4, d_out, d_sink) ||
        run_mma_sync<8>(8, d_out, d_sink) || run_mma_sync<8>(16, d_out, d_sink))
        return 1;
    return 0;
}
