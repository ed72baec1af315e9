// Device helpers shared by the libonmf kernels: bounded waits, the error
// word, BF16 packing and thin inline-PTX wrappers for the sm_103a data-movement
// and tensor-core instructions the kernels use.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace onmf {

// Bits of the per-state device error word.
enum : int {
    ERR_INPUT = 1,    // a frame value was negative, NaN or Inf
    ERR_NUMERIC = 2,  // the dictionary step produced a non-finite W
    ERR_TIMEOUT = 4,  // a bounded wait (grid barrier, bulk copy) ran out
    ERR_CONFIG = 8,   // the launch did not have the shape the kernel needs
};

// Every device-side wait gives up after this many nanoseconds of
// %globaltimer and reports ERR_TIMEOUT instead of spinning forever.
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Whether this CTA has flagged an error since the kernel started
// (flag_error sets it; kernels with grid barriers clear it at entry with
// cta_err_init). A CTA that arrives at a grid barrier with it set also sets
// the barrier counter's top bit, so that every CTA waiting there learns of
// the error from the word it polls, with no second read of the error word.
static __shared__ int s_cta_err;

__device__ __forceinline__ void flag_error(int *err, int bits) {
    atomicOr(err, bits);
    s_cta_err = 1;
}

__device__ __forceinline__ int read_error(const int *err) {
    return *reinterpret_cast<const volatile int *>(err);
}

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_gpu_add(unsigned *p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Top bit of a grid barrier counter: some CTA arrived with an error (or
// gave up waiting); the low 31 bits count the arrivals of the launch.
constexpr unsigned kBarErrBit = 0x80000000u;

// At kernel entry, before any flag_error: an error word that is already set
// (an earlier launch on the same state) counts as this CTA's own, so the
// kernel leaves at its first grid barrier.
__device__ __forceinline__ void cta_err_init(const int *err) {
    if (threadIdx.x == 0) s_cta_err = read_error(err) != 0 ? 1 : 0;
    __syncthreads();
}

// Thread 0: arrive at a grid barrier (after a CTA barrier), carrying this
// CTA's error state in the top bit. The bit is set before the release add,
// so a CTA that sees the full count also sees the bit.
__device__ __forceinline__ void grid_arrive_t0(unsigned *counter) {
    if (s_cta_err) atomicOr(counter, kBarErrBit);
    red_release_gpu_add(counter, 1u);
}

// Thread 0: wait until `target` CTAs have arrived or the error bit is set;
// false on the error bit or on timeout (the CTA then flags ERR_TIMEOUT and
// sets the bit, so the others stop waiting too).
__device__ __forceinline__ bool grid_wait_t0(unsigned *counter, unsigned target, int *err) {
    const uint64_t t0 = global_ns();
    unsigned spins = 0;
    for (;;) {
        const unsigned c = ld_acquire_gpu(counter);
        if (c & kBarErrBit) return false;
        if (c >= target) return true;
        if (++spins > 1024) __nanosleep(32);
        if ((spins & 255u) == 0 && global_ns() - t0 > kWaitLimitNs) {
            flag_error(err, ERR_TIMEOUT);
            atomicOr(counter, kBarErrBit);
            return false;
        }
    }
}

// Grid-wide barrier for a cooperative (co-resident) launch. `epoch` counts
// the barriers this CTA has passed; the counter must be zero at launch.
// Thread 0 arrives with a release reduction after the CTA barrier and waits
// with acquire loads before the next CTA barrier; release and acquire are
// cumulative, so the writes of the whole CTA before the barrier are visible
// to every CTA after it. Every CTA returns false, and callers leave the
// kernel, when some CTA arrived with an error flagged (the counter's top
// bit: all of them see it, so all leave at the same barrier); an error this
// CTA flags after arriving travels with its next arrival. The wait is
// bounded: on timeout the CTA flags ERR_TIMEOUT and returns false.
__device__ __forceinline__ bool grid_sync(unsigned *counter, unsigned nblocks,
                                          unsigned &epoch, int *err) {
    __syncthreads();
    ++epoch;
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        grid_arrive_t0(counter);
        s_ok = grid_wait_t0(counter, epoch * nblocks, err) ? 1 : 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// The two halves of grid_sync, for a CTA that has work to do between its
// arrival and its wait (work that reads nothing other CTAs write in this
// phase). grid_arrive releases the CTA's writes made before it; grid_wait
// returns false on a reported error or timeout, like grid_sync.
__device__ __forceinline__ void grid_arrive(unsigned *counter, unsigned &epoch) {
    __syncthreads();
    ++epoch;
    if (threadIdx.x == 0) grid_arrive_t0(counter);
}

__device__ __forceinline__ bool grid_wait(unsigned *counter, unsigned nblocks, unsigned epoch,
                                          int *err) {
    __shared__ int s_okw;
    if (threadIdx.x == 0) s_okw = grid_wait_t0(counter, epoch * nblocks, err) ? 1 : 0;
    __syncthreads();
    return s_okw != 0;
}

// %globaltimer (ns, one clock for all SMs) of thread 0 into
// stamps[(m * gridDim.x + blockIdx.x) * ONMF_STAMP_PTS + i] (phase-timing
// builds; compiled out otherwise).
#ifndef ONMF_STAMP_PTS
#define ONMF_STAMP_PTS 48  // points per (minibatch, CTA) record
#endif
#ifdef ONMF_PHASE_STAMPS
#define ONMF_STAMP(stamps, m, i)                                                              \
    do {                                                                                      \
        if ((stamps) && threadIdx.x == 0 && (m) < 128)                                        \
            (stamps)[((long long)(m) * gridDim.x + blockIdx.x) * ONMF_STAMP_PTS + (i)] =      \
                (long long)global_ns();                                                       \
    } while (0)
#else
#define ONMF_STAMP(stamps, m, i) \
    do {                          \
    } while (0)
#endif

// ---------------------------------------------------------------- BF16

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// ------------------------------------------------- tensor core (mma.sync)

// D = A * B + C for one m16n8k16 tile, BF16 inputs, FP32 accumulate.
__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4],
                                               uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t (&r)[4], const void *row_addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(row_addr)));
}

__device__ __forceinline__ void ldmatrix_x4_trans(uint32_t (&r)[4], const void *row_addr) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(row_addr)));
}

// Store four 8x8 b16 matrices transposed: lane L supplies the row address of
// row (L & 7) of matrix (L >> 3); register i holds this thread's pair
// (row lane/4, columns 2*(lane%4), +1) of matrix i before transposition.
__device__ __forceinline__ void stmatrix_x4_trans(void *row_addr, uint32_t r0, uint32_t r1,
                                                  uint32_t r2, uint32_t r3) {
    asm volatile("stmatrix.sync.aligned.m8n8.x4.trans.shared.b16 [%0], {%1,%2,%3,%4};\n" ::"r"(
                     smem_u32(row_addr)),
                 "r"(r0), "r"(r1), "r"(r2), "r"(r3)
                 : "memory");
}

// Approximate reciprocal (MUFU, about 1 ulp); used where the result is
// rounded to BF16 afterwards.
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ------------------------------------------------------- async copies

// 16-byte global->shared copy; src_bytes < 16 zero-fills the rest.
__device__ __forceinline__ void cp_async16(void *smem_dst, const void *gmem_src,
                                           int src_bytes = 16) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(smem_dst)),
                 "l"(gmem_src), "r"(src_bytes)
                 : "memory");
}

// 4-byte global->shared copy (no alignment beyond 4 bytes needed).
__device__ __forceinline__ void cp_async4(void *smem_dst, const void *gmem_src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_u32(smem_dst)),
                 "l"(gmem_src)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Wait until at most the most recent group is still in flight.
__device__ __forceinline__ void cp_async_wait_group1() {
    asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}

// mbarrier + bulk (TMA engine) copies.
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_shared() {
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile(
        "{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
            smem_u32(bar)),
        "r"(bytes)
        : "memory");
}

// Bulk copy of `bytes` (multiple of 16, both addresses 16-byte aligned)
// from global to this CTA's shared memory, completing on `bar`.
__device__ __forceinline__ void bulk_g2s(void *smem_dst, const void *gmem_src, unsigned bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];\n" ::"r"(smem_u32(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase. Returns false (and flags ERR_TIMEOUT)
// if the phase did not complete within the limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, int *err) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    unsigned spins = 0;
    while (!mbar_try_wait(bar, parity)) {
        if ((++spins & 255u) == 0 && global_ns() - t0 > kWaitLimitNs) {
            flag_error(err, ERR_TIMEOUT);
            return false;
        }
    }
    return true;
}

// ------------------------------------------ thread-block clusters (DSMEM)

__device__ __forceinline__ unsigned cluster_ctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_nctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// Cluster-wide barrier of all threads of all CTAs in the cluster; release
// and acquire order the shared::cluster stores issued before it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n"
                 "barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
}

// Address in CTA `rank`'s shared memory of the local shared address `a`.
__device__ __forceinline__ uint32_t map_rank(uint32_t a, unsigned rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_cluster_f32x2(uint32_t a, float x, float y) {
    asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(x), "f"(y) : "memory");
}

__device__ __forceinline__ void st_cluster_u32(uint32_t a, uint32_t v) {
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

__device__ __forceinline__ void st_cluster_v4(uint32_t a, uint4 v) {
    asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w)
                 : "memory");
}

__device__ __forceinline__ void st_cluster_f32x4(uint32_t a, float x, float y, float z, float w) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(x), "f"(y),
                 "f"(z), "f"(w)
                 : "memory");
}

__device__ __forceinline__ void st_cluster_f32(uint32_t a, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__host__ __device__ constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }
__host__ __device__ constexpr int ceil_div(int x, int m) { return (x + m - 1) / m; }

}  // namespace onmf
