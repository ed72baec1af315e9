// Host-side launchers of the libonmf kernels (C++ linkage, internal).
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "onmf_kernels.cuh"

namespace onmf {

int64_t kernel_launches();
cudaError_t configure_kernels();
size_t max_dynamic_smem();
size_t online_smem_bytes(const Shape &s, int prec);
size_t tile_smem_bytes(const Shape &s, int prec);
size_t batch_stats_smem_bytes(int prec);
cudaError_t max_coresident_blocks(int prec, int ks, size_t smem, int *blocks_per_sm);

cudaError_t launch_online(const StepArgs &a, int prec, int grid, size_t smem, cudaStream_t stream);
cudaError_t launch_tiles(const TileArgs &a, int prec, int grid, size_t smem, cudaStream_t stream);
cudaError_t launch_prepare(const Shape &s, const float *Wcm, float *Wrm, __nv_bfloat16 *Wimg,
                           float *swpart, cudaStream_t stream, __nv_bfloat16 *Wrow = nullptr);
bool tc_shape_supported(const Shape &s);
const void *serve_gather_fn();                // serving phase 0 (frames to the device)
const void *serve_fn(int prec, int ks);       // serving phase 1 (h-solve)
const void *serve_any_fn();                   // phase 1 over every dictionary size at once
const void *serve_stats_fn(int prec);         // serving phase 2 (statistics, W')
const void *serve_rescale_fn(int prec);       // serving phase 3 (rescale, loss)
cudaError_t launch_sum(const double *x, long long n, double *out, int accumulate,
                       cudaStream_t stream);
cudaError_t launch_batch_stats(const Shape &s, int prec, const void *Pg, const void *Qg,
                               const void *Hg, long long betap, long long N, int nchunks,
                               float *part, int grid, cudaStream_t stream);
cudaError_t launch_batch_wstep(const Shape &s, const float *part, int nchunks, float *W,
                               cudaStream_t stream);
cudaError_t launch_batch_normalize(const Shape &s, int normalize, float *W, float *scale, int *err,
                                   cudaStream_t stream);
cudaError_t launch_batch_scale_h(int K, long long N, float *H, const float *scale,
                                 cudaStream_t stream);
cudaError_t launch_batch_h0(const Shape &s, const float *V, long long ldv, long long N, float eps,
                            const float *swpart, float *H, cudaStream_t stream);
// h-solve variant for a shape and an onmf_hsolve choice (PREC_FP32 unless
// mixed; -1 if the shape does not allow the choice).
int select_prec(bool mixed, const Shape &s, int hsolve);

// Cluster h-solve (PREC_CL): C CTAs per cluster.
struct ClusterTiles {
    int C = 0, grid = 0;  // CTAs per cluster (0: shape not covered), CTAs
    size_t smem = 0;
    long long slots = 0;  // loss slots: 32-frame tiles x C
};
// Launch geometry of the cluster tile kernel for n frames.
ClusterTiles cluster_tiles(const Shape &s, long long n);
size_t cluster_smem_bytes(const Shape &s, int C, bool online);
int cluster_max_active(const Shape &s, int C, bool online);
int cluster_choose(const Shape &s, long long frames, int num_sms, size_t smem_limit, bool online);
cudaError_t launch_online_cluster(const StepArgs &a, int C, int grid, size_t smem,
                                  cudaStream_t stream);
cudaError_t launch_tiles_cluster(const TileArgs &a, int C, int grid, size_t smem,
                                 cudaStream_t stream);

// Row gather/scatter by an index list (NULL: consecutive rows from `first`).
cudaError_t launch_gather_rows(float *dst, long long ld_dst, const float *src, long long ld_src,
                               const long long *idx, long long first, long long n, int width,
                               cudaStream_t stream);
cudaError_t launch_scatter_rows(float *dst, long long ld_dst, const float *src, long long ld_src,
                                const long long *idx, long long first, long long n, int width,
                                cudaStream_t stream);
cudaError_t launch_index_rows(long long *dst, const long long *idx, long long first, long long n,
                              cudaStream_t stream);
// Rows of F floats from mapped host memory (src, leading dimension lds) to a
// dense device buffer, by kPullCtas CTAs.
constexpr int kPullCtas = 16;
cudaError_t launch_pull_rows(float *dst, int F, const float *src, long long lds, long long n,
                             cudaStream_t stream);

cudaError_t launch_wait_selftest(int which, unsigned *counter, int *err,
                                 unsigned long long *elapsed, cudaStream_t stream);

}  // namespace onmf
