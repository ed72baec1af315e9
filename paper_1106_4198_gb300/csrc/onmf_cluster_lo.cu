// Cluster h-solve kernels for 1..8 k16 slabs (K up to 128); a separate
// translation unit so the variants compile in parallel.
#include "onmf_cluster_step.cuh"

namespace onmf {

const void *cluster_online_lo(int ks) {
    static const void *const fns[] = {
        (const void *)online_cluster_kernel<1>,
        (const void *)online_cluster_kernel<2>,
        (const void *)online_cluster_kernel<3>,
        (const void *)online_cluster_kernel<4>,
        (const void *)online_cluster_kernel<5>,
        (const void *)online_cluster_kernel<6>,
        (const void *)online_cluster_kernel<7>,
        (const void *)online_cluster_kernel<8>};
    return (ks >= 1 && ks <= 8) ? fns[ks - 1] : nullptr;
}

const void *cluster_tile_lo(int ks) {
    static const void *const fns[] = {
        (const void *)tile_cluster_kernel<1>,
        (const void *)tile_cluster_kernel<2>,
        (const void *)tile_cluster_kernel<3>,
        (const void *)tile_cluster_kernel<4>,
        (const void *)tile_cluster_kernel<5>,
        (const void *)tile_cluster_kernel<6>,
        (const void *)tile_cluster_kernel<7>,
        (const void *)tile_cluster_kernel<8>};
    return (ks >= 1 && ks <= 8) ? fns[ks - 1] : nullptr;
}

}  // namespace onmf
