// Cluster h-solve kernels for 9..16 k16 slabs (K from 129 to 256); a separate
// translation unit so the variants compile in parallel.
#include "onmf_cluster_step.cuh"

namespace onmf {

const void *cluster_online_hi(int ks) {
    static const void *const fns[] = {
        (const void *)online_cluster_kernel<9>,
        (const void *)online_cluster_kernel<10>,
        (const void *)online_cluster_kernel<11>,
        (const void *)online_cluster_kernel<12>,
        (const void *)online_cluster_kernel<13>,
        (const void *)online_cluster_kernel<14>,
        (const void *)online_cluster_kernel<15>,
        (const void *)online_cluster_kernel<16>};
    return (ks >= 9 && ks <= 16) ? fns[ks - 9] : nullptr;
}

const void *cluster_tile_hi(int ks) {
    static const void *const fns[] = {
        (const void *)tile_cluster_kernel<9>,
        (const void *)tile_cluster_kernel<10>,
        (const void *)tile_cluster_kernel<11>,
        (const void *)tile_cluster_kernel<12>,
        (const void *)tile_cluster_kernel<13>,
        (const void *)tile_cluster_kernel<14>,
        (const void *)tile_cluster_kernel<15>,
        (const void *)tile_cluster_kernel<16>};
    return (ks >= 9 && ks <= 16) ? fns[ks - 9] : nullptr;
}

}  // namespace onmf
