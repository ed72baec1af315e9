// Mixed-precision (BF16 tensor-core) step kernels for 1..4 k16 slabs
// (K up to 64); a separate translation unit so the variants compile in
// parallel.
#include "onmf_step.cuh"

namespace onmf {

const void *mixed_online_lo(int ks) {
    switch (ks) {
    case 1: return (const void *)online_kernel<PREC_MIXED, 1>;
    case 2: return (const void *)online_kernel<PREC_MIXED, 2>;
    case 3: return (const void *)online_kernel<PREC_MIXED, 3>;
    case 4: return (const void *)online_kernel<PREC_MIXED, 4>;
    }
    return nullptr;
}

const void *mixed_tile_lo(int ks) {
    switch (ks) {
    case 1: return (const void *)tile_kernel<PREC_MIXED, 1>;
    case 2: return (const void *)tile_kernel<PREC_MIXED, 2>;
    case 3: return (const void *)tile_kernel<PREC_MIXED, 3>;
    case 4: return (const void *)tile_kernel<PREC_MIXED, 4>;
    }
    return nullptr;
}

}  // namespace onmf
