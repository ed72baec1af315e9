// Mixed-precision (BF16 tensor-core) step kernels for 5..8 k16 slabs
// (K up to 128); a separate translation unit so the variants compile in
// parallel.
#include "onmf_step.cuh"

namespace onmf {

const void *mixed_online_hi(int ks) {
    switch (ks) {
    case 5: return (const void *)online_kernel<PREC_MIXED, 5>;
    case 6: return (const void *)online_kernel<PREC_MIXED, 6>;
    case 7: return (const void *)online_kernel<PREC_MIXED, 7>;
    case 8: return (const void *)online_kernel<PREC_MIXED, 8>;
    }
    return nullptr;
}

const void *mixed_tile_hi(int ks) {
    switch (ks) {
    case 5: return (const void *)tile_kernel<PREC_MIXED, 5>;
    case 6: return (const void *)tile_kernel<PREC_MIXED, 6>;
    case 7: return (const void *)tile_kernel<PREC_MIXED, 7>;
    case 8: return (const void *)tile_kernel<PREC_MIXED, 8>;
    }
    return nullptr;
}

}  // namespace onmf
