// Mixed-precision step and tile kernels with the penalties of Section 2.2
// ("Extensions") on the mma.sync h-solve, for 1..8 k16 slabs; a translation
// unit of their own so they compile in parallel with the others and leave
// the unpenalized instantiations untouched.
#include "onmf_step.cuh"

namespace onmf {

const void *mixed_online_pen(int ks) {
    switch (ks) {
    case 1: return (const void *)online_kernel<PREC_MIXED, 1, true>;
    case 2: return (const void *)online_kernel<PREC_MIXED, 2, true>;
    case 3: return (const void *)online_kernel<PREC_MIXED, 3, true>;
    case 4: return (const void *)online_kernel<PREC_MIXED, 4, true>;
    case 5: return (const void *)online_kernel<PREC_MIXED, 5, true>;
    case 6: return (const void *)online_kernel<PREC_MIXED, 6, true>;
    case 7: return (const void *)online_kernel<PREC_MIXED, 7, true>;
    case 8: return (const void *)online_kernel<PREC_MIXED, 8, true>;
    }
    return nullptr;
}

const void *mixed_tile_pen(int ks) {
    switch (ks) {
    case 1: return (const void *)tile_kernel<PREC_MIXED, 1, true>;
    case 2: return (const void *)tile_kernel<PREC_MIXED, 2, true>;
    case 3: return (const void *)tile_kernel<PREC_MIXED, 3, true>;
    case 4: return (const void *)tile_kernel<PREC_MIXED, 4, true>;
    case 5: return (const void *)tile_kernel<PREC_MIXED, 5, true>;
    case 6: return (const void *)tile_kernel<PREC_MIXED, 6, true>;
    case 7: return (const void *)tile_kernel<PREC_MIXED, 7, true>;
    case 8: return (const void *)tile_kernel<PREC_MIXED, 8, true>;
    }
    return nullptr;
}

}  // namespace onmf
