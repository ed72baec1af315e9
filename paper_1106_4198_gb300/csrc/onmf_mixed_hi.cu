// Mixed-precision step kernels for 5..8 k16 slabs (K up to 128): the
// mma.sync h-solve (PREC_MIXED) and the tcgen05 h-solve (PREC_TC); a separate
// translation unit so the variants compile in parallel.
#include "onmf_serve.cuh"
#include "onmf_step.cuh"

namespace onmf {

const void *mixed_online_hi(int prec, int ks) {
    switch (ks) {
    case 5: return prec == PREC_TC ? (const void *)online_kernel<PREC_TC, 5>
                                   : (const void *)online_kernel<PREC_MIXED, 5>;
    case 6: return prec == PREC_TC ? (const void *)online_kernel<PREC_TC, 6>
                                   : (const void *)online_kernel<PREC_MIXED, 6>;
    case 7: return prec == PREC_TC ? (const void *)online_kernel<PREC_TC, 7>
                                   : (const void *)online_kernel<PREC_MIXED, 7>;
    case 8: return prec == PREC_TC ? (const void *)online_kernel<PREC_TC, 8>
                                   : (const void *)online_kernel<PREC_MIXED, 8>;
    }
    return nullptr;
}

const void *mixed_tile_hi(int prec, int ks) {
    switch (ks) {
    case 5: return prec == PREC_TC ? (const void *)tile_kernel<PREC_TC, 5>
                                   : (const void *)tile_kernel<PREC_MIXED, 5>;
    case 6: return prec == PREC_TC ? (const void *)tile_kernel<PREC_TC, 6>
                                   : (const void *)tile_kernel<PREC_MIXED, 6>;
    case 7: return prec == PREC_TC ? (const void *)tile_kernel<PREC_TC, 7>
                                   : (const void *)tile_kernel<PREC_MIXED, 7>;
    case 8: return prec == PREC_TC ? (const void *)tile_kernel<PREC_TC, 8>
                                   : (const void *)tile_kernel<PREC_MIXED, 8>;
    }
    return nullptr;
}

const void *mixed_serve_hi(int ks) {
    switch (ks) {
    case 5: return (const void *)serve_hsolve_kernel<PREC_MIXED, 5>;
    case 6: return (const void *)serve_hsolve_kernel<PREC_MIXED, 6>;
    case 7: return (const void *)serve_hsolve_kernel<PREC_MIXED, 7>;
    case 8: return (const void *)serve_hsolve_kernel<PREC_MIXED, 8>;
    }
    return nullptr;
}

}  // namespace onmf
