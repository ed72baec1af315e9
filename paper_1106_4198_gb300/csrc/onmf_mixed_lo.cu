// Mixed-precision step kernels for 1..4 k16 slabs (K up to 64): the
// mma.sync h-solve (PREC_MIXED) and the tcgen05 h-solve (PREC_TC); a separate
// translation unit so the variants compile in parallel.
#include "onmf_serve.cuh"
#include "onmf_step.cuh"

namespace onmf {

const void *mixed_online_lo(int prec, int ks) {
    switch (ks) {
    case 1: return prec == PREC_TC ? (const void *)online_kernel<PREC_TC, 1>
                                   : (const void *)online_kernel<PREC_MIXED, 1>;
    case 2: return prec == PREC_TC ? (const void *)online_kernel<PREC_TC, 2>
                                   : (const void *)online_kernel<PREC_MIXED, 2>;
    case 3: return prec == PREC_TC ? (const void *)online_kernel<PREC_TC, 3>
                                   : (const void *)online_kernel<PREC_MIXED, 3>;
    case 4: return prec == PREC_TC ? (const void *)online_kernel<PREC_TC, 4>
                                   : (const void *)online_kernel<PREC_MIXED, 4>;
    }
    return nullptr;
}

const void *mixed_tile_lo(int prec, int ks) {
    switch (ks) {
    case 1: return prec == PREC_TC ? (const void *)tile_kernel<PREC_TC, 1>
                                   : (const void *)tile_kernel<PREC_MIXED, 1>;
    case 2: return prec == PREC_TC ? (const void *)tile_kernel<PREC_TC, 2>
                                   : (const void *)tile_kernel<PREC_MIXED, 2>;
    case 3: return prec == PREC_TC ? (const void *)tile_kernel<PREC_TC, 3>
                                   : (const void *)tile_kernel<PREC_MIXED, 3>;
    case 4: return prec == PREC_TC ? (const void *)tile_kernel<PREC_TC, 4>
                                   : (const void *)tile_kernel<PREC_MIXED, 4>;
    }
    return nullptr;
}

const void *mixed_serve_lo(int ks) {
    switch (ks) {
    case 1: return (const void *)serve_hsolve_kernel<PREC_MIXED, 1>;
    case 2: return (const void *)serve_hsolve_kernel<PREC_MIXED, 2>;
    case 3: return (const void *)serve_hsolve_kernel<PREC_MIXED, 3>;
    case 4: return (const void *)serve_hsolve_kernel<PREC_MIXED, 4>;
    }
    return nullptr;
}

}  // namespace onmf
