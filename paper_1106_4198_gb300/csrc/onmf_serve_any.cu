// The serving h-solve over chunks of every dictionary size in one launch
// (serve_hsolve_any_kernel), in a translation unit of its own: it inlines
// the mma.sync h-solve for every k16-slab count, so it compiles in parallel
// with the per-size instantiations.
#include "onmf_serve.cuh"

namespace onmf {

const void *serve_any_fn() { return (const void *)serve_hsolve_any_kernel<PREC_MIXED>; }

}  // namespace onmf
