// Composite-grid FAC kernel instances for 2 right-hand sides.
#include "fac_multi.cuh"

namespace amgdd {

cudaError_t launch_fac_multi_2(const FacParams &P, int nsub, int variant, cudaStream_t st)
{
    return P.fp32 ? launch_fac_r_typed<float, 2>(P, nsub, variant, st)
                  : launch_fac_r_typed<double, 2>(P, nsub, variant, st);
}

}  // namespace amgdd
