// Composite-grid FAC kernel instances for 4 right-hand sides.
#include "fac_multi.cuh"

namespace amgdd {

cudaError_t launch_fac_multi_4(const FacParams &P, int nsub, int variant, cudaStream_t st)
{
    return P.fp32 ? launch_fac_r_typed<float, 4>(P, nsub, variant, st)
                  : launch_fac_r_typed<double, 4>(P, nsub, variant, st);
}

}  // namespace amgdd
