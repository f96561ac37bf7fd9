// Composite-grid FAC kernel instances for 1 right-hand side.
#include "fac_multi.cuh"

namespace amgdd {

cudaError_t launch_fac_multi_1(const FacParams &P, int nsub, int variant, cudaStream_t st)
{
    return P.fp32 ? launch_fac_r_typed<float, 1>(P, nsub, variant, st)
                  : launch_fac_r_typed<double, 1>(P, nsub, variant, st);
}

}  // namespace amgdd
