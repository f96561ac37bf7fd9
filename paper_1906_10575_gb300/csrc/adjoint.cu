// Gradient of a quadratic form of the 7-point variable-coefficient diffusion
// operator with respect to its node coefficients: for A(kappa) assembled with
// harmonic-mean face coefficients c_ij = 2 k_i k_j / (k_i + k_j) (a face to the
// Dirichlet boundary uses k_i),
//   g_m = d(-lam^T A x)/d k_m
//       = -( sum_{j nbr m} 2 k_j^2 / (k_m + k_j)^2 (lam_m - lam_j)(x_m - x_j)
//            + (number of boundary faces of m) lam_m x_m ),
// i.e. the outer product -lam x^T restricted to the stencil and chained
// through the face coefficients. With x = A^{-1} b and lam = A^{-1} dL/dx
// (A is symmetric) it is dL/dk. One thread per node, no atomics.
#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "../../include/amgdd.h"

namespace amgdd {
void set_last_error(const std::string &msg);
}

namespace {

__global__ void k_kappa_grad(int nx, int ny, int nz, const double *__restrict__ kap, const double *__restrict__ x,
                             const double *__restrict__ lam, double *__restrict__ g)
{
    const int64_t n = (int64_t)nx * ny * nz;
    for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < n; m += (int64_t)gridDim.x * blockDim.x) {
        const int i = (int)(m % nx);
        const int j = (int)((m / nx) % ny);
        const int k = (int)(m / ((int64_t)nx * ny));
        const double km = kap[m], lm = lam[m], xm = x[m];
        const int64_t sx = 1, sy = nx, sz = (int64_t)nx * ny;
        // neighbours in ascending index order: -z, -y, -x, +x, +y, +z
        const bool has[6] = {k > 0, j > 0, i > 0, i < nx - 1, j < ny - 1, k < nz - 1};
        const int64_t off[6] = {-sz, -sy, -sx, sx, sy, sz};
        double s = 0.0;
        int nb = 0;
        for (int q = 0; q < 6; ++q) {
            if (!has[q]) {
                ++nb;
                continue;
            }
            const int64_t o = m + off[q];
            const double kj = kap[o];
            const double den = (km + kj) * (km + kj);
            const double w = (2.0 * kj * kj) / den;
            s = s + w * ((lm - lam[o]) * (xm - x[o]));
        }
        s = s + (double)nb * (lm * xm);
        g[m] = -s;
    }
}

}  // namespace

extern "C" amgdd_status amgdd_kappa_grad_3d(int32_t nx, int32_t ny, int32_t nz, const double *kappa, const double *x,
                                            const double *lam, double *grad, void *stream)
{
    if (nx <= 0 || ny <= 0 || nz <= 0) {
        amgdd::set_last_error("grid sizes must be positive");
        return AMGDD_ERR_INVALID_ARG;
    }
    if (!kappa || !x || !lam || !grad) {
        amgdd::set_last_error("null pointer");
        return AMGDD_ERR_INVALID_ARG;
    }
    const int64_t n = (int64_t)nx * ny * nz;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 152 * 32) blocks = 152 * 32;
    k_kappa_grad<<<(int)blocks, 256, 0, (cudaStream_t)stream>>>(nx, ny, nz, kappa, x, lam, grad);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        amgdd::set_last_error(std::string("gradient kernel: ") + cudaGetErrorString(e));
        return AMGDD_ERR_CUDA;
    }
    return AMGDD_OK;
}
