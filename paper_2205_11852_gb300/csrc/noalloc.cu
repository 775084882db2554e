// tpcf_lc_cov_noalloc: the float64 LC covariance with its scratch in a
// fixed, file-scope device array instead of context workspace.
//
// For callers that must not allocate device memory once they are running:
// services that size all of their GPU memory at start-up and treat any later
// cudaMalloc as a failure, and code that must not trigger the implicit device
// synchronisation that cudaMalloc / cudaFree can cause.  The caller passes
// only its inputs and outputs; nothing is allocated or freed here.
#include <cmath>

#include "tpcf_internal.h"

namespace tpcf {
namespace {

// Scratch of the float64 LC covariance: centred residuals of the three
// variants, their means and the three Gram blocks (the layout the existing
// float64 launcher expects).  Every GPU that loads the library holds this
// array until the process exits.
constexpr size_t NOALLOC_SCRATCH_DOUBLES = size_t(1) << 21;   // 16 MiB
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

// Device address of the scratch array in the current device's context.  In
// host code the array's name is only a host-side stand-in; the address is
// looked up on every call (a host-side table lookup once the module is
// loaded), so it stays right after cudaDeviceReset or a context change.
cudaError_t scratch_on_current_device(double **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = (double *)p;
    return cudaSuccess;
}

}  // namespace

size_t noalloc_scratch_doubles(int n_mock, int nbin)
{
    return 3 * (size_t)n_mock * nbin + 3 * (size_t)nbin + 3 * (size_t)nbin * nbin;
}

}  // namespace tpcf

extern "C" int tpcf_lc_cov_noalloc(const double *xi_a1, const double *xi_a2, const double *xi_b, int n_mock,
                                   int nbin, int M_a, double M, double *C_lc, double *Ca, double *Cb, double *A,
                                   double *B, void *stream)
{
    using namespace tpcf;
    if (!xi_a1 || !xi_a2 || !xi_b || !C_lc) return TPCF_ERR_ARG;
    if (n_mock < 2 || nbin < 1 || M_a < 1 || !(M >= (double)M_a)) return TPCF_ERR_ARG;
    if (noalloc_scratch_doubles(n_mock, nbin) > NOALLOC_SCRATCH_DOUBLES) return TPCF_ERR_RANGE;
    double *scratch = nullptr;
    cudaError_t e = scratch_on_current_device(&scratch);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TPCF_ERR_CUDA;
    }
    // every scratch element is written before it is read (means, residuals,
    // all Gram entries), so nothing needs clearing between calls
    e = launch_lc_fp64(xi_a1, xi_a2, xi_b, n_mock, nbin, scratch, M_a, M, C_lc, Ca, Cb, A, B,
                       (cudaStream_t)stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TPCF_ERR_CUDA;
    }
    return TPCF_OK;
}
