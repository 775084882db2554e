// Split-precision Gram products for the LC covariance on the tensor cores.
#include "tpcf_internal.h"

namespace tpcf {

size_t lc_split_work_bytes(int n_mock, int nbin, int precision)
{
    (void)precision;
    return 256 + 3 * (size_t)n_mock * nbin * 8 + 3 * (size_t)nbin * 8 + 3 * (size_t)nbin * nbin * 8;
}

cudaError_t launch_lc_split(const double *, const double *, const double *, int, int, int, void *, size_t, int,
                            double, double *, double *, double *, double *, double *, cudaStream_t)
{
    return cudaErrorNotSupported;
}

}  // namespace tpcf
