"""GB300 pair counts, split Landy-Szalay estimator and linear-construction
(LC) covariance of the two-point correlation function.

The computation lives in the CUDA library ``_build/libtpcf.so`` (C ABI in
``include/tpcf.h``); this package is its thin ctypes binding.  Importing the
package loads the library and fails if it has not been built.
"""
from ._binding import (  # noqa: F401
    EXPORTED, TPCF_BATCHED, TPCF_BF16X3, TPCF_DD, TPCF_DR, TPCF_ERR_ARG, TPCF_ERR_CUDA, TPCF_ERR_NOMEM,
    TPCF_ERR_RANGE, TPCF_ERR_STATE, TPCF_ERR_TIMEOUT, TPCF_FP64, TPCF_HOST_INPUT, TPCF_KERNEL_AUTO,
    TPCF_KERNEL_DIRECT, TPCF_KERNEL_GENERAL, TPCF_LOS_MIDPOINT, TPCF_LOS_X, TPCF_OK, TPCF_OPEN,
    TPCF_OPT_AUTOTUNE, TPCF_OPT_GRAPHS, TPCF_OPT_HOST_GROUP_KB, TPCF_OPT_KERNEL, TPCF_OPT_TEST_SKIP_MMA,
    TPCF_OPT_WAIT_LIMIT,
    TPCF_PER_LAUNCH, TPCF_PERIODIC, TPCF_RR, TPCF_TF32X3,
    TPCF_WARN_EMPTY_BIN, Context, TpcfArgError, TpcfError, lib, make_binning, tpcf_multipole_matrix,
    tpcf_thresholds, validate_count_args,
)

lib()
