"""GB300-native HHL state-vector simulation (Zheng, Chen, Yang & Li, PESGM 2024).

Thin Python binding of ``libqsim_gb300.so`` (C ABI in ``include/qsim.h``): argument
marshalling only; every step of the simulation runs in the library's CUDA kernels.  PyTorch is
used for device memory and streams.  There is no CPU fallback: if the shared library is
missing the import of a binding raises ``QsimLibraryMissing``.
"""
from ._binding import (  # noqa: F401
    QSIM_C64,
    QSIM_C128,
    QsimError,
    QsimLibraryMissing,
    Batch,
    Circuit,
    hhl_batch_autotune,
    hhl_batch_create,
    qsim_apply_batched,
    qsim_batch_create,
    HHLCircuit,
    Pool,
    hhl_build,
    hhl_build_spectral,
    hhl_prepare_state,
    hhl_run,
    hhl_readout,
    library,
    library_path,
    qsim_apply,
    qsim_device_status,
    qsim_launch_count,
    qsim_launch_counts,
    qsim_fuse,
    qsim_hermitian_eig,
    qsim_autotune,
    qsim_tune_get,
    qsim_tune_reset,
    qsim_tune_set,
    qsim_tune_table,
    QSIM_TUNE_DFT_TMA,
    QSIM_TUNE_DFT_LANES,
    QSIM_TUNE_DFT_PREFETCH,
    QSIM_TUNE_DENSE_TC,
    QSIM_TUNE_FUSE_WIDTH,
    QSIM_TUNE_DFT_L2PROMO,
    QSIM_TUNE_DFT_MERGE,
    QSIM_TUNE_TUNED,
    qsim_version,
)
