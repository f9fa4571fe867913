"""GB300-native extended convolution and correlation (arXiv 2006.13188).

The compute lives in libextconv.so (CUDA kernels for sm_103a behind the C ABI
in include/extconv.h); this package is its thin Python binding.
"""
from ._binding import (  # noqa: F401
    EXT_FILTER_ANALYTIC_GAUSSPOW, EXT_FILTER_SAMPLED, EXT_FILTER_TABLE, EXT_PREC_BF16X3, EXT_PREC_FP32,
    EXPORTED, ExtError, FilterSO2, LIB_PATH, Plan, ext_conv_so2, ext_corr_so2, ext_corr_so2_components,
    ext_filter_so2_decompose, ext_sweep_so2, ext_sweep_so2_noalloc, ext_conv_scale, ext_batch_corr_so2,
    ext_so3_channels, ext_so3_wigner, ext_corr_so3_components, ext_sweep_so3, ext_corr_so3, ext_conv_so3,
    ext_conv_similarity, so3_pack_tables, lib,
    MLP, ext_mlp_forward, ext_mlp_grads, ext_mlp_train, ext_so3_upper_bound, ext_so3_refined_bound, ext_so3_gather, ext_so3_augment,
    ext_so3_refine, ext_so3_propose, ext_corr_so3_propose, ext_gradient_field, ext_consensus_radius,
    ext_consensus_filter, ext_ght_detect, ext_conv_so2_normalized, ext_filter_so2_energy, ext_corr_so2_subset,
    EXT_PREC_DEFAULT, EXT_FAULT_ALLOC, EXT_FAULT_NONE, EXT_TUNE_OFF, EXT_TUNE_ON, ext_mlp_checkpoint_info,
    ext_select_components, BatchDescriptors, ext_sweep_so3_grid, ext_corr_so3_grid,
)
