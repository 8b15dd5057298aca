"""Seeded synthetic inputs for the ACI library and its tests.

This package produces the input tensor trains (TTs) of the paper's workloads:
quantics TTs of Fourier fields (Sec. 3.2, Eq. (fourierseries) and Eq. (quanticsrep)),
Gaussians (Sec. 3.1, Eq. (gaussians)) and uniform random TTs (Sec. 3.3). It holds
none of the ACI method's arithmetic: only data generation (exact block-sum TTs of
Fourier modes, TT-SVD compression) and plain TT evaluation used to check results.
Both the CPU oracle and the CUDA path read their inputs from here.
"""

from .tt import (
    TT, tt_ranks, tt_full, tt_eval, tt_block_sum, tt_svd_round, tt_from_dense,
    tt_random_uniform, quantics_points,
)
from .fields import (
    fourier_config1, fourier_config2, fourier_config3, fourier_paper_1d,
    gaussian_pair, random_tt_pair, config_inputs, CONFIG_NAMES,
)

__all__ = [
    "TT", "tt_ranks", "tt_full", "tt_eval", "tt_block_sum", "tt_svd_round", "tt_from_dense",
    "tt_random_uniform", "quantics_points",
    "fourier_config1", "fourier_config2", "fourier_config3", "fourier_paper_1d",
    "gaussian_pair", "random_tt_pair", "config_inputs", "CONFIG_NAMES",
]
