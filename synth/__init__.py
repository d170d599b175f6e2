"""Seeded synthetic multi-echo (multi-coil) MRI volumes.

This module only draws inputs: phantom magnitude, smooth field map, coil
sensitivities, noise and the support mask, and synthesises the echo images by
the forward signal model (Sec. II, Eq. 1: y = e^{i w t} s x + noise).  It holds
none of the estimator's arithmetic (no cost, gradient, curvature, factor or
solver), so both the FP64 oracle and the CUDA path may take their inputs from it.
"""
from .volumes import (Volume, make_volume, ellipsoid_mask, small_config, full_config,
                      diff_config, batch_configs, TE_MS, make_wf_volume, wf_config, fat_spectrum,
                      WF_TE_MS, phantom_config, full8_small_config, full1_config)

__all__ = ["Volume", "make_volume", "ellipsoid_mask", "small_config", "full_config",
           "diff_config", "batch_configs", "TE_MS", "make_wf_volume", "wf_config", "fat_spectrum",
           "WF_TE_MS", "phantom_config", "full8_small_config", "full1_config"]
