"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module produces raw samples only: dense images and wavefronts, per-axis
sample vectors and scalar parameters.  It contains none of the method's
arithmetic (no quantics map, no SVD, no MPO, no propagation), so both sides can
draw their inputs from it without sharing any part of the computation.

Every generator takes an explicit integer seed; the default seeds are
``23089 + config_index`` so each workload is reproducible on any machine.
"""
from .fields import (  # noqa: F401
    SEED_BASE,
    gaussian_random_field_image,
    gaussian_beam_with_rectangles,
    separable_phase_factors,
    kolmogorov_phase_screen,
    batched_item_specs,
    batched_item_field,
    rectangles_target,
    smooth_random_phase_mask_factors,
    random_mps_sites,
    random_unitary_sites,
    physical_constants,
    pupil_field,
)
