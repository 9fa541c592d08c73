"""GB300-native differentiable free-space propagation of sampled optical fields.

The computation lives in the CUDA library libtop.so (C ABI in include/top.h);
this package builds it (``build.build()``) and binds it for torch CUDA tensors
(``binding``) and autograd (``autograd``).
"""
from .binding import (Modulation, Stage, top_fused_chain, top_fused_chain_backward, top_coherence_intensity, top_coherence_intensity_backward, top_modulate,  # noqa: F401
                      top_modulate_backward, top_mse_loss, top_plan_query, top_propagate, top_propagate_backward,
                      top_propagate_coherence, top_propagate_coherence_backward, top_propagate_intensity,
                      top_propagate_intensity_backward, top_intensity, top_intensity_backward, top_propagate_noalloc, top_propagate_overlap, top_propagate_ragged, top_overlap_loss, top_resample, top_resample_backward, top_zcritical)
from .binding import (autotune_clear, autotune_get, autotune_load, autotune_save, autotune_set,  # noqa: F401
                      top_autotune)
from .binding import (circular_polarizer, linear_polarizer, top_field_power, top_jones,  # noqa: F401
                      top_jones_backward, waveplate)
from ._lib import TopError  # noqa: F401
