"""Seeded synthetic image and noise generator.

Serves both the CUDA path's tests/benchmark and the oracle's tests.  It holds
none of the denoiser's arithmetic (no pyramid, no structure tensor, no
filtering): only clean-image synthesis and noise draws.

Clean images stand in for the paper's natural-image training/test sets
(Section 4, "Experimental results": Berkeley test images, Internet training
images), which are not available: piecewise-smooth random polygons (even-odd
fill) with per-polygon linear colour gradients, about 30 % of them filled with
an oriented sinusoid of period 4-32 px, over a per-channel linear-gradient
background, clipped to [0, 1].  Images are planar float32 ``[3][H][W]`` RGB.
"""
from .images import (clean_image, awgn, signal_dependent_noise, gain_field,
                     quantize8, noisy_pair, batch_pairs)

__all__ = ["clean_image", "awgn", "signal_dependent_noise", "gain_field",
           "quantize8", "noisy_pair", "batch_pairs"]
