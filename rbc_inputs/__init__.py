"""Seeded input generators shared by the oracle side and the CUDA side.

This package holds only inputs: the coefficient tensors (U, V, W) of published
bilinear formulas, the seeded perturbation that turns an exact formula into an
approximate one, and seeded matrix generators.  It holds none of the method's
arithmetic (no encoding, no products, no decoding, no random draws of the
randomization itself).
"""
from .formulas import (  # noqa: F401
    strassen, laderman, classical_formula, perturbed, ones_rank1, gaussian_formula,
    formula_by_name,
)
from .matrices import (  # noqa: F401
    gaussian, uniform, scaled_hard, adversarial, hilbert, matrix_pair,
)
