"""FP64 CPU oracle (test infrastructure only; never on the product path)."""
from . import rbc_oracle  # noqa: F401
