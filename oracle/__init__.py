"""FP64 CPU oracle (test infrastructure only; see tp_oracle)."""
from . import tp_oracle  # noqa: F401
