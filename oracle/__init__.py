"""Plain FP64 CPU oracle of the hot path (test infrastructure only; see orc.py)."""
