"""FP64 CPU oracle for the FFM hot path: test infrastructure only (see oracle.py)."""
