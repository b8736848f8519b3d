"""FP64 CPU oracle for HOQRI (test infrastructure only; see oracle.py)."""
