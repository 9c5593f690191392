"""Plain FP64 CPU oracle for Parallel CFR -- test infrastructure only (see oracle.py)."""
