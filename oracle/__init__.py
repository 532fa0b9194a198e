"""FP64 reference oracle for the ACSE hot path (test infrastructure only)."""
