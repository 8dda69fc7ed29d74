"""FP64 CPU oracle of the implicit TDGL step (test infrastructure only)."""
