"""FP64 CPU oracle of the SIPF-W step (test infrastructure only)."""
