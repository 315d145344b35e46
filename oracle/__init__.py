"""FP64 CPU oracle of the split time step (test infrastructure only)."""
