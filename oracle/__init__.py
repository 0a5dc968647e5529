"""FP64 CPU oracle of the neural radiance cache hot path (test infrastructure only)."""
