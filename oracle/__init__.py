"""FP64 CPU oracle of the Fossen vehicle step — test infrastructure, not part of the product."""
