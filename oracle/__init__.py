"""CPU FP64 oracle of ChASE (test infrastructure only; never imported by the product library)."""
