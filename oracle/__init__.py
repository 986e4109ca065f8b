"""CPU FP64 oracle (test infrastructure only; see bspline_oracle)."""
