"""CPU FP64 oracle (test infrastructure only; see st_oracle)."""
