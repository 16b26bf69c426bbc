"""FP64 CPU oracle (test infrastructure only; see vif_oracle)."""
