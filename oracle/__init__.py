"""FP64 CPU oracle (test infrastructure only; see fc_oracle.py)."""
