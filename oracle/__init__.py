"""FP64 CPU oracle (test infrastructure only; see qfd_oracle.py's header)."""
