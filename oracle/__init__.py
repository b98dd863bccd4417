"""CPU oracle (test infrastructure only; see dgsem_oracle)."""
