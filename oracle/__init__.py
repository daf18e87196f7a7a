"""CPU oracle for the PSD solver (test infrastructure only; see psd_oracle)."""
