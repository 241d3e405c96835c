"""CPU FP64 SPH oracle: test infrastructure only (see oracle/sph_oracle.c)."""
