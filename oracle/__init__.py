"""The GFMC oracle: test infrastructure only (see oracle.py and gfmc_oracle.c)."""
