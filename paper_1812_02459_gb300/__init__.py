"""GB300-native fractional-step MRT lattice Boltzmann solver (arXiv:1812.02459)."""
