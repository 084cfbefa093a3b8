"""GB300-native hybrid lattice Boltzmann scheme for binary mixtures (arXiv:0902.3921)."""
