"""GB300-native lattice gauge fixing (Schroeck & Vogt, arXiv:1212.5221)."""
