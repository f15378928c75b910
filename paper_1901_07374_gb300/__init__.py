"""GB300-native damage-weighted Total-Lagrangian SPH step (arXiv 1901.07374)."""
