"""B300-native preconditioned Bi-CGSTAB Poisson solver (arxiv 2503.08935)."""
