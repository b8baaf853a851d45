"""GB300-native parallel-in-time multigrid preconditioned FGMRES for augmented systems."""
