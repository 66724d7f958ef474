"""GB300-native SEM Poisson operator and CG solve behind a C-ABI library."""
