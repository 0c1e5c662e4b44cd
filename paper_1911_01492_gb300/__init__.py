"""GB300-native matrix-free SIPG-DG operator and CG solvers (placeholder)."""
