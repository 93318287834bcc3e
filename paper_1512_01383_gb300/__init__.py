"""GB300-native lifted PDHG solver (arXiv 1512.01383)."""
