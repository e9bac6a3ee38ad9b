"""GB300-native multi-objective Digital Annealer (arXiv 2205.13399)."""
