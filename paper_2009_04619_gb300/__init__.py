"""GB300-native 25-point acoustic wave step with fused PML (arXiv 2009.04619)."""
