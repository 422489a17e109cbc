"""GB300-native multi-time-step PD / continuum coupling (arXiv 2403.03605)."""
