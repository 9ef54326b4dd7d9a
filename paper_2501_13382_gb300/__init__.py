"""libgbt: GB300-native Gaussian beam summation (arXiv 2501.13382)."""
