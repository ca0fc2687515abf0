"""GB300-native Fourier Poisson solver (FLUPS method, arXiv 2211.07777)."""
