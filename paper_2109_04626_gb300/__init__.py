"""GB300-native PC-stable skeleton search (arXiv 2109.04626), reversed-order schedule."""
