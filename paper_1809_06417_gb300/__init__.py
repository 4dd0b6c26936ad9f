"""GB300-native radiative-transport flame volume reconstruction (arXiv 1809.06417)."""
