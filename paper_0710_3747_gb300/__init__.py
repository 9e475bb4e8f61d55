"""GB300-native random-phase pure-state spin dynamics (arXiv:0710.3747)."""
