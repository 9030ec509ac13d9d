"""GB300-native block-space map H for m-simplex domains (arXiv 2208.11617)."""
