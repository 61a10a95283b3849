"""B300-native vesicle-suspension boundary-integral hot path (arXiv 2606.25569)."""
