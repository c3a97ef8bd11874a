"""GB300-native Faceted HyperSARA PDFB hot path (arXiv 2003.07358)."""
