"""GB300-native batched IGA-FEM element-matrix integration (arxiv 2207.00280)."""
