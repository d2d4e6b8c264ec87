"""GB300-native constrained Delaunay refinement (the per-round refinement step of gQM3D)."""
