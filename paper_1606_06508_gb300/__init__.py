"""Batched accurate normalization of vectors and quaternions on GB300 (arXiv 1606.06508)."""
