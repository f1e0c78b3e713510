"""Alias-table construction and sampling on GB300 (placeholder; binding added with the CUDA library)."""
