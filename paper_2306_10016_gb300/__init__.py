"""Hybrid dealiased convolution on GB300 (placeholder; binding added below)."""
