"""Comparison paths timed beside the engine (not part of the product)."""
