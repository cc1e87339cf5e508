"""Exact GB300 assignment solver (Kuhn-Munkres and batched KM)."""
