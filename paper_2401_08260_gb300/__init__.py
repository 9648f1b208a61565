"""Sliced fast kernel summation on GB300 (sm_103a)."""
