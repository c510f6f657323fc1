"""GB300 median-threshold-bitmap (MTB) exposure alignment."""
