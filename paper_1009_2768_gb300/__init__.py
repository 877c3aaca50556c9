"""GB300-native TRMC-R (recursive Time Relaxed Monte Carlo) collision step."""
