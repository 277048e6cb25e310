"""GB300-native Parallel Toplesets Propagation (PTP) geodesic distances."""
