"""GB300-native transit-model hot path (placeholder; the CUDA binding follows)."""
