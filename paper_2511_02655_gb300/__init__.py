"""GB300-native softened-gravity N-body hot path (placeholder; binding added next)."""
