"""GB300-native BSGD hot path (placeholder; the binding is added next)."""
