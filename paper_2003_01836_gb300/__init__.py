"""GB300-native barycentric Lagrange treecode (placeholder until the binding lands)."""
