"""GB300-native fast Hankel tensor-vector products (placeholder, filled below)."""
