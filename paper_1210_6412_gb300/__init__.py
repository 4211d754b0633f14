"""GB300-native reachability-probability solver (placeholder, binding follows)."""
