"""GB300-native FilterReg hot path (placeholder; the binding is added with the C-ABI)."""
