"""GB300-native hash group-by and hash join (C-ABI library + thin binding)."""
