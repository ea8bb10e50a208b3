"""GB300-native multi-patch FC-SDNN spatial operator (C-ABI library + thin binding)."""
