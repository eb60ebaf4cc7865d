"""GB300-native RoofGS renderer (binding is filled in by the runtime module)."""
