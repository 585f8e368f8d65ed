"""GB300-native REDO (Rapid Exponentiation using Discrete Operators)."""
