"""GB300-native exact brute-force k-NN graph engine (Komarov, Dashti, D'Souza,
"Fast k-NNG construction with GPU-based quick multi-select").

The compute path is the C-ABI library ``libknn.so`` built from ``csrc/``; this
package's binding only marshals arguments into it. Importing the package does
not load the library: the first call does, and fails loudly when it is missing.
"""
__all__ = ["inputs"]
