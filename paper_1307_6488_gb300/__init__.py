"""GB300-native BSSN right-hand side, Kreiss-Oliger dissipation and RK4
library (hand-written sm_103a CUDA behind a C ABI).

The compute path lives in ``libbssn.so`` (built from ``csrc/``); the Python
module ``binding`` only marshals arguments to it. ``inputs`` builds seeded
synthetic initial data.
"""
__all__ = ["binding", "inputs"]
