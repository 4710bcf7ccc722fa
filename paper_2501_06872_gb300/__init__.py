"""GB300-native graph transposition (CSR -> CSC).

The compute path is the C-ABI library ``libgt.so`` built from ``csrc/`` for
sm_103a; :mod:`.binding` marshals arguments to it.  There is no CPU fallback:
if the library is missing, calls raise.
"""

__all__ = ["binding"]
