"""GB300 (sm_103a) implementation of the convex-programming method for top-k
locally densest subgraphs (edge density, LDS) and locally triangle-densest
subgraphs (LTDS).

The compute path is the C-ABI library ``liblds.so`` built from ``csrc/``; the
Python binding in :mod:`.lds` only marshals arguments.  Importing this package
loads nothing; :func:`.lds.load` loads the library and raises if it is missing.
"""
__all__ = ["lds", "synth"]
