"""GB300-native ProbeSim: single-source and top-k SimRank on dynamic directed graphs.

The compute path is ``libprobesim.so`` (hand-written sm_103a CUDA behind a C ABI, declared in
``include/probesim.h``).  ``probesim`` is its thin ctypes binding; ``synth`` holds the seeded synthetic
graph and query generators.  Importing the package loads nothing; ``probesim.load()`` loads the
library and raises if it is missing.
"""
__all__ = ["probesim", "synth"]
