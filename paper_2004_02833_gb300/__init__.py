"""GB300-native staggered-grid P_N time step (StaRMAP, arXiv 2004.02833).

The compute path is the CUDA library ``librtpn.so`` built from ``csrc/``; ``rtpn`` is its thin
ctypes binding.  ``synth`` produces the seeded synthetic inputs, ``showcase`` runs the reactor-like
convergence study of Section 5.2, and ``halo`` holds the slab decomposition and ghost-plane exchange
of the multi-rank step.  Importing this package does not load the library; ``rtpn.lib()`` does, and
raises if it is missing.
"""
__all__ = ["rtpn", "synth", "showcase", "halo"]
