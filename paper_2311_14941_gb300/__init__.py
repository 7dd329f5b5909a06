"""GB300-native stiff finite-rate chemistry integration (constant-pressure homogeneous reactors).

Importing the package is cheap: the CUDA library is loaded on first use of
:mod:`paper_2311_14941_gb300.chem`.  :mod:`paper_2311_14941_gb300.synth` builds seeded synthetic
mechanisms and cell fields.
"""
__all__ = ["chem", "synth"]
