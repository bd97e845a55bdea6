"""GB300-native parallel community detection (PLP, PLM, PLMR, EPP).

The compute path is the CUDA library built from ``csrc/`` and reached through
the C-ABI declared in ``include/cd.h``; :mod:`.cd` is its Python binding and
:mod:`.synth` holds the seeded input generators.  Importing the package does
not load the library; the binding loads it on first use and raises if it is
missing.
"""
