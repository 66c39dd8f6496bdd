"""GB300-native compressed Deep Potential (DP-SE_a) energy / force / virial path.

The compute runs in the CUDA library ``libdp.so`` (built from ``csrc/``) behind
the C-ABI declared in ``include/dp.h``; :mod:`.dp` is its thin Python binding
and :mod:`.inputs` holds the seeded synthetic-input generators.
"""
