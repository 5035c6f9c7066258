"""GB300-native staggered Kahler-Dirac multigrid (arXiv:2212.12559).

The solver lives in the CUDA shared library ``libsmg.so`` built from
``csrc/``; ``binding`` wraps its C ABI.  ``inputs`` draws the seeded synthetic
gauge fields and sources.  Importing this package does not load the library;
``binding.load()`` does, and fails loudly when it is missing.
"""
