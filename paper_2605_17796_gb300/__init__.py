"""GB300 (sm_103a) implementation of LEAD's data-parallel decoding path.

The computation lives in the C-ABI library liblead.so (include/lead.h); ``lead`` is its
Python binding and ``pipeline`` a batched driver (sampling, decoding, checking) used by the
benchmark and the tests. ``build`` compiles the library.
"""
