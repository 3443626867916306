"""GB300 ferrofluid dipolar Barnes-Hut library.

``ff``    - binding of the CUDA library libff.so (include/ff.h)
``synth`` - seeded synthetic ensembles shaped like the paper's workloads

Importing the package loads nothing; ``ff.lib()`` loads libff.so and raises if
it has not been built.
"""
__all__ = ["ff", "synth"]
