"""GB300-native Mu3e online event selection (arXiv:2206.11535).

The package holds the CUDA library (``csrc/``, built to ``libm3e.so``), its thin
ctypes binding (``m3e``) and the synthetic frame generator (``gen``).  Importing the
package loads nothing; ``paper_2206_11535_gb300.m3e`` loads the shared library and
fails loudly when it has not been built.
"""
__version__ = "0.1.0"
