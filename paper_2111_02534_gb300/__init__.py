"""GB300-native tensor-product scheme for three-body bound states (arXiv 2111.02534).

Importing the package is light: the CUDA library is loaded by
``paper_2111_02534_gb300.tps`` (the ctypes binding), which raises if the
compiled extension is missing.
"""
__all__ = ["inputs"]
