"""GB300-native time step of the DPRI urban-flow LES (arXiv 1504.02264).

The compute path is a C-ABI CUDA library (``include/les.h``); ``les`` holds its
thin ctypes binding and ``scene`` the seeded synthetic inputs.  Importing the
package loads nothing; ``paper_1504_02264_gb300.les`` loads the library.
"""
__all__ = ["scene", "les"]
