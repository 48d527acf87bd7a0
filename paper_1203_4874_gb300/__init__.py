"""CBP deblurring on one GB300 (sm_103a): CUDA library libcbp + ctypes binding.

The method is Thorpe et al., "A Co-Prime Blur Scheme for Data Security in
Video Surveillance" (arXiv 1203.4874).  ``cbp`` holds the binding of the C ABI
declared in ``include/cbp.h``; ``build`` compiles the library in-tree.
"""
from . import cbp  # noqa: F401
