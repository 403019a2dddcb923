"""GB300-native BioFVM-B LOD diffusion-decay step (arXiv 2602.05017).

The compute path is ``libbiofvm.so`` (hand-written sm_103a CUDA kernels behind a C ABI, see
``include/biofvm.h``); ``binding`` wraps it with ctypes and torch device memory.  Importing this
package does not load the library; ``from paper_2602_05017_gb300 import binding`` does, and fails
loudly if it has not been built.
"""
__all__ = ["inputs", "binding", "build"]
