"""GB300-native (sm_103a) 3D Gaussian Splatting training hot path.

The compute path is the C-ABI library ``libgs.so`` built from ``csrc/``; the
Python modules here only marshal arguments (``binding``), manage device
buffers and streams (``engine``), and draw synthetic inputs (``synth``).
Importing the package loads nothing; ``binding.lib()`` loads the library and
raises if it has not been built.
"""
__all__ = ["synth"]
