"""GB300 (sm_103a) library for explicit time steps of d-dimensional linear PDEs held in
hierarchical Tucker or CP format (arXiv:1803.10270).

The compute path is the C-ABI shared library built from ``csrc/`` (``build.py``);
``htgpu`` is its ctypes binding.  Importing this package loads nothing: call
``htgpu.load()`` (done implicitly by the binding's functions).
"""
__all__ = ["htgpu", "inputs", "build"]
