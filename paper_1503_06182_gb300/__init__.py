"""GB300-native VEGAS (the data-parallel hot path of arXiv:1503.06182).

The compute path is the CUDA library ``libgvegas.so`` (built in-tree from
``csrc/``); ``vegas`` is its thin ctypes binding and ``autograd`` the PyTorch
``autograd.Function`` over the adjoint.  ``workloads`` holds the seeded
synthetic inputs only.  Importing the package does not load the library; the
first binding call does, and it raises if the library is missing.
"""
__all__ = ["vegas", "workloads", "autograd"]
