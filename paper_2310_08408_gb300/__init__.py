"""GB300-native differentiable free-space optics: RS / VRS / CZT / VCZT propagation, optical
elements and camera losses with hand-written adjoints (XLuminA, arXiv 2310.08408, hot path).

The compute path is the C-ABI CUDA library ``libxl.so`` (built from ``csrc/``); ``xl`` is its
thin ctypes binding and ``autograd`` wraps it in ``torch.autograd.Function``s. Importing this
package loads nothing; the library is loaded on first use and a missing library raises.
"""
