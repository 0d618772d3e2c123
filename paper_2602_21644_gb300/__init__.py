"""GB300-native MP-aware differentiable Gaussian splatting (DAGS-SLAM hot path).

The compute lives in the CUDA library ``libdags.so`` (built from ``csrc/``,
C ABI declared in ``include/dags.h``); ``dags`` is its thin ctypes binding,
``autograd`` wraps forward/backward in a ``torch.autograd.Function`` and
``synth`` makes seeded synthetic scenes and ``state`` dumps and restores run
state (.npz). Importing the package loads nothing;
the library is loaded on first use and its absence is an error.
"""
__all__ = ["dags", "autograd", "synth", "state"]
