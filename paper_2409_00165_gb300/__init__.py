"""FOS on GB300: Mie + Monte Carlo photon transport + MLP surrogate (arxiv 2409.00165).

The compute path is the CUDA library ``libfos.so`` (sources in ``csrc/``) behind the
C ABI declared in ``include/fos.h``; ``fos`` is its thin ctypes binding.  The library
is loaded on first use, not at import.
"""
__all__ = ["fos", "workloads"]
