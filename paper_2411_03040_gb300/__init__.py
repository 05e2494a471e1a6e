"""GB300-native line radiative transfer hot path (Magritte, arXiv 2411.03040).

The compute path is the CUDA library ``libmgt.so`` behind the C-ABI declared in
``include/magritte_gpu.h``; ``paper_2411_03040_gb300.mgt`` is its thin ctypes
binding (import it explicitly; importing this package loads nothing native).
``paper_2411_03040_gb300.synth`` generates seeded synthetic input models.
"""
__all__ = ["synth", "mgt"]
