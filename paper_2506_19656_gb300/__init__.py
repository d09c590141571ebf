"""xv: GPU encoder analysis for spatiotemporal Earth-data cubes (GB300, sm_103a).

The compute path is the CUDA library ``libxv.so`` behind the C ABI declared in
``include/xv.h``; ``paper_2506_19656_gb300.xv`` is its thin Python binding.
Importing this package does not load the library; the binding does, and it
raises if the library is missing.
"""
__all__ = ["synth", "xv"]
