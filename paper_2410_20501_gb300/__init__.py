"""GB300-native particle-mesh force step (PySCo, arXiv 2410.20501).

The compute path is the CUDA library ``_lib/libpmgb.so`` (sources in ``csrc/``,
C ABI in ``include/pm_api.h``); ``pm`` is its thin ctypes binding over torch
device memory and streams.  ``inputs`` draws seeded synthetic inputs.
The binding is imported lazily so that input generation works without a GPU.
"""
__all__ = ["pm", "inputs", "build"]
