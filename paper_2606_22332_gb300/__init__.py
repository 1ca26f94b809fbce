"""GB300-native tactile contact query and noise model (Tactile Genesis, arxiv 2606.22332).

The compute path is the CUDA library ``csrc/libtg.so`` behind the C-ABI in
``include/tg.h``; :mod:`paper_2606_22332_gb300.tg` is its thin ctypes binding.
:mod:`paper_2606_22332_gb300.workload` creates seeded synthetic inputs.
Submodules load lazily so that the input generator imports without a GPU.
"""
__all__ = ["tg", "workload"]
