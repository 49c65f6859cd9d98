"""FP64 CPU oracle of the DNSLABIB flow step and its ventilation metrics.

Test infrastructure only: used by ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``.
It shares no code with the CUDA library and never imports it.
"""
